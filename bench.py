#!/usr/bin/env python3
"""GFMC throughput benchmark on GB300: spin updates/s at L = 32, M = 1024.

Workload (one chain, synthetic): double-exchange model at infinite Hund
coupling on a 32^3 periodic cubic lattice, t = 1, spins uniform on the sphere
(seed 0), beta = 20/t, mu = -2t, Jackson kernel, M = 1024 moments, sequential
sweep with Philox proposals (seed 1).  A "step" is one block of
``--updates-per-step`` consecutive single-spin updates of the sweep (each
update = 511 fused 7-vector stencil steps + moments + FFT + quadrature +
Metropolis + patch), i.e. one pass of the whole hot path over that block.

The headline ``value`` is the FP64 path (all arithmetic in FP64); the same run
also times the FP32-mixed path and reports it under ``fp32_mixed``.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gfmc|reference]

Under torchrun each rank runs an independent replica chain (chain_id = rank):
the path shards by chains, with no data-path collective ("replicas only").
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "spin updates/s at L=32,M=1024 (FP64 vs FP32-mixed); stencil GB/s; p99 sweep latency"
UNIT = "spin updates/s"

# Algorithmic work of one site in one fused stencil step of the doubling
# (M/2 - 1 steps), recursion on the 7 unit vectors:
#   stencil  7 x (6 complex MACs + 2r - r_prev)      = 7 x (6 x 8 + 4)   = 364 flop
#   Gram     28 <r_m|r_m> (7 real diagonal) + 28 <r_m|r_m+1>
#            = 7 x 3 + 21 x 6 + 28 x 6                                     = 315 flop
#   sums     112 real partial products added once                           = 112 flop
# and on the proposal's two vectors o, v: 2 x 52 stencil + 8 real products of
# 3 flop + 8 sums = 136 flop.
FLOP_PER_SITE_STEP = 364 + 315 + 112
FLOP_PER_SITE_STEP_PROPOSAL = 2 * 52 + 8 * 3 + 8
# With L even the periodic cubic lattice is bipartite: r_m of vector o lives on
# one parity and r_m of its 6 neighbours on the other, so half of the stencil
# terms and most Gram products above are zero by construction.  What is left,
# per pair of sites (one of each parity) and step:
#   stencil  7 vector-site updates x 52                                     = 364 flop
#   Gram     7 real diagonals x 3 + 15 pairs among the neighbours x 6
#            + 6 products <r_m^o|r_m+1^k> x 6                              = 147 flop
#   sums     49 nonzero real entries                                          = 49 flop
# i.e. 280 flop per site and step: the work the FP64 engine does on even L.
FLOP_PER_SITE_STEP_BIPARTITE = (364 + 147 + 49) / 2


# Bytes of one site in one step of the doubling: read r_m and r_{m-1}, write
# r_{m+1} for each of the nv vectors (3 nv complex values) plus the site's
# spinor (3 reals), B_upd = (M/2) N (21 s_c + s_chi): 180 B FP32, 360 B FP64
# for the 7 unit vectors.  The checkerboard recursion of the FP32 engine
# (M - 2 steps over half the sites each) moves exactly these values.
def bytes_per_site_step(real_bytes: int, nv: int = 7) -> int:
    return 3 * nv * 2 * real_bytes + 3 * real_bytes


def update_work(L: int, M: int, real_bytes: int, nv: int = 7):
    N = L ** 3
    steps = M // 2 - 1
    flop = FLOP_PER_SITE_STEP if nv == 7 else FLOP_PER_SITE_STEP_PROPOSAL
    return steps * N * flop, steps * N * bytes_per_site_step(real_bytes, nv)


def update_flop_nonzero(L: int, M: int) -> float:
    """Flop of one update of the FP64 engine without the terms that vanish by
    parity (L even; the full count for odd L)."""
    per = FLOP_PER_SITE_STEP_BIPARTITE if L % 2 == 0 else FLOP_PER_SITE_STEP
    return (M // 2 - 1) * L ** 3 * per


# DRAM bytes (read + write) of one engine launch in the bench's launch
# configuration (FP64: 16 updates; FP32-mixed: 64), each from one ncu capture
# (`ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum` of run_case with
# that many updates).  They hold only for the engine sources they were taken
# from: bench.py reports them as roofline.traffic while the hash of those
# sources is unchanged and the launch has that many updates, and null
# otherwise.
TRAFFIC_SOURCES = ("gfmc_engine.cuh", "gfmc_k64.cu", "gfmc_k32.cu", "gfmc_internal.h", "gfmc_vcluster.cuh",
                   "gfmc_kvc.cu")
TRAFFIC_HASH = "f1314c5534c2c5a7"
TRAFFIC_PER_LAUNCH = {"fp64": (16, 6818304 + 2359296), "fp32_mixed": (64, 1485312 + 26880)}


def engine_sources_hash() -> str:
    import hashlib
    csrc = os.path.join(ROOT, "paper_1303_6016_gb300", "csrc")
    inner = "".join(hashlib.sha256(open(os.path.join(csrc, f), "rb").read()).hexdigest() + "  " +
                    os.path.join("paper_1303_6016_gb300", "csrc", f) + "\n" for f in TRAFFIC_SOURCES)
    return hashlib.sha256(inner.encode()).hexdigest()[:16]


def traffic_per_launch(precision: str, updates: int):
    try:
        if engine_sources_hash() != TRAFFIC_HASH:
            return None
    except OSError:
        return None
    n, b = TRAFFIC_PER_LAUNCH[precision]
    return float(b) if updates == n else None


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# FP64 / FP32 vector (non-tensor) ALU peaks of GB300, derived from the unit
# counts and the maximum SM clock: 152 SMs x 2070 MHz x 2 flop per FMA x
# FMA lanes per SM per clock (FP32: 128; FP64: 2, from the 1.25 TFLOP/s figure).
def alu_peak_tflops(precision: str, sm_mhz: float = 2070.0) -> float:
    lanes = 2.0 if precision == "fp64" else 128.0
    return 152 * sm_mhz * 1e6 * 2 * lanes / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = list(self.rows)

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(n_gpus: int):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, world, local, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value: float) -> float:
    if dist is None:
        return value
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(world: int, steps: int, updates_per_step: int, max_total_ms: float) -> float:
    """Whole-job updates/s: every rank ran `steps` blocks of updates on its own
    replica chain; the slowest rank's device time bounds the job."""
    return world * steps * updates_per_step / (max_total_ms / 1000.0)


def l2_copy_gbs(n_bytes: int = 32 << 20, copies: int = 40, replays: int = 10) -> float:
    """Measured L2-resident copy bandwidth (read + write bytes): `copies` copies
    of a 32 MiB buffer into another (64 MiB in all, inside the 129 MB L2)
    captured in a CUDA graph so no launch gaps are timed; CUDA events."""
    import torch
    x = torch.ones(n_bytes // 4, dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(3):
            y.copy_(x)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(copies):
            y.copy_(x)
    g.replay()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(replays):
        g.replay()
    b.record()
    b.synchronize()
    return 2.0 * n_bytes * copies * replays / (a.elapsed_time(b) / 1000.0) / 1e9


def sweep_latency(gfmc, inputs, stream, L, M, precision, sweeps, warmup=2):
    """p50 / p99 of full-sweep device time (CUDA events) on an L^3 chain."""
    import torch
    sp = inputs.uniform_sphere(L, 0)
    ch = gfmc.Chain(L, sp, M=M, beta=20.0, mu=-2.0, seed=1, precision=precision, stream=stream.cuda_stream)
    N = L ** 3
    for _ in range(warmup):
        ch.updates_into(N)
    per = []
    for _ in range(sweeps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        ch.updates_into(N)
        e.record(stream)
        e.synchronize()
        per.append(s.elapsed_time(e))
    ch.close()
    per.sort()
    p99 = per[min(len(per) - 1, int(math.ceil(0.99 * len(per))) - 1)]
    return {"L": L, "M": M, "precision": precision, "sweeps": sweeps, "p50_ms": statistics.median(per),
            "p99_ms": p99}


def run_batching(stream, steps, warmup, updates, flush, recursion="unit_vectors", graphs=True, compensated=False):
    """64 independent FP32-mixed chains, L from {8,12,16,24,32}, T ~ U[0.02, 0.2],
    M = 1024, in team-engine launches planned by the autotuner; a step runs
    `updates` updates of every chain (`compensated`: Dot2 Gram sums)."""
    import torch
    from paper_1303_6016_gb300 import batch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    chains, Ls, Ts = batch.c4_chains(M=1024, recursion=recursion, compensated=compensated)
    tuner = batch.Autotuner(M=1024, precision="fp32_mixed", recursion=recursion, compensated=compensated)
    runner = batch.BatchRunner(chains, tuner)
    plan = runner.plan([updates] * len(chains))
    tune_s = time.perf_counter() - t0
    for _ in range(warmup):
        runner.run(updates)
    per = []
    for k in range(steps):
        flush.fill_(k)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        runner.run(updates)
        e.record()
        e.synchronize()
        per.append(s.elapsed_time(e))
    total = sum(per)
    teams = {}
    for w, tc in plan:
        for i, t in zip(w, tc):
            teams.setdefault(int(Ls[i]), set()).add(int(t))  # 0: shares a one-CTA team
    n = len(chains)
    nv = 2 if recursion == "proposal" else 7
    _, bytes_u = zip(*[update_work(int(L), 1024, 4, nv) for L in Ls])
    graph = None
    if graphs and len(plan) == 1:
        # the same step captured once in a CUDA graph (gfmc_plan_*) and replayed
        from paper_1303_6016_gb300 import gfmc
        w, tc = plan[0]
        order = list(w)
        with gfmc.Plan([chains[i] for i in order], [updates] * n, list(tc), schedule="teams") as gp:
            gp.launch(warmup)
            gp.sync(trace=False)
            perg = []
            for k in range(steps):
                flush.fill_(k)
                s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s.record()
                gp.launch(1)
                e.record()
                e.synchronize()
                perg.append(s.elapsed_time(e))
            gp.sync(trace=False)
        graph = {"value": n * updates * steps / (sum(perg) / 1000.0), "unit": UNIT,
                 "ms_per_step": sum(perg) / steps,
                 "note": "one CUDA graph launch per step (gfmc_plan_launch), no host work between steps"}
    for ch in chains:
        ch.close()
    return {"value": n * updates * steps / (total / 1000.0), "unit": UNIT, "chains": n, "graph": graph,
            "updates_per_chain_per_step": updates, "ms_per_step": total / steps,
            "launches_per_step": len(plan), "team_ctas_by_L": {str(k): sorted(v) for k, v in sorted(teams.items())},
            "shared_ctas": sum(1 for w, tc in plan for k in range(len(tc)) if tc[k] == 1 and k + 1 < len(tc)
                               and tc[k + 1] == 0),
            "lattice_counts": {str(int(L)): int((Ls == L).sum()) for L in sorted(set(Ls.tolist()))},
            "stencil_gbs": sum(bytes_u) * updates / (total / steps / 1000.0) / 1e9,
            "autotune_s": tune_s, "recursion": recursion, "compensated": compensated,
            "config": "64 chains, L uniform from {8,12,16,24,32} (seed 4), T uniform in [0.02, 0.2] t, "
                      "mu = -2t, M = 1024, FP32-mixed, spins uniform (seed = chain index)"}


def run_batching_clusters(stream, steps, warmup, updates, flush, graphs=True):
    """The 64-chain batching workload on thread-block clusters (proposal-vector
    recursion, FP32-mixed): each chain's lattice in the shared memory of the
    smallest cluster that holds it; a step runs `updates` updates of every
    chain."""
    import torch
    from paper_1303_6016_gb300 import batch
    chains, Ls, Ts = batch.c4_chains(M=1024, recursion="proposal")
    t0 = time.perf_counter()
    tuner = batch.ClusterTuner(M=1024, precision="fp32_mixed")
    runner = batch.ClusterRunner(chains, tuner, updates=updates)
    tune_s = time.perf_counter() - t0
    for _ in range(warmup):
        runner.run(updates)
    per = []
    for k in range(steps):
        flush.fill_(k)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        runner.run(updates)
        e.record()
        e.synchronize()
        per.append(s.elapsed_time(e))
    total = sum(per)
    n = len(chains)
    by_L = {str(int(L)): c for L, c in sorted(zip(Ls, runner.cluster_ctas))}
    # the same steps captured once in a CUDA graph (gfmc_plan_*) and replayed
    graph = None
    if graphs:
        from paper_1303_6016_gb300 import gfmc
        ordered, sizes = runner.ordered()
        with gfmc.Plan(ordered, [updates] * n, sizes, schedule="clusters") as plan:
            plan.launch(warmup)
            plan.sync(trace=False)
            perg = []
            for k in range(steps):
                flush.fill_(k)
                s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s.record()
                plan.launch(1)
                e.record()
                e.synchronize()
                perg.append(s.elapsed_time(e))
            plan.sync(trace=False)
        totg = sum(perg)
        graph = {"value": n * updates * steps / (totg / 1000.0), "unit": UNIT, "ms_per_step": totg / steps,
                 "note": "one CUDA graph launch per step (gfmc_plan_launch), no host work between steps"}
    for ch in chains:
        ch.close()
    _, bytes_u = zip(*[update_work(int(L), 1024, 4, 2) for L in Ls])
    return {"value": n * updates * steps / (total / 1000.0), "unit": UNIT, "chains": n,
            "updates_per_chain_per_step": updates, "ms_per_step": total / steps,
            "stencil_gbs": sum(bytes_u) * updates / (total / steps / 1000.0) / 1e9,
            "graph": graph,
            "cluster_ctas_by_L": by_L, "recursion": "proposal", "autotune_s": tune_s,
            "tuned_ms_per_step": runner.makespan * 1e3 if runner.makespan else None,
            "config": "the batching workload (64 chains, L from {8,12,16,24,32}, M = 1024, FP32-mixed), "
                      "each chain on one thread-block cluster holding its lattice in shared memory"}


def time_device(ch, stream, U, steps, warmup, flush, dist, sampler=None):
    """Device-timed steps: CUDA events on the chain's stream around each step,
    a 256 MiB L2 flush between steps outside the events."""
    import torch
    for _ in range(warmup):
        ch.updates_into(U)
    barrier(dist)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if sampler:
        sampler.start()
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(k)
        starts[k].record(stream)
        ch.updates_into(U)
        ends[k].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    barrier(dist)
    per = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    return per, clocks


def time_e2e(ch, stream, U, steps, spins0):
    """End to end through the public API with pinned host buffers: upload the
    chain state, run the block of updates with host traces, read the spins."""
    import numpy as np
    import torch
    N = ch.N
    h_spins = torch.empty((N, 2), dtype=torch.float64, pin_memory=True).numpy()
    h_out = torch.empty((N, 2), dtype=torch.float64, pin_memory=True).numpy()
    h_dec = torch.empty(U, dtype=torch.uint8, pin_memory=True).numpy()
    h_dom = torch.empty(U, dtype=torch.float64, pin_memory=True).numpy()
    h_spins[:] = spins0
    counter = ch.counter
    torch.cuda.synchronize()
    per = []
    for _ in range(steps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        ch.set_state(h_spins, counter)
        ch.updates_into(U, decisions=h_dec, d_omega=h_dom)
        ch.get_spins(h_out)
        e.record(stream)
        e.synchronize()
        per.append(s.elapsed_time(e))
        h_spins[:] = h_out
        counter += U
    h2d = N * 16
    d2h = U * (1 + 8) + N * 16 + 8 + 8
    assert np.isfinite(h_dom).all()
    return per, h2d, d2h


def cpu_baseline(L, M, spins, n_updates, threads):
    """The oracle on `threads` host threads (its site and node loops; results
    are bitwise the same for any count)."""
    from oracle import oracle as O
    O.build()
    O.set_threads(threads)
    t0 = time.perf_counter()
    O.updates(L, spins, n_updates, M, beta=20.0, chem=-2.0, seed=1)
    dt = time.perf_counter() - t0
    used = O.max_threads()
    return n_updates / dt, dt, used


def run_reference(args, rank, world, dist):
    """The oracle (plain C, FP64, OpenMP over all host threads) on the same
    workload: the reference arm, on rank 0 only."""
    if rank != 0:
        return 0
    from paper_1303_6016_gb300 import inputs
    L, M = args.L, args.M
    spins = inputs.uniform_sphere(L, 0)
    from oracle import oracle as O
    O.build()
    O.set_threads(os.cpu_count() or 1)
    cores = O.max_threads()
    U = 1
    per = []
    s = spins.copy()
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        res = O.updates(L, s, U, M, beta=20.0, chem=-2.0, seed=1, upd0=k * U)
        dt = time.perf_counter() - t0
        s = res["spins"]
        if k >= args.warmup:
            per.append(dt * 1000.0)
    ms = statistics.mean(per)
    value = U / (ms / 1000.0)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(L, M, U, "fp64"), l2="not applicable: the CPU oracle"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{U} update per step from the start of sweep 0 at L={L}, M={M}, "
                                   f"OpenMP over the oracle's site and node loops on {cores} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(L, M, U, precision):
    return {"workload": f"GFMC single chain, L={L} (N={L ** 3}) periodic cubic, M={M} Jackson moments, "
                        "t=1, beta=20/t, mu=-2t, spins uniform on the sphere (seed 0), sequential sweep, "
                        "Philox proposals (seed 1)",
            "L": L, "M": M, "updates_per_step": U, "precision": precision,
            "l2": "flushed between timed steps (256 MiB write); the chain's working set is L2-resident "
                  "within a step"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gfmc", choices=["gfmc", "reference"])
    ap.add_argument("--L", type=int, default=32)
    ap.add_argument("--M", type=int, default=1024)
    ap.add_argument("--updates-per-step", type=int, default=0)
    ap.add_argument("--mixed-updates-per-step", type=int, default=0)
    ap.add_argument("--cpu-updates", type=int, default=6)
    ap.add_argument("--cpu-updates-all", type=int, default=40)
    ap.add_argument("--sweeps-l32", type=int, default=0,
                    help="also time this many full FP32-mixed sweeps of the L=32 chain (each ~30 s)")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-latency", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-variant", action="store_true")
    ap.add_argument("--no-l16", action="store_true", help="skip the single-chain L=16 leg")
    ap.add_argument("--no-graph", action="store_true",
                    help="skip the CUDA-graph replays of the batch steps")
    ap.add_argument("--batch-updates", type=int, default=4)
    ap.add_argument("--latency-sweeps", type=int, default=5)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local, dist = dist_setup(args.gpus)
    if args.impl == "reference":
        return run_reference(args, rank, world, dist)

    import torch
    from paper_1303_6016_gb300 import build, gfmc, inputs
    if rank == 0 or world == 1:
        build.build()
    barrier(dist)
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    L, M, N = args.L, args.M, args.L ** 3
    spins = inputs.uniform_sphere(L, 0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    U = args.updates_per_step or 16
    Um = args.mixed_updates_per_step or 64
    peaks = load_peaks()

    # ---- FP64 headline ----
    ch = gfmc.Chain(L, spins, M=M, beta=20.0, mu=-2.0, seed=1, chain_id=rank, stream=stream.cuda_stream)
    sampler = ClockSampler(local)
    per, clocks = time_device(ch, stream, U, args.steps, args.warmup, flush, dist, sampler)
    total_ms = max_over_ranks(dist, sum(per))
    value = aggregate(world, args.steps, U, total_ms)
    ms_step = total_ms / args.steps
    flop_u, bytes_u = update_work(L, M, 8)
    flop_nz = update_flop_nonzero(L, M)
    launch_s = statistics.mean(per) / 1000.0
    achieved_tf = U * flop_nz / launch_s / 1e12
    derived_tf = alu_peak_tflops("fp64", clocks.get("sm_max_mhz") or 2070.0) if clocks else alu_peak_tflops("fp64")
    peak_tf = gfmc.fma_peak_tflops("fp64", repeats=3, stream=stream.cuda_stream)
    # what the FP64 pipe needs at the engine's occupancy (one CTA of 256 per SM)
    issue = {"chains16_warps8": gfmc.fp64_issue_rate(16, 8, stream=stream.cuda_stream),
             "chains1_warps4": gfmc.fp64_issue_rate(1, 4, stream=stream.cuda_stream),
             "chains4_warps8_lanes12": gfmc.fp64_issue_rate(4, 8, lanes=12, stream=stream.cuda_stream),
             "unit": "FP64 fma warp-lane slots per SM clock (gfmc_measure_fp64_issue)",
             "note": "one dependent chain on each of 4 warps keeps the pipe as busy as 16 chains on 8, and a "
                     "warp of 12 active lanes costs 32 lanes' slots: the engine's rate is set by its count of "
                     "warp-level FP64 instructions"}
    e2e_per, h2d, d2h = time_e2e(ch, stream, U, max(3, args.steps // 2), ch.get_spins())
    e2e_value = U / (statistics.mean(e2e_per) / 1000.0) * world
    vec_bytes = 2 * 7 * L ** 3 * 16
    footprint = {"device_bytes": ch.device_bytes, "vector_bytes": vec_bytes,
                 "beyond_vectors": ch.device_bytes - vec_bytes,
                 "note": "device memory of the FP64 chain's handle (gfmc_device_bytes); the Gram sums of the "
                         "doubling are one [M/2-1][112] fixed-point array whatever the number of CTAs"}
    ch.close()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(L, M, U, "fp64"), parallelism=f"replicas{world}"),
        "stencil_gbs": U * bytes_u / launch_s / 1e9,
        "latency_ms_per_update": {"p50": statistics.median(per) / U, "p99": sorted(per)[-1] / U},
        "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                     "frac": achieved_tf / peak_tf, "traffic": traffic_per_launch("fp64", U),
                     "traffic_unit": "bytes per launch (DRAM read + write, ncu)",
                     "flop_per_update": flop_nz,
                     "flop_note": "flop of the update without the terms that vanish by parity on the bipartite "
                                  "lattice (280 per site and step of the M/2-1 doubling steps at even L; the "
                                  "count with them, 791, gives flop_full_per_update)",
                     "flop_full_per_update": flop_u,
                     "peak_source": "measured in this run: gfmc_measure_fma_peak (own kernel, 16 independent "
                                    "double fma chains per thread, one CTA of 256 on every SM, best of 3, CUDA "
                                    "events; it retires the pipe's 2 warp-lane slots per SM clock, see "
                                    "fp64_issue)",
                     "peak_derived": derived_tf,
                     "peak_derived_source": "152 SMs x max SM clock x 2 FP64 FMA lanes per SM x 2 flop",
                     "flop_s8d_per_update": (M // 2) * L ** 3 * 830,
                     "frac_s8d": U * (M // 2) * L ** 3 * 830 / launch_s / 1e12 / peak_tf,
                     "s8d_note": "the survey's per-update count (M/2) N 830 counts the products that vanish by "
                                 "parity, which this engine does not execute; against it the fraction exceeds 1",
                     "fp64_issue": issue},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps,
        "clocks": clocks,
        "footprint": footprint,
    }

    # ---- FP32-mixed ----
    if not args.no_mixed:
        chm = gfmc.Chain(L, spins, M=M, beta=20.0, mu=-2.0, seed=1, chain_id=rank, precision="fp32_mixed",
                         stream=stream.cuda_stream)
        perm, clocks_m = time_device(chm, stream, Um, args.steps, args.warmup, flush, dist, ClockSampler(local))
        tot_m = max_over_ranks(dist, sum(perm))
        flop_m, bytes_m = update_work(L, M, 4)
        launch_m = statistics.mean(perm) / 1000.0
        gbs = Um * bytes_m / launch_m / 1e9
        l2 = l2_copy_gbs()
        line["fp32_mixed"] = {
            "value": aggregate(world, args.steps, Um, tot_m), "unit": UNIT, "updates_per_step": Um,
            "ms_per_step": tot_m / args.steps, "stencil_gbs": gbs,
            "latency_ms_per_update": {"p50": statistics.median(perm) / Um, "p99": sorted(perm)[-1] / Um},
            "roofline": {"bound": "l2", "achieved": gbs, "peak": l2, "unit": "GB/s",
                         "frac": gbs / l2, "traffic": traffic_per_launch("fp32_mixed", Um),
                         "peak_source": "measured in this run: graph-replayed copies of a 32 MiB "
                                        "L2-resident buffer (read + write bytes, CUDA events)",
                         "hbm_frac": gbs / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None},
            "alu_tflops": Um * flop_m / launch_m / 1e12, "clocks": clocks_m,
            "gpu_launches": args.steps,
        }
        if L == 32 and L % 2 == 0:
            # the vector-cluster engine's bound: its per-step exchange between CTAs,
            # measured alone (no arithmetic) in this run
            floor = gfmc.cluster_exchange_cycles(steps=2000, repeats=3, stream=stream.cuda_stream)
            mhz = (clocks_m or {}).get("sm_mhz") or 2070.0
            step_cycles = launch_m / Um / (M - 1) * mhz * 1e6
            line["fp32_mixed"]["exchange_floor"] = {
                "cycles_per_step": floor, "engine_cycles_per_step": step_cycles,
                "floor_over_step": floor / step_cycles,
                "updates_per_s_at_floor": mhz * 1e6 / (floor * (M - 1)),
                "note": "gfmc_measure_cluster_exchange: the engine's exchange pattern and volume (4 KB per CTA "
                        "and step over st.async + mbarrier in 4x4 tori of 16 CTAs, 7 clusters) with no "
                        "arithmetic; the engine takes M - 1 steps per update (moments read off the "
                        "recursion), engine cycles per step include the update's tail"}
        chm.close()

    if not args.no_l16:
        # the single-chain workload's smaller lattice: L=16 (N=4096), same M, both precisions
        L16, spins16 = 16, inputs.uniform_sphere(16, 0)
        l16 = {"L": L16, "M": M, "note": "single chain, uniform spins (seed 0), M=1024; the FP32-mixed chain "
                                          "runs the grid engine (the vector-cluster engine is for L=32)"}
        for prec, u16 in (("fp64", 64), ("fp32_mixed", 64)):
            c16 = gfmc.Chain(L16, spins16, M=M, beta=20.0, mu=-2.0, seed=1, chain_id=rank, precision=prec,
                             stream=stream.cuda_stream)
            per16, _ = time_device(c16, stream, u16, max(3, args.steps // 2), args.warmup, flush, dist)
            c16.close()
            tot16 = max_over_ranks(dist, sum(per16))
            _, b16 = update_work(L16, M, 8 if prec == "fp64" else 4)
            l16[prec] = {"value": aggregate(world, max(3, args.steps // 2), u16, tot16), "unit": UNIT,
                         "updates_per_step": u16, "ms_per_update": statistics.mean(per16) / u16,
                         "stencil_gbs": u16 * b16 / (statistics.mean(per16) / 1000.0) / 1e9}
        line["single_chain_L16"] = l16

    if not args.no_variant:
        # the paper's recursion on the proposal's vectors (o, v; o+v and o+iv by linearity)
        chv = gfmc.Chain(L, spins, M=M, beta=20.0, mu=-2.0, seed=1, chain_id=rank, recursion="proposal",
                         stream=stream.cuda_stream)
        Uv = 4 * U
        perv, clocks_v = time_device(chv, stream, Uv, args.steps, args.warmup, flush, dist, ClockSampler(local))
        totv = max_over_ranks(dist, sum(perv))
        chv.close()
        chm2 = gfmc.Chain(L, spins, M=M, beta=20.0, mu=-2.0, seed=1, chain_id=rank, recursion="proposal",
                          precision="fp32_mixed", stream=stream.cuda_stream)
        perv2, _ = time_device(chm2, stream, Um, args.steps, args.warmup, flush, dist)
        totv2 = max_over_ranks(dist, sum(perv2))
        chm2.close()
        line["proposal_recursion"] = {
            "note": "the paper's recursion on the proposal's vectors o, v (o+v, o+iv by linearity): "
                    "2 recursions + 8 real dot products per site and step instead of 7 + 112",
            "fp64": {"value": aggregate(world, args.steps, Uv, totv), "unit": UNIT, "updates_per_step": Uv,
                     "ms_per_update": totv / args.steps / Uv, "clocks": clocks_v},
            "fp32_mixed": {"value": aggregate(world, args.steps, Um, totv2), "unit": UNIT, "updates_per_step": Um,
                           "ms_per_update": totv2 / args.steps / Um}}

    if not args.no_batch:
        graphs = not args.no_graph
        line["batching"] = run_batching(stream, max(3, args.steps // 2), 3, args.batch_updates, flush,
                                        graphs=graphs)
        if not args.no_variant:
            line["batching_proposal_recursion"] = run_batching(stream, max(3, args.steps // 2), 3,
                                                               args.batch_updates, flush, "proposal", graphs)
            line["batching_clusters"] = run_batching_clusters(stream, max(3, args.steps // 2), 3,
                                                              args.batch_updates, flush, graphs)
            comp = run_batching(stream, max(3, args.steps // 2), 3, args.batch_updates, flush,
                                graphs=graphs, compensated=True)
            line["batching_compensated"] = {k: comp[k] for k in ("value", "unit", "ms_per_step", "graph",
                                                                 "launches_per_step", "compensated")}
            line["batching_compensated"]["note"] = ("the batching workload with Dot2 compensated Gram sums "
                                                    "(gfmc_options.compensated); the cost of the extra "
                                                    "accuracy against batching.value")

    if not args.no_mixed:
        # FP32-mixed against the FP64 path on the same chain: Delta Omega error per
        # update (target <= 1e-4 t) and moment error by band of n
        from paper_1303_6016_gb300 import precision_report
        prec = precision_report.run(L=L, Ms=(M,), n_sites=4)
        line["fp32_mixed"]["error_vs_fp64"] = [
            {"spins": r["spins"], "M": r["M"],
             **{name: {k: v[k] for k in ("domega_err_max", "domega_rel_err_max", "moment_err_by_n")}
                for name, v in r["variants"].items()}} for r in prec]
        line["fp32_mixed"]["error_vs_fp64_note"] = (
            "default: the vector-cluster engine (moments read off the recursion); grid_plain: the doubling's "
            "Gram products in FP32 warp sums; grid_compensated: the same with Dot2 products and sums")

    if not args.no_serving:
        from paper_1303_6016_gb300 import serving
        line["serving"] = serving.sweep(rates=(10, 100, 1000), seconds=3.0, K=2, drain_s=8.0)
        if not args.no_variant:
            line["serving_unit_vectors"] = serving.sweep(rates=(10, 100, 1000), seconds=3.0, K=2, drain_s=8.0,
                                                         recursion="unit_vectors")

    if not args.no_latency:
        line["sweep_latency"] = [sweep_latency(gfmc, inputs, stream, 8, M, prec, args.latency_sweeps)
                                 for prec in ("fp64", "fp32_mixed")]
        line["sweep_latency_note"] = ("full sequential sweeps of an 8^3 chain; at L=32 a sweep is "
                                      "32768 updates, i.e. 32768 x latency_ms_per_update")
        if args.sweeps_l32 > 0:
            line["sweep_latency_L32"] = sweep_latency(gfmc, inputs, stream, L, M, "fp32_mixed", args.sweeps_l32,
                                                      warmup=0)

    if rank == 0 and world == 1 and not args.no_cpu:
        ncores = os.cpu_count() or 1
        v, dt, used = cpu_baseline(L, M, spins, args.cpu_updates_all, ncores)
        v1, dt1, _ = cpu_baseline(L, M, spins, args.cpu_updates, 1)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": used, "kind": "oracle",
                                "sample": f"first {args.cpu_updates_all} updates of sweep 0 at L={L}, M={M} "
                                          f"({dt:.1f} s; plain C, FP64, OpenMP over the site and node loops "
                                          f"on {used} of {ncores} host threads)",
                                "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                                                  "sample": f"first {args.cpu_updates} updates of sweep 0 "
                                                            f"({dt1:.1f} s, one thread)"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
