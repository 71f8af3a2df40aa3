"""Serving: Poisson-arrival requests over a pool of chains, continuous batching.

A request asks to continue one chain by K updates.  Chains are kept resident
on the GPU across requests; a chain becomes resident (is created) when its
first request is admitted and its device footprint fits the HBM budget --
otherwise the request waits.  Admitted requests go to a free slot of the
device-resident request loop (``gfmc.Server``), chosen by the chain's lattice
size, so requests that arrive while others run start as soon as a slot and
their chain are free, and their work overlaps on the device.

    python -m paper_1303_6016_gb300.serving --rates 10 100 1000 --seconds 6

Jobs compute Delta Omega and decisions only, so the chains use the recursion
on the proposal's vectors by default (identical results, see gfmc.h).

Reported per arrival rate: requests completed, p50 / p99 latency (arrival to
completion, host clock), aggregate spin updates/s, requests left waiting when
admission stops (``drain`` seconds after the last arrival).
"""
from __future__ import annotations

import argparse
import json
import math
import time
from collections import deque

import numpy as np

from . import gfmc, inputs

# Slots of the request loop (CTAs each); 144 of the 152 SMs, the rest stay free
# for the set-up kernels of chains created while the server runs.
SLOTS = [32] + [16] * 2 + [8] * 6 + [4] * 6 + [2] * 4


def job_work(L: int, M: int, precision: str) -> float:
    """Relative cost of one update: sites x recursion steps, FP64 weighted by
    the FP64/FP32 throughput ratio of the team engine (about 4)."""
    return L ** 3 * M * (4.0 if precision == "fp64" else 1.0)


def preferred_team(L: int, M: int = 1024, precision: str = "fp32_mixed") -> int:
    """Slot size for a job: the costliest jobs (FP64 at the largest L and M)
    get the widest slot so that they do not set the tail latency alone."""
    w = job_work(L, M, precision)
    if w >= 2.0e8:
        return 32
    if w >= 4.0e7:
        return 16
    if w >= 1.0e7:
        return 8
    if w >= 2.5e6:
        return 4
    return 2


def footprint(L: int, M: int, precision: str) -> int:
    """Device bytes of one chain before it is created (the allocations of
    gfmc_create: spins and bonds, the two recursion buffers, the Gram sums
    (M/2 - 1) x 112 x 8 bytes, moments and tables); once created, the chain's
    own count (Chain.device_bytes) replaces the estimate."""
    N = L ** 3
    vec = 16 if precision == "fp64" else 8
    return (16 * N + 36 * N + 14 * N * vec + (M // 2 - 1) * 112 * 8 + 49 * M * 16 + 200 * M
            + 24 * 1024 + 3 * 1024 * 9 + 64 * 1024)


def pool_specs(n: int = 24, seed: int = 5, Ls=range(8, 49), Ms=(512, 1024, 2048)):
    rng = np.random.default_rng(seed)
    Ls = list(Ls)
    return [{"L": int(rng.choice(Ls)), "M": int(rng.choice(Ms)),
             "precision": "fp64" if rng.random() < 0.5 else "fp32_mixed", "chain_id": c} for c in range(n)]


def arrivals(rate: float, seconds: float, n_chains: int, seed: int = 5):
    rng = np.random.default_rng(seed + int(rate))
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= seconds:
            return out
        out.append((t, int(rng.integers(n_chains))))


class Scheduler:
    def __init__(self, specs, hbm_budget: float, K: int = 2, slots=SLOTS, max_M: int = 2048,
                 recursion: str = "proposal"):
        self.specs = specs
        self.recursion = recursion
        self.K = K
        self.budget = hbm_budget
        self.used = 0.0
        self.chains = {}
        self.busy_chain = set()
        self.slots = list(slots)
        self.free = set(range(len(self.slots)))
        self.running = {}  # slot -> (request arrival time, chain index)
        self.server = gfmc.Server(self.slots, max_M=max_M)

    def close(self):
        self.server.close()
        for ch in self.chains.values():
            ch.close()

    def _resident(self, c):
        if c in self.chains:
            return True
        sp = self.specs[c]
        fb = footprint(sp["L"], sp["M"], sp["precision"])
        if self.used + fb > self.budget:
            return False
        self.chains[c] = gfmc.Chain(sp["L"], inputs.uniform_sphere(sp["L"], 100 + c), M=sp["M"],
                                    precision=sp["precision"], beta=20.0, mu=-2.0, seed=1, chain_id=c,
                                    stream=0, recursion=self.recursion)
        self.used += self.chains[c].device_bytes
        return True

    def _slot_for(self, c):
        sp = self.specs[c]
        L = sp["L"]
        want = preferred_team(L, sp["M"], sp["precision"])
        cand = sorted((s for s in self.free if self.slots[s] <= L ** 3),
                      key=lambda s: (abs(self.slots[s] - want), -self.slots[s]))
        return cand[0] if cand else None

    def run(self, reqs, seconds: float, drain_s: float = 120.0):
        waiting = deque()
        lat, done_updates, i = [], 0, 0
        t0 = time.perf_counter()
        while True:
            now = time.perf_counter() - t0
            while i < len(reqs) and reqs[i][0] <= now:
                waiting.append(reqs[i])
                i += 1
            admitting = now <= seconds + drain_s
            # admit in arrival order; a request whose chain is busy or not yet
            # resident waits without blocking the ones behind it
            for _ in range(len(waiting) if admitting else 0):
                t_arr, c = waiting.popleft()
                if c in self.busy_chain or not self._resident(c):
                    waiting.append((t_arr, c))
                    continue
                s = self._slot_for(c)
                if s is None:
                    waiting.append((t_arr, c))
                    continue
                self.server.submit(s, self.chains[c], self.K, trace=False)
                self.free.discard(s)
                self.busy_chain.add(c)
                self.running[s] = (t_arr, c)
            for s in list(self.running):
                if self.server.poll(s) is not None:
                    t_arr, c = self.running.pop(s)
                    lat.append(time.perf_counter() - t0 - t_arr)
                    done_updates += self.K
                    self.free.add(s)
                    self.busy_chain.discard(c)
            if not self.running and i >= len(reqs) and (not waiting or not admitting):
                break
            time.sleep(0.0005)
        elapsed = time.perf_counter() - t0
        lat.sort()

        def pct(p):
            return lat[min(len(lat) - 1, max(0, int(math.ceil(p * len(lat))) - 1))] if lat else None

        return {"requests": len(reqs), "completed": len(lat), "left_waiting": len(waiting),
                "p50_s": pct(0.50), "p99_s": pct(0.99), "updates_per_s": done_updates / elapsed,
                "elapsed_s": elapsed, "resident_chains": len(self.chains), "hbm_used_gb": self.used / 1e9}


def sweep(rates=(10, 100, 1000), seconds: float = 6.0, K: int = 2, n_chains: int = 24,
          hbm_budget_gb: float = 4.0, drain_s: float = 30.0, recursion: str = "proposal"):
    specs = pool_specs(n_chains)
    out = []
    for r in rates:
        sch = Scheduler(specs, hbm_budget_gb * 1e9, K=K, recursion=recursion)
        try:
            res = sch.run(arrivals(r, seconds, n_chains), seconds, drain_s)
        finally:
            sch.close()
        res["rate_req_s"] = r
        out.append(res)
    return {"requests": f"continue one of {n_chains} chains by K={K} updates; L uniform in 8..48, "
                        "M in {512,1024,2048}, FP64 or FP32-mixed 50/50 (seed 5); Poisson arrivals",
            "slots": SLOTS, "hbm_budget_gb": hbm_budget_gb, "recursion": recursion, "results": out}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--rates", type=float, nargs="+", default=[10, 100, 1000])
    ap.add_argument("--seconds", type=float, default=6.0)
    ap.add_argument("--K", type=int, default=2)
    ap.add_argument("--chains", type=int, default=24)
    ap.add_argument("--hbm-gb", type=float, default=4.0)
    ap.add_argument("--drain", type=float, default=30.0)
    ap.add_argument("--recursion", default="proposal", choices=["proposal", "unit_vectors"])
    a = ap.parse_args(argv)
    from . import build
    build.build()
    print(json.dumps(sweep(a.rates, a.seconds, a.K, a.chains, a.hbm_gb, a.drain, a.recursion)))


if __name__ == "__main__":
    main()
