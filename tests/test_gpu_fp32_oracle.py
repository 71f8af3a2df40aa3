"""FP32-mixed chains of every multi-chain schedule replayed by the oracle.

The batching and serving workloads run FP32-mixed chains; here each schedule
-- team batches, thread-block cluster batches, CUDA-graph plans of both, and
server jobs -- runs chains of the batching workload's lattice sizes (L = 8,
12, 16, 24, 32 at M = 1024) and the oracle (FP64) follows the GPU's decisions
update by update (Algorithm 1; independent chains, Sec. 3.2).

Tolerances (FP32 recursion vectors, FP64 above them):
  Delta Omega  <= 1e-4 t per update
  decisions    identical except where |exp(-beta dO) - u| < 1e-4
"""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_6016_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-4
TIE = 1e-4
M = 1024
SIZES = (8, 12, 16, 24, 32)
BETAS = (50.0, 12.0, 20.0, 8.0, 30.0)  # temperatures in [0.02 t, 0.2 t]


@pytest.fixture(scope="module")
def G():
    from paper_1303_6016_gb300 import build, gfmc
    build.build()
    gfmc.load()
    return gfmc


def replay(L, sp, beta, seed, chain_id, decisions, d_omega, upd0=0):
    n = decisions.size
    res = O.updates(L, sp, n, M, beta=beta, chem=-2.0, seed=seed, chain_id=chain_id, upd0=upd0,
                    forced=decisions.astype(np.int8))
    own = res["ratio"] > res["u"]
    for q in range(n):
        assert abs(d_omega[q] - res["d_omega"][q]) <= TOL, (L, q, d_omega[q], res["d_omega"][q])
        if own[q] != bool(decisions[q]):
            assert abs(res["ratio"][q] - res["u"][q]) < TIE, (L, q)
    return res


def make_chains(G, recursion, seed):
    chains, sps = [], []
    for c, (L, beta) in enumerate(zip(SIZES, BETAS)):
        sp = inputs.uniform_sphere(L, 60 + c)
        sps.append(sp)
        chains.append(G.Chain(L, sp, M=M, beta=beta, mu=-2.0, precision="fp32_mixed", seed=seed, chain_id=c,
                              recursion=recursion))
    return chains, sps


def test_team_batch(G):
    """One launch, a team of CTAs per chain (one-CTA teams keep the small
    lattices in shared memory), the team sizes the batch autotuner picks."""
    chains, sps = make_chains(G, "unit_vectors", seed=4)
    n = 3
    outs = G.run_batch(chains, n, team_ctas=[1, 1, 1, 2, 6])
    for c, L in enumerate(SIZES):
        replay(L, sps[c], BETAS[c], 4, c, outs[c]["decisions"], outs[c]["d_omega"])
        chains[c].close()


def test_cluster_batch(G):
    """Chains on the proposal's vectors, each on one thread-block cluster that
    holds its lattice in shared memory (the cluster sizes of the tuner)."""
    chains, sps = make_chains(G, "proposal", seed=5)
    n = 3
    outs = G.run_clusters(chains, n, cluster_ctas=[4, 2, 2, 8, 8])
    for c, L in enumerate(SIZES):
        replay(L, sps[c], BETAS[c], 5, c, outs[c]["decisions"], outs[c]["d_omega"])
        chains[c].close()


@pytest.mark.parametrize("schedule,recursion,ctas", [("teams", "unit_vectors", [1, 1, 1, 2, 6]),
                                                     ("clusters", "proposal", [4, 2, 2, 8, 8])])
def test_graph_plans(G, schedule, recursion, ctas):
    """A step captured in a CUDA graph and replayed twice; the two steps'
    traces are replayed by the oracle from the start."""
    chains, sps = make_chains(G, recursion, seed=6)
    per = 2
    traces = [([], []) for _ in SIZES]
    with G.Plan(chains, [per] * len(SIZES), ctas, schedule=schedule) as plan:
        for _ in range(2):
            plan.launch(1)
            for c, r in enumerate(plan.sync()):
                traces[c][0].append(r["decisions"].copy())
                traces[c][1].append(r["d_omega"].copy())
    for c, L in enumerate(SIZES):
        dec, dom = np.concatenate(traces[c][0]), np.concatenate(traces[c][1])
        replay(L, sps[c], BETAS[c], 6, c, dec, dom)
        chains[c].close()


def test_server_jobs(G):
    """FP32-mixed jobs of three lattice sizes side by side in the serving loop."""
    sizes, betas = (12, 24, 32), (12.0, 8.0, 30.0)
    chains, sps = [], []
    for c, (L, beta) in enumerate(zip(sizes, betas)):
        sp = inputs.uniform_sphere(L, 70 + c)
        sps.append(sp)
        chains.append(G.Chain(L, sp, M=M, beta=beta, mu=-2.0, precision="fp32_mixed", seed=7, chain_id=c))
    n = 3
    with G.Server([4, 8, 16], max_M=M) as srv:
        for k, ch in enumerate(chains):
            srv.submit(k, ch, n)
        res, t0 = {}, time.time()
        while len(res) < len(sizes):
            for k in range(len(sizes)):
                if k not in res:
                    r = srv.poll(k)
                    if r is not None:
                        res[k] = r
            assert time.time() - t0 < 120.0, "server jobs did not finish"
            time.sleep(0.001)
    for c, L in enumerate(sizes):
        replay(L, sps[c], betas[c], 7, c, res[c]["decisions"], res[c]["d_omega"])
        chains[c].close()
