"""Batch plans: one step of a batch captured in a CUDA graph (gfmc_plan_*).

A plan's steps run the same kernels on the same inputs as gfmc_run_batch /
gfmc_run_clusters called once per step, so the traces and the spins must be
bitwise equal to that step-by-step run; FP64 chains are also replayed by the
oracle (Delta Omega 1e-10 |dO| + 1e-13 a, decisions identical except near
ties |exp(-beta dO) - u| < 1e-9).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_6016_gb300 import inputs

pytestmark = pytest.mark.gpu

A = 6.05


def dom_tol(ref):
    return 1e-10 * abs(ref) + 1e-13 * A


@pytest.fixture(scope="module")
def G():
    from paper_1303_6016_gb300 import build, gfmc
    build.build()
    gfmc.load()
    return gfmc


def make(G, specs, M, recursion):
    return [G.Chain(L, inputs.uniform_sphere(L, s), M=M, precision=prec, beta=15.0, mu=-2.0, seed=3, chain_id=c,
                    recursion=recursion) for c, (L, prec, s) in enumerate(specs)]


def oracle_replay(L, sp, M, dec, dom, seed, chain_id, beta=15.0):
    n = dec.size
    res = O.updates(L, sp, n, M, beta=beta, chem=-2.0, seed=seed, chain_id=chain_id, forced=dec.astype(np.int8))
    own = res["ratio"] > res["u"]
    for q in range(n):
        assert abs(dom[q] - res["d_omega"][q]) <= dom_tol(res["d_omega"][q]), (q, dom[q], res["d_omega"][q])
        if own[q] != bool(dec[q]):
            assert abs(res["ratio"][q] - res["u"][q]) < 1e-9
    return res


@pytest.mark.parametrize("schedule", ["clusters", "teams"])
def test_plan_steps_equal_step_by_step_calls_and_the_oracle(G, schedule):
    M, steps = 64, 3
    if schedule == "clusters":
        specs = [(6, "fp64", 61), (8, "fp64", 62), (8, "fp32_mixed", 63)]
        ctas, recursion, run = [1, 2, 1], "proposal", G.run_clusters
    else:
        specs = [(6, "fp32_mixed", 61), (8, "fp32_mixed", 62), (5, "fp32_mixed", 63)]
        ctas, recursion, run = [2, 1, 1], "unit_vectors", G.run_batch
    n = [10, 8, 12]
    ref, got = make(G, specs, M, recursion), make(G, specs, M, recursion)
    ref_steps = [run(ref, n, ctas) for _ in range(steps)]
    traces = []
    with G.Plan(got, n, ctas, schedule=schedule) as plan:
        for _ in range(steps):
            plan.launch(1)
            traces.append(plan.sync())
    for c in range(len(specs)):
        for k in range(steps):
            assert np.array_equal(traces[k][c]["decisions"], ref_steps[k][c]["decisions"]), (c, k)
            assert np.array_equal(traces[k][c]["d_omega"], ref_steps[k][c]["d_omega"]), (c, k)
        assert np.array_equal(got[c].get_spins(), ref[c].get_spins())
        assert got[c].counter == ref[c].counter == steps * n[c]
        L, prec, s = specs[c]
        if prec == "fp64":
            dec = np.concatenate([traces[k][c]["decisions"] for k in range(steps)])
            dom = np.concatenate([traces[k][c]["d_omega"] for k in range(steps)])
            oracle_replay(L, inputs.uniform_sphere(L, s), M, dec, dom, seed=3, chain_id=c)
    for ch in ref + got:
        ch.close()


def test_many_steps_in_one_launch(G):
    """Steps enqueued back to back (no host work between them) end where the
    same number of separate calls ends; sync returns the last step."""
    M, steps, n = 64, 5, [6, 4]
    specs = [(8, "fp32_mixed", 71), (6, "fp64", 72)]
    ref, got = make(G, specs, M, "proposal"), make(G, specs, M, "proposal")
    for _ in range(steps):
        last = G.run_clusters(ref, n, [1, 1])
    with G.Plan(got, n, [1, 1], schedule="clusters") as plan:
        plan.launch(steps)
        out = plan.sync()
    for c in range(len(specs)):
        assert np.array_equal(out[c]["d_omega"], last[c]["d_omega"])
        assert np.array_equal(got[c].get_spins(), ref[c].get_spins())
        assert got[c].counter == steps * n[c]
    for ch in ref + got:
        ch.close()


def test_plan_owns_its_chains(G):
    from paper_1303_6016_gb300.gfmc import GfmcError
    chains = make(G, [(6, "fp64", 81)], 64, "proposal")
    plan = G.Plan(chains, [4], [1], schedule="clusters")
    with pytest.raises(GfmcError, match="belongs to a plan"):
        G.Plan(chains, [4], [1], schedule="clusters")
    plan.close()
    with G.Plan(chains, [4], [1], schedule="clusters") as again:  # released by destroy
        again.launch(1)
        again.sync()
    chains[0].close()
