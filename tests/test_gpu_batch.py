"""Batched chains (one launch, one team of CTAs per chain) against the oracle
and against the same chains run alone.

Tolerances as in test_gpu_parity: FP64 Delta Omega 1e-10 |dO| + 1e-13 a with
identical decisions except near ties |exp(-beta dO) - u| < 1e-9 (the oracle
follows the GPU's decisions); FP32-mixed Delta Omega 1e-4 t.
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


def oracle_replay(L, sp, M, beta, seed, chain_id, out):
    n = out["decisions"].size
    res = O.updates(L, sp, n, M, beta=beta, chem=-2.0, seed=seed, chain_id=chain_id,
                    forced=out["decisions"].astype(np.int8))
    own = res["ratio"] > res["u"]
    for q in range(n):
        assert abs(out["d_omega"][q] - res["d_omega"][q]) <= dom_tol(res["d_omega"][q]), (L, q)
        if own[q] != bool(out["decisions"][q]):
            assert abs(res["ratio"][q] - res["u"][q]) < 1e-9


def test_fp64_batch_matches_oracle_per_chain(G):
    """Chains of different L, beta and team size in one launch; each chain's
    trace is replayed by the oracle."""
    specs = [(4, 20.0, 1), (5, 8.0, 2), (6, 12.0, 1), (8, 20.0, 3), (8, 5.0, 1), (12, 15.0, 2)]
    M = 64
    chains, sps = [], []
    for c, (L, beta, _) in enumerate(specs):
        sp = inputs.uniform_sphere(L, 10 + c)
        sps.append(sp)
        chains.append(G.Chain(L, sp, M=M, beta=beta, mu=-2.0, seed=3, chain_id=c))
    n = [L ** 3 if L <= 5 else 60 for (L, _, _) in specs]
    outs = G.run_batch(chains, n, team_ctas=[t for (_, _, t) in specs])
    for c, (L, beta, _) in enumerate(specs):
        oracle_replay(L, sps[c], M, beta, 3, c, outs[c])
        assert chains[c].counter == n[c]
        assert outs[c]["n_accepted"] == int(outs[c]["decisions"].sum())
    for ch in chains:
        ch.close()


def test_batch_continues_where_single_chain_stops(G):
    """The batch starts from each chain's counter and state: run alone for a
    while, then in a batch, equals the oracle for the whole run."""
    L, M = 6, 64
    sp = inputs.uniform_sphere(L, 33)
    ch = G.Chain(L, sp, M=M, beta=20.0, mu=-2.0, seed=9, chain_id=4)
    first = ch.updates(50)
    other = G.Chain(4, inputs.uniform_sphere(4, 1), M=M, beta=20.0, mu=-2.0, seed=9, chain_id=5)
    second = G.run_batch([ch, other], [70, 10], team_ctas=[2, 1])[0]
    full = {"decisions": np.concatenate([first["decisions"], second["decisions"]]),
            "d_omega": np.concatenate([first["d_omega"], second["d_omega"]])}
    oracle_replay(L, sp, M, 20.0, 9, 4, full)
    ch.close()
    other.close()


def test_fp32_alone_equals_in_the_mix(G):
    """FP32-mixed chains: in a mixed batch (shared-memory and L2 teams) each
    gives the Delta Omega trace it gives alone, within 1e-4 t."""
    specs = [(8, 1), (12, 1), (16, 4), (10, 2)]
    M = 128
    alone, mix = [], []
    for c, (L, tc) in enumerate(specs):
        sp = inputs.uniform_sphere(L, 20 + c)
        with G.Chain(L, sp, M=M, precision="fp32_mixed", seed=2, chain_id=c) as ch:
            alone.append(ch.updates(40))
        mix.append(G.Chain(L, sp, M=M, precision="fp32_mixed", seed=2, chain_id=c))
    outs = G.run_batch(mix, 40, team_ctas=[t for (_, t) in specs])
    for c in range(len(specs)):
        d = np.abs(outs[c]["d_omega"] - alone[c]["d_omega"])
        same = outs[c]["decisions"] == alone[c]["decisions"]
        # traces may only part where a decision is a near tie; up to there they agree
        k = int(np.argmin(same)) if not same.all() else same.size
        assert d[:k].max() <= 1e-4, (c, d[:k].max())
        assert k >= 10
    for ch in mix:
        ch.close()


def test_shared_memory_team_equals_global_team(G):
    L, M = 8, 128
    sp = inputs.uniform_sphere(L, 44)
    a = G.Chain(L, sp, M=M, precision="fp32_mixed", seed=5)
    b = G.Chain(L, sp, M=M, precision="fp32_mixed", seed=5)
    oa, ob = G.run_batch([a, b], 30, team_ctas=[1, 2])  # team of 1: lattice in shared memory
    k = int(np.argmin(oa["decisions"] == ob["decisions"])) if (oa["decisions"] != ob["decisions"]).any() else 30
    assert np.abs(oa["d_omega"][:k] - ob["d_omega"][:k]).max() <= 1e-5
    a.close()
    b.close()


def test_batch_rejects_oversubscription_and_bad_team(G):
    L, M = 32, 64
    sp = inputs.uniform_sphere(L, 0)
    chains = [G.Chain(L, sp, M=M, precision="fp32_mixed", chain_id=c) for c in range(2)]
    with pytest.raises(G.GfmcError) as e:
        G.run_batch(chains, 1, team_ctas=[152, 152])  # more CTAs than the device holds at once
    assert e.value.status == G.GFMC_EINVAL
    with pytest.raises(G.GfmcError) as e:
        G.run_batch(chains, 1, team_ctas=[0, 1])  # a shared team needs a one-CTA team before it
    assert e.value.status == G.GFMC_EINVAL
    with pytest.raises(G.GfmcError) as e:
        G.run_batch(chains, 1, team_ctas=[2, 0])  # ... not a two-CTA one
    assert e.value.status == G.GFMC_EINVAL
    prop = G.Chain(8, inputs.uniform_sphere(8, 0), M=M, precision="fp32_mixed", recursion="proposal")
    with pytest.raises(G.GfmcError) as e:
        G.run_batch([chains[0], prop], 1, team_ctas=[1, 0])  # ... nor one on another recursion
    assert e.value.status == G.GFMC_EINVAL
    assert all(ch.counter == 0 for ch in chains + [prop])
    for ch in chains + [prop]:
        ch.close()


@pytest.mark.parametrize("prec,recursion", [("fp32_mixed", "unit_vectors"), ("fp64", "unit_vectors"),
                                            ("fp32_mixed", "proposal")])
def test_chains_sharing_a_cta_equal_the_chains_alone(G, prec, recursion):
    """Chains with team size 0 run after the chain before them on its one CTA:
    each gives bitwise the trace and spins it gives alone on a one-CTA team,
    with multi-CTA teams before, between and after the shared ones (lattices
    in shared memory and in global memory, ragged update counts)."""
    M = 64
    specs = [(6, 2, 5), (8, 1, 7), (5, 0, 4), (12, 0, 9), (4, 0, 3), (10, 3, 6), (7, 1, 8), (9, 0, 5), (6, 2, 4)]
    mk = lambda c, L: G.Chain(L, inputs.uniform_sphere(L, 60 + c), M=M, precision=prec, seed=9, chain_id=c,
                              recursion=recursion, beta=12.0)
    mix = [mk(c, L) for c, (L, _, _) in enumerate(specs)]
    outs = G.run_batch(mix, [n for (_, _, n) in specs], team_ctas=[t for (_, t, _) in specs])
    for c, (L, t, n) in enumerate(specs):
        with mk(c, L) as alone:
            ref = G.run_batch([alone], [n], team_ctas=[max(t, 1)])[0]
            spins = alone.get_spins()
        assert np.array_equal(outs[c]["decisions"], ref["decisions"]), c
        assert np.array_equal(outs[c]["d_omega"], ref["d_omega"]), c
        assert np.array_equal(mix[c].get_spins(), spins), c
        assert mix[c].counter == n
    for ch in mix:
        ch.close()


def test_batch_plan_with_shared_ctas_equals_calls(G):
    """A graph-captured step of a batch with a shared one-CTA team equals the
    same step run by gfmc_run_batch."""
    M, n = 64, [5, 3, 4, 6]
    specs = [(8, 2), (6, 1), (5, 0), (7, 0)]
    mk = lambda c, L: G.Chain(L, inputs.uniform_sphere(L, 80 + c), M=M, precision="fp32_mixed", seed=2,
                              chain_id=c)
    ref = [mk(c, L) for c, (L, _) in enumerate(specs)]
    got = [mk(c, L) for c, (L, _) in enumerate(specs)]
    tcs = [t for (_, t) in specs]
    for _ in range(2):
        last = G.run_batch(ref, n, team_ctas=tcs)
    with G.Plan(got, n, tcs, schedule="teams") as plan:
        plan.launch(2)
        out = plan.sync()
    for c in range(len(specs)):
        assert np.array_equal(out[c]["d_omega"], last[c]["d_omega"]), c
        assert np.array_equal(got[c].get_spins(), ref[c].get_spins()), c
    for ch in ref + got:
        ch.close()


def test_batch_magnetisation_is_the_definition(G):
    """After a full sweep the engine's |sum_i S_i| / N equals the value computed
    here from the spins read back (Algorithm 1, the measurement line)."""
    L, M = 5, 64
    ch = G.Chain(L, inputs.uniform_sphere(L, 3), M=M, seed=4)
    out = G.run_batch([ch], [2 * L ** 3], team_ctas=[2])[0]
    assert out["magnetization"].shape == (2,)
    s = ch.get_spins()
    v = np.stack([np.sin(s[:, 0]) * np.cos(s[:, 1]), np.sin(s[:, 0]) * np.sin(s[:, 1]), np.cos(s[:, 0])], 1)
    assert out["magnetization"][-1] == pytest.approx(np.linalg.norm(v.sum(0)) / L ** 3, abs=1e-13)
    ch.close()


def test_temperature_scan_orders_at_low_temperature(G):
    """From a ferromagnetic start the chain stays ordered far below the ordering
    temperature and disorders far above it (Algorithm 1, Sec. 4)."""
    from paper_1303_6016_gb300 import mt_scan
    res = mt_scan.scan(Ls=(4,), Ts=(0.02, 2.0), sweeps=14, warmup=6, M=64, start="cold")
    m = {p["T"]: p["M_mean"] for p in res["points"]}
    assert m[0.02] > 0.8 and m[2.0] < 0.4, m


def test_proposal_recursion_batch_matches_oracle(G):
    """Chains with the recursion on the proposal's vectors, in one batch with
    unit-vector chains, shared-memory and L2 teams; each replayed by the oracle."""
    specs = [(4, 20.0, 1, "proposal"), (6, 12.0, 2, "proposal"), (8, 20.0, 1, "unit_vectors"),
             (8, 9.0, 3, "proposal"), (12, 15.0, 1, "proposal")]
    M = 64
    chains, sps = [], []
    for c, (L, beta, _, rec) in enumerate(specs):
        sp = inputs.uniform_sphere(L, 60 + c)
        sps.append(sp)
        chains.append(G.Chain(L, sp, M=M, beta=beta, mu=-2.0, seed=4, chain_id=c, recursion=rec))
    n = 50
    outs = G.run_batch(chains, n, team_ctas=[t for (_, _, t, _) in specs])
    for c, (L, beta, _, _) in enumerate(specs):
        oracle_replay(L, sps[c], M, beta, 4, c, outs[c])
    for ch in chains:
        ch.close()
