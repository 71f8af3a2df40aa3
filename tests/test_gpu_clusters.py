"""Chains on thread-block clusters (gfmc_run_clusters): the lattice of a chain
in the distributed shared memory of one cluster, recursion on the proposal's
vectors.

FP64 chains are replayed by the oracle (Delta Omega 1e-10 |dO| + 1e-13 a,
decisions identical except near ties |exp(-beta dO) - u| < 1e-9); FP32-mixed
chains give the Delta Omega trace the same chain gives alone on the
single-chain engine within 1e-4 t, up to the first decision that parts at a
near tie.
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


def agree_until_tie(a, b, tol, min_k):
    same = a["decisions"] == b["decisions"]
    k = same.size if same.all() else int(np.argmin(same))
    assert k >= min_k
    if k:
        assert np.abs(a["d_omega"][:k] - b["d_omega"][:k]).max() <= tol


def test_fp64_clusters_match_oracle_at_every_cluster_size(G):
    """Every cluster size, slabs of 1 to 4 z-planes per CTA, several groups in
    flight at once; each chain replayed by the oracle."""
    specs = [(4, 1, 20.0), (4, 2, 10.0), (4, 4, 20.0), (8, 8, 15.0), (16, 16, 20.0),
             (6, 2, 12.0), (12, 4, 20.0), (8, 1, 9.0), (16, 4, 12.0)]
    M, n = 64, 40
    chains, sps = [], []
    for c, (L, _, beta) in enumerate(specs):
        sp = inputs.uniform_sphere(L, 70 + c)
        sps.append(sp)
        chains.append(G.Chain(L, sp, M=M, beta=beta, mu=-2.0, seed=7, chain_id=c, recursion="proposal"))
    outs = G.run_clusters(chains, n, [C for (_, C, _) in specs])
    for c, (L, _, beta) in enumerate(specs):
        oracle_replay(L, sps[c], M, beta, 7, c, outs[c])
        assert chains[c].counter == n
        assert outs[c]["n_accepted"] == int(outs[c]["decisions"].sum())
    for ch in chains:
        ch.close()


def test_clusters_continue_a_chain_and_a_full_sweep_measures(G):
    """A chain run alone, then on a cluster, then again alone, is the oracle's
    chain for the whole run; the magnetisation after each full sweep is the
    definition evaluated on the spins read back."""
    L, M = 4, 64
    sp = inputs.uniform_sphere(L, 8)
    ch = G.Chain(L, sp, M=M, beta=20.0, mu=-2.0, seed=2, chain_id=1, recursion="proposal")
    first = ch.updates(20)
    second = G.run_clusters([ch], [2 * L ** 3 - 20], [4])[0]
    third = ch.updates(15)
    full = {k: np.concatenate([first[k], second[k], third[k]]) for k in ("decisions", "d_omega")}
    oracle_replay(L, sp, M, 20.0, 2, 1, full)
    ch.close()

    ch = G.Chain(L, sp, M=M, beta=20.0, mu=-2.0, seed=2, chain_id=1, recursion="proposal")
    out = G.run_clusters([ch], [2 * L ** 3], [2])[0]
    assert out["magnetization"].shape == (2,)
    s = ch.get_spins()
    v = np.stack([np.sin(s[:, 0]) * np.cos(s[:, 1]), np.sin(s[:, 0]) * np.sin(s[:, 1]), np.cos(s[:, 0])], 1)
    assert out["magnetization"][-1] == pytest.approx(np.linalg.norm(v.sum(0)) / L ** 3, abs=1e-13)
    ch.close()


def test_fp32_clusters_equal_the_chain_alone(G):
    """FP32-mixed chains on clusters of 1 to 16 CTAs against the same chains on
    the single-chain engine."""
    specs = [(8, 1), (8, 4), (12, 4), (16, 1), (16, 2), (16, 8), (16, 16)]
    M, n = 128, 40
    mix, alone = [], []
    for c, (L, _) in enumerate(specs):
        sp = inputs.uniform_sphere(L, 30 + c)
        with G.Chain(L, sp, M=M, precision="fp32_mixed", seed=2, chain_id=c, recursion="proposal") as ch:
            alone.append(ch.updates(n))
        mix.append(G.Chain(L, sp, M=M, precision="fp32_mixed", seed=2, chain_id=c, recursion="proposal"))
    outs = G.run_clusters(mix, n, [C for (_, C) in specs])
    for c in range(len(specs)):
        agree_until_tie(outs[c], alone[c], 1e-4, 10)
    for ch in mix:
        ch.close()


def test_full_size_lattice_on_clusters_of_8_and_16(G):
    """The L=32, M=1024 lattice held by a 16-CTA cluster (2048 sites per CTA)
    and by an 8-CTA cluster (4096 sites, the shared memory nearly full),
    FP32-mixed, against the single-chain engine; FP64 L=24 against the oracle
    for its first updates (8 CTAs of 3 planes)."""
    L, M, n = 32, 1024, 6
    sp = inputs.uniform_sphere(L, 0)
    with G.Chain(L, sp, M=M, precision="fp32_mixed", seed=1, recursion="proposal") as ch:
        alone = ch.updates(n)
    for C in (16, 8):
        with G.Chain(L, sp, M=M, precision="fp32_mixed", seed=1, recursion="proposal") as ch:
            out = G.run_clusters([ch], n, [C])[0]
        agree_until_tie(out, alone, 1e-4, 3)

    L, M, n = 24, 512, 3
    sp = inputs.uniform_sphere(L, 5)
    with G.Chain(L, sp, M=M, seed=1, recursion="proposal") as ch:
        out = G.run_clusters([ch], n, [8])[0]
    oracle_replay(L, sp, M, 20.0, 1, 0, out)


def test_clusters_reject_bad_requests(G):
    M = 64
    unit = G.Chain(4, inputs.uniform_sphere(4, 0), M=M)
    prop = G.Chain(6, inputs.uniform_sphere(6, 0), M=M, recursion="proposal")
    big = G.Chain(32, inputs.uniform_sphere(32, 0), M=M, recursion="proposal")
    unit8 = G.Chain(8, inputs.uniform_sphere(8, 0), M=M, recursion="proposal")
    for chains, C in (([unit], [2]),      # unit-vector recursion
                      ([prop], [16]),     # 16 does not divide L = 6
                      ([unit8], [16]),    # divides N = 512 but not L = 8: no whole planes
                      ([prop], [3]),      # not a cluster size
                      ([big], [2]),       # FP64 L=32 does not fit in two CTAs' shared memory
                      ([prop, prop], [1, 1])):  # the same chain twice
        with pytest.raises(G.GfmcError) as e:
            G.run_clusters(chains, 1, C)
        assert e.value.status == G.GFMC_EINVAL
    assert prop.counter == 0 and big.counter == 0
    for ch in (unit, prop, big, unit8):
        ch.close()


def test_smallest_cluster_and_cluster_runner(G):
    """The smallest cluster that holds a lattice, and the runner that puts every
    chain on its smallest cluster (FP64 chains replayed by the oracle)."""
    from paper_1303_6016_gb300 import batch
    assert G.cluster_min_ctas(8, 1024) == 1
    assert G.cluster_min_ctas(32, 1024) == 8   # 4096 sites x 56 B per CTA
    c24 = G.cluster_min_ctas(24, 1024)
    assert 24 % c24 == 0 and c24 > 1
    assert G.cluster_min_ctas(32, 1024, "fp64") == 16  # 2048 sites x 112 B per CTA
    for args in ((64, 1024), (8, 100), (2, 64)):
        with pytest.raises(G.GfmcError) as e:
            G.cluster_min_ctas(*args)
        assert e.value.status == G.GFMC_EINVAL
    specs = [(6, 12.0), (8, 20.0), (12, 9.0)]
    M, n = 64, 30
    chains, sps = [], []
    for c, (L, beta) in enumerate(specs):
        sp = inputs.uniform_sphere(L, 90 + c)
        sps.append(sp)
        chains.append(G.Chain(L, sp, M=M, beta=beta, mu=-2.0, seed=5, chain_id=c, recursion="proposal"))
    runner = batch.ClusterRunner(chains)
    assert runner.cluster_ctas == [1, 1, 1]
    outs = runner.run(n, trace=True)
    for c, (L, beta) in enumerate(specs):
        oracle_replay(L, sps[c], M, beta, 5, c, outs[c])
    for ch in chains:
        ch.close()
