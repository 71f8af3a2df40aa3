"""FP32-mixed chains with compensated Gram dot products (gfmc_options.compensated:
Dot2 -- error-free FP32 products and sums carried as (hi, lo) pairs through
the warp sums, FP64 above) against the oracle, on every engine that forms
the doubling's dot products (Eq. mu2): the grid single-chain engine, team
batches, thread-block cluster batches and graph plans.

Tolerances as for plain FP32-mixed: moments 2e-5, Delta Omega 1e-4 t,
decisions identical except where |exp(-beta dO) - u| < 1e-4.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_6016_gb300 import inputs

pytestmark = pytest.mark.gpu

MOM_TOL = 2e-5
TOL = 1e-4
TIE = 1e-4


@pytest.fixture(scope="module")
def G():
    from paper_1303_6016_gb300 import build, gfmc
    build.build()
    gfmc.load()
    return gfmc


def replay(L, sp, M, beta, seed, chain_id, out):
    n = out["decisions"].size
    res = O.updates(L, sp, n, M, beta=beta, chem=-2.0, seed=seed, chain_id=chain_id,
                    forced=out["decisions"].astype(np.int8))
    own = res["ratio"] > res["u"]
    for q in range(n):
        assert abs(out["d_omega"][q] - res["d_omega"][q]) <= TOL, (L, q)
        if own[q] != bool(out["decisions"][q]):
            assert abs(res["ratio"][q] - res["u"][q]) < TIE


@pytest.mark.parametrize("L,M,recursion", [(8, 256, "unit_vectors"), (12, 512, "unit_vectors"),
                                           (32, 1024, "unit_vectors"), (8, 256, "proposal")])
def test_single_chain_grid_engine(G, L, M, recursion):
    sp = inputs.uniform_sphere(L, 11)
    o = L ** 3 // 3 + 1
    with G.Chain(L, sp, M=M, beta=20.0, mu=-2.0, precision="fp32_mixed", engine="grid", compensated=True,
                 recursion=recursion) as ch:
        ref = O.moments(L, sp, o, M)
        if recursion == "unit_vectors":
            got = ch.moments(o)
            assert np.abs(got - ref).max() <= MOM_TOL
        d = ch.delta_omega(o, 1.9, 0.8)
        dref, _ = O.delta_omega_from_moments(L, sp, ref, O.kernel(M), o, 1.9, 0.8, beta=20.0, chem=-2.0)
        assert abs(d - dref) <= TOL
        if L <= 12:
            out = ch.updates(20)
            replay(L, sp, M, 20.0, 1, 0, out)


@pytest.mark.parametrize("runner,recursion,ctas", [("teams", "unit_vectors", [1, 2, 4]),
                                                   ("teams", "proposal", [1, 2, 4]),
                                                   ("clusters", "proposal", [2, 2, 4]),
                                                   ("plan", "unit_vectors", [1, 2, 4])])
def test_batches(G, runner, recursion, ctas):
    sizes, M, n = (8, 12, 16), 512, 6
    chains, sps = [], []
    for c, L in enumerate(sizes):
        sp = inputs.uniform_sphere(L, 80 + c)
        sps.append(sp)
        chains.append(G.Chain(L, sp, M=M, beta=15.0, mu=-2.0, precision="fp32_mixed", seed=8, chain_id=c,
                              recursion=recursion, compensated=True))
    if runner == "teams":
        outs = G.run_batch(chains, n, team_ctas=ctas)
    elif runner == "clusters":
        outs = G.run_clusters(chains, n, cluster_ctas=ctas)
    else:
        with G.Plan(chains, [n] * len(sizes), ctas, schedule="teams") as plan:
            plan.launch(1)
            outs = plan.sync()
    for c, L in enumerate(sizes):
        replay(L, sps[c], M, 15.0, 8, c, outs[c])
        chains[c].close()


def test_mixed_kinds_and_the_server_are_refused(G):
    L, M = 8, 64
    a = G.Chain(L, inputs.uniform_sphere(L, 1), M=M, precision="fp32_mixed", compensated=True)
    b = G.Chain(L, inputs.uniform_sphere(L, 2), M=M, precision="fp32_mixed")
    with pytest.raises(G.GfmcError) as e:
        G.run_batch([a, b], 2, team_ctas=[1, 1])
    assert e.value.status == G.GFMC_EINVAL
    with G.Server([2], max_M=M) as srv:
        with pytest.raises(G.GfmcError) as e:
            srv.submit(0, a, 2)
        assert e.value.status == G.GFMC_EINVAL
    with pytest.raises(G.GfmcError) as e:
        G.Chain(L, inputs.uniform_sphere(L, 1), M=M, precision="fp64", compensated=True)
    assert e.value.status == G.GFMC_EINVAL
    a.close()
    b.close()
