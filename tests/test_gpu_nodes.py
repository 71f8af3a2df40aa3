"""The Green's function and the Delta Omega quadrature on K = 2M Chebyshev
nodes (gfmc_options.nodes), against the oracle on the same nodes.

The engine takes the K-point FFT of the zero-padded damped moments (Eq.
green_fft with the nodes theta_k = pi (k + 1/2)/K); the oracle sums Eq. green
directly at each of the K nodes and takes the 7x7 determinant.  Tolerances as
for the default K = M: FP64 Delta Omega 1e-10 |dO| + 1e-13 a, decisions
identical except near ties |exp(-beta dO) - u| < 1e-9, FP32-mixed 1e-4 t.
"""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_6016_gb300 import inputs

pytestmark = pytest.mark.gpu

A = 6.05
TIE = 1e-9


def dom_tol(ref):
    return 1e-10 * abs(ref) + 1e-13 * A


@pytest.fixture(scope="module")
def G():
    from paper_1303_6016_gb300 import build, gfmc
    build.build()
    gfmc.load()
    return gfmc


def replay(L, sp0, M, K, out, n, seed, chain_id=0, beta=20.0):
    """The oracle follows the GPU's decisions; every Delta Omega must agree and
    every decision that differs must be a near tie."""
    res = O.updates(L, sp0, n, M, beta=beta, chem=-2.0, seed=seed, chain_id=chain_id, nodes=K,
                    forced=out["decisions"].astype(np.int8))
    own = res["ratio"] > res["u"]
    for q in range(n):
        assert abs(out["d_omega"][q] - res["d_omega"][q]) <= dom_tol(res["d_omega"][q]), \
            (q, out["d_omega"][q], res["d_omega"][q])
        if own[q] != bool(out["decisions"][q]):
            assert abs(res["ratio"][q] - res["u"][q]) < TIE
    return res


@pytest.mark.parametrize("L,M,ncta,recursion", [(4, 256, 0, "unit_vectors"), (6, 128, 3, "unit_vectors"),
                                                (8, 64, 0, "proposal"), (4, 2048, 0, "unit_vectors")])
def test_delta_omega_on_2m_nodes_matches_oracle(G, L, M, ncta, recursion):
    sp = inputs.uniform_sphere(L, 31)
    rng = np.random.default_rng(8)
    with G.Chain(L, sp, M=M, beta=20.0, mu=-2.0, num_ctas=ncta, recursion=recursion, nodes=2 * M) as ch:
        assert ch.K == 2 * M
        for o in (0, L ** 3 // 2, L ** 3 - 1):
            th, ph = float(np.arccos(1 - 2 * rng.random())), float(2 * np.pi * rng.random())
            got = ch.delta_omega(o, th, ph)
            ref = O.delta_omega(L, sp, o, th, ph, M, beta=20.0, chem=-2.0, nodes=2 * M)
            assert abs(got - ref) <= dom_tol(ref), (o, got, ref)
        # the identity proposal stays exactly zero on the finer grid
        assert ch.delta_omega(5, sp[5, 0], sp[5, 1]) == 0.0


def test_2m_nodes_differ_from_m_nodes(G):
    """The option is live: the same proposal on M and on 2M nodes gives the two
    oracle values, which differ by the M-node rule's quadrature error."""
    L, M = 6, 256
    sp = inputs.uniform_sphere(L, 0)
    o, th, ph = 17, 0.2, 4.0
    got = {}
    for K in (M, 2 * M):
        with G.Chain(L, sp, M=M, beta=5.0, mu=-2.0, nodes=K) as ch:
            got[K] = ch.delta_omega(o, th, ph)
        ref = O.delta_omega(L, sp, o, th, ph, M, beta=5.0, chem=-2.0, nodes=K)
        assert abs(got[K] - ref) <= dom_tol(ref)
    assert abs(got[M] - got[2 * M]) > 1e-6


def test_sweep_on_2m_nodes_fp64(G):
    L, M = 4, 128
    sp = inputs.uniform_sphere(L, 3)
    with G.Chain(L, sp, M=M, beta=20.0, mu=-2.0, seed=4, nodes=2 * M) as ch:
        out = ch.sweep(1)
        spins = ch.get_spins()
    res = replay(L, sp, M, 2 * M, out, L ** 3, seed=4)
    np.testing.assert_allclose(spins, res["spins"], rtol=0, atol=1e-15)


def test_fp32_mixed_on_2m_nodes(G):
    L, M = 8, 256
    sp = inputs.make("vmf", L, seed=2)
    with G.Chain(L, sp, M=M, beta=20.0, mu=-2.0, precision="fp32_mixed", nodes=2 * M) as ch:
        for o, th, ph in ((0, 1.1, 0.3), (300, 2.6, 5.0)):
            d = ch.delta_omega(o, th, ph)
            assert abs(d - O.delta_omega(L, sp, o, th, ph, M, beta=20.0, chem=-2.0, nodes=2 * M)) <= 1e-4


def test_batch_and_clusters_on_2m_nodes(G):
    """Team batches and thread-block clusters size their work areas by the
    nodes: chains on 2M nodes give the oracle's trace there too."""
    M, n = 64, 24
    specs = [(6, 2, 41), (5, 1, 42)]
    chains = [G.Chain(L, inputs.uniform_sphere(L, s), M=M, beta=20.0, mu=-2.0, seed=6, chain_id=c, nodes=2 * M)
              for c, (L, _, s) in enumerate(specs)]
    outs = G.run_batch(chains, [n] * len(chains), team_ctas=[tc for (_, tc, _) in specs])
    for c, (L, _, s) in enumerate(specs):
        replay(L, inputs.uniform_sphere(L, s), M, 2 * M, outs[c], n, seed=6, chain_id=c)
    for ch in chains:
        ch.close()
    L, s = 8, 43
    with G.Chain(L, inputs.uniform_sphere(L, s), M=M, beta=20.0, mu=-2.0, seed=6, chain_id=7,
                 recursion="proposal", nodes=2 * M) as ch:
        C = G.cluster_min_ctas(L, 2 * M, "fp64")
        out = G.run_clusters([ch], [n], [C])[0]
    replay(L, inputs.uniform_sphere(L, s), M, 2 * M, out, n, seed=6, chain_id=7)


def test_server_job_on_2m_nodes(G):
    M, n, L = 64, 20, 6
    sp = inputs.uniform_sphere(L, 44)
    ch = G.Chain(L, sp, M=M, beta=20.0, mu=-2.0, seed=8, chain_id=2, nodes=2 * M)
    with G.Server([2], max_M=2 * M) as srv:
        srv.submit(0, ch, n)
        t0 = time.time()
        out = None
        while out is None:
            out = srv.poll(0)
            assert time.time() - t0 < 120.0, "server job did not finish"
            time.sleep(0.001)
    replay(L, sp, M, 2 * M, out, n, seed=8, chain_id=2)
    ch.close()


def test_full_size_delta_omega_on_2m_nodes(G):
    L, M = 32, 1024
    sp = inputs.uniform_sphere(L, 0)
    o, th, ph = 12345, 2.1, 0.7
    with G.Chain(L, sp, M=M, beta=20.0, mu=-2.0, nodes=2 * M) as ch:
        d = ch.delta_omega(o, th, ph)
    mu = O.moments(L, sp, o, M)
    dref, _ = O.delta_omega_from_moments(L, sp, mu, O.kernel(M), o, th, ph, beta=20.0, chem=-2.0,
                                         nodes=2 * M)
    assert abs(d - dref) <= dom_tol(dref)


def test_largest_moment_count_on_2m_nodes(G):
    """M = 4096 on K = 8192 nodes: the largest FFT (128 KB of shared memory)."""
    L, M = 4, 4096
    sp = inputs.uniform_sphere(L, 77)
    with G.Chain(L, sp, M=M, beta=20.0, mu=-2.0, nodes=2 * M) as ch:
        d = ch.delta_omega(9, 2.0, 1.0)
    ref = O.delta_omega(L, sp, 9, 2.0, 1.0, M, beta=20.0, chem=-2.0, nodes=2 * M)
    assert abs(d - ref) <= dom_tol(ref)
