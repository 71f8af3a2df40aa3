"""GPU parity of the FP32-mixed single-chain engine on seven thread-block
clusters (gfmc_options.engine = GFMC_ENGINE_VECTOR_CLUSTERS, L = 32): moments
read off the plain Chebyshev recursion of each unit vector (Eq. recursive),
against the oracle and against the grid engine.

Tolerances (FP32 recursion vectors, FP64 above them):
  moments       <= 2e-5 absolute, element by element (6e-8 rounding per step,
                   values <= 1, the Chebyshev recursion is stable)
  Delta Omega   <= 1e-4 t
  decisions     identical except where |exp(-beta dO) - u| < 1e-4 (the FP32
                   error in dO, ~1e-7 t, moves exp(-beta dO) by ~1e-5 at beta = 20)
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_6016_gb300 import inputs

pytestmark = pytest.mark.gpu

L = 32
MOM_TOL = 2e-5
DOM_TOL = 1e-4
TIE32 = 1e-4


@pytest.fixture(scope="module")
def G():
    from paper_1303_6016_gb300 import build, gfmc
    build.build()
    gfmc.load()
    return gfmc


def vc_chain(G, sp, M, **kw):
    kw.setdefault("beta", 20.0)
    kw.setdefault("mu", -2.0)
    return G.Chain(L, sp, M=M, precision="fp32_mixed", engine="vector_clusters", **kw)


def site(x, y, z):
    return x + L * (y + L * z)


# sites whose 7-site stars cross the pencils of the 4 x 4 cluster split (y, z
# multiples of 8), the periodic wrap in every direction, and the z-pairs
SITES = [site(0, 0, 0), site(31, 31, 31), site(5, 7, 8), site(16, 8, 15), site(3, 20, 23), site(31, 0, 16),
         site(12, 15, 1)]


def test_moments_match_oracle_M256(G):
    M = 256
    sp = inputs.uniform_sphere(L, 0)
    with vc_chain(G, sp, M) as ch:
        for o in SITES:
            got = ch.moments(o)
            ref = O.moments(L, sp, o, M)
            err = np.abs(got - ref).max()
            assert err <= MOM_TOL, (o, err)
            # mu_0 = delta and mu_1 = Htilde are exact entries
            np.testing.assert_array_equal(got[:, :, 0], np.eye(7))
            assert np.abs(got[:, :, 1] - ref[:, :, 1]).max() <= 1e-7


def test_moments_full_size_M1024_match_oracle(G):
    """The benchmark's workload (L = 32, M = 1024) on three sites."""
    M = 1024
    sp = inputs.uniform_sphere(L, 0)
    with vc_chain(G, sp, M) as ch:
        for o in (12345, SITES[2], SITES[5]):
            got = ch.moments(o)
            ref = O.moments(L, sp, o, M)
            err = np.abs(got - ref).max()
            assert err <= MOM_TOL, (o, err)


def test_moments_ferromagnet_closed_form(G):
    """All spins along z: mu_n^{jk} = (1/N) sum_q cos(q.(r_j - r_k)) T_n(eps_q / a)."""
    M, A = 128, 6.05
    q = 2 * np.pi * np.arange(L) / L
    Q = np.stack(np.meshgrid(q, q, q, indexing="ij"), axis=-1).reshape(-1, 3)
    eps = -2.0 * np.cos(Q).sum(axis=1)
    R = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])
    with vc_chain(G, inputs.ferromagnet(L), M) as ch:
        got = ch.moments(site(7, 8, 23))
    Tn = np.cos(np.arange(M)[:, None] * np.arccos(eps / A)[None, :])
    for j in range(7):
        for k in range(7):
            ref = Tn @ np.cos(Q @ (R[j] - R[k])) / L ** 3
            assert np.abs(got[j, k] - ref).max() <= MOM_TOL


@pytest.mark.parametrize("kind,M,kernel,nodes", [("uniform", 256, "jackson", 0), ("vmf", 256, "jackson", 0),
                                                 ("uniform", 128, "lorentz", 0), ("uniform", 128, "jackson", 256),
                                                 ("uniform", 1024, "jackson", 0)])
def test_delta_omega_matches_oracle(G, kind, M, kernel, nodes):
    sp = inputs.make(kind, L, seed=0 if kind == "uniform" else 2)
    rng = np.random.default_rng(11)
    K = nodes or M
    with vc_chain(G, sp, M, kernel=kernel, nodes=nodes) as ch:
        for o in SITES[:3]:
            th, ph = float(np.arccos(1 - 2 * rng.random())), float(2 * np.pi * rng.random())
            d = ch.delta_omega(o, th, ph)
            mu = O.moments(L, sp, o, M)
            dref, _ = O.delta_omega_from_moments(L, sp, mu, O.kernel(M, kind=1 if kernel == "lorentz" else 0),
                                                 o, th, ph, beta=20.0, chem=-2.0, nodes=K)
            assert abs(d - dref) <= DOM_TOL, (o, d, dref)


def test_agrees_with_the_grid_engine(G):
    """The two FP32-mixed engines (direct entries vs the doubling's Gram sums)."""
    M = 256
    sp = inputs.uniform_sphere(L, 3)
    o = SITES[3]
    with vc_chain(G, sp, M) as a, G.Chain(L, sp, M=M, beta=20.0, mu=-2.0, precision="fp32_mixed",
                                          engine="grid") as b:
        assert np.abs(a.moments(o) - b.moments(o)).max() <= 2 * MOM_TOL
        assert abs(a.delta_omega(o, 0.4, 5.0) - b.delta_omega(o, 0.4, 5.0)) <= DOM_TOL


def replay(sp0, M, out, n, upd0=0, seed=1):
    res = O.updates(L, sp0, n, M, beta=20.0, chem=-2.0, seed=seed, upd0=upd0,
                    forced=out["decisions"].astype(np.int8))
    own = res["ratio"] > res["u"]
    gdec = out["decisions"].astype(bool)
    for q in range(n):
        assert abs(out["d_omega"][q] - res["d_omega"][q]) <= DOM_TOL, (q, out["d_omega"][q], res["d_omega"][q])
        if own[q] != gdec[q]:
            assert abs(res["ratio"][q] - res["u"][q]) < TIE32, (q, res["ratio"][q], res["u"][q])
    return res


def test_updates_replayed_by_oracle(G):
    """Sequential updates from a sweep's start: the oracle follows the GPU's
    decisions and agrees on every Delta Omega; the spins agree after the run."""
    M, n = 128, 12
    sp = inputs.uniform_sphere(L, 0)
    with vc_chain(G, sp, M, seed=1) as ch:
        out = ch.updates(n)
        spins = ch.get_spins()
    res = replay(sp, M, out, n)
    assert 0 < int(out["decisions"].sum()) < n
    np.testing.assert_allclose(spins, res["spins"], rtol=0, atol=1e-15)


def test_updates_across_a_sweep_end(G):
    """Updates N-3 .. N+2: the last sites of a sweep, the magnetisation after
    it, and the first sites of the next sweep (the patched bonds in use)."""
    M, n = 64, 6
    N = L ** 3
    sp = inputs.uniform_sphere(L, 6)
    with vc_chain(G, sp, M, seed=3) as ch:
        ch.set_state(sp, N - 3)
        out = ch.updates(n)
    res = replay(sp, M, out, n, upd0=N - 3, seed=3)
    assert out["magnetization"].shape == (1,)
    assert out["magnetization"][0] == pytest.approx(res["magnetization"][0], abs=1e-13)


def test_reruns_are_bitwise_identical(G):
    M = 64
    sp = inputs.uniform_sphere(L, 5)
    outs = []
    for _ in range(2):
        with vc_chain(G, sp, M) as ch:
            outs.append((ch.updates(5), ch.moments(SITES[1])))
    np.testing.assert_array_equal(outs[0][0]["d_omega"], outs[1][0]["d_omega"])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])


def test_timeout_status_and_recovery(G):
    """CTA 0 of the first cluster withholds its faces: its neighbours run out
    of a short budget, the launch ends with GFMC_ETIMEOUT, and the handle
    gives the same answer afterwards."""
    M = 64
    sp = inputs.uniform_sphere(L, 0)
    with vc_chain(G, sp, M) as ch:
        ref = ch.delta_omega(3, 1.0, 1.0)
        ch.set_wait_budget(20_000_000)
        ch.inject_stall(True)
        with pytest.raises(G.GfmcError) as e:
            ch.delta_omega(3, 1.0, 1.0)
        assert e.value.status == G.GFMC_ETIMEOUT
        ch.set_wait_budget(4_000_000_000)
        assert ch.delta_omega(3, 1.0, 1.0) == ref


def test_engine_option_is_checked(G):
    with pytest.raises(G.GfmcError) as e:
        G.Chain(16, inputs.uniform_sphere(16, 0), M=64, precision="fp32_mixed", engine="vector_clusters")
    assert e.value.status == G.GFMC_EINVAL
    with pytest.raises(G.GfmcError) as e:
        G.Chain(L, inputs.uniform_sphere(L, 0), M=64, precision="fp64", engine="vector_clusters")
    assert e.value.status == G.GFMC_EINVAL
