"""GPU parity: the CUDA engine (through the C ABI) against the oracle.

Tolerances (stated here, derived in the design notes):
  FP64 moments            |mu_gpu - mu_oracle| <= 1e-12 absolute, element by element
  FP64 Delta Omega        |dO_gpu - dO_oracle| <= 1e-10 |dO_oracle| + 1e-13 a
  decisions               identical, except where |exp(-beta dO) - u| < 1e-9
  FP32-mixed moments      <= 2e-5 absolute (FP32 recursion vectors)
  FP32-mixed Delta Omega  <= 1e-4 t
The GPU takes routes the oracle does not (doubling of Eq. mu2, FFT of
Eq. green_fft, 2x2 determinant of Eq. d_z_green, stencil summation order), so
agreement is across independent routes.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_6016_gb300 import inputs

pytestmark = pytest.mark.gpu

A = 6.05
MOM_TOL = 1e-12
TIE = 1e-9


def dom_tol(ref):
    return 1e-10 * abs(ref) + 1e-13 * A


@pytest.fixture(scope="module")
def G():
    from paper_1303_6016_gb300 import build, gfmc
    build.build()
    gfmc.load()
    return gfmc


def chain(G, L, spins, M, **kw):
    kw.setdefault("beta", 20.0)
    kw.setdefault("mu", -2.0)
    return G.Chain(L, spins, M=M, **kw)


# ---------------------------------------------------------------------------
# moments
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L,M,ncta", [(3, 32, 0), (4, 256, 0), (5, 64, 2), (8, 128, 0), (8, 64, 5),
                                      (12, 64, 0), (8, 128, 2), (6, 64, 1)])
def test_moments_fp64_match_oracle(G, L, M, ncta):
    """(8, 128, 2): 256-site tiles whose parity classes fill all 128 staging
    positions, on the split instantiation; (6, 64, 1): one 216-site tile, whose
    halo-only prefetch window is empty."""
    sp = inputs.uniform_sphere(L, 0)
    with chain(G, L, sp, M, num_ctas=ncta) as ch:
        for o in sorted({0, 1, L ** 3 // 2 + 3, L ** 3 - 1}):
            got = ch.moments(o)
            ref = O.moments(L, sp, o, M)
            err = np.abs(got - ref).max()
            assert err <= MOM_TOL, (o, err)


def test_moments_ferromagnet_closed_form_L16(G):
    L, M = 16, 256
    q = 2 * np.pi * np.arange(L) / L
    Q = np.stack(np.meshgrid(q, q, q, indexing="ij"), axis=-1).reshape(-1, 3)
    eps = -2.0 * np.cos(Q).sum(axis=1)
    R = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])
    with chain(G, L, inputs.ferromagnet(L), M) as ch:
        got = ch.moments(1234)
    Tn = np.cos(np.arange(M)[:, None] * np.arccos(eps / A)[None, :])  # [M, N]
    for j in range(7):
        for k in range(7):
            ref = Tn @ np.cos(Q @ (R[j] - R[k])) / L ** 3
            assert np.abs(got[j, k] - ref).max() <= MOM_TOL


# ---------------------------------------------------------------------------
# Delta Omega
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L,M,ncta,kernel", [(4, 256, 0, "jackson"), (6, 128, 3, "jackson"),
                                             (8, 256, 0, "jackson"), (6, 128, 0, "lorentz")])
def test_delta_omega_fp64_matches_oracle(G, L, M, ncta, kernel):
    sp = inputs.uniform_sphere(L, 1)
    kind = 0 if kernel == "jackson" else 1
    rng = np.random.default_rng(3)
    with chain(G, L, sp, M, num_ctas=ncta, kernel=kernel) as ch:
        for o in (0, L ** 3 // 3, L ** 3 - 1):
            th, ph = float(np.arccos(1 - 2 * rng.random())), float(2 * np.pi * rng.random())
            got = ch.delta_omega(o, th, ph)
            ref = O.delta_omega(L, sp, o, th, ph, M, beta=20.0, chem=-2.0, kernel_kind=kind, lam=4.0)
            assert abs(got - ref) <= dom_tol(ref), (o, got, ref)


def test_identity_proposal_is_exactly_zero(G):
    L, M = 6, 128
    sp = inputs.uniform_sphere(L, 2)
    with chain(G, L, sp, M) as ch:
        for o in (0, 100):
            assert ch.delta_omega(o, sp[o, 0], sp[o, 1]) == 0.0


# ---------------------------------------------------------------------------
# sweeps: identical decisions (near ties excepted), Delta Omega traces
# ---------------------------------------------------------------------------

def check_trace_against_oracle(L, sp0, M, gpu, n, beta=20.0, seed=1, chain_id=0, upd0=0):
    """Replay the GPU's decisions in the oracle and compare each update."""
    res = O.updates(L, sp0, n, M, beta=beta, chem=-2.0, seed=seed, chain_id=chain_id, upd0=upd0,
                    forced=gpu["decisions"].astype(np.int8))
    own = res["ratio"] > res["u"]
    gdec = gpu["decisions"].astype(bool)
    for q in range(n):
        assert abs(gpu["d_omega"][q] - res["d_omega"][q]) <= dom_tol(res["d_omega"][q]), \
            (q, gpu["d_omega"][q], res["d_omega"][q])
        if own[q] != gdec[q]:
            assert abs(res["ratio"][q] - res["u"][q]) < TIE, (q, res["ratio"][q], res["u"][q])
    return res


def test_sweep_L4_M256_fp64(G):
    """One full sequential sweep of 64 updates at L = 4, M = 256, beta = 20, mu = -2."""
    L, M = 4, 256
    sp = inputs.uniform_sphere(L, 0)
    with chain(G, L, sp, M, seed=1) as ch:
        out = ch.sweep(1)
        spins = ch.get_spins()
    res = check_trace_against_oracle(L, sp, M, out, L ** 3)
    np.testing.assert_allclose(spins, res["spins"], rtol=0, atol=1e-15)
    assert out["n_accepted"] == int(out["decisions"].sum())
    assert out["magnetization"].shape == (1,)
    assert out["magnetization"][0] == pytest.approx(res["magnetization"][0], abs=1e-13)


def test_sweep_L6_multi_cta_fp64(G):
    L, M = 6, 128
    sp = inputs.uniform_sphere(L, 4)
    with chain(G, L, sp, M, seed=7, chain_id=3, num_ctas=4) as ch:
        out = ch.sweep(1)
    check_trace_against_oracle(L, sp, M, out, L ** 3, seed=7, chain_id=3)


def test_resume_equals_uninterrupted(G):
    """Checkpoint/resume: k updates, save (spins, counter), restore into a new
    chain, continue; equals the uninterrupted run bit for bit."""
    L, M = 5, 64
    sp = inputs.uniform_sphere(L, 9)
    with chain(G, L, sp, M) as ch:
        full = ch.updates(2 * L ** 3)
        s_full = ch.get_spins()
    with chain(G, L, sp, M) as ch:
        first = ch.updates(77)
        saved, ctr = ch.get_spins(), ch.counter
    with chain(G, L, sp, M) as ch2:
        ch2.set_state(saved, ctr)
        second = ch2.updates(2 * L ** 3 - 77)
        s_res = ch2.get_spins()
    np.testing.assert_array_equal(np.concatenate([first["decisions"], second["decisions"]]),
                                  full["decisions"])
    np.testing.assert_array_equal(np.concatenate([first["d_omega"], second["d_omega"]]), full["d_omega"])
    np.testing.assert_array_equal(s_res, s_full)


def test_reruns_are_bitwise_identical(G):
    L, M = 8, 64
    sp = inputs.uniform_sphere(L, 5)
    outs = []
    for _ in range(2):
        with chain(G, L, sp, M) as ch:
            outs.append((ch.updates(100), ch.moments(17)))
    np.testing.assert_array_equal(outs[0][0]["d_omega"], outs[1][0]["d_omega"])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])


# ---------------------------------------------------------------------------
# FP32-mixed path
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["uniform", "vmf"])
def test_fp32_mixed_against_oracle(G, kind):
    L, M = 8, 256
    sp = inputs.make(kind, L, seed=0 if kind == "uniform" else 2)
    rng = np.random.default_rng(8)
    with chain(G, L, sp, M, precision="fp32_mixed") as ch:
        for o in (0, 200, 511):
            got = ch.moments(o)
            ref = O.moments(L, sp, o, M)
            assert np.abs(got - ref).max() <= 2e-5
            th, ph = float(np.arccos(1 - 2 * rng.random())), float(2 * np.pi * rng.random())
            d = ch.delta_omega(o, th, ph)
            dref = O.delta_omega(L, sp, o, th, ph, M, beta=20.0, chem=-2.0)
            assert abs(d - dref) <= 1e-4


# ---------------------------------------------------------------------------
# full size (L = 32, M = 1024) in the launch configuration the benchmark times
# ---------------------------------------------------------------------------

def test_full_size_sampled_moments_and_delta_fp64(G):
    L, M = 32, 1024
    sp = inputs.uniform_sphere(L, 0)
    with chain(G, L, sp, M) as ch:
        o = 12345
        got = ch.moments(o)
        ref = O.moments(L, sp, o, M)
        assert np.abs(got - ref).max() <= MOM_TOL
        th, ph = 2.1, 0.7
        d = ch.delta_omega(o, th, ph)
        dref, _ = O.delta_omega_from_moments(L, sp, ref, O.kernel(M), o, th, ph, beta=20.0, chem=-2.0)
        assert abs(d - dref) <= dom_tol(dref)


def test_full_size_first_updates_fp64(G):
    L, M, n = 32, 1024, 3
    sp = inputs.uniform_sphere(L, 0)
    with chain(G, L, sp, M, seed=1) as ch:
        out = ch.updates(n)
    check_trace_against_oracle(L, sp, M, out, n)


def test_full_size_fp32_mixed_delta(G):
    L, M = 32, 1024
    sp = inputs.uniform_sphere(L, 0)
    o, th, ph = 777, 1.2, 4.4
    with chain(G, L, sp, M, precision="fp32_mixed") as ch:
        d = ch.delta_omega(o, th, ph)
    dref = O.delta_omega(L, sp, o, th, ph, M, beta=20.0, chem=-2.0)
    assert abs(d - dref) <= 1e-4


# ---------------------------------------------------------------------------
# error handling on the GPU
# ---------------------------------------------------------------------------

def test_bad_site_and_timeout_status(G):
    L, M = 8, 64
    sp = inputs.uniform_sphere(L, 0)
    with chain(G, L, sp, M, num_ctas=4) as ch:
        with pytest.raises(G.GfmcError) as e:
            ch.moments(L ** 3)
        assert e.value.status == G.GFMC_EINVAL
        ref = ch.delta_omega(3, 1.0, 1.0)
        # a flag that nothing sets: the neighbours of CTA 0 exhaust a short budget
        ch.set_wait_budget(20_000_000)
        ch.inject_stall(True)
        with pytest.raises(G.GfmcError) as e:
            ch.delta_omega(3, 1.0, 1.0)
        assert e.value.status == G.GFMC_ETIMEOUT
        # the handle stays usable and gives the same answer afterwards
        ch.set_wait_budget(4_000_000_000)
        assert ch.delta_omega(3, 1.0, 1.0) == ref


def test_fp32_timeout_status(G):
    """FP32-mixed: CTA 0 withholds its tagged values, the CTAs reading them run
    out of a short budget and the launch ends with GFMC_ETIMEOUT; the handle
    stays usable and gives the same answer afterwards."""
    L, M = 8, 64
    sp = inputs.uniform_sphere(L, 0)
    with chain(G, L, sp, M, num_ctas=4, precision="fp32_mixed") as ch:
        ref = ch.delta_omega(3, 1.0, 1.0)
        ch.set_wait_budget(20_000_000)
        ch.inject_stall(True)
        with pytest.raises(G.GfmcError) as e:
            ch.delta_omega(3, 1.0, 1.0)
        assert e.value.status == G.GFMC_ETIMEOUT
        ch.set_wait_budget(4_000_000_000)
        assert ch.delta_omega(3, 1.0, 1.0) == ref


# ---------------------------------------------------------------------------
# the paper's recursion on the proposal's vectors (o, v; o+v and o+iv by linearity)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L,M,ncta,prec", [(4, 256, 0, "fp64"), (6, 128, 3, "fp64"), (8, 256, 0, "fp64"),
                                           (8, 256, 0, "fp32_mixed")])
def test_proposal_recursion_delta_omega_matches_oracle(G, L, M, ncta, prec):
    sp = inputs.uniform_sphere(L, 11)
    rng = np.random.default_rng(12)
    with chain(G, L, sp, M, num_ctas=ncta, recursion="proposal", precision=prec) as ch:
        for o in (0, L ** 3 // 2, L ** 3 - 1):
            th, ph = float(np.arccos(1 - 2 * rng.random())), float(2 * np.pi * rng.random())
            got = ch.delta_omega(o, th, ph)
            ref = O.delta_omega(L, sp, o, th, ph, M, beta=20.0, chem=-2.0)
            tol = dom_tol(ref) if prec == "fp64" else 1e-4
            assert abs(got - ref) <= tol, (o, got, ref)
        # the 7x7 moments call still runs on the unit vectors
        assert np.abs(ch.moments(5) - O.moments(L, sp, 5, M)).max() <= (MOM_TOL if prec == "fp64" else 2e-5)


def test_proposal_recursion_sweep_matches_oracle(G):
    L, M = 6, 128
    sp = inputs.uniform_sphere(L, 13)
    with chain(G, L, sp, M, seed=2, recursion="proposal") as ch:
        out = ch.sweep(1)
    check_trace_against_oracle(L, sp, M, out, L ** 3, seed=2)


def test_proposal_recursion_full_size_fp64(G):
    L, M, n = 32, 1024, 3
    sp = inputs.uniform_sphere(L, 0)
    with chain(G, L, sp, M, seed=1, recursion="proposal") as ch:
        out = ch.updates(n)
    check_trace_against_oracle(L, sp, M, out, n)


# ---------------------------------------------------------------------------
# edges: chains with more sites than threads per CTA, extreme M, Lorentz sweep
# ---------------------------------------------------------------------------

def test_multi_site_chain_matches_oracle(G):
    """L = 36 (N = 46656 > 256 x 152 CTAs): every call of the chain runs the
    engine's multi-site variant."""
    L, M = 36, 64
    sp = inputs.uniform_sphere(L, 21)
    with chain(G, L, sp, M, seed=5) as ch:
        o = 30000
        assert np.abs(ch.moments(o) - O.moments(L, sp, o, M)).max() <= MOM_TOL
        d = ch.delta_omega(o, 0.9, 5.5)
        dref = O.delta_omega(L, sp, o, 0.9, 5.5, M, beta=20.0, chem=-2.0)
        assert abs(d - dref) <= dom_tol(dref)
        out = ch.updates(3)
    check_trace_against_oracle(L, sp, M, out, 3, seed=5)


@pytest.mark.parametrize("M", [16, 4096])
def test_extreme_M(G, M):
    L = 4
    sp = inputs.uniform_sphere(L, 22)
    with chain(G, L, sp, M) as ch:
        assert np.abs(ch.moments(9) - O.moments(L, sp, 9, M)).max() <= MOM_TOL
        d = ch.delta_omega(9, 2.0, 1.0)
    dref = O.delta_omega(L, sp, 9, 2.0, 1.0, M, beta=20.0, chem=-2.0)
    assert abs(d - dref) <= dom_tol(dref)


def test_lorentz_sweep_matches_oracle(G):
    L, M = 5, 128
    sp = inputs.uniform_sphere(L, 23)
    with chain(G, L, sp, M, kernel="lorentz", lorentz_lambda=3.0, seed=9) as ch:
        out = ch.sweep(1)
    res = O.updates(L, sp, L ** 3, M, beta=20.0, chem=-2.0, seed=9, kernel_kind=1, lam=3.0,
                    forced=out["decisions"].astype(np.int8))
    own = res["ratio"] > res["u"]
    for q in range(L ** 3):
        assert abs(out["d_omega"][q] - res["d_omega"][q]) <= dom_tol(res["d_omega"][q])
        if own[q] != bool(out["decisions"][q]):
            assert abs(res["ratio"][q] - res["u"][q]) < TIE


# ---------------------------------------------------------------------------
# tile layouts of the single-chain engines: the FP64 engine's prefetched runs
# of sites (ragged tiles, tiles across plane boundaries, y-wrap rows) and the
# FP32 engine with and without warp 7 as the flag helper (tiles of <= 224
# sites or more)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L,ncta", [(20, 0), (10, 7), (24, 152), (9, 5), (16, 17), (16, 0), (20, 152), (14, 0)])
def test_fp64_tile_layouts_match_oracle(G, L, ncta):
    """Tile layouts of the FP64 engine: odd L (no bipartite step) and
    bipartite tiles, the (vector, site) items of a step filling part of one
    pass or spilling into a second -- (20, 0), (16, 0): 64-site tiles; (20,
    152): ragged 52/53-site tiles; (14, 0): 65-site tiles -- and tiles of at
    least 128 sites on the split instantiation (halo-only prefetch, group sums
    beside the units): (10, 7), 142/143 sites; (16, 17), 240/241 sites."""
    M = 64
    sp = inputs.uniform_sphere(L, 40 + L)
    with chain(G, L, sp, M, num_ctas=ncta, seed=3) as ch:
        N = L ** 3
        for o in (0, N // 3 + 1, N - 1):
            assert np.abs(ch.moments(o) - O.moments(L, sp, o, M)).max() <= MOM_TOL, o
        out = ch.updates(6)
    check_trace_against_oracle(L, sp, M, out, 6, seed=3)


@pytest.mark.parametrize("L,ncta", [(8, 2), (8, 3), (12, 9)])
def test_fp32_with_and_without_the_helper_warp(G, L, ncta):
    """(8, 2): 256-site tiles, no helper; (8, 3) and (12, 9): tiles within 7
    warps, warp 7 publishes and polls.  Delta Omega within 1e-4 t of the oracle."""
    M = 64
    sp = inputs.uniform_sphere(L, 50 + ncta)
    with chain(G, L, sp, M, num_ctas=ncta, precision="fp32_mixed", seed=4) as ch:
        out = ch.updates(5)
    res = O.updates(L, sp, 5, M, beta=20.0, chem=-2.0, seed=4, forced=out["decisions"].astype(np.int8))
    assert np.abs(out["d_omega"] - res["d_omega"]).max() <= 1e-4


def test_torch_tensor_spins_give_the_same_chain(G):
    """Spins as a torch tensor on the GPU or the host, or as numpy: the same chain."""
    torch = pytest.importorskip("torch")
    L, M = 6, 64
    sp = inputs.uniform_sphere(L, 21)
    outs = []
    for arg in (sp, torch.tensor(sp), torch.tensor(sp, device="cuda")):
        with chain(G, L, arg, M, seed=5) as ch:
            out = ch.updates(8)
            ch.set_state(arg, 0)
            outs.append((out["d_omega"], ch.moments(9)))
    for d, mu in outs[1:]:
        np.testing.assert_array_equal(d, outs[0][0])
        np.testing.assert_array_equal(mu, outs[0][1])
