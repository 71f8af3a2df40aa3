"""Pins of the oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each check uses an independent
route -- the paper's own printed hopping formula (Eq. ht), dense
diagonalisation with numpy, closed forms of the ferromagnet, the sum rule of
the Green's function, the determinant identity of Eq. green_delta, the exact
grand potential of Sec. 2.1, or a second Philox written from its published
definition.  Each test names the passage it pins.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_6016_gb300 import inputs

A = 6.05  # spectral scale a = 6.05 |t|


# --------------------------------------------------------------------------
# independent constructions used by the pins
# --------------------------------------------------------------------------

def coords(L, i):
    return i % L, (i // L) % L, i // (L * L)


def paper_hamiltonian(L, spins, t=1.0):
    """H built from the hopping exactly as printed in Eq. ht (paper's gauge),
    H = -sum t_ij c_i^dag c_j (Eq. 2), neighbours enumerated from coordinates."""
    N = L ** 3
    H = np.zeros((N, N), dtype=np.complex128)
    for i in range(N):
        x, y, z = coords(L, i)
        for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            j = (x + dx) % L + L * (((y + dy) % L) + L * ((z + dz) % L))
            ti, pi_ = spins[i]
            tj, pj = spins[j]
            tij = (math.cos((ti - tj) / 2) * math.cos((pi_ - pj) / 2)
                   + 1j * math.cos((ti + tj) / 2) * math.sin((pi_ - pj) / 2))
            H[i, j] += -t * tij
    return H


def to_bj_gauge(Hp, spins):
    """The paper's spinor is e^{-i phi/2} times the (cos, e^{i phi} sin) spinor,
    so H_paper = D H D^dag with D = diag(e^{i phi/2})."""
    d = np.exp(0.5j * spins[:, 1])
    return d.conj()[:, None] * Hp * d[None, :]


def local7(L, o):
    x, y, z = coords(L, o)
    out = [o]
    for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
        out.append((x + dx) % L + L * (((y + dy) % L) + L * ((z + dz) % L)))
    return np.array(out)


def cheb_T(n, x):
    return np.cos(n * np.arccos(np.clip(x, -1.0, 1.0)))


def exact_delta_omega(L, spins, site, th, ph, beta, chem, t=1.0):
    """Omega(S') - Omega(S) from the eigenvalues (Sec. 2.1, S_eff = beta Omega)."""
    s2 = spins.copy()
    s2[site] = (th, ph)
    e1 = np.linalg.eigvalsh(paper_hamiltonian(L, spins, t))
    e2 = np.linalg.eigvalsh(paper_hamiltonian(L, s2, t))

    def omega(e):
        x = -beta * (e - chem)
        return -np.sum(np.where(x > 0, x + np.log1p(np.exp(-np.abs(x))),
                                np.log1p(np.exp(np.minimum(x, 0))))) / beta

    return omega(e2) - omega(e1)


# --------------------------------------------------------------------------
# lattice and Hamiltonian (Sec. 2.1, Eqs. 2 and ht)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("L", [3, 4, 5])
def test_local_sites_match_coordinates(L):
    for o in range(0, L ** 3, max(1, L ** 3 // 17)):
        assert list(O.local_sites(L, o)) == list(local7(L, o))


@pytest.mark.parametrize("L", [3, 4])
def test_hamiltonian_equals_paper_hopping_up_to_gauge(L):
    sp = inputs.uniform_sphere(L, 3)
    H = O.dense_htilde(L, sp) * A
    Hp = paper_hamiltonian(L, sp)
    np.testing.assert_allclose(H, to_bj_gauge(Hp, sp), atol=1e-14)
    assert np.abs(H - H.conj().T).max() == 0.0
    ev = np.linalg.eigvalsh(H)
    np.testing.assert_allclose(ev, np.linalg.eigvalsh(Hp), atol=1e-12)
    assert np.abs(ev).max() < A  # the rescaled spectrum lies inside (-1, 1)


@pytest.mark.parametrize("L", [4, 5])
def test_ferromagnet_spectrum_closed_form(L):
    H = O.dense_htilde(L, inputs.ferromagnet(L)) * A
    q = 2 * np.pi * np.arange(L) / L
    eq = -2.0 * (np.cos(q)[:, None, None] + np.cos(q)[None, :, None] + np.cos(q)[None, None, :])
    np.testing.assert_allclose(np.linalg.eigvalsh(H), np.sort(eq.ravel()), atol=1e-12)


# --------------------------------------------------------------------------
# moments (Sec. 2.2: mu_m = <i|T_m(H~)|i>, Eq. recursive, Eq. mu2)
# --------------------------------------------------------------------------

def test_moments_match_dense_diagonalisation():
    L, M = 4, 96
    sp = inputs.uniform_sphere(L, 0)
    Ht = to_bj_gauge(paper_hamiltonian(L, sp), sp) / A
    ev, U = np.linalg.eigh(Ht)
    for o in (0, 21, 63):
        mu = O.moments(L, sp, o, M)
        loc = local7(L, o)
        Uj = U[loc, :]
        for n in range(M):
            ref = (Uj * cheb_T(n, ev)[None, :]) @ Uj.conj().T
            np.testing.assert_allclose(mu[:, :, n], ref, atol=1e-12, rtol=0)


def test_moment_invariants():
    L, M = 4, 64
    sp = inputs.uniform_sphere(L, 5)
    o = 9
    mu = O.moments(L, sp, o, M)
    np.testing.assert_array_equal(mu[:, :, 0], np.eye(7))
    Ht = to_bj_gauge(paper_hamiltonian(L, sp), sp) / A
    loc = local7(L, o)
    np.testing.assert_allclose(mu[:, :, 1], Ht[np.ix_(loc, loc)], atol=1e-15)
    # mu_2^{jj} = 2 sum_l |H~_jl|^2 - 1
    np.testing.assert_allclose(np.diagonal(mu[:, :, 2]).real,
                               2 * np.sum(np.abs(Ht[loc, :]) ** 2, axis=1) - 1, atol=1e-14)
    np.testing.assert_allclose(mu, np.conj(np.transpose(mu, (1, 0, 2))), atol=1e-13)
    assert np.abs(mu).max() <= 1.0 + 1e-12


def test_bipartite_parity_even_L():
    """Even L: the cubic lattice is bipartite, so <j|T_n|k> vanishes when
    n + dist(j, k) is odd, and when n < dist(j, k) (light cone)."""
    L, M = 6, 40
    sp = inputs.uniform_sphere(L, 1)
    mu = O.moments(L, sp, 100, M)
    dist = np.array([[0, 1, 1, 1, 1, 1, 1]] + [[1] + [0 if a == b else 2 for b in range(1, 7)]
                                               for a in range(1, 7)])
    for n in range(M):
        for j in range(7):
            for k in range(7):
                if (n + dist[j, k]) % 2 == 1 or n < dist[j, k]:
                    assert mu[j, k, n] == 0.0


@pytest.mark.parametrize("L,M", [(4, 128), (6, 64), (8, 48)])
def test_ferromagnet_moments_closed_form(L, M):
    """All theta = 0: H = -t x adjacency, eps_q = -2t sum cos q_a, and
    <j|T_n(H~)|k> = (1/N) sum_q cos(q.(r_j - r_k)) T_n(eps_q / a)."""
    o = L ** 3 // 3
    mu = O.moments(L, inputs.ferromagnet(L), o, M)
    q = 2 * np.pi * np.arange(L) / L
    Q = np.stack(np.meshgrid(q, q, q, indexing="ij"), axis=-1).reshape(-1, 3)
    eps = -2.0 * np.cos(Q).sum(axis=1)
    R = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])
    for n in range(M):
        Tn = cheb_T(n, eps / A)
        for j in range(7):
            for k in range(7):
                ref = np.mean(np.cos(Q @ (R[j] - R[k])) * Tn)
                assert abs(mu[j, k, n] - ref) < 1e-12


def test_doubling_identity_holds_for_direct_moments():
    """Eq. mu2: mu_{2m} = 2<r_m|r_m> - mu_0 and mu_{2m+1} = 2<r_m|r_{m+1}> - mu_1,
    with the r_m built here by numpy from the paper's Hamiltonian."""
    L, M = 4, 64
    sp = inputs.uniform_sphere(L, 7)
    o = 33
    mu = O.moments(L, sp, o, M)
    Ht = to_bj_gauge(paper_hamiltonian(L, sp), sp) / A
    loc = local7(L, o)
    R = [np.eye(L ** 3)[:, loc].astype(complex)]
    R.append(Ht @ R[0])
    for m in range(2, M // 2 + 1):
        R.append(2 * Ht @ R[-1] - R[-2])
    for m in range(M // 2):
        np.testing.assert_allclose(mu[:, :, 2 * m], 2 * R[m].conj().T @ R[m] - mu[:, :, 0],
                                   atol=1e-12)
        np.testing.assert_allclose(mu[:, :, 2 * m + 1],
                                   2 * R[m].conj().T @ R[m + 1] - mu[:, :, 1], atol=1e-12)


# --------------------------------------------------------------------------
# kernels g_n
# --------------------------------------------------------------------------

@pytest.mark.parametrize("M", [16, 256, 1024])
def test_jackson_kernel_closed_forms_and_positivity(M):
    g = O.kernel(M, 0)
    assert g[0] == pytest.approx(1.0, abs=1e-15)
    assert g[1] == pytest.approx(math.cos(math.pi / (M + 1)), abs=1e-15)
    assert np.all(np.diff(g) < 0) and g[-1] > 0
    # the Jackson-smoothed delta function is positive and normalised
    x = np.cos(np.pi * (np.arange(2 * M) + 0.5) / (2 * M))
    n = np.arange(M)
    for y in (0.0, 0.37, -0.81):
        K = g[0] + 2 * np.sum((g[1:, None] * cheb_T(n[1:, None], x[None, :])
                               * cheb_T(n[1:, None], y)), axis=0)
        assert K.min() > -1e-10
        # int K(x,y) dx / (pi sqrt(1-x^2)) = 1 by Chebyshev-Gauss (exact here)
        assert np.mean(K) == pytest.approx(1.0, abs=1e-12)


def test_lorentz_kernel_values():
    M, lam = 128, 4.0
    g = O.kernel(M, 1, lam)
    assert g[0] == pytest.approx(1.0, abs=1e-15)
    assert g[M // 2] == pytest.approx(1.0 / (2.0 * math.cosh(lam / 2)), rel=1e-14)
    assert np.all(np.diff(g) < 0)


# --------------------------------------------------------------------------
# Green's function (Eq. green) and determinant (Eq. green_delta, Eq. d_z_green)
# --------------------------------------------------------------------------

def test_green_single_level_sum_rule_and_far_field():
    """One level at eps: mu_n = T_n(eps).  The Chebyshev-Gauss sum of Im G over
    the nodes is pi mu_0 exactly (sum rule), and away from eps the damped series
    approaches 1/(eps - w) (G = (H - z)^{-1})."""
    M, eps = 4096, 0.31
    g = O.kernel(M, 0)
    mu = np.zeros((7, 7, M), dtype=np.complex128)
    mu[0, 0, :] = cheb_T(np.arange(M), eps)
    ks = np.arange(0, M, 7)
    G = np.array([O.green7(mu, g, int(k))[0, 0] for k in ks])
    w = np.cos(np.pi * (ks + 0.5) / M)
    far = np.abs(w - eps) > 0.2
    np.testing.assert_allclose(G[far].real, 1.0 / (eps - w[far]), rtol=2e-4, atol=2e-4)
    assert np.abs(G[far].imag).max() < 1e-4
    assert np.all(G.imag > -1e-12)  # Im G = pi rho >= 0 for the damped series
    # full-node sum rule at a smaller M (exact identity)
    M2 = 256
    g2 = O.kernel(M2, 0)
    mu2 = np.zeros((7, 7, M2), dtype=np.complex128)
    mu2[0, 0, :] = cheb_T(np.arange(M2), eps)
    th = np.pi * (np.arange(M2) + 0.5) / M2
    s = sum(math.sin(th[k]) * O.green7(mu2, g2, k)[0, 0].imag for k in range(M2))
    assert s * math.pi / M2 == pytest.approx(math.pi, abs=1e-12)


def test_det7_matches_library_determinant():
    rng = np.random.default_rng(11)
    for _ in range(20):
        Amat = rng.normal(size=(7, 7)) + 1j * rng.normal(size=(7, 7))
        np.testing.assert_allclose(O.det7(Amat), np.linalg.det(Amat), rtol=1e-12)


def test_det_equals_eigenvalue_ratio_product():
    """Eq. green_delta: Det[1 + G(z) Delta] = prod (eps'_i - z)/(eps_i - z), with
    the exact G(z) = (H - z)^{-1} and the oracle's local 7x7 Delta."""
    L = 4
    sp = inputs.uniform_sphere(L, 2)
    o, th, ph = 22, 2.2, 5.1
    Ht = to_bj_gauge(paper_hamiltonian(L, sp), sp) / A
    sp2 = sp.copy()
    sp2[o] = (th, ph)
    Ht2 = to_bj_gauge(paper_hamiltonian(L, sp2), sp2) / A
    e1, e2 = np.linalg.eigvalsh(Ht), np.linalg.eigvalsh(Ht2)
    D = O.delta7(L, sp, o, th, ph)
    loc = local7(L, o)
    np.testing.assert_allclose(D, (Ht2 - Ht)[np.ix_(loc, loc)], atol=1e-15)
    for z in (-0.5 + 0.05j, 0.1 + 0.02j, 0.63 + 0.2j):
        G = np.linalg.inv(Ht - z * np.eye(L ** 3))[np.ix_(loc, loc)]
        ref = np.prod((e2 - z) / (e1 - z))
        assert abs(O.det_one_plus_gd(G, D) - ref) < 1e-11 * max(1.0, abs(ref))


def test_det_7x7_equals_2x2_reduction():
    """Eq. d_z_green: with |v> = Delta|o>, Det[1 + G Delta]
    = (1 + G_ov)(1 + G_vo) - G_oo G_vv, for any G."""
    L = 4
    sp = inputs.uniform_sphere(L, 4)
    rng = np.random.default_rng(5)
    for o, th, ph in ((0, 1.0, 2.0), (37, 2.9, 0.4)):
        D = O.delta7(L, sp, o, th, ph)
        v = D[:, 0]
        e0 = np.eye(7)[:, 0]
        for _ in range(5):
            G = rng.normal(size=(7, 7)) + 1j * rng.normal(size=(7, 7))
            Gov, Gvo = e0 @ G @ v, v.conj() @ G @ e0
            Goo, Gvv = G[0, 0], v.conj() @ G @ v
            ref = (1 + Gov) * (1 + Gvo) - Goo * Gvv
            assert abs(O.det_one_plus_gd(G, D) - ref) < 1e-12 * max(1, abs(ref))


# --------------------------------------------------------------------------
# Delta Omega (Eq. d_seff2)
# --------------------------------------------------------------------------

def test_identity_proposal_gives_zero():
    L, M = 4, 64
    sp = inputs.uniform_sphere(L, 0)
    for o in (0, 13):
        assert O.delta_omega(L, sp, o, sp[o, 0], sp[o, 1], M) == 0.0


def test_delta_omega_is_rotation_invariant():
    """A rotation of every spin and of the proposal about z leaves every hopping
    <chi_i|chi_j> unchanged, so Delta Omega must agree to rounding.  A general
    rotation leaves the spectra unchanged but moves the proposed spinor's gauge
    relative to the old one at o; det(1 + G Delta) only ignores that gauge for
    the exact G, so with the KPM G it agrees within the expansion's error."""
    L, M = 4, 128
    sp = inputs.uniform_sphere(L, 8)
    o, th, ph = 10, 1.9, 0.7

    def rot(s, ax, ang):
        v = np.stack([np.sin(s[:, 0]) * np.cos(s[:, 1]), np.sin(s[:, 0]) * np.sin(s[:, 1]),
                      np.cos(s[:, 0])], axis=1)
        ax = np.asarray(ax, float) / np.linalg.norm(ax)
        K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
        Rm = np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K
        w = v @ Rm.T
        return np.stack([np.arccos(np.clip(w[:, 2], -1, 1)), np.arctan2(w[:, 1], w[:, 0]) % (2 * np.pi)],
                        axis=1)

    ref = O.delta_omega(L, sp, o, th, ph, M)
    both = np.vstack([sp, [[th, ph]]])
    r = rot(both, (0.0, 0.0, 1.0), 1.1)
    got = O.delta_omega(L, r[:-1], o, r[-1, 0], r[-1, 1], M)
    assert abs(got - ref) < 1e-12
    r = rot(both, (0.3, -1.0, 0.5), 1.1)
    got = O.delta_omega(L, r[:-1], o, r[-1, 0], r[-1, 1], M)
    assert abs(got - ref) < 1e-4


@pytest.mark.parametrize("beta", [1.0, 2.0, 5.0])
def test_delta_omega_converges_to_exact_diagonalisation(beta):
    """KPM Delta Omega against Omega(S') - Omega(S) from the eigenvalues (Sec. 2.1)
    on a 6^3 lattice; the error falls as M grows while the Jackson-smoothed phase
    is resolved by the nodes (max increment well below pi)."""
    L, chem = 6, -2.0
    sp = inputs.uniform_sphere(L, 0)
    total = {128: 0.0, 512: 0.0}
    for o, th, ph in ((0, 1.0, 2.0), (5, 2.5, 0.3), (17, 0.2, 4.0)):
        exact = exact_delta_omega(L, sp, o, th, ph, beta, chem)
        for M in (128, 256, 512):
            mu = O.moments(L, sp, o, M)
            d, inc = O.delta_omega_from_moments(L, sp, mu, O.kernel(M), o, th, ph, beta=beta,
                                                chem=chem)
            assert inc < 1.0
            if M >= 256:
                assert abs(d - exact) < 5e-4, (o, M, d, exact)
            if M in total:
                total[M] += abs(d - exact)
    assert total[512] < total[128]


@pytest.mark.parametrize("factor", [1, 2, 4])
def test_green_sum_rule_on_finer_node_grids(factor):
    """K >= M nodes theta_k = pi (k + 1/2)/K (the FFT nodes of Sec. 2.2 on a
    finer grid): sin(theta) Im G(w) is a polynomial of degree M - 1 in w, so the
    K-node Chebyshev-Gauss rule gives the sum rule pi g_0 mu_0 exactly for every
    K >= M / 2."""
    M, eps = 256, -0.47
    K = factor * M
    g = O.kernel(M, 0)
    mu = np.zeros((7, 7, M), dtype=np.complex128)
    mu[0, 0, :] = cheb_T(np.arange(M), eps)
    th = np.pi * (np.arange(K) + 0.5) / K
    s = sum(math.sin(th[k]) * O.green7(mu, g, k, nodes=K)[0, 0].imag for k in range(K))
    assert s * math.pi / K == pytest.approx(math.pi * g[0], abs=1e-12)
    # and the far field 1/(eps - w) is sampled at the K-grid's own nodes
    ks = np.arange(3, K, 97)
    w = np.cos(th[ks])
    G = np.array([O.green7(mu, g, int(k), nodes=K)[0, 0] for k in ks])
    far = np.abs(w - eps) > 0.3
    np.testing.assert_allclose(G[far].real, 1.0 / (eps - w[far]), rtol=5e-3, atol=5e-3)


def test_identity_proposal_gives_zero_on_2m_nodes():
    L, M = 4, 64
    sp = inputs.uniform_sphere(L, 0)
    for o in (0, 13):
        assert O.delta_omega(L, sp, o, sp[o, 0], sp[o, 1], M, nodes=2 * M) == 0.0


@pytest.mark.parametrize("beta", [1.0, 5.0, 20.0])
def test_2m_nodes_converge_to_exact_diagonalisation(beta):
    """Delta Omega with the Green's function and the quadrature on K = 2M nodes
    against Omega(S') - Omega(S) from the eigenvalues (Sec. 2.1) on a 6^3
    lattice, and against the same expansion on 8M nodes: doubling the nodes
    takes out most of the quadrature error of the M-node rule."""
    L, chem = 6, -2.0
    sp = inputs.uniform_sphere(L, 0)
    q_m = q_2m = 0.0
    for o, th, ph in ((0, 1.0, 2.0), (5, 2.5, 0.3), (17, 0.2, 4.0)):
        exact = exact_delta_omega(L, sp, o, th, ph, beta, chem)
        for M in (256, 512):
            mu = O.moments(L, sp, o, M)
            g = O.kernel(M)
            d = {K: O.delta_omega_from_moments(L, sp, mu, g, o, th, ph, beta=beta, chem=chem, nodes=K)[0]
                 for K in (M, 2 * M, 8 * M)}
            tol = 5e-4 if beta < 20 else 3.5e-3  # site 17 at beta = 20 sits on a sharp feature
            assert abs(d[2 * M] - exact) < tol, (o, M, d[2 * M], exact)
            q_m += abs(d[M] - d[8 * M])
            q_2m += abs(d[2 * M] - d[8 * M])
    assert q_2m < 0.05 * q_m, (q_2m, q_m)


# --------------------------------------------------------------------------
# Philox4x32-10 and the Metropolis sweep (Algorithm 1)
# --------------------------------------------------------------------------

def _philox_ref(ctr, key):
    """Philox4x32-10 restated from its published definition (Salmon et al., SC'11):
    ten rounds of two 32x32->64 multiplies with an xor-permutation, key bumped by
    the Weyl constants between rounds."""
    MASK = 0xFFFFFFFF
    c = list(ctr)
    k0, k1 = key
    for r in range(10):
        if r:
            k0 = (k0 + 0x9E3779B9) & MASK
            k1 = (k1 + 0xBB67AE85) & MASK
        p0 = 0xD2511F53 * c[0]
        p1 = 0xCD9E8D57 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k0) & MASK, p1 & MASK, ((p0 >> 32) ^ c[3] ^ k1) & MASK, p0 & MASK]
    return c


def test_philox_matches_second_implementation():
    rng = np.random.default_rng(0)
    for _ in range(200):
        ctr = [int(v) for v in rng.integers(0, 2 ** 32, 4)]
        key = [int(v) for v in rng.integers(0, 2 ** 32, 2)]
        assert O.philox4x32_10(ctr, key) == _philox_ref(ctr, key)


def test_philox_known_answers():
    """Philox4x32-10 against the known-answer vectors published with the
    generator (Salmon, Moraes, Dror, Shaw, SC'11, and the known-answer file of
    its reference distribution, Random123): a wrong multiplier, Weyl constant,
    round count or output permutation changes every one of them."""
    kat = [
        ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for ctr, key, want in kat:
        assert O.philox4x32_10(list(ctr), list(key)) == list(want)


def test_results_do_not_depend_on_the_thread_count():
    """The oracle's parallel loops (sites of Htilde x and of the recursion,
    nodes of the Green's function) leave every result bitwise unchanged."""
    L, M = 6, 128
    sp = inputs.uniform_sphere(L, 3)
    nmax = max(2, O.max_threads())
    out = {}
    for n in (1, nmax):
        O.set_threads(n)
        mu = O.moments(L, sp, 17, M)
        d = O.delta_omega(L, sp, 17, 1.1, 0.4, M, beta=20.0, chem=-2.0)
        res = O.updates(L, sp, 6, M, beta=20.0, chem=-2.0, seed=1)
        out[n] = (mu, d, res["d_omega"], res["spins"])
    O.set_threads(nmax)
    a, b = out[1], out[nmax]
    np.testing.assert_array_equal(a[0], b[0])
    assert a[1] == b[1]
    np.testing.assert_array_equal(a[2], b[2])
    np.testing.assert_array_equal(a[3], b[3])


def test_draws_are_uniform():
    n = 20000
    d = np.array([O.draw(1, 0, u) for u in range(n)])
    cos_t = np.cos(d[:, 0])
    for col in (0.5 * (1 - cos_t), d[:, 1] / (2 * np.pi), d[:, 2]):
        assert col.min() >= 0.0 and col.max() < 1.0
        counts = np.histogram(col, bins=20, range=(0, 1))[0]
        chi2 = np.sum((counts - n / 20) ** 2 / (n / 20))
        assert chi2 < 50.0  # 19 dof, p ~ 1e-4
    # distinct chains draw distinct streams
    assert O.draw(1, 0, 5) != O.draw(1, 1, 5)


def test_updates_follow_metropolis_rule():
    L, M = 3, 32
    sp = inputs.uniform_sphere(L, 0)
    res = O.updates(L, sp, 2 * L ** 3, M, beta=20.0)
    acc = res["decisions"].astype(bool)
    np.testing.assert_array_equal(acc, res["ratio"] > res["u"])
    np.testing.assert_allclose(res["ratio"], np.exp(-20.0 * res["d_omega"]), rtol=1e-15)
    assert 0 < acc.sum() < acc.size
    assert res["magnetization"].shape == (2,)
    # replay: spins change exactly at accepted updates, to the drawn proposal
    s = sp.copy()
    for q in range(acc.size):
        th, ph, u = O.draw(1, 0, q)
        assert u == res["u"][q]
        if acc[q]:
            s[q % L ** 3] = (th, ph)
    np.testing.assert_array_equal(s, res["spins"])
    assert res["magnetization"][-1] == pytest.approx(O.magnetization(L, s), abs=0)
    # forced decisions are honoured
    forced = np.full(acc.size, -1, dtype=np.int8)
    forced[3] = 1 - acc[3]
    res2 = O.updates(L, sp, 4, M, beta=20.0, forced=forced[:4])
    assert res2["decisions"][3] == 1 - acc[3]


def test_magnetization_limits():
    assert O.magnetization(4, inputs.ferromagnet(4)) == pytest.approx(1.0, abs=1e-15)
    assert O.magnetization(8, inputs.uniform_sphere(8, 0)) < 0.1


def test_grand_potential_limits_and_particle_number():
    """Pins of Omega(beta, mu) = -(1/beta) sum ln(1 + e^{-beta(e - mu)}) that do
    not restate it: the zero-temperature limit sum_{e < mu} (e - mu) (error at
    most n ln2 / beta), the high-temperature expansion of ln(1 + e^x) =
    ln 2 + x/2 + x^2/8 + O(x^4), and -dOmega/dmu = N = sum of Fermi factors."""
    rng = np.random.default_rng(3)
    e = np.sort(rng.uniform(-6.0, 6.0, 40))
    mu = -0.7
    # T -> 0: the occupied levels' e - mu
    for beta in (1e3, 1e5):
        om = O.grand_potential(e, beta, mu)
        assert abs(om - np.sum(np.minimum(e - mu, 0.0))) <= len(e) * np.log(2.0) / beta
    # T -> infinity: -(1/beta) (n ln2 + sum x/2 + sum x^2/8), x = -beta (e - mu)
    beta = 1e-3
    x = -beta * (e - mu)
    hot = -(len(e) * np.log(2.0) + x.sum() / 2 + (x ** 2).sum() / 8) / beta
    assert O.grand_potential(e, beta, mu) == pytest.approx(hot, abs=len(e) * np.max(np.abs(x)) ** 4 / beta)
    # particle number: centred difference in mu against the Fermi sum
    for beta in (0.5, 5.0, 20.0):
        h = 1e-5
        n_fd = -(O.grand_potential(e, beta, mu + h) - O.grand_potential(e, beta, mu - h)) / (2 * h)
        fermi = np.sum(1.0 / (1.0 + np.exp(beta * (e - mu))))
        assert n_fd == pytest.approx(fermi, rel=1e-7, abs=1e-7)


def test_grand_potential_matches_definition():
    e = np.linspace(-5, 5, 11)
    for beta in (0.5, 20.0, 200.0):
        ref = -np.sum(np.log1p(np.exp(np.clip(-beta * (e + 2.0), -700, 700)))) / beta
        if beta < 100:
            assert O.grand_potential(e, beta, -2.0) == pytest.approx(ref, rel=1e-13)
        else:
            assert np.isfinite(O.grand_potential(e, beta, -2.0))
