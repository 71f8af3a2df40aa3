"""ctypes wrapper of the GFMC oracle (TEST INFRASTRUCTURE ONLY).

The oracle is the plain FP64 CPU restatement of the GFMC single-spin update of
arXiv:1303.6016 (Sec. 2.2 and Algorithm 1) in ``gfmc_oracle.c``.  Only the
tests, the smoke check and the CPU-baseline leg of the benchmark may import
this module.  It shares nothing with the CUDA path: it neither imports the
package nor is imported by it.

Array conventions (numpy):
  spins    float64 [N, 2]   (theta, phi) per site, N = L**3, site = x + L*(y + L*z)
  moments  complex128 [7, 7, M]   mu[j, k, n] = <l_j| T_n(Htilde) |l_k>
           local order 0 = o, 1 = +x, 2 = -x, 3 = +y, 4 = -y, 5 = +z, 6 = -z
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gfmc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, strict IEEE: no fast-math), with
    OpenMP when the compiler has it (the site and node loops then run on
    ``set_threads`` threads; results are bitwise the same for any count)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off"]
        try:
            subprocess.check_call(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base + [_SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        d = ctypes.POINTER(ctypes.c_double)
        i8 = ctypes.POINTER(ctypes.c_int8)
        u8 = ctypes.POINTER(ctypes.c_uint8)
        u32 = ctypes.POINTER(ctypes.c_uint32)
        lp = ctypes.POINTER(ctypes.c_long)
        c_int, c_long, c_double = ctypes.c_int, ctypes.c_long, ctypes.c_double
        L.orc_local_sites.argtypes = [c_int, c_long, lp]
        L.orc_dense_htilde.argtypes = [c_int, d, c_double, c_double, d]
        L.orc_apply_htilde.argtypes = [c_int, d, c_double, c_double, d, d]
        L.orc_moments.argtypes = [c_int, d, c_double, c_double, c_long, c_int, d]
        L.orc_kernel.argtypes = [c_int, c_int, c_double, d]
        L.orc_green7.argtypes = [c_int, c_int, d, d, c_int, d]
        L.orc_delta7.argtypes = [c_int, d, c_double, c_double, c_long, c_double, c_double, d]
        L.orc_det_one_plus_gd.argtypes = [d, d, d]
        L.orc_det7.argtypes = [d, d]
        L.orc_delta_omega_from_moments.argtypes = [c_int, d, c_double, c_double, c_double,
                                                   c_double, c_int, c_int, d, d, c_long, c_double,
                                                   c_double, d, d]
        L.orc_delta_omega.argtypes = [c_int, d, c_double, c_double, c_double, c_double, c_int,
                                      c_int, c_int, c_double, c_long, c_double, c_double, d]
        L.orc_grand_potential.argtypes = [c_long, d, c_double, c_double]
        L.orc_grand_potential.restype = c_double
        L.orc_philox4x32_10.argtypes = [u32, u32, u32]
        L.orc_philox4x32_10.restype = None
        L.orc_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, d, d, d]
        L.orc_draw.restype = None
        L.orc_magnetization.argtypes = [c_int, d]
        L.orc_magnetization.restype = c_double
        L.orc_set_threads.argtypes = [c_int]
        L.orc_set_threads.restype = None
        L.orc_max_threads.argtypes = []
        L.orc_max_threads.restype = c_int
        L.orc_updates.argtypes = [c_int, d, c_double, c_double, c_double, c_double, c_int, c_int,
                                  c_int, c_double, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                  c_long, i8, u8, d, d, d, lp]
        _lib = L
    return _lib


def set_threads(n: int) -> None:
    """Threads of the oracle's site and node loops (1: single-threaded)."""
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    """Threads the next oracle call will use (1 without OpenMP)."""
    return int(lib().orc_max_threads())


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(st, what):
    if st != 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


def _spins(spins):
    s = np.ascontiguousarray(spins, dtype=np.float64).reshape(-1, 2)
    return s


DEFAULT_SCALE = 6.05  # a = 6.05 |t|


def local_sites(L: int, o: int) -> np.ndarray:
    out = (ctypes.c_long * 7)()
    lib().orc_local_sites(L, o, out)
    return np.array(list(out), dtype=np.int64)


def dense_htilde(L, spins, t=1.0, a=None):
    a = DEFAULT_SCALE * abs(t) if a is None else a
    N = L ** 3
    H = np.zeros((N, N), dtype=np.complex128)
    s = _spins(spins)
    _check(lib().orc_dense_htilde(L, _dp(s), t, a, _dp(H.view(np.float64))), "dense_htilde")
    return H


def apply_htilde(L, spins, x, t=1.0, a=None):
    a = DEFAULT_SCALE * abs(t) if a is None else a
    s = _spins(spins)
    x = np.ascontiguousarray(x, dtype=np.complex128)
    y = np.zeros_like(x)
    _check(lib().orc_apply_htilde(L, _dp(s), t, a, _dp(x.view(np.float64)),
                                  _dp(y.view(np.float64))), "apply_htilde")
    return y


def moments(L, spins, site, M, t=1.0, a=None):
    a = DEFAULT_SCALE * abs(t) if a is None else a
    s = _spins(spins)
    mu = np.zeros((7, 7, M), dtype=np.complex128)
    _check(lib().orc_moments(L, _dp(s), t, a, site, M, _dp(mu.view(np.float64))), "moments")
    return mu


def kernel(M, kind=0, lam=4.0):
    g = np.zeros(M, dtype=np.float64)
    _check(lib().orc_kernel(kind, M, lam, _dp(g)), "kernel")
    return g


def green7(mu, g, k, nodes=None):
    """7x7 Green's matrix at node k of `nodes` (default M) Chebyshev nodes."""
    mu = np.ascontiguousarray(mu, dtype=np.complex128)
    g = np.ascontiguousarray(g, dtype=np.float64)
    M = mu.shape[-1]
    K = M if nodes is None else int(nodes)
    G = np.zeros((7, 7), dtype=np.complex128)
    _check(lib().orc_green7(M, K, _dp(mu.view(np.float64)), _dp(g), k, _dp(G.view(np.float64))),
           "green7")
    return G


def delta7(L, spins, site, theta_new, phi_new, t=1.0, a=None):
    a = DEFAULT_SCALE * abs(t) if a is None else a
    s = _spins(spins)
    D = np.zeros((7, 7), dtype=np.complex128)
    _check(lib().orc_delta7(L, _dp(s), t, a, site, theta_new, phi_new,
                            _dp(D.view(np.float64))), "delta7")
    return D


def det_one_plus_gd(G, D):
    G = np.ascontiguousarray(G, dtype=np.complex128)
    D = np.ascontiguousarray(D, dtype=np.complex128)
    out = np.zeros(2)
    lib().orc_det_one_plus_gd(_dp(G.view(np.float64)), _dp(D.view(np.float64)), _dp(out))
    return complex(out[0], out[1])


def det7(A):
    A = np.ascontiguousarray(A, dtype=np.complex128)
    out = np.zeros(2)
    lib().orc_det7(_dp(A.view(np.float64)), _dp(out))
    return complex(out[0], out[1])


def delta_omega_from_moments(L, spins, mu, g, site, theta_new, phi_new, t=1.0, chem=-2.0,
                             beta=20.0, a=None, nodes=None):
    a = DEFAULT_SCALE * abs(t) if a is None else a
    s = _spins(spins)
    mu = np.ascontiguousarray(mu, dtype=np.complex128)
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros(1)
    inc = np.zeros(1)
    K = mu.shape[-1] if nodes is None else int(nodes)
    _check(lib().orc_delta_omega_from_moments(L, _dp(s), t, chem, beta, a, mu.shape[-1], K,
                                              _dp(mu.view(np.float64)), _dp(g), site,
                                              theta_new, phi_new, _dp(out), _dp(inc)),
           "delta_omega_from_moments")
    return float(out[0]), float(inc[0])


def delta_omega(L, spins, site, theta_new, phi_new, M, t=1.0, chem=-2.0, beta=20.0, a=None,
                kernel_kind=0, lam=4.0, nodes=None):
    a = DEFAULT_SCALE * abs(t) if a is None else a
    s = _spins(spins)
    out = np.zeros(1)
    K = M if nodes is None else int(nodes)
    _check(lib().orc_delta_omega(L, _dp(s), t, chem, beta, a, M, K, kernel_kind, lam, site,
                                 theta_new, phi_new, _dp(out)), "delta_omega")
    return float(out[0])


def grand_potential(eps, beta, chem):
    e = np.ascontiguousarray(eps, dtype=np.float64)
    return lib().orc_grand_potential(e.size, _dp(e), beta, chem)


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def draw(seed, chain_id, upd):
    th, ph, u = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().orc_draw(seed, chain_id, upd, ctypes.byref(th), ctypes.byref(ph), ctypes.byref(u))
    return th.value, ph.value, u.value


def magnetization(L, spins):
    s = _spins(spins)
    return lib().orc_magnetization(L, _dp(s))


def updates(L, spins, n_updates, M, t=1.0, chem=-2.0, beta=20.0, a=None, kernel_kind=0,
            lam=4.0, seed=1, chain_id=0, upd0=0, forced=None, nodes=None):
    """Run n_updates sequential updates (Green's function and quadrature on
    `nodes` Chebyshev nodes, default M); returns a dict with the new spins and
    traces."""
    a = DEFAULT_SCALE * abs(t) if a is None else a
    s = _spins(spins).copy()
    n = int(n_updates)
    dec = np.zeros(n, dtype=np.uint8)
    dom = np.zeros(n, dtype=np.float64)
    ru = np.zeros((n, 2), dtype=np.float64)
    N = L ** 3
    mag = np.zeros(n // N + 2, dtype=np.float64)
    nmag = ctypes.c_long(0)
    fp = None
    if forced is not None:
        f = np.ascontiguousarray(forced, dtype=np.int8)
        fp = f.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))
    K = M if nodes is None else int(nodes)
    _check(lib().orc_updates(L, _dp(s), t, chem, beta, a, M, K, kernel_kind, lam, seed, chain_id,
                             upd0, n, fp, dec.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                             _dp(dom), _dp(ru), _dp(mag), ctypes.byref(nmag)), "updates")
    return {"spins": s, "decisions": dec, "d_omega": dom, "ratio": ru[:, 0], "u": ru[:, 1],
            "magnetization": mag[: nmag.value]}
