"""Python binding of libgfmc.so (the C ABI in include/gfmc.h).

Argument marshalling only: every step of a GFMC update runs in the CUDA
kernels behind the C ABI.  The library must have been built
(``python -m paper_1303_6016_gb300.build`` or ``__graft_entry__.build()``);
without it every call raises -- there is no CPU fallback.

    from paper_1303_6016_gb300 import gfmc, inputs
    ch = gfmc.Chain(L=16, spins=inputs.uniform_sphere(16, 0), M=1024, beta=20.0, mu=-2.0)
    mu = ch.moments(site=0)                       # complex128 [7, 7, M]
    dO = ch.delta_omega(0, theta_new, phi_new)    # float, units of t
    out = ch.updates(4096)                         # decisions, Delta Omega trace, ...
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgfmc.so")

GFMC_OK, GFMC_EINVAL, GFMC_ENOMEM, GFMC_ECUDA, GFMC_ETIMEOUT, GFMC_ENUMERIC = range(6)
PRECISIONS = {"fp64": 0, "fp32_mixed": 1}
KERNELS = {"jackson": 0, "lorentz": 1}
RECURSIONS = {"unit_vectors": 0, "proposal": 1}
ENGINES = {"auto": 0, "grid": 1, "vector_clusters": 2}

# Names exported by libgfmc.so; include/gfmc.h declares exactly these.
EXPORTS = ("gfmc_default_options", "gfmc_create", "gfmc_moments", "gfmc_delta_omega",
           "gfmc_updates", "gfmc_sweep", "gfmc_get_spins", "gfmc_set_state", "gfmc_get_counter", "gfmc_device_bytes",
           "gfmc_set_wait_budget", "gfmc_inject_stall", "gfmc_last_error", "gfmc_destroy",
           "gfmc_delta_omega_noalloc", "gfmc_run_batch", "gfmc_run_clusters", "gfmc_cluster_min_ctas",
           "gfmc_plan_create", "gfmc_plan_launch", "gfmc_plan_sync", "gfmc_plan_destroy",
           "gfmc_server_create",
           "gfmc_server_submit",
           "gfmc_server_poll", "gfmc_server_last_error", "gfmc_server_destroy",
           "gfmc_measure_fma_peak", "gfmc_measure_fp64_issue", "gfmc_measure_cluster_exchange")


class GfmcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"gfmc status {status}: {message}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("kernel", ctypes.c_int),
                ("lorentz_lambda", ctypes.c_double), ("spectral_scale", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("chain_id", ctypes.c_uint32),
                ("stream", ctypes.c_void_p), ("num_ctas", ctypes.c_int), ("recursion", ctypes.c_int),
                ("nodes", ctypes.c_int), ("engine", ctypes.c_int), ("compensated", ctypes.c_int)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libgfmc.so and declare its signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA engine first "
                           "(python -m paper_1303_6016_gb300.build); there is no fallback")
    L = ctypes.CDLL(path)
    vp, d, i64, u64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_uint64
    L.gfmc_default_options.argtypes = [ctypes.POINTER(Options)]
    L.gfmc_default_options.restype = None
    L.gfmc_create.argtypes = [ctypes.c_int, d, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                              ctypes.c_int, ctypes.POINTER(Options), ctypes.POINTER(vp)]
    L.gfmc_moments.argtypes = [vp, i64, d]
    L.gfmc_delta_omega.argtypes = [vp, i64, ctypes.c_double, ctypes.c_double, d]
    L.gfmc_updates.argtypes = [vp, i64, ctypes.POINTER(u64), ctypes.POINTER(ctypes.c_uint8), d, d,
                               ctypes.POINTER(i64)]
    L.gfmc_sweep.argtypes = [vp, ctypes.c_int, ctypes.POINTER(u64), d, ctypes.POINTER(ctypes.c_uint8), d]
    L.gfmc_get_spins.argtypes = [vp, d]
    L.gfmc_set_state.argtypes = [vp, d, u64]
    L.gfmc_get_counter.argtypes = [vp, ctypes.POINTER(u64)]
    L.gfmc_device_bytes.argtypes = [vp, ctypes.POINTER(u64)]
    L.gfmc_set_wait_budget.argtypes = [vp, i64]
    L.gfmc_inject_stall.argtypes = [vp, ctypes.c_int]
    L.gfmc_last_error.argtypes = [vp]
    L.gfmc_last_error.restype = ctypes.c_char_p
    L.gfmc_destroy.argtypes = [vp]
    L.gfmc_destroy.restype = None
    L.gfmc_delta_omega_noalloc.argtypes = [ctypes.c_int, vp, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, i64, ctypes.c_double, ctypes.c_double, vp, vp,
                                           ctypes.c_char_p, ctypes.c_size_t]
    L.gfmc_delta_omega_noalloc.restype = ctypes.c_int
    L.gfmc_run_batch.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(u64), ctypes.POINTER(ctypes.POINTER(ctypes.c_uint8)),
                                 ctypes.POINTER(ctypes.POINTER(ctypes.c_double)),
                                 ctypes.POINTER(ctypes.POINTER(ctypes.c_double)), ctypes.POINTER(i64), vp]
    L.gfmc_run_batch.restype = ctypes.c_int
    L.gfmc_run_clusters.argtypes = L.gfmc_run_batch.argtypes
    L.gfmc_run_clusters.restype = ctypes.c_int
    L.gfmc_cluster_min_ctas.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.gfmc_cluster_min_ctas.restype = ctypes.c_int
    L.gfmc_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int),
                                   ctypes.c_int, ctypes.POINTER(vp)]
    L.gfmc_plan_create.restype = ctypes.c_int
    L.gfmc_plan_launch.argtypes = [vp, ctypes.c_int, vp]
    L.gfmc_plan_launch.restype = ctypes.c_int
    L.gfmc_plan_sync.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(ctypes.POINTER(ctypes.c_uint8)),
                                 ctypes.POINTER(ctypes.POINTER(ctypes.c_double)),
                                 ctypes.POINTER(ctypes.POINTER(ctypes.c_double)), ctypes.POINTER(i64)]
    L.gfmc_plan_sync.restype = ctypes.c_int
    L.gfmc_plan_destroy.argtypes = [vp]
    L.gfmc_plan_destroy.restype = None
    L.gfmc_server_create.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.POINTER(vp)]
    L.gfmc_server_create.restype = ctypes.c_int
    L.gfmc_server_submit.argtypes = [vp, ctypes.c_int, vp, i64, ctypes.POINTER(ctypes.c_uint8), d]
    L.gfmc_server_submit.restype = ctypes.c_int
    L.gfmc_server_poll.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(u64)]
    L.gfmc_server_poll.restype = ctypes.c_int
    L.gfmc_server_last_error.argtypes = [vp]
    L.gfmc_server_last_error.restype = ctypes.c_char_p
    L.gfmc_server_destroy.argtypes = [vp]
    L.gfmc_server_destroy.restype = None
    L.gfmc_measure_fma_peak.argtypes = [ctypes.c_int, ctypes.c_int, d, vp]
    L.gfmc_measure_fma_peak.restype = ctypes.c_int
    L.gfmc_measure_fp64_issue.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, d, vp]
    L.gfmc_measure_fp64_issue.restype = ctypes.c_int
    L.gfmc_measure_cluster_exchange.argtypes = [ctypes.c_int, ctypes.c_int, d, vp]
    L.gfmc_measure_cluster_exchange.restype = ctypes.c_int
    for name in ("gfmc_create", "gfmc_moments", "gfmc_delta_omega", "gfmc_updates", "gfmc_sweep",
                 "gfmc_get_spins", "gfmc_set_state", "gfmc_get_counter", "gfmc_device_bytes", "gfmc_set_wait_budget",
                 "gfmc_inject_stall"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _host_spins(spins) -> np.ndarray:
    """Spins (theta, phi) as a contiguous host float64 [N][2] array, from a numpy
    array or a torch tensor on any device (the library copies host spins)."""
    if hasattr(spins, "detach") and hasattr(spins, "cpu"):
        spins = spins.detach().cpu().numpy()
    return np.ascontiguousarray(spins, dtype=np.float64).reshape(-1, 2)


def current_stream_handle():
    """The raw cudaStream_t of torch's current stream, or None (default stream)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream) or None
    except Exception:  # torch absent or without CUDA
        pass
    return None


class Chain:
    """One GFMC Markov chain resident on the GPU (a gfmc_t handle)."""

    def __init__(self, L: int, spins, t: float = 1.0, mu: float = -2.0, beta: float = 20.0,
                 M: int = 256, precision: str = "fp64", kernel: str = "jackson",
                 lorentz_lambda: float = 4.0, spectral_scale: float = 0.0, seed: int = 1,
                 chain_id: int = 0, stream=None, num_ctas: int = 0, recursion: str = "unit_vectors",
                 nodes: int = 0, engine: str = "auto", compensated: bool = False):
        lib = load()
        self.L, self.N, self.M = int(L), int(L) ** 3, int(M)
        self.K = int(nodes) if nodes else self.M  # Chebyshev nodes of G and of the quadrature
        self.t, self.mu, self.beta = float(t), float(mu), float(beta)
        self.precision = precision
        self.recursion = recursion
        opt = Options()
        lib.gfmc_default_options(ctypes.byref(opt))
        opt.precision = PRECISIONS[precision]
        opt.kernel = KERNELS[kernel]
        opt.lorentz_lambda = float(lorentz_lambda)
        opt.spectral_scale = float(spectral_scale)
        opt.seed = int(seed)
        opt.chain_id = int(chain_id)
        s = current_stream_handle() if stream is None else stream
        opt.stream = s if s else None
        opt.num_ctas = int(num_ctas)
        opt.recursion = RECURSIONS[recursion]
        opt.nodes = int(nodes)
        opt.engine = ENGINES[engine]
        opt.compensated = 1 if compensated else 0
        self.engine = engine
        self.compensated = bool(compensated)
        sp = _host_spins(spins)
        if sp.shape[0] != self.N:
            raise ValueError(f"spins has {sp.shape[0]} rows, expected N = {self.N}")
        h = ctypes.c_void_p()
        st = lib.gfmc_create(self.L, _dp(sp), self.t, self.mu, self.beta, self.M, ctypes.byref(opt),
                             ctypes.byref(h))
        if st != GFMC_OK:
            raise GfmcError(st, lib.gfmc_last_error(None).decode())
        self._h = h
        self._lib = lib

    # -- helpers --
    def _check(self, st):
        if st != GFMC_OK:
            raise GfmcError(st, self._lib.gfmc_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gfmc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- API --
    def moments(self, site: int) -> np.ndarray:
        mu = np.zeros((7, 7, self.M), dtype=np.complex128)
        self._check(self._lib.gfmc_moments(self._h, int(site), _dp(mu.view(np.float64))))
        return mu

    def delta_omega(self, site: int, theta_new: float, phi_new: float) -> float:
        out = np.zeros(1)
        self._check(self._lib.gfmc_delta_omega(self._h, int(site), float(theta_new), float(phi_new),
                                               _dp(out)))
        return float(out[0])

    def updates(self, n: int, trace: bool = True) -> dict:
        n = int(n)
        acc = ctypes.c_uint64(0)
        nmag = ctypes.c_int64(0)
        dec = np.zeros(n if trace else 0, dtype=np.uint8)
        dom = np.zeros(n if trace else 0, dtype=np.float64)
        mag = np.zeros(n // self.N + 2, dtype=np.float64)
        self._check(self._lib.gfmc_updates(
            self._h, n, ctypes.byref(acc),
            dec.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)) if trace else None,
            _dp(dom) if trace else None, _dp(mag), ctypes.byref(nmag)))
        return {"n_accepted": int(acc.value), "decisions": dec, "d_omega": dom,
                "magnetization": mag[: nmag.value]}

    def updates_into(self, n: int, decisions=None, d_omega=None, magnetization=None) -> tuple:
        """gfmc_updates writing into caller-owned (e.g. pinned) numpy buffers;
        returns (n_accepted, n_magnetisations)."""
        acc = ctypes.c_uint64(0)
        nmag = ctypes.c_int64(0)
        self._check(self._lib.gfmc_updates(
            self._h, int(n), ctypes.byref(acc),
            decisions.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)) if decisions is not None else None,
            _dp(d_omega) if d_omega is not None else None,
            _dp(magnetization) if magnetization is not None else None, ctypes.byref(nmag)))
        return int(acc.value), int(nmag.value)

    def sweep(self, n_sweeps: int = 1, trace: bool = True) -> dict:
        return self.updates(int(n_sweeps) * self.N, trace=trace)

    def get_spins(self, out=None) -> np.ndarray:
        if out is None:
            out = np.zeros((self.N, 2), dtype=np.float64)
        self._check(self._lib.gfmc_get_spins(self._h, _dp(out)))
        return out

    def set_state(self, spins, counter: int):
        sp = _host_spins(spins)
        self._check(self._lib.gfmc_set_state(self._h, _dp(sp), int(counter)))

    def set_wait_budget(self, cycles: int):
        self._check(self._lib.gfmc_set_wait_budget(self._h, int(cycles)))

    def inject_stall(self, enable: bool = True):
        self._check(self._lib.gfmc_inject_stall(self._h, 1 if enable else 0))

    @property
    def device_bytes(self) -> int:
        """Bytes of device memory the handle holds."""
        b = ctypes.c_uint64(0)
        self._check(self._lib.gfmc_device_bytes(self._h, ctypes.byref(b)))
        return int(b.value)

    @property
    def counter(self) -> int:
        c = ctypes.c_uint64(0)
        self._check(self._lib.gfmc_get_counter(self._h, ctypes.byref(c)))
        return int(c.value)


def fma_peak_tflops(precision: str = "fp64", repeats: int = 3, stream=None) -> float:
    """Fused multiply-add throughput of the current GPU (gfmc_measure_fma_peak)."""
    lib = load()
    out = np.zeros(1)
    st = lib.gfmc_measure_fma_peak(PRECISIONS[precision], int(repeats), _dp(out), stream)
    if st != GFMC_OK:
        raise GfmcError(st, "gfmc_measure_fma_peak failed")
    return float(out[0])


def fp64_issue_rate(chains: int, warps: int, lanes: int = 32, repeats: int = 2, stream=None) -> float:
    """FP64 fma warp-lane slots an SM retires per clock at one CTA of 256
    threads per SM (gfmc_measure_fp64_issue)."""
    lib = load()
    out = np.zeros(1)
    st = lib.gfmc_measure_fp64_issue(int(chains), int(warps), int(lanes), int(repeats), _dp(out), stream)
    if st != GFMC_OK:
        raise GfmcError(st, "gfmc_measure_fp64_issue failed")
    return float(out[0])


def cluster_exchange_cycles(steps: int = 2000, repeats: int = 3, stream=None) -> float:
    """SM cycles per step of the FP32 vector-cluster engine's exchange alone
    (gfmc_measure_cluster_exchange)."""
    lib = load()
    out = np.zeros(1)
    st = lib.gfmc_measure_cluster_exchange(int(steps), int(repeats), _dp(out), stream)
    if st != GFMC_OK:
        raise GfmcError(st, "gfmc_measure_cluster_exchange failed")
    return float(out[0])


def run_clusters(chains, n_updates, cluster_ctas, trace=True, stream=None) -> list:
    """Chains on the proposal-vector recursion, each on one thread-block
    cluster holding its lattice in shared memory (gfmc_run_clusters)."""
    return run_batch(chains, n_updates, cluster_ctas, trace, stream, _fn="gfmc_run_clusters")


SCHEDULES = {"teams": 0, "clusters": 1}


class Plan:
    """One step of a batch captured in a CUDA graph (gfmc_plan_*): every chain
    runs n_updates[c] updates per step; launch() enqueues steps, sync() waits
    and returns the last step's results per chain.  While the plan exists its
    chains belong to it."""

    def __init__(self, chains, n_updates, ctas, schedule: str = "clusters"):
        lib = load()
        self._lib = lib
        self.chains = list(chains)
        n = len(self.chains)
        self.n_updates = [int(u) for u in (n_updates if hasattr(n_updates, "__len__") else [n_updates] * n)]
        H = (ctypes.c_void_p * n)(*[c._h.value for c in self.chains])
        NU = (ctypes.c_int64 * n)(*self.n_updates)
        TC = (ctypes.c_int * n)(*[int(t) for t in ctas])
        h = ctypes.c_void_p()
        st = lib.gfmc_plan_create(H, n, NU, TC, SCHEDULES[schedule], ctypes.byref(h))
        if st != GFMC_OK:
            raise GfmcError(st, lib.gfmc_last_error(None).decode())
        self._h = h
        self._stream = None
        self._decs = [np.zeros(u, dtype=np.uint8) for u in self.n_updates]
        self._doms = [np.zeros(u, dtype=np.float64) for u in self.n_updates]

    def launch(self, n_steps: int = 1, stream=None):
        if stream is None:
            stream = current_stream_handle()
        st = self._lib.gfmc_plan_launch(self._h, int(n_steps), stream)
        if st != GFMC_OK:
            raise GfmcError(st, self._lib.gfmc_last_error(None).decode())

    def sync(self, trace: bool = True) -> list:
        n = len(self.chains)
        acc = (ctypes.c_uint64 * n)()
        NM = (ctypes.c_int64 * n)()
        DP = (ctypes.POINTER(ctypes.c_uint8) * n)(*[d.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
                                                      for d in self._decs]) if trace else None
        OP = (ctypes.POINTER(ctypes.c_double) * n)(*[_dp(d) for d in self._doms]) if trace else None
        st = self._lib.gfmc_plan_sync(self._h, acc, DP, OP, None, NM)
        if st != GFMC_OK:
            raise GfmcError(st, self._lib.gfmc_last_error(None).decode())
        return [{"n_accepted": int(acc[c]), "decisions": self._decs[c].copy() if trace else None,
                 "d_omega": self._doms[c].copy() if trace else None} for c in range(n)]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.gfmc_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cluster_min_ctas(L: int, M: int, precision: str = "fp32_mixed") -> int:
    """Smallest cluster size that holds an L^3 lattice with M moments."""
    lib = load()
    out = ctypes.c_int(0)
    st = lib.gfmc_cluster_min_ctas(int(L), int(M), PRECISIONS[precision], ctypes.byref(out))
    if st != GFMC_OK:
        raise GfmcError(st, lib.gfmc_last_error(None).decode())
    return out.value


def run_batch(chains, n_updates, team_ctas=None, trace=True, stream=None, _fn="gfmc_run_batch") -> list:
    """One launch over several chains (each on its own team of CTAs).
    Returns one dict per chain with n_accepted and, if trace, the decisions and
    Delta Omega trace."""
    lib = load()
    n = len(chains)
    H = (ctypes.c_void_p * n)(*[c._h.value for c in chains])
    NU = (ctypes.c_int64 * n)(*[int(u) for u in (n_updates if hasattr(n_updates, "__len__") else [n_updates] * n)])
    TC = (ctypes.c_int * n)(*[int(t) for t in team_ctas]) if team_ctas is not None else None
    acc = (ctypes.c_uint64 * n)()
    decs = [np.zeros(int(NU[c]), dtype=np.uint8) for c in range(n)]
    doms = [np.zeros(int(NU[c]), dtype=np.float64) for c in range(n)]
    DP = (ctypes.POINTER(ctypes.c_uint8) * n)(*[d.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)) for d in decs])
    OP = (ctypes.POINTER(ctypes.c_double) * n)(*[_dp(d) for d in doms])
    mags = [np.zeros(int(NU[c]) // chains[c].N + 2, dtype=np.float64) for c in range(n)]
    MP = (ctypes.POINTER(ctypes.c_double) * n)(*[_dp(m) for m in mags])
    NM = (ctypes.c_int64 * n)()
    if stream is None:
        stream = current_stream_handle()
    st = getattr(lib, _fn)(H, n, NU, TC, acc, DP if trace else None, OP if trace else None, MP, NM, stream)
    if st != GFMC_OK:
        raise GfmcError(st, lib.gfmc_last_error(None).decode())
    return [{"n_accepted": int(acc[c]), "decisions": decs[c], "d_omega": doms[c],
             "magnetization": mags[c][: int(NM[c])]} for c in range(n)]


class Server:
    """A device-resident request loop (gfmc_server_t) with n slots of CTAs."""

    def __init__(self, slot_ctas, max_M: int = 2048):
        self._lib = load()
        self.slot_ctas = [int(c) for c in slot_ctas]
        arr = (ctypes.c_int * len(self.slot_ctas))(*self.slot_ctas)
        h = ctypes.c_void_p()
        st = self._lib.gfmc_server_create(len(self.slot_ctas), arr, int(max_M), ctypes.byref(h))
        if st != GFMC_OK:
            raise GfmcError(st, self._lib.gfmc_server_last_error(None).decode())
        self._h = h
        self._bufs = {}

    def _check(self, st):
        if st != GFMC_OK:
            raise GfmcError(st, self._lib.gfmc_server_last_error(self._h).decode())

    def submit(self, slot: int, chain: "Chain", n_updates: int, trace: bool = True):
        n = int(n_updates)
        dec = np.zeros(n if trace else 0, dtype=np.uint8)
        dom = np.zeros(n if trace else 0, dtype=np.float64)
        self._check(self._lib.gfmc_server_submit(
            self._h, int(slot), chain._h, n,
            dec.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)) if trace else None,
            _dp(dom) if trace else None))
        # the library writes into these buffers when the job is polled done:
        # keep them alive until then (only once the submit has succeeded)
        self._bufs[slot] = (dec, dom)

    def poll(self, slot: int):
        """None while the slot's job runs; else a dict with its results."""
        done = ctypes.c_int(0)
        acc = ctypes.c_uint64(0)
        st = self._lib.gfmc_server_poll(self._h, int(slot), ctypes.byref(done), ctypes.byref(acc))
        if st != GFMC_OK:
            self._bufs.pop(slot, None)
            raise GfmcError(st, self._lib.gfmc_server_last_error(self._h).decode())
        if not done.value:
            return None
        dec, dom = self._bufs.pop(slot, (np.zeros(0, np.uint8), np.zeros(0)))
        return {"n_accepted": int(acc.value), "decisions": dec, "d_omega": dom}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gfmc_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
