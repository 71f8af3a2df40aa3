"""gfmc_delta_omega_noalloc: Delta Omega with no allocation of any kind.

Some callers cannot allocate device memory while they run -- a plugin's
enqueue step inside a framework that owns the device memory pool, code under a
fixed memory budget, code that must not let cudaMalloc synchronise the device.
They own their input and output buffers and call this entry point, whose
scratch is a fixed device array inside the library.  These tests call it
through the C ABI: twice in a row against the handle based gfmc_delta_omega,
against the oracle (at the largest accepted size and with the Lorentz kernel),
and with the device's free memory read around a call that is not the first,
all within the Delta Omega tolerance of the parity tests.  They live in their
own file so that pytest collects them last.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_6016_gb300 import inputs

pytestmark = pytest.mark.gpu

A = 6.05


def tol(ref):
    return 1e-10 * abs(ref) + 1e-13 * A


@pytest.fixture(scope="module")
def lib():
    from paper_1303_6016_gb300 import build, gfmc
    build.build()
    return gfmc.load()


def test_noalloc_matches_handle_entry_point_on_two_calls(lib):
    torch = pytest.importorskip("torch")
    from paper_1303_6016_gb300 import gfmc
    L, M = 8, 256
    sp = inputs.uniform_sphere(L, 6)
    cases = [(5, 1.1, 2.3), (301, 2.7, 0.4)]
    with gfmc.Chain(L, sp, M=M, beta=20.0, mu=-2.0, stream=None) as ch:
        refs = [ch.delta_omega(o, th, ph) for o, th, ph in cases]
    # caller-owned device buffers: the spins in, one double out
    d_spins = torch.tensor(sp, dtype=torch.float64, device="cuda")
    d_out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    msg = ctypes.create_string_buffer(256)
    for (o, th, ph), ref in zip(cases, refs):
        st = lib.gfmc_delta_omega_noalloc(L, d_spins.data_ptr(), 1.0, -2.0, 20.0, M, 0, 0.0, 0.0, o, th, ph,
                                          d_out.data_ptr(), None, msg, len(msg))
        assert st == 0, msg.value.decode()
        got = float(d_out.item())
        assert abs(got - ref) <= tol(ref), (o, got, ref)


@pytest.mark.parametrize("L,M", [(32, 1024), (22, 256)])
def test_noalloc_rejects_sizes_beyond_its_scratch(lib, L, M):
    """More CTAs of 256 sites than the scratch is laid out for (L = 22, 32)."""
    torch = pytest.importorskip("torch")
    d_spins = torch.zeros((L ** 3, 2), dtype=torch.float64, device="cuda")
    d_out = torch.zeros(1, dtype=torch.float64, device="cuda")
    msg = ctypes.create_string_buffer(256)
    st = lib.gfmc_delta_omega_noalloc(L, d_spins.data_ptr(), 1.0, -2.0, 20.0, M, 0, 0.0, 0.0, 0, 1.0, 1.0,
                                      d_out.data_ptr(), None, msg, len(msg))
    assert st == 1  # GFMC_EINVAL
    assert "needs" in msg.value.decode() and "static scratch holds" in msg.value.decode()


def _call(lib, L, d_spins, M, o, th, ph, d_out, kernel=0, lam=0.0):
    msg = ctypes.create_string_buffer(256)
    st = lib.gfmc_delta_omega_noalloc(L, d_spins.data_ptr(), 1.0, -2.0, 20.0, M, kernel, lam, 0.0, o, th, ph,
                                      d_out.data_ptr(), None, msg, len(msg))
    assert st == 0, msg.value.decode()
    return float(d_out.item())


@pytest.mark.parametrize("L,M,kernel", [(8, 256, 0), (12, 1024, 0), (20, 4096, 0), (6, 128, 1)])
def test_noalloc_matches_the_oracle(lib, L, M, kernel):
    """Against the oracle directly, at the largest accepted size (L = 20 on
    all 32 CTAs, with the largest M) and with the Lorentz kernel."""
    torch = pytest.importorskip("torch")
    sp = inputs.uniform_sphere(L, 7)
    d_spins = torch.tensor(sp, dtype=torch.float64, device="cuda")
    d_out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(3)
    for o in (0, L ** 3 // 2 + 1):
        th, ph = float(np.arccos(1 - 2 * rng.random())), float(2 * np.pi * rng.random())
        got = _call(lib, L, d_spins, M, o, th, ph, d_out, kernel=kernel, lam=4.0 if kernel else 0.0)
        ref = O.delta_omega(L, sp, o, th, ph, M, beta=20.0, chem=-2.0, kernel_kind=kernel, lam=4.0)
        assert abs(got - ref) <= tol(ref), (L, M, o, got, ref)


def test_noalloc_second_call_allocates_nothing(lib):
    """Free device memory is the same before and after a call that is not the
    first one on the device."""
    torch = pytest.importorskip("torch")
    L, M = 12, 1024
    sp = inputs.uniform_sphere(L, 8)
    d_spins = torch.tensor(sp, dtype=torch.float64, device="cuda")
    d_out = torch.zeros(1, dtype=torch.float64, device="cuda")
    first = _call(lib, L, d_spins, M, 100, 1.0, 1.0, d_out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    second = _call(lib, L, d_spins, M, 100, 1.0, 1.0, d_out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert second == first
