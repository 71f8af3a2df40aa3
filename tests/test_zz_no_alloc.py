"""gfmc_delta_omega_noalloc: Delta Omega with no allocation of any kind.

Some callers cannot allocate device memory while they run -- a plugin's
enqueue step inside a framework that owns the device memory pool, code under a
fixed memory budget, code that must not let cudaMalloc synchronise the device.
They own their input and output buffers and call this entry point, whose
scratch is a fixed device array inside the library.  This test calls it
through the C ABI twice in a row and checks each result against the handle
based gfmc_delta_omega within the Delta Omega tolerance of the parity tests.
It lives in its own file so that pytest collects it last.
"""
import ctypes

import pytest

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


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    torch = pytest.importorskip("torch")
    L, M = 32, 1024
    d_spins = torch.zeros((L ** 3, 2), dtype=torch.float64, device="cuda")
    d_out = torch.zeros(1, dtype=torch.float64, device="cuda")
    msg = ctypes.create_string_buffer(256)
    st = lib.gfmc_delta_omega_noalloc(L, d_spins.data_ptr(), 1.0, -2.0, 20.0, M, 0, 0.0, 0.0, 0, 1.0, 1.0,
                                      d_out.data_ptr(), None, msg, len(msg))
    assert st == 1  # GFMC_EINVAL
    assert "needs" in msg.value.decode() and "static scratch holds" in msg.value.decode()
