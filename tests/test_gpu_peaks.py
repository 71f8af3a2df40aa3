"""The library's own measurement kernels (include/gfmc_peaks.h): the FMA
throughput that divides the FP64 engine's rate, the FP64 pipe's issue rate at
that engine's occupancy, and the exchange of the FP32 vector-cluster engine
timed alone.  They time the hardware, so the checks are
ranges that any working GB300 meets, and the argument errors."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_1303_6016_gb300 import build, gfmc
    build.build()
    gfmc.load()
    return gfmc


def test_fma_peak_is_in_the_device_range(G):
    # FP64: a few hundred SMs x 2 DFMA per clock x ~2 GHz; FP32 about 64x more
    f64 = G.fma_peak_tflops("fp64", repeats=2)
    f32 = G.fma_peak_tflops("fp32_mixed", repeats=2)
    assert 0.3 < f64 < 3.0
    assert 10.0 < f32 < 200.0
    assert f32 > 20 * f64


def test_fp64_pipe_is_shared_by_the_sm(G):
    """At one CTA of 256 threads per SM the FP64 pipe is as busy with one
    dependent chain on each of 4 warps as with 16 chains on 8, and a warp with
    12 active lanes costs a full warp's slots: the FP64 engines are bound by
    their count of warp instructions, not by latency or by lanes."""
    full = G.fp64_issue_rate(16, 8)
    one = G.fp64_issue_rate(1, 4)
    part = G.fp64_issue_rate(4, 8, lanes=12)
    assert 0.5 < full < 4.0  # a handful of FP64 lanes per SM and clock
    assert one > 0.9 * full
    assert part > 0.9 * full


def test_cluster_exchange_floor(G):
    """A step of the exchange alone takes a few hundred to a few thousand
    cycles: more than one DSMEM round trip, far less than the engine's
    budget."""
    c = G.cluster_exchange_cycles(steps=500, repeats=2)
    assert 100.0 < c < 20000.0


def test_argument_errors(G):
    import ctypes
    lib = G.load()
    out = ctypes.c_double(0.0)
    assert lib.gfmc_measure_fp64_issue(3, 8, 32, 1, ctypes.byref(out), None) == G.GFMC_EINVAL
    assert lib.gfmc_measure_fp64_issue(4, 9, 32, 1, ctypes.byref(out), None) == G.GFMC_EINVAL
    assert lib.gfmc_measure_fp64_issue(4, 8, 33, 1, ctypes.byref(out), None) == G.GFMC_EINVAL
    assert lib.gfmc_measure_cluster_exchange(1, 1, ctypes.byref(out), None) == G.GFMC_EINVAL
    assert lib.gfmc_measure_cluster_exchange(10, 0, ctypes.byref(out), None) == G.GFMC_EINVAL
    assert lib.gfmc_measure_cluster_exchange(10, 1, None, None) == G.GFMC_EINVAL
    assert lib.gfmc_measure_fma_peak(7, 1, ctypes.byref(out), None) == G.GFMC_EINVAL
