"""The C ABI: libgfmc.so builds, loads, exports every function include/gfmc.h
declares, and rejects bad arguments before touching a GPU (no compute here)."""
import ctypes
import os
import re
import shutil

import numpy as np
import pytest

from paper_1303_6016_gb300 import gfmc, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]

needs_nvcc = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


def declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(gfmc_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1303_6016_gb300 import build
    build.build()
    return gfmc.load()


@needs_nvcc
def test_header_and_binding_agree():
    assert declared_functions() == sorted(gfmc.EXPORTS)


@needs_nvcc
def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


@needs_nvcc
def test_default_options(lib):
    opt = gfmc.Options()
    lib.gfmc_default_options(ctypes.byref(opt))
    assert opt.precision == 0 and opt.kernel == 0 and opt.seed == 1 and opt.num_ctas == 0


@needs_nvcc
@pytest.mark.parametrize("L,M,beta,t,msg", [
    (2, 256, 20.0, 1.0, "L = 2"),
    (99, 256, 20.0, 1.0, "L = 99"),
    (4, 100, 20.0, 1.0, "M = 100"),
    (4, 8, 20.0, 1.0, "M = 8"),
    (4, 256, 0.0, 1.0, "beta"),
    (4, 256, float("nan"), 1.0, "beta"),
    (4, 256, 20.0, 0.0, "t = 0"),
])
def test_create_rejects_bad_arguments(lib, L, M, beta, t, msg):
    sp = inputs.uniform_sphere(max(L, 3), 0)
    h = ctypes.c_void_p()
    st = lib.gfmc_create(L, sp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), t, -2.0, beta, M, None,
                         ctypes.byref(h))
    assert st == gfmc.GFMC_EINVAL
    assert not h.value
    assert msg in lib.gfmc_last_error(None).decode()


@needs_nvcc
def test_create_rejects_bad_spins_and_scale(lib):
    sp = inputs.uniform_sphere(4, 0)
    sp[5, 0] = 4.0  # theta > pi
    h = ctypes.c_void_p()
    st = lib.gfmc_create(4, sp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1.0, -2.0, 20.0, 64, None,
                         ctypes.byref(h))
    assert st == gfmc.GFMC_EINVAL and "spin 5" in lib.gfmc_last_error(None).decode()
    opt = gfmc.Options()
    lib.gfmc_default_options(ctypes.byref(opt))
    opt.spectral_scale = 5.0  # must exceed 6|t|
    sp = inputs.uniform_sphere(4, 0)
    st = lib.gfmc_create(4, sp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1.0, -2.0, 20.0, 64,
                         ctypes.byref(opt), ctypes.byref(h))
    assert st == gfmc.GFMC_EINVAL and "spectral scale" in lib.gfmc_last_error(None).decode()


@needs_nvcc
@pytest.mark.parametrize("nodes", [3 * 64, 64 // 2, 4 * 64, -1])
def test_create_rejects_bad_node_counts(lib, nodes):
    """gfmc_options.nodes: 0, M or 2M; anything else is rejected before any device work."""
    sp = inputs.uniform_sphere(4, 0)
    opt = gfmc.Options()
    lib.gfmc_default_options(ctypes.byref(opt))
    assert opt.nodes == 0
    opt.nodes = nodes
    h = ctypes.c_void_p()
    st = lib.gfmc_create(4, sp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1.0, -2.0, 20.0, 64,
                         ctypes.byref(opt), ctypes.byref(h))
    assert st == gfmc.GFMC_EINVAL and "nodes" in lib.gfmc_last_error(None).decode()
    assert not h.value


@needs_nvcc
def test_null_handle_is_rejected(lib):
    out = np.zeros(2)
    assert lib.gfmc_delta_omega(None, 0, 0.0, 0.0, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) \
        == gfmc.GFMC_EINVAL
    assert b"invalid handle" in lib.gfmc_last_error(None)
    lib.gfmc_destroy(None)  # a no-op


def test_binding_fails_loudly_without_library(tmp_path):
    missing = str(tmp_path / "libgfmc.so")
    saved = gfmc._lib
    gfmc._lib = None
    try:
        with pytest.raises(RuntimeError, match="no fallback"):
            gfmc.load(missing)
    finally:
        gfmc._lib = saved
