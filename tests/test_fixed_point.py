"""The engines' fixed-point Gram partials: fixed58(x) = round(x 2^58), ties to
even, from the bits of x with integer operations only (csrc/gfmc_engine.cuh),
and its range check |x| <= 16.  The function's own source is compiled for the
host with g++ and compared with the C library's llrint(x * 2^58) (exact
scaling, then the current rounding mode, round-to-nearest-even) on random
values over 86 binades, exact ties and their neighbours, the range boundary,
subnormals, zeros and non-finite values."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_1303_6016_gb300", "csrc", "gfmc_engine.cuh")

PRELUDE = r"""
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
static long long dbits(double x) { long long b; std::memcpy(&b, &x, 8); return b; }
#define __double_as_longlong dbits
#define __device__
#define __forceinline__ inline
"""

DRIVER = r"""
int main()
{
    std::mt19937_64 g(7);
    long bad = 0, n = 0;
    auto chk = [&](double x) {
        bool ok;
        const long long q = fixed58(x, ok);
        const bool ok_ref = std::fabs(x) <= 16.0;
        ++n;
        if (ok != ok_ref) { if (bad < 5) std::printf("range %a\n", x); ++bad; return; }
        if (!ok) return;
        const long long r = std::llrint(x * 0x1p58);
        if (q != r) { if (bad < 5) std::printf("value %a: %lld vs %lld\n", x, q, r); ++bad; }
    };
    std::uniform_real_distribution<double> u(-1.0, 1.0);
    for (int e = -80; e <= 5; ++e)
        for (int i = 0; i < 20000; ++i) chk(std::ldexp(u(g), e));
    for (int i = 0; i < 200000; ++i) {
        const long long k = (long long)(g() >> 12);
        const int s = 59 + (int)(g() % 40);
        const double x = std::ldexp((double)(2 * k + 1), -s);  // an exact tie of x 2^58 when s == 59
        if (std::fabs(x) <= 16.0) {
            chk(x); chk(-x); chk(std::nextafter(x, 0.0)); chk(std::nextafter(x, 1e9));
        }
    }
    const double sp[] = {0.0, -0.0, 16.0, -16.0, std::nextafter(16.0, 20.0), -std::nextafter(16.0, 20.0),
                         std::nextafter(16.0, 0.0), INFINITY, -INFINITY, NAN, 4.9e-324, -4.9e-324, 2.2e-308,
                         0x1p-59, -0x1p-59, 0x1p-60, 0x1.8p-59, 0x1.8p-58, 0x1.4p-58, 3 * 0x1p-59, 1.0, -1.0,
                         0.5, 0x1p-58, 4.0, -4.0};
    for (double x : sp) chk(x);
    std::printf("checked %ld, bad %ld\n", n, bad);
    return bad != 0;
}
"""


def extract_fixed58() -> str:
    src = open(HEADER).read()
    m = re.search(r"__device__ __forceinline__ long long fixed58\(double x, bool& ok\)\n\{.*?\n\}\n", src, re.S)
    assert m, "fixed58 not found in gfmc_engine.cuh"
    return m.group(0)


def test_fixed58_matches_llrint(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "fixed58.cpp"
    src.write_text(PRELUDE + extract_fixed58() + DRIVER)
    exe = tmp_path / "fixed58"
    subprocess.run([cxx, "-O2", "-std=c++17", "-o", str(exe), str(src)], check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "bad 0" in r.stdout
