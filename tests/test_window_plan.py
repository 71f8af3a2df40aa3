"""The host's plan of the FP64 engine's prefetch windows (plan_windows in
csrc/gfmc_api.cu): per CTA, the sites its stencil reads, as runs of
consecutive sites that the helper warp copies into shared memory.  The
function's own source is compiled for the host and its runs checked on the
tilings the engine uses (tile c = [c N / ncta, (c + 1) N / ncta)):
* the runs of a CTA are sorted, disjoint and maximal;
* every neighbour of every tile site is in a run -- or, for the halo-only plan
  of the split instantiation, in the tile itself;
* a halo-only plan holds no tile site, a full plan holds every one, and no
  plan holds a site that is neither a tile site nor a neighbour of one;
* max_len is the largest number of sites of one CTA."""
import re
import shutil
import subprocess

import pytest

from test_fixed_point import ROOT

API = f"{ROOT}/paper_1303_6016_gb300/csrc/gfmc_api.cu"

PRELUDE = r"""
#include <algorithm>
#include <cstdio>
#include <set>
#include <vector>
struct int2 { int x, y; };
static int2 make_int2(int x, int y) { return int2{x, y}; }
"""

DRIVER = r"""
static int nbr(int i, int d, int L)
{
    const int x = i % L, y = (i / L) % L, z = i / (L * L);
    switch (d) {
    case 0: return (x + 1) % L + L * (y + L * z);
    case 1: return (x + L - 1) % L + L * (y + L * z);
    case 2: return x + L * ((y + 1) % L + L * z);
    case 3: return x + L * ((y + L - 1) % L + L * z);
    case 4: return x + L * (y + L * ((z + 1) % L));
    default: return x + L * (y + L * ((z + L - 1) % L));
    }
}

static int check(int L, int ncta, bool halo)
{
    const int N = L * L * L;
    std::vector<int> start(ncta + 1), ptr;
    for (int c = 0; c <= ncta; ++c) start[c] = (int)(((long long)c * N) / ncta);
    std::vector<int2> wins;
    int max_len = -1;
    plan_windows(L, ncta, start, ptr, wins, max_len, halo);
    int bad = 0, longest = 0;
    if ((int)ptr.size() != ncta + 1 || ptr[0] != 0 || ptr[ncta] != (int)wins.size()) return 1;
    for (int c = 0; c < ncta; ++c) {
        std::set<int> in, need;
        int total = 0;
        for (int w = ptr[c]; w < ptr[c + 1]; ++w) {
            const int2 r = wins[w];
            if (r.y < 1) ++bad;
            if (w > ptr[c] && r.x <= wins[w - 1].x + wins[w - 1].y) ++bad;  // sorted, disjoint, maximal
            for (int s = r.x; s < r.x + r.y; ++s) in.insert(s);
            total += r.y;
        }
        longest = std::max(longest, total);
        for (int i = start[c]; i < start[c + 1]; ++i) {
            need.insert(i);
            for (int d = 0; d < 6; ++d) need.insert(nbr(i, d, L));
        }
        for (int s : need) {
            const bool own = s >= start[c] && s < start[c + 1];
            if (halo && own) { if (in.count(s)) ++bad; }
            else if (!in.count(s)) ++bad;
        }
        for (int s : in)
            if (!need.count(s)) ++bad;
    }
    if (longest != max_len) ++bad;
    std::printf("L=%d ncta=%d halo=%d: %d CTAs, max_len %d, bad %d\n", L, ncta, (int)halo, ncta, max_len, bad);
    return bad;
}

int main()
{
    const int cases[][2] = {{32, 152}, {32, 64}, {24, 152}, {24, 108}, {16, 64}, {16, 17}, {10, 7}, {8, 2},
                            {6, 1}, {20, 152}, {14, 42}, {3, 1}, {5, 2}};
    int bad = 0;
    for (auto& c : cases)
        for (int h = 0; h < 2; ++h) bad += check(c[0], c[1], h != 0);
    return bad != 0;
}
"""


def extract_plan_windows() -> str:
    src = open(API).read()
    m = re.search(r"void plan_windows\(int L, int ncta.*?\n\}\n", src, re.S)
    assert m, "plan_windows not found in gfmc_api.cu"
    return m.group(0)


def test_window_plan_covers_every_neighbour(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "plan.cpp"
    src.write_text(PRELUDE + extract_plan_windows() + DRIVER)
    exe = tmp_path / "plan"
    subprocess.run([cxx, "-O2", "-std=c++17", "-o", str(exe), str(src)], check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("bad 0") == 26, r.stdout
