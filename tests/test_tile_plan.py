"""The host's tile plan of the single-chain engines (plan_tiles in
csrc/gfmc_api.cu): tile c = [c N / ncta, (c + 1) N / ncta), and for each
CTA the list of the other CTAs that own a neighbour of one of its sites --
the CTAs whose flags it waits for before each stencil step, so a CTA missing
from the list would let a step read stale values.  The function's own source
is compiled for the host and checked against a brute-force list on the
engine's tilings: exactly the owners of the neighbours, no duplicates, never
the CTA itself.  A contiguous tiling of the cubic lattice depends on at most 6
CTAs per tile here, far below the limit the plan refuses beyond (the driver
checks either outcome against the brute-force count)."""
import re
import shutil
import subprocess

import pytest

from test_fixed_point import ROOT

API = f"{ROOT}/paper_1303_6016_gb300/csrc/gfmc_api.cu"
INTERNAL = f"{ROOT}/paper_1303_6016_gb300/csrc/gfmc_internal.h"

PRELUDE = r"""
#include <cstdio>
#include <set>
#include <vector>
enum gfmc_status { GFMC_OK = 0, GFMC_EINVAL = 1 };
struct gfmc_ctx { int N, L; };
static gfmc_status fail(gfmc_ctx*, gfmc_status st, const char*, ...) { return st; }
namespace gfmc { constexpr int kMaxNbrCta = %d; }
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

static int check(int L, int ncta)
{
    gfmc_ctx h{L * L * L, L};
    const int N = h.N;
    std::vector<int> start, ptr, idx;
    const gfmc_status st = plan_tiles(&h, ncta, start, ptr, idx);
    // brute force: the owners of the neighbours of each tile's sites
    std::vector<int> owner(N);
    std::vector<std::set<int>> want(ncta);
    int most = 0;
    for (int c = 0; c < ncta; ++c)
        for (int i = (int)(((long long)c * N) / ncta); i < (int)(((long long)(c + 1) * N) / ncta); ++i) owner[i] = c;
    for (int i = 0; i < N; ++i)
        for (int d = 0; d < 6; ++d)
            if (owner[nbr(i, d, L)] != owner[i]) want[owner[i]].insert(owner[nbr(i, d, L)]);
    for (auto& w : want) most = w.size() > (size_t)most ? (int)w.size() : most;
    int bad = 0;
    if (most > gfmc::kMaxNbrCta) {
        bad += st != GFMC_EINVAL;
    } else {
        bad += st != GFMC_OK;
        if ((int)start.size() != ncta + 1 || start[0] != 0 || start[ncta] != N) return 1;
        for (int c = 0; c < ncta; ++c) {
            if (start[c] != (int)(((long long)c * N) / ncta)) ++bad;
            std::set<int> got(idx.begin() + ptr[c], idx.begin() + ptr[c + 1]);
            if ((int)got.size() != ptr[c + 1] - ptr[c]) ++bad;  // duplicates
            if (got != want[c]) ++bad;
        }
    }
    std::printf("L=%d ncta=%d: most %d, bad %d\n", L, ncta, most, bad);
    return bad;
}

int main()
{
    const int cases[][2] = {{32, 152}, {32, 64}, {32, 512}, {24, 152}, {16, 64}, {16, 17}, {10, 7}, {8, 2},
                            {6, 1}, {20, 152}, {14, 42}, {3, 1}, {3, 27}, {5, 2}, {4, 64}};
    int bad = 0;
    for (auto& c : cases) bad += check(c[0], c[1]);
    return bad != 0;
}
"""


def extract(path: str, pattern: str) -> str:
    m = re.search(pattern, open(path).read(), re.S)
    assert m, f"{pattern} not found in {path}"
    return m.group(0)


def test_tile_plan_lists_exactly_the_neighbour_ctas(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    limit = int(re.search(r"constexpr int kMaxNbrCta = (\d+);", open(INTERNAL).read()).group(1))
    fn = extract(API, r"gfmc_status plan_tiles\(gfmc_ctx\* h, int ncta.*?\n\}\n")
    src = tmp_path / "tiles.cpp"
    src.write_text(PRELUDE.replace("%d", str(limit)) + fn + DRIVER)
    exe = tmp_path / "tiles"
    subprocess.run([cxx, "-O2", "-std=c++17", "-o", str(exe), str(src)], check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("bad 0") == 15, r.stdout
