"""The stored sweep of the smallest workload (tests/golden/sweep_L4_M256.txt,
written from the oracle by tests/golden/make_golden.py): the oracle still
reproduces it, and the GPU engine matches it (Delta Omega within
1e-10 |dO| + 1e-13 a, decisions identical except near ties
|exp(-beta dO) - u| < 1e-9)."""
import os

import numpy as np
import pytest

from oracle import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "sweep_L4_M256.txt")
L, M, BETA, CHEM, SEED = 4, 256, 20.0, -2.0, 1
A = 6.05


def load():
    spins, upd, mag = [], [], None
    for line in open(GOLDEN):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "spin":
            spins.append((float(f[2]), float(f[3])))
        elif f[0] == "update":
            upd.append((int(f[2]), float(f[3]), float(f[4]), float(f[5]), float(f[6]), float(f[7]), int(f[8])))
        elif f[0] == "magnetization":
            mag = float(f[1])
    return np.array(spins), upd, mag


def test_oracle_reproduces_the_stored_sweep():
    sp, upd, mag = load()
    res = O.updates(L, sp, L ** 3, M, beta=BETA, chem=CHEM, seed=SEED)
    for q, (site, th, ph, dom, ratio, u, acc) in enumerate(upd):
        assert site == q % L ** 3
        assert (th, ph, u) == O.draw(SEED, 0, q)
        assert abs(res["d_omega"][q] - dom) <= 1e-13 * max(1.0, abs(dom))
        assert int(res["decisions"][q]) == acc
    assert res["magnetization"][0] == pytest.approx(mag, abs=1e-14)


@pytest.mark.gpu
def test_gpu_sweep_matches_the_stored_sweep():
    from paper_1303_6016_gb300 import build, gfmc
    build.build()
    sp, upd, mag = load()
    with gfmc.Chain(L, sp, M=M, beta=BETA, mu=CHEM, seed=SEED) as ch:
        out = ch.sweep(1)
    for q, (site, th, ph, dom, ratio, u, acc) in enumerate(upd):
        assert abs(out["d_omega"][q] - dom) <= 1e-10 * abs(dom) + 1e-13 * A, (q, out["d_omega"][q], dom)
        if int(out["decisions"][q]) != acc:
            assert abs(ratio - u) < 1e-9
    if np.array_equal(out["decisions"], np.array([a for *_, a in upd], dtype=np.uint8)):
        assert out["magnetization"][0] == pytest.approx(mag, abs=1e-13)
