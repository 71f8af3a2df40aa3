"""Write the stored expected values under tests/golden/ from the oracle.

    python tests/golden/make_golden.py

The paper prints no worked numerical example of the update, so the stored
values are the oracle's (the plain FP64 CPU restatement in oracle/, pinned by
tests/test_oracle_pins.py): one full sequential sweep of the smallest
workload -- L = 4 (N = 64) periodic, t = 1, spins uniform on the sphere
(seed 0), a = 6.05, Jackson kernel, M = 256, beta = 20, mu = -2, Philox
proposals and Metropolis draws (seed 1, chain 0) -- with every update's
proposal, Delta Omega, acceptance ratio, uniform and decision, and the
magnetisation after the sweep (Algorithm 1; Sec. 2.2 for Delta Omega).
Only oracle/ and the seeded input generator are called.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1303_6016_gb300 import inputs  # noqa: E402

L, M, BETA, CHEM, SEED, CHAIN = 4, 256, 20.0, -2.0, 1, 0
PATH = os.path.join(HERE, "sweep_L4_M256.txt")


def main():
    O.build()
    sp = inputs.uniform_sphere(L, 0)
    res = O.updates(L, sp, L ** 3, M, beta=BETA, chem=CHEM, seed=SEED, chain_id=CHAIN)
    with open(PATH, "w") as f:
        f.write("# One sequential sweep, L=4 (N=64), t=1, a=6.05, Jackson, M=256, beta=20, mu=-2,\n")
        f.write("# Philox seed 1, chain 0 (Algorithm 1; Delta Omega by Eq. d_seff2), written by\n")
        f.write("# tests/golden/make_golden.py from oracle/ (the paper prints no worked example).\n")
        f.write("# initial spins: site theta phi\n")
        for i, (th, ph) in enumerate(sp):
            f.write(f"spin {i} {float(th)!r} {float(ph)!r}\n")
        f.write("# updates: q site theta_new phi_new d_omega ratio u accepted\n")
        for q in range(L ** 3):
            th, ph, u = O.draw(SEED, CHAIN, q)
            f.write(f"update {q} {q % L ** 3} {float(th)!r} {float(ph)!r} {float(res['d_omega'][q])!r} "
                    f"{float(res['ratio'][q])!r} {float(res['u'][q])!r} {int(res['decisions'][q])}\n")
        f.write(f"magnetization {float(res['magnetization'][0])!r}\n")
    print(PATH)


if __name__ == "__main__":
    main()
