"""Run a fixed block of GFMC updates on one chain (for profiling and timing).

    python -m paper_1303_6016_gb300.run_case --L 32 --M 1024 --precision fp64 --updates 1

Builds the engine if needed, creates one chain from seeded uniform-sphere
spins (seed 0), runs the updates through the C ABI and prints a summary line.
"""
from __future__ import annotations

import argparse
import time

from . import build, gfmc, inputs


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=32)
    ap.add_argument("--M", type=int, default=1024)
    ap.add_argument("--precision", default="fp64", choices=sorted(gfmc.PRECISIONS))
    ap.add_argument("--updates", type=int, default=1)
    ap.add_argument("--spins", default="uniform", choices=["uniform", "vmf", "fm"])
    ap.add_argument("--beta", type=float, default=20.0)
    ap.add_argument("--mu", type=float, default=-2.0)
    ap.add_argument("--num-ctas", type=int, default=0)
    ap.add_argument("--recursion", default="unit_vectors", choices=sorted(gfmc.RECURSIONS))
    ap.add_argument("--engine", default="auto", choices=sorted(gfmc.ENGINES))
    ap.add_argument("--compensated", action="store_true")
    ap.add_argument("--team", type=int, default=0,
                    help="run the updates as a one-chain batch on a team of this many CTAs")
    ap.add_argument("--cluster", type=int, default=0,
                    help="run the updates on a thread-block cluster of this many CTAs (proposal recursion)")
    a = ap.parse_args(argv)
    build.build()
    sp = inputs.make(a.spins, a.L, seed=0 if a.spins != "vmf" else 2)
    with gfmc.Chain(a.L, sp, M=a.M, beta=a.beta, mu=a.mu, precision=a.precision,
                    num_ctas=a.num_ctas, recursion=a.recursion, engine=a.engine,
                    compensated=a.compensated) as ch:
        t0 = time.perf_counter()
        if a.cluster > 0:
            out = gfmc.run_clusters([ch], [a.updates], [a.cluster])[0]
        elif a.team > 0:
            out = gfmc.run_batch([ch], [a.updates], team_ctas=[a.team])[0]
        else:
            out = ch.updates(a.updates)
        dt = time.perf_counter() - t0
    print(f"L={a.L} M={a.M} {a.precision}: {a.updates} updates in {dt * 1e3:.2f} ms, "
          f"{out['n_accepted']} accepted, first dOmega {out['d_omega'][0]:.6e}")


if __name__ == "__main__":
    main()
