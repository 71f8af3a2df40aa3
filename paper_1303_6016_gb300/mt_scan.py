"""Magnetisation against temperature (Algorithm 1; the validation of Sec. 4).

For each lattice size L and temperature T one chain starts from a cold
(ferromagnetic) or hot (uniform-sphere) configuration and runs S sweeps;
after each sweep the engine measures M = |sum_i S_i| / N, and the first `warmup` sweeps are dropped before
averaging (Sec. 3.2: warm-up sweeps are discarded).  All chains run together:
every launch of the batch engine advances each chain by one sweep.

    python -m paper_1303_6016_gb300.mt_scan --L 4 6 8 --T 0.02 0.05 0.1 0.2 0.4 \\
        --sweeps 80 --warmup 20 [--M 256] [--mu 0] [--precision fp32_mixed]

The paper prints no numbers for this curve (its figure is not in the text),
so the output is a qualitative reproduction: ordered (M near 1) at low T,
disordered (M ~ 1/sqrt(N)) at high T.  A hot start quenched far below the
ordering temperature freezes into a disordered state within the sweeps one
can afford (acceptance collapses; the oracle shows the same), hence the cold
start by default.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import gfmc, inputs


def scan(Ls=(4, 6, 8), Ts=(0.02, 0.05, 0.08, 0.1, 0.12, 0.15, 0.2, 0.3), sweeps=80, warmup=20, M=256,
         mu=0.0, precision="fp32_mixed", team_ctas=None, seed=7, start="cold"):
    chains, keys = [], []
    for L in Ls:
        for T in Ts:
            c = len(chains)
            sp = inputs.ferromagnet(L) if start == "cold" else inputs.uniform_sphere(L, seed + c)
            chains.append(gfmc.Chain(L, sp, M=M, beta=1.0 / T, mu=mu, precision=precision, seed=seed,
                                     chain_id=c))
            keys.append((L, T))
    tcs = team_ctas or [1] * len(chains)
    series = [[] for _ in chains]
    acc = np.zeros(len(chains))
    for s in range(sweeps):
        out = gfmc.run_batch(chains, [ch.N for ch in chains], team_ctas=tcs, trace=False)
        for c, r in enumerate(out):
            series[c].extend(r["magnetization"].tolist())
            if s >= warmup:
                acc[c] += r["n_accepted"] / chains[c].N
    res = []
    for c, (L, T) in enumerate(keys):
        m = np.array(series[c][warmup:])
        res.append({"L": L, "T": T, "M_mean": float(m.mean()), "M_sem": float(m.std(ddof=1) / np.sqrt(len(m))),
                    "acceptance": float(acc[c] / max(1, sweeps - warmup))})
    for ch in chains:
        ch.close()
    return {"mu": mu, "M": M, "precision": precision, "sweeps": sweeps, "warmup": warmup, "start": start,
            "points": res}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, nargs="+", default=[4, 6, 8])
    ap.add_argument("--T", type=float, nargs="+", default=[0.02, 0.05, 0.08, 0.1, 0.12, 0.15, 0.2, 0.3])
    ap.add_argument("--sweeps", type=int, default=80)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--M", type=int, default=256)
    ap.add_argument("--mu", type=float, default=0.0)
    ap.add_argument("--precision", default="fp32_mixed")
    ap.add_argument("--start", default="cold", choices=["cold", "hot"])
    a = ap.parse_args(argv)
    from . import build
    build.build()
    print(json.dumps(scan(a.L, a.T, a.sweeps, a.warmup, a.M, a.mu, a.precision, start=a.start)))


if __name__ == "__main__":
    main()
