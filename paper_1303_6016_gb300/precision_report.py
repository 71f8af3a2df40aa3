"""Error of the FP32-mixed paths against the FP64 path on the L = 32 workloads.

    python -m paper_1303_6016_gb300.precision_report [--L 32] [--M 1024 2048] [--sites 6]
                                                     [--json out.json]

For each spin distribution (uniform on the sphere, seed 0; von Mises-Fisher
about +z with kappa = 5, seed 2) and each M, on a sample of sites it reports
  * the moment error |mu_mixed - mu_fp64| as a function of n (maximum over the
    49 entries and the sampled sites, in bands of n),
  * the Delta Omega error |dO_mixed - dO_fp64| for a seeded proposal at each
    sampled site,
for three FP32-mixed arithmetics: the default engine (at L = 32 the vector
clusters, moments read off the recursion with no dot products), the grid
engine's doubling with plain FP32 warp sums of the Gram products, and the
same with compensated (Dot2) products and sums.  The FP64 path itself is
checked against the oracle by the parity tests.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import build, gfmc, inputs


def proposal(q):
    """A seeded proposal direction uniform on the sphere for sample q."""
    rng = np.random.default_rng(1000 + q)
    return float(np.arccos(1 - 2 * rng.random())), float(2 * math.pi * rng.random())


def run(L=32, Ms=(1024, 2048), n_sites=6, kinds=("uniform", "vmf")):
    build.build()
    N = L ** 3
    out = []
    sites = [int(s) for s in np.linspace(0, N - 1, n_sites).astype(int)]
    for kind in kinds:
        sp = inputs.make(kind, L, seed=0 if kind == "uniform" else 2)
        for M in Ms:
            bands = [(0, 64), (64, 256), (256, M // 2), (M // 2, M)]
            variants = {"default": {}, "grid_plain": {"engine": "grid"},
                        "grid_compensated": {"engine": "grid", "compensated": True}}
            with gfmc.Chain(L, sp, M=M, precision="fp64") as c64:
                ref = {o: c64.moments(o) for o in sites}
                dref = {q: c64.delta_omega(o, *proposal(q)) for q, o in enumerate(sites)}
            rows = {}
            for name, kw in variants.items():
                band_err = np.zeros(len(bands))
                dom_err, dom_rel = [], []
                with gfmc.Chain(L, sp, M=M, precision="fp32_mixed", **kw) as c32:
                    for q, o in enumerate(sites):
                        err = np.abs(c32.moments(o) - ref[o]).max(axis=(0, 1))
                        for b, (lo, hi) in enumerate(bands):
                            band_err[b] = max(band_err[b], float(err[lo:hi].max()))
                        d32 = c32.delta_omega(o, *proposal(q))
                        dom_err.append(abs(d32 - dref[q]))
                        dom_rel.append(abs(d32 - dref[q]) / max(abs(dref[q]), 1e-300))
                rows[name] = {"moment_err_by_n": {f"[{lo},{hi})": float(e) for (lo, hi), e in zip(bands, band_err)},
                              "domega_err_max": float(max(dom_err)), "domega_err_mean": float(np.mean(dom_err)),
                              "domega_rel_err_max": float(max(dom_rel))}
            out.append(dict({"spins": kind, "L": L, "M": M, "sites": sites}, **rows["default"],
                            variants=rows))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=32)
    ap.add_argument("--M", type=int, nargs="+", default=[1024, 2048])
    ap.add_argument("--sites", type=int, default=6)
    ap.add_argument("--json", default="")
    a = ap.parse_args(argv)
    res = run(a.L, tuple(a.M), a.sites)
    for r in res:
        print(json.dumps(r))
    if a.json:
        with open(a.json, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
