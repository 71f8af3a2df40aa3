"""Batches of independent chains on one GPU: team-size autotuning and packing.

Independent Monte Carlo chains share nothing (Sec. 3.2: the sweep loop splits
into independent chains), so a batch runs all of them in one launch of the
team engine, each chain on its own team of CTAs (``gfmc_run_batch``), or --
for chains on the proposal-vector recursion -- each on one thread-block
cluster that holds its lattice in shared memory (``ClusterRunner``,
``gfmc_run_clusters``).

The autotuner measures, on the device, the time of one update of a probe
chain of each lattice size at candidate team sizes, then shares the device's
CTAs among the chains of a batch so that the slowest chain finishes first as
early as possible (greedy: repeatedly double the team of the chain with the
longest projected time while the CTAs last).  Chains that do not fit in one
launch are run in waves.

    from paper_1303_6016_gb300 import batch
    tuner = batch.Autotuner(M=1024, precision="fp32_mixed")
    runner = batch.BatchRunner(chains, tuner)
    out = runner.run(updates_per_chain=8)
"""
from __future__ import annotations

import time

import numpy as np

from . import gfmc, inputs

CANDIDATES = (1, 2, 4, 8, 16, 32, 64)


def device_ctas() -> int:
    """CTAs of the team engine resident at once (one per SM)."""
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


class Autotuner:
    """Per-lattice-size update times of the team engine at candidate team sizes."""

    def __init__(self, M: int, precision: str = "fp32_mixed", candidates=CANDIDATES, probe_updates: int = 2,
                 beta: float = 20.0, mu: float = -2.0, recursion: str = "unit_vectors"):
        self.M, self.precision, self.recursion = M, precision, recursion
        self.candidates = tuple(candidates)
        self.probe_updates = probe_updates
        self.beta, self.mu = beta, mu
        self.table = {}  # L -> {team size: seconds per update}

    def measure(self, L: int) -> dict:
        if L in self.table:
            return self.table[L]
        import torch
        sp = inputs.uniform_sphere(L, 0)
        res = {}
        with gfmc.Chain(L, sp, M=self.M, precision=self.precision, beta=self.beta, mu=self.mu,
                        recursion=self.recursion) as ch:
            for tc in self.candidates:
                if tc > min(L ** 3, 1024) or tc > device_ctas():
                    continue
                gfmc.run_batch([ch], 1, team_ctas=[tc], trace=False)  # warm-up, plans the team
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                gfmc.run_batch([ch], self.probe_updates, team_ctas=[tc], trace=False)
                res[tc] = (time.perf_counter() - t0) / self.probe_updates
        self.table[L] = res
        return res

    def allocate(self, Ls, budget: int, work=None) -> list:
        """Team sizes for chains of lattice sizes Ls within `budget` CTAs.
        work[c] is the number of updates chain c will run (default equal)."""
        work = [1.0] * len(Ls) if work is None else list(work)
        tables = [self.measure(L) for L in Ls]
        tc = [min(t) for t in tables]
        used = sum(tc)
        if used > budget:
            raise ValueError(f"{len(Ls)} chains need at least {used} CTAs, the device holds {budget}")

        def proj(c):
            return tables[c][tc[c]] * work[c]

        while True:
            order = sorted(range(len(Ls)), key=proj, reverse=True)
            grown = False
            for c in order[:1]:
                bigger = [t for t in tables[c] if t > tc[c]]
                if not bigger:
                    break
                nxt = min(bigger)
                if used - tc[c] + nxt <= budget and tables[c][nxt] < tables[c][tc[c]]:
                    used += nxt - tc[c]
                    tc[c] = nxt
                    grown = True
            if not grown:
                return tc


class BatchRunner:
    """Runs a list of chains as batches of the team engine."""

    def __init__(self, chains, tuner: Autotuner, budget: int = 0):
        self.chains = list(chains)
        self.tuner = tuner
        self.budget = budget or device_ctas()

    def plan(self, updates):
        """Waves of (chain indices, team sizes) that each fit the device."""
        Ls = [c.L for c in self.chains]
        need = [min(self.tuner.measure(L)) for L in Ls]
        waves, cur, used = [], [], 0
        for i in sorted(range(len(Ls)), key=lambda i: -Ls[i]):
            if used + need[i] > self.budget and cur:
                waves.append(cur)
                cur, used = [], 0
            cur.append(i)
            used += need[i]
        if cur:
            waves.append(cur)
        plan = []
        for w in waves:
            tc = self.tuner.allocate([Ls[i] for i in w], self.budget, [updates[i] for i in w])
            plan.append((w, tc))
        return plan

    def run(self, updates_per_chain, trace: bool = False):
        n = len(self.chains)
        updates = list(updates_per_chain) if hasattr(updates_per_chain, "__len__") else [updates_per_chain] * n
        out = [None] * n
        for w, tc in self.plan(updates):
            res = gfmc.run_batch([self.chains[i] for i in w], [updates[i] for i in w], team_ctas=tc, trace=trace)
            for k, i in enumerate(w):
                out[i] = dict(res[k], team_ctas=tc[k])
        return out


class ClusterRunner:
    """Runs chains with the recursion on the proposal's vectors on
    thread-block clusters (gfmc_run_clusters): each chain on the smallest
    cluster whose shared memory holds its lattice -- the fewest SMs per chain,
    hence the most chains in flight -- all chains in one call (one launch per
    cluster size and precision, the launches overlapping)."""

    def __init__(self, chains):
        self.chains = list(chains)
        self.cluster_ctas = [gfmc.cluster_min_ctas(c.L, max(c.M, c.K), c.precision) for c in self.chains]

    def run(self, updates_per_chain, trace: bool = False):
        n = len(self.chains)
        updates = list(updates_per_chain) if hasattr(updates_per_chain, "__len__") else [updates_per_chain] * n
        res = gfmc.run_clusters(self.chains, updates, self.cluster_ctas, trace=trace)
        return [dict(r, cluster_ctas=c) for r, c in zip(res, self.cluster_ctas)]


def c4_chains(n_chains: int = 64, M: int = 1024, precision: str = "fp32_mixed", seed: int = 4,
              sizes=(8, 12, 16, 24, 32), tmin: float = 0.02, tmax: float = 0.2, mu: float = -2.0,
              recursion: str = "unit_vectors"):
    """The batching workload: n_chains independent chains with L drawn from
    `sizes` and temperatures uniform in [tmin, tmax] (seeded), spins uniform on
    the sphere (seed = chain index), M moments, FP32-mixed by default."""
    rng = np.random.default_rng(seed)
    Ls = rng.choice(sizes, size=n_chains)
    Ts = rng.uniform(tmin, tmax, size=n_chains)
    chains = [gfmc.Chain(int(L), inputs.uniform_sphere(int(L), c), M=M, precision=precision, beta=1.0 / T,
                         mu=mu, seed=1, chain_id=c, recursion=recursion) for c, (L, T) in enumerate(zip(Ls, Ts))]
    return chains, Ls, Ts
