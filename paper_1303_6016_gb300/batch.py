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
early as possible (greedy: repeatedly grow the team of the chain with the
longest projected time to the next probed size while the CTAs last, small
chains sharing one CTA one after another when that frees CTAs for the large
ones).  Chains that do not
fit in one launch are run in waves.

    from paper_1303_6016_gb300 import batch
    tuner = batch.Autotuner(M=1024, precision="fp32_mixed")
    runner = batch.BatchRunner(chains, tuner)
    out = runner.run(updates_per_chain=8)
"""
from __future__ import annotations

import time

import numpy as np

from . import gfmc, inputs

# team sizes the autotuner probes (the tiles are contiguous site ranges, so any
# size works; the in-between sizes let a large chain's team grow in small steps)
CANDIDATES = (1, 2, 3, 4, 5, 6, 8, 12, 16, 24, 32, 64)


def device_ctas() -> int:
    """CTAs of the team engine resident at once (one per SM)."""
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


class Autotuner:
    """Per-lattice-size update times of the team engine at candidate team sizes."""

    def __init__(self, M: int, precision: str = "fp32_mixed", candidates=CANDIDATES, probe_updates: int = 2,
                 beta: float = 20.0, mu: float = -2.0, recursion: str = "unit_vectors", compensated: bool = False):
        self.M, self.precision, self.recursion = M, precision, recursion
        self.compensated = compensated
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
                        recursion=self.recursion, compensated=self.compensated) as ch:
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

    def allocate(self, Ls, budget: int, work=None, sizes=None) -> list:
        """Team sizes for chains of lattice sizes Ls within `budget` CTAs.
        work[c] is the number of updates chain c will run (default equal);
        sizes, if given, restricts the team sizes considered."""
        work = [1.0] * len(Ls) if work is None else list(work)
        tables = [{k: v for k, v in self.measure(L).items() if sizes is None or k in sizes} for L in Ls]
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

    def pack(self, Ls, budget: int, work=None, kinds=None):
        """As allocate, but small chains may share one CTA and run one after
        another (gfmc_run_batch's team size 0), which leaves CTAs to the large
        chains.  Greedy on the projected time of each unit (a team of one
        chain, or a shared one-CTA team: the sum of its chains' one-CTA
        times): grow the slowest unit's team; when the CTAs run out, merge the
        two fastest one-CTA units while the merged unit stays faster than the
        slowest; only chains of one kind (recursion) share a CTA.  Returns
        (order, team sizes): chain order[k] gets tc[k] CTAs, 0 meaning after
        order[k-1] on its CTA."""
        work = [1.0] * len(Ls) if work is None else list(work)
        kinds = [0] * len(Ls) if kinds is None else list(kinds)
        tables = [self.measure(L) for L in Ls]
        units = [[min(t), [c]] for c, t in enumerate(tables)]  # [team size, chains]
        used = sum(u[0] for u in units)
        if used > budget:
            raise ValueError(f"{len(Ls)} chains need at least {used} CTAs, the device holds {budget}")

        def t_unit(u):
            if len(u[1]) == 1:
                c = u[1][0]
                return tables[c][u[0]] * work[c]
            return sum(tables[c][1] * work[c] for c in u[1])

        while True:
            units.sort(key=t_unit, reverse=True)
            top = units[0]
            t_max = t_unit(top)
            if len(top[1]) > 1:
                break
            c = top[1][0]
            bigger = sorted(t for t in tables[c] if t > top[0])
            if not bigger or tables[c][bigger[0]] >= tables[c][top[0]]:
                break
            nxt = bigger[0]
            need = used + nxt - top[0] - budget
            while need > 0:
                ones = sorted((u for u in units[1:] if u[0] == 1 and all(1 in tables[k] for k in u[1])), key=t_unit)
                pair = None
                for x in range(len(ones)):
                    for y in range(x + 1, len(ones)):
                        if kinds[ones[x][1][0]] == kinds[ones[y][1][0]]:
                            if pair is None or t_unit(ones[x]) + t_unit(ones[y]) < t_unit(pair[0]) + t_unit(pair[1]):
                                pair = (ones[x], ones[y])
                            break
                if pair is None or t_unit(pair[0]) + t_unit(pair[1]) >= t_max:
                    break
                a, b = pair
                a[1].extend(b[1])
                units.remove(b)
                used -= 1
                need -= 1
            if need > 0:
                break
            used += nxt - top[0]
            top[0] = nxt
        order, tc = [], []
        for size, members in units:
            for k, c in enumerate(members):
                order.append(c)
                tc.append(size if k == 0 else 0)
        return order, tc


class BatchRunner:
    """Runs a list of chains as batches of the team engine."""

    def __init__(self, chains, tuner: Autotuner, budget: int = 0):
        self.chains = list(chains)
        self.tuner = tuner
        self.budget = budget or device_ctas()
        self._plans = {}

    def candidates(self, w, updates):
        """Distinct team plans (order, team sizes) for the chains w of one
        wave: packed (small chains sharing CTAs), every probed size without
        sharing, and power-of-two sizes only."""
        Ls = [self.chains[i].L for i in w]
        work = [updates[i] for i in w]
        out = [self.tuner.pack(Ls, self.budget, work, [self.chains[i].recursion for i in w])]
        ident = list(range(len(w)))
        out.append((ident, self.tuner.allocate(Ls, self.budget, work)))
        out.append((ident, self.tuner.allocate(Ls, self.budget, work, sizes=(1, 2, 4, 8, 16, 32, 64))))
        seen, uniq = set(), []
        for order, tc in out:
            key = tuple(zip(order, tc))
            if key not in seen:
                seen.add(key)
                uniq.append((order, tc))
        return uniq

    def choose(self, w, updates):
        """The fastest candidate plan of wave w, each timed for one step on
        probe chains of the wave's lattice sizes and recursions (the probe
        times of chains alone do not show how the chains of a full batch
        share the L2)."""
        import torch
        cands = self.candidates(w, updates)
        if len(cands) == 1:
            return cands[0]
        t = self.tuner
        probes = [gfmc.Chain(self.chains[i].L, inputs.uniform_sphere(self.chains[i].L, 0), M=t.M,
                             precision=t.precision, beta=t.beta, mu=t.mu, recursion=self.chains[i].recursion,
                             compensated=self.chains[i].compensated, chain_id=k) for k, i in enumerate(w)]
        best = None
        try:
            for order, tc in cands:
                chs = [probes[k] for k in order]
                nu = [updates[w[k]] for k in order]
                gfmc.run_batch(chs, nu, team_ctas=tc, trace=False)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                gfmc.run_batch(chs, nu, team_ctas=tc, trace=False)
                dt = time.perf_counter() - t0
                if best is None or dt < best[0]:
                    best = (dt, order, tc)
        finally:
            for p in probes:
                p.close()
        return best[1], best[2]

    def plan(self, updates):
        """Waves of (chain indices, team sizes) that each fit the device
        (chosen once per list of update counts)."""
        key = tuple(updates)
        if key not in self._plans:
            self._plans[key] = self._plan(updates)
        return self._plans[key]

    def _plan(self, updates):
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
            order, tc = self.choose(w, updates)
            plan.append(([w[k] for k in order], tc))
        return plan

    def run(self, updates_per_chain, trace: bool = False):
        n = len(self.chains)
        updates = list(updates_per_chain) if hasattr(updates_per_chain, "__len__") else [updates_per_chain] * n
        out = [None] * n
        for w, tc in self.plan(updates):
            res = gfmc.run_batch([self.chains[i] for i in w], [updates[i] for i in w], team_ctas=tc, trace=trace)
            for k, i in enumerate(w):
                out[i] = dict(res[k], team_ctas=tc[k])  # 0: shares the CTA of the chain before it
        return out


CLUSTER_SIZES = (1, 2, 4, 8, 16)


def list_schedule(jobs, sms: int) -> float:
    """Makespan of jobs (cluster CTAs, seconds) started in the given order on
    `sms` SMs, each as soon as enough SMs are free, later jobs filling gaps
    that earlier ones cannot use (the device's cluster dispatch)."""
    import heapq
    now, free, running, waiting = 0.0, sms, [], list(jobs)
    while waiting or running:
        k = 0
        while k < len(waiting):
            C, d = waiting[k]
            if C <= free:
                free -= C
                heapq.heappush(running, (now + d, C))
                waiting.pop(k)
            else:
                k += 1
        if not running:
            raise ValueError("a job needs more SMs than the device has")
        now, C = heapq.heappop(running)
        free += C
        while running and running[0][0] <= now:
            free += heapq.heappop(running)[1]
    return now


class ClusterTuner:
    """Update times of the cluster engine per lattice size and cluster size,
    measured on the device, and the choice of cluster sizes and launch order
    for a batch: every assignment of a size to each lattice class is run
    through the list-scheduling model and the one with the shortest makespan
    wins; chains launch longest first."""

    def __init__(self, M: int, precision: str = "fp32_mixed", probe_updates: int = 2, beta: float = 20.0,
                 mu: float = -2.0, nodes: int = 0):
        self.M, self.precision, self.probe_updates = M, precision, probe_updates
        self.beta, self.mu, self.nodes = beta, mu, nodes
        self.table = {}  # L -> {cluster size: seconds per update}

    def measure(self, L: int) -> dict:
        if L in self.table:
            return self.table[L]
        import torch
        K = self.nodes or self.M
        cmin = gfmc.cluster_min_ctas(L, max(self.M, K), self.precision)
        res = {}
        with gfmc.Chain(L, inputs.uniform_sphere(L, 0), M=self.M, precision=self.precision, beta=self.beta,
                        mu=self.mu, recursion="proposal", nodes=self.nodes) as ch:
            for C in CLUSTER_SIZES:
                if C < cmin or L % C:
                    continue
                gfmc.run_clusters([ch], [1], [C], trace=False)  # warm-up
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                gfmc.run_clusters([ch], [self.probe_updates], [C], trace=False)
                res[C] = (time.perf_counter() - t0) / self.probe_updates
        self.table[L] = res
        return res

    def rank(self, Ls, updates, sms: int = 0, top: int = 0):
        """Assignments (cluster size per chain, launch order, modelled makespan)
        sorted by the modelled makespan; the first `top` (all if 0)."""
        import itertools
        sms = sms or device_ctas()
        classes = sorted(set(int(L) for L in Ls))
        tables = {L: self.measure(L) for L in classes}
        out = []
        for pick in itertools.product(*[sorted(tables[L]) for L in classes]):
            size = dict(zip(classes, pick))
            dur = [updates[c] * tables[int(L)][size[int(L)]] for c, L in enumerate(Ls)]
            order = sorted(range(len(Ls)), key=lambda c: -dur[c])
            span = list_schedule([(size[int(Ls[c])], dur[c]) for c in order], sms)
            out.append(([size[int(L)] for L in Ls], order, span))
        out.sort(key=lambda x: x[2])
        return out[:top] if top else out

    def choose(self, Ls, updates, sms: int = 0):
        """The assignment with the shortest modelled makespan."""
        return self.rank(Ls, updates, sms, top=1)[0]

    def choose_measured(self, chains, updates, top: int = 8):
        """The model's `top` assignments and the smallest-cluster one, each timed
        for one step on probe chains of the batch's lattice sizes (the model
        does not know how the device places clusters on its GPCs); the fastest
        wins.  Returns (sizes, order, measured seconds per step)."""
        import torch
        Ls = [c.L for c in chains]
        n = len(chains)
        cands = self.rank(Ls, updates, top=top)
        smallest = [min(self.measure(int(L))) for L in Ls]
        cands.append((smallest, sorted(range(n), key=lambda c: -updates[c] * self.table[int(Ls[c])][smallest[c]]),
                      None))
        probes = [gfmc.Chain(c.L, inputs.uniform_sphere(c.L, 0), M=self.M, precision=self.precision, beta=self.beta,
                             mu=self.mu, recursion="proposal", nodes=self.nodes, chain_id=k)
                  for k, c in enumerate(chains)]
        best = None
        try:
            for sizes, order, _ in cands:
                chs = [probes[i] for i in order]
                cs = [sizes[i] for i in order]
                nu = [updates[i] for i in order]
                gfmc.run_clusters(chs, nu, cs, trace=False)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                gfmc.run_clusters(chs, nu, cs, trace=False)
                dt = time.perf_counter() - t0
                if best is None or dt < best[2]:
                    best = (sizes, order, dt)
        finally:
            for p in probes:
                p.close()
        return best


class ClusterRunner:
    """Runs chains with the recursion on the proposal's vectors on
    thread-block clusters (gfmc_run_clusters).  With a ClusterTuner the
    cluster sizes and the launch order are the fastest, timed on probe
    chains, of the list-scheduling model's best assignments and the
    smallest-cluster one; without one each chain takes the smallest cluster
    whose shared memory holds its lattice (the fewest SMs per chain)."""

    def __init__(self, chains, tuner: "ClusterTuner" = None, updates: int = 4):
        self.chains = list(chains)
        n = len(self.chains)
        if tuner is None:
            self.cluster_ctas = [gfmc.cluster_min_ctas(c.L, max(c.M, c.K), c.precision) for c in self.chains]
            self.order = list(range(n))
            self.makespan = None
        else:
            self.cluster_ctas, self.order, self.makespan = tuner.choose_measured(self.chains, [updates] * n)

    def ordered(self):
        """(chains, cluster sizes) in launch order."""
        return [self.chains[i] for i in self.order], [self.cluster_ctas[i] for i in self.order]

    def run(self, updates_per_chain, trace: bool = False):
        n = len(self.chains)
        updates = list(updates_per_chain) if hasattr(updates_per_chain, "__len__") else [updates_per_chain] * n
        chs, cs = self.ordered()
        res = gfmc.run_clusters(chs, [updates[i] for i in self.order], cs, trace=trace)
        out = [None] * n
        for k, i in enumerate(self.order):
            out[i] = dict(res[k], cluster_ctas=self.cluster_ctas[i])
        return out


def c4_chains(n_chains: int = 64, M: int = 1024, precision: str = "fp32_mixed", seed: int = 4,
              sizes=(8, 12, 16, 24, 32), tmin: float = 0.02, tmax: float = 0.2, mu: float = -2.0,
              recursion: str = "unit_vectors", compensated: bool = False):
    """The batching workload: n_chains independent chains with L drawn from
    `sizes` and temperatures uniform in [tmin, tmax] (seeded), spins uniform on
    the sphere (seed = chain index), M moments, FP32-mixed by default
    (`compensated`: Dot2 sums of the Gram products)."""
    rng = np.random.default_rng(seed)
    Ls = rng.choice(sizes, size=n_chains)
    Ts = rng.uniform(tmin, tmax, size=n_chains)
    chains = [gfmc.Chain(int(L), inputs.uniform_sphere(int(L), c), M=M, precision=precision, beta=1.0 / T,
                         mu=mu, seed=1, chain_id=c, recursion=recursion, compensated=compensated)
              for c, (L, T) in enumerate(zip(Ls, Ts))]
    return chains, Ls, Ts
