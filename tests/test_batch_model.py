"""The cluster-schedule model of the batch runner (host logic, no GPU): the
list-scheduling makespan and the tuner's choice of cluster sizes and launch
order."""
import pytest

def test_list_schedule_model():
    from paper_1303_6016_gb300.batch import list_schedule
    assert list_schedule([(4, 1.0), (4, 1.0)], 4) == 2.0
    assert list_schedule([(2, 1.0), (2, 1.0)], 4) == 1.0
    # a wide job first, then narrow ones fill the gaps it leaves
    assert list_schedule([(3, 2.0), (1, 1.0), (1, 1.0)], 4) == 2.0
    # a job that must wait for SMs starts when enough are free
    assert list_schedule([(3, 2.0), (2, 1.0)], 4) == 3.0
    with pytest.raises(ValueError):
        list_schedule([(8, 1.0)], 4)


def test_cluster_tuner_picks_the_shortest_modelled_makespan():
    from paper_1303_6016_gb300.batch import ClusterTuner, list_schedule
    tuner = ClusterTuner(M=1024)
    # seconds per update at each cluster size (measured on a GB300 for the
    # 64-chain workload's lattice sizes, M = 1024, FP32-mixed)
    tuner.table = {8: {1: 0.836e-3, 2: 0.68e-3, 4: 0.571e-3}, 12: {1: 1.608e-3, 2: 1.099e-3, 4: 0.838e-3},
                   16: {1: 2.513e-3, 2: 1.547e-3, 4: 0.999e-3, 8: 0.727e-3, 16: 0.841e-3},
                   24: {4: 2.266e-3, 8: 1.57e-3}, 32: {8: 2.554e-3, 16: 1.752e-3}}
    Ls = [8] * 8 + [12] * 11 + [16] * 17 + [24] * 10 + [32] * 18
    sizes, order, span = tuner.choose(Ls, [4] * len(Ls), sms=152)
    smallest = {8: 1, 12: 1, 16: 1, 24: 4, 32: 8}
    base = list_schedule(sorted([(smallest[L], 4 * tuner.table[L][smallest[L]]) for L in Ls],
                                key=lambda j: -j[0]), 152)
    assert span < base
    assert sorted(order) == list(range(len(Ls)))
    durs = [4 * tuner.table[Ls[c]][sizes[c]] for c in order]
    assert durs == sorted(durs, reverse=True)
    assert all(tuner.table[L].get(C) is not None for L, C in zip(Ls, sizes))


def test_team_packer_shares_ctas_and_shortens_the_slowest_team():
    """Small chains share one-CTA teams (team size 0 after a 1) so that the
    large chains' teams can grow: the packed plan fits the budget, every chain
    appears once, every 0 follows a one-CTA team, and the slowest unit is no
    slower than the plan without sharing."""
    from paper_1303_6016_gb300.batch import Autotuner
    tuner = Autotuner.__new__(Autotuner)
    # seconds per update at each team size (the team engine's shape: about
    # 1/n for large lattices, flat for small ones)
    base = {8: 3.4e-3, 12: 9.2e-3, 16: 18e-3, 24: 59e-3, 32: 134e-3}
    tuner.table = {L: {n: t / n + 1.5e-3 * (n > 1) for n in (1, 2, 3, 4, 5, 6, 8, 12, 16)} for L, t in base.items()}
    Ls = [8] * 8 + [12] * 11 + [16] * 17 + [24] * 10 + [32] * 18
    budget = 152
    plain = tuner.allocate(Ls, budget)
    order, tc = tuner.pack(Ls, budget)
    assert sorted(order) == list(range(len(Ls)))
    assert sum(tc) <= budget and tc[0] >= 1
    units = []
    for k, (c, t) in enumerate(zip(order, tc)):
        if t == 0:
            assert tc[k - 1] in (0, 1)
            units[-1][1].append(c)
        else:
            units.append((t, [c]))

    def t_unit(u):
        t, cs = u
        return tuner.table[Ls[cs[0]]][t] if len(cs) == 1 else sum(tuner.table[Ls[c]][1] for c in cs)

    t_plain = max(tuner.table[L][t] for L, t in zip(Ls, plain))
    t_packed = max(t_unit(u) for u in units)
    assert any(len(cs) > 1 for _, cs in units)
    assert t_packed < t_plain
