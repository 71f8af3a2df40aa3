"""The serving loop's host logic (paper_1303_6016_gb300/serving.py) on CPU,
with the device server and chains replaced by fakes: admission by the HBM
budget (a chain becomes resident only while the budget holds it, and once),
the choice of a slot (never more CTAs than the chain has sites; the preferred
width when it is free), and the request loop (every request served, a chain
never in two slots at once, requests of a busy chain waiting without blocking
the others)."""
import pytest

from paper_1303_6016_gb300 import serving


class FakeChain:
    def __init__(self, L, spins, M, precision, **kw):
        self.L, self.M, self.precision = L, M, precision
        self.device_bytes = serving.footprint(L, M, precision)

    def close(self):
        pass


class FakeServer:
    """Each job completes on its third poll."""

    def __init__(self, slots, max_M):
        self.slots = list(slots)
        self.jobs = {}
        self.busy = set()
        self.log = []

    def submit(self, s, chain, K, trace=False):
        assert s not in self.jobs, "slot submitted while busy"
        assert id(chain) not in self.busy, "chain in two slots at once"
        assert self.slots[s] <= chain.L ** 3, "slot wider than the chain's sites"
        self.jobs[s] = [3, chain]
        self.busy.add(id(chain))
        self.log.append((s, chain.L, K))

    def poll(self, s):
        job = self.jobs[s]
        job[0] -= 1
        if job[0] > 0:
            return None
        del self.jobs[s]
        self.busy.discard(id(job[1]))
        return {}

    def close(self):
        pass


@pytest.fixture
def fakes(monkeypatch):
    monkeypatch.setattr(serving.gfmc, "Server", FakeServer)
    monkeypatch.setattr(serving.gfmc, "Chain", FakeChain)


SPECS = [{"L": 16, "M": 1024, "precision": "fp64", "chain_id": 0},
         {"L": 24, "M": 512, "precision": "fp32_mixed", "chain_id": 1},
         {"L": 48, "M": 2048, "precision": "fp64", "chain_id": 2},
         {"L": 3, "M": 512, "precision": "fp32_mixed", "chain_id": 3}]


def test_admission_respects_the_budget(fakes):
    fp = [serving.footprint(s["L"], s["M"], s["precision"]) for s in SPECS]
    sch = serving.Scheduler(SPECS, hbm_budget=fp[0] + fp[1] + fp[3] + 1)
    assert sch._resident(0) and sch._resident(1)
    assert not sch._resident(2)  # the L = 48 chain does not fit what is left
    assert sch._resident(3)
    used = sch.used
    assert used == fp[0] + fp[1] + fp[3] <= sch.budget
    assert sch._resident(0) and sch.used == used  # already resident: not charged again
    sch.close()


def test_slot_choice(fakes):
    sch = serving.Scheduler(SPECS, hbm_budget=1e12)
    # L = 3 (27 sites): never the 32-CTA slot; a cheap job prefers 2-CTA slots
    s = sch._slot_for(3)
    assert sch.slots[s] == serving.preferred_team(3, 512, "fp32_mixed") == 2
    # the costliest job (FP64, L = 48, M = 2048) takes the widest slot
    s = sch._slot_for(2)
    assert sch.slots[s] == 32
    # with only the wide slot free, the L = 3 chain cannot use it
    sch.free = {sch.slots.index(32)}
    assert sch._slot_for(3) is None
    sch.close()


def test_request_loop_serves_every_request(fakes):
    sch = serving.Scheduler(SPECS, hbm_budget=1e12, K=2)
    # repeated requests for chain 0 arrive together: they must run one after another
    reqs = [(0.0, 0), (0.0, 0), (0.0, 1), (0.001, 3), (0.002, 0), (0.003, 2)]
    out = sch.run(reqs, seconds=0.05, drain_s=2.0)
    assert out["completed"] == len(reqs) and out["left_waiting"] == 0
    assert len(sch.server.log) == len(reqs)
    assert all(k == 2 for _, _, k in sch.server.log)
    assert out["p50_s"] is not None and out["p99_s"] >= out["p50_s"]
    sch.close()
