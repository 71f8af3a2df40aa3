"""The serving loop (device-resident request loop with slots).

Jobs that run side by side in the server give the results the same chains
give alone: FP64 jobs are replayed by the oracle (Delta Omega 1e-10 |dO| +
1e-13 a, decisions identical except near ties), FP32-mixed jobs match the
same chain run alone within 1e-4 t.  Every poll loop has a host deadline.
"""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_6016_gb300 import inputs

pytestmark = pytest.mark.gpu

A = 6.05


def dom_tol(ref):
    return 1e-10 * abs(ref) + 1e-13 * A


@pytest.fixture(scope="module")
def G():
    from paper_1303_6016_gb300 import build, gfmc
    build.build()
    gfmc.load()
    return gfmc


def wait_all(server, slots, deadline_s=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(slots):
        for s in slots:
            if s not in out:
                r = server.poll(s)
                if r is not None:
                    out[s] = r
        assert time.time() - t0 < deadline_s, "server jobs did not finish"
        time.sleep(0.001)
    return out


def test_jobs_in_the_mix_match_oracle_and_alone(G):
    specs = [(6, "fp64", 1), (8, "fp64", 4), (5, "fp64", 2), (8, "fp32_mixed", 1), (12, "fp32_mixed", 4)]
    M = 64
    n = 40
    chains = []
    for c, (L, prec, _) in enumerate(specs):
        chains.append(G.Chain(L, inputs.uniform_sphere(L, 50 + c), M=M, precision=prec, seed=6, chain_id=c,
                              beta=15.0))
    with G.Server([tc for (_, _, tc) in specs], max_M=M) as srv:
        for k, ch in enumerate(chains):
            srv.submit(k, ch, n)
        res = wait_all(srv, list(range(len(specs))))
    for c, (L, prec, _) in enumerate(specs):
        out = res[c]
        assert chains[c].counter == n
        sp = inputs.uniform_sphere(L, 50 + c)
        if prec == "fp64":
            ref = O.updates(L, sp, n, M, beta=15.0, chem=-2.0, seed=6, chain_id=c,
                            forced=out["decisions"].astype(np.int8))
            for q in range(n):
                assert abs(out["d_omega"][q] - ref["d_omega"][q]) <= dom_tol(ref["d_omega"][q])
                if bool(ref["ratio"][q] > ref["u"][q]) != bool(out["decisions"][q]):
                    assert abs(ref["ratio"][q] - ref["u"][q]) < 1e-9
        else:
            with G.Chain(L, sp, M=M, precision=prec, seed=6, chain_id=c, beta=15.0) as alone:
                a = alone.updates(n)
            same = a["decisions"] == out["decisions"]
            k = n if same.all() else int(np.argmin(same))
            assert k >= 10
            assert np.abs(a["d_omega"][:k] - out["d_omega"][:k]).max() <= 1e-4
    for ch in chains:
        ch.close()


def test_consecutive_jobs_continue_the_chain_and_idle_relaunch(G):
    L, M = 6, 64
    sp = inputs.uniform_sphere(L, 77)
    with G.Chain(L, sp, M=M, seed=8) as alone:
        full = alone.updates(60)
    ch = G.Chain(L, sp, M=M, seed=8)
    with G.Server([2, 1], max_M=M) as srv:
        srv.submit(0, ch, 25)
        r1 = wait_all(srv, [0])[0]
        time.sleep(2.5)  # longer than the idle budget: the launch ends by itself
        srv.submit(1, ch, 35)  # the next submit starts it again
        r2 = wait_all(srv, [1])[1]
    d = np.concatenate([r1["d_omega"], r2["d_omega"]])
    dec = np.concatenate([r1["decisions"], r2["decisions"]])
    same = dec == full["decisions"]
    k = 60 if same.all() else int(np.argmin(same))
    assert k >= 30
    assert np.abs(d[:k] - full["d_omega"][:k]).max() <= dom_tol(1.0)
    assert ch.counter == 60
    ch.close()


def test_idle_slot_takes_a_job_while_another_slot_is_busy(G):
    """A slot idle for longer than the idle budget stays in the launch while
    another slot works, so a job posted to it runs at once instead of waiting
    for the busy slot's job and a relaunch."""
    long_ch = G.Chain(12, inputs.uniform_sphere(12, 5), M=1024, seed=3)   # FP64, about 77 ms per update on 1 CTA
    short_ch = G.Chain(6, inputs.uniform_sphere(6, 6), M=64, seed=4)
    with G.Server([1, 1], max_M=1024) as srv:
        srv.submit(0, long_ch, 60)
        time.sleep(1.6)  # longer than the idle budget: slot 1 has been idle since the launch
        t0 = time.time()
        srv.submit(1, short_ch, 5)
        r1 = None
        while r1 is None:
            r1 = srv.poll(1)
            assert time.time() - t0 < 120.0, "server job did not finish"
            time.sleep(0.001)
        dt = time.time() - t0
        assert srv.poll(0) is None, "the long job ended first: lengthen it"
        assert dt < 0.5, dt
        wait_all(srv, [0])
    assert long_ch.counter == 60 and short_ch.counter == 5
    long_ch.close()
    short_ch.close()


def test_busy_slot_and_busy_chain_are_rejected(G):
    L, M = 8, 64
    a = G.Chain(L, inputs.uniform_sphere(L, 1), M=M)
    b = G.Chain(L, inputs.uniform_sphere(L, 2), M=M)
    with G.Server([1, 1], max_M=M) as srv:
        srv.submit(0, a, 200)
        with pytest.raises(G.GfmcError) as e:
            srv.submit(0, b, 5)  # slot 0 busy
        assert e.value.status == G.GFMC_EINVAL
        with pytest.raises(G.GfmcError) as e:
            srv.submit(1, a, 5)  # chain a already has a job
        assert e.value.status == G.GFMC_EINVAL
        wait_all(srv, [0])
    a.close()
    b.close()


def test_proposal_recursion_jobs_match_oracle(G):
    specs = [(6, "fp64", 2), (8, "fp64", 1)]
    M, n = 64, 30
    chains = [G.Chain(L, inputs.uniform_sphere(L, 90 + c), M=M, precision=prec, seed=3, chain_id=c,
                      recursion="proposal") for c, (L, prec, _) in enumerate(specs)]
    with G.Server([tc for (_, _, tc) in specs], max_M=M) as srv:
        for k, ch in enumerate(chains):
            srv.submit(k, ch, n)
        res = wait_all(srv, [0, 1])
    for c, (L, _, _) in enumerate(specs):
        out = res[c]
        ref = O.updates(L, inputs.uniform_sphere(L, 90 + c), n, M, beta=20.0, chem=-2.0, seed=3, chain_id=c,
                        forced=out["decisions"].astype(np.int8))
        for q in range(n):
            assert abs(out["d_omega"][q] - ref["d_omega"][q]) <= dom_tol(ref["d_omega"][q])
            if bool(ref["ratio"][q] > ref["u"][q]) != bool(out["decisions"][q]):
                assert abs(ref["ratio"][q] - ref["u"][q]) < 1e-9
    for ch in chains:
        ch.close()
