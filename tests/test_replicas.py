"""Replica chains across ranks (the only multi-GPU form of the path): the
benchmark's rank set-up, max-over-ranks timing and whole-job aggregation, run
as two gloo ranks on the CPU; and a rank that dies before the timing
collective, which the surviving rank must see as an error (no hang)."""
import datetime
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})


def _worker_max(rank, world, port, q):
    _env(rank, world, port)
    r, w, local, dist = bench.dist_setup(world)
    assert (r, w, local) == (rank, world, rank)
    local_ms = [1000.0, 1250.0][rank]  # the slower replica bounds the job
    mx = bench.max_over_ranks(dist, local_ms)
    bench.barrier(dist)
    q.put((rank, mx, bench.aggregate(w, steps=10, updates_per_step=16, max_total_ms=mx)))
    dist.destroy_process_group()


def test_two_rank_max_and_aggregate():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker_max, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, mx, value in got:
        assert mx == 1250.0
        assert value == pytest.approx(2 * 10 * 16 / 1.25)


def _worker_dies(rank, world, port, q):
    _env(rank, world, port)
    import torch.distributed as dist
    dist.init_process_group("gloo", timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        os._exit(3)  # a replica that dies between steps, before the timing collective
    try:
        bench.max_over_ranks(dist, 1.0)
        q.put(("no error", rank))
    except Exception as e:  # the survivor learns of it on the host
        q.put(("error", type(e).__name__))


def test_dead_replica_is_detected_by_survivor():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker_dies, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert procs[1].exitcode == 3
    status, _ = q.get(timeout=5)
    assert status == "error"

