"""The multi-rank logic of bench.py on CPU with two gloo ranks: replicas
(weak scaling, no data-path collective), the max over ranks of the timed
region and the whole-job rate; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as tdist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist()
    local_ms = 100.0 + 37.5 * r                     # each rank's own timed region
    tdist.barrier()
    slowest = bench.max_over_ranks(local_ms, tdist)
    rate = bench.job_rate(ws, 20000 * 5, slowest / 1e3)
    q.put((r, ws, local, slowest, rate, bench.replica_event_id(r)))
    tdist.barrier()
    tdist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_sum_the_work():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = 100.0 + 37.5 * (world - 1)
    for r, (rank, ws, local, s, rate, eid) in enumerate(res):
        assert rank == r and ws == world and local == r
        assert s == pytest.approx(slowest)
        assert rate == pytest.approx(world * 20000 * 5 / (slowest / 1e3))
    assert len({eid for *_, eid in res}) == world        # each replica has its own event id


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    ns = type("A", (), dict(workload="tile", steps=1, warmup=0))()
    bench.run_reference(ns)                              # returns at once on rank 1
    assert capsys.readouterr().out == ""
    assert bench.max_over_ranks(3.5) == 3.5              # alone: no collective


def test_gpus_must_match_the_launched_ranks():
    sys.path.insert(0, ROOT)
    import bench
    bench.check_ranks(1, 1)
    bench.check_ranks(4, 4)
    for gpus, world in ((2, 1), (1, 2), (8, 4)):
        with pytest.raises(SystemExit, match="torch.distributed.run"):
            bench.check_ranks(gpus, world)
