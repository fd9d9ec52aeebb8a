"""The multi-GPU bookkeeping (independent tanks, one per rank) with two gloo
ranks on CPU: the barrier, the maximum of the ranks' times and the job
throughput counting every rank's nodes; and a rank that fails before the
barrier, which the other rank learns of as RankFailure within the process
group's timeout instead of waiting forever."""
import os
import socket
import time

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    from paper_2209_10411_gb300 import replicas
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = replicas.rank_env()
        assert (r, w, local) == (rank, world, rank)
        replicas.barrier(w)
        ms = 10.0 + 3.0 * rank              # the slower rank's time must count
        ms_max = replicas.max_over_ranks(ms, w)
        value = replicas.aggregate_throughput(1000.0, w, ms_max)
        with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as fh:
            fh.write("%r %r\n" % (ms_max, value))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    vals = [open(tmp_path / ("rank%d.txt" % r)).read().split() for r in range(world)]
    for ms_max, value in vals:
        assert float(ms_max) == 13.0
        assert abs(float(value) - 1000.0 * 2 / 13e-3) < 1e-6


def _failing_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    from paper_2209_10411_gb300 import replicas
    replicas.init_process_group("gloo", timeout_s=5.0, rank=rank, world_size=world)
    if rank == 1:
        raise SystemExit(3)          # this rank fails between steps, with nothing in flight
    t0 = time.time()
    try:
        replicas.barrier(world)
        outcome = "passed"
    except replicas.RankFailure:
        outcome = "detected"
    with open(os.path.join(out_dir, "rank0.txt"), "w") as fh:
        fh.write("%s %.1f\n" % (outcome, time.time() - t0))
    try:
        dist.destroy_process_group()
    except Exception:
        pass


@pytest.mark.timeout(120)
def test_failed_rank_is_detected(tmp_path):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=90)
    assert procs[1].exitcode == 3
    assert procs[0].exitcode == 0
    outcome, waited = open(tmp_path / "rank0.txt").read().split()
    assert outcome == "detected" and float(waited) < 60.0
