"""The N > 1 path of the benchmark on CPU (gloo, world size 2): the path has
no exchange step, so N GPUs run N independent replicas and the job's
frames/s is N x steps over the slowest rank's timed region; the reference
arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        assert (r, w, local) == (rank, world, rank)
        # rank k timed 10 frames in 100 (k + 1) ms: the job waits for the slowest rank
        value, job_ms = bench.replica_throughput(100.0 * (rank + 1), 10, world)
        out[rank] = (value, job_ms)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_gloo():
    world = 2
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for value, job_ms in res.values():
        assert job_ms == 200.0
        assert abs(value - world * 10 / 0.2) < 1e-9      # 100 frames/s for the job


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    value, job_ms = bench.replica_throughput(250.0, 5, 1)
    assert job_ms == 250.0 and abs(value - 20.0) < 1e-12


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup = 1, 0
    assert bench.run_reference(Args()) is None
    assert capsys.readouterr().out == ""
