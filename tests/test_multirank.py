"""Multi-rank host logic of the benchmark on CPU (gloo, 2 ranks): the job's
time is the slowest rank's and the rate counts every rank's units (weak
scaling of independent replicas); the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took r + 1 seconds for its 100 units
    rate, secs = bench.whole_job_rate(rank + 1.0, 100.0, world, device="cpu")
    out.put((rank, rate, secs))
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_rate_two_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, rate, secs in res:
        assert secs == pytest.approx(2.0)          # the slowest rank
        assert rate == pytest.approx(2 * 100.0 / 2.0)


def test_single_rank_rate():
    assert bench.whole_job_rate(4.0, 100.0, 1) == (25.0, 4.0)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup = 1, 0
    bench.run_reference(Args())
    assert capsys.readouterr().out == ""
