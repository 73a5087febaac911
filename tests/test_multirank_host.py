"""Host logic of `bench.py --gpus N` (N independent replicas, one process per
GPU) checked with world-size-2 gloo process groups on the CPU: the job's time
is the slowest rank's, the job's throughput counts every rank's samples, and
the reference arm runs on rank 0 only.  No GPU is used."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = 10.0 + 7.5 * rank                       # rank 1 is the slower one
    job = bench.slowest_rank_ms(mine, world, "cpu")
    value = bench.job_msamples_per_s(1e6, job, world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, job, value))


def test_two_replicas_report_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [17.5, 17.5]
    # 2 ranks x 1e6 samples in 17.5 ms
    assert res[0][2] == pytest.approx(2 * 1e6 / 17.5e-3 / 1e6)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank_ms(3.25, 1, "cpu") == 3.25
    assert bench.job_msamples_per_s(2e6, 4.0, 1) == pytest.approx(500.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    bench.run_reference(bench.parse_args())       # returns without work or output
    assert capsys.readouterr().out == ""
