"""The multi-rank host logic of bench.py on CPU, with two real gloo ranks.

bench.py runs one process per GPU (torchrun); each rank advances its own
replica (weak scaling), the slowest rank's time is the job's time (a max over
ranks), and rank 0 alone prints. The reference arm runs on rank 0 only; the
other ranks exit without work.
"""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as tdist
    import bench
    tdist.init_process_group("gloo", rank=rank, world_size=2)
    r, world, local = bench.dist_env()
    times = bench.max_over_ranks([10.0 + 5.0 * rank, 7.0 - rank], world, device="cpu")
    rate = bench.whole_job_rate(1000, world, 20, times[0] / 1e3)
    tdist.barrier()
    tdist.destroy_process_group()
    out.put((r, world, local, times, rate))


def test_two_gloo_ranks_share_the_slowest_time():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, port, out)) for r in range(2)]
    for pr in procs:
        pr.start()
    got = sorted(out.get(timeout=120) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    for rank, (r, world, local, times, rate) in enumerate(got):
        assert (r, world, local) == (rank, 2, rank)
        assert times == [15.0, 7.0]                        # the max over the two ranks
        assert rate == pytest.approx(1000 * 2 * 20 / 0.015)  # all ranks' particles, slowest time


def test_single_rank_needs_no_process_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    assert bench.dist_env() == (0, 1, 0)
    assert bench.max_over_ranks([3.5, 1.0], 1) == [3.5, 1.0]
    assert bench.whole_job_rate(4_000_000, 1, 200, 0.5) == 4_000_000 * 200 / 0.5


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(None) is None           # returns before touching its arguments
    assert capsys.readouterr().out == ""
