"""The replica path of bench.py with two ranks on the CPU (gloo): every rank times its own solves,
the job time is the slowest rank's, and the job time per solve counts the solves of all ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    r, w = bench.dist_init("gloo")
    assert (r, w) == (rank, world)
    my_ms = 100.0 + 50.0 * rank          # rank 1 is slower
    mx = bench.dist_max(my_ms)
    tot = bench.dist_sum(8.0)
    bench.dist_barrier()
    out[rank] = (mx, tot, bench.job_ms_per_unit(mx, 8 * 5, w))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for rank in (0, 1):
        mx, tot, per = out[rank]
        assert mx == 150.0
        assert tot == 16.0
        assert per == pytest.approx(150.0 / 80.0)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(bench.parse_args(["--impl", "reference", "--steps", "1", "--warmup", "0"]))
    assert capsys.readouterr().out == ""
