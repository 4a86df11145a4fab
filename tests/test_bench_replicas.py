"""The multi-GPU path of bench.py is N independent replicas: ranks meet only
for a barrier and the maximum of their step times.  Checked here with two
gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    r, w = bench.dist_init(world, backend="gloo")
    bench.barrier(w)
    ms = 10.0 + 5.0 * r                       # rank 1 is the slow replica
    slowest = bench.allmax(ms, w)
    out[r] = (r, w, slowest, bench.replica_value(1000, w, slowest))
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_step():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in range(world):
        rank, w, slowest, value = res[r]
        assert w == world and slowest == 15.0
        # whole-job throughput: both replicas' points over the slowest time
        assert abs(value - 2.0 * 1000 * world / 15e-3 / 1e6) < 1e-12


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        warmup, steps = 3, 1

    bench.run_reference(Args())
    assert capsys.readouterr().out == ""
