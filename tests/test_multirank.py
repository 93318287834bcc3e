"""The replica path of bench.py at world size 2 on CPU (gloo): each rank
solves its own instance, the job time is the slowest rank's, and only rank 0
runs the reference arm."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    m = bench.max_over_ranks(10.0 * (rank + 1), "cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, m))


def test_max_over_ranks_gloo_world2():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 20.0, 1: 20.0}


def test_max_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5


def test_reference_arm_runs_on_rank0_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(argparse.Namespace(steps=1, warmup=0)) == 0
    assert capsys.readouterr().out == ""


def test_all_cores_oracle_leg_runs_every_worker():
    """The all-cores CPU leg of bench.py: spawned workers, each running the
    unmodified oracle on its own crop; the throughput counts every worker's
    units over the wall time of the whole map."""
    sys.path.insert(0, ROOT)
    import bench
    f = bench.make_input(0)
    n, reps = bench.cpu_sample_all_cores(f, 24, 3, reps=2, workers=2)
    assert n == 2 and len(reps) == 2
    for value, wall in reps:
        assert wall > 0 and value > 0
        assert abs(value - 2 * 24 * 24 * bench.K_INT * 3 / wall / 1e9) <= 1e-12 * value
