"""The N > 1 host logic of bench.py (replicas, one rank per GPU) with two
gloo ranks on the CPU: the slowest rank's time and all ranks' launches make
the whole-job numbers; the reference arm runs on rank 0 only."""
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


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    allreduce = bench.make_allreduce(dist, "cpu")
    # rank r took 100 (r + 1) ms for 2 solves and launched 1000 + r kernels
    res = bench.aggregate(100.0 * (rank + 1), 1000 + rank, 2, world, allreduce, dist)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, res))


def test_whole_job_numbers_over_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        max_ms, launches, value = results[r]
        assert max_ms == 200.0                 # the slowest rank
        assert launches == 2001                # both ranks' kernels
        assert value == pytest.approx(2 * 2 / 0.2)


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    max_ms, launches, value = bench.aggregate(250.0, 7, 1, 1, bench.make_allreduce(None, "cpu"), None)
    assert (max_ms, launches) == (250.0, 7) and value == pytest.approx(4.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        pass
    bench.run_reference(A(), rank=1, world=2)      # returns before any work
    assert capsys.readouterr().out == ""
