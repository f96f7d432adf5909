"""The N > 1 path of bench.py on CPU: full-matrix sweeps do not shard, so N GPUs run N independent
replicas; the job's time is the slowest rank's and the value counts every rank's solves.  Checked
with two gloo ranks (no GPU)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = 1.0 + rank  # rank 1 is the slow one
    t = bench.max_over_ranks(elapsed, "cpu")
    out.put((rank, t, bench.whole_job_value(world, 3, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.0, 2.0]          # both ranks see the max
    assert all(abs(r[2] - 3.0) < 1e-12 for r in res)  # 2 ranks x 3 solves / 2 s


def test_single_process_is_a_no_op():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.25, "cpu") == 1.25
    assert bench.whole_job_value(1, 4, 2.0) == 2.0


def test_reference_arm_prints_only_on_rank_zero(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        size = 8
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
