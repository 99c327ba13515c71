"""The N-replica host logic of bench.py on CPU (gloo, world size 2): the timed region's length is
the slowest rank's, the whole-job rate counts every rank's solves, and the reference arm runs on
rank 0 only.  The solve does not shard (replicas only), so there is no data-path collective to
test; no GPU is used.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = bench.max_over_ranks(1.0 + rank, dist, "cpu")     # rank 1 is the slower one
        out.put((rank, elapsed, bench.replica_rate(world, 10, elapsed)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_count_every_solve():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.0, 2.0]                 # both see the slower rank's time
    assert [r[2] for r in res] == [10.0, 10.0]               # 2 ranks x 10 solves / 2 s


def test_one_rank_needs_no_collective():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_rate(1, 50, 0.5) == 100.0


def test_reference_arm_runs_on_rank_zero_only():
    class Args:
        steps, warmup, gpus, ref_iters = 1, 0, 2, 1
    assert bench.run_reference(Args(), world=2, rank=1) == 0     # returns at once, no work
