"""The multi-GPU bench path is replicas only: each rank orthogonalizes its own
block, with no collective on the data path; the ranks only agree on the
slowest rank's time.  This checks that host logic with two gloo ranks on the
CPU (no GPU)."""
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


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        my_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        mx = bench.max_over_ranks(my_ms, "cpu")
        val = bench.weak_scaling_value(ws, 1e9, mx)
        q.put((rank, ws, r, mx, val))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_agree_on_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ws, r, mx, val in res:
        assert ws == 2 and r == rank
        assert mx == 15.0  # the max over ranks
        assert val == pytest.approx(2 * 1e9 / 15e-3 / 1e9)  # whole-job GB/s over both replicas


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.weak_scaling_value(1, 2e9, 1000.0) == pytest.approx(2.0)
    assert bench.alu_peak_tflops() == pytest.approx(64 * 152 * 2.07e9 / 10 * 2 / 1e12)
