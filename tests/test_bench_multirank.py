"""The multi-process side of bench.py on CPU (gloo, world size 2): the whole-job
time is the slowest rank's and the work is summed over ranks; the reference arm
runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, work = bench.aggregate(10.0 + 5.0 * rank, 1000.0 * (rank + 1), dist, "cpu")
    q.put((rank, ms, work))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_max_time_sum_work_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, work in got:
        assert ms == 15.0 and work == 3000.0


def test_aggregate_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.aggregate(3.5, 42.0, None) == (3.5, 42.0)


def test_reference_arm_nonzero_rank_exits_without_output():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
