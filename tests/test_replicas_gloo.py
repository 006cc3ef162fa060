"""The multi-GPU bench path on CPU: one process per GPU, each a replica of the
whole workload (the screen does not shard: no data-path collective).  Two
gloo ranks check the one cross-rank step, the slowest-rank reduction that
turns per-rank times into the whole-job number, and that a non-zero rank of
the reference arm exits without work."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.slowest_rank(times[rank], world, device="cpu")
        out[rank] = (t, t / (4 * world))  # 4 screens per rank -> whole-job ms per screen
    finally:
        dist.destroy_process_group()


def test_slowest_rank_over_two_gloo_ranks():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(2, port, [30.0, 42.5], out), nprocs=2, join=True)
    assert out[0] == out[1] == (42.5, 42.5 / 8)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank(12.5, 1) == 12.5


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
