"""The multi-rank path of bench.py on the CPU: the path has no exchange step
on one GPU, so N ranks run N independent replicas and only the timing is
combined (the slowest rank's time, the units of all ranks).  Two gloo ranks
on 127.0.0.1 check that aggregation; a non-zero rank of the reference arm
exits at once without work."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: 10 ms per step more than rank r-1, 1000 * (r + 1) particle-steps
        elapsed, units = bench.aggregate_replicas(100.0 + 10.0 * rank, 1000.0 * (rank + 1))
        results[rank] = (elapsed, units)
    finally:
        dist.destroy_process_group()


def test_aggregate_replicas_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        results = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, results), nprocs=world, join=True)
        got = dict(results)
    for rank in range(world):
        elapsed, units = got[rank]
        assert elapsed == pytest.approx(110.0)  # the slowest rank
        assert units == pytest.approx(3000.0)   # both ranks' units


def test_aggregate_replicas_without_process_group():
    import bench
    assert bench.aggregate_replicas(12.5, 400) == (12.5, 400.0)


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                         env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == ""
