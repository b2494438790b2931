"""The benchmark's N > 1 path on the CPU: two replicas as gloo ranks on
127.0.0.1 combine their figures as the whole-job rule says (the largest time
over ranks, the units summed), and under torchrun only rank 0 of the
reference arm does work and prints."""
import os
import socket
import subprocess
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        times, units = bench.whole_job([1.0 + rank, 10.0 - rank], [100.0 * (rank + 1), 7.0])
        assert times == [float(world), 10.0], times
        assert units == [100.0 * world * (world + 1) / 2, 7.0 * world], units
    finally:
        dist.destroy_process_group()


def test_whole_job_over_two_gloo_ranks():
    mp.spawn(_rank, args=(2, _free_port()), nprocs=2, join=True)


def test_whole_job_on_one_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job([2.5, 3.0], [11.0]) == ([2.5, 3.0], [11.0])


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "sod",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True, cwd=ROOT, env=env,
                         timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [l for l in out.stdout.splitlines() if l.startswith("{")]
