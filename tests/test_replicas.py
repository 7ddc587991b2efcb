"""The N > 1 path of bench.py on CPU: replicas are independent, so the only
exchange is the timing reduction (max of the time, sum of the units) that
bench.whole_job performs; tested here with world_size 2 over gloo.  The
reference arm must leave every rank but 0 without work."""
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took 1 + r seconds for 100 (r + 1) units
    out[rank] = bench.whole_job(1.0 + rank, 100.0 * (rank + 1), world)
    dist.destroy_process_group()


def test_whole_job_over_two_ranks():
    world = 2
    with mp.get_context("spawn").Manager() as m:  # no fork of a process that may hold a CUDA context
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        for r in range(world):
            sec, units, value = out[r]
            assert sec == 2.0 and units == 300.0 and value == 150.0


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job(2.0, 10.0, 1) == (2.0, 10.0, 5.0)


def test_reference_arm_on_rank_one_does_no_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
