"""The N > 1 path of bench.py on CPU: world_size 2 over gloo (127.0.0.1).

Rays shard into independent replicas with no data-path collective; the only
cross-rank step is the timing aggregation (max over ranks) and rank 0's
report.  These run the same helpers bench.py uses under torchrun."""

import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) * 10 ms for the timed steps and r + 0.5 s end to end
        total_ms, e2e_s = bench.max_over_ranks([(rank + 1) * 10.0, rank + 0.5],
                                               torch.device("cpu"))
        dist.barrier()
        out[rank] = (total_ms, e2e_s, bench.job_rate(1000, world, 2, total_ms))
    finally:
        dist.destroy_process_group()


def test_timing_is_the_slowest_rank_and_rate_counts_all_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        total_ms, e2e_s, rate = out[r]
        assert total_ms == 20.0 and e2e_s == 1.5
        # 1000 units per rank per step, 2 steps, 2 ranks over 20 ms
        assert rate == pytest.approx(1000 * 2 * 2 / 0.020)


def test_reference_arm_on_a_nonzero_rank_does_no_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
