"""The multi-rank host logic of the benchmark, on CPU ranks over gloo (world size 2).

The path runs as independent replicas (one per GPU, no collective on the data path); what the
ranks share is the timing: the job's step time is the maximum over the ranks and its rate is the
units all ranks processed per second of that time.  The reference arm runs on rank 0 alone.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.whole_job_rate(10.0 + 2.5 * rank, 1000, world, dist, "cpu")
    with open(os.path.join(outdir, "r%d.json" % rank), "w") as f:
        json.dump({"ms": ms, "value": value}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_single_rank_rate():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.whole_job_rate(12.5, 1000, 1)
    assert ms == 12.5 and value == pytest.approx(1000 / 12.5e-3)


def test_two_ranks_take_the_slowest_rank(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / ("r%d.json" % r))) for r in range(world)]
    for r in res:                          # every rank sees the slowest rank's time
        assert r["ms"] == 12.5
        assert r["value"] == pytest.approx(world * 1000 / 12.5e-3)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""
