"""Host-side logic of bench.py, on CPU: the multi-rank plumbing (gloo,
world size 2: each rank gets its own independent link window, the elapsed
time is the maximum over ranks) and the reference arm's JSON line."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    win = bench.window_for(rank, n=1 << 12)
    elapsed = 1.0 + rank  # rank 1 is the slow one
    mx = bench.dist_max(elapsed, world)
    bench.dist_barrier(world)
    with open(out_path % rank, "w") as f:
        json.dump({"max": mx, "first": win.pairs[:4].tolist()}, f)
    dist.destroy_process_group()


def test_two_ranks_get_independent_links_and_max_time(tmp_path):
    import torch.multiprocessing as mp
    port = 29500 + (os.getpid() % 1000)
    out = str(tmp_path / "rank%d.json")
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    r0 = json.load(open(out % 0))
    r1 = json.load(open(out % 1))
    assert r0["max"] == r1["max"] == 2.0
    assert r0["first"] != r1["first"]  # different seeds per link


def test_reference_arm_prints_one_json_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
           "--warmup", "3", "--ref-sample", "65536"]
    res = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "Gpps" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_reference_sample_bounds_the_run():
    """The reference arm's default sample keeps a run of --steps K near 55
    samples of 2^22 pairs (a few minutes of oracle work), never below 2^18."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.ref_sample_for(5, 5) == 1 << 22
    assert bench.ref_sample_for(50, 5) == 1 << 22
    for steps in (100, 200, 1000, 10_000):
        s = bench.ref_sample_for(steps, 5)
        assert (1 << 18) <= s < (1 << 22)
        assert s * (steps + 5) <= 55 * (1 << 22) or s == 1 << 18

