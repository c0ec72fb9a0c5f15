"""The multi-rank logic of shard.py on CPU: gloo ranks (world size 2 and 4)
exchange the DHLAs and pairs of one window through torch.distributed, with
the CPU oracle in place of the GPU steps, and the result is checked against
the oracle run on the whole window.

* Stream split then OR merge (§4.2): each rank builds the DHLA of its part
  of the window; after or_allreduce every rank holds the DHLA of the whole
  window, and its report is the whole window's.
* Key partition (§5): each rank's pairs go to the rank owning their key
  (key & (world - 1)) in each direction; each rank's DHLA and its own hits
  equal the oracle's on the pairs of its keys, and together the ranks
  report every super point the oracle finds among all keys' partitions."""
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SEED = 0x5A4E


def _setup(rank, world, port):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _np_or_parts(dst, src, words, count):
    import torch
    a = src.numpy().view(np.uint32).reshape(count, words)
    dst.copy_(torch.from_numpy(np.bitwise_or.reduce(a, axis=0).view(np.int32)))


def _np_partition(direction, pairs, parts):
    import torch
    p = pairs.numpy().view(np.uint32).reshape(-1, 2)
    key = p[:, direction]
    part = key & np.uint32(parts - 1)
    order = np.argsort(part, kind="stable")
    kp = p[order][:, [direction, 1 - direction]]
    counts = np.bincount(part, minlength=parts)
    return torch.from_numpy(np.ascontiguousarray(kp).reshape(-1).view(np.int32)), counts


def _workload():
    from paper_1803_11449_gb300 import traffic as T
    w = T.WORKLOADS["tiny"].with_(dirs=2, n=(1 << 18) + 3, planted=16, planted_c=("uniform", 1500, 4000))
    return w, T.make_window(w, 404).pairs


def _or_rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    _setup(rank, world, port)
    import oracle as O
    from paper_1803_11449_gb300 import shard
    w, pairs = _workload()
    op = O.params_from(w.sketch(), seed=SEED)
    mine = np.array_split(pairs, world)[rank]
    grid = O.new_grid(op)
    O.update(op, grid, mine)
    merged = shard.or_allreduce(torch.from_numpy(grid.view(np.int32)), or_parts=_np_or_parts)
    merged = merged.numpy().view(np.uint32)
    whole = O.new_grid(op)
    O.update(op, whole, pairs)
    rep = O.close_window(op, merged)
    ref = O.close_window(op, whole)
    with open(out % rank, "w") as f:
        json.dump({"grid_equal": bool(np.array_equal(merged, whole)),
                   "ips_equal": bool(np.array_equal(rep["ip"], ref["ip"])),
                   "est_equal": bool(np.array_equal(rep["est"], ref["est"])),
                   "hits": int(rep["n_hits"])}, f)
    dist.destroy_process_group()


def _part_rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    _setup(rank, world, port)
    import oracle as O
    from paper_1803_11449_gb300 import shard
    w, pairs = _workload()
    op = O.params_from(w.sketch(), seed=SEED)
    mine = np.array_split(pairs, world)[rank]
    t = torch.from_numpy(np.ascontiguousarray(mine).reshape(-1).view(np.int32))
    halves = []
    received = []
    for d in range(2):
        kp = shard.exchange_by_key(t, d, partition=_np_partition).numpy().view(np.uint32).reshape(-1, 2)
        received.append(kp)
        src_dst = kp if d == 0 else kp[:, ::-1]      # back to (src, dst) for the oracle
        g = O.new_grid(op)
        O.update(op, g, np.ascontiguousarray(src_dst))
        halves.append(g.reshape(2, -1)[d])
    grid = np.concatenate(halves)
    rep = O.close_window(op, grid)
    # the oracle on the pairs of this rank's keys, from the whole window
    ref_halves = []
    for d in range(2):
        sub = pairs[(pairs[:, d] & np.uint32(world - 1)) == rank]
        g = O.new_grid(op)
        O.update(op, g, sub)
        ref_halves.append(g.reshape(2, -1)[d])
    ref = O.close_window(op, np.concatenate(ref_halves))
    own = (rep["ip"] & np.uint32(world - 1)) == rank
    own_ref = (ref["ip"] & np.uint32(world - 1)) == rank
    hits = np.zeros(int(own.sum()), dtype=[("ip", "<u4"), ("dir", "<u4")])
    hits["ip"], hits["dir"] = rep["ip"][own], rep["dir"][own]
    assert np.array_equal(shard.own_hits(hits, rank, world), hits)
    gathered = [None] * world
    dist.all_gather_object(gathered, [(int(d), int(i)) for d, i in zip(rep["dir"][own], rep["ip"][own])])
    with open(out % rank, "w") as f:
        json.dump({"keys_owned": all(bool(np.all((kp[:, 0] & np.uint32(world - 1)) == rank)) for kp in received),
                   "grid_equal": bool(np.array_equal(grid, np.concatenate(ref_halves))),
                   "own_equal": bool(np.array_equal(rep["ip"][own], ref["ip"][own_ref]) and
                                     np.array_equal(rep["est"][own], ref["est"][own_ref])),
                   "union": sorted(set(tuple(x) for g in gathered for x in g)),
                   "received": int(sum(len(k) for k in received))}, f)
    dist.destroy_process_group()


def _spawn(fn, world, tmp_path):
    import torch.multiprocessing as mp
    port = 29600 + (os.getpid() % 500) + 7 * world
    out = str(tmp_path / f"{fn.__name__}_%d.json")
    mp.start_processes(fn, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    return [json.load(open(out % r)) for r in range(world)]


@pytest.mark.parametrize("world", [2, 4])
def test_or_merge_across_ranks_gives_the_whole_windows_report(O, tmp_path, world):
    res = _spawn(_or_rank, world, tmp_path)
    assert all(r["grid_equal"] and r["ips_equal"] and r["est_equal"] for r in res)
    assert res[0]["hits"] > 10


@pytest.mark.parametrize("world", [2, 4])
def test_key_partition_across_ranks(O, tmp_path, world):
    res = _spawn(_part_rank, world, tmp_path)
    w, pairs = _workload()
    assert all(r["keys_owned"] and r["grid_equal"] and r["own_equal"] for r in res)
    assert sum(r["received"] for r in res) == 2 * len(pairs)   # every pair, once per direction
    union = res[0]["union"]
    assert all(r["union"] == union for r in res) and len(union) > 10
    # the planted super points with at least 2 theta peers are found by their owners
    from paper_1803_11449_gb300 import traffic as T
    win = T.make_window(w, 404)
    found = {(d, ip) for d, ip in union}
    for ip, d, c in zip(win.planted_ip, win.planted_dir, win.planted_c):
        if c >= 2 * w.theta:
            assert (int(d), int(ip)) in found
