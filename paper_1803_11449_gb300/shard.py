"""One detection window over several GPUs, one process per GPU.

Two ways to spread the work follow from the paper (see include/sd.h for the
device steps):

* Stream split, then merge (§4.2: local DHLAs merged into a global DHLA,
  read as a bitwise OR).  Each rank runs sd_update on its part of the
  window; ``merge_across`` then ORs the ranks' DHLAs so that every rank holds
  the DHLA of the whole window (``or_allreduce``: a reduce-scatter by
  all-to-all, whose parts the library ORs with sd_or_words, and an
  all-gather; no collective library offers a bitwise-OR reduction).  Any rank
  can then close the window and gets the report of the whole stream.
* Key partition (§5: hosts divided by the low bits of their address).  Each
  rank groups its pairs by the key of each direction (sd_partition_pairs)
  and ``exchange_by_key`` sends every group to the rank owning those keys
  (all-to-all); ``update_partitioned`` feeds the received pairs with
  sd_update_dir.  Each rank's DHLA holds its own keys only; ``own_hits``
  keeps the hits of those keys (others are estimator collisions).

The collectives go through ``torch.distributed`` (NCCL between GPUs).  The
device steps default to the library's kernels; the collective logic takes
them as arguments so that it can also run on CPU tensors over gloo.
"""
from __future__ import annotations

import numpy as np

from . import sd


def _or_parts_device(dst, src, words: int, count: int) -> None:
    import torch
    if not (dst.is_cuda and src.is_cuda):
        raise RuntimeError("or_allreduce: the default OR step runs on the GPU; pass or_parts for CPU tensors")
    sd.sd_or_words(dst, src, words, count, torch.cuda.current_stream())


def or_allreduce(words, group=None, or_parts=None):
    """Bitwise-OR all-reduce of a 1-D tensor of 32-bit DHLA words over the
    group: every rank gets the OR of all ranks' tensors.  Rank j receives
    part j of every rank's words (all-to-all), ORs them (``or_parts(dst,
    src, words, count)``: dst = OR of `count` arrays of `words` words laid
    end to end in src), and the ORed parts are all-gathered."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    if world == 1:
        return words
    or_parts = or_parts or _or_parts_device
    n = words.numel()
    part = -(-n // (4 * world)) * 4          # words per part, a multiple of 4
    padded = part * world
    send = words if n == padded else torch.cat([words, words.new_zeros(padded - n)])
    recv = torch.empty_like(send)
    dist.all_to_all_single(recv, send, group=group)
    mine = torch.empty(part, dtype=words.dtype, device=words.device)
    or_parts(mine, recv, part, world)
    full = torch.empty(padded, dtype=words.dtype, device=words.device)
    dist.all_gather_into_tensor(full, mine, group=group)
    return full[:n]


def merge_across(h, group=None):
    """OR the DHLAs of h on every rank of the group into each of them (§4.2
    merge): afterwards every rank's h holds the DHLA of the union of the
    ranks' streams.  Blocks until the merged DHLA is in h."""
    import torch
    p = h.params
    words = p.dirs * sd.sd_grid_words(p)
    image = torch.empty(words, dtype=torch.int32, device=f"cuda:{p.device}")
    sd.sd_export_grid(h, image)
    sd.sd_sync(h)
    merged = or_allreduce(image, group)
    torch.cuda.current_stream().synchronize()
    sd.sd_or_grid(h, merged)
    sd.sd_sync(h)


def _partition_device(h, direction: int, pairs, parts: int):
    import torch
    out = torch.empty_like(pairs)
    counts = sd.sd_partition_pairs(h, direction, pairs, parts, out)
    return out, counts


def exchange_by_key(pairs, direction: int, group=None, h=None, partition=None):
    """Send each of this rank's (src, dst) pairs to the rank that owns its key
    of `direction` (key & (world - 1), world a power of two) and return the
    (key, peer) pairs this rank owns, as a 1-D 32-bit tensor.  `partition(
    direction, pairs, parts) -> (grouped (key, peer) words, pairs per part)`
    defaults to sd_partition_pairs on h's device."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    if world & (world - 1):
        raise ValueError("exchange_by_key: the number of ranks must be a power of two")
    if partition is None:
        grouped, counts = _partition_device(h, direction, pairs, world)
    else:
        grouped, counts = partition(direction, pairs, world)
    dev = grouped.device
    send_counts = torch.as_tensor(np.asarray(counts, dtype=np.int64) * 2, device=dev)
    recv_counts = torch.empty_like(send_counts)
    dist.all_to_all_single(recv_counts, send_counts, group=group)
    rc = [int(x) for x in recv_counts.cpu()]
    sc = [int(x) for x in send_counts.cpu()]
    recv = torch.empty(sum(rc), dtype=grouped.dtype, device=dev)
    dist.all_to_all_single(recv, grouped, output_split_sizes=rc, input_split_sizes=sc, group=group)
    return recv


def update_partitioned(h, pairs, group=None):
    """Key-partitioned Algorithm 1: for each direction, this rank's pairs go
    to the ranks owning their keys and the pairs of this rank's keys are fed
    to h with sd_update_dir."""
    for d in range(h.params.dirs):
        mine = exchange_by_key(pairs, d, group, h=h)
        sd.sd_update_dir(h, d, mine)


def own_hits(hits, rank: int, world: int):
    """The hits of a key-partitioned rank's own keys (ip & (world - 1) ==
    rank): a rank's DHLA has the full counts of those keys only."""
    return hits[(hits["ip"] & np.uint32(world - 1)) == np.uint32(rank)]
