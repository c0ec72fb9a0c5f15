"""Autotuner for the update kernel's launch knobs (sd_tuning).

Each candidate setting is timed with CUDA events on the handle's stream over
the caller's own pair buffer, starting from an empty DHLA every time (a
window close clears it), and the fastest setting is applied to the handle.
"""
from __future__ import annotations

import itertools

from . import sd

MODES = (0, 1, 2, 3, 4, 5, 6)
UNROLLS = (1, 2, 4)
THREADS = (256, 512, 1024)
FILTERS = (12, 13, 14)   # log2 entries of the shared-memory filter (modes 3, 4)


BINNED = [dict(bin_slice_log2=sl, bin_tile_pairs=tp, bin_chunk_log2=ch, bin_slack_pct=100)
          for sl in (13, 14, 15) for tp in (512, 1024, 2048) for ch in (21, 22, 23, 24)]

PLANES = [dict(plane_tile_pairs=tp, plane_round_log2=rd, plane_unit_log2=un)
          for tp in (1024, 2048, 4096) for rd in (21, 22, 23, 24) for un in (13, 14, 15, 16)]


def _space(modes, unrolls, threads, filters):
    for mode in modes:
        if mode == 5:
            for b in BINNED:
                yield dict(mode=5, **b)
            continue
        if mode == 6:
            for b in PLANES:
                yield dict(mode=6, **b)
            continue
        for unroll, nthr in itertools.product(unrolls, threads):
            for flog in (filters if mode >= 3 else (13,)):
                yield dict(mode=mode, unroll=unroll, block_threads=nthr, filter_log2=flog)


def autotune(h, pairs_dev, stream, reps: int = 3, modes=MODES, unrolls=UNROLLS, threads=THREADS,
             filters=FILTERS, verbose: bool = False) -> dict:
    """Time every setting of the search space on `pairs_dev`; apply and
    return the best as a dict with its knobs, "ms" and "table"."""
    import torch

    table = []
    for knobs in _space(modes, unrolls, threads, filters):
        try:
            sd.sd_set_tuning(h, **knobs)
        except sd.SdError:
            continue  # a setting this DHLA cannot take (e.g. a binning tile too large)
        times = []
        for _ in range(reps):
            sd.sd_close_window(h)  # clears the DHLA: every trial starts from zero
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sd.sd_update(h, pairs_dev)
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
        ms = sorted(times)[len(times) // 2]
        table.append(dict(knobs, ms=ms))
        if verbose:
            print(table[-1], flush=True)
    sd.sd_close_window(h)
    best = min(table, key=lambda r: r["ms"])
    sd.sd_set_tuning(h, **{k: v for k, v in best.items() if k != "ms"})
    return dict(best, table=table)


BATCHED = [dict(bin_chunk_log2=ch, bin_batch_mib=mib, bin_tile_pairs=tp)
           for ch in (20, 21, 22, 23, 24) for mib in (1024, 4096, 8192) for tp in (1024, 2048)]


def autotune_many(hs, pairs_list, stream, reps: int = 2, space=None, verbose: bool = False) -> dict:
    """Time sd_update_many over the caller's links for every batched-update
    setting (the driver hs[0]'s chunk, bins per round and tile), each trial
    from empty DHLAs (sd_close_many clears them); apply the best to every
    handle and return it as a dict with "ms" and "table"."""
    import torch

    table = []
    for knobs in (space or BATCHED):
        try:
            for h in hs:
                sd.sd_set_tuning(h, mode=5, **knobs)
        except sd.SdError:
            continue
        times = []
        for _ in range(reps):
            sd.sd_close_many(hs)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sd.sd_update_many(hs, pairs_list)
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
        table.append(dict(knobs, ms=min(times)))
        if verbose:
            print(table[-1], flush=True)
    sd.sd_close_many(hs)
    best = min(table, key=lambda r: r["ms"])
    for h in hs:
        sd.sd_set_tuning(h, mode=5, **{k: v for k, v in best.items() if k != "ms"})
    return dict(best, table=table)
