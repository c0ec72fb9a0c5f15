"""Autotuner for the update kernel's launch knobs (sd_tuning).

Each candidate setting is timed over the caller's own pair buffer as one
whole window -- the update, then the close -- starting from an empty DHLA
every time, and the fastest setting is applied to the handle.  The close is
in the timed region because the plane-binned mode (6) folds its plane-major
copy into the DHLA there; the rest of the close is the same for every
setting.
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
          for tp in (4096, 8192) for rd in (22, 24, 26) for un in (13, 14, 15, 16)]


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
    """Time every setting of the search space on `pairs_dev` (one window:
    sd_update, then sd_close_window, wall time after the stream is idle);
    apply and return the best as a dict with its knobs, "ms" and "table"."""
    import time

    import torch

    table = []
    for knobs in _space(modes, unrolls, threads, filters):
        try:
            sd.sd_set_tuning(h, **knobs)
        except sd.SdError:
            continue  # a setting this DHLA cannot take (e.g. a binning tile too large)
        times = []
        sd.sd_close_window(h)  # clears the DHLA: every trial starts from zero
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sd.sd_update(h, pairs_dev)
            sd.sd_close_window(h)
            times.append(1e3 * (time.perf_counter() - t0))
        ms = sorted(times)[len(times) // 2]
        table.append(dict(knobs, ms=ms))
        if verbose:
            print(table[-1], flush=True)
    sd.sd_close_window(h)
    best = min(table, key=lambda r: r["ms"])
    sd.sd_set_tuning(h, **{k: v for k, v in best.items() if k != "ms"})
    return dict(best, table=table)


BATCHED = ([dict(mode=5, bin_chunk_log2=ch, bin_batch_mib=mib, bin_tile_pairs=tp)
            for ch in (21, 22, 23, 24) for mib in (1024, 8192) for tp in (1024, 2048)] +
           [dict(mode=6, plane_round_log2=rd, bin_batch_mib=mib)
            for rd in (22, 24, 26) for mib in (1, 8192)])


def autotune_many(hs, pairs_list, stream, reps: int = 2, space=None, verbose: bool = False) -> dict:
    """Time sd_update_many then sd_close_many over the caller's links for
    every batched setting (mode 5: the driver hs[0]'s chunk, bins per round
    and tile; mode 6: its round and the bins of its lanes -- 1 MiB allows one
    lane), each trial from empty DHLAs; apply the best to every handle (the
    mode to all, the knobs to each) and return it as a dict with "ms" and
    "table"."""
    import time

    import torch

    table = []
    for knobs in (space or BATCHED):
        try:
            for h in hs:
                sd.sd_set_tuning(h, **knobs)
        except sd.SdError:
            continue
        times = []
        sd.sd_close_many(hs)
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sd.sd_update_many(hs, pairs_list)
            sd.sd_close_many(hs)
            times.append(1e3 * (time.perf_counter() - t0))
        table.append(dict(knobs, ms=min(times)))
        if verbose:
            print(table[-1], flush=True)
    best = min(table, key=lambda r: r["ms"])
    for h in hs:
        sd.sd_set_tuning(h, **{k: v for k, v in best.items() if k != "ms"})
    return dict(best, table=table)
