"""The autotuner's search spaces on CPU: every setting lies within the ranges
sd_set_tuning accepts (include/sd.h), so that a trial is skipped only for a
DHLA shape that cannot take it, never for a malformed setting, and the
default plane-mode knobs are among the single-window candidates."""
from paper_1803_11449_gb300 import tune


def _plane_ok(k):
    return (k.get("plane_tile_pairs", 8192) in (1024, 2048, 4096, 8192)
            and 10 <= k.get("plane_round_log2", 26) <= 28
            and 8 <= k.get("plane_unit_log2", 14) <= 24)


def test_single_window_space_is_within_the_accepted_ranges():
    space = list(tune._space(tune.MODES, tune.UNROLLS, tune.THREADS, tune.FILTERS))
    assert {k["mode"] for k in space} == set(tune.MODES)
    for k in space:
        if k["mode"] == 6:
            assert _plane_ok(k)
        elif k["mode"] == 5:
            assert 10 <= k["bin_slice_log2"] <= 15 and 12 <= k["bin_chunk_log2"] <= 28
            assert k["bin_tile_pairs"] & (k["bin_tile_pairs"] - 1) == 0 and 64 <= k["bin_tile_pairs"] <= 2048
        else:
            assert k["unroll"] in (1, 2, 4) and 64 <= k["block_threads"] <= 1024 and k["block_threads"] % 32 == 0
            assert 8 <= k["filter_log2"] <= 14
    defaults = dict(mode=6, plane_tile_pairs=8192, plane_round_log2=26, plane_unit_log2=14)
    assert any(all(k.get(f) == v for f, v in defaults.items()) for k in space)


def test_batched_space_covers_both_binned_modes():
    modes = {k["mode"] for k in tune.BATCHED}
    assert modes == {5, 6}
    for k in tune.BATCHED:
        assert k["bin_batch_mib"] >= 1
        if k["mode"] == 6:
            assert _plane_ok(k)
        else:
            assert 12 <= k["bin_chunk_log2"] <= 28
    # one lane (a budget below one round's bins) and the default lanes are both tried
    assert {k["bin_batch_mib"] for k in tune.BATCHED if k["mode"] == 6} == {1, 8192}
