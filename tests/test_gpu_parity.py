"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer results (DHLA bits, ZR, hot sets, |K|, K, reported addresses, SZ)
must be identical; psi and the Eq. 4 estimates are evaluated from identical
integers by the same double formulas on the host and must be bit-identical
too.  Inputs come from the seeded traffic generator only.
"""
import numpy as np
import pytest

from paper_1803_11449_gb300 import traffic as T

pytestmark = pytest.mark.gpu

SEED = 0x5EED5EED


@pytest.fixture(scope="module")
def sd():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1803_11449_gb300 import build as b
    b.build()
    from paper_1803_11449_gb300 import sd as mod
    mod.lib()
    return mod


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    return torch


def _oracle_run(O, w, pairs, seed, **caps):
    op = O.params_from(w.sketch(), seed=seed, **caps)
    og = O.new_grid(op)
    O.update(op, og, pairs)
    ref = O.close_window(op, og, want_cands=True)
    return op, og, ref


def _dev(torch_mod, pairs):
    return torch_mod.from_numpy(np.ascontiguousarray(pairs).reshape(-1).view(np.int32)).cuda()


def _grids(sd, h):
    return np.concatenate([sd.sd_get_grid(h, d) for d in range(h.params.dirs)])


def _assert_report_equal(O, rep, ref, p):
    assert rep.n_cand == ref["n_cand"]
    assert [rep.dir_flags(d) for d in range(p.dirs)] == ref["flags"]
    assert np.array_equal(rep.zr, ref["zr"])
    assert np.array_equal(rep.n_hot, ref["n_hot"])
    assert rep.psi == ref["psi"]
    assert rep.n_hits_total == ref["n_hits"]
    assert np.array_equal(rep.hits["dir"], ref["dir"])
    assert np.array_equal(rep.hits["ip"], ref["ip"])
    assert np.array_equal(rep.hits["sz"], ref["sz"])
    assert np.array_equal(rep.hits["est"], ref["est"])   # bit-exact doubles


def _full_check(sd, O, torch_mod, w, win, seed=SEED, tuning=None, **caps):
    p = sd.params_for(w, seed, cuda_stream=torch_mod.cuda.current_stream().cuda_stream, **caps)
    h = sd.sd_create(p)
    try:
        if tuning:
            sd.sd_set_tuning(h, **tuning)
        sd.sd_update(h, _dev(torch_mod, win.pairs))
        grid = _grids(sd, h)
        rep = sd.sd_close_window(h)
        hot = [[sd.sd_get_hot(h, d, i) for i in range(p.r)] for d in range(p.dirs)]
        cands = [sd.sd_get_candidates(h, d) for d in range(p.dirs)]
        after = _grids(sd, h)
    finally:
        sd.sd_destroy(h)
    op, og, ref = _oracle_run(O, w, win.pairs, seed, **caps)
    assert np.array_equal(grid, og), "DHLA bits differ"
    assert not after.any(), "DHLA not cleared by the close"
    _assert_report_equal(O, rep, ref, p)
    for d in range(p.dirs):
        z0, _ = O.row_stats(op, og, d)
        he, nhe = O.hot_sets(op, z0)
        for i in range(p.r):
            assert np.array_equal(np.flatnonzero(hot[d][i]), he[i, :nhe[i]])
        if ref["flags"][d] == 0:
            nk, ks = cands[d]
            assert nk == ref["n_cand"][d]
            assert np.array_equal(np.sort(ks), ref["cands"][d])
    return rep, ref


def test_tiny_window_full_parity(sd, O, torch_mod):
    w = T.WORKLOADS["tiny"]
    rep, ref = _full_check(sd, O, torch_mod, w, T.make_window(w, T.window_seed(1)))
    assert ref["n_hits"] > 20


@pytest.mark.parametrize("mode,unroll,threads,flog", [
    (0, 1, 256, 13), (0, 4, 1024, 13), (1, 2, 512, 13), (2, 2, 512, 13), (2, 4, 256, 13),
    (1, 1, 128, 13), (3, 2, 512, 13), (3, 1, 1024, 14), (3, 4, 256, 8), (4, 2, 512, 12),
    (4, 1, 64, 8), (5, 2, 512, 13), (6, 2, 512, 13)])
def test_update_variants_give_identical_grids(sd, O, torch_mod, mode, unroll, threads, flog):
    w = T.WORKLOADS["tiny"].with_(dirs=2, n=(1 << 19) + 3)
    win = T.make_window(w, 8)
    _full_check(sd, O, torch_mod, w, win,
                tuning=dict(mode=mode, unroll=unroll, block_threads=threads, filter_log2=flog))


def test_filter_modes_on_heavy_hitters(sd, O, torch_mod):
    """A few hosts carry most of the traffic, so the shared-memory filter of
    modes 3 and 4 is hit constantly and blocks see bits others have set; in
    the binned mode 5 a few slices get most bit-sets and their bins overflow
    into the atomic fallback."""
    w = T.WORKLOADS["core"].with_(n=1 << 21, src_pool=64, zipf_s=1.3, dst_pool=1 << 12,
                                  planted=4, planted_c=("uniform", 3000, 5000))
    win = T.make_window(w, 19)
    for tuning in (dict(mode=3, filter_log2=10), dict(mode=4, filter_log2=10),
                   dict(mode=5, bin_chunk_log2=19, bin_slack_pct=0xFFFFFFFF),
                   dict(mode=5, bin_chunk_log2=21, bin_slack_pct=400),
                   dict(mode=6, plane_round_log2=19, plane_unit_log2=10),
                   dict(mode=6, plane_round_log2=21, plane_unit_log2=20, plane_tile_pairs=1024)):
        _full_check(sd, O, torch_mod, w, win, tuning=tuning)


@pytest.mark.parametrize("slice_log2,tile,chunk_log2,slack", [
    (14, 1024, 23, 100), (10, 256, 16, 0xFFFFFFFF), (15, 512, 18, 50), (12, 64, 12, 10),
    (13, 2048, 20, 100)])
def test_binned_update_variants(sd, O, torch_mod, slice_log2, tile, chunk_log2, slack):
    """Mode 5 with slices, tiles, rounds and bin slack from tiny (many rounds,
    overflowing bins) to large; ragged pair count."""
    w = T.WORKLOADS["tiny"].with_(dirs=2, n=(1 << 19) + 5)
    win = T.make_window(w, 23)
    _full_check(sd, O, torch_mod, w, win,
                tuning=dict(mode=5, bin_slice_log2=slice_log2, bin_tile_pairs=tile,
                            bin_chunk_log2=chunk_log2, bin_slack_pct=slack))


@pytest.mark.parametrize("tile,round_log2,unit_log2", [
    (4096, 22, 15), (1024, 10, 8), (2048, 16, 12), (4096, 13, 24), (1024, 18, 9)])
@pytest.mark.parametrize("dirs", [1, 2])
def test_plane_update_variants(sd, O, torch_mod, tile, round_log2, unit_log2, dirs):
    """Mode 6 (binned by estimator bit) with tiles, rounds and apply units
    from tiny (many rounds of one partial tile; apply units of 256 keys, so
    a plane's bin is split over many blocks) to one round; ragged pair
    count."""
    w = T.WORKLOADS["tiny"].with_(dirs=dirs, n=(1 << 19) + 5)
    win = T.make_window(w, 23)
    _full_check(sd, O, torch_mod, w, win,
                tuning=dict(mode=6, plane_tile_pairs=tile, plane_round_log2=round_log2,
                            plane_unit_log2=unit_log2))


@pytest.mark.parametrize("read_before_close", [True, False])
def test_plane_update_keeps_bits_across_calls_and_modes(sd, O, torch_mod, read_before_close):
    """The DHLA of a handle in mode 6 is its DHLA plus the pending planes:
    updates of several calls, a switch to another mode in mid-window, a
    checkpoint read (which folds the planes) and more mode-6 updates all
    end in Algorithm 1's DHLA of the whole stream.  Without a read right
    before the close, the close's fold (which also computes the row
    statistics) merges pending planes into a DHLA that already holds bits."""
    w = T.WORKLOADS["tiny"].with_(dirs=2)
    win = T.make_window(w, 71)
    parts = np.array_split(win.pairs, 5)
    p = sd.params_for(w, SEED, cuda_stream=torch_mod.cuda.current_stream().cuda_stream)
    h = sd.sd_create(p)
    try:
        assert sd.sd_get_tuning(h).mode == 6
        sd.sd_update(h, _dev(torch_mod, parts[0]))
        sd.sd_update(h, _dev(torch_mod, parts[1]))
        sd.sd_set_tuning(h, mode=5)
        sd.sd_update(h, _dev(torch_mod, parts[2]))
        mid = _grids(sd, h)
        sd.sd_set_tuning(h, mode=6)
        sd.sd_update(h, _dev(torch_mod, parts[3]))
        sd.sd_set_tuning(h, mode=1)
        sd.sd_update(h, _dev(torch_mod, parts[4]))
        sd.sd_set_tuning(h, mode=6)
        if not read_before_close:
            sd.sd_update(h, _dev(torch_mod, parts[4]))  # pending planes again (the same pairs: no new bits)
        grid = _grids(sd, h) if read_before_close else None
        rep = sd.sd_close_window(h)
        after = _grids(sd, h)
    finally:
        sd.sd_destroy(h)
    op = O.params_from(w.sketch(), seed=SEED)
    og = O.new_grid(op)
    O.update(op, og, np.concatenate(parts[:3]))
    assert np.array_equal(mid, og)
    _, og, ref = _oracle_run(O, w, win.pairs, SEED)
    assert (grid is None or np.array_equal(grid, og)) and not after.any()
    _assert_report_equal(O, rep, ref, p)


def test_plane_bins_follow_shifting_traffic(sd, O, torch_mod):
    """Mode 6 lays out each round's bins from the previous round's counts.
    Traffic that changes between rounds overflows them: rounds of uniform
    pairs, then a flood to one destination from distinct sources (all its
    outbound keys fall in one plane), then uniform pairs again (planes the
    flood left nearly empty get many keys).  Keys beyond a bin's room set
    their bits directly; the DHLA and the report still equal the oracle's."""
    w = T.WORKLOADS["core"].with_(n=3 << 18)
    rng = np.random.default_rng(5)
    uni = rng.integers(0, 2**32, size=(1 << 18, 2), dtype=np.uint64).astype(np.uint32)
    flood = np.empty((1 << 18, 2), np.uint32)
    flood[:, 0] = T.mix32(np.arange(1 << 18, dtype=np.uint32) + np.uint32(7))
    flood[:, 1] = 0xC0A80101
    uni2 = rng.integers(0, 2**32, size=(1 << 18, 2), dtype=np.uint64).astype(np.uint32)
    pairs = np.concatenate([uni, flood, uni2])
    win = _window_of(w, pairs)
    rep, ref = _full_check(sd, O, torch_mod, w, win,
                           tuning=dict(mode=6, plane_round_log2=15, plane_unit_log2=12))
    hit = rep.hits[(rep.hits["ip"] == 0xC0A80101) & (rep.hits["dir"] == 1)]
    assert len(hit) == 1


@pytest.mark.parametrize("mode", [1, 3, 5, 6])
def test_ragged_and_misaligned_inputs(sd, O, torch_mod, mode):
    """Odd pair counts and buffers starting 8 or 4 bytes past a 16-byte
    boundary take the head/tail and unaligned paths."""
    w = T.WORKLOADS["tiny"].with_(dirs=2)
    win = T.make_window(w, 21)
    n = len(win.pairs)
    flat = _dev(torch_mod, win.pairs)
    op = O.params_from(w.sketch(), seed=SEED)
    for off_words, count in ((0, n - 7), (2, n - 2), (1, 5), (2, 1), (0, 1), (3, 999)):
        p = sd.params_for(w, SEED, cuda_stream=torch_mod.cuda.current_stream().cuda_stream)
        h = sd.sd_create(p)
        sd.sd_set_tuning(h, mode=mode, bin_chunk_log2=16)
        try:
            if off_words % 2 == 0:
                view = flat[off_words: off_words + 2 * count]
                sd.sd_update(h, view)
                sub = win.pairs[off_words // 2: off_words // 2 + count]
            else:
                # a buffer whose pairs start on an odd word
                buf = torch_mod.zeros(2 * count + 1, dtype=torch_mod.int32, device="cuda")
                buf[1:] = flat[: 2 * count]
                sd.sd_update(h, buf[1:])
                sub = win.pairs[:count]
            grid = _grids(sd, h)
        finally:
            sd.sd_destroy(h)
        og = O.new_grid(op)
        O.update(op, og, sub)
        assert np.array_equal(grid, og), (off_words, count)


def test_empty_window_and_split_updates(sd, O, torch_mod):
    w = T.WORKLOADS["tiny"]
    win = T.make_window(w, 5)
    p = sd.params_for(w, SEED, cuda_stream=torch_mod.cuda.current_stream().cuda_stream)
    h = sd.sd_create(p)
    try:
        rep0 = sd.sd_close_window(h)        # nothing fed: no hot estimators, no hits
        assert rep0.n_hits_total == 0 and rep0.n_cand == [0] and rep0.flags == 0
        assert rep0.psi == [0.0]
        sd.sd_update(h, np.zeros(0, dtype=np.uint32))
        dev = _dev(torch_mod, win.pairs)
        for part in torch_mod.tensor_split(dev, 9):
            if part.numel() % 2:
                continue
            sd.sd_update(h, part)
        # tensor_split may cut a pair; feed the whole stream again (idempotent)
        sd.sd_update(h, dev)
        grid = sd.sd_get_grid(h, 0)
        rep = sd.sd_close_window(h)
    finally:
        sd.sd_destroy(h)
    op, og, ref = _oracle_run(O, w, win.pairs, SEED)
    assert np.array_equal(grid, og)
    _assert_report_equal(O, rep, ref, p)


@pytest.mark.parametrize("pinned", [False, True])
def test_host_pointer_ingest(sd, O, torch_mod, pinned):
    """Host buffers (pageable or pinned) go through the chunked staging path;
    small chunks force many double-buffered copies."""
    w = T.WORKLOADS["tiny"].with_(dirs=2)
    win = T.make_window(w, 6)
    p = sd.params_for(w, SEED, stage_pairs=40_000,
                      cuda_stream=torch_mod.cuda.current_stream().cuda_stream)
    h = sd.sd_create(p)
    try:
        if pinned:
            host = torch_mod.from_numpy(win.pairs.reshape(-1).view(np.int32)).pin_memory()
            sd.sd_update(h, host)
        else:
            sd.sd_update(h, win.pairs.reshape(-1))
        grid = _grids(sd, h)
        rep = sd.sd_close_window(h)
    finally:
        sd.sd_destroy(h)
    op, og, ref = _oracle_run(O, w, win.pairs, SEED)
    assert np.array_equal(grid, og)
    _assert_report_equal(O, rep, ref, p)


def _small_core(**kw):
    base = dict(n=1 << 22, planted=40, planted_c=("loguniform", 1024, 20000), src_pool=1 << 20,
                dst_pool=1 << 22)
    base.update(kw)
    return base


@pytest.mark.parametrize("name", ["core", "paper"])
def test_core_and_paper_parameters_small_window(sd, O, torch_mod, name):
    w = T.WORKLOADS[name].with_(**_small_core())
    _full_check(sd, O, torch_mod, w, T.make_window(w, 99))


@pytest.mark.parametrize("mode", [None, 1, 5, 6])
def test_core_link_window_full_size(sd, O, torch_mod, mode):
    """The benchmarked workload itself: 2^26 pairs, g=512, r=4, k=16, both
    directions; the default launch configuration and the update modes the
    benchmark may pick."""
    w = T.WORKLOADS["core"]
    win = _core_window()
    rep, ref = _full_check(sd, O, torch_mod, w, win, tuning=None if mode is None else dict(mode=mode))
    assert rep.n_hits_total > 500


def test_stress_sketch_beyond_l2(sd, O, torch_mod):
    """The stress sketch (g=1024, r=4, k=18, alpha=7: 2 x 128 MiB, larger than
    L2; 2048 binning slices) on 2^25 pairs of stress-shaped traffic (flows of
    8 packets), in the benchmark's launch configuration (binned, 2^24-pair
    rounds) and with a round that ends mid-window."""
    w = T.WORKLOADS["stress"]
    win = T.make_window(w, T.window_seed(5), n=(1 << 25) + 12345)
    rep, ref = _full_check(sd, O, torch_mod, w, win)
    assert rep.n_hits_total > 100 and ref["flags"] == [0, 0]


@pytest.mark.parametrize("g,r,k,alpha,theta,n,pool,planted,c", [
    (32, 8, 8, 4, 40, 6000, 1 << 10, 2, (120, 200)),       # one word per estimator, the most rows,
                                                           # 256 estimators, 2^16 preimages per (c0, c1)
    (64, 6, 10, 6, 80, 40_000, 1 << 12, 3, (250, 400)),
    (32, 8, 8, 6, 40, 6000, 1 << 10, 2, (120, 200)),       # the last block starts at bit 36 (empty)
    (4096, 3, 16, 16, 1024, 1 << 18, 1 << 15, 6, (3072, 6144)),  # 128 words per estimator, blocks
                                                                 # that do not overlap
    (32, 3, 24, 8, 40, 1 << 18, 1 << 16, 6, (120, 240)),   # 2^24 estimators: 3 x 64 MiB per direction,
                                                           # hot row 2 too large for shared memory
])
def test_edge_sketch_shapes(sd, O, torch_mod, g, r, k, alpha, theta, n, pool, planted, c):
    """The extremes of the parameter space (g = 32 and 4096, r = 3 and 8,
    k = 8 and 24) on both directions, in the default launch configuration."""
    w = T.WORKLOADS["tiny"].with_(g=g, r=r, k=k, alpha=alpha, theta=theta, dirs=2, n=n, src_pool=pool,
                                  dst_pool=pool, planted=planted, planted_c=("uniform",) + c)
    win = T.make_window(w, 61)
    rep, ref = _full_check(sd, O, torch_mod, w, win)
    assert ref["flags"] == [0, 0] and rep.n_hits_total > 0


def _window_of(w, pairs):
    return T.Window(pairs=np.ascontiguousarray(pairs, dtype=np.uint32), planted_ip=np.zeros(0, np.uint32),
                    planted_dir=np.zeros(0, np.uint8), planted_c=np.zeros(0, np.int64), workload=w, seed=0)


def test_degenerate_windows(sd, O, torch_mod):
    """One pair repeated 2^20 times (every bit-set of the window lands in the
    same 8 words: the bins overflow into the atomic fallback), and one source
    with 2^20 distinct destinations (its estimators fill completely: SZ = 0,
    an infinite Eq. 4 estimate, reported by both sides)."""
    w = T.WORKLOADS["core"].with_(n=1 << 20)
    same = np.tile(np.array([[0x0A000001, 0xC0A80001]], np.uint32), (1 << 20, 1))
    rep, ref = _full_check(sd, O, torch_mod, w, _window_of(w, same))
    assert rep.n_hits_total == 0
    one = np.empty((1 << 20, 2), np.uint32)
    one[:, 0] = 0x0A000002
    one[:, 1] = T.mix32(np.arange(1 << 20, dtype=np.uint32))
    rep, ref = _full_check(sd, O, torch_mod, w, _window_of(w, one))
    hit = rep.hits[(rep.hits["ip"] == 0x0A000002) & (rep.hits["dir"] == 0)]
    assert len(hit) == 1 and hit["sz"][0] == 0 and np.isinf(hit["est"][0])


_CORE = {}


def _core_window():
    if "win" not in _CORE:
        _CORE["win"] = T.make_window(T.WORKLOADS["core"], T.window_seed(2))
    return _CORE["win"]


def test_paper_parameter_full_window_overloads_quickly(sd, O, torch_mod):
    """The paper's own sketch (g=1024, r=5, k=14, alpha=6: 10 MiB per
    direction) on the full 2^26-pair core-link window: it saturates, most
    estimators are hot and |K| is far above cand_cap.  Both sides flag the
    overload the same way (|K| reported as cand_cap + 1), and the close
    stops once K passes its capacity instead of enumerating ~10^9
    candidates: under 5 ms."""
    import time
    w = T.WORKLOADS["paper"]
    win = _core_window()   # the same traffic recipe and seed as the core window
    p = sd.params_for(w, SEED, cuda_stream=torch_mod.cuda.current_stream().cuda_stream)
    dev = _dev(torch_mod, win.pairs)
    h = sd.sd_create(p)
    try:
        sd.sd_update(h, dev)
        grid = _grids(sd, h)
        rep = sd.sd_close_window(h)
        times = []
        for _ in range(3):    # the same window again, timed without first-use allocations
            sd.sd_update(h, dev)
            sd.sd_sync(h)
            t0 = time.perf_counter()
            again = sd.sd_close_window(h)
            times.append(time.perf_counter() - t0)
            assert again.flags == rep.flags and again.n_cand == rep.n_cand
    finally:
        sd.sd_destroy(h)
    op, og, ref = _oracle_run(O, w, win.pairs, SEED)
    assert np.array_equal(grid, og), "DHLA bits differ"
    _assert_report_equal(O, rep, ref, p)
    assert all(f & O.FLAG_OVERLOAD_CANDS for f in ref["flags"])
    assert rep.n_cand == [(p.cand_cap or (1 << 20)) + 1] * 2 and rep.rc == sd.SD_ERR_OVERLOAD
    assert min(times) < 5e-3, times


def test_saturated_row(sd, O, torch_mod):
    w = T.WORKLOADS["tiny"]
    win = T.make_window(w, 3)
    p = sd.params_for(w, SEED, cuda_stream=torch_mod.cuda.current_stream().cuda_stream)
    op = O.params_from(w.sketch(), seed=SEED)
    og = O.new_grid(op)
    O.update(op, og, win.pairs)
    rw = og.size // p.r
    og[2 * rw: 3 * rw] = 0xFFFFFFFF          # row 2 completely set
    h = sd.sd_create(p)
    try:
        sd.sd_set_grid(h, 0, og)
        rep = sd.sd_close_window(h)
    finally:
        sd.sd_destroy(h)
    ref = O.close_window(op, og)
    assert rep.rc == sd.SD_ERR_SATURATED
    assert rep.dir_flags(0) == sd.SD_FLAG_SATURATED == ref["flags"][0]
    assert rep.psi[0] == -1.0 and rep.n_hits_total == 0
    assert np.array_equal(rep.zr, ref["zr"])


def test_overload_caps(sd, O, torch_mod):
    """Each cap on each side of its boundary: the work bound |HE(0)| 2^(32-k)
    against pair_cap, and |K| against cand_cap (an overloaded |K| is
    reported as cand_cap + 1 by both sides)."""
    w = T.WORKLOADS["tiny"]
    win = T.make_window(w, T.window_seed(1))
    _, _, full = _oracle_run(O, w, win.pairs, SEED)
    work = int(full["n_hot"][0][0]) << (32 - w.k)
    nk = full["n_cand"][0]
    for caps in (dict(pair_cap=work - 1), dict(pair_cap=work), dict(cand_cap=nk - 1), dict(cand_cap=nk),
                 dict(cand_cap=nk // 5)):
        rep, ref = _full_check(sd, O, torch_mod, w, win, **caps)
        if ref["flags"][0]:
            assert rep.rc == sd.SD_ERR_OVERLOAD and rep.n_hits_total == 0
        if "cand_cap" in caps and caps["cand_cap"] < nk:
            assert rep.n_cand[0] == caps["cand_cap"] + 1


def test_report_cap_truncates_in_order(sd, O, torch_mod):
    w = T.WORKLOADS["tiny"]
    win = T.make_window(w, T.window_seed(1))
    p = sd.params_for(w, SEED, report_cap=17, cuda_stream=torch_mod.cuda.current_stream().cuda_stream)
    h = sd.sd_create(p)
    try:
        sd.sd_update(h, _dev(torch_mod, win.pairs))
        rep = sd.sd_close_window(h)
    finally:
        sd.sd_destroy(h)
    _, _, ref = _oracle_run(O, w, win.pairs, SEED)
    assert rep.rc == sd.SD_ERR_REPORT_OVERFLOW
    assert rep.n_hits_total == ref["n_hits"] and len(rep.hits) == 17
    assert np.array_equal(rep.hits["ip"], ref["ip"][:17])
    assert np.array_equal(rep.hits["est"], ref["est"][:17])


@pytest.mark.parametrize("p_full,least", [(0.0465, 8192), (0.066, 65536), (0.11, 1 << 19)])
def test_many_hits_take_the_multi_block_sort(sd, O, torch_mod, p_full, least):
    """A DHLA where a fraction p of the estimators of each row are full: |K|
    is about p^4 2^32, every candidate has SZ = 0 and is reported, and more
    than one block sorts: up to 2^19 hits by the sample sort (buckets split
    at sampled keys, each sorted by one block), more by sorted segments
    merged in pairwise passes."""
    w = T.WORKLOADS["core"].with_(dirs=1, g=256)
    rng = np.random.default_rng(12)
    cells = rng.random((w.r, 1 << w.k)) < p_full
    grid = np.zeros((w.r, 1 << w.k, w.g // 32), dtype=np.uint32)
    grid[cells] = 0xFFFFFFFF
    grid[~cells, 0] = 1   # every other estimator keeps g-1 zero bits
    grid = grid.reshape(-1)
    cap = 1 << 17 if least < (1 << 19) else 1 << 20
    p = sd.params_for(w, SEED, cand_cap=cap,
                      cuda_stream=torch_mod.cuda.current_stream().cuda_stream)
    h = sd.sd_create(p)
    try:
        sd.sd_set_grid(h, 0, grid)
        rep = sd.sd_close_window(h)
    finally:
        sd.sd_destroy(h)
    op = O.params_from(w.sketch(), seed=SEED, cand_cap=cap)
    ref = O.close_window(op, grid)
    assert ref["n_hits"] > least
    _assert_report_equal(O, rep, ref, p)


def test_checkpoint_resume(sd, O, torch_mod):
    """Snapshot the DHLA mid-window, restore it in a fresh handle, finish the
    window there: same report as an uninterrupted run."""
    w = T.WORKLOADS["tiny"].with_(dirs=2)
    win = T.make_window(w, 31)
    half = len(win.pairs) // 2
    stream = torch_mod.cuda.current_stream().cuda_stream
    p = sd.params_for(w, SEED, cuda_stream=stream)
    a = sd.sd_create(p)
    b = sd.sd_create(p)
    try:
        sd.sd_update(a, _dev(torch_mod, win.pairs[:half]))
        snap = [sd.sd_get_grid(a, d) for d in range(2)]
        for d in range(2):
            sd.sd_set_grid(b, d, snap[d])
        sd.sd_update(b, _dev(torch_mod, win.pairs[half:]))
        rep = sd.sd_close_window(b)
    finally:
        sd.sd_destroy(a)
        sd.sd_destroy(b)
    _, _, ref = _oracle_run(O, w, win.pairs, SEED)
    _assert_report_equal(O, rep, ref, p)


def test_merge_of_monitors_equals_union(sd, O, torch_mod):
    """§4.2 merge of local DHLAs (read as bitwise OR): three monitors each see
    part of the traffic; the merged DHLA reports what one monitor seeing all
    of it would."""
    w = T.WORKLOADS["tiny"].with_(dirs=2)
    win = T.make_window(w, 41)
    parts = np.array_split(win.pairs, 3)
    stream = torch_mod.cuda.current_stream().cuda_stream
    p = sd.params_for(w, SEED, cuda_stream=stream)
    hs = [sd.sd_create(p) for _ in parts]
    try:
        for h, part in zip(hs, parts):
            sd.sd_update(h, _dev(torch_mod, part))
        sd.sd_merge(hs[0], hs[1])
        sd.sd_merge(hs[0], hs[2])
        grid = _grids(sd, hs[0])
        rep = sd.sd_close_window(hs[0])
    finally:
        for h in hs:
            sd.sd_destroy(h)
    _, og, ref = _oracle_run(O, w, win.pairs, SEED)
    assert np.array_equal(grid, og)
    _assert_report_equal(O, rep, ref, p)


def test_consecutive_windows_are_independent(sd, O, torch_mod):
    w = T.WORKLOADS["tiny"].with_(dirs=2)
    wins = [T.make_window(w, s) for s in (51, 52, 53)]
    p = sd.params_for(w, SEED, cuda_stream=torch_mod.cuda.current_stream().cuda_stream)
    h = sd.sd_create(p)
    try:
        reps = []
        for win in wins:
            sd.sd_update(h, _dev(torch_mod, win.pairs))
            reps.append(sd.sd_close_window(h))
    finally:
        sd.sd_destroy(h)
    for win, rep in zip(wins, reps):
        _, _, ref = _oracle_run(O, w, win.pairs, SEED)
        _assert_report_equal(O, rep, ref, p)
        assert rep.n_pairs == len(win.pairs)
