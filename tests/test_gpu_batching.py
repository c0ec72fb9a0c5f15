"""Batched windows of many links (sd_update_many, sd_close_many): every
link's DHLA and report must be exactly what the oracle gives for that link
alone, and exactly what the one-window-at-a-time path gives."""
import numpy as np
import pytest

from paper_1803_11449_gb300 import traffic as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sd():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1803_11449_gb300 import build as b
    b.build()
    from paper_1803_11449_gb300 import sd as mod
    mod.lib()
    return mod


def _dev(pairs):
    import torch
    return torch.from_numpy(np.ascontiguousarray(pairs).reshape(-1).view(np.int32)).cuda()


def _oracle(O, w, pairs, seed):
    op = O.params_from(w.sketch(), seed=seed)
    og = O.new_grid(op)
    O.update(op, og, pairs)
    return og, O.close_window(op, og)


def _same_report(rep, ref, dirs):
    assert rep.n_cand == ref["n_cand"]
    assert [rep.dir_flags(d) for d in range(dirs)] == ref["flags"]
    assert np.array_equal(rep.zr, ref["zr"]) and rep.psi == ref["psi"]
    assert np.array_equal(rep.hits["ip"], ref["ip"]) and np.array_equal(rep.hits["sz"], ref["sz"])
    assert np.array_equal(rep.hits["dir"], ref["dir"])
    assert np.array_equal(rep.hits["est"], ref["est"])


@pytest.mark.parametrize("tuning", [dict(mode=5), dict(mode=5, bin_chunk_log2=17), dict(mode=1),
                                    dict(mode=5, bin_batch_mib=1), dict(mode=5, bin_chunk_log2=14, bin_batch_mib=4),
                                    dict(mode=6), dict(mode=6, plane_round_log2=14),
                                    dict(mode=6, plane_round_log2=16, plane_tile_pairs=1024),
                                    dict(mode=6, bin_batch_mib=1)])
def test_batched_links_equal_each_link_alone(sd, O, tuning):
    """Seven links of uneven sizes (one of them much larger than a round's
    share), each with its own traffic and its own hash seed."""
    w = T.WORKLOADS["tiny"].with_(dirs=2)
    sizes = [1 << 14, 3 + (1 << 16), 200_001, 1 << 12, 1 << 19, 77_777, 5]
    seeds = [1000 + i for i in range(len(sizes))]
    wins = [T.make_window(w.with_(n=max(n, 64), planted=4 if n > 1000 else 0), s, n=n)
            for n, s in zip(sizes, seeds)]
    hs = [sd.sd_create(sd.params_for(w, s)) for s in seeds]
    try:
        for h in hs:
            sd.sd_set_tuning(h, **tuning)
        devs = [_dev(win.pairs) for win in wins]
        sd.sd_update_many(hs, devs)
        grids = [np.concatenate([sd.sd_get_grid(h, d) for d in range(2)]) for h in hs]
        reps = sd.sd_close_many(hs)
    finally:
        for h in hs:
            sd.sd_destroy(h)
    for win, s, g, rep in zip(wins, seeds, grids, reps):
        og, ref = _oracle(O, w, win.pairs, s)
        assert np.array_equal(g, og)
        _same_report(rep, ref, 2)
        assert rep.n_pairs == len(win.pairs)


def test_plane_batches_across_round_sizes(sd, O):
    """Plane-mode members whose bin layouts come from rounds of other sizes:
    each link first updates alone (one round of its whole part, through its
    own bins), then in batches driven by a handle with 2^14-pair rounds
    (layouts too large for the driver's bins are scaled down), then with
    2^18-pair rounds (scaled up from the 2^14-pair rounds), then alone
    again; a member in mode 5 takes its own update inside the batches.
    Every DHLA and report equals the oracle's on the link's whole stream."""
    w = T.WORKLOADS["tiny"].with_(dirs=2)
    sizes = [1 << 19, 300_001, 150_000, 1 << 17]
    seeds = [3000 + i for i in range(len(sizes))]
    wins = [T.make_window(w.with_(n=n, planted=4), s, n=n) for n, s in zip(sizes, seeds)]
    drv = sd.sd_create(sd.params_for(w, 1))
    hs = [sd.sd_create(sd.params_for(w, s)) for s in seeds]
    try:
        sd.sd_set_tuning(hs[3], mode=5)
        cuts = [0, 0, 0, 0]
        keep = []  # the device buffers stay alive until the handles' streams have read them

        def feed(frac, batched):
            parts = []
            for i, win in enumerate(wins):
                end = int(len(win.pairs) * frac)
                parts.append(_dev(win.pairs[cuts[i]:end]))
                cuts[i] = end
            keep.append(parts)
            if batched:
                sd.sd_update_many([drv] + hs, [_dev(np.zeros((0, 2), np.uint32))] + parts)
            else:
                for h, p in zip(hs, parts):
                    sd.sd_update(h, p)

        feed(0.3, False)
        sd.sd_set_tuning(drv, mode=6, plane_round_log2=14)
        feed(0.5, True)
        feed(0.6, True)
        sd.sd_set_tuning(drv, mode=6, plane_round_log2=18)
        feed(0.9, True)
        feed(1.0, False)
        grids = [np.concatenate([sd.sd_get_grid(h, d) for d in range(2)]) for h in hs]
        reps = sd.sd_close_many(hs)
    finally:
        for h in hs + [drv]:
            sd.sd_destroy(h)
    for win, s, g, rep in zip(wins, seeds, grids, reps):
        og, ref = _oracle(O, w, win.pairs, s)
        assert np.array_equal(g, og)
        _same_report(rep, ref, 2)
        assert rep.n_pairs == len(win.pairs)


def test_plane_batch_lanes_with_handles_on_one_stream(sd, O):
    """Members that share the driver's CUDA stream, dealt to the batch's
    side lanes: each lane waits for the stream's earlier work and the
    stream for every lane, so a second batch and the closes see every bit."""
    import torch
    w = T.WORKLOADS["tiny"].with_(dirs=2)
    stream = torch.cuda.Stream()
    sizes = [300_000, 250_000, 200_000, 150_000, 100_000, 5000]
    seeds = [4000 + i for i in range(len(sizes))]
    wins = [T.make_window(w.with_(n=n, planted=4), s, n=n) for n, s in zip(sizes, seeds)]
    hs = [sd.sd_create(sd.params_for(w, s, cuda_stream=stream.cuda_stream)) for s in seeds]
    try:
        devs = [_dev(win.pairs) for win in wins]
        half = [d[: 2 * (len(d) // 4)] for d in devs]
        rest = [d[2 * (len(d) // 4):] for d in devs]
        sd.sd_update_many(hs, half)
        sd.sd_update_many(hs, rest)
        grids = [np.concatenate([sd.sd_get_grid(h, d) for d in range(2)]) for h in hs]
        reps = sd.sd_close_many(hs)
    finally:
        for h in hs:
            sd.sd_destroy(h)
    for win, s, g, rep in zip(wins, seeds, grids, reps):
        og, ref = _oracle(O, w, win.pairs, s)
        assert np.array_equal(g, og)
        _same_report(rep, ref, 2)


def test_close_many_equals_close_window_on_core_links(sd, O):
    """Core-link sketches (both directions, 2^16 estimators of 512 bits):
    three links closed together report what each reports alone."""
    w = T.WORKLOADS["core"].with_(n=1 << 20, planted=20, planted_c=("loguniform", 1024, 20000),
                                  src_pool=1 << 18, dst_pool=1 << 20)
    wins = [T.make_window(w, s) for s in (7, 8, 9)]
    seeds = [71, 72, 73]
    alone = []
    for win, s in zip(wins, seeds):
        h = sd.sd_create(sd.params_for(w, s))
        try:
            sd.sd_update(h, _dev(win.pairs))
            alone.append(sd.sd_close_window(h))
        finally:
            sd.sd_destroy(h)
    hs = [sd.sd_create(sd.params_for(w, s)) for s in seeds]
    try:
        sd.sd_update_many(hs, [_dev(win.pairs) for win in wins])
        together = sd.sd_close_many(hs)
    finally:
        for h in hs:
            sd.sd_destroy(h)
    for a, b, win, s in zip(alone, together, wins, seeds):
        assert a.n_cand == b.n_cand and a.flags == b.flags
        assert np.array_equal(a.hits, b.hits)
        _, ref = _oracle(O, w, win.pairs, s)
        _same_report(b, ref, 2)


def test_close_many_mixed_shapes_and_restores(sd, O):
    """Handles of different shapes, or with the staged-join restore, close
    one by one inside sd_close_many; handles of one shape close in batched
    launches.  Every report equals the oracle's."""
    import torch
    w1 = T.WORKLOADS["tiny"].with_(dirs=1)
    w2 = T.WORKLOADS["tiny"].with_(dirs=2)
    cases = [(w1, 31, 0), (w2, 32, 0), (w2, 33, 1), (w2, 34, 0)]
    wins = [T.make_window(w.with_(n=1 << 18, planted=6), s) for w, s, _ in cases]
    for group in (cases, [c for c in cases if c[0] is w2 and c[2] == 0]):
        hs = [sd.sd_create(sd.params_for(w, s)) for w, s, _ in group]
        try:
            for h, (_, _, restore) in zip(hs, group):
                sd.sd_set_tuning(h, mode=5, restore=restore)
            for h, (w, s, _) in zip(hs, group):
                win = wins[[c[1] for c in cases].index(s)]
                sd.sd_update(h, _dev(win.pairs))
            torch.cuda.synchronize()
            reps = sd.sd_close_many(hs)
            again = sd.sd_close_many(hs)  # empty windows after the close
        finally:
            for h in hs:
                sd.sd_destroy(h)
        for rep, r2, (w, s, _) in zip(reps, again, group):
            win = wins[[c[1] for c in cases].index(s)]
            _, ref = _oracle(O, w, win.pairs, s)
            _same_report(rep, ref, w.dirs)
            assert r2.n_pairs == 0 and len(r2.hits) == 0


def _batch_window(args):
    link, n, planted = args
    w = T.WORKLOADS["core"].with_(n=n, planted=planted)
    return T.make_window(w, T.window_seed(3, link=link)).pairs


def test_batching_workload_full_size_sampled(sd, O):
    """The batching benchmark's workload at full size (64 links, lognormal
    window sizes clipped to [256K, 64M], 50-300 planted each, core-link
    sketches) in the benchmark's launch configuration; the smallest, the
    median and the largest link are checked against the oracle in full, and
    every link's pair count and flags are checked."""
    import multiprocessing as mp

    rng = np.random.default_rng(0x5D5A0300)
    sizes = np.clip(np.exp(rng.normal(np.log(4 << 20), 1.0, size=64)), 256 << 10, 64 << 20)
    sizes = (sizes.astype(np.int64) // 2) * 2
    planted = rng.integers(50, 301, size=64)
    jobs = [(i, int(n), int(p)) for i, (n, p) in enumerate(zip(sizes, planted))]
    with mp.get_context("spawn").Pool(8) as pool:
        wins = pool.map(_batch_window, jobs)
    w = T.WORKLOADS["core"]
    seed = T.window_seed(2)
    hs = [sd.sd_create(sd.params_for(w, seed)) for _ in wins]
    try:
        sd.sd_update_many(hs, [_dev(p) for p in wins])
        reps = sd.sd_close_many(hs)
    finally:
        for h in hs:
            sd.sd_destroy(h)
    order = np.argsort(sizes)
    for i in range(64):
        assert reps[i].n_pairs == len(wins[i]) and reps[i].flags == 0
    for i in (order[0], order[32], order[-1]):
        _, ref = _oracle(O, w, wins[i], seed)
        _same_report(reps[i], ref, 2)


def test_update_many_mixed_members_and_close_many_arguments(sd, O):
    """sd_update_many members that cannot join the binned batch (host-memory
    pairs, another DHLA shape, no pairs) take the single-handle path; the
    results still equal the oracle's.  sd_close_many rejects a handle given
    twice and accepts an empty list."""
    w = T.WORKLOADS["tiny"].with_(dirs=2)
    w1 = T.WORKLOADS["tiny"].with_(dirs=1)
    wins = [T.make_window(w.with_(n=100_000, planted=4), s) for s in (51, 52, 53)]
    hs = [sd.sd_create(sd.params_for(w, 51)), sd.sd_create(sd.params_for(w, 52)),
          sd.sd_create(sd.params_for(w1, 53)), sd.sd_create(sd.params_for(w, 54))]
    try:
        pairs = [_dev(wins[0].pairs), np.ascontiguousarray(wins[1].pairs), _dev(wins[2].pairs),
                 np.zeros((0, 2), np.uint32)]
        sd.sd_update_many(hs, pairs)
        reps = sd.sd_close_many(hs)
        with pytest.raises(sd.SdError):
            sd.sd_close_many([hs[0], hs[1], hs[0]])
        assert sd.sd_close_many([]) == []
    finally:
        for h in hs:
            sd.sd_destroy(h)
    for rep, win, ww, s in zip(reps[:3], wins, (w, w, w1), (51, 52, 53)):
        _, ref = _oracle(O, ww, win.pairs, s)
        _same_report(rep, ref, ww.dirs)
    assert reps[3].n_pairs == 0 and len(reps[3].hits) == 0
