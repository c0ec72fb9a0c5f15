"""The device steps of a detection spread over GPUs, on one GPU with virtual
shards, against the CPU oracle.

Stream split then merge (§4.2, the merge of local DHLAs read as a bitwise
OR): shards update their part of the window, their DHLA images are ORed with
sd_or_words (the reduction step of an OR all-reduce) and ORed into one handle
with sd_or_grid; the merged DHLA and its report equal the whole window's.

Key partition (§5, hosts divided by the low bits of their address): each
direction's pairs are grouped by key with sd_partition_pairs and fed to the
shard owning those keys with sd_update_dir; each shard's report, kept to its
own keys, equals the oracle's on that shard's pairs."""
import numpy as np
import pytest

from paper_1803_11449_gb300 import traffic as T

pytestmark = pytest.mark.gpu

SEED = 0x5A4D


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


def _oracle_grid(O, op, pairs):
    og = O.new_grid(op)
    O.update(op, og, pairs)
    return og


@pytest.mark.parametrize("shards", [2, 3, 8])
def test_stream_split_then_or_merge_equals_the_whole_window(sd, O, shards):
    import torch
    w = T.WORKLOADS["tiny"].with_(dirs=2)
    win = T.make_window(w, 77)
    p = sd.params_for(w, SEED)
    words = p.dirs * sd.sd_grid_words(p)
    parts = np.array_split(win.pairs, shards)
    hs = [sd.sd_create(p) for _ in range(shards)]
    merged_h = sd.sd_create(p)
    try:
        images = torch.zeros(shards * words, dtype=torch.int32, device="cuda")
        for i, (h, part) in enumerate(zip(hs, parts)):
            if i % 2:
                sd.sd_set_tuning(h, mode=5)   # shards may bin either way
            sd.sd_update(h, _dev(part))
            sd.sd_export_grid(h, images[i * words:(i + 1) * words])
        for h in hs:
            sd.sd_sync(h)
        merged = torch.zeros(words, dtype=torch.int32, device="cuda")
        sd.sd_or_words(merged, images, words, shards)
        torch.cuda.synchronize()
        sd.sd_or_grid(merged_h, merged)
        grid = np.concatenate([sd.sd_get_grid(merged_h, d) for d in range(p.dirs)])
        rep = sd.sd_close_window(merged_h)
    finally:
        for h in hs + [merged_h]:
            sd.sd_destroy(h)
    op = O.params_from(w.sketch(), seed=SEED)
    og = _oracle_grid(O, op, win.pairs)
    assert np.array_equal(grid, og), "the OR of the shards' DHLAs differs from the whole window's"
    ref = O.close_window(op, og)
    assert rep.n_hits_total == ref["n_hits"] and rep.n_cand == ref["n_cand"]
    assert np.array_equal(rep.hits["ip"], ref["ip"]) and np.array_equal(rep.hits["est"], ref["est"])


def test_or_words_of_ragged_parts(sd):
    """The reduction over count parts, word by word, on random images."""
    import torch
    rng = np.random.default_rng(3)
    words, count = 4 * 12345, 5
    src = rng.integers(0, 2**32, size=(count, words), dtype=np.uint64).astype(np.uint32)
    src[rng.random(src.shape) < 0.7] = 0
    out = torch.zeros(words, dtype=torch.int32, device="cuda")
    sd.sd_or_words(out, torch.from_numpy(src.reshape(-1).view(np.int32)).cuda(), words, count)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), np.bitwise_or.reduce(src, axis=0))


@pytest.mark.parametrize("parts", [1, 4])
def test_key_partition_reports_each_shards_keys(sd, O, parts):
    import torch
    w = T.WORKLOADS["tiny"].with_(dirs=2, n=(1 << 19) + 7, planted=24)
    win = T.make_window(w, 91)
    p = sd.params_for(w, SEED)
    dev = _dev(win.pairs)
    hs = [sd.sd_create(p) for _ in range(parts)]
    try:
        segs = {}
        for d in range(2):
            out = torch.empty_like(dev)
            counts = sd.sd_partition_pairs(hs[0], d, dev, parts, out)
            keys = win.pairs[:, d]
            assert list(counts) == [int(np.sum((keys & (parts - 1)) == q)) for q in range(parts)]
            got = out.cpu().numpy().view(np.uint32).reshape(-1, 2)
            off = np.concatenate([[0], np.cumsum(counts)])
            for q in range(parts):
                seg = got[off[q]:off[q + 1]]
                assert np.all((seg[:, 0] & (parts - 1)) == q)
                want = win.pairs[(keys & (parts - 1)) == q][:, [d, 1 - d]]
                assert np.array_equal(np.sort(seg.view(np.uint64).ravel()), np.sort(want.copy().view(np.uint64).ravel()))
                segs[d, q] = out[2 * off[q]:2 * off[q + 1]]
        reps = []
        for q, h in enumerate(hs):
            for d in range(2):
                sd.sd_update_dir(h, d, segs[d, q])
            reps.append(sd.sd_close_window(h))
    finally:
        for h in hs:
            sd.sd_destroy(h)
    op = O.params_from(w.sketch(), seed=SEED)
    total = 0
    for q, rep in enumerate(reps):
        halves = []
        for d in range(2):
            sub = win.pairs[(win.pairs[:, d] & (parts - 1)) == q]
            halves.append(_oracle_grid(O, op, sub).reshape(2, -1)[d])
        ref = O.close_window(op, np.concatenate(halves))
        mine = (rep.hits["ip"] & (parts - 1)) == q
        theirs = (ref["ip"] & (parts - 1)) == q
        for f, g in (("dir", "dir"), ("ip", "ip"), ("sz", "sz"), ("est", "est")):
            assert np.array_equal(rep.hits[f][mine], ref[g][theirs]), (q, f)
        assert rep.n_pairs == int(np.sum((win.pairs[:, 0] & (parts - 1)) == q))
        total += int(np.sum(mine))
    assert total > 0
