"""sd_update_noalloc, the binned update for callers that cannot allocate
device memory (an ingest thread on a latency budget, or a program whose
device memory belongs to another allocator).  Its scratch is a fixed array
inside the library, shared by every call and keeping the last call's
contents.  Through the C ABI, the tests check that two calls in a row give
exactly the DHLA of Algorithm 1 (the CPU oracle's) and of sd_update; that a
DHLA near the 4096-slice limit (bins of about a thousand entries) and a
window whose bit-sets all land in one slice (its bin overflows into the
atomic fallback) come out bit-exact; and that what does not fit, or lives
on the host, is refused.  This file is collected last so a run that stops
at the first failure has run every other test first."""
import numpy as np
import pytest

from paper_1803_11449_gb300 import traffic as T

pytestmark = pytest.mark.gpu

SEED = 0x0A110C


@pytest.fixture(scope="module")
def sd():
    import torch
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    from paper_1803_11449_gb300 import build as b
    b.build()
    from paper_1803_11449_gb300 import sd as mod
    return mod


def _reference_grid(sd, w, pairs_dev):
    p = sd.params_for(w, SEED)
    h = sd.sd_create(p)
    try:
        sd.sd_update(h, pairs_dev)
        return np.concatenate([sd.sd_get_grid(h, d) for d in range(p.dirs)])
    finally:
        sd.sd_destroy(h)


def _oracle_grid(O, w, pairs):
    op = O.params_from(w.sketch(), seed=SEED)
    og = O.new_grid(op)
    O.update(op, og, pairs)
    return og


def _noalloc(sd, torch, p, pairs_dev, stream):
    words = p.dirs * sd.sd_grid_words(p)
    grid = torch.zeros(words, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    rc = sd.sd_update_noalloc(p, grid, pairs_dev, stream)
    assert rc == sd.SD_OK, rc
    stream.synchronize()
    return grid.cpu().numpy().view(np.uint32)


def test_noalloc_update_matches_the_oracle_on_two_calls_in_a_row(sd, O):
    import torch
    w = T.WORKLOADS["core"].with_(n=(1 << 21) + 3, planted=30, planted_c=("loguniform", 1024, 20000),
                                  src_pool=1 << 18, dst_pool=1 << 21)
    p = sd.params_for(w, SEED)
    stream = torch.cuda.Stream()
    for call, seed in enumerate((101, 202)):
        win = T.make_window(w, seed)
        pairs = torch.from_numpy(win.pairs.reshape(-1).view(np.int32)).cuda()
        got = _noalloc(sd, torch, p, pairs, stream)
        assert np.array_equal(got, _oracle_grid(O, w, win.pairs)), f"call {call}: DHLA differs from the oracle's"
        assert np.array_equal(got, _reference_grid(sd, w, pairs)), f"call {call}: DHLA differs from sd_update's"


def test_noalloc_near_the_slice_limit_and_with_overflowing_bins(sd, O):
    """g=2048, r=4, k=18, both directions: 2 x 256 MiB of DHLA = 4096 slices
    of 128 KiB, the most the scratch takes (about a thousand entries per
    bin, many rounds).  Then one pair repeated 2^20 times on the core
    sketch: every bit-set of a direction falls in the same words, so those
    slices' bins overflow and the rest goes through the atomic fallback."""
    import torch
    stream = torch.cuda.Stream()
    w = T.WORKLOADS["core"].with_(g=2048, r=4, k=18, alpha=7, n=1 << 20, src_pool=1 << 16,
                                  dst_pool=1 << 20, planted=8, planted_c=("uniform", 3000, 6000))
    p = sd.params_for(w, SEED)
    assert p.dirs * sd.sd_grid_words(p) == 4096 << 15
    win = T.make_window(w, 303)
    got = _noalloc(sd, torch, p, torch.from_numpy(win.pairs.reshape(-1).view(np.int32)).cuda(), stream)
    assert np.array_equal(got, _oracle_grid(O, w, win.pairs))
    del got
    w = T.WORKLOADS["core"].with_(n=1 << 20)
    same = np.tile(np.array([[0x0A000001, 0xC0A80001]], np.uint32), (1 << 20, 1))
    p = sd.params_for(w, SEED)
    got = _noalloc(sd, torch, p, torch.from_numpy(same.reshape(-1).view(np.int32)).cuda(), stream)
    og = _oracle_grid(O, w, same)
    assert np.array_equal(got, og) and int(np.unpackbits(og.view(np.uint8)).sum()) == 2 * w.r


def test_noalloc_rejects_what_does_not_fit_or_is_not_on_the_device(sd):
    import torch
    big = sd.sd_default_params(g=4096, r=8, k=20, alpha=4, dirs=2)   # 2 x 512 MiB of DHLA
    assert sd.sd_check_params(big) == 0
    grid = torch.zeros(16, dtype=torch.int32, device="cuda")
    pairs = torch.zeros(2, dtype=torch.int32, device="cuda")
    assert sd.sd_update_noalloc(big, grid, pairs) == sd.SD_ERR_TOO_LARGE
    small = sd.sd_default_params()
    host_pairs = torch.zeros(2, dtype=torch.int32)
    dgrid = torch.zeros(small.dirs * sd.sd_grid_words(small), dtype=torch.int32, device="cuda")
    assert sd.sd_update_noalloc(small, dgrid, host_pairs) == sd.SD_ERR_ARG
    assert sd.sd_update_noalloc(small, dgrid.cpu(), pairs) == sd.SD_ERR_ARG
