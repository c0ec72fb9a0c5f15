"""sd_update_noalloc, the binned update for callers that cannot allocate
device memory (an ingest thread on a latency budget, or a program whose
device memory belongs to another allocator).  Its scratch is a fixed array
inside the library, shared by every call and keeping the last call's
contents; the test checks, through the C ABI, that two calls in a row give
exactly the DHLA that sd_update builds.  This file is collected last so a
run that stops at the first failure has run every other test first."""
import numpy as np
import pytest

from paper_1803_11449_gb300 import traffic as T

pytestmark = pytest.mark.gpu

SEED = 0x0A110C


def _reference_grid(sd, torch, w, pairs_dev):
    p = sd.params_for(w, SEED)
    h = sd.sd_create(p)
    try:
        sd.sd_update(h, pairs_dev)
        return np.concatenate([sd.sd_get_grid(h, d) for d in range(p.dirs)])
    finally:
        sd.sd_destroy(h)


def test_noalloc_update_matches_sd_update_on_two_calls_in_a_row():
    import torch
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    from paper_1803_11449_gb300 import build as b
    b.build()
    from paper_1803_11449_gb300 import sd

    w = T.WORKLOADS["core"].with_(n=(1 << 21) + 3, planted=30, planted_c=("loguniform", 1024, 20000),
                                  src_pool=1 << 18, dst_pool=1 << 21)
    p = sd.params_for(w, SEED)
    words = p.dirs * sd.sd_grid_words(p)
    stream = torch.cuda.Stream()
    for call, seed in enumerate((101, 202)):
        win = T.make_window(w, seed)
        pairs = torch.from_numpy(win.pairs.reshape(-1).view(np.int32)).cuda()
        expected = _reference_grid(sd, torch, w, pairs)
        grid = torch.zeros(words, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        rc = sd.sd_update_noalloc(p, grid, pairs, stream)
        assert rc == sd.SD_OK, (call, rc)
        stream.synchronize()
        got = grid.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, expected), f"call {call}: DHLA differs from sd_update's"


def test_noalloc_rejects_what_does_not_fit():
    import torch
    from paper_1803_11449_gb300 import sd
    big = sd.sd_default_params(g=4096, r=8, k=20, alpha=4, dirs=2)   # 2 x 512 MiB of DHLA
    assert sd.sd_check_params(big) == 0
    grid = torch.zeros(16, dtype=torch.int32, device="cuda")
    pairs = torch.zeros(2, dtype=torch.int32, device="cuda")
    assert sd.sd_update_noalloc(big, grid, pairs) == sd.SD_ERR_TOO_LARGE
