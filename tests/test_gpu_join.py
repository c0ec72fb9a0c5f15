"""The paper's staged join restore on the GPU (tuning restore = 1, §4.2,
Algorithms 3 and 4) against the CPU oracle: the candidate set K, the hot
sets and the report must be identical to the oracle's, and K must equal the
oracle's own literal staged join."""
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


def _run(sd, w, pairs, seed, restore, **caps):
    p = sd.params_for(w, seed, **caps)
    h = sd.sd_create(p)
    try:
        sd.sd_set_tuning(h, mode=5, restore=restore)
        assert sd.sd_get_tuning(h).restore == restore
        sd.sd_update(h, _dev(pairs))
        rep = sd.sd_close_window(h)
        cands = [sd.sd_get_candidates(h, d) for d in range(p.dirs)]
    finally:
        sd.sd_destroy(h)
    return p, rep, cands


def _check(sd, O, w, win, seed=0x10A1):
    p, rep, cands = _run(sd, w, win.pairs, seed, restore=1)
    op = O.params_from(w.sketch(), seed=seed)
    og = O.new_grid(op)
    O.update(op, og, win.pairs)
    ref = O.close_window(op, og, want_cands=True)
    assert [rep.dir_flags(d) for d in range(p.dirs)] == ref["flags"] == [0] * p.dirs
    assert rep.n_cand == ref["n_cand"]
    assert np.array_equal(rep.n_hot, ref["n_hot"]) and rep.psi == ref["psi"]
    for f in ("dir", "ip", "sz", "est"):
        assert np.array_equal(rep.hits[f], ref[f])
    for d in range(p.dirs):
        nk, ks = cands[d]
        assert nk == ref["n_cand"][d]
        assert np.array_equal(np.sort(ks), ref["cands"][d])
        # the oracle's literal staged join reaches the same K
        z0, _ = O.row_stats(op, og, d)
        he, nhe = O.hot_sets(op, z0)
        nj, kj = O.restore_join(op, d, he, nhe)
        assert nj == nk and np.array_equal(np.sort(kj), np.sort(ks))
    # and the default restore gives the same report
    _, rep0, _ = _run(sd, w, win.pairs, seed, restore=0)
    assert np.array_equal(rep0.hits, rep.hits) and rep0.n_cand == rep.n_cand
    return rep, ref


@pytest.mark.parametrize("dirs", [1, 2])
def test_join_tiny(sd, O, dirs):
    """g=256 r=4 k=12 alpha=10: two bits of overlap between neighbouring
    blocks, so the intermediate lists are large relative to K."""
    w = T.WORKLOADS["tiny"].with_(dirs=dirs)
    rep, ref = _check(sd, O, w, T.make_window(w, T.window_seed(1)))
    assert ref["n_hits"] > 20


def test_join_paper_parameters(sd, O):
    """The paper's g=1024 r=5 k=14 alpha=6 (three join stages after the
    first) on core-link traffic."""
    w = T.WORKLOADS["paper"].with_(n=1 << 21, planted=60)
    rep, ref = _check(sd, O, w, T.make_window(w, T.window_seed(6)))
    assert ref["n_hits"] > 10


def test_join_three_rows(sd, O):
    """r = 3 (k = alpha = 16): the first stage is the last one, and the
    blocks do not overlap at all."""
    w = T.WORKLOADS["tiny"].with_(r=3, k=16, alpha=16, theta=512, dirs=2, n=1 << 18, planted=6,
                                  planted_c=("uniform", 2000, 4000))
    _check(sd, O, w, T.make_window(w, 33))


def test_join_overloads(sd, O):
    w = T.WORKLOADS["tiny"].with_(dirs=1)
    win = T.make_window(w, T.window_seed(1))
    # intermediate buffers of 4 cand_cap entries overflow: the direction is
    # flagged, reports nothing, and gives |K| as cand_cap + 1
    p, rep, _ = _run(sd, w, win.pairs, 5, restore=1, cand_cap=64)
    assert rep.dir_flags(0) & sd.SD_FLAG_OVERLOAD_CANDS and len(rep.hits) == 0
    assert rep.n_cand[0] == 65
    # first-stage tuples |HE(0)||HE(1)||HE(2)| above pair_cap while the
    # common work bound |HE(0)| 2^(32-k) stays within it (k = 16 and hot
    # lists of about 300: |HE(1)||HE(2)| > 2^16)
    w = T.WORKLOADS["core"].with_(n=1 << 22, planted=40, planted_c=("loguniform", 1024, 20000),
                                  src_pool=1 << 20, dst_pool=1 << 22)
    win = T.make_window(w, 99)
    n = [int(x) for x in O.close_window(*_oracle_grid(O, w, win.pairs, 5))["n_hot"][0][:3]]
    cap = n[0] * n[1] * n[2] - 1
    assert (n[0] << (32 - w.k)) <= cap
    p, rep, _ = _run(sd, w, win.pairs, 5, restore=1, pair_cap=cap)
    assert rep.dir_flags(0) & sd.SD_FLAG_OVERLOAD_PAIRS and rep.n_cand[0] == 0
    p, rep, _ = _run(sd, w, win.pairs, 5, restore=0, pair_cap=cap)
    assert rep.dir_flags(0) == 0 and len(rep.hits) > 0


def _oracle_grid(O, w, pairs, seed):
    op = O.params_from(w.sketch(), seed=seed)
    og = O.new_grid(op)
    O.update(op, og, pairs)
    return op, og
