"""The seeded traffic generator: determinism, Zipf shape, planted degrees."""
import math

import numpy as np
from scipy import stats

from paper_1803_11449_gb300 import traffic as T


def test_same_seed_same_window():
    w = T.WORKLOADS["tiny"].with_(n=1 << 14)
    a, b = T.make_window(w, 9), T.make_window(w, 9)
    c = T.make_window(w, 10)
    assert np.array_equal(a.pairs, b.pairs) and not np.array_equal(a.pairs, c.pairs)
    assert a.pairs.shape == (1 << 14, 2) and a.pairs.dtype == np.uint32


def test_zipf_sampler_matches_pmf():
    """Rejection-inversion must reproduce P(k) ~ k^-s exactly (chi-square)."""
    rng = np.random.default_rng(0)
    for N, s in ((20, 1.1), (50, 1.0), (30, 0.8)):
        x = T.zipf_ranks(rng, 200_000, N, s)
        assert x.min() >= 1 and x.max() <= N
        pmf = np.arange(1, N + 1, dtype=float) ** -s
        pmf /= pmf.sum()
        obs = np.bincount(x, minlength=N + 1)[1:]
        assert stats.chisquare(obs, pmf * x.size).pvalue > 1e-4


def test_mix32_is_a_bijection_on_a_block():
    idx = np.arange(1 << 20, dtype=np.uint32)
    assert np.unique(T.mix32(idx)).size == idx.size


def test_planted_degrees_are_exact():
    w = T.WORKLOADS["core"].with_(n=1 << 20, planted=12, planted_c=("loguniform", 1024, 8000),
                                  src_pool=1 << 16, dst_pool=1 << 20)
    win = T.make_window(w, 4)
    for d in (0, 1):
        hosts, counts = T.exact_cardinality(win.pairs, d)
        lookup = dict(zip(hosts.tolist(), counts.tolist()))
        for ip, pd, c in zip(win.planted_ip, win.planted_dir, win.planted_c):
            if pd == d:
                assert lookup[int(ip)] == c
    assert set(win.planted_dir.tolist()) == {0, 1}


def test_loguniform_planted_range_and_budget():
    w = T.WORKLOADS["core"].with_(n=1 << 20, planted=200)
    win = T.make_window(w, 1)
    assert win.planted_c.sum() <= w.planted_share * w.n
    w2 = T.WORKLOADS["core"].with_(n=1 << 26, planted=300)
    c = T._planted_counts(np.random.default_rng(3), w2, w2.n)
    assert c.min() >= 1024 and c.max() <= 200_000
    # log-uniform: log c roughly uniform
    assert abs(np.mean(np.log(c)) - (math.log(1024) + math.log(200_000)) / 2) < 0.5
