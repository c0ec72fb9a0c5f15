"""Pins for the oracle's hash group (§3.2, Eq. 2 and Eq. 3; restrictions in §3.3).

Each test checks the oracle against something other than itself: published
generator output, the paper's reconstruction claim, the algebra of odd
multipliers, or uniformity statistics.
"""
import os

import numpy as np
import pytest
from scipy import stats

HERE = os.path.dirname(os.path.abspath(__file__))

CONFIGS = [  # (g, r, k, alpha)
    (256, 4, 12, 10),   # tiny
    (512, 4, 16, 8),    # core
    (1024, 5, 14, 6),   # the paper's §5 parameters
    (1024, 4, 18, 7),   # stress
    (64, 3, 16, 16),    # alpha = k: no overlap between blocks
    (128, 6, 10, 6),    # (r-2)alpha + k > 32: last block runs past bit 31
    (64, 8, 8, 6),      # the last block starts at bit 36: Eq. 2's shift leaves nothing
]


def _golden(name):
    vals = []
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                vals.append(int(line, 0))
    return vals


def test_splitmix64_matches_published_output(O):
    assert O.splitmix64_stream(0, 3) == _golden("splitmix64_seed0.txt")


def test_hash_constants_are_odd_and_direction_specific(O):
    for seed in (0, 1, 0xDEADBEEF, 2**63 + 5):
        a0, a1, _ = O.hash_constants(seed, 0)
        b0, b1, _ = O.hash_constants(seed, 1)
        assert a0 & 1 and a1 & 1 and b0 & 1 and b1 & 1
        assert (a0, a1) != (b0, b1)


def test_inverse_of_odd_multiplier(O):
    rng = np.random.default_rng(7)
    for a in rng.integers(0, 2**31, size=200) * 2 + 1:
        inv = O.inverse_odd(int(a))
        assert (int(a) * inv) % 2**32 == 1


def _blocks(O, p, a):
    """BL(i) for i = 1..r-1 by Eq. 3: DH_i(a) xor DH_0(a)."""
    h0 = O.dh(p, 0, 0, a)
    return [O.dh(p, 0, i, a) ^ h0 for i in range(1, p.r)]


@pytest.mark.parametrize("g,r,k,alpha", CONFIGS)
def test_eq3_blocks_restore_the_key(O, g, r, k, alpha):
    """§3.3: with alpha <= k and (r-2)alpha + k >= 32, a0 is restored from its
    r-1 bit blocks by comparing the k-alpha overlapping bits of neighbours and
    concatenating.  The reconstruction here is written from that description
    alone; a wrong shift, index or mask in Eq. 2 breaks it."""
    p = O.make_params(g, r, k, alpha, 1024.0, seed=99)
    assert O.check_params(p)
    rng = np.random.default_rng(k * 31 + r)
    keys = list(rng.integers(0, 2**32, size=300, dtype=np.uint64)) + [0, 1, 2**32 - 1, 2**31]
    ov = k - alpha
    for a in keys:
        a = int(a)
        bl = _blocks(O, p, a)
        assert all(0 <= b < 2**k for b in bl)
        # neighbouring blocks agree on their k - alpha shared bits
        for i in range(len(bl) - 1):
            assert (bl[i] >> alpha) == (bl[i + 1] & ((1 << ov) - 1))
        rec = bl[0]
        for i in range(1, len(bl)):
            rec |= (bl[i] >> ov) << (i - 1) * alpha + k
        assert rec == a


@pytest.mark.parametrize("g,r,k,alpha", CONFIGS[:4])
def test_dh0_preimages(O, g, r, k, alpha):
    """A0 odd makes a -> A0*a mod 2^32 a bijection, so each CL_0 has exactly
    2^(32-k) preimages a = A0^-1 ((CL_0 << (32-k)) | t)."""
    p = O.make_params(g, r, k, alpha, 1024.0, seed=5)
    A0, _, _ = O.hash_constants(p.seed, 0)
    inv = O.inverse_odd(A0)
    rng = np.random.default_rng(1)
    for c in rng.integers(0, 2**k, size=40):
        for t in rng.integers(0, 2**(32 - k), size=20):
            a = (inv * ((int(c) << (32 - k)) | int(t))) % 2**32
            assert O.dh(p, 0, 0, a) == c


@pytest.mark.parametrize("g,r,k,alpha", CONFIGS[:4])
def test_dh_rows_are_uniform(O, g, r, k, alpha):
    """§3.2 requirement 1: every estimator of an LA is used with the same
    probability.  Chi-square over 16 buckets of each row's index, for random
    keys and for consecutive keys."""
    p = O.make_params(g, r, k, alpha, 1024.0, seed=11)
    rng = np.random.default_rng(3)
    for keys in (rng.integers(0, 2**32, size=4000, dtype=np.uint64), np.arange(4000) + 0x0A000000):
        for i in range(r):
            idx = np.array([O.dh(p, 0, i, int(a)) for a in keys])
            assert idx.min() >= 0 and idx.max() < 2**k
            counts = np.bincount(idx >> (k - 4), minlength=16)
            assert stats.chisquare(counts).pvalue > 1e-6


def test_h1_is_uniform_over_g_bits(O):
    """§3.2: H1 spreads a host's peers uniformly over the g bits of an
    estimator, also when the peers are structured the way addresses are:
    one subnet (only the low bits differ) or one host number in many
    networks (only the high bits differ)."""
    for g in (256, 512, 1024):
        p = O.make_params(g, 4, 16, 8, 1024.0, seed=3)
        rng = np.random.default_rng(g)
        for ys in (rng.integers(0, 2**32, size=60000, dtype=np.uint64),
                   0x0A000000 + np.arange(60000, dtype=np.uint64),
                   (np.arange(60000, dtype=np.uint64) << np.uint64(16)) | np.uint64(0x0101)):
            bits = np.array([O.h1(p, 0, int(y)) for y in ys])
            assert bits.min() >= 0 and bits.max() < g
            counts = np.bincount(bits * 16 // g, minlength=16)
            assert stats.chisquare(counts).pvalue > 1e-6


def test_parameter_restrictions(O):
    mk = O.make_params
    assert O.check_params(mk(1024, 5, 14, 6, 1024, 0))          # §5 choice
    assert not O.check_params(mk(1024, 5, 14, 15, 1024, 0))     # alpha > k
    assert not O.check_params(mk(1024, 5, 14, 5, 1024, 0))      # (r-2)alpha + k = 29 < 32
    assert not O.check_params(mk(1000, 4, 16, 8, 1024, 0))      # g not a power of two
    assert not O.check_params(mk(512, 2, 16, 16, 1024, 0))      # r < 3
    assert not O.check_params(mk(512, 4, 25, 8, 1024, 0))       # k beyond the layout


def test_default_alpha_reproduces_the_papers_choice():
    from paper_1803_11449_gb300.traffic import default_alpha
    assert default_alpha(14, 5) == 6      # §5: r=5, k=14, alpha=6
    assert default_alpha(16, 4) == 8
    assert default_alpha(12, 4) == 10
    assert default_alpha(18, 4) == 7
