"""Pins for the oracle's window close: hot estimators and Zmin (Algorithm 2),
psi (Lemma 1 and the w(i)' average of §3.3), Eq. 4 (Theorem 1), the restore
(Algorithm 2 / Algorithms 3-4) and the report."""
import math

import numpy as np
import pytest

from paper_1803_11449_gb300 import traffic as T


def _grid_with_weights(O, p, weights):
    """A one-direction grid whose estimator (i, j) has exactly weights[i][j]
    one bits (the lowest bits)."""
    cw = p.g // 32
    grid = O.new_grid(p).reshape(p.r, 1 << p.k, cw)
    bits = np.zeros((p.r, 1 << p.k, p.g), dtype=np.uint8)
    w = np.asarray(weights)
    ar = np.arange(p.g)
    bits[:] = (ar[None, None, :] < w[:, :, None])
    packed = np.packbits(bits, axis=2, bitorder="little").view(np.uint32)
    grid[:] = packed
    return grid.reshape(-1)


def test_psi_closed_form(O):
    """Lemma 1: psi = 1 - e^(-w/(g 2^k)); with w' the mean of the per-row
    w(i)' = -g 2^k ln(ZR(i)/(g 2^k)), psi = 1 - (prod_i ZR(i)/(g 2^k))^(1/r).
    Rows at exactly half density give psi = 1/2."""
    p = O.make_params(256, 4, 10, 8, 1024.0, seed=1)
    half = np.full((p.r, 1 << p.k), p.g // 2)
    grid = _grid_with_weights(O, p, half)
    _, zr = O.row_stats(p, grid, 0)
    assert list(zr) == [(1 << p.k) * p.g // 2] * p.r
    assert abs(O.psi(p, zr) - 0.5) < 1e-14

    rng = np.random.default_rng(0)
    dens = [0.1, 0.35, 0.6, 0.85]
    w = np.stack([rng.binomial(p.g, d, size=1 << p.k) for d in dens])
    grid = _grid_with_weights(O, p, w)
    _, zr = O.row_stats(p, grid, 0)
    G = p.g * (1 << p.k)
    assert list(zr) == [int(G - w[i].sum()) for i in range(p.r)]
    geo = math.prod(int(z) / G for z in zr) ** (1.0 / p.r)
    assert abs(O.psi(p, zr) - (1.0 - geo)) < 1e-12


def test_saturated_row_has_no_psi(O):
    p = O.make_params(256, 4, 10, 8, 1024.0, seed=1)
    w = np.full((p.r, 1 << p.k), 7)
    w[2] = p.g
    grid = _grid_with_weights(O, p, w)
    _, zr = O.row_stats(p, grid, 0)
    assert zr[2] == 0 and O.psi(p, zr) < 0
    res = O.close_window(p, grid)
    assert res["flags"][0] == O.FLAG_SATURATED and res["n_hits"] == 0


def test_hot_threshold_is_strict(O):
    """Algorithm 2: Zmin = g e^(-theta/g) and an estimator is hot when
    z_0 < Zmin.  For g = theta = 1024, Zmin = 1024/e = 376.7..., so z_0 = 376 is
    hot and 377 is not."""
    p = O.make_params(1024, 4, 8, 8, 1024.0, seed=1)
    assert abs(O.zmin(1024, 1024.0) - 1024 / math.e) < 1e-9
    w = np.zeros((p.r, 1 << p.k), dtype=np.int64)
    w[:, 5] = 1024 - 376
    w[:, 9] = 1024 - 377
    w[:, 200] = 1024          # full estimator: z_0 = 0
    grid = _grid_with_weights(O, p, w)
    z0, _ = O.row_stats(p, grid, 0)
    he, nhe = O.hot_sets(p, z0)
    for i in range(p.r):
        assert list(he[i, :nhe[i]]) == [5, 200]


def test_eq4_special_cases(O):
    """Eq. 4, C = -g ln(SZ / (g - g psi^r)): with psi = 0 it is the linear
    estimator of Eq. 1, -g ln(z_0/g); SZ = 0 gives +inf; SZ = g(1 - psi^r)
    gives 0; it decreases in SZ."""
    g, r = 1024, 5
    for z in (1, 17, 376, 1023):
        assert abs(O.estimate(g, r, 0.0, z) - (-g * math.log(z / g))) < 1e-9 * g
    assert O.estimate(g, r, 0.3, 0) == math.inf
    psi = 0.5
    zero_at = g * (1 - psi ** r)
    assert float(zero_at).is_integer()
    assert O.estimate(g, r, psi, int(zero_at)) == 0.0
    vals = [O.estimate(g, r, 0.37, z) for z in range(0, g + 1)]
    assert all(a > b for a, b in zip(vals, vals[1:]))


def test_eq4_inverts_the_expected_zero_count(O):
    """Theorem 1's model: a host with c peers keeps a bit of ULE at zero when
    none of its c peers hashed there ((1 - 1/g)^c) and the bit is not set in
    all r estimators by other hosts (1 - psi^r), so E[SZ] = g (1 - 1/g)^c
    (1 - psi^r).  Eq. 4 maps that SZ back to -g c ln(1 - 1/g) (= c to within
    c/2g) for any g, r, c and psi; psi is solved here so that E[SZ] is the
    integer the oracle takes."""
    rng = np.random.default_rng(4)
    for _ in range(200):
        g = int(2 ** rng.integers(5, 13))
        r = int(rng.integers(3, 9))
        c = float(rng.uniform(0, 4 * g))
        own = g * (1 - 1 / g) ** c          # expected zero bits of the host's own estimator
        if own < 2:
            continue
        sz = int(rng.integers(1, int(own)))  # any integer below it fixes psi
        psi = (1 - sz / own) ** (1 / r)
        want = -g * c * math.log1p(-1 / g)
        got = O.estimate(g, r, psi, sz)
        assert abs(got - want) <= 1e-9 * max(1.0, abs(want)), (g, r, c, psi, sz)


def test_theorem1_removes_shared_bits(O):
    """Theorem 1 model: a host's r estimators each hold its own c peers plus
    bits set by other hosts independently with probability psi.  ULE is the
    AND of the r estimators, SZ its zero count, and Eq. 4 then estimates c.
    Simulated here without the oracle; the oracle's Eq. 4 must be unbiased to
    within 3% (dropping the exponent r, or psi, is off by tens of percent)."""
    g, r, psi, c = 1024, 4, 0.3, 1500
    rng = np.random.default_rng(42)
    ests = []
    for _ in range(400):
        own = np.zeros(g, dtype=bool)
        own[rng.integers(0, g, size=c)] = True
        ule = own.copy()
        other = np.ones(g, dtype=bool)
        for _ in range(r):
            other &= rng.random(g) < psi
        ule |= other
        sz = int(g - ule.sum())
        ests.append(O.estimate(g, r, psi, sz))
    assert abs(np.mean(ests) / c - 1) < 0.03


def _hot_from_keys(O, p, keys, extra=0, seed=0):
    """z_0 arrays in which exactly the estimators of `keys` (plus `extra`
    random ones per row) are hot."""
    z0 = np.full((p.r, 1 << p.k), p.g, dtype=np.uint32)
    for a in keys:
        for i in range(p.r):
            z0[i, O.dh(p, 0, i, int(a))] = 0
    rng = np.random.default_rng(seed)
    for i in range(p.r):
        z0[i, rng.integers(0, 1 << p.k, size=extra)] = 0
    return O.hot_sets(p, z0)


@pytest.mark.parametrize("g,r,k,alpha", [(256, 4, 12, 10), (512, 4, 16, 8), (1024, 5, 14, 6),
                                         (64, 3, 16, 16), (128, 6, 10, 6)])
def test_every_host_restores_to_itself(O, g, r, k, alpha):
    """§3.2: a0 can be restored from LE(a0).  When the estimators of a set P
    of hosts are hot, the join of Algorithm 2 (staged as in Algorithms 3-4)
    and the preimage enumeration both return a superset of P, and every
    restored host has all r estimators hot."""
    p = O.make_params(g, r, k, alpha, 1024.0, seed=123)
    rng = np.random.default_rng(k + r)
    P = rng.choice(2**32, size=25, replace=False)
    he, nhe = _hot_from_keys(O, p, P, extra=20, seed=k)
    hot = [set(he[i, :nhe[i]].tolist()) for i in range(p.r)]
    nj, kj = O.restore_join(p, 0, he, nhe)
    npre, kp = O.restore_preimage(p, 0, he, nhe)
    assert nj == npre and np.array_equal(kj, kp)
    assert set(P.tolist()) <= set(kj.tolist())
    for a in kj:
        assert all(O.dh(p, 0, i, int(a)) in hot[i] for i in range(p.r))


def test_restore_routines_agree_across_parameter_space(O):
    """§3.3 allows any r >= 3 and alpha with alpha <= k and (r-2) alpha + k
    >= 32.  For seeded random parameter sets across that space (not only the
    default alpha), the staged join and the preimage enumeration return the
    same K, which holds every host whose estimators were made hot, and every
    member of K has all r estimators hot."""
    rng = np.random.default_rng(2018)
    done = 0
    while done < 16:
        r = int(rng.integers(3, 9))
        k = int(rng.integers(14, 21))
        lo = -(-(32 - k) // (r - 2))
        if lo > k:
            continue
        alpha = int(rng.integers(max(1, lo), k + 1))
        p = O.make_params(64, r, k, alpha, 1024.0, seed=int(rng.integers(1 << 62)))
        assert O.check_params(p), (r, k, alpha)
        P = rng.choice(2**32, size=8, replace=False)
        he, nhe = _hot_from_keys(O, p, P, extra=12, seed=done)
        hot = [set(he[i, :nhe[i]].tolist()) for i in range(p.r)]
        _, kj = O.restore_join(p, 0, he, nhe)
        _, kp = O.restore_preimage(p, 0, he, nhe)
        assert np.array_equal(kj, kp), (r, k, alpha)
        assert set(P.tolist()) <= set(kj.tolist())
        assert all(O.dh(p, 0, i, int(a)) in hot[i] for a in kj for i in range(p.r))
        done += 1


def test_join_stops_at_bit_31(O):
    """Algorithm 3 joins BL(1) and the new bits of BL(2) into bits [0, k +
    alpha) of a0.  With k + alpha > 32, a tuple whose BL(2) sets a bit at or
    above 32 names no IPv4 address and restores nothing; cut to 32 bits it
    would name a host whose row-2 estimator is not hot.  Hand-built hot sets
    around one host a: its own CL_0 and CL_1, and in row 2 such a tuple's
    estimator, a's own, or both."""
    p = O.make_params(64, 3, 20, 16, 1024.0, seed=77)
    assert O.check_params(p)
    a = 0xC0A81234
    c0, c1, c2 = (O.dh(p, 0, i, a) for i in range(3))
    past_31 = c0 ^ (((a >> 16) & 0xFFFF) | (0x5 << 16))  # BL(2) with bits 32-35 set
    assert past_31 != c2
    he = np.zeros((p.r, 1 << p.k), dtype=np.uint32)
    he[0, 0], he[1, 0] = c0, c1
    for row2, expect in (([past_31], []), ([c2], [a]), (sorted([past_31, c2]), [a])):
        he[2, :len(row2)] = row2
        nhe = np.array([1, 1, len(row2)], dtype=np.uint32)
        _, kj = O.restore_join(p, 0, he, nhe)
        _, kp = O.restore_preimage(p, 0, he, nhe)
        assert kj.tolist() == kp.tolist() == expect


@pytest.mark.slow
def test_restore_and_report_equal_exhaustive_sweep(O):
    """The restored set K equals {a in [0, 2^32) : DH_i(a) in HE(i) for all i}
    and the report equals {a : all estimators hot and C(a) >= theta}, both by
    sweeping the whole key space; the staged join agrees as well."""
    w = T.WORKLOADS["tiny"]
    win = T.make_window(w, T.window_seed(1))
    p = O.params_from(w.sketch(), seed=1234)
    grid = O.new_grid(p)
    O.update(p, grid, win.pairs)
    res = O.close_window(p, grid, want_cands=True)
    z0, _ = O.row_stats(p, grid, 0)
    he, nhe = O.hot_sets(p, z0)
    nj, kj = O.restore_join(p, 0, he, nhe)
    ip, sz, kb = O.report_brute(p, grid, 0)
    assert res["n_cand"][0] == nj == len(kb)
    assert np.array_equal(res["cands"][0], kb) and np.array_equal(kj, kb)
    assert np.array_equal(res["ip"], ip) and np.array_equal(res["sz"], sz)
    assert res["n_hits"] > 0


def _small_core(n=1 << 22, planted=40):
    return T.WORKLOADS["core"].with_(n=n, planted=planted, planted_c=("loguniform", 1024, 20000),
                                     src_pool=1 << 20, dst_pool=1 << 22)


@pytest.mark.parametrize("name", ["tiny", "small-core"])
def test_planted_super_points_are_found(O, name):
    """§3.2: when a0 is a super point its estimators are hot, so it is
    restored.  Every planted host with at least 2 theta distinct peers must
    be reported in its own direction."""
    w = T.WORKLOADS["tiny"] if name == "tiny" else _small_core()
    win = T.make_window(w, 77)
    p = O.params_from(w.sketch(), seed=2024)
    grid = O.new_grid(p)
    O.update(p, grid, win.pairs)
    res = O.close_window(p, grid)
    assert res["flags"] == [0] * p.dirs
    got = set(zip(res["dir"].tolist(), res["ip"].tolist()))
    strong = [(int(d), int(a)) for a, d, c in zip(win.planted_ip, win.planted_dir, win.planted_c)
              if c >= 2 * p.theta]
    assert strong and all(s in got for s in strong)
    # every reported estimate is at least theta, ordered by (dir, ip)
    assert np.all(res["est"] >= p.theta)
    key = res["dir"].astype(np.uint64) << np.uint64(32) | res["ip"].astype(np.uint64)
    assert np.all(np.diff(key.astype(np.int64)) > 0)


def test_accuracy_statistics_small_core(O):
    """Definition 2 (FPR, FNR) against exact cardinalities; informational
    bounds only (the paper's own accuracy figures are not recoverable)."""
    w = _small_core()
    win = T.make_window(w, 5)
    p = O.params_from(w.sketch(), seed=99)
    grid = O.new_grid(p)
    O.update(p, grid, win.pairs)
    res = O.close_window(p, grid)
    for d in range(p.dirs):
        hosts, counts = T.exact_cardinality(win.pairs, d)
        truth = set(hosts[counts > p.theta].tolist())
        rep = set(res["ip"][res["dir"] == d].tolist())
        N = max(1, len(truth))
        fnr = len(truth - rep) / N
        fpr = len(rep - truth) / N
        assert fnr < 0.2, (d, fnr, fpr, len(truth))


def test_overload_flags(O):
    """Overload reading (the paper has no bound): the restore work bound
    |HE(0)| 2^(32-k) above pair_cap skips the restore; |K| above cand_cap
    drops the direction's hits and reports |K| as cand_cap + 1.  Both caps
    are checked on each side of their boundary."""
    w = T.WORKLOADS["tiny"]
    win = T.make_window(w, T.window_seed(1))
    p = O.params_from(w.sketch(), seed=1234)
    grid = O.new_grid(p)
    O.update(p, grid, win.pairs)
    full = O.close_window(p, grid)
    nk = full["n_cand"][0]
    work = int(full["n_hot"][0][0]) << (32 - w.k)
    p2 = O.params_from(w.sketch(), seed=1234, pair_cap=work - 1)
    r2 = O.close_window(p2, grid)
    assert r2["flags"][0] == O.FLAG_OVERLOAD_PAIRS and r2["n_hits"] == 0 and r2["n_cand"][0] == 0
    p2b = O.params_from(w.sketch(), seed=1234, pair_cap=work)
    assert O.close_window(p2b, grid)["flags"][0] == 0
    p3 = O.params_from(w.sketch(), seed=1234, cand_cap=nk - 1)
    r3 = O.close_window(p3, grid)
    assert r3["flags"][0] == O.FLAG_OVERLOAD_CANDS and r3["n_hits"] == 0
    assert r3["n_cand"][0] == nk
    p3b = O.params_from(w.sketch(), seed=1234, cand_cap=nk // 3)
    r3b = O.close_window(p3b, grid)
    assert r3b["flags"][0] == O.FLAG_OVERLOAD_CANDS and r3b["n_cand"][0] == nk // 3 + 1
    p4 = O.params_from(w.sketch(), seed=1234, cand_cap=nk)
    r4 = O.close_window(p4, grid)
    assert r4["flags"][0] == 0 and r4["n_hits"] == full["n_hits"] and r4["n_cand"][0] == nk


def test_overloaded_restore_stops_at_the_cap(O):
    """A DHLA whose estimators are all full: every key is in K (|K| = 2^32),
    so the close must flag the overload after cand_cap + 1 members instead of
    walking the whole key space."""
    import time
    w = T.WORKLOADS["tiny"]
    p = O.params_from(w.sketch(), seed=77, cand_cap=1 << 16)
    grid = np.full(O.new_grid(p).shape, 0xFFFFFFFF, dtype=np.uint32)
    grid[::w.g // 32] = 0xFFFFFFFE   # one zero bit per estimator: ZR(i) = 2^k, psi defined
    t0 = time.perf_counter()
    r = O.close_window(p, grid)
    assert time.perf_counter() - t0 < 5.0
    assert r["flags"][0] == O.FLAG_OVERLOAD_CANDS and r["n_cand"][0] == (1 << 16) + 1
    assert list(r["n_hot"][0]) == [1 << w.k] * w.r and r["n_hits"] == 0
