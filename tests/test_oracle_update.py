"""Pins for the oracle's Algorithm 1 (Update DHLA) and the grid it builds."""
import numpy as np
import pytest


def _single_key_pairs(key, peers, direction=0):
    peers = np.asarray(peers, dtype=np.uint32)
    keys = np.full(peers.size, key, dtype=np.uint32)
    return np.stack([keys, peers] if direction == 0 else [peers, keys], axis=1)


def _cells(O, p, grid):
    cw = p.g // 32
    return grid.reshape(p.dirs, p.r, 1 << p.k, cw)


@pytest.mark.parametrize("n", [1, 37, 300, 2000])
def test_single_key_closed_form(O, n):
    """One host with n distinct peers in an empty DHLA: Algorithm 1 selects
    one bit per peer (shared by all r rows) and sets it in exactly one
    estimator per row.  So the grid has exactly one non-zero estimator per
    row, the r estimators are identical, ULE equals each of them, and
    SZ = g - popcount of that estimator."""
    p = O.make_params(512, 4, 16, 8, 1024.0, seed=21)
    rng = np.random.default_rng(n)
    peers = rng.choice(2**32, size=n, replace=False)
    key = 0xC0A80001
    grid = O.new_grid(p)
    O.update(p, grid, _single_key_pairs(key, peers))
    cells = _cells(O, p, grid)[0]
    nz = [np.flatnonzero(cells[i].any(axis=1)) for i in range(p.r)]
    assert all(len(x) == 1 for x in nz)
    for i in range(p.r):
        assert nz[i][0] == O.dh(p, 0, i, key)
    first = cells[0, nz[0][0]]
    for i in range(1, p.r):
        assert np.array_equal(cells[i, nz[i][0]], first)
    ones = int(np.unpackbits(first.view(np.uint8)).sum())
    assert 1 <= ones <= min(n, p.g)
    assert O.sz(p, grid, 0, key) == p.g - ones


def test_linear_counting_expectation(O):
    """Eq. 1's model (and the proof of Lemma 1): after n distinct peers, the
    expected number of zero bits in a g-bit estimator is g (1 - 1/g)^n.
    Averaged over 400 independent hosts in an otherwise sparse grid, the
    mean z_0 must lie within 4 standard errors of that value."""
    g, n = 256, 200
    p = O.make_params(g, 4, 12, 10, 1024.0, seed=77)
    rng = np.random.default_rng(5)
    z = []
    keys = rng.choice(2**32, size=400, replace=False)
    for key in keys:
        grid = O.new_grid(p)
        O.update(p, grid, _single_key_pairs(int(key), rng.choice(2**32, size=n, replace=False)))
        z.append(O.sz(p, grid, 0, int(key)))
    z = np.array(z, dtype=float)
    expect = g * (1 - 1 / g) ** n
    assert abs(z.mean() - expect) < 4 * z.std(ddof=1) / np.sqrt(z.size)


def test_grid_depends_only_on_the_set_of_pairs(O):
    """Algorithm 1 only sets bits (§3.3: no data conflict), so the DHLA is a
    function of the set of distinct pairs: independent of order, of
    duplicates and of how the stream is split into batches; and grids built
    from two halves merge by bitwise OR into the grid of the whole."""
    from paper_1803_11449_gb300 import traffic as T
    w = T.WORKLOADS["tiny"].with_(dirs=2, n=1 << 16)
    win = T.make_window(w, 3)
    p = O.params_from(w.sketch(), seed=17)
    ref = O.new_grid(p)
    O.update(p, ref, win.pairs)
    assert ref.any()

    rng = np.random.default_rng(0)
    shuffled = O.new_grid(p)
    O.update(p, shuffled, win.pairs[rng.permutation(len(win.pairs))])
    assert np.array_equal(shuffled, ref)

    dup = O.new_grid(p)
    O.update(p, dup, np.concatenate([win.pairs, win.pairs[::3]]))
    assert np.array_equal(dup, ref)

    split = O.new_grid(p)
    for part in np.array_split(win.pairs, 7):
        O.update(p, split, part)
    assert np.array_equal(split, ref)

    a, b = O.new_grid(p), O.new_grid(p)
    O.update(p, a, win.pairs[: len(win.pairs) // 3])
    O.update(p, b, win.pairs[len(win.pairs) // 3:])
    assert np.array_equal(a | b, ref)


def test_directions_key_on_src_and_dst(O):
    """Direction 0 records src hosts' peers, direction 1 dst hosts' peers: a
    scanner (one src, many dst) fills one estimator per row in direction 0
    only, with the popcount of a g-bit linear estimator of its peer count."""
    p = O.make_params(512, 4, 16, 8, 1024.0, seed=8, dirs=2)
    rng = np.random.default_rng(2)
    peers = rng.choice(2**32, size=3000, replace=False)
    scanner = 0x0B0B0B0B
    grid = O.new_grid(p)
    O.update(p, grid, _single_key_pairs(scanner, peers, direction=0))
    cells = _cells(O, p, grid)
    out_full = [int(np.unpackbits(cells[0, i, O.dh(p, 0, i, scanner)].view(np.uint8)).sum())
                for i in range(p.r)]
    assert min(out_full) > 0.9 * p.g
    # inbound: every peer is a distinct dst host with a single src -> 1 bit each
    in_pop = np.unpackbits(cells[1].view(np.uint8)).reshape(p.r, -1).sum(axis=1)
    assert in_pop.max() <= 3000 and in_pop.min() > 2800


def test_sz_counts_zeros_of_the_and(O):
    """§3.2, Definition 1: ULE(a0) is the bitwise AND of a0's r estimators
    and SZ(a0) its number of zero bits.  Estimators built here by hand: a
    common set of 100 bits in all r, plus bits of their own in each row (and
    a neighbour estimator full), so the AND keeps exactly the common 100."""
    p = O.make_params(512, 4, 16, 8, 1024.0, seed=31)
    a0 = 0x0A0B0C0D
    bits = np.zeros((p.r, 1 << p.k, p.g), dtype=np.uint8)
    common = np.arange(3, 503, 5)  # 100 bits
    for i in range(p.r):
        j = O.dh(p, 0, i, a0)
        bits[i, j, common] = 1
        bits[i, j, (common + 1 + i) % p.g] = 1   # row-specific bits
        bits[i, (j + 1) % (1 << p.k), :] = 1     # a full neighbour estimator
    grid = np.packbits(bits, axis=2, bitorder="little").view(np.uint32).reshape(-1).copy()
    assert O.sz(p, grid, 0, a0) == p.g - 100
    # a host none of whose estimators share a bit with a0's: SZ = g unless
    # it lands on a0's or a neighbour's estimator in every row
    b0 = 0x01020304
    cells = [O.dh(p, 0, i, b0) for i in range(p.r)]
    if all(bits[i, c].sum() == 0 for i, c in enumerate(cells)):
        assert O.sz(p, grid, 0, b0) == p.g

