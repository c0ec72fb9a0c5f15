"""The serving engine (continuous batching over many links, admission
under an HBM budget): every window a link closes in the mix must report
exactly what the oracle gives for that window of that link alone, and what
the same link reports when it is served alone."""
import numpy as np
import pytest

from paper_1803_11449_gb300 import traffic as T

pytestmark = pytest.mark.gpu

WINDOW = 1 << 16


@pytest.fixture(scope="module")
def mods():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1803_11449_gb300 import build as b
    b.build()
    from paper_1803_11449_gb300 import sd, serving
    sd.lib()
    return sd, serving


def _workload():
    return T.WORKLOADS["tiny"].with_(dirs=2, theta=512, planted=4, planted_c=("uniform", 3000, 6000))


def _streams():
    w = _workload()
    lens = [3 * WINDOW + 1234, 2 * WINDOW, 150_001, WINDOW - 7, 4 * WINDOW + 999, 90_000]
    seeds = [500 + i for i in range(len(lens))]
    pairs = [T.make_window(w.with_(n=n), s, n=n).pairs for n, s in zip(lens, seeds)]
    return w, seeds, pairs


def _batches(rng, n):
    """Cut a stream of n pairs into batches of 1 .. 20000 pairs."""
    cuts, at = [], 0
    while at < n:
        m = int(min(n - at, rng.integers(1, 20001)))
        cuts.append((at, at + m))
        at += m
    return cuts


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1).view(np.int32)).cuda()


def _expected(O, w, seed, pairs):
    """Oracle reports of consecutive windows of WINDOW pairs (the last one
    partial), each over a fresh DHLA."""
    out = []
    for a in range(0, len(pairs), WINDOW):
        op = O.params_from(w.sketch(), seed=seed)
        og = O.new_grid(op)
        O.update(op, og, pairs[a:a + WINDOW])
        out.append(O.close_window(op, og))
    return out


def _same(rep, ref):
    assert rep.n_cand == ref["n_cand"]
    assert [rep.dir_flags(d) for d in range(2)] == ref["flags"]
    assert np.array_equal(rep.zr, ref["zr"]) and rep.psi == ref["psi"]
    assert np.array_equal(rep.hits["ip"], ref["ip"]) and np.array_equal(rep.hits["sz"], ref["sz"])
    assert np.array_equal(rep.hits["dir"], ref["dir"]) and np.array_equal(rep.hits["est"], ref["est"])


def _serve(mods, w, seeds, pairs, links, budget_links, rng, chunk_log2=21, mode=None):
    sd, serving = mods
    srv = serving.Server(w, WINDOW, hbm_budget=1 << 40, bin_chunk_log2=chunk_log2, mode=mode)
    srv.budget = srv.fixed + budget_links * srv.link_bytes()
    for i in links:
        srv.open_link(i, seeds[i])
    todo = {i: _batches(rng, len(pairs[i])) for i in links}
    dev = {i: _dev(pairs[i]) for i in links}
    # interleave the links' batches in a random order, a step every few batches
    order = [i for i in links for _ in todo[i]]
    rng.shuffle(order)
    nxt = {i: 0 for i in links}
    for j, i in enumerate(order):
        a, b = todo[i][nxt[i]]
        nxt[i] += 1
        srv.submit(i, dev[i][2 * a:2 * b], arrival=float(j))
        if j % 5 == 4:
            srv.step()
        if nxt[i] == len(todo[i]) and i == links[0]:
            srv.close_link(i)  # the first link leaves early: a waiting link takes its slot
    srv.drain()
    srv.shutdown()
    assert not srv.links and srv.used == 0
    got = {}
    for r in srv.reports:
        got.setdefault(r.link, {})[r.window] = r
    return srv, got


@pytest.mark.parametrize("mode,chunk_log2", [(6, 21), (6, 13), (5, 21)])
def test_served_windows_equal_oracle_and_alone(mods, O, mode, chunk_log2):
    """Plane rounds (mode 6; with 2^13-pair rounds a batch of a link takes
    several) and slice-binned rounds (mode 5) of the batched update."""
    w, seeds, pairs = _streams()
    rng = np.random.default_rng(11)
    links = list(range(len(pairs)))
    srv, got = _serve(mods, w, seeds, pairs, links, budget_links=3, rng=rng, chunk_log2=chunk_log2, mode=mode)
    assert srv.mode == mode
    assert srv.pairs_done == sum(len(p) for p in pairs)
    n_hits = 0
    for i in links:
        ref = _expected(O, w, seeds[i], pairs[i])
        assert sorted(got[i]) == list(range(len(ref)))
        for k, rr in enumerate(ref):
            rep = got[i][k].report
            assert rep.n_pairs == min(WINDOW, len(pairs[i]) - k * WINDOW)
            _same(rep, rr)
            n_hits += len(rep.hits)
    assert n_hits > 0
    # the link with the most windows, served alone with other batch cuts,
    # reports the same windows
    _, alone = _serve(mods, w, seeds, pairs, [4], budget_links=1, rng=np.random.default_rng(3), mode=mode)
    for k, r in alone[4].items():
        assert np.array_equal(r.report.hits, got[4][k].report.hits)
        assert r.report.n_cand == got[4][k].report.n_cand


@pytest.mark.parametrize("mode", [5, 6])
def test_admission_respects_budget(mods, mode):
    sd, serving = mods
    w = _workload()
    bins = 64 << 20
    probe = serving.Server(w, WINDOW, hbm_budget=1 << 40, bin_bytes=bins, mode=mode)
    fixed, lb = probe.fixed, probe.link_bytes()
    scratch = sd.sd_scratch_bytes(probe.driver, 1 << 20)
    if mode == 5:
        assert fixed >= scratch >= bins
    else:  # the bins of one round of 2^22 pairs: at least 9/8 of its 2^23 keys
        assert fixed >= scratch >= 4 * (9 << 20)
    probe.shutdown()
    grid = 2 * 4 * sd.sd_grid_words(sd.params_for(w, 1))
    assert fixed > 0 and lb > 2 * grid  # the DHLA and its plane-major copy
    with pytest.raises(ValueError):
        serving.Server(w, WINDOW, hbm_budget=fixed - 1, bin_bytes=bins, mode=mode)  # not even the engine fits
    srv = serving.Server(w, WINDOW, hbm_budget=fixed + lb - 1, bin_bytes=bins, mode=mode)
    with pytest.raises(ValueError):
        srv.open_link("a", 1)  # one link does not fit
    srv.shutdown()
    srv = serving.Server(w, WINDOW, hbm_budget=fixed + 2 * lb, bin_bytes=bins, mode=mode)
    assert srv.open_link("a", 1) and srv.open_link("b", 2)
    assert not srv.open_link("c", 3)
    assert list(srv.waiting) == ["c"] and srv.used == fixed + 2 * lb
    srv.close_link("a")
    assert "c" in srv.admitted and not srv.waiting
    srv.shutdown()
    assert srv.used == 0


def test_ring_fed_links_equal_oracle(mods, O):
    """Links fed through device rings of R pairs (R not a multiple of the
    window, so windows and ring wraps fall at different places)."""
    import torch
    sd, serving = mods
    w, seeds, pairs = _streams()
    links = [0, 2, 4]
    R = 50_000
    srv = serving.Server(w, WINDOW, hbm_budget=1 << 40)
    rings, dev, at = {}, {}, {}
    for i in links:
        srv.open_link(i, seeds[i])
        rings[i] = torch.zeros(2 * R, dtype=torch.int32, device="cuda")
        srv.attach_ring(i, rings[i])
        dev[i] = _dev(pairs[i])
        at[i] = 0
    rng = np.random.default_rng(5)
    while any(at[i] < len(pairs[i]) for i in links):
        for i in links:
            L = srv.links[i]
            free = R - (L.head - L.tail)
            c = int(min(free, len(pairs[i]) - at[i], rng.integers(1, 30001)))
            if c <= 0:
                continue
            # the producer writes pairs at..at+c-1 into ring slots (at mod R), wrapping
            with torch.cuda.stream(srv.stream):
                done = 0
                while done < c:
                    pos = (at[i] + done) % R
                    m = min(c - done, R - pos)
                    rings[i][2 * pos:2 * (pos + m)].copy_(dev[i][2 * (at[i] + done):2 * (at[i] + done + m)])
                    done += m
            srv.advance(i, c)
            at[i] += c
        srv.step()
    srv.drain()
    srv.shutdown()
    got = {}
    for r in srv.reports:
        got.setdefault(r.link, {})[r.window] = r.report
    for i in links:
        ref = _expected(O, w, seeds[i], pairs[i])
        assert sorted(got[i]) == list(range(len(ref)))
        for k, rr in enumerate(ref):
            _same(got[i][k], rr)
    with pytest.raises(ValueError):
        srv2 = serving.Server(w, WINDOW, hbm_budget=1 << 40)
        srv2.open_link("x", 1)
        srv2.attach_ring("x", rings[0])
        srv2.advance("x", R + 1)


def test_serving_full_size_windows_sampled(mods, O):
    """Serving at the benchmark's sizes: core-link sketches, 2^26-pair
    windows, batches uniform in [64K, 4M] pairs, a 2 GiB budget with half for
    bins and 2^22-pair shares; a link carrying a DDoS victim (2M spoofed
    sources) and a plain link are served together and each link's first
    window equals the oracle's report for those pairs alone."""
    import torch
    sd, serving = mods
    W = 1 << 26
    w = T.WORKLOADS["core"].with_(n=W, planted=100)
    wins = [T.make_window(w, T.window_seed(4, link=i)).pairs for i in range(2)]
    rng = np.random.default_rng(9)
    victim = np.uint32(0xC0A80001)
    pos = rng.choice(W, size=2_000_000, replace=False)
    wins[0][pos, 0] = T.ip_of(0x7000_0000, np.arange(2_000_000), 12345)
    wins[0][pos, 1] = victim
    srv = serving.Server(w, W, hbm_budget=2 << 30)
    seeds = [T.window_seed(4, link=i) for i in range(2)]
    for i in range(2):
        srv.open_link(i, seeds[i])
    dev = [_dev(p) for p in wins]
    at = [0, 0]
    while min(at) < W:
        for i in range(2):
            m = int(min(W - at[i], rng.integers(1 << 16, (1 << 22) + 1)))
            if m:
                srv.submit(i, dev[i][2 * at[i]:2 * (at[i] + m)])
                at[i] += m
        srv.step()
    srv.drain()
    srv.shutdown()
    got = {r.link: r.report for r in srv.reports if r.window == 0}
    for i in range(2):
        _, ref = O_close(O, w, wins[i], seeds[i])
        _same(got[i], ref)
    hits0 = got[0].hits
    assert ((hits0["ip"] == victim) & (hits0["dir"] == 1)).any()


def O_close(O, w, pairs, seed):
    op = O.params_from(w.sketch(), seed=seed)
    og = O.new_grid(op)
    O.update(op, og, pairs)
    return og, O.close_window(op, og)
