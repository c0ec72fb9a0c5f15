"""Host logic of the serving engine on CPU: window cuts, ring wrap-around,
admission under a budget, and the closing thread, with the C-ABI calls
replaced by a recording fake (no GPU).  Each fake close returns the pairs
its handle received since the previous close, so every window can be
checked to be exactly `window_pairs` consecutive pairs of its link."""
import contextlib

import numpy as np
import pytest
import torch

from paper_1803_11449_gb300 import serving


class _FakeSd:
    """The subset of the binding the engine calls."""

    class Handle:
        def __init__(self, seed):
            self.seed = seed
            self.got = []

    def __init__(self, link_bytes=100, scratch=1000):
        self.link_bytes = link_bytes
        self.scratch = scratch
        self.created = 0
        self.live = 0
        self.tuned = []

    def params_for(self, workload, seed, **kw):
        return dict(seed=seed, **kw)

    def sd_device_bytes(self, p):
        return self.link_bytes

    def sd_create(self, p):
        self.created += 1
        self.live += 1
        return self.Handle(p["seed"])

    def sd_destroy(self, h):
        self.live -= 1

    def sd_set_tuning(self, h, **kw):
        assert kw["mode"] in (5, 6)
        self.tuned.append(kw)

    def sd_get_tuning(self, h):
        class _T:
            mode = 6
        return _T()

    def sd_scratch_bytes(self, h, links):
        return self.scratch

    def sd_sync(self, h):
        pass

    def sd_update_many(self, hs, bufs):
        assert len(set(map(id, hs))) == len(hs)
        for h, b in zip(hs, bufs):
            h.got.append(b.numpy().reshape(-1, 2).copy())

    def sd_close_many(self, hs):
        out = []
        for h in hs:
            out.append(np.concatenate(h.got) if h.got else np.zeros((0, 2), np.int32))
            h.got = []
        return out

    def sd_close_window(self, h):
        return self.sd_close_many([h])[0]


@pytest.fixture
def fake(monkeypatch):
    class _Stream:
        cuda_stream = 0

    real_zeros = torch.zeros
    monkeypatch.setattr(torch.cuda, "Stream", lambda device=None: _Stream())
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch, "zeros", lambda *a, **k: real_zeros(*a, **{x: v for x, v in k.items() if x != "device"}))
    f = _FakeSd()
    monkeypatch.setattr(serving, "sd", f)
    return f


def _stream(n, link):
    x = np.arange(2 * n, dtype=np.int64).reshape(n, 2) + (link << 24)
    return x.astype(np.int32)


def _windows(srv, link):
    got = sorted((r.window, r.report) for r in srv.reports if r.link == link)
    return [w for _, w in got]


def test_batches_cut_at_window_boundaries(fake):
    W = 1000
    srv = serving.Server({}, W, hbm_budget=10_000)
    streams = {i: _stream(3 * W + 123, i) for i in range(3)}
    for i in streams:
        assert srv.open_link(i, seed=i)
    rng = np.random.default_rng(1)
    at = {i: 0 for i in streams}
    while any(at[i] < len(streams[i]) for i in streams):
        for i in streams:
            m = int(min(len(streams[i]) - at[i], rng.integers(1, 700)))
            if m:
                srv.submit(i, torch.from_numpy(streams[i][at[i]:at[i] + m].reshape(-1)))
                at[i] += m
        srv.step()
    srv.drain()
    srv.shutdown()
    for i, s in streams.items():
        ws = _windows(srv, i)
        assert [len(w) for w in ws] == [W, W, W, 123]
        assert np.array_equal(np.concatenate(ws), s)
    assert fake.live == 0 and srv.used == 0


def test_ring_wraps_and_rejects_overrun(fake):
    W, R = 1000, 777
    srv = serving.Server({}, W, hbm_budget=10_000)
    srv.open_link("a", seed=1)
    ring = torch.zeros(2 * R, dtype=torch.int32)
    srv.attach_ring("a", ring)
    s = _stream(2500, 5)
    at = 0
    while at < len(s):
        L = srv.links["a"]
        c = int(min(R - (L.head - L.tail), len(s) - at, 500))
        for q in range(c):  # the producer writes pair j to slot j mod R
            ring[2 * ((at + q) % R): 2 * ((at + q) % R) + 2] = torch.from_numpy(s[at + q])
        srv.advance("a", c)
        at += c
        srv.step()
    with pytest.raises(ValueError):
        srv.advance("a", R + 1)
    srv.drain()
    srv.shutdown()
    ws = _windows(srv, "a")
    assert [len(w) for w in ws] == [1000, 1000, 500]
    assert np.array_equal(np.concatenate(ws), s)


def test_admission_order_and_budget(fake):
    srv = serving.Server({}, 100, hbm_budget=(100 + 1000) + 2 * 100)  # the engine (sketch + bins), then two links
    assert srv.open_link("a", 1) and srv.open_link("b", 2)
    assert not srv.open_link("c", 3) and not srv.open_link("d", 4)
    srv.submit("c", torch.from_numpy(_stream(50, 3).reshape(-1)))  # queued while waiting
    assert list(srv.waiting) == ["c", "d"]
    srv.close_link("b")
    assert "c" in srv.admitted and list(srv.waiting) == ["d"]
    srv.close_link("d")  # never admitted: dropped with its queue
    srv.drain()
    srv.shutdown()
    assert len(_windows(srv, "c")[0]) == 50 and fake.live == 0
    with pytest.raises(ValueError):
        serving.Server({}, 100, hbm_budget=999)


def test_server_as_context_manager_releases_everything(fake):
    with serving.Server({}, 10, hbm_budget=10_000) as srv:
        srv.open_link("a", 1)
        srv.submit("a", torch.from_numpy(_stream(25, 1).reshape(-1)))
        srv.step()
    assert fake.live == 0 and srv.used == 0 and not srv.links
    assert [len(w) for w in _windows(srv, "a")] == [10, 10, 5]


def test_failed_close_raises_and_shutdown_frees_everything(fake):
    """A close that fails on the closing thread (an error from the library,
    injected here on the host) is raised by the step that collects it; its
    links are not left waiting for a close that will never come, and
    shutdown frees every handle, then raises the first error."""
    real = fake.sd_close_many
    calls = {"n": 0}

    def flaky(hs):
        calls["n"] += 1
        if calls["n"] == 2:
            raise RuntimeError("injected close failure")
        return real(hs)

    fake.sd_close_many = flaky
    W = 100
    srv = serving.Server({}, W, hbm_budget=10_000)
    for lid in ("a", "b"):
        srv.open_link(lid, seed=1)
    with pytest.raises(RuntimeError, match="injected"):
        for k in range(20):
            for lid in ("a", "b"):
                srv.submit(lid, torch.from_numpy(_stream(W, k).reshape(-1)))
            srv.step()
        srv.drain()
    assert not any(L.closing for L in srv.links.values())
    srv.submit("a", torch.from_numpy(_stream(30, 99).reshape(-1)))
    srv.shutdown()  # the other closes succeed again
    assert fake.live == 0 and srv.used == 0 and not srv.links

    fake.sd_close_many = lambda hs: (_ for _ in ()).throw(RuntimeError("injected close failure"))
    srv = serving.Server({}, W, hbm_budget=10_000)
    for lid in ("a", "b", "c"):
        srv.open_link(lid, seed=2)
        srv.submit(lid, torch.from_numpy(_stream(W // 2, 7).reshape(-1)))
    with pytest.raises(RuntimeError, match="injected"):
        srv.shutdown()
    assert fake.live == 0 and srv.used == 0 and not srv.links and srv.driver is None

