"""Serving loop: many monitored links feeding packet batches, each admitted
link's DHLA resident on the device, a window closed every `window_pairs`
pairs of a link.

The engine does continuous batching: every step takes all batches that
have arrived for every admitted link that is not closing, cuts them at
window boundaries, and runs them in one batched update (sd_update_many);
the windows that filled during the step are closed together
(sd_close_many) by a closing thread while the next steps update the other
links.  Each link's handle has its own CUDA stream, so a close waits only
for the update that filled its window; the link itself rejoins the steps
once its report is on the host.  The batched update runs on a driver
handle of the same shape that holds no link (its bins serve every step);
the budget covers the driver, its bins for the largest round, and the
admitted links' sketches.  A link is admitted when its sketch fits the
budget; the others keep their batches queued, in arrival order, until a
slot frees (a link leaves).  All GPU work goes through the C ABI; this
module only schedules.

A link takes its pairs either as submitted batches (device tensors, queued
in order) or from a ring of pairs in device memory that a producer fills
(attach_ring, then advance by the pairs written); a step takes a ring's
pairs up to the window boundary or the ring's end, whichever comes first.

Each window report carries two latencies: the close (from the end of the
update that completed the window to the report on the host) and, when the
caller stamped its batches with arrival times, from the arrival of the
window's last batch to the report.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from concurrent.futures import ThreadPoolExecutor

from . import sd


@dataclasses.dataclass
class WindowReport:
    link: object
    window: int
    report: sd.Report
    close_s: float          # end of the completing update -> report on the host
    done_at: float          # perf_counter() when the report was on the host
    last_arrival: float     # arrival stamp of the window's last batch (0 if unstamped)


class _Link:
    def __init__(self, seed):
        self.seed = seed
        self.h = None                        # handle while admitted
        self.stream = None                   # the handle's CUDA stream
        self.filled = 0                      # pairs in the open window
        self.window = 0                      # index of the open window
        self.closing = False                 # its full window is being closed
        self.pending = collections.deque()   # [pairs tensor (2n words), arrival stamp]
        self.last_arrival = 0.0
        self.ring = None                     # device ring of pairs (2R words)
        self.head = 0                        # pairs written to the ring
        self.tail = 0                        # pairs applied from the ring

    def has_work(self):
        return bool(self.pending) or self.head > self.tail


class Server:
    """Serve links with per-link sketches of one shape (`workload`, a
    traffic.Workload or a dict of its sketch parameters).  hbm_budget is in
    bytes; bin_chunk_log2 sets the most pairs a link gives one binned round.
    The update is the library's default for the shape (mode 6, binned by
    bit plane, where one plane fits; `mode=5` asks for the slice binning):
    in mode 6 the links' rounds run on up to four lanes, each with the bins
    of one round (as many lanes as bin_bytes holds); in mode 5 a round
    takes as many links as bin_bytes of bins (default: half the budget)
    hold at their actual shares."""

    def __init__(self, workload, window_pairs: int, hbm_budget: int, device: int = 0,
                 bin_chunk_log2: int = 22, bin_bytes: int | None = None, cand_cap: int = 1 << 18,
                 stream=None, mode: int | None = None):
        import torch
        self.torch = torch
        self.workload = workload
        self.window_pairs = int(window_pairs)
        self.budget = int(hbm_budget)
        self.device = device
        self.stream = stream or torch.cuda.Stream(device=device)
        self.cand_cap = cand_cap
        self.bin_chunk_log2 = bin_chunk_log2
        self.links: dict = {}                  # every open link, admitted or waiting
        self.admitted: dict = {}               # link id -> _Link with a handle
        self.waiting = collections.deque()     # link ids waiting for admission
        self.used = 0
        self.reports: list[WindowReport] = []
        self.pairs_done = 0
        self.steps = 0
        self._bytes = None
        self._closer = ThreadPoolExecutor(1)
        self._closing = collections.deque()    # (future, link ids) in submission order
        self.bin_bytes = int(bin_bytes) if bin_bytes is not None else self.budget // 2
        self.driver = sd.sd_create(self._params(0, self.stream, cand_cap=1024))
        self.mode = sd.sd_get_tuning(self.driver).mode if mode is None else int(mode)
        if self.mode not in (5, 6):
            sd.sd_destroy(self.driver)
            self.driver = None
            self._closer.shutdown()
            raise ValueError("the engine's batched update is binned: mode 5 or 6")
        self._tune(self.driver, bin_batch_mib=max(1, self.bin_bytes >> 20))
        self.fixed = (sd.sd_device_bytes(self._params(0, self.stream, cand_cap=1024)) +
                      sd.sd_scratch_bytes(self.driver, 1 << 20))
        if self.fixed > self.budget:
            sd.sd_destroy(self.driver)
            self.driver = None
            self._closer.shutdown()
            raise ValueError(f"the engine's own memory ({self.fixed} bytes) is above the budget {self.budget}")
        self.used = self.fixed
        self._empty = torch.zeros(0, dtype=torch.int32, device=f"cuda:{device}")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.shutdown()
        return False

    # ---------------------------------------------------------- admission
    def _tune(self, h, **extra):
        if self.mode == 6:
            sd.sd_set_tuning(h, mode=6, plane_round_log2=self.bin_chunk_log2, **extra)
        else:
            sd.sd_set_tuning(h, mode=5, bin_chunk_log2=self.bin_chunk_log2, **extra)

    def _params(self, seed, stream, cand_cap=None):
        return sd.params_for(self.workload, seed, device=self.device, cand_cap=cand_cap or self.cand_cap,
                             cuda_stream=stream.cuda_stream)

    def link_bytes(self) -> int:
        """Device bytes of one link's handle (its DHLA and close buffers)."""
        if self._bytes is None:
            self._bytes = sd.sd_device_bytes(self._params(0, self.stream))
        return self._bytes

    def _admit(self, lid) -> None:
        L = self.links[lid]
        L.stream = self.torch.cuda.Stream(device=self.device)
        L.h = sd.sd_create(self._params(L.seed, L.stream))
        self._tune(L.h)
        self.admitted[lid] = L
        self.used += self.link_bytes()

    def _admit_waiting(self) -> None:
        while self.waiting and self.used + self.link_bytes() <= self.budget:
            self._admit(self.waiting.popleft())

    def open_link(self, link_id, seed: int) -> bool:
        """Open `link_id` with hash seed `seed`; it is admitted now if its
        sketch fits the budget and no link waits before it, else it queues.
        Returns True when admitted now."""
        if link_id in self.links:
            raise ValueError(f"link {link_id!r} is already open")
        if self.fixed + self.link_bytes() > self.budget:
            raise ValueError(f"one link needs {self.link_bytes()} bytes; the budget {self.budget} "
                             f"leaves {self.budget - self.fixed}")
        self.links[link_id] = _Link(seed)
        self.waiting.append(link_id)
        self._admit_waiting()
        return link_id in self.admitted

    def close_link(self, link_id) -> WindowReport | None:
        """Feed the link's queued pairs, close its open window (if it holds
        pairs), free its slot and admit waiting links.  A link that was
        never admitted is dropped with its queue."""
        L = self.links[link_id]
        out = None
        if L.h is not None:
            while L.closing and self._closing:
                self._collect(block=True)
            while L.has_work():
                self._feed([link_id], flush=True)
            if L.filled:
                reps, close_s, done_at = self._close_now([L.h])
                out = WindowReport(link_id, L.window, reps[0], close_s, done_at, L.last_arrival)
                self.reports.append(out)
        self._release(link_id)
        return out

    def _release(self, link_id) -> None:
        """Free the link's handle (if admitted) or its place in the queue,
        forget the link and admit waiting links."""
        L = self.links.pop(link_id)
        if L.h is not None:
            sd.sd_destroy(L.h)
            L.h = None
            del self.admitted[link_id]
            self.used -= self.link_bytes()
        else:
            self.waiting.remove(link_id)
        self._admit_waiting()

    # --------------------------------------------------------------- work
    def submit(self, link_id, pairs, arrival: float = 0.0) -> None:
        """Queue a batch of (src, dst) pairs (a device tensor of 2n 4-byte
        words, kept alive by the engine until applied) for an open link."""
        if pairs.numel() % 2:
            raise ValueError("a batch holds whole (src, dst) pairs")
        if pairs.numel():
            if pairs.is_cuda:
                pairs.record_stream(self.stream)  # read on the engine's stream
            self.links[link_id].pending.append([pairs, arrival])

    def attach_ring(self, link_id, ring) -> None:
        """Make a device tensor of 2R 4-byte words (R pairs) the link's
        input ring; the producer writes pair j to slot j mod R.  A slot is
        free again once a step has enqueued the update that reads it, so the
        producer writes on the engine's stream (`Server.stream`, where the
        batched updates run) or orders its writes after that stream."""
        if ring.numel() % 2 or not ring.numel():
            raise ValueError("a ring holds a positive number of (src, dst) pairs")
        L = self.links[link_id]
        if L.pending:
            raise ValueError("the link already takes submitted batches")
        L.ring, L.head, L.tail = ring, 0, 0

    def advance(self, link_id, n_pairs: int, arrival: float = 0.0) -> None:
        """The producer wrote `n_pairs` more pairs to the link's ring."""
        L = self.links[link_id]
        if L.head + n_pairs - L.tail > L.ring.numel() // 2:
            raise ValueError("ring overrun: the producer is a full ring ahead of the engine")
        L.head += int(n_pairs)
        L.last_arrival = arrival

    def pending_pairs(self) -> int:
        return sum(sum(b.numel() // 2 for b, _ in L.pending) + L.head - L.tail for L in self.links.values())

    def _feed(self, lids, flush=False):
        """Take each link's queued pairs up to the end of its open window
        (a batch that crosses the boundary is split, its rest waits) and
        apply them in one batched update.  Returns the links whose window
        is full; with flush, closes them here (the caller's thread)."""
        hs, bufs, full = [self.driver], [self._empty], []
        for lid in lids:
            L = self.links[lid]
            parts = []
            if L.ring is not None and L.head > L.tail and L.filled < self.window_pairs:
                R = L.ring.numel() // 2
                pos = L.tail % R
                m = min(L.head - L.tail, self.window_pairs - L.filled, R - pos)
                parts.append(L.ring[2 * pos: 2 * (pos + m)])
                L.tail += m
                L.filled += m
            while L.pending and L.filled < self.window_pairs:
                b, at = L.pending[0]
                n = b.numel() // 2
                room = self.window_pairs - L.filled
                if n <= room:
                    parts.append(b)
                    L.pending.popleft()
                    L.filled += n
                    L.last_arrival = at
                else:
                    parts.append(b[: 2 * room])
                    L.pending[0][0] = b[2 * room:]
                    L.filled += room
                    L.last_arrival = at
            if parts:
                with self.torch.cuda.stream(self.stream):
                    buf = parts[0] if len(parts) == 1 else self.torch.cat(parts)
                hs.append(L.h)
                bufs.append(buf)
                self.pairs_done += buf.numel() // 2
            if L.filled >= self.window_pairs:
                full.append(lid)
        if len(hs) > 1:
            sd.sd_update_many(hs, bufs)
        if flush and full:
            self._finish(full, *self._close_now([self.links[lid].h for lid in full]))
        return full

    @staticmethod
    def _close_now(handles):
        """Close the windows of `handles` (each handle's stream already
        waits for the update that filled it).  Returns (reports, close
        seconds, completion time)."""
        for h in handles:
            sd.sd_sync(h)  # the completing update is done: the close latency starts here
        t0 = time.perf_counter()
        reps = sd.sd_close_many(handles)
        t1 = time.perf_counter()
        return reps, t1 - t0, t1

    def _finish(self, lids, reps, close_s, done_at) -> list[WindowReport]:
        out = []
        for lid, rep in zip(lids, reps):
            L = self.links[lid]
            out.append(WindowReport(lid, L.window, rep, close_s, done_at, L.last_arrival))
            L.window += 1
            L.filled = 0
            L.closing = False
        self.reports += out
        return out

    def _collect(self, block=False) -> list[WindowReport]:
        """Reports of the closes that have finished (block: wait for the
        oldest one when none has)."""
        out = []
        while self._closing and (self._closing[0][0].done() or (block and not out)):
            fut, lids = self._closing.popleft()
            try:
                res = fut.result()
            except BaseException:
                # the close failed: its links hold a full window, no longer
                # closing (a later close of the link tries again)
                for lid in lids:
                    self.links[lid].closing = False
                raise
            out += self._finish(lids, *res)
        return out

    def step(self) -> list[WindowReport]:
        """One engine step: collect finished closes, run one batched update
        over every ready link's arrived pairs, and hand the windows it
        filled to the closing thread.  With nothing to update, wait for the
        oldest close in flight instead."""
        self.steps += 1
        out = self._collect()
        ready = [lid for lid, L in self.admitted.items() if not L.closing and L.has_work()]
        if not ready:
            if self._closing:
                out += self._collect(block=True)
            return out
        full = self._feed(ready)
        if full:
            for lid in full:
                self.links[lid].closing = True
            fut = self._closer.submit(self._close_now, [self.links[lid].h for lid in full])
            self._closing.append((fut, full))
        return out

    def drain(self) -> list[WindowReport]:
        """Steps until no admitted link has queued pairs and no close is
        in flight."""
        out = []
        while self._closing or any(L.has_work() for L in self.admitted.values()):
            out += self.step()
        return out

    def shutdown(self) -> list[WindowReport]:
        """Close every link (admitted links first, then those that get
        admitted as slots free) and free every handle.  A close or update
        that fails does not stop the others: its link is freed without a
        report, and the first error is raised once everything is freed."""
        out, err = [], None
        while self._closing:
            try:
                out += self._collect(block=True)
            except Exception as e:  # noqa: BLE001 - re-raised below
                err = err or e
        while self.links:
            lid = next(iter(self.admitted), None)
            if lid is None:
                self._admit_waiting()
                lid = next(iter(self.admitted))
            try:
                r = self.close_link(lid)
            except Exception as e:  # noqa: BLE001 - re-raised below
                err = err or e
                if lid in self.links:
                    self.links[lid].pending.clear()
                    self._release(lid)
                continue
            if r:
                out.append(r)
        if self.driver is not None:
            sd.sd_destroy(self.driver)
            self.driver = None
            self.used -= self.fixed
            self._closer.shutdown()
        if err is not None:
            raise err
        return out
