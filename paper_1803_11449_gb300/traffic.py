"""Seeded synthetic packet-pair traffic for super-point detection.

This module draws the inputs only: ``(src, dst)`` uint32 IP pairs shaped like
a core-link window (Zipf-distributed sources, uniform destinations, planted
super points with an exact number of distinct peers, shuffled order).  It
holds none of the detection method's arithmetic, so both the CUDA path and
the CPU oracle can be fed from it.

The CAIDA OC192 trace used in the paper (§5) is not available; these
workloads stand in for it.  Every draw comes from ``numpy.random.Generator``
(PCG64) seeded by the caller, so a (workload, seed) pair always yields the
same window.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Index ranges of the host roles before mixing; disjoint ranges give disjoint
# IP sets because the mixer below is a bijection of uint32.
_ROLE_SRC = 0x00000000
_ROLE_DST = 0x20000000
_ROLE_PLANTED = 0x70000000
_ROLE_PEER = 0x80000000


@dataclasses.dataclass(frozen=True)
class Workload:
    """Sketch parameters plus the traffic recipe of one window."""
    name: str
    # sketch (g bits per estimator, r rows, 2^k estimators per row, alpha)
    g: int
    r: int
    k: int
    alpha: int
    theta: float
    dirs: int
    # traffic
    n: int                      # pairs in the window
    src_pool: int               # distinct natural sources
    zipf_s: float               # Zipf exponent of the source ranks
    dst_pool: int | None        # distinct natural destinations (None: uniform over 2^32)
    planted: int                # planted super points
    planted_c: tuple            # ("uniform"|"loguniform", lo, hi) distinct peers each
    pkts_per_flow: int = 1      # packets per natural flow
    planted_share: float = 0.5  # planted pairs are scaled to at most this share of n

    def sketch(self) -> dict:
        return dict(g=self.g, r=self.r, k=self.k, alpha=self.alpha, theta=self.theta,
                    dirs=self.dirs)

    def with_(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


def default_alpha(k: int, r: int) -> int:
    """Smallest alpha with (r-2)*alpha + k >= 32 (the §3.3 restriction)."""
    return -(-(32 - k) // (r - 2))


WORKLOADS = {
    # 1 window of 2^20 pairs; 2^16 Zipf(1.1) sources, uniform 32-bit dsts;
    # 20 planted with 1,500-4,000 peers; 4 x 2^12 estimators of 256 bits.
    "tiny": Workload("tiny", g=256, r=4, k=12, alpha=10, theta=1024, dirs=1, n=1 << 20,
                     src_pool=1 << 16, zipf_s=1.1, dst_pool=None, planted=20,
                     planted_c=("uniform", 1500, 4000)),
    # core-link window: 2^26 pairs, 2^24 Zipf(1.05) sources, 2^26 dsts, 500
    # planted log-uniform in [1,024, 200,000]; 4 x 2^16 x 512 bits, both dirs.
    "core": Workload("core", g=512, r=4, k=16, alpha=8, theta=1024, dirs=2, n=1 << 26,
                     src_pool=1 << 24, zipf_s=1.05, dst_pool=1 << 26, planted=500,
                     planted_c=("loguniform", 1024, 200_000)),
    # the paper's own parameters (§5: g=1024, r=5, alpha=6, k=14) on core traffic
    "paper": Workload("paper", g=1024, r=5, k=14, alpha=6, theta=1024, dirs=2, n=1 << 26,
                      src_pool=1 << 24, zipf_s=1.05, dst_pool=1 << 26, planted=500,
                      planted_c=("loguniform", 1024, 200_000)),
    # stress: 2^30 pairs, 2^28 Zipf(1.0) sources, 2^30 dsts, 10^4 planted,
    # 4 x 2^18 x 1024 bits (128 MiB per direction); 8 packets per flow.
    "stress": Workload("stress", g=1024, r=4, k=18, alpha=7, theta=1024, dirs=2, n=1 << 30,
                       src_pool=1 << 28, zipf_s=1.0, dst_pool=1 << 30, planted=10_000,
                       planted_c=("loguniform", 1024, 10_000_000), pkts_per_flow=8),
}


def mix32(x: np.ndarray) -> np.ndarray:
    """A bijection of uint32 (xor-shift / odd-multiply rounds), used to turn
    role indices into scattered IP addresses."""
    x = np.asarray(x, dtype=np.uint32).copy()
    x ^= x >> np.uint32(16)
    x *= np.uint32(0x7FEB352D)
    x ^= x >> np.uint32(15)
    x *= np.uint32(0x846CA68B)
    x ^= x >> np.uint32(16)
    return x


def ip_of(role: int, idx: np.ndarray, salt: int) -> np.ndarray:
    idx = np.asarray(idx, dtype=np.uint64)
    raw = ((np.uint64(role) + idx) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    return mix32(raw ^ np.uint32(salt))


def zipf_ranks(rng: np.random.Generator, size: int, N: int, s: float) -> np.ndarray:
    """Ranks in [1, N] with P(k) proportional to k^-s, by rejection-inversion
    (Hörmann and Derflinger, "Rejection-inversion to generate variates from
    monotone discrete distributions", 1996).  Vectorised: rejected draws are
    redrawn until none remain."""
    one_s = 1.0 - s

    def helper1(x):  # log1p(x)/x, -> 1 at 0
        out = np.ones_like(x)
        nz = np.abs(x) > 1e-8
        out[nz] = np.log1p(x[nz]) / x[nz]
        return out

    def helper2(x):  # expm1(x)/x, -> 1 at 0
        out = np.ones_like(x)
        nz = np.abs(x) > 1e-8
        out[nz] = np.expm1(x[nz]) / x[nz]
        return out

    def H(x):  # an antiderivative of x^-s
        lx = np.log(x)
        return helper2(one_s * lx) * lx

    def Hinv(u):
        t = np.maximum(u * one_s, -1.0)
        return np.exp(helper1(t) * u)

    def h(x):
        return np.exp(-s * np.log(x))

    f = lambda v: np.array([v], dtype=np.float64)  # noqa: E731
    hx1 = H(f(1.5))[0] - 1.0
    hN = H(f(N + 0.5))[0]
    shift = 2.0 - Hinv(H(f(2.5)) - h(f(2.0)))[0]
    out = np.empty(size, dtype=np.int64)
    todo = np.arange(size, dtype=np.int64)
    while todo.size:
        u = hN + rng.random(todo.size) * (hx1 - hN)
        x = Hinv(u)
        kk = np.clip(np.floor(x + 0.5), 1, N)
        ok = (kk - x <= shift) | (u >= H(kk + 0.5) - h(kk))
        out[todo[ok]] = kk[ok].astype(np.int64)
        todo = todo[~ok]
    return out


@dataclasses.dataclass
class Window:
    pairs: np.ndarray          # uint32 [n, 2] (src, dst)
    planted_ip: np.ndarray     # uint32 [P]
    planted_dir: np.ndarray    # uint8 [P]: 0 = scanner-like src, 1 = victim-like dst
    planted_c: np.ndarray      # int64 [P]: exact distinct peers
    workload: Workload
    seed: int


def _planted_counts(rng, w: Workload, n: int) -> np.ndarray:
    kind, lo, hi = w.planted_c
    if w.planted == 0:
        return np.zeros(0, dtype=np.int64)
    if kind == "uniform":
        c = rng.integers(lo, hi + 1, size=w.planted)
    else:
        c = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=w.planted))).astype(np.int64)
    budget = int(w.planted_share * n)
    tot = int(c.sum())
    if tot > budget:  # keep the window size fixed: shrink all planted degrees alike
        c = np.maximum(1, (c * (budget / tot)).astype(np.int64))
    return c.astype(np.int64)


def make_window(w: Workload | str, seed: int, n: int | None = None) -> Window:
    """Draw one window of ``n`` pairs (default ``w.n``)."""
    if isinstance(w, str):
        w = WORKLOADS[w]
    n = w.n if n is None else int(n)
    rng = np.random.default_rng(seed)
    salt = int(rng.integers(0, 2**32))
    c = _planted_counts(rng, w, n)
    P = c.size
    keys = ip_of(_ROLE_PLANTED, np.arange(P), salt)
    pdir = (np.arange(P) % 2).astype(np.uint8) if w.dirs == 2 else np.zeros(P, dtype=np.uint8)
    npl = int(c.sum())
    peers = ip_of(_ROLE_PEER, np.arange(npl), salt)
    owner = np.repeat(np.arange(P), c)
    okey = keys[owner]
    odir = pdir[owner]
    psrc = np.where(odir == 0, okey, peers)
    pdst = np.where(odir == 0, peers, okey)

    n_nat = n - npl
    m = max(1, w.pkts_per_flow)
    flows = -(-n_nat // m)
    src = ip_of(_ROLE_SRC, zipf_ranks(rng, flows, w.src_pool, w.zipf_s) - 1, salt)
    if w.dst_pool is None:
        dst = rng.integers(0, 2**32, size=flows, dtype=np.uint64).astype(np.uint32)
    else:
        dst = ip_of(_ROLE_DST, rng.integers(0, w.dst_pool, size=flows), salt)
    if m > 1:
        src = np.repeat(src, m)[:n_nat]
        dst = np.repeat(dst, m)[:n_nat]

    pairs = np.empty((n, 2), dtype=np.uint32)
    pairs[:npl, 0] = psrc
    pairs[:npl, 1] = pdst
    pairs[npl:, 0] = src
    pairs[npl:, 1] = dst
    pairs = pairs[rng.permutation(n)]
    return Window(pairs=np.ascontiguousarray(pairs), planted_ip=keys, planted_dir=pdir,
                  planted_c=c, workload=w, seed=seed)


def exact_cardinality(pairs: np.ndarray, direction: int):
    """Distinct peers per host: (hosts, counts), for direction 0 (src keyed)
    or 1 (dst keyed).  Exact, by sorting the 64-bit (key, peer) values."""
    key = pairs[:, direction].astype(np.uint64)
    peer = pairs[:, 1 - direction].astype(np.uint64)
    u = np.unique((key << np.uint64(32)) | peer)
    hosts, counts = np.unique((u >> np.uint64(32)).astype(np.uint32), return_counts=True)
    return hosts, counts


def window_seed(workload_index: int, link: int = 0) -> int:
    """Seed convention: 0x5D5A0000 + workload index, + (link << 8) per link."""
    return 0x5D5A0000 + workload_index + (link << 8)
