"""CPU oracle for DHSA super-point detection (arxiv 1803.11449).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path (the
CUDA library and its Python binding) never imports this package.

The arithmetic lives in ``sd_oracle.c`` (plain single-threaded C, fp64 where
floating point appears); this module compiles it with gcc and wraps it with
ctypes, marshalling numpy arrays.  Each wrapper names the part of the paper
the C routine follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SD_ORACLE_SRC builds the oracle from another copy of the C source instead:
# the mutation tests plant one mistake in a copy and run the pins against it.
_SRC = os.environ.get("SD_ORACLE_SRC") or os.path.join(_HERE, "sd_oracle.c")
_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(_SRC)), "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

FLAG_SATURATED = 1
FLAG_OVERLOAD_PAIRS = 2
FLAG_OVERLOAD_CANDS = 4


def build(force: bool = False) -> str:
    """Compile ``sd_oracle.c`` into ``_build/liboracle.so`` (gcc -O3).

    ``-ffp-contract=off`` keeps every double expression rounded step by step,
    as written, on every host architecture.
    """
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [("g", ctypes.c_uint32), ("r", ctypes.c_uint32), ("k", ctypes.c_uint32),
                ("alpha", ctypes.c_uint32), ("dirs", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("theta", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("pair_cap", ctypes.c_uint64),
                ("cand_cap", ctypes.c_uint64)]


class Summary(ctypes.Structure):
    _fields_ = [("zr", (ctypes.c_uint64 * 8) * 2), ("psi", ctypes.c_double * 2),
                ("n_hot", (ctypes.c_uint32 * 8) * 2), ("n_cand", ctypes.c_uint64 * 2),
                ("flags", ctypes.c_uint32 * 2), ("n_hits", ctypes.c_uint64)]


_P = ctypes.POINTER
_u32p = _P(ctypes.c_uint32)
_u64p = _P(ctypes.c_uint64)
_f64p = _P(ctypes.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            sig = {
                "or_splitmix64": (ctypes.c_uint64, [_u64p]),
                "or_hash_constants": (None, [ctypes.c_uint64, ctypes.c_uint32, _u32p, _u64p, _u64p]),
                "or_dh0": (ctypes.c_uint32, [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]),
                "or_dh": (ctypes.c_uint32, [ctypes.c_uint32] * 5),
                "or_h1": (ctypes.c_uint32, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                            ctypes.c_uint32]),
                "or_check_params": (ctypes.c_int, [_P(Params)]),
                "or_grid_words": (ctypes.c_uint64, [_P(Params)]),
                "or_update": (None, [_P(Params), _u32p, _u32p, ctypes.c_uint64]),
                "or_row_stats": (None, [_P(Params), _u32p, ctypes.c_uint32, _u32p, _u64p]),
                "or_zmin": (ctypes.c_double, [ctypes.c_uint32, ctypes.c_double]),
                "or_hot_sets": (None, [_P(Params), _u32p, _u32p, _u32p]),
                "or_psi": (ctypes.c_double, [_P(Params), _u64p]),
                "or_estimate": (ctypes.c_double, [ctypes.c_uint32, ctypes.c_uint32,
                                                  ctypes.c_double, ctypes.c_uint32]),
                "or_sz": (ctypes.c_uint32, [_P(Params), _u32p, ctypes.c_uint32, ctypes.c_uint32]),
                "or_inverse_odd": (ctypes.c_uint32, [ctypes.c_uint32]),
                "or_restore_join": (ctypes.c_uint64, [_P(Params), ctypes.c_uint32, _u32p, _u32p,
                                                      _u32p, ctypes.c_uint64]),
                "or_restore_preimage": (ctypes.c_uint64, [_P(Params), ctypes.c_uint32, _u32p,
                                                          _u32p, _u32p, ctypes.c_uint64]),
                "or_close_window": (ctypes.c_uint64, [_P(Params), _u32p, _P(Summary), _u32p,
                                                      _u32p, _u32p, _f64p, ctypes.c_uint64,
                                                      _u32p]),
                "or_report_brute": (ctypes.c_uint64, [_P(Params), _u32p, ctypes.c_uint32, _u32p,
                                                      _u32p, ctypes.c_uint64, _u32p,
                                                      ctypes.c_uint64, _u64p]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _ptr(a: np.ndarray, ctype=ctypes.c_uint32):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_P(ctype))


def make_params(g, r, k, alpha, theta, seed, dirs=1, pair_cap=1 << 32, cand_cap=1 << 20) -> Params:
    return Params(g=g, r=r, k=k, alpha=alpha, dirs=dirs, reserved=0, theta=float(theta),
                  seed=seed, pair_cap=pair_cap, cand_cap=cand_cap)


def params_from(cfg: dict, seed: int, **over) -> Params:
    d = dict(g=cfg["g"], r=cfg["r"], k=cfg["k"], alpha=cfg["alpha"], theta=cfg["theta"],
             dirs=cfg["dirs"])
    d.update(over)
    return make_params(seed=seed, **d)


def check_params(p: Params) -> bool:
    return lib().or_check_params(ctypes.byref(p)) == 0


def splitmix64_stream(seed: int, count: int) -> list[int]:
    st = ctypes.c_uint64(seed)
    return [lib().or_splitmix64(ctypes.byref(st)) for _ in range(count)]


def hash_constants(seed: int, direction: int):
    A0, A1, B1 = ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_uint64()
    lib().or_hash_constants(seed, direction, ctypes.byref(A0), ctypes.byref(A1), ctypes.byref(B1))
    return A0.value, A1.value, B1.value


def dh(p: Params, direction: int, i: int, x: int) -> int:
    """Eq. 2 (DH_0 for i = 0)."""
    A0, _, _ = hash_constants(p.seed, direction)
    return lib().or_dh(A0, p.k, p.alpha, i, x)


def h1(p: Params, direction: int, y: int) -> int:
    _, A1, B1 = hash_constants(p.seed, direction)
    return lib().or_h1(A1, B1, p.g, y)


def grid_words(p: Params) -> int:
    return int(lib().or_grid_words(ctypes.byref(p)))


def new_grid(p: Params) -> np.ndarray:
    return np.zeros(grid_words(p), dtype=np.uint32)


def update(p: Params, grid: np.ndarray, pairs: np.ndarray) -> None:
    """Algorithm 1 over every (src, dst) pair, for each direction."""
    pairs = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1)
    assert pairs.size % 2 == 0 and grid.dtype == np.uint32 and grid.size == grid_words(p)
    lib().or_update(ctypes.byref(p), _ptr(grid), _ptr(pairs), pairs.size // 2)


def row_stats(p: Params, grid: np.ndarray, direction: int):
    """Returns (z0[r, 2^k], ZR[r])."""
    z0 = np.empty((p.r, 1 << p.k), dtype=np.uint32)
    zr = np.empty(p.r, dtype=np.uint64)
    lib().or_row_stats(ctypes.byref(p), _ptr(grid), direction, _ptr(z0), _ptr(zr, ctypes.c_uint64))
    return z0, zr


def zmin(g: int, theta: float) -> float:
    return lib().or_zmin(g, theta)


def hot_sets(p: Params, z0: np.ndarray):
    """Returns (he[r, 2^k] padded lists, nhe[r]) with HE(i) = he[i, :nhe[i]]."""
    z0 = np.ascontiguousarray(z0, dtype=np.uint32)
    he = np.zeros((p.r, 1 << p.k), dtype=np.uint32)
    nhe = np.zeros(p.r, dtype=np.uint32)
    lib().or_hot_sets(ctypes.byref(p), _ptr(z0), _ptr(he), _ptr(nhe))
    return he, nhe


def psi(p: Params, zr) -> float:
    zr = np.ascontiguousarray(zr, dtype=np.uint64)
    return lib().or_psi(ctypes.byref(p), _ptr(zr, ctypes.c_uint64))


def estimate(g: int, r: int, psi_: float, sz: int) -> float:
    """Eq. 4."""
    return lib().or_estimate(g, r, psi_, sz)


def sz(p: Params, grid: np.ndarray, direction: int, a0: int) -> int:
    return lib().or_sz(ctypes.byref(p), _ptr(grid), direction, a0)


def inverse_odd(a: int) -> int:
    return lib().or_inverse_odd(a)


def _restore(fn, p, direction, he, nhe, cap):
    he = np.ascontiguousarray(he, dtype=np.uint32)
    nhe = np.ascontiguousarray(nhe, dtype=np.uint32)
    out = np.zeros(max(cap, 1), dtype=np.uint32)
    n = fn(ctypes.byref(p), direction, _ptr(he), _ptr(nhe), _ptr(out), cap)
    if n == 2**64 - 1:
        raise MemoryError("oracle restore ran out of memory")
    return int(n), out[:min(n, cap)].copy()


def restore_join(p, direction, he, nhe, cap=1 << 22):
    return _restore(lib().or_restore_join, p, direction, he, nhe, cap)


def restore_preimage(p, direction, he, nhe, cap=1 << 22):
    return _restore(lib().or_restore_preimage, p, direction, he, nhe, cap)


def close_window(p: Params, grid: np.ndarray, hit_cap: int = 1 << 20, want_cands: bool = False):
    """Algorithm 2 + the §4.2 estimation step.  Returns a dict with the per
    direction row statistics, psi, hot counts, |K|, flags and the hits ordered
    by (dir, ip)."""
    s = Summary()
    hd = np.zeros(hit_cap, dtype=np.uint32)
    hi = np.zeros(hit_cap, dtype=np.uint32)
    hs = np.zeros(hit_cap, dtype=np.uint32)
    he = np.zeros(hit_cap, dtype=np.float64)
    cands = np.zeros(p.dirs * p.cand_cap, dtype=np.uint32) if want_cands else None
    n = lib().or_close_window(ctypes.byref(p), _ptr(grid), ctypes.byref(s), _ptr(hd), _ptr(hi),
                              _ptr(hs), _ptr(he, ctypes.c_double), hit_cap,
                              _ptr(cands) if want_cands else None)
    if n == 2**64 - 1:
        raise MemoryError("oracle close ran out of memory")
    m = min(n, hit_cap)
    out = {
        "zr": np.array([[s.zr[d][i] for i in range(p.r)] for d in range(p.dirs)], dtype=np.uint64),
        "psi": [s.psi[d] for d in range(p.dirs)],
        "n_hot": np.array([[s.n_hot[d][i] for i in range(p.r)] for d in range(p.dirs)]),
        "n_cand": [int(s.n_cand[d]) for d in range(p.dirs)],
        "flags": [int(s.flags[d]) for d in range(p.dirs)],
        "n_hits": int(n),
        "dir": hd[:m].copy(), "ip": hi[:m].copy(), "sz": hs[:m].copy(), "est": he[:m].copy(),
    }
    if want_cands:
        out["cands"] = [cands[d * p.cand_cap: d * p.cand_cap + min(out["n_cand"][d], p.cand_cap)]
                        .copy() for d in range(p.dirs)]
    return out


def report_brute(p: Params, grid: np.ndarray, direction: int, cap: int = 1 << 20):
    """Exhaustive sweep of all 2^32 keys: returns (report ips, their SZ, K)."""
    ip = np.zeros(cap, dtype=np.uint32)
    szs = np.zeros(cap, dtype=np.uint32)
    kk = np.zeros(cap, dtype=np.uint32)
    nk = ctypes.c_uint64(0)
    n = lib().or_report_brute(ctypes.byref(p), _ptr(grid), direction, _ptr(ip), _ptr(szs), cap,
                              _ptr(kk), cap, ctypes.byref(nk))
    if n == 2**64 - 1:
        raise ValueError("saturated grid or out of memory")
    return ip[:min(n, cap)].copy(), szs[:min(n, cap)].copy(), kk[:min(nk.value, cap)].copy()
