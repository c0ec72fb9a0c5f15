"""Python binding of the sd C ABI (``include/sd.h``): argument marshalling only.

Every function keeps its C name and forwards to ``_build/libsd.so``; all
computation happens in the library's CUDA kernels.  The library must have
been built (``paper_1803_11449_gb300.build.build()`` or
``__graft_entry__.build()``): importing the binding without it raises, there
is no fallback.

Pair buffers may be torch tensors (CUDA or CPU) or numpy arrays of 2n
4-byte words, interleaved (src, dst).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsd.so")

SD_OK = 0
SD_ERR_ARG = -1
SD_ERR_NOMEM = -2
SD_ERR_CUDA = -3
SD_ERR_SATURATED = -4
SD_ERR_OVERLOAD = -5
SD_ERR_REPORT_OVERFLOW = -6
SD_ERR_TOO_LARGE = -7

SD_FLAG_SATURATED = 1
SD_FLAG_OVERLOAD_PAIRS = 2
SD_FLAG_OVERLOAD_CANDS = 4
SD_FLAG_REPORT_OVERFLOW = 8

# every function the header declares, in declaration order
EXPORTS = ["sd_default_params", "sd_check_params", "sd_grid_words", "sd_device_bytes", "sd_create",
           "sd_update", "sd_close_window", "sd_close_many", "sd_update_many", "sd_scratch_bytes", "sd_sync", "sd_destroy",
           "sd_last_error", "sd_get_grid",
           "sd_set_grid", "sd_get_hot", "sd_get_candidates", "sd_merge", "sd_kernel_launches",
           "sd_get_tuning", "sd_set_tuning", "sd_update_noalloc", "sd_update_dir", "sd_export_grid",
           "sd_or_grid", "sd_or_words", "sd_partition_pairs"]


class sd_params(ctypes.Structure):
    _fields_ = [("g", ctypes.c_uint32), ("r", ctypes.c_uint32), ("k", ctypes.c_uint32),
                ("alpha", ctypes.c_uint32), ("theta", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("dirs", ctypes.c_uint32), ("device", ctypes.c_int32),
                ("pair_cap", ctypes.c_uint64), ("cand_cap", ctypes.c_uint64),
                ("report_cap", ctypes.c_uint64), ("stage_pairs", ctypes.c_uint64),
                ("cuda_stream", ctypes.c_void_p)]


class sd_hit(ctypes.Structure):
    _fields_ = [("ip", ctypes.c_uint32), ("sz", ctypes.c_uint32), ("dir", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("est", ctypes.c_double)]


class sd_report(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_uint64), ("zr", (ctypes.c_uint64 * 8) * 2),
                ("psi", ctypes.c_double * 2), ("n_hot", (ctypes.c_uint32 * 8) * 2),
                ("n_cand", ctypes.c_uint64 * 2), ("zhot", ctypes.c_uint32),
                ("szmax", ctypes.c_uint32 * 2), ("flags", ctypes.c_uint32),
                ("n_hits_total", ctypes.c_uint64), ("n_hits", ctypes.c_uint64),
                ("hits", ctypes.POINTER(sd_hit))]


class sd_tuning(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_uint32), ("block_threads", ctypes.c_uint32),
                ("blocks_per_sm", ctypes.c_uint32), ("unroll", ctypes.c_uint32),
                ("filter_log2", ctypes.c_uint32), ("bin_slice_log2", ctypes.c_uint32),
                ("bin_tile_pairs", ctypes.c_uint32), ("bin_chunk_log2", ctypes.c_uint32),
                ("bin_slack_pct", ctypes.c_uint32), ("restore", ctypes.c_uint32),
                ("bin_batch_mib", ctypes.c_uint32), ("plane_tile_pairs", ctypes.c_uint32),
                ("plane_round_log2", ctypes.c_uint32), ("plane_unit_log2", ctypes.c_uint32)]


HIT_DTYPE = np.dtype([("ip", "<u4"), ("sz", "<u4"), ("dir", "<u4"), ("reserved", "<u4"),
                      ("est", "<f8")])
assert HIT_DTYPE.itemsize == ctypes.sizeof(sd_hit)


class SdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sd error {code}: {msg}")
        self.code = code


_P = ctypes.POINTER
_VP = ctypes.c_void_p
_lock = threading.Lock()
_lib = None


def lib():
    """Load libsd.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"the sd CUDA library is not built ({LIB_PATH} missing); "
                                   "run paper_1803_11449_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            sig = {
                "sd_default_params": (ctypes.c_int, [_P(sd_params)]),
                "sd_check_params": (ctypes.c_int, [_P(sd_params)]),
                "sd_grid_words": (ctypes.c_uint64, [_P(sd_params)]),
                "sd_device_bytes": (ctypes.c_uint64, [_P(sd_params)]),
                "sd_create": (ctypes.c_int, [_P(sd_params), _P(_VP)]),
                "sd_update": (ctypes.c_int, [_VP, _VP, ctypes.c_uint64]),
                "sd_close_window": (ctypes.c_int, [_VP, _P(sd_report)]),
                "sd_close_many": (ctypes.c_int, [_P(_VP), ctypes.c_uint32, _P(sd_report),
                                                 _P(ctypes.c_int)]),
                "sd_update_many": (ctypes.c_int, [_P(_VP), _P(_VP), _P(ctypes.c_uint64),
                                                  ctypes.c_uint32]),
                "sd_sync": (ctypes.c_int, [_VP]),
                "sd_destroy": (ctypes.c_int, [_VP]),
                "sd_last_error": (ctypes.c_char_p, [_VP]),
                "sd_get_grid": (ctypes.c_int, [_VP, ctypes.c_uint32, _VP]),
                "sd_set_grid": (ctypes.c_int, [_VP, ctypes.c_uint32, _VP]),
                "sd_get_hot": (ctypes.c_int, [_VP, ctypes.c_uint32, ctypes.c_uint32, _VP]),
                "sd_get_candidates": (ctypes.c_int64, [_VP, ctypes.c_uint32, _VP, ctypes.c_uint64]),
                "sd_merge": (ctypes.c_int, [_VP, _VP]),
                "sd_kernel_launches": (ctypes.c_uint64, []),
                "sd_scratch_bytes": (ctypes.c_uint64, [_VP, ctypes.c_uint32]),
                "sd_get_tuning": (ctypes.c_int, [_VP, _P(sd_tuning)]),
                "sd_set_tuning": (ctypes.c_int, [_VP, _P(sd_tuning)]),
                "sd_update_noalloc": (ctypes.c_int, [_P(sd_params), _VP, _VP, ctypes.c_uint64, _VP]),
                "sd_update_dir": (ctypes.c_int, [_VP, ctypes.c_uint32, _VP, ctypes.c_uint64]),
                "sd_export_grid": (ctypes.c_int, [_VP, _VP]),
                "sd_or_grid": (ctypes.c_int, [_VP, _VP]),
                "sd_or_words": (ctypes.c_int, [_VP, _VP, ctypes.c_uint64, ctypes.c_uint32, _VP]),
                "sd_partition_pairs": (ctypes.c_int, [_VP, ctypes.c_uint32, _VP, ctypes.c_uint64,
                                                      ctypes.c_uint32, _VP, _P(ctypes.c_uint64)]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc: int, h=None, ok=(SD_OK,)):
    if rc not in ok:
        msg = lib().sd_last_error(h)
        raise SdError(rc, msg.decode() if msg else "")
    return rc


# ------------------------------------------------------------------ params
def sd_default_params(**over) -> sd_params:
    p = sd_params()
    _check(lib().sd_default_params(ctypes.byref(p)))
    for key, val in over.items():
        if key == "cuda_stream" and val is not None and not isinstance(val, int):
            val = val.cuda_stream  # a torch.cuda.Stream
        setattr(p, key, val)
    return p


def sd_check_params(p: sd_params) -> int:
    return lib().sd_check_params(ctypes.byref(p))


def sd_grid_words(p: sd_params) -> int:
    return int(lib().sd_grid_words(ctypes.byref(p)))


def sd_device_bytes(p: sd_params) -> int:
    return int(lib().sd_device_bytes(ctypes.byref(p)))


# ------------------------------------------------------------------ handle
class Handle:
    """An ``sd_handle*`` with its parameters."""

    def __init__(self, ptr: int, params: sd_params):
        self.ptr = ptr
        self.params = params

    @property
    def _as_parameter_(self):
        return ctypes.c_void_p(self.ptr)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        sd_destroy(self)
        return False


def sd_create(p: sd_params) -> Handle:
    out = _VP()
    rc = lib().sd_create(ctypes.byref(p), ctypes.byref(out))
    _check(rc, None)
    return Handle(out.value, p)


def sd_destroy(h: Handle) -> None:
    if h is not None and h.ptr:
        lib().sd_destroy(h.ptr)
        h.ptr = 0


def sd_last_error(h: Handle | None = None) -> str:
    msg = lib().sd_last_error(h.ptr if h else None)
    return msg.decode() if msg else ""


def sd_sync(h: Handle) -> None:
    _check(lib().sd_sync(h.ptr), h.ptr)


def _buffer(pairs):
    """(address, number of pairs, keep-alive) of a pair buffer."""
    try:
        import torch
        if isinstance(pairs, torch.Tensor):
            assert pairs.element_size() == 4 and pairs.is_contiguous(), \
                "pairs must be a contiguous tensor of 4-byte words"
            return pairs.data_ptr(), pairs.numel() // 2, pairs
    except ImportError:  # pragma: no cover
        pass
    a = np.ascontiguousarray(pairs)
    assert a.itemsize == 4, "pairs must hold 4-byte words"
    return a.ctypes.data, a.size // 2, a


def sd_update(h: Handle, pairs) -> None:
    """Algorithm 1 over every (src, dst) pair of `pairs`."""
    ptr, n, _keep = _buffer(pairs)
    _check(lib().sd_update(h.ptr, ptr if n else None, n), h.ptr)


@dataclasses.dataclass
class Report:
    rc: int
    n_pairs: int
    zr: np.ndarray          # [dirs, r]
    psi: list
    n_hot: np.ndarray       # [dirs, r]
    n_cand: list
    zhot: int
    szmax: list
    flags: int
    n_hits_total: int
    hits: np.ndarray        # structured HIT_DTYPE, ordered by (dir, ip)

    def dir_flags(self, d: int) -> int:
        return (self.flags >> (8 * d)) & 0xFF


def sd_close_window(h: Handle, allow=(SD_OK, SD_ERR_SATURATED, SD_ERR_OVERLOAD,
                                      SD_ERR_REPORT_OVERFLOW)) -> Report:
    """Close the window; returns the report (codes in `allow` do not raise)."""
    rep = sd_report()
    rc = lib().sd_close_window(h.ptr, ctypes.byref(rep))
    _check(rc, h.ptr, ok=allow)
    return _report_of(h, rc, rep)


def _report_of(h: Handle, rc: int, rep: sd_report) -> Report:
    p = h.params
    n = int(rep.n_hits)
    if n:
        addr = ctypes.cast(rep.hits, ctypes.c_void_p).value
        raw = (ctypes.c_char * (n * HIT_DTYPE.itemsize)).from_address(addr)
        hits = np.frombuffer(raw, dtype=HIT_DTYPE, count=n).copy()  # the handle reuses its buffer
    else:
        hits = np.zeros(0, dtype=HIT_DTYPE)
    zr = np.frombuffer(rep.zr, dtype=np.uint64).reshape(2, 8)[: p.dirs, : p.r].copy()
    n_hot = np.frombuffer(rep.n_hot, dtype=np.uint32).reshape(2, 8)[: p.dirs, : p.r].astype(np.int64)
    return Report(
        rc=rc, n_pairs=int(rep.n_pairs), zr=zr, psi=list(rep.psi)[: p.dirs], n_hot=n_hot,
        n_cand=[int(x) for x in list(rep.n_cand)[: p.dirs]], zhot=int(rep.zhot),
        szmax=[int(x) for x in list(rep.szmax)[: p.dirs]], flags=int(rep.flags),
        n_hits_total=int(rep.n_hits_total), hits=hits)


def sd_update_many(hs, pairs_list) -> None:
    """Algorithm 1 for many handles at once (batched rounds, see sd.h)."""
    n = len(hs)
    bufs = [_buffer(p) for p in pairs_list]
    arr_h = (_VP * n)(*[h.ptr for h in hs])
    arr_p = (_VP * n)(*[b[0] if b[1] else None for b in bufs])
    arr_n = (ctypes.c_uint64 * n)(*[b[1] for b in bufs])
    _check(lib().sd_update_many(arr_h, arr_p, arr_n, n), hs[0].ptr if hs else None)


def sd_close_many(hs) -> list:
    """Close the windows of many handles at once; one Report per handle."""
    n = len(hs)
    arr_h = (_VP * n)(*[h.ptr for h in hs])
    reps = (sd_report * n)()
    rcs = (ctypes.c_int * n)()
    rc = lib().sd_close_many(arr_h, n, reps, rcs)
    if rc not in (SD_OK, SD_ERR_SATURATED, SD_ERR_OVERLOAD, SD_ERR_REPORT_OVERFLOW):
        _check(rc, hs[0].ptr)
    return [_report_of(h, int(rcs[i]), reps[i]) for i, h in enumerate(hs)]


def sd_get_grid(h: Handle, direction: int) -> np.ndarray:
    out = np.empty(sd_grid_words(h.params), dtype=np.uint32)
    _check(lib().sd_get_grid(h.ptr, direction, out.ctypes.data), h.ptr)
    return out


def sd_set_grid(h: Handle, direction: int, words: np.ndarray) -> None:
    a = np.ascontiguousarray(words, dtype=np.uint32)
    assert a.size == sd_grid_words(h.params)
    _check(lib().sd_set_grid(h.ptr, direction, a.ctypes.data), h.ptr)


def sd_get_hot(h: Handle, direction: int, row: int) -> np.ndarray:
    """Row `row`'s hot bitmap as of the last close, unpacked to a bool array."""
    nw = max(1, (1 << h.params.k) // 32)
    out = np.empty(nw, dtype=np.uint32)
    _check(lib().sd_get_hot(h.ptr, direction, row, out.ctypes.data), h.ptr)
    return np.unpackbits(out.view(np.uint8), bitorder="little")[: 1 << h.params.k].astype(bool)


def sd_get_candidates(h: Handle, direction: int, cap: int | None = None):
    """(|K|, the stored members of K, unordered) as of the last close."""
    cap = int(h.params.cand_cap or (1 << 20)) if cap is None else cap
    out = np.empty(max(cap, 1), dtype=np.uint32)
    n = lib().sd_get_candidates(h.ptr, direction, out.ctypes.data, cap)
    _check(int(n) if n < 0 else SD_OK, h.ptr)
    return int(n), out[: min(int(n), cap)].copy()


def sd_merge(dst: Handle, src: Handle) -> None:
    _check(lib().sd_merge(dst.ptr, src.ptr), dst.ptr)


def sd_scratch_bytes(h: Handle, links: int = 1) -> int:
    """Device bytes of the binned update's scratch of h (see sd.h)."""
    return int(lib().sd_scratch_bytes(h.ptr, links))


def sd_kernel_launches() -> int:
    return int(lib().sd_kernel_launches())


def sd_get_tuning(h: Handle) -> sd_tuning:
    t = sd_tuning()
    _check(lib().sd_get_tuning(h.ptr, ctypes.byref(t)), h.ptr)
    return t


def sd_set_tuning(h: Handle, mode=0, block_threads=0, blocks_per_sm=0, unroll=0, filter_log2=0,
                  bin_slice_log2=0, bin_tile_pairs=0, bin_chunk_log2=0, bin_slack_pct=0, restore=0,
                  bin_batch_mib=0, plane_tile_pairs=0, plane_round_log2=0, plane_unit_log2=0) -> None:
    t = sd_tuning(mode=mode, block_threads=block_threads, blocks_per_sm=blocks_per_sm, unroll=unroll,
                  filter_log2=filter_log2, bin_slice_log2=bin_slice_log2,
                  bin_tile_pairs=bin_tile_pairs, bin_chunk_log2=bin_chunk_log2,
                  bin_slack_pct=bin_slack_pct, restore=restore, bin_batch_mib=bin_batch_mib,
                  plane_tile_pairs=plane_tile_pairs, plane_round_log2=plane_round_log2,
                  plane_unit_log2=plane_unit_log2)
    _check(lib().sd_set_tuning(h.ptr, ctypes.byref(t)), h.ptr)


def sd_update_dir(h: Handle, direction: int, pairs) -> None:
    """Algorithm 1 for one direction of (key, peer) pairs (see include/sd.h)."""
    ptr, n, _keep = _buffer(pairs)
    if n == 0:
        return
    _check(lib().sd_update_dir(h.ptr, direction, ptr, n), h.ptr)


def sd_export_grid(h: Handle, dst) -> None:
    """Queue a copy of h's DHLA (both directions) into the device tensor dst."""
    ptr, _, _keep = _buffer(dst)
    _check(lib().sd_export_grid(h.ptr, ptr), h.ptr)


def sd_or_grid(h: Handle, src) -> None:
    """Queue h's DHLA |= the DHLA image in the device tensor src."""
    ptr, _, _keep = _buffer(src)
    _check(lib().sd_or_grid(h.ptr, ptr), h.ptr)


def sd_or_words(dst, src, words: int, count: int, stream=None) -> None:
    """dst[:words] = OR of the count word arrays laid end to end in src (device tensors)."""
    d, _, _k1 = _buffer(dst)
    s_, _, _k2 = _buffer(src)
    st = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(lib().sd_or_words(d, s_, words, count, st))


def sd_partition_pairs(h: Handle, direction: int, pairs, parts: int, out) -> np.ndarray:
    """Group device pairs by the key of `direction` (& (parts - 1)) into the
    device tensor out as (key, peer) pairs; returns the pairs per part."""
    ptr, n, _keep = _buffer(pairs)
    optr, _, _k2 = _buffer(out)
    counts = (ctypes.c_uint64 * parts)()
    _check(lib().sd_partition_pairs(h.ptr, direction, ptr if n else None, n, parts, optr if n else None,
                                    counts), h.ptr)
    return np.array(counts[:], dtype=np.int64)


def sd_update_noalloc(p: sd_params, grid, pairs, stream=None) -> int:
    """Binned update into a caller-owned device DHLA `grid` (torch tensor of
    dirs * sd_grid_words(p) 4-byte words) with no device allocation; returns
    the C status code.  See include/sd.h for the scratch rules."""
    gptr, _, _g = _buffer(grid)
    ptr, n, _keep = _buffer(pairs)
    s = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    return lib().sd_update_noalloc(ctypes.byref(p), gptr, ptr if n else None, n, s)


def params_for(workload, seed: int, device: int = 0, **over) -> sd_params:
    """sd_params of a traffic.Workload's sketch."""
    s = workload.sketch() if hasattr(workload, "sketch") else dict(workload)
    return sd_default_params(g=s["g"], r=s["r"], k=s["k"], alpha=s["alpha"], theta=float(s["theta"]),
                             dirs=s["dirs"], seed=seed, device=device, **over)
