"""Benchmark of one detection window per step: sd_update over the window's
pairs (Algorithm 1) and sd_close_window (Algorithm 2 + §4.2), through the C
ABI.

Prints one JSON line (rank 0).  `value` is whole-job packets per second
(Gpps) with the pairs already resident in HBM; `e2e` is the same metric with
the pairs fed from pinned host memory through sd_update (host->device copies
inside the timed region) and the report read back.  `roofline` covers the
dominant kernel (the update): algorithmic bytes = 8 per pair, over its CUDA
event time, against the measured HBM copy bandwidth.

--impl reference times the CPU oracle (test infrastructure) on a bounded
sample of the same workload, as the reference arm.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1803_11449_gb300 import traffic as T  # noqa: E402

WORKLOAD = "core"
WORKLOAD_DESC = ("core-link window: 2^26 (src,dst) uint32 pairs, 2^24 Zipf(1.05) sources, 2^26 "
                 "destinations, 500 planted super points (1,024-200,000 peers); DHLA g=512 r=4 "
                 "k=16 alpha=8 (16 MiB per direction, L2-resident), theta=1024, both directions")
DESCS = {
    "core": WORKLOAD_DESC,
    "paper": ("the paper's sketch parameters on core-link traffic: 2^26 (src,dst) uint32 pairs, 2^24 "
              "Zipf(1.05) sources, 2^26 destinations, 500 planted super points (1,024-200,000 peers); "
              "DHLA g=1024 r=5 k=14 alpha=6 (10 MiB per direction), theta=1024, both directions"),
    "stress": ("stress window: 2^30 (src,dst) uint32 pairs in flows of 8 packets, 2^28 Zipf(1.0) sources, "
               "2^30 destinations, 10^4 planted super points (1,024-10^7 peers); DHLA g=1024 r=4 k=18 "
               "alpha=7 (128 MiB per direction, larger than L2), theta=1024, both directions"),
    "tiny": ("small window: 2^20 (src,dst) uint32 pairs, 2^16 Zipf(1.1) sources, uniform destinations, "
             "20 planted super points (1,500-4,000 peers); DHLA g=256 r=4 k=12 alpha=10, theta=1024, "
             "outbound only"),
}
BYTES_PER_PAIR = 8
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e specification, for context beside the measured copy rate
GBITS_PER_PACKET = 800 * 8 / 1e9   # 800-byte average packet (§1, §5)
CPU_SAMPLE_PAIRS = 1 << 26


UPDATE_KERNELS = {5: "k_bin+k_apply", 6: "k_plane_bin+k_plane_apply"}
UPDATE_SOURCES = {5: ["sd_binned.cu", "sd_common.cuh"], 6: ["sd_plane.cu", "sd_common.cuh"]}
UPDATE_PROFILES = {5: "update_binned_core_window.txt", 6: "update_plane_core_window.txt"}


def source_sha256(mode: int) -> str:
    """sha256 of the update kernels' sources of a tuning mode, in order."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1803_11449_gb300", "csrc")
    h = hashlib.sha256()
    for f in UPDATE_SOURCES.get(mode, ["sd_update.cu", "sd_common.cuh"]):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(mode: int, n: int):
    """DRAM bytes per launch set of the update for `n` pairs, from the
    committed ncu summary of the same kernel source; None when no summary
    matches the current source (the counters no longer describe it)."""
    digest = source_sha256(mode)
    name = UPDATE_PROFILES.get(mode, "update_inplace_core_window.txt")
    # the counters were taken for one mode-5 round; in-place modes have none committed
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    fields = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line:
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip()
    if fields.get("source_sha256") != digest or "dram_bytes_per_pair" not in fields:
        return None
    return float(fields["dram_bytes_per_pair"]) * n


def ref_sample_for(steps: int, warmup: int) -> int:
    """Pairs per step of the reference arm: 2^22 (about a second of oracle
    work) while the whole run stays near 55 such samples, then halved down to
    2^18, so that long runs still end within a few minutes."""
    sample = 1 << 22
    while sample > (1 << 18) and sample * (steps + warmup) > 55 * (1 << 22):
        sample >>= 1
    return sample


def l2_reduction_ceiling():
    """Random L2 reductions per second measured on this GPU (the in-place
    update's bound), from the committed ncu summary of k_update mode 0 on
    uniform pairs; None when the summary is absent."""
    path = os.path.join(ROOT, "profiles", "update_inplace_uniform_l2_atomics.txt")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        for line in fh:
            m = re.search(r"->\s*([0-9.]+e[0-9]+) L2 reductions/s", line)
            if m:
                return float(m.group(1))
    return None


def l2_roofline(ops_per_pair: int, n: int, t_upd: float) -> dict:
    """Bit-sets per second of the update beside the measured random-L2
    reduction rate, the ceiling of any in-place update."""
    achieved = ops_per_pair * n / t_upd
    ceiling = l2_reduction_ceiling()
    out = {"ops_per_pair": ops_per_pair, "achieved_ops_per_s": achieved}
    if ceiling:
        out.update({"in_place_ceiling_ops_per_s": ceiling, "vs_in_place_ceiling": achieved / ceiling,
                    "ceiling_source": "profiles/update_inplace_uniform_l2_atomics.txt (measured: one "
                                      "red.or per bit-set, uniform pairs, L2 at 84.5% of peak)"})
    return out


def ceilings_lib():
    """libsd_ceilings.so: microbenchmarks of the rates that bound the update."""
    import ctypes
    from paper_1803_11449_gb300 import build as b
    b.build()
    L = ctypes.CDLL(b.CEILINGS_LIB)
    d = ctypes.POINTER(ctypes.c_double)
    L.sdc_smem_or_rate.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, d]
    L.sdc_l2_rates.argtypes = [ctypes.c_uint64, d, d, d]
    L.sdc_host_link.argtypes = [ctypes.c_uint64, d, d, d]
    return L


def smem_or_ceiling(words_log2: int = 13) -> float | None:
    """Random shared-memory atomic ORs per second on this GPU (the bound of
    the apply step, which sets every bit that way), measured now: the best
    of a few block shapes."""
    import ctypes
    L = ceilings_lib()
    best = None
    for threads, bps in ((512, 2), (512, 4), (1024, 2)):
        v = ctypes.c_double()
        if L.sdc_smem_or_rate(words_log2, threads, bps, ctypes.byref(v)) == 0:
            best = max(best or 0.0, v.value)
    return best


def run_ceilings(args, rank, world, local):
    """The rates that bound the update, measured on this GPU (one JSON line)."""
    import ctypes
    import torch
    torch.cuda.set_device(local)
    if rank != 0:
        return
    L = ceilings_lib()
    out = {"gpu": torch.cuda.get_device_name(local), "smem_atomic_or_per_s": {}}
    for lw in (13, 15):
        for threads, bps in ((256, 4), (512, 2), (512, 4), (1024, 1), (1024, 2)):
            if (4 << lw) * bps > 200 * 1024:
                continue
            v = ctypes.c_double()
            if L.sdc_smem_or_rate(lw, threads, bps, ctypes.byref(v)) == 0:
                out["smem_atomic_or_per_s"][f"{4 << lw >> 10} KiB, {threads} threads x {bps} blocks/SM"] = v.value
    out["l2"] = {}
    for mib in (32, 64, 96):
        r, w_, b_ = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        if L.sdc_l2_rates(mib << 20, ctypes.byref(r), ctypes.byref(w_), ctypes.byref(b_)) == 0:
            out["l2"][f"{mib} MiB"] = {"read_gbs": r.value, "write_gbs": w_.value, "bulk_or_gbs": b_.value}
    h2d, pr, pg = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    if L.sdc_host_link(1 << 30, ctypes.byref(h2d), ctypes.byref(pr), ctypes.byref(pg)) == 0:
        out["host_link_gbs"] = {"h2d_pinned_copy": h2d.value, "kernel_reads_pinned": pr.value,
                                "kernel_reads_pageable": pg.value,
                                "pairs_per_s_at_h2d": h2d.value * 1e9 / BYTES_PER_PAIR}
    print(json.dumps(out), flush=True)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class _Nvml:
    """Read-only NVML queries through ctypes (SM clock, its maximum, power,
    clock-event reasons); None when the library is absent."""
    SM = 1

    def __init__(self, index: int):
        import ctypes
        self.ct = ctypes
        self.L = ctypes.CDLL("libnvidia-ml.so.1")
        if self.L.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        if self.L.nvmlDeviceGetHandleByIndex_v2(index, ctypes.byref(self.h)) != 0:
            raise OSError("no NVML handle")
        fn = getattr(self.L, "nvmlDeviceGetCurrentClocksEventReasons", None)
        self.reasons_fn = fn or self.L.nvmlDeviceGetCurrentClocksThrottleReasons

    def sample(self):
        c = self.ct
        mhz, mx, mw, rs = c.c_uint(), c.c_uint(), c.c_uint(), c.c_ulonglong()
        if self.L.nvmlDeviceGetClockInfo(self.h, self.SM, c.byref(mhz)) != 0:
            return None
        self.L.nvmlDeviceGetMaxClockInfo(self.h, self.SM, c.byref(mx))
        self.L.nvmlDeviceGetPowerUsage(self.h, c.byref(mw))
        self.reasons_fn(self.h, c.byref(rs))
        return (float(mhz.value), float(mx.value), mw.value / 1000.0, int(rs.value))

    def close(self):
        self.L.nvmlShutdown()


class ClockSampler:
    """SM clock and clock-event reasons sampled during the timed region
    (read-only queries): NVML every 2 ms from a thread, else nvidia-smi
    every 10 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clock-event reason bits
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    def __init__(self, index: int, period_s: float = 0.002):
        self.index = index
        self.period = period_s
        self.proc = None
        self.tmp = None
        self.nvml = None
        self.rows = []
        self.thread = None
        self.stop = None

    def __enter__(self):
        import threading
        try:
            self.nvml = _Nvml(self.index)
        except (OSError, AttributeError):
            self.nvml = None
        if self.nvml is not None:
            self.stop = threading.Event()

            def run():
                while not self.stop.is_set():
                    r = self.nvml.sample()
                    if r is not None:
                        self.rows.append(r)
                    self.stop.wait(self.period)
            self.thread = threading.Thread(target=run, daemon=True)
            self.thread.start()
            return self
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "10"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.thread is not None:
            self.stop.set()
            self.thread.join(timeout=5)
            self.nvml.close()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.nvml is not None:
            if not self.rows:
                return None
            reasons = sorted({n for r in self.rows for n, b in self.BITS.items() if r[3] & b})
            return {"sm_mhz": statistics.median(r[0] for r in self.rows),
                    "sm_max_mhz": max(r[1] for r in self.rows), "reasons": reasons,
                    "samples": len(self.rows), "power_w_max": max(r[2] for r in self.rows),
                    "source": f"NVML every {self.period * 1e3:.0f} ms"}
        if self.proc is None or self.tmp is None:
            return None
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows),
                "source": "nvidia-smi every 10 ms"}


def dist_setup(n_gpus: int):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def dist_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


TRAFFIC = "core"


def window_for(rank: int, n: int | None = None):
    """Each rank processes its own link: an independent window (weak scaling)."""
    if TRAFFIC == "uniform":
        n = n or T.WORKLOADS[WORKLOAD].n
        rng = np.random.default_rng(T.window_seed(2, link=rank))
        pairs = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
        return T.Window(pairs=pairs, planted_ip=np.zeros(0, np.uint32),
                        planted_dir=np.zeros(0, np.uint8), planted_c=np.zeros(0, np.int64),
                        workload=T.WORKLOADS[WORKLOAD], seed=0)
    return T.make_window(WORKLOAD, T.window_seed(2, link=rank), n=n)




def cpu_oracle_rate(pairs: np.ndarray, sample: int, parts: dict | None = None):
    """The oracle, as it stands, on the first `sample` pairs of the window:
    update then close, single-threaded.  Returns (pairs/s, seconds); the
    update and close seconds go to `parts` when given."""
    import oracle as O
    O.build()
    w = T.WORKLOADS[WORKLOAD]
    op = O.params_from(w.sketch(), seed=T.window_seed(2))
    grid = O.new_grid(op)
    sub = np.ascontiguousarray(pairs[:sample])
    t0 = time.perf_counter()
    O.update(op, grid, sub)
    t1 = time.perf_counter()
    O.close_window(op, grid)
    dt = time.perf_counter() - t0
    if parts is not None:
        parts.update(update_s=t1 - t0, close_s=dt - (t1 - t0))
    return sample / dt, dt


def _oracle_part(args):
    """Worker of the parallel CPU baseline: the oracle's Algorithm 1 over one
    contiguous part of the pairs (read from shared memory) into a new grid."""
    import oracle as O
    from multiprocessing import shared_memory
    name, n, lo, hi, sketch, seed = args
    shm = shared_memory.SharedMemory(name=name)
    try:
        pairs = np.ndarray((n, 2), dtype=np.uint32, buffer=shm.buf)
        op = O.params_from(sketch, seed=seed)
        grid = O.new_grid(op)
        O.update(op, grid, pairs[lo:hi])
        return grid
    finally:
        shm.close()


def cpu_oracle_parallel(pairs: np.ndarray, workers: int):
    """The oracle with the window split over `workers` processes: each
    builds a grid from its part (Algorithm 1), the grids are OR-merged (the
    grid of the union stream) and the oracle closes the window.  Returns
    (pairs/s, seconds)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    import oracle as O
    O.build()
    w = T.WORKLOADS[WORKLOAD]
    seed = T.window_seed(2)
    n = len(pairs)
    shm = shared_memory.SharedMemory(create=True, size=pairs.nbytes)
    try:
        np.ndarray(pairs.shape, dtype=np.uint32, buffer=shm.buf)[:] = pairs
        bounds = np.linspace(0, n, workers + 1).astype(np.int64)
        jobs = [(shm.name, n, int(bounds[i]), int(bounds[i + 1]), w.sketch(), seed) for i in range(workers)]
        with mp.get_context("spawn").Pool(workers) as pool:
            pool.map(_oracle_part, [(shm.name, n, 0, 1, w.sketch(), seed)] * workers)  # start the workers
            t0 = time.perf_counter()
            grids = pool.map(_oracle_part, jobs)
            grid = grids[0]
            for g in grids[1:]:
                grid |= g
            O.close_window(O.params_from(w.sketch(), seed=seed), grid)
            dt = time.perf_counter() - t0
    finally:
        shm.close()
        shm.unlink()
    return n / dt, dt


def run_reference(args, rank, world):
    if rank != 0:
        return
    win = window_for(0)
    times = []
    rate = None
    for i in range(args.warmup + args.steps):
        r, dt = cpu_oracle_rate(win.pairs, args.ref_sample)
        if i >= args.warmup:
            times.append(dt)
            rate = r
    total = sum(times)
    value = args.steps * args.ref_sample / total / 1e9
    line = {
        "impl": "reference", "metric": "packets/s (Gpps)", "value": value, "unit": "Gpps",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "pairs_per_step": args.ref_sample},
        "cpu_baseline": {"value": value, "unit": "Gpps", "cores": 1, "kind": "oracle",
                         "sample": f"first {args.ref_sample} pairs of the window, update + close"},
        "e2e": {"value": value, "unit": "Gpps", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local):
    import torch

    from paper_1803_11449_gb300 import build as b
    b.build()
    from paper_1803_11449_gb300 import sd

    torch.cuda.set_device(local)
    win = window_for(rank, n=args.pairs)
    n = len(win.pairs)
    pairs_dev = torch.from_numpy(win.pairs.reshape(-1).view(np.int32)).cuda()
    pairs_host = torch.from_numpy(win.pairs.reshape(-1).view(np.int32)).pin_memory()
    # one explicit stream shared by the library and the timing events
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    w = T.WORKLOADS[WORKLOAD]
    p = sd.params_for(w, seed=T.window_seed(2), device=local, cuda_stream=stream.cuda_stream)
    h = sd.sd_create(p)
    tuned = None
    if args.tuning:
        knobs = {kv.split("=")[0]: int(kv.split("=")[1], 0) for kv in args.tuning.split(",")}
        knobs.setdefault("mode", sd.sd_get_tuning(h).mode)
        sd.sd_set_tuning(h, **knobs)
    elif args.mode is not None or args.unroll or args.threads:
        sd.sd_set_tuning(h, mode=args.mode if args.mode is not None else sd.sd_get_tuning(h).mode,
                         unroll=args.unroll, block_threads=args.threads)
    elif args.autotune:
        from paper_1803_11449_gb300.tune import autotune
        tuned = autotune(h, pairs_dev, stream, verbose=args.verbose)
    # a second sketch of the same link on its own stream: window w+1 is
    # ingested while window w closes (two DHLAs in turn, as a monitor that
    # keeps counting during a close would run)
    stream2 = torch.cuda.Stream()
    h2 = sd.sd_create(sd.params_for(w, seed=T.window_seed(2), device=local, cuda_stream=stream2.cuda_stream))
    t1 = sd.sd_get_tuning(h)
    sd.sd_set_tuning(h2, **{f: getattr(t1, f) for f, _ in sd.sd_tuning._fields_})
    hs, streams = (h, h2), (stream, stream2)

    def timed(steps, pipelined):
        """`steps` windows, each sd_update then sd_close_window; pipelined:
        the two sketches alternate and window w's close overlaps window
        w+1's update.  Returns (elapsed s, per-update s, last report)."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_mid = torch.cuda.Event()
        t_start.record(stream)
        stream2.wait_event(t_start)
        rep = None
        for i in range(steps):
            k = (i & 1) if pipelined else 0
            ev[i][0].record(streams[k])
            sd.sd_update(hs[k], pairs_dev)
            ev[i][1].record(streams[k])
            if not pipelined:
                rep = sd.sd_close_window(hs[0])
            elif i > 0:
                rep = sd.sd_close_window(hs[1 - k])
        if pipelined:
            rep = sd.sd_close_window(hs[(steps - 1) & 1])
        t_mid.record(stream2)
        stream.wait_event(t_mid)
        t_end.record(stream)
        torch.cuda.synchronize()
        return t_start.elapsed_time(t_end) / 1e3, [a.elapsed_time(b_) / 1e3 for a, b_ in ev], rep

    for _ in range(max(1, args.warmup // 2)):
        timed(2, True)
        timed(2, False)
    torch.cuda.synchronize()

    close_ms = []
    dist_barrier(world)
    torch.cuda.synchronize()
    launches0 = sd.sd_kernel_launches()
    with ClockSampler(local) as clk:
        elapsed, upd, rep = timed(args.steps, not args.sequential)
    launches = sd.sd_kernel_launches() - launches0
    dist_barrier(world)
    elapsed_max = dist_max(elapsed, world)
    value = world * args.steps * n / elapsed_max / 1e9
    # the other schedule, for reference
    el2, upd2, _ = timed(args.steps, args.sequential)
    el2_max = dist_max(el2, world)
    # the roofline takes the update kernels alone (the sequential schedule);
    # in the pipelined one a close overlaps them
    upd_alone, upd_piped = (upd, upd2) if args.sequential else (upd2, upd)
    other = world * args.steps * n / el2_max / 1e9

    # window-close latency on its own: the update has finished when the
    # clock starts; the report is on the host when it stops
    for _ in range(max(args.steps, 20)):
        sd.sd_update(h, pairs_dev)
        torch.cuda.synchronize()
        c0 = time.perf_counter()
        sd.sd_close_window(h)
        close_ms.append(1e3 * (time.perf_counter() - c0))

    # end to end: pinned host pairs through sd_update (H2D in the timed
    # region), report back to the host in sd_close_window.  In the pipelined
    # schedule a second host thread closes window w (its own sketch) while
    # the main thread ingests window w+1 into the other sketch, so the
    # host-to-device link does not wait for the close.
    from concurrent.futures import ThreadPoolExecutor

    def e2e_run(steps, pipelined):
        d2h = 0
        if not pipelined:
            for _ in range(steps):
                sd.sd_update(h, pairs_host)
                d2h += 296 + 8 * sd.sd_close_window(h).n_hits_total
            return d2h
        with ThreadPoolExecutor(1) as ex:
            fut = None
            for i in range(steps):
                sd.sd_update(hs[i & 1], pairs_host)
                if fut is not None:
                    d2h += 296 + 8 * fut.result().n_hits_total
                fut = ex.submit(sd.sd_close_window, hs[i & 1])
            d2h += 296 + 8 * fut.result().n_hits_total
        return d2h

    e2e_run(2, not args.sequential)
    torch.cuda.synchronize()
    dist_barrier(world)
    e0 = time.perf_counter()
    d2h = e2e_run(args.e2e_steps, not args.sequential)
    torch.cuda.synchronize()
    e_el = dist_max(time.perf_counter() - e0, world)
    e2e = world * args.e2e_steps * n / e_el / 1e9
    # the other schedule, for reference
    e2e_run(2, args.sequential)
    torch.cuda.synchronize()
    dist_barrier(world)
    e0 = time.perf_counter()
    e2e_run(args.e2e_steps, args.sequential)
    torch.cuda.synchronize()
    e2e_other = world * args.e2e_steps * n / dist_max(time.perf_counter() - e0, world) / 1e9
    tuning = sd.sd_get_tuning(h)
    sd.sd_destroy(h)
    sd.sd_destroy(h2)

    peak, peak_kind = measured_peaks()
    t_upd = statistics.mean(upd_alone)
    # the on-chip bound of the binned updates: r * dirs random shared-memory
    # atomic ORs per pair (the apply step), against their rate measured now
    onchip = None
    if tuning.mode in (5, 6):
        ceiling = smem_or_ceiling()
        achieved_ops = p.r * p.dirs * n / t_upd
        onchip = {"bound": "shared-memory atomic ORs", "ops_per_pair": p.r * p.dirs,
                  "achieved_ops_per_s": achieved_ops, "peak_ops_per_s": ceiling,
                  "frac": achieved_ops / ceiling if ceiling else None,
                  "peak_source": "sdc_smem_or_rate (random 32-bit atomic ORs into shared memory), measured in "
                                 "this run"}
    achieved = BYTES_PER_PAIR * n / t_upd / 1e9
    clocks = clk.summary()
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        parts = {}
        r, dt = cpu_oracle_rate(win.pairs, args.cpu_sample, parts)
        cpu = {"value": r / 1e9, "unit": "Gpps", "cores": 1, "kind": "oracle",
               "sample": f"first {args.cpu_sample} pairs of the window: oracle update + close "
                         f"({dt:.1f} s, single thread: update {parts['update_s']:.2f} s, "
                         f"close {parts['close_s']:.2f} s)",
               "update_gpps": args.cpu_sample / parts["update_s"] / 1e9, "close_s": parts["close_s"]}
        workers = os.cpu_count() or 1
        rp, dtp = cpu_oracle_parallel(win.pairs, workers)
        cpu["parallel"] = {"value": rp / 1e9, "unit": "Gpps", "cores": workers,
                           "sample": f"the whole window split over {workers} processes, one grid each, "
                                     f"OR-merged, then the oracle's close ({dtp:.1f} s)"}
    line = {
        "metric": "packets/s (Gpps)", "value": value, "unit": "Gpps", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "pairs_per_step_per_gpu": n,
                   "l2": (f"inputs larger than L2 ({BYTES_PER_PAIR * n / 2**20:.0f} MiB of pairs per step)"
                          if BYTES_PER_PAIR * n > 129e6 else
                          f"inputs of {BYTES_PER_PAIR * n / 2**20:.0f} MiB fit L2 and are not flushed: "
                          "a development number, not a bench value"),
                   "parallelism": f"{world} independent link(s), one per GPU",
                   "traffic": args.traffic,
                   "tuning": dict({f: getattr(tuning, f) for f, _ in tuning._fields_},
                                  autotuned=tuned is not None)},
        "schedule": ("sequential: one sketch, each window's close before the next update" if args.sequential else
                     "pipelined: two sketches of the link in turn, window w closes while w+1 is ingested"),
        ("pipelined" if args.sequential else "sequential"): {"value": other, "unit": "Gpps",
                                                             "ms_per_step": 1e3 * el2_max / args.steps,
                                                             "e2e": e2e_other},
        "gbps_at_800B": value * 1e9 * GBITS_PER_PACKET,
        "close_latency_ms": {"p50": float(np.percentile(close_ms, 50)),
                             "p99": float(np.percentile(close_ms, 99)), "samples": len(close_ms)},
        "update_ms": 1e3 * t_upd,
        "update_ms_in_pipeline": 1e3 * statistics.mean(upd_piped),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": profiled_traffic(tuning.mode, n) if WORKLOAD == "core" else None,
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "nominal": NOMINAL_HBM_GBS,
                     "kernel": UPDATE_KERNELS.get(tuning.mode, "k_update"),
                     "timed": "CUDA events around each sd_update of the sequential schedule "
                              "(the update kernels alone on the library's stream)",
                     "peak_source": f"hbm_gbs, {peak_kind}",
                     "algorithmic_bytes_per_pair": BYTES_PER_PAIR},
        "l2_random_op_roofline": l2_roofline(p.r * p.dirs, n, t_upd),
        "onchip_roofline": onchip,
        "e2e": {"value": e2e, "unit": "Gpps", "h2d_bytes_per_step": BYTES_PER_PAIR * n,
                "d2h_bytes_per_step": int(d2h / max(1, args.e2e_steps))},
        "gpu_launches": launches,
        "clocks": clocks,
        "report": {"hits": int(rep.n_hits_total), "n_cand": rep.n_cand,
                   "n_hot_row0": [int(x) for x in rep.n_hot[:, 0]]},
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def run_shard(args, rank, world, local):
    """One core window split over the ranks' GPUs (strong scaling): rank r
    updates the r-th contiguous part of the window, the DHLAs are OR-merged
    across ranks (shard.merge_across: all-to-all, the library's OR, an
    all-gather), and the window is closed.  Every rank closes the merged
    DHLA (the same report everywhere, and each rank's DHLA is cleared for the
    next window); the elapsed time is the maximum over ranks."""
    import torch
    import torch.distributed as dist

    from paper_1803_11449_gb300 import build as b
    b.build()
    from paper_1803_11449_gb300 import sd, shard

    torch.cuda.set_device(local)
    win = window_for(0, n=args.pairs)          # the same window on every rank
    n = len(win.pairs)
    part = np.array_split(win.pairs, world)[rank]
    mine = torch.from_numpy(np.ascontiguousarray(part).reshape(-1).view(np.int32)).cuda()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    w = T.WORKLOADS[WORKLOAD]
    h = sd.sd_create(sd.params_for(w, seed=T.window_seed(2), device=local, cuda_stream=stream.cuda_stream))
    group = dist.group.WORLD if world > 1 else None

    def step():
        sd.sd_update(h, mine)
        if world > 1:
            shard.merge_across(h, group)
        return sd.sd_close_window(h)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    dist_barrier(world)
    launches0 = sd.sd_kernel_launches()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            rep = step()
        torch.cuda.synchronize()
        elapsed = time.perf_counter() - t0
    launches = sd.sd_kernel_launches() - launches0
    dist_barrier(world)
    el = dist_max(elapsed, world)
    sd.sd_destroy(h)
    if rank != 0:
        return
    value = args.steps * n / el / 1e9
    line = {
        "metric": "packets/s (Gpps)", "value": value, "unit": "Gpps", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "pairs_per_step": n, "pairs_per_step_per_gpu": len(part),
                   "parallelism": f"one window split over {world} GPU(s); DHLAs OR-merged across GPUs "
                                  "(all-to-all, OR kernel, all-gather) before the close"},
        "timed": "host clock around sd_update + merge + sd_close_window per step (report on the host)",
        "gpu_launches": launches, "clocks": clk.summary(),
        "report": {"hits": int(rep.n_hits_total), "n_cand": rep.n_cand},
    }
    print(json.dumps(line), flush=True)


def run_noalloc(args, rank, world, local):
    """sd_update_noalloc (the binned update with its scratch in a fixed
    array inside the library) on the core window, beside sd_update in the
    same binned mode (5) and in the default mode: CUDA events around each
    call, pairs resident in HBM (one JSON line)."""
    import torch

    from paper_1803_11449_gb300 import build as b
    b.build()
    from paper_1803_11449_gb300 import sd

    torch.cuda.set_device(local)
    win = window_for(rank, n=args.pairs)
    n = len(win.pairs)
    dev = torch.from_numpy(win.pairs.reshape(-1).view(np.int32)).cuda()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    w = T.WORKLOADS[WORKLOAD]
    p = sd.params_for(w, seed=T.window_seed(2), device=local, cuda_stream=stream.cuda_stream)
    grid = torch.zeros(p.dirs * sd.sd_grid_words(p), dtype=torch.int32, device="cuda")

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            e.record(stream)
            e.synchronize()
            ts.append(a.elapsed_time(e))
        return statistics.median(ts)

    def noalloc():
        rc = sd.sd_update_noalloc(p, grid, dev, stream)
        assert rc == sd.SD_OK, rc
    timed(noalloc, args.warmup)
    t_na = timed(noalloc, args.steps)
    out = {"metric": "sd_update_noalloc, pairs/s (Gpairs/s)", "n_pairs": n, "workload": WORKLOAD_DESC,
           "noalloc_ms": t_na, "noalloc_gpps": n / t_na / 1e6}
    for mode in (5, None):
        h = sd.sd_create(p)
        if mode is not None:
            sd.sd_set_tuning(h, mode=mode)
        timed(lambda: sd.sd_update(h, dev), args.warmup)
        t = timed(lambda: sd.sd_update(h, dev), args.steps)
        key = "sd_update_mode5" if mode == 5 else f"sd_update_default_mode{sd.sd_get_tuning(h).mode}"
        out[key + "_ms"] = t
        out[key + "_gpps"] = n / t / 1e6
        sd.sd_destroy(h)
    if rank == 0:
        print(json.dumps(out), flush=True)


def _batch_window(args):
    """(pairs, planted count) of link `link` of the batching workload."""
    link, n, planted = args
    w = T.WORKLOADS[WORKLOAD].with_(n=n, planted=planted)
    return T.make_window(w, T.window_seed(3, link=link)).pairs


def run_batching(args, rank, world, local):
    """Many links of uneven size: one window at a time through one handle
    versus all links batched (sd_update_many + sd_close_many).  Every link
    uses the core-link sketch; links differ by traffic."""
    import multiprocessing as mp

    rng = np.random.default_rng(0x5D5A0300 + rank)
    sizes = np.clip(np.exp(rng.normal(np.log(4 << 20), 1.0, size=args.links)), 256 << 10, 64 << 20)
    sizes = (sizes.astype(np.int64) // 2) * 2
    planted = rng.integers(50, 301, size=args.links)
    jobs = [(rank * args.links + i, int(n), int(p)) for i, (n, p) in enumerate(zip(sizes, planted))]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        wins = pool.map(_batch_window, jobs)

    import torch

    from paper_1803_11449_gb300 import build as b
    b.build()
    from paper_1803_11449_gb300 import sd

    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    devs = [torch.from_numpy(wn.reshape(-1).view(np.int32)).cuda() for wn in wins]
    total = int(sum(len(wn) for wn in wins))
    w = T.WORKLOADS[WORKLOAD]
    seed = T.window_seed(2)
    hs = [sd.sd_create(sd.params_for(w, seed=seed, device=local, cuda_stream=stream.cuda_stream))
          for _ in wins]
    one = hs[0]
    tuned = None
    if args.autotune:
        from paper_1803_11449_gb300.tune import autotune_many
        tuned = autotune_many(hs, devs, stream, verbose=args.verbose)

    def one_at_a_time():
        lat = []
        for d in devs:
            sd.sd_update(one, d)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sd.sd_close_window(one)
            lat.append(time.perf_counter() - t0)
        return lat

    def batched():
        sd.sd_update_many(hs, devs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sd.sd_close_many(hs)
        return time.perf_counter() - t0

    for _ in range(max(1, args.warmup // 3)):
        one_at_a_time()
        batched()
    torch.cuda.synchronize()
    t_one, t_bat, lat_one, lat_bat = [], [], [], []
    for _ in range(args.batch_reps):
        t0 = time.perf_counter()
        lat_one += one_at_a_time()
        torch.cuda.synchronize()
        t_one.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        lat_bat.append(batched())
        torch.cuda.synchronize()
        t_bat.append(time.perf_counter() - t0)
    tuning = {f: getattr(sd.sd_get_tuning(one), f) for f, _ in sd.sd_tuning._fields_}
    for h in hs:
        sd.sd_destroy(h)
    one_v = dist_max(min(t_one), world)
    bat_v = dist_max(min(t_bat), world)
    if rank != 0:
        return
    line = {
        "metric": "packets/s (Gpps), batched windows", "value": world * total / bat_v / 1e9,
        "unit": "Gpps", "n_gpus": args.gpus, "steps": args.batch_reps, "warmup": args.warmup,
        "ms_per_step": 1e3 * bat_v, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"batching: {args.links} links, window sizes lognormal (median 4M pairs, "
                               "clipped to [256K, 64M]), 50-300 planted each, core-link sketch per link",
                   "pairs_per_step_per_gpu": total,
                   "tuning": tuning, "autotuned": tuned is not None},
        "one_window_at_a_time": {"value": world * total / one_v / 1e9, "unit": "Gpps",
                                 "ms_per_step": 1e3 * one_v,
                                 "close_ms_per_window": {"p50": 1e3 * float(np.percentile(lat_one, 50)),
                                                         "p99": 1e3 * float(np.percentile(lat_one, 99))}},
        "batched_close_ms_all_links": {"p50": 1e3 * float(np.percentile(lat_bat, 50)),
                                       "p99": 1e3 * float(np.percentile(lat_bat, 99))},
    }
    print(json.dumps(line), flush=True)


def _serve_window(args):
    """Traffic of serving link `link` (one window, cycled through its ring):
    core-link traffic with 50-300 planted hosts; link 0 also carries a DDoS
    victim (one dst, `ddos` distinct spoofed srcs) and link 1 a scanner (one
    src, `scan` distinct dsts), written over random positions."""
    link, n, planted, ddos, scan = args
    w = T.WORKLOADS[WORKLOAD].with_(n=n, planted=planted)
    win = T.make_window(w, T.window_seed(4, link=link))
    pairs = win.pairs
    rng = np.random.default_rng(T.window_seed(4, link=link) ^ 0xDD05)
    special = None
    if link == 0 and ddos:
        victim = np.uint32(rng.integers(0, 2**32))
        pos = rng.choice(n, size=ddos, replace=False)
        pairs[pos, 0] = T.ip_of(0x7000_0000, np.arange(ddos), int(rng.integers(0, 2**32)))
        pairs[pos, 1] = victim
        special = (1, int(victim))
    elif link == 1 and scan:
        scanner = np.uint32(rng.integers(0, 2**32))
        pos = rng.choice(n, size=scan, replace=False)
        pairs[pos, 0] = scanner
        pairs[pos, 1] = T.ip_of(0x7100_0000, np.arange(scan), int(rng.integers(0, 2**32)))
        special = (0, int(scanner))
    return pairs, special


def run_serving(args, rank, world, local):
    """The serving engine in real time: `serve_links` links, each with its
    sketch resident under an HBM budget, take Poisson arrivals of batches of
    uniform [64K, 4M] pairs (sharing `serve_load` Gpps offered) into a
    device ring (the link's synthetic traffic, one window long, cycled);
    the engine (continuous batching, a window closed every `window_pairs`
    pairs of a link) runs for `serve_seconds`.  Reports the served rate,
    pairs dropped at full rings, the close latency (end of the completing
    update to the report on the host) and the latency from the arrival of a
    window's last batch to its report."""
    import multiprocessing as mp

    W, nl = args.window_pairs, args.serve_links
    rng = np.random.default_rng(0x5D5A0400 + rank)
    planted = rng.integers(50, 301, size=nl)
    jobs = [(rank * nl + i, W, int(p), args.serve_ddos, args.serve_scan) for i, p in enumerate(planted)]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        gen = pool.map(_serve_window, jobs)
    wins = [g[0] for g in gen]
    special = {i: g[1] for i, g in enumerate(gen) if g[1] is not None}
    rate = args.serve_load * 1e9 / nl                            # pairs/s per link
    lo, hi = 1 << 16, 1 << 22
    T_run = args.serve_seconds
    arr_t, arr_n = [], []
    for _ in range(nl):
        m = int(T_run * rate / ((lo + hi) / 2) * 1.3) + 16
        t = np.cumsum(rng.exponential((lo + hi) / 2 / rate, size=m))
        k = int(np.searchsorted(t, T_run))
        arr_t.append(t[:k])
        arr_n.append(rng.integers(lo, hi + 1, size=k))

    import torch

    from paper_1803_11449_gb300 import build as b
    b.build()
    from paper_1803_11449_gb300 import serving

    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    rings = [torch.from_numpy(wn.reshape(-1).view(np.int32)).cuda() for wn in wins]
    del wins
    srv = serving.Server(T.WORKLOADS[WORKLOAD], W, hbm_budget=int(args.serve_budget_gb * (1 << 30)),
                         device=local, stream=stream, bin_chunk_log2=args.serve_chunk_log2)
    admitted = 0
    for i in range(nl):
        admitted += srv.open_link(i, T.window_seed(4, link=rank * nl + i))
        srv.attach_ring(i, rings[i])
    # warm-up: one window on every admitted link
    for i in srv.admitted:
        srv.advance(i, W)
    srv.drain()
    torch.cuda.synchronize()
    found = {i: any(int(ip) == sp[1] for ip, d in zip(r.report.hits["ip"], r.report.hits["dir"]) if d == sp[0])
             for i, sp in special.items() for r in srv.reports if r.link == i}
    srv.reports.clear()
    base = {i: srv.links[i].tail for i in srv.admitted}
    win0 = {i: srv.links[i].window for i in srv.admitted}
    acc = {i: [] for i in srv.admitted}             # accepted batches: (pairs served after it, arrival)
    nxt = {i: 0 for i in srv.admitted}
    dropped = offered = 0
    clock = ClockSampler(local)
    t0 = time.perf_counter()
    with clock:
        while True:
            now = time.perf_counter() - t0
            if now >= T_run and srv.pending_pairs() == 0:
                break
            for i in srv.admitted:
                L = srv.links[i]
                while nxt[i] < len(arr_t[i]) and arr_t[i][nxt[i]] <= now:
                    n = int(arr_n[i][nxt[i]])
                    offered += n
                    if L.head + n - L.tail <= W:
                        srv.advance(i, n)
                        acc[i].append((L.head - base[i], arr_t[i][nxt[i]]))
                    else:
                        dropped += n
                    nxt[i] += 1
            if srv.pending_pairs():
                srv.step()
            elif now < T_run:
                time.sleep(20e-6)
        torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    srv.drain()  # the reports of closes still in flight
    served = sum(srv.links[i].tail - base[i] for i in srv.admitted)
    lat = []
    for r in srv.reports:
        end = (r.window - win0[r.link] + 1) * W
        a = acc[r.link]
        j = next((q for q, (cum, _) in enumerate(a) if cum >= end), None)
        if j is not None:
            lat.append(r.done_at - t0 - a[j][1])
    close = [r.close_s for r in srv.reports]
    n_win = len(srv.reports)
    steps = srv.steps
    admitted_links = list(srv.admitted)
    srv.shutdown()
    # the same offered load, one window at a time: each batch through
    # sd_update of its link's handle as it comes, each full window closed
    # with sd_close_window before the next batch is taken
    alone = _one_at_a_time(args, admitted_links, rings, arr_t, arr_n, T_run, local, stream, rank, nl)
    value = dist_max(elapsed, world)
    if rank != 0:
        return
    pct = lambda a, q: 1e3 * float(np.percentile(a, q)) if len(a) else None
    line = {
        "metric": "packets/s (Gpps), served under Poisson arrivals", "value": world * served / value / 1e9,
        "unit": "Gpps", "n_gpus": args.gpus, "steps": steps, "warmup": 1,
        "ms_per_step": 1e3 * elapsed / max(1, steps), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"serving: {nl} links, Poisson batches of uniform [64K, 4M] pairs sharing "
                               f"{args.serve_load} Gpps offered, a window closed every {W} pairs per link, "
                               f"core-link sketch per link, HBM budget {args.serve_budget_gb} GiB, "
                               f"DDoS victim ({args.serve_ddos} srcs) on link 0, scanner ({args.serve_scan} "
                               f"dsts) on link 1, {T_run} s",
                   "window_pairs": W, "offered_gpps": args.serve_load, "links": nl, "admitted": admitted},
        "offered_pairs": int(offered), "served_pairs": int(served), "dropped_pairs": int(dropped),
        "windows_closed": n_win, "attacks_reported_in_warmup_window": {str(k): v for k, v in found.items()},
        "latency_ms_last_arrival_to_report": {"p50": pct(lat, 50), "p99": pct(lat, 99), "n": len(lat)},
        "close_ms": {"p50": pct(close, 50), "p99": pct(close, 99)},
        "one_window_at_a_time": alone,
        "clocks": clock.summary(),
    }
    print(json.dumps(line), flush=True)


def _one_at_a_time(args, links, rings, arr_t, arr_n, T_run, local, stream, rank, nl):
    """The serving workload without the engine: one handle per link, every
    arriving batch fed by sd_update as it comes (oldest first), a link's
    window closed by sd_close_window as soon as it is full, all on one
    stream, one call at a time.  A batch that would leave a link with more
    than one window of arrived pairs not yet fed is dropped, as the engine's
    ring would.  Returns served Gpps,
    dropped pairs and the latency from a window's last batch to its report."""
    import heapq

    from paper_1803_11449_gb300 import sd

    W = args.window_pairs
    w = T.WORKLOADS[WORKLOAD]
    hs = {}
    for i in links:
        h = sd.sd_create(sd.params_for(w, seed=T.window_seed(4, link=rank * nl + i), device=local,
                                       cuda_stream=stream.cuda_stream))
        # batches are at most 2^22 pairs: bins for rounds of that size
        sd.sd_set_tuning(h, mode=sd.sd_get_tuning(h).mode, plane_round_log2=22)
        hs[i] = h
    fill = {i: 0 for i in links}          # pairs of the open window
    tail = {i: 0 for i in links}          # ring offset of the next pair
    backlog = {i: 0 for i in links}       # accepted, not yet fed
    events = []                           # (arrival, link, pairs): a global arrival-order queue
    for i in links:
        for t, n in zip(arr_t[i], arr_n[i]):
            events.append((float(t), i, int(n)))
    events.sort()
    queue = []
    served = dropped = 0
    lat, close = [], []
    nxt = 0

    def feed(i, n):
        ring = rings[i]
        off = tail[i] % W
        take = min(n, W - off)
        sd.sd_update(hs[i], ring[2 * off:2 * (off + take)])
        if take < n:
            sd.sd_update(hs[i], ring[:2 * (n - take)])
        tail[i] += n

    # warm-up: one window on every link
    for i in links:
        feed(i, W)
        sd.sd_close_window(hs[i])
    tail = {i: 0 for i in links}
    torch_sync = __import__("torch").cuda.synchronize
    torch_sync()
    t0 = time.perf_counter()
    while True:
        now = time.perf_counter() - t0
        while nxt < len(events) and events[nxt][0] <= now:
            t, i, n = events[nxt]
            nxt += 1
            if backlog[i] + n <= W:       # the engine's ring holds one window of arrived pairs
                heapq.heappush(queue, (t, i, n))
                backlog[i] += n
            else:
                dropped += n
        if not queue:
            if now >= T_run and nxt >= len(events):
                break
            time.sleep(20e-6)
            continue
        t, i, n = heapq.heappop(queue)
        backlog[i] -= n
        while n:
            take = min(n, W - fill[i])
            feed(i, take)
            fill[i] += take
            served += take
            n -= take
            if fill[i] == W:
                c0 = time.perf_counter()
                sd.sd_close_window(hs[i])
                done = time.perf_counter()
                close.append(done - c0)
                lat.append(done - t0 - t)
                fill[i] = 0
    torch_sync()
    elapsed = time.perf_counter() - t0
    for h in hs.values():
        sd.sd_destroy(h)
    pct = lambda a, q: 1e3 * float(np.percentile(a, q)) if len(a) else None
    return {"value": served / elapsed / 1e9, "unit": "Gpps", "served_pairs": int(served),
            "dropped_pairs": int(dropped), "windows_closed": len(close),
            "latency_ms_last_arrival_to_report": {"p50": pct(lat, 50), "p99": pct(lat, 99), "n": len(lat)},
            "close_ms": {"p50": pct(close, 50), "p99": pct(close, 99)},
            "schedule": "plain sd_update per batch and sd_close_window per full window, one call at a time, "
                        "one stream"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--cpu-sample", type=int, default=CPU_SAMPLE_PAIRS)
    ap.add_argument("--ref-sample", type=int, default=0,
                    help="pairs per reference step (default: 2^22, fewer for long runs so that the "
                         "reference arm stays within a few minutes)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--pairs", type=int, default=None,
                    help="pairs per window (default: the workload's 2^26); profiling only")
    ap.add_argument("--mode", type=int, default=None)
    ap.add_argument("--unroll", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--tuning", default="",
                    help="update-kernel knobs, e.g. mode=5,bin_slice_log2=15,bin_chunk_log2=24")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the update kernel's launch knobs by timing them first")
    ap.add_argument("--traffic", default="core", choices=["core", "uniform"],
                    help="uniform: every pair random (no Zipf, no planted hosts)")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--sequential", action="store_true",
                    help="one sketch: each window closes before the next is ingested")
    ap.add_argument("--batching", action="store_true",
                    help="many links of uneven size: batched versus one window at a time")
    ap.add_argument("--links", type=int, default=64)
    ap.add_argument("--batch-reps", type=int, default=3)
    ap.add_argument("--workload", default="core", choices=sorted(DESCS),
                    help="window and sketch configuration of the default mode")
    ap.add_argument("--serving", action="store_true",
                    help="the serving engine in real time under Poisson arrivals")
    ap.add_argument("--noalloc", action="store_true",
                    help="time sd_update_noalloc beside sd_update on the window")
    ap.add_argument("--ceilings", action="store_true",
                    help="measure the on-chip and host-link rates that bound the update")
    ap.add_argument("--shard", action="store_true",
                    help="one window split over the GPUs, DHLAs OR-merged across them (strong scaling)")
    ap.add_argument("--serve-links", type=int, default=16)
    ap.add_argument("--window-pairs", type=int, default=1 << 26)
    ap.add_argument("--serve-load", type=float, default=10.0, help="offered Gpps, all links")
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    ap.add_argument("--serve-budget-gb", type=float, default=2.0)
    ap.add_argument("--serve-chunk-log2", type=int, default=22)
    ap.add_argument("--serve-ddos", type=int, default=2_000_000)
    ap.add_argument("--serve-scan", type=int, default=500_000)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if not args.ref_sample:
        args.ref_sample = ref_sample_for(args.steps, args.warmup)
    global TRAFFIC, WORKLOAD, WORKLOAD_DESC
    TRAFFIC = args.traffic
    if not (args.batching or args.serving):
        WORKLOAD, WORKLOAD_DESC = args.workload, DESCS[args.workload]
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.batching:
        run_batching(args, rank, world, local)
    elif args.serving:
        run_serving(args, rank, world, local)
    elif args.shard:
        run_shard(args, rank, world, local)
    elif args.ceilings:
        run_ceilings(args, rank, world, local)
    elif args.noalloc:
        run_noalloc(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
