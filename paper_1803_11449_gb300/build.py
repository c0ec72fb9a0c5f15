"""Build the CUDA library ``_build/libsd.so`` for GB300 (sm_103a) with nvcc.

The translation units are compiled in parallel and linked into one shared
library with the CUDA runtime linked statically, so the library loads on a
machine without a GPU (the driver is only needed at the first CUDA call).
Host code is compiled with ``-ffp-contract=off`` so the double-precision
formulas evaluated on the host round step by step, as written.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libsd.so")
# microbenchmarks of the rates that bound the update (the benchmark's
# roofline lines); a library of its own, not part of the detection API
CEILINGS_SRC = "sd_ceilings.cu"
CEILINGS_LIB = os.path.join(OUT_DIR, "libsd_ceilings.so")
SOURCES = ["sd_update.cu", "sd_binned.cu", "sd_plane.cu", "sd_fold.cu", "sd_close.cu", "sd_join.cu", "sd_shard.cu",
           "sd_api.cu", "sd_noalloc.cu"]
HEADERS = [os.path.join(CSRC, "sd_common.cuh"), os.path.join(INCLUDE, "sd.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off,-fno-fast-math",
                "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the sd library")


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if needed) and return the path of libsd.so."""
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    objs, procs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + HEADERS):
            cmd = [cc] + FLAGS + ["-c", s, "-o", o]
            if verbose:
                print(" ".join(cmd))
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((cmd, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"))
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    if force or procs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    csrc = os.path.join(CSRC, CEILINGS_SRC)
    if force or _stale(CEILINGS_LIB, [csrc]):
        tmp = CEILINGS_LIB + f".tmp{os.getpid()}"
        cmd = [cc] + FLAGS + ["-shared", csrc, "-o", tmp]
        res = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if res.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + res.stdout.decode(errors="replace"))
        os.replace(tmp, CEILINGS_LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
