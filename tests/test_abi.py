"""The C-ABI library: it builds, loads without a GPU, exports every symbol the
header declares, and its host-only parameter logic agrees with the paper's
restrictions (§3.3).  No compute call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sdmod():
    from paper_1803_11449_gb300 import build as b
    b.build()
    from paper_1803_11449_gb300 import sd
    sd.lib()
    return sd


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w \*]*?\b(sd_\w+)\s*\(", text, flags=re.M)
    return names


def test_every_declared_symbol_is_exported(sdmod):
    names = _declared()
    assert "sd_create" in names and "sd_close_window" in names
    L = ctypes.CDLL(sdmod.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(sdmod.EXPORTS)


def test_struct_sizes_match_the_header(sdmod):
    # sizes derived by hand from the field lists in include/sd.h (LP64)
    assert ctypes.sizeof(sdmod.sd_params) == 80
    assert ctypes.sizeof(sdmod.sd_hit) == 24
    assert ctypes.sizeof(sdmod.sd_report) == 272
    assert ctypes.sizeof(sdmod.sd_tuning) == 56


def test_default_params_and_grid_words(sdmod):
    p = sdmod.sd_default_params()
    assert (p.g, p.r, p.k, p.alpha, p.dirs, p.theta) == (512, 4, 16, 8, 2, 1024.0)
    assert sdmod.sd_check_params(p) == 0
    assert sdmod.sd_grid_words(p) == 4 * (1 << 16) * 16
    assert sdmod.sd_device_bytes(p) > 2 * 4 * sdmod.sd_grid_words(p)


def test_param_checks_agree_with_the_oracle(sdmod, O):
    rng = np.random.default_rng(0)
    for _ in range(400):
        g = int(2 ** rng.integers(4, 14))
        r = int(rng.integers(2, 10))
        k = int(rng.integers(0, 27))
        a = int(rng.integers(0, 28))
        th = float(rng.choice([1024.0, 0.0, -3.0, 7.5]))
        p = sdmod.sd_default_params(g=g, r=r, k=k, alpha=a, theta=th, dirs=int(rng.integers(0, 4)))
        op = O.make_params(g, r, k, a, th, 0, dirs=p.dirs)
        assert (sdmod.sd_check_params(p) == 0) == O.check_params(op), (g, r, k, a, th, p.dirs)
        if sdmod.sd_check_params(p) == 0:
            assert sdmod.sd_grid_words(p) * p.dirs == O.grid_words(op)
        else:
            assert sdmod.sd_grid_words(p) == 0


def test_create_rejects_invalid_parameters_without_touching_a_gpu(sdmod):
    p = sdmod.sd_default_params(alpha=3)  # (r-2) alpha + k = 22 < 32
    with pytest.raises(sdmod.SdError) as e:
        sdmod.sd_create(p)
    assert e.value.code == sdmod.SD_ERR_ARG
    assert "invalid parameters" in sdmod.sd_last_error(None)


def test_entry_points_reject_null_arguments_without_touching_a_gpu(sdmod):
    """The header's error contract for missing arguments: every entry point
    that takes a handle or a buffer returns SD_ERR_ARG for NULL (a NULL
    handle to sd_destroy is a no-op, an empty batch is SD_OK) before any
    CUDA call, so the checks hold on a machine without a GPU."""
    L = sdmod.lib()
    ARG, OK = sdmod.SD_ERR_ARG, sdmod.SD_OK
    buf = (ctypes.c_uint32 * 64)()
    rep = sdmod.sd_report()
    tun = sdmod.sd_tuning()
    assert L.sd_update(None, buf, 1) == ARG
    assert L.sd_close_window(None, ctypes.byref(rep)) == ARG
    assert L.sd_sync(None) == ARG
    assert L.sd_destroy(None) == OK
    assert L.sd_get_grid(None, 0, buf) == ARG
    assert L.sd_set_grid(None, 0, buf) == ARG
    assert L.sd_get_hot(None, 0, 0, buf) == ARG
    assert L.sd_get_candidates(None, 0, buf, 64) == ARG
    assert L.sd_merge(None, None) == ARG
    assert L.sd_get_tuning(None, ctypes.byref(tun)) == ARG
    assert L.sd_set_tuning(None, ctypes.byref(tun)) == ARG
    assert L.sd_scratch_bytes(None, 1) == 0
    assert L.sd_check_params(None) == ARG
    assert L.sd_update_many(None, None, None, 0) == OK
    assert L.sd_update_many(None, None, None, 2) == ARG
    assert L.sd_close_many(None, 0, None, None) == OK
    assert L.sd_close_many(None, 2, None, None) == ARG
    p = sdmod.sd_default_params()
    assert L.sd_update_noalloc(ctypes.byref(p), None, buf, 1, None) == ARG  # no DHLA
    assert L.sd_update_noalloc(None, buf, buf, 1, None) == ARG              # no parameters
    assert L.sd_update_dir(None, 0, buf, 1) == ARG
    assert L.sd_export_grid(None, buf) == ARG
    assert L.sd_or_grid(None, buf) == ARG
    assert L.sd_or_words(None, buf, 4, 1, None) == ARG
    assert L.sd_or_words(buf, buf, 3, 1, None) == ARG                    # words not a multiple of 4
    counts = (ctypes.c_uint64 * 4)()
    assert L.sd_partition_pairs(None, 0, buf, 1, 4, buf, counts) == ARG
    assert isinstance(L.sd_last_error(None), bytes)
