"""The C-ABI library builds, loads and exports every symbol include/fwr.h
declares; argument errors are reported before any device work (CPU only)."""

import ctypes
import os
import re

import numpy as np
import pytest

from paper_1705_04298_gb300 import build_lib, fwr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fwr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fwr_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(fwr.LIB_PATH):
        build_lib.build()
    return fwr.load()


def test_every_declared_symbol_is_exported_and_bound(lib):
    names = _declared()
    assert "fwr_plan_create" in names and "fwr_reconstruct" in names
    for name in names:
        assert hasattr(lib, name), name
        assert name in fwr.SIGNATURES, name
    assert set(fwr.SIGNATURES) == set(names)


def test_status_strings(lib):
    for code, name in fwr.STATUS.items():
        assert lib.fwr_status_string(code).decode() == name


def _create(lib, n=16, pad=2.0, mask=None, filt=0, nv=0.0, r0=1.0, L0=10.0):
    m = np.ones((n, n), np.uint8) if mask is None else np.ascontiguousarray(mask, np.uint8)
    h = ctypes.c_void_p()
    code = lib.fwr_plan_create(ctypes.byref(h), n, pad, m.ctypes.data_as(ctypes.c_void_p), filt, nv, r0, L0)
    return code, h


def test_invalid_plans_rejected_before_device_work(lib):
    ARG, UNSUP = 1, 2
    assert _create(lib, n=1)[0] == ARG
    assert _create(lib, n=16, pad=1.0)[0] == ARG          # N = 16 < n + 2
    assert _create(lib, n=16, pad=0.5)[0] == ARG
    assert _create(lib, n=16, pad=float("nan"))[0] == ARG
    assert _create(lib, n=16, mask=np.zeros((16, 16)))[0] == ARG
    assert _create(lib, n=16, filt=7)[0] == ARG
    assert _create(lib, n=16, nv=-1.0)[0] == ARG
    assert _create(lib, n=16, filt=1, r0=0.0)[0] == ARG
    assert _create(lib, n=16, filt=1, L0=-3.0)[0] == ARG
    assert _create(lib, n=300, pad=2.0)[0] == UNSUP        # N = 1024
    code, h = _create(lib, n=16)
    assert code == 0 or code == 3  # plan needs a device; without one it is a CUDA error
    if code == 0:
        lib.fwr_plan_destroy(h)


def test_null_plan_calls(lib):
    assert lib.fwr_plan_grid(None) == -1
    assert lib.fwr_plan_valid_count(None) == -1
    assert lib.fwr_reconstruct(None, None, 0, 0, None, None) == 1
    assert lib.fwr_reconstruct_ex(None, None, None, 0, 0, None, None, None) == 1
    assert lib.fwr_plan_set_option(None, 1, 0.0) == 1
    assert lib.fwr_fft2(48, None, None, 1, 0, None) == 1
    assert lib.fwr_fft2(32, None, None, 0, 0, None) == 0
    assert lib.fwr_plan_shape(None) == -1 and lib.fwr_plan_ctas(None) == -1 and lib.fwr_plan_l2_persist(None) == -1
    assert lib.fwr_plan_set_option(None, fwr.OPT_L2_PERSIST, 1.0) == 1
    assert lib.fwr_l2_persist_reset(-1) == 1  # no such device
    assert lib.fwr_plan_autotune(None, None, 1, 1, None, None, None) == 1
    lib.fwr_plan_destroy(None)


def test_python_constants_match_the_header():
    """Every #define of include/fwr.h that the binding mirrors has the same
    value in fwr.py (option keys and their values, filters, limits)."""
    src = open(os.path.join(ROOT, "include", "fwr.h")).read()
    defines = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+FWR_([A-Z0-9_]+)\s+(-?\d+)", src)}
    mirrored = {
        "OPT_PERIODIC": fwr.OPT_PERIODIC, "OPT_TRANSFORM": fwr.OPT_TRANSFORM, "OPT_G_MODEL": fwr.OPT_G_MODEL,
        "OPT_PIXEL": fwr.OPT_PIXEL, "OPT_EXTENSION": fwr.OPT_EXTENSION, "G_AVERAGED": fwr.G_AVERAGED,
        "G_FRIED": fwr.G_FRIED, "EXT_ZERO": fwr.EXT_ZERO, "EXT_HUDGIN": fwr.EXT_HUDGIN,
        "PERIODIC_BEFORE_EACH_FFT": fwr.PERIODIC_BEFORE_EACH_FFT, "PERIODIC_FINAL_ONLY": fwr.PERIODIC_FINAL_ONLY,
        "PERIODIC_NONE": fwr.PERIODIC_NONE, "TRANSFORM_FFT": fwr.TRANSFORM_FFT,
        "TRANSFORM_DFT_BF16X3": fwr.TRANSFORM_DFT_BF16X3, "TRANSFORM_DFT_BF16X6": fwr.TRANSFORM_DFT_BF16X6,
        "OPT_SHAPE": fwr.OPT_SHAPE, "OPT_CTAS": fwr.OPT_CTAS, "OPT_L2_PERSIST": fwr.OPT_L2_PERSIST,
    }
    for name, value in mirrored.items():
        assert defines.get(name) == value, name
