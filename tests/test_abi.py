"""The C-ABI library builds, loads and exports every entry point that
include/mf.h declares; host-side descriptor validation (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2003_02978_gb300 import build
    build.build()
    from paper_2003_02978_gb300._native import lib as _lib
    return _lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mf_[a-z_]+)\s*\(", src)))


def test_header_declares_api():
    names = declared_functions()
    for n in ("mf_plan", "mf_retrieve", "mf_destroy", "mf_plan_status", "mf_retrieve_host",
              "mf_background", "mf_status_string", "mf_last_error", "mf_profile",
              "mf_profile_read", "mf_num_partitions"):
        assert n in names


def test_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_flag_values_match_the_binding():
    import paper_2003_02978_gb300 as mfg
    src = open(os.path.join(ROOT, "include", "mf.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in
            re.finditer(r"#define MF_([A-Z_]+)\s+(\d+)u", src)}
    for name in ("ALBEDO", "SPARSE", "LITERAL", "PENALTY_NO_ALBEDO", "PERSISTENT"):
        assert defs[name] == getattr(mfg, name), name


def test_status_strings(lib):
    for s in range(0, 9):
        assert lib.mf_status_string(s)


def _desc(**kw):
    from paper_2003_02978_gb300._native import MfDesc
    d = dict(rows=100, cols=4, bands_total=72, band_lo=0, band_hi=72, col_group=1, layout=0,
             precision=0, flags=3)
    d.update(kw)
    return MfDesc(**d)


@pytest.mark.parametrize("kw,code", [
    (dict(rows=0), 1), (dict(cols=-1), 1), (dict(band_lo=10, band_hi=8), 1),
    (dict(band_hi=80), 1), (dict(col_group=0), 1), (dict(layout=3), 8),
    (dict(precision=7), 1), (dict(precision=1, bands_total=128, band_hi=128), 8),
    (dict(precision=1, bands_total=32, band_hi=32), 8), (dict(precision=1, band_lo=12), 8),
    (dict(flags=1 << 9), 1), (dict(flags=3 | 4 | 16), 1),  # MF_PERSISTENT with MF_LITERAL
    (dict(band_lo=2, band_hi=74, bands_total=80), 8),
    (dict(band_lo=0, band_hi=6), 8), (dict(bands_total=200, band_hi=200), 8),
])
def test_descriptor_validation(lib, kw, code):
    h = ctypes.c_void_p()
    assert lib.mf_plan(ctypes.byref(_desc(**kw)), ctypes.byref(h)) == code
    assert h.value is None
    assert lib.mf_last_error()


def test_batched_plan_validation(lib):
    from paper_2003_02978_gb300._native import MfDesc
    h = ctypes.c_void_p()
    rows = (ctypes.c_int64 * 3)(100, 200, 300)
    assert lib.mf_plan_batched(ctypes.byref(_desc(rows=601)), rows, 3, ctypes.byref(h)) == 1
    assert b"sum of the line rows" in lib.mf_last_error()
    bad = (ctypes.c_int64 * 3)(100, -5, 505)
    assert lib.mf_plan_batched(ctypes.byref(_desc(rows=600)), bad, 3, ctypes.byref(h)) == 1
    assert lib.mf_plan_batched(ctypes.byref(_desc(rows=600)), rows, 0, ctypes.byref(h)) == 1
    assert lib.mf_plan_batched(ctypes.byref(_desc(rows=600)), None, 3, ctypes.byref(h)) == 1
    assert lib.mf_num_lines(None) == -1
    assert lib.mf_plan_ex(None, None, 1, None, ctypes.byref(h)) == 1
    assert lib.mf_plan_ex(ctypes.byref(_desc(rows=601)), rows, 3, None, ctypes.byref(h)) == 1
    assert lib.mf_retrieve_batched(None, None, None, None, 1e-9, None, None, None, None) == 1


def test_null_arguments(lib):
    assert lib.mf_plan(None, None) == 1
    assert lib.mf_retrieve(None, None, None, 1.0, 1.0, 1, None, None, None, None, None) == 1
    assert lib.mf_plan_status(None, None) == 1
    assert lib.mf_num_partitions(None) == -1
