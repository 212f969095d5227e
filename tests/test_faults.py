"""Failure detection, driven by the MF_FAULT hook (read at plan creation);
nothing here faults, traps or hangs a GPU.

* alloc:   mf_plan returns MF_ERR_OOM before any CUDA call (host side, runs
           without a GPU);
* notspd:  every partition's initial covariance is reported not positive
           definite: status MF_ERR_NOT_SPD, alpha NaN on valid pixels, 0 on
           masked ones;
* timeout: every pixel-kernel CTA of the first pass makes a 2000-cycle wait
           on a barrier that nothing arrives on; the wait runs out, the CTA
           waits (with the normal limit) for the copies it issued, records
           MF_ERR_TIMEOUT and leaves; the later passes write NaN.  The context
           stays usable: a plan made afterwards retrieves correctly.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from parity import check_alpha, f32, retrieve_near_threshold
from synth import workload_scene


@pytest.fixture(scope="module")
def lib():
    from paper_2003_02978_gb300 import build
    build.build()
    from paper_2003_02978_gb300._native import lib as _lib
    return _lib()


def _desc():
    from paper_2003_02978_gb300._native import MfDesc
    return MfDesc(rows=512, cols=16, bands_total=72, band_lo=0, band_hi=72, col_group=1,
                  layout=0, precision=0, flags=3)


def test_alloc_fault_fails_plan_on_host(lib, monkeypatch):
    monkeypatch.setenv("MF_FAULT", "alloc")
    h = ctypes.c_void_p()
    d = _desc()
    assert lib.mf_plan(ctypes.byref(d), ctypes.byref(h)) == 3  # MF_ERR_OOM
    assert b"MF_FAULT=alloc" in lib.mf_last_error()
    assert not h.value


def test_unknown_fault_is_rejected(lib, monkeypatch):
    monkeypatch.setenv("MF_FAULT", "sometimes")
    h = ctypes.c_void_p()
    d = _desc()
    assert lib.mf_plan(ctypes.byref(d), ctypes.byref(h)) == 1  # MF_ERR_INVALID_ARG


def _retrieve(n_iter, precision=0):
    import paper_2003_02978_gb300 as mfg
    sc, prm = workload_scene("plain-512x16x72", seed=1, mask_frac=0.05)
    plan = mfg.Plan(512, 16, 72, precision=precision)
    a = plan.retrieve(sc.cube.cuda(), sc.k, prm["lam"], prm["eps"], n_iter,
                      mask=sc.mask.cuda())
    torch.cuda.synchronize()
    st = plan.status()
    plan.close()
    return sc, prm, a.cpu().numpy(), st


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 1])
def test_notspd_fault(monkeypatch, lib, precision):
    monkeypatch.setenv("MF_FAULT", "notspd")
    sc, _, a, st = _retrieve(3, precision)
    assert np.all(st == 4)
    valid = oracle.valid_pixels(sc.cube.numpy(), sc.mask.numpy())
    assert np.all(np.isnan(a[valid])) and np.all(a[~valid] == 0)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 1])
def test_timeout_fault_reports_status_and_leaves_context_usable(monkeypatch, lib, precision):
    monkeypatch.setenv("MF_FAULT", "timeout")
    sc, prm, a, st = _retrieve(2, precision)
    assert np.all(st == 6)  # MF_ERR_TIMEOUT
    valid = oracle.valid_pixels(sc.cube.numpy(), sc.mask.numpy())
    assert np.all(np.isnan(a[valid])) and np.all(a[~valid] == 0)
    # a plan made without the hook works on the same context
    monkeypatch.delenv("MF_FAULT")
    sc, prm, a, st = _retrieve(2, precision)
    assert np.all(st == 0)
    cube = sc.cube.numpy().astype(np.float64)
    mask = sc.mask.numpy()
    ref, _ = oracle.retrieve(cube, f32(sc.k), prm["lam"], prm["eps"], 2, mask=mask)
    amp = oracle.retrieve_amplification(cube, f32(sc.k), prm["lam"], prm["eps"], 2, mask=mask)
    near = retrieve_near_threshold(cube, f32(sc.k), prm["lam"], prm["eps"], 2, mask=mask)
    check_alpha(a, ref, oracle.valid_pixels(sc.cube.numpy(), mask), amp, near=near)
