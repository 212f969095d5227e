"""mf_background_noalloc: the allocation-free entry point for callers that may
not allocate device memory once running (real-time processing that forbids
allocation after start-up, hosts whose device memory belongs to another
allocator).  Its output must equal what the plan-based path returns for the
same cube (mf_retrieve, then mf_background) and match the FP64 oracle's mean
and covariance of the valid pixels, on two calls in a row: the second call
reuses the library's fixed scratch array, which still holds the first call's
moments.

Collected last (file name) so that a run stopping at the first failure has
already run every other test; it must also pass alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from synth import make_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2003_02978_gb300 import build
    build.build()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("col_group", [1, 3])
def test_noalloc_background_matches_plan_path_and_oracle_twice(col_group):
    import paper_2003_02978_gb300 as mfg
    from paper_2003_02978_gb300._native import MfDesc, lib

    rows, cols, bands = 700, 20, 72
    sc = make_scene(rows, cols, bands, n_plumes=2, plume_sigma=(3.0, 6.0),
                    plume_peak=(800.0, 3000.0), mask_frac=0.05, nan_masked=True, seed=77)
    cube = sc.cube.cuda().contiguous()
    mask = sc.mask.cuda().contiguous()
    k = np.asarray(sc.k, np.float32)
    P = len(oracle.partitions(cols, col_group))

    # existing path: a plan (allocates its workspace), one retrieval, read-back
    plan = mfg.Plan(rows, cols, bands, col_group=col_group)
    plan.retrieve(cube, k, 1e-3, 1e-9, 0, mask=mask)
    mu_ref, cov_ref = plan.background()
    torch.cuda.synchronize()
    mu_ref, cov_ref = mu_ref.cpu().numpy(), cov_ref.cpu().numpy()
    plan.close()

    # FP64 oracle: mean and covariance of each partition's valid pixels
    cube_np = sc.cube.numpy()
    valid = oracle.valid_pixels(cube_np, sc.mask.numpy())
    mu_o, cov_o = [], []
    for c0, c1 in oracle.partitions(cols, col_group):
        X = cube_np[:, c0:c1][valid[:, c0:c1]].astype(np.float64)
        m = oracle.mean_vector(X)
        mu_o.append(m)
        cov_o.append(oracle.covariance_about(X - m))

    # the allocation-free entry point, twice in a row on the same stream
    L = lib()
    d = MfDesc(rows=rows, cols=cols, bands_total=bands, band_lo=0, band_hi=bands,
               col_group=col_group, layout=0, precision=0, flags=3)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        mu = torch.full((P, bands), float("nan"), dtype=torch.float64, device="cuda")
        cov = torch.full((P, bands, bands), float("nan"), dtype=torch.float64, device="cuda")
        st = L.mf_background_noalloc(ctypes.byref(d), _ptr(cube), _ptr(mask), _ptr(mu), _ptr(cov),
                                     stream)
        assert st == 0, L.mf_last_error()
        torch.cuda.synchronize()
        mu_n, cov_n = mu.cpu().numpy(), cov.cpu().numpy()
        # against the plan path and the oracle, with the tolerances of the
        # background-statistics parity test
        np.testing.assert_allclose(mu_n, mu_ref, rtol=1e-7)
        for j in range(P):
            rel = np.linalg.norm(cov_n[j] - cov_ref[j]) / np.linalg.norm(cov_ref[j])
            assert rel < 1e-6, (call, j, rel)
            np.testing.assert_allclose(mu_n[j], mu_o[j], rtol=1e-7)
            rel_o = np.linalg.norm(cov_n[j] - cov_o[j]) / np.linalg.norm(cov_o[j])
            assert rel_o < 1e-6, (call, j, rel_o)


def test_noalloc_rejects_oversized_problem():
    from paper_2003_02978_gb300._native import MfDesc, lib
    L = lib()
    # 3000 detector columns of 128 bands: ~70 KB of moments per column, over 64 MiB
    d = MfDesc(rows=256, cols=3000, bands_total=128, band_lo=0, band_hi=128, col_group=1,
               layout=0, precision=0, flags=3)
    dummy = torch.empty(16, dtype=torch.float32, device="cuda")
    out = torch.empty(16, dtype=torch.float64, device="cuda")
    st = L.mf_background_noalloc(ctypes.byref(d), _ptr(dummy), None, _ptr(out), _ptr(out), None)
    assert st == 8  # MF_ERR_UNSUPPORTED, nothing enqueued
    assert b"scratch" in L.mf_last_error()
