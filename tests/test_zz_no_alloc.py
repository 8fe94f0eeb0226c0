"""The allocation-free update entry point, checked against the ordinary one.

fv_patch_batch_update_noalloc serves callers that cannot call cudaMalloc
where they step their patches (for example host code running while a CUDA
graph is captured, or a plugin whose device memory belongs to a pooling
allocator).  It keeps its intermediates in a built-in 64 MiB device array
instead of memory it allocates.  This test calls it through the C ABI twice
in a row (the second call consumes the first call's output, so the array's
left-over contents from the first call must not leak into the second) and
compares both results with fv_patch_batch_update on a batch created with
fv_batch_create, within the FP64 tolerance of the other parity tests.  It
passes alone in a fresh process and after the rest of the suite.
"""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_16731_gb300 import build, fvbatch
    build.build()
    return fvbatch


def _rel_linf(a, b, N):
    a = a.reshape(-1, N)
    b = b.reshape(-1, N)
    return max(float(np.max(np.abs(a[:, k] - b[:, k])) / np.max(np.abs(b[:, k]))) for k in range(N))


@pytest.mark.parametrize("dim,p,T,precision", [(2, 16, 200, 0), (3, 6, 40, 0), (2, 8, 300, 1)])
def test_no_alloc_update_matches_batch_update_twice(lib, dim, p, T, precision):
    import torch
    from paper_2306_16731_gb300 import inputs
    fb = lib
    w = inputs.uniform_batch(dim, [p] * T, seed=31 + dim, dx=np.linspace(0.01, 0.05, T))
    dtype = torch.float64 if precision == fb.FV_F64 else torch.float32
    N = dim + 2
    q0 = torch.from_numpy(w.Q0).to("cuda", dtype)
    dx = torch.tensor(w.dx, device="cuda")
    dt = torch.full((T,), 1e-3, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream

    # reference: two steps through a batch created the usual way
    b = fb.FVBatch(dim, [p] * T, precision=precision, stream=stream)
    r1, r2 = q0.clone(), q0.clone()
    lam_r = torch.zeros(T, dtype=torch.float64, device="cuda")
    dtn_r = torch.zeros_like(lam_r)
    b.update(q0, r1, dx, dt, lam_r, dtn_r, 0.4)
    b.update(r1, r2, dx, dtn_r, lam_r, None, 0.4)
    torch.cuda.synchronize()
    b.close()

    # the allocation-free entry point, two calls in a row
    o1, o2 = q0.clone(), q0.clone()
    lam_n = torch.zeros_like(lam_r)
    dtn_n = torch.zeros_like(lam_r)
    fb.fv_patch_batch_update_noalloc(dim, T, p, precision, fb.FV_HALO_FIXED, 1.4, q0, o1,
                                     dx, dt, lam_n, dtn_n, 0.4, stream)
    fb.fv_patch_batch_update_noalloc(dim, T, p, precision, fb.FV_HALO_FIXED, 1.4, o1, o2,
                                     dx, dtn_n, lam_n, None, 0.4, stream)
    torch.cuda.synchronize()

    tol = TOL if precision == fb.FV_F64 else 1e-6
    for got, ref in ((o1, r1), (o2, r2)):
        g = got.double().cpu().numpy()
        r = ref.double().cpu().numpy()
        assert _rel_linf(g, r, N) <= tol
    assert np.max(np.abs(lam_n.cpu().numpy() - lam_r.cpu().numpy()) / lam_r.cpu().numpy()) <= tol
    assert np.max(np.abs(dtn_n.cpu().numpy() - dtn_r.cpu().numpy()) / dtn_r.cpu().numpy()) <= tol


def test_no_alloc_rejects_batches_beyond_its_array(lib):
    import torch
    fb = lib
    q = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(fb.FVError) as ei:
        fb.fv_patch_batch_update_noalloc(2, 100000, 16, fb.FV_F64, fb.FV_HALO_FIXED, 1.4,
                                         q, q.clone(), q, q)
    assert ei.value.code == fb.FV_EINVAL
    assert "64 MiB" in str(ei.value)
