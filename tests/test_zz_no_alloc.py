"""The allocation-free update entry point, checked against the ordinary one
and against the FP64 oracle.

fv_patch_batch_update_noalloc serves callers that cannot call cudaMalloc
where they step their patches (for example host code running while a CUDA
graph is captured, or a plugin whose device memory belongs to a pooling
allocator).  It keeps its intermediates in a built-in 64 MiB device array
instead of memory it allocates.  This test calls it through the C ABI twice
in a row (the second call consumes the first call's output, so the array's
left-over contents from the first call must not leak into the second) and
compares both results with fv_patch_batch_update on a batch created with
fv_batch_create, within the tolerance of the other parity tests for the
precision, and with the oracle's two steps.  Fixed and periodic halos, FP64,
FP32 and BF16 storage are covered; a warmed-up call must leave the device's
free memory unchanged.  It passes alone in a fresh process and after the
rest of the suite.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

# rel L-inf tolerance against the ordinary update (the same cascade kernels,
# so in practice identical) and against the oracle, per precision
TOL = {0: 1e-12, 1: 1e-5, 2: 5e-2}


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_16731_gb300 import build, fvbatch
    build.build()
    oracle.build()
    return fvbatch


def _rel_linf(a, b, dim, p, T):
    N = dim + 2
    sh = (T,) + (p + 2,) * dim + (N,)
    core = (slice(None),) + (slice(1, -1),) * dim
    a = np.asarray(a, dtype=np.float64).reshape(sh)[core].reshape(-1, N)
    b = np.asarray(b, dtype=np.float64).reshape(sh)[core].reshape(-1, N)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("dim,p,T,precision,halo", [(2, 16, 200, 0, 0), (3, 6, 40, 0, 0), (2, 8, 300, 1, 0),
                                                    (2, 16, 120, 0, 1), (3, 8, 30, 1, 1), (2, 8, 100, 2, 0),
                                                    (3, 4, 50, 2, 1)])
def test_no_alloc_update_matches_batch_update_twice(lib, dim, p, T, precision, halo):
    import torch
    from paper_2306_16731_gb300 import inputs
    fb = lib
    w = inputs.uniform_batch(dim, [p] * T, seed=31 + dim, dx=np.linspace(0.01, 0.05, T), halo_mode=halo)
    dtype = {0: torch.float64, 1: torch.float32, 2: torch.bfloat16}[precision]
    q0 = torch.from_numpy(w.Q0).to("cuda").to(dtype)
    dx = torch.tensor(w.dx, device="cuda")
    dt = torch.full((T,), 1e-3, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream

    # a zero-patch call primes the entry point on this device (no buffers)
    fb.fv_patch_batch_update_noalloc(dim, 0, p, precision, halo, 1.4, None, None, None, None, None, None,
                                     0.4, stream)

    # reference: two steps through a batch created the usual way
    b = fb.FVBatch(dim, [p] * T, precision=precision, halo_mode=halo, form=fb.FV_FORM_CASCADE, stream=stream)
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
    lam_1 = torch.zeros_like(lam_r)
    fb.fv_patch_batch_update_noalloc(dim, T, p, precision, halo, 1.4, q0, o1,
                                     dx, dt, lam_1, dtn_n, 0.4, stream)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    fb.fv_patch_batch_update_noalloc(dim, T, p, precision, halo, 1.4, o1, o2,
                                     dx, dtn_n, lam_n, None, 0.4, stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before        # nothing allocated

    tol = TOL[precision]
    for got, ref in ((o1, r1), (o2, r2)):
        assert _rel_linf(got.double().cpu().numpy(), ref.double().cpu().numpy(), dim, p, T) <= tol
    assert np.max(np.abs(lam_n.cpu().numpy() - lam_r.cpu().numpy()) / lam_r.cpu().numpy()) <= tol
    assert np.max(np.abs(dtn_n.cpu().numpy() - dtn_r.cpu().numpy()) / dtn_r.cpu().numpy()) <= tol

    # the oracle's two steps from the same (rounded) start, with the first
    # step's CFL time steps feeding the second
    start = q0.double().cpu().numpy()
    s1, l1 = oracle.batch_step(dim, w.patch_size, w.dx, [1e-3] * T, start, halo_mode=halo)
    d1 = oracle.cfl_time_step(dim, l1, w.dx, 0.4)
    s2, l2 = oracle.batch_step(dim, w.patch_size, w.dx, d1, s1, halo_mode=halo)
    assert _rel_linf(o1.double().cpu().numpy(), s1, dim, p, T) <= tol
    assert _rel_linf(o2.double().cpu().numpy(), s2, dim, p, T) <= 2 * tol
    assert np.max(np.abs(lam_1.cpu().numpy() - l1) / l1) <= tol
    assert np.max(np.abs(lam_n.cpu().numpy() - l2) / l2) <= 2 * tol


def test_no_alloc_rejects_batches_beyond_its_array(lib):
    import torch
    fb = lib
    q = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(fb.FVError) as ei:
        fb.fv_patch_batch_update_noalloc(2, 100000, 16, fb.FV_F64, fb.FV_HALO_FIXED, 1.4,
                                         q, q.clone(), q, q)
    assert ei.value.code == fb.FV_EINVAL
    assert "64 MiB" in str(ei.value)
