"""The reduced-precision kernels sit at their precision's floor.

``tests/test_precision_floor.py`` shows, without a GPU, where float32
arithmetic (and bfloat16 storage) puts the error of the scheme against the
FP64 oracle.  Here the CUDA kernels run the same patches for the same
steps, and their error in each norm -- per unknown and state-normalised --
must stay within a small factor of that floor: rounding in another order
gives errors of the same size, a fault in a kernel gives errors far larger.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2306_16731_gb300 import inputs
from tests import fp_emulation as fe
from tests.gpu_util import gpu_run, initial_fp64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_16731_gb300 import build
    build.build()
    oracle.build()


def _norms(got_flat, ref_flat, w):
    p = int(w.patch_size[0])
    N = w.dim + 2
    shape = (w.num_patches,) + (p + 2,) * w.dim + (N,)
    core = (slice(None),) + (slice(1, -1),) * w.dim
    g = np.asarray(got_flat, dtype=np.float64).reshape(shape)[core].reshape(-1, N)
    r = np.asarray(ref_flat, dtype=np.float64).reshape(shape)[core].reshape(-1, N)
    state = float(np.max(np.abs(g - r)) / np.max(np.abs(r)))
    per = np.array([np.max(np.abs(g[:, k] - r[:, k])) / np.max(np.abs(r[:, k])) for k in range(N)])
    return state, per


@pytest.mark.parametrize("cfg,T,precision", [(3, 64, 1), (3, 64, 2), (2, 16, 1), (5, 2, 1)])
def test_kernel_error_is_at_the_precision_floor(cfg, T, precision):
    w = inputs.config(cfg, num_patches=T)
    start = initial_fp64(w.Q0, precision)
    ref, _, _ = oracle.batch_run(w.dim, w.patch_size, w.dx, start, w.steps, w.gamma, w.halo_mode, w.cfl)
    got, _, _, desc = gpu_run(w, precision, 0, w.steps, use_graph=True)
    p = int(w.patch_size[0])
    Q32 = start.astype(np.float32).reshape((T,) + (p + 2,) * w.dim + (w.dim + 2,))
    emu = fe.run(Q32, w.dim, w.dx, w.steps, w.gamma, w.halo_mode == inputs.PERIODIC, w.cfl,
                 storage="bf16" if precision == 2 else None)
    gs, gp = _norms(got, ref, w)
    es, ep = _norms(emu.reshape(-1), ref, w)
    print("%s precision %d (%s): kernel state %.2e per unknown %s | emulated floor state %.2e per unknown %s"
          % (w.name, precision, desc.split()[0], gs, " ".join("%.1e" % e for e in gp), es,
             " ".join("%.1e" % e for e in ep)))
    # within 4x of the floor in every unknown (plus FP32 rounding of the
    # smallest representable relative error, for unknowns the floor puts
    # near zero)
    assert np.all(gp <= 4.0 * ep + 1e-6), (gp, ep)
    assert gs <= 4.0 * es + 1e-7, (gs, es)
    if precision == 1:
        assert gs <= 1e-5
