"""The seeded synthetic workloads follow the stated recipe: value ranges of
the uniform primitives, the density pulse of the periodic 8^3 workload, the
edge-length and mesh-width distributions of the uneven batch, and prefix
stability (the first k patches of a workload do not depend on its size)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2306_16731_gb300 import inputs


def _primitives(w):
    N = w.dim + 2
    q = w.Q0.reshape(-1, N).astype(np.float64)
    rho = q[:, 0]
    u = q[:, 1:1 + w.dim] / rho[:, None]
    p = (inputs.GAMMA - 1.0) * (q[:, -1] - 0.5 * np.sum(q[:, 1:1 + w.dim] * u, axis=1))
    return rho, u, p


@pytest.mark.parametrize("index,npatch", [(1, 64), (2, 40), (5, 3)])
def test_uniform_primitives_lie_in_their_ranges(index, npatch):
    w = inputs.config(index, num_patches=npatch)
    rho, u, p = _primitives(w)
    eps = 1e-12
    assert rho.min() >= 0.5 - eps and rho.max() <= 1.5 + eps
    assert p.min() >= 0.5 - eps and p.max() <= 1.5 + eps
    assert np.abs(u).max() <= 0.5 + eps
    # spread over the ranges (not a constant field)
    assert rho.max() - rho.min() > 0.9 and np.abs(u).max() > 0.45


def test_periodic_pulse_has_the_stated_amplitude_and_noise():
    w = inputs.config(3, num_patches=6)
    assert w.halo_mode == inputs.PERIODIC and w.dim == 3 and set(w.patch_size) == {8}
    rho, u, p = _primitives(w)
    assert np.abs(u).max() <= 1e-3 + 1e-12
    assert np.abs(p - 1.0).max() <= 1e-3 + 1e-12
    assert rho.min() >= 1.0 - 1e-3 - 1e-12 and rho.max() <= 1.2 + 1e-3 + 1e-12
    # the peak sits at the patch centre, a corner of the eight central
    # volumes (even edge): their centres are half a volume off it per axis,
    # so rho there is 1 + 0.2 exp(-3 (h/2)^2 / (0.2 p h)^2) up to the noise
    r = rho.reshape(6, 10, 10, 10)[:, 1:-1, 1:-1, 1:-1]
    peak = 1.0 + 0.2 * np.exp(-3 * 0.25 / (0.2 * 8) ** 2)
    assert np.abs(r[:, 3:5, 3:5, 3:5] - peak).max() <= 1e-3 + 1e-12
    corner = r[:, [0, -1]][:, :, [0, -1]][:, :, :, [0, -1]]
    assert corner.max() < 1.01


def test_uneven_batch_draws_edges_and_mesh_widths_uniformly():
    w = inputs.config(4, num_patches=20000)
    sizes, counts = np.unique(w.patch_size, return_counts=True)
    assert list(sizes) == [4, 8, 16, 32]
    assert np.all(np.abs(counts / counts.sum() - 0.25) < 0.02)
    ks = np.round(-np.log(w.dx) / np.log(3.0)).astype(int)
    assert np.allclose(w.dx, 3.0 ** -ks, rtol=0, atol=0)
    kv, kc = np.unique(ks, return_counts=True)
    assert list(kv) == [1, 2, 3, 4]
    assert np.all(np.abs(kc / kc.sum() - 0.25) < 0.02)


@pytest.mark.parametrize("index", [1, 3, 4])
def test_first_patches_do_not_depend_on_the_batch_size(index):
    a = inputs.config(index, num_patches=7)
    b = inputs.config(index, num_patches=12)
    n = len(a.Q0)
    assert np.array_equal(a.patch_size, b.patch_size[:7]) and np.array_equal(a.dx, b.dx[:7])
    assert np.array_equal(a.Q0, b.Q0[:n])


def test_single_precision_storage_is_the_rounded_double_draw():
    a = inputs.config(2, num_patches=5)
    b = inputs.config(2, num_patches=5, dtype=np.float32)
    assert b.Q0.dtype == np.float32
    assert np.array_equal(b.Q0, a.Q0.astype(np.float32))
