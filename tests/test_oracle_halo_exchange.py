"""Pins of the oracle's halo exchange between patches of a batch.

A periodic domain cut into a grid of equal patches, whose face halos are
filled from their neighbours before each step, must step exactly like the
whole domain held as one periodic patch: each volume sees the same
neighbour values and the same arithmetic (bitwise, for a common dt).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests._helpers import cons_from_prim, interior


def grid_neighbours(G, dim):
    """Neighbour table of a periodic G^dim grid of patches (index = x + G y (+ G^2 z))."""
    T = G ** dim
    nb = np.zeros((T, 2 * dim), dtype=np.int32)
    for i in range(T):
        c = [(i // G ** a) % G for a in range(dim)]
        for a in range(dim):
            for s, off in ((0, -1), (1, +1)):
                d = list(c)
                d[a] = (d[a] + off) % G
                nb[i, 2 * a + s] = sum(d[b] * G ** b for b in range(dim))
    return nb


def split_domain(big, G, p, dim):
    """Interior of a (G p)^dim domain -> flat batch of G^dim patches with NaN halos."""
    N = dim + 2
    parts = []
    for i in range(G ** dim):
        c = [(i // G ** a) % G for a in range(dim)]
        patch = np.full((p + 2,) * dim + (N,), np.nan)
        sl = tuple(slice(c[dim - 1 - ax] * p, (c[dim - 1 - ax] + 1) * p) for ax in range(dim))
        interior(patch, dim)[...] = big[sl]
        parts.append(patch.reshape(-1))
    return np.concatenate(parts)


def join_domain(flat, G, p, dim):
    N = dim + 2
    big = np.zeros((G * p,) * dim + (N,))
    per = (p + 2) ** dim * N
    for i in range(G ** dim):
        c = [(i // G ** a) % G for a in range(dim)]
        patch = flat[i * per:(i + 1) * per].reshape((p + 2,) * dim + (N,))
        sl = tuple(slice(c[dim - 1 - ax] * p, (c[dim - 1 - ax] + 1) * p) for ax in range(dim))
        big[sl] = interior(patch, dim)
    return big


@pytest.mark.parametrize("dim,G,p", [(2, 3, 4), (2, 2, 5), (3, 2, 3)])
def test_patch_grid_with_exchange_steps_like_one_periodic_patch(dim, G, p):
    rng = np.random.default_rng(100 + dim)
    n = G * p
    shape = (n,) * dim
    big = cons_from_prim(rng.uniform(0.5, 1.5, shape), rng.uniform(-0.5, 0.5, shape + (dim,)),
                         rng.uniform(0.5, 1.5, shape))
    nb = grid_neighbours(G, dim)
    T = G ** dim
    sizes = [p] * T
    h, dt = 0.1, 0.01
    flat = split_domain(big, G, p, dim)
    whole = np.zeros((n + 2,) * dim + (dim + 2,))
    interior(whole, dim)[...] = big
    for _ in range(4):
        flat = oracle.halo_exchange(dim, sizes, nb, flat)
        flat, _ = oracle.batch_step(dim, sizes, [h] * T, [dt] * T, flat, halo_mode=oracle.FIXED)
        whole_flat, _ = oracle.batch_step(dim, [n], [h], [dt], whole.reshape(-1), halo_mode=oracle.PERIODIC)
        whole = whole_flat.reshape(whole.shape)
    assert np.array_equal(join_domain(flat, G, p, dim), interior(whole, dim))


def test_exchange_writes_only_face_halos_with_neighbours():
    rng = np.random.default_rng(7)
    p, dim = 3, 2
    flat = rng.uniform(1.0, 2.0, 2 * (p + 2) ** 2 * 4)
    nb = np.array([[-1, 1, -1, -1], [0, -1, -1, -1]], dtype=np.int32)   # patch 0 | patch 1 along x
    out = oracle.halo_exchange(dim, [p, p], nb, flat)
    a = flat.reshape(2, p + 2, p + 2, 4)
    b = out.reshape(2, p + 2, p + 2, 4)
    assert np.array_equal(b[0, 1:-1, p + 1], a[1, 1:-1, 1])       # +x halo of 0 = column 0 of 1
    assert np.array_equal(b[1, 1:-1, 0], a[0, 1:-1, p])            # -x halo of 1 = column p-1 of 0
    changed = np.any(b != a, axis=-1)
    expect = np.zeros(changed.shape, bool)
    expect[0, 1:-1, p + 1] = True
    expect[1, 1:-1, 0] = True
    assert np.array_equal(changed, expect & np.any(b != a, axis=-1)) and not np.any(changed & ~expect)


def test_exchange_rejects_nonconforming_neighbours():
    with pytest.raises(RuntimeError):
        oracle.halo_exchange(2, [3, 4], np.array([[-1, 1, -1, -1], [0, -1, -1, -1]]), np.zeros(25 * 4 + 36 * 4))
