"""Test-side helpers: build patches from primitive variables, compare states.

These only prepare inputs and compare outputs; they hold no step of the
finite-volume update.
"""
from __future__ import annotations

import numpy as np

GAMMA = 1.4


def cons_from_prim(rho, vel, p, gamma=GAMMA):
    """Conserved (rho, rho u_1..rho u_d, E) from primitives, last axis = unknowns."""
    rho = np.asarray(rho, dtype=np.float64)
    vel = np.asarray(vel, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    d = vel.shape[-1]
    out = np.empty(rho.shape + (d + 2,))
    out[..., 0] = rho
    out[..., 1:1 + d] = rho[..., None] * vel
    out[..., d + 1] = p / (gamma - 1.0) + 0.5 * rho * np.sum(vel * vel, axis=-1)
    return out


def prim_from_cons(Q, dim, gamma=GAMMA):
    rho = Q[..., 0]
    vel = Q[..., 1:1 + dim] / rho[..., None]
    p = (gamma - 1.0) * (Q[..., dim + 1] - 0.5 * np.sum(Q[..., 1:1 + dim] * vel, axis=-1))
    return rho, vel, p


def random_patch(rng, dim, p, gamma=GAMMA):
    """One halo-inclusive patch [(p+2)]*dim + [dim+2] with the uniform
    distributions of the benchmark workloads."""
    shape = (p + 2,) * dim
    rho = rng.uniform(0.5, 1.5, shape)
    vel = rng.uniform(-0.5, 0.5, shape + (dim,))
    pr = rng.uniform(0.5, 1.5, shape)
    return cons_from_prim(rho, vel, pr, gamma)


def interior(Q, dim):
    return Q[(slice(1, -1),) * dim]


def rel_linf(a, b, dim):
    """max over unknowns k of max|a_k - b_k| / max|b_k| (interior volumes)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    errs = []
    for k in range(dim + 2):
        den = np.max(np.abs(b[..., k]))
        errs.append(np.max(np.abs(a[..., k] - b[..., k])) / (den if den > 0 else 1.0))
    return max(errs)


def patches_interior(flat, dim, patch_size):
    """List of interior arrays of every patch of a flat state."""
    p = np.asarray(patch_size, dtype=np.int64)
    off = np.concatenate([[0], np.cumsum((dim + 2) * (p + 2) ** dim)])
    out = []
    for i in range(len(p)):
        shape = (int(p[i]) + 2,) * dim + (dim + 2,)
        out.append(interior(np.asarray(flat[off[i]:off[i + 1]]).reshape(shape), dim))
    return out


def state_rel_linf(a, b):
    """Relative L-infinity error of a state: the largest |a - b| over volumes
    and unknowns divided by the largest |b| over volumes and unknowns."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0))


def _interiors(a, b, dim, patch_size):
    N = dim + 2
    A = np.concatenate([x.reshape(-1, N) for x in patches_interior(a, dim, patch_size)])
    B = np.concatenate([x.reshape(-1, N) for x in patches_interior(b, dim, patch_size)])
    return A, B


def batch_rel_linf(a, b, dim, patch_size):
    """Relative L-infinity error over the interiors of a whole batch
    (normalised by the oracle state's largest magnitude, all unknowns)."""
    A, B = _interiors(a, b, dim, patch_size)
    return state_rel_linf(A, B)


def batch_rel_linf_components(a, b, dim, patch_size):
    """Per-unknown relative L-infinity errors (each unknown normalised by its
    own largest magnitude), for reporting."""
    A, B = _interiors(a, b, dim, patch_size)
    return [float(np.max(np.abs(A[:, k] - B[:, k])) / max(np.max(np.abs(B[:, k])), 1e-300))
            for k in range(dim + 2)]
