"""Reduced-precision restatement of the finite-volume step (test-side only).

It answers one question: how far from the FP64 oracle does the scheme land
when its arithmetic is carried out in float32 (or with the state rounded to
bfloat16 after every step), independently of how the CUDA kernels schedule
that arithmetic?  A kernel whose error sits at this floor is as accurate as
the precision allows; a kernel far above it has a fault of its own.

It is written from the scheme as the oracle's header states it (arXiv
2306.16731, Sec. 2.2: Rusanov faces of Eq. 2, the update with the flux
difference formed first and summed over x, y, z, the per-patch maximum
eigenvalue of the new state; Sec. 5: ideal-gas Euler), vectorised with numpy
over a batch of equal patches.  It shares no code with the CUDA library and
is not part of the oracle: nothing outside ``tests/`` imports it.  In float64
it reproduces the oracle (a test checks that), so in float32 it differs from
the oracle only by rounding.
"""
from __future__ import annotations

import numpy as np


def bf16_round(a) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned
    as float32 (finite inputs)."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).reshape(a.shape)


def _wrap_halos(Q, dim):
    """Periodic halos: halo index -1 <- interior p-1, halo index p <- interior 0,
    axis by axis (so edges and corners wrap too; they are never read)."""
    E = Q.shape[1]
    for ax in range(1, dim + 1):
        lo = [slice(None)] * Q.ndim
        hi = [slice(None)] * Q.ndim
        lo[ax], hi[ax] = 0, E - 1
        src_lo = [slice(None)] * Q.ndim
        src_hi = [slice(None)] * Q.ndim
        src_lo[ax], src_hi[ax] = E - 2, 1
        Q[tuple(lo)] = Q[tuple(src_lo)]
        Q[tuple(hi)] = Q[tuple(src_hi)]


def _primitives(Q, dim, g):
    """Velocities, pressure and sound speed in the array's own precision."""
    ct = Q.dtype.type
    rho = Q[..., 0]
    u = [Q[..., 1 + a] / rho for a in range(dim)]
    kin = np.zeros_like(rho)
    for a in range(dim):
        kin = kin + Q[..., 1 + a] * u[a]
    pres = (ct(g) - ct(1.0)) * (Q[..., dim + 1] - ct(0.5) * kin)
    snd = np.sqrt(ct(g) * pres / rho)
    return u, pres, snd


def _flux(Q, dim, u, pres, n):
    """Physical flux along axis n, unknowns on the last axis."""
    F = np.empty_like(Q)
    F[..., 0] = Q[..., 1 + n]
    for a in range(dim):
        F[..., 1 + a] = Q[..., 1 + a] * u[n] + (pres if a == n else 0)
    F[..., dim + 1] = (Q[..., dim + 1] + pres) * u[n]
    return F


def step(Q, dim, dt, h, gamma=1.4, periodic=False):
    """One step of a batch of equal patches Q[T, (p+2,)*dim, N] (z, y, x, k),
    in Q's dtype.  dt and h are per-patch float64 arrays.  Returns the new
    state (halos: fixed ones copied, periodic ones left for the next wrap)
    and the per-patch maximum eigenvalue of the new interior as float64."""
    ct = Q.dtype.type
    Q = np.array(Q, copy=True)
    if periodic:
        _wrap_halos(Q, dim)
    T, E = Q.shape[0], Q.shape[1]
    p = E - 2
    u, pres, snd = _primitives(Q, dim, gamma)
    inner = slice(1, p + 1)
    acc = None
    for n in range(dim):                       # x, y, z
        ax = dim - n                           # array axis of spatial axis n
        F = _flux(Q, dim, u, pres, n)
        lam = np.abs(u[n]) + snd
        # faces between array indices i and i+1 along ax, i = 0..p; the
        # other spatial axes restricted to the interior
        sel = [slice(None)] + [inner] * dim
        sel[ax] = slice(0, p + 1)
        selR = list(sel)
        selR[ax] = slice(1, p + 2)
        QL, QR = Q[tuple(sel)], Q[tuple(selR)]
        FL, FR = F[tuple(sel)], F[tuple(selR)]
        lmax = np.maximum(lam[tuple(sel)], lam[tuple(selR)])[..., None]
        Fh = ct(0.5) * (FL + FR) - ct(0.5) * lmax * (QR - QL)
        hi = [slice(None)] * (dim + 2)
        lo = [slice(None)] * (dim + 2)
        hi[ax], lo[ax] = slice(1, p + 1), slice(0, p)
        d = Fh[tuple(hi)] - Fh[tuple(lo)]
        acc = d if acc is None else acc + d
    scale = (np.asarray(dt, dtype=np.float64).astype(ct) / np.asarray(h, dtype=np.float64).astype(ct))
    scale = scale.reshape((T,) + (1,) * (dim + 1))
    out = Q.copy()
    core = (slice(None),) + (inner,) * dim
    out[core] = Q[core] - scale * acc
    un, pn, cn = _primitives(out[core], dim, gamma)
    lam_new = np.abs(un[0]) + cn
    for n in range(1, dim):
        lam_new = np.maximum(lam_new, np.abs(un[n]) + cn)
    lam_max = lam_new.reshape(T, -1).max(axis=1).astype(np.float64)
    return out, lam_max


def max_eigenvalue(Q, dim, gamma=1.4):
    """Per-patch maximum of |u_n| + c over the interior and all directions."""
    p = Q.shape[1] - 2
    core = (slice(None),) + (slice(1, p + 1),) * dim
    u, _, c = _primitives(Q[core], dim, gamma)
    lam = np.abs(u[0]) + c
    for n in range(1, dim):
        lam = np.maximum(lam, np.abs(u[n]) + c)
    return lam.reshape(Q.shape[0], -1).max(axis=1).astype(np.float64)


def run(Q, dim, h, steps, gamma=1.4, periodic=False, cfl=0.4, storage=None):
    """``steps`` CFL-chained steps in Q's dtype; the time step is formed in
    float64 from the eigenvalue maximum (dt = cfl h / (d lambda)), as the
    reduced-precision kernels do.  ``storage`` = "bf16" rounds the state to
    bfloat16 before the first step and after every step (float32 arithmetic
    in between)."""
    h = np.asarray(h, dtype=np.float64)
    cur = np.array(Q, copy=True)
    if storage == "bf16":
        cur = bf16_round(cur)
    dt = cfl * h / (dim * max_eigenvalue(cur, dim, gamma))
    for _ in range(steps):
        cur, lam = step(cur, dim, dt, h, gamma, periodic)
        if storage == "bf16":
            cur = bf16_round(cur)
        dt = cfl * h / (dim * lam)
    return cur
