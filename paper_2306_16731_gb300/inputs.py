"""Seeded synthetic workloads for the batched finite-volume patch update.

This module is shared by the tests, the benchmark and the smoke check: both
the CUDA path and the FP64 oracle take their inputs from here.  It holds no
arithmetic of the method itself (no flux, eigenvalue, update or time step),
only the input recipe: draw primitive variables with numpy's PCG64 and
convert them to the conserved variables of the Euler equations
(rho, rho u_1..rho u_d, E) with E = p/(gamma-1) + 1/2 rho |u|^2.

Draw order: per patch, per volume in storage order (halo volumes included),
per primitive (rho, u_1..u_d, p).  The state layout is the array of
structures ``Q[patch][z][y][x][k]`` with a one-volume halo (Sec. 4 of the
paper); patch ``i`` starts at element ``sum_{j<i} (d+2) (p_j+2)^d``.

The five workloads below stand in for the paper's miniapp inputs, which the
paper does not give: Euler, d in {2, 3}, small patches, FP64 array of
structures, at the sizes of the benchmark plan.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

FIXED = 0
PERIODIC = 1
GAMMA = 1.4
CFL = 0.4


@dataclass
class Workload:
    name: str
    dim: int
    patch_size: np.ndarray          # int32 [T]
    dx: np.ndarray                  # float64 [T]
    halo_mode: int
    steps: int
    Q0: np.ndarray                  # flat AoS state with halo, float64 or float32
    gamma: float = GAMMA
    cfl: float = CFL
    seed: int = 0
    notes: dict = field(default_factory=dict)

    @property
    def num_patches(self) -> int:
        return int(len(self.patch_size))

    @property
    def unknowns(self) -> int:
        return self.dim + 2

    @property
    def interior_volumes(self) -> int:
        return int(np.sum(self.patch_size.astype(np.int64) ** self.dim))

    def offsets(self) -> np.ndarray:
        return patch_offsets(self.dim, self.patch_size)


def patch_offsets(dim: int, patch_size) -> np.ndarray:
    p = np.asarray(patch_size, dtype=np.int64).reshape(-1)
    return np.concatenate([[0], np.cumsum((dim + 2) * (p + 2) ** dim)]).astype(np.int64)


def _to_conserved(prim: np.ndarray, dim: int, gamma: float, out: np.ndarray) -> None:
    """prim[..., (rho, u_1..u_d, p)] -> out[..., (rho, rho u_1..rho u_d, E)]."""
    rho = prim[:, 0]
    vel = prim[:, 1:1 + dim]
    pres = prim[:, dim + 1]
    out[:, 0] = rho
    out[:, 1:1 + dim] = rho[:, None] * vel
    out[:, dim + 1] = pres / (gamma - 1.0) + 0.5 * rho * np.sum(vel * vel, axis=1)


def _uniform_states(rng, ncells: int, dim: int, gamma: float, out: np.ndarray,
                    chunk: int = 1 << 22) -> None:
    """rho, p ~ U[0.5, 1.5), u_k ~ U[-0.5, 0.5): out[ncells, d+2] conserved."""
    lo = np.array([0.5] + [-0.5] * dim + [0.5])
    for s in range(0, ncells, chunk):
        e = min(ncells, s + chunk)
        prim = rng.random((e - s, dim + 2)) + lo
        tmp = np.empty((e - s, dim + 2), dtype=np.float64)
        _to_conserved(prim, dim, gamma, tmp)
        out[s:e] = tmp


def _gaussian_pulse_states(rng, T: int, p: int, dx: float, gamma: float,
                           out: np.ndarray) -> None:
    """3D pulse: rho = 1 + 0.2 exp(-|x - x_c|^2 / w^2), w = 0.2 p dx, x_c the
    patch centre, cell centres (i + 1/2) dx; u = 0, p = 1; then iid
    U[-1e-3, 1e-3) noise on rho, each u_k and p."""
    dim = 3
    e = p + 2
    idx = np.arange(-1, p + 1, dtype=np.float64)
    xc = (idx + 0.5) * dx
    L = p * dx
    w = 0.2 * L
    z, y, x = np.meshgrid(xc, xc, xc, indexing="ij")
    r2 = (x - 0.5 * L) ** 2 + (y - 0.5 * L) ** 2 + (z - 0.5 * L) ** 2
    base = np.zeros((e ** 3, dim + 2))
    base[:, 0] = 1.0 + 0.2 * np.exp(-r2.reshape(-1) / (w * w))
    base[:, dim + 1] = 1.0
    ncell = e ** 3
    for i in range(T):
        prim = base + (2.0 * rng.random((ncell, dim + 2)) - 1.0) * 1e-3
        tmp = np.empty_like(prim)
        _to_conserved(prim, dim, gamma, tmp)
        out[i * ncell:(i + 1) * ncell] = tmp


def config(index: int, dtype=np.float64, num_patches: int | None = None) -> Workload:
    """Workload ``index`` in 1..5 (see module docstring and the design notes).

    ``num_patches`` keeps only the first patches (same values as the full
    workload, since draws run patch by patch); ``dtype`` is the storage
    type of ``Q0`` (the float64 draws are rounded once)."""
    seed = index
    rng = np.random.Generator(np.random.PCG64(seed))
    if index == 1:
        dim, T, p, dxv, halo, steps = 2, 64, 3, 0.1, FIXED, 10
        name = "2d_p3_T64_fp64"
    elif index == 2:
        dim, T, p, dxv, halo, steps = 2, 16384, 16, 0.01, FIXED, 100
        name = "2d_p16_T16384"
    elif index == 3:
        dim, T, p, dxv, halo, steps = 3, 4096, 8, 1.0 / 8.0, PERIODIC, 50
        name = "3d_p8_T4096_periodic_pulse"
    elif index == 4:
        dim, T, halo, steps = 2, 50000, FIXED, 200
        name = "2d_uneven_T50000"
        j = rng.integers(2, 6, size=T)           # p = 2^j, j uniform on {2,3,4,5}
        k = rng.integers(1, 5, size=T)           # dx = 3^-k, k uniform on {1..4}
        psz = (2 ** j).astype(np.int32)
        dxa = 3.0 ** (-k.astype(np.float64))
    elif index == 5:
        dim, T, p, dxv, halo, steps = 3, 32768, 16, 0.01, FIXED, 20
        name = "3d_p16_T32768"
    else:
        raise ValueError("workload index must be 1..5")

    if index != 4:
        psz = np.full(T, p, dtype=np.int32)
        dxa = np.full(T, dxv, dtype=np.float64)
    if num_patches is not None:
        T = int(num_patches)
        psz = psz[:T].copy()
        dxa = dxa[:T].copy()

    N = dim + 2
    off = patch_offsets(dim, psz)
    ncells = int(off[-1]) // N
    Q = np.empty((ncells, N), dtype=dtype)
    if index == 3:
        _gaussian_pulse_states(rng, T, int(psz[0]), float(dxa[0]), GAMMA, Q)
    else:
        _uniform_states(rng, ncells, dim, GAMMA, Q)
    return Workload(name=name, dim=dim, patch_size=psz, dx=dxa, halo_mode=halo,
                    steps=steps, Q0=Q.reshape(-1), seed=seed)


def uniform_batch(dim: int, patch_size, seed: int, dx=0.1, dtype=np.float64,
                  halo_mode: int = FIXED, steps: int = 1) -> Workload:
    """Ad-hoc batch with the uniform value distributions of workload 1 for
    arbitrary (possibly ragged) patch sizes."""
    psz = np.asarray(patch_size, dtype=np.int32).reshape(-1)
    T = len(psz)
    rng = np.random.Generator(np.random.PCG64(seed))
    off = patch_offsets(dim, psz)
    ncells = int(off[-1]) // (dim + 2)
    Q = np.empty((ncells, dim + 2), dtype=dtype)
    _uniform_states(rng, ncells, dim, GAMMA, Q)
    dxa = np.broadcast_to(np.asarray(dx, dtype=np.float64), (T,)).copy()
    return Workload(name="uniform_%dd" % dim, dim=dim, patch_size=psz, dx=dxa,
                    halo_mode=halo_mode, steps=steps, Q0=Q.reshape(-1), seed=seed)


def shallow_water_batch(patch_size, seed: int, dx=0.1, dtype=np.float64, halo_mode: int = FIXED,
                        bottom: float = 0.2, depth_noise: float = 0.05, speed: float = 0.3) -> Workload:
    """2D shallow water batch, Q = (h, hu, hv, b) per volume (halo volumes
    included): a perturbed lake over a random bottom, b ~ U[-bottom, bottom],
    h = 1 - b + U[-depth_noise, depth_noise], u, v ~ U[-speed, speed]."""
    psz = np.asarray(patch_size, dtype=np.int32).reshape(-1)
    T = len(psz)
    rng = np.random.Generator(np.random.PCG64(seed))
    ncells = int(np.sum((psz.astype(np.int64) + 2) ** 2))
    b = rng.uniform(-bottom, bottom, ncells)
    h = 1.0 - b + rng.uniform(-depth_noise, depth_noise, ncells)
    u = rng.uniform(-speed, speed, ncells)
    v = rng.uniform(-speed, speed, ncells)
    Q = np.stack([h, h * u, h * v, b], axis=1).astype(dtype)
    dxa = np.broadcast_to(np.asarray(dx, dtype=np.float64), (T,)).copy()
    return Workload(name="shallow_water_2d", dim=2, patch_size=psz, dx=dxa, halo_mode=halo_mode,
                    steps=1, Q0=Q.reshape(-1), seed=seed)


def patch_view(w: Workload, Q: np.ndarray, i: int) -> np.ndarray:
    """Patch ``i`` of a flat state as an array [(p+2)]*d + [d+2] (z, y, x, k)."""
    off = w.offsets()
    p = int(w.patch_size[i])
    shape = [p + 2] * w.dim + [w.dim + 2]
    return Q[off[i]:off[i + 1]].reshape(shape)


def interior(dim: int, patch: np.ndarray) -> np.ndarray:
    """Interior volumes of one patch view."""
    return patch[(slice(1, -1),) * dim]
