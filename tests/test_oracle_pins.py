"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks a property
that the finite-volume step of Sec. 2.2 (Rusanov flux, Eq. 2) must have on
the Euler equations, a closed form from linear stability theory, a value
worked out by hand, or an independent brute-force evaluation.  A dropped
term, a wrong sign, a swapped index or a transposed operand anywhere in the
oracle fails at least one of them.
"""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

import oracle
from tests._helpers import (GAMMA, cons_from_prim, prim_from_cons, random_patch,
                            interior, rel_linf)

EPS = np.finfo(np.float64).eps


def step1(Q, dim, dt, h=1.0, halo_mode=oracle.FIXED):
    """One oracle step on a single patch array [(p+2)]*d + [d+2]."""
    p = Q.shape[0] - 2
    out, lam = oracle.batch_step(dim, [p], [h], [dt], Q.reshape(-1), GAMMA, halo_mode)
    return out.reshape(Q.shape), lam[0]


# ------------------------------------------------------------ free stream

@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("mode", [oracle.FIXED, oracle.PERIODIC])
def test_free_stream_is_preserved_bitwise(dim, mode):
    rng = np.random.default_rng(11 + dim)
    p = 5
    for _ in range(3):
        q = random_patch(rng, dim, 1)[(0,) * dim]          # one random state
        Q = np.broadcast_to(q, (p + 2,) * dim + (dim + 2,)).copy()
        out, _ = step1(Q, dim, dt=rng.uniform(0.01, 0.3), h=rng.uniform(0.01, 1.0),
                       halo_mode=mode)
        assert np.array_equal(interior(out, dim), interior(Q, dim))


# ------------------------------------------------------- conservation

@pytest.mark.parametrize("dim,p", [(2, 7), (3, 4)])
def test_periodic_patch_conserves_totals(dim, p):
    rng = np.random.default_rng(5)
    Q = random_patch(rng, dim, p)
    h = 0.1
    tot0 = interior(Q, dim).reshape(-1, dim + 2).sum(axis=0)
    mag = np.abs(interior(Q, dim)).reshape(-1, dim + 2).sum(axis=0)
    steps = 8
    cur = Q
    for s in range(steps):
        lam = oracle.batch_max_eigenvalue(dim, [p], cur.reshape(-1))[0]
        dt = 0.4 * h / (dim * lam)
        cur, _ = step1(cur, dim, dt, h, oracle.PERIODIC)
    tot = interior(cur, dim).reshape(-1, dim + 2).sum(axis=0)
    bound = 8 * p ** dim * EPS * mag * steps
    assert np.all(np.abs(tot - tot0) <= bound), (tot - tot0, bound)
    # the same patch with fixed halos is NOT conservative: fluxes through
    # the patch boundary change the totals (guards against a vacuous test)
    fixed, _ = step1(Q, dim, 0.4 * h / (dim * 3.0), h, oracle.FIXED)
    dtot = interior(fixed, dim).reshape(-1, dim + 2).sum(axis=0) - tot0
    assert np.max(np.abs(dtot)) > 1e-6


# ------------------------------------------------------------- symmetry

def _mirror(Q, dim, axis):
    """Reflect a patch along spatial axis (0 = x): flip that array axis and
    negate the momentum along it."""
    arr_axis = dim - 1 - axis                     # arrays are (z, y, x, k)
    M = np.flip(Q, axis=arr_axis).copy()
    M[..., 1 + axis] *= -1.0
    return M


def _swap_axes(Q, dim, a, b):
    """Exchange spatial axes a and b together with the two momenta."""
    M = np.swapaxes(Q, dim - 1 - a, dim - 1 - b).copy()
    M[..., [1 + a, 1 + b]] = M[..., [1 + b, 1 + a]]
    return M


@pytest.mark.parametrize("dim", [2, 3])
def test_mirror_symmetry_is_bitwise(dim):
    rng = np.random.default_rng(21)
    Q = random_patch(rng, dim, 6)
    out, _ = step1(Q, dim, dt=0.05, h=0.2)
    for axis in range(dim):
        mo, _ = step1(_mirror(Q, dim, axis), dim, dt=0.05, h=0.2)
        assert np.array_equal(interior(mo, dim), interior(_mirror(out, dim, axis), dim))


@pytest.mark.parametrize("dim,a,b,exact", [(2, 0, 1, True), (3, 0, 1, True),
                                          (3, 1, 2, False), (3, 0, 2, False)])
def test_axis_permutation_symmetry(dim, a, b, exact):
    rng = np.random.default_rng(31)
    Q = random_patch(rng, dim, 5)
    out, _ = step1(Q, dim, dt=0.05, h=0.2)
    so, _ = step1(_swap_axes(Q, dim, a, b), dim, dt=0.05, h=0.2)
    want = interior(_swap_axes(out, dim, a, b), dim)
    got = interior(so, dim)
    if exact:      # the x and y differences are added first, in either order
        assert np.array_equal(got, want)
    else:          # the z difference joins in a different order
        assert rel_linf(got, want, dim) < 4 * EPS


@pytest.mark.parametrize("dim", [2, 3])
def test_periodic_translation_invariance(dim):
    rng = np.random.default_rng(41)
    p = 6
    Q = random_patch(rng, dim, p)
    out, _ = step1(Q, dim, dt=0.04, h=0.1, halo_mode=oracle.PERIODIC)
    for axis in range(dim):
        arr_axis = dim - 1 - axis
        R = Q.copy()
        interior(R, dim)[...] = np.roll(interior(Q, dim), 2, axis=arr_axis)
        ro, _ = step1(R, dim, dt=0.04, h=0.1, halo_mode=oracle.PERIODIC)
        assert np.array_equal(interior(ro, dim),
                              np.roll(interior(out, dim), 2, axis=arr_axis))


def test_fixed_halo_is_copied_unchanged():
    rng = np.random.default_rng(51)
    Q = random_patch(rng, 2, 4)
    out, _ = step1(Q, 2, dt=0.05, h=0.2)
    mask = np.ones(Q.shape[:2], dtype=bool)
    mask[1:-1, 1:-1] = False
    assert np.array_equal(out[mask], Q[mask])


# ------------------------------------------------------ hand-worked value

def _read_golden(name):
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    rows = {}
    with open(path) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                parts = line.split()
                rows[parts[0]] = np.array([float(v) for v in parts[1:]])
    return rows


def test_hand_worked_single_volume():
    g = _read_golden("hand_worked_p1_2d.txt")
    Q = np.zeros((3, 3, 4))

    def put(j, i, row):
        Q[j, i] = cons_from_prim(row[0], row[1:3], row[3])

    put(1, 1, g["interior"])
    put(1, 0, g["left"])
    put(1, 2, g["right"])
    put(0, 1, g["lower"])
    put(2, 1, g["upper"])
    Q[0, 0] = Q[0, 2] = Q[2, 0] = Q[2, 2] = np.nan     # corners are never read
    out, _ = step1(Q, 2, dt=0.1, h=1.0)
    np.testing.assert_allclose(out[1, 1], g["expected"], rtol=2e-15, atol=4e-16)


# ---------------------------------------------------- eigenvalue and CFL

def test_max_eigenvalue_and_cfl_closed_form():
    # rho = 1.4, p = 1 gives c = 1; rho = 5.6, p = 1 gives c = 1/2.
    Q = np.zeros((4, 4, 4))
    Q[...] = cons_from_prim(1.4, [0.0, 0.0], 1.0)
    Q[1, 1] = cons_from_prim(1.4, [0.2, -0.9], 1.0)      # lam_y = 1.9  (largest)
    Q[2, 2] = cons_from_prim(5.6, [1.3, 0.0], 1.0)       # lam_x = 1.8
    Q[0, 1] = cons_from_prim(1.4, [0.0, 7.0], 1.0)       # halo: must be ignored
    Q[1, 3] = cons_from_prim(1.4, [-9.0, 0.0], 1.0)      # halo: must be ignored
    lam = oracle.batch_max_eigenvalue(2, [2], Q.reshape(-1))[0]
    assert abs(lam - 1.9) <= 2 * EPS * 1.9
    dt = oracle.cfl_time_step(2, [lam], [0.3], 0.4)[0]
    assert abs(dt - 0.4 * 0.3 / (2 * 1.9)) <= 4 * EPS * dt
    # the step reports the maximum eigenvalue of its NEW state
    _, lam_new = oracle.batch_step(2, [2], [1.0], [0.0], Q.reshape(-1))
    assert lam_new[0] == lam


# -------------------------------------------- linear (von Neumann) modes

def _eigenmodes(dim, n, rho0, vel0, p0, gamma=GAMMA):
    """Right eigenvectors (conserved variables) and eigenvalues of the Euler
    flux Jacobian along axis n at the base state, from the linearised
    primitive system: acoustic (1, +-c/rho, c^2) with speed u_n +- c,
    entropy (1, 0, 0) and shear (tangential velocity) with speed u_n."""
    c = math.sqrt(gamma * p0 / rho0)
    modes = []

    def to_cons(drho, dvel, dp):
        dq = np.zeros(dim + 2)
        dq[0] = drho
        dq[1:1 + dim] = np.asarray(vel0) * drho + rho0 * np.asarray(dvel)
        dq[dim + 1] = dp / (gamma - 1.0) + 0.5 * np.dot(vel0, vel0) * drho \
            + rho0 * np.dot(vel0, dvel)
        return dq

    for s in (+1.0, -1.0):
        dv = np.zeros(dim)
        dv[n] = s * c / rho0
        modes.append((to_cons(1.0, dv, c * c), vel0[n] + s * c))
    modes.append((to_cons(1.0, np.zeros(dim), 0.0), vel0[n]))
    for t in range(dim):
        if t != n:
            dv = np.zeros(dim)
            dv[t] = 1.0
            modes.append((to_cons(0.0, dv, 0.0), vel0[n]))
    return modes, c


@pytest.mark.parametrize("dim,axis", [(2, 0), (2, 1), (3, 0), (3, 1), (3, 2)])
def test_linear_modes_follow_von_neumann_amplification(dim, axis):
    """Small-amplitude eigenmodes on a periodic patch evolve as G(theta)^n with
    G = 1 - i (a dt/h) sin(theta) - (alpha dt/h) (1 - cos(theta)),
    a the mode's wave speed and alpha = |u_n| + c the Rusanov coefficient."""
    p = 16 if dim == 2 else 8
    rho0, p0 = 1.3, 0.9
    vel0 = np.array([0.31, -0.23, 0.17][:dim])
    modes, c0 = _eigenmodes(dim, axis, rho0, vel0, p0)
    h, dt, nsteps, m = 0.05, 0.005, 6, 1
    eps = 1e-7
    theta = 2 * math.pi * m / p
    alpha = abs(vel0[axis]) + c0
    base = cons_from_prim(rho0, vel0, p0)
    coord = np.arange(-1, p + 1)
    shape = (p + 2,) * dim
    jj = np.meshgrid(*([coord] * dim), indexing="ij")[dim - 1 - axis]   # index along axis
    for r, a in modes:
        Q = np.broadcast_to(base, shape + (dim + 2,)).copy()
        Q += eps * np.cos(theta * jj)[..., None] * r
        cur = Q
        for _ in range(nsteps):
            cur, _ = step1(cur, dim, dt, h, oracle.PERIODIC)
        G = 1 - 1j * (a * dt / h) * math.sin(theta) - (alpha * dt / h) * (1 - math.cos(theta))
        want = np.real((G ** nsteps) * np.exp(1j * theta * jj))[..., None] * r
        got = (cur - base) / eps
        err = np.max(np.abs(interior(got, dim) - interior(want, dim)))
        assert err < 1e-5 * np.max(np.abs(r)), (a, err)
        # the mode really changed: amplitude decay is visible
        assert abs(abs(G) ** nsteps - 1) > 1e-3


# --------------------------------------------------------- contact wave

@pytest.mark.parametrize("dim", [2, 3])
def test_contact_keeps_velocity_and_pressure(dim):
    """Uniform velocity and pressure with any density: Rusanov on the Euler
    equations keeps u and p unchanged (momentum and energy fluxes are affine
    in the mass flux on such data)."""
    rng = np.random.default_rng(61)
    p = 6
    shape = (p + 2,) * dim
    vel = np.array([0.4, -0.25, 0.1][:dim])
    Q = cons_from_prim(rng.uniform(0.5, 1.5, shape), np.broadcast_to(vel, shape + (dim,)),
                       np.full(shape, 0.8))
    cur = Q
    for _ in range(5):
        cur, _ = step1(cur, dim, dt=0.02, h=0.1, halo_mode=oracle.PERIODIC)
    rho, v, pr = prim_from_cons(interior(cur, dim), dim)
    assert np.max(np.abs(v - vel)) < 1e-13
    assert np.max(np.abs(pr - 0.8)) < 1e-13
    assert np.max(np.abs(rho - interior(Q, dim)[..., 0])) > 1e-3   # density moved


# ------------------------------------------------- first-order convergence

def _advected_sine_error(p):
    """rho = 1 + 0.2 sin(2 pi x), u = 0.5, v = 0, p = 1 on a periodic unit
    patch (data constant in y), run to t = 0.25; L1 error of rho against the
    exact cell averages of the translated profile."""
    h = 1.0 / p
    xe = np.arange(p + 1) * h                   # cell edges
    avg = lambda t: 1.0 + 0.2 * (np.cos(2 * np.pi * (xe[:-1] - 0.5 * t))
                                 - np.cos(2 * np.pi * (xe[1:] - 0.5 * t))) / (2 * np.pi * h)
    rho = np.zeros((p + 2, p + 2))
    rho[1:-1, 1:-1] = avg(0.0)[None, :]
    rho[0], rho[-1], rho[:, 0], rho[:, -1] = 1.0, 1.0, 1.0, 1.0
    Q = cons_from_prim(rho, np.broadcast_to([0.5, 0.0], (p + 2, p + 2, 2)), np.ones((p + 2, p + 2)))
    t, tend = 0.0, 0.25
    cur = Q
    while t < tend - 1e-14:
        lam = oracle.batch_max_eigenvalue(2, [p], cur.reshape(-1))[0]
        dt = min(0.4 * h / (2 * lam), tend - t)
        cur, _ = step1(cur, 2, dt, h, oracle.PERIODIC)
        t += dt
    err = np.abs(cur[1:-1, 1:-1, 0] - avg(tend)[None, :])
    return float(np.mean(err))


@pytest.mark.slow
def test_first_order_convergence_on_moving_contact():
    errs = [_advected_sine_error(p) for p in (16, 32, 64, 128)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert 0.9 <= orders[-1] <= 1.1, orders
    assert errs[-1] < errs[0] / 6


# ------------------------------------------------ independent brute force

def _brute_force_step(Q, dim, dt, h, gamma=GAMMA):
    """Face-major re-evaluation written directly from the formulas, sharing
    nothing with the oracle's volume-major loops."""
    p = Q.shape[0] - 2
    N = dim + 2
    out = Q.copy()
    acc = np.zeros((p,) * dim + (N,))

    def flux(q, n):
        rho = q[0]
        u = q[1:1 + dim] / rho
        pr = (gamma - 1) * (q[-1] - 0.5 * rho * np.dot(u, u))
        c = math.sqrt(gamma * pr / rho)
        F = u[n] * q
        F[1 + n] += pr
        F[-1] += pr * u[n]
        return F, abs(u[n]) + c

    for n in range(dim):
        arr = dim - 1 - n
        # every face normal to n once: the left face of each volume, plus the
        # right face of the last volume of each line
        for idx in np.ndindex(*((p,) * dim)):
            faces = [idx[arr]] + ([p] if idx[arr] == p - 1 else [])
            for f in faces:
                left = list(idx)
                left[arr] = f - 1
                right = list(idx)
                right[arr] = f
                qL = Q[tuple(x + 1 for x in left)]
                qR = Q[tuple(x + 1 for x in right)]
                FL, lL = flux(qL, n)
                FR, lR = flux(qR, n)
                Fh = 0.5 * (FL + FR) - 0.5 * max(lL, lR) * (qR - qL)
                if f - 1 >= 0:
                    acc[tuple(left)] += Fh           # right face of the left volume
                if f <= p - 1:
                    acc[tuple(right)] -= Fh          # left face of the right volume
    interior(out, dim)[...] = interior(Q, dim) - (dt / h) * acc
    return out


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2)])
def test_matches_independent_brute_force(dim, p):
    rng = np.random.default_rng(71 + p)
    Q = random_patch(rng, dim, p)
    got, _ = step1(Q, dim, dt=0.03, h=0.1)
    want = _brute_force_step(Q, dim, dt=0.03, h=0.1)
    assert rel_linf(interior(got, dim), interior(want, dim), dim) < 1e-14


# ----------------------------------------------------- batches and runs

def test_batch_of_ragged_patches_equals_patchwise_steps():
    rng = np.random.default_rng(81)
    sizes = [1, 3, 4, 2, 5]
    patches = [random_patch(rng, 2, s) for s in sizes]
    flat = np.concatenate([q.reshape(-1) for q in patches])
    dx = [0.1, 0.2, 0.3, 0.05, 0.11]
    dt = [0.01, 0.02, 0.005, 0.001, 0.03]
    out, lam = oracle.batch_step(2, sizes, dx, dt, flat)
    off = oracle.patch_offsets(2, sizes)
    for i, q in enumerate(patches):
        one, l1 = step1(q, 2, dt[i], dx[i])
        assert np.array_equal(out[off[i]:off[i + 1]], one.reshape(-1))
        assert lam[i] == l1


def test_run_chains_cfl_time_steps():
    rng = np.random.default_rng(91)
    q = random_patch(rng, 2, 4)
    Qf, lam, dt = oracle.batch_run(2, [4], [0.1], q.reshape(-1), steps=3)
    cur = q.reshape(-1)
    l = oracle.batch_max_eigenvalue(2, [4], cur)
    for _ in range(3):
        d = oracle.cfl_time_step(2, l, [0.1], 0.4)
        cur, l = oracle.batch_step(2, [4], [0.1], d, cur)
    assert np.array_equal(Qf, cur)
    assert np.array_equal(lam, l)
    assert np.array_equal(dt, oracle.cfl_time_step(2, l, [0.1], 0.4))


@pytest.mark.parametrize("index,npatch", [(1, 64), (3, 4), (4, 40), (5, 1)])
def test_workloads_stay_physical(index, npatch):
    from paper_2306_16731_gb300 import inputs
    w = inputs.config(index, num_patches=npatch)
    steps = min(w.steps, 10)
    Qf, lam, dt = oracle.batch_run(w.dim, w.patch_size, w.dx, w.Q0, steps,
                                   halo_mode=w.halo_mode)
    for q in patches_of(w, Qf):
        rho, _, pr = prim_from_cons(q, w.dim)
        assert np.all(rho > 0) and np.all(pr > 0)
    assert np.all(np.isfinite(lam)) and np.all(dt > 0)


def patches_of(w, flat):
    from tests._helpers import patches_interior
    return patches_interior(flat, w.dim, w.patch_size)


# ------------------------------------------------- conservation totals

@pytest.mark.parametrize("dim", [2, 3])
def test_batch_totals_closed_form_exclude_halos(dim):
    """Per-patch totals of a ragged batch of constant patches: p_i^d copies of
    the patch's state q_i summed, so exactly p_i^d q_i (the values have few
    significant bits, so every partial sum is exact).  The halo volumes hold
    a different value that would show in the totals if any were summed."""
    sizes = [1, 3, 2, 5] if dim == 2 else [1, 3, 2, 4]
    N = dim + 2
    states = [np.array([1.5, -0.25, 0.75, 2.5, 0.125][:N]) * (i + 1) for i in range(len(sizes))]
    parts = []
    for p, q in zip(sizes, states):
        a = np.full((p + 2,) * dim + (N,), 1.0e6)
        a[(slice(1, -1),) * dim] = q
        parts.append(a.reshape(-1))
    tot = oracle.batch_totals(dim, sizes, np.concatenate(parts))
    want = np.array([p ** dim * q for p, q in zip(sizes, states)])
    assert np.array_equal(np.asarray(tot).reshape(len(sizes), N), want)


@pytest.mark.parametrize("dim", [2, 3])
def test_batch_totals_are_interior_sums(dim):
    """Random ragged patches: the totals equal a brute-force sum over each
    patch's interior slice, and changing one halo volume (of any face) or
    one interior volume of the last plane changes exactly what it should."""
    rng = np.random.default_rng(71 + dim)
    sizes = [3, 5, 2] if dim == 3 else [4, 7, 1, 6]
    N = dim + 2
    pats = [random_patch(rng, dim, p) for p in sizes]
    flat = np.concatenate([q.reshape(-1) for q in pats])
    tot = np.asarray(oracle.batch_totals(dim, sizes, flat)).reshape(len(sizes), N)
    for i, q in enumerate(pats):
        brute = interior(q, dim).reshape(-1, N).sum(axis=0)
        assert np.allclose(tot[i], brute, rtol=1e-13, atol=0)
    # halo volumes on every face do not count
    for axis in range(dim):
        for side in (0, -1):
            mod = [q.copy() for q in pats]
            idx = [slice(1, -1)] * dim
            idx[axis] = side
            mod[0][tuple(idx)] += 100.0
            t2 = np.asarray(oracle.batch_totals(dim, sizes, np.concatenate([q.reshape(-1) for q in mod])))
            assert np.array_equal(t2.reshape(len(sizes), N), tot)
    # the last interior plane along the slowest axis does count
    mod = [q.copy() for q in pats]
    idx = [slice(1, -1)] * dim
    idx[0] = -2
    mod[-1][tuple(idx)] += 1.0
    t3 = np.asarray(oracle.batch_totals(dim, sizes, np.concatenate([q.reshape(-1) for q in mod]))).reshape(len(sizes), N)
    p = sizes[-1]
    assert np.allclose(t3[-1] - tot[-1], p ** (dim - 1), rtol=1e-12)
    assert np.array_equal(t3[:-1], tot[:-1])
