"""Pins of the oracle's generic-PDE step (Eq. 1 with a non-conservative
product and a source): two-dimensional shallow water over a bathymetry b
with a Coriolis force, Q = (h, hu, hv, b).

Each pin is a property the method has by construction or a special case
with a closed form:
  * free stream (flat bottom, no rotation) is kept bitwise;
  * a uniform state over a flat bottom sees only the source: one explicit
    Euler step of the rotation ODE, hu' = hu + dt f hv, hv' = hv - dt f hu,
    and the momentum norm grows by sqrt(1 + (f dt)^2);
  * a lake at rest (h + b constant, no velocity) over an arbitrary bottom
    keeps zero momentum: the pressure-flux difference and the averaged
    non-conservative product cancel exactly, which fixes the sign, the one
    half and the averaged state of that product; its depth changes only by
    the Rusanov dissipation, a closed form for zero velocity;
  * mass is conserved on periodic patches, momentum too over a flat bottom
    without rotation; the bathymetry is never changed;
  * mirroring x (hu -> -hu, f -> -f) commutes with the step;
  * the eigenvalue is |u_n| + sqrt(g h).
A mutation test plants one mistake at a time in the oracle's source and
checks that one of these pins fails.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from oracle import fv_oracle

G = 9.81
SRC = os.path.join(os.path.dirname(fv_oracle.__file__), "fv_oracle.c")


def _patch(rng, p, h_range=(0.5, 1.5), vel=0.5, bottom=0.3, flat=False):
    e = p + 2
    Q = np.empty((e, e, 4))
    Q[..., 0] = rng.uniform(*h_range, (e, e))
    Q[..., 1] = Q[..., 0] * rng.uniform(-vel, vel, (e, e))
    Q[..., 2] = Q[..., 0] * rng.uniform(-vel, vel, (e, e))
    Q[..., 3] = 0.0 if flat else rng.uniform(-bottom, bottom, (e, e))
    return Q


def _step(Qs, h=0.1, dt=0.004, f=0.0, mode=oracle.FIXED):
    Qs = [np.asarray(q) for q in Qs]
    p = [q.shape[0] - 2 for q in Qs]
    out, lam = oracle.swe_batch_step(p, [h] * len(Qs), [dt] * len(Qs),
                                     np.concatenate([q.reshape(-1) for q in Qs]), G, f, mode)
    res, o = [], 0
    for q in Qs:
        res.append(out[o:o + q.size].reshape(q.shape))
        o += q.size
    return res, lam


@pytest.mark.parametrize("mode", [oracle.FIXED, oracle.PERIODIC])
def test_swe_free_stream_is_bitwise(mode):
    Q = np.tile(np.array([1.3, 0.4, -0.2, 0.25]), (7, 7, 1))
    (out,), _ = _step([Q], mode=mode)
    assert np.array_equal(out[1:-1, 1:-1], Q[1:-1, 1:-1])


@pytest.mark.parametrize("f", [0.7, -1.3])
def test_swe_coriolis_on_a_uniform_state_is_one_euler_step_of_the_rotation(f):
    hu, hv, dt = 0.37, -0.81, 0.004
    Q = np.tile(np.array([1.1, hu, hv, 0.05]), (6, 6, 1))
    (out,), _ = _step([Q], dt=dt, f=f)
    inner = out[1:-1, 1:-1]
    assert np.array_equal(inner[..., 0], np.full((4, 4), 1.1))
    assert np.array_equal(inner[..., 1], np.full((4, 4), hu + dt * (f * hv)))
    assert np.array_equal(inner[..., 2], np.full((4, 4), hv + dt * (-f * hu)))
    # explicit Euler on a rotation scales the momentum by sqrt(1 + (f dt)^2)
    norm = np.hypot(inner[..., 1], inner[..., 2])
    assert np.allclose(norm, np.hypot(hu, hv) * np.sqrt(1.0 + (f * dt) ** 2), rtol=1e-14, atol=0)


@pytest.mark.parametrize("f", [0.0, 0.9])
def test_swe_lake_at_rest_keeps_zero_momentum_over_any_bottom(f):
    rng = np.random.default_rng(3)
    p, eta, h_cell, dt = 9, 2.0, 0.1, 0.004
    b = rng.uniform(-0.6, 0.6, (p + 2, p + 2))
    Q = np.zeros((p + 2, p + 2, 4))
    Q[..., 0] = eta - b
    Q[..., 3] = b
    (out,), _ = _step([Q], h=h_cell, dt=dt, f=f)
    inner = out[1:-1, 1:-1]
    scale = dt / h_cell * 0.5 * G * np.max(Q[..., 0]) ** 2
    assert np.max(np.abs(inner[..., 1])) <= 1e-14 * scale
    assert np.max(np.abs(inner[..., 2])) <= 1e-14 * scale
    # depth: with zero velocity only the Rusanov dissipation acts on h
    h = Q[..., 0]
    c = np.sqrt(G * h)
    expect = h[1:-1, 1:-1].copy()
    for axis in (0, 1):            # array axis 0 is y, 1 is x
        lo = [slice(1, -1), slice(1, -1)]
        hi = [slice(1, -1), slice(1, -1)]
        lo[axis] = slice(0, -2)
        hi[axis] = slice(2, None)
        hc, hl, hr = h[1:-1, 1:-1], h[tuple(lo)], h[tuple(hi)]
        lr = np.maximum(c[1:-1, 1:-1], c[tuple(hi)])
        ll = np.maximum(c[tuple(lo)], c[1:-1, 1:-1])
        expect = expect + dt / h_cell * 0.5 * (lr * (hr - hc) - ll * (hc - hl))
    assert np.allclose(inner[..., 0], expect, rtol=1e-13, atol=0)


def test_swe_periodic_patch_conserves_mass_and_keeps_the_bottom():
    rng = np.random.default_rng(5)
    Q = _patch(rng, 8)
    (out,), _ = _step([Q], f=0.6, mode=oracle.PERIODIC)
    m0, m1 = Q[1:-1, 1:-1, 0].sum(), out[1:-1, 1:-1, 0].sum()
    assert abs(m1 - m0) <= 64 * np.finfo(float).eps * np.abs(Q[1:-1, 1:-1, 0]).sum()
    assert np.array_equal(out[1:-1, 1:-1, 3], Q[1:-1, 1:-1, 3])


def test_swe_flat_bottom_without_rotation_conserves_momentum_on_periodic_patches():
    rng = np.random.default_rng(6)
    Q = _patch(rng, 8, flat=True)
    (out,), _ = _step([Q], mode=oracle.PERIODIC)
    for k in (1, 2):
        d = out[1:-1, 1:-1, k].sum() - Q[1:-1, 1:-1, k].sum()
        assert abs(d) <= 256 * np.finfo(float).eps * (np.abs(Q[1:-1, 1:-1, :3]).sum())


def test_swe_mirror_in_x_commutes_with_the_step():
    rng = np.random.default_rng(8)
    Q = _patch(rng, 7)
    M = Q[:, ::-1].copy()
    M[..., 1] = -M[..., 1]
    (a,), _ = _step([Q], f=0.8)
    (bm,), _ = _step([M], f=-0.8)
    back = bm[:, ::-1].copy()
    back[..., 1] = -back[..., 1]
    assert np.allclose(back[1:-1, 1:-1], a[1:-1, 1:-1], rtol=0, atol=1e-15 * np.abs(a).max())


def test_swe_eigenvalue_is_velocity_plus_gravity_wave_speed():
    rng = np.random.default_rng(9)
    Q = _patch(rng, 6)
    lam = oracle.swe_batch_max_eigenvalue([6], Q.reshape(-1), G)
    h = Q[1:-1, 1:-1, 0]
    u = np.abs(Q[1:-1, 1:-1, 1] / h)
    v = np.abs(Q[1:-1, 1:-1, 2] / h)
    assert lam[0] == pytest.approx(np.max(np.maximum(u, v) + np.sqrt(G * h)), rel=1e-15)


def test_swe_fixed_halo_is_copied_and_patches_are_independent():
    rng = np.random.default_rng(10)
    A, B = _patch(rng, 5), _patch(rng, 9)
    (a2, b2), _ = _step([A, B], f=0.4)
    (a1,), _ = _step([A], f=0.4)
    assert np.array_equal(a2, a1)
    halo = np.ones(A.shape[:2], bool)
    halo[1:-1, 1:-1] = False
    assert np.array_equal(a2[halo], A[halo])


# --------------------------------------------------------------- mutations

def _swe_pins():
    return [
        ("free_stream_fixed", lambda: test_swe_free_stream_is_bitwise(oracle.FIXED)),
        ("free_stream_periodic", lambda: test_swe_free_stream_is_bitwise(oracle.PERIODIC)),
        ("coriolis", lambda: test_swe_coriolis_on_a_uniform_state_is_one_euler_step_of_the_rotation(0.7)),
        ("lake_at_rest", lambda: test_swe_lake_at_rest_keeps_zero_momentum_over_any_bottom(0.0)),
        ("lake_at_rest_rotating", lambda: test_swe_lake_at_rest_keeps_zero_momentum_over_any_bottom(0.9)),
        ("mass", test_swe_periodic_patch_conserves_mass_and_keeps_the_bottom),
        ("momentum", test_swe_flat_bottom_without_rotation_conserves_momentum_on_periodic_patches),
        ("mirror", test_swe_mirror_in_x_commutes_with_the_step),
        ("eigenvalue", test_swe_eigenvalue_is_velocity_plus_gravity_wave_speed),
        ("halo", test_swe_fixed_halo_is_copied_and_patches_are_independent),
    ]


SWE_MUTANTS = {
    "ncp_sign": ("D[1] = n == 0 ? g * hbar * (QR[3] - QL[3]) : 0.0;",
                 "D[1] = n == 0 ? -g * hbar * (QR[3] - QL[3]) : 0.0;"),
    "ncp_without_half": ("acc[k] += (Fr[k] - Fl[k]) + 0.5 * (Dr[k] + Dl[k]);",
                         "acc[k] += (Fr[k] - Fl[k]) + (Dr[k] + Dl[k]);"),
    "ncp_left_state": ("double hbar = 0.5 * (QL[0] + QR[0]);", "double hbar = QL[0];"),
    "ncp_wrong_axis": ("D[2] = n == 1 ? g * hbar * (QR[3] - QL[3]) : 0.0;",
                       "D[2] = n == 0 ? g * hbar * (QR[3] - QL[3]) : 0.0;"),
    "coriolis_sign": ("double S[SWE_N] = {0.0, f * qc[2], -f * qc[1], 0.0};",
                      "double S[SWE_N] = {0.0, -f * qc[2], f * qc[1], 0.0};"),
    "coriolis_components_swapped": ("double S[SWE_N] = {0.0, f * qc[2], -f * qc[1], 0.0};",
                                    "double S[SWE_N] = {0.0, f * qc[1], -f * qc[2], 0.0};"),
    "pressure_without_half": ("F[1] = q[1] * un + (n == 0 ? 0.5 * g * h * h : 0.0);",
                              "F[1] = q[1] * un + (n == 0 ? g * h * h : 0.0);"),
    "wave_speed_without_g": ("return fabs(q[1 + n] / h) + sqrt(g * h);", "return fabs(q[1 + n] / h) + sqrt(h);"),
    # the bottom gets the Rusanov dissipation and is updated like an unknown
    "bottom_evolved_like_an_unknown": [("for (int k = 0; k < 3; ++k)\n        Fhat[k] = 0.5",
                                        "for (int k = 0; k < 4; ++k)\n        Fhat[k] = 0.5"),
                                       ("    Fhat[3] = 0.0;\n}", "}"),
                                       ("Qout[c * SWE_N + 3] = qc[3];", "Qout[c * SWE_N + 3] = qc[3] - scale * acc[3];")],
    "source_scaled_by_dt_over_h": ("qc[k] - scale * acc[k] + dt * S[k];", "qc[k] - scale * acc[k] + scale * S[k];"),
    "swe_left_neighbour_always_x": ("int lo[2] = {i, j}, hi[2] = {i, j};\n                lo[n] -= 1;",
                                    "int lo[2] = {i, j}, hi[2] = {i, j};\n                lo[0] -= 1;"),
}


def _failing(lib_path):
    failed = []
    with fv_oracle.use_library(lib_path):
        for name, fn in _swe_pins():
            try:
                fn()
            except Exception:
                failed.append(name)
    return failed


def test_unmodified_swe_oracle_passes_every_pin(tmp_path):
    assert _failing(fv_oracle.compile_source(SRC, str(tmp_path / "clean.so"))) == []


@pytest.mark.parametrize("name", sorted(SWE_MUTANTS))
def test_planted_swe_mistake_is_caught(name, tmp_path):
    edits = SWE_MUTANTS[name]
    src = open(SRC).read()
    for old, new in (edits if isinstance(edits, list) else [edits]):
        assert old in src, "mutation anchor not found: %r" % old
        src = src.replace(old, new)
    path = tmp_path / ("m_%s.c" % name)
    path.write_text(src)
    lib = fv_oracle.compile_source(str(path), str(tmp_path / ("m_%s.so" % name)))
    assert _failing(lib), "no pin caught the planted mistake %s" % name
