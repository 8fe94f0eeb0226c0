"""The oracle's pins must catch plausible mistakes.

Each case copies the oracle's C source to a temporary folder, plants one
mistake by a textual edit (a dropped term, a wrong sign, a swapped index, a
wrong coefficient), compiles it, routes the oracle module to the mutant and
runs the pins of ``test_oracle_pins``.  At least one pin must fail for every
mutant; the unmodified source must pass all of them.
"""
from __future__ import annotations

import os

import pytest

import oracle
from oracle import fv_oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(fv_oracle.__file__), "fv_oracle.c")

MUTANTS = {
    "dissipation_coefficient_1": ("- 0.5 * lam * (QR[k] - QL[k])", "- 1.0 * lam * (QR[k] - QL[k])"),
    "dissipation_sign": ("- 0.5 * lam * (QR[k] - QL[k])", "+ 0.5 * lam * (QR[k] - QL[k])"),
    "central_weight": ("0.5 * (FL[k] + FR[k])", "0.5 * (FL[k] + FL[k])"),
    "update_scale_dt_times_h": ("double scale = dt / h;", "double scale = dt * h;"),
    "update_sign": ("Q[c * N + q] - scale * acc[q]", "Q[c * N + q] + scale * acc[q]"),
    "flux_difference_sign": ("acc[q] += Fright[q] - Fleft[q];", "acc[q] += Fleft[q] - Fright[q];"),
    "pressure_missing_in_momentum_flux": ("(a == n ? pres : 0.0)", "0.0"),
    "pressure_on_wrong_momentum": ("(a == n ? pres : 0.0)", "(a == 0 ? pres : 0.0)"),
    "energy_flux_without_pressure": ("(q[dim + 1] + pres) * u[n]", "q[dim + 1] * u[n]"),
    "mass_flux_always_x": ("F[0] = q[1 + n];", "F[0] = q[1];"),
    "kinetic_energy_factor": ("(E - 0.5 * kin)", "(E - kin)"),
    "gamma_minus_one": ("*pres = (gamma - 1.0) *", "*pres = (gamma - 0.5) *"),
    "sound_speed_without_gamma": ("sqrt(gamma * (*pres) / rho)", "sqrt((*pres) / rho)"),
    "eigenvalue_without_abs": ("return fabs(u[n]) + snd;", "return u[n] + snd;"),
    "eigenvalue_min_not_max": ("lamL > lamR ? lamL : lamR", "lamL < lamR ? lamL : lamR"),
    "left_neighbour_always_x": ("lo[n] -= 1;", "lo[0] -= 1;"),
    "right_neighbour_always_x": ("hi[n] += 1;", "hi[0] += 1;"),
    "periodic_wrap_swapped": ("src[axis] = idx[axis] == -1 ? p - 1 : 0;",
                              "src[axis] = idx[axis] == -1 ? 0 : p - 1;"),
    "cfl_without_dimension": ("((double)dim * lambda[i])", "(lambda[i])"),
    "totals_include_x_halo": ("for (int ii = 0; ii < P; ++ii) {\n                    const double *c = Q + off[i]",
                              "for (int ii = -1; ii <= P; ++ii) {\n                    const double *c = Q + off[i]"),
    "totals_include_y_halo": ("for (int j = 0; j < P; ++j)\n                for (int ii = 0; ii < P; ++ii) {\n                    const double *c",
                              "for (int j = -1; j < P; ++j)\n                for (int ii = 0; ii < P; ++ii) {\n                    const double *c"),
    "totals_skip_last_z_plane": ("int kmax = dim == 3 ? P - 1 : 0;", "int kmax = dim == 3 ? P - 2 : 0;"),
    "totals_wrong_patch_offset": ("const double *c = Q + off[i] + cell_index", "const double *c = Q + off[0] + cell_index"),
    "max_eigenvalue_over_first_direction_only": ("for (int n = 0; n < dim; ++n) {\n                    double l",
                                                 "for (int n = 0; n < 1; ++n) {\n                    double l"),
}


def _pin_checks():
    """(name, callable) for every fast pin, with fixed parameters."""
    c = []
    for dim in (2, 3):
        for mode in (oracle.FIXED, oracle.PERIODIC):
            c.append(("free_stream_%d_%d" % (dim, mode),
                      lambda dim=dim, mode=mode: pins.test_free_stream_is_preserved_bitwise(dim, mode)))
        c.append(("mirror_%d" % dim, lambda dim=dim: pins.test_mirror_symmetry_is_bitwise(dim)))
        c.append(("translation_%d" % dim, lambda dim=dim: pins.test_periodic_translation_invariance(dim)))
        c.append(("contact_%d" % dim, lambda dim=dim: pins.test_contact_keeps_velocity_and_pressure(dim)))
    c.append(("conservation_2", lambda: pins.test_periodic_patch_conserves_totals(2, 7)))
    c.append(("conservation_3", lambda: pins.test_periodic_patch_conserves_totals(3, 4)))
    for args in [(2, 0, 1, True), (3, 0, 1, True), (3, 1, 2, False), (3, 0, 2, False)]:
        c.append(("permutation_%s" % (args,), lambda a=args: pins.test_axis_permutation_symmetry(*a)))
    for dim, axis in [(2, 0), (2, 1), (3, 0), (3, 1), (3, 2)]:
        c.append(("von_neumann_%d_%d" % (dim, axis),
                  lambda dim=dim, axis=axis: pins.test_linear_modes_follow_von_neumann_amplification(dim, axis)))
    c.append(("hand_worked", pins.test_hand_worked_single_volume))
    c.append(("eigenvalue_cfl", pins.test_max_eigenvalue_and_cfl_closed_form))
    c.append(("fixed_halo", pins.test_fixed_halo_is_copied_unchanged))
    for dim in (2, 3):
        c.append(("totals_closed_form_%d" % dim, lambda dim=dim: pins.test_batch_totals_closed_form_exclude_halos(dim)))
        c.append(("totals_interior_sums_%d" % dim, lambda dim=dim: pins.test_batch_totals_are_interior_sums(dim)))
    return c


def _failing_pins(lib_path):
    failed = []
    with fv_oracle.use_library(lib_path):
        for name, fn in _pin_checks():
            try:
                fn()
            except Exception:      # an assertion or a numerical blow-up both count
                failed.append(name)
    return failed


def test_unmodified_oracle_passes_every_pin(tmp_path):
    out = fv_oracle.compile_source(SRC, str(tmp_path / "clean.so"))
    assert _failing_pins(out) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert old in src, "mutation anchor not found: %r" % old
    mutated = src.replace(old, new)
    path = tmp_path / ("m_%s.c" % name)
    path.write_text(mutated)
    lib = fv_oracle.compile_source(str(path), str(tmp_path / ("m_%s.so" % name)))
    failed = _failing_pins(lib)
    assert failed, "no pin caught the planted mistake %s" % name
