"""Where reduced precision itself puts the error, independent of any kernel.

The error target for the FP32 forms is a relative L-infinity of 1e-5 against
the FP64 oracle.  Two norms are reported for it:

* per unknown: max over volumes of |Q_k - Q_k^oracle| divided by max over
  volumes of |Q_k^oracle|, for each unknown k (the plan's definition);
* state-normalised: max over volumes and unknowns of |Q - Q^oracle| divided
  by max over volumes and unknowns of |Q^oracle|.

On the 3D pulse workload (4,096 periodic 8^3 patches, 50 steps) the momenta
end near 6e-5 while pressure fluxes are O(1), so float32 rounding of the
pressure flux differences alone moves the momenta by ~5e-8 absolute: the
per-unknown norm then divides that by 6e-5.  These tests run a float32
restatement of the step (``tests/fp_emulation.py``, numpy, no CUDA) from the
same start and show that this floor is the precision's, not a kernel's: the
emulation misses the per-unknown target on the momenta by the same order as
the CUDA kernels do (8.4e-4), while meeting the state-normalised one.  The
same emulation with the state rounded to bfloat16 after every step gives the
floor of the BF16-storage form.  The GPU tests compare the kernels' errors
with these floors directly.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2306_16731_gb300 import inputs
from tests import fp_emulation as fe


def _as_batch(w, flat):
    p = int(w.patch_size[0])
    return np.asarray(flat).reshape((w.num_patches,) + (p + 2,) * w.dim + (w.dim + 2,))


def _norms(got, ref, dim):
    """(state-normalised, per-unknown list) over the interiors."""
    core = (slice(None),) + (slice(1, -1),) * dim
    N = dim + 2
    g = np.asarray(got, dtype=np.float64)[core].reshape(-1, N)
    r = np.asarray(ref, dtype=np.float64)[core].reshape(-1, N)
    state = float(np.max(np.abs(g - r)) / np.max(np.abs(r)))
    per = [float(np.max(np.abs(g[:, k] - r[:, k])) / np.max(np.abs(r[:, k]))) for k in range(N)]
    return state, per


def _oracle_run(w, start64, steps):
    ref, _, _ = oracle.batch_run(w.dim, w.patch_size, w.dx, start64.reshape(-1), steps, w.gamma,
                                 w.halo_mode, w.cfl)
    return _as_batch(w, ref)


@pytest.mark.parametrize("cfg,T", [(1, 64), (2, 6), (3, 6)])
def test_emulation_in_float64_is_the_oracle(cfg, T):
    """The restatement is the oracle's scheme: in float64 one step gives the
    oracle's state and eigenvalues bitwise, and a CFL-chained run agrees to
    rounding."""
    w = inputs.config(cfg, num_patches=T)
    Q = _as_batch(w, w.Q0)
    lam0 = oracle.batch_max_eigenvalue(w.dim, w.patch_size, w.Q0)
    assert np.array_equal(fe.max_eigenvalue(Q, w.dim), lam0)
    dt = oracle.cfl_time_step(w.dim, lam0, w.dx, w.cfl)
    ref, lam = oracle.batch_step(w.dim, w.patch_size, w.dx, dt, w.Q0, w.gamma, w.halo_mode)
    got, glam = fe.step(Q, w.dim, dt, w.dx, w.gamma, w.halo_mode == inputs.PERIODIC)
    core = (slice(None),) + (slice(1, -1),) * w.dim
    assert np.array_equal(got[core], _as_batch(w, ref)[core])
    assert np.array_equal(glam, lam)
    run = fe.run(Q, w.dim, w.dx, 5, w.gamma, w.halo_mode == inputs.PERIODIC, w.cfl)
    state, _ = _norms(run, _oracle_run(w, Q, 5), w.dim)
    assert state <= 1e-14


def test_float32_floor_on_the_3d_pulse():
    """3D pulse, first 16 patches, 50 steps in float32: the state-normalised
    error meets 1e-5 by two orders, but the momenta miss the per-unknown 1e-5
    by more than an order of magnitude -- the CUDA kernels' 7e-4..8.4e-4 on
    these unknowns is this floor."""
    w = inputs.config(3, dtype=np.float32, num_patches=16)
    Q32 = _as_batch(w, w.Q0)
    ref = _oracle_run(w, Q32.astype(np.float64), w.steps)
    emu = fe.run(Q32, 3, w.dx, w.steps, w.gamma, True, w.cfl)
    state, per = _norms(emu, ref, 3)
    print("float32 emulation, 3D pulse: state %.2e, per unknown %s" % (state, " ".join("%.2e" % e for e in per)))
    assert state <= 1e-6
    assert per[0] <= 1e-6 and per[4] <= 1e-6                 # density and energy meet it
    for k in (1, 2, 3):                                       # the momenta cannot
        assert 1e-4 <= per[k] <= 5e-3, (k, per[k])


@pytest.mark.parametrize("cfg,T", [(2, 8), (1, 64)])
def test_float32_meets_the_per_unknown_target_on_uniform_data(cfg, T):
    """Where no unknown is near zero (the uniform random workloads) float32
    meets 1e-5 in both norms after the workload's full step count."""
    w = inputs.config(cfg, dtype=np.float32, num_patches=T)
    Q32 = _as_batch(w, w.Q0)
    ref = _oracle_run(w, Q32.astype(np.float64), w.steps)
    emu = fe.run(Q32, w.dim, w.dx, w.steps, w.gamma, False, w.cfl)
    state, per = _norms(emu, ref, w.dim)
    assert state <= 1e-6 and max(per) <= 1e-6, (state, per)


def test_bf16_storage_floor_on_the_3d_pulse():
    """BF16 storage: the state is rounded to 8 significant bits after every
    step, a relative error of at most 2^-8 per value and step.  If the step
    does not amplify errors in the maximum norm (the Rusanov scheme under its
    CFL condition), S steps stay within S * 2^-8 of the state's magnitude:
    0.195 after 50 steps -- the stated bound.  The emulation lands at ~2e-2
    (rounding errors partly cancel), which is where the CUDA kernel is."""
    w = inputs.config(3, dtype=np.float32, num_patches=16)
    Q32 = _as_batch(w, w.Q0)
    start = fe.bf16_round(Q32)
    ref = _oracle_run(w, start.astype(np.float64), w.steps)
    emu = fe.run(Q32, 3, w.dx, w.steps, w.gamma, True, w.cfl, storage="bf16")
    state, per = _norms(emu, ref, 3)
    print("bf16-storage emulation, 3D pulse: state %.2e, per unknown %s"
          % (state, " ".join("%.2e" % e for e in per)))
    bound = w.steps * 2.0 ** -8
    assert 5e-3 <= state <= bound
    assert max(per[1:4]) > 1e-2                               # momenta: far above 1e-5


def test_bf16_round_is_round_to_nearest_even():
    """The rounding the BF16-storage emulation relies on: exact for values
    with 8 significant bits, ties to even, monotone."""
    exact = np.array([1.0, 1.5, -2.75, 0.0078125, 255.0 * 2.0 ** -7], dtype=np.float32)
    assert np.array_equal(fe.bf16_round(exact), exact)
    ulp = 2.0 ** -7
    ties = np.array([1.0 + ulp / 2, 1.0 + 3 * ulp / 2], dtype=np.float32)
    assert np.array_equal(fe.bf16_round(ties), np.array([1.0, 1.0 + 2 * ulp], dtype=np.float32))
    x = np.sort(np.random.default_rng(0).uniform(-3, 3, 4096).astype(np.float32))
    r = fe.bf16_round(x)
    assert np.all(np.diff(r) >= 0) and np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -8)
