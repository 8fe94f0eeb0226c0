"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (relative L-infinity over interior volumes: the largest error
over volumes and unknowns divided by the largest magnitude of the oracle's
state; per-unknown values are printed for the record):
  FP64 forms                       1e-12
  FP32 state and arithmetic        1e-5   (after the workload's full step count)
  BF16 storage, FP32 arithmetic    stated (each step rounds the state to 8 bits
                                   of mantissa); asserted below 5e-2
The oracle for reduced precision starts from the GPU's rounded initial state
widened to FP64; each side chains its own CFL time steps, so time-step drift
counts as error.  Large workloads run whole on the GPU, in the launch
configuration the benchmark times, and are checked on seeded samples of
patches: patches are independent, so the oracle run on the sample is exact.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2306_16731_gb300 import inputs
from tests._helpers import batch_rel_linf, batch_rel_linf_components, patches_interior
from tests.gpu_util import gpu_run, initial_fp64, subset, take_patches, to_device, torch_dtype

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 5e-2}
FORMS = {"fused": 0, "cascade": 1, "tile": 2}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_16731_gb300 import build
    build.build()
    oracle.build()


def _oracle(w, precision, steps, Q0=None):
    Q0 = w.Q0 if Q0 is None else Q0
    start = initial_fp64(Q0, precision)
    return oracle.batch_run(w.dim, w.patch_size, w.dx, start, steps, gamma=w.gamma,
                            halo_mode=w.halo_mode, cfl=w.cfl)


def _supported(w, precision, form):
    from paper_2306_16731_gb300 import fvbatch as fb
    try:
        b = fb.FVBatch(w.dim, w.patch_size, precision=precision, halo_mode=w.halo_mode, form=form)
        b.close()
        return True
    except fb.FVError as e:
        if e.code == fb.FV_EUNSUPPORTED:
            return False
        raise


def _check(w, precision, form, steps, use_graph=False, sample=None, tune=False):
    if not _supported(w, precision, form):
        pytest.skip("form %d has no kernel for these shapes" % form)
    got, lam, dtn, desc = gpu_run(w, precision, form, steps, use_graph=use_graph, tune=tune)
    if sample is None:
        ref, lam_ref, dt_ref = _oracle(w, precision, steps)
        got_s, psz = got, w.patch_size
        lam_g, dt_g = lam, dtn
    else:
        sw = subset(w, sample)
        ref, lam_ref, dt_ref = _oracle(sw, precision, steps)
        got_s, psz = take_patches(w, got, sample), sw.patch_size
        lam_g, dt_g = lam[sample], dtn[sample]
    err = batch_rel_linf(got_s, ref, w.dim, psz)
    comps = batch_rel_linf_components(got_s, ref, w.dim, psz)
    print("%s precision %d form %d: rel Linf %.3e, per unknown %s"
          % (w.name, precision, form, err, " ".join("%.2e" % c for c in comps)))
    tol = TOL[precision]
    assert err <= tol, "%s: rel Linf %.3e > %.1e (%s)" % (w.name, err, tol, desc)
    lam_err = np.max(np.abs(lam_g - lam_ref) / lam_ref) if len(lam_ref) else 0.0
    dt_err = np.max(np.abs(dt_g - dt_ref) / dt_ref) if len(dt_ref) else 0.0
    assert lam_err <= tol and dt_err <= tol, (lam_err, dt_err)
    return err


# ------------------------------------------------------------- workloads

@pytest.mark.parametrize("form", ["cascade", "tile", "fused"])
def test_workload1_fp64(form):
    w = inputs.config(1)
    _check(w, 0, FORMS[form], w.steps)


@pytest.mark.parametrize("form", ["cascade", "tile", "fused"])
def test_workload2_fp64_first_patches(form):
    w = inputs.config(2, num_patches=300)
    _check(w, 0, FORMS[form], w.steps)


@pytest.mark.parametrize("form,precision", [("fused", 1), ("fused", 0), ("cascade", 0),
                                            ("tile", 1)])
def test_workload2_full_size_sampled(form, precision):
    """16,384 patches of 16x16, 100 steps, graph-captured, as the benchmark runs it."""
    w = inputs.config(2, dtype=np.float64)
    sample = np.sort(np.random.default_rng(2).choice(w.num_patches, 24, replace=False))
    _check(w, precision, FORMS[form], w.steps, use_graph=True, sample=sample)


@pytest.mark.parametrize("precision", [1, 2])
def test_workload3_periodic_pulse(precision):
    w = inputs.config(3, num_patches=200)
    _check(w, precision, FORMS["fused"], w.steps)


def test_workload3_full_size_sampled():
    w = inputs.config(3)
    sample = np.sort(np.random.default_rng(3).choice(w.num_patches, 32, replace=False))
    _check(w, 1, FORMS["fused"], w.steps, use_graph=True, sample=sample)


def test_workload4_uneven_full_size_sampled():
    """50,000 patches of edge 4..32 with per-patch dx, 200 steps in one graph."""
    w = inputs.config(4, dtype=np.float32)
    rng = np.random.default_rng(4)
    sample = []
    for p in (4, 8, 16, 32):               # every size class is sampled
        cand = np.flatnonzero(w.patch_size == p)
        sample += list(rng.choice(cand, 8, replace=False))
    sample = np.sort(np.array(sample))
    _check(w, 1, FORMS["fused"], w.steps, use_graph=True, sample=sample, tune=True)


@pytest.mark.slow
def test_workload5_full_size_sampled():
    """32,768 patches of 16^3 (3.8 GB FP32 state), 20 steps."""
    w = inputs.config(5, dtype=np.float32)
    sample = np.sort(np.random.default_rng(5).choice(w.num_patches, 6, replace=False))
    _check(w, 1, FORMS["fused"], w.steps, use_graph=True, sample=sample)


# ------------------------------------------------------------ edge cases

def _refuses_fused(w, precision, form="fused"):
    """A form refuses a batch it has no kernel for, at creation, with
    FV_EUNSUPPORTED (the caller then picks another form; the loop cascade
    takes every batch)."""
    from paper_2306_16731_gb300 import fvbatch as fb
    with pytest.raises(fb.FVError) as e:
        fb.FVBatch(w.dim, w.patch_size, precision=precision, halo_mode=w.halo_mode, form=FORMS[form])
    assert e.value.code == fb.FV_EUNSUPPORTED


@pytest.mark.parametrize("form", ["cascade", "tile", "fused"])
@pytest.mark.parametrize("dim,sizes", [(2, [1, 2, 3, 5, 7, 16, 17, 31, 32, 33, 4, 8]),
                                       (3, [1, 2, 3, 4, 5, 8, 6, 7, 16, 24, 10])])
@pytest.mark.parametrize("precision", [0, 1])
def test_ragged_batches(form, dim, sizes, precision):
    w = inputs.uniform_batch(dim, sizes, seed=100 + dim, dx=np.linspace(0.05, 0.2, len(sizes)))
    if not _supported(w, precision, FORMS[form]):
        # fused 2D sweeps serve edges <= 32, fused 3D sweeps edges <= 16 (and
        # uniform multiples of 8 up to 32), the patch-wise kernel patches
        # that fit one block's shared memory: a batch with a larger patch is
        # refused, and the rest of it runs in that form
        _refuses_fused(w, precision, form)
        while not _supported(w, precision, FORMS[form]):
            w = subset(w, np.flatnonzero(w.patch_size < w.patch_size.max()))
        assert w.num_patches >= len(sizes) - 3
    _check(w, precision, FORMS[form], 7)


@pytest.mark.parametrize("precision", [0, 1])
def test_periodic_ragged(precision):
    w = inputs.uniform_batch(2, [3, 8, 16, 5], seed=7, halo_mode=inputs.PERIODIC)
    _check(w, precision, FORMS["fused"], 9)
    w3 = inputs.uniform_batch(3, [3, 8, 4], seed=8, halo_mode=inputs.PERIODIC)
    _check(w3, precision, FORMS["fused"], 5)


def test_single_volume_patch():
    w = inputs.uniform_batch(2, [1], seed=1)
    for form in FORMS.values():
        _check(w, 0, form, 3)


@pytest.mark.parametrize("dim,p", [(2, 1024), (3, 128)])
def test_maximum_edge_length(dim, p):
    """The largest edges the batch accepts run on the loop cascade; the
    fused form has no kernel for them and says so."""
    w = inputs.uniform_batch(dim, [p], seed=9, dx=0.01)
    _check(w, 0, FORMS["cascade"], 1)
    _check(w, 1, FORMS["cascade"], 1)
    _refuses_fused(w, 1)


def test_empty_batch_is_a_no_op():
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    b = fb.FVBatch(2, [], precision=0)
    assert b.state_elems() == 0
    q = torch.zeros(4, dtype=torch.float64, device="cuda")
    b.update(q, q.clone(), q, q)
    b.max_eigenvalue(q, q)
    b.status()
    b.close()


def test_free_stream_is_exact_on_gpu():
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    for dim, sizes in ((2, [16, 5, 32]), (3, [8, 3])):
        w = inputs.uniform_batch(dim, sizes, seed=3)
        N = dim + 2
        state = np.tile(w.Q0[:N], len(w.Q0) // N)
        for precision in (0, 1, 2):
            for form in FORMS.values():
                if not _supported(w, precision, form):
                    continue
                got, _, _, _ = gpu_run(w, precision, form, 4, Q0=state)
                want = initial_fp64(state, precision)
                for a, b in zip(patches_interior(got, dim, w.patch_size),
                                patches_interior(want, dim, w.patch_size)):
                    assert np.array_equal(a, b), (dim, precision, form)


def test_graph_replay_equals_eager_bitwise():
    w = inputs.config(2, num_patches=500)
    for form in FORMS.values():
        if not _supported(w, 1, form):
            continue
        a = gpu_run(w, 1, form, 12, use_graph=False)
        b = gpu_run(w, 1, form, 12, use_graph=True)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_forms_agree_closely_fp32():
    w = inputs.config(2, num_patches=200)
    res = [gpu_run(w, 1, f, 10)[0] for f in FORMS.values() if _supported(w, 1, f)]
    for r in res[1:]:
        assert batch_rel_linf(r, res[0], w.dim, w.patch_size) < 1e-5


def test_fixed_halo_of_output_is_untouched_or_copied():
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    w = inputs.uniform_batch(2, [4, 6], seed=5)
    for form in FORMS.values():
        if not _supported(w, 0, form):
            continue
        b = fb.FVBatch(2, w.patch_size, precision=0, form=form)
        q = torch.from_numpy(w.Q0.copy()).cuda()
        out = torch.full_like(q, 7.25)
        dx = torch.full((2,), 0.1, dtype=torch.float64, device="cuda")
        dt = torch.full((2,), 0.01, dtype=torch.float64, device="cuda")
        b.update(q, out, dx, dt)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        off = w.offsets()
        for i, p in enumerate(w.patch_size):
            patch = o[off[i]:off[i + 1]].reshape(p + 2, p + 2, 4)
            inp = w.Q0[off[i]:off[i + 1]].reshape(p + 2, p + 2, 4)
            mask = np.ones((p + 2, p + 2), bool)
            mask[1:-1, 1:-1] = False
            untouched = np.all(patch[mask] == 7.25, axis=-1)
            copied = np.all(patch[mask] == inp[mask], axis=-1)
            assert np.all(untouched | copied)
            assert np.all(patch[1:-1, 1:-1] != 7.25)
        b.close()


def test_periodic_conservation_on_gpu():
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    w = inputs.uniform_batch(3, [8, 6, 8], seed=12, halo_mode=inputs.PERIODIC)
    b = fb.FVBatch(3, w.patch_size, precision=0, halo_mode=inputs.PERIODIC)
    q = torch.from_numpy(w.Q0.copy()).cuda()
    t0 = torch.zeros(3 * 5, dtype=torch.float64, device="cuda")
    b.conserved_totals(q, t0)
    got, _, _, _ = gpu_run(w, 0, None, 10)
    t1 = torch.zeros_like(t0)
    b.conserved_totals(torch.from_numpy(got).cuda(), t1)
    torch.cuda.synchronize()
    ref = oracle.batch_totals(3, w.patch_size, w.Q0).reshape(-1)
    assert np.allclose(t0.cpu().numpy(), ref, rtol=1e-14, atol=1e-13)
    drift = np.abs(t1.cpu().numpy() - t0.cpu().numpy())
    mag = np.abs(oracle.batch_totals(3, w.patch_size, np.abs(w.Q0)).reshape(-1))
    bound = 8 * 8 ** 3 * np.finfo(np.float64).eps * mag * 10     # per-step round-off bound x steps
    assert np.all(drift <= bound), (drift, bound)
    b.close()


# -------------------------------------------------------- error handling

def test_nonphysical_state_is_reported():
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    w = inputs.uniform_batch(2, [8, 8], seed=2)
    Q = w.Q0.copy()
    Q[4 * 33] = -1.0                     # negative density at (x, y) = (2, 2) of patch 0
    for form in FORMS.values():
        if not _supported(w, 0, form):
            continue
        b = fb.FVBatch(2, w.patch_size, precision=0, form=form)
        q = torch.from_numpy(Q).cuda()
        out = q.clone()
        dx = torch.full((2,), 0.1, dtype=torch.float64, device="cuda")
        dt = torch.full((2,), 1e-4, dtype=torch.float64, device="cuda")
        lam = torch.zeros(2, dtype=torch.float64, device="cuda")
        b.max_eigenvalue(q, lam)
        with pytest.raises(fb.FVError) as ei:
            b.status()
        assert ei.value.code == fb.FV_ENONPHYSICAL
        b.update(q, out, dx, dt, lam)
        with pytest.raises(fb.FVError) as ei:
            b.status()
        assert ei.value.code == fb.FV_ENONPHYSICAL
        b.status()                       # the flag was cleared
        b.close()


def test_invalid_device_arguments():
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    b = fb.FVBatch(2, [4, 4], precision=0)
    n = b.state_elems()
    q = torch.zeros(n + 2, dtype=torch.float64, device="cuda")
    dx = torch.ones(2, dtype=torch.float64, device="cuda")
    for args in [(q, q), (q[:n], q[1:n + 1]), (q[1:], q[:n].clone())]:
        with pytest.raises(fb.FVError) as ei:
            b.update(args[0], args[1], dx, dx)
        assert ei.value.code == fb.FV_EINVAL
    with pytest.raises(fb.FVError) as ei:
        b.update(q[:n], q[:n].clone(), None, dx)
    assert ei.value.code == fb.FV_EINVAL
    with pytest.raises(fb.FVError) as ei:
        b.update(q[:n], q[:n].clone(), dx, dx, None, dx, cfl=-1.0)
    assert ei.value.code == fb.FV_EINVAL
    with pytest.raises(fb.FVError) as ei:
        b.set_form(9)
    assert ei.value.code == fb.FV_EINVAL
    b.close()


@pytest.mark.parametrize("p,T,precision", [(16, 3001, 1), (8, 1500, 1), (32, 700, 1), (4, 900, 1),
                                           (8, 700, 0), (16, 300, 0)])
def test_launch_shapes_are_bitwise_identical(p, T, precision):
    """Every launch shape the tuner can pick (one warp per item, counter-fed
    persistent warps, round-robin streaming warps; 16 warps per block included,
    which the FP64 row rings do not fit in shared memory and the launcher
    narrows) computes the same bits."""
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    w = inputs.uniform_batch(2, [p] * T, seed=40 + p, dx=0.02, dtype=np.float32 if precision == 1 else np.float64)
    results = []
    for shape in [(4, 0), (2, -1), (4, -2), (1, -2), (16, -2), (16, -1), (8, 1), (16, 0)]:
        b = fb.FVBatch(2, w.patch_size, precision=precision)
        b.set_launch_shape(*shape)
        qa = torch.from_numpy(w.Q0).cuda()
        qb = qa.clone()
        dx = torch.tensor(w.dx, device="cuda")
        lam = torch.zeros(T, dtype=torch.float64, device="cuda")
        dta, dtb = torch.zeros_like(lam), torch.zeros_like(lam)
        b.max_eigenvalue(qa, lam)
        b.cfl_time_step(lam, dx, 0.4, dta)
        b.run(qa, qb, dx, dta, dtb, lam, 5, 0.4, use_graph=shape[1] == -2)
        b.status()
        results.append((qb.cpu().numpy(), lam.cpu().numpy()))
        b.close()
    for q, l in results[1:]:
        assert np.array_equal(q, results[0][0]) and np.array_equal(l, results[0][1])
    # and the result is right
    ref, _, _ = oracle.batch_run(2, w.patch_size, w.dx, w.Q0.astype(np.float64), 5)
    assert batch_rel_linf(results[0][0], ref, 2, w.patch_size) < TOL[precision]


@pytest.mark.parametrize("p,T,precision,halo", [(16, 700, 1, inputs.FIXED), (8, 333, 2, inputs.FIXED),
                                                (32, 61, 1, inputs.PERIODIC), (4, 130, 1, inputs.FIXED),
                                                (16, 5, 2, inputs.PERIODIC)])
def test_sweep_ring_depths_are_bitwise_identical(p, T, precision, halo):
    """Every staging depth of the 2D sweep (4, 6 or 8 rows in flight per
    warp), with one-item-per-warp and persistent shapes, computes the same
    bits over five CFL-chained steps, and the result is the oracle's."""
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    w = inputs.uniform_batch(2, [p] * T, seed=80 + p, dx=np.linspace(0.01, 0.03, T), halo_mode=halo)
    results = []
    for ring, shape in [(0, (4, 0)), (4, (2, 0)), (6, (4, 0)), (4, (1, -1)), (6, (16, 1)), (8, (8, -1))]:
        b = fb.FVBatch(2, w.patch_size, precision=precision, halo_mode=halo)
        b.set_launch_shape(*shape)
        b.set_sweep_ring(ring)
        assert ("ring=%d" % (ring or 8)) in b.describe()
        qa = to_device(w.Q0, precision)
        qb = qa.clone()
        dx = torch.tensor(w.dx, device="cuda")
        lam = torch.zeros(T, dtype=torch.float64, device="cuda")
        dta, dtb = torch.zeros_like(lam), torch.zeros_like(lam)
        b.max_eigenvalue(qa, lam)
        b.cfl_time_step(lam, dx, 0.4, dta)
        b.run(qa, qb, dx, dta, dtb, lam, 5, 0.4, use_graph=ring == 6)
        b.status()
        results.append((qb.to(torch.float64).cpu().numpy(), lam.cpu().numpy(), dtb.cpu().numpy()))
        b.close()
    for r in results[1:]:
        for a_, b_ in zip(r, results[0]):
            assert np.array_equal(a_, b_)
    ref, lam_ref, _ = _oracle(w, precision, 5)
    assert batch_rel_linf(results[0][0], ref, 2, w.patch_size) <= TOL[precision]
    assert np.max(np.abs(results[0][1] - lam_ref) / lam_ref) <= TOL[precision]


def test_sweep_ring_is_refused_where_it_has_no_choice():
    from paper_2306_16731_gb300 import fvbatch as fb
    for dim, sizes, prec in ((2, [16] * 4, 0), (2, [16, 8], 1), (2, [12] * 3, 1), (3, [8] * 2, 1)):
        b = fb.FVBatch(dim, sizes, precision=prec)
        with pytest.raises(fb.FVError) as e:
            b.set_sweep_ring(4)
        assert e.value.code == fb.FV_EUNSUPPORTED
        assert "ring=8" in b.describe()
        b.set_sweep_ring(0)                       # the default is always accepted
        b.close()
    b = fb.FVBatch(2, [16] * 4, precision=1)
    with pytest.raises(fb.FVError) as e:
        b.set_sweep_ring(5)
    assert e.value.code == fb.FV_EINVAL
    b.close()


def test_tuner_records_shape_and_ring_depth(tmp_path, monkeypatch):
    """fv_batch_tune times launch shapes and ring depths together (every
    candidate checked bitwise against the first), keeps the fastest, and
    writes it -- ring depth included -- to the tuning cache file."""
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("FVBATCH_TUNE_CACHE", str(cache))
    w = inputs.uniform_batch(2, [16] * 777, seed=91, dx=0.02, dtype=np.float32)
    b = fb.FVBatch(2, w.patch_size, precision=1)
    qa = torch.from_numpy(w.Q0).cuda()
    scratch = qa.clone()
    dx = torch.tensor(w.dx, device="cuda")
    dt = torch.full((777,), 1e-3, dtype=torch.float64, device="cuda")
    b.tune(qa, scratch, dx, dt)
    desc = b.describe()
    line = [ln for ln in cache.read_text().splitlines() if "T777|" in ln and "prec1" in ln]
    assert len(line) == 1
    key, wpb, bps, ring = line[0].split()
    assert ("warps_per_block=%s blocks_per_sm=%s ring=%d" % (wpb, bps, int(ring) or 8)) in desc
    b.close()


def test_tuner_picks_a_shape_and_keeps_results(tmp_path, monkeypatch):
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    w = inputs.config(2, num_patches=2000, dtype=np.float32)
    a = gpu_run(w, 1, 0, 6, tune=False)
    b = gpu_run(w, 1, 0, 6, tune=True)
    assert np.array_equal(a[0], b[0])


@pytest.mark.parametrize("p,T", [(8, 300), (16, 40)])
def test_3d_block_kernel_periodic_conservation_and_graph(p, T):
    """The 8x8-block 3D kernel (uniform edge multiple of 8): periodic patches
    conserve their totals to round-off, graph replay equals eager launches
    bitwise, and the state matches the oracle."""
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    w = inputs.uniform_batch(3, [p] * T, seed=60 + p, halo_mode=inputs.PERIODIC, dtype=np.float32)
    eager = gpu_run(w, 1, 0, 6, use_graph=False)
    graph = gpu_run(w, 1, 0, 6, use_graph=True)
    assert "sweep3d" in eager[3]
    assert np.array_equal(eager[0], graph[0]) and np.array_equal(eager[1], graph[1])
    ref, _, _ = oracle.batch_run(3, w.patch_size, w.dx, initial_fp64(w.Q0, 1), 6, halo_mode=inputs.PERIODIC)
    assert batch_rel_linf(eager[0], ref, 3, w.patch_size) < 1e-5
    b = fb.FVBatch(3, w.patch_size, precision=0, halo_mode=inputs.PERIODIC)
    t0 = torch.zeros(T * 5, dtype=torch.float64, device="cuda")
    t1 = torch.zeros_like(t0)
    b.conserved_totals(torch.from_numpy(initial_fp64(w.Q0, 1)).cuda(), t0)
    b.conserved_totals(torch.from_numpy(eager[0]).cuda(), t1)
    torch.cuda.synchronize()
    mag = oracle.batch_totals(3, w.patch_size, np.abs(initial_fp64(w.Q0, 1))).reshape(-1)
    # FP32 arithmetic: a few float ulps of each volume's magnitude per step
    bound = 6 * 8 * np.finfo(np.float32).eps * mag + 1e-12
    assert np.all(np.abs(t1.cpu().numpy() - t0.cpu().numpy()) <= bound)
    b.close()


@pytest.mark.parametrize("p,halo,T", [(8, inputs.FIXED, 40), (16, inputs.FIXED, 9), (16, inputs.PERIODIC, 7),
                                      (24, inputs.FIXED, 5), (32, inputs.PERIODIC, 3)])
@pytest.mark.parametrize("precision", [1, 2])
def test_3d_block_kernel_bulk_plane_copies(p, halo, T, precision):
    """The 8x8-block 3D kernel fetches each plane of a device-resident uniform
    batch by one bulk copy (BF16 planes, whose bytes are not multiples of
    16, through the range widened to 16-byte boundaries), and the planes of
    mapped host buffers by per-thread chunk copies.  Both give the same bits,
    for compiled (8, 16) and run-time (24, 32) edges, and match the oracle."""
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    w = inputs.uniform_batch(3, [p] * T, seed=140 + p, dx=np.linspace(0.02, 0.04, T), halo_mode=halo)
    b = fb.FVBatch(3, w.patch_size, precision=precision, halo_mode=halo)
    if p != 8 or halo != inputs.PERIODIC:
        assert "sweep3d_b8" in b.describe()
    qa = to_device(w.Q0, precision)
    qb = torch.zeros_like(qa)
    dx = torch.tensor(w.dx, device="cuda")
    dt = torch.full((T,), 1e-3, dtype=torch.float64, device="cuda")
    lam = torch.zeros(T, dtype=torch.float64, device="cuda")
    dtn = torch.zeros_like(lam)
    b.update(qa, qb, dx, dt, lam, dtn, 0.4)
    torch.cuda.synchronize()
    hin = qa.cpu().pin_memory()
    hout = torch.zeros_like(hin).pin_memory()
    hl = torch.zeros(T, dtype=torch.float64).pin_memory()
    hd = torch.zeros(T, dtype=torch.float64).pin_memory()
    b.update_host(hin, hout, dx.cpu().pin_memory(), dt.cpu().pin_memory(), hl, hd, 0.4, 0)   # mapped buffers
    got = patches_interior(qb.to(torch.float64).cpu().numpy(), 3, w.patch_size)
    mapped = patches_interior(hout.to(torch.float64).numpy(), 3, w.patch_size)
    assert all(np.array_equal(g, m) for g, m in zip(got, mapped))
    assert np.array_equal(hl.numpy(), lam.cpu().numpy()) and np.array_equal(hd.numpy(), dtn.cpu().numpy())
    ref, lam_ref = oracle.batch_step(3, w.patch_size, w.dx, [1e-3] * T, initial_fp64(w.Q0, precision), halo_mode=halo)
    tol = TOL[precision] if precision == 1 else 1e-2
    assert batch_rel_linf(qb.to(torch.float64).cpu().numpy(), ref, 3, w.patch_size) <= tol
    assert np.max(np.abs(lam.cpu().numpy() - lam_ref) / lam_ref) <= tol
    b.close()


@pytest.mark.parametrize("dim,p", [(2, 16), (2, 8), (3, 8)])
def test_bfloat16_storage_error_is_stated_and_bounded(dim, p):
    w = inputs.uniform_batch(dim, [p] * 64, seed=70 + p, dx=0.02)
    got, lam, dtn, desc = gpu_run(w, 2, 0, 10)
    ref, lam_ref, _ = oracle.batch_run(dim, w.patch_size, w.dx, initial_fp64(w.Q0, 2), 10)
    err = batch_rel_linf(got, ref, dim, w.patch_size)
    print("bf16 storage dim %d p %d: rel Linf after 10 steps %.3e (%s)" % (dim, p, err, desc))
    assert err < 5e-2


def test_uneven_3d_batch_mixes_kernels_correctly():
    w = inputs.uniform_batch(3, [8, 4, 8, 6, 3, 8, 5], seed=80, dx=np.linspace(0.05, 0.1, 7))
    for precision in (0, 1):
        _check(w, precision, FORMS["fused"], 5)


def _grid_neighbours(G, dim, open_faces=()):
    from tests.test_oracle_halo_exchange import grid_neighbours
    nb = grid_neighbours(G, dim)
    for (i, f) in open_faces:
        nb[i, f] = -1
    return nb


@pytest.mark.parametrize("dim,G,p,precision", [(2, 5, 8, 0), (2, 4, 16, 1), (3, 2, 8, 0), (3, 2, 6, 2)])
def test_halo_exchange_is_bitwise_the_oracle_exchange(dim, G, p, precision):
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    T = G ** dim
    w = inputs.uniform_batch(dim, [p] * T, seed=90 + dim)
    nb = _grid_neighbours(G, dim, open_faces=[(0, 0), (1, 3)])
    b = fb.FVBatch(dim, w.patch_size, precision=precision)
    b.set_neighbours(nb.tolist())
    q = to_device(w.Q0, precision)
    b.halo_exchange(q)
    torch.cuda.synchronize()
    got = q.to(torch.float64).cpu().numpy()
    want = oracle.halo_exchange(dim, w.patch_size, nb, initial_fp64(w.Q0, precision))
    assert np.array_equal(got, want)
    b.close()


def _oracle_grid_run(w, nb, steps, precision):
    Q = initial_fp64(w.Q0, precision)
    lam = oracle.batch_max_eigenvalue(w.dim, w.patch_size, Q)
    for _ in range(steps):
        dt = oracle.cfl_time_step(w.dim, lam, w.dx, w.cfl)
        Q = oracle.halo_exchange(w.dim, w.patch_size, nb, Q)
        Q, lam = oracle.batch_step(w.dim, w.patch_size, w.dx, dt, Q, w.gamma, w.halo_mode)
    return Q, lam


@pytest.mark.parametrize("form", ["fused", "cascade", "tile"])
@pytest.mark.parametrize("dim,G,p,precision", [(2, 6, 16, 0), (2, 4, 8, 1), (3, 2, 8, 0)])
def test_patch_grid_with_neighbours_matches_oracle(form, dim, G, p, precision):
    """Patches wired as a periodic grid (two faces left open to their own
    halos): the fused 2D kernels read neighbours in-kernel, every other
    kernel gets an exchange before each update inside fv_batch_run."""
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    T = G ** dim
    w = inputs.uniform_batch(dim, [p] * T, seed=110 + dim + p, dx=np.linspace(0.01, 0.02, T))
    nb = _grid_neighbours(G, dim, open_faces=[(0, 1), (T - 1, 2)])
    if not _supported(w, precision, FORMS[form]):
        pytest.skip("no kernel")
    b = fb.FVBatch(dim, w.patch_size, precision=precision, form=FORMS[form])
    b.set_neighbours(nb.tolist())
    qa = to_device(w.Q0, precision)
    qb = qa.clone()
    dx = torch.tensor(w.dx, device="cuda")
    lam = torch.zeros(T, dtype=torch.float64, device="cuda")
    dta, dtb = torch.zeros_like(lam), torch.zeros_like(lam)
    b.max_eigenvalue(qa, lam)
    b.cfl_time_step(lam, dx, w.cfl, dta)
    steps = 7
    b.run(qa, qb, dx, dta, dtb, lam, steps, w.cfl, use_graph=True)
    b.status()
    got = (qb if steps % 2 else qa).to(torch.float64).cpu().numpy()
    ref, lam_ref = _oracle_grid_run(w, nb, steps, precision)
    err = batch_rel_linf(got, ref, dim, w.patch_size)
    assert err <= TOL[precision], (err, b.describe())
    assert np.max(np.abs(lam.cpu().numpy() - lam_ref) / lam_ref) <= TOL[precision]
    b.close()


def test_neighbour_table_is_validated():
    from paper_2306_16731_gb300 import fvbatch as fb
    b = fb.FVBatch(2, [4, 4, 8], precision=0)
    for bad in ([[5, -1, -1, -1]] * 3, [[2, -1, -1, -1], [-1] * 4, [-1] * 4], [[-2, -1, -1, -1]] * 3):
        with pytest.raises(fb.FVError) as ei:
            b.set_neighbours(bad)
        assert ei.value.code == fb.FV_EINVAL
    with pytest.raises(fb.FVError):
        import torch
        b.halo_exchange(torch.zeros(8, device="cuda"))      # no table registered
    b.set_neighbours([[1, -1, -1, -1], [-1, 0, -1, -1], [-1] * 4])
    b.set_neighbours(None)
    b.close()


@pytest.mark.parametrize("dim,sizes,precision,halo", [(2, [16] * 700, 1, inputs.FIXED), (3, [8] * 90, 1, inputs.FIXED),
                                                      (3, [8] * 90, 1, inputs.PERIODIC),
                                                      (3, [8] * 70, 2, inputs.PERIODIC),
                                                      (2, [16] * 64, 0, inputs.FIXED),
                                                      (2, [8, 16, 4, 8, 32] * 7, 1, inputs.FIXED)])
def test_host_state_update_matches_device_update(dim, sizes, precision, halo):
    """fv_patch_batch_update_host (pipelined chunks of host-to-device copy,
    update, device-to-host copy, or with 0 chunks the kernels working on the
    mapped host buffers directly) gives the device update's interiors,
    eigenvalues and time steps bitwise, for any chunk count."""
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    w = inputs.uniform_batch(dim, sizes, seed=130 + dim, dx=0.02, halo_mode=halo)
    T = w.num_patches
    dtype = torch_dtype(precision)
    b = fb.FVBatch(dim, w.patch_size, precision=precision, halo_mode=halo)
    qa = torch.from_numpy(w.Q0).to("cuda", dtype)
    qb = qa.clone()
    dx = torch.tensor(w.dx, device="cuda")
    dt = torch.full((T,), 2e-3, dtype=torch.float64, device="cuda")
    lam = torch.zeros(T, dtype=torch.float64, device="cuda")
    dtn = torch.zeros_like(lam)
    b.update(qa, qb, dx, dt, lam, dtn, 0.4)
    torch.cuda.synchronize()
    ref = patches_interior(qb.to(torch.float64).cpu().numpy(), dim, w.patch_size)
    hin = qa.cpu().pin_memory()
    for chunks in (1, 4, 7, 0):
        hout = torch.zeros_like(hin).pin_memory()
        hl = torch.zeros(T, dtype=torch.float64).pin_memory()
        hd = torch.zeros(T, dtype=torch.float64).pin_memory()
        b.update_host(hin, hout, dx.cpu().pin_memory(), dt.cpu().pin_memory(), hl, hd, 0.4, chunks)
        got = patches_interior(hout.to(torch.float64).numpy(), dim, w.patch_size)
        if dim == 3 and halo == inputs.PERIODIC and chunks == 0:
            # mapped host buffers run the 8x8-block kernel instead of the
            # one-warp periodic kernel (whose bulk copies address device
            # memory only): same scheme, other rounding
            tol = 1e-6 if precision == 1 else 1e-2
            assert batch_rel_linf(hout.to(torch.float64).numpy(), qb.to(torch.float64).cpu().numpy(), dim,
                                  w.patch_size) < tol
            assert np.allclose(hl.numpy(), lam.cpu().numpy(), rtol=tol, atol=0)
            continue
        assert all(np.array_equal(g, r) for g, r in zip(got, ref)), chunks
        assert np.array_equal(hl.numpy(), lam.cpu().numpy()) and np.array_equal(hd.numpy(), dtn.cpu().numpy())
    # and the host path's result is the oracle's step from the same start
    oref, olam = oracle.batch_step(dim, w.patch_size, w.dx, [2e-3] * T, initial_fp64(w.Q0, precision),
                                   halo_mode=halo)
    assert batch_rel_linf(hout.to(torch.float64).numpy(), oref, dim, w.patch_size) <= TOL[precision]
    assert np.max(np.abs(hl.numpy() - olam) / olam) <= TOL[precision]
    b.close()


def _host_chain_setup(dim, sizes, precision, halo, seed, form="fused"):
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    w = inputs.uniform_batch(dim, sizes, seed=seed, dx=np.linspace(0.02, 0.03, len(sizes)), halo_mode=halo)
    T = w.num_patches
    b = fb.FVBatch(dim, w.patch_size, precision=precision, halo_mode=halo, form=FORMS[form])
    q0 = torch.from_numpy(w.Q0).to(torch_dtype(precision))
    lam0 = torch.zeros(T, dtype=torch.float64, device="cuda")
    dt0 = torch.zeros_like(lam0)
    dx = torch.tensor(w.dx, device="cuda")
    b.max_eigenvalue(q0.cuda(), lam0)
    b.cfl_time_step(lam0, dx, w.cfl, dt0)
    torch.cuda.synchronize()
    return w, b, q0, dt0.cpu()


@pytest.mark.parametrize("dim,sizes,precision,halo,form", [(2, [16] * 300, 1, inputs.FIXED, "fused"),
                                                           (3, [8] * 40, 1, inputs.PERIODIC, "fused"),
                                                           (3, [16] * 12, 1, inputs.FIXED, "fused"),
                                                           (2, [8, 16, 4] * 5, 0, inputs.FIXED, "fused"),
                                                           (2, [16] * 64, 2, inputs.FIXED, "fused"),
                                                           (3, [8] * 16, 2, inputs.PERIODIC, "fused"),
                                                           (2, [8] * 40, 0, inputs.FIXED, "cascade"),
                                                           (3, [4] * 20, 1, inputs.FIXED, "tile")])
def test_host_time_stepping_equals_per_step_calls_and_the_oracle(dim, sizes, precision, halo, form):
    """fv_patch_batch_run_host: S CFL-chained steps with the state in host
    memory, every step copied in and out, the chunks' chains overlapping
    across steps.  Bitwise the same final state, time steps and eigenvalues
    as S calls of fv_patch_batch_update_host with the buffers alternated,
    for 1, 3 and 8 chunks, and within the precision's tolerance of the
    oracle's S CFL-chained steps; fixed halos come back unchanged."""
    import torch
    S = 5
    w, b, q0, dt0 = _host_chain_setup(dim, sizes, precision, halo, 150 + dim, form)
    T = w.num_patches
    pin = lambda t: t.clone().pin_memory()
    hdx = pin(torch.from_numpy(w.dx.copy()))
    # reference: S single-step calls
    rq = [pin(q0), pin(q0)]
    rdt = [pin(dt0), pin(torch.zeros(T, dtype=torch.float64))]
    rlam = pin(torch.zeros(T, dtype=torch.float64))
    for s_ in range(S):
        i = s_ & 1
        b.update_host(rq[i], rq[1 - i], hdx, rdt[i], rlam, rdt[1 - i], w.cfl, 4)
    ref_q, ref_dt = rq[S & 1], rdt[S & 1]
    for chunks in (1, 3, 8):
        hq = [pin(q0), pin(q0)]
        hdt = [pin(dt0), pin(torch.zeros(T, dtype=torch.float64))]
        hlam = pin(torch.zeros(T, dtype=torch.float64))
        b.run_host(hq[0], hq[1], hdx, hdt[0], hdt[1], hlam, S, w.cfl, chunks)
        got = patches_interior(hq[S & 1].to(torch.float64).numpy(), dim, w.patch_size)
        ref = patches_interior(ref_q.to(torch.float64).numpy(), dim, w.patch_size)
        assert all(np.array_equal(g, r) for g, r in zip(got, ref)), chunks
        assert np.array_equal(hdt[S & 1].numpy(), ref_dt.numpy()), chunks
        assert np.array_equal(hlam.numpy(), rlam.numpy()), chunks
        if halo == inputs.FIXED:
            assert torch.equal(hq[S & 1], ref_q)                          # halos included
            assert_halos_equal(hq[S & 1].to(torch.float64).numpy(), initial_fp64(w.Q0, precision), dim,
                               w.patch_size)
    b.status()
    b.close()
    oref, olam, _ = oracle.batch_run(dim, w.patch_size, w.dx, initial_fp64(w.Q0, precision), S, gamma=w.gamma,
                                     halo_mode=halo, cfl=w.cfl)
    # BF16 storage rounds the state every step: within S * 2^-8 of the state
    tol = TOL[precision] if precision != 2 else S * 2.0 ** -8
    assert batch_rel_linf(ref_q.to(torch.float64).numpy(), oref, dim, w.patch_size) <= tol
    assert np.max(np.abs(rlam.numpy() - olam) / olam) <= tol


def assert_halos_equal(a, b, dim, sizes):
    """Every halo volume of the batch state a equals b's."""
    off = 0
    for p in sizes:
        n = (int(p) + 2) ** dim * (dim + 2)
        pa = a[off:off + n].reshape((int(p) + 2,) * dim + (dim + 2,))
        pb = b[off:off + n].reshape((int(p) + 2,) * dim + (dim + 2,))
        mask = np.ones((int(p) + 2,) * dim, bool)
        mask[(slice(1, -1),) * dim] = False
        assert np.array_equal(pa[mask], pb[mask])
        off += n


@pytest.mark.parametrize("dim,G,p,form", [(3, 2, 8, "fused"), (2, 4, 16, "fused"), (2, 3, 8, "tile")])
def test_host_time_stepping_on_a_neighbour_grid_equals_fv_batch_run(dim, G, p, form):
    """With a neighbour table, fv_patch_batch_run_host fills the face halos
    from the neighbours before each step (where the kernel does not read
    them itself), as fv_batch_run does on device buffers: the same interiors,
    eigenvalues and time steps bitwise, and the oracle's grid run."""
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    T = G ** dim
    S = 5
    w = inputs.uniform_batch(dim, [p] * T, seed=180 + dim + p, dx=np.linspace(0.01, 0.02, T))
    nb = _grid_neighbours(G, dim, open_faces=[(0, 1), (T - 1, 2)])
    b = fb.FVBatch(dim, w.patch_size, precision=1, form=FORMS[form])
    b.set_neighbours(nb.tolist())
    q0 = torch.from_numpy(w.Q0).to(torch.float32)
    dx = torch.tensor(w.dx, device="cuda")
    lam = torch.zeros(T, dtype=torch.float64, device="cuda")
    dta, dtb = torch.zeros_like(lam), torch.zeros_like(lam)
    b.max_eigenvalue(q0.cuda(), lam)
    b.cfl_time_step(lam, dx, w.cfl, dta)
    dt0 = dta.cpu()
    qa, qb = q0.cuda(), q0.cuda()
    b.run(qa, qb, dx, dta, dtb, lam, S, w.cfl, use_graph=False)
    ref_q = (qb if S % 2 else qa).cpu()
    ref_dt, ref_lam = (dtb if S % 2 else dta).cpu(), lam.cpu()
    pin = lambda t: t.clone().pin_memory()
    hq = [pin(q0), pin(q0)]
    hdt = [pin(dt0), pin(torch.zeros(T, dtype=torch.float64))]
    hl = pin(torch.zeros(T, dtype=torch.float64))
    b.run_host(hq[0], hq[1], pin(dx.cpu()), hdt[0], hdt[1], hl, S, w.cfl, 4)
    b.status()
    got = patches_interior(hq[S & 1].to(torch.float64).numpy(), dim, w.patch_size)
    ref = patches_interior(ref_q.to(torch.float64).numpy(), dim, w.patch_size)
    assert all(np.array_equal(g, r) for g, r in zip(got, ref))
    assert torch.equal(hdt[S & 1], ref_dt) and torch.equal(hl, ref_lam)
    oref, olam = _oracle_grid_run(w, nb, S, 1)
    assert batch_rel_linf(hq[S & 1].to(torch.float64).numpy(), oref, dim, w.patch_size) <= TOL[1]
    b.close()


def test_host_time_stepping_rejects_bad_arguments_and_handles_no_steps():
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    w, b, q0, dt0 = _host_chain_setup(2, [16] * 8, 1, inputs.FIXED, 160)
    pin = lambda t: t.clone().pin_memory()
    hq = [pin(q0), pin(q0)]
    hdx = pin(torch.from_numpy(w.dx.copy()))
    hdt = [pin(dt0), pin(dt0)]
    before = hq[0].clone()
    b.run_host(hq[0], hq[1], hdx, hdt[0], hdt[1], None, 0, 0.4, 4)            # no steps: nothing moves
    assert torch.equal(hq[0], before)
    for kw in ({"steps": -1}, {"chunks": 0}, {"chunks": 65}, {"cfl": 0.0}):
        args = dict(steps=2, cfl=0.4, chunks=4)
        args.update(kw)
        with pytest.raises(fb.FVError) as e:
            b.run_host(hq[0], hq[1], hdx, hdt[0], hdt[1], None, args["steps"], args["cfl"], args["chunks"])
        assert e.value.code == fb.FV_EINVAL
    with pytest.raises(fb.FVError) as e:
        b.run_host(hq[0], hq[0], hdx, hdt[0], hdt[1], None, 2, 0.4, 4)          # Q_a is Q_b
    assert e.value.code == fb.FV_EINVAL
    with pytest.raises(fb.FVError) as e:
        b.run_host(hq[0], hq[1], hdx, hdt[0], hdt[0], None, 2, 0.4, 4)          # dt_a is dt_b
    assert e.value.code == fb.FV_EINVAL
    with pytest.raises(fb.FVError) as e:
        b.run_host(hq[0], None, hdx, hdt[0], hdt[1], None, 2, 0.4, 4)
    assert e.value.code == fb.FV_EINVAL
    b.close()


@pytest.mark.parametrize("chunks", [1, 4])
def test_chained_host_updates_keep_fixed_halos_and_match_the_oracle(chunks):
    """Single-step host updates chained by the caller (output of one the
    input of the next): with fixed halos the staged output carries the
    input's halo volumes back, so the chain is the oracle's."""
    import torch
    S = 4
    w, b, q0, dt0 = _host_chain_setup(2, [16] * 64, 1, inputs.FIXED, 170)
    T = w.num_patches
    pin = lambda t: t.clone().pin_memory()
    hdx = pin(torch.from_numpy(w.dx.copy()))
    hq = [pin(q0), pin(torch.full_like(q0, float("nan")))]                  # output halos start as NaN
    hdt = [pin(dt0), pin(torch.zeros(T, dtype=torch.float64))]
    hlam = pin(torch.zeros(T, dtype=torch.float64))
    for s_ in range(S):
        i = s_ & 1
        b.update_host(hq[i], hq[1 - i], hdx, hdt[i], hlam, hdt[1 - i], w.cfl, chunks)
    b.status()
    assert_halos_equal(hq[S & 1].to(torch.float64).numpy(), initial_fp64(w.Q0, 1), 2, w.patch_size)
    oref, olam, _ = oracle.batch_run(2, w.patch_size, w.dx, initial_fp64(w.Q0, 1), S, gamma=w.gamma,
                                     halo_mode=inputs.FIXED, cfl=w.cfl)
    assert batch_rel_linf(hq[S & 1].to(torch.float64).numpy(), oref, 2, w.patch_size) <= TOL[1]
    assert np.max(np.abs(hlam.numpy() - olam) / olam) <= TOL[1]
    b.close()


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("T", [1, 5, 37, 700])
def test_periodic_8cubed_warp_kernel_shapes_and_oracle(precision, T):
    """Periodic 8^3 patches run the one-warp-per-patch kernel (bulk-copied
    plane ring, packed pair arithmetic).  Every launch shape gives the same
    bits, including shapes where one warp walks several patches (its copy
    ring then runs across patches); the state and eigenvalues match the
    oracle's periodic step from the same (rounded) start."""
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    w = inputs.uniform_batch(3, [8] * T, seed=90 + T, dx=np.linspace(0.05, 0.1, T),
                             halo_mode=inputs.PERIODIC)
    dtype = torch_dtype(precision)
    results = []
    for shape in [(4, 0), (1, 0), (3, 0), (16, -1), (1, 1), (2, 1), (8, 2)]:
        b = fb.FVBatch(3, w.patch_size, precision=precision, halo_mode=inputs.PERIODIC)
        b.set_launch_shape(*shape)
        assert "fused_kernel=sweep3d_p8" in b.describe()
        qa = to_device(w.Q0, precision)
        qb = torch.zeros_like(qa)
        dx = torch.tensor(w.dx, device="cuda")
        dt = torch.full((T,), 2e-3, dtype=torch.float64, device="cuda")
        lam = torch.zeros(T, dtype=torch.float64, device="cuda")
        dtn = torch.zeros_like(lam)
        b.update(qa, qb, dx, dt, lam, dtn, 0.4)
        b.status()
        results.append((qb.to(torch.float64).cpu().numpy(), lam.cpu().numpy(), dtn.cpu().numpy()))
        b.close()
    for q, l, d in results[1:]:
        assert np.array_equal(patches_interior(q, 3, w.patch_size), patches_interior(results[0][0], 3, w.patch_size))
        assert np.array_equal(l, results[0][1]) and np.array_equal(d, results[0][2])
    q0 = initial_fp64(w.Q0, precision)
    ref, lam_ref = oracle.batch_step(3, w.patch_size, w.dx, [2e-3] * T, q0, halo_mode=inputs.PERIODIC)
    tol = 1e-5 if precision == 1 else 2e-2
    assert batch_rel_linf(results[0][0], ref, 3, w.patch_size) < tol
    assert np.max(np.abs(results[0][1] - lam_ref) / lam_ref) < (1e-5 if precision == 1 else 2e-2)
    assert np.allclose(results[0][2], 0.4 * np.asarray(w.dx) / (3 * results[0][1]), rtol=1e-15, atol=0)
    # rows are written whole: x-halo volumes of interior rows hold the wrapped values
    E = 10
    qf = results[0][0].reshape(T, E, E, E, 5)
    assert np.array_equal(qf[:, 1:-1, 1:-1, E - 1], qf[:, 1:-1, 1:-1, 1])
    assert np.array_equal(qf[:, 1:-1, 1:-1, 0], qf[:, 1:-1, 1:-1, E - 2])


def test_periodic_8cubed_warp_kernel_agrees_with_tile_form():
    w = inputs.uniform_batch(3, [8] * 200, seed=97, halo_mode=inputs.PERIODIC, dtype=np.float32)
    fused = gpu_run(w, 1, FORMS["fused"], 8)
    tile = gpu_run(w, 1, FORMS["tile"], 8)
    assert "sweep3d_p8" in fused[3]
    ref, _, _ = oracle.batch_run(3, w.patch_size, w.dx, initial_fp64(w.Q0, 1), 8, halo_mode=inputs.PERIODIC)
    e_f = batch_rel_linf(fused[0], ref, 3, w.patch_size)
    e_t = batch_rel_linf(tile[0], ref, 3, w.patch_size)
    print("periodic 8^3 FP32 after 8 steps: warp kernel %.2e, tile form %.2e" % (e_f, e_t))
    assert e_f < 1e-5 and e_t < 1e-5
    assert batch_rel_linf(fused[0], tile[0], 3, w.patch_size) < 1e-5


@pytest.mark.parametrize("p,halo,kernel", [(8, inputs.PERIODIC, "sweep3d_p8"), (16, inputs.FIXED, "sweep3d_b8")])
def test_bounded_copy_wait_reports_timeout_and_context_survives(p, halo, kernel):
    """A plane wait that can never complete (the test hook makes it expect 16
    bytes more than its copy delivers) gives up after its 1 s bound: the
    update reports FV_ETIMEOUT, nothing faults, and the next normal update
    on the same context matches the oracle.  Both kernels that fetch planes
    by bulk copies: the one-warp periodic 8^3 kernel and the 8x8-block
    kernel (16^3, fixed halos)."""
    import time
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    T = 6
    w = inputs.uniform_batch(3, [p] * T, seed=99, halo_mode=halo, dtype=np.float32)
    b = fb.FVBatch(3, w.patch_size, precision=1, halo_mode=halo)
    assert kernel in b.describe()
    qa = to_device(w.Q0, 1)
    qb = torch.zeros_like(qa)
    dx = torch.tensor(w.dx, device="cuda")
    dt = torch.full((T,), 1e-3, dtype=torch.float64, device="cuda")
    lam = torch.zeros(T, dtype=torch.float64, device="cuda")
    b.test_wait_expiry(True)
    t0 = time.perf_counter()
    b.update(qa, qb, dx, dt, lam, None, 0.4)
    with pytest.raises(fb.FVError) as ei:
        b.status()
    elapsed = time.perf_counter() - t0
    assert ei.value.code == fb.FV_ETIMEOUT
    assert 0.9 < elapsed < 20.0
    b.test_wait_expiry(False)
    b.update(qa, qb, dx, dt, lam, None, 0.4)
    b.status()
    ref, lam_ref = oracle.batch_step(3, w.patch_size, w.dx, [1e-3] * T, initial_fp64(w.Q0, 1), halo_mode=halo)
    assert batch_rel_linf(qb.to(torch.float64).cpu().numpy(), ref, 3, w.patch_size) < 1e-5
    b.close()


def _one_update(w, precision, form, layout=0, dt=1e-3):
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    T = w.num_patches
    b = fb.FVBatch(w.dim, w.patch_size, precision=precision, halo_mode=w.halo_mode, form=form)
    b.set_cascade_layout(layout)
    qa = to_device(w.Q0, precision)
    qb = qa.clone()
    dx = torch.tensor(np.asarray(w.dx, dtype=np.float64), device="cuda")
    dtv = torch.full((T,), dt, dtype=torch.float64, device="cuda")
    lam = torch.zeros(T, dtype=torch.float64, device="cuda")
    dtn = torch.zeros_like(lam)
    b.update(qa, qb, dx, dtv, lam, dtn, 0.4)
    b.status()
    desc = b.describe()
    out = (qb.to(torch.float64).cpu().numpy(), lam.cpu().numpy(), dtn.cpu().numpy(), desc)
    b.close()
    return out


@pytest.mark.parametrize("dim,sizes,halo", [(2, [3, 16, 5, 8, 1, 32, 7] * 3, inputs.FIXED),
                                            (2, [16] * 40, inputs.PERIODIC),
                                            (3, [4, 8, 3, 6] * 3, inputs.FIXED),
                                            (3, [8] * 9, inputs.PERIODIC)])
@pytest.mark.parametrize("precision", [0, 1])
def test_cascade_temporaries_layout_does_not_change_bits(dim, sizes, halo, precision):
    """AoS, SoA and AoSoA temporaries (the paper's App. C ablation) store the
    same values in different places: the update is bitwise identical."""
    w = inputs.uniform_batch(dim, sizes, seed=101 + dim, dx=0.05, halo_mode=halo)
    ref = _one_update(w, precision, FORMS["cascade"], 0)
    for layout in (1, 2):
        got = _one_update(w, precision, FORMS["cascade"], layout)
        assert ("cascade_layout=%s" % ("soa" if layout == 1 else "aosoa")) in got[3]
        for a, b in zip(got[:3], ref[:3]):
            assert np.array_equal(a, b)
    # and it is the right update
    q0 = initial_fp64(w.Q0, precision)
    oref, lref = oracle.batch_step(dim, w.patch_size, w.dx, [1e-3] * w.num_patches, q0, halo_mode=halo)
    assert batch_rel_linf(ref[0], oref, dim, w.patch_size) < TOL[precision]


@pytest.mark.parametrize("dim,sizes,halo", [(2, [3, 16, 5, 8, 1, 32, 7] * 2, inputs.FIXED),
                                            (2, [8] * 30, inputs.PERIODIC),
                                            (3, [4, 8, 3, 6, 5], inputs.FIXED),
                                            (3, [6] * 7, inputs.PERIODIC)])
@pytest.mark.parametrize("precision,layout", [(0, 0), (1, 0), (0, 1), (1, 2)])
def test_taskgraph_form_is_bitwise_the_batched_cascade(dim, sizes, halo, precision, layout):
    """The task-graph realisation runs the batched kernels restricted to one
    patch (and axis) per node, so its state, eigenvalues and time steps are
    bitwise those of the batched realisation."""
    w = inputs.uniform_batch(dim, sizes, seed=111 + dim, dx=0.05, halo_mode=halo)
    ref = _one_update(w, precision, FORMS["cascade"], layout)
    got = _one_update(w, precision, 3, layout)
    assert "form=taskgraph" in got[3]
    for a, b in zip(got[:3], ref[:3]):
        assert np.array_equal(a, b)
    # and it is the oracle's step (dt = 1e-3 for every patch)
    oref, olam = oracle.batch_step(dim, w.patch_size, w.dx, [1e-3] * w.num_patches, initial_fp64(w.Q0, precision),
                                   halo_mode=halo)
    assert batch_rel_linf(got[0], oref, dim, w.patch_size) <= TOL[precision]
    assert np.max(np.abs(got[1] - olam) / olam) <= TOL[precision]


def test_taskgraph_form_multi_step_run_equals_cascade():
    """fv_batch_run with the task-graph form (one graph launch per step; a
    requested outer graph is not captured) chains CFL steps like the cascade."""
    w = inputs.uniform_batch(2, [8, 16, 4] * 10, seed=121, dx=0.02)
    a = gpu_run(w, 0, FORMS["cascade"], 5)
    b = gpu_run(w, 0, 3, 5, use_graph=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    ref, lam_ref, dt_ref = _oracle(w, 0, 5)
    assert batch_rel_linf(b[0], ref, 2, w.patch_size) <= TOL[0]
    assert np.max(np.abs(b[1] - lam_ref) / lam_ref) <= TOL[0] and np.max(np.abs(b[2] - dt_ref) / dt_ref) <= TOL[0]


# ------------------------------------------------- generic PDE (Eq. 1): shallow water

SWE_G, SWE_F = 9.81, 0.6


def _swe_batch(w, precision, form=None):
    from paper_2306_16731_gb300 import fvbatch as fb
    return fb.FVBatch(2, w.patch_size, precision=precision, halo_mode=w.halo_mode, form=form,
                      pde=fb.FV_PDE_SHALLOW_WATER, params=[SWE_G, SWE_F])


@pytest.mark.parametrize("halo", [inputs.FIXED, inputs.PERIODIC])
@pytest.mark.parametrize("precision", [0, 1])
def test_shallow_water_step_matches_oracle(halo, precision):
    """One step of the generic-PDE kernel (Rusanov flux, averaged
    non-conservative product, Coriolis source) against the oracle, with the
    eigenvalues and CFL time steps of the new state."""
    import torch
    w = inputs.shallow_water_batch([3, 8, 16, 5, 32, 1, 12] * 3, seed=131 + halo, dx=np.linspace(0.02, 0.1, 21),
                                   halo_mode=halo)
    T = w.num_patches
    b = _swe_batch(w, precision)
    assert "pde=shallow_water" in b.describe() and "form=tile" in b.describe()
    q0 = initial_fp64(w.Q0, precision)
    lam0 = oracle.swe_batch_max_eigenvalue(w.patch_size, q0, SWE_G)
    dt = 0.4 * w.dx / (2 * lam0)
    qa = to_device(w.Q0, precision)
    qb = qa.clone()
    dx = torch.tensor(w.dx, device="cuda")
    dtv = torch.tensor(dt, device="cuda")
    lam = torch.zeros(T, dtype=torch.float64, device="cuda")
    dtn = torch.zeros_like(lam)
    lg = torch.zeros_like(lam)
    b.max_eigenvalue(qa, lg)
    b.update(qa, qb, dx, dtv, lam, dtn, 0.4)
    b.status()
    ref, lref = oracle.swe_batch_step(w.patch_size, w.dx, dt, q0, SWE_G, SWE_F, halo)
    got = qb.to(torch.float64).cpu().numpy()
    tol = 1e-12 if precision == 0 else 1e-5
    assert batch_rel_linf(got, ref, 2, w.patch_size) < tol
    assert np.max(np.abs(lg.cpu().numpy() - lam0) / lam0) < tol
    assert np.max(np.abs(lam.cpu().numpy() - lref) / lref) < tol
    assert np.allclose(dtn.cpu().numpy(), 0.4 * w.dx / (2 * lam.cpu().numpy()), rtol=1e-15, atol=0)
    # the bathymetry is a parameter: copied bitwise
    for g_, q_ in zip(patches_interior(got, 2, w.patch_size), patches_interior(q0, 2, w.patch_size)):
        assert np.array_equal(g_[..., 3], q_[..., 3])
    b.close()


def test_shallow_water_cfl_chained_run_and_graph_replay():
    """Ten CFL-chained steps on the GPU (eager and as one CUDA graph, bitwise
    equal) against the oracle chained the same way."""
    w = inputs.shallow_water_batch([16] * 30 + [7] * 11, seed=141, dx=0.05)
    steps = 10
    from paper_2306_16731_gb300 import fvbatch as fb
    res = []
    for use_graph in (False, True):
        import torch
        b = _swe_batch(w, 0)
        qa = to_device(w.Q0, 0)
        qb = qa.clone()
        dx = torch.tensor(w.dx, device="cuda")
        lam = torch.zeros(w.num_patches, dtype=torch.float64, device="cuda")
        dta, dtb = torch.zeros_like(lam), torch.zeros_like(lam)
        b.max_eigenvalue(qa, lam)
        b.cfl_time_step(lam, dx, 0.4, dta)
        b.run(qa, qb, dx, dta, dtb, lam, steps, 0.4, use_graph)
        b.status()
        res.append(((qb if steps % 2 else qa).cpu().numpy(), lam.cpu().numpy()))
        b.close()
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    q = w.Q0.astype(np.float64)
    lamo = oracle.swe_batch_max_eigenvalue(w.patch_size, q, SWE_G)
    for _ in range(steps):
        dt = 0.4 * w.dx / (2 * lamo)
        q, lamo = oracle.swe_batch_step(w.patch_size, w.dx, dt, q, SWE_G, SWE_F, w.halo_mode)
    assert batch_rel_linf(res[0][0], q, 2, w.patch_size) < 1e-12


@pytest.mark.parametrize("form", ["fused", "tile"])
def test_shallow_water_lake_at_rest_keeps_zero_momentum_on_gpu(form):
    import torch
    w = inputs.shallow_water_batch([16] * 8, seed=151, dx=0.1, depth_noise=0.0, speed=0.0, bottom=0.5)
    b = _swe_batch(w, 0, FORMS[form])
    assert ("form=%s" % form) in b.describe()
    qa = to_device(w.Q0, 0)
    qb = qa.clone()
    dx = torch.tensor(w.dx, device="cuda")
    dt = torch.full((8,), 0.004, dtype=torch.float64, device="cuda")
    b.update(qa, qb, dx, dt, None, None, 0.4)
    b.status()
    got = qb.cpu().numpy().reshape(-1, 4)
    scale = 0.004 / 0.1 * 0.5 * SWE_G * np.max(w.Q0.reshape(-1, 4)[:, 0]) ** 2
    assert np.max(np.abs(got[:, 1:3])) <= 1e-13 * scale
    b.close()


def test_shallow_water_rejects_what_it_does_not_cover():
    from paper_2306_16731_gb300 import fvbatch as fb
    with pytest.raises(fb.FVError) as e:
        fb.FVBatch(3, [4], pde=fb.FV_PDE_SHALLOW_WATER, params=[9.81, 0.0])
    assert e.value.code == fb.FV_EINVAL
    with pytest.raises(fb.FVError) as e:
        fb.FVBatch(2, [4], precision=fb.FV_BF16_F32, pde=fb.FV_PDE_SHALLOW_WATER, params=[9.81, 0.0])
    assert e.value.code == fb.FV_EUNSUPPORTED
    with pytest.raises(fb.FVError) as e:
        fb.FVBatch(2, [4], pde=fb.FV_PDE_SHALLOW_WATER, params=[-1.0, 0.0])
    assert e.value.code == fb.FV_EINVAL
    b = fb.FVBatch(2, [4, 12], pde=fb.FV_PDE_SHALLOW_WATER, params=[9.81, 0.0])
    assert "form=tile" in b.describe()                    # edge 12: no fused sweep
    for form in (fb.FV_FORM_FUSED, fb.FV_FORM_CASCADE, fb.FV_FORM_TASKGRAPH):
        with pytest.raises(fb.FVError) as e:
            b.set_form(form)
        assert e.value.code == fb.FV_EUNSUPPORTED
    b.close()
    b = fb.FVBatch(2, [4, 8], pde=fb.FV_PDE_SHALLOW_WATER, params=[9.81, 0.0])
    assert "form=fused" in b.describe() and "fused_kernel=sweep_pde" in b.describe()
    for form in (fb.FV_FORM_CASCADE, fb.FV_FORM_TASKGRAPH):
        with pytest.raises(fb.FVError) as e:
            b.set_form(form)
        assert e.value.code == fb.FV_EUNSUPPORTED
    b.set_form(fb.FV_FORM_TILE)
    b.set_form(fb.FV_FORM_FUSED)
    b.close()


def _swe_one_step(b, w, precision, dt):
    import torch
    T = w.num_patches
    qa = to_device(w.Q0, precision)
    qb = qa.clone()
    lam = torch.zeros(T, dtype=torch.float64, device="cuda")
    dtn = torch.zeros_like(lam)
    b.update(qa, qb, torch.tensor(w.dx, device="cuda"), torch.tensor(dt, device="cuda"), lam, dtn, 0.4)
    b.status()
    return qb.to(torch.float64).cpu().numpy(), lam.cpu().numpy(), dtn.cpu().numpy()


@pytest.mark.parametrize("halo", [inputs.FIXED, inputs.PERIODIC])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("sizes", [[4, 8, 16, 32] * 5, [16] * 67])
def test_shallow_water_fused_sweep_matches_oracle(halo, precision, sizes):
    """The fused row sweep of the generic PDE (edges 4, 8, 16, 32): one step
    against the oracle -- Rusanov flux, averaged non-conservative product,
    Coriolis source -- with the eigenvalues and CFL steps of the new state and
    the bathymetry copied bitwise; and within the same tolerance of the
    patch-wise form on the same batch."""
    w = inputs.shallow_water_batch(sizes, seed=171 + halo + len(sizes), dx=np.linspace(0.02, 0.1, len(sizes)),
                                   halo_mode=halo)
    b = _swe_batch(w, precision)
    assert "form=fused" in b.describe() and "fused_kernel=sweep_pde" in b.describe()
    q0 = initial_fp64(w.Q0, precision)
    lam0 = oracle.swe_batch_max_eigenvalue(w.patch_size, q0, SWE_G)
    dt = 0.4 * w.dx / (2 * lam0)
    got, lam, dtn = _swe_one_step(b, w, precision, dt)
    ref, lref = oracle.swe_batch_step(w.patch_size, w.dx, dt, q0, SWE_G, SWE_F, halo)
    tol = 1e-12 if precision == 0 else 1e-5
    assert batch_rel_linf(got, ref, 2, w.patch_size) < tol
    assert np.max(np.abs(lam - lref) / lref) < tol
    assert np.allclose(dtn, 0.4 * w.dx / (2 * lam), rtol=1e-15, atol=0)
    for g_, q_ in zip(patches_interior(got, 2, w.patch_size), patches_interior(q0, 2, w.patch_size)):
        assert np.array_equal(g_[..., 3], q_[..., 3])
    b.set_form(FORMS["tile"])                             # the patch-wise form on the same batch
    tile, _, _ = _swe_one_step(b, w, precision, dt)
    assert batch_rel_linf(got, tile, 2, w.patch_size) < tol
    b.close()


def test_shallow_water_fused_sweep_chained_graph_and_launch_shapes():
    """Ten CFL-chained fused steps: eager and as one CUDA graph bitwise equal,
    every launch shape bitwise equal, and the oracle chained the same way
    within FP64 tolerance."""
    import torch
    w = inputs.shallow_water_batch([16] * 40 + [8] * 21 + [32] * 5, seed=181, dx=0.05)
    steps = 10
    res = []
    for shape, use_graph in (((4, 0), False), ((4, 0), True), ((2, -1), False), ((8, 1), True), ((1, 0), False)):
        b = _swe_batch(w, 0)
        b.set_launch_shape(*shape)
        qa = to_device(w.Q0, 0)
        qb = qa.clone()
        dx = torch.tensor(w.dx, device="cuda")
        lam = torch.zeros(w.num_patches, dtype=torch.float64, device="cuda")
        dta, dtb = torch.zeros_like(lam), torch.zeros_like(lam)
        b.max_eigenvalue(qa, lam)
        b.cfl_time_step(lam, dx, 0.4, dta)
        b.run(qa, qb, dx, dta, dtb, lam, steps, 0.4, use_graph)
        b.status()
        res.append(((qb if steps % 2 else qa).cpu().numpy(), lam.cpu().numpy()))
        b.close()
    for r in res[1:]:
        assert np.array_equal(r[0], res[0][0]) and np.array_equal(r[1], res[0][1])
    q = w.Q0.astype(np.float64)
    lamo = oracle.swe_batch_max_eigenvalue(w.patch_size, q, SWE_G)
    for _ in range(steps):
        dt = 0.4 * w.dx / (2 * lamo)
        q, lamo = oracle.swe_batch_step(w.patch_size, w.dx, dt, q, SWE_G, SWE_F, w.halo_mode)
    assert batch_rel_linf(res[0][0], q, 2, w.patch_size) < 1e-12


# ------------------------------------------------- patches as separate host allocations

def _host_patches(w, precision, fill=None):
    """One page-locked allocation per patch (the input state, or a sentinel)."""
    import torch
    dt = torch_dtype(precision)
    off = w.offsets()
    out = []
    for i in range(w.num_patches):
        n = int(off[i + 1] - off[i])
        t = torch.empty(n, dtype=dt, pin_memory=True)
        if fill is None:
            t.copy_(torch.from_numpy(np.asarray(w.Q0[off[i]:off[i + 1]], dtype=np.float64)).to(dt))
        else:
            t.fill_(fill)
        out.append(t)
    return out


@pytest.mark.parametrize("dim,sizes,precision,halo", [(2, [16] * 60 + [8] * 20 + [5, 3, 32], 1, inputs.FIXED),
                                                      (2, [16] * 40, 0, inputs.PERIODIC),
                                                      (3, [8] * 30, 1, inputs.PERIODIC),
                                                      (3, [6, 4, 8, 5] * 4, 0, inputs.FIXED)])
@pytest.mark.parametrize("flags", [0, 2])
def test_scattered_host_patches_match_the_device_update(dim, sizes, precision, halo, flags):
    """Patches held as separate page-locked host allocations, gathered by a
    kernel (flags 0) or copied one by one (flags 2), updated and their
    interiors written back: bitwise the device update of the same batch, two
    ping-pong steps; output halos are not written."""
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    w = inputs.uniform_batch(dim, sizes, seed=161 + dim, dx=0.04, halo_mode=halo)
    T = w.num_patches
    ins = _host_patches(w, precision)
    outs = _host_patches(w, precision, fill=-7.0)
    b = fb.FVBatch(dim, w.patch_size, precision=precision, halo_mode=halo)
    b.set_host_patches(ins, outs)
    dx = torch.tensor(w.dx).pin_memory()
    dt = torch.full((T,), 1e-3, dtype=torch.float64).pin_memory()
    lam = torch.zeros(T, dtype=torch.float64).pin_memory()
    dtn = torch.zeros_like(lam).pin_memory()
    b.update_scattered(dx, dt, lam, dtn, 0.4, flags)
    # reference: the device update of the contiguous batch
    qa = to_device(w.Q0, precision)
    qb = qa.clone()
    ddx, ddt = dx.cuda(), dt.cuda()
    rl, rn = torch.zeros(T, dtype=torch.float64, device="cuda"), torch.zeros(T, dtype=torch.float64, device="cuda")
    b.update(qa, qb, ddx, ddt, rl, rn, 0.4)
    b.status()
    ref = qb.to(torch.float64).cpu().numpy()
    got = np.concatenate([t.to(torch.float64).numpy() for t in outs])
    gi, ri = patches_interior(got, dim, w.patch_size), patches_interior(ref, dim, w.patch_size)
    for g_, r_ in zip(gi, ri):
        assert np.array_equal(g_, r_)
    # the gathered update is the oracle's step
    q0 = initial_fp64(w.Q0, precision)
    o1, ol1 = oracle.batch_step(dim, w.patch_size, w.dx, [1e-3] * T, q0, halo_mode=halo)
    assert batch_rel_linf(got, o1, dim, w.patch_size) <= TOL[precision]
    assert np.max(np.abs(lam.numpy() - ol1) / ol1) <= TOL[precision]
    assert np.array_equal(lam.numpy(), rl.cpu().numpy()) and np.array_equal(dtn.numpy(), rn.cpu().numpy())
    # halo volumes of the output patches keep the sentinel
    for t, p in zip(outs, w.patch_size):
        shape = (int(p) + 2,) * dim + (dim + 2,)
        a = t.to(torch.float64).numpy().reshape(shape)
        mask = np.ones(shape[:-1], bool)
        mask[(slice(1, -1),) * dim] = False
        assert np.all(a[mask] == -7.0)
    # second step the other way round (outputs read, inputs written); fixed
    # halos are held in both ping-pong buffers, so the output patches get the
    # input patches' halo volumes first
    for t_in, t_out, p in zip(ins, outs, w.patch_size):
        shape = (int(p) + 2,) * dim + (dim + 2,)
        mask = np.ones(shape[:-1], bool)
        mask[(slice(1, -1),) * dim] = False
        t_out.numpy().reshape(shape)[mask] = t_in.numpy().reshape(shape)[mask]
    b.update_scattered(dx, dt, lam, dtn, 0.4, flags | fb.FV_SCATTER_SWAP)
    qa2 = qa.clone()
    b.update(qb, qa2, ddx, ddt, rl, rn, 0.4)
    b.status()
    got2 = np.concatenate([t.to(torch.float64).numpy() for t in ins])
    for g_, r_ in zip(patches_interior(got2, dim, w.patch_size),
                      patches_interior(qa2.to(torch.float64).cpu().numpy(), dim, w.patch_size)):
        assert np.array_equal(g_, r_)
    # second step against the oracle's second step (fixed halos as given)
    o2, _ = oracle.batch_step(dim, w.patch_size, w.dx, [1e-3] * T, o1, halo_mode=halo)
    assert batch_rel_linf(got2, o2, dim, w.patch_size) <= 2 * TOL[precision]
    b.set_host_patches(None, None)
    b.close()


def test_scattered_registration_rejects_pageable_memory():
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    w = inputs.uniform_batch(2, [4, 4], seed=171)
    b = fb.FVBatch(2, w.patch_size)
    pageable = [np.zeros(144), np.zeros(144)]
    pinned = _host_patches(w, 0)
    with pytest.raises(fb.FVError) as e:
        b.set_host_patches([a.ctypes.data for a in pageable], pinned)
    assert e.value.code == fb.FV_EINVAL
    with pytest.raises(fb.FVError) as e:
        b.set_host_patches(pinned, pinned)             # aliasing
    assert e.value.code == fb.FV_EINVAL
    dx = torch.full((2,), 0.1, dtype=torch.float64).pin_memory()
    with pytest.raises(fb.FVError) as e:
        b.update_scattered(dx, dx)                      # nothing registered
    assert e.value.code == fb.FV_EINVAL
    b.close()


def test_new_entry_points_handle_empty_batches_and_bad_arguments():
    """Empty batches go through the task-graph form, the scattered host
    patches and the generic PDE without work; invalid layouts, flags and
    forms are refused."""
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    b = fb.FVBatch(2, [], form=3)
    b.set_cascade_layout(fb.FV_LAYOUT_SOA)
    b.update(z, torch.zeros_like(z), z, z, z, z, 0.4)
    b.set_host_patches([], [])
    hz = torch.zeros(1, dtype=torch.float64).pin_memory()
    b.update_scattered(hz, hz)
    b.status()
    with pytest.raises(fb.FVError) as e:
        b.set_cascade_layout(3)
    assert e.value.code == fb.FV_EINVAL
    b.close()
    s = fb.FVBatch(2, [], pde=fb.FV_PDE_SHALLOW_WATER, params=[9.81, 0.1])
    s.update(z, torch.zeros_like(z), z, z, z, z, 0.4)
    s.status()
    s.close()
    w = inputs.uniform_batch(2, [4, 4], seed=181)
    b = fb.FVBatch(2, w.patch_size)
    ins = _host_patches(w, 0)
    outs = _host_patches(w, 0, fill=0.0)
    b.set_host_patches(ins, outs)
    dx = torch.full((2,), 0.1, dtype=torch.float64).pin_memory()
    with pytest.raises(fb.FVError) as e:
        b.update_scattered(dx, dx, None, None, 0.4, 4)            # unknown flag
    assert e.value.code == fb.FV_EINVAL
    with pytest.raises(fb.FVError) as e:
        fb.FVBatch(2, [4], pde=7, params=[1.0])
    assert e.value.code == fb.FV_EINVAL
    b.close()


@pytest.mark.parametrize("chunks", [0, 3])
def test_shallow_water_host_state_update_matches_device_update(chunks):
    """The host-state update (pipelined copies, or kernels on the mapped host
    buffers) drives the generic-PDE kernel like the device update."""
    import torch
    w = inputs.shallow_water_batch([16] * 20 + [8] * 9, seed=191, dx=0.05)
    T = w.num_patches
    b = _swe_batch(w, 1)
    hin = torch.from_numpy(w.Q0.astype(np.float32)).pin_memory()
    hout = torch.zeros_like(hin).pin_memory()
    dx = torch.tensor(w.dx).pin_memory()
    dt = torch.full((T,), 2e-3, dtype=torch.float64).pin_memory()
    lam = torch.zeros(T, dtype=torch.float64).pin_memory()
    dtn = torch.zeros_like(lam).pin_memory()
    b.update_host(hin, hout, dx, dt, lam, dtn, 0.4, chunks)
    qa = hin.cuda()
    qb = qa.clone()
    rl = torch.zeros(T, dtype=torch.float64, device="cuda")
    rn = torch.zeros_like(rl)
    b.update(qa, qb, dx.cuda(), dt.cuda(), rl, rn, 0.4)
    b.status()
    for g_, r_ in zip(patches_interior(hout.numpy(), 2, w.patch_size),
                      patches_interior(qb.cpu().numpy(), 2, w.patch_size)):
        assert np.array_equal(g_, r_)
    assert np.array_equal(lam.numpy(), rl.cpu().numpy()) and np.array_equal(dtn.numpy(), rn.cpu().numpy())
    b.close()


@pytest.mark.parametrize("halo", [inputs.FIXED, inputs.PERIODIC])
def test_shallow_water_host_time_stepping_equals_per_step_calls(halo):
    """fv_patch_batch_run_host drives the generic-PDE kernel (uniform batch:
    chunk chains over the fused shallow-water sweep) exactly like per-step
    host updates with the buffers alternated (fixed halos carried along,
    periodic ones rebuilt by the kernel every step)."""
    import torch
    S = 3
    w = inputs.shallow_water_batch([16] * 40, seed=193, dx=0.05, halo_mode=halo)
    T = w.num_patches
    b = _swe_batch(w, 1)
    pin = lambda t: t.clone().pin_memory()
    q0 = torch.from_numpy(w.Q0.astype(np.float32))
    dx = pin(torch.tensor(w.dx))
    dt0 = torch.full((T,), 2e-3, dtype=torch.float64)
    rq, rdt = [pin(q0), pin(q0)], [pin(dt0), pin(torch.zeros(T, dtype=torch.float64))]
    rl = pin(torch.zeros(T, dtype=torch.float64))
    for s_ in range(S):
        i = s_ & 1
        b.update_host(rq[i], rq[1 - i], dx, rdt[i], rl, rdt[1 - i], 0.4, 4)
    for chunks in (1, 4):
        hq, hdt = [pin(q0), pin(q0)], [pin(dt0), pin(torch.zeros(T, dtype=torch.float64))]
        hl = pin(torch.zeros(T, dtype=torch.float64))
        b.run_host(hq[0], hq[1], dx, hdt[0], hdt[1], hl, S, 0.4, chunks)
        got = patches_interior(hq[S & 1].numpy(), 2, w.patch_size)
        ref = patches_interior(rq[S & 1].numpy(), 2, w.patch_size)
        assert all(np.array_equal(g_, r_) for g_, r_ in zip(got, ref))
        if halo == inputs.FIXED:
            assert torch.equal(hq[S & 1], rq[S & 1])
        assert torch.equal(hdt[S & 1], rdt[S & 1]) and torch.equal(hl, rl)
    b.status()
    b.close()


def test_out_of_memory_paths_fail_cleanly_and_batches_stay_usable():
    """Device allocation failures (made on the host with the test hook) give
    FV_ENOMEM at every call that allocates; nothing half-made stays behind,
    so the same call succeeds once the hook is disarmed."""
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    w = inputs.uniform_batch(2, [8] * 12, seed=201, dx=0.05)
    T = w.num_patches
    try:
        fb.fv_test_fail_device_alloc(1)
        with pytest.raises(fb.FVError) as e:
            fb.FVBatch(2, w.patch_size)                       # metadata block
        assert e.value.code == fb.FV_ENOMEM
        fb.fv_test_fail_device_alloc(0)
        b = fb.FVBatch(2, w.patch_size)
        fb.fv_test_fail_device_alloc(1)
        with pytest.raises(fb.FVError) as e:
            b.set_form(fb.FV_FORM_CASCADE)                    # cascade scratch
        assert e.value.code == fb.FV_ENOMEM and "form=fused" in b.describe()
        nb = [[-1, -1, -1, -1]] * T
        fb.fv_test_fail_device_alloc(1)
        with pytest.raises(fb.FVError) as e:
            b.set_neighbours(nb)                              # neighbour table
        assert e.value.code == fb.FV_ENOMEM
        hin = torch.from_numpy(w.Q0).pin_memory()
        hout = torch.zeros_like(hin).pin_memory()
        dx = torch.tensor(w.dx).pin_memory()
        dt = torch.full((T,), 1e-3, dtype=torch.float64).pin_memory()
        for k in (1, 2, 3):                                   # each staging buffer in turn
            fb.fv_test_fail_device_alloc(k)
            with pytest.raises(fb.FVError) as e:
                b.update_host(hin, hout, dx, dt, None, None, 0.4, 2)
            assert e.value.code == fb.FV_ENOMEM
        ins = _host_patches(w, 0)
        outs = _host_patches(w, 0, fill=0.0)
        fb.fv_test_fail_device_alloc(1)
        with pytest.raises(fb.FVError) as e:
            b.set_host_patches(ins, outs)                     # patch address table
        assert e.value.code == fb.FV_ENOMEM
        qa = torch.from_numpy(w.Q0).cuda()
        scratch = qa.clone()
        ddx, ddt = dx.cuda(), dt.cuda()
        for k in (1, 2):                                      # tuner buffers
            fb.fv_test_fail_device_alloc(k)
            with pytest.raises(fb.FVError) as e:
                b.tune(qa, scratch, ddx, ddt)
            assert e.value.code == fb.FV_ENOMEM
        fb.fv_test_fail_device_alloc(0)
        # every call works now, and gives the right update
        b.set_form(fb.FV_FORM_CASCADE)
        b.set_neighbours(nb)
        b.set_neighbours(None)
        b.update_host(hin, hout, dx, dt, None, None, 0.4, 2)
        b.set_host_patches(ins, outs)
        b.set_form(fb.FV_FORM_FUSED)
        b.tune(qa, scratch, ddx, ddt)
        qb = qa.clone()
        b.update(qa, qb, ddx, ddt)
        b.status()
        ref, _ = oracle.batch_step(2, w.patch_size, w.dx, [1e-3] * T, w.Q0)
        assert batch_rel_linf(qb.cpu().numpy(), ref, 2, w.patch_size) < 1e-12
        assert batch_rel_linf(hout.numpy(), ref, 2, w.patch_size) < 1e-12
        b.close()
    finally:
        fb.fv_test_fail_device_alloc(0)


def test_double_destroy_is_refused():
    from paper_2306_16731_gb300 import fvbatch as fb
    h = fb.fv_batch_create(2, [4, 4])
    fb.fv_batch_destroy(h)
    with pytest.raises(fb.FVError) as e:
        fb.fv_batch_destroy(h)
    assert e.value.code == fb.FV_EINVAL


def test_non_finite_time_step_is_reported():
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    w = inputs.uniform_batch(2, [8, 8], seed=211)
    for form in FORMS.values():
        b = fb.FVBatch(2, w.patch_size, precision=0, form=form)
        q = torch.from_numpy(w.Q0).cuda()
        out = q.clone()
        dx = torch.full((2,), 0.1, dtype=torch.float64, device="cuda")
        dt = torch.tensor([float("nan"), 1e-4], dtype=torch.float64, device="cuda")
        lam = torch.zeros(2, dtype=torch.float64, device="cuda")
        b.update(q, out, dx, dt, lam)
        with pytest.raises(fb.FVError) as e:
            b.status()
        assert e.value.code == fb.FV_ENONPHYSICAL
        b.close()


def test_host_update_graph_replays_new_contents_and_falls_back_for_pageable_buffers():
    """The chunked host-state update is captured as a CUDA graph per set of
    host buffers and replayed: a replay must read the buffers' current
    contents (a chain of steps through the same two buffers, fixed halos put
    back between steps, equals the same chain of device updates), a change
    of launch shape drops the graph, and pageable buffers (not capturable)
    run the same pipeline eagerly."""
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    w = inputs.uniform_batch(2, [16] * 600, seed=141, dx=0.02)
    T = w.num_patches
    b = fb.FVBatch(2, w.patch_size, precision=fb.FV_F32)
    dx = torch.tensor(w.dx, device="cuda")
    dt = torch.full((T,), 1e-3, dtype=torch.float64, device="cuda")
    # device reference: three steps, ping-pong
    qs = [torch.from_numpy(w.Q0).to("cuda", torch.float32), None]
    qs[1] = qs[0].clone()
    lam = torch.zeros(T, dtype=torch.float64, device="cuda")
    for s in range(3):
        b.update(qs[s & 1], qs[1 - (s & 1)], dx, dt, lam, None, 0.4)
    torch.cuda.synchronize()
    ref = patches_interior(qs[1].to(torch.float64).cpu().numpy(), 2, w.patch_size)
    ref_lam = lam.cpu().numpy().copy()

    def host_chain(pin, shape_change=False):
        mk = (lambda t: t.pin_memory()) if pin else (lambda t: t)
        h = [mk(torch.from_numpy(w.Q0.astype(np.float32))), None]
        h[1] = mk(h[0].clone())
        hdx, hdt = mk(dx.cpu()), mk(dt.cpu())
        hl = mk(torch.zeros(T, dtype=torch.float64))
        q0 = w.Q0.astype(np.float32).reshape(T, 18, 18, 4)
        for s in range(3):
            if shape_change and s == 1:
                b.set_launch_shape(2, 0)
            b.update_host(h[s & 1], h[1 - (s & 1)], hdx, hdt, hl, None, 0.4, 4)
            # the halos of Q_out_host are unspecified: put the fixed halos
            # back before the buffer is the next step's input
            o = h[1 - (s & 1)].numpy().reshape(T, 18, 18, 4)
            o[:, [0, 17]] = q0[:, [0, 17]]
            o[:, :, [0, 17]] = q0[:, :, [0, 17]]
        return patches_interior(h[1].to(torch.float64).numpy(), 2, w.patch_size), hl.numpy()

    for pin, change in ((True, False), (True, True), (False, False)):
        got, gl = host_chain(pin, change)
        assert all(np.array_equal(g, r) for g, r in zip(got, ref)), (pin, change)
        assert np.array_equal(gl, ref_lam), (pin, change)
    b.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_uneven_2d_batch_runs_as_one_launch_when_edges_are_compiled(precision):
    """An uneven 2D batch whose edges are all 4, 8, 16 or 32 is updated by one
    launch over every size class (items dispatched on their edge); with a
    runtime edge among them it falls back to one launch per class.  Both
    match the oracle, fixed and periodic, and every launch shape gives the
    same bits."""
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    rng = np.random.default_rng(77)
    for sizes, launches in ((rng.choice([4, 8, 16, 32], 900), 1), (np.r_[rng.choice([4, 8, 16], 300), [5] * 7], 4)):
        for halo in (inputs.FIXED, inputs.PERIODIC):
            w = inputs.uniform_batch(2, sizes, seed=170 + halo, dx=np.linspace(0.05, 0.2, len(sizes)),
                                     halo_mode=halo, dtype=np.float32 if precision == 1 else np.float64)
            T = w.num_patches
            results = []
            for shape in ((4, 0), (2, -1), (8, 1)):
                b = fb.FVBatch(2, w.patch_size, precision=precision, halo_mode=halo)
                b.set_launch_shape(*shape)
                assert b.launches_per_update() == launches
                qa = to_device(w.Q0, precision)
                qb = qa.clone()
                dx = torch.tensor(w.dx, device="cuda")
                dt = torch.full((T,), 1e-3, dtype=torch.float64, device="cuda")
                lam = torch.zeros(T, dtype=torch.float64, device="cuda")
                b.update(qa, qb, dx, dt, lam, None, 0.4)
                b.status()
                results.append((qb.to(torch.float64).cpu().numpy(), lam.cpu().numpy()))
                b.close()
            for q, l in results[1:]:
                assert np.array_equal(q, results[0][0]) and np.array_equal(l, results[0][1])
            ref, lam_ref = oracle.batch_step(2, w.patch_size, w.dx, [1e-3] * T, initial_fp64(w.Q0, precision),
                                             halo_mode=halo)
            assert batch_rel_linf(results[0][0], ref, 2, w.patch_size) < TOL[precision]
            assert np.max(np.abs(results[0][1] - lam_ref) / lam_ref) < TOL[precision]
