"""GPU-side helpers for the parity tests: run the CUDA path through the C ABI
on a seeded workload, and run the FP64 oracle on the same inputs.

Inputs come from ``paper_2306_16731_gb300.inputs``; expected values come
only from ``oracle/``.  Nothing here computes a step of the method.
"""
from __future__ import annotations

import numpy as np

from paper_2306_16731_gb300 import inputs

PREC_NP = {0: np.float64, 1: np.float32}


def torch_dtype(precision):
    import torch
    return {0: torch.float64, 1: torch.float32, 2: torch.bfloat16}[precision]


def to_device(Q0, precision):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(Q0, dtype=np.float64))
    return t.to(device="cuda", dtype=torch_dtype(precision)).contiguous()


def initial_fp64(Q0, precision):
    """The state the GPU starts from, widened to FP64 (the oracle's start)."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(Q0, dtype=np.float64)).to(torch_dtype(precision))
    return t.to(torch.float64).numpy()


def gpu_run(w, precision, form, steps, use_graph=False, tune=False, Q0=None):
    """CFL-chained run of ``steps`` steps.  Returns (Q_final float64 numpy,
    lambda of the final state, dt_next, batch description)."""
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    Q0 = w.Q0 if Q0 is None else Q0
    T = w.num_patches
    b = fb.FVBatch(w.dim, w.patch_size, precision=precision, halo_mode=w.halo_mode,
                   gamma=w.gamma, form=form)
    try:
        qa = to_device(Q0, precision)
        qb = qa.clone()
        dx = torch.tensor(np.asarray(w.dx, dtype=np.float64), device="cuda")
        lam = torch.zeros(max(T, 1), dtype=torch.float64, device="cuda")
        dta = torch.zeros_like(lam)
        dtb = torch.zeros_like(lam)
        if tune:
            b.max_eigenvalue(qa, lam)
            b.cfl_time_step(lam, dx, w.cfl, dta)
            scratch = qa.clone()
            b.tune(qa, scratch, dx, dta)
            del scratch
        b.max_eigenvalue(qa, lam)
        b.cfl_time_step(lam, dx, w.cfl, dta)
        b.run(qa, qb, dx, dta, dtb, lam, steps, w.cfl, use_graph)
        b.status()
        torch.cuda.synchronize()
        final = qb if steps % 2 == 1 else qa
        dtn = dtb if steps % 2 == 1 else dta
        desc = b.describe()
        return (final.to(torch.float64).cpu().numpy(), lam[:T].cpu().numpy(),
                dtn[:T].cpu().numpy(), desc)
    finally:
        b.close()


def subset(w, idx):
    """Workload made of patches ``idx`` of ``w`` (exact for the oracle, since
    patches are independent)."""
    off = w.offsets()
    parts = [w.Q0[off[i]:off[i + 1]] for i in idx]
    return inputs.Workload(name=w.name + "_subset", dim=w.dim,
                           patch_size=w.patch_size[idx].copy(), dx=w.dx[idx].copy(),
                           halo_mode=w.halo_mode, steps=w.steps,
                           Q0=np.concatenate(parts) if parts else w.Q0[:0].copy(),
                           gamma=w.gamma, cfl=w.cfl, seed=w.seed)


def take_patches(w, flat, idx):
    off = w.offsets()
    return np.concatenate([flat[off[i]:off[i + 1]] for i in idx])
