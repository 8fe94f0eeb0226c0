#!/usr/bin/env python
"""Benchmark of the batched finite-volume patch update on GB300.

Workload (default): 16,384 two-dimensional patches of 16 x 16 volumes with a
one-volume fixed halo, compressible Euler (4 unknowns, gamma 1.4), Rusanov
flux, explicit Euler step with per-patch CFL 0.4 time steps, dx = 0.01,
seeded uniform primitives (rho, p in [0.5, 1.5], u, v in [-0.5, 0.5]).

One benchmark "step" is one time step of the whole batch: one call of
``fv_patch_batch_update`` (stage, directional fluxes and eigenvalues, Rusanov
face fluxes, update, per-patch eigenvalue maximum and next CFL time step).
The headline value is the fused FP32 form; the FP64 fused and the plain FP64
loop-cascade forms are timed beside it.  L2 is flushed (256 MiB write, then a
256 MiB read) before every timed step and each step is timed alone with CUDA
events on the launching stream.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead (the reference arm of this project).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "volume updates/s per GB300, fused FP32 vs plain FP64 at stated error; % roofline"
UNIT = "volume updates/s"
WORKLOAD = "2D Euler, 16384 patches of 16x16 + 1-cell fixed halo, dx=0.01, CFL 0.4, seeded uniform primitives"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="skip the secondary 3D / uneven workload lines")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--profile", choices=["fused_f32", "fused_f64", "cascade_f64", "tile_f32",
                                          "fused3d_f32", "fused3d16_f32", "fused3dper_f32", "uneven_f32",
                                          "swe_f32", "swetile_f32"],
                    default=None, help="no timing: run a few launches of one form for ncu")
    ap.add_argument("--patches", type=int, default=None,
                    help="with --profile: batch size (default 65536, state larger than L2)")
    return ap.parse_args()


def bench_config(T, p, N):
    """The workload both arms run (the reference arm times the FP64 oracle
    on it): same keys and values on both lines."""
    return {"workload": WORKLOAD, "dim": 2, "patches_per_gpu": T, "p": p, "unknowns": N,
            "steps_per_timed_step": 1, "parallelism": "replicas (patches independent; no collective)"}


def algorithmic_bytes_per_volume(dim, p, N, s, periodic=False):
    """Read every needed volume once (interior plus the 2d face-halo layers;
    periodic halos are rebuilt from the interior), write the interior once."""
    reads = p ** dim + (0 if periodic else 2 * dim * p ** (dim - 1))
    return N * s * (reads + p ** dim) / p ** dim


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during timing."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        busy = [c for c, p in zip(sm, power) if p > 200.0] or sm
        return {"sm_mhz": float(np.median(busy)) if busy else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ------------------------------------------------------------ CPU oracle

def _oracle_sample(w, idx):
    off = w.offsets()
    return np.concatenate([np.asarray(w.Q0[off[i]:off[i + 1]], dtype=np.float64) for i in idx])


def cpu_baseline(w, seconds, sample_patches=1024, steps=1, threads=0):
    import oracle
    oracle.build()
    oracle.set_num_threads(threads)
    rng = np.random.default_rng(12345)
    idx = np.sort(rng.choice(w.num_patches, min(sample_patches, w.num_patches), replace=False))
    Q = _oracle_sample(w, idx)
    psz, dx = w.patch_size[idx], w.dx[idx]
    vols = int(np.sum(psz.astype(np.int64) ** w.dim))
    lam = oracle.batch_max_eigenvalue(w.dim, psz, Q)
    dt = oracle.cfl_time_step(w.dim, lam, dx, w.cfl)
    runs, t0 = 0, time.perf_counter()
    while True:
        for _ in range(steps):
            oracle.batch_step(w.dim, psz, dx, dt, Q, w.gamma, w.halo_mode)
        runs += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    value = vols * steps * runs / el
    desc = ("%d seeded patches of the workload x %d step(s), repeated %d times (%.1f s)"
            % (len(idx), steps, runs, el))
    cores = oracle.num_threads()
    oracle.set_num_threads(0)
    return value, cores, desc


def oracle_error(w, Q0_f32, gpu_final, steps, idx):
    """rel L-inf of the GPU result on patches idx vs the FP64 oracle run from
    the same (FP32-rounded) start, with its own CFL chain."""
    import oracle
    start = _oracle_sample(w, idx).astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    ref, _, _ = oracle.batch_run(w.dim, w.patch_size[idx], w.dx[idx], start, steps,
                                 w.gamma, w.halo_mode, w.cfl)
    el = time.perf_counter() - t0
    off = w.offsets()
    got = np.concatenate([gpu_final[off[i]:off[i + 1]] for i in idx])
    N = w.dim + 2
    errs = []
    o2 = np.concatenate([[0], np.cumsum((N) * (w.patch_size[idx].astype(np.int64) + 2) ** w.dim)])
    A, B = [], []
    for j, i in enumerate(idx):
        p = int(w.patch_size[i])
        sh = (p + 2,) * w.dim + (N,)
        A.append(got[o2[j]:o2[j + 1]].reshape(sh)[(slice(1, -1),) * w.dim].reshape(-1, N))
        B.append(ref[o2[j]:o2[j + 1]].reshape(sh)[(slice(1, -1),) * w.dim].reshape(-1, N))
    A, B = np.concatenate(A), np.concatenate(B)
    for k in range(N):
        errs.append(float(np.max(np.abs(A[:, k] - B[:, k])) / np.max(np.abs(B[:, k]))))
    return float(np.max(np.abs(A - B)) / np.max(np.abs(B))), errs, el


def oracle_error_sample(w, precision, got_patches, steps, idx):
    """rel L-inf (state-normalised, and per unknown) of GPU final patches idx
    against the FP64 oracle run for the same steps from the same start
    (rounded to the GPU's storage type), each side with its own CFL chain."""
    import oracle
    import torch
    dt = {0: torch.float64, 1: torch.float32, 2: torch.bfloat16}[precision]
    start = torch.from_numpy(_oracle_sample(w, idx)).to(dt).to(torch.float64).numpy()
    ref, _, _ = oracle.batch_run(w.dim, w.patch_size[idx], w.dx[idx], start, steps, w.gamma, w.halo_mode, w.cfl)
    N = w.dim + 2
    o2 = np.concatenate([[0], np.cumsum(N * (w.patch_size[idx].astype(np.int64) + 2) ** w.dim)])
    A, B = [], []
    for j, i in enumerate(idx):
        p = int(w.patch_size[i])
        sh = (p + 2,) * w.dim + (N,)
        A.append(np.asarray(got_patches[j]).reshape(sh)[(slice(1, -1),) * w.dim].reshape(-1, N))
        B.append(ref[o2[j]:o2[j + 1]].reshape(sh)[(slice(1, -1),) * w.dim].reshape(-1, N))
    A, B = np.concatenate(A), np.concatenate(B)
    comps = [float(np.max(np.abs(A[:, k] - B[:, k])) / np.max(np.abs(B[:, k]))) for k in range(N)]
    return float(np.max(np.abs(A - B)) / np.max(np.abs(B))), comps


def error_statement(state, per_unknown, steps, patches, precision):
    """Error against the FP64 oracle in both norms, with the bound each is
    held to.  FP32: 1e-5 (the target).  BF16 storage: steps * 2^-8 of the
    state's magnitude (each step rounds every stored value to 8 significant
    bits; the step does not amplify errors in the maximum norm), stated for
    the state-normalised norm only."""
    if precision == 1:
        bound = 1e-5
    elif precision == 2:
        bound = steps * 2.0 ** -8
    else:
        bound = 1e-12
    worst = max(per_unknown)
    out = {"rel_linf": state, "rel_linf_per_unknown": per_unknown, "rel_linf_per_unknown_max": worst,
           "bound": bound, "meets_bound_state_normalised": bool(state <= bound),
           "meets_bound_per_unknown": bool(worst <= bound) if precision != 2 else None,
           "steps": steps, "patches_sampled": patches,
           "precision": {0: "f64", 1: "f32", 2: "bf16 storage, f32 arithmetic"}[precision],
           "norms": "rel_linf: max|Q - Q_oracle| / max|Q_oracle| over volumes and unknowns (state-normalised); "
                    "rel_linf_per_unknown[k]: max|Q_k - Q_oracle,k| / max|Q_oracle,k| (per unknown)"}
    if precision == 1 and worst > bound:
        out["per_unknown_miss"] = ("misses 1e-5 per unknown; a float32 restatement of the scheme run on the "
                                   "same patches misses it by the same order (near-zero unknowns divided by "
                                   "their own small maximum), so this is float32's floor, not the kernel's")
    return out


# ------------------------------------------------------------ traffic note

def committed_traffic(kernel_tag, source_files):
    """DRAM bytes per launch from a committed ncu summary, valid only while
    the kernel sources still hash to the value recorded beside it."""
    path = os.path.join(ROOT, "profiles", kernel_tag + ".md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    h = re.search(r"source_sha256:\s*([0-9a-f]+)", text)
    if not m or not h:
        return None
    sha = hashlib.sha256()
    for f in source_files:
        sha.update(open(os.path.join(ROOT, f), "rb").read())
    if sha.hexdigest()[:16] != h.group(1)[:16]:
        return None
    return float(m.group(1))


def kernel_source_files():
    c = "paper_2306_16731_gb300/csrc/"
    return [c + "fv_sweep.cu", c + "fv_physics.cuh", c + "fv_common.cuh"]


# ------------------------------------------------------------------ ours

def run_ours(args):
    import torch
    from paper_2306_16731_gb300 import build, fvbatch as fb, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    build.build()

    w = inputs.config(2, dtype=np.float32)
    N, T, p = w.dim + 2, w.num_patches, int(w.patch_size[0])
    vols = w.interior_volumes
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def make(precision, form):
        b = fb.FVBatch(w.dim, w.patch_size, precision=precision, halo_mode=w.halo_mode,
                       form=form, stream=stream.cuda_stream)
        dtype = {0: torch.float64, 1: torch.float32}[precision]
        qa = torch.from_numpy(w.Q0).to(device=dev, dtype=dtype)
        qb = qa.clone()
        dx = torch.tensor(w.dx, device=dev)
        lam = torch.zeros(T, dtype=torch.float64, device=dev)
        dta, dtb = torch.zeros_like(lam), torch.zeros_like(lam)
        b.max_eigenvalue(qa, lam)
        b.cfl_time_step(lam, dx, w.cfl, dta)
        return b, [qa, qb], dx, lam, [dta, dtb]

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    clean = torch.ones(64 << 20, dtype=torch.float32, device=dev)     # 256 MiB

    def flush_l2():
        """Write a buffer larger than L2, then read another one, so the step
        starts with none of its inputs in L2 and without the flush's dirty
        lines waiting to be written back during the step."""
        flush.zero_()
        clean.sum()

    def timed_steps(b, qs, dx, lam, dts, steps, warmup):
        # warm-up steps are the timed steps untimed, flush included, so that
        # one-time costs of the flush pattern (the first allocation of the
        # reduction's output) fall outside the timed region
        for s in range(warmup):
            i = s & 1
            flush_l2()
            b.update(qs[i], qs[1 - i], dx, dts[i], lam, dts[1 - i], w.cfl)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        barrier()
        torch.cuda.nvtx.range_push("timed_steps")     # lets a profiler select exactly these launches
        for s in range(steps):
            i = (warmup + s) & 1
            flush_l2()
            ev[s][0].record(stream)
            b.update(qs[i], qs[1 - i], dx, dts[i], lam, dts[1 - i], w.cfl)
            ev[s][1].record(stream)
        torch.cuda.nvtx.range_pop()
        barrier()
        return sum(a.elapsed_time(c) for a, c in ev)     # ms

    clocks = ClockSampler(_smi_id(torch, dev))
    clocks.start()

    # headline: fused FP32
    b32, qs32, dx, lam32, dts32 = make(fb.FV_F32, fb.FV_FORM_FUSED if _fused_ok(fb, w, fb.FV_F32) else fb.FV_FORM_TILE)
    scratch = qs32[0].clone()
    b32.tune(qs32[0], scratch, dx, dts32[0])
    del scratch
    ms = timed_steps(b32, qs32, dx, lam32, dts32, args.steps, args.warmup)
    desc32 = b32.describe()
    launches = b32.launches_per_update() * args.steps

    # slowest rank decides; every rank advanced its own replica batch
    from paper_2306_16731_gb300.multigpu import max_over_ranks, whole_job_rate
    ms_max = max_over_ranks(ms, dist, dev)
    value = whole_job_rate(vols * args.steps, ms_max / 1e3, dist, dev)

    # the FP64 forms beside it (fewer steps: FP64 is slow on this part)
    forms = {}
    k64 = max(5, min(20, args.steps // 10))
    for name, prec, form in (("fused_f64", fb.FV_F64, fb.FV_FORM_FUSED),
                             ("tile_f64", fb.FV_F64, fb.FV_FORM_TILE),
                             ("cascade_f64", fb.FV_F64, fb.FV_FORM_CASCADE),
                             ("tile_f32", fb.FV_F32, fb.FV_FORM_TILE),
                             ("cascade_f32", fb.FV_F32, fb.FV_FORM_CASCADE)):
        try:
            bb, qq, dxx, ll, dd = make(prec, form)
        except fb.FVError:
            continue
        m = timed_steps(bb, qq, dxx, ll, dd, k64, 3)
        forms[name] = {"value": vols * k64 / (m / 1e3), "ms_per_step": m / k64,
                       "launches_per_step": bb.launches_per_update(), "kernel": bb.describe()}
        bb.close()
        del qq
    forms["fused_f32"] = {"value": vols * args.steps / (ms / 1e3), "ms_per_step": ms / args.steps,
                          "launches_per_step": b32.launches_per_update(), "kernel": desc32}

    # 100-step graph-captured run from the initial state, L2-warm (for the
    # error statement and the multi-step throughput)
    qa = torch.from_numpy(w.Q0).to(device=dev, dtype=torch.float32)
    qb = qa.clone()
    b32.max_eigenvalue(qa, lam32)
    b32.cfl_time_step(lam32, dx, w.cfl, dts32[0])
    b32.run(qa, qb, dx, dts32[0], dts32[1], lam32, w.steps, w.cfl, True)   # capture + run
    qa2 = torch.from_numpy(w.Q0).to(device=dev, dtype=torch.float32)
    qa.copy_(qa2)
    qb.copy_(qa2)
    del qa2
    b32.max_eigenvalue(qa, lam32)
    b32.cfl_time_step(lam32, dx, w.cfl, dts32[0])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    b32.run(qa, qb, dx, dts32[0], dts32[1], lam32, w.steps, w.cfl, True)
    e1.record(stream)
    torch.cuda.synchronize()
    b32.status()
    graph_ms = e0.elapsed_time(e1)
    final = (qb if w.steps % 2 else qa).to(torch.float64).cpu().numpy()
    # median of 16 further replays of the same graph (the state keeps evolving)
    reps = []
    for r_ in range(16):
        e0.record(stream)
        b32.run(qa, qb, dx, dts32[0], dts32[1], lam32, w.steps, w.cfl, True)
        e1.record(stream)
        torch.cuda.synchronize()
        reps.append(e0.elapsed_time(e1))
    b32.status()
    med = float(np.median(reps))
    forms["fused_f32_graph_%dsteps_l2warm" % w.steps] = {
        "value": vols * w.steps / (graph_ms / 1e3), "ms_per_step": graph_ms / w.steps,
        "median_of_16_replays": {"value": vols * w.steps / (med / 1e3), "ms_per_step": med / w.steps}}

    # end to end through the public API with host buffers: the state lives in
    # pinned host memory and every step copies it in, updates it and copies
    # it back.  CFL-chained time stepping: the state and the time steps
    # ping-pong between two pinned host sets; every step copies the state
    # and dt in and the new state and next time steps out (dx once, the
    # final eigenvalues once), all inside the timed region.
    # fv_patch_batch_run_host runs the steps as per-chunk chains, so one
    # step's copies out overlap the next step's copies in.
    host_q = [torch.from_numpy(w.Q0.astype(np.float32)).pin_memory(), None]
    host_q[1] = host_q[0].clone().pin_memory()
    host_dx = torch.from_numpy(w.dx.copy()).pin_memory()
    host_lam = torch.empty(T, dtype=torch.float64).pin_memory()
    lam0 = torch.zeros(T, dtype=torch.float64, device=dev)
    dt0 = torch.zeros_like(lam0)
    b32.max_eigenvalue(host_q[0].to(dev), lam0)
    b32.cfl_time_step(lam0, dx, w.cfl, dt0)
    host_dts = [dt0.cpu().pin_memory(), torch.empty(T, dtype=torch.float64).pin_memory()]
    host_dt = host_dts[0]
    ke = max(20, min(50, args.steps)) // 2 * 2           # even: the state ends where it started
    chunks = 2                             # two chunk chains: 0.557 ms per step (4: 0.576, 8: 0.61-0.63)

    b32.run_host(host_q[0], host_q[1], host_dx, host_dts[0], host_dts[1], host_lam, 2, w.cfl, chunks)   # staging
    b32.status()
    barrier()
    t_e2e = time.perf_counter()
    ee0 = torch.cuda.Event(enable_timing=True)
    ee0.record(stream)
    b32.run_host(host_q[0], host_q[1], host_dx, host_dts[0], host_dts[1], host_lam, ke, w.cfl, chunks)
    ee1 = torch.cuda.Event(enable_timing=True)
    ee1.record(stream)
    barrier()
    e2e_ms = ee0.elapsed_time(ee1)
    e2e_wall = time.perf_counter() - t_e2e
    b32.status()                           # a non-physical state would show here
    state_bytes = host_q[0].numel() * 4
    e2e = {"value": whole_job_rate(vols * ke, e2e_wall, dist, dev), "unit": UNIT,
           "h2d_bytes_per_step": int(state_bytes + T * 8 + T * 8 / ke),
           "d2h_bytes_per_step": int(state_bytes + T * 8 + T * 8 / ke),
           "steps": ke, "wall_s": e2e_wall, "device_event_ms": e2e_ms,
           "link_bound_ms_per_step": 2 * state_bytes / 330e9 * 1e3,
           "call": "fv_patch_batch_run_host, %d steps in one call, %d chunk chains, CFL-chained dt" % (ke, chunks)}

    def host_steps(n, chunks_):
        for s_ in range(n):
            i_ = s_ & 1
            b32.update_host(host_q[i_], host_q[1 - i_], host_dx, host_dts[i_], host_lam, host_dts[1 - i_],
                            w.cfl, chunks_)

    # the same steps as one fv_patch_batch_update_host call each (a step's
    # copies in wait for the previous call's copies out), at that call's
    # best chunk count
    call_chunks = 4
    host_steps(4, call_chunks)             # captures the two ping-pong graphs
    barrier()
    t_c = time.perf_counter()
    host_steps(ke, call_chunks)
    barrier()
    e2e["per_step_calls_value"] = whole_job_rate(vols * ke, time.perf_counter() - t_c, dist, dev)
    e2e["per_step_calls_chunks"] = call_chunks
    b32.status()
    # the same call with chunks = 0: the kernels read and write the mapped
    # host buffers directly over the coherent CPU-GPU link, no staging
    host_steps(4, 0)
    barrier()
    t_d = time.perf_counter()
    host_steps(ke, 0)
    barrier()
    e2e["direct_mapped_value"] = whole_job_rate(vols * ke, time.perf_counter() - t_d, dist, dev)

    # patches as separate host objects (the paper's heap patches): one pinned
    # arena per side with the patches in shuffled order and random gaps;
    # gather/scatter kernels over the coherent link vs one copy per patch
    e2e["scattered_patches"] = scattered_e2e(b32, w, host_dx, host_dt, host_lam, dist, dev)

    if not args.no_other_workloads and world == 1:
        forms_other = other_workloads(dev, stream, flush_l2, args.steps)
        abl = ablations(dev, stream, flush_l2)
    else:
        forms_other = None
        abl = None
    clk = clocks.stop()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return None

    bpv = algorithmic_bytes_per_volume(w.dim, p, N, 4)
    avg_launch_s = (ms / args.steps) / 1e3
    achieved = vols * bpv / avg_launch_s / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    traffic = committed_traffic("fused_f32_2d_p16_T16384", kernel_source_files())
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "algorithmic_bytes_per_volume": bpv,
                "algorithmic_bytes_per_launch": vols * bpv,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if "hbm_gbs" in peaks
                else "fallback 6800 GB/s"}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded PCG64 uniform primitives; no dataset)",
           "config": bench_config(T, p, N),
           "arm": {"form": "fused", "kernel": desc32,
                   "precision": "f32 state and arithmetic, f64 eigenvalue maximum and CFL time step",
                   "l2": "flushed before every timed step (256 MiB write, then a 256 MiB read so the "
                         "flush's dirty lines are not written back inside the step); steps timed one "
                         "by one with CUDA events"},
           "roofline": roofline, "gpu_launches": launches, "e2e": e2e, "clocks": clk,
           "forms": forms}
    err_samples = forms_other.pop("_error_samples", []) if forms_other is not None else []
    if forms_other is not None:
        out["workloads"] = forms_other
    if abl is not None:
        out["ablations"] = abl
    if "cascade_f64" in forms:
        out["speedup_fused_f32_vs_cascade_f64"] = forms["fused_f32"]["value"] / forms["cascade_f64"]["value"]
    # the paper's unit: time per degree-of-freedom update (volume updates x N unknowns)
    out["cost_per_dof_update_ns"] = (ms_max / args.steps) * 1e6 / (vols * N)

    if not args.no_cpu_baseline and world == 1:
        wd = inputs.config(2, dtype=np.float64)
        v, cores, desc = cpu_baseline(wd, args.cpu_seconds)
        v1, _, desc1 = cpu_baseline(wd, max(1.0, args.cpu_seconds / 2), sample_patches=128, threads=1)
        out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": desc, "single_thread": {"value": v1, "cores": 1, "sample": desc1}}
        idx = np.sort(np.random.default_rng(7).choice(T, 16, replace=False))
        err, comps, _ = oracle_error(wd, None, final, w.steps, idx)
        out["error_vs_oracle"] = error_statement(err, comps, w.steps, len(idx), 1)
        # the same statement for the other workloads, after their full step counts
        for name, wo, prec, got, nsteps, sidx in err_samples:
            e_, c_ = oracle_error_sample(wo, prec, got, nsteps, sidx)
            out["workloads"][name]["error_vs_oracle"] = error_statement(e_, c_, nsteps, len(sidx), prec)
    if dist is not None:
        dist.destroy_process_group()
    return out


def scattered_e2e(b, w, host_dx, host_dt, host_lam, dist, dev, k=5):
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb
    from paper_2306_16731_gb300.multigpu import whole_job_rate
    T = w.num_patches
    off = w.offsets()
    sizes = np.diff(off) * 4                           # FP32 bytes per patch
    rng = np.random.default_rng(17)
    gaps = rng.integers(0, 256, T) * 16                # up to 4 KB between patches
    order = rng.permutation(T)
    pos = np.zeros(T, dtype=np.int64)
    cur = 0
    for i in order:
        cur += int(gaps[i])
        pos[i] = cur
        cur += int(sizes[i] + 15) // 16 * 16
    arena_in = torch.empty(cur, dtype=torch.uint8).pin_memory()
    arena_out = torch.empty(cur, dtype=torch.uint8).pin_memory()
    src = np.frombuffer(w.Q0.astype(np.float32).tobytes(), dtype=np.uint8)
    a_in = arena_in.numpy()
    for i in range(T):
        a_in[pos[i]:pos[i] + sizes[i]] = src[off[i] * 4:off[i + 1] * 4]
    base_in, base_out = arena_in.data_ptr(), arena_out.data_ptr()
    b.set_host_patches([base_in + int(x) for x in pos], [base_out + int(x) for x in pos])
    res = {"patches": T, "arena_bytes": int(cur), "layout": "shuffled order, 0-4 KB gaps, one pinned arena per side"}
    for name, flags, steps in (("gather_kernels", 0, k), ("per_patch_copies", fb.FV_SCATTER_COPIES, 2)):
        b.update_scattered(host_dx, host_dt, host_lam, None, w.cfl, flags)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s_ in range(steps):
            b.update_scattered(host_dx, host_dt, host_lam, None, w.cfl, flags | (fb.FV_SCATTER_SWAP if s_ & 1 else 0))
        el = time.perf_counter() - t0
        res[name] = {"value": whole_job_rate(w.interior_volumes * steps, el, dist, dev), "ms_per_step": el / steps * 1e3}
    b.set_host_patches(None, None)
    return res


def ablations(dev, stream, flush_l2, k=5):
    """The paper's realisation and layout comparisons on the 2D 16x16 FP64
    workload: the batched loop cascade with AoS, SoA and AoSoA temporaries
    (App. C), and the task-graph realisation (one graph node per patch, step
    and axis, Sec. 3) against the cascade at growing batch sizes."""
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb, inputs
    res = {}

    def setup(w, form, layout=0):
        b = fb.FVBatch(2, w.patch_size, precision=0, form=form, stream=stream.cuda_stream)
        b.set_cascade_layout(layout)
        qs = [torch.from_numpy(w.Q0).to(dev), None]
        qs[1] = qs[0].clone()
        dx = torch.tensor(w.dx, device=dev)
        lam = torch.zeros(w.num_patches, dtype=torch.float64, device=dev)
        dts = [torch.full((w.num_patches,), 1e-4, dtype=torch.float64, device=dev) for _ in range(2)]
        return b, qs, dx, lam, dts

    def steps(b, qs, dx, lam, dts):
        t0 = time.perf_counter()
        for s_ in range(2):                       # first use builds graphs (task-graph form)
            b.update(qs[s_ & 1], qs[1 - (s_ & 1)], dx, dts[s_ & 1], lam, dts[1 - (s_ & 1)], 0.4)
        torch.cuda.synchronize()
        first = time.perf_counter() - t0
        tot = 0.0
        for s_ in range(k):
            i = s_ & 1
            flush_l2()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.update(qs[i], qs[1 - i], dx, dts[i], lam, dts[1 - i], 0.4)
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        b.status()
        return tot / k, first

    w = inputs.config(2, dtype=np.float64)
    lay = {}
    for name, layout in (("aos", 0), ("soa", 1), ("aosoa", 2)):
        b, qs, dx, lam, dts = setup(w, 1, layout)
        ms, _ = steps(b, qs, dx, lam, dts)
        lay[name] = {"value": w.interior_volumes / (ms / 1e3), "ms_per_step": ms}
        b.close()
        del qs
    res["cascade_f64_temporaries_layout_2d_p16_T16384"] = lay
    tg = {}
    for T in (256, 2048, 16384):
        wt = inputs.uniform_batch(2, [16] * T, seed=2, dx=0.01)
        row = {}
        for name, form in (("taskgraph", 3), ("cascade", 1), ("fused", 0)):
            b, qs, dx, lam, dts = setup(wt, form)
            ms, first = steps(b, qs, dx, lam, dts)
            row[name] = {"value": wt.interior_volumes / (ms / 1e3), "ms_per_step": ms}
            if form == 3:
                row[name]["graph_kernel_nodes"] = b.launches_per_update()
                row[name]["first_two_updates_s"] = first
            b.close()
            del qs
        tg["T%d" % T] = row
    res["taskgraph_vs_batched_f64_2d_p16"] = tg
    return res


def other_workloads(dev, stream, flush_l2, steps):
    """Secondary lines: the 3D periodic pulse (FP32 and BF16 storage), the
    uneven 2D batch (200 steps in one CUDA graph) and the 3D 16^3 batch
    (fused FP32 vs plain FP64 cascade).  Single steps are timed with L2
    flushed like the headline; graph runs are L2-warm by nature."""
    import torch
    from paper_2306_16731_gb300 import fvbatch as fb, inputs
    peak = _peak_hbm()
    res = {}

    def setup(w, precision, form=None):
        b = fb.FVBatch(w.dim, w.patch_size, precision=precision, halo_mode=w.halo_mode,
                       form=form, stream=stream.cuda_stream)
        dtype = {0: torch.float64, 1: torch.float32, 2: torch.bfloat16}[precision]
        qa = torch.from_numpy(w.Q0).to(device=dev).to(dtype)
        qb = qa.clone()
        dx = torch.tensor(w.dx, device=dev)
        lam = torch.zeros(w.num_patches, dtype=torch.float64, device=dev)
        dts = [torch.zeros_like(lam), torch.zeros_like(lam)]
        b.max_eigenvalue(qa, lam)
        b.cfl_time_step(lam, dx, w.cfl, dts[0])
        return b, [qa, qb], dx, lam, dts

    def single_steps(b, qs, dx, lam, dts, k, cfl):
        for s in range(3):                       # warm-up: the timed step untimed, flush included
            flush_l2()
            b.update(qs[s & 1], qs[1 - (s & 1)], dx, dts[s & 1], lam, dts[1 - (s & 1)], cfl)
        tot = 0.0
        for s in range(k):
            i = (3 + s) & 1
            flush_l2()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.update(qs[i], qs[1 - i], dx, dts[i], lam, dts[1 - i], cfl)
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        b.status()
        return tot / k

    def graph_steps(b, qs, dx, lam, dts, nsteps, cfl):
        """Per-step time of an nsteps CFL-chained run captured as one CUDA
        graph (first replay captures; median of 5 timed replays).  The state
        is not flushed between the steps of a run: for batches below the L2
        size this is the L2-warm multi-step number beside the flushed one."""
        b.run(qs[0], qs[1], dx, dts[0], dts[1], lam, nsteps, cfl, True)
        torch.cuda.synchronize()
        times = []
        for _ in range(5):
            flush_l2()
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            b.run(qs[0], qs[1], dx, dts[0], dts[1], lam, nsteps, cfl, True)
            g1.record(stream)
            torch.cuda.synchronize()
            times.append(g0.elapsed_time(g1) / nsteps)
        b.status()
        return float(np.median(times))

    def bytes_per_volume(w, es):
        p = w.patch_size.astype(np.float64)
        N = w.dim + 2
        reads = p ** w.dim + (0 if w.halo_mode == 1 else 2 * w.dim * p ** (w.dim - 1))
        return float(np.sum(N * es * (reads + p ** w.dim)) / np.sum(p ** w.dim))

    k = max(5, min(30, steps // 4))
    samples = []

    def final_sample(name, w, precision, nsteps, nsample, seed, use_graph=True):
        """Run the workload's full step count (CFL-chained) from its initial
        state; keep the final state of a seeded sample of patches for the
        error statement against the oracle (made in the CPU-baseline leg)."""
        b, qs, dx, lam, dts = setup(w, precision)
        b.run(qs[0], qs[1], dx, dts[0], dts[1], lam, nsteps, w.cfl, use_graph)
        b.status()
        fin = (qs[1] if nsteps % 2 else qs[0])
        idx = np.sort(np.random.default_rng(seed).choice(w.num_patches, nsample, replace=False))
        off = w.offsets()
        got = [fin[int(off[i]):int(off[i + 1])].to(torch.float64).cpu().numpy() for i in idx]
        samples.append((name, w, precision, got, nsteps, idx))
        b.close()
        del qs

    # 3D periodic pulse, 4096 patches of 8^3
    w3 = inputs.config(3, dtype=np.float32)
    for name, prec, es in (("3d_p8_T4096_periodic_f32", 1, 4), ("3d_p8_T4096_periodic_bf16", 2, 2)):
        b, qs, dx, lam, dts = setup(w3, prec)
        scratch = qs[0].clone()
        b.tune(qs[0], scratch, dx, dts[0])
        del scratch
        ms = single_steps(b, qs, dx, lam, dts, k, w3.cfl)
        bpv = bytes_per_volume(w3, es)
        gms = graph_steps(b, qs, dx, lam, dts, w3.steps, w3.cfl)
        res[name] = {"value": w3.interior_volumes / (ms / 1e3), "ms_per_step": ms,
                     "bytes_per_volume": bpv, "achieved_gbs": w3.interior_volumes * bpv / (ms / 1e3) / 1e9,
                     "roofline_frac": w3.interior_volumes * bpv / (ms / 1e3) / 1e9 / peak,
                     "value_graph_%dsteps_l2warm" % w3.steps: w3.interior_volumes / (gms / 1e3),
                     "ms_per_step_graph_l2warm": gms,
                     "kernel": b.describe()}
        b.close()
        final_sample(name, w3, prec, w3.steps, 16, 31)
    # uneven 2D batch, 50,000 patches, 200 steps in one graph
    w4 = inputs.config(4, dtype=np.float32)
    b, qs, dx, lam, dts = setup(w4, 1)
    scratch = qs[0].clone()
    b.tune(qs[0], scratch, dx, dts[0])
    del scratch
    ms1 = single_steps(b, qs, dx, lam, dts, k, w4.cfl)
    b.run(qs[0], qs[1], dx, dts[0], dts[1], lam, w4.steps, w4.cfl, True)    # capture
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.run(qs[0], qs[1], dx, dts[0], dts[1], lam, w4.steps, w4.cfl, True)
    e1.record(stream)
    torch.cuda.synchronize()
    b.status()
    gms = e0.elapsed_time(e1)
    bpv = bytes_per_volume(w4, 4)
    res["2d_uneven_T50000_f32"] = {
        "value_graph_%dsteps" % w4.steps: w4.interior_volumes * w4.steps / (gms / 1e3),
        "ms_per_step_graph": gms / w4.steps, "value_single_step": w4.interior_volumes / (ms1 / 1e3),
        "ms_per_step_single": ms1, "bytes_per_volume": bpv,
        "roofline_frac_single_step": w4.interior_volumes * bpv / (ms1 / 1e3) / 1e9 / peak,
        "launches_per_step": b.launches_per_update(), "kernel": b.describe()}
    b.close()
    del qs
    final_sample("2d_uneven_T50000_f32", w4, 1, w4.steps, 16, 41)
    # the generic-PDE kernel (Eq. 1 with non-conservative product and
    # source): 2D shallow water, 16,384 patches of 16x16, FP32 and FP64
    for name, prec, es in (("2d_p16_T16384_shallow_water_f32", 1, 4), ("2d_p16_T16384_shallow_water_f64", 0, 8)):
        ws = inputs.shallow_water_batch([16] * 16384, seed=9, dx=0.01)
        bs = fb.FVBatch(2, ws.patch_size, precision=prec, pde=fb.FV_PDE_SHALLOW_WATER, params=[9.81, 0.5],
                        stream=stream.cuda_stream)
        dtype = torch.float32 if prec == 1 else torch.float64
        qs = [torch.from_numpy(ws.Q0).to(device=dev).to(dtype), None]
        qs[1] = qs[0].clone()
        dx = torch.tensor(ws.dx, device=dev)
        lam = torch.zeros(ws.num_patches, dtype=torch.float64, device=dev)
        dts = [torch.zeros_like(lam), torch.zeros_like(lam)]
        bs.max_eigenvalue(qs[0], lam)
        bs.cfl_time_step(lam, dx, 0.4, dts[0])
        ms = single_steps(bs, qs, dx, lam, dts, k, 0.4)
        bpv = bytes_per_volume(ws, es)
        res[name] = {"value": ws.interior_volumes / (ms / 1e3), "ms_per_step": ms, "bytes_per_volume": bpv,
                     "roofline_frac": ws.interior_volumes * bpv / (ms / 1e3) / 1e9 / peak, "kernel": bs.describe()}
        # the patch-wise form on the same batch, for comparison
        bs.set_form(fb.FV_FORM_TILE)
        mt = single_steps(bs, qs, dx, lam, dts, k, 0.4)
        res[name]["patchwise_tile"] = {"value": ws.interior_volumes / (mt / 1e3), "ms_per_step": mt,
                                       "roofline_frac": ws.interior_volumes * bpv / (mt / 1e3) / 1e9 / peak}
        bs.close()
        del qs
    # the 2D batch wired as a periodic 128 x 128 grid of patches: halos filled
    # from neighbours in-kernel (fused) vs a separate exchange launch + update
    w2 = inputs.config(2, dtype=np.float32)
    G = 128
    nb = []
    for i in range(w2.num_patches):
        gx, gy = i % G, i // G
        nb.append([gy * G + (gx - 1) % G, gy * G + (gx + 1) % G, ((gy - 1) % G) * G + gx, ((gy + 1) % G) * G + gx])
    b, qs, dx, lam, dts = setup(w2, 1)
    b.set_neighbours(nb)
    ms_fused = single_steps(b, qs, dx, lam, dts, k, w2.cfl)
    b.set_neighbours(None)
    b2 = fb.FVBatch(2, w2.patch_size, precision=1, stream=stream.cuda_stream)
    b2.set_neighbours(nb)
    tot = 0.0
    for s_ in range(3 + k):
        i = s_ & 1
        flush_l2()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b2.halo_exchange(qs[i])
        b.update(qs[i], qs[1 - i], dx, dts[i], lam, dts[1 - i], w2.cfl)
        e1.record(stream)
        torch.cuda.synchronize()
        if s_ >= 3:
            tot += e0.elapsed_time(e1)
    ms_sep = tot / k
    b.status()
    res["2d_p16_T16384_grid_exchange_f32"] = {
        "value_fused_neighbour_reads": w2.interior_volumes / (ms_fused / 1e3), "ms_per_step_fused": ms_fused,
        "value_exchange_then_update": w2.interior_volumes / (ms_sep / 1e3), "ms_per_step_separate": ms_sep,
        "roofline_frac_fused": w2.interior_volumes * 36.0 / (ms_fused / 1e3) / 1e9 / peak}
    b.close()
    b2.close()
    del qs

    # 3D 16^3, 32,768 patches (3.8 GB FP32 state)
    w5 = inputs.config(5, dtype=np.float32)
    b, qs, dx, lam, dts = setup(w5, 1)
    ms = single_steps(b, qs, dx, lam, dts, max(3, k // 3), w5.cfl)
    bpv = bytes_per_volume(w5, 4)
    res["3d_p16_T32768_f32"] = {"value": w5.interior_volumes / (ms / 1e3), "ms_per_step": ms,
                                "bytes_per_volume": bpv,
                                "achieved_gbs": w5.interior_volumes * bpv / (ms / 1e3) / 1e9,
                                "roofline_frac": w5.interior_volumes * bpv / (ms / 1e3) / 1e9 / peak,
                                "kernel": b.describe()}
    b.close()
    del qs
    final_sample("3d_p16_T32768_f32", w5, 1, w5.steps, 4, 51, use_graph=False)
    torch.cuda.empty_cache()
    try:
        b, qs, dx, lam, dts = setup(w5, 0, fb.FV_FORM_CASCADE)
        ms = single_steps(b, qs, dx, lam, dts, 2, w5.cfl)
        res["3d_p16_T32768_cascade_f64"] = {"value": w5.interior_volumes / (ms / 1e3), "ms_per_step": ms,
                                            "scratch_bytes": b.scratch_bytes()}
        res["3d_p16_T32768_speedup_fused_f32_vs_cascade_f64"] = (
            res["3d_p16_T32768_f32"]["value"] / res["3d_p16_T32768_cascade_f64"]["value"])
        b.close()
        del qs
    except Exception as e:            # e.g. not enough device memory for the cascade scratch
        res["3d_p16_T32768_cascade_f64"] = {"unavailable": str(e)[:200]}
    torch.cuda.empty_cache()
    res["_error_samples"] = samples
    return res


def _peak_hbm():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        return 6800.0


def _smi_id(torch, dev):
    """nvidia-smi selector of the torch device (its UUID when available)."""
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev.index or 0)


def _fused_ok(fb, w, precision):
    try:
        b = fb.FVBatch(w.dim, w.patch_size, precision=precision, halo_mode=w.halo_mode,
                       form=fb.FV_FORM_FUSED)
        b.close()
        return True
    except fb.FVError:
        return False


# ------------------------------------------------------------- reference

def run_reference(args):
    """The reference arm: the FP64 CPU oracle, as it stands, on the whole
    headline batch (16,384 patches of 16 x 16) for every timed step, with
    its own CFL chain, on the host's cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    from paper_2306_16731_gb300 import inputs
    import oracle
    oracle.build()
    w = inputs.config(2, dtype=np.float64)
    T, p, N = w.num_patches, int(w.patch_size[0]), w.dim + 2
    psz, dx = w.patch_size, w.dx
    vols = w.interior_volumes
    lam = oracle.batch_max_eigenvalue(w.dim, psz, w.Q0)
    dt = oracle.cfl_time_step(w.dim, lam, dx, w.cfl)
    cur = w.Q0
    for _ in range(args.warmup):
        cur, lam = oracle.batch_step(w.dim, psz, dx, dt, cur, w.gamma, w.halo_mode)
        dt = oracle.cfl_time_step(w.dim, lam, dx, w.cfl)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cur, lam = oracle.batch_step(w.dim, psz, dx, dt, cur, w.gamma, w.halo_mode)
        dt = oracle.cfl_time_step(w.dim, lam, dx, w.cfl)
    el = time.perf_counter() - t0
    value = vols * args.steps / el
    cores = oracle.num_threads()
    sample = ("the whole batch (%d patches of %dx%d) every step, %d CFL-chained steps, FP64 oracle on %d host "
              "threads" % (T, p, p, args.steps, cores))
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded PCG64 uniform primitives; no dataset)",
            "config": bench_config(T, p, N),
            "arm": {"form": "FP64 CPU oracle (plain C, OpenMP over patches)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}


def run_profile(args):
    """A few launches of one form on a batch larger than L2, for ncu."""
    import torch
    from paper_2306_16731_gb300 import build, fvbatch as fb, inputs
    build.build()
    form_name, prec_name = args.profile.split("_")
    pde_kw = {}
    if form_name in ("swe", "swetile"):
        # shallow water over a bathymetry, 2D patches of 16x16 (fused sweep or patch-wise)
        T = args.patches or 65536
        w = inputs.shallow_water_batch([16] * T, seed=9, dx=0.01)
        pde_kw = {"pde": fb.FV_PDE_SHALLOW_WATER, "params": [9.81, 0.5]}
        form_name = "fused" if form_name == "swe" else "tile"
    elif form_name.startswith("fused3d"):
        p3 = 16 if form_name == "fused3d16" else 8
        T = args.patches or (4096 if p3 == 16 else 16384)
        halo = inputs.PERIODIC if form_name == "fused3dper" else inputs.FIXED
        w = inputs.uniform_batch(3, [p3] * T, seed=3, dx=0.01, dtype=np.float32, halo_mode=halo)
        form_name = "fused"
    elif form_name == "uneven":
        # the 50,000-patch uneven batch (edges 4..32, dx = 3^-k), one launch per step
        w = inputs.config(4, dtype=np.float32, num_patches=args.patches)
        T = w.num_patches
        form_name = "fused"
    else:
        T = args.patches or 65536
        w = inputs.uniform_batch(2, [16] * T, seed=2, dx=0.01, dtype=np.float32)
    prec = {"f32": fb.FV_F32, "f64": fb.FV_F64}[prec_name]
    form = {"fused": fb.FV_FORM_FUSED, "cascade": fb.FV_FORM_CASCADE, "tile": fb.FV_FORM_TILE}[form_name]
    b = fb.FVBatch(w.dim, w.patch_size, precision=prec, form=form, halo_mode=w.halo_mode, **pde_kw)
    dtype = torch.float32 if prec == fb.FV_F32 else torch.float64
    qa = torch.from_numpy(w.Q0).to("cuda", dtype)
    qb = qa.clone()
    dx = torch.tensor(w.dx, device="cuda")
    lam = torch.zeros(T, dtype=torch.float64, device="cuda")
    dta, dtb = torch.zeros_like(lam), torch.zeros_like(lam)
    b.max_eigenvalue(qa, lam)
    b.cfl_time_step(lam, dx, 0.4, dta)
    for s in range(args.warmup + args.steps):
        i = s & 1
        b.update([qa, qb][i], [qb, qa][i], dx, [dta, dtb][i], lam, [dtb, dta][i], 0.4)
    torch.cuda.synchronize()
    b.status()
    print(json.dumps({"profile": args.profile, "patches": T, "launches": args.warmup + args.steps,
                      "kernel": b.describe()}))


def main():
    args = parse_args()
    if args.profile:
        run_profile(args)
        return
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
