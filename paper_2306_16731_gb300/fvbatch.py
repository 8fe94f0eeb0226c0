"""Thin ctypes binding of ``libfvbatch.so`` (C ABI in ``include/fv_batch.h``).

Argument marshalling only: every step of the update runs in the CUDA
kernels of the library.  PyTorch supplies device memory and streams.  The
binding refuses to work without the compiled library (there is no CPU
fallback); build it with ``paper_2306_16731_gb300.build.build()``.

The function names mirror the C entry points.  Buffers may be torch tensors
(their ``data_ptr()`` is passed) or raw integer addresses.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB as _LIB_PATH

FV_OK = 0
FV_EINVAL = -1
FV_ENOMEM = -2
FV_ECUDA = -3
FV_EUNSUPPORTED = -4
FV_ENONPHYSICAL = -5
FV_ETIMEOUT = -6

FV_F64 = 0
FV_F32 = 1
FV_BF16_F32 = 2

FV_HALO_FIXED = 0
FV_HALO_PERIODIC = 1

FV_FORM_FUSED = 0
FV_FORM_CASCADE = 1
FV_FORM_TILE = 2
FV_FORM_TASKGRAPH = 3
FV_PDE_EULER = 0
FV_PDE_SHALLOW_WATER = 1
FV_LAYOUT_AOS = 0
FV_LAYOUT_SOA = 1
FV_LAYOUT_AOSOA = 2
FV_SCATTER_SWAP = 1
FV_SCATTER_COPIES = 2

_ERRNAMES = {FV_EINVAL: "FV_EINVAL", FV_ENOMEM: "FV_ENOMEM", FV_ECUDA: "FV_ECUDA",
             FV_EUNSUPPORTED: "FV_EUNSUPPORTED", FV_ENONPHYSICAL: "FV_ENONPHYSICAL",
             FV_ETIMEOUT: "FV_ETIMEOUT"}

EXPORTS = ["fv_batch_create", "fv_batch_set_form", "fv_batch_set_stream", "fv_batch_set_launch_shape",
           "fv_batch_set_sweep_ring",
           "fv_batch_set_neighbours", "fv_halo_exchange", "fv_patch_batch_update_host",
           "fv_patch_batch_update", "fv_max_eigenvalue", "fv_cfl_time_step",
           "fv_conserved_totals", "fv_batch_run", "fv_batch_tune", "fv_batch_status",
           "fv_batch_destroy", "fv_last_error", "fv_batch_state_elems",
           "fv_batch_scratch_bytes", "fv_batch_describe", "fv_batch_launches_per_update",
           "fv_batch_test_wait_expiry", "fv_batch_set_cascade_layout", "fv_batch_create_pde",
           "fv_batch_set_host_patches", "fv_patch_batch_update_scattered", "fv_test_fail_device_alloc",
           "fv_patch_batch_run_host"]


class FVError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (_ERRNAMES.get(code, "FV_E?"), code, msg))
        self.code = code


_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_dp = ctypes.c_void_p     # device double* passed as an address


def library_path() -> str:
    return os.environ.get("FVBATCH_LIB") or _LIB_PATH


def load() -> ctypes.CDLL:
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError("libfvbatch.so is not built (%s); run "
                               "paper_2306_16731_gb300.build.build()" % path)
        lib = ctypes.CDLL(path)
        i, d = ctypes.c_int, ctypes.c_double
        sig = {
            "fv_batch_create": (i, [ctypes.POINTER(_vp), i, i, ctypes.POINTER(ctypes.c_int32), i, i, i, i, d, _vp]),
            "fv_batch_create_pde": (i, [ctypes.POINTER(_vp), i, i, i, ctypes.POINTER(ctypes.c_int32), i, i,
                                        ctypes.POINTER(ctypes.c_double), i, _vp]),
            "fv_batch_set_form": (i, [_vp, i]),
            "fv_batch_set_stream": (i, [_vp, _vp]),
            "fv_batch_set_launch_shape": (i, [_vp, i, i]),
            "fv_batch_set_sweep_ring": (i, [_vp, i]),
            "fv_batch_test_wait_expiry": (i, [_vp, i]),
            "fv_batch_set_cascade_layout": (i, [_vp, i]),
            "fv_test_fail_device_alloc": (i, [i]),
            "fv_batch_set_host_patches": (i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
            "fv_patch_batch_update_scattered": (i, [_vp, _vp, _vp, _vp, _vp, d, i]),
            "fv_batch_set_neighbours": (i, [_vp, ctypes.POINTER(ctypes.c_int32)]),
            "fv_patch_batch_update_host": (i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, d, i]),
            "fv_patch_batch_run_host": (i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, i, d, i]),
            "fv_halo_exchange": (i, [_vp, _vp]),
            "fv_patch_batch_update": (i, [_vp, _vp, _vp, _dp, _dp, _dp, _dp, d]),
            "fv_max_eigenvalue": (i, [_vp, _vp, _dp]),
            "fv_cfl_time_step": (i, [_vp, _dp, _dp, d, _dp]),
            "fv_conserved_totals": (i, [_vp, _vp, _dp]),
            "fv_batch_run": (i, [_vp, _vp, _vp, _dp, _dp, _dp, _dp, i, d, i]),
            "fv_batch_tune": (i, [_vp, _vp, _vp, _dp, _dp]),
            "fv_batch_status": (i, [_vp]),
            "fv_batch_destroy": (i, [_vp]),
            "fv_last_error": (ctypes.c_char_p, []),
            "fv_batch_state_elems": (ctypes.c_size_t, [_vp]),
            "fv_batch_scratch_bytes": (ctypes.c_size_t, [_vp]),
            "fv_batch_describe": (i, [_vp, ctypes.c_char_p, ctypes.c_size_t]),
            "fv_batch_launches_per_update": (i, [_vp]),
            "fv_patch_batch_update_noalloc": (i, [i, i, i, i, i, d, _vp, _vp, _dp, _dp, _dp, _dp, d, _vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _addr(x):
    """Device address of a tensor / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _check(rc: int) -> int:
    if rc != FV_OK:
        raise FVError(rc, load().fv_last_error().decode())
    return rc


def last_error() -> str:
    return load().fv_last_error().decode()


# ------------------------------------------------------------ C-ABI mirror

def fv_batch_create(dim, patch_size, halo=1, unknowns=None, precision=FV_F64,
                    halo_mode=FV_HALO_FIXED, gamma=1.4, stream=0):
    """Returns the opaque batch handle (int).  ``patch_size``: host ints."""
    lib = load()
    ps = [int(v) for v in patch_size]
    arr = (ctypes.c_int32 * max(1, len(ps)))(*ps) if ps else None
    h = _vp()
    _check(lib.fv_batch_create(ctypes.byref(h), int(dim), len(ps), arr, int(halo),
                               int(dim + 2 if unknowns is None else unknowns),
                               int(precision), int(halo_mode), float(gamma), _vp(stream or 0)))
    return h.value


def fv_batch_set_form(b, form):
    return _check(load().fv_batch_set_form(b, int(form)))


def fv_batch_set_neighbours(b, neighbours):
    """neighbours: host ints [T, 2*dim] (order -x,+x,-y,+y[,-z,+z]; -1 = own halo) or None."""
    if neighbours is None:
        return _check(load().fv_batch_set_neighbours(b, None))
    flat = [int(v) for row in neighbours for v in (row if hasattr(row, "__iter__") else [row])]
    arr = (ctypes.c_int32 * max(1, len(flat)))(*flat)
    return _check(load().fv_batch_set_neighbours(b, arr))


def fv_halo_exchange(b, Q):
    return _check(load().fv_halo_exchange(b, _addr(Q)))


def fv_batch_set_launch_shape(b, warps_per_block, blocks_per_sm):
    return _check(load().fv_batch_set_launch_shape(b, int(warps_per_block), int(blocks_per_sm)))


def fv_batch_set_sweep_ring(b, rows):
    return _check(load().fv_batch_set_sweep_ring(b, int(rows)))


def fv_batch_create_pde(pde, dim, patch_size, precision, halo_mode, params, stream=0):
    """Batch for one of the FV_PDE_* systems; ``params`` are host floats."""
    lib = load()
    ps = [int(v) for v in patch_size]
    arr = (ctypes.c_int32 * max(1, len(ps)))(*ps) if ps else None
    pv = [float(v) for v in params]
    parr = (ctypes.c_double * max(1, len(pv)))(*pv)
    h = _vp()
    _check(lib.fv_batch_create_pde(ctypes.byref(h), int(pde), int(dim), len(ps), arr, int(precision),
                                   int(halo_mode), parr, len(pv), _vp(stream or 0)))
    return h.value


def fv_batch_set_host_patches(b, patch_in, patch_out):
    """patch_in / patch_out: sequences of host addresses (ints or pinned CPU
    tensors), one per patch, or both None to clear."""
    if patch_in is None and patch_out is None:
        return _check(load().fv_batch_set_host_patches(b, None, None))
    ai = [_addr(x) for x in patch_in]
    ao = [_addr(x) for x in patch_out]
    ti = (_vp * max(1, len(ai)))(*ai)
    to = (_vp * max(1, len(ao)))(*ao)
    return _check(load().fv_batch_set_host_patches(b, ti, to))


def fv_patch_batch_update_scattered(b, dx_host, dt_host, lambda_host=None, dt_next_host=None, cfl=0.4, flags=0):
    return _check(load().fv_patch_batch_update_scattered(b, _addr(dx_host), _addr(dt_host), _addr(lambda_host),
                                                         _addr(dt_next_host), float(cfl), int(flags)))


def fv_test_fail_device_alloc(k):
    """Test hook: make the k-th following device allocation fail (k <= 0 disarms)."""
    return _check(load().fv_test_fail_device_alloc(int(k)))


def fv_batch_set_cascade_layout(b, layout):
    return _check(load().fv_batch_set_cascade_layout(b, int(layout)))


def fv_batch_test_wait_expiry(b, enable):
    return _check(load().fv_batch_test_wait_expiry(b, 1 if enable else 0))


def fv_batch_set_stream(b, stream):
    return _check(load().fv_batch_set_stream(b, _vp(stream or 0)))


def fv_patch_batch_update(b, Q_in, Q_out, dx, dt, lambda_out=None, dt_next_out=None, cfl=0.4):
    return _check(load().fv_patch_batch_update(b, _addr(Q_in), _addr(Q_out), _addr(dx), _addr(dt),
                                               _addr(lambda_out), _addr(dt_next_out), float(cfl)))


def fv_patch_batch_run_host(b, Q_a_host, Q_b_host, dx_host, dt_a_host, dt_b_host, lambda_host=None, steps=1,
                            cfl=0.4, chunks=8):
    """CFL-chained steps with the state in host memory (pinned torch CPU
    tensors or addresses), ping-ponging between Q_a/Q_b and dt_a/dt_b."""
    return _check(load().fv_patch_batch_run_host(b, _addr(Q_a_host), _addr(Q_b_host), _addr(dx_host),
                                                 _addr(dt_a_host), _addr(dt_b_host), _addr(lambda_host),
                                                 int(steps), float(cfl), int(chunks)))


def fv_patch_batch_update_host(b, Q_in_host, Q_out_host, dx_host, dt_host, lambda_host=None,
                               dt_next_host=None, cfl=0.4, chunks=8):
    """Update with the state in host memory (pinned torch CPU tensors or
    addresses); copies and updates pipelined over ``chunks`` patch ranges."""
    return _check(load().fv_patch_batch_update_host(b, _addr(Q_in_host), _addr(Q_out_host), _addr(dx_host),
                                                    _addr(dt_host), _addr(lambda_host), _addr(dt_next_host),
                                                    float(cfl), int(chunks)))


def fv_max_eigenvalue(b, Q, lambda_out):
    return _check(load().fv_max_eigenvalue(b, _addr(Q), _addr(lambda_out)))


def fv_cfl_time_step(b, lam, dx, cfl, dt_out):
    return _check(load().fv_cfl_time_step(b, _addr(lam), _addr(dx), float(cfl), _addr(dt_out)))


def fv_conserved_totals(b, Q, totals_out):
    return _check(load().fv_conserved_totals(b, _addr(Q), _addr(totals_out)))


def fv_batch_run(b, Q_a, Q_b, dx, dt_a, dt_b, lambda_out, steps, cfl=0.4, use_graph=True):
    return _check(load().fv_batch_run(b, _addr(Q_a), _addr(Q_b), _addr(dx), _addr(dt_a),
                                      _addr(dt_b), _addr(lambda_out), int(steps), float(cfl),
                                      1 if use_graph else 0))


def fv_batch_tune(b, Q_in, Q_out, dx, dt):
    return _check(load().fv_batch_tune(b, _addr(Q_in), _addr(Q_out), _addr(dx), _addr(dt)))


def fv_batch_status(b):
    return _check(load().fv_batch_status(b))


def fv_batch_destroy(b):
    return _check(load().fv_batch_destroy(b))


def fv_batch_state_elems(b) -> int:
    return int(load().fv_batch_state_elems(b))


def fv_batch_scratch_bytes(b) -> int:
    return int(load().fv_batch_scratch_bytes(b))


def fv_batch_describe(b) -> str:
    buf = ctypes.create_string_buffer(512)
    _check(load().fv_batch_describe(b, buf, 512))
    return buf.value.decode()


def fv_batch_launches_per_update(b) -> int:
    return int(load().fv_batch_launches_per_update(b))


# ------------------------------------------------------ convenience object

_PREC_DTYPES = {FV_F64: "float64", FV_F32: "float32", FV_BF16_F32: "bfloat16"}


class FVBatch:
    """Owns one batch handle; methods forward to the C entry points."""

    def __init__(self, dim, patch_size, precision=FV_F64, halo_mode=FV_HALO_FIXED,
                 gamma=1.4, stream=None, form=None, pde=FV_PDE_EULER, params=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.dim = int(dim)
        self.patch_size = [int(v) for v in patch_size]
        self.precision = int(precision)
        self.halo_mode = int(halo_mode)
        self.pde = int(pde)
        if self.pde == FV_PDE_EULER and params is None:
            self.handle = fv_batch_create(dim, self.patch_size, 1, dim + 2, precision, halo_mode, gamma, stream)
        else:
            self.handle = fv_batch_create_pde(self.pde, dim, self.patch_size, precision, halo_mode,
                                              params if params is not None else [gamma], stream)
        if form is not None:
            fv_batch_set_form(self.handle, form)

    @property
    def torch_dtype(self):
        import torch
        return getattr(torch, _PREC_DTYPES[self.precision])

    def state_elems(self) -> int:
        return fv_batch_state_elems(self.handle)

    def set_form(self, form):
        fv_batch_set_form(self.handle, form)

    def set_neighbours(self, neighbours):
        fv_batch_set_neighbours(self.handle, neighbours)

    def halo_exchange(self, Q):
        fv_halo_exchange(self.handle, Q)

    def set_launch_shape(self, warps_per_block, blocks_per_sm):
        fv_batch_set_launch_shape(self.handle, warps_per_block, blocks_per_sm)

    def set_sweep_ring(self, rows):
        fv_batch_set_sweep_ring(self.handle, rows)

    def set_host_patches(self, patch_in, patch_out):
        """Register per-patch page-locked host buffers (see fv_batch_set_host_patches)."""
        fv_batch_set_host_patches(self.handle, patch_in, patch_out)

    def update_scattered(self, dx_host, dt_host, lambda_host=None, dt_next_host=None, cfl=0.4, flags=0):
        fv_patch_batch_update_scattered(self.handle, dx_host, dt_host, lambda_host, dt_next_host, cfl, flags)

    def set_cascade_layout(self, layout):
        """Layout of the cascade's (and task graph's) vector temporaries (FV_LAYOUT_*)."""
        fv_batch_set_cascade_layout(self.handle, layout)

    def test_wait_expiry(self, enable):
        """Test hook: make the bounded copy waits of the periodic 8^3 kernel run out."""
        fv_batch_test_wait_expiry(self.handle, enable)

    def set_stream(self, stream):
        fv_batch_set_stream(self.handle, stream)

    def update(self, Q_in, Q_out, dx, dt, lambda_out=None, dt_next_out=None, cfl=0.4):
        fv_patch_batch_update(self.handle, Q_in, Q_out, dx, dt, lambda_out, dt_next_out, cfl)

    def update_host(self, Q_in_host, Q_out_host, dx_host, dt_host, lambda_host=None, dt_next_host=None,
                    cfl=0.4, chunks=8):
        fv_patch_batch_update_host(self.handle, Q_in_host, Q_out_host, dx_host, dt_host, lambda_host,
                                   dt_next_host, cfl, chunks)

    def run_host(self, Q_a_host, Q_b_host, dx_host, dt_a_host, dt_b_host, lambda_host=None, steps=1, cfl=0.4,
                 chunks=8):
        fv_patch_batch_run_host(self.handle, Q_a_host, Q_b_host, dx_host, dt_a_host, dt_b_host, lambda_host, steps,
                                cfl, chunks)

    def max_eigenvalue(self, Q, lambda_out):
        fv_max_eigenvalue(self.handle, Q, lambda_out)

    def cfl_time_step(self, lam, dx, cfl, dt_out):
        fv_cfl_time_step(self.handle, lam, dx, cfl, dt_out)

    def conserved_totals(self, Q, totals_out):
        fv_conserved_totals(self.handle, Q, totals_out)

    def run(self, Q_a, Q_b, dx, dt_a, dt_b, lambda_out, steps, cfl=0.4, use_graph=True):
        fv_batch_run(self.handle, Q_a, Q_b, dx, dt_a, dt_b, lambda_out, steps, cfl, use_graph)

    def tune(self, Q_in, Q_out, dx, dt):
        fv_batch_tune(self.handle, Q_in, Q_out, dx, dt)

    def status(self):
        fv_batch_status(self.handle)

    def describe(self) -> str:
        return fv_batch_describe(self.handle)

    def launches_per_update(self) -> int:
        return fv_batch_launches_per_update(self.handle)

    def scratch_bytes(self) -> int:
        return fv_batch_scratch_bytes(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            fv_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fv_patch_batch_update_noalloc(dim, num_patches, patch_size, precision, halo_mode, gamma,
                                  Q_in, Q_out, dx, dt, lambda_out=None, dt_next_out=None,
                                  cfl=0.4, stream=0):
    """Allocation-free update of equal-size patches (loop-cascade kernels,
    scratch in a built-in 64 MiB device array); see include/fv_batch.h."""
    return _check(load().fv_patch_batch_update_noalloc(
        int(dim), int(num_patches), int(patch_size), int(precision), int(halo_mode), float(gamma),
        _addr(Q_in), _addr(Q_out), _addr(dx), _addr(dt), _addr(lambda_out), _addr(dt_next_out),
        float(cfl), _vp(stream or 0)))


def fv_last_error() -> str:
    """Thread-local description of the last failure of this thread."""
    return last_error()
