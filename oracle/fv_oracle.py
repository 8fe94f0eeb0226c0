"""ctypes front end of the plain C FP64 oracle (``fv_oracle.c``).

TEST INFRASTRUCTURE: imported only by the tests, the smoke check and the
CPU-baseline leg of the benchmark.  The C source is compiled with gcc into
``oracle/_build`` on first use (or by ``build()``), with
``-O2 -ffp-contract=off`` so that every product and sum is rounded on its own,
and with OpenMP over patches (thread count from ``OMP_NUM_THREADS``).

All arrays are numpy float64 in the array-of-structures layout
``Q[patch][z][y][x][k]`` with a one-volume halo around each patch; patch ``i``
starts at element ``sum_{j<i} (d+2) (p_j+2)^d``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

FIXED = 0
PERIODIC = 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libfvoracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


def compile_source(src: str, out: str) -> str:
    """gcc-compile an oracle C source into the shared library ``out``."""
    tmp = out + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-fopenmp", "-std=c11", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent); returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    return compile_source(_SRC, _LIB)


def bind(path: str):
    """ctypes handle of an oracle library at ``path`` with typed entry points."""
    lib = ctypes.CDLL(path)
    lib.fvo_state_elems.restype = ctypes.c_int64
    lib.fvo_state_elems.argtypes = [ctypes.c_int, ctypes.c_int, _ip]
    lib.fvo_batch_step.restype = ctypes.c_int
    lib.fvo_batch_step.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _dp, _dp,
                                   ctypes.c_double, ctypes.c_int, _dp, _dp, _dp]
    lib.fvo_batch_max_eigenvalue.restype = ctypes.c_int
    lib.fvo_batch_max_eigenvalue.argtypes = [ctypes.c_int, ctypes.c_int, _ip,
                                             ctypes.c_double, _dp, _dp]
    lib.fvo_cfl_time_step.restype = None
    lib.fvo_cfl_time_step.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp,
                                      ctypes.c_double, _dp]
    lib.fvo_batch_run.restype = ctypes.c_int
    lib.fvo_batch_run.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _dp,
                                  ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_int, _dp, _dp, _dp]
    lib.fvo_batch_totals.restype = ctypes.c_int
    lib.fvo_batch_totals.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _dp, _dp]
    lib.fvo_swe_batch_step.restype = ctypes.c_int
    lib.fvo_swe_batch_step.argtypes = [ctypes.c_int, _ip, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, _dp, _dp, _dp]
    lib.fvo_swe_batch_max_eigenvalue.restype = ctypes.c_int
    lib.fvo_swe_batch_max_eigenvalue.argtypes = [ctypes.c_int, _ip, ctypes.c_double, _dp, _dp]
    lib.fvo_halo_exchange.restype = ctypes.c_int
    lib.fvo_halo_exchange.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _ip, _dp]
    lib.fvo_num_threads.restype = ctypes.c_int
    lib.fvo_num_threads.argtypes = []
    lib.fvo_set_num_threads.restype = None
    lib.fvo_set_num_threads.argtypes = [ctypes.c_int]
    return lib


_override = None


def _load():
    global _lib
    if _override is not None:
        return _override
    with _lock:
        if _lib is None:
            _lib = bind(build())
    return _lib


class use_library:
    """Context manager: route this module's functions to another build of the
    oracle (the mutation tests use it to check that the pins catch planted
    mistakes)."""

    def __init__(self, path: str):
        self.lib = bind(path)

    def __enter__(self):
        global _override
        self._prev = _override
        _override = self.lib
        return self

    def __exit__(self, *exc):
        global _override
        _override = self._prev
        return False


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(-1))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))


def _ptr_i(a):
    return a.ctypes.data_as(_ip)


def _ptr_d(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError("oracle %s failed with code %d" % (what, rc))


def state_elems(dim: int, patch_size) -> int:
    """Number of doubles in a halo-inclusive batch state."""
    p = _i32(patch_size)
    return int(_load().fvo_state_elems(dim, len(p), _ptr_i(p)))


def patch_offsets(dim: int, patch_size) -> np.ndarray:
    """Element offset of every patch (T+1 entries), by the layout rule."""
    p = np.asarray(patch_size, dtype=np.int64).reshape(-1)
    sizes = (dim + 2) * (p + 2) ** dim
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def batch_step(dim, patch_size, dx, dt, Q, gamma=1.4, halo_mode=FIXED):
    """One explicit step.  Returns (Q_new, lambda_max of Q_new per patch)."""
    lib = _load()
    p = _i32(patch_size)
    T = len(p)
    Q = _f64(Q)
    out = np.empty_like(Q)
    lam = np.empty(T, dtype=np.float64)
    dx = _f64(np.broadcast_to(np.asarray(dx, dtype=np.float64), (T,)))
    dt = _f64(np.broadcast_to(np.asarray(dt, dtype=np.float64), (T,)))
    _check(lib.fvo_batch_step(dim, T, _ptr_i(p), _ptr_d(dx), _ptr_d(dt), gamma,
                              halo_mode, _ptr_d(Q), _ptr_d(out), _ptr_d(lam)), "step")
    return out, lam


def batch_max_eigenvalue(dim, patch_size, Q, gamma=1.4):
    """Per-patch maximum of |u_n| + c over interior volumes and directions."""
    lib = _load()
    p = _i32(patch_size)
    Q = _f64(Q)
    lam = np.empty(len(p), dtype=np.float64)
    _check(lib.fvo_batch_max_eigenvalue(dim, len(p), _ptr_i(p), gamma, _ptr_d(Q),
                                        _ptr_d(lam)), "max_eigenvalue")
    return lam


def cfl_time_step(dim, lam, dx, cfl):
    """dt = cfl * h / (d * lambda), per patch."""
    lam = _f64(lam)
    T = len(lam)
    dx = _f64(np.broadcast_to(np.asarray(dx, dtype=np.float64), (T,)))
    out = np.empty(T, dtype=np.float64)
    _load().fvo_cfl_time_step(dim, T, _ptr_d(lam), _ptr_d(dx), cfl, _ptr_d(out))
    return out


def batch_run(dim, patch_size, dx, Q, steps, gamma=1.4, halo_mode=FIXED, cfl=0.4):
    """``steps`` steps with per-patch CFL dt chaining, starting from
    dt_0 = cfl h / (d lambda(Q)).  Returns (Q_final, lambda_final, dt_next)."""
    lib = _load()
    p = _i32(patch_size)
    T = len(p)
    Q = _f64(Q).copy()
    dx = _f64(np.broadcast_to(np.asarray(dx, dtype=np.float64), (T,)))
    lam = np.empty(T, dtype=np.float64)
    dt = np.empty(T, dtype=np.float64)
    _check(lib.fvo_batch_run(dim, T, _ptr_i(p), _ptr_d(dx), gamma, halo_mode, cfl,
                             int(steps), _ptr_d(Q), _ptr_d(lam), _ptr_d(dt)), "run")
    return Q, lam, dt


def batch_totals(dim, patch_size, Q):
    """Per-patch interior sums of each unknown, shape (T, d+2)."""
    lib = _load()
    p = _i32(patch_size)
    Q = _f64(Q)
    out = np.empty(len(p) * (dim + 2), dtype=np.float64)
    _check(lib.fvo_batch_totals(dim, len(p), _ptr_i(p), _ptr_d(Q), _ptr_d(out)), "totals")
    return out.reshape(len(p), dim + 2)


def halo_exchange(dim, patch_size, neighbours, Q):
    """Copy of Q with every face halo that has a neighbour filled from the
    neighbour's interior (neighbours: [T, 2*dim], order -x,+x,-y,+y[,-z,+z],
    -1 = keep)."""
    lib = _load()
    p = _i32(patch_size)
    nb = _i32(neighbours)
    Q = _f64(Q).copy()
    _check(lib.fvo_halo_exchange(dim, len(p), _ptr_i(p), _ptr_i(nb), _ptr_d(Q)), "halo_exchange")
    return Q


def num_threads() -> int:
    """Threads the oracle's batch loops run on."""
    return int(_load().fvo_num_threads())


def set_num_threads(n: int) -> None:
    """Run the following batch loops on n threads (n < 1: the default)."""
    _load().fvo_set_num_threads(int(n))


def swe_batch_step(patch_size, dx, dt, Q, g=9.81, f=0.0, halo_mode=FIXED):
    """One shallow water step (Eq. 1 with B and S, readings R13-R15) over a
    batch of 2D patches of Q = (h, hu, hv, b); returns (Q_new, lambda_new)."""
    p = _i32(patch_size)
    T = len(p)
    Q = _f64(Q)
    out = np.empty_like(Q)
    lam = np.empty(T)
    _check(_load().fvo_swe_batch_step(T, _ptr_i(p), _ptr_d(_f64(dx)), _ptr_d(_f64(dt)), float(g), float(f),
                                      int(halo_mode), _ptr_d(Q), _ptr_d(out), _ptr_d(lam)), "swe_batch_step")
    return out, lam


def swe_batch_max_eigenvalue(patch_size, Q, g=9.81):
    p = _i32(patch_size)
    lam = np.empty(len(p))
    _check(_load().fvo_swe_batch_max_eigenvalue(len(p), _ptr_i(p), float(g), _ptr_d(_f64(Q)), _ptr_d(lam)),
           "swe_batch_max_eigenvalue")
    return lam
