"""Host-side checks of the C ABI that need no GPU: the library builds, loads
and exports every entry point that ``include/*.h`` declares, and argument
validation that happens before any CUDA call returns the documented codes.
"""
from __future__ import annotations

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2306_16731_gb300 import build, fvbatch
    build.build()
    return fvbatch.load()


def _declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(fv_[a-z0-9_]+)\s*\(",
                            text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("fv_batch_create", "fv_patch_batch_update", "fv_max_eigenvalue",
                     "fv_batch_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_binding_mirrors_declared_names(lib):
    from paper_2306_16731_gb300 import fvbatch
    for n in _declared_functions():
        assert hasattr(fvbatch, n), n


def _create(lib, dim=2, sizes=(4,), halo=1, unknowns=None, precision=0, halo_mode=0, gamma=1.4,
            out=True):
    arr = (ctypes.c_int32 * len(sizes))(*sizes) if sizes is not None else None
    h = ctypes.c_void_p()
    return lib.fv_batch_create(ctypes.byref(h) if out else None, dim, len(sizes or ()), arr, halo,
                               dim + 2 if unknowns is None else unknowns, precision, halo_mode,
                               gamma, None)


@pytest.mark.parametrize("kwargs,code", [
    (dict(dim=4), -1),
    (dict(dim=1), -1),
    (dict(halo=2), -1),
    (dict(halo=0), -1),
    (dict(unknowns=5), -1),
    (dict(dim=3, unknowns=4), -1),
    (dict(precision=7), -1),
    (dict(halo_mode=3), -1),
    (dict(gamma=1.0), -1),
    (dict(gamma=float("nan")), -1),
    (dict(sizes=(4, 0, 3)), -1),
    (dict(sizes=(4, -2)), -1),
    (dict(sizes=(2000,)), -1),
    (dict(dim=3, sizes=(200,)), -1),
    (dict(out=False), -1),
])
def test_create_rejects_bad_arguments(lib, kwargs, code):
    assert _create(lib, **kwargs) == code
    assert lib.fv_last_error().decode() != ""


def test_null_batch_is_rejected_or_ignored(lib):
    assert lib.fv_batch_destroy(None) == 0
    assert lib.fv_patch_batch_update(None, None, None, None, None, None, None, 0.4) == -1
    assert lib.fv_max_eigenvalue(None, None, None) == -1
    assert lib.fv_batch_status(None) == -1
    assert lib.fv_batch_state_elems(None) == 0
    assert lib.fv_patch_batch_update_host(None, None, None, None, None, None, None, 0.4, 4) == -1
    assert lib.fv_patch_batch_run_host(None, None, None, None, None, None, None, 5, 0.4, 4) == -1


def _declared_arities():
    """Parameter count of every fv_* declaration in include/*.h."""
    arity = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"\b(fv_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S):
            params = m.group(2).strip()
            arity[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return arity


def test_binding_argument_counts_match_the_header(lib):
    """The ctypes signatures the binding registers have as many arguments as
    the header's declarations (catches a parameter added on one side only)."""
    arity = _declared_arities()
    assert set(arity) >= set(_declared_functions()) - {"fv_last_error"}
    registered = {n: getattr(lib, n).argtypes for n in arity}
    assert all(v is not None for v in registered.values()), [n for n, v in registered.items() if v is None]
    mismatched = {n: (k, len(registered[n])) for n, k in arity.items() if len(registered[n]) != k}
    assert mismatched == {}
