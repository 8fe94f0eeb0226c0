"""FP64 CPU oracle for the batched finite-volume patch update.

Test infrastructure: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  It shares no code with
the CUDA library in ``paper_2306_16731_gb300``.
"""
from .fv_oracle import (  # noqa: F401
    build,
    state_elems,
    patch_offsets,
    batch_step,
    batch_max_eigenvalue,
    cfl_time_step,
    batch_run,
    batch_totals,
    halo_exchange,
    swe_batch_step,
    swe_batch_max_eigenvalue,
    num_threads,
    set_num_threads,
    FIXED,
    PERIODIC,
)
