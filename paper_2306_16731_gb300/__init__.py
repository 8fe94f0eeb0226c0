"""GB300-native (sm_103a) batched finite-volume patch update.

One explicit time step of many small Cartesian patches with a one-volume
halo: Rusanov face fluxes on the compressible Euler equations, the volume
update and the per-patch CFL eigenvalue (arXiv:2306.16731).  The compute
path is the CUDA library ``libfvbatch.so`` (C ABI in ``include/fv_batch.h``)
reached through the ctypes binding in :mod:`.fvbatch`.

Submodules are imported lazily so that the input generators
(:mod:`.inputs`) can be used without the compiled library.
"""

__all__ = ["build", "fvbatch", "inputs"]
