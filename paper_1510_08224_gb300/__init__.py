"""GB300 solver for the double-distribution non-orthogonal MRT lattice
Boltzmann method for incompressible thermal flow (Liu, He, Li & Li,
arXiv:1510.08224).

The hot path is one fused CUDA kernel per time step (sm_103a) behind the C ABI
of ``include/nomrt_lbm.h``; :mod:`.lbm` is its ctypes binding.
"""
from .lbm import (BATCH_KINDS, EXPORTED, Batch, LBMError, Lattice, STORAGE, STORAGE_BYTES, SIDES, STEP_VARIANTS, load, make_params,
                  lbm_footprint_bytes, library_path, probe_fp64_rate, residual_fields_noalloc, step_kernel_count, step_kernels, validate)

__all__ = ["BATCH_KINDS", "EXPORTED", "Batch", "LBMError", "Lattice", "STORAGE", "STORAGE_BYTES", "SIDES", "STEP_VARIANTS", "load", "make_params",
           "lbm_footprint_bytes", "library_path", "probe_fp64_rate", "residual_fields_noalloc", "step_kernel_count", "step_kernels", "validate"]
