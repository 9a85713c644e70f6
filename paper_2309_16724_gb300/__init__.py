"""GB300 (sm_103a) SU(2) two-site DMRG H.psi and Davidson (arXiv:2309.16724).

The compute lives in ``libsu2dmrg.so`` (C++ host tables + CUDA kernels,
C-ABI in ``include/su2dmrg.h``); ``_lib`` is its ctypes binding and
``workload`` turns the seeded synthetic configurations into library calls.
"""
from ._lib import (SU2_FP64, SU2_MODEL_AB_INITIO, SU2_MODEL_CASIMIR_N, SU2_MODEL_CASIMIR_S2, SU2_MODEL_HEISENBERG,
                   SU2_MODEL_QC_SKELETON, SU2_SITE_ORBITAL, SU2_SITE_SPIN_HALF, SU2_SPLIT_BF16, SU2_SPLIT_FP8, Context,
                   Davidson, Environment, Sectors, Su2Error, Sweep, apply_heff, apply_heff_host, apply_heff_static_scratch, hash_group,
                   build_environment,
                   build_sectors, davidson_create, davidson_step, diag_heff, energy, lib)

__all__ = [
    "SU2_FP64", "SU2_SPLIT_BF16", "SU2_SPLIT_FP8", "SU2_MODEL_AB_INITIO", "SU2_MODEL_HEISENBERG", "SU2_MODEL_QC_SKELETON", "SU2_MODEL_CASIMIR_S2",
    "SU2_MODEL_CASIMIR_N", "SU2_SITE_SPIN_HALF", "SU2_SITE_ORBITAL", "Context", "Sectors", "Environment",
    "Davidson", "Su2Error", "Sweep", "apply_heff", "apply_heff_host", "apply_heff_static_scratch", "hash_group", "diag_heff", "build_sectors", "build_environment",
    "davidson_create", "davidson_step", "energy", "lib",
]
