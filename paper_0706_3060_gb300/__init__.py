"""GB300-native (sm_103a) all-pairs N-body forces and leapfrog, after
Elsen et al., "N-Body Simulations on GPUs" (arXiv 0706.3060).

The numerical work runs in ``libnbody.so`` (hand-written CUDA kernels behind the
C ABI of ``include/nbody.h``); this package only marshals torch tensors into
that ABI. There is no CPU fallback: calls raise if the library is not built.
"""
from . import _lib
from .checkpoint import load_state, save_state
from ._lib import (ACC_VALID, ACCUMULATE, COMPUTE_POT, FIXED_POINT, LAW_GRAV, LAW_LJC,
                   LAW_LJC_LINEAR, NO_COMPENSATION, PRECISE_RSQRT, TABLE_BATCHED,
                   TABLE_GRAV_FIXED, TABLE_JERK, TABLE_VJP_GRAV, TABLE_VJP_LJC,
                   TABLE_VJP_LJC_LINEAR, TILE_PACKED, TILE_SYMMETRIC, NBodyError)
from .api import (COULOMB_K, BatchPlan, adjoint, adjoint_leapfrog, forces, forces_batched,
                  forces_jerk, forces_subset, hermite_step,
                  get_config, pack_grav, pack_ljc, params, release, set_tuned, step, sync_check,
                  tile_count, tile_info, timing_enable, timing_read, tune_table, version,
                  workspace_size)

__all__ = [
    "ACC_VALID", "ACCUMULATE", "COMPUTE_POT", "LAW_GRAV", "LAW_LJC", "LAW_LJC_LINEAR",
    "TABLE_BATCHED", "TABLE_GRAV_FIXED", "TABLE_JERK", "TABLE_VJP_GRAV", "TABLE_VJP_LJC",
    "TABLE_VJP_LJC_LINEAR",
    "FIXED_POINT", "NO_COMPENSATION",
    "PRECISE_RSQRT", "NBodyError", "COULOMB_K", "BatchPlan", "adjoint", "adjoint_leapfrog",
    "forces", "forces_batched", "forces_jerk", "forces_subset", "hermite_step", "get_config", "pack_grav", "pack_ljc", "params", "release",
    "set_tuned", "step", "sync_check", "tile_count", "tile_info", "timing_enable",
    "timing_read", "tune_table", "version", "save_state", "load_state", "workspace_size",
]
