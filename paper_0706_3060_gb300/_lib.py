"""ctypes binding of libnbody.so (the C ABI declared in include/nbody.h).

Argument marshalling only: every numerical step runs in the library's CUDA
kernels. Loading fails loudly if the library has not been built; there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnbody.so")

NBODY_OK = 0
STATUS = {0: "NBODY_OK", 1: "NBODY_EINVAL", 2: "NBODY_EALIGN", 3: "NBODY_ENOMEM",
          4: "NBODY_ECUDA", 5: "NBODY_ETIMEOUT", 6: "NBODY_EUNSUPPORTED"}

LAW_GRAV = 0
LAW_LJC = 1
LAW_LJC_LINEAR = 2
TABLE_BATCHED = 3  # tile table of the batched mixed-law kernel

COMPUTE_POT = 1 << 0
PRECISE_RSQRT = 1 << 1
NO_COMPENSATION = 1 << 2
ACC_VALID = 1 << 3
ACCUMULATE = 1 << 4
FIXED_POINT = 1 << 5
TABLE_GRAV_FIXED = 4  # tile table of the fixed-point gravity kernels
TABLE_VJP_GRAV = 5  # tile table of the gravity VJP kernels (nbody_adjoint*)
TABLE_VJP_LJC = 6  # tile table of the LJC VJP kernels
TABLE_JERK = 7  # tile table of the acceleration + jerk kernels
TABLE_VJP_LJC_LINEAR = 8  # tile table of the LJC(linear) VJP kernels

TILE_PACKED = 1  # nbody_tile_info kind bits
TILE_SYMMETRIC = 2

# Every symbol include/nbody.h declares.
EXPORTS = (
    "nbody_version", "nbody_last_error", "nbody_release", "nbody_check",
    "nbody_pack_grav", "nbody_pack_ljc", "nbody_forces", "nbody_step",
    "nbody_batch_plan_create", "nbody_batch_plan_destroy", "nbody_batch_plan_particles",
    "nbody_batch_run", "nbody_forces_batched", "nbody_adjoint", "nbody_adjoint_leapfrog",
    "nbody_tile_count", "nbody_tile_info", "nbody_set_tuned", "nbody_get_config",
    "nbody_timing_enable", "nbody_timing_read", "nbody_peak_probe", "nbody_forces_static",
    "nbody_forces_subset", "nbody_forces_jerk", "nbody_hermite_step", "nbody_selftest_timeout",
    "nbody_tune", "nbody_workspace_size",
)


class NBodyParams(ctypes.Structure):
    _fields_ = [("law", ctypes.c_int32), ("flags", ctypes.c_uint32), ("G", ctypes.c_float),
                ("eps2", ctypes.c_float), ("tile", ctypes.c_int32), ("jsplit", ctypes.c_int32)]


class NBodySystem(ctypes.Structure):
    _fields_ = [("offset", ctypes.c_int64), ("n", ctypes.c_int32), ("law", ctypes.c_int32),
                ("G", ctypes.c_float), ("eps2", ctypes.c_float), ("dt", ctypes.c_float),
                ("reserved", ctypes.c_int32)]


class NBodyError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libnbody.so (raises if it is missing: build it with build.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(
                f"{p} not found: the CUDA library must be built first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(p)
        vp, i64, i32, u32, f32, f64 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_uint32, ctypes.c_float, ctypes.c_double)
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        pp = ctypes.POINTER(NBodyParams)
        sig = {
            "nbody_version": ([], ctypes.c_int),
            "nbody_last_error": ([], ctypes.c_char_p),
            "nbody_release": ([], ctypes.c_int),
            "nbody_check": ([vp], ctypes.c_int),
            "nbody_pack_grav": ([vp, vp, vp, vp, vp, i64, vp], ctypes.c_int),
            "nbody_pack_ljc": ([vp, vp, vp, vp, f64, vp, i64, vp], ctypes.c_int),
            "nbody_forces": ([vp, vp, vp, vp, i64, pp, vp], ctypes.c_int),
            "nbody_forces_static": ([vp, vp, vp, i64, pp, vp], ctypes.c_int),
            "nbody_forces_subset": ([vp, vp, vp, i64, vp, i64, pp, vp], ctypes.c_int),
            "nbody_forces_jerk": ([vp, vp, vp, vp, i64, pp, vp], ctypes.c_int),
            "nbody_hermite_step": ([vp, vp, vp, vp, i64, f32, i32, pp, vp], ctypes.c_int),
            "nbody_selftest_timeout": ([i64, vp], ctypes.c_int),
            "nbody_step": ([vp, vp, vp, vp, i64, f32, i32, i32, vp, vp, vp, pp, vp],
                           ctypes.c_int),
            "nbody_batch_plan_create": ([ctypes.POINTER(NBodySystem), i32, u32, i32,
                                         ctypes.POINTER(vp)], ctypes.c_int),
            "nbody_batch_plan_destroy": ([vp], ctypes.c_int),
            "nbody_batch_plan_particles": ([vp], i64),
            "nbody_batch_run": ([vp, vp, vp, vp, vp, i32, u32, i32, vp], ctypes.c_int),
            "nbody_forces_batched": ([ctypes.POINTER(NBodySystem), i32, vp, vp, vp, vp, i32,
                                      u32, vp], ctypes.c_int),
            "nbody_adjoint": ([vp, vp, vp, vp, vp, vp, i32, f32, i64, pp, vp], ctypes.c_int),
            "nbody_adjoint_leapfrog": ([vp, vp, i64, i32, f32, i32, vp, vp, vp, vp, i32, pp, vp],
                                       ctypes.c_int),
            "nbody_tile_count": ([i32], ctypes.c_int),
            "nbody_tile_info": ([i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                 ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)],
                                ctypes.c_int),
            "nbody_set_tuned": ([i32, i32, i32, i32], ctypes.c_int),
            "nbody_timing_enable": ([i32], ctypes.c_int),
            "nbody_peak_probe": ([i32, i32, ctypes.POINTER(f64), ctypes.POINTER(f64)],
                                 ctypes.c_int),
            "nbody_timing_read": ([i32, ctypes.POINTER(i64), ctypes.POINTER(f64)], ctypes.c_int),
            "nbody_get_config": ([i32, i64, ctypes.POINTER(i32), ctypes.POINTER(i32)],
                                 ctypes.c_int),
            "nbody_tune": ([i32, vp, vp, i64, f32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                            ctypes.POINTER(f32), vp], ctypes.c_int),
            "nbody_workspace_size": ([pp, i64, i32, ctypes.POINTER(ctypes.c_size_t)],
                                     ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        del dp, fp
        _lib = lib
        return _lib


def check(status: int, where: str) -> None:
    """Raise NBodyError for a non-OK status, with the library's message."""
    if status != NBODY_OK:
        msg = load().nbody_last_error()
        raise NBodyError(status, where, msg.decode() if msg else "")
