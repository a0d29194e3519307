"""Python API over the C ABI: same names as include/nbody.h, torch tensors in.

PyTorch supplies device memory and the current CUDA stream; every numerical
step runs in libnbody.so. Tensors must be contiguous float32 ``(n, 4)``
(positions/masses ``pos_m``, velocities, accelerations, LJC parameters
``prm``), on the GPU, or -- for :func:`forces` and :func:`step` -- all on the
host, in which case the library stages them through device memory.
"""
from __future__ import annotations

import ctypes
import math

import torch

from . import _lib
from ._lib import (ACC_VALID, ACCUMULATE, COMPUTE_POT, FIXED_POINT, LAW_GRAV, LAW_LJC,
                   LAW_LJC_LINEAR, NO_COMPENSATION, PRECISE_RSQRT, TILE_PACKED, TILE_SYMMETRIC,
                   NBodyParams, NBodySystem, check, load)

COULOMB_K = 332.0637  # kcal A / (mol e^2): units A, kcal/mol, e, amu (AKMA time)


_tuned_done = False


def _lib():
    """The loaded library, with the stored tuning table of this GPU installed once."""
    global _tuned_done
    lib = load()
    if not _tuned_done:
        _tuned_done = True
        try:
            from . import tune
            tune.load_cache()
        except Exception:  # a missing or foreign cache only means default tiles
            pass
    return lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None, device=None):
    if stream is not None:
        return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)
    if device is not None and device.type == "cuda":
        return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    return ctypes.c_void_p(0)


def _check4(t, name):
    if t is None:
        return
    if t.dtype != torch.float32 or t.dim() != 2 or t.shape[1] != 4 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 (n, 4) tensor")


def params(law=LAW_GRAV, G=1.0, eps=0.0, pot=False, precise=False, compensated=True,
           tile=-1, jsplit=0, acc_valid=False, accumulate=False, fixed=False) -> NBodyParams:
    flags = FIXED_POINT if fixed else 0
    flags |= COMPUTE_POT if pot else 0
    flags |= PRECISE_RSQRT if precise else 0
    flags |= 0 if compensated else NO_COMPENSATION
    flags |= ACC_VALID if acc_valid else 0
    flags |= ACCUMULATE if accumulate else 0
    return NBodyParams(int(law), flags, float(G), float(eps) ** 2, int(tile), int(jsplit))


def version() -> int:
    return load().nbody_version()


def release() -> None:
    check(load().nbody_release(), "nbody_release")


def sync_check(stream=None) -> None:
    """Synchronize and raise if a kernel recorded an error (e.g. a timeout)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    check(load().nbody_check(_stream(stream, dev)), "nbody_check")


# ---------------------------------------------------------------------------
# Packing
# ---------------------------------------------------------------------------
def pack_grav(x: torch.Tensor, m: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """(n, 3) float64 positions and (n,) float64 masses on the GPU -> (n, 4) float32."""
    x = x.to(torch.float64)
    n = x.shape[0]
    cols = [x[:, k].contiguous() for k in range(3)]
    m = m.to(torch.float64).contiguous()
    out = torch.empty((n, 4), dtype=torch.float32, device=x.device) if out is None else out
    check(load().nbody_pack_grav(_ptr(cols[0]), _ptr(cols[1]), _ptr(cols[2]), _ptr(m), _ptr(out),
                                 n, _stream(stream, x.device)), "nbody_pack_grav")
    return out


def pack_ljc(q, sigma, eps, types, kq=COULOMB_K / 80.0, out=None, stream=None):
    """Per-particle charges, sigma, epsilon (float64) and int32 types on the GPU ->
    (n, 4) float32 prm = (q sqrt(kq), sigma / 2, sqrt(24 eps), type)."""
    q = q.to(torch.float64).contiguous()
    sigma = sigma.to(torch.float64).contiguous()
    eps = eps.to(torch.float64).contiguous()
    types = types.to(torch.int32).contiguous()
    n = q.shape[0]
    out = torch.empty((n, 4), dtype=torch.float32, device=q.device) if out is None else out
    check(load().nbody_pack_ljc(_ptr(q), _ptr(sigma), _ptr(eps), _ptr(types), float(kq),
                                _ptr(out), n, _stream(stream, q.device)), "nbody_pack_ljc")
    return out


# ---------------------------------------------------------------------------
# Forces and leapfrog
# ---------------------------------------------------------------------------
def forces(pos_m, prm=None, *, law=None, G=1.0, eps=0.0, pot=False, precise=False,
           compensated=True, tile=-1, jsplit=0, out=None, out_lo=None, want_lo=False,
           fixed=False, stream=None):
    """One all-pairs force evaluation. Returns acc (n, 4) = (ax, ay, az, phi), or
    (acc, acc_lo) with ``want_lo``."""
    _check4(pos_m, "pos_m")
    _check4(prm, "prm")
    law = (LAW_LJC if prm is not None else LAW_GRAV) if law is None else law
    n = pos_m.shape[0]
    acc = torch.empty_like(pos_m) if out is None else out
    lo = (torch.empty_like(pos_m) if out_lo is None else out_lo) if want_lo else None
    p = params(law, G, eps, pot, precise, compensated, tile, jsplit, fixed=fixed)
    check(_lib().nbody_forces(_ptr(pos_m), _ptr(prm), _ptr(acc), _ptr(lo), n, ctypes.byref(p),
                              _stream(stream, pos_m.device)), "nbody_forces")
    return (acc, lo) if want_lo else acc


def forces_subset(pos_m, idx, prm=None, *, law=None, G=1.0, eps=0.0, pot=False, precise=False,
                  compensated=True, tile=-1, jsplit=0, out=None, stream=None):
    """Forces on the particles ``idx`` (int32 tensor of indices) against all
    particles: returns (len(idx), 4) accelerations in the order of ``idx``."""
    _check4(pos_m, "pos_m")
    _check4(prm, "prm")
    law = (LAW_LJC if prm is not None else LAW_GRAV) if law is None else law
    idx = idx.to(torch.int32).contiguous()
    acc = torch.empty((idx.shape[0], 4), dtype=torch.float32, device=pos_m.device) \
        if out is None else out
    p = params(law, G, eps, pot, precise, compensated, tile, jsplit)
    check(_lib().nbody_forces_subset(_ptr(pos_m), _ptr(prm), _ptr(idx), idx.shape[0], _ptr(acc),
                                     pos_m.shape[0], ctypes.byref(p),
                                     _stream(stream, pos_m.device)), "nbody_forces_subset")
    return acc


def forces_jerk(pos_m, vel, *, G=1.0, eps=0.0, compensated=True, tile=-1, jsplit=0,
                fixed=False, stream=None):
    """Acceleration and jerk (Table 1 GAJ): returns (acc, jerk), each (n, 4).
    ``tile`` indexes tile table 7 (-1: tuned/default). ``fixed=True`` (eps > 0):
    the symmetric tiles add their per-block partials exactly in fixed point."""
    _check4(pos_m, "pos_m")
    _check4(vel, "vel")
    acc = torch.empty_like(pos_m)
    jerk = torch.empty_like(pos_m)
    p = params(LAW_GRAV, G, eps, compensated=compensated, tile=tile, jsplit=jsplit,
               fixed=fixed)
    check(_lib().nbody_forces_jerk(_ptr(pos_m), _ptr(vel), _ptr(acc), _ptr(jerk), pos_m.shape[0],
                                   ctypes.byref(p), _stream(stream, pos_m.device)),
          "nbody_forces_jerk")
    return acc, jerk


def hermite_step(pos_m, vel, acc, jerk, *, dt, nsteps=1, G=1.0, eps=0.0, acc_valid=False,
                 compensated=True, tile=-1, jsplit=0, fixed=False, stream=None):
    """``nsteps`` fourth-order Hermite steps in place; acc/jerk receive (a, j) at exit."""
    for t, nm in ((pos_m, "pos_m"), (vel, "vel"), (acc, "acc"), (jerk, "jerk")):
        _check4(t, nm)
    p = params(LAW_GRAV, G, eps, compensated=compensated, acc_valid=acc_valid, tile=tile,
               jsplit=jsplit, fixed=fixed)
    check(_lib().nbody_hermite_step(_ptr(pos_m), _ptr(vel), _ptr(acc), _ptr(jerk),
                                    pos_m.shape[0], float(dt), int(nsteps), ctypes.byref(p),
                                    _stream(stream, pos_m.device)), "nbody_hermite_step")


def step(pos_m, vel, acc, prm=None, *, dt, nsteps=1, law=None, G=1.0, eps=0.0,
         report_every=0, acc_valid=False, pot=False, precise=False, compensated=True,
         tile=-1, jsplit=0, trace=None, diag=None, state_lo=None, fixed=False, stream=None):
    """``nsteps`` KDK leapfrog steps in place on (pos_m, vel); acc receives a(x_T).

    ``state_lo`` (2n, 4) float32, zero-initialised by the caller, turns on the
    compensated two-float state update (low parts of x, then of v).

    Returns the FP64 diagnostics (rows of K, U, Px, Py, Pz, Lx, Ly, Lz) as a
    float64 tensor when ``report_every`` > 0, else None.
    """
    for t, nm in ((pos_m, "pos_m"), (vel, "vel"), (acc, "acc"), (prm, "prm"), (trace, "trace")):
        if t is not None and nm != "trace":
            _check4(t, nm)
    law = (LAW_LJC if prm is not None else LAW_GRAV) if law is None else law
    n = pos_m.shape[0]
    rows = nsteps // report_every + 1 if report_every > 0 else 0
    if rows and diag is None:
        diag = torch.zeros((rows, 8), dtype=torch.float64, device=pos_m.device)
    p = params(law, G, eps, pot, precise, compensated, tile, jsplit, acc_valid, fixed=fixed)
    check(_lib().nbody_step(_ptr(pos_m), _ptr(vel), _ptr(acc), _ptr(prm), n, float(dt),
                            int(nsteps), int(report_every), _ptr(diag) if rows else None,
                            _ptr(trace), _ptr(state_lo), ctypes.byref(p),
                            _stream(stream, pos_m.device)),
          "nbody_step")
    return diag if rows else None


# ---------------------------------------------------------------------------
# Batched ensembles
# ---------------------------------------------------------------------------
class BatchPlan:
    """Work list + graph cache for many independent systems (nbody_batch_plan)."""

    def __init__(self, systems, precise=False, compensated=True, tile=-1):
        """systems: iterable of dicts with offset, n, law, G, eps, dt."""
        lib = _lib()
        systems = list(systems)
        arr = (NBodySystem * len(systems))()
        for k, s in enumerate(systems):
            arr[k] = NBodySystem(int(s["offset"]), int(s["n"]), int(s["law"]),
                                 float(s.get("G", 1.0)), float(s.get("eps", 0.0)) ** 2,
                                 float(s["dt"]), 0)
        flags = (PRECISE_RSQRT if precise else 0) | (0 if compensated else NO_COMPENSATION)
        h = ctypes.c_void_p()
        check(lib.nbody_batch_plan_create(arr, len(systems), flags, int(tile), ctypes.byref(h)),
              "nbody_batch_plan_create")
        self._h = h
        self.systems = systems
        self.total = int(lib.nbody_batch_plan_particles(h))

    def run(self, pos_m, vel, acc, prm=None, nsteps=0, acc_valid=False, graph=True,
            stream=None):
        check(load().nbody_batch_run(self._h, _ptr(pos_m), _ptr(vel), _ptr(acc), _ptr(prm),
                                     int(nsteps), ACC_VALID if acc_valid else 0, int(bool(graph)),
                                     _stream(stream, pos_m.device)), "nbody_batch_run")

    def close(self):
        if getattr(self, "_h", None):
            load().nbody_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def forces_batched(systems, pos_m, vel, acc, prm=None, nsteps=0, acc_valid=False, stream=None):
    """One-shot batched run (plan, run, destroy); synchronizes."""
    lib = _lib()
    systems = list(systems)
    arr = (NBodySystem * len(systems))()
    for k, s in enumerate(systems):
        arr[k] = NBodySystem(int(s["offset"]), int(s["n"]), int(s["law"]), float(s.get("G", 1.0)),
                             float(s.get("eps", 0.0)) ** 2, float(s["dt"]), 0)
    check(lib.nbody_forces_batched(arr, len(systems), _ptr(pos_m), _ptr(vel), _ptr(acc),
                                   _ptr(prm), int(nsteps), ACC_VALID if acc_valid else 0,
                                   _stream(stream, pos_m.device)), "nbody_forces_batched")


# ---------------------------------------------------------------------------
# Adjoint
# ---------------------------------------------------------------------------
def adjoint(pos_m, lam, prm=None, *, law=None, G=1.0, eps=0.0, alpha=1.0, grad_x=None,
            grad_m=None, grad_types=None, ntypes=4, accumulate=False, tile=-1, jsplit=0,
            compensated=True, fixed=False, stream=None):
    """One force VJP: returns (grad_x (n,4), grad_m (n,), grad_types (2*ntypes,) or None).
    ``tile`` indexes tile table 5 (gravity), 6 (LJC) or 8 (LJC linear); -1:
    tuned/default. ``compensated=False`` sets NBODY_NO_COMPENSATION (plain FP32
    per-tile sums); ``fixed=True`` sets NBODY_FIXED_POINT (gravity, eps > 0: the
    symmetric tiles add their per-block partials exactly in fixed point)."""
    _check4(pos_m, "pos_m")
    _check4(lam, "lam")
    law = (LAW_LJC if prm is not None else LAW_GRAV) if law is None else law
    n = pos_m.shape[0]
    dev = pos_m.device
    gx = torch.zeros_like(pos_m) if grad_x is None else grad_x
    gm = torch.zeros(n, dtype=torch.float32, device=dev) if grad_m is None else grad_m
    gt = grad_types
    if gt is None and law in (LAW_LJC, LAW_LJC_LINEAR):
        gt = torch.zeros(2 * ntypes, dtype=torch.float64, device=dev)
    p = params(law, G, eps, compensated=compensated, accumulate=accumulate, tile=tile,
               jsplit=jsplit, fixed=fixed)
    check(_lib().nbody_adjoint(_ptr(pos_m), _ptr(prm), _ptr(lam), _ptr(gx), _ptr(gm), _ptr(gt),
                               int(ntypes), float(alpha), n, ctypes.byref(p),
                               _stream(stream, dev)), "nbody_adjoint")
    return gx, gm, gt


def adjoint_leapfrog(xs, lam_x, lam_v, prm=None, *, k, dt, first, law=None, G=1.0, eps=0.0,
                     grad_m=None, grad_types=None, ntypes=4, tile=-1, jsplit=0, stream=None):
    """Reverse sweep over k stored positions xs ((k or more) * n, 4); updates
    lam_x, lam_v, grad_m, grad_types in place."""
    n = lam_x.shape[0]
    law = (LAW_LJC if prm is not None else LAW_GRAV) if law is None else law
    p = params(law, G, eps, tile=tile, jsplit=jsplit)
    check(_lib().nbody_adjoint_leapfrog(_ptr(xs), _ptr(prm), n, int(k), float(dt), int(first),
                                        _ptr(lam_x), _ptr(lam_v), _ptr(grad_m), _ptr(grad_types),
                                        int(ntypes), ctypes.byref(p),
                                        _stream(stream, lam_x.device)),
          "nbody_adjoint_leapfrog")


# ---------------------------------------------------------------------------
# Tiles / tuning
# ---------------------------------------------------------------------------
def tile_count(law: int) -> int:
    c = load().nbody_tile_count(int(law))
    if c < 0:
        check(-c, "nbody_tile_count")
    return c


def tile_info(law: int, tile: int) -> dict:
    vals = [ctypes.c_int32() for _ in range(5)]
    check(load().nbody_tile_info(int(law), int(tile), *[ctypes.byref(v) for v in vals]),
          "nbody_tile_info")
    d = dict(zip(("threads", "i_per_thread", "j_lanes", "j_tile", "kind"),
                 (v.value for v in vals)))
    d["packed"] = bool(d["kind"] & TILE_PACKED)
    d["symmetric"] = bool(d["kind"] & TILE_SYMMETRIC)
    return d


def set_tuned(law: int, n: int, tile: int, jsplit: int = 0) -> None:
    check(load().nbody_set_tuned(int(law), int(math.floor(math.log2(max(n, 1)))), int(tile),
                                 int(jsplit)), "nbody_set_tuned")


def get_config(law: int, n: int) -> tuple[int, int]:
    t, j = ctypes.c_int32(), ctypes.c_int32()
    check(_lib().nbody_get_config(int(law), int(n), ctypes.byref(t), ctypes.byref(j)),
          "nbody_get_config")
    return t.value, j.value


def workspace_size(n: int, *, law=LAW_GRAV, eps=0.0, tile=-1, jsplit=0, fixed=False,
                   compensated=True, report_rows=0) -> int:
    """Device scratch bytes a forces/step call with these settings requests from
    the library's per-stream workspace (nbody_workspace_size)."""
    b = ctypes.c_size_t()
    p = params(law, 1.0, eps, compensated=compensated, tile=tile, jsplit=jsplit, fixed=fixed)
    check(_lib().nbody_workspace_size(ctypes.byref(p), int(n), int(report_rows), ctypes.byref(b)),
          "nbody_workspace_size")
    return b.value


def tune_table(table: int, pos_m, prm=None, *, eps=0.01, reps=5, stream=None) -> dict:
    """Autotune tile table ``table`` at n = len(pos_m) in the library (nbody_tune):
    installs and returns the fastest (tile, jsplit) with its median milliseconds."""
    _check4(pos_m, "pos_m")
    t, j, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    check(_lib().nbody_tune(int(table), _ptr(pos_m), _ptr(prm), pos_m.shape[0], float(eps) ** 2,
                            int(reps), ctypes.byref(t), ctypes.byref(j), ctypes.byref(ms),
                            _stream(stream, pos_m.device)), "nbody_tune")
    return {"tile": t.value, "jsplit": j.value, "ms": ms.value}


# ---------------------------------------------------------------------------
# Kernel timers
# ---------------------------------------------------------------------------
def timing_enable(on: bool = True) -> None:
    check(load().nbody_timing_enable(int(bool(on))), "nbody_timing_enable")


def timing_read(which: int = 0) -> tuple[int, float]:
    """(launches, total device ms) of force (0) or VJP (1) kernels since the last read."""
    n, ms = ctypes.c_int64(), ctypes.c_double()
    check(load().nbody_timing_read(int(which), ctypes.byref(n), ctypes.byref(ms)),
          "nbody_timing_read")
    return n.value, ms.value
