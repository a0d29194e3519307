"""Helpers shared by the GPU parity tests: build inputs from the seeded
workloads, convert them to the library's float4 layout, and measure the
per-particle relative error against the FP64 oracle."""
from __future__ import annotations

import numpy as np
import torch

import workloads

TOL_RMS = 1e-5   # RMS_i |a_gpu - a_ref| / |a_ref|  (FP32 pair math, compensated sums)
TOL_MAX = 1e-4   # max_i of the same


def dev():
    return torch.device("cuda", 0)


def lib():
    import paper_0706_3060_gb300 as nb
    return nb


def grav_tensors(g: workloads.GravInput, device=None):
    """pos_m, vel (n, 4) float32 on the device from the FP32-rounded input."""
    device = device or dev()
    x, v, m = g.f32()
    pos = np.concatenate([x, m[:, None]], axis=1).astype(np.float32)
    vel = np.concatenate([v, np.zeros((g.n, 1), np.float32)], axis=1)
    return (torch.from_numpy(pos).to(device).contiguous(),
            torch.from_numpy(vel).to(device).contiguous())


def ljc_tensors(s: workloads.LJCInput, device=None):
    """pos_m, vel, prm on the device; prm is packed by the library's kernel from
    the FP32-rounded per-particle q, sigma, eps (as doubles)."""
    nb = lib()
    device = device or dev()
    x, v, m, q, sig_t, eps_t = s.f32()
    pos = torch.from_numpy(np.concatenate([x, m[:, None]], 1).astype(np.float32)).to(device)
    vel = torch.from_numpy(np.concatenate([v, np.zeros((s.n, 1), np.float32)], 1)).to(device)
    qd = torch.from_numpy(q.astype(np.float64)).to(device)
    sd = torch.from_numpy(sig_t.astype(np.float64)[s.types]).to(device)
    ed = torch.from_numpy(eps_t.astype(np.float64)[s.types]).to(device)
    td = torch.from_numpy(s.types.astype(np.int32)).to(device)
    prm = nb.pack_ljc(qd, sd, ed, td, kq=ljc_kq(s))
    return pos.contiguous(), vel.contiguous(), prm


def ljc_kq(s: workloads.LJCInput) -> float:
    return 332.0637 / s.dielectric


def oracle_ljc_system(s: workloads.LJCInput):
    import oracle
    x, v, m, q, sig_t, eps_t = s.f32_as_f64()
    return oracle.LJCSystem(m, q, s.types, sig_t, eps_t, ljc_kq(s)), x, v


def rel_errors(got, ref):
    """Per-particle relative L2 error |got_i - ref_i| / |ref_i|."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    num = np.linalg.norm(got - ref, axis=1)
    den = np.linalg.norm(ref, axis=1)
    den = np.where(den == 0, 1.0, den)
    return num / den


def assert_forces_close(got, ref, rms=TOL_RMS, mx=TOL_MAX, what=""):
    e = rel_errors(got, ref)
    r, m = float(np.sqrt(np.mean(e * e))), float(e.max())
    assert r <= rms and m <= mx, f"{what}: rms rel err {r:.3e} (tol {rms}), max {m:.3e} (tol {mx})"
    return r, m


def traj_errors(got, ref):
    """Per-particle error scaled by the RMS norm of the reference."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.sqrt(np.mean(np.sum(ref * ref, axis=1)))
    e = np.linalg.norm(got - ref, axis=1) / scale
    return float(np.sqrt(np.mean(e * e))), float(e.max())


# Per-particle parity of VJPs and gradients. Each output is a sum over all
# particles of terms of both signs (J^T lambda with a random lambda, the scalar
# mass derivative), so at a few particles it cancels to nearly zero and a plain
# relative error would divide an FP32 rounding error of the size of the terms by
# a vanishing value. The denominator is floored at a fraction of the RMS output
# magnitude: 1% for 3-vector outputs, 10% for scalar ones (which cancel more).
FLOOR_VEC = 0.01
FLOOR_SCALAR = 0.1
GRAD_TOL_RMS = 1e-4  # reverse-leapfrog gradients: FP32 x_T against a 0.01 residual
GRAD_TOL_MAX = 1e-3


def floored_errors(got, ref, floor):
    """|got_i - ref_i| / max(|ref_i|, floor * RMS_j |ref_j|), per particle (row)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    n = ref.shape[0]
    got = got.reshape(n, -1)
    ref = ref.reshape(n, -1)
    num = np.linalg.norm(got - ref, axis=1)
    den = np.linalg.norm(ref, axis=1)
    rms = float(np.sqrt(np.mean(den * den)))
    return num / np.maximum(den, max(floor * rms, 1e-300))


def assert_per_particle(got, ref, floor, rms=TOL_RMS, mx=TOL_MAX, what=""):
    """RMS and max of floored_errors within (rms, mx); returns them."""
    e = floored_errors(got, ref, floor)
    r, m = float(np.sqrt(np.mean(e * e))), float(e.max())
    assert r <= rms and m <= mx, (f"{what}: per-particle rms {r:.3e} (tol {rms}), "
                                  f"max {m:.3e} (tol {mx}), floor {floor}")
    return r, m


def assert_vjp_close(gx, gm, rg, rm, what=""):
    """A force VJP (J^T lambda, mass derivative) against the oracle, per particle."""
    assert_per_particle(gx, rg, FLOOR_VEC, what=f"{what} J^T lambda")
    assert_per_particle(gm, rm, FLOOR_SCALAR, what=f"{what} d/dm")


def assert_types_close(got_t, rs, re, rtol=1e-4, what=""):
    """Per-type sigma and epsilon derivatives (2 x ntypes), each entry against its
    own magnitude floored at 10% of the RMS of its kind."""
    got_t = np.asarray(got_t, dtype=np.float64)
    nt = len(rs)
    assert_per_particle(got_t[:nt], rs, FLOOR_SCALAR, rms=rtol, mx=rtol, what=f"{what} d/dsigma")
    assert_per_particle(got_t[nt:], re, FLOOR_SCALAR, rms=rtol, mx=rtol, what=f"{what} d/deps")


def assert_grads_close(gx, gv, gm, ref, what=""):
    """Reverse-leapfrog gradients against the oracle's, per particle."""
    assert_per_particle(gx, ref["x0"], FLOOR_SCALAR, GRAD_TOL_RMS, GRAD_TOL_MAX, f"{what} dL/dx0")
    assert_per_particle(gv, ref["v0"], FLOOR_SCALAR, GRAD_TOL_RMS, GRAD_TOL_MAX, f"{what} dL/dv0")
    assert_per_particle(gm, ref["m"], FLOOR_SCALAR, GRAD_TOL_RMS, GRAD_TOL_MAX, f"{what} dL/dm")


def as_f32(a):
    """FP64 copy of the FP32 rounding of `a` (what the GPU side was given)."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)
