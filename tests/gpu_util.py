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
