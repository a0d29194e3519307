"""nbody_forces_static: the force evaluation for callers that cannot allocate
device memory (fixed budgets, foreign allocators, real-time loops). It must give
the same accelerations as nbody_forces, call after call, from its one static
scratch array. This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import workloads
from gpu_util import TOL_MAX, TOL_RMS, dev, grav_tensors, lib, ljc_tensors, rel_errors

pytestmark = pytest.mark.gpu


def _static(pos, prm, acc, params):
    from paper_0706_3060_gb300 import _lib
    L = _lib.load()
    st = L.nbody_forces_static(ctypes.c_void_p(pos.data_ptr()),
                               ctypes.c_void_p(prm.data_ptr()) if prm is not None else None,
                               ctypes.c_void_p(acc.data_ptr()), pos.shape[0],
                               ctypes.byref(params), ctypes.c_void_p(
                                   torch.cuda.current_stream().cuda_stream))
    return st


def _close(a, b):
    e = rel_errors(a[:, :3].double().cpu().numpy(), b[:, :3].double().cpu().numpy())
    assert np.sqrt(np.mean(e * e)) <= TOL_RMS and e.max() <= TOL_MAX


def test_static_scratch_matches_nbody_forces_twice():
    nb = lib()
    # two calls in a row with different inputs and sizes share the one array
    for n, seed in ((70001, 1), (3001, 2)):
        g = workloads.plummer(n, seed=seed, eps=0.01)
        pos, _ = grav_tensors(g)
        eps = float(np.float32(g.eps))
        ref = nb.forces(pos, eps=eps, pot=True)
        acc = torch.full_like(pos, float("nan"))
        p = nb.params(nb.LAW_GRAV, 1.0, eps, pot=True)
        assert _static(pos, None, acc, p) == 0
        torch.cuda.synchronize()
        _close(acc, ref)
        e = np.abs(acc[:, 3].double().cpu().numpy() - ref[:, 3].double().cpu().numpy())
        assert np.all(e <= 1e-5 * np.abs(ref[:, 3].double().cpu().numpy()))


def test_static_scratch_ljc_and_rejects_oversize():
    nb = lib()
    s = workloads.ljc_sphere(2000, seed=5)
    pos, _, prm = ljc_tensors(s)
    ref = nb.forces(pos, prm)
    for _ in range(2):
        acc = torch.zeros_like(pos)
        assert _static(pos, prm, acc, nb.params(nb.LAW_LJC)) == 0
        torch.cuda.synchronize()
        _close(acc, ref)
    # a size beyond the static scratch is refused before any GPU work
    small = torch.zeros((8, 4), device=dev())
    p = nb.params(nb.LAW_GRAV)
    from paper_0706_3060_gb300 import _lib
    L = _lib.load()
    st = L.nbody_forces_static(ctypes.c_void_p(small.data_ptr()), None,
                               ctypes.c_void_p(small.data_ptr()), 4_000_000, ctypes.byref(p),
                               None)
    assert st == 1 and b"static scratch" in L.nbody_last_error()
