"""nbody_forces_static: the force evaluation for callers that cannot allocate
device memory -- code under a memory budget fixed at start-up, a process whose
device allocator belongs to another framework, or a real-time loop that must not
block in cudaMalloc. Its scratch is one static array inside the library, shared
by every call.

Checked here, through the C ABI: per-particle parity with the FP64 oracle and
agreement with nbody_forces on two calls in a row (and a repeat of the first,
bit for bit, after another call has overwritten the array); the sizes where the
tuned symmetric tile falls back to a one-sided tile whose automatic j-split would
not fit (the plan must shrink it); that a call allocates nothing; and that a
timeout recorded on the device before a call is still reported by nbody_check
after it. This file is collected last on purpose, so that a run stopping at the
first failure has run every other test first."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_util import (TOL_MAX, TOL_RMS, assert_forces_close, dev, grav_tensors, lib,
                      ljc_tensors, oracle_ljc_system)

pytestmark = pytest.mark.gpu


def _L():
    from paper_0706_3060_gb300 import api
    return api._lib()  # the library, with the stored tuning table installed


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _static(pos, prm, acc, params):
    return _L().nbody_forces_static(ctypes.c_void_p(pos.data_ptr()),
                                    ctypes.c_void_p(prm.data_ptr()) if prm is not None else None,
                                    ctypes.c_void_p(acc.data_ptr()), pos.shape[0],
                                    ctypes.byref(params), _stream())


def _run_static(pos, prm, params):
    acc = torch.full_like(pos, float("nan"))
    assert _static(pos, prm, acc, params) == 0, _L().nbody_last_error()
    assert _L().nbody_check(_stream()) == 0, _L().nbody_last_error()
    return acc


def _grav_case(n, seed):
    g = workloads.plummer(n, seed=seed, eps=0.01)
    pos, _ = grav_tensors(g)
    x, _, m = g.f32_as_f64()
    return g, pos, x, m, float(np.float32(g.eps))


def test_static_matches_oracle_and_nbody_forces_twice():
    nb = lib()
    cases = [_grav_case(70001, 1), _grav_case(3001, 2)]
    first = None
    for k, (g, pos, x, m, eps) in enumerate(cases):
        p = nb.params(nb.LAW_GRAV, 1.0, eps, pot=True)
        acc = _run_static(pos, None, p)
        if k == 0:
            first = acc.clone()
        got = acc.double().cpu().numpy()
        idx = np.random.default_rng(k).choice(g.n, size=min(g.n, 1024), replace=False)
        ref_a, ref_phi = oracle.grav_accel(x, m, eps=eps, idx=idx, potential=True)
        assert_forces_close(got[idx, :3], ref_a, what=f"static vs oracle n={g.n}")
        assert np.all(np.abs(got[idx, 3] - ref_phi) <= 1e-5 * np.abs(ref_phi))
        # and against the allocating entry point on every particle
        ref = nb.forces(pos, eps=eps, pot=True).double().cpu().numpy()
        assert_forces_close(got[:, :3], ref[:, :3], what=f"static vs nbody_forces n={g.n}")
    # the array now holds the second call's data: repeating the first call gives
    # the same bits as before
    again = _run_static(cases[0][1], None, nb.params(nb.LAW_GRAV, 1.0, cases[0][4], pot=True))
    assert torch.equal(again, first)


@pytest.mark.parametrize("law", ["ljc", "ljclin"])
def test_static_ljc_twice_against_oracle(law):
    nb = lib()
    s = workloads.ljc_sphere(2000, seed=5)
    if law == "ljc":
        pos, _, prm = ljc_tensors(s)
        sysm, x, _ = oracle_ljc_system(s)
        code = nb.LAW_LJC
    else:
        K = 332.0637
        xf, _, mf, q, st, et = s.f32()
        pos = torch.from_numpy(np.concatenate([xf, mf[:, None]], 1).astype(np.float32)).to(dev())
        prm = nb.pack_ljc(torch.from_numpy(q.astype(np.float64)).to(dev()),
                          torch.from_numpy(st.astype(np.float64)[s.types]).to(dev()),
                          torch.from_numpy(et.astype(np.float64)[s.types]).to(dev()),
                          torch.from_numpy(s.types).to(dev()), kq=K / 4.0)
        x, _, md, qd, sd, ed = s.f32_as_f64()
        sysm = oracle.LJCSystem(md, qd, s.types, sd, ed, K / 4.0, linear=True)
        code = nb.LAW_LJC_LINEAR
    ref = sysm.accel(x)
    for _ in range(2):
        acc = _run_static(pos.contiguous(), prm, nb.params(code))
        assert_forces_close(acc[:, :3].double().cpu().numpy(), ref, what=f"static {law}")
        assert_forces_close(acc[:, :3].double().cpu().numpy(),
                            nb.forces(pos.contiguous(), prm, law=code)[:, :3].double().cpu().numpy(),
                            what=f"static vs nbody_forces {law}")


@pytest.mark.parametrize("n", [131072, 262144, 524288])
def test_static_shrinks_the_split_where_the_tuned_tile_is_symmetric(n):
    """With a symmetric tile as the tuned choice the call falls back to a
    one-sided tile and must cut its automatic j-split to what the scratch holds."""
    nb = lib()
    sym = [t for t in range(nb.tile_count(nb.LAW_GRAV))
           if nb.tile_info(nb.LAW_GRAV, t)["symmetric"]][-1]
    old = nb.get_config(nb.LAW_GRAV, n)
    nb.set_tuned(nb.LAW_GRAV, n, sym, 0)
    try:
        g = workloads.plummer(n, seed=11, eps=workloads.plummer_softening(n))
        pos, _ = grav_tensors(g)
        eps = float(np.float32(g.eps))
        acc = _run_static(pos, None, nb.params(nb.LAW_GRAV, 1.0, eps))
        x, _, m = g.f32_as_f64()
        idx = np.random.default_rng(n).choice(n, size=512, replace=False)
        ref = oracle.grav_accel(x, m, eps=eps, idx=idx)
        assert_forces_close(acc[idx, :3].double().cpu().numpy(), ref, what=f"static n={n}")
    finally:
        nb.set_tuned(nb.LAW_GRAV, n, old[0], old[1])


def test_static_allocates_nothing():
    nb = lib()
    g, pos, _, _, eps = _grav_case(262144, 3)
    p = nb.params(nb.LAW_GRAV, 1.0, eps)
    acc = torch.empty_like(pos)
    assert _static(pos, None, acc, p) == 0  # warm-up: modules loaded, address looked up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    allocs0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for _ in range(2):
        assert _static(pos, None, acc, p) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == allocs0
    assert torch.all(torch.isfinite(acc))


def test_recorded_timeout_survives_a_static_call():
    """A bounded wait that ran out (the self-test's mbarrier that nothing
    completes) is recorded in the device error word; a following static call
    must not clear it, and nbody_check reports it once."""
    nb = lib()
    L = _L()
    g, pos, _, _, eps = _grav_case(5000, 4)
    p = nb.params(nb.LAW_GRAV, 1.0, eps)
    acc = torch.empty_like(pos)
    assert L.nbody_check(_stream()) == 0
    assert L.nbody_selftest_timeout(2_000_000, _stream()) == 0
    assert _static(pos, None, acc, p) == 0
    assert L.nbody_check(_stream()) == 5  # NBODY_ETIMEOUT
    assert L.nbody_check(_stream()) == 0
    assert _static(pos, None, acc, p) == 0
    assert L.nbody_check(_stream()) == 0


def test_static_rejects_oversize_and_symmetric_tiles():
    nb = lib()
    L = _L()
    small = torch.zeros((8, 4), device=dev())
    p = nb.params(nb.LAW_GRAV)
    st = L.nbody_forces_static(ctypes.c_void_p(small.data_ptr()), None,
                               ctypes.c_void_p(small.data_ptr()), 4_000_000, ctypes.byref(p),
                               None)
    assert st == 1 and b"static scratch" in L.nbody_last_error()
    sym = [t for t in range(nb.tile_count(nb.LAW_GRAV))
           if nb.tile_info(nb.LAW_GRAV, t)["symmetric"]][0]
    p = nb.params(nb.LAW_GRAV, tile=sym)
    assert _static(small, None, small, p) == 1
    assert b"one-sided" in L.nbody_last_error()
