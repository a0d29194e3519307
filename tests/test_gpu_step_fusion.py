"""GPU: the launch-saving forms of nbody_step give the same bits as the plain ones.

Within one call, every step after the first reads the pair-interleaved source
copy that the previous step's finalize wrote with the drifted positions (and, for
the symmetric gravity tiles that accumulate in fixed point, the accumulators that
finalize zeroed again); a call that starts from the caller's acceleration
(acc_valid) has its first half-kick and drift done by the interleave launch; and
report steps add their FP64 diagnostics in the finalize's last block. Checks, for
every compiled tile of each law at a ragged size:

- k steps in one call equal, bit for bit, one call without steps followed by k
  calls of one step from the returned acceleration (each of which builds its
  source copy from scratch, through the fused kick-drift where the tile is packed),
  with and without the two-float state;
- the diagnostic rows equal FP64 sums over the state and potential they describe.
"""
import numpy as np
import pytest
import torch

import workloads
from gpu_util import grav_tensors, lib, ljc_tensors

pytestmark = pytest.mark.gpu

N_RAGGED = 2049   # odd: the last source pair holds the far-away massless pad
STEPS = 5


def _tiles(table):
    return list(range(lib().tile_count(table)))


def _system(law, n, seed):
    nb = lib()
    if law == nb.LAW_GRAV:
        g = workloads.plummer(n, seed=seed, eps=0.01)
        pos, vel = grav_tensors(g)
        return pos, vel, None, dict(eps=float(np.float32(g.eps)), dt=1e-3)
    s = workloads.ljc_sphere(n, seed=seed)
    pos, vel, prm = ljc_tensors(s)
    return pos, vel, prm, dict(law=law, dt=1e-4)


def _run_both(law, tile, two_float, **extra):
    nb = lib()
    pos, vel, prm, kw = _system(law, N_RAGGED, seed=61 + law)
    kw.update(extra)
    n = pos.shape[0]
    p1, v1 = pos.clone(), vel.clone()
    a1 = torch.empty_like(p1)
    lo1 = torch.zeros((2 * n, 4), device=pos.device) if two_float else None
    nb.step(p1, v1, a1, prm, nsteps=STEPS, tile=tile, state_lo=lo1, **kw)
    p2, v2 = pos.clone(), vel.clone()
    a2 = torch.empty_like(p2)
    lo2 = torch.zeros_like(lo1) if two_float else None
    nb.step(p2, v2, a2, prm, nsteps=0, tile=tile, state_lo=lo2, **kw)
    for _ in range(STEPS):
        nb.step(p2, v2, a2, prm, nsteps=1, tile=tile, acc_valid=True, state_lo=lo2, **kw)
    assert torch.equal(p1, p2), "positions"
    assert torch.equal(v1, v2), "velocities"
    assert torch.equal(a1[:, :3], a2[:, :3]), "accelerations"
    if two_float:
        assert torch.equal(lo1, lo2), "two-float low parts"


@pytest.mark.parametrize("two_float", [False, True])
def test_gravity_one_call_equals_single_steps(two_float):
    nb = lib()
    for tile in _tiles(nb.LAW_GRAV):
        _run_both(nb.LAW_GRAV, tile, two_float)


def test_gravity_symmetric_plain_sums_one_call_equals_single_steps():
    """The symmetric tiles with one partial slot per block (no fixed point)."""
    nb = lib()
    for tile in _tiles(nb.LAW_GRAV):
        if nb.tile_info(nb.LAW_GRAV, tile)["symmetric"]:
            _run_both(nb.LAW_GRAV, tile, False, compensated=False)


def test_gravity_fixed_point_one_call_equals_single_steps():
    nb = lib()
    for tile in _tiles(nb.TABLE_GRAV_FIXED):
        _run_both(nb.LAW_GRAV, tile, False, fixed=True)


@pytest.mark.parametrize("linear", [False, True])
def test_ljc_one_call_equals_single_steps(linear):
    nb = lib()
    law = nb.LAW_LJC_LINEAR if linear else nb.LAW_LJC
    for tile in _tiles(law):
        _run_both(law, tile, tile % 2 == 1)


def _diag_ref(pos, vel, acc, law):
    """K, U, P, L in FP64 from the FP32 state and potential; the scale of each row
    for the tolerance (the sum of the terms' magnitudes)."""
    x = pos[:, :3].double().cpu().numpy()
    m = pos[:, 3].double().cpu().numpy()
    v = vel[:, :3].double().cpu().numpy()
    w = acc[:, 3].double().cpu().numpy()
    ke = 0.5 * m * np.sum(v * v, axis=1)
    pe = 0.5 * m * w if law == 0 else 0.5 * w
    mv = m[:, None] * v
    lm = m[:, None] * np.cross(x, v)
    val = np.concatenate([[ke.sum(), pe.sum()], mv.sum(0), lm.sum(0)])
    scale = np.concatenate([[np.abs(ke).sum(), np.abs(pe).sum()], np.abs(mv).sum(0),
                            np.abs(lm).sum(0)])
    return val, scale


@pytest.mark.parametrize("n", [3000, 70001])
@pytest.mark.parametrize("law", [0, 1, 2])
def test_diagnostics_summed_in_the_finalize(law, n):
    """Rows at step 0 and at the last step against FP64 sums over the state they
    describe (70001 particles: more finalize blocks than its threads, so each
    thread of the last block adds several block rows)."""
    nb = lib()
    pos, vel, prm, kw = _system(law, n, seed=71 + law)
    kw.pop("law", None)
    steps = 2
    p, v = pos.clone(), vel.clone()
    a = torch.empty_like(p)
    d = nb.step(p, v, a, prm, law=law, nsteps=steps, report_every=steps, **kw)
    d = d.cpu().numpy()
    assert d.shape == (2, 8)
    a0 = nb.forces(pos, prm, law=law, pot=True, eps=kw.get("eps", 0.0))
    for row, (x_, v_, a_) in zip(d, ((pos, vel, a0), (p, v, a))):
        ref, scale = _diag_ref(x_, v_, a_, law)
        np.testing.assert_array_less(np.abs(row - ref), 1e-11 * scale + 1e-300)


@pytest.mark.parametrize("law", [0, 1])
def test_step_loop_replays_from_a_cuda_graph(law):
    """A multi-step call (its launches chained as programmatic dependent launches,
    the finalize preparing each next step's sources) captured in a CUDA graph and
    replayed gives the bits of the same call issued eagerly, report rows included."""
    nb = lib()
    pos, vel, prm, kw = _system(law, N_RAGGED, seed=91 + law)
    kw.pop("law", None)
    steps = 4
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    p1, v1 = pos.clone(), vel.clone()
    a1 = torch.empty_like(p1)
    d1 = torch.zeros((3, 8), dtype=torch.float64, device=pos.device)
    with torch.cuda.stream(s):  # eager, and sizes the capturing stream's workspace
        nb.step(p1, v1, a1, prm, law=law, nsteps=steps, report_every=2, diag=d1, **kw)
    s.synchronize()
    p2, v2 = pos.clone(), vel.clone()
    a2 = torch.empty_like(p2)
    d2 = torch.zeros_like(d1)
    p0, v0 = p2.clone(), v2.clone()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        nb.step(p2, v2, a2, prm, law=law, nsteps=steps, report_every=2, diag=d2, **kw)
    p2.copy_(p0)
    v2.copy_(v0)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(p1, p2) and torch.equal(v1, v2) and torch.equal(a1[:, :3], a2[:, :3])
    assert torch.equal(d1, d2)
