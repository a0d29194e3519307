"""GPU parity of the Newton-symmetric gravity tiles (each unordered pair evaluated
once and applied to both particles) against the FP64 oracle: block sizes 512
and 1024, every ragged case of one and several blocks (odd N ends with the pad
particle), eps = 0 with the self pair masked on diagonal blocks, the potential,
both rsqrt modes, leapfrog trajectories, run-to-run bitwise reproducibility,
and the planning rules (no subsets, a cap on the partial-sum memory)."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_util import assert_forces_close, dev, grav_tensors, lib, traj_errors

pytestmark = pytest.mark.gpu


def _sym_tiles():
    nb = lib()
    tiles = [t for t in range(nb.tile_count(nb.LAW_GRAV))
             if nb.tile_info(nb.LAW_GRAV, t)["symmetric"]]
    assert tiles, "no symmetric gravity tile compiled"
    return tiles


def _ref(g, potential=False):
    x, _, m = g.f32_as_f64()
    return oracle.grav_accel(x, m, G=g.G, eps=float(np.float32(g.eps)), potential=potential)


@pytest.mark.parametrize("n", [1, 2, 3, 511, 512, 513, 1023, 1024, 1025, 2047, 2049, 5001])
def test_symmetric_tiles_ragged_sizes(n):
    nb = lib()
    g = workloads.plummer(n, seed=500 + n, eps=0.01)
    pos, _ = grav_tensors(g)
    eps = float(np.float32(g.eps))
    for tile in _sym_tiles():
        info = nb.tile_info(nb.LAW_GRAV, tile)
        assert info["j_tile"] == info["threads"] * info["i_per_thread"]
        for precise in (False, True):
            acc = nb.forces(pos, eps=eps, pot=True, precise=precise, tile=tile)
            torch.cuda.synchronize()
            a = acc.cpu().numpy()
            assert np.all(np.isfinite(a)), f"tile {tile} n {n}"
            if n == 1:
                assert np.all(a == 0.0)
                continue
            ref, phi = _ref(g, potential=True)
            assert_forces_close(a[:, :3], ref, what=f"tile={tile} n={n} precise={precise}")
            e = np.abs(a[:, 3] - phi) / np.abs(phi)
            assert np.sqrt(np.mean(e * e)) <= 1e-5 and e.max() <= 1e-4


def test_symmetric_unsoftened_few_body():
    """eps = 0: the diagonal block drops the self pair by index, off-diagonal blocks
    never meet it; three bodies in one block and across two blocks of 512."""
    nb = lib()
    rng = np.random.default_rng(9)
    for n in (2, 3, 600):
        x = rng.normal(size=(n, 3))
        m = rng.uniform(0.5, 2.0, n)
        pos = torch.from_numpy(np.concatenate([x, m[:, None]], 1).astype(np.float32)).to(dev())
        xd = pos[:, :3].double().cpu().numpy()
        md = pos[:, 3].double().cpu().numpy()
        ref, phi = oracle.grav_accel(xd, md, G=1.5, eps=0.0, potential=True)
        for tile in _sym_tiles():
            a = nb.forces(pos.contiguous(), G=1.5, eps=0.0, pot=True, tile=tile).cpu().numpy()
            assert np.all(np.isfinite(a))
            assert_forces_close(a[:, :3], ref, what=f"eps=0 tile={tile} n={n}")
            np.testing.assert_allclose(a[:, 3], phi, rtol=1e-5)


def test_symmetric_momentum_and_reproducibility():
    """The pair term is applied to both particles, so sum m_i a_i is the FP32
    rounding of a sum of cancelling terms; two calls agree bit for bit."""
    nb = lib()
    g = workloads.plummer(20000, seed=21, eps=0.01)
    pos, _ = grav_tensors(g)
    eps = float(np.float32(g.eps))
    for tile in _sym_tiles():
        a1 = nb.forces(pos, eps=eps, tile=tile)
        a2 = nb.forces(pos, eps=eps, tile=tile)
        assert torch.equal(a1, a2)
        a = a1[:, :3].double().cpu().numpy()
        m = pos[:, 3].double().cpu().numpy()
        p = np.abs((m[:, None] * a).sum(0))
        scale = np.sum(m[:, None] * np.abs(a), 0)
        assert np.all(p <= 1e-6 * scale), (p, scale)


def test_symmetric_leapfrog_matches_oracle():
    nb = lib()
    g = workloads.plummer(3001, seed=31, eps=0.01)
    eps = float(np.float32(g.eps))
    x, v, m = g.f32_as_f64()
    sysm = oracle.GravSystem(m, G=g.G, eps=eps)
    xs, vs = oracle.leapfrog(sysm, x, v, 1e-3, 10, store=True)
    for tile in _sym_tiles():
        pos, vel = grav_tensors(g)
        acc = torch.empty_like(pos)
        nb.step(pos, vel, acc, dt=1e-3, nsteps=10, eps=eps, tile=tile)
        ex = traj_errors(pos[:, :3].cpu().numpy(), xs[-1])
        ev = traj_errors(vel[:, :3].cpu().numpy(), vs[-1])
        assert ex[0] <= 1e-6 and ex[1] <= 1e-5, (tile, ex)
        assert ev[0] <= 1e-5 and ev[1] <= 1e-4, (tile, ev)


def test_symmetric_planning_rules():
    nb = lib()
    t = _sym_tiles()[0]
    g = workloads.plummer(4096, seed=41, eps=0.01)
    pos, _ = grav_tensors(g)
    idx = torch.arange(0, 4096, 7, dtype=torch.int32, device=dev())
    # targets that are not the sources: refused for an explicit symmetric tile
    with pytest.raises(nb.NBodyError):
        nb.forces_subset(pos, idx, eps=0.01, tile=t)
    # partials above the cap (one float4 per particle and block, 4 GiB)
    B = nb.tile_info(nb.LAW_GRAV, t)["j_tile"]
    n_big = 1 << 20
    assert (n_big // B) * n_big * 16 > 4 << 30
    with pytest.raises(nb.NBodyError):
        nb.workspace_size(n_big, eps=0.01, tile=t)
    assert nb.workspace_size(1 << 16, eps=0.01, tile=t) > 0
    # a tuned symmetric tile above the cap falls back to the default one-sided tile
    old = nb.get_config(nb.LAW_GRAV, n_big)
    old_small = nb.get_config(nb.LAW_GRAV, 4096)
    try:
        nb.set_tuned(nb.LAW_GRAV, n_big, t, 0)
        assert nb.workspace_size(n_big, eps=0.01) > 0
        nb.set_tuned(nb.LAW_GRAV, 4096, t, 0)
        acc = nb.forces_subset(pos, idx, eps=0.01)  # subset: falls back as well
        ref = oracle.grav_accel(*[a.astype(np.float64) for a in (g.f32()[0], g.f32()[2])],
                                eps=0.01, idx=idx.cpu().numpy())
        assert_forces_close(acc[:, :3].cpu().numpy(), ref, what="subset fallback")
    finally:
        nb.set_tuned(nb.LAW_GRAV, n_big, *old)
        nb.set_tuned(nb.LAW_GRAV, 4096, *old_small)
