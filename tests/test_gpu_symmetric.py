"""GPU parity of the Newton-symmetric gravity tiles (each unordered pair evaluated
once and applied to both particles) against the FP64 oracle: gravity forces
(blocks of 512, 768 and 1024), LJC forces with constant and linear dielectric
(blocks of 256 to 1024), the gravity and LJC force VJPs and acceleration + jerk
(blocks of 128 to 512), every ragged case
of one and several blocks (odd N ends with the pad particle), eps = 0 with the
self pair masked on diagonal blocks, the potential, both rsqrt modes, leapfrog
trajectories, run-to-run bitwise reproducibility, and the planning rules (no
subsets, a cap on the partial-sum memory)."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_util import (FLOOR_SCALAR, as_f32, assert_forces_close, assert_grads_close,
                      assert_per_particle, assert_types_close, assert_vjp_close, dev,
                      grav_tensors, lib, oracle_ljc_system, traj_errors)

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
    # slot partials above the cap (one float4 per particle and block; at most
    # 16 GiB): unsoftened gravity and plain sums keep per-block slots
    B = nb.tile_info(nb.LAW_GRAV, t)["j_tile"]
    n_big = 1 << 21
    assert (n_big // B) * n_big * 16 > 16 << 30
    for kw in ({"eps": 0.0}, {"eps": 0.01, "compensated": False}):
        with pytest.raises(nb.NBodyError):
            nb.workspace_size(n_big, tile=t, **kw)
    assert nb.workspace_size(1 << 16, eps=0.0, tile=t) > 0
    # softened gravity accumulates atomically: O(n) scratch, no cap
    ws = nb.workspace_size(n_big, eps=0.01, tile=t)
    assert 0 < ws < 128 * n_big, ws
    # a tuned symmetric tile above the cap falls back to the default one-sided tile
    old = nb.get_config(nb.LAW_GRAV, n_big)
    old_small = nb.get_config(nb.LAW_GRAV, 4096)
    try:
        nb.set_tuned(nb.LAW_GRAV, n_big, t, 0)
        assert nb.workspace_size(n_big, eps=0.0) > 0
        nb.set_tuned(nb.LAW_GRAV, 4096, t, 0)
        acc = nb.forces_subset(pos, idx, eps=0.01)  # subset: falls back as well
        ref = oracle.grav_accel(*[a.astype(np.float64) for a in (g.f32()[0], g.f32()[2])],
                                eps=0.01, idx=idx.cpu().numpy())
        assert_forces_close(acc[:, :3].cpu().numpy(), ref, what="subset fallback")
    finally:
        nb.set_tuned(nb.LAW_GRAV, n_big, *old)
        nb.set_tuned(nb.LAW_GRAV, 4096, *old_small)


def _sym_vjp_tiles():
    nb = lib()
    tiles = [t for t in range(nb.tile_count(nb.TABLE_VJP_GRAV))
             if nb.tile_info(nb.TABLE_VJP_GRAV, t)["symmetric"]]
    assert tiles, "no symmetric gravity VJP tile compiled"
    return tiles



@pytest.mark.parametrize("n", [1, 2, 3, 255, 256, 257, 511, 512, 513, 1025, 3001])
def test_symmetric_vjp_ragged_sizes(n):
    nb = lib()
    g = workloads.plummer(n, seed=700 + n, eps=0.01)
    pos, _ = grav_tensors(g)
    eps = float(np.float32(g.eps))
    lam = np.random.default_rng(n).standard_normal((n, 4)).astype(np.float32)
    x, _, m = g.f32_as_f64()
    rg, rm = oracle.grav_vjp(x, m, lam[:, :3].astype(np.float64), G=0.7, eps=eps)
    for tile in _sym_vjp_tiles():
        gx, gm, _ = nb.adjoint(pos, torch.from_numpy(lam).to(dev()), G=0.7, eps=eps, tile=tile)
        gxh, gmh = gx[:, :3].cpu().numpy(), gm.cpu().numpy()
        assert np.all(np.isfinite(gxh)) and np.all(np.isfinite(gmh))
        if n == 1:
            assert np.all(gxh == 0.0) and np.all(gmh == 0.0)
            continue
        assert_vjp_close(gxh, gmh, rg, rm, what=str((tile, n)))


def test_symmetric_vjp_unsoftened_and_repeatable():
    """eps = 0: only the diagonal blocks meet the self pair, masked there."""
    nb = lib()
    rng = np.random.default_rng(12)
    for n in (3, 700):
        x = rng.normal(size=(n, 3))
        m = rng.uniform(0.5, 2.0, n)
        pos = torch.from_numpy(np.concatenate([x, m[:, None]], 1).astype(np.float32)).to(dev())
        lam = rng.standard_normal((n, 4)).astype(np.float32)
        xd = pos[:, :3].double().cpu().numpy()
        md = pos[:, 3].double().cpu().numpy()
        rg, rm = oracle.grav_vjp(xd, md, lam[:, :3].astype(np.float64), eps=0.0)
        for tile in _sym_vjp_tiles():
            lt = torch.from_numpy(lam).to(dev())
            gx, gm, _ = nb.adjoint(pos.contiguous(), lt, eps=0.0, tile=tile)
            gx2, gm2, _ = nb.adjoint(pos.contiguous(), lt, eps=0.0, tile=tile)
            assert torch.equal(gx, gx2) and torch.equal(gm, gm2)
            assert_vjp_close(gx[:, :3].cpu().numpy(), gm.cpu().numpy(), rg, rm, what=str((tile, n)))


def test_symmetric_vjp_planning_rules():
    """One partial slot per block (no softening, or plain sums asked for) is
    refused where the slots pass the cap; the fixed-point path, which softened
    gravity takes there, has none (it runs at 2^20 in
    test_symmetric_vjp_fixed_point_at_two_to_the_twenty); fixed point without
    softening is refused."""
    nb = lib()
    t = _sym_vjp_tiles()[0]
    B = nb.tile_info(nb.TABLE_VJP_GRAV, t)["j_tile"]
    n_big = 1 << 21  # partials (n / B) x n x 16 B far above the 16 GiB cap
    assert (n_big // B) * n_big * 16 > 16 << 30
    pos = torch.zeros((n_big, 4), device=dev())
    pos[:, 0] = torch.arange(n_big, device=dev(), dtype=torch.float32)
    with pytest.raises(nb.NBodyError):
        nb.adjoint(pos, torch.zeros_like(pos), eps=0.0, tile=t)
    with pytest.raises(nb.NBodyError):
        nb.adjoint(pos, torch.zeros_like(pos), eps=0.01, tile=t, compensated=False)
    small = torch.zeros((8, 4), device=dev())
    with pytest.raises(nb.NBodyError):
        nb.adjoint(small, small, eps=0.0, tile=t, fixed=True)


@pytest.mark.parametrize("n", [257, 3001])
def test_symmetric_vjp_fixed_point_and_slots(n):
    """Softened gravity: the exact fixed-point sums (fixed=True), the per-block
    slots with compensation (default at this size) and without (compensated=False)
    of every symmetric VJP tile and source split against the oracle; the
    fixed-point result is bitwise repeatable."""
    nb = lib()
    g = workloads.plummer(n, seed=800 + n, eps=0.01)
    pos, _ = grav_tensors(g)
    eps = float(np.float32(g.eps))
    lam = np.random.default_rng(n).standard_normal((n, 4)).astype(np.float32)
    lt = torch.from_numpy(lam).to(dev())
    x, _, m = g.f32_as_f64()
    rg, rm = oracle.grav_vjp(x, m, lam[:, :3].astype(np.float64), G=1.3, eps=eps)
    for tile in _sym_vjp_tiles():
        for jsplit in (0, 2, 4):
            for mode in ("fixed", "slots", "plain"):
                kw = dict(fixed=mode == "fixed", compensated=mode != "plain")
                gx, gm, _ = nb.adjoint(pos, lt, G=1.3, eps=eps, tile=tile, jsplit=jsplit, **kw)
                assert_vjp_close(gx[:, :3].cpu().numpy(), gm.cpu().numpy(), rg, rm,
                                 what=str((tile, jsplit, mode)))
                if mode == "fixed":
                    gx2, gm2, _ = nb.adjoint(pos, lt, G=1.3, eps=eps, tile=tile,
                                             jsplit=jsplit, **kw)
                    assert torch.equal(gx, gx2) and torch.equal(gm, gm2)


@pytest.mark.slow
def test_symmetric_vjp_fixed_point_at_two_to_the_twenty():
    """N = 2^20, blocks of 512 in 2 parts: one slot per block and part would take
    32 GiB (above the cap), so the softened VJP takes the fixed-point sums (64 B
    per particle); 48 seeded particles against the oracle's rows, computed one by
    one."""
    nb = lib()
    n = 1 << 20
    g = workloads.plummer(n, seed=9, eps=workloads.plummer_softening(n))
    pos, _ = grav_tensors(g)
    eps = float(np.float32(g.eps))
    lam = np.random.default_rng(9).standard_normal((n, 4)).astype(np.float32)
    tile = [t for t in _sym_vjp_tiles()
            if nb.tile_info(nb.TABLE_VJP_GRAV, t)["j_tile"] == 512][0]
    gx, gm, _ = nb.adjoint(pos, torch.from_numpy(lam).to(dev()), eps=eps, tile=tile, jsplit=2)
    idx = np.sort(np.random.default_rng(10).choice(n, 48, replace=False))
    x, _, m = g.f32_as_f64()
    rg, rm = oracle.grav_vjp(x, m, lam[:, :3].astype(np.float64), eps=eps, idx=idx)
    it = torch.from_numpy(idx).to(dev())
    assert_vjp_close(gx[it, :3].cpu().numpy(), gm[it].cpu().numpy(), rg, rm, what="2^20")


def test_symmetric_forces_and_vjp_in_reverse_leapfrog():
    """The checkpointed reverse leapfrog (torch.autograd.Function) with the
    Newton-symmetric force tile in the forward pass and recompute and each
    symmetric VJP tile in the reverse sweep (installed as the tuned entries for
    N = 1024), against the FP64 oracle's gradient."""
    nb = lib()
    from paper_0706_3060_gb300.autograd import leapfrog
    g = workloads.plummer(1024, seed=4, eps=0.01)
    eps = float(np.float32(g.eps))
    target = workloads.perturbed_target(g.f32_as_f64()[0], seed=4)
    x, v, m = g.f32_as_f64()
    sysm = oracle.GravSystem(m, eps=eps)
    xs, _ = oracle.leapfrog(sysm, x, v, 1e-4, 60, store=True)
    ref = oracle.adjoint_leapfrog(sysm, x, v, 1e-4, 60, oracle.target_loss_grad(xs[-1], as_f32(target)),
                                  xs=xs)
    old_f = nb.get_config(nb.LAW_GRAV, 1024)
    old_v = nb.get_config(nb.TABLE_VJP_GRAV, 1024)
    try:
        nb.set_tuned(nb.LAW_GRAV, 1024, _sym_tiles()[-1], 0)
        for tile in _sym_vjp_tiles():
            nb.set_tuned(nb.TABLE_VJP_GRAV, 1024, tile, 0)
            xf, vf, mf = g.f32()
            d = dev()
            x0 = torch.from_numpy(xf).to(d).requires_grad_(True)
            v0 = torch.from_numpy(vf).to(d).requires_grad_(True)
            m0 = torch.from_numpy(mf).to(d).requires_grad_(True)
            xT, _ = leapfrog(x0, v0, m0, dt=1e-4, nsteps=60, k=20, eps=eps)
            tgt = torch.from_numpy(target.astype(np.float32)).to(d)
            (((xT - tgt) ** 2).sum() / 1024).backward()
            nb.sync_check()
            assert_grads_close(x0.grad.cpu().numpy(), v0.grad.cpu().numpy(), m0.grad.cpu().numpy(), ref, what=str(tile))
    finally:
        nb.set_tuned(nb.LAW_GRAV, 1024, *old_f)
        nb.set_tuned(nb.TABLE_VJP_GRAV, 1024, *old_v)


def _sym_ljc_tiles(law):
    nb = lib()
    return [t for t in range(nb.tile_count(law)) if nb.tile_info(law, t)["symmetric"]]


@pytest.mark.parametrize("linear", [False, True])
@pytest.mark.parametrize("n", [2, 3, 255, 256, 257, 513, 1025, 3001])
def test_symmetric_ljc_ragged_sizes(n, linear):
    """Table 1 LJC(constant) (dielectric 80) and LJC(linear) (D = 4) through every
    symmetric tile, with the potential and both rsqrt modes."""
    nb = lib()
    law = nb.LAW_LJC_LINEAR if linear else nb.LAW_LJC
    D = 4.0 if linear else 80.0
    s = workloads.ljc_sphere(n, seed=800 + n)
    x, v, m, q, st, et = s.f32()
    d = dev()
    pos = torch.from_numpy(np.concatenate([x, m[:, None]], 1).astype(np.float32)).to(d)
    prm = nb.pack_ljc(torch.from_numpy(q.astype(np.float64)).to(d),
                      torch.from_numpy(st.astype(np.float64)[s.types]).to(d),
                      torch.from_numpy(et.astype(np.float64)[s.types]).to(d),
                      torch.from_numpy(s.types).to(d), kq=332.0637 / D)
    sysm = oracle.LJCSystem(m.astype(np.float64), q.astype(np.float64), s.types,
                            st.astype(np.float64), et.astype(np.float64), 332.0637 / D,
                            linear=linear)
    ref, phi = sysm.accel(x.astype(np.float64), potential=True)
    tiles = _sym_ljc_tiles(law)
    assert tiles
    for tile in tiles:
        for precise in (False, True):
            acc = nb.forces(pos.contiguous(), prm, law=law, pot=True, precise=precise,
                            tile=tile).cpu().numpy()
            assert np.all(np.isfinite(acc)), (tile, n)
            assert_forces_close(acc[:, :3], ref, what=f"LJC linear={linear} tile={tile} n={n}")
            e = np.abs(acc[:, 3] - phi) / np.maximum(np.abs(phi), 1e-3 * np.abs(phi).max())
            assert np.sqrt(np.mean(e * e)) <= 1e-5 and e.max() <= 1e-4, (tile, n)


@pytest.mark.parametrize("n", [2, 3, 255, 256, 257, 513, 1025, 3001])
def test_symmetric_jerk_ragged_sizes(n):
    """Acceleration + jerk (Table 1 GAJ) through every symmetric tile of its table."""
    nb = lib()
    g = workloads.plummer(n, seed=900 + n, eps=0.01)
    pos, vel = grav_tensors(g)
    eps = float(np.float32(g.eps))
    x, v, m = g.f32_as_f64()
    ra, rj = oracle.grav_jerk(x, v, m, G=1.3, eps=eps)
    tiles = _sym_ljc_tiles(nb.TABLE_JERK)
    assert tiles
    for tile in tiles:
        for fixed in (False, True):  # per-block slots; exact fixed-point sums
            acc, jerk = nb.forces_jerk(pos, vel, G=1.3, eps=eps, tile=tile, fixed=fixed)
            what = f"tile {tile} n {n} fixed {fixed}"
            assert_forces_close(acc[:, :3].cpu().numpy(), ra, what=f"GAJ acc {what}")
            assert_forces_close(jerk[:, :3].cpu().numpy(), rj, what=f"GAJ jerk {what}")
            if fixed:
                acc2, jerk2 = nb.forces_jerk(pos, vel, G=1.3, eps=eps, tile=tile, fixed=True)
                assert torch.equal(acc, acc2) and torch.equal(jerk, jerk2)


def test_symmetric_jerk_unsoftened_and_hermite():
    """eps = 0 (self pair masked on diagonal blocks; the closed-form two-body jerk)
    and fourth-order Hermite steps through each symmetric jerk tile against the
    FP64 oracle's Hermite integrator."""
    nb = lib()
    pos = torch.tensor([[0, 0, 0, 5.0], [3, 4, 0, 2.0]], dtype=torch.float32, device=dev())
    vel = torch.tensor([[0, 0, 0, 0], [1, 0, 0, 0]], dtype=torch.float32, device=dev())
    g = workloads.plummer(2048, seed=23, eps=0.01)
    eps = float(np.float32(g.eps))
    x, v, m = g.f32_as_f64()
    xr, vr = oracle.hermite(x, v, m, 1e-3, 10, eps=eps)
    for tile in _sym_ljc_tiles(nb.TABLE_JERK):
        _, jerk = nb.forces_jerk(pos, vel, eps=0.0, tile=tile)
        np.testing.assert_allclose(jerk[0, :3].cpu().numpy(), [-0.00128, -0.02304, 0.0],
                                   rtol=2e-6, atol=1e-9)
        for fixed in (False, True):
            p, vv = grav_tensors(g)
            acc = torch.empty_like(p)
            jk = torch.empty_like(p)
            nb.hermite_step(p, vv, acc, jk, dt=1e-3, nsteps=10, eps=eps, tile=tile,
                            fixed=fixed)
            ex = traj_errors(p[:, :3].cpu().numpy(), xr)
            ev = traj_errors(vv[:, :3].cpu().numpy(), vr)
            assert ex[0] <= 1e-6 and ex[1] <= 1e-5, (tile, fixed, ex)
            assert ev[0] <= 1e-5 and ev[1] <= 1e-4, (tile, fixed, ev)
    with pytest.raises(nb.NBodyError):  # no bound without softening
        nb.forces_jerk(pos, vel, eps=0.0, fixed=True)


@pytest.mark.slow
def test_symmetric_jerk_fixed_point_at_two_to_the_twenty():
    """N = 2^20, blocks of 512: the two partial blocks of one slot per particle and
    block would take 64 GiB (above the cap), so the softened evaluation takes the
    fixed-point sums (128 B per particle); 48 seeded particles against the oracle."""
    nb = lib()
    n = 1 << 20
    g = workloads.plummer(n, seed=11, eps=workloads.plummer_softening(n))
    pos, vel = grav_tensors(g)
    eps = float(np.float32(g.eps))
    tile = [t for t in _sym_ljc_tiles(nb.TABLE_JERK)
            if nb.tile_info(nb.TABLE_JERK, t)["j_tile"] == 512][0]
    acc, jerk = nb.forces_jerk(pos, vel, eps=eps, tile=tile)
    idx = np.sort(np.random.default_rng(12).choice(n, 48, replace=False))
    x, v, m = g.f32_as_f64()
    ra, rj = oracle.grav_jerk(x, v, m, eps=eps, idx=idx)
    it = torch.from_numpy(idx).to(dev())
    assert_forces_close(acc[it, :3].cpu().numpy(), ra, what="GAJ acc 2^20")
    assert_forces_close(jerk[it, :3].cpu().numpy(), rj, what="GAJ jerk 2^20")


@pytest.mark.parametrize("linear", [False, True])
@pytest.mark.parametrize("n", [2, 3, 127, 128, 129, 257, 1025, 3001])
def test_symmetric_ljc_vjp_ragged_sizes(n, linear):
    """LJC VJP with mass and per-type sigma/epsilon derivatives (both dielectric
    models) through every symmetric tile, against the oracle."""
    nb = lib()
    law = nb.LAW_LJC_LINEAR if linear else nb.LAW_LJC
    table = nb.TABLE_VJP_LJC_LINEAR if linear else nb.TABLE_VJP_LJC
    D = 4.0 if linear else 80.0
    s = workloads.ljc_sphere(n, seed=950 + n)
    x, v, m, q, st, et = s.f32()
    d = dev()
    pos = torch.from_numpy(np.concatenate([x, m[:, None]], 1).astype(np.float32)).to(d)
    prm = nb.pack_ljc(torch.from_numpy(q.astype(np.float64)).to(d),
                      torch.from_numpy(st.astype(np.float64)[s.types]).to(d),
                      torch.from_numpy(et.astype(np.float64)[s.types]).to(d),
                      torch.from_numpy(s.types).to(d), kq=332.0637 / D)
    sysm = oracle.LJCSystem(m.astype(np.float64), q.astype(np.float64), s.types,
                            st.astype(np.float64), et.astype(np.float64), 332.0637 / D,
                            linear=linear)
    lam = np.random.default_rng(n).standard_normal((n, 4)).astype(np.float32)
    rg, rm, rs, re = sysm.vjp(x.astype(np.float64), lam[:, :3].astype(np.float64))
    tiles = _sym_ljc_tiles(table)
    assert tiles
    for tile in tiles:
        gx, gm, gt = nb.adjoint(pos.contiguous(), torch.from_numpy(lam).to(d), prm, law=law,
                                tile=tile)
        assert_vjp_close(gx[:, :3].cpu().numpy(), gm.cpu().numpy(), rg, rm, what=str((tile, n)))
        got_t = gt.cpu().numpy()
        present = np.unique(s.types)
        assert_types_close(np.concatenate([got_t[:4][present], got_t[4:][present]]), rs[present], re[present], what=str((tile, n)))


def test_symmetric_ljc_reverse_leapfrog():
    """LJC reverse leapfrog (torch.autograd.Function) with each symmetric LJC
    VJP tile and the symmetric LJC force tile installed as the tuned entries for
    the size, against the FP64 oracle's gradients (positions, velocities,
    masses, per-type sigma and epsilon)."""
    nb = lib()
    from paper_0706_3060_gb300.autograd import leapfrog
    s = workloads.ljc_sphere(300, seed=14, radius=20.0)
    x, v, m, q, st, et = s.f32()
    d = dev()
    dt, T = 1e-4, 12
    target = workloads.perturbed_target(x.astype(np.float64), seed=4)
    sysm, xo, vo = oracle_ljc_system(s)
    xs, _ = oracle.leapfrog(sysm, xo, vo, dt, T, store=True)
    ref = oracle.adjoint_leapfrog(sysm, xo, vo, dt, T, oracle.target_loss_grad(xs[-1], as_f32(target)),
                                  xs=xs)
    old_f = nb.get_config(nb.LAW_LJC, 300)
    old_v = nb.get_config(nb.TABLE_VJP_LJC, 300)
    try:
        nb.set_tuned(nb.LAW_LJC, 300, _sym_ljc_tiles(nb.LAW_LJC)[0], 0)
        for tile in _sym_ljc_tiles(nb.TABLE_VJP_LJC):
            nb.set_tuned(nb.TABLE_VJP_LJC, 300, tile, 0)
            x0 = torch.from_numpy(x).to(d).requires_grad_(True)
            v0 = torch.from_numpy(v).to(d).requires_grad_(True)
            m0 = torch.from_numpy(m).to(d).requires_grad_(True)
            sig = torch.from_numpy(st).to(d).requires_grad_(True)
            eps = torch.from_numpy(et).to(d).requires_grad_(True)
            xT, _ = leapfrog(x0, v0, m0, dt=dt, nsteps=T, k=5, law=nb.LAW_LJC,
                             q=torch.from_numpy(q.astype(np.float64)).to(d),
                             types=torch.from_numpy(s.types).to(d), sig_t=sig, eps_t=eps)
            loss = ((xT - torch.from_numpy(target.astype(np.float32)).to(d)) ** 2).sum() / 300
            loss.backward()
            nb.sync_check()
            assert_grads_close(x0.grad.cpu().numpy(), v0.grad.cpu().numpy(), m0.grad.cpu().numpy(), ref, what=str(tile))
            assert_per_particle(sig.grad.cpu().numpy(), ref["sig_t"], FLOOR_SCALAR, 1e-3, 1e-3, "sig_t")
            assert_per_particle(eps.grad.cpu().numpy(), ref["eps_t"], FLOOR_SCALAR, 1e-3, 1e-3, "eps_t")
    finally:
        nb.set_tuned(nb.LAW_LJC, 300, *old_f)
        nb.set_tuned(nb.TABLE_VJP_LJC, 300, *old_v)


@pytest.mark.parametrize("n", [2, 3, 511, 1025, 3001])
def test_symmetric_fixed_point(n):
    """64-bit fixed-point partials (Sec. 3.2) from the symmetric tiles: oracle
    accuracy for forces and potential, bitwise repeatable, and 10 leapfrog steps."""
    nb = lib()
    tiles = _sym_ljc_tiles(nb.TABLE_GRAV_FIXED)
    assert tiles
    g = workloads.plummer(n, seed=1100 + n, eps=0.01)
    pos, _ = grav_tensors(g)
    eps = float(np.float32(g.eps))
    ref, phi = _ref(g, potential=True)
    for tile in tiles:
        a = nb.forces(pos, eps=eps, fixed=True, pot=True, tile=tile)
        b = nb.forces(pos, eps=eps, fixed=True, pot=True, tile=tile)
        assert torch.equal(a, b)
        assert_forces_close(a[:, :3].cpu().numpy(), ref, what=f"fixed sym tile={tile} n={n}")
        e = np.abs(a[:, 3].cpu().numpy() - phi) / np.abs(phi)
        assert e.max() <= 1e-4, (tile, n)
    if n >= 1000:
        x, v, m = g.f32_as_f64()
        sysm = oracle.GravSystem(m, G=g.G, eps=eps)
        xs, vs = oracle.leapfrog(sysm, x, v, 1e-3, 10, store=True)
        for tile in tiles:
            p, vel = grav_tensors(g)
            acc = torch.empty_like(p)
            nb.step(p, vel, acc, dt=1e-3, nsteps=10, eps=eps, fixed=True, tile=tile)
            ex = traj_errors(p[:, :3].cpu().numpy(), xs[-1])
            assert ex[0] <= 1e-6 and ex[1] <= 1e-5, (tile, ex)


@pytest.mark.parametrize("n", [3, 700, 1025, 3001, 8192])
@pytest.mark.parametrize("jsplit", [2, 4, 8])
def test_symmetric_source_split(n, jsplit):
    """The source split (each block's sources cut into 2, 4 or 8 parts, one CTA
    each, the finalize counting only the slots a particle receives) for every
    symmetric force tile: gravity with the potential, fixed point, and LJC."""
    nb = lib()
    g = workloads.plummer(n, seed=1300 + n, eps=0.01)
    pos, _ = grav_tensors(g)
    eps = float(np.float32(g.eps))
    ref, phi = _ref(g, potential=True)
    for tile in _sym_tiles():
        a = nb.forces(pos, eps=eps, pot=True, tile=tile, jsplit=jsplit)
        b = nb.forces(pos, eps=eps, pot=True, tile=tile, jsplit=jsplit)
        assert torch.equal(a, b)
        assert_forces_close(a[:, :3].cpu().numpy(), ref, what=f"tile={tile} split={jsplit} n={n}")
        e = np.abs(a[:, 3].cpu().numpy() - phi) / np.abs(phi)
        assert e.max() <= 1e-4, (tile, jsplit, n)
    for tile in _sym_ljc_tiles(nb.TABLE_GRAV_FIXED):
        a = nb.forces(pos, eps=eps, fixed=True, tile=tile, jsplit=jsplit)
        assert_forces_close(a[:, :3].cpu().numpy(), ref, what=f"fixed tile={tile} split={jsplit}")
    s = workloads.ljc_sphere(n, seed=1400 + n)
    x, v, m, q, st, et = s.f32()
    d = dev()
    lpos = torch.from_numpy(np.concatenate([x, m[:, None]], 1).astype(np.float32)).to(d)
    prm = nb.pack_ljc(torch.from_numpy(q.astype(np.float64)).to(d),
                      torch.from_numpy(st.astype(np.float64)[s.types]).to(d),
                      torch.from_numpy(et.astype(np.float64)[s.types]).to(d),
                      torch.from_numpy(s.types).to(d))
    sysm, xo, _ = oracle_ljc_system(s)
    lref = sysm.accel(xo)
    for tile in _sym_ljc_tiles(nb.LAW_LJC):
        a = nb.forces(lpos.contiguous(), prm, tile=tile, jsplit=jsplit)
        assert_forces_close(a[:, :3].cpu().numpy(), lref, what=f"LJC tile={tile} split={jsplit}")


def test_symmetric_split_leapfrog():
    nb = lib()
    g = workloads.plummer(3001, seed=31, eps=0.01)
    eps = float(np.float32(g.eps))
    x, v, m = g.f32_as_f64()
    sysm = oracle.GravSystem(m, G=g.G, eps=eps)
    xs, vs = oracle.leapfrog(sysm, x, v, 1e-3, 10, store=True)
    for tile in _sym_tiles():
        pos, vel = grav_tensors(g)
        acc = torch.empty_like(pos)
        nb.step(pos, vel, acc, dt=1e-3, nsteps=10, eps=eps, tile=tile, jsplit=4)
        ex = traj_errors(pos[:, :3].cpu().numpy(), xs[-1])
        assert ex[0] <= 1e-6 and ex[1] <= 1e-5, (tile, ex)


@pytest.mark.parametrize("n", [3, 700, 1025, 3001])
@pytest.mark.parametrize("jsplit", [2, 4])
def test_symmetric_vjp_source_split(n, jsplit):
    """The gravity VJP with each block's sources cut into parts (one CTA each, the
    finalize walking the slots a particle receives), every symmetric VJP tile."""
    nb = lib()
    g = workloads.plummer(n, seed=1500 + n, eps=0.01)
    pos, _ = grav_tensors(g)
    eps = float(np.float32(g.eps))
    lam = np.random.default_rng(n).standard_normal((n, 4)).astype(np.float32)
    x, _, m = g.f32_as_f64()
    rg, rm = oracle.grav_vjp(x, m, lam[:, :3].astype(np.float64), eps=eps)
    for tile in _sym_vjp_tiles():
        lt = torch.from_numpy(lam).to(dev())
        gx, gm, _ = nb.adjoint(pos, lt, eps=eps, tile=tile, jsplit=jsplit)
        gx2, gm2, _ = nb.adjoint(pos, lt, eps=eps, tile=tile, jsplit=jsplit)
        assert torch.equal(gx, gx2) and torch.equal(gm, gm2)
        assert_vjp_close(gx[:, :3].cpu().numpy(), gm.cpu().numpy(), rg, rm, what=str((tile, jsplit, n)))


def test_symmetric_vjp_split_in_reverse_leapfrog():
    """The reverse leapfrog with a split symmetric VJP installed as the tuned entry."""
    nb = lib()
    from paper_0706_3060_gb300.autograd import leapfrog
    g = workloads.plummer(1024, seed=4, eps=0.01)
    eps = float(np.float32(g.eps))
    target = workloads.perturbed_target(g.f32_as_f64()[0], seed=4)
    x, v, m = g.f32_as_f64()
    sysm = oracle.GravSystem(m, eps=eps)
    xs, _ = oracle.leapfrog(sysm, x, v, 1e-4, 60, store=True)
    ref = oracle.adjoint_leapfrog(sysm, x, v, 1e-4, 60, oracle.target_loss_grad(xs[-1], as_f32(target)),
                                  xs=xs)
    old_v = nb.get_config(nb.TABLE_VJP_GRAV, 1024)
    try:
        nb.set_tuned(nb.TABLE_VJP_GRAV, 1024, _sym_vjp_tiles()[0], 2)
        xf, vf, mf = g.f32()
        d = dev()
        x0 = torch.from_numpy(xf).to(d).requires_grad_(True)
        v0 = torch.from_numpy(vf).to(d).requires_grad_(True)
        m0 = torch.from_numpy(mf).to(d).requires_grad_(True)
        xT, _ = leapfrog(x0, v0, m0, dt=1e-4, nsteps=60, k=20, eps=eps)
        tgt = torch.from_numpy(target.astype(np.float32)).to(d)
        (((xT - tgt) ** 2).sum() / 1024).backward()
        nb.sync_check()
        assert_grads_close(x0.grad.cpu().numpy(), v0.grad.cpu().numpy(), m0.grad.cpu().numpy(), ref, what="")
    finally:
        nb.set_tuned(nb.TABLE_VJP_GRAV, 1024, *old_v)


def test_symmetric_no_compensation_is_honoured():
    """NBODY_NO_COMPENSATION on the Newton-symmetric tiles adds their per-block
    partials in plain FP32 (128 blocks here): the bits differ from the compensated
    default, and both stay within the force tolerance of the oracle."""
    nb = lib()
    n = 65536
    g = workloads.plummer(n, seed=31, eps=workloads.plummer_softening(n))
    pos, _ = grav_tensors(g)
    eps = float(np.float32(g.eps))
    x, _, m = g.f32_as_f64()
    idx = np.random.default_rng(31).choice(n, 512, replace=False)
    ref = oracle.grav_accel(x, m, eps=eps, idx=idx)
    sym = [t for t in range(nb.tile_count(nb.LAW_GRAV))
           if nb.tile_info(nb.LAW_GRAV, t)["symmetric"]]
    for t in sym:
        a = nb.forces(pos, eps=eps, tile=t)
        b = nb.forces(pos, eps=eps, tile=t, compensated=False)
        assert not torch.equal(a, b), t
        for acc in (a, b):
            assert_forces_close(acc[idx, :3].double().cpu().numpy(), ref, what=f"tile {t}")


def test_symmetric_gravity_beyond_the_slot_cap():
    """Softened gravity at N = 2^21 through the Newton-symmetric tile with blocks of
    1024: per-block FP32 slots would need nb x N x 16 B = 32 GiB (above the cap), the
    fixed-point atomic accumulation needs 32 B per particle. 512 sampled targets
    against the oracle, and the same bits on a second call."""
    nb = lib()
    n = 1 << 21
    t = [k for k in _sym_tiles() if nb.tile_info(nb.LAW_GRAV, k)["j_tile"] == 1024][-1]
    g = workloads.plummer(n, seed=13, eps=workloads.plummer_softening(n))
    pos, _ = grav_tensors(g)
    eps = float(np.float32(g.eps))
    assert nb.workspace_size(n, eps=eps, tile=t) < 128 * n
    with pytest.raises(nb.NBodyError):  # the slot path at this size is refused
        nb.workspace_size(n, eps=eps, tile=t, compensated=False)
    acc = nb.forces(pos, eps=eps, tile=t, pot=True)
    again = nb.forces(pos, eps=eps, tile=t, pot=True)
    assert torch.equal(acc, again)
    x, _, m = g.f32_as_f64()
    idx = np.random.default_rng(21).choice(n, 512, replace=False)
    ref, phi = oracle.grav_accel(x, m, eps=eps, idx=idx, potential=True)
    got = acc[torch.from_numpy(idx).to(dev())].double().cpu().numpy()
    assert_forces_close(got[:, :3], ref, what="N = 2^21 symmetric")
    assert np.all(np.abs(got[:, 3] - phi) <= 1e-5 * np.abs(phi))


def test_symmetric_gravity_tiny_softening():
    """The fixed-point accumulation's grid follows the a-priori bound ~M / eps^2, so
    with eps = 1e-6 (system size / eps ~ 1e6) one 64-bit word per component would
    round each per-block partial to 2^-23 absolute, far coarser than FP32 for the
    outer particles; the integer part plus the 2^-32 fraction word keep every
    partial exact. Sampled targets against the oracle at the force tolerance."""
    nb = lib()
    n = 32768
    g = workloads.plummer(n, seed=17, eps=1e-6)
    pos, _ = grav_tensors(g)
    eps = float(np.float32(g.eps))
    x, _, m = g.f32_as_f64()
    idx = np.random.default_rng(17).choice(n, 1024, replace=False)
    ref = oracle.grav_accel(x, m, eps=eps, idx=idx)
    for t in _sym_tiles():
        acc = nb.forces(pos, eps=eps, tile=t)
        assert_forces_close(acc[idx, :3].double().cpu().numpy(), ref, what=f"eps 1e-6 tile {t}")
