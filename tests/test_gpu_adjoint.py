"""GPU parity of the reverse-mode path: single force VJPs (gravity and LJC, with
mass and per-type sigma/epsilon derivatives) against the FP64 oracle's
block-by-block Jacobian transpose, and the checkpointed reverse leapfrog
(torch.autograd.Function) against the oracle's reverse leapfrog and against
central finite differences of the oracle's FP64 loss."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_util import (FLOOR_SCALAR, GRAD_TOL_MAX, GRAD_TOL_RMS, as_f32, assert_grads_close,
                      assert_per_particle, assert_types_close, assert_vjp_close, dev,
                      grav_tensors, lib, ljc_tensors, oracle_ljc_system, traj_errors)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [3, 257, 1000, 9000, 9001])
def test_grav_vjp(n):
    nb = lib()
    g = workloads.plummer(n, seed=60 + n, eps=0.01)
    pos, _ = grav_tensors(g)
    lam = np.random.default_rng(n).standard_normal((n, 4)).astype(np.float32)
    gx, gm, _ = nb.adjoint(pos, torch.from_numpy(lam).to(dev()), eps=float(np.float32(g.eps)),
                           alpha=1.0)
    x, _, m = g.f32_as_f64()
    rg, rm = oracle.grav_vjp(x, m, lam[:, :3].astype(np.float64), eps=float(np.float32(g.eps)))
    assert_vjp_close(gx[:, :3].cpu().numpy(), gm.cpu().numpy(), rg, rm, what=f"n={n}")


@pytest.mark.parametrize("tile", range(17))
@pytest.mark.parametrize("jsplit", [0, 3])
def test_grav_vjp_every_tile(tile, jsplit):
    """Every compiled gravity VJP tile (packed and scalar, j-lanes, unrolls) at a
    ragged size spanning several j-tiles and slices, against the oracle."""
    nb = lib()
    n = 1500
    g = workloads.plummer(n, seed=61, eps=0.01)
    pos, _ = grav_tensors(g)
    lam = np.random.default_rng(7).standard_normal((n, 4)).astype(np.float32)
    gx, gm, _ = nb.adjoint(pos, torch.from_numpy(lam).to(dev()), eps=float(np.float32(g.eps)),
                           tile=tile, jsplit=jsplit)
    x, _, m = g.f32_as_f64()
    rg, rm = oracle.grav_vjp(x, m, lam[:, :3].astype(np.float64), eps=float(np.float32(g.eps)))
    assert_vjp_close(gx[:, :3].cpu().numpy(), gm.cpu().numpy(), rg, rm, what=str(tile))


@pytest.mark.parametrize("tile", range(12))
def test_ljc_vjp_every_tile(tile):
    nb = lib()
    n = 700
    s = workloads.ljc_sphere(n, seed=71)
    pos, _, prm = ljc_tensors(s)
    lam = np.random.default_rng(8).standard_normal((n, 4)).astype(np.float32)
    gx, gm, gt = nb.adjoint(pos, torch.from_numpy(lam).to(dev()), prm, tile=tile)
    sysm, x, _ = oracle_ljc_system(s)
    rg, rm, rs, re = sysm.vjp(x, lam[:, :3].astype(np.float64))
    assert_vjp_close(gx[:, :3].cpu().numpy(), gm.cpu().numpy(), rg, rm, what=str(tile))
    got_t = gt.cpu().numpy()
    assert_types_close(got_t, rs, re, what=str(tile))


def test_vjp_bad_tile_is_rejected():
    nb = lib()
    pos = torch.zeros((8, 4), device=dev())
    with pytest.raises(nb.NBodyError):
        nb.adjoint(pos, torch.zeros_like(pos), tile=nb.tile_count(nb.TABLE_VJP_GRAV))


def test_grav_vjp_alpha_and_accumulate():
    nb = lib()
    g = workloads.plummer(500, seed=3, eps=0.02)
    pos, _ = grav_tensors(g)
    lam = torch.randn((500, 4), device=dev())
    gx1, gm1, _ = nb.adjoint(pos, lam, eps=float(np.float32(g.eps)), alpha=1.0)
    gx2, gm2, _ = nb.adjoint(pos, lam, eps=float(np.float32(g.eps)), alpha=0.5)
    nb.adjoint(pos, lam, eps=float(np.float32(g.eps)), alpha=0.5, grad_x=gx2, grad_m=gm2,
               accumulate=True)
    torch.testing.assert_close(gx2[:, :3], gx1[:, :3], rtol=1e-5, atol=1e-6)
    torch.testing.assert_close(gm2, gm1, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("n", [20, 600, 3000, 8192])
def test_ljc_vjp(n):
    """LJC VJP with mass and per-type derivatives; n = 8192 is the molecular
    workload itself (seed 2) in the launch configuration the bench times."""
    nb = lib()
    s = workloads.ljc_sphere(n, seed=2 if n == 8192 else 70 + n)
    pos, _, prm = ljc_tensors(s)
    lam = np.random.default_rng(n).standard_normal((n, 4)).astype(np.float32)
    gx, gm, gt = nb.adjoint(pos, torch.from_numpy(lam).to(dev()), prm, alpha=1.0)
    sysm, x, _ = oracle_ljc_system(s)
    rg, rm, rs, re = sysm.vjp(x, lam[:, :3].astype(np.float64))
    assert_vjp_close(gx[:, :3].cpu().numpy(), gm.cpu().numpy(), rg, rm, what=f"n={n}")
    got_t = gt.cpu().numpy()
    assert_types_close(got_t, rs, re)


def _grav_autograd_grads(g, dt, nsteps, k, target, want_xT=False):
    nb = lib()
    from paper_0706_3060_gb300.autograd import leapfrog
    x, v, m = g.f32()
    d = dev()
    x0 = torch.from_numpy(x).to(d).requires_grad_(True)
    v0 = torch.from_numpy(v).to(d).requires_grad_(True)
    m0 = torch.from_numpy(m).to(d).requires_grad_(True)
    xT, _ = leapfrog(x0, v0, m0, dt=dt, nsteps=nsteps, k=k, eps=float(np.float32(g.eps)))
    tgt = torch.from_numpy(target.astype(np.float32)).to(d)
    loss = ((xT - tgt) ** 2).sum() / xT.shape[0]
    loss.backward()
    nb.sync_check()
    out = (x0.grad.cpu().numpy(), v0.grad.cpu().numpy(), m0.grad.cpu().numpy(),
           float(loss.detach()))
    return out + (xT.detach().double().cpu().numpy(),) if want_xT else out


def test_reverse_leapfrog_vs_oracle_gradient():
    """N = 1024 Plummer, 60 steps at dt = 1e-4, checkpoints every 20 steps."""
    g = workloads.plummer(1024, seed=4, eps=0.01)
    target = workloads.perturbed_target(g.f32_as_f64()[0], seed=4)
    gx, gv, gm, _ = _grav_autograd_grads(g, 1e-4, 60, 20, target)
    x, v, m = g.f32_as_f64()
    sysm = oracle.GravSystem(m, eps=float(np.float32(g.eps)))
    xs, _ = oracle.leapfrog(sysm, x, v, 1e-4, 60, store=True)
    ref = oracle.adjoint_leapfrog(sysm, x, v, 1e-4, 60, oracle.target_loss_grad(xs[-1], as_f32(target)),
                                  xs=xs)
    assert_grads_close(gx, gv, gm, ref, what="")


def test_reverse_leapfrog_checkpoint_invariance():
    """k = 7 (ragged last chunk) and k = 60 (one chunk) give the same gradients."""
    g = workloads.plummer(777, seed=9, eps=0.02)
    target = workloads.perturbed_target(g.f32_as_f64()[0], seed=4)
    a = _grav_autograd_grads(g, 1e-4, 60, 7, target)
    b = _grav_autograd_grads(g, 1e-4, 60, 60, target)
    for u, w in zip(a[:3], b[:3]):
        np.testing.assert_allclose(u, w, rtol=1e-5, atol=1e-9 * np.abs(w).max())


def test_reverse_leapfrog_vs_finite_differences():
    """Directional central differences (h = 1e-4) of the FP64 oracle loss."""
    g = workloads.plummer(256, seed=12, eps=0.05)
    dt, T = 1e-3, 40
    target = workloads.perturbed_target(g.f32_as_f64()[0], seed=4)
    gx, gv, gm, _ = _grav_autograd_grads(g, dt, T, 20, target)
    x, v, m = g.f32_as_f64()
    eps = float(np.float32(g.eps))

    def loss(x0, v0, m0):
        xT, _ = oracle.leapfrog(oracle.GravSystem(m0, eps=eps), x0, v0, dt, T)
        return oracle.target_loss(xT, as_f32(target))

    h = 1e-4
    for d in workloads.random_directions((256, 7), 4, seed=5):
        dx, dv, dm = d[:, :3], d[:, 3:6], d[:, 6] * 1e-2
        fd = (loss(x + h * dx, v + h * dv, m + h * dm) - loss(x - h * dx, v - h * dv, m - h * dm)) / (2 * h)
        an = np.sum(gx * dx) + np.sum(gv * dv) + np.sum(gm * dm)
        assert abs(fd - an) <= 1e-3 * abs(an) + 1e-9, (fd, an)


def test_ljc_reverse_leapfrog_vs_oracle():
    nb = lib()
    from paper_0706_3060_gb300.autograd import leapfrog
    s = workloads.ljc_sphere(300, seed=14, radius=20.0)
    x, v, m, q, st, et = s.f32()
    d = dev()
    x0 = torch.from_numpy(x).to(d).requires_grad_(True)
    v0 = torch.from_numpy(v).to(d).requires_grad_(True)
    m0 = torch.from_numpy(m).to(d).requires_grad_(True)
    sig = torch.from_numpy(st).to(d).requires_grad_(True)
    eps = torch.from_numpy(et).to(d).requires_grad_(True)
    dt, T = 1e-4, 12
    xT, _ = leapfrog(x0, v0, m0, dt=dt, nsteps=T, k=5, law=nb.LAW_LJC,
                     q=torch.from_numpy(q.astype(np.float64)).to(d),
                     types=torch.from_numpy(s.types).to(d), sig_t=sig, eps_t=eps)
    target = workloads.perturbed_target(x.astype(np.float64), seed=4)
    loss = ((xT - torch.from_numpy(target.astype(np.float32)).to(d)) ** 2).sum() / 300
    loss.backward()
    sysm, xo, vo = oracle_ljc_system(s)
    xs, _ = oracle.leapfrog(sysm, xo, vo, dt, T, store=True)
    ref = oracle.adjoint_leapfrog(sysm, xo, vo, dt, T, oracle.target_loss_grad(xs[-1], as_f32(target)),
                                  xs=xs)
    assert_grads_close(x0.grad.cpu().numpy(), v0.grad.cpu().numpy(), m0.grad.cpu().numpy(), ref, what="")
    assert_per_particle(sig.grad.cpu().numpy(), ref["sig_t"], FLOOR_SCALAR, 1e-3, 1e-3, "sig_t")
    assert_per_particle(eps.grad.cpu().numpy(), ref["eps_t"], FLOOR_SCALAR, 1e-3, 1e-3, "eps_t")


def test_adjoint_workload_size_one_chunk():
    """The adjoint workload's size (Plummer N = 16384, eps = 0.04 N^-1/3, dt = 1e-4)
    over one 20-step checkpoint chunk, against the FP64 oracle's gradient."""
    n = 16384
    g = workloads.plummer(n, seed=4, eps=workloads.plummer_softening(n))
    target = workloads.perturbed_target(g.f32_as_f64()[0], seed=4)
    gx, gv, gm, _ = _grav_autograd_grads(g, 1e-4, 20, 20, target)
    x, v, m = g.f32_as_f64()
    sysm = oracle.GravSystem(m, eps=float(np.float32(g.eps)))
    xs, _ = oracle.leapfrog(sysm, x, v, 1e-4, 20, store=True)
    ref = oracle.adjoint_leapfrog(sysm, x, v, 1e-4, 20, oracle.target_loss_grad(xs[-1], as_f32(target)),
                                  xs=xs)
    assert_grads_close(gx, gv, gm, ref, what="")


GOLDEN_ADJOINT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                              "adjoint_plummer16384.json")


def _adjoint_workload():
    n = 16384
    g = workloads.plummer(n, seed=4, eps=workloads.plummer_softening(n))
    target = workloads.perturbed_target(g.f32_as_f64()[0], seed=4)
    return g, target


def _fd_directions(n, golden):
    d = workloads.random_directions((n, 7), len(golden["fd"]), seed=golden["dir_seed"])
    return [np.concatenate([di[:, :6], di[:, 6:7] * 1e-2], axis=1) for di in d]


def _check_fd(gx, gv, gm, golden):
    """GPU gradient along each stored direction against central differences
    (h = 1e-4) of the oracle's FP64 loss: within 1e-3 of the derivative plus 1e-6
    of the gradient's norm (a unit direction can make the derivative itself small)."""
    gnorm = float(np.sqrt(np.sum(gx * gx) + np.sum(gv * gv) + np.sum((gm * 1e-2) ** 2)))
    for k, d in enumerate(_fd_directions(gx.shape[0], golden)):
        an = float(np.sum(gx * d[:, :3]) + np.sum(gv * d[:, 3:6]) + np.sum(gm * d[:, 6]))
        fd = golden["fd"][k]["fd"]
        assert abs(fd - an) <= 1e-3 * abs(fd) + 1e-6 * gnorm, (k, fd, an, gnorm)


def test_adjoint_workload_against_stored_oracle():
    """The adjoint workload in the bench's configuration (Plummer N = 16384,
    200 KDK steps at dt = 1e-4, checkpoints every 20, tuned tiles) against the
    oracle's answer stored by tests/golden/make_adjoint_golden.py: the loss, the
    gradient of 256 seeded particles per particle, and directional derivatives
    against central differences of the oracle loss along 4 seeded directions."""
    golden = json.load(open(GOLDEN_ADJOINT))
    g, target = _adjoint_workload()
    gx, gv, gm, loss = _grav_autograd_grads(g, golden["dt"], golden["steps"], golden["k"],
                                            target)
    assert abs(loss - golden["loss"]) <= 1e-5 * golden["loss"], (loss, golden["loss"])
    idx = np.asarray(golden["index"])
    ref = {"x0": np.asarray(golden["x0"]), "v0": np.asarray(golden["v0"]),
           "m": np.asarray(golden["m"])}
    # the floor of the per-particle metric comes from the full gradient's RMS
    for key, got in (("x0", gx[idx]), ("v0", gv[idx]), ("m", gm[idx])):
        num = np.linalg.norm(np.reshape(got, (len(idx), -1)) - np.reshape(ref[key], (len(idx), -1)),
                             axis=1)
        den = np.linalg.norm(np.reshape(ref[key], (len(idx), -1)), axis=1)
        e = num / np.maximum(den, FLOOR_SCALAR * golden["rms"][key])
        assert np.sqrt(np.mean(e * e)) <= GRAD_TOL_RMS and e.max() <= GRAD_TOL_MAX, (key, e.max())
    _check_fd(gx, gv, gm, golden)


@pytest.mark.slow
def test_adjoint_workload_full_against_oracle():
    """The same workload on every particle: the GPU's x_T against the oracle's
    FP64 trajectory, and dL/dx0, dL/dv0, dL/dm against the oracle's reverse
    leapfrog (every state stored, two VJPs per step) element by element. The
    oracle sweep takes a few minutes on the host cores."""
    golden = json.load(open(GOLDEN_ADJOINT))
    g, target = _adjoint_workload()
    T, dt, k = golden["steps"], golden["dt"], golden["k"]
    gx, gv, gm, loss, xT = _grav_autograd_grads(g, dt, T, k, target, want_xT=True)
    x, v, m = g.f32_as_f64()
    sysm = oracle.GravSystem(m, eps=float(np.float32(g.eps)))
    xs, _ = oracle.leapfrog(sysm, x, v, dt, T, store=True)
    r, mx = traj_errors(xT, xs[-1])
    assert r <= 1e-6 and mx <= 1e-5, (r, mx)
    ref = oracle.adjoint_leapfrog(sysm, x, v, dt, T, oracle.target_loss_grad(xs[-1], as_f32(target)),
                                  xs=xs)
    assert_grads_close(gx, gv, gm, ref, what="full adjoint workload")
    _check_fd(gx, gv, gm, golden)


def test_adjoint_workload_translation_identities():
    """The full adjoint workload in the bench's configuration (N = 16384, 200 steps
    at dt = 1e-4, checkpoints every 20): properties that hold at any size. The
    forces are translation invariant, so shifting every x0 by e shifts x_T by e
    and boosting every v0 by e shifts x_T by T dt e; hence
      sum_i dL/dx0_i = (2/N) sum_i (x_T,i - x*_i),  sum_i dL/dv0_i = T dt times it."""
    nb = lib()
    from paper_0706_3060_gb300.autograd import leapfrog
    n, T, dt = 16384, 200, 1e-4
    g = workloads.plummer(n, seed=4, eps=workloads.plummer_softening(n))
    target = workloads.perturbed_target(g.f32_as_f64()[0], seed=4)
    x, v, m = g.f32()
    d = dev()
    x0 = torch.from_numpy(x).to(d).requires_grad_(True)
    v0 = torch.from_numpy(v).to(d).requires_grad_(True)
    m0 = torch.from_numpy(m).to(d).requires_grad_(True)
    xT, _ = leapfrog(x0, v0, m0, dt=dt, nsteps=T, k=20, eps=float(np.float32(g.eps)))
    loss = ((xT - torch.from_numpy(target.astype(np.float32)).to(d)) ** 2).sum() / n
    loss.backward()
    nb.sync_check()
    resid = (xT.detach().double().cpu().numpy() - target).sum(axis=0) * 2.0 / n
    sx = x0.grad.double().cpu().numpy().sum(axis=0)
    sv = v0.grad.double().cpu().numpy().sum(axis=0)
    scale = np.abs(x0.grad.double().cpu().numpy()).sum(axis=0)
    assert np.all(np.abs(sx - resid) <= 1e-5 * scale + 1e-12), (sx, resid)
    assert np.all(np.abs(sv - T * dt * resid) <= 1e-5 * T * dt * scale + 1e-12), (sv, resid)


def test_every_family_bitwise_repeatable():
    """Fixed-order reductions: the same call twice gives identical bits for the
    LJC forces, both VJPs and acceleration + jerk (a race in a ring stage or a
    reduction would show up here)."""
    nb = lib()
    s = workloads.ljc_sphere(3000, seed=72)
    lpos, _, prm = ljc_tensors(s)
    g = workloads.plummer(5000, seed=73, eps=0.01)
    pos, vel = grav_tensors(g)
    lam = torch.randn((5000, 4), device=dev())
    llam = torch.randn((3000, 4), device=dev())
    runs = [
        lambda: (nb.forces(lpos, prm),),
        lambda: nb.adjoint(lpos, llam, prm)[:2],
        lambda: nb.adjoint(pos, lam, eps=0.01)[:2],
        lambda: nb.forces_jerk(pos, vel, eps=0.01),
    ]
    for k, fn in enumerate(runs):
        a = [t.clone() for t in fn()]
        b = [t.clone() for t in fn()]
        for u, w in zip(a, b):
            assert torch.equal(u, w), k


def _ljclin_setup(n, seed):
    """Positions, masses and LJ(linear) parameters packed with kq = k_e / 4 (the
    dielectric 4 r), and the matching oracle system."""
    nb = lib()
    K = 332.0637
    s = workloads.ljc_sphere(n, seed=seed)
    x, v, m, q, st, et = s.f32()
    d = dev()
    pos = torch.from_numpy(np.concatenate([x, m[:, None]], 1).astype(np.float32)).to(d)
    prm = nb.pack_ljc(torch.from_numpy(q.astype(np.float64)).to(d),
                      torch.from_numpy(st.astype(np.float64)[s.types]).to(d),
                      torch.from_numpy(et.astype(np.float64)[s.types]).to(d),
                      torch.from_numpy(s.types).to(d), kq=K / 4.0)
    xd, vd, md, qd, std, etd = s.f32_as_f64()
    sysm = oracle.LJCSystem(md, qd, s.types, std, etd, K / 4.0, linear=True)
    return s, pos.contiguous(), prm, sysm, xd, vd


@pytest.mark.parametrize("tile", range(7))
@pytest.mark.parametrize("n", [600, 3001])
def test_ljc_linear_vjp_every_tile(tile, n):
    """LJC(linear) VJP (dielectric 4 r) with mass and per-type derivatives, every
    tile of its table, against the oracle."""
    nb = lib()
    s, pos, prm, sysm, x, _ = _ljclin_setup(n, 80 + n)
    lam = np.random.default_rng(n).standard_normal((n, 4)).astype(np.float32)
    gx, gm, gt = nb.adjoint(pos, torch.from_numpy(lam).to(dev()), prm,
                            law=nb.LAW_LJC_LINEAR, tile=tile)
    rg, rm, rs, re = sysm.vjp(x, lam[:, :3].astype(np.float64))
    assert_vjp_close(gx[:, :3].cpu().numpy(), gm.cpu().numpy(), rg, rm, what=str(tile))
    got_t = gt.cpu().numpy()
    assert_types_close(got_t, rs, re, what=str(tile))


def test_ljc_linear_reverse_leapfrog_vs_oracle():
    nb = lib()
    from paper_0706_3060_gb300.autograd import leapfrog
    s = workloads.ljc_sphere(300, seed=15, radius=20.0)
    x, v, m, q, st, et = s.f32()
    d = dev()
    x0 = torch.from_numpy(x).to(d).requires_grad_(True)
    v0 = torch.from_numpy(v).to(d).requires_grad_(True)
    m0 = torch.from_numpy(m).to(d).requires_grad_(True)
    sig = torch.from_numpy(st).to(d).requires_grad_(True)
    eps = torch.from_numpy(et).to(d).requires_grad_(True)
    dt, T = 1e-4, 12
    xT, _ = leapfrog(x0, v0, m0, dt=dt, nsteps=T, k=5, law=nb.LAW_LJC_LINEAR,
                     q=torch.from_numpy(q.astype(np.float64)).to(d),
                     types=torch.from_numpy(s.types).to(d), sig_t=sig, eps_t=eps)
    target = workloads.perturbed_target(x.astype(np.float64), seed=4)
    loss = ((xT - torch.from_numpy(target.astype(np.float32)).to(d)) ** 2).sum() / 300
    loss.backward()
    xo, vo, mo, qo, so, eo = s.f32_as_f64()
    sysm = oracle.LJCSystem(mo, qo, s.types, so, eo, 332.0637 / 4.0, linear=True)
    xs, _ = oracle.leapfrog(sysm, xo, vo, dt, T, store=True)
    ref = oracle.adjoint_leapfrog(sysm, xo, vo, dt, T, oracle.target_loss_grad(xs[-1], as_f32(target)),
                                  xs=xs)
    assert_grads_close(x0.grad.cpu().numpy(), v0.grad.cpu().numpy(), m0.grad.cpu().numpy(), ref, what="")
    assert_per_particle(sig.grad.cpu().numpy(), ref["sig_t"], FLOOR_SCALAR, 1e-3, 1e-3, "sig_t")
    assert_per_particle(eps.grad.cpu().numpy(), ref["eps_t"], FLOOR_SCALAR, 1e-3, 1e-3, "eps_t")
