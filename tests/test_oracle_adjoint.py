"""Pins for the FP64 vector-Jacobian products and the reverse-mode leapfrog.

J^T lam is checked by the dot-product identity <lam, J u> = <J^T lam, u> with
J u taken by central finite differences of the force law; parameter
derivatives by finite differences of lam . a; the whole reverse leapfrog by
central finite differences of the loss along seeded random directions and,
for N = 8, component by component.
"""
import numpy as np
import pytest

import oracle
import workloads


def _grav_case(n=24, seed=21):
    g = workloads.plummer(n, seed=seed)
    m = g.m * np.linspace(0.6, 1.4, n)
    return g.x, g.v, m


def _ljc_case(n=20, seed=22):
    s = workloads.ljc_sphere(n, seed=seed, radius=6.0)
    return s


def test_grav_vjp_dot_product_identity():
    x, _, m = _grav_case()
    sysm = oracle.GravSystem(m, G=1.0, eps=0.05)
    rng = np.random.default_rng(3)
    lam = rng.standard_normal(x.shape)
    g, _ = sysm.vjp(x, lam)
    for _ in range(4):
        u = rng.standard_normal(x.shape)
        h = 1e-6
        Ju = (sysm.accel(x + h * u) - sysm.accel(x - h * u)) / (2 * h)
        assert abs(np.sum(lam * Ju) - np.sum(g * u)) <= 1e-7 * np.abs(g * u).sum()


def test_grav_vjp_rows_gather_equals_scatter():
    """The row-subset VJP gathers each row from the blocks (i, k) and (k, k); the
    full one scatters every ordered pair into the rows it touches. Two loop
    structures written apart: the same numbers to rounding, duplicate and
    unsorted indices included, unequal masses and G != 1."""
    rng = np.random.default_rng(17)
    n = 257
    x = rng.standard_normal((n, 3))
    m = rng.uniform(0.2, 2.0, n)
    lam = rng.standard_normal((n, 3))
    g, gm = oracle.grav_vjp(x, m, lam, G=0.7, eps=0.03)
    idx = np.array([256, 0, 5, 100, 100, 17])
    gr, gmr = oracle.grav_vjp(x, m, lam, G=0.7, eps=0.03, idx=idx)
    scale_g = np.abs(g).max()
    assert np.abs(gr - g[idx]).max() <= 1e-12 * scale_g
    assert np.abs(gmr - gm[idx]).max() <= 1e-12 * np.abs(gm).max()


def test_grav_mass_derivative():
    x, _, m = _grav_case()
    rng = np.random.default_rng(4)
    lam = rng.standard_normal(x.shape)
    _, gm = oracle.grav_vjp(x, m, lam, eps=0.05)
    dm = rng.standard_normal(m.shape) * 1e-3
    h = 1e-4
    fd = (np.sum(lam * oracle.grav_accel(x, m + h * dm, eps=0.05))
          - np.sum(lam * oracle.grav_accel(x, m - h * dm, eps=0.05))) / (2 * h)
    assert abs(fd - gm @ dm) <= 1e-9 * np.abs(gm * dm).sum()


@pytest.mark.parametrize("linear", [False, True])
def test_ljc_vjp_dot_product_and_parameters(linear):
    """J^T lam against central differences of the oracle's forces, for both
    dielectric models (constant eps_r = 80; linear D r with D = 4)."""
    s = _ljc_case()
    kq = oracle.COULOMB_K / (4.0 if linear else 80.0)
    sysm = oracle.LJCSystem(s.m, s.q, s.types, s.sig_t, s.eps_t, kq, linear=linear)
    rng = np.random.default_rng(5)
    lam = rng.standard_normal(s.x.shape)
    g, gm, gs, ge = sysm.vjp(s.x, lam)
    h = 1e-6
    for _ in range(3):
        u = rng.standard_normal(s.x.shape)
        Ju = (sysm.accel(s.x + h * u) - sysm.accel(s.x - h * u)) / (2 * h)
        assert abs(np.sum(lam * Ju) - np.sum(g * u)) <= 1e-6 * np.abs(g * u).sum()

    def lam_a(m=s.m, sig_t=s.sig_t, eps_t=s.eps_t):
        return np.sum(lam * oracle.LJCSystem(m, s.q, s.types, sig_t, eps_t, kq,
                                             linear=linear).accel(s.x))

    for t in range(len(s.sig_t)):
        e = np.zeros_like(s.sig_t)
        e[t] = 1.0
        fd = (lam_a(sig_t=s.sig_t + h * e) - lam_a(sig_t=s.sig_t - h * e)) / (2 * h)
        assert abs(fd - gs[t]) <= 1e-6 * max(1.0, abs(gs[t]))
        fd = (lam_a(eps_t=s.eps_t + 1e-7 * e) - lam_a(eps_t=s.eps_t - 1e-7 * e)) / 2e-7
        assert abs(fd - ge[t]) <= 1e-5 * max(1.0, abs(ge[t]))
    dm = rng.standard_normal(s.m.shape) * 1e-2
    fd = (lam_a(m=s.m + h * dm) - lam_a(m=s.m - h * dm)) / (2 * h)
    assert abs(fd - gm @ dm) <= 1e-6 * np.abs(gm * dm).sum()


def _loss_grav(x0, v0, m, target, dt, T, eps):
    sysm = oracle.GravSystem(m, eps=eps)
    xT, _ = oracle.leapfrog(sysm, x0, v0, dt, T)
    return oracle.target_loss(xT, target)


def test_reverse_leapfrog_full_fd_n8():
    x, v, m = _grav_case(8, seed=30)
    eps, dt, T = 0.05, 1e-3, 20
    sysm = oracle.GravSystem(m, eps=eps)
    xs, _ = oracle.leapfrog(sysm, x, v, dt, T, store=True)
    target = workloads.perturbed_target(x, seed=4)
    grad = oracle.adjoint_leapfrog(sysm, x, v, dt, T, oracle.target_loss_grad(xs[-1], target),
                                   xs=xs)
    h = 1e-4
    for name, arr in (("x0", x), ("v0", v), ("m", m)):
        fd = np.zeros_like(arr)
        flat = arr.reshape(-1)
        for k in range(flat.size):
            p, q = arr.copy().reshape(-1), arr.copy().reshape(-1)
            p[k] += h
            q[k] -= h
            args = {"x0": x, "v0": v, "m": m}
            args[name] = p.reshape(arr.shape)
            lp = _loss_grav(args["x0"], args["v0"], args["m"], target, dt, T, eps)
            args[name] = q.reshape(arr.shape)
            lm = _loss_grav(args["x0"], args["v0"], args["m"], target, dt, T, eps)
            fd.reshape(-1)[k] = (lp - lm) / (2 * h)
        scale = np.abs(fd).max()
        np.testing.assert_allclose(grad[name], fd, atol=1e-6 * scale, rtol=1e-5)


def test_reverse_leapfrog_directional_fd():
    x, v, m = _grav_case(48, seed=31)
    eps, dt, T = 0.02, 1e-3, 40
    sysm = oracle.GravSystem(m, eps=eps)
    xs, _ = oracle.leapfrog(sysm, x, v, dt, T, store=True)
    target = workloads.perturbed_target(x, seed=4)
    grad = oracle.adjoint_leapfrog(sysm, x, v, dt, T, oracle.target_loss_grad(xs[-1], target),
                                   xs=xs)
    h = 1e-4
    dirs = workloads.random_directions((48, 7), 8, seed=5)
    for d in dirs:
        dx, dv, dm = d[:, :3], d[:, 3:6], d[:, 6] * 1e-2
        lp = _loss_grav(x + h * dx, v + h * dv, m + h * dm, target, dt, T, eps)
        lm = _loss_grav(x - h * dx, v - h * dv, m - h * dm, target, dt, T, eps)
        fd = (lp - lm) / (2 * h)
        an = np.sum(grad["x0"] * dx) + np.sum(grad["v0"] * dv) + np.sum(grad["m"] * dm)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-12), (fd, an)


@pytest.mark.parametrize("linear", [False, True])
def test_reverse_leapfrog_ljc_directional_fd(linear):
    s = workloads.ljc_sphere(12, seed=23, radius=5.0)
    kq = oracle.COULOMB_K / (4.0 if linear else 80.0)
    dt, T = 2e-3, 10

    def loss(x0, v0, sig_t, eps_t):
        sysm = oracle.LJCSystem(s.m, s.q, s.types, sig_t, eps_t, kq, linear=linear)
        xT, _ = oracle.leapfrog(sysm, x0, v0, dt, T)
        return oracle.target_loss(xT, target)

    target = workloads.perturbed_target(s.x, seed=4)
    sysm = oracle.LJCSystem(s.m, s.q, s.types, s.sig_t, s.eps_t, kq, linear=linear)
    xs, _ = oracle.leapfrog(sysm, s.x, s.v, dt, T, store=True)
    grad = oracle.adjoint_leapfrog(sysm, s.x, s.v, dt, T,
                                   oracle.target_loss_grad(xs[-1], target), xs=xs)
    h = 1e-5
    rng = np.random.default_rng(9)
    for _ in range(4):
        dx = rng.standard_normal(s.x.shape)
        dv = rng.standard_normal(s.x.shape)
        ds = rng.standard_normal(s.sig_t.shape) * 0.1
        de = rng.standard_normal(s.eps_t.shape) * 0.01
        lp = loss(s.x + h * dx, s.v + h * dv, s.sig_t + h * ds, s.eps_t + h * de)
        lm = loss(s.x - h * dx, s.v - h * dv, s.sig_t - h * ds, s.eps_t - h * de)
        fd = (lp - lm) / (2 * h)
        an = (np.sum(grad["x0"] * dx) + np.sum(grad["v0"] * dv) + grad["sig_t"] @ ds
              + grad["eps_t"] @ de)
        assert abs(fd - an) <= 1e-5 * max(abs(an), 1e-12), (fd, an)


@pytest.mark.parametrize("n", [2, 5])
def test_grav_vjp_tiny_brute_force(n):
    # Build the full 3n x 3n Jacobian by finite differences and multiply.
    x, _, m = _grav_case(n, seed=40 + n)
    sysm = oracle.GravSystem(m, eps=0.1)
    h = 1e-6
    J = np.zeros((3 * n, 3 * n))
    for k in range(3 * n):
        e = np.zeros(3 * n)
        e[k] = h
        J[:, k] = ((sysm.accel(x + e.reshape(n, 3)) - sysm.accel(x - e.reshape(n, 3)))
                   .reshape(-1) / (2 * h))
    lam = np.random.default_rng(n).standard_normal((n, 3))
    g, _ = sysm.vjp(x, lam)
    np.testing.assert_allclose(g.reshape(-1), J.T @ lam.reshape(-1), rtol=1e-6,
                               atol=1e-8 * np.abs(J).max())
