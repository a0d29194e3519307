"""Pins for the FP64 LJ + Coulomb oracle (Table 1 "LJC(constant)").

The paper prints the Lennard-Jones term as a bare scalar; the oracle reads it
as the standard 12-6 potential. These tests pin that reading to the textbook
facts of the 12-6 potential (zero force at r = 2^(1/6) sigma, well depth
-epsilon, zero energy at r = sigma), Coulomb's law, Lorentz-Berthelot mixing,
Newton's third law and F = -grad U.
"""
import numpy as np

import oracle
import workloads


def _pair(r, q=(0.0, 0.0), sig=(3.0, 3.0), eps=(0.1, 0.1), kq=1.0):
    x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    return oracle.ljc_force(x, np.array(q), np.array(sig), np.array(eps), kq=kq,
                            potential=True)


def test_lj_minimum_and_zero_crossing():
    sigma, eps = 3.0, 0.1
    rmin = 2.0 ** (1.0 / 6.0) * sigma
    f, phi = _pair(rmin, sig=(sigma, sigma), eps=(eps, eps))
    # force scale 24 eps / sigma ~ 0.8; zero to rounding at the minimum
    assert np.all(np.abs(f) < 1e-14)
    np.testing.assert_allclose(phi, [-eps, -eps], rtol=1e-13)
    f, phi = _pair(sigma, sig=(sigma, sigma), eps=(eps, eps))
    np.testing.assert_allclose(phi, [0.0, 0.0], atol=1e-15)
    # at r = sigma the force is repulsive: (24 eps / sigma) (2 - 1) = 0.8 along -x on atom 0
    np.testing.assert_allclose(f[0], [-0.8, 0.0, 0.0], rtol=1e-13)
    np.testing.assert_allclose(f[1], [0.8, 0.0, 0.0], rtol=1e-13)


def test_lorentz_berthelot_mixing():
    # sigma_12 = (3 + 2) / 2 = 2.5, eps_12 = sqrt(0.2 * 0.05) = 0.1
    rmin = 2.0 ** (1.0 / 6.0) * 2.5
    f, phi = _pair(rmin, sig=(3.0, 2.0), eps=(0.2, 0.05))
    assert np.all(np.abs(f) < 1e-14)
    np.testing.assert_allclose(phi, [-0.1, -0.1], rtol=1e-13)


def test_coulomb_only():
    # kq q1 q2 / r^2 with kq = 332.0637 / 80, q = (0.5, -0.4), r = 4 A:
    # |F| = 4.15079625 * 0.2 / 16 = 0.05188495..., attractive
    kq = 332.0637 / 80.0
    f, phi = _pair(4.0, q=(0.5, -0.4), eps=(0.0, 0.0), kq=kq)
    np.testing.assert_allclose(f[0], [0.0518849531250, 0.0, 0.0], rtol=1e-12)
    np.testing.assert_allclose(f[1], [-0.0518849531250, 0.0, 0.0], rtol=1e-12)
    np.testing.assert_allclose(phi, [-0.20753981250, -0.20753981250], rtol=1e-12)


def test_newton_third_law_and_gradient():
    s = workloads.ljc_sphere(200, seed=12)
    sig, eps = s.sig_t[s.types], s.eps_t[s.types]
    kq = oracle.COULOMB_K / 80.0
    f = oracle.ljc_force(s.x, s.q, sig, eps, kq)
    assert np.all(np.abs(f.sum(axis=0)) <= 1e-13 * np.abs(f).sum())
    # Moving x_i changes U only through the pairs (i, j), so dU/dx_i = dphi_i/dx_i;
    # differencing phi_i instead of the whole U keeps the rounding error small.
    h = 1e-5
    for i in (0, 17, 199):
        for a in range(3):
            xp, xm = s.x.copy(), s.x.copy()
            xp[i, a] += h
            xm[i, a] -= h
            _, pp = oracle.ljc_force(xp, s.q, sig, eps, kq, idx=[i], potential=True)
            _, pm = oracle.ljc_force(xm, s.q, sig, eps, kq, idx=[i], potential=True)
            dU = (pp[0] - pm[0]) / (2 * h)
            assert abs(-dU - f[i, a]) <= 1e-6 * max(1e-3, np.abs(f[i]).max())


def test_permutation_invariance():
    s = workloads.ljc_sphere(150, seed=13)
    sig, eps = s.sig_t[s.types], s.eps_t[s.types]
    f = oracle.ljc_force(s.x, s.q, sig, eps)
    p = np.random.default_rng(2).permutation(150)
    fp = oracle.ljc_force(s.x[p], s.q[p], sig[p], eps[p])
    np.testing.assert_allclose(fp, f[p], rtol=1e-11, atol=1e-13)


def test_generator_constraints():
    s = workloads.ljc_sphere(2000, seed=2)
    d2 = np.sum((s.x[:, None, :] - s.x[None, :, :]) ** 2, axis=-1)
    np.fill_diagonal(d2, np.inf)
    assert d2.min() >= 1.0
    r = 45.0 * (2000 / 8192) ** (1 / 3)
    assert np.max(np.linalg.norm(s.x, axis=1)) <= r
    assert abs(s.q.sum()) < 1e-12 and np.all(np.abs(s.q) <= 1.6)
    assert np.all((s.sig_t >= 2.5) & (s.sig_t <= 3.8))
    assert np.all((s.eps_t >= 0.05) & (s.eps_t <= 0.2))


def test_linear_dielectric_coulomb_hand_values():
    # Table 1 LJC(linear) with dielectric D r, D = 4: kq = 332.0637 / 4 = 83.015925.
    # Energy kq q1 q2 / r^2 = 83.015925 * (-0.2) / 16 = -1.0376990625,
    # force magnitude 2 kq |q1 q2| / r^3 = 2 * 83.015925 * 0.2 / 64 = 0.518849531...
    kq = 332.0637 / 4.0
    x = np.array([[0.0, 0.0, 0.0], [4.0, 0.0, 0.0]])
    f, phi = oracle.ljc_force(x, np.array([0.5, -0.4]), np.array([3.0, 3.0]), np.zeros(2),
                              kq=kq, potential=True, linear=True)
    np.testing.assert_allclose(f[0], [0.51884953125, 0.0, 0.0], rtol=1e-12)
    np.testing.assert_allclose(phi, [-1.0376990625, -1.0376990625], rtol=1e-12)


def test_linear_dielectric_force_is_minus_gradient():
    s = workloads.ljc_sphere(150, seed=15)
    sig, eps = s.sig_t[s.types], s.eps_t[s.types]
    kq = 332.0637 / 4.0
    f = oracle.ljc_force(s.x, s.q, sig, eps, kq, linear=True)
    assert np.all(np.abs(f.sum(axis=0)) <= 1e-13 * np.abs(f).sum())
    h = 1e-5
    for i in (3, 77):
        for a in range(3):
            xp, xm = s.x.copy(), s.x.copy()
            xp[i, a] += h
            xm[i, a] -= h
            _, pp = oracle.ljc_force(xp, s.q, sig, eps, kq, idx=[i], potential=True, linear=True)
            _, pm = oracle.ljc_force(xm, s.q, sig, eps, kq, idx=[i], potential=True, linear=True)
            assert abs(-(pp[0] - pm[0]) / (2 * h) - f[i, a]) <= 1e-6 * max(1e-3, np.abs(f[i]).max())
