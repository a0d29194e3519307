"""Pins for the FP64 gravity oracle (Eq. 1, Table 1 "Gravity (accel)").

Each test ties the oracle to something other than its own formula: hand-worked
two-body numbers, the closed-form energy of a Plummer sphere, Newton's third
law, F = -grad U, the far-field monopole limit and symmetry invariances.
"""
import math

import numpy as np
import pytest

import oracle
import workloads


def test_two_body_hand_values():
    # Bodies at (0,0,0) and (3,4,0), |r| = 5, masses 5 and 2, G = 1.5, eps = 0.
    # a_0 = G m_1 (x_1 - x_0) / 125 = 3 (3,4,0) / 125 = (0.072, 0.096, 0)
    # a_1 = G m_0 (x_0 - x_1) / 125 = 7.5 (-3,-4,0) / 125 = (-0.18, -0.24, 0)
    # phi_0 = -G m_1 / 5 = -0.6, phi_1 = -G m_0 / 5 = -1.5
    x = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    m = np.array([5.0, 2.0])
    acc, phi = oracle.grav_accel(x, m, G=1.5, eps=0.0, potential=True)
    np.testing.assert_allclose(acc, [[0.072, 0.096, 0.0], [-0.18, -0.24, 0.0]], rtol=1e-15,
                               atol=1e-17)
    np.testing.assert_allclose(phi, [-0.6, -1.5], rtol=1e-15)


def test_two_body_softened_hand_values():
    # Same pair with eps = sqrt(11): s^2 = 25 + 11 = 36, s = 6, s^3 = 216.
    # a_0 = 3 (3,4,0) / 216, phi_0 = -3 / 6 = -0.5 ; a_1 = 7.5 (-3,-4,0)/216
    x = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    m = np.array([5.0, 2.0])
    acc, phi = oracle.grav_accel(x, m, G=1.5, eps=math.sqrt(11.0), potential=True)
    np.testing.assert_allclose(acc[0], [9.0 / 216, 12.0 / 216, 0.0], rtol=1e-14, atol=1e-17)
    np.testing.assert_allclose(acc[1], [-22.5 / 216, -30.0 / 216, 0.0], rtol=1e-14,
                               atol=1e-17)
    np.testing.assert_allclose(phi, [-0.5, -1.25], rtol=1e-14)


def test_single_particle_and_self_exclusion():
    acc, phi = oracle.grav_accel([[1.0, 2.0, 3.0]], [4.0], eps=0.0, potential=True)
    assert np.all(acc == 0.0) and np.all(phi == 0.0)


def test_high_precision_brute_force():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    g = workloads.plummer(12, seed=11)
    x, m = g.x, g.m * np.linspace(0.5, 1.5, 12)
    G, eps = 1.3, 0.05
    acc, phi = oracle.grav_accel(x, m, G=G, eps=eps, potential=True)
    for i in range(12):
        ax = [mp.mpf(0)] * 3
        p = mp.mpf(0)
        for j in range(12):
            if i == j:
                continue
            r = [mp.mpf(x[i, a]) - mp.mpf(x[j, a]) for a in range(3)]
            s2 = r[0] ** 2 + r[1] ** 2 + r[2] ** 2 + mp.mpf(eps) ** 2
            for a in range(3):
                ax[a] -= mp.mpf(m[j]) * r[a] / s2 ** mp.mpf(1.5)
            p -= mp.mpf(m[j]) / mp.sqrt(s2)
        ref = np.array([float(G * v) for v in ax])
        assert np.linalg.norm(acc[i] - ref) <= 1e-14 * np.linalg.norm(ref)
        assert abs(phi[i] - float(G * p)) <= 1e-14 * abs(float(G * p))


def test_newton_third_law():
    g = workloads.plummer(512, seed=1)
    acc = oracle.grav_accel(g.x, g.m, eps=0.01)
    total = np.sum(g.m[:, None] * acc, axis=0)
    scale = np.sum(g.m[:, None] * np.abs(acc))
    assert np.all(np.abs(total) <= 1e-14 * scale)


def test_force_is_minus_gradient_of_potential():
    g = workloads.plummer(40, seed=7)
    sysm = oracle.GravSystem(g.m, G=1.0, eps=0.02)
    acc = sysm.accel(g.x)
    h = 1e-5
    rng = np.random.default_rng(0)
    for i in rng.choice(40, 6, replace=False):
        for a in range(3):
            xp, xm = g.x.copy(), g.x.copy()
            xp[i, a] += h
            xm[i, a] -= h
            dU = (sysm.potential_energy(xp) - sysm.potential_energy(xm)) / (2 * h)
            # -dU/dx_i = m_i a_i
            assert abs(-dU - g.m[i] * acc[i, a]) <= 1e-7 * abs(g.m[i]) * np.abs(acc[i]).max()


def test_plummer_potential_energy_closed_form_and_virial():
    # Infinite Plummer sphere with G = M = a = 1: U = -3 pi / 32 = -0.29452...
    # and the equilibrium distribution function is in virial balance, 2K = -U.
    g = workloads.plummer(8192, seed=3)
    sysm = oracle.GravSystem(g.m, G=1.0, eps=0.0)
    d = oracle.diagnostics(sysm, g.x, g.v)
    assert abs(d["U"] / (-3.0 * math.pi / 32.0) - 1.0) < 0.03
    assert abs(2.0 * d["K"] / -d["U"] - 1.0) < 0.05


def test_far_field_monopole():
    g = workloads.plummer(200, seed=5)
    x = np.vstack([g.x * 0.1, [[0.0, 0.0, 1000.0]]])
    m = np.append(g.m, 1e-9)
    acc, phi = oracle.grav_accel(x, m, G=2.0, eps=0.0, idx=[200], potential=True)
    M = g.m.sum()
    # phi -> -G M / r and a -> -G M r_hat / r^2 up to quadrupole terms (r_cluster/r)^2
    assert abs(phi[0] / (-2.0 * M / 1000.0) - 1.0) < 1e-6
    np.testing.assert_allclose(acc[0], [0.0, 0.0, -2.0 * M / 1000.0 ** 2], rtol=1e-5,
                               atol=1e-11)


def test_permutation_translation_rotation_invariance():
    g = workloads.plummer(300, seed=9)
    acc = oracle.grav_accel(g.x, g.m, eps=0.01)
    perm = np.random.default_rng(1).permutation(300)
    acc_p = oracle.grav_accel(g.x[perm], g.m[perm], eps=0.01)
    np.testing.assert_allclose(acc_p, acc[perm], rtol=1e-12, atol=1e-14)
    acc_t = oracle.grav_accel(g.x + np.array([0.3, -0.2, 0.7]), g.m, eps=0.01)
    np.testing.assert_allclose(acc_t, acc, rtol=1e-10, atol=1e-12)
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    acc_r = oracle.grav_accel(g.x @ R.T, g.m, eps=0.01)
    np.testing.assert_allclose(acc_r, acc @ R.T, rtol=1e-10, atol=1e-12)


def test_subset_matches_full():
    g = workloads.plummer(257, seed=2)
    acc, phi = oracle.grav_accel(g.x, g.m, eps=0.01, potential=True)
    idx = [0, 5, 256, 100]
    a2, p2 = oracle.grav_accel(g.x, g.m, eps=0.01, idx=idx, potential=True)
    np.testing.assert_array_equal(a2, acc[idx])
    np.testing.assert_array_equal(p2, phi[idx])


def test_softening_limit():
    # eps -> 0 recovers the unsoftened sum (continuity at a fixed configuration)
    g = workloads.plummer(64, seed=4)
    a0 = oracle.grav_accel(g.x, g.m, eps=0.0)
    a1 = oracle.grav_accel(g.x, g.m, eps=1e-7)
    np.testing.assert_allclose(a1, a0, rtol=1e-6, atol=1e-9)


def test_thread_count_does_not_change_the_forces():
    """Each target's sum runs in index order inside one thread, so the oracle's
    forces are bitwise the same on one thread and on all of them."""
    g = workloads.plummer(300, seed=17)
    prev = oracle.set_threads(None)
    try:
        oracle.set_threads(1)
        a1 = oracle.grav_accel(g.x, g.m, eps=0.01)
        oracle.set_threads(max(2, prev))
        a2 = oracle.grav_accel(g.x, g.m, eps=0.01)
    finally:
        oracle.set_threads(prev)
    assert np.array_equal(a1, a2)
