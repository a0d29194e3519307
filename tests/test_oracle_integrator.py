"""Pins for the FP64 kick-drift-kick leapfrog (the update step of Sec. 1).

Kepler's two-body orbit in closed form (solved through Kepler's equation)
gives second-order convergence; the energy error of a Plummer cluster scales
as dt^2; the scheme is time-reversible and conserves momentum.
"""
import math

import numpy as np

import oracle
import workloads


def _kepler_orbit(t, a=1.0, e=0.5, mu=1.0):
    """Relative position of a bound Kepler orbit at time t (periapsis at t=0)."""
    n = math.sqrt(mu / a ** 3)
    M = n * t
    E = M
    for _ in range(60):
        E -= (E - e * math.sin(E) - M) / (1.0 - e * math.cos(E))
    return np.array([a * (math.cos(E) - e), a * math.sqrt(1 - e * e) * math.sin(E), 0.0])


def _kepler_run(dt, T, e=0.5):
    m1, m2 = 0.7, 0.3
    a = 1.0
    rp = a * (1 - e)
    vp = math.sqrt((m1 + m2) * (1 + e) / (a * (1 - e)))
    rel_x = np.array([rp, 0.0, 0.0])
    rel_v = np.array([0.0, vp, 0.0])
    x = np.array([-m2 / (m1 + m2) * rel_x, m1 / (m1 + m2) * rel_x])
    v = np.array([-m2 / (m1 + m2) * rel_v, m1 / (m1 + m2) * rel_v])
    sysm = oracle.GravSystem([m1, m2], G=1.0, eps=0.0)
    xT, _ = oracle.leapfrog(sysm, x, v, dt, int(round(T / dt)))
    rel = xT[1] - xT[0]
    return np.linalg.norm(rel - _kepler_orbit(T, a, e, m1 + m2))


def test_kepler_second_order_convergence():
    period = 2 * math.pi
    errs = [_kepler_run(period / k, period) for k in (400, 800, 1600)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, errs
    assert errs[2] < 1e-3


def test_energy_error_scales_as_dt_squared():
    g = workloads.plummer(64, seed=8)
    sysm = oracle.GravSystem(g.m, eps=0.05)
    E0 = oracle.diagnostics(sysm, g.x, g.v)["E"]
    errs = []
    for dt in (2e-3, 1e-3):
        xs, vs = oracle.leapfrog(sysm, g.x, g.v, dt, int(round(0.2 / dt)), store=True)
        errs.append(max(abs(oracle.diagnostics(sysm, x, v)["E"] - E0)
                        for x, v in zip(xs[::10], vs[::10])))
    assert 3.0 < errs[0] / errs[1] < 5.0, errs


def test_time_reversibility_and_momentum():
    g = workloads.plummer(32, seed=6)
    sysm = oracle.GravSystem(g.m, eps=0.05)
    x1, v1 = oracle.leapfrog(sysm, g.x, g.v, 1e-3, 50)
    x2, v2 = oracle.leapfrog(sysm, x1, -v1, 1e-3, 50)
    np.testing.assert_allclose(x2, g.x, atol=1e-12)
    np.testing.assert_allclose(-v2, g.v, atol=1e-12)
    P0 = np.sum(g.m[:, None] * g.v, axis=0)
    P1 = np.sum(g.m[:, None] * v1, axis=0)
    np.testing.assert_allclose(P1, P0, atol=1e-15)


def test_diagnostics_hand_values():
    """K, P and L of two particles worked by hand (distinct masses, motion in
    different planes), so that a swapped cross product, a dropped mass or a
    missing factor 1/2 each change a printed value:
      m1 = 3 at (1, 0, 0) moving (0, 2, 0):  m x x v = 3 (0, 0, 2) = (0, 0, 6)
      m2 = 2 at (0, 0, 1) moving (1, 0, 0):  m x x v = 2 (0, 1, 0) = (0, 2, 0)
    L = (0, 2, 6); P = (2, 6, 0); K = 3 * 4 / 2 + 2 * 1 / 2 = 7."""
    x = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    v = np.array([[0.0, 2.0, 0.0], [1.0, 0.0, 0.0]])
    sysm = oracle.GravSystem(np.array([3.0, 2.0]), eps=0.0)
    d = oracle.diagnostics(sysm, x, v)
    np.testing.assert_array_equal(d["L"], [0.0, 2.0, 6.0])
    np.testing.assert_array_equal(d["P"], [2.0, 6.0, 0.0])
    assert d["K"] == 7.0
    # U of the pair: -G m1 m2 / r with r = sqrt(2)
    assert abs(d["U"] + 6.0 / math.sqrt(2.0)) <= 1e-15 * 6.0


def test_angular_momentum_of_a_circular_orbit():
    """Two bodies on a circular orbit about their resting centre of mass, moving
    counter-clockwise in the x-y plane: L = mu r v_rel along +z, with
    mu = m1 m2 / (m1 + m2) and v_rel = sqrt(G (m1 + m2) / r) (closed form)."""
    m1, m2, r, G = 0.7, 0.3, 2.0, 1.0
    vrel = math.sqrt(G * (m1 + m2) / r)
    rel_x, rel_v = np.array([r, 0.0, 0.0]), np.array([0.0, vrel, 0.0])
    x = np.array([-m2 / (m1 + m2) * rel_x, m1 / (m1 + m2) * rel_x])
    v = np.array([-m2 / (m1 + m2) * rel_v, m1 / (m1 + m2) * rel_v])
    sysm = oracle.GravSystem(np.array([m1, m2]), G=G, eps=0.0)
    L = oracle.diagnostics(sysm, x, v)["L"]
    mu = m1 * m2 / (m1 + m2)
    np.testing.assert_allclose(L, [0.0, 0.0, mu * r * vrel], rtol=1e-15, atol=1e-16)
    # a quarter period later the orbit has turned; L is the same vector
    period = 2.0 * math.pi * r / vrel
    xs, vs = oracle.leapfrog(sysm, x, v, period / 4000.0, 1000)
    np.testing.assert_allclose(oracle.diagnostics(sysm, xs, vs)["L"], L, rtol=1e-13,
                               atol=1e-15)


def test_leapfrog_conserves_angular_momentum_to_rounding():
    """Central pair forces change sum m x x v by sum_(i<j) (x_i - x_j) x F_ij = 0 in a
    kick, and a drift adds m v x v = 0, so KDK conserves L exactly up to FP64
    rounding, while the energy (not conserved by KDK) drifts."""
    g = workloads.plummer(64, seed=8)
    sysm = oracle.GravSystem(g.m, eps=0.02)
    L0 = oracle.diagnostics(sysm, g.x, g.v)["L"]
    x, v = oracle.leapfrog(sysm, g.x, g.v, 1e-2, 200)
    L1 = oracle.diagnostics(sysm, x, v)["L"]
    scale = float(np.sum(g.m * np.linalg.norm(np.cross(g.x, g.v), axis=1)))
    assert np.all(np.abs(L1 - L0) <= 1e-13 * scale), (L0, L1)
    assert np.linalg.norm(L0) > 1e-3 * scale  # a rotating sample: the check is not 0 = 0


def _kepler_hermite(dt, T, e=0.5):
    m1, m2 = 0.7, 0.3
    rp = 1.0 - e
    vp = math.sqrt((m1 + m2) * (1 + e) / (1.0 - e))
    rel_x = np.array([rp, 0.0, 0.0])
    rel_v = np.array([0.0, vp, 0.0])
    x = np.array([-m2 / (m1 + m2) * rel_x, m1 / (m1 + m2) * rel_x])
    v = np.array([-m2 / (m1 + m2) * rel_v, m1 / (m1 + m2) * rel_v])
    xT, _ = oracle.hermite(x, v, np.array([m1, m2]), dt, int(round(T / dt)), eps=0.0)
    return np.linalg.norm((xT[1] - xT[0]) - _kepler_orbit(T, 1.0, e, m1 + m2))


def test_hermite_fourth_order_on_kepler():
    """The Hermite scheme on acceleration + jerk converges at fourth order: halving dt
    divides the error by about 16 (the closed-form Kepler orbit is the reference)."""
    period = 2 * math.pi
    errs = [_kepler_hermite(period / k, period) for k in (200, 400, 800)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 13.0 < r1 < 19.0 and 13.0 < r2 < 19.0, errs
    assert errs[2] < 1e-6


def test_hermite_conserves_momentum_and_energy():
    g = workloads.plummer(48, seed=21)
    sysm = oracle.GravSystem(g.m, eps=0.05)
    xs, vs = oracle.hermite(g.x, g.v, g.m, 1e-3, 100, eps=0.05, store=True)
    E0 = oracle.diagnostics(sysm, xs[0], vs[0])["E"]
    E1 = oracle.diagnostics(sysm, xs[-1], vs[-1])["E"]
    assert abs(E1 - E0) <= 1e-9 * abs(E0)
    P = np.sum(g.m[:, None] * vs[-1], axis=0)
    np.testing.assert_allclose(P, np.sum(g.m[:, None] * g.v, axis=0), atol=1e-15)
