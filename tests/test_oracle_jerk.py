"""Pins for the FP64 acceleration-and-jerk oracle (Table 1 "Gravity (accel & jerk)"):
hand-worked two-body values, the jerk as the time derivative of the acceleration
along uniform motion (central differences), Newton's third law, and agreement of
the acceleration part with Eq. 1."""
import numpy as np

import oracle
import workloads


def test_two_body_hand_values():
    # x0 = 0, x1 = (3,4,0), v0 = 0, v1 = (1,0,0), m1 = 2, G = 1, eps = 0:
    # r = (3,4,0), u = (1,0,0), r.u = 3, s = 5
    # j_0 = 2 [ (1,0,0)/125 - 3*3*(3,4,0)/3125 ] = (-0.00128, -0.02304, 0)
    x = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    v = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    m = np.array([5.0, 2.0])
    a, j = oracle.grav_jerk(x, v, m, G=1.0, eps=0.0)
    np.testing.assert_allclose(a[0], [6.0 / 125, 8.0 / 125, 0.0], rtol=1e-15)
    np.testing.assert_allclose(j[0], [-0.00128, -0.02304, 0.0], rtol=1e-13, atol=1e-18)
    # body 1 sees u = -(1,0,0), r = -(3,4,0), r.u = 3: j_1 = 5 [(-1,0,0)/125 + 9 (3,4,0)/3125]
    np.testing.assert_allclose(j[1], [5 * (-0.008 + 0.00864), 5 * 0.01152, 0.0], rtol=1e-13)


def test_jerk_is_time_derivative_of_acceleration():
    g = workloads.plummer(64, seed=3)
    m = g.m * np.linspace(0.5, 1.5, 64)
    a, j = oracle.grav_jerk(g.x, g.v, m, G=1.3, eps=0.05)
    h = 1e-5
    ap = oracle.grav_accel(g.x + h * g.v, m, G=1.3, eps=0.05)
    am = oracle.grav_accel(g.x - h * g.v, m, G=1.3, eps=0.05)
    fd = (ap - am) / (2 * h)
    np.testing.assert_allclose(j, fd, rtol=1e-6, atol=1e-8 * np.abs(j).max())
    np.testing.assert_allclose(a, oracle.grav_accel(g.x, m, G=1.3, eps=0.05), rtol=1e-13,
                               atol=1e-16)


def test_newton_third_law_for_jerk():
    g = workloads.plummer(200, seed=4)
    _, j = oracle.grav_jerk(g.x, g.v, g.m, eps=0.01)
    assert np.all(np.abs(np.sum(g.m[:, None] * j, axis=0)) <= 1e-14 * np.sum(g.m[:, None] * np.abs(j)))


def test_target_subset_matches_full():
    g = workloads.plummer(200, seed=23)
    v = np.random.default_rng(2).standard_normal((200, 3))
    a, j = oracle.grav_jerk(g.x, v, g.m, eps=0.02)
    idx = np.array([199, 0, 57, 58])
    a2, j2 = oracle.grav_jerk(g.x, v, g.m, eps=0.02, idx=idx)
    assert np.array_equal(a2, a[idx]) and np.array_equal(j2, j[idx])
