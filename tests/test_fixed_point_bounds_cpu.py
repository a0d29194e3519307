"""The a-priori bounds behind the fixed-point scales (CPU, FP64).

The Newton-symmetric gravity kernels add their per-block partials as 64-bit
fixed point, scaled by the largest 2^S that keeps every sum a particle can reach
below 2^62. The scale comes from a bound on the sum of the magnitudes of a
particle's pair terms (every partial sum is smaller still):

- forces (Eq. 1): |m_j d / s^3| <= m_j max_r r / (r^2 + eps^2)^(3/2)
  = m_j 2 / (3 sqrt(3) eps^2), and |m_j / s| <= m_j / eps;
- the force VJP: |y^3 (I - 3 y^2 d d^T) w| <= 2 y^3 |w| <= 2 / eps^3 |w| with
  w = m_k lam_j - m_j lam_k (the matrix has eigenvalues 1 and 1 - 3 r^2 / s^2,
  which lies in (-2, 1]), and |(lam_j . d) y^3| <= |lam_j| 2 / (3 sqrt(3) eps^2).

Here every pair term is evaluated in FP64 and the sums of their magnitudes are
checked against those bounds, on random systems and on the configurations that
come closest: partners at r = eps / sqrt(2), where r / s^3 peaks, and at r = 0 for
the VJP matrix (s = eps, y^3 = 1 / eps^3)."""
import math

import numpy as np
import pytest

C = 2.0 / (3.0 * math.sqrt(3.0))  # max of r / (r^2 + 1)^(3/2)


def _pair_terms(x, m, lam, eps):
    """Per pair (k, j != k): the force term m_j d / s^3, the potential term m_j / s,
    the VJP term y^3 (w - 3 y^2 (d . w) d) and the VJP mass term (lam_j . d) y^3."""
    d = x[None, :, :] - x[:, None, :]                      # d[k, j] = x_j - x_k
    s2 = np.sum(d * d, axis=2) + eps * eps
    y = 1.0 / np.sqrt(s2)
    np.fill_diagonal(y, 0.0)
    y3 = y ** 3
    f = m[None, :, None] * d * y3[:, :, None]
    phi = m[None, :] * y
    w = m[:, None, None] * lam[None, :, :] - m[None, :, None] * lam[:, None, :]
    dw = np.sum(d * w, axis=2)
    g = y3[:, :, None] * (w - 3.0 * (y * y * dw)[:, :, None] * d)
    gm = np.sum(lam[None, :, :] * d, axis=2) * y3
    return f, phi, g, gm


def _check(x, m, lam, eps):
    f, phi, g, gm = _pair_terms(x, m, lam, eps)
    M, mmax = np.abs(m).sum(), np.abs(m).max()
    ln = np.linalg.norm(lam, axis=1)
    L, lmax = ln.sum(), ln.max()
    # forces: per component and for the norm of each term
    assert np.linalg.norm(f, axis=2).sum(axis=1).max() <= M * C / eps**2 * (1 + 1e-12)
    assert np.abs(phi).sum(axis=1).max() <= M / eps * (1 + 1e-12)
    # VJP
    assert np.linalg.norm(g, axis=2).sum(axis=1).max() <= (
        2.0 * (mmax * L + lmax * M) / eps**3 * (1 + 1e-12))
    assert np.abs(gm).sum(axis=1).max() <= C * L / eps**2 * (1 + 1e-12)
    return f, g, gm


@pytest.mark.parametrize("seed", range(6))
def test_bounds_hold_on_random_systems(seed):
    rng = np.random.default_rng(seed)
    n = 60
    x = rng.standard_normal((n, 3)) * rng.uniform(0.01, 1.0)
    m = rng.uniform(0.1, 2.0, n)
    lam = rng.standard_normal((n, 3))
    _check(x, m, lam, eps=rng.uniform(0.005, 0.2))


def test_bounds_are_reached_at_the_extreme_configurations():
    """Partners at r = eps / sqrt(2) put every force term and every VJP mass term
    at its largest magnitude C / eps^2, which the bounds count for each pair. For
    the VJP matrix term, y^3 max(1, |1 - 3 r^2 y^2|) peaks at r = 0 at 1 / eps^3: a
    coincident pair reaches |w| / eps^3, half the bound's 2 |w| / eps^3 (the 2 is
    the matrix norm taken at its worst over r, apart from y^3)."""
    eps = 0.01
    # one target, six partners on the axes at r = eps / sqrt(2): all terms add up
    # only along one axis, so the sum of magnitudes is what the bound counts
    r = eps / math.sqrt(2.0)
    pts = [np.zeros(3)] + [r * v for v in np.eye(3)] + [-r * v for v in np.eye(3)]
    x = np.array(pts)
    m = np.ones(len(pts))
    lam = np.zeros_like(x)
    lam[1:, 0] = 1.0
    f, g, gm = _check(x, m, lam, eps)
    per_term = np.linalg.norm(f[0], axis=1)[1:]
    np.testing.assert_allclose(per_term, C / eps**2, rtol=1e-12)   # each term at the max
    # VJP: the mass term of the target reaches |lam_j| r / s^3 = C / eps^2 per partner
    # along the axis where lam_j is parallel to d
    np.testing.assert_allclose(np.abs(gm[0, 1]), C / eps**2, rtol=1e-12)
    # coincident pair: y = 1 / eps, the matrix is the identity, |term| = |w| / eps^3
    x2 = np.zeros((2, 3))
    m2 = np.array([1.0, 1.0])
    lam2 = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    _, g2, _ = _check(x2, m2, lam2, eps)
    np.testing.assert_allclose(np.linalg.norm(g2[1, 0]), 1.0 / eps**3, rtol=1e-12)
