"""Pins of the oracle's proximity operators (no GPU).

Each prox is checked against the optimality condition of its definition
(§4.1: prox_f(x) = argmin_z f(z) + 1/2 ||x - z||^2) and, for the soft
threshold, against brute-force minimisation on a grid.  The l2-ball
projection follows the set B of §4.3; the formula printed as eq. prox2
projects onto a ball around 0 instead, which the last test shows.
"""
import numpy as np
import pytest

from oracle import prox
from paper_1307_4370_gb300 import inputs


def test_soft_threshold_optimality():
    rng = np.random.default_rng(0)
    a = inputs.random_vis(2000, rng)
    lam = rng.uniform(0.0, 1.5, a.size)
    r = prox.soft_threshold(a, lam)
    zero = np.abs(r) == 0
    # r = 0 exactly when |a| <= lam; otherwise a - r = lam r/|r| (the subgradient of lam|.|)
    assert np.array_equal(zero, np.abs(a) <= lam)
    nz = ~zero
    assert np.allclose(a[nz] - r[nz], lam[nz] * r[nz] / np.abs(r[nz]), atol=1e-14)
    assert np.all(prox.soft_threshold(np.zeros(3, complex), 0.5) == 0)


def test_soft_threshold_brute_force():
    rng = np.random.default_rng(1)
    g = np.linspace(-2, 2, 801)
    Z = g[None, :] + 1j * g[:, None]
    for _ in range(6):
        a = complex(*rng.uniform(-1.5, 1.5, 2))
        lam = rng.uniform(0.1, 1.0)
        obj = lam * np.abs(Z) + 0.5 * np.abs(a - Z) ** 2
        zbest = Z.ravel()[np.argmin(obj)]
        assert abs(prox.soft_threshold(np.array([a]), lam)[0] - zbest) <= 2 * (g[1] - g[0])


def test_l2_ball_projection():
    rng = np.random.default_rng(2)
    M = 500
    y = inputs.random_vis(M, rng)
    eps = 3.0
    r = y + 2.0 * inputs.random_vis(M, rng)  # outside: ||r - y|| ~ 2 sqrt(M)
    p = prox.project_l2_ball(r, y, eps)
    assert np.linalg.norm(p - y) == pytest.approx(eps, rel=1e-13)
    assert np.allclose(prox.project_l2_ball(p, y, eps), p, atol=1e-14)  # idempotent
    inside = y + 0.05 * inputs.random_vis(M, rng)
    assert np.array_equal(prox.project_l2_ball(inside, y, eps), inside)
    # obtuse-angle condition Re <r - P r, z - P r> <= 0 for points z of B
    for _ in range(20):
        d = inputs.random_vis(M, rng)
        z = y + rng.uniform(0, eps) * d / np.linalg.norm(d)
        assert np.vdot(r - p, z - p).real <= 1e-9


def test_printed_prox2_is_not_the_projection():
    # min(1, eps/||r||) r is generally outside B = {||y - r|| <= eps}.
    rng = np.random.default_rng(3)
    y = 5.0 + inputs.random_vis(100, rng)
    r = y + inputs.random_vis(100, rng)
    eps = 1.0
    printed = min(1.0, eps / np.linalg.norm(r)) * r
    assert np.linalg.norm(y - printed) > eps
    assert np.linalg.norm(y - prox.project_l2_ball(r, y, eps)) <= eps * (1 + 1e-14)


def test_positive_orthant_projection():
    rng = np.random.default_rng(4)
    a = inputs.random_vis(1000, rng)
    p = prox.project_positive(a)
    assert np.all(p.imag == 0) and np.all(p.real >= 0)
    assert np.array_equal(prox.project_positive(p), p)
    # obtuse-angle condition against random points of the orthant
    for _ in range(20):
        z = np.abs(rng.standard_normal(a.size)).astype(complex)
        assert np.vdot(a - p, z - p).real <= 1e-12
