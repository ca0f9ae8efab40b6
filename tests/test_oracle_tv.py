"""Pins of the oracle's weighted TV and its prox (no GPU).

* TV of images with a closed-form value (constant, a step edge, a ramp).
* L and L^T are adjoint (the dual maps of Beck & Teboulle 2009).
* The prox: the identity cases, the two-pixel closed form, and on a small
  image the FGP result against an independent solver (L-BFGS on the
  smoothed weighted TV, smoothing continued to 1e-7).
"""
import numpy as np
import pytest
from scipy import optimize

from oracle import tv


def test_tv_closed_forms():
    m, n = 6, 8
    assert tv.tv_norm(np.full((m, n), 3.0 + 1j)) == 0.0
    step = np.zeros((m, n))
    step[:, n // 2:] = 2.5
    assert tv.tv_norm(step) == pytest.approx(2.5 * m, rel=1e-15)
    a, b = 0.7, -1.3
    ramp = a * np.arange(m)[:, None] + b * np.arange(n)[None, :]
    want = (m - 1) * (n - 1) * np.hypot(a, b) + (n - 1) * abs(b) + (m - 1) * abs(a)
    assert tv.tv_norm(ramp) == pytest.approx(want, rel=1e-14)
    w = np.full((m, n), 0.5)
    assert tv.tv_norm(ramp, w) == pytest.approx(0.5 * want, rel=1e-14)
    # complex differences count by modulus: i * x has the same TV as x
    assert tv.tv_norm(1j * ramp) == pytest.approx(want, rel=1e-14)


def test_L_and_LT_are_adjoint():
    rng = np.random.default_rng(1)
    m, n = 7, 5
    x = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    p = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    q = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    p[-1, :] = 0
    q[:, -1] = 0
    g1, g2 = tv.op_LT(x)
    lhs = np.vdot(tv.op_L(p, q), x)
    rhs = np.vdot(p, g1) + np.vdot(q, g2)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # L^T is minus the gradient
    d1, d2 = tv.grad(x)
    assert np.array_equal(g1, -d1) and np.array_equal(g2, -d2)


def test_prox_identity_cases():
    rng = np.random.default_rng(2)
    b = rng.standard_normal((5, 5)) + 1j * rng.standard_normal((5, 5))
    assert np.array_equal(tv.prox_tv(b, 0.0), b)
    c = np.full((5, 5), 1.5 - 0.5j)
    assert np.allclose(tv.prox_tv(c, 0.7), c, rtol=0, atol=1e-15)


@pytest.mark.parametrize("b1,b2,lam,w", [(0.0, 3.0, 0.5, 1.0), (1.0, 1.4, 0.5, 1.0), (2.0, -1.0, 0.3, 0.5),
                                         (1 + 1j, -2 + 0.5j, 0.4, 1.0)])
def test_prox_two_pixels_closed_form(b1, b2, lam, w):
    # One difference: min 1/2|x1-b1|^2 + 1/2|x2-b2|^2 + lam w |x2 - x1| moves both
    # values towards each other by lam w (or to the mean when they are closer).
    b = np.array([[b1], [b2]], dtype=np.complex128)
    weights = np.array([[w], [w]])
    x = tv.prox_tv(b, lam, weights, iters=500)
    d = b2 - b1
    if abs(d) <= 2 * lam * w:
        want = np.full(2, (b1 + b2) / 2)
    else:
        u = d / abs(d)
        want = np.array([b1 + lam * w * u, b2 - lam * w * u])
    assert np.allclose(x.ravel(), want, rtol=0, atol=1e-9)


def prox_objective(x, b, lam, w):
    return 0.5 * np.sum(np.abs(x - b) ** 2) + lam * tv.tv_norm(x, w)


def smoothed_prox(b, lam, w):
    """Independent reference: minimise 1/2||x - b||^2 + lam sum w sqrt(|grad x|^2 + mu^2)
    (smooth and strictly convex) by L-BFGS, continuing mu down to 1e-7."""
    m, n = b.shape
    x = b.ravel().copy()
    for mu in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7):
        def f(v, mu=mu):
            X = v.reshape(m, n)
            d1, d2 = tv.grad(X)
            sq = np.sqrt(d1 ** 2 + d2 ** 2 + mu ** 2)
            g = X - b
            c1, c2 = lam * w * d1 / sq, lam * w * d2 / sq
            g[:-1, :] -= c1[:-1, :]
            g[1:, :] += c1[:-1, :]
            g[:, :-1] -= c2[:, :-1]
            g[:, 1:] += c2[:, :-1]
            return 0.5 * np.sum((X - b) ** 2) + lam * np.sum(w * sq), g.ravel()
        x = optimize.minimize(f, x, jac=True, method="L-BFGS-B",
                              options={"maxiter": 20000, "ftol": 1e-16, "gtol": 1e-13}).x
    return x.reshape(m, n)


def test_prox_against_independent_solver():
    rng = np.random.default_rng(3)
    m, n = 4, 5
    b = rng.uniform(0, 1, (m, n))
    b[:, 3:] += 1.0
    w = rng.uniform(0.5, 1.5, (m, n))
    lam = 0.15
    x_fgp = tv.prox_tv(b, lam, w, iters=3000)
    x_ref = smoothed_prox(b, lam, w)
    f_fgp, f_ref = prox_objective(x_fgp, b, lam, w), prox_objective(x_ref, b, lam, w)
    assert f_fgp <= f_ref + 1e-9
    assert np.max(np.abs(x_fgp - x_ref)) < 1e-5
    # FGP converges: the default inner count is already close
    f20 = prox_objective(tv.prox_tv(b, lam, w), b, lam, w)
    assert f_fgp <= f20 <= f_fgp * (1 + 1e-2)
