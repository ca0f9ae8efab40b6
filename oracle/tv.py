"""Weighted total variation and its proximity operator (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

§3.3 (eq. tvproblem) and §5 define the TV prior ||x||_TV = ||grad x||_1 with
|grad x| the gradient magnitude (isotropic, Rudin et al. 1992), and its
weighted form ||W grad x||_1 for the reweighted problem; SOPT computes the
prox of the weighted TV with the fast gradient projection of Beck & Teboulle
(2009) applied to the dual problem.  This module follows that construction.

Discrete gradient (Neumann boundary): for an m x n image x,

    (grad x)_{i,j} = (d1, d2),  d1 = x_{i+1,j} - x_{i,j} (0 on the last row),
                                d2 = x_{i,j+1} - x_{i,j} (0 on the last column),
    ||W grad x||_1 = sum_{i,j} w_{i,j} sqrt(|d1|^2 + |d2|^2)

(moduli of complex differences: x in C^N is R^2 per pixel, §4.1).  With the
dual pair (p, q) (p on the first m - 1 rows, q on the first n - 1 columns,
zero elsewhere) the two linear maps of Beck & Teboulle are

    L(p, q)_{i,j} = p_{i,j} + q_{i,j} - p_{i-1,j} - q_{i,j-1}   (= -div),
    L^T(x)        = (x_{i,j} - x_{i+1,j},  x_{i,j} - x_{i,j+1})  (= -grad),

and prox_{lam TV_W}(b) = argmin_x 1/2 ||x - b||^2 + lam ||W grad x||_1 is
x = b - lam L(p, q) at the solution of the dual, found by fast projected
gradient (FGP) with step 1/(8 lam) onto the set |(p, q)_{i,j}| <= w_{i,j}:

    (r, s) = (p0, q0) = 0, t = 1; for k = 1..K:
        (p, q)_k = Proj[(r, s) + 1/(8 lam) L^T(b - lam L(r, s))]
        t' = (1 + sqrt(1 + 4 t^2)) / 2
        (r, s) = (p, q)_k + ((t - 1) / t') ((p, q)_k - (p, q)_{k-1}); t = t'
    x = b - lam L(p_K, q_K)

Pinned by ``tests/test_oracle_tv.py``: TV of closed-form images, the
adjointness of L and L^T, prox optimality against an independent
constrained solver, and the identity cases.
"""
from __future__ import annotations

import numpy as np

FGP_ITERS = 20  # inner iterations per prox (the paper gives none; the reading taken here)


def grad(x: np.ndarray):
    """Forward differences (d1, d2) with zeros on the last row / column."""
    x = np.asarray(x)
    d1 = np.zeros_like(x)
    d2 = np.zeros_like(x)
    d1[:-1, :] = x[1:, :] - x[:-1, :]
    d2[:, :-1] = x[:, 1:] - x[:, :-1]
    return d1, d2


def tv_norm(x: np.ndarray, w: np.ndarray | None = None) -> float:
    """||W grad x||_1 (isotropic)."""
    d1, d2 = grad(x)
    mag = np.sqrt(np.abs(d1) ** 2 + np.abs(d2) ** 2)
    return float(np.sum(mag if w is None else np.asarray(w) * mag))


def grad_magnitude(x: np.ndarray) -> np.ndarray:
    """|grad x| per pixel."""
    d1, d2 = grad(x)
    return np.sqrt(np.abs(d1) ** 2 + np.abs(d2) ** 2)


def op_L(p: np.ndarray, q: np.ndarray) -> np.ndarray:
    """L(p, q) = p_{i,j} + q_{i,j} - p_{i-1,j} - q_{i,j-1}, with p on rows 0..m-2 and
    q on columns 0..n-2 (their last row / column are not part of the dual)."""
    out = np.zeros(np.shape(p), dtype=np.result_type(p, q, np.float64))
    out[:-1, :] += p[:-1, :]
    out[:, :-1] += q[:, :-1]
    out[1:, :] -= p[:-1, :]
    out[:, 1:] -= q[:, :-1]
    return out


def op_LT(x: np.ndarray):
    """L^T(x) = (x_{i,j} - x_{i+1,j}, x_{i,j} - x_{i,j+1}), zero on the last row / column."""
    d1, d2 = grad(x)
    return -d1, -d2


def project_dual(p: np.ndarray, q: np.ndarray, w: np.ndarray | None):
    """Projection of each pair (p_ij, q_ij) onto the disc of radius w_ij (1 without weights)."""
    mag = np.sqrt(np.abs(p) ** 2 + np.abs(q) ** 2)
    rad = np.ones_like(mag) if w is None else np.asarray(w, dtype=np.float64)
    f = np.where(mag > rad, rad / np.where(mag > 0, mag, 1.0), 1.0)
    return p * f, q * f


def prox_tv(b: np.ndarray, lam: float, w: np.ndarray | None = None, iters: int = FGP_ITERS) -> np.ndarray:
    """prox_{lam ||W grad .||_1}(b) by FGP on the dual (Beck & Teboulle 2009)."""
    b = np.asarray(b, dtype=np.complex128)
    if lam <= 0.0:
        return b.copy()
    p = np.zeros_like(b)
    q = np.zeros_like(b)
    r, s = p.copy(), q.copy()
    t = 1.0
    for _ in range(iters):
        g1, g2 = op_LT(b - lam * op_L(r, s))
        p_new, q_new = project_dual(r + g1 / (8.0 * lam), s + g2 / (8.0 * lam), w)
        p_new[-1, :] = 0.0
        q_new[:, -1] = 0.0
        t_new = (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0
        c = (t - 1.0) / t_new
        r = p_new + c * (p_new - p)
        s = q_new + c * (q_new - q)
        p, q, t = p_new, q_new, t_new
    return b - lam * op_L(p, q)
