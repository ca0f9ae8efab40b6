"""Proximity operators of the three SDMM functions (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

§4.4 gives, for f1(r) = ||W r||_1 = sum_j w_j |r_j| (eq. prox1), the
entrywise complex soft threshold prox_{lam |.|}(a) = a/|a| (|a| - lam)^+,
applied with lam = gamma w_j; at a = 0 it returns 0.

For f2 = indicator of B = {r : ||y - r||_2 <= eps} the paper prints
min(1, eps/||r||) r (eq. prox2), which projects onto a ball centred at 0,
not at y.  The projection onto B as defined in §4.3 is

    P_B(r) = y + min(1, eps / ||r - y||) (r - y),

and that is what is computed here (identity when r is inside B).

For f3 = indicator of the positive orthant (eq. prox3): complex vectors are
treated as real vectors of twice the length (§4.1), so the orthant of
R_+^N inside C^N is {x : Im x = 0, Re x >= 0} and the projection is
max(Re a, 0) + 0i.

Pinned by ``tests/test_oracle_prox.py`` against brute-force minimisation of
the prox objective and the projection optimality conditions.
"""
from __future__ import annotations

import numpy as np


def soft_threshold(a: np.ndarray, lam) -> np.ndarray:
    """prox of lam |.| entrywise: a/|a| (|a| - lam)^+ (0 where a = 0)."""
    a = np.asarray(a, dtype=np.complex128)
    mag = np.abs(a)
    shrink = np.maximum(mag - lam, 0.0)
    scale = np.divide(shrink, mag, out=np.zeros_like(mag), where=mag > 0)
    return a * scale


def project_l2_ball(r: np.ndarray, y: np.ndarray, eps: float) -> np.ndarray:
    """P_B(r) for B = {r : ||r - y||_2 <= eps}."""
    d = np.asarray(r, dtype=np.complex128) - y
    nd = np.sqrt(np.sum(np.abs(d) ** 2))
    if nd <= eps:
        return np.array(r, dtype=np.complex128)
    return y + (eps / nd) * d


def project_l2_balls(r: np.ndarray, y: np.ndarray, eps, offsets) -> np.ndarray:
    """Block by block P_{B_i}, B_i = {r_i : ||r_i - y_i||_2 <= eps_i}: the data
    constraints of the distributed form (§4.5 eq. dbp1), blocks
    r[offsets[i]:offsets[i+1]] as in eq. blocks."""
    out = np.empty(len(r), dtype=np.complex128)
    for i in range(len(eps)):
        sl = slice(offsets[i], offsets[i + 1])
        out[sl] = project_l2_ball(r[sl], y[sl], eps[i])
    return out


def project_positive(a: np.ndarray) -> np.ndarray:
    """Projection onto {x real, x >= 0}: max(Re a, 0)."""
    return np.maximum(np.real(a), 0.0).astype(np.complex128)
