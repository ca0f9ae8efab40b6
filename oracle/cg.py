"""Conjugate gradient for the SDMM x-update (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Algorithm 1 step 5 solves Q x = sum_i x_i with Q = sum_i L_i^H L_i (§4.3
eq. qp1, eq. upd1).  With L1 = Psi^H (a Parseval frame), L2 = Phi, L3 = I,
Q = Phi^H Phi + 2I (§4.4), Hermitian positive definite; §4.4 solves it with
the conjugate gradient method (Saad 2003).  The paper does not fix the start
or the step count: the reading taken here warm-starts from the previous x-hat and takes a
fixed number k of steps.  Inner products are Hermitian, <a, b> = a^H b.

Standard CG (Saad 2003, Algorithm 6.18) in complex128:

    r = b - Q x;  p = r;  rho = <r, r>
    repeat k times:
        q = Q p;  alpha = rho / <p, q>;  x += alpha p;  r -= alpha q
        rho' = <r, r>;  p = r + (rho'/rho) p;  rho = rho'

Pinned by ``tests/test_oracle_cg.py`` against a dense solve of Q assembled
column by column.
"""
from __future__ import annotations

from typing import Callable

import numpy as np


def vdot(a: np.ndarray, b: np.ndarray) -> complex:
    """a^H b over all entries."""
    return complex(np.vdot(a.ravel(), b.ravel()))


def cg(apply_q: Callable[[np.ndarray], np.ndarray], b: np.ndarray, x0: np.ndarray,
       iters: int) -> tuple[np.ndarray, float]:
    """``iters`` CG steps on Q x = b from x0; returns (x, ||b - Q x|| recurrence)."""
    x = np.array(x0, dtype=np.complex128)
    r = b - apply_q(x)
    p = r.copy()
    rho = vdot(r, r).real
    for _ in range(iters):
        if rho == 0.0:
            break
        q = apply_q(p)
        alpha = rho / vdot(p, q).real
        x = x + alpha * p
        r = r - alpha * q
        rho_new = vdot(r, r).real
        p = r + (rho_new / rho) * p
        rho = rho_new
    return x, float(np.sqrt(rho))
