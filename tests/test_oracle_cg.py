"""Pins of the oracle's conjugate-gradient x-update (no GPU).

Q = Phi^H Phi + 2I (§4.4) is assembled column by column on a tiny problem and
the CG result is compared with a dense solve.
"""
import numpy as np
import pytest

from oracle import cg, measurement as me
from paper_1307_4370_gb300 import inputs


def test_cg_random_hpd_matrix():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((30, 30)) + 1j * rng.standard_normal((30, 30))
    Q = A.conj().T @ A + 2 * np.eye(30)
    b = rng.standard_normal(30) + 1j * rng.standard_normal(30)
    x, res = cg.cg(lambda v: Q @ v, b, np.zeros(30, complex), 60)
    assert np.allclose(x, np.linalg.solve(Q, b), rtol=0, atol=1e-10 * np.abs(x).max())
    assert res < 1e-8


def test_cg_on_gram_operator_against_dense_solve():
    n, J, M = 8, 4, 96
    rng = np.random.default_rng(1)
    uv = inputs.uniform_uv(M, rng)

    def apply_q(v):
        return me.phi_adj(me.phi(v, uv, J), uv, n, J) + 2.0 * v

    cols = []
    for k in range(n * n):
        e = np.zeros(n * n, complex)
        e[k] = 1
        cols.append(apply_q(e.reshape(n, n)).ravel())
    Q = np.array(cols).T
    assert np.allclose(Q, Q.conj().T, atol=1e-13)            # Hermitian
    assert np.min(np.linalg.eigvalsh(Q)) >= 2.0 - 1e-12        # >= 2I
    b = inputs.random_image(n, rng)
    x0 = inputs.random_image(n, rng)
    x, _ = cg.cg(apply_q, b, x0, 2 * n * n)
    want = np.linalg.solve(Q, b.ravel()).reshape(n, n)
    assert np.allclose(x, want, rtol=0, atol=1e-10 * np.abs(want).max())
    # residual after k steps decreases in the Q-norm of the error
    errs = []
    for k in (1, 3, 6, 12):
        xk, _ = cg.cg(apply_q, b, x0, k)
        e = (xk - want).ravel()
        errs.append(np.vdot(e, Q @ e).real)
    assert all(e1 > e2 for e1, e2 in zip(errs, errs[1:]))
