"""Pins of the oracle's SARA dictionary (no GPU).

§3.3 (concatenation of Dirac and db1..db8) and §4.4 (Parseval frame, so that
Psi Psi^H = I): each W_p is checked as an explicit orthogonal matrix, the
synthesis as its transpose, the frame as Parseval, and one Haar level by hand.
"""
import numpy as np
import pytest

from oracle import sara
from paper_1307_4370_gb300 import inputs


def as_matrix(fn, n):
    cols = []
    for k in range(n * n):
        e = np.zeros(n * n, dtype=np.complex128)
        e[k] = 1.0
        cols.append(fn(e.reshape(n, n)).ravel())
    return np.array(cols).T


@pytest.mark.parametrize("p", range(1, 9))
def test_dwt_is_orthogonal_matrix(p):
    # n = 16 with 4 levels: the level-2..4 lengths 8, 4, 2 are shorter than most filters.
    n, levels = 16, 4
    W = as_matrix(lambda x: sara.dwt2(x, p, levels), n)
    Wt = as_matrix(lambda c: sara.idwt2(c, p, levels), n)
    assert np.max(np.abs(W.imag)) == 0.0
    assert np.allclose(W.T @ W, np.eye(n * n), atol=1e-12)
    assert np.allclose(Wt, W.T, atol=1e-13)


def test_haar_one_level_by_hand():
    x = np.array([[1.0, 2.0], [3.0, 5.0]])
    a, b, c, d = x.ravel()
    c_ = sara.dwt2(x, 1, 1).real
    want = np.array([[a + b + c + d, a - b + c - d], [a + b - c - d, a - b - c + d]]) / 2
    assert np.allclose(c_, want, atol=1e-15)


def test_haar_levels_mallat_layout():
    # Three Haar levels of a constant 8x8 image: all energy (norm 8) in the top-left coefficient.
    x = np.ones((8, 8))
    c = sara.dwt2(x, 1, 3).real
    assert c[0, 0] == pytest.approx(8.0, abs=1e-14)
    c[0, 0] = 0.0
    assert np.max(np.abs(c)) < 1e-14


def test_shift_covariance_one_level():
    # One periodic level commutes with a circular shift by 2 pixels (1 coefficient).
    rng = np.random.default_rng(0)
    x = inputs.random_image(16, rng)
    for p in (2, 5, 8):
        c = sara.dwt2(x, p, 1)
        cs = sara.dwt2(np.roll(x, -2, axis=1), p, 1)
        assert np.allclose(cs[:, :8], np.roll(c[:, :8], -1, axis=1), atol=1e-13)
        assert np.allclose(cs[:, 8:], np.roll(c[:, 8:], -1, axis=1), atol=1e-13)


@pytest.mark.parametrize("n", [16, 64])
def test_parseval_frame(n):
    rng = np.random.default_rng(n)
    x = inputs.random_image(n, rng)
    al = sara.sara_analysis(x, 4)
    assert al.shape == (9, n, n)
    assert np.allclose(al[0], x / 3.0, atol=1e-15)
    assert np.linalg.norm(al) == pytest.approx(np.linalg.norm(x), rel=1e-13)
    assert np.allclose(sara.sara_synthesis(al, 4), x, atol=1e-12)
    # synthesis is the adjoint of analysis
    b = rng.standard_normal(al.shape) + 1j * rng.standard_normal(al.shape)
    lhs = np.vdot(b, al)
    rhs = np.vdot(sara.sara_synthesis(b, 4), x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_single_basis_subsets():
    rng = np.random.default_rng(5)
    x = inputs.random_image(16, rng)
    al = sara.sara_analysis(x, 4, bases=(8,))
    assert np.allclose(al[0], sara.dwt2(x, 8, 4), atol=1e-15)
    al = sara.sara_analysis(x, 4, bases=(0,))
    assert np.allclose(al[0], x, atol=0)
