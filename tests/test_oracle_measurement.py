"""Pins of the oracle's measurement operator Phi = G F D Z (no GPU).

Phi approximates the direct non-uniform DFT (§3.1 eqs. ri1/ri4, §5 eq.
opmodel); the tolerance is the interpolation error of the Kaiser-Bessel
kernel, which the tests measure and bound (J = 4: 1e-3, J = 6: 2e-5).
"""
import numpy as np
import pytest

from oracle import measurement as me
from paper_1307_4370_gb300 import inputs

NUFFT_BOUND = {4: 1e-3, 6: 2e-5}


def nudft_loop(x, uv):
    """The definition, one term at a time (tiny inputs)."""
    n = x.shape[0]
    y = np.zeros(uv.shape[0], dtype=np.complex128)
    for m in range(uv.shape[0]):
        s = 0j
        for r in range(n):
            for c in range(n):
                s += x[r, c] * np.exp(-1j * (uv[m, 0] * (r - n // 2) + uv[m, 1] * (c - n // 2)))
        y[m] = s / (2 * n)
    return y


def test_nudft_matches_definition():
    rng = np.random.default_rng(1)
    x = inputs.random_image(8, rng)
    uv = inputs.uniform_uv(7, rng)
    assert np.allclose(me.nudft(x, uv), nudft_loop(x, uv), rtol=0, atol=1e-13)


def test_nudft_single_pixel():
    # A unit pixel at offset l gives exp(-i u.l) / (2n).
    n = 16
    x = np.zeros((n, n), dtype=np.complex128)
    x[3, 11] = 1.0
    uv = inputs.uniform_uv(50, np.random.default_rng(2))
    l = np.array([3 - n // 2, 11 - n // 2])
    want = np.exp(-1j * uv @ l) / (2 * n)
    assert np.allclose(me.nudft(x, uv), want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("n,J,M", [(8, 4, 300), (16, 4, 500), (16, 6, 500), (64, 4, 2048), (64, 6, 2048)])
def test_phi_against_nudft(n, J, M):
    rng = np.random.default_rng(n * 100 + J)
    x = inputs.random_image(n, rng)
    uv = inputs.uniform_uv(M, rng)
    y = me.phi(x, uv, J)
    yd = me.nudft(x, uv)
    err = np.linalg.norm(y - yd) / np.linalg.norm(yd)
    assert err <= NUFFT_BOUND[J]
    # the approximation is not exact either: a scale or sign slip would give O(1)
    assert err > 1e-9
    v = inputs.random_vis(M, rng)
    xa = me.phi_adj(v, uv, n, J)
    xd = me.nudft_adj(v, uv, n)
    assert np.linalg.norm(xa - xd) / np.linalg.norm(xd) <= NUFFT_BOUND[J]


@pytest.mark.parametrize("n,J", [(16, 4), (32, 6), (64, 6)])
def test_adjoint_identity(n, J):
    rng = np.random.default_rng(7 + n)
    M = 3 * n * n // 2
    uv = inputs.uniform_uv(M, rng)
    x = inputs.random_image(n, rng)
    v = inputs.random_vis(M, rng)
    lhs = np.vdot(v, me.phi(x, uv, J))
    rhs = np.vdot(me.phi_adj(v, uv, n, J), x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_centre_pixel_is_flat():
    # A unit pixel at the image centre (l = 0) has the constant transform 1/(2n).
    n, J = 32, 6
    x = np.zeros((n, n), dtype=np.complex128)
    x[n // 2, n // 2] = 1.0
    uv = inputs.uniform_uv(400, np.random.default_rng(3))
    y = me.phi(x, uv, J)
    assert np.max(np.abs(y - 1.0 / (2 * n))) <= NUFFT_BOUND[J] / (2 * n) * 5


def test_wraparound_frequencies():
    # Frequencies at the edge of [-pi, pi) use footprints that wrap the grid.
    n, J = 16, 6
    rng = np.random.default_rng(4)
    x = inputs.random_image(n, rng)
    e = np.float32(np.pi) - np.float32(1e-3)
    uv = np.array([[-np.pi, -np.pi], [e, e], [-np.pi, e], [e, 0.0], [0.0, -np.pi]], dtype=np.float64)
    y = me.phi(x, uv, J)
    yd = me.nudft(x, uv)
    assert np.linalg.norm(y - yd) / np.linalg.norm(yd) <= NUFFT_BOUND[J]


# ---------------------------------------------------------------------------
# Gaussian kernel and primary beam (Phi = G F D Z B, §5 eq. opmodel)
# ---------------------------------------------------------------------------
# Interpolation error of the Gaussian kernel against the direct transform,
# measured with this oracle on uniform frequencies (n = 16, 64): 9.5e-3 (J=4),
# 9.7e-4 (J=6), 9.8e-5 (J=8); roughly a decade per two taps, as expected of
# Gaussian gridding at oversampling 2.
GAUSS_BOUND = {4: 2e-2, 6: 2e-3, 8: 2e-4}


@pytest.mark.parametrize("n", [16, 64])
@pytest.mark.parametrize("J", [4, 6, 8])
def test_gauss_phi_against_nudft(n, J):
    rng = np.random.default_rng(10 * n + J)
    uv = inputs.uniform_uv(400, rng)
    x = inputs.random_image(n, rng)
    beam = 0.5 + rng.uniform(0, 1, (n, n))
    want = me.nudft(x, uv, beam=beam)
    got = me.phi(x, uv, J, kernel="gauss", beam=beam)
    assert np.linalg.norm(got - want) <= GAUSS_BOUND[J] * np.linalg.norm(want)
    if J < 8:  # more taps interpolate better
        got2 = me.phi(x, uv, J + 2, kernel="gauss", beam=beam)
        assert np.linalg.norm(got2 - want) < 0.3 * np.linalg.norm(got - want)


@pytest.mark.parametrize("kernel", ["kb", "gauss"])
def test_adjoint_identity_with_beam(kernel):
    rng = np.random.default_rng(7)
    n, J = 32, 6
    uv = inputs.uniform_uv(300, rng)
    x = inputs.random_image(n, rng)
    y = inputs.random_vis(300, rng)
    beam = rng.uniform(0.1, 1.0, (n, n))
    lhs = np.vdot(y, me.phi(x, uv, J, kernel, beam))
    rhs = np.vdot(me.phi_adj(y, uv, n, J, kernel, beam), x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_unit_beam_is_no_beam():
    rng = np.random.default_rng(8)
    n, J = 16, 4
    uv = inputs.uniform_uv(100, rng)
    x = inputs.random_image(n, rng)
    y = inputs.random_vis(100, rng)
    one = np.ones((n, n))
    assert np.array_equal(me.phi(x, uv, J, "gauss", one), me.phi(x, uv, J, "gauss"))
    assert np.array_equal(me.phi_adj(y, uv, n, J, "gauss", one), me.phi_adj(y, uv, n, J, "gauss"))
    # a beam that blanks half the image removes that half from every visibility
    half = np.zeros((n, n))
    half[:, : n // 2] = 1.0
    x2 = x.copy()
    x2[:, n // 2:] = 0.0
    assert np.allclose(me.phi(x, uv, J, "kb", half), me.phi(x2, uv, J, "kb"), rtol=0, atol=1e-15)
