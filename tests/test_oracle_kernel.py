"""Pins of the oracle's Kaiser-Bessel kernel and unitary FFT (no GPU).

The closed-form transform g_hat that D divides by (§5 eq. opmodel) is checked
against numerical quadrature of g itself; the FFT (a library primitive inside
the oracle) against the DFT written as a double loop.
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import kaiser_bessel as kb
from oracle import measurement as me


@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
@pytest.mark.parametrize("J", [2, 4, 6, 8])
@pytest.mark.parametrize("f", [0.0, 0.03125, 0.1, 0.2, 0.25])
def test_transform_matches_quadrature(J, f):
    # g is even, so its transform is the cosine integral over [-J/2, J/2].
    val, err = integrate.quad(lambda t: kb.kb_kernel(t, J) * np.cos(2 * np.pi * f * t),
                              -J / 2, J / 2, epsabs=1e-14, epsrel=1e-14, limit=200)
    assert abs(kb.kb_transform(f, J) - val) <= 1e-12 * abs(val)


@pytest.mark.parametrize("J", [4, 6])
def test_kernel_shape(J):
    # Normalised to 1 at the centre, 1/I0(beta) at the support edge, zero outside.
    beta = kb.kb_beta(J)
    assert kb.kb_kernel(0.0, J) == pytest.approx(1.0, abs=1e-15)
    assert kb.kb_kernel(J / 2, J) == pytest.approx(1.0 / np.i0(beta), rel=1e-14)
    assert kb.kb_kernel(J / 2 + 1e-9, J) == 0.0
    t = np.linspace(-J / 2, J / 2, 101)
    assert np.allclose(kb.kb_kernel(t, J), kb.kb_kernel(-t, J), rtol=0, atol=1e-15)


def test_beta_values():
    # Beatty et al. (2005) shape rule at oversampling 2: beta(4) ~ 8.9962, beta(6) ~ 13.8551.
    assert kb.kb_beta(4) == pytest.approx(8.99615, abs=1e-4)
    assert kb.kb_beta(6) == pytest.approx(13.85510, abs=1e-4)


def direct_dft2(g):
    L0, L1 = g.shape
    X = np.zeros_like(g, dtype=np.complex128)
    for k0 in range(L0):
        for k1 in range(L1):
            s = 0j
            for j0 in range(L0):
                for j1 in range(L1):
                    s += g[j0, j1] * np.exp(-2j * np.pi * (k0 * j0 / L0 + k1 * j1 / L1))
            X[k0, k1] = s
    return X / np.sqrt(L0 * L1)


@pytest.mark.parametrize("L", [8, 12, 16, 24])
def test_fft_against_direct_dft(L):
    rng = np.random.default_rng(L)
    g = rng.standard_normal((L, L)) + 1j * rng.standard_normal((L, L))
    X = me.fft2_unitary(g)
    assert np.max(np.abs(X - direct_dft2(g))) <= 1e-13 * np.max(np.abs(X)) * L
    # unitary: Parseval, and the inverse undoes it
    assert np.linalg.norm(X) == pytest.approx(np.linalg.norm(g), rel=1e-13)
    assert np.allclose(me.ifft2_unitary(X), g, rtol=0, atol=1e-13 * np.abs(g).max())


def test_deapodisation_profile():
    # g_hat(l / 2n) over l = -n/2..n/2-1: largest at l = 0, even about 0.
    n = 64
    gh = kb.deapodisation(n, 6)
    assert np.argmax(gh) == n // 2
    assert np.allclose(gh[1:], gh[1:][::-1], rtol=1e-14)


# ---------------------------------------------------------------------------
# The paper's Gaussian kernel (§5)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("J", [4, 6, 8])
@pytest.mark.parametrize("f", [0.0, 0.05, 0.125, 0.25])
def test_gauss_transform_matches_quadrature(J, f):
    # g_hat is the transform of the untruncated Gaussian: integrate over R,
    # as twice the integral over [0, t_max] with exp(-b t_max^2) = e^-80 (the
    # rest of the tail is below 1e-35 of the value)
    b = kb.gauss_b(J)
    t_max = np.sqrt(80.0 / b)
    val, _ = integrate.quad(lambda t: 2.0 * np.exp(-b * t * t) * np.cos(2 * np.pi * f * t), 0.0, t_max,
                            epsabs=0.0, epsrel=1e-13, limit=400)
    assert abs(kb.gauss_transform(f, J) - val) <= 1e-12 * abs(val)


@pytest.mark.parametrize("J", [4, 6, 8])
def test_gauss_kernel_shape(J):
    # exp(-b t^2) with b = pi (alpha - 1/2) / (alpha J / 2): 1 at the centre,
    # exp(-3 pi J / 8) at the support edge (alpha = 2), zero outside, even.
    assert kb.gauss_b(J) == pytest.approx(0.75 * np.pi / (J / 2), rel=1e-15)
    assert kb.gauss_kernel(0.0, J) == 1.0
    assert kb.gauss_kernel(J / 2, J) == pytest.approx(np.exp(-3 * np.pi * J / 8), rel=1e-14)
    assert kb.gauss_kernel(J / 2 + 1e-9, J) == 0.0
    t = np.linspace(-J / 2, J / 2, 101)
    assert np.array_equal(kb.gauss_kernel(t, J), kb.gauss_kernel(-t, J))
    assert np.array_equal(kb.kernel(t, J, "gauss"), kb.gauss_kernel(t, J))
    assert np.array_equal(kb.kernel(t, J, "kb"), kb.kb_kernel(t, J))


def test_gauss_deapodisation_profile():
    n = 64
    gh = kb.deapodisation(n, 6, "gauss")
    l = np.arange(n) - n // 2
    assert np.allclose(gh, kb.gauss_transform(l / (2 * n), 6), rtol=1e-15, atol=0)
    assert np.argmax(gh) == n // 2
