"""Kaiser-Bessel interpolation kernel of the gridding operator G (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

§5 eq. opmodel builds Phi = G F D Z B with G a compactly supported
convolutional interpolation kernel in the frequency plane and D the diagonal
of 1/g_hat, g_hat being the inverse Fourier transform of the continuous
kernel.  The paper uses a Gaussian kernel; this build uses a Kaiser-Bessel
kernel of support J cells, whose transform has a closed form.

    g(t)     = I0(beta * sqrt(1 - (2t/J)^2)) / I0(beta),   |t| <= J/2,  else 0
    g_hat(f) = int g(t) exp(-2 pi i f t) dt
             = J sinh(sqrt(beta^2 - (pi J f)^2)) / (I0(beta) sqrt(beta^2 - (pi J f)^2))

with beta = pi sqrt((J/alpha)^2 (alpha - 1/2)^2 - 0.8) for oversampling
alpha = 2 (the shape rule of Beatty, Nishimura & Pauly 2005; the paper
gives none).  f is in cycles per grid cell; pixel l of an n-pixel axis on
the 2n-point grid sits at f = l / (2n), |f| <= 1/4.

Pinned by ``tests/test_oracle_kernel.py``: the closed form against numerical
quadrature of g, and the interpolation against a direct DFT.
"""
from __future__ import annotations

import numpy as np

OVERSAMPLE = 2


def kb_beta(J: int, alpha: float = OVERSAMPLE) -> float:
    """Kaiser-Bessel shape parameter for support J and oversampling alpha."""
    return float(np.pi * np.sqrt((J / alpha) ** 2 * (alpha - 0.5) ** 2 - 0.8))


def kb_kernel(t: np.ndarray, J: int) -> np.ndarray:
    """g(t): the 1-D kernel sampled at offsets t (cells), zero outside |t| <= J/2."""
    beta = kb_beta(J)
    t = np.asarray(t, dtype=np.float64)
    s = 1.0 - (2.0 * t / J) ** 2
    inside = s >= 0.0
    val = np.i0(beta * np.sqrt(np.where(inside, s, 0.0))) / np.i0(beta)
    return np.where(inside, val, 0.0)


def kb_transform(f: np.ndarray, J: int) -> np.ndarray:
    """g_hat(f), the continuous Fourier transform of g (cycles per cell).

    Valid while (pi J f)^2 < beta^2, which holds for |f| <= 1/4 and J >= 2.
    """
    beta = kb_beta(J)
    f = np.asarray(f, dtype=np.float64)
    a = np.sqrt(beta ** 2 - (np.pi * J * f) ** 2)
    return J * np.sinh(a) / (np.i0(beta) * a)


def deapodisation(n: int, J: int) -> np.ndarray:
    """g_hat(l / (2n)) for the pixel offsets l = -n/2 .. n/2-1 of one axis.

    D = diag(1 / (g_hat(l1/2n) g_hat(l2/2n))) is separable; this returns the
    per-axis factor g_hat (the caller divides by the outer product).
    """
    l = np.arange(n) - n // 2
    return kb_transform(l / (OVERSAMPLE * n), J)
