"""Kaiser-Bessel interpolation kernel of the gridding operator G (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

§5 eq. opmodel builds Phi = G F D Z B with G a compactly supported
convolutional interpolation kernel in the frequency plane and D the diagonal
of 1/g_hat, g_hat being the inverse Fourier transform of the continuous
kernel.  The paper uses a Gaussian kernel; the reading taken here is a Kaiser-Bessel
kernel of support J cells, whose transform has a closed form.

    g(t)     = I0(beta * sqrt(1 - (2t/J)^2)) / I0(beta),   |t| <= J/2,  else 0
    g_hat(f) = int g(t) exp(-2 pi i f t) dt
             = J sinh(sqrt(beta^2 - (pi J f)^2)) / (I0(beta) sqrt(beta^2 - (pi J f)^2))

with beta = pi sqrt((J/alpha)^2 (alpha - 1/2)^2 - 0.8) for oversampling
alpha = 2 (the shape rule of Beatty, Nishimura & Pauly 2005; the paper
gives none).  f is in cycles per grid cell; pixel l of an n-pixel axis on
the 2n-point grid sits at f = l / (2n), |f| <= 1/4.

The paper's own kernel, a compactly supported Gaussian (§5), is here too:

    g(t)     = exp(-b t^2),   |t| <= J/2,  else 0
    g_hat(f) = sqrt(pi / b) exp(-pi^2 f^2 / b)   (transform of the untruncated
                                                  Gaussian; the truncation is
                                                  part of the interpolation error)

with b = pi (alpha - 1/2) / (alpha J/2): the Gaussian width of Greengard &
Lee (2004, "Accelerating the nonuniform FFT") for oversampling alpha and
spreading half-width J/2, written in grid cells.  The paper gives no width.

Pinned by ``tests/test_oracle_kernel.py``: the closed forms against numerical
quadrature, and the interpolation against a direct DFT.
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


def deapodisation(n: int, J: int, name: str = "kb") -> np.ndarray:
    """g_hat(l / (2n)) for the pixel offsets l = -n/2 .. n/2-1 of one axis.

    D = diag(1 / (g_hat(l1/2n) g_hat(l2/2n))) is separable; this returns the
    per-axis factor g_hat (the caller divides by the outer product).
    """
    l = np.arange(n) - n // 2
    f = l / (OVERSAMPLE * n)
    return kb_transform(f, J) if name == "kb" else gauss_transform(f, J)


# ---------------------------------------------------------------------------
# Gaussian kernel (the paper's choice, §5)
# ---------------------------------------------------------------------------
KERNELS = ("kb", "gauss")


def gauss_b(J: int, alpha: float = OVERSAMPLE) -> float:
    """Gaussian rate b of g(t) = exp(-b t^2) for support J and oversampling alpha."""
    return float(np.pi * (alpha - 0.5) / (alpha * J / 2.0))


def gauss_kernel(t: np.ndarray, J: int) -> np.ndarray:
    """g(t) = exp(-b t^2) at offsets t (cells), zero outside |t| <= J/2."""
    t = np.asarray(t, dtype=np.float64)
    return np.where(np.abs(t) <= J / 2.0, np.exp(-gauss_b(J) * t * t), 0.0)


def gauss_transform(f: np.ndarray, J: int) -> np.ndarray:
    """g_hat(f) of the untruncated Gaussian (cycles per cell)."""
    b = gauss_b(J)
    f = np.asarray(f, dtype=np.float64)
    return np.sqrt(np.pi / b) * np.exp(-np.pi ** 2 * f * f / b)


def kernel(t: np.ndarray, J: int, name: str = "kb") -> np.ndarray:
    """The interpolation kernel g of G by name ("kb" or "gauss")."""
    return kb_kernel(t, J) if name == "kb" else gauss_kernel(t, J)


def transform(f: np.ndarray, J: int, name: str = "kb") -> np.ndarray:
    """g_hat of the named kernel."""
    return kb_transform(f, J) if name == "kb" else gauss_transform(f, J)
