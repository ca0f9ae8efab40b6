"""Visibility simulation and the l2 bound of §6 (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

§6: visibilities are corrupted by i.i.d. complex Gaussian noise at an input
SNR, ISNR = 20 log10(||y0|| / ||n||) = 30 dB, and the bound of eq. delta is
eps^2 = (2M + 4 sqrt(M)) sigma_n^2 / 2, sigma_n^2 / 2 being the variance of
the real and of the imaginary part.  The reading taken here sets
sigma_n = ||y0|| / sqrt(M) * 10^(-ISNR/20) (so the expected ||n|| matches the
ISNR) and scales unit-variance draws by it.  SNR of a reconstruction is
20 log10(||x|| / ||x - x_hat||) (§6).
"""
from __future__ import annotations

import numpy as np

from . import measurement, sara, sdmm


def noise_sigma(y0: np.ndarray, isnr_db: float) -> float:
    """sigma_n for the requested input SNR."""
    return float(np.linalg.norm(y0) / np.sqrt(y0.size) * 10.0 ** (-isnr_db / 20.0))


def l2_bound(M: int, sigma_n: float) -> float:
    """eps = sqrt((2M + 4 sqrt(M)) sigma_n^2 / 2)."""
    return float(np.sqrt((2.0 * M + 4.0 * np.sqrt(M)) * sigma_n ** 2 / 2.0))


def snr_db(x: np.ndarray, x_hat: np.ndarray) -> float:
    """Reconstruction SNR of §6."""
    return float(20.0 * np.log10(np.linalg.norm(x) / np.linalg.norm(x - x_hat)))


def visibilities(x_true: np.ndarray, uv: np.ndarray, J: int, noise_unit: np.ndarray,
                 isnr_db: float, kernel: str = "kb", beam=None) -> tuple[np.ndarray, float]:
    """y = Phi x + n and eps, with n = sigma_n * noise_unit."""
    y0 = measurement.phi(x_true.astype(np.complex128), uv, J, kernel, beam)
    sig = noise_sigma(y0, isnr_db)
    return y0 + sig * noise_unit, l2_bound(y0.size, sig)


def operators(uv: np.ndarray, n: int, J: int, levels: int = 4,
              bases=sara.ALL_BASES, kernel: str = "kb", beam=None) -> sdmm.Operators:
    """The operators of eq. cvx2 for one problem (interpolation kernel and
    primary beam of Phi = G F D Z B selectable)."""
    return sdmm.Operators(
        phi=lambda x: measurement.phi(x, uv, J, kernel, beam),
        phi_adj=lambda y: measurement.phi_adj(y, uv, n, J, kernel, beam),
        psi_adj=lambda x: sara.sara_analysis(x, levels, bases),
        psi=lambda a: sara.sara_synthesis(a, levels, bases),
    )
