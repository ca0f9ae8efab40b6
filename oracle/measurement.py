"""Measurement operator Phi = G F D Z B and its adjoint (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

§3.1 eq. ri4 models the visibilities as y = Phi x + n; §5 eq. opmodel writes
Phi = G F D Z B with B the primary beam (the identity in every experiment of
§6), Z the zero padding onto an oversampled grid (oversampling 2 per axis,
so N' = 4N), D the diagonal deapodisation 1/g_hat, F the unitary 2-D DFT and
G the convolutional interpolation onto the continuous frequencies.

Conventions (the paper fixes none of them; these are the readings taken here):

* image x is n x n, x[r, c] is the pixel at offset l = (r - n/2, c - n/2);
* a visibility frequency u = (u0, u1) is in radians per pixel, in [-pi, pi)^2,
  with u0 paired with the row offset; the target of Phi is the direct
  transform (1/(2n)) sum_l x_l exp(-i u.l) (the sign of eq. ri1);
* Z places pixel l at grid cell (l mod 2n) per axis;
* F is X[k] = (1/(2n)) sum_j g[j] exp(-2 pi i k.j / (2n)), natural order;
* G: kappa = u 2n / (2 pi); the footprint of a visibility is the J cells
  floor(kappa) - J/2 + 1 .. floor(kappa) + J/2 of each axis (indices mod
  2n) weighted by g(kappa - k) of ``kaiser_bessel`` (Kaiser-Bessel by
  default, or the paper's Gaussian with ``kernel="gauss"``);
* B: an optional real n x n primary beam multiplying the image (default the
  identity, as in all of §6).

``phi_adj`` is the exact transpose-conjugate of each factor in reverse
order: Z^T D F^H G^T.

Pinned by ``tests/test_oracle_measurement.py``: against the direct
non-uniform DFT below within the interpolation error, the adjoint identity,
and special cases.
"""
from __future__ import annotations

import numpy as np

from .kaiser_bessel import OVERSAMPLE, deapodisation
from .kaiser_bessel import kernel as interp_kernel


def _pad_rows(n: int) -> np.ndarray:
    """Grid row (or column) of each image row: (r - n/2) mod 2n."""
    return (np.arange(n) - n // 2) % (OVERSAMPLE * n)


def footprint(uv: np.ndarray, n: int, J: int):
    """First footprint cell k0 (M, 2) and kappa (M, 2) of each visibility."""
    L = OVERSAMPLE * n
    kappa = np.asarray(uv, dtype=np.float64) * (L / (2.0 * np.pi))
    k0 = np.floor(kappa).astype(np.int64) - J // 2 + 1
    return k0, kappa


def zero_pad_deapodise(x: np.ndarray, J: int, kernel: str = "kb") -> np.ndarray:
    """D Z x: the image divided by g_hat, placed on the 2n x 2n grid."""
    n = x.shape[0]
    L = OVERSAMPLE * n
    gh = deapodisation(n, J, kernel)
    g = np.zeros((L, L), dtype=np.complex128)
    rows = _pad_rows(n)
    g[np.ix_(rows, rows)] = x / np.outer(gh, gh)
    return g


def crop_deapodise(g: np.ndarray, n: int, J: int, kernel: str = "kb") -> np.ndarray:
    """Z^T D g: the image pixels of a grid, divided by g_hat."""
    gh = deapodisation(n, J, kernel)
    rows = _pad_rows(n)
    return g[np.ix_(rows, rows)] / np.outer(gh, gh)


def fft2_unitary(g: np.ndarray) -> np.ndarray:
    """F: unitary forward 2-D DFT (numpy's FFT, scaled by 1/sqrt(N'))."""
    return np.fft.fft2(g) / np.sqrt(g.size)


def ifft2_unitary(X: np.ndarray) -> np.ndarray:
    """F^H: unitary inverse 2-D DFT."""
    return np.fft.ifft2(X) * np.sqrt(X.size)


def _axis_weights(k0: np.ndarray, kappa: np.ndarray, J: int, kernel: str = "kb"):
    """Per-axis kernel weights g(kappa - k0 - a), a = 0..J-1, as J arrays of (M, 2)."""
    return [interp_kernel(kappa - (k0 + a), J, kernel) for a in range(J)]


def degrid(X: np.ndarray, uv: np.ndarray, J: int, kernel: str = "kb") -> np.ndarray:
    """G: y_m = sum_{a,b < J} g(kappa_m0 - k0_m0 - a) g(kappa_m1 - k0_m1 - b) X[k0 + (a, b)]."""
    L = X.shape[0]
    k0, kappa = footprint(uv, L // OVERSAMPLE, J)
    w = _axis_weights(k0, kappa, J, kernel)
    y = np.zeros(k0.shape[0], dtype=np.complex128)
    for a in range(J):
        k_r = (k0[:, 0] + a) % L
        for b in range(J):
            k_c = (k0[:, 1] + b) % L
            y += w[a][:, 0] * w[b][:, 1] * X[k_r, k_c]
    return y


def grid(y: np.ndarray, uv: np.ndarray, n: int, J: int, kernel: str = "kb") -> np.ndarray:
    """G^T: X[k] = sum_m g(kappa_m0 - k0) g(kappa_m1 - k1) y_m (G is real)."""
    L = OVERSAMPLE * n
    k0, kappa = footprint(uv, n, J)
    w = _axis_weights(k0, kappa, J, kernel)
    y = np.asarray(y, dtype=np.complex128)
    X = np.zeros(L * L, dtype=np.complex128)
    for a in range(J):
        k_r = (k0[:, 0] + a) % L
        for b in range(J):
            k_c = (k0[:, 1] + b) % L
            v = w[a][:, 0] * w[b][:, 1] * y
            cell = k_r * L + k_c
            X += np.bincount(cell, weights=v.real, minlength=L * L)
            X += 1j * np.bincount(cell, weights=v.imag, minlength=L * L)
    return X.reshape(L, L)


def phi(x: np.ndarray, uv: np.ndarray, J: int, kernel: str = "kb", beam: np.ndarray | None = None) -> np.ndarray:
    """Phi x = G F D Z B x for an n x n image x and M frequencies uv."""
    bx = x if beam is None else np.asarray(beam, dtype=np.float64) * x
    return degrid(fft2_unitary(zero_pad_deapodise(bx, J, kernel)), uv, J, kernel)


def phi_adj(y: np.ndarray, uv: np.ndarray, n: int, J: int, kernel: str = "kb",
            beam: np.ndarray | None = None) -> np.ndarray:
    """Phi^H y = B Z^T D F^H G^T y, an n x n image (B is real and diagonal)."""
    x = crop_deapodise(ifft2_unitary(grid(y, uv, n, J, kernel)), n, J, kernel)
    return x if beam is None else np.asarray(beam, dtype=np.float64) * x


def nudft(x: np.ndarray, uv: np.ndarray, beam: np.ndarray | None = None) -> np.ndarray:
    """Direct non-uniform DFT, (1/(2n)) sum_l x_l exp(-i u.l).

    This is the quantity Phi approximates (eq. ri1 without DDEs, sampled on
    the pixel grid as in eq. ri4), with the 1/(2n) of the unitary DFT on the
    oversampled grid.  O(M N): for small inputs only.
    """
    n = x.shape[0]
    if beam is not None:
        x = np.asarray(beam, dtype=np.float64) * x
    l = np.arange(n) - n // 2
    uv = np.asarray(uv, dtype=np.float64)
    e0 = np.exp(-1j * np.outer(uv[:, 0], l))  # (M, n)
    e1 = np.exp(-1j * np.outer(uv[:, 1], l))
    return np.einsum("mr,rc,mc->m", e0, x, e1) / (OVERSAMPLE * n)


def nudft_adj(y: np.ndarray, uv: np.ndarray, n: int) -> np.ndarray:
    """Adjoint of ``nudft``."""
    l = np.arange(n) - n // 2
    uv = np.asarray(uv, dtype=np.float64)
    e0 = np.exp(1j * np.outer(uv[:, 0], l))
    e1 = np.exp(1j * np.outer(uv[:, 1], l))
    return np.einsum("m,mr,mc->rc", y, e0, e1) / (OVERSAMPLE * n)
