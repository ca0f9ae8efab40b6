"""SARA dictionary Psi = [Dirac, db1, ..., db8] and its adjoint (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

§3.3 defines the SARA dictionary as the concatenation of q bases
Psi = [Psi_1, ..., Psi_q], here the Dirac basis and the orthonormal
Daubechies bases db1..db8 (q = 9, D = 9N).  §4.4 needs Psi Psi^H = I (a
Parseval frame) so that Q = Phi^H Phi + 2I; the plain concatenation of nine
orthonormal bases has Psi Psi^H = 9 I, so it is scaled here by
1/sqrt(q).  Hence

    Psi^H x   = (1/sqrt q) [x; W_1 x; ...; W_8 x]            (analysis, C^N -> C^D)
    Psi alpha = (1/sqrt q) (alpha_0 + sum_b W_b^T alpha_b)   (synthesis)

W_p is the periodic, separable 2-D orthonormal DWT with the Daubechies-p
filters over ``levels`` levels (4 in every workload).  One level on an L x L
block: the 1-D step a[i] = sum_m h[m] s[(2i + m) mod L],
d[i] = sum_m g[m] s[(2i + m) mod L], with output [a | d], is applied along
each row, then along each column; the next level works on the top-left
(low-low) quarter (Mallat layout).  Indices wrap modulo the current length,
also when the filter is longer than the signal (db8 on 8 samples).

Pinned by ``tests/test_oracle_sara.py``: orthogonality of every W_p as a
matrix, Parseval, the Dirac plane, and the one-level Haar case by hand.
"""
from __future__ import annotations

import numpy as np

from .daubechies import daubechies_highpass, daubechies_lowpass

ALL_BASES = tuple(range(9))  # 0 = Dirac, p = db_p


def _analysis_axis(s: np.ndarray, h: np.ndarray, g: np.ndarray, axis: int) -> np.ndarray:
    """One periodic analysis step along ``axis``: [a | d]."""
    L = s.shape[axis]
    i2 = 2 * np.arange(L // 2)
    a = np.zeros_like(np.take(s, i2, axis=axis))
    d = np.zeros_like(a)
    for m in range(h.size):
        sm = np.take(s, (i2 + m) % L, axis=axis)
        a = a + h[m] * sm
        d = d + g[m] * sm
    return np.concatenate([a, d], axis=axis)


def _synthesis_axis(c: np.ndarray, h: np.ndarray, g: np.ndarray, axis: int) -> np.ndarray:
    """Transpose of ``_analysis_axis``: s[(2i + m) mod L] += h[m] a[i] + g[m] d[i]."""
    L = c.shape[axis]
    a = np.take(c, np.arange(L // 2), axis=axis)
    d = np.take(c, np.arange(L // 2, L), axis=axis)
    s = np.moveaxis(np.zeros_like(c), axis, 0)
    a0 = np.moveaxis(a, axis, 0)
    d0 = np.moveaxis(d, axis, 0)
    i2 = 2 * np.arange(L // 2)
    for m in range(h.size):
        np.add.at(s, (i2 + m) % L, h[m] * a0 + g[m] * d0)
    return np.moveaxis(s, 0, axis)


def dwt2(x: np.ndarray, p: int, levels: int) -> np.ndarray:
    """W_p x: periodic 2-D orthonormal DWT, Mallat layout."""
    h = daubechies_lowpass(p)
    g = daubechies_highpass(h)
    out = np.array(x, dtype=np.complex128)
    L = out.shape[0]
    for _ in range(levels):
        blk = _analysis_axis(out[:L, :L], h, g, axis=1)  # rows
        blk = _analysis_axis(blk, h, g, axis=0)          # then columns
        out[:L, :L] = blk
        L //= 2
    return out


def idwt2(c: np.ndarray, p: int, levels: int) -> np.ndarray:
    """W_p^T c (= W_p^{-1} c since W_p is orthogonal)."""
    h = daubechies_lowpass(p)
    g = daubechies_highpass(h)
    out = np.array(c, dtype=np.complex128)
    n = out.shape[0]
    for lev in reversed(range(levels)):
        L = n >> lev
        blk = _synthesis_axis(out[:L, :L], h, g, axis=0)  # transpose order:
        blk = _synthesis_axis(blk, h, g, axis=1)          # columns, then rows
        out[:L, :L] = blk
    return out


def sara_analysis(x: np.ndarray, levels: int = 4, bases=ALL_BASES) -> np.ndarray:
    """Psi^H x, shape (q, n, n): plane b is basis bases[b] (0 = Dirac)."""
    q = len(bases)
    planes = [np.array(x, dtype=np.complex128) if b == 0 else dwt2(x, b, levels) for b in bases]
    return np.stack(planes) / np.sqrt(q)


def sara_synthesis(alpha: np.ndarray, levels: int = 4, bases=ALL_BASES) -> np.ndarray:
    """Psi alpha for alpha of shape (q, n, n)."""
    q = len(bases)
    x = np.zeros(alpha.shape[1:], dtype=np.complex128)
    for k, b in enumerate(bases):
        x += alpha[k] if b == 0 else idwt2(alpha[k], b, levels)
    return x / np.sqrt(q)
