"""Daubechies-p orthonormal wavelet filters by spectral factorisation (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

§3.3 names the first eight orthonormal Daubechies bases (db1..db8) as the
wavelet part of the SARA dictionary; the paper gives no coefficients.  They
follow from the published construction (Daubechies 1988; Ten Lectures on
Wavelets, 1992, §6.1):

  |m0(w)|^2 = cos^{2p}(w/2) P(sin^2(w/2)),  P(y) = sum_{k<p} C(p-1+k, k) y^k,

m0 = ((1 + e^{-iw})/2)^p L(e^{-iw}) with |L|^2 = P.  Each root y_k of P maps
to a reciprocal pair of zeros of L through y = (2 - z - 1/z)/4; taking the
zero inside the unit circle of every pair gives the minimum-phase filter.
The low-pass filter h (length 2p) is the coefficient list of
(z + 1)^p prod_k (z - z_k) in descending powers of z, scaled so that
sum h = sqrt(2).  The high-pass filter is g[m] = (-1)^m h[2p - 1 - m].

Convention: with this ordering the analysis step is the correlation
a[i] = sum_m h[m] s[2i + m]; db2 is ((1+r3), (3+r3), (3-r3), (1-r3)) / (4 sqrt 2).

Pinned by ``tests/test_oracle_daubechies.py``: orthonormality, the sum rule,
p vanishing moments, and the closed forms of db1, db2 and db3.
"""
from __future__ import annotations

from math import comb

import numpy as np


def daubechies_lowpass(p: int) -> np.ndarray:
    """Low-pass filter h of the Daubechies-p wavelet (length 2p, float64)."""
    if p < 1:
        raise ValueError("p >= 1")
    # P(y) coefficients, ascending powers, then numpy wants descending.
    P = np.array([comb(p - 1 + k, k) for k in range(p)], dtype=np.float64)
    zeros = []
    if p > 1:
        for yk in np.roots(P[::-1]):
            # z + 1/z = 2 - 4 y  ->  z^2 - (2 - 4y) z + 1 = 0
            c = 2.0 - 4.0 * yk
            disc = np.sqrt(c * c - 4.0 + 0j)
            z1, z2 = (c + disc) / 2.0, (c - disc) / 2.0
            zeros.append(z1 if abs(z1) < 1.0 else z2)
    q = np.poly(np.concatenate([-np.ones(p), np.array(zeros, dtype=np.complex128)]))
    h = np.real(q)
    return h * (np.sqrt(2.0) / h.sum())


def daubechies_highpass(h: np.ndarray) -> np.ndarray:
    """g[m] = (-1)^m h[len(h) - 1 - m]."""
    m = np.arange(h.size)
    return ((-1.0) ** m) * h[::-1]
