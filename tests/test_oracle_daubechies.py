"""Pins of the oracle's Daubechies filters (no GPU).

Orthonormality (double-shift orthogonality), the sum rule, p vanishing moments
of the high-pass filter and the minimum-phase choice determine db_p uniquely;
db1, db2 and db3 are also checked against their published closed forms
(Daubechies 1988).
"""
import numpy as np
import pytest

from oracle import daubechies as dbm


def test_db1_haar():
    assert np.allclose(dbm.daubechies_lowpass(1), [2 ** -0.5, 2 ** -0.5], atol=1e-15)


def test_db2_closed_form():
    r3 = np.sqrt(3.0)
    want = np.array([1 + r3, 3 + r3, 3 - r3, 1 - r3]) / (4 * np.sqrt(2.0))
    assert np.allclose(dbm.daubechies_lowpass(2), want, rtol=0, atol=1e-14)


def test_db3_closed_form():
    r10 = np.sqrt(10.0)
    s = np.sqrt(5 + 2 * r10)
    want = np.array([1 + r10 + s, 5 + r10 + 3 * s, 10 - 2 * r10 + 2 * s,
                     10 - 2 * r10 - 2 * s, 5 + r10 - 3 * s, 1 + r10 - s]) / (16 * np.sqrt(2.0))
    assert np.allclose(dbm.daubechies_lowpass(3), want, rtol=0, atol=1e-14)


@pytest.mark.parametrize("p", range(1, 9))
def test_filter_identities(p):
    h = dbm.daubechies_lowpass(p)
    g = dbm.daubechies_highpass(h)
    assert h.size == 2 * p
    assert h.sum() == pytest.approx(np.sqrt(2.0), abs=1e-13)
    for m in range(p):
        dot = np.dot(h[: h.size - 2 * m], h[2 * m:])
        assert dot == pytest.approx(1.0 if m == 0 else 0.0, abs=1e-13)
        assert np.dot(g[: g.size - 2 * m], h[2 * m:]) == pytest.approx(0.0, abs=1e-13)
        assert np.dot(h[: h.size - 2 * m], g[2 * m:]) == pytest.approx(0.0, abs=1e-13)
    k = np.arange(2 * p, dtype=np.float64)
    for j in range(p):
        # vanishing moments, scaled by the size of the terms
        assert abs(np.sum(k ** j * g)) <= 1e-11 * max(1.0, np.sum(np.abs(k ** j * g)))


@pytest.mark.parametrize("p", range(2, 9))
def test_minimum_phase(p):
    # sum_m h[m] z^(2p-1-m) = (z + 1)^p q(z): the remainder of the division is zero
    # and every zero of q lies strictly inside the unit circle.
    h = dbm.daubechies_lowpass(p)
    q, rem = np.polydiv(h, np.poly(-np.ones(p)))
    assert np.max(np.abs(rem)) < 1e-12
    assert q.size == p
    assert np.all(np.abs(np.roots(q)) < 1.0 - 1e-6)
