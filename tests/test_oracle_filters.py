"""Pins of the oracle's Daubechies filters (Section 4's dictionary Db1..Db8 + Haar).

The paper names the bases only; the filters are fixed by Daubechies'
construction (orthonormality, K vanishing moments, extremal phase) and by the
closed forms of Db2 and Db3 (Daubechies 1988, Comm. Pure Appl. Math. 41).
"""

import numpy as np
import pytest

from oracle import daubechies


@pytest.mark.parametrize("K", range(1, 9))
def test_normalisation_and_shift_orthogonality(K):
    h = daubechies.daubechies(K)
    assert len(h) == 2 * K
    assert abs(h.sum() - np.sqrt(2.0)) < 1e-14
    for m in range(0, K):
        s = float(np.dot(h[: len(h) - 2 * m], h[2 * m:]))
        assert abs(s - (1.0 if m == 0 else 0.0)) < 5e-15, (K, m, s)


@pytest.mark.parametrize("K", range(1, 9))
def test_vanishing_moments(K):
    h = daubechies.daubechies(K)
    F = len(h)
    n = np.arange(F, dtype=float)
    g = np.array([(-1) ** i * h[F - 1 - i] for i in range(F)])
    for p in range(K):
        scale = np.sum(np.abs(g) * n ** p)
        assert abs(np.sum(g * n ** p)) < 1e-13 * max(scale, 1.0), (K, p)
    # the K-th moment does not vanish (exactly K vanishing moments)
    assert abs(np.sum(g * n ** K)) > 1e-6


@pytest.mark.parametrize("K", range(2, 9))
def test_extremal_phase(K):
    # zeros of sum h_n z^n other than the K-fold zero at z = -1 lie outside the unit circle
    h = daubechies.daubechies(K)
    q = np.polynomial.polynomial.polydiv(h, np.polynomial.polynomial.polypow([1.0, 1.0], K))
    assert np.max(np.abs(q[1])) < 1e-12
    zs = np.polynomial.polynomial.polyroots(q[0])
    assert np.all(np.abs(zs) > 1.0 + 1e-6)


def test_db1_is_haar():
    assert np.array_equal(daubechies.daubechies(1), daubechies.HAAR)
    assert np.max(np.abs(daubechies.HAAR - np.sqrt(0.5))) <= 2.3e-16


def test_db2_closed_form():
    s3 = np.sqrt(3.0)
    ref = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4 * np.sqrt(2.0))
    assert np.max(np.abs(daubechies.daubechies(2) - ref)) < 1e-15


def test_db3_closed_form():
    s10 = np.sqrt(10.0)
    r = np.sqrt(5 + 2 * s10)
    ref = np.array([1 + s10 + r, 5 + s10 + 3 * r, 10 - 2 * s10 + 2 * r,
                    10 - 2 * s10 - 2 * r, 5 + s10 - 3 * r, 1 + s10 - r]) / (16 * np.sqrt(2.0))
    assert np.max(np.abs(daubechies.daubechies(3) - ref)) < 1e-15


def test_dictionary_mask():
    d = daubechies.dictionary(0x1FF)
    assert [n for n, _ in d] == [f"db{k}" for k in range(1, 9)] + ["haar"]
    assert [n for n, _ in daubechies.dictionary(0b100000101)] == ["db1", "db3", "haar"]
