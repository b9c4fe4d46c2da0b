"""Daubechies orthonormal filters DbK (K vanishing moments, length 2K).

TEST INFRASTRUCTURE (part of the oracle).

Construction from the definition (Daubechies 1988, the spectral
factorisation): the low-pass response is
``m0(w) = ((1 + e^{-iw})/2)^K L(w)`` with
``|L(w)|^2 = P(sin^2(w/2))``, ``P(y) = sum_{k<K} C(K-1+k, k) y^k``.
With ``z = e^{-iw}``, ``sin^2(w/2) = (2 - z - 1/z)/4``, so every root y_j of
P gives the pair of zeros ``z, 1/z`` of ``z^2 - (2 - 4 y_j) z + 1``.  The
extremal-phase choice keeps, from each pair, the zero outside the unit circle
of ``H(z) = sum_n h_n z^n``; this gives the filters with their energy at the
start (h_0 = (1 + sqrt 3)/(4 sqrt 2) for K = 2).  The filter is normalised to
``sum_n h_n = sqrt(2)``.

The wavelet dictionary of the paper's Section 4 is Db1..Db8 plus a Haar basis
(Db1 and Haar are the same filter).
"""

from __future__ import annotations

from math import comb

import numpy as np


def _polish_root(coef_inc, z, iters=8):
    # Newton refinement of a root of sum_k coef_inc[k] z^k
    p = np.polynomial.Polynomial(coef_inc)
    dp = p.deriv()
    for _ in range(iters):
        d = dp(z)
        if d == 0:
            break
        z = z - p(z) / d
    return z


def daubechies(K: int) -> np.ndarray:
    """Low-pass taps h_0..h_{2K-1} of DbK (extremal phase)."""
    if K < 1:
        raise ValueError("K >= 1")
    if K == 1:
        return np.array([1.0, 1.0]) / np.sqrt(2.0)
    pc = [float(comb(K - 1 + k, k)) for k in range(K)]  # increasing powers of y
    yroots = np.roots(pc[::-1]).astype(complex)
    yroots = np.array([_polish_root(pc, y) for y in yroots])
    zeros = []
    for y in yroots:
        b = 1.0 - 2.0 * y
        disc = np.sqrt(b * b - 1.0 + 0j)
        z1, z2 = b + disc, b - disc
        zeros.append(z1 if abs(z1) > 1.0 else z2)
    q = np.poly(zeros)[::-1]  # prod (z - z_j), increasing powers
    q = np.real_if_close(q, tol=1e6).real
    hp = np.convolve([float(comb(K, n)) for n in range(K + 1)], q)
    return hp * np.sqrt(2.0) / hp.sum()


HAAR = np.array([1.0, 1.0]) / np.sqrt(2.0)


def dictionary(mask: int = 0x1FF):
    """Filters of the bases selected by ``mask``: bit K-1 for DbK (K = 1..8),
    bit 8 for the Haar basis.  Returns a list of (name, taps)."""
    out = []
    for K in range(1, 9):
        if mask >> (K - 1) & 1:
            out.append((f"db{K}", daubechies(K)))
    if mask >> 8 & 1:
        out.append(("haar", HAAR.copy()))
    return out
