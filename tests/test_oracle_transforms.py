"""Pins of the oracle's FFT, wavelet transform and DCT.

- FFT: equals numpy's FFT (a library routine the oracle does not call).
- Wavelets: each basis of W_s is orthonormal, W^T W = W W^T = I, which is what
  Eq. Qlsimp needs (W_s^T W_s = n_s I for a union of n_s bases); it equals the
  dense matrix assembled from the definition; constants have no detail
  coefficients (first vanishing moment); Haar on 2 x 2 has a closed form.
- DCT: orthonormal and equal to scipy's orthonormal DCT-II.
"""

import numpy as np
import pytest
import scipy.fft

import oracle
from oracle import daubechies
from tests import _dense


def test_fft2_matches_numpy():
    rng = np.random.default_rng(0)
    for N in (2, 8, 16, 64):
        x = rng.normal(size=(3, N, N)) + 1j * rng.normal(size=(3, N, N))
        assert np.max(np.abs(oracle.fft2(x) - np.fft.fft2(x))) < 1e-12 * N * N
        assert np.max(np.abs(oracle.fft2(x, inverse=True) - np.fft.ifft2(x) * N * N)) < 1e-12 * N * N


@pytest.mark.parametrize("N,J", [(16, 1), (16, 2), (16, 3), (32, 3), (64, 3), (8, 3)])
@pytest.mark.parametrize("K", [1, 2, 5, 8])
def test_dwt_orthonormal(N, J, K):
    h = daubechies.daubechies(K)
    rng = np.random.default_rng(N * 100 + J * 10 + K)
    x = rng.normal(size=(2, N, N))
    z = oracle.dwt2(x, h, J)
    assert abs(np.linalg.norm(z) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)
    assert np.max(np.abs(oracle.dwt2(z, h, J, inverse=True) - x)) < 1e-12
    zz = rng.normal(size=(2, N, N))
    assert np.max(np.abs(oracle.dwt2(oracle.dwt2(zz, h, J, inverse=True), h, J) - zz)) < 1e-12
    # analysis and synthesis are transposes: <W x, z> = <x, W^T z>
    assert abs(np.vdot(z, zz) - np.vdot(x, oracle.dwt2(zz, h, J, inverse=True))) < 1e-10


@pytest.mark.parametrize("N,J,K", [(8, 1, 2), (8, 2, 4), (8, 3, 8), (16, 2, 3)])
def test_dwt_equals_dense_definition(N, J, K):
    h = daubechies.daubechies(K)
    W = _dense.dwt_matrix(h, N, J)
    x = np.random.default_rng(7).normal(size=(N, N))
    assert np.max(np.abs(oracle.dwt2(x, h, J).ravel() - W @ x.ravel())) < 1e-13
    z = np.random.default_rng(8).normal(size=(N, N))
    assert np.max(np.abs(oracle.dwt2(z, h, J, inverse=True).ravel() - W.T @ z.ravel())) < 1e-13


@pytest.mark.parametrize("K", range(1, 9))
def test_dwt_of_constant(K):
    # sum h = sqrt 2 and sum g = 0: a constant c maps to c 2^J in the coarse block, 0 elsewhere
    N, J = 32, 3
    h = daubechies.daubechies(K)
    z = oracle.dwt2(np.full((N, N), 1.5), h, J)
    M = N >> J
    assert np.max(np.abs(z[:M, :M] - 1.5 * 2 ** J)) < 1e-12
    z[:M, :M] = 0.0
    assert np.max(np.abs(z)) < 1e-12


def test_haar_2x2_closed_form():
    x = np.array([[1.0, 2.0], [3.0, 5.0]])
    z = oracle.dwt2(x, daubechies.HAAR, 1)
    a, b, c, d = 1.0, 2.0, 3.0, 5.0
    ref = 0.5 * np.array([[a + b + c + d, a - b + c - d], [a + b - c - d, a - b - c + d]])
    assert np.max(np.abs(z - ref)) < 1e-15


@pytest.mark.parametrize("L", [2, 8, 15, 32, 64])
def test_dct_orthonormal_and_scipy(L):
    C = oracle.dct_matrix(L)
    assert np.max(np.abs(C @ C.T - np.eye(L))) < 1e-14
    x = np.random.default_rng(L).normal(size=(L, 5))
    assert np.max(np.abs(C @ x - scipy.fft.dct(x, type=2, norm="ortho", axis=0))) < 1e-13
