"""Dense operators for tiny cubes, built in the tests from their definitions.

These matrices are the brute-force side of the oracle's pins: they are
assembled here element by element (no call into the oracle's transforms), so
a wrong index, sign or transpose in the oracle shows up as a mismatch.
"""

import numpy as np


def conv_matrix(psf2d: np.ndarray) -> np.ndarray:
    """H for one band: (H x)[i] = sum_j psf[(i - j + N/2) mod N] x[j] in 2-D
    (circular convolution with the PSF whose peak is at (N/2, N/2))."""
    N = psf2d.shape[0]
    H = np.zeros((N * N, N * N))
    for r in range(N):
        for c in range(N):
            for rr in range(N):
                for cc in range(N):
                    H[r * N + c, rr * N + cc] = psf2d[(r - rr + N // 2) % N, (c - cc + N // 2) % N]
    return H


def analysis_1d(h: np.ndarray, M: int) -> np.ndarray:
    """Periodic one-level analysis matrix: rows i < M/2 give the low-pass
    a_i = sum_n h_n x[(2i+n) mod M]; rows M/2 + i the high-pass with
    g_n = (-1)^n h_{F-1-n}."""
    F = len(h)
    A = np.zeros((M, M))
    for i in range(M // 2):
        for n in range(F):
            A[i, (2 * i + n) % M] += h[n]
            A[M // 2 + i, (2 * i + n) % M] += (-1) ** n * h[F - 1 - n]
    return A


def dwt_matrix(h: np.ndarray, N: int, J: int) -> np.ndarray:
    """Dense N^2 x N^2 matrix of the J-level separable periodic 2-D transform:
    at level j the top-left M x M block (M = N / 2^(j-1)) becomes A_M B A_M^T."""
    W = np.eye(N * N)
    for j in range(1, J + 1):
        M = N >> (j - 1)
        A = analysis_1d(h, M)
        lev = np.zeros((N * N, N * N))
        for col in range(N * N):
            img = np.zeros((N, N))
            img.flat[col] = 1.0
            out = img.copy()
            out[:M, :M] = A @ img[:M, :M] @ A.T
            lev[:, col] = out.ravel()
        W = lev @ W
    return W


def dct_matrix(L: int) -> np.ndarray:
    """Orthonormal DCT-II: C[k, l] = a_k cos(pi (2l+1) k / (2L))."""
    C = np.zeros((L, L))
    for k in range(L):
        a = np.sqrt(1.0 / L) if k == 0 else np.sqrt(2.0 / L)
        for l in range(L):
            C[k, l] = a * np.cos(np.pi * (2 * l + 1) * k / (2 * L))
    return C


def linear_conv_matrix(psf2d: np.ndarray) -> np.ndarray:
    """H for one band with a PSF that does not wrap: (H x)[i] = sum_j psf[i - j + N/2] x[j]
    in 2-D, the PSF taken as zero outside its N x N support (linear, "same"-size
    convolution)."""
    N = psf2d.shape[0]
    H = np.zeros((N * N, N * N))
    for r in range(N):
        for c in range(N):
            for rr in range(N):
                for cc in range(N):
                    u, v = r - rr + N // 2, c - cc + N // 2
                    if 0 <= u < N and 0 <= v < N:
                        H[r * N + c, rr * N + cc] = psf2d[u, v]
    return H
