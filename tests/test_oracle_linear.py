"""Pins of the oracle's step I for a non-circulant H (linear convolution) and
its conjugate gradient solve (Algorithm 1's comment; Hestenes-Stiefel, as the
paper's Section 3 cites).

- H x and H^T x through the 2N FFT equal the dense linear ("same"-size)
  convolution matrix, assembled element by element, and its transpose.
- k conjugate gradient iterations from a given start equal k iterations of the
  textbook recurrence run with the dense Q = H^T H + rho I (so a finite-iteration
  iterate, not only the converged answer, is pinned), band by band.
- Run long enough, the solve equals the dense solution of Q x = b.
- With a delta PSF the linear and circular convolutions are both the identity:
  the linear-mode ADMM equals the circular-mode ADMM.
- With exact step I (CG run to convergence) the linear-mode ADMM keeps He and
  Yuan's merit non-increasing.
"""

import numpy as np
import pytest

import oracle
from paper_1504_06847_gb300 import synth
from tests import _dense

PRM = dict(mu_eps=0.003, mu_s=0.04, mu_nu=0.015, rho_P=0.7, rho_T=1.3, rho_V=1.9, rho_S=0.6)


def _cube(N=8, L=3, seed=41):
    c = synth.make_cube(N, L, n_sources=2, n_antennas=10, seed=seed)
    return c


def test_operator_equals_dense_linear_convolution():
    c = _cube(N=8, L=3)
    pb = oracle.Problem(c.psf, c.y, PRM, J=2, conv="linear", cg_iters=5)
    x = np.random.default_rng(2).normal(size=c.y.shape)
    hx, htx = pb.apply_H(x), pb.apply_H(x, adjoint=True)
    for l in range(pb.L):
        H = _dense.linear_conv_matrix(c.psf[l])
        assert np.max(np.abs(hx[l].ravel() - H @ x[l].ravel())) < 1e-12
        assert np.max(np.abs(htx[l].ravel() - H.T @ x[l].ravel())) < 1e-12
        assert np.max(np.abs(pb.HtY[l].ravel() - H.T @ c.y[l].ravel())) < 1e-12
    # the linear and circular operators differ (the PSF does not wrap)
    assert np.max(np.abs(hx[0].ravel() - _dense.conv_matrix(c.psf[0]) @ x[0].ravel())) > 1e-3


def _dense_cg(Q, b, x, iters):
    r = b - Q @ x
    p = r.copy()
    g = r @ r
    for _ in range(iters):
        if g == 0.0:
            break
        q = Q @ p
        pq = p @ q
        if not pq > 0.0:
            break
        a = g / pq
        x = x + a * p
        r = r - a * q
        g2 = r @ r
        p = r + (g2 / g) * p
        g = g2
    return x


@pytest.mark.parametrize("iters", [1, 3, 12])
def test_cg_iterates_equal_the_textbook_recurrence(iters):
    c = _cube(N=8, L=3, seed=42)
    pb = oracle.Problem(c.psf, c.y, PRM, J=2, conv="linear")
    rng = np.random.default_rng(3)
    b = rng.normal(size=c.y.shape)
    x0 = rng.normal(size=c.y.shape)
    X = pb.solve(b, x0=x0, cg_iters=iters)
    for l in range(pb.L):
        H = _dense.linear_conv_matrix(c.psf[l])
        Q = H.T @ H + pb.rho_bar * np.eye(pb.N ** 2)
        ref = _dense_cg(Q, b[l].ravel(), x0[l].ravel(), iters)
        assert np.max(np.abs(X[l].ravel() - ref)) < 1e-11 * max(1.0, np.abs(ref).max())


def test_cg_converges_to_the_dense_solve():
    c = _cube(N=16, L=2, seed=43)
    pb = oracle.Problem(c.psf, c.y, PRM, J=2, conv="linear")
    b = np.random.default_rng(4).normal(size=c.y.shape)
    X = pb.solve(b, cg_iters=200)
    for l in range(pb.L):
        H = _dense.linear_conv_matrix(c.psf[l])
        x = np.linalg.solve(H.T @ H + pb.rho_bar * np.eye(pb.N ** 2), b[l].ravel())
        assert np.max(np.abs(X[l].ravel() - x)) < 1e-10 * np.abs(x).max()


def test_delta_psf_linear_equals_circular():
    N, L = 16, 3
    psf = np.zeros((L, N, N))
    psf[:, N // 2, N // 2] = 1.0
    y = np.random.default_rng(5).normal(size=(L, N, N))
    lin = oracle.Problem(psf, y, PRM, J=2, conv="linear", cg_iters=3)
    cir = oracle.Problem(psf, y, PRM, J=2)
    a, _ = lin.run(12)
    b, _ = cir.run(12)
    for k in a:
        assert np.max(np.abs(a[k] - b[k])) < 1e-12, k


def test_merit_monotone_with_exact_step_I():
    c = _cube(N=16, L=4, seed=44)
    pb = oracle.Problem(c.psf, c.y, synth.WORKLOAD_PARAMS, J=2, conv="linear", cg_iters=150)
    _, H = pb.run(25, hist=True)
    E = H[:, 2]
    assert np.all(E[2:] <= E[1:-1] * (1 + 1e-8) + 1e-20 * E[1]), E
    assert H[-1, 0] < 1e-2 * H[0, 0]
