"""Pins of the oracle's spectral dictionary as a union of m_nu orthonormal
bases (Section 3, step V: W_nu W_nu^T = m_nu I, so S = C / (m_nu rho_V + rho_S))
and of its second basis, the Chebyshev polynomial basis Section 4 suggests,
made orthonormal on the equispaced bands (the discrete Chebyshev, or Gram,
polynomials).

- The Chebyshev matrix is orthonormal, its rows of degree 0 and 1 have closed
  forms, and row k is a polynomial of degree exactly k in the band position.
- With m_nu = 2 (DCT + Chebyshev) steps IV and V are the minimisers of the
  augmented Lagrangian (IV by the prox closed form per basis, V by a dense
  least-squares solve of the stacked system).
- The iteration converges to the optimum of the problem with both spectral
  terms, computed independently from its Fenchel dual on a tiny cube.
- He and Yuan's merit, with (m_nu rho_V + rho_S) ||dS||^2, stays monotone.
"""

import numpy as np
import pytest
import scipy.optimize

import oracle
from oracle import daubechies
from paper_1504_06847_gb300 import synth
from tests import _dense

PRM = dict(mu_eps=0.003, mu_s=0.07, mu_nu=0.02, rho_P=0.7, rho_T=1.3, rho_V=1.9, rho_S=0.6)


@pytest.mark.parametrize("L", [2, 3, 8, 15, 32, 64])
def test_chebyshev_basis_orthonormal_with_closed_forms(L):
    P = oracle.chebyshev_matrix(L)
    assert np.max(np.abs(P @ P.T - np.eye(L))) < 1e-12
    assert np.max(np.abs(P[0] - 1 / np.sqrt(L))) < 1e-15
    l = np.arange(L)
    t1 = (2 * l - (L - 1)) / np.sqrt(L * (L * L - 1) / 3.0)
    assert np.max(np.abs(P[1] - t1)) < 1e-14


@pytest.mark.parametrize("L", [8, 15])
def test_chebyshev_rows_have_exact_degree(L):
    P = oracle.chebyshev_matrix(L)
    t = np.linspace(-1, 1, L)
    for k in range(L):
        fit = np.polynomial.chebyshev.chebfit(t, P[k], k)
        assert np.max(np.abs(np.polynomial.chebyshev.chebval(t, fit) - P[k])) < 1e-10
        if k > 0:
            low = np.polynomial.chebyshev.chebfit(t, P[k], k - 1)
            assert np.max(np.abs(np.polynomial.chebyshev.chebval(t, low) - P[k])) > 1e-3


def test_steps_IV_and_V_with_two_spectral_bases():
    c = synth.make_cube(8, 5, n_sources=2, n_antennas=10, seed=51)
    pb = oracle.Problem(c.psf, c.y, PRM, J=2, spectral=("dct", "cheb"))
    rng = np.random.default_rng(52)
    st = pb.zero_state()
    for k in st:
        st[k][...] = 0.1 * rng.normal(size=st[k].shape)
    old = {k: v.copy() for k, v in st.items()}
    X = 0.2 * rng.normal(size=st["X"].shape)
    pb.primal_dual(X, st)
    p = pb.params
    Cs = [_dense.dct_matrix(pb.L), oracle.chebyshev_matrix(pb.L)]
    tau = p["mu_nu"] / p["rho_V"]
    for j, C in enumerate(Cs):
        SW = np.einsum("kl,lij->kij", C, old["S"])
        t = SW - old["GV"][j] / p["rho_V"]
        assert np.max(np.abs(st["V"][j] - np.sign(t) * np.maximum(np.abs(t) - tau, 0.0))) < 1e-14
    # V: S = argmin sum_j rho_V/2 ||V_j - S W_j + G_Vj/rho_V||^2 + rho_S/2 ||S - X + G_S/rho_S||^2
    A = np.vstack([np.sqrt(p["rho_V"]) * C for C in Cs] + [np.sqrt(p["rho_S"]) * np.eye(pb.L)])
    for i in range(pb.N):
        for jj in range(pb.N):
            rhs = np.concatenate([np.sqrt(p["rho_V"]) * (st["V"][j][:, i, jj] + old["GV"][j][:, i, jj] / p["rho_V"])
                                  for j in range(2)] +
                                 [np.sqrt(p["rho_S"]) * (X[:, i, jj] - old["GS"][:, i, jj] / p["rho_S"])])
            s_ref = np.linalg.lstsq(A, rhs, rcond=None)[0]
            assert np.max(np.abs(st["S"][:, i, jj] - s_ref)) < 1e-13
    # VI: each Gamma_Vj moves by rho_V (V_j - S+ W_j)
    for j, C in enumerate(Cs):
        ref = old["GV"][j] + p["rho_V"] * (st["V"][j] - np.einsum("kl,lij->kij", C, st["S"]))
        assert np.max(np.abs(st["GV"][j] - ref)) < 1e-13


def _dual_optimum(c, params, J, mask, spectral):
    """x* of 1/2||y-Hx||^2 + mu_eps/2||x||^2 + mu_s sum_k ||W_k x||_1 + mu_nu sum_j ||x W_j||_1 + 1_{R+}(x)
    from its bounded dual (see tests/test_oracle_admm.py), with one mu_nu block per spectral basis."""
    L, N = c.y.shape[0], c.y.shape[-1]
    n = N * N * L
    Hd = np.zeros((n, n))
    for l in range(L):
        Hd[l * N * N:(l + 1) * N * N, l * N * N:(l + 1) * N * N] = _dense.conv_matrix(c.psf[l])
    Ws = [np.kron(np.eye(L), _dense.dwt_matrix(h, N, J)) for _, h in daubechies.dictionary(mask)]
    Cn = [np.kron(C, np.eye(N * N)) for C in spectral]
    K = np.vstack(Ws + Cn + [np.eye(n)])
    Q0 = Hd.T @ Hd + params["mu_eps"] * np.eye(n)
    q = Hd.T @ c.y.ravel()
    w, U = np.linalg.eigh(Q0)
    Qmh = U @ np.diag(w ** -0.5) @ U.T
    nb, nm = len(Ws), len(Cn)
    lb = np.concatenate([-params["mu_s"] * np.ones(nb * n), -params["mu_nu"] * np.ones(nm * n), -np.inf * np.ones(n)])
    ub = np.concatenate([params["mu_s"] * np.ones(nb * n), params["mu_nu"] * np.ones(nm * n), np.zeros(n)])
    r = scipy.optimize.lsq_linear(Qmh @ K.T, Qmh @ q, bounds=(lb, ub), method="bvls", tol=1e-15, max_iter=200000)
    lam = r.x
    xs = np.linalg.solve(Q0, q - K.T @ lam)
    dual = -0.5 * (q - K.T @ lam) @ np.linalg.solve(Q0, q - K.T @ lam) + 0.5 * c.y.ravel() @ c.y.ravel()
    xp = np.maximum(xs, 0.0)
    primal = (0.5 * np.sum((c.y.ravel() - Hd @ xp) ** 2) + 0.5 * params["mu_eps"] * xp @ xp
              + params["mu_s"] * sum(np.abs(W @ xp).sum() for W in Ws)
              + params["mu_nu"] * sum(np.abs(C @ xp).sum() for C in Cn))
    return xs.reshape(c.y.shape), primal - dual


def test_converges_to_brute_force_optimum_with_two_spectral_bases():
    c = synth.make_cube(8, 4, n_sources=2, n_antennas=12, seed=21)
    params = dict(mu_eps=0.01, mu_s=0.05, mu_nu=0.02, rho_P=1.0, rho_T=1.0, rho_V=1.0, rho_S=1.0)
    xs, gap = _dual_optimum(c, params, 1, 0x107, [_dense.dct_matrix(4), oracle.chebyshev_matrix(4)])
    assert gap < 1e-9
    pb = oracle.Problem(c.psf, c.y, params, J=1, mask=0x107, spectral=("dct", "cheb"))
    st, _ = pb.run(60000)
    assert np.max(np.abs(st["X"] - xs)) < 1e-6


def test_merit_monotone_with_two_spectral_bases():
    c = synth.workload("64x64x8")
    pb = oracle.Problem(c.psf, c.y, synth.WORKLOAD_PARAMS, spectral=("dct", "cheb"))
    _, H = pb.run(30, hist=True)
    E = H[:, 2]
    assert np.all(E[2:] <= E[1:-1] * (1 + 1e-10) + 1e-20 * E[1]), E
    assert H[-1, 0] < 1e-2 * H[0, 0]
