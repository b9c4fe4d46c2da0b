"""Pins of the oracle's whole ADMM iteration (Algorithm 1).

- He and Yuan's merit for two-block ADMM (SIAM J. Numer. Anal. 2015): with
  the blocks (X, V) | (P, T, S) that Algorithm 1 updates in this order,
  E_k = rho_P||dP||^2 + rho_T||dT||^2 + (rho_V + rho_S)||dS||^2
        + sum_c ||dGamma_c||^2 / rho_c is non-increasing.
- Convergence to the optimum of the convex problem (Eqs. costreg, eq:RegAll),
  computed independently by a bounded-variable least-squares solve of its
  Fenchel dual on tiny cubes and certified by a duality gap.
- Special cases with closed forms: H = I without sparsity terms gives
  X* = max(0, Y / (1 + mu_eps)); a Tikhonov solution that is already positive
  gives X* = (H^T H + mu_eps I)^-1 H^T Y.
- The optimality relations of step VI hold at every iteration.
"""

import numpy as np
import pytest
import scipy.optimize

import oracle
from paper_1504_06847_gb300 import synth
from tests import _dense


def _merit_is_monotone(H, rel=1e-10):
    # non-increasing from the second iteration on, down to the FP64 rounding floor
    E = H[:, 2]
    floor = 1e-20 * E[1]
    return np.all(E[2:] <= E[1:-1] * (1 + rel) + floor)


@pytest.mark.parametrize("params", [synth.WORKLOAD_PARAMS, synth.PAPER_PARAMS])
def test_merit_monotone_64x64x8(params):
    c = synth.workload("64x64x8")
    pb = oracle.Problem(c.psf, c.y, params)
    st, H = pb.run(40, hist=True)
    assert _merit_is_monotone(H), H[:, 2]
    assert H[-1, 0] < 1e-2 * H[0, 0]  # primal residual falls
    # invariants of step VI after the last iteration
    C = oracle.dct_matrix(pb.L)
    assert st["GP"].min() >= -1e-12
    assert np.abs(st["GT"]).max() <= params["mu_s"] + 1e-12
    assert np.max(np.abs(st["GS"] - np.einsum("kl,kij->lij", C, st["GV"]))) < 1e-12


def test_reconstruction_beats_dirty_image():
    c = synth.workload("64x64x8")
    pb = oracle.Problem(c.psf, c.y, synth.WORKLOAD_PARAMS)
    st, _ = pb.run(50)
    err = np.linalg.norm(st["X"] - c.sky) / np.linalg.norm(c.sky)
    assert err < 0.1


def _dual_optimum(c, params, J, mask):
    """x* of min 1/2||y-Hx||^2 + mu_eps/2||x||^2 + mu_s||W_s x||_1 + mu_nu||x W_nu||_1 + 1_{R+}(x)
    via its dual: max over |u| <= mu_s, |v| <= mu_nu, w <= 0 of
    -1/2 (q - K^T lam)^T Q0^-1 (q - K^T lam), q = H^T y, Q0 = H^T H + mu_eps I,
    K = [W_s; W_nu; I]; then x* = Q0^-1 (q - K^T lam*)."""
    L, N = c.y.shape[0], c.y.shape[-1]
    n = N * N * L
    Hd = np.zeros((n, n))
    for l in range(L):
        Hd[l * N * N:(l + 1) * N * N, l * N * N:(l + 1) * N * N] = _dense.conv_matrix(c.psf[l])
    from oracle import daubechies
    Ws = [np.kron(np.eye(L), _dense.dwt_matrix(h, N, J)) for _, h in daubechies.dictionary(mask)]
    Cn = np.kron(_dense.dct_matrix(L), np.eye(N * N))
    K = np.vstack(Ws + [Cn, np.eye(n)])
    Q0 = Hd.T @ Hd + params["mu_eps"] * np.eye(n)
    q = Hd.T @ c.y.ravel()
    w, U = np.linalg.eigh(Q0)
    Qmh = U @ np.diag(w ** -0.5) @ U.T
    nb = len(Ws)
    lb = np.concatenate([-params["mu_s"] * np.ones(nb * n), -params["mu_nu"] * np.ones(n), -np.inf * np.ones(n)])
    ub = np.concatenate([params["mu_s"] * np.ones(nb * n), params["mu_nu"] * np.ones(n), np.zeros(n)])
    r = scipy.optimize.lsq_linear(Qmh @ K.T, Qmh @ q, bounds=(lb, ub), method="bvls", tol=1e-15,
                                  max_iter=200000)
    lam = r.x
    xs = np.linalg.solve(Q0, q - K.T @ lam)
    dual = -0.5 * (q - K.T @ lam) @ np.linalg.solve(Q0, q - K.T @ lam) + 0.5 * c.y.ravel() @ c.y.ravel()
    xp = np.maximum(xs, 0.0)
    primal = (0.5 * np.sum((c.y.ravel() - Hd @ xp) ** 2) + 0.5 * params["mu_eps"] * xp @ xp
              + params["mu_s"] * sum(np.abs(W @ xp).sum() for W in Ws) + params["mu_nu"] * np.abs(Cn @ xp).sum())
    return xs.reshape(c.y.shape), primal - dual


@pytest.mark.parametrize("J,mask,iters", [(1, 0x107, 60000), (2, 0x10B, 60000)])
def test_converges_to_brute_force_optimum(J, mask, iters):
    c = synth.make_cube(8, 4, n_sources=2, n_antennas=12, seed=21)
    params = dict(mu_eps=0.01, mu_s=0.05, mu_nu=0.02, rho_P=1.0, rho_T=1.0, rho_V=1.0, rho_S=1.0)
    xs, gap = _dual_optimum(c, params, J, mask)
    assert gap < 1e-9
    pb = oracle.Problem(c.psf, c.y, params, J=J, mask=mask)
    st, _ = pb.run(iters)
    assert np.max(np.abs(st["X"] - xs)) < 1e-6


@pytest.mark.slow
def test_converges_to_brute_force_optimum_full_dictionary():
    c = synth.make_cube(8, 4, n_sources=2, n_antennas=12, seed=21)
    params = dict(mu_eps=0.01, mu_s=0.05, mu_nu=0.02, rho_P=1.0, rho_T=1.0, rho_V=1.0, rho_S=1.0)
    xs, gap = _dual_optimum(c, params, 1, 0x1FF)
    assert gap < 1e-9
    pb = oracle.Problem(c.psf, c.y, params, J=1, mask=0x1FF)
    st, _ = pb.run(100000)
    assert np.max(np.abs(st["X"] - xs)) < 1e-6


def test_identity_psf_without_sparsity():
    N, L = 16, 4
    rng = np.random.default_rng(1)
    psf = np.zeros((L, N, N))
    psf[:, N // 2, N // 2] = 1.0
    y = rng.normal(size=(L, N, N))
    params = dict(mu_eps=0.05, mu_s=0.0, mu_nu=0.0, rho_P=1.0, rho_T=1.0, rho_V=1.0, rho_S=1.0)
    pb = oracle.Problem(psf, y, params, J=2)
    st, H = pb.run(3000, hist=True)
    assert np.max(np.abs(st["X"] - np.maximum(0.0, y / (1 + params["mu_eps"])))) < 1e-9
    assert _merit_is_monotone(H)


def test_tikhonov_special_case():
    N, L = 16, 3
    r2 = ((np.arange(N) - N // 2)[:, None] ** 2 + (np.arange(N) - N // 2)[None, :] ** 2)
    psf = np.stack([np.exp(-r2 / (2 * (0.6 + 0.2 * l) ** 2)) for l in range(L)])
    x = 1.0 + 0.2 * np.random.default_rng(4).uniform(size=(L, N, N))
    c = synth.Cube(sky=x, psf=psf, y=np.zeros_like(x), nu=np.ones(L), sigma=0.0)
    mu = 0.05
    ref = np.empty_like(x)
    for l in range(L):
        H = _dense.conv_matrix(psf[l])
        c.y[l] = (H @ x[l].ravel()).reshape(N, N)
        ref[l] = np.linalg.solve(H.T @ H + mu * np.eye(N * N), H.T @ c.y[l].ravel()).reshape(N, N)
    assert ref.min() > 0
    params = dict(mu_eps=mu, mu_s=0.0, mu_nu=0.0, rho_P=1.0, rho_T=1.0, rho_V=1.0, rho_S=1.0)
    pb = oracle.Problem(c.psf, c.y, params, J=2, mask=0x103)
    st, _ = pb.run(2000)
    assert np.max(np.abs(st["X"] - ref)) < 1e-9
