"""Pins of the oracle's ADMM steps against the augmented Lagrangian of
Eqs. admm1/admm2 (Section 3), minimised here by brute force.

Each primal step of Algorithm 1 is the exact minimiser of the augmented
Lagrangian in one variable, the others fixed.  The tests build that
minimisation independently of the oracle's step formulas: stacked dense least
squares for the quadratic steps (I and V) and a vectorised golden-section
search for the separable non-smooth ones (II, III, IV).  Step VI is pinned by
the optimality relations it must produce (Boyd et al. 2011, Sec. 3.3):
Gamma_P >= 0 with Gamma_P P = 0, |Gamma_T| <= mu_s with Gamma_T = -mu_s sign(T)
on T != 0, Gamma_S = Gamma_V W_nu^T, and |Gamma_V + rho_V (S+ - S) W_nu| <= mu_nu.
"""

import numpy as np
import pytest

import oracle
from paper_1504_06847_gb300 import synth
from tests import _dense

PRM = dict(mu_eps=0.003, mu_s=0.07, mu_nu=0.02, rho_P=0.7, rho_T=1.3, rho_V=1.9, rho_S=0.6)


def _problem(N=8, L=3, J=2, seed=11, mask=0x1FF, params=PRM):
    c = synth.make_cube(N, L, n_sources=2, n_antennas=10, seed=seed)
    return c, oracle.Problem(c.psf, c.y, params, J=J, mask=mask)


def _random_state(pb, seed=3, scale=0.1):
    rng = np.random.default_rng(seed)
    st = pb.zero_state()
    for k in st:
        st[k][...] = scale * rng.normal(size=st[k].shape)
    return st


def golden_min(f, lo, hi, iters=160):
    """Vectorised golden-section minimisation of a convex elementwise f on [lo, hi]."""
    g = (np.sqrt(5.0) - 1.0) / 2.0
    a, b = lo.copy(), hi.copy()
    c = b - g * (b - a)
    d = a + g * (b - a)
    fc, fd = f(c), f(d)
    for _ in range(iters):
        left = fc < fd
        b = np.where(left, d, b)
        a = np.where(left, a, c)
        d_new = np.where(left, c, a + g * (b - a))
        c_new = np.where(left, b - g * (b - a), d)
        c, d = c_new, d_new
        fc, fd = f(c), f(d)
    return 0.5 * (a + b)


def test_setup_against_dense_operator():
    c, pb = _problem()
    for l in range(pb.L):
        H = _dense.conv_matrix(c.psf[l])
        assert np.max(np.abs(pb.HtY[l].ravel() - H.T @ c.y[l].ravel())) < 1e-12
        # hhat is the 2-D DFT of the PSF's first column of H
        assert np.max(np.abs((pb.hre[l] + 1j * pb.him[l]) - np.fft.fft2(H[:, 0].reshape(pb.N, pb.N)))) < 1e-12


def test_binary_mask_psf_gives_two_valued_filter():
    # The synthetic PSF is Re(ifft2(mask)) / peak with a Hermitian binary mask, so
    # its DFT is mask * N^2 / count: exactly two values.
    c, pb = _problem(N=16, L=2)
    for l in range(pb.L):
        hh = pb.hre[l]
        vals = np.unique(np.round(hh, 9))
        assert len(vals) == 2 and vals[0] == 0.0
        assert np.max(np.abs(pb.him[l])) < 1e-12


def _step_I_minimiser(pb, psf, y, st):
    """Per band, the X minimising the augmented Lagrangian with the other
    variables fixed, as stacked dense least squares."""
    p = pb.params
    N = pb.N
    Ws = [_dense.dwt_matrix(h, N, pb.J) for _, h in pb.bases]
    I = np.eye(N * N)
    out = []
    for l in range(pb.L):
        H = _dense.conv_matrix(psf[l])
        rows = [H, np.sqrt(p["mu_eps"]) * I, np.sqrt(p["rho_P"]) * I, np.sqrt(p["rho_S"]) * I]
        rhs = [y[l].ravel(), np.zeros(N * N),
               np.sqrt(p["rho_P"]) * (st["P"][l] + st["GP"][l] / p["rho_P"]).ravel(),
               np.sqrt(p["rho_S"]) * (st["S"][l] + st["GS"][l] / p["rho_S"]).ravel()]
        for k, W in enumerate(Ws):
            rows.append(np.sqrt(p["rho_T"]) * W)
            rhs.append(np.sqrt(p["rho_T"]) * (st["T"][k, l] + st["GT"][k, l] / p["rho_T"]).ravel())
        out.append(np.linalg.lstsq(np.vstack(rows), np.concatenate(rhs), rcond=None)[0])
    return out


@pytest.mark.parametrize("mask", [0x1FF, 0x0A2])
def test_step_I_is_the_X_minimiser(mask):
    c, pb = _problem(mask=mask)
    st = _random_state(pb)
    X = pb.solve(pb.make_b(st))
    for l, x_ref in enumerate(_step_I_minimiser(pb, c.psf, c.y, st)):
        assert np.max(np.abs(X[l].ravel() - x_ref)) < 1e-11 * max(1.0, np.abs(x_ref).max())


def test_asymmetric_psf_setup_and_step_I():
    # The recipe's PSFs are point-symmetric about (N/2, N/2), so for them
    # H^T = H and a missing conjugate in H^T y or in the filter goes unseen;
    # this PSF has no symmetry.
    rng = np.random.default_rng(5)
    N, L = 8, 3
    psf = rng.uniform(-0.3, 0.3, size=(L, N, N))
    psf[:, N // 2, N // 2] = 1.0
    y = rng.normal(size=(L, N, N))
    pb = oracle.Problem(psf, y, PRM, J=2)
    for l in range(L):
        H = _dense.conv_matrix(psf[l])
        assert np.abs(H - H.T).max() > 0.1
        assert np.max(np.abs(pb.HtY[l].ravel() - H.T @ y[l].ravel())) < 1e-12
    st = _random_state(pb)
    X = pb.solve(pb.make_b(st))
    for l, x_ref in enumerate(_step_I_minimiser(pb, psf, y, st)):
        assert np.max(np.abs(X[l].ravel() - x_ref)) < 1e-11 * max(1.0, np.abs(x_ref).max())


def test_step_I_against_dense_lu_and_cg():
    # Fourier-diagonal solve (Section 3) vs (H^T H + rho I)^-1 b, 16 x 16 x 4
    c, pb = _problem(N=16, L=4)
    b = np.random.default_rng(5).normal(size=(pb.L, pb.N, pb.N))
    X = pb.solve(b)
    for l in range(pb.L):
        H = _dense.conv_matrix(c.psf[l])
        Q = H.T @ H + pb.rho_bar * np.eye(pb.N ** 2)
        x_lu = np.linalg.solve(Q, b[l].ravel())
        assert np.max(np.abs(X[l].ravel() - x_lu)) < 1e-12
        # conjugate gradient (Hestenes-Stiefel), as Algorithm 1's comment suggests
        x = np.zeros(pb.N ** 2)
        r = b[l].ravel() - Q @ x
        d = r.copy()
        for _ in range(200):
            Qd = Q @ d
            a = (r @ r) / (d @ Qd)
            x = x + a * d
            r_new = r - a * Qd
            if np.linalg.norm(r_new) < 1e-15:
                break
            d = r_new + (r_new @ r_new) / (r @ r) * d
            r = r_new
        assert np.max(np.abs(X[l].ravel() - x)) < 1e-12


def test_steps_II_to_V_are_the_minimisers():
    c, pb = _problem()
    st = _random_state(pb, seed=4)
    old = {k: v.copy() for k, v in st.items()}
    X = 0.2 * np.random.default_rng(9).normal(size=st["X"].shape)
    pb.primal_dual(X, st)
    p = pb.params
    # II: P = argmin 1_{R+}(P) + <G_P, P - X> + rho_P/2 ||P - X||^2  (elementwise)
    t = X - old["GP"] / p["rho_P"]
    f = lambda u: np.where(u < 0, np.inf, 0.5 * (u - t) ** 2)
    lo, hi = np.zeros_like(t), np.abs(t) + 1.0
    P_ref = golden_min(f, lo, hi)
    assert np.max(np.abs(st["P"] - P_ref)) < 3e-8  # golden section resolves u to ~sqrt(eps)
    # III: T_k = argmin mu_s |T| + <G_T, T - W_k X> + rho_T/2 ||T - W_k X||^2
    for k, (_, h) in enumerate(pb.bases):
        Z = oracle.dwt2(X, h, pb.J)
        f = lambda u: p["mu_s"] * np.abs(u) + old["GT"][k] * (u - Z) + 0.5 * p["rho_T"] * (u - Z) ** 2
        span = np.abs(Z) + np.abs(old["GT"][k]) / p["rho_T"] + 1.0
        T_ref = golden_min(f, -span, span)
        assert np.max(np.abs(st["T"][k] - T_ref)) < 3e-8  # golden section resolves u to ~sqrt(eps)
    # IV (old S): V = argmin mu_nu |V| + <G_V, V - S W_nu> + rho_V/2 ||V - S W_nu||^2
    C = _dense.dct_matrix(pb.L)
    SW = np.einsum("kl,lij->kij", C, old["S"])
    f = lambda u: p["mu_nu"] * np.abs(u) + old["GV"] * (u - SW) + 0.5 * p["rho_V"] * (u - SW) ** 2
    span = np.abs(SW) + np.abs(old["GV"]) / p["rho_V"] + 1.0
    V_ref = golden_min(f, -span, span)
    assert np.max(np.abs(st["V"] - V_ref)) < 3e-8  # golden section resolves u to ~sqrt(eps)
    # V: S = argmin <G_V, V - S W_nu> + rho_V/2||V - S W_nu||^2 + <G_S, S - X> + rho_S/2||S - X||^2
    A = np.vstack([np.sqrt(p["rho_V"]) * C, np.sqrt(p["rho_S"]) * np.eye(pb.L)])
    for i in range(pb.N):
        for j in range(pb.N):
            rhs = np.concatenate([np.sqrt(p["rho_V"]) * (st["V"][:, i, j] + old["GV"][:, i, j] / p["rho_V"]),
                                  np.sqrt(p["rho_S"]) * (X[:, i, j] - old["GS"][:, i, j] / p["rho_S"])])
            s_ref = np.linalg.lstsq(A, rhs, rcond=None)[0]
            assert np.max(np.abs(st["S"][:, i, j] - s_ref)) < 1e-13


def test_step_VI_optimality_relations():
    c, pb = _problem(N=16, L=4, J=3)
    st = _random_state(pb, seed=6)
    S_old = st["S"].copy()
    X = 0.2 * np.random.default_rng(2).normal(size=st["X"].shape)
    pb.primal_dual(X, st)
    p = pb.params
    tol = 1e-12
    assert st["GP"].min() >= -tol
    assert np.max(np.abs(st["GP"] * st["P"])) < tol
    assert np.abs(st["GT"]).max() <= p["mu_s"] + tol
    nz = st["T"] != 0
    assert np.max(np.abs(st["GT"][nz] + p["mu_s"] * np.sign(st["T"][nz]))) < tol
    C = _dense.dct_matrix(pb.L)
    assert np.max(np.abs(st["GS"] - np.einsum("kl,kij->lij", C, st["GV"]))) < tol
    g = st["GV"] + p["rho_V"] * np.einsum("kl,lij->kij", C, st["S"] - S_old)
    assert np.abs(g).max() <= p["mu_nu"] + tol
    nz = st["V"] != 0
    assert np.max(np.abs(g[nz] + p["mu_nu"] * np.sign(st["V"][nz]))) < tol
