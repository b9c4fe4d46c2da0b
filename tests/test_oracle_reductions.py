"""Pins of the oracle's per-iteration reductions (the values every residual
and objective parity check of the CUDA path is compared with).

After each of the first iterations of Algorithm 1 the oracle reports, in
FP64, the primal residual, the dual residual of Boyd et al. (2011, Sec. 3.3)
for the two-block split (X, V) | (P, T, S) of Section 3, the objective of
Eqs. costreg and eq:RegAll, and the summed squared change of the four
multipliers.  Here each is rebuilt from the oracle's state arrays before and
after the iteration with dense operators assembled in the tests (H from the
PSF element by element, every W_k as the dense matrix of its J-level
transform, W_nu as the dense DCT-II matrix), so a dropped factor (the 1/2 of
the data fit, a rho), a transposed operand (W_nu against W_nu^T), a basis
missing from a sum or the wrong S (old against new) in a term shows up as a
mismatch:

  r^2 = ||P-X||^2 + sum_k ||T_k - W_k X||^2 + ||V - S W_nu||^2 + ||S-X||^2
  s^2 = ||rho_P dP + rho_T sum_k W_k^T dT_k + rho_S dS||^2 + rho_V^2 ||dS W_nu||^2
  F   = 1/2||Y - H X||^2 + mu_eps/2 ||X||^2 + mu_s sum_k ||W_k X||_1 + mu_nu ||X W_nu||_1
  sum_c ||dGamma_c||^2 over Gamma_P, every Gamma_T,k, Gamma_V and Gamma_S.
"""

import numpy as np
import pytest

import oracle
from oracle import daubechies
from paper_1504_06847_gb300 import synth
from tests import _dense

# distinct penalties, so that a rho taken for another one is seen
PRM = dict(mu_eps=0.003, mu_s=0.04, mu_nu=0.015, rho_P=0.7, rho_T=1.3, rho_V=1.9, rho_S=0.6)


def _dense_ops(c, J, mask, conv="circular"):
    L, N = c.y.shape[0], c.y.shape[-1]
    build = _dense.linear_conv_matrix if conv == "linear" else _dense.conv_matrix
    H = [build(c.psf[l]) for l in range(L)]
    W = [_dense.dwt_matrix(h, N, J) for _, h in daubechies.dictionary(mask)]
    return H, W, _dense.dct_matrix(L)


def _apply_bands(M, cube):
    """M (N^2 x N^2) applied to every band image of cube [L, N, N]."""
    L, N = cube.shape[0], cube.shape[-1]
    return np.stack([(M @ cube[l].ravel()).reshape(N, N) for l in range(L)])


def _spectral(C, cube):
    """cube W_nu: (X W_nu)[k] = sum_l C[k, l] X[l] for every pixel."""
    return np.einsum("kl,lij->kij", C, cube)


def _reductions(c, H, W, C, prev, st, p):
    """C: the spectral basis matrix, or a list of them (a union of bases)."""
    Cs = C if isinstance(C, list) else [C]
    X, P, T, S = st["X"], st["P"], st["T"], st["S"]
    V = st["V"] if len(Cs) > 1 else [st["V"]]
    Z = [_apply_bands(Wk, X) for Wk in W]
    primal = (np.sum((P - X) ** 2) + sum(np.sum((T[k] - Z[k]) ** 2) for k in range(len(W)))
              + sum(np.sum((V[j] - _spectral(Cj, S)) ** 2) for j, Cj in enumerate(Cs)) + np.sum((S - X) ** 2))
    dP, dS = P - prev["P"], S - prev["S"]
    sx = p["rho_P"] * dP + p["rho_S"] * dS
    for k, Wk in enumerate(W):
        sx = sx + p["rho_T"] * _apply_bands(Wk.T, T[k] - prev["T"][k])
    dual = np.sum(sx ** 2) + p["rho_V"] ** 2 * sum(np.sum(_spectral(Cj, dS) ** 2) for Cj in Cs)
    HX = np.stack([(H[l] @ X[l].ravel()).reshape(X.shape[1:]) for l in range(X.shape[0])])
    objective = (0.5 * np.sum((c.y - HX) ** 2) + 0.5 * p["mu_eps"] * np.sum(X ** 2)
                 + p["mu_s"] * sum(np.abs(z).sum() for z in Z)
                 + p["mu_nu"] * sum(np.abs(_spectral(Cj, X)).sum() for Cj in Cs))
    dgamma = sum(np.sum((st[g] - prev[g]) ** 2) for g in ("GP", "GT", "GV", "GS"))
    merit = (p["rho_P"] * np.sum(dP ** 2) + p["rho_T"] * np.sum((T - prev["T"]) ** 2)
             + (len(Cs) * p["rho_V"] + p["rho_S"]) * np.sum(dS ** 2)
             + sum(np.sum((st[g] - prev[g]) ** 2) / p[r]
                   for g, r in (("GP", "rho_P"), ("GT", "rho_T"), ("GV", "rho_V"), ("GS", "rho_S"))))
    return {0: primal, 1: dual, 2: merit, 3: objective, 4: X.min(), 5: np.sum(X ** 2), 6: dgamma}


@pytest.mark.parametrize("N,L,J,mask,seed,conv", [(8, 4, 2, 0x1FF, 31, "circular"), (16, 4, 3, 0x1FF, 32, "circular"),
                                                   (16, 3, 2, 0x0A5, 33, "circular"), (8, 3, 2, 0x1FF, 35, "linear")])
def test_history_matches_dense_reductions(N, L, J, mask, seed, conv):
    c = synth.make_cube(N, L, n_sources=2, n_antennas=12, seed=seed)
    pb = oracle.Problem(c.psf, c.y, PRM, J=J, mask=mask, conv=conv, cg_iters=4)
    H, W, C = _dense_ops(c, J, mask, conv)
    st = pb.zero_state()
    for it in range(3):
        prev = {k: v.copy() for k, v in st.items()}
        hist = pb.iterate(st, 1, hist=True)[0]
        ref = _reductions(c, H, W, C, prev, st, PRM)
        for q, v in ref.items():
            assert abs(hist[q] - v) <= 1e-12 * max(abs(v), 1e-300) + 1e-300, (it, q, hist[q], v)
        assert hist[1] > 0 and hist[0] > 0


def test_history_with_two_spectral_bases():
    c = synth.make_cube(8, 5, n_sources=2, n_antennas=12, seed=36)
    pb = oracle.Problem(c.psf, c.y, PRM, J=2, spectral=("dct", "cheb"))
    H, W, C = _dense_ops(c, 2, 0x1FF)
    Cs = [C, oracle.chebyshev_matrix(5)]
    st = pb.zero_state()
    for it in range(3):
        prev = {k: v.copy() for k, v in st.items()}
        hist = pb.iterate(st, 1, hist=True)[0]
        ref = _reductions(c, H, W, Cs, prev, st, PRM)
        for q, v in ref.items():
            assert abs(hist[q] - v) <= 1e-12 * max(abs(v), 1e-300) + 1e-300, (it, q, hist[q], v)


def test_dual_residual_sees_each_term():
    """Each of the three change terms of the dual residual contributes: the
    reference value moves when any one of them is dropped, so agreement above
    is not carried by a subset."""
    c = synth.make_cube(8, 4, n_sources=2, n_antennas=12, seed=34)
    pb = oracle.Problem(c.psf, c.y, PRM, J=2)
    H, W, C = _dense_ops(c, 2, 0x1FF)
    st = pb.zero_state()
    pb.iterate(st, 1)
    prev = {k: v.copy() for k, v in st.items()}
    hist = pb.iterate(st, 1, hist=True)[0]
    full = _reductions(c, H, W, C, prev, st, PRM)[1]
    assert abs(hist[1] - full) <= 1e-12 * full
    for drop in ("P", "T", "S"):
        cut = dict(prev)
        cut[drop] = st[drop]  # no change in that variable
        assert abs(_reductions(c, H, W, C, cut, st, PRM)[1] - full) > 1e-6 * full, drop
