"""FP64 PyTorch restatement of the unrolled ADMM (Algorithm 1) for reference
gradients.

TEST INFRASTRUCTURE (part of the oracle; see oracle/__init__.py).  It states
the same steps as mf_oracle.c with differentiable torch operations, so that
autograd gives d||X_K - X_true||^2 / d(y, mu_s, mu_nu, rho) for K unrolled
iterations from the zero state, with the four penalties tied to one rho.
The subgradient choices follow from the operations used: d max(0,t)/dt and
d S_tau(t)/dt are 1 only where the inequality is strict.  It is pinned by the
tests to the C oracle's forward and to central finite differences of it.
"""

from __future__ import annotations

import numpy as np
import torch

from . import daubechies

DT = torch.float64


def _level_analysis(x, h):
    """One 2-D level on the last two dims (M x M): rows then columns,
    a_i = sum_n h_n x[(2i+n) mod M], d_i = sum_n g_n x[(2i+n) mod M]."""
    M = x.shape[-1]
    F = len(h)
    hh = torch.tensor(h, dtype=DT)
    gg = torch.tensor([(-1) ** n * h[F - 1 - n] for n in range(F)], dtype=DT)
    idx = torch.tensor([[(2 * i + n) % M for n in range(F)] for i in range(M // 2)])
    def rows(v):
        w = v[..., idx]  # (..., M, M/2, F)
        return torch.cat([w @ hh, w @ gg], dim=-1)
    y = rows(x)
    return rows(y.transpose(-1, -2)).transpose(-1, -2)


def _level_synthesis(z, h):
    """Transpose of _level_analysis: x[(2i+n) mod M] += h_n a_i + g_n d_i, columns then rows."""
    M = z.shape[-1]
    F = len(h)
    hh = torch.tensor(h, dtype=DT)
    gg = torch.tensor([(-1) ** n * h[F - 1 - n] for n in range(F)], dtype=DT)
    tgt = torch.tensor([(2 * i + n) % M for i in range(M // 2) for n in range(F)])
    def rows(v):
        a, d = v[..., : M // 2], v[..., M // 2:]
        contrib = a[..., :, None] * hh + d[..., :, None] * gg  # (..., M/2, F)
        contrib = contrib.reshape(*contrib.shape[:-2], -1)
        out = torch.zeros(*v.shape[:-1], M, dtype=DT)
        return out.index_add(-1, tgt, contrib)
    y = rows(z.transpose(-1, -2)).transpose(-1, -2)
    return rows(y)


def dwt(x, h, J):
    N = x.shape[-1]
    z = x
    for j in range(1, J + 1):
        M = N >> (j - 1)
        blk = _level_analysis(z[..., :M, :M], h)
        z = torch.cat([torch.cat([blk, z[..., :M, M:]], -1), z[..., M:, :]], -2)
    return z


def idwt(z, h, J):
    N = z.shape[-1]
    x = z
    for j in range(J, 0, -1):
        M = N >> (j - 1)
        blk = _level_synthesis(x[..., :M, :M], h)
        x = torch.cat([torch.cat([blk, x[..., :M, M:]], -1), x[..., M:, :]], -2)
    return x


def dct_matrix(L):
    k = np.arange(L)[:, None]
    l = np.arange(L)[None, :]
    C = np.where(k == 0, np.sqrt(1.0 / L), np.sqrt(2.0 / L)) * np.cos(np.pi * (2 * l + 1) * k / (2 * L))
    return torch.tensor(C, dtype=DT)


def soft(t, tau):
    return torch.sign(t) * torch.relu(t.abs() - tau)


def unrolled(psf, y, mu_s, mu_nu, rho, K, mu_eps=0.001, J=3, mask=0x1FF):
    """X after K iterations of Algorithm 1 from the zero state (all tensors FP64;
    psf is a constant, y, mu_s, mu_nu, rho may require grad)."""
    bases = [h for _, h in daubechies.dictionary(mask)]
    ns = len(bases)
    L, N = y.shape[0], y.shape[-1]
    h0 = torch.fft.ifftshift(torch.as_tensor(psf, dtype=DT), dim=(-2, -1))
    hh = torch.fft.fft2(h0)
    yhat = torch.fft.fft2(y)
    HtY = torch.fft.ifft2(torch.conj(hh) * yhat).real
    rho_bar = mu_eps + 2 * rho + ns * rho
    C = dct_matrix(L)
    dctb = lambda a: torch.einsum("kl,lij->kij", C, a)
    idctb = lambda a: torch.einsum("kl,kij->lij", C, a)
    zero = torch.zeros(L, N, N, dtype=DT)
    P, V, S, GP, GV, GS = zero, zero, zero, zero, zero, zero
    T = [zero] * ns
    GT = [zero] * ns
    X = zero
    for _ in range(K):
        b = HtY + GP + rho * P + GS + rho * S
        for k, h in enumerate(bases):
            b = b + idwt(GT[k] + rho * T[k], h, J)
        X = torch.fft.ifft2(torch.fft.fft2(b) / (hh.abs() ** 2 + rho_bar)).real
        P = torch.relu(X - GP / rho)
        Z = [dwt(X, h, J) for h in bases]
        T = [soft(Z[k] - GT[k] / rho, mu_s / rho) for k in range(ns)]
        V = soft(dctb(S) - GV / rho, mu_nu / rho)
        S = (idctb(GV + rho * V) - GS + rho * X) / (2 * rho)
        GP = GP + rho * (P - X)
        GT = [GT[k] + rho * (T[k] - Z[k]) for k in range(ns)]
        GV = GV + rho * (V - dctb(S))
        GS = GS + rho * (S - X)
    return X


def loss_and_grads(psf, y, x_true, mu_s, mu_nu, rho, K, **kw):
    """(loss, dL/dy, dL/dmu_s, dL/dmu_nu, dL/drho) for L = ||X_K - x_true||^2."""
    yt = torch.tensor(np.asarray(y), dtype=DT, requires_grad=True)
    ms = torch.tensor(float(mu_s), dtype=DT, requires_grad=True)
    mn = torch.tensor(float(mu_nu), dtype=DT, requires_grad=True)
    rh = torch.tensor(float(rho), dtype=DT, requires_grad=True)
    X = unrolled(psf, yt, ms, mn, rh, K, **kw)
    loss = ((X - torch.as_tensor(x_true, dtype=DT)) ** 2).sum()
    loss.backward()
    return (loss.item(), yt.grad.numpy(), ms.grad.item(), mn.grad.item(), rh.grad.item(), X.detach().numpy())
