"""torch.autograd.Function over the unrolled ADMM (differentiable form).

X_K = unrolled(plan, y, mu_s, mu_nu, rho, n_iter): the X of the last step I
after n_iter iterations of Algorithm 1 from the zero state, with the four
penalties tied to rho.  Gradients with respect to y, mu_s, mu_nu and rho come
from the library's reverse pass (mf_admm_backward), which re-runs the forward
with per-iteration checkpoints; PyTorch only carries the tensors.
"""

from __future__ import annotations

import torch

from . import Plan


class ADMMUnrolled(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, mu_s, mu_nu, rho, plan, n_iter, kw):
        r = float(rho)
        plan.iterate(y, n_iter, mu_s=float(mu_s), mu_nu=float(mu_nu), rho_P=r, rho_T=r, rho_V=r, rho_S=r, **kw)
        x = plan.x().clone()
        ctx.save_for_backward(y, mu_s, mu_nu, rho)
        ctx.plan, ctx.n_iter, ctx.kw = plan, n_iter, kw
        return x

    @staticmethod
    def backward(ctx, gx):
        y, mu_s, mu_nu, rho = ctx.saved_tensors
        dy, dms, dmn, dr = ctx.plan.backward(y, ctx.n_iter, gx.to(y.dtype), mu_s=float(mu_s), mu_nu=float(mu_nu),
                                             rho=float(rho), **ctx.kw)
        t = lambda v, ref: torch.tensor(v, dtype=ref.dtype, device=ref.device)
        return dy, t(dms, mu_s), t(dmn, mu_nu), t(dr, rho), None, None, None


def unrolled(plan: Plan, y, mu_s, mu_nu, rho, n_iter: int = 20, **kw):
    """Differentiable X_K (see the module docstring); mu_s, mu_nu, rho are 0-d tensors."""
    return ADMMUnrolled.apply(y, mu_s, mu_nu, rho, plan, n_iter, kw)
