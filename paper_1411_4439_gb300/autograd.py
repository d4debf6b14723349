"""Differentiable solve x = (M^dag M)^-1 b on the full lattice.

M(mu) = 2m + D(mu) with the chemical potential on the temporal hops. The
backward pass does one adjoint solve and forms the link force in the CUDA
library:

  lambda = (M^dag M)^-1 g          (g = dL/dRe x + i dL/dIm x, A Hermitian)
  y = M x,  z = M lambda
  dL/db  = lambda
  dL/dU  = -[F_1(y, lambda) + F_1(z, x)]      (hop 1)
  dL/dN  = -[F_3(y, lambda) + F_3(z, x)]      (hop 3)
  dL/dm  = -2 Re sum_k (<y_k, lambda_k> + <z_k, x_k>)
  dL/dmu = -Re sum_k (<y_k, M' lambda_k> + <z_k, M' x_k>),   M' = dM/dmu

with F_h(a, b)[mu][x] = f a(x) b(x+h mu)^dag - b(x) a(x+h mu)^dag / f
(f = e^{h mu} on temporal links). These follow from
dL = -Re[y^dag dM lambda + z^dag dM x]. Gradients use PyTorch's convention
for complex tensors (d/dRe + i d/dIm). Everything runs in FP64 on the GPU.
"""
from __future__ import annotations

import torch

from . import hisq as H


def _split(t):
    return [t[k] for k in range(t.shape[0])]


class HisqSolve(torch.autograd.Function):
    """x = (M(mu)^dag M(mu))^-1 b for a bundle b of shape (n, 2 V_h, 3), complex128.

    U, N: canonical complex128 links (4, Lt, Lz, Ly, Lx, 3, 3) on the GPU;
    mass, mu: 0-d float64 tensors. Vectors are parity-blocked (even sites first).
    """

    @staticmethod
    def forward(ctx, U, N, mass, mu, b, tol=1e-12):
        L = (U.shape[4], U.shape[3], U.shape[2], U.shape[1])
        g = H.hisq_gauge_load(L, U.detach().contiguous(), N.detach().contiguous(), prec=H.HISQ_F64)
        m, muf = float(mass), float(mu)
        bb = b.detach().contiguous()
        x = torch.zeros_like(bb)
        p = H.cg_params(inner_prec=H.HISQ_F64, even_odd=0)
        H.hisq_cg_solve(g, m, muf, _split(bb), _split(x), tol, p)
        ctx.gauge = g
        ctx.scalars = (m, muf, tol)
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        g = ctx.gauge
        m, muf, tol = ctx.scalars
        gx = gx.contiguous()
        lam = torch.zeros_like(gx)
        p = H.cg_params(inner_prec=H.HISQ_F64, even_odd=0)
        H.hisq_cg_solve(g, m, muf, _split(gx), _split(lam), tol, p)
        y = torch.empty_like(x)
        z = torch.empty_like(x)
        H.hisq_apply_m(g, m, muf, H.HISQ_OP_M, _split(x), _split(y), H.HISQ_F64)
        H.hisq_apply_m(g, m, muf, H.HISQ_OP_M, _split(lam), _split(z), H.HISQ_F64)
        grad_U = grad_N = grad_m = grad_mu = None
        Ls = g.L
        shape = (4, Ls[3], Ls[2], Ls[1], Ls[0], 3, 3)
        if ctx.needs_input_grad[0]:
            grad_U = torch.zeros(shape, dtype=torch.complex128, device=x.device)
            H.hisq_link_force(g, muf, 1, _split(y), _split(lam), -1.0, grad_U)
            H.hisq_link_force(g, muf, 1, _split(z), _split(x), -1.0, grad_U)
        if ctx.needs_input_grad[1]:
            grad_N = torch.zeros(shape, dtype=torch.complex128, device=x.device)
            H.hisq_link_force(g, muf, 3, _split(y), _split(lam), -1.0, grad_N)
            H.hisq_link_force(g, muf, 3, _split(z), _split(x), -1.0, grad_N)
        if ctx.needs_input_grad[2]:
            s = H.hisq_cdot(g, _split(y), _split(lam)) + H.hisq_cdot(g, _split(z), _split(x))
            grad_m = torch.tensor(-2.0 * float(s.real.sum()), dtype=torch.float64)
        if ctx.needs_input_grad[3]:
            dl = torch.empty_like(x)
            dx = torch.empty_like(x)
            H.hisq_apply_m(g, m, muf, H.HISQ_OP_DM_DMU, _split(lam), _split(dl), H.HISQ_F64)
            H.hisq_apply_m(g, m, muf, H.HISQ_OP_DM_DMU, _split(x), _split(dx), H.HISQ_F64)
            s = H.hisq_cdot(g, _split(y), _split(dl)) + H.hisq_cdot(g, _split(z), _split(dx))
            grad_mu = torch.tensor(-float(s.real.sum()), dtype=torch.float64)
        H.hisq_gauge_free(g)
        ctx.gauge = None
        return grad_U, grad_N, grad_m, grad_mu, lam, None


def hisq_solve(U, N, mass, mu, b, tol=1e-12):
    """Differentiable x = (M^dag M)^-1 b (see HisqSolve)."""
    mass = mass if torch.is_tensor(mass) else torch.tensor(float(mass), dtype=torch.float64)
    mu = mu if torch.is_tensor(mu) else torch.tensor(float(mu), dtype=torch.float64)
    return HisqSolve.apply(U, N, mass, mu, b, tol)
