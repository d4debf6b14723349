"""Stochastic trace estimates of Eq. 2 on the GPU.

The mu-derivatives of ln Z (Eq. 1) reduce to traces of words such as
Tr(M' M^-1), Tr(M'' M^-1), Tr(M' M^-1 M' M^-1), with M^(k) = d^k M / dmu^k.
Each trace is estimated by noise vectors eta with E[eta eta^dag] = 1:

    Tr(W) ~ (1/N) sum_k eta_k^dag W eta_k .

``trace_word_bilinears`` returns the per-vector bilinears for one bundle of
noise vectors; averaging them over bundles gives the estimate. Every step is
a C-ABI call: M^-1 v = (M^dag M)^-1 M^dag v by hisq_cg_solve on the full
lattice, the derivative operators by hisq_apply_m, the dot products by
hisq_cdot.
"""
from __future__ import annotations

import numpy as np
import torch

from . import hisq as H


def _split(t):
    return [t[k] for k in range(t.shape[0])]


def apply_minv(g, mass: float, mu: float, v: torch.Tensor, tol: float = 1e-12,
               inner_prec: int = H.HISQ_F64, stream=None) -> torch.Tensor:
    """M(mu)^-1 v for parity-blocked complex128 vectors (n, 2 V_h, 3)."""
    mdv = torch.empty_like(v)
    H.hisq_apply_m(g, mass, mu, H.HISQ_OP_MDAG, _split(v), _split(mdv), H.HISQ_F64, stream)
    x = torch.zeros_like(v)
    p = H.cg_params(inner_prec=inner_prec, even_odd=0)
    H.hisq_cg_solve(g, mass, mu, _split(mdv), _split(x), tol, p, stream)
    return x


def trace_word_bilinears(g, mass: float, mu: float, eta: torch.Tensor, orders, tol: float = 1e-12,
                         inner_prec: int = H.HISQ_F64, stream=None) -> np.ndarray:
    """eta_k^dag (M^(n1) M^-1)(M^(n2) M^-1)...(M^(nj) M^-1) eta_k for each vector k.

    eta: complex128 CUDA tensor (n, 2 V_h, 3), parity-blocked; orders =
    (n1, ..., nj) with 1 <= n_i <= 4. The handle g must hold FP64 links for
    inner_prec = HISQ_F64 (or links of inner_prec for a mixed solve).
    """
    v = eta.contiguous()
    for order in reversed(list(orders)):
        if not 1 <= int(order) <= 4:
            raise ValueError("derivative orders must be 1..4")
        x = apply_minv(g, mass, mu, v, tol, inner_prec, stream)
        w = torch.empty_like(x)
        H.hisq_apply_m(g, mass, mu, H.HISQ_OP_DM_DMU + int(order) - 1, _split(x), _split(w),
                       H.HISQ_F64, stream)
        v = w
    return H.hisq_cdot(g, _split(eta.contiguous()), _split(v), stream)


def estimate_trace(g, mass: float, mu: float, eta_bundles, orders, tol: float = 1e-12,
                   inner_prec: int = H.HISQ_F64):
    """Mean and standard error of Tr(word) over all noise vectors of the bundles."""
    vals = np.concatenate([trace_word_bilinears(g, mass, mu, e, orders, tol, inner_prec)
                           for e in eta_bundles])
    n = vals.size
    err = vals.std(ddof=1) / np.sqrt(n) if n > 1 else float("nan")
    return complex(vals.mean()), float(err)
