"""Stochastic trace bilinears of Eq. 2 on the GPU against the FP64 oracle."""
import numpy as np
import pytest

import hisq_inputs as gen
from oracle import hisq_oracle as O

pytestmark = pytest.mark.gpu


def blocked(v_full, L):
    return np.concatenate([O.to_half(v_full, L, 0), O.to_half(v_full, L, 1)], axis=1)


@pytest.mark.parametrize("orders", [(1,), (2,), (1, 1), (3,), (4,), (2, 1)])
@pytest.mark.parametrize("mu", [0.0, 0.1])
def test_trace_word_bilinears_match_oracle(gpu_lib, orders, mu):
    import torch
    from paper_1411_4439_gb300.trace import trace_word_bilinears
    H = gpu_lib
    L, m = (4, 4, 4, 6), 0.1
    U, N = gen.hisq_links(L, seed=101)
    eta = O.to_full(gen.z2_source(L, 3, seed=102), L, 0) + O.to_full(gen.z2_source(L, 3, seed=103), L, 1)
    g = H.hisq_gauge_load(L, torch.from_numpy(U).cuda(), torch.from_numpy(N).cuda(), prec=H.HISQ_F64)
    try:
        got = trace_word_bilinears(g, m, mu, torch.from_numpy(blocked(eta, L)).cuda(), orders, tol=1e-13)
    finally:
        H.hisq_gauge_free(g)
    ref = O.trace_word_bilinear(U, N, eta, m, mu, orders, tol=1e-14)
    assert np.allclose(got, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())


def test_apply_m_derivatives_match_oracle(gpu_lib):
    import torch
    H = gpu_lib
    L, mu = (4, 6, 8, 10), 0.2
    U, N = gen.hisq_links(L, seed=104)
    v = O.to_full(gen.gaussian_source(L, 2, seed=105), L, 0) + O.to_full(gen.gaussian_source(L, 2, seed=106), L, 1)
    vb = torch.from_numpy(blocked(v, L)).cuda()
    for prec, tol in ((H.HISQ_F64, 1e-13), (H.HISQ_F32, 1e-6)):
        g = H.hisq_gauge_load(L, torch.from_numpy(U).cuda(), torch.from_numpy(N).cuda(), prec=prec,
                              recon_U=18, recon_N=18)
        try:
            src = vb if prec == H.HISQ_F64 else vb.to(torch.complex64)
            for op, ref in ((H.HISQ_OP_M, O.apply_M(U, N, v, 0.07, mu)),
                            (H.HISQ_OP_MDAG, O.apply_Mdag(U, N, v, 0.07, mu)),
                            (H.HISQ_OP_DM_DMU, O.apply_dnM_dmun(U, N, v, mu, 1)),
                            (H.HISQ_OP_D2M_DMU2, O.apply_dnM_dmun(U, N, v, mu, 2)),
                            (H.HISQ_OP_D3M_DMU3, O.apply_dnM_dmun(U, N, v, mu, 3)),
                            (H.HISQ_OP_D4M_DMU4, O.apply_dnM_dmun(U, N, v, mu, 4))):
                w = torch.empty_like(src)
                H.hisq_apply_m(g, 0.07, mu, op, [src[0], src[1]], [w[0], w[1]], prec)
                torch.cuda.synchronize()
                got = w.cpu().numpy().astype(np.complex128)
                exp = blocked(ref, L)
                assert np.linalg.norm(got - exp) <= tol * np.linalg.norm(exp), (prec, op)
        finally:
            H.hisq_gauge_free(g)
