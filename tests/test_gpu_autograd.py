"""Differentiable solve: GPU gradients against the FP64 oracle.

Loss L = sum_k Re c_k^dag x_k with x = (M^dag M)^-1 b on the full lattice.
Gradients with respect to link entries, the mass, mu and b are compared with
central finite differences of the oracle's L (h = 1e-6), and the mu and mass
derivatives with the trace forms -2 Re <M x, M' x> and -4 Re <x, M x>
(for c = b) that the stochastic estimators of Eq. 2 use.
"""
import numpy as np
import pytest

import hisq_inputs as gen
from oracle import hisq_oracle as O

pytestmark = pytest.mark.gpu


def blocked(v_full, L):
    return np.concatenate([O.to_half(v_full, L, 0), O.to_half(v_full, L, 1)], axis=1)


def unblocked(v_blk, L):
    vh = v_blk.shape[1] // 2
    return O.to_full(v_blk[:, :vh], L, 0) + O.to_full(v_blk[:, vh:], L, 1)


def oracle_loss(U, N, m, mu, b_full, c_full):
    x, _ = O.cg(lambda q: O.apply_MdagM(U, N, q, m, mu), b_full, tol=1e-14)
    return float(np.sum(np.conj(c_full) * x).real)


def gpu_grads(gpu_lib, U, N, m, mu, b_full, c_full, L):
    import torch
    from paper_1411_4439_gb300.autograd import hisq_solve
    dU = torch.from_numpy(U).cuda().requires_grad_(True)
    dN = torch.from_numpy(N).cuda().requires_grad_(True)
    tm = torch.tensor(m, dtype=torch.float64, requires_grad=True)
    tmu = torch.tensor(mu, dtype=torch.float64, requires_grad=True)
    tb = torch.from_numpy(blocked(b_full, L)).cuda().requires_grad_(True)
    tc = torch.from_numpy(blocked(c_full, L)).cuda()
    x = hisq_solve(dU, dN, tm, tmu, tb, tol=1e-13)
    loss = (torch.conj(tc) * x).real.sum()
    loss.backward()
    return (dU.grad.cpu().numpy(), dN.grad.cpu().numpy(), float(tm.grad), float(tmu.grad),
            unblocked(tb.grad.cpu().numpy(), L), float(loss), unblocked(x.detach().cpu().numpy(), L))


def test_gradients_match_oracle_finite_differences(gpu_lib):
    L, m, mu = (4, 4, 4, 6), 0.1, 0.1
    U, N = gen.hisq_links(L, seed=91)
    rng = np.random.default_rng(92)
    shape = (2,) + O.grid_shape(L) + (3,)
    b = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)
    c = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)
    gU, gN, gm, gmu, gb, loss, x = gpu_grads(gpu_lib, U, N, m, mu, b, c, L)
    L0 = oracle_loss(U, N, m, mu, b, c)
    assert abs(loss - L0) <= 1e-10 * abs(L0)
    h = 1e-6

    def fd(fn):
        return (fn(+h) - fn(-h)) / (2 * h)

    scale_U = np.abs(gU).max()
    scale_N = np.abs(gN).max()
    for trial in range(4):
        idx = tuple(int(rng.integers(0, s)) for s in U.shape)
        for field, grad, scale in (("U", gU, scale_U), ("N", gN, scale_N)):
            def perturb(d, unit):
                U2, N2 = U.copy(), N.copy()
                (U2 if field == "U" else N2)[idx] += unit * d
                return oracle_loss(U2, N2, m, mu, b, c)
            g_re = fd(lambda d: perturb(d, 1.0))
            g_im = fd(lambda d: perturb(d, 1j))
            assert abs(grad[idx] - (g_re + 1j * g_im)) <= 2e-4 * scale, (field, idx)
    g_m = fd(lambda d: oracle_loss(U, N, m + d, mu, b, c))
    g_mu = fd(lambda d: oracle_loss(U, N, m, mu + d, b, c))
    assert abs(gm - g_m) <= 1e-5 * max(1.0, abs(g_m))
    assert abs(gmu - g_mu) <= 1e-5 * max(1.0, abs(g_mu))
    # dL/db = (M^dag M)^-1 c (the operator is Hermitian)
    lam, _ = O.cg(lambda q: O.apply_MdagM(U, N, q, m, mu), c, tol=1e-14)
    assert np.linalg.norm(gb - lam) <= 1e-9 * np.linalg.norm(lam)


@pytest.mark.parametrize("L,n,m,mu", [((4, 6, 8, 10), 2, 0.05, 0.1), ((16, 16, 16, 16), 4, 0.05, 0.1)])
def test_trace_forms_of_mass_and_mu_derivatives(gpu_lib, L, n, m, mu):
    """With c = b = eta: dL/dmu = -2 Re <M x, M' x>, dL/dm = -4 Re <x, M x>."""
    eta = O.to_full(gen.z2_source(L, n, seed=93), L, 0) + O.to_full(gen.z2_source(L, n, seed=94), L, 1)
    U, N = gen.hisq_links(L, seed=95)
    gU, gN, gm, gmu, gb, loss, x = gpu_grads(gpu_lib, U, N, m, mu, eta, eta, L)
    res = O.true_relative_residual(lambda q: O.apply_MdagM(U, N, q, m, mu), x, eta)
    assert np.all(res <= 1e-10)
    Mx = O.apply_M(U, N, x, m, mu)
    trace_mu = -2.0 * float(np.vdot(Mx, O.apply_dM_dmu(U, N, x, mu)).real)
    trace_m = -4.0 * float(np.vdot(x, Mx).real)
    assert abs(gmu - trace_mu) <= 1e-8 * abs(trace_mu)
    assert abs(gm - trace_m) <= 1e-8 * abs(trace_m)
