"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test ties the oracle to something other than itself: the numbers printed
in Table 1, the closed-form spectrum of the free field, anti-hermiticity of
Eq. 3, gauge covariance, a dense library solve, and exact reconstruction of
unitary links. None of them needs a GPU.
"""
import numpy as np
import pytest

import hisq_inputs as gen
from oracle import hisq_oracle as O
from conftest import read_golden

LATTICES = [(8, 8, 8, 8), (4, 6, 8, 10)]


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def gaussian_full(L, n, seed):
    rng = np.random.default_rng(seed)
    shape = (n,) + O.grid_shape(L) + (3,)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)


def coords(L):
    Lt, Lz, Ly, Lx = O.grid_shape(L)
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly),
                             np.arange(Lx), indexing="ij")
    return x, y, z, t


def plane_wave(L, k, chi):
    """e^{i p.x} chi with p_mu = 2 pi k_mu / L_mu (mu < 3), p_t = (2 k_t + 1) pi / Lt."""
    x, y, z, t = coords(L)
    p = [2 * np.pi * k[0] / L[0], 2 * np.pi * k[1] / L[1], 2 * np.pi * k[2] / L[2],
         (2 * k[3] + 1) * np.pi / L[3]]
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return ph[None, ..., None] * np.asarray(chi)[None, None, None, None, None, :], p


def free_s(p, c1, c3, mu_chem=0.0):
    s = [2 * c1 * np.sin(q) + 2 * c3 * np.sin(3 * q) for q in p[:3]]
    q = p[3] - 1j * mu_chem
    s.append(2 * c1 * np.sin(q) + 2 * c3 * np.sin(3 * q))
    return s


# ---------------------------------------------------------------------------
# Table 1 and the intensity statements of Sec. 1 / Sec. 3 (golden fixtures)
# ---------------------------------------------------------------------------

def test_table1_arithmetic_intensity():
    rows = read_golden("table1_arithmetic_intensity.txt")
    assert len(rows) == 7
    for n, full, r14 in rows:
        n = int(n)
        assert round(O.dslash_intensity(n, 18), 2) == pytest.approx(float(full), abs=1e-9)
        assert round(O.dslash_intensity(n, 14), 2) == pytest.approx(float(r14), abs=1e-9)


def test_intensity_statements():
    g = {r[0]: [float(v) for v in r[1:]] for r in read_golden("intensity_statements.txt")}
    limit = O.dslash_flops(1) / ((16 * 6 + 6) * 4)
    assert abs(limit - g["limit"][0]) <= g["limit"][1]
    assert abs(O.dslash_intensity(8, 18) / limit - g["frac_n8"][0]) <= g["frac_n8"][1]
    for f in (18, 14):
        frac1 = O.dslash_intensity(1, f) / limit
        assert g["frac_n1_lo"][0] <= frac1 <= g["frac_n1_hi"][0]
    ratio = O.dslash_intensity(4, 14) / O.dslash_intensity(1, 14)
    assert abs(ratio - g["ratio_r14_4_over_1"][0]) <= g["ratio_r14_4_over_1"][1]


def test_flop_count_by_operation_census():
    # one complex multiply = 4 mul + 2 add, one complex add = 2 add
    assert O.MATVEC_FLOPS == 9 * (4 + 2) + 6 * 2
    assert O.dslash_flops(1) == 1146


# ---------------------------------------------------------------------------
# Geometry: the half-lattice index h = i // 2 within one parity
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L", LATTICES)
def test_half_index_is_lex_over_two(L):
    x, y, z, t = coords(L)
    lex = x + L[0] * (y + L[1] * (z + L[2] * t))
    for p in (0, 1):
        field = lex.astype(np.complex128)[None, ..., None] * np.ones(3)
        half = O.to_half(field, L, p)
        vh = lex.size // 2
        assert half.shape == (1, vh, 3)
        h_of = (half[0, :, 0].real.astype(np.int64)) // 2
        np.testing.assert_array_equal(h_of, np.arange(vh))
        par = (x + y + z + t) % 2
        sel = lex[par == p]
        np.testing.assert_array_equal(np.sort(sel), half[0, :, 0].real.astype(np.int64))
        back = O.to_full(half, L, p)
        np.testing.assert_array_equal(back[0][par == p], field[0][par == p])
        assert np.all(back[0][par != p] == 0)


# ---------------------------------------------------------------------------
# P1: free field. -D^2 acts on plane waves as sum_mu s_mu(p)^2.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L", LATTICES)
@pytest.mark.parametrize("mu_chem", [0.0, 0.3])
def test_free_field_plane_wave_spectrum(L, mu_chem):
    c1, c3 = 9.0 / 8.0, -1.0 / 24.0
    U, N = gen.free_field_links(L, c1, c3)
    rng = np.random.default_rng(5)
    for trial in range(4):
        k = [int(rng.integers(0, L[m])) for m in range(4)]
        chi = rng.standard_normal(3) + 1j * rng.standard_normal(3)
        v, p = plane_wave(L, k, chi)
        lam = sum(s * s for s in free_s(p, c1, c3, mu_chem))
        Dv = O.dslash(U, N, v, mu_chem)
        DDv = O.dslash(U, N, Dv, mu_chem)
        assert rel(-DDv, lam * v) < 1e-12


@pytest.mark.parametrize("L", LATTICES)
def test_free_field_even_odd_eigenvector_and_one_step_cg(L):
    c1, c3, m = 9.0 / 8.0, -1.0 / 24.0, 0.05
    U, N = gen.free_field_links(L, c1, c3)
    k = [1, 2, 0, 1]
    v, p = plane_wave(L, k, [1.0, 0.5j, -0.25])
    lam = 4 * m * m + sum(s * s for s in free_s(p, c1, c3)).real
    ve = O.to_half(v, L, 0)
    Av = O.apply_Ae(U, N, ve, L, m)
    assert rel(Av, lam * ve) < 1e-12
    x, iters = O.cg(lambda q: O.apply_Ae(U, N, q, L, m), ve, tol=1e-12)
    assert iters[0] == 1
    assert rel(x, ve / lam) < 1e-12


# ---------------------------------------------------------------------------
# P2: anti-hermiticity <w, D v> = -<D w, v>; D(mu)^dag = -D(-mu)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L", LATTICES)
@pytest.mark.parametrize("mu_chem", [0.0, 0.2])
def test_anti_hermiticity(L, mu_chem):
    U, N = gen.hisq_links(L, seed=11)
    v = gaussian_full(L, 2, 1)
    w = gaussian_full(L, 2, 2)
    lhs = np.vdot(w, O.dslash(U, N, v, mu_chem))
    rhs = -np.vdot(O.dslash(U, N, w, -mu_chem), v)
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(w) * np.linalg.norm(v) * 10


@pytest.mark.parametrize("L", LATTICES)
def test_parity_blocks_adjoint(L):
    U, N = gen.hisq_links(L, seed=12)
    a_e = gen.gaussian_source(L, 2, 3)
    b_o = gen.gaussian_source(L, 2, 4)
    lhs = np.vdot(a_e, O.dslash_parity(U, N, b_o, L, 0))      # <a_e, D_eo b_o>
    rhs = -np.vdot(O.dslash_parity(U, N, a_e, L, 1), b_o)     # -<D_oe a_e, b_o>
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(a_e) * np.linalg.norm(b_o)


def test_dslash_is_parity_off_diagonal():
    L = (4, 6, 8, 10)
    U, N = gen.hisq_links(L, seed=13)
    v = gaussian_full(L, 1, 5)
    ve = O.to_full(O.to_half(v, L, 0), L, 0)
    Dve = O.dslash(U, N, ve)
    assert np.all(Dve[:, O.parity_mask(L, 0)] == 0)


# ---------------------------------------------------------------------------
# P3: gauge covariance U -> g U g'^dag, N -> g N g'''^dag, v -> g v
# ---------------------------------------------------------------------------

def gauge_transform(L, U, N, g):
    gd = np.conj(np.swapaxes(g, -1, -2))
    U2 = np.empty_like(U)
    N2 = np.empty_like(N)
    for mu in range(4):
        U2[mu] = g @ U[mu] @ O.shift(gd, mu, +1, 0)
        N2[mu] = g @ N[mu] @ O.shift(gd, mu, +3, 0)
    return U2, N2


@pytest.mark.parametrize("L", LATTICES)
@pytest.mark.parametrize("mu_chem", [0.0, 0.25])
def test_gauge_covariance(L, mu_chem):
    U, N = gen.hisq_links(L, seed=21)
    g = gen.random_su3_field(L, seed=22)
    U2, N2 = gauge_transform(L, U, N, g)
    v = gaussian_full(L, 2, 7)
    gv = np.einsum("tzyxij,ntzyxj->ntzyxi", g, v)
    lhs = O.dslash(U2, N2, gv, mu_chem)
    rhs = np.einsum("tzyxij,ntzyxj->ntzyxi", g, O.dslash(U, N, v, mu_chem))
    assert rel(lhs, rhs) < 1e-13


def test_gauge_covariance_of_cg_solution():
    L, m = (4, 4, 4, 6), 0.1
    U, N = gen.hisq_links(L, seed=23)
    g = gen.random_su3_field(L, seed=24)
    U2, N2 = gauge_transform(L, U, N, g)
    b = gen.z2_source(L, 1, 25)
    # g restricted to even sites, as a (V_h, 3, 3) stack
    mask = O.parity_mask(L, 0)
    g_e = g[mask]
    x, _ = O.cg(lambda q: O.apply_Ae(U, N, q, L, m), b, tol=1e-13)
    gb = np.einsum("hij,nhj->nhi", g_e, b)
    x2, _ = O.cg(lambda q: O.apply_Ae(U2, N2, q, L, m), gb, tol=1e-13)
    assert rel(x2, np.einsum("hij,nhj->nhi", g_e, x)) < 1e-10


# ---------------------------------------------------------------------------
# P4 / P6: dense library solve, hermiticity and positivity of the CG system
# ---------------------------------------------------------------------------

def test_dense_even_odd_system_matches_library_solve():
    L, m = (4, 4, 4, 4), 0.05
    U, N = gen.hisq_links(L, seed=31)
    vh = 128
    A = O.dense_matrix(lambda q: O.apply_Ae(U, N, q, L, m), (vh, 3))
    assert A.shape == (384, 384)
    assert np.abs(A - A.conj().T).max() < 1e-13
    ev = np.linalg.eigvalsh(A)
    assert ev.min() >= 4 * m * m * (1 - 1e-10)
    # A_e = 4m^2 + D_oe^dag D_oe with D_oe the odd<-even block of the dense D
    Doe = O.dense_matrix(lambda q: O.dslash_parity(U, N, q, L, 1), (vh, 3))
    assert np.abs(A - (4 * m * m * np.eye(384) + Doe.conj().T @ Doe)).max() < 1e-12
    b = gen.z2_source(L, 2, 32)
    x_lu = np.linalg.solve(A, b.reshape(2, -1).T).T.reshape(b.shape)
    x_cg, iters = O.cg(lambda q: O.apply_Ae(U, N, q, L, m), b, tol=1e-13)
    assert rel(x_cg, x_lu) < 1e-10
    assert np.all(O.true_relative_residual(lambda q: O.apply_Ae(U, N, q, L, m), x_cg, b) < 1e-12)


def test_light_mass_cg_solution_matches_refined_dense_solve():
    # At the mixed-precision configuration's mass the system is ill conditioned;
    # the oracle's CG (iterated residual 1e-13) must still give the solution
    # to far better than the 1e-8 the GPU solutions are held to. Reference: a
    # dense library solve refined once with a long-double residual.
    L, m = (4, 4, 4, 4), 0.0025
    U, N = gen.hisq_links(L, seed=71)
    vh = 128
    A = O.dense_matrix(lambda q: O.apply_Ae(U, N, q, L, m), (vh, 3))
    ev = np.linalg.eigvalsh(A)
    assert ev[-1] / ev[0] > 1e4                          # ill conditioned indeed
    b = gen.gaussian_source(L, 2, 72)
    B = b.reshape(2, -1).T
    X = np.linalg.solve(A, B)
    R = B.astype(np.clongdouble) - A.astype(np.clongdouble) @ X.astype(np.clongdouble)
    X = X + np.linalg.solve(A, R.astype(np.complex128))
    x_ref = X.T.reshape(b.shape)
    x_cg, _ = O.cg(lambda q: O.apply_Ae(U, N, q, L, m), b, tol=1e-13)
    for k in range(2):
        assert rel(x_cg[k], x_ref[k]) < 1e-9


def test_dense_full_lattice_normal_system_with_mu():
    L, m, mu = (4, 4, 4, 4), 0.1, 0.1
    U, N = gen.hisq_links(L, seed=33)
    shape = O.grid_shape(L) + (3,)
    M = O.dense_matrix(lambda q: O.apply_M(U, N, q, m, mu), shape)
    Md = O.dense_matrix(lambda q: O.apply_Mdag(U, N, q, m, mu), shape)
    assert np.abs(Md - M.conj().T).max() < 1e-13          # M^dag is the adjoint of M
    A = O.dense_matrix(lambda q: O.apply_MdagM(U, N, q, m, mu), shape)
    assert np.abs(A - M.conj().T @ M).max() < 1e-12
    rng = np.random.default_rng(34)
    b = rng.standard_normal((1,) + shape) + 1j * rng.standard_normal((1,) + shape)
    x_lu = np.linalg.solve(A, b.reshape(1, -1).T).T.reshape(b.shape)
    x_cg, _ = O.cg(lambda q: O.apply_MdagM(U, N, q, m, mu), b, tol=1e-13)
    assert rel(x_cg, x_lu) < 1e-9


def test_full_lattice_solve_equals_even_odd_at_zero_mu():
    L, m = (4, 4, 4, 6), 0.1
    U, N = gen.hisq_links(L, seed=35)
    b_e = gen.z2_source(L, 1, 36)
    x_e, _ = O.cg(lambda q: O.apply_Ae(U, N, q, L, m), b_e, tol=1e-13)
    b_full = O.to_full(b_e, L, 0)
    x_full, _ = O.cg(lambda q: O.apply_MdagM(U, N, q, m, 0.0), b_full, tol=1e-13)
    assert rel(O.to_half(x_full, L, 0), x_e) < 1e-10
    assert np.linalg.norm(O.to_half(x_full, L, 1)) < 1e-10 * np.linalg.norm(x_e)


@pytest.mark.parametrize("L", [(8, 8, 8, 8)])
def test_hermitian_positive_system_random_vectors(L):
    m = 0.05
    U, N = gen.hisq_links(L, seed=41)
    u = gen.gaussian_source(L, 1, 42)
    v = gen.gaussian_source(L, 1, 43)
    Au = O.apply_Ae(U, N, u, L, m)
    Av = O.apply_Ae(U, N, v, L, m)
    assert abs(np.vdot(u, Av) - np.conj(np.vdot(v, Au))) < 1e-12 * np.linalg.norm(u) * np.linalg.norm(v) * 10
    assert np.vdot(v, Av).real >= 4 * m * m * np.vdot(v, v).real


# ---------------------------------------------------------------------------
# CG behaviour per rhs
# ---------------------------------------------------------------------------

def test_cg_per_rhs_freezing_and_zero_source():
    L, m = (4, 4, 4, 4), 0.05
    U, N = gen.hisq_links(L, seed=51)
    b = gen.z2_source(L, 3, 52)
    b[1] = 0.0
    x, iters = O.cg(lambda q: O.apply_Ae(U, N, q, L, m), b, tol=1e-11)
    assert iters[1] == 0 and np.all(x[1] == 0)
    # per-rhs solutions equal the single-rhs solves
    for k in (0, 2):
        xk, _ = O.cg(lambda q: O.apply_Ae(U, N, q, L, m), b[k:k + 1], tol=1e-11)
        assert rel(x[k], xk[0]) < 1e-14


# ---------------------------------------------------------------------------
# P7: link compression round trips and rejection
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L", LATTICES)
def test_r14_round_trip_on_naik_links(L):
    U, N = gen.hisq_links(L, seed=61)
    packed = O.compress_r14(N)
    assert packed.shape == N.shape[:-2] + (14,)
    back = O.reconstruct_r14(packed)
    assert np.abs(back - N).max() < 5e-14
    z = packed[..., 12] + 1j * packed[..., 13]
    assert np.allclose(np.abs(z), 24.0, rtol=1e-12)     # |z| = 1/|c| for N = c W, W in U(3)
    # r14 also holds for U(3)-type links after a gauge transform
    g = gen.random_su3_field(L, seed=62)
    _, N2 = gauge_transform(L, U, N, g)
    assert np.abs(O.reconstruct_r14(O.compress_r14(N2)) - N2).max() < 5e-14


@pytest.mark.parametrize("L", LATTICES)
def test_r12_round_trip_on_fat_links(L):
    U, N = gen.hisq_links(L, seed=63)
    back = O.reconstruct_r12(O.compress_r12(U), L, 0.9, hop=1)
    assert np.abs(back - U).max() < 5e-14
    # Naik links are U(3), not sign * SU(3): r12 must not reproduce them
    backN = O.reconstruct_r12(O.compress_r12(N), L, 1.0 / 24.0, hop=3)
    assert np.abs(backN - N).max() > 1e-3


def test_reconstruct_rejects_non_unitary():
    rng = np.random.default_rng(64)
    m = rng.standard_normal((10, 3, 3)) + 1j * rng.standard_normal((10, 3, 3))
    back = O.reconstruct_r14(O.compress_r14(m))
    assert np.abs(back - m).max() > 1e-2


def test_link_sign_matches_generator_phases():
    # sigma in the r12 reconstruction equals the sign folded into the links
    L = (4, 6, 8, 10)
    U, _ = gen.hisq_links(L, seed=65)
    det = np.linalg.det(U)
    sig = np.sign((det / 0.9 ** 3).real)
    assert np.array_equal(sig, O.link_sign(L, 1))


@pytest.mark.parametrize("mu_chem", [0.0, 0.15])
def test_site_evaluation_matches_array_form(mu_chem):
    L = (4, 6, 8, 10)
    U, N = gen.hisq_links(L, seed=71)
    v = gaussian_full(L, 3, 72)
    w = O.dslash(U, N, v, mu_chem)
    rng = np.random.default_rng(73)
    sites = [tuple(int(rng.integers(0, L[m])) for m in range(4)) for _ in range(25)]
    ws = O.dslash_at_sites(U, N, v, sites, mu_chem)
    for s, (x, y, z, t) in enumerate(sites):
        assert np.abs(ws[:, s] - w[:, t, z, y, x]).max() < 1e-13


@pytest.mark.parametrize("mu_chem", [0.0, 0.2])
def test_mu_derivative_is_finite_difference_of_dslash(mu_chem):
    L = (4, 4, 4, 6)
    U, N = gen.hisq_links(L, seed=81)
    v = gaussian_full(L, 2, 82)
    h = 1e-5
    fd = (O.dslash(U, N, v, mu_chem + h) - O.dslash(U, N, v, mu_chem - h)) / (2 * h)
    assert rel(O.apply_dM_dmu(U, N, v, mu_chem), fd) < 1e-9
    # and d(M^dag)/dmu is the adjoint of dM/dmu
    w = gaussian_full(L, 2, 83)
    fd_dag = (O.apply_Mdag(U, N, w, 0.1, mu_chem + h) - O.apply_Mdag(U, N, w, 0.1, mu_chem - h)) / (2 * h)
    assert abs(np.vdot(v, fd_dag) - np.vdot(O.apply_dM_dmu(U, N, v, mu_chem), w)) < 1e-8 * np.linalg.norm(v) * np.linalg.norm(w)


@pytest.mark.parametrize("order", [2, 3, 4])
def test_higher_mu_derivatives_are_finite_differences(order):
    L = (4, 4, 4, 6)
    U, N = gen.hisq_links(L, seed=84)
    v = gaussian_full(L, 1, 85)
    mu, h = 0.1, 1e-4
    fd = (O.apply_dnM_dmun(U, N, v, mu + h, order - 1) - O.apply_dnM_dmun(U, N, v, mu - h, order - 1)) / (2 * h)
    assert rel(O.apply_dnM_dmun(U, N, v, mu, order), fd) < 1e-6


def test_trace_word_matches_dense_trace():
    """With all unit vectors as noise the bilinear sum is the exact trace of the word."""
    L, m, mu = (4, 4, 4, 4), 0.2, 0.1
    U, N = gen.hisq_links(L, seed=86)
    shape = O.grid_shape(L) + (3,)
    dim = int(np.prod(shape))
    Md = O.dense_matrix(lambda q: O.apply_M(U, N, q, m, mu), shape)
    D1 = O.dense_matrix(lambda q: O.apply_dnM_dmun(U, N, q, mu, 1), shape)
    D2 = O.dense_matrix(lambda q: O.apply_dnM_dmun(U, N, q, mu, 2), shape)
    Mi = np.linalg.inv(Md)
    exact_1 = np.trace(D1 @ Mi)
    exact_11 = np.trace(D1 @ Mi @ D1 @ Mi)
    exact_2 = np.trace(D2 @ Mi)
    # a random subset of unit vectors gives the same partial sums as the dense matrices
    rng = np.random.default_rng(87)
    idx = rng.choice(dim, size=6, replace=False)
    eta = np.zeros((6, dim), dtype=complex)
    eta[np.arange(6), idx] = 1.0
    eta = eta.reshape((6,) + shape)
    for orders, W in (((1,), D1 @ Mi), ((1, 1), D1 @ Mi @ D1 @ Mi), ((2,), D2 @ Mi)):
        got = O.trace_word_bilinear(U, N, eta, m, mu, orders)
        assert np.allclose(got, W[idx, idx], rtol=1e-9, atol=1e-11)
    assert abs(exact_1) > 0 and abs(exact_11) > 0 and abs(exact_2) > 0


# ---------------------------------------------------------------------------
# The residual checker that decides every CG parity test: pinned to a residual
# fixed independently of it (a dense matrix product and numpy's own norm, and
# the closed-form eigenvalue of the free field)
# ---------------------------------------------------------------------------

def test_true_relative_residual_equals_dense_residual_of_a_perturbed_solution():
    L, m = (4, 4, 4, 4), 0.05
    U, N = gen.hisq_links(L, seed=61)
    vh = 128
    A = O.dense_matrix(lambda q: O.apply_Ae(U, N, q, L, m), (vh, 3))
    rng = np.random.default_rng(62)
    n = 3
    # rhs of very different norms, so that a norm taken over all rhs together
    # or a missing division by |b| shows
    b = gen.z2_source(L, n, 63) * np.array([1.0, 1e-3, 250.0])[:, None, None]
    x_lu = np.linalg.solve(A, b.reshape(n, -1).T).T
    delta = rng.standard_normal(x_lu.shape) + 1j * rng.standard_normal(x_lu.shape)
    delta *= np.array([1e-6, 1e-9, 1e-2])[:, None]      # residuals of about 1e-5 .. 1e-9
    x = (x_lu + delta).reshape(b.shape)
    want = np.array([np.linalg.norm(A @ delta[k]) / np.linalg.norm(b[k].ravel()) for k in range(n)])
    got = O.true_relative_residual(lambda q: O.apply_Ae(U, N, q, L, m), x, b)
    assert got.shape == (n,)
    # x_lu is exact to ~1e-15 relative, far below the planted residuals
    np.testing.assert_allclose(got, want, rtol=1e-6)
    # a squared norm (|r|^2/|b|^2) or |r|^2/|b| would be off by orders of magnitude
    assert np.all(got > 1e-10) and np.all(got < 1e-3)


@pytest.mark.parametrize("c", [0.0, 0.5, 1.5])
def test_true_relative_residual_of_a_free_field_eigenvector(c):
    # b an eigenvector of A_e with eigenvalue lam (closed form) and x = c b / lam:
    # b - A x = (1 - c) b, so the relative residual is |1 - c| exactly
    L, m = (8, 8, 8, 8), 0.05
    c1, c3 = 9.0 / 8.0, -1.0 / 24.0
    U, N = gen.free_field_links(L, c1, c3)
    v, p = plane_wave(L, [1, 2, 0, 1], [1.0, 0.5j, -0.25])
    lam = 4 * m * m + sum(s * s for s in free_s(p, c1, c3)).real
    b = np.concatenate([O.to_half(v, L, 0), 3.0 * O.to_half(v, L, 0)])
    x = np.concatenate([c * b[:1] / lam, np.zeros_like(b[1:])])
    got = O.true_relative_residual(lambda q: O.apply_Ae(U, N, q, L, m), x, b)
    np.testing.assert_allclose(got, [abs(1.0 - c), 1.0], rtol=0, atol=1e-12)


# ---------------------------------------------------------------------------
# The reading of "FP16 link storage": 16-bit fixed point per stored component,
# not IEEE half. A model of the mixed-precision solver (half spinors with a
# per-rhs scale, FP32 solution increment, FP64 reliable update every 50
# iterations or when the residual fell by 10x) on the light-mass system
# m = 0.0025 converges with fixed-point links and fails with IEEE-half links.
# ---------------------------------------------------------------------------

def _links_ieee_half(a):
    return a.real.astype(np.float16).astype(np.float64) + 1j * a.imag.astype(np.float16).astype(np.float64)


def _links_fixed16(a):
    # one scale per stored complex component (i, j) of the field: the largest
    # |Re| or |Im| of that component over the field maps to 32767
    out = np.empty_like(a)
    for i in range(3):
        for j in range(3):
            c = a[..., i, j]
            s = max(np.abs(c.real).max(), np.abs(c.imag).max()) / 32767.0
            out[..., i, j] = (np.rint(c.real / s) + 1j * np.rint(c.imag / s)) * s
    return out


def _half_store(v, scale):
    w = v * scale
    return (w.real.astype(np.float16).astype(np.float64) + 1j * w.imag.astype(np.float16).astype(np.float64)) / scale


def _mv(M, v):
    # dense matrix-vector product without a threaded BLAS (stays fast on busy hosts)
    return np.einsum("ij,j->i", M, v)


def _mixed_cg_model(Doe, Deo, A, b, m, tol=1e-10, maxiter=12000, every=50, delta=0.1):
    """(iterations, final true relative residual) of the storage model."""
    m2 = 4 * m * m
    x = np.zeros_like(b)
    bb = np.vdot(b, b).real
    s = 1.0 / np.abs(b).max()
    r = _half_store(b, s)
    p = r.copy()
    xl = np.zeros_like(b)
    rr = np.vdot(r, r).real
    rr_rel, since, res = rr, 0, 1.0
    for it in range(1, maxiter + 1):
        t = _half_store(_mv(Doe, p), s)
        Ap = _half_store(m2 * p - _mv(Deo, t), s)
        alpha = rr / np.vdot(p, Ap).real
        r = _half_store(r - alpha * Ap, s)
        xl = (xl + alpha * p).astype(np.complex64).astype(np.complex128)
        rr_new = np.vdot(r, r).real
        beta, rr = rr_new / rr, rr_new
        p = _half_store(r + beta * p, s)
        since += 1
        if since >= every or rr <= delta * delta * rr_rel:
            x, xl = x + xl, np.zeros_like(xl)
            rt = b - _mv(A, x)                  # FP64 true residual
            res = np.sqrt(np.vdot(rt, rt).real / bb)
            if res <= tol or not np.isfinite(res) or res > 1e2:
                return it, res
            s = 1.0 / np.abs(rt).max()
            r, p = _half_store(rt, s), _half_store(p, s)
            rr = rr_rel = np.vdot(r, r).real
            since = 0
    return maxiter, res


@pytest.mark.parametrize("seed", [1, 4])
def test_sixteen_bit_fixed_point_links_converge_where_ieee_half_links_fail(seed):
    L, m = (4, 4, 4, 4), 0.0025
    U, N = gen.hisq_links(L, seed=seed)
    vh = 128

    def blocks(Uq, Nq):
        Doe = O.dense_matrix(lambda q: O.dslash_parity(Uq, Nq, q, L, 1), (vh, 3))
        Deo = O.dense_matrix(lambda q: O.dslash_parity(Uq, Nq, q, L, 0), (vh, 3))
        return Doe, Deo

    Doe, Deo = blocks(U, N)
    A = 4 * m * m * np.eye(3 * vh) - Deo @ Doe
    b = gen.gaussian_source(L, 1, seed + 100)[0].ravel()
    it_ref, res_ref = _mixed_cg_model(Doe, Deo, A, b, m)
    assert res_ref <= 1e-10
    it_fx, res_fx = _mixed_cg_model(*blocks(_links_fixed16(U), _links_fixed16(N)), A, b, m)
    assert res_fx <= 1e-10 and it_fx <= 1.3 * it_ref
    _, res_half = _mixed_cg_model(*blocks(_links_ieee_half(U), _links_ieee_half(N)), A, b, m)
    assert not res_half <= 1e-10


def test_algorithmic_bytes_are_the_table_1_model_without_the_neighbour_rereads():
    """Sec. 1 (Table 1) counts 16 neighbour reads and one write per rhs; read
    once from DRAM, the input costs one read, so the minimum is that model
    minus 15 re-reads of 6 reals per rhs. Hand values: FP32 18/14 at n = 8 is
    8 * 32 * 4 + 12 * 8 * 4 = 1408 B, FP16 (16-bit links) 704 B."""
    for n in (1, 2, 4, 8, 16):
        for f_n in (18, 14):
            assert (O.dslash_bytes_algorithmic(n, 18, f_n, 4, 4)
                    == O.dslash_bytes_no_reuse(n, f_n, 18, 4) - n * 15 * 6 * 4)
    assert O.dslash_bytes_algorithmic(8, 18, 14, 4, 4) == 1408
    assert O.dslash_bytes_algorithmic(8, 18, 14, 2, 2) == 704
