"""The bundle spinor layout: packing, the bundle Dslash and the bundle CG.

The layout is checked byte for byte against its definition (include/hisq.h,
hisq_layout) written out here in numpy; the Dslash against the FP64 oracle
element by element (relative L2 per rhs: FP32 1e-6, FP16 3e-3); every built
thread mapping and kernel variant on ragged lattices (V_h not a multiple of
the 128-thread block); the configuration lattice 48^3x12 with FP16 storage
on sampled sites; and the CG on the bundle against the oracle.
"""
import numpy as np
import pytest

import hisq_inputs as gen
from oracle import hisq_oracle as O
from conftest import rel_l2

pytestmark = pytest.mark.gpu

TOL = {1: 1e-6, 2: 3e-3}
WIDTH = {1: 2, 2: 4}
_cache = {}


def links(L, seed=3):
    key = (L, seed)
    if key not in _cache:
        _cache[key] = gen.hisq_links(L, seed=seed)
    return _cache[key]


def load(H, L, prec, ru, rn, seed=3):
    import torch
    U, N = links(L, seed)
    return H.hisq_gauge_load(L, torch.from_numpy(U).cuda(), torch.from_numpy(N).cuda(),
                             prec=prec, recon_U=ru, recon_N=rn)


def rounded(v, prec):
    """The values the storage keeps: FP32 by one rounding; FP16 as the kernels
    convert, FP64 -> FP32 -> FP16 (both round to nearest even)."""
    re, im = v.real.astype(np.float32), v.imag.astype(np.float32)
    if prec == 2:
        re, im = re.astype(np.float16), im.astype(np.float16)
    return re, im


def bundle_reference(v, prec):
    """Bundle of v (n, V_h, 3) by the layout's definition: chunk (g, c, h)
    holds the W real parts of rhs gW .. gW+W-1, then their imaginary parts."""
    n, vh, _ = v.shape
    W = WIDTH[prec]
    re, im = rounded(v, prec)
    re = re.reshape(n // W, W, vh, 3).transpose(0, 3, 2, 1)   # (G, 3, V_h, W)
    im = im.reshape(n // W, W, vh, 3).transpose(0, 3, 2, 1)
    return np.ascontiguousarray(np.concatenate([re, im], axis=-1))


def pack(H, g, v, prec):
    import torch
    n = v.shape[0]
    src = [torch.from_numpy(np.ascontiguousarray(v[k])).cuda() for k in range(n)]
    dt = torch.float32 if prec == 1 else torch.float16
    b = torch.empty(H.hisq.bundle_bytes(g, n, prec) // (4 if prec == 1 else 2), dtype=dt, device="cuda")
    H.hisq_bundle_pack(g, src, prec, b)
    return b


def unpack(H, g, b, n, prec):
    import torch
    vh = int(np.prod(g.L)) // 2
    dst = [torch.empty(vh, 3, dtype=torch.complex128, device="cuda") for _ in range(n)]
    H.hisq_bundle_unpack(g, b, prec, dst)
    torch.cuda.synchronize()
    return np.stack([t.cpu().numpy() for t in dst])


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("n", [4, 8, 16])
def test_pack_follows_the_layout_definition_and_unpacks_exactly(gpu_lib, prec, n):
    H = gpu_lib
    L = (4, 6, 8, 10)
    g = load(H, L, prec, 18, 14)
    try:
        v = gen.gaussian_source(L, n, seed=200 + n) * 3.0
        b = pack(H, g, v, prec)
        ref = bundle_reference(v, prec)
        got = b.cpu().numpy().reshape(ref.shape)
        np.testing.assert_array_equal(got, ref)            # bit-exact
        back = unpack(H, g, b, n, prec)
        re, im = rounded(v, prec)
        np.testing.assert_array_equal(back, re.astype(np.float64) + 1j * im.astype(np.float64))
    finally:
        H.hisq_gauge_free(g)


def test_bundle_calls_reject_bad_shapes(gpu_lib):
    import torch
    H = gpu_lib
    L = (4, 6, 8, 10)
    g = load(H, L, 2, 18, 14)
    try:
        v = gen.gaussian_source(L, 6, seed=1)
        src = [torch.from_numpy(np.ascontiguousarray(v[k])).cuda() for k in range(6)]
        b = torch.empty(H.hisq.bundle_bytes(g, 6, 2) // 2, dtype=torch.float16, device="cuda")
        with pytest.raises(H.HisqError, match="multiple of 4"):
            H.hisq_bundle_pack(g, src, 2, b)              # FP16 chunks hold 4 rhs
        with pytest.raises(ValueError):
            H.hisq_bundle_pack(g, [s.to(torch.complex64) for s in src[:4]], 2, b)
    finally:
        H.hisq_gauge_free(g)


VARIANTS = [(1, 18, 18), (1, 18, 14), (1, 12, 14), (1, 14, 14),
            (2, 18, 18), (2, 18, 14), (2, 12, 14), (2, 14, 14)]


# (4, 6, 10, 8): Lz > Lt, so the kernels visit the (z, t) planes with z slow
@pytest.mark.parametrize("L", [(4, 6, 8, 10), (8, 8, 8, 8), (4, 6, 10, 8)])
@pytest.mark.parametrize("prec,ru,rn", VARIANTS)
def test_bundle_dslash_matches_oracle(gpu_lib, L, prec, ru, rn):
    import torch
    H = gpu_lib
    U, N = links(L)
    g = load(H, L, prec, ru, rn)
    try:
        for n in (4, 8, 16):
            v = gen.gaussian_source(L, n, seed=210 + n)
            b = pack(H, g, v, prec)
            for parity in (0, 1):
                w = torch.full_like(b, float("nan"))
                H.hisq_dslash_ex(g, 0.0, b, w, parity, prec, H.HISQ_BUNDLE, n=n)
                got = unpack(H, g, w, n, prec)
                ref = O.dslash_parity(U, N, v, L, parity)
                for k in range(n):
                    assert rel_l2(got[k], ref[k]) < TOL[prec], (n, parity, k)
    finally:
        H.hisq_gauge_free(g)


# every bundle mapping built for U r18 / N r14: (rhs per thread, min blocks, flags)
MAPPINGS = [(8, 3, 0), (4, 4, 0), (8, 3, 128), (8, 2, 0), (4, 3, 0), (4, 4, 128),
            (8, 1, 0), (8, 1, 8), (8, 2, 8), (4, 3, 8),
            (8, 2, 128), (8, 4, 128), (4, 3, 128), (8, 2, 136), (8, 3, 136), (4, 3, 136), (4, 4, 136),
            (8, 2, 4), (8, 3, 4), (8, 4, 4), (8, 2, 4 | 16), (8, 3, 4 | 16), (4, 4, 4),
            (8, 3, 4 | 128), (8, 4, 4 | 128), (8, 3, 4 | 128 | 16), (8, 4, 4 | 128 | 16), (4, 4, 4 | 128 | 16)]


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("rpt,minb,flags", MAPPINGS)
def test_every_bundle_mapping_matches_oracle(gpu_lib, prec, rpt, minb, flags):
    import torch
    H = gpu_lib
    L = (6, 4, 8, 10)
    U, N = links(L)
    g = load(H, L, prec, 18, 14)
    try:
        H.hisq_set_dslash_mapping(g, rpt, minb, flags)
        for n in (8, 16):
            if n % rpt or n // rpt > 4:
                continue
            v = gen.z2_source(L, n, seed=230 + n)
            b = pack(H, g, v, prec)
            w = torch.full_like(b, float("nan"))
            H.hisq_dslash_ex(g, 0.0, b, w, 1, prec, H.HISQ_BUNDLE, n=n)
            got = unpack(H, g, w, n, prec)
            ref = O.dslash_parity(U, N, v, L, 1)
            for k in range(n):
                assert rel_l2(got[k], ref[k]) < TOL[prec], (n, k)
    finally:
        H.hisq_gauge_free(g)


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("mu", [0.2, -0.3])
def test_bundle_dslash_chemical_potential(gpu_lib, prec, mu):
    import torch
    H = gpu_lib
    L = (4, 6, 8, 10)
    U, N = links(L)
    g = load(H, L, prec, 18, 14)
    try:
        n = 8
        v = gen.gaussian_source(L, n, seed=240)
        b = pack(H, g, v, prec)
        for parity in (0, 1):
            w = torch.empty_like(b)
            H.hisq_dslash_ex(g, mu, b, w, parity, prec, H.HISQ_BUNDLE, n=n)
            got = unpack(H, g, w, n, prec)
            ref = O.dslash_parity(U, N, v, L, parity, mu)
            for k in range(n):
                assert rel_l2(got[k], ref[k]) < TOL[prec]
    finally:
        H.hisq_gauge_free(g)


def _sample_sites(L, count, seed, parity):
    rng = np.random.default_rng(seed)
    sites = []
    while len(sites) < count:
        c = tuple(int(rng.integers(0, L[m])) for m in range(4))
        if sum(c) % 2 == parity:
            sites.append(c)
    corners = [(0, 0, 0, 0), (L[0] - 1, L[1] - 1, L[2] - 1, L[3] - 1), (1, 0, 0, L[3] - 1),
               (L[0] - 2, 1, L[2] - 1, 0), (0, L[1] - 3, 2, L[3] - 2)]
    sites += [c for c in corners if sum(c) % 2 == parity]
    hidx = [(c[0] + L[0] * (c[1] + L[1] * (c[2] + L[2] * c[3]))) // 2 for c in sites]
    return sites, hidx


@pytest.mark.parametrize("prec", [2, 1])
def test_configuration_lattice_bundle_dslash_on_sampled_sites(gpu_lib, prec):
    """48^3x12, n = 8, U r18 / N r14: the mixed-precision configuration's field
    (16-bit links with field-wide component scales) in the launch the CG uses."""
    import torch
    H = gpu_lib
    L = (48, 48, 48, 12)
    U, N = gen.hisq_links(L, seed=1)
    n = 8
    v = gen.gaussian_source(L, n, seed=2)
    g = H.hisq_gauge_load(L, torch.from_numpy(U).cuda(), torch.from_numpy(N).cuda(),
                          prec=prec, recon_U=18, recon_N=14)
    try:
        b = pack(H, g, v, prec)
        w = torch.empty_like(b)
        H.hisq_dslash_ex(g, 0.0, b, w, 0, prec, H.HISQ_BUNDLE, n=n)
        got = unpack(H, g, w, n, prec)
        assert np.all(np.isfinite(got))
        sites, hidx = _sample_sites(L, 96, 11, 0)
        ref = O.dslash_at_sites(U, N, O.to_full(v, L, 1), sites)
        for k in range(n):
            assert rel_l2(got[k, hidx], ref[k]) < TOL[prec], k
    finally:
        H.hisq_gauge_free(g)


@pytest.mark.parametrize("prec,ru,rn,mass", [(1, 18, 14, 0.05), (2, 18, 14, 0.05), (2, 12, 14, 0.1)])
def test_bundle_cg_matches_oracle(gpu_lib, prec, ru, rn, mass):
    import torch
    H = gpu_lib
    L = (4, 6, 8, 10)
    U, N = links(L)
    g = load(H, L, prec, ru, rn)
    try:
        n = 8
        b = gen.z2_source(L, n, seed=250)
        b[3] = 0.0                                       # a zero source rests from the start
        bt = [torch.from_numpy(b[k]).cuda() for k in range(n)]
        xt = [torch.empty_like(t) for t in bt]
        p = H.cg_params(inner_prec=prec, spinor_layout=H.HISQ_BUNDLE)
        st = H.hisq_cg_solve(g, mass, 0.0, bt, xt, 1e-10, p)
        x = np.stack([t.cpu().numpy() for t in xt])
        A = lambda q: O.apply_Ae(U, N, q, L, mass)
        res = O.true_relative_residual(A, x, b)
        assert np.all(res <= 1e-10), res
        assert np.all(x[3] == 0)
        x_ref, _ = O.cg(A, b, tol=1e-13)
        for k in range(n):
            if k != 3:
                assert rel_l2(x[k], x_ref[k]) <= 1e-8, k
        assert st.total_iters > 0
    finally:
        H.hisq_gauge_free(g)


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("rpt,minb,flags", [(8, 3, 0), (8, 3, 4), (8, 4, 4 | 128), (8, 3, 4 | 128 | 16),
                                            (4, 4, 0)])
def test_bundle_cg_with_a_forced_mapping(gpu_lib, prec, rpt, minb, flags):
    """The CG's second Dslash carries the x epilogue and Re<x, out> (the CG on
    A = 4m^2 - D_eo D_oe): the epilogue of every kernel kind against the
    oracle's solve."""
    import torch
    H = gpu_lib
    L = (4, 6, 8, 10)
    mass = 0.05
    U, N = links(L)
    g = load(H, L, prec, 18, 14)
    try:
        H.hisq_set_dslash_mapping(g, rpt, minb, flags)
        assert H.hisq_get_dslash_mapping_ex(g, 8, prec, H.HISQ_BUNDLE) == (rpt, minb, flags)
        n = 8
        b = gen.z2_source(L, n, seed=251)
        bt = [torch.from_numpy(b[k]).cuda() for k in range(n)]
        xt = [torch.empty_like(t) for t in bt]
        p = H.cg_params(inner_prec=prec, spinor_layout=H.HISQ_BUNDLE)
        H.hisq_cg_solve(g, mass, 0.0, bt, xt, 1e-10, p)
        x = np.stack([t.cpu().numpy() for t in xt])
        A = lambda q: O.apply_Ae(U, N, q, L, mass)
        assert np.all(O.true_relative_residual(A, x, b) <= 1e-10)
        x_ref, _ = O.cg(A, b, tol=1e-13)
        for k in range(n):
            assert rel_l2(x[k], x_ref[k]) <= 1e-8, k
    finally:
        H.hisq_gauge_free(g)


def test_profiled_solve_times_every_launch_and_still_converges(gpu_lib):
    """profile_kernels runs the iterations from the host with CUDA events
    around the four launches; the solve itself is unchanged."""
    import torch
    H = gpu_lib
    L = (4, 6, 8, 10)
    mass = 0.05
    U, N = links(L)
    g = load(H, L, 2, 18, 14)
    try:
        n = 8
        b = gen.z2_source(L, n, seed=252)
        bt = [torch.from_numpy(b[k]).cuda() for k in range(n)]
        xt = [torch.empty_like(t) for t in bt]
        p = H.cg_params(inner_prec=2, spinor_layout=H.HISQ_BUNDLE, profile_kernels=1)
        st = H.hisq_cg_solve(g, mass, 0.0, bt, xt, 1e-10, p)
        assert 0 < st.profiled_iters < st.total_iters
        assert all(st.kernel_us[k] > 0 for k in range(4))
        x = np.stack([t.cpu().numpy() for t in xt])
        A = lambda q: O.apply_Ae(U, N, q, L, mass)
        assert np.all(O.true_relative_residual(A, x, b) <= 1e-10)
        st0 = H.hisq_cg_solve(g, mass, 0.0, bt, xt, 1e-10, H.cg_params(inner_prec=2, spinor_layout=H.HISQ_BUNDLE))
        assert st0.profiled_iters == 0 and abs(st0.total_iters - st.total_iters) <= 10
    finally:
        H.hisq_gauge_free(g)


def test_unconverged_solve_returns_the_solution_its_residual_reports(gpu_lib):
    """At the iteration cap (HISQ_ENOCONV) x holds, per rhs, the solution at
    the lowest FP64 residual reached, and stats report that residual."""
    import torch
    H = gpu_lib
    L = (4, 6, 8, 10)
    mass = 0.01
    U, N = links(L)
    g = load(H, L, 2, 18, 14)
    try:
        n = 8
        b = gen.z2_source(L, n, seed=253)
        bt = [torch.from_numpy(b[k]).cuda() for k in range(n)]
        xt = [torch.empty_like(t) for t in bt]
        p = H.cg_params(inner_prec=2, spinor_layout=H.HISQ_BUNDLE, maxiter=40, reliable_every=20)
        with pytest.raises(H.HisqError) as ei:
            H.hisq_cg_solve(g, mass, 0.0, bt, xt, 1e-10, p)
        assert ei.value.status == H.hisq.HISQ_ENOCONV
        st = ei.value.stats
        x = np.stack([t.cpu().numpy() for t in xt])
        A = lambda q: O.apply_Ae(U, N, q, L, mass)
        res = O.true_relative_residual(A, x, b)
        for k in range(n):
            assert 0 < st.true_rel_res[k] < 1.0
            assert abs(res[k] / st.true_rel_res[k] - 1.0) < 1e-6, (k, res[k], st.true_rel_res[k])
    finally:
        H.hisq_gauge_free(g)


# lattices whose (z, t) planes are whole 128-site runs (the tile applies),
# one of them with Lz > Lt; and one where the launcher falls back
@pytest.mark.parametrize("L", [(16, 16, 10, 8), (8, 32, 4, 6), (16, 16, 8, 8), (4, 6, 8, 10)])
@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("minb", [2, 3])
def test_xy_tile_bundle_dslash_matches_oracle(gpu_lib, L, prec, minb):
    """HISQ_MAP_TILE_XY: the x and y hops read a shared-memory tile of whole
    x-rows (Eq. 3 on a bundle); n = 8 uses the tile, n = 16 (two rhs groups)
    the plain loop; both against the oracle on both parities."""
    import torch
    H = gpu_lib
    U, N = links(L)
    g = load(H, L, prec, 18, 14)
    try:
        H.hisq_set_dslash_mapping(g, 8, minb, H.HISQ_MAP_TILE_XY)
        assert H.hisq_get_dslash_mapping_ex(g, 8, prec, H.HISQ_BUNDLE) == (8, minb, H.HISQ_MAP_TILE_XY)
        for n in (8, 16):
            v = gen.gaussian_source(L, n, seed=260 + n)
            b = pack(H, g, v, prec)
            for parity in (0, 1):
                w = torch.full_like(b, float("nan"))
                H.hisq_dslash_ex(g, 0.0, b, w, parity, prec, H.HISQ_BUNDLE, n=n)
                got = unpack(H, g, w, n, prec)
                ref = O.dslash_parity(U, N, v, L, parity)
                for k in range(n):
                    assert rel_l2(got[k], ref[k]) < TOL[prec], (n, parity, k)
    finally:
        H.hisq_gauge_free(g)
