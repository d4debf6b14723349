"""GPU Dslash, normal operator and link packing against the FP64 oracle.

Element-by-element relative L2 error per rhs, with the bounds stated for the
storage precisions: FP64 1e-13, FP32 1e-6, FP16 3e-3.
"""
import numpy as np
import pytest

import hisq_inputs as gen
from oracle import hisq_oracle as O
from conftest import from_dev, rel_l2, to_dev

pytestmark = pytest.mark.gpu

TOL = {0: 1e-13, 1: 1e-6, 2: 3e-3}
VARIANTS = [  # (prec, recon_U, recon_N)
    (0, 18, 18),
    (1, 18, 18), (1, 18, 14), (1, 12, 14), (1, 14, 14),
    (2, 18, 18), (2, 18, 14), (2, 12, 14), (2, 14, 14),
]
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


# (4, 6, 10, 8): Lz > Lt, so the kernels visit the (z, t) planes with z slow
@pytest.mark.parametrize("L", [(4, 6, 8, 10), (8, 8, 8, 8), (4, 4, 4, 4), (4, 6, 10, 8)])
@pytest.mark.parametrize("prec,ru,rn", VARIANTS)
def test_dslash_matches_oracle(gpu_lib, L, prec, ru, rn):
    import torch
    H = gpu_lib
    U, N = links(L)
    g = load(H, L, prec, ru, rn)
    try:
        for n in (1, 3, 8):
            v = gen.gaussian_source(L, n, seed=10 + n)
            for parity in (0, 1):
                vd = [to_dev(v[k], prec) for k in range(n)]
                wd = [torch.empty_like(t) for t in vd]
                H.hisq_dslash(g, vd, wd, parity, prec)
                torch.cuda.synchronize()
                ref = O.dslash_parity(U, N, v, L, parity)
                for k in range(n):
                    assert rel_l2(from_dev(wd[k]), ref[k]) < TOL[prec], (n, parity, k)
    finally:
        H.hisq_gauge_free(g)


@pytest.mark.parametrize("prec,ru,rn", [(0, 18, 18), (1, 18, 14), (1, 12, 14), (2, 14, 14)])
@pytest.mark.parametrize("mu", [0.2, -0.35])
def test_dslash_chemical_potential(gpu_lib, prec, ru, rn, mu):
    import torch
    H = gpu_lib
    L = (4, 6, 8, 10)
    U, N = links(L)
    g = load(H, L, prec, ru, rn)
    try:
        n = 2
        v = gen.gaussian_source(L, n, seed=21)
        for parity in (0, 1):
            vd = [to_dev(v[k], prec) for k in range(n)]
            wd = [torch.empty_like(t) for t in vd]
            H.hisq_dslash_ex(g, mu, vd, wd, parity, prec)
            torch.cuda.synchronize()
            ref = O.dslash_parity(U, N, v, L, parity, mu)
            for k in range(n):
                assert rel_l2(from_dev(wd[k]), ref[k]) < TOL[prec]
    finally:
        H.hisq_gauge_free(g)


@pytest.mark.parametrize("prec,ru,rn", [(0, 18, 18), (1, 18, 14), (2, 18, 14)])
@pytest.mark.parametrize("n", [16, 12, 6])
def test_every_thread_mapping_gives_the_same_result(gpu_lib, prec, ru, rn, n):
    """Each rhs-per-thread split of the bundle matches the oracle (n up to 16)."""
    import torch
    H = gpu_lib
    L = (4, 6, 8, 10)
    U, N = links(L)
    g = load(H, L, prec, ru, rn)
    try:
        v = gen.z2_source(L, n, seed=31)
        ref = O.dslash_parity(U, N, v, L, 0)
        vd = [to_dev(v[k], prec) for k in range(n)]
        maxr = 4 if prec == 0 else 8
        for rpt in (1, 2, 4, 8):
            if rpt > maxr or n % rpt or n // rpt > 8:
                continue
            H.hisq_set_dslash_mapping(g, rpt)
            wd = [torch.full_like(t, float("nan")) for t in vd]
            H.hisq_dslash(g, vd, wd, 0, prec)
            torch.cuda.synchronize()
            for k in range(n):
                assert rel_l2(from_dev(wd[k]), ref[k]) < TOL[prec], (rpt, k)
    finally:
        H.hisq_gauge_free(g)


@pytest.mark.parametrize("prec,ru,rn", [(0, 18, 18), (1, 18, 14), (2, 18, 14)])
def test_normal_operator_matches_oracle(gpu_lib, prec, ru, rn):
    import torch
    H = gpu_lib
    L = (8, 8, 8, 8)
    U, N = links(L)
    m = 0.05
    g = load(H, L, prec, ru, rn)
    try:
        n = 4
        v = gen.gaussian_source(L, n, seed=41)
        vd = [to_dev(v[k], prec) for k in range(n)]
        wd = [torch.empty_like(t) for t in vd]
        H.hisq_mdagm(g, m, vd, wd, prec)
        torch.cuda.synchronize()
        ref = O.apply_Ae(U, N, v, L, m)
        for k in range(n):
            assert rel_l2(from_dev(wd[k]), ref[k]) < TOL[prec] * (1 if prec else 10)
    finally:
        H.hisq_gauge_free(g)


def test_free_field_eigenvector_on_gpu(gpu_lib):
    """Plane waves are eigenvectors of A_e with eigenvalue 4m^2 + sum s_mu(p)^2."""
    import torch
    H = gpu_lib
    L = (8, 8, 8, 8)
    c1, c3, m = 9 / 8, -1 / 24, 0.05
    U, N = gen.free_field_links(L, c1, c3)
    Lt, Lz, Ly, Lx = O.grid_shape(L)
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    k = (1, 3, 2, 0)
    p = [2 * np.pi * k[0] / Lx, 2 * np.pi * k[1] / Ly, 2 * np.pi * k[2] / Lz, (2 * k[3] + 1) * np.pi / Lt]
    wave = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))[None, ..., None] * np.array([1, 2j, -1])
    ve = O.to_half(wave, L, 0)
    lam = 4 * m * m + sum((2 * c1 * np.sin(q) + 2 * c3 * np.sin(3 * q)) ** 2 for q in p)
    g = H.hisq_gauge_load(L, torch.from_numpy(U).cuda(), torch.from_numpy(N).cuda(), prec=0)
    try:
        vd = [to_dev(ve[0], 0)]
        wd = [torch.empty_like(vd[0])]
        H.hisq_mdagm(g, m, vd, wd, 0)
        torch.cuda.synchronize()
        assert rel_l2(from_dev(wd[0]), lam * ve[0]) < 1e-13
    finally:
        H.hisq_gauge_free(g)


@pytest.mark.parametrize("recon", [18, 14, 12])
def test_link_compress_and_reconstruct(gpu_lib, recon):
    import torch
    H = gpu_lib
    L = (4, 6, 8, 10)
    U, N = links(L)
    src = U if recon == 12 else N
    V = int(np.prod(L))
    d_links = torch.from_numpy(src).cuda()
    packed = torch.empty((4, V, recon), dtype=torch.float64, device="cuda")
    err = H.hisq_link_compress(L, d_links, recon, packed)
    assert err < 1e-13
    ref = {18: lambda a: a.view(np.float64).reshape(a.shape[:-2] + (18,)),
           14: O.compress_r14, 12: O.compress_r12}[recon](src)
    assert np.abs(packed.cpu().numpy().reshape(ref.shape) - ref).max() < 1e-13
    back = torch.empty_like(d_links)
    H.hisq_link_reconstruct(L, packed, recon, back)
    torch.cuda.synchronize()
    assert np.abs(back.cpu().numpy() - src).max() < 5e-14


def test_loader_rejects_links_the_compression_cannot_hold(gpu_lib):
    import torch
    H = gpu_lib
    L = (4, 4, 4, 4)
    U, N = links(L)
    rng = np.random.default_rng(5)
    junk = (rng.standard_normal(N.shape) + 1j * rng.standard_normal(N.shape)) * 0.1
    dU, dN, dJ = (torch.from_numpy(a).cuda() for a in (U, N, junk))
    with pytest.raises(H.HisqError) as e:
        H.hisq_gauge_load(L, dU, dJ, prec=1, recon_U=18, recon_N=14)
    assert e.value.status == H.hisq.HISQ_ERECON
    # Naik links are U(3), not sign * scale * SU(3): R12 must reject them as fat links
    with pytest.raises(H.HisqError) as e:
        H.hisq_gauge_load(L, dN, dN, prec=1, recon_U=12, recon_N=14)
    assert e.value.status == H.hisq.HISQ_ERECON
    # a host-resident load gives the same handle contents as a device load
    g1 = H.hisq_gauge_load(L, U, N, prec=1, recon_U=12, recon_N=14)
    H.hisq_gauge_free(g1)


def test_full_size_dslash_sampled_sites(gpu_lib):
    """32^3x8, n = 8, FP32 with R14 Naik links: check 64 sampled output sites."""
    import torch
    H = gpu_lib
    L = (32, 32, 32, 8)
    U, N = gen.hisq_links(L, seed=1)
    n = 8
    v = gen.z2_source(L, n, seed=2)
    g = H.hisq_gauge_load(L, torch.from_numpy(U).cuda(), torch.from_numpy(N).cuda(),
                          prec=1, recon_U=18, recon_N=14)
    try:
        vd = [to_dev(v[k], 1) for k in range(n)]
        wd = [torch.empty_like(t) for t in vd]
        H.hisq_dslash(g, vd, wd, 0, 1)
        torch.cuda.synchronize()
        w = np.stack([from_dev(t) for t in wd])
        vfull = O.to_full(v, L, 1)
        rng = np.random.default_rng(9)
        sites, hidx = [], []
        while len(sites) < 64:
            c = [int(rng.integers(0, L[m])) for m in range(4)]
            if sum(c) % 2 == 0:
                sites.append(tuple(c))
                hidx.append((c[0] + L[0] * (c[1] + L[1] * (c[2] + L[2] * c[3]))) // 2)
        # include the corners, where every hop wraps
        for c in [(0, 0, 0, 0), (31, 31, 31, 7), (1, 0, 0, 7), (30, 1, 31, 0)]:
            if sum(c) % 2 == 0:
                sites.append(c)
                hidx.append((c[0] + L[0] * (c[1] + L[1] * (c[2] + L[2] * c[3]))) // 2)
        ref = O.dslash_at_sites(U, N, vfull, sites)
        got = w[:, hidx]
        assert rel_l2(got, ref) < 1e-6
        assert np.all(np.isfinite(w))
    finally:
        H.hisq_gauge_free(g)


@pytest.mark.parametrize("prec,ru,rn", [(0, 18, 18), (1, 18, 14), (1, 12, 14), (2, 18, 14)])
@pytest.mark.parametrize("mu", [0.0, 0.15])
def test_soa_layout_matches_oracle(gpu_lib, prec, ru, rn, mu):
    """Colour-plane layout [3][V_h]: same operator, different addressing."""
    import torch
    H = gpu_lib
    L = (4, 6, 8, 10)
    U, N = links(L)
    g = load(H, L, prec, ru, rn)
    try:
        for n in (3, 8):
            v = gen.gaussian_source(L, n, seed=50 + n)
            for parity in (0, 1):
                vs = np.ascontiguousarray(np.swapaxes(v, 1, 2))        # (n, 3, V_h)
                vd = [to_dev(vs[k], prec) for k in range(n)]
                wd = [torch.full_like(t, float("nan")) for t in vd]
                H.hisq_dslash_ex(g, mu, vd, wd, parity, prec, H.HISQ_SOA)
                torch.cuda.synchronize()
                ref = O.dslash_parity(U, N, v, L, parity, mu)
                for k in range(n):
                    got = np.swapaxes(from_dev(wd[k]), 0, 1)
                    assert rel_l2(got, ref[k]) < TOL[prec], (n, parity, k)
    finally:
        H.hisq_gauge_free(g)


@pytest.mark.parametrize("rpt,minb", [(1, 4), (2, 3), (4, 2), (4, 3), (8, 2)])
def test_every_built_mapping_matches_oracle(gpu_lib, rpt, minb):
    import torch
    H = gpu_lib
    L = (8, 8, 8, 8)
    U, N = links(L)
    g = load(H, L, 1, 18, 14)
    try:
        H.hisq_set_dslash_mapping(g, rpt, minb)
        n = 8
        v = gen.z2_source(L, n, seed=61)
        ref = O.dslash_parity(U, N, v, L, 1)
        for layout in (H.HISQ_AOS, H.HISQ_SOA):
            src = v if layout == H.HISQ_AOS else np.ascontiguousarray(np.swapaxes(v, 1, 2))
            vd = [to_dev(src[k], 1) for k in range(n)]
            wd = [torch.full_like(t, float("nan")) for t in vd]
            H.hisq_dslash_ex(g, 0.0, vd, wd, 1, 1, layout)
            torch.cuda.synchronize()
            for k in range(n):
                got = from_dev(wd[k])
                got = got if layout == H.HISQ_AOS else np.swapaxes(got, 0, 1)
                assert rel_l2(got, ref[k]) < 1e-6
    finally:
        H.hisq_gauge_free(g)


@pytest.mark.parametrize("L", [(16, 16, 4, 6), (32, 8, 6, 4)])
@pytest.mark.parametrize("prec,ru,rn", [(1, 18, 14), (1, 12, 14), (1, 18, 18), (2, 18, 14), (2, 14, 14)])
def test_staged_link_kernel_matches_oracle(gpu_lib, L, prec, ru, rn):
    """Links staged in shared memory by bulk copies: every mapping, both layouts, mu."""
    import torch
    H = gpu_lib
    U, N = links(L)
    g = load(H, L, prec, ru, rn)
    try:
        for n, rpt, minb in ((8, 8, 2), (8, 8, 3), (8, 4, 2), (4, 4, 3), (4, 4, 2)):
            H.hisq_set_dslash_mapping(g, rpt, minb, H.HISQ_MAP_STAGED)
            assert H.hisq_get_dslash_mapping(g, n, prec) == (rpt, minb, H.HISQ_MAP_STAGED)
            v = gen.gaussian_source(L, n, seed=70 + n)
            for layout in (H.HISQ_AOS, H.HISQ_SOA):
                for parity, mu in ((0, 0.0), (1, 0.0), (0, 0.2)):
                    src = v if layout == H.HISQ_AOS else np.ascontiguousarray(np.swapaxes(v, 1, 2))
                    vd = [to_dev(src[k], prec) for k in range(n)]
                    wd = [torch.full_like(t, float("nan")) for t in vd]
                    H.hisq_dslash_ex(g, mu, vd, wd, parity, prec, layout)
                    torch.cuda.synchronize()
                    ref = O.dslash_parity(U, N, v, L, parity, mu)
                    for k in range(n):
                        got = from_dev(wd[k])
                        got = got if layout == H.HISQ_AOS else np.swapaxes(got, 0, 1)
                        assert rel_l2(got, ref[k]) < TOL[prec], (n, rpt, minb, layout, parity, mu, k)
    finally:
        H.hisq_gauge_free(g)


def test_staged_mapping_falls_back_where_the_tile_does_not_fit(gpu_lib):
    H = gpu_lib
    g = load(H, (8, 8, 8, 8), 1, 18, 14)      # an x-y plane holds 32 sites < one 128-site tile
    try:
        H.hisq_set_dslash_mapping(g, 8, 2, H.HISQ_MAP_STAGED)
        assert H.hisq_get_dslash_mapping(g, 8, 1)[2] & H.HISQ_MAP_STAGED == 0
    finally:
        H.hisq_gauge_free(g)


def test_staged_cg_solve_matches_oracle(gpu_lib):
    import torch
    H = gpu_lib
    L, m = (16, 16, 4, 6), 0.05
    U, N = links(L)
    b = gen.z2_source(L, 8, seed=81)
    g = load(H, L, 1, 18, 14)
    try:
        H.hisq_set_dslash_mapping(g, 8, 2, H.HISQ_MAP_STAGED)
        bt = [torch.from_numpy(b[k]).cuda() for k in range(8)]
        xt = [torch.zeros_like(t) for t in bt]
        H.hisq_cg_solve(g, m, 0.0, bt, xt, 1e-10, H.cg_params(inner_prec=1))
        x = np.stack([t.cpu().numpy() for t in xt])
    finally:
        H.hisq_gauge_free(g)
    res = O.true_relative_residual(lambda q: O.apply_Ae(U, N, q, L, m), x, b)
    assert np.all(res <= 1e-10)


def test_autotuner_keeps_a_correct_mapping(gpu_lib):
    import torch
    H = gpu_lib
    L = (16, 16, 4, 6)
    U, N = links(L)
    g = load(H, L, 1, 18, 14)
    try:
        for n in (8, 4, 3):
            best = H.hisq.hisq_autotune_dslash(g, n, 1, H.HISQ_AOS, reps=3)
            assert best["seconds"] > 0
            got = H.hisq_get_dslash_mapping(g, n, 1)
            assert got == (best["rhs_per_thread"], best["min_blocks"], best["flags"])
            v = gen.gaussian_source(L, n, seed=90 + n)
            vd = [to_dev(v[k], 1) for k in range(n)]
            wd = [torch.full_like(t, float("nan")) for t in vd]
            H.hisq_dslash(g, vd, wd, 1, 1)
            torch.cuda.synchronize()
            ref = O.dslash_parity(U, N, v, L, 1)
            for k in range(n):
                assert rel_l2(from_dev(wd[k]), ref[k]) < 1e-6
    finally:
        H.hisq_gauge_free(g)


PIPE_MAPPINGS = [(8, 1, 1), (4, 2, 1), (4, 1, 2), (4, 2, 2)]   # (rpt, minb, depth)


@pytest.mark.parametrize("prec,ru,rn", [(1, 18, 14), (1, 12, 14), (1, 18, 18), (1, 14, 14),
                                        (2, 18, 14), (2, 12, 14)])
def test_pipelined_kernel_matches_oracle(gpu_lib, prec, ru, rn):
    """Loads of the next hops in flight: every built mapping, both layouts, mu, parities,
    bundles that use one and two rhs groups, on a lattice with a ragged last block."""
    import torch
    H = gpu_lib
    L = (6, 10, 4, 6)                       # V_h = 720: not a multiple of the block
    U, N = links(L)
    g = load(H, L, prec, ru, rn)
    try:
        for rpt, minb, depth in PIPE_MAPPINGS:
            flag = H.HISQ_MAP_PIPELINED if depth == 1 else H.HISQ_MAP_PIPELINED2
            H.hisq_set_dslash_mapping(g, rpt, minb, flag)
            for n in sorted({rpt, 2 * rpt}):
                assert H.hisq_get_dslash_mapping(g, n, prec) == (rpt, minb, flag)
                v = gen.gaussian_source(L, n, seed=90 + n)
                for layout in (H.HISQ_AOS, H.HISQ_SOA):
                    for parity, mu in ((0, 0.0), (1, 0.0), (1, -0.25)):
                        src = v if layout == H.HISQ_AOS else np.ascontiguousarray(np.swapaxes(v, 1, 2))
                        vd = [to_dev(src[k], prec) for k in range(n)]
                        wd = [torch.full_like(t, float("nan")) for t in vd]
                        H.hisq_dslash_ex(g, mu, vd, wd, parity, prec, layout)
                        torch.cuda.synchronize()
                        ref = O.dslash_parity(U, N, v, L, parity, mu)
                        for k in range(n):
                            got = from_dev(wd[k])
                            got = got if layout == H.HISQ_AOS else np.swapaxes(got, 0, 1)
                            assert rel_l2(got, ref[k]) < TOL[prec], (rpt, minb, depth, n, layout, parity, mu, k)
    finally:
        H.hisq_gauge_free(g)


def test_pipelined_mapping_in_solve_and_mu_derivative(gpu_lib):
    """The CG runs the pipelined kernel; the temporal-only operator d M / d mu,
    which the pipelined kernel does not serve, falls back to the register kernel."""
    import torch
    H = gpu_lib
    L, m, mu = (8, 8, 8, 8), 0.05, 0.2
    U, N = links(L)
    b = gen.z2_source(L, 8, seed=91)
    g = load(H, L, 1, 18, 14)
    try:
        H.hisq_set_dslash_mapping(g, 8, 1, H.HISQ_MAP_PIPELINED)
        bt = [torch.from_numpy(b[k]).cuda() for k in range(8)]
        xt = [torch.zeros_like(t) for t in bt]
        H.hisq_cg_solve(g, m, 0.0, bt, xt, 1e-10, H.cg_params(inner_prec=1))
        x = np.stack([t.cpu().numpy() for t in xt])
        v = O.to_full(gen.gaussian_source(L, 8, seed=92), L, 0) + \
            O.to_full(gen.gaussian_source(L, 8, seed=93), L, 1)
        vb = np.concatenate([O.to_half(v, L, 0), O.to_half(v, L, 1)], axis=1)
        src = [torch.from_numpy(vb[k]).cuda().to(torch.complex64) for k in range(8)]
        for op, order in ((H.HISQ_OP_M, 0), (H.HISQ_OP_DM_DMU, 1)):
            w = [torch.empty_like(t) for t in src]
            H.hisq_apply_m(g, m, mu, op, src, w, 1)
            torch.cuda.synchronize()
            ref = O.apply_M(U, N, v, m, mu) if order == 0 else O.apply_dnM_dmun(U, N, v, mu, 1)
            exp = np.concatenate([O.to_half(ref, L, 0), O.to_half(ref, L, 1)], axis=1)
            for k in range(8):
                assert rel_l2(w[k].cpu().numpy(), exp[k]) < 1e-6, (op, k)
    finally:
        H.hisq_gauge_free(g)
    res = O.true_relative_residual(lambda q: O.apply_Ae(U, N, q, L, m), x, b)
    assert np.all(res <= 1e-10)


def test_tuned_gauge_load_picks_an_exact_compression(gpu_lib):
    """The compression tuner only keeps pairs that hold the links; its handle
    computes the oracle's Dslash and the choice is cached for the shape."""
    import torch
    H = gpu_lib
    L = (16, 16, 4, 6)
    U, N = links(L)
    n = 8
    dU, dN = torch.from_numpy(U).cuda(), torch.from_numpy(N).cuda()
    g = H.hisq_gauge_load_tuned(L, dU, dN, prec=1, n=n)
    try:
        assert (g.recon_U, g.recon_N) in ((18, 18), (18, 14), (12, 14), (14, 14))
        v = gen.gaussian_source(L, n, seed=95)
        vd = [to_dev(v[k], 1) for k in range(n)]
        wd = [torch.empty_like(t) for t in vd]
        H.hisq_dslash(g, vd, wd, 0, 1)
        torch.cuda.synchronize()
        ref = O.dslash_parity(U, N, v, L, 0)
        for k in range(n):
            assert rel_l2(from_dev(wd[k]), ref[k]) < 1e-6
        g2 = H.hisq_gauge_load_tuned(L, dU, dN, prec=1, n=n)
        try:
            assert (g2.recon_U, g2.recon_N) == (g.recon_U, g.recon_N)
        finally:
            H.hisq_gauge_free(g2)
        best = H.hisq_autotune_bundle(g, 8, 1)
        assert best["n"] in (1, 2, 4, 8) and best["seconds_per_rhs"] > 0
    finally:
        H.hisq_gauge_free(g)
    # fat links 0.9 x U(3) (not SU(3)): R12 cannot hold them, the tuner must skip it
    Ualt = (-0.9 * 24.0) * N
    g = H.hisq_gauge_load_tuned((16, 16, 4, 6), torch.from_numpy(Ualt).cuda(), dN, prec=1, n=4)
    try:
        assert g.recon_U != 12
        v = gen.gaussian_source(L, 4, seed=96)
        vd = [to_dev(v[k], 1) for k in range(4)]
        wd = [torch.empty_like(t) for t in vd]
        H.hisq_dslash(g, vd, wd, 1, 1)
        torch.cuda.synchronize()
        ref = O.dslash_parity(Ualt, N, v, L, 1)
        for k in range(4):
            assert rel_l2(from_dev(wd[k]), ref[k]) < 1e-6
    finally:
        H.hisq_gauge_free(g)
