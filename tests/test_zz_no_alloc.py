"""hisq_cdot_noalloc: the FP64 per-rhs dot product for callers that cannot allocate.

Callers whose device memory belongs entirely to another allocator, or that
cannot accept the device synchronisation of cudaMalloc, use this variant of
hisq_cdot; its reduction scratch is a fixed device array inside the library.
The GPU test compares it, through the C ABI, with hisq_cdot (which allocates
its scratch on the handle) on two calls in a row. This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest

from conftest import lib_built


def test_rejects_bundles_beyond_the_static_scratch():
    lib_built()
    import paper_1411_4439_gb300 as H
    lib = H.hisq.library()
    ptrs = (ctypes.c_void_p * 17)()
    out = (ctypes.c_double * 34)()
    st = lib.hisq_cdot_noalloc(ptrs, ptrs, 17, 48, out, None)
    assert st == H.hisq.HISQ_EINVAL
    assert "16" in H.hisq.hisq_last_error()


@pytest.mark.gpu
def test_matches_the_allocating_entry_point_on_two_calls(gpu_lib):
    import torch
    import hisq_inputs as gen
    H = gpu_lib
    L = (4, 6, 8, 10)
    U, N = gen.hisq_links(L, seed=111)
    g = H.hisq_gauge_load(L, torch.from_numpy(U).cuda(), torch.from_numpy(N).cuda(), prec=H.HISQ_F64)
    try:
        for call, n in enumerate((5, 16)):
            a = torch.from_numpy(gen.gaussian_source(L, n, seed=112 + call)).cuda()
            b = torch.from_numpy(gen.gaussian_source(L, n, seed=113 + call)).cuda()
            av, bv = [a[k] for k in range(n)], [b[k] for k in range(n)]
            ref = H.hisq_cdot(g, av, bv)
            got = H.hisq_cdot_noalloc(av, bv)
            assert got.shape == (n,)
            assert np.allclose(got, ref, rtol=1e-13, atol=0.0)
            exact = np.sum(np.conj(a.cpu().numpy()) * b.cpu().numpy(), axis=(1, 2))
            assert np.allclose(got, exact, rtol=1e-12)
    finally:
        H.hisq_gauge_free(g)


def test_rejects_non_fp64_and_host_vectors_before_any_launch():
    import torch
    import paper_1411_4439_gb300 as H
    host = [np.zeros((8, 3), dtype=np.complex128)]
    with pytest.raises(ValueError):
        H.hisq_cdot_noalloc(host, host)          # numpy arrays are host memory
    c64 = [torch.zeros(8, 3, dtype=torch.complex64)]
    with pytest.raises(ValueError):
        H.hisq_cdot_noalloc(c64, c64)
    with pytest.raises(ValueError):
        H.hisq_cdot(None, c64, c64)              # checked before the handle is used


@pytest.mark.gpu
def test_largest_block_count_and_after_a_solve_on_the_same_stream(gpu_lib):
    """A length that launches the largest grid the reduction uses (8 blocks
    per SM for one rhs), and a call queued right behind a CG solve on the
    same stream (the solve's own reductions share nothing with this scratch)."""
    import torch
    import hisq_inputs as gen
    H = gpu_lib
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    length = 2 * 8 * sms * 256                     # complex numbers: > 8 SMs' worth of 256-thread blocks
    rng = np.random.default_rng(5)
    a = rng.standard_normal(length) + 1j * rng.standard_normal(length)
    b = rng.standard_normal(length) + 1j * rng.standard_normal(length)
    at, bt = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    got = H.hisq_cdot_noalloc([at], [bt])
    assert np.allclose(got, [np.vdot(a, b)], rtol=1e-12)
    L = (4, 6, 8, 10)
    U, N = gen.hisq_links(L, seed=121)
    g = H.hisq_gauge_load(L, torch.from_numpy(U).cuda(), torch.from_numpy(N).cuda(), prec=H.HISQ_F32,
                          recon_U=18, recon_N=14)
    try:
        src = torch.from_numpy(gen.z2_source(L, 4, seed=122)).cuda()
        xs = [torch.zeros_like(src[k]) for k in range(4)]
        stream = torch.cuda.current_stream()
        H.hisq_cg_solve(g, 0.1, 0.0, [src[k] for k in range(4)], xs, 1e-10,
                        H.cg_params(inner_prec=H.HISQ_F32), stream=stream)
        got = H.hisq_cdot_noalloc(xs, [src[k] for k in range(4)], stream=stream)
        want = [np.vdot(xs[k].cpu().numpy(), src[k].cpu().numpy()) for k in range(4)]
        assert np.allclose(got, want, rtol=1e-12)
    finally:
        H.hisq_gauge_free(g)
