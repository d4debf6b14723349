// CG vector updates on the rhs-interleaved bundle layout (see
// dslash_bundle.cuh): the same operations as blas.cu, with the W rhs of a
// 16-byte chunk updated together, each with its own alpha_k, beta_k and
// masks. Vectors are [G][3][V_h] chunks (G = n / W groups); the grid is
// (blocks per group, G), every block streams a strided share of one group.
// Per-rhs sums: per thread in FP32, across the warp in FP32, across warps and
// blocks in FP64 in a fixed order (deterministic).
//
// FP64 vectors (the reliable-update side: b, x, r) stay one [V_h][3] block
// per rhs, as in blas.cu.
#include "hisq_internal.cuh"
#include "reduce.cuh"

namespace hisq {

namespace {

constexpr int kThreads = 256;

// One chunk of W rhs of storage S as complex numbers, and back.
template <typename S> struct Chunk;
template <> struct Chunk<float> {
    static constexpr int W = 2;
    __device__ static void get(const uint4& c, float2 (&v)[2]) {
        v[0] = make_float2(__uint_as_float(c.x), __uint_as_float(c.z));
        v[1] = make_float2(__uint_as_float(c.y), __uint_as_float(c.w));
    }
    __device__ static uint4 put(const float2 (&v)[2]) {
        return make_uint4(__float_as_uint(v[0].x), __float_as_uint(v[1].x), __float_as_uint(v[0].y),
                          __float_as_uint(v[1].y));
    }
    __device__ static void round(float2 (&)[2]) {}
};
__device__ __forceinline__ float2 h2f2(unsigned u) {
    __half2 h;
    memcpy(&h, &u, 4);
    return __half22float2(h);
}
__device__ __forceinline__ unsigned f2h2(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    unsigned u;
    memcpy(&u, &h, 4);
    return u;
}
template <> struct Chunk<__half> {
    static constexpr int W = 4;
    __device__ static void get(const uint4& c, float2 (&v)[4]) {
        const float2 r01 = h2f2(c.x), r23 = h2f2(c.y), i01 = h2f2(c.z), i23 = h2f2(c.w);
        v[0] = make_float2(r01.x, i01.x);
        v[1] = make_float2(r01.y, i01.y);
        v[2] = make_float2(r23.x, i23.x);
        v[3] = make_float2(r23.y, i23.y);
    }
    __device__ static uint4 put(const float2 (&v)[4]) {
        return make_uint4(f2h2(v[0].x, v[1].x), f2h2(v[2].x, v[3].x), f2h2(v[0].y, v[1].y),
                          f2h2(v[2].y, v[3].y));
    }
    __device__ static void round(float2 (&v)[4]) {
#pragma unroll
        for (int l = 0; l < 4; ++l) v[l] = __half22float2(__floats2half2_rn(v[l].x, v[l].y));
    }
};

// The solution increment x_lo: FP32, W rhs per chunk of 8 W bytes
// (real parts of the W rhs, then imaginary parts).
template <int W>
__device__ __forceinline__ void xlo_get(const float* b, long long i, float2 (&v)[W]) {
    const float4* p = reinterpret_cast<const float4*>(b + (size_t)i * 2 * W);
    if constexpr (W == 2) {
        const float4 t = __ldg(p);
        v[0] = make_float2(t.x, t.z);
        v[1] = make_float2(t.y, t.w);
    } else {
        const float4 re = __ldg(p), im = __ldg(p + 1);
        v[0] = make_float2(re.x, im.x);
        v[1] = make_float2(re.y, im.y);
        v[2] = make_float2(re.z, im.z);
        v[3] = make_float2(re.w, im.w);
    }
}
template <int W>
__device__ __forceinline__ void xlo_put(float* b, long long i, const float2 (&v)[W]) {
    float4* p = reinterpret_cast<float4*>(b + (size_t)i * 2 * W);
    if constexpr (W == 2) {
        p[0] = make_float4(v[0].x, v[1].x, v[0].y, v[1].y);
    } else {
        p[0] = make_float4(v[0].x, v[1].x, v[2].x, v[3].x);
        p[1] = make_float4(v[0].y, v[1].y, v[2].y, v[3].y);
    }
}

// Per-rhs sums of a block (NV values per thread, value j of group blockIdx.y
// is rhs blockIdx.y * NV + j) into the partial slots; in the last block,
// s_vals[0 .. G * NV) holds the grid sums. Returns true in the last block.
template <int NV>
__device__ bool group_reduce_arrive(const RedScratch& red, float (&val)[NV], int groups, double* s_vals) {
    __shared__ double s_w[NV][kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const float t = warp_sum(val[j]);
        if (lane == 0) s_w[j][warp] = (double)t;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        const int j = threadIdx.x;
        double acc = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) acc += s_w[j][w];
        red.partials[(size_t)(blockIdx.y * NV + j) * kMaxRedBlocks + blockIdx.x] = acc;
    }
    if (!last_block_arrive(red.counter, gridDim.x * gridDim.y)) return false;
    finish_values(red, groups * NV, gridDim.x, [](int) { return false; }, s_vals);
    return true;
}

// r -= alpha Ap (moving rhs) ; rr' = |r|^2 of the stored r ; finish: beta.
template <typename S>
__global__ void __launch_bounds__(kThreads, 4) update_r_b_kernel(BlasArgs a, uint4* r, const uint4* Ap) {
    constexpr int W = Chunk<S>::W;
    const int g = blockIdx.y;
    const long long nch = a.len;   // chunks per group: 3 V_h
    const size_t off = (size_t)g * nch;
    float alpha[W], val[W];
    bool mv[W], any = false;
#pragma unroll
    for (int l = 0; l < W; ++l) {
        const int k = g * W + l;
        mv[l] = moving(a.cg, k);
        alpha[l] = mv[l] ? (float)a.cg->alpha[k] : 0.f;
        val[l] = 0.f;
        any = any || mv[l];
    }
    if (any) {
        // U chunks per thread and pass, all loads issued before the first use
        constexpr int U = 4;
        const long long stride = (long long)gridDim.x * blockDim.x;
        for (long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; i0 < nch; i0 += U * stride) {
            uint4 rc[U], ac[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long i = i0 + u * stride;
                if (i < nch) {
                    rc[u] = __ldg(r + off + i);
                    ac[u] = __ldg(Ap + off + i);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long i = i0 + u * stride;
                if (i >= nch) break;
                float2 rv[W], av[W];
                Chunk<S>::get(rc[u], rv);
                Chunk<S>::get(ac[u], av);
#pragma unroll
                for (int l = 0; l < W; ++l) {
                    if (!mv[l]) continue;   // a resting rhs keeps its residual
                    rv[l].x = fmaf(-alpha[l], av[l].x, rv[l].x);
                    rv[l].y = fmaf(-alpha[l], av[l].y, rv[l].y);
                }
                r[off + i] = Chunk<S>::put(rv);
                Chunk<S>::round(rv);   // the norm is that of the stored residual
#pragma unroll
                for (int l = 0; l < W; ++l) val[l] = fmaf(rv[l].x, rv[l].x, fmaf(rv[l].y, rv[l].y, val[l]));
            }
        }
    }
    __shared__ double s_vals[kMaxRedVals];
    if (group_reduce_arrive<W>(a.red, val, gridDim.y, s_vals)) finish_cg_beta(a.cg, s_vals, a.n);
}

// x_lo += alpha p ; p = r + beta p (moving rhs), both from the old p.
template <typename S>
__global__ void __launch_bounds__(kThreads, 4) update_px_b_kernel(BlasArgs a, float* x, const uint4* r, uint4* p) {
    constexpr int W = Chunk<S>::W;
    const int g = blockIdx.y;
    const long long nch = a.len;
    const size_t off = (size_t)g * nch;
    float alpha[W], beta[W];
    bool mv[W], any_x = false, any_p = false;
#pragma unroll
    for (int l = 0; l < W; ++l) {
        const int k = g * W + l;
        alpha[l] = (float)a.cg->alpha[k];
        mv[l] = moving(a.cg, k);
        beta[l] = (float)a.cg->beta[k];
        any_x = any_x || alpha[l] != 0.f;
        any_p = any_p || mv[l];
    }
    if (!any_x && !any_p) return;
    // U chunks per thread and pass, all loads issued before the first use
    constexpr int U = 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; i0 < nch; i0 += U * stride) {
        uint4 pc[U], rc[U];
        float2 xv[U][W];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long i = i0 + u * stride;
            if (i < nch) {
                pc[u] = __ldg(p + off + i);
                if (any_x) xlo_get<W>(x, (long long)off + i, xv[u]);
                if (any_p) rc[u] = __ldg(r + off + i);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long i = i0 + u * stride;
            if (i >= nch) break;
            float2 pv[W];
            Chunk<S>::get(pc[u], pv);
            if (any_x) {
#pragma unroll
                for (int l = 0; l < W; ++l) {
                    if (alpha[l] == 0.f) continue;
                    xv[u][l].x = fmaf(alpha[l], pv[l].x, xv[u][l].x);
                    xv[u][l].y = fmaf(alpha[l], pv[l].y, xv[u][l].y);
                }
                xlo_put<W>(x, (long long)off + i, xv[u]);
            }
            if (any_p) {
                float2 rv[W];
                Chunk<S>::get(rc[u], rv);
#pragma unroll
                for (int l = 0; l < W; ++l) {
                    if (mv[l]) {
                        pv[l].x = fmaf(beta[l], pv[l].x, rv[l].x);
                        pv[l].y = fmaf(beta[l], pv[l].y, rv[l].y);
                    }
                }
                p[off + i] = Chunk<S>::put(pv);
            }
        }
    }
}

// x_hi (FP64, [V_h][3] per rhs) += x_lo / scale ; x_lo = 0 (active rhs).
template <int W>
__global__ void __launch_bounds__(kThreads) accum_b_kernel(BlasArgs a, double2* x_hi, float* x_lo, int vh) {
    const int g = blockIdx.y;
    const long long nch = a.len;
    const size_t off = (size_t)g * nch;
    bool act[W], any = false;
    double inv[W];
#pragma unroll
    for (int l = 0; l < W; ++l) {
        const int k = g * W + l;
        act[l] = a.cg->active[k] != 0;
        inv[l] = 1.0 / a.cg->scale[k];
        any = any || act[l];
    }
    if (!any) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nch;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i / vh);
        const long long h = i - (long long)c * vh;
        float2 lo[W];
        xlo_get<W>(x_lo, (long long)off + i, lo);
#pragma unroll
        for (int l = 0; l < W; ++l) {
            if (!act[l]) continue;
            double2* xp = x_hi + (size_t)(g * W + l) * a.len + 3 * h + c;
            double2 v = *xp;
            v.x = fma((double)lo[l].x, inv[l], v.x);
            v.y = fma((double)lo[l].y, inv[l], v.y);
            *xp = v;
            lo[l] = make_float2(0.f, 0.f);
        }
        xlo_put<W>(x_lo, (long long)off + i, lo);
    }
}

// r_lo = scale r_hi ; p_lo = reset ? r_lo : p_lo * scale / scale_old ;
// rr = rr_rel = |r_lo|^2 (active rhs; the others keep their vectors).
template <typename S>
__global__ void __launch_bounds__(kThreads) rescale_b_kernel(BlasArgs a, const double2* r_hi, uint4* r_lo,
                                                             uint4* p_lo, int reset_all, int vh) {
    constexpr int W = Chunk<S>::W;
    const int g = blockIdx.y;
    const long long nch = a.len;
    const size_t off = (size_t)g * nch;
    bool act[W], reset[W];
    double sc[W];
    float ratio[W], val[W];
#pragma unroll
    for (int l = 0; l < W; ++l) {
        const int k = g * W + l;
        act[l] = a.cg->active[k] != 0;
        reset[l] = reset_all != 0 || a.cg->reset_p[k] != 0;
        sc[l] = a.cg->scale[k];
        ratio[l] = (float)(a.cg->scale[k] / a.cg->scale_old[k]);
        val[l] = 0.f;
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nch;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i / vh);
        const long long h = i - (long long)c * vh;
        float2 rv[W], pv[W];
        Chunk<S>::get(__ldg(r_lo + off + i), rv);
        Chunk<S>::get(__ldg(p_lo + off + i), pv);
#pragma unroll
        for (int l = 0; l < W; ++l) {
            if (!act[l]) continue;
            const double2 hv = __ldg(r_hi + (size_t)(g * W + l) * a.len + 3 * h + c);
            rv[l] = make_float2((float)(hv.x * sc[l]), (float)(hv.y * sc[l]));
        }
        r_lo[off + i] = Chunk<S>::put(rv);
        Chunk<S>::round(rv);   // the stored values define rr
#pragma unroll
        for (int l = 0; l < W; ++l) {
            if (!act[l]) continue;
            val[l] = fmaf(rv[l].x, rv[l].x, fmaf(rv[l].y, rv[l].y, val[l]));
            if (reset[l]) {
                pv[l] = rv[l];
            } else {
                pv[l].x *= ratio[l];
                pv[l].y *= ratio[l];
            }
        }
        p_lo[off + i] = Chunk<S>::put(pv);
    }
    __shared__ double s_vals[kMaxRedVals];
    if (group_reduce_arrive<W>(a.red, val, gridDim.y, s_vals)) {
        const int t = threadIdx.x;
        if (t < a.n) {
            if (a.cg->active[t]) {
                a.cg->rr[t] = s_vals[t];
                a.cg->rr_rel[t] = s_vals[t];
            }
            a.cg->frozen[t] = 0;
            a.cg->reset_p[t] = 0;
        }
    }
}

// FP64 [V_h][3] per rhs <-> bundle chunks of storage S (pack rounds).
template <typename S>
__global__ void __launch_bounds__(kThreads) pack_b_kernel(const BundlePtrs src, uint4* dst, long long vh) {
    constexpr int W = Chunk<S>::W;
    const int g = blockIdx.y;
    const long long nch = 3 * vh;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nch;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i / vh);
        const long long h = i - (long long)c * vh;
        float2 v[W];
#pragma unroll
        for (int l = 0; l < W; ++l) {
            const double2 d = __ldg(src.p[g * W + l] + 3 * h + c);
            v[l] = make_float2((float)d.x, (float)d.y);
        }
        dst[(size_t)g * nch + i] = Chunk<S>::put(v);
    }
}

template <typename S>
__global__ void __launch_bounds__(kThreads) unpack_b_kernel(const uint4* src, const BundlePtrs dst, long long vh) {
    constexpr int W = Chunk<S>::W;
    const int g = blockIdx.y;
    const long long nch = 3 * vh;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nch;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i / vh);
        const long long h = i - (long long)c * vh;
        float2 v[W];
        Chunk<S>::get(__ldg(src + (size_t)g * nch + i), v);
#pragma unroll
        for (int l = 0; l < W; ++l)
            const_cast<double2*>(dst.p[g * W + l])[3 * h + c] = make_double2((double)v[l].x, (double)v[l].y);
    }
}

// At most per_sm blocks per SM over all groups, one chunk per thread.
dim3 bundle_grid(long long chunks, int groups, int per_sm = 8) {
    long long b = (chunks + kThreads - 1) / kThreads;
    long long cap = ((long long)per_sm * device_sm_count() + groups - 1) / groups;
    if (cap < 1) cap = 1;
    if (b > cap) b = cap;
    if (b > kMaxRedBlocks) b = kMaxRedBlocks;
    if (b < 1) b = 1;
    return dim3((unsigned)b, (unsigned)groups);
}

}  // namespace

int bundle_width(int prec) { return prec == HISQ_F32 ? 2 : prec == HISQ_F16 ? 4 : 0; }

#define HISQ_BUNDLE_SWITCH(prec, CALL)                       \
    switch (prec) {                                          \
        case HISQ_F32: { using S = float; CALL; break; }     \
        case HISQ_F16: { using S = __half; CALL; break; }    \
        default: return cudaErrorInvalidValue;               \
    }

// a.len is the number of chunks per group (3 V_h); a.n the number of rhs.
cudaError_t launch_cg_update_r_bundle(const BlasArgs& a, int prec, void* r, const void* Ap, cudaStream_t s) {
    const int W = bundle_width(prec);
    if (W == 0 || a.n % W) return cudaErrorInvalidValue;
    // one wave of 4 blocks per SM (64 registers a thread), four chunks a pass
    HISQ_BUNDLE_SWITCH(prec, (update_r_b_kernel<S><<<bundle_grid(a.len, a.n / W, 4), kThreads, 0, s>>>(
                                 a, (uint4*)r, (const uint4*)Ap)));
    return cudaGetLastError();
}

cudaError_t launch_cg_update_px_bundle(const BlasArgs& a, int prec, void* x, const void* r, void* p,
                                       cudaStream_t s) {
    const int W = bundle_width(prec);
    if (W == 0 || a.n % W) return cudaErrorInvalidValue;
    // one wave of 4 blocks per SM, two chunks a pass
    HISQ_BUNDLE_SWITCH(prec, (update_px_b_kernel<S><<<bundle_grid(a.len, a.n / W, 4), kThreads, 0, s>>>(
                                 a, (float*)x, (const uint4*)r, (uint4*)p)));
    return cudaGetLastError();
}

cudaError_t launch_accum_solution_bundle(const BlasArgs& a, int prec, double2* x_hi, void* x_lo, int vh,
                                         cudaStream_t s) {
    const int W = bundle_width(prec);
    if (W == 0 || a.n % W) return cudaErrorInvalidValue;
    if (W == 2)
        accum_b_kernel<2><<<bundle_grid(a.len, a.n / W), kThreads, 0, s>>>(a, x_hi, (float*)x_lo, vh);
    else
        accum_b_kernel<4><<<bundle_grid(a.len, a.n / W), kThreads, 0, s>>>(a, x_hi, (float*)x_lo, vh);
    return cudaGetLastError();
}

cudaError_t launch_reliable_rescale_bundle(const BlasArgs& a, int prec, const double2* r_hi, void* r_lo,
                                           void* p_lo, int reset_p, int vh, cudaStream_t s) {
    const int W = bundle_width(prec);
    if (W == 0 || a.n % W) return cudaErrorInvalidValue;
    HISQ_BUNDLE_SWITCH(prec, (rescale_b_kernel<S><<<bundle_grid(a.len, a.n / W), kThreads, 0, s>>>(
                                 a, r_hi, (uint4*)r_lo, (uint4*)p_lo, reset_p, vh)));
    return cudaGetLastError();
}

// ptrs.p[0 .. n): FP64 vectors [V_h][3] (device pointers).
cudaError_t launch_bundle_pack(const BundlePtrs& ptrs, int n, int prec, long long vh, void* bundle,
                               cudaStream_t s) {
    const int W = bundle_width(prec);
    if (W == 0 || n % W) return cudaErrorInvalidValue;
    HISQ_BUNDLE_SWITCH(prec, (pack_b_kernel<S><<<bundle_grid(3 * vh, n / W), kThreads, 0, s>>>(
                                 ptrs, (uint4*)bundle, vh)));
    return cudaGetLastError();
}

cudaError_t launch_bundle_unpack(const void* bundle, const BundlePtrs& ptrs, int n, int prec, long long vh,
                                 cudaStream_t s) {
    const int W = bundle_width(prec);
    if (W == 0 || n % W) return cudaErrorInvalidValue;
    HISQ_BUNDLE_SWITCH(prec, (unpack_b_kernel<S><<<bundle_grid(3 * vh, n / W), kThreads, 0, s>>>(
                                 (const uint4*)bundle, ptrs, vh)));
    return cudaGetLastError();
}

}  // namespace hisq
