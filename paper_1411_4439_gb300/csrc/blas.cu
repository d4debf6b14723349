// Fused CG vector updates and FP64 reductions (the BLAS-1 part of the CG).
//
// Vectors of the bundle are one contiguous block [n][len] of complex numbers
// (len = 3 V_h). The grid is (blocks per rhs, n): block (b, k) streams a
// strided share of rhs k with 16-byte loads, so every kernel is a pure HBM
// stream. Per-rhs sums are formed per thread in the storage arithmetic (FP32
// for F32/F16, FP64 for F64), reduced across the warp in that precision and
// across warps and blocks in FP64, in a fixed order.
#include "hisq_internal.cuh"
#include "reduce.cuh"

namespace hisq {

namespace {

// VEC complex numbers per 16-byte access of each storage type.
template <typename S> struct Vec;
template <> struct Vec<double> {
    static constexpr int N = 1;
    using R = double;
    __device__ static void load(const void* b, long long i, double2 (&v)[1]) {
        v[0] = __ldg(reinterpret_cast<const double2*>(b) + i);
    }
    __device__ static void store(void* b, long long i, const double2 (&v)[1]) {
        reinterpret_cast<double2*>(b)[i] = v[0];
    }
    __device__ static void round(double2 (&)[1]) {}
};
template <> struct Vec<float> {
    static constexpr int N = 2;
    using R = float;
    __device__ static void load(const void* b, long long i, float2 (&v)[2]) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(b) + i);
        v[0] = make_float2(t.x, t.y);
        v[1] = make_float2(t.z, t.w);
    }
    __device__ static void store(void* b, long long i, const float2 (&v)[2]) {
        reinterpret_cast<float4*>(b)[i] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    }
    __device__ static void round(float2 (&)[2]) {}
};
template <> struct Vec<__half> {
    static constexpr int N = 4;
    using R = float;
    __device__ static void load(const void* b, long long i, float2 (&v)[4]) {
        const uint4 t = __ldg(reinterpret_cast<const uint4*>(b) + i);
        const unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            __half2 h;
            memcpy(&h, &w[c], 4);
            v[c] = __half22float2(h);
        }
    }
    __device__ static void store(void* b, long long i, const float2 (&v)[4]) {
        unsigned w[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const __half2 h = __float22half2_rn(v[c]);
            memcpy(&w[c], &h, 4);
        }
        reinterpret_cast<uint4*>(b)[i] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    // the values a store leaves in memory
    __device__ static void round(float2 (&v)[4]) {
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = __half22float2(__float22half2_rn(v[c]));
    }
};

// FP64 vectors read VEC complex numbers at a time to match a storage chunk.
template <int N>
__device__ __forceinline__ void load64(const double2* b, long long i, double2 (&v)[N]) {
#pragma unroll
    for (int c = 0; c < N; ++c) v[c] = __ldg(b + i * N + c);
}
template <int N>
__device__ __forceinline__ void store64(double2* b, long long i, const double2 (&v)[N]) {
#pragma unroll
    for (int c = 0; c < N; ++c) b[i * N + c] = v[c];
}

template <typename RC> struct CxOf;
template <> struct CxOf<float> { using T = float2; };
template <> struct CxOf<double> { using T = double2; };

constexpr int kThreads = 256;

// Reduce nv per-thread values of rhs blockIdx.y into partial slots, arrive,
// and in the last block fill s_vals[0 .. n*nv). Returns true in the last block.
template <typename R, int NV>
__device__ bool block_reduce_arrive(const RedScratch& red, R (&val)[NV], int n, const bool (&is_max)[NV],
                                    double* s_vals) {
    __shared__ double s_w[NV][kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const R t = is_max[j] ? warp_max(val[j]) : warp_sum(val[j]);
        if (lane == 0) s_w[j][warp] = (double)t;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        const int j = threadIdx.x;
        double acc = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) acc = is_max[j] ? fmax(acc, s_w[j][w]) : acc + s_w[j][w];
        red.partials[(size_t)(blockIdx.y * NV + j) * kMaxRedBlocks + blockIdx.x] = acc;
    }
    if (!last_block_arrive(red.counter, gridDim.x * gridDim.y)) return false;
    finish_values(red, n * NV, gridDim.x, [](int v) { return (NV == 2) && (v & 1); }, s_vals);
    return true;
}

// The low-precision solution increment x_lo is kept in at least FP32: it
// collects alpha p over up to a reliable-update cycle, and in FP16 the small
// increments would round away against its growing value.
template <typename S> struct XType { using T = S; };
template <> struct XType<__half> { using T = float; };

// N complex numbers of an FP32 / FP64 vector starting at complex index i * N.
template <typename SX, int N> struct XVec;
template <int N> struct XVec<float, N> {
    static_assert(N % 2 == 0, "FP32 chunks hold pairs of complex numbers");
    __device__ static void load(const void* b, long long i, float2 (&v)[N]) {
#pragma unroll
        for (int c = 0; c < N / 2; ++c) {
            const float4 t = __ldg(reinterpret_cast<const float4*>(b) + i * (N / 2) + c);
            v[2 * c] = make_float2(t.x, t.y);
            v[2 * c + 1] = make_float2(t.z, t.w);
        }
    }
    __device__ static void store(void* b, long long i, const float2 (&v)[N]) {
#pragma unroll
        for (int c = 0; c < N / 2; ++c)
            reinterpret_cast<float4*>(b)[i * (N / 2) + c] =
                make_float4(v[2 * c].x, v[2 * c].y, v[2 * c + 1].x, v[2 * c + 1].y);
    }
};
template <int N> struct XVec<double, N> {
    __device__ static void load(const void* b, long long i, double2 (&v)[N]) {
#pragma unroll
        for (int c = 0; c < N; ++c) v[c] = __ldg(reinterpret_cast<const double2*>(b) + i * N + c);
    }
    __device__ static void store(void* b, long long i, const double2 (&v)[N]) {
#pragma unroll
        for (int c = 0; c < N; ++c) reinterpret_cast<double2*>(b)[i * N + c] = v[c];
    }
};

// r -= alpha Ap ; rr' = |r|^2 of the stored residual ; finish: beta = rr'/rr.
// The solution update waits for update_px, which reads p before it changes.
template <typename S>
__global__ void __launch_bounds__(kThreads) update_r_kernel(BlasArgs a, void* r, const void* Ap) {
    using V = Vec<S>;
    using R = typename V::R;
    using RC = typename CxOf<R>::T;
    constexpr int N = V::N;
    const int k = blockIdx.y;
    const long long nch = a.len / N;
    const long long off = (long long)k * nch;
    R val[1] = {(R)0};
    if (moving(a.cg, k)) {
        const R alpha = (R)a.cg->alpha[k];
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nch;
             i += (long long)gridDim.x * blockDim.x) {
            RC rv[N], av[N];
            V::load(r, off + i, rv);
            V::load(Ap, off + i, av);
#pragma unroll
            for (int c = 0; c < N; ++c) {
                rv[c].x = fma(-alpha, av[c].x, rv[c].x);
                rv[c].y = fma(-alpha, av[c].y, rv[c].y);
            }
            V::store(r, off + i, rv);
            V::round(rv);   // the norm is that of the stored residual
#pragma unroll
            for (int c = 0; c < N; ++c) val[0] = fma(rv[c].x, rv[c].x, fma(rv[c].y, rv[c].y, val[0]));
        }
    }
    __shared__ double s_vals[kMaxRedVals];
    const bool mx[1] = {false};
    if (block_reduce_arrive<R, 1>(a.red, val, a.n, mx, s_vals)) finish_cg_beta(a.cg, s_vals, a.n);
}

// x += alpha p ; p = r + beta p, both from the old p, in one pass. alpha is
// zero for an rhs that did not move this iteration; an rhs frozen by this
// iteration's finish still takes its x update but keeps p.
template <typename S>
__global__ void __launch_bounds__(kThreads) update_px_kernel(BlasArgs a, void* x, const void* r, void* p) {
    using V = Vec<S>;
    using R = typename V::R;
    using RC = typename CxOf<R>::T;
    using X = XVec<typename XType<S>::T, V::N>;
    constexpr int N = V::N;
    const int k = blockIdx.y;
    const R alpha = (R)a.cg->alpha[k];
    const bool move = moving(a.cg, k);
    const bool upd_x = alpha != (R)0;
    if (!move && !upd_x) return;
    const long long nch = a.len / N;
    const long long off = (long long)k * nch;
    const R beta = (R)a.cg->beta[k];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nch;
         i += (long long)gridDim.x * blockDim.x) {
        RC pv[N];
        V::load(p, off + i, pv);
        if (upd_x) {
            RC xv[N];
            X::load(x, off + i, xv);
#pragma unroll
            for (int c = 0; c < N; ++c) {
                xv[c].x = fma(alpha, pv[c].x, xv[c].x);
                xv[c].y = fma(alpha, pv[c].y, xv[c].y);
            }
            X::store(x, off + i, xv);
        }
        if (move) {
            RC rv[N];
            V::load(r, off + i, rv);
#pragma unroll
            for (int c = 0; c < N; ++c) {
                pv[c].x = fma(beta, pv[c].x, rv[c].x);
                pv[c].y = fma(beta, pv[c].y, rv[c].y);
            }
            V::store(p, off + i, pv);
        }
    }
}

// x_hi += x_lo / scale ; x_lo = 0   (FP64 solution accumulation)
template <typename S>
__global__ void __launch_bounds__(kThreads) accum_kernel(BlasArgs a, double2* x_hi, void* x_lo) {
    using V = Vec<S>;
    using R = typename V::R;
    using RC = typename CxOf<R>::T;
    using X = XVec<typename XType<S>::T, V::N>;
    constexpr int N = V::N;
    const int k = blockIdx.y;
    if (!a.cg->active[k]) return;
    const long long nch = a.len / N;
    const long long off = (long long)k * nch;
    const double inv = 1.0 / a.cg->scale[k];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nch;
         i += (long long)gridDim.x * blockDim.x) {
        RC lo[N];
        double2 hi[N];
        X::load(x_lo, off + i, lo);
        load64<N>(x_hi, off + i, hi);
#pragma unroll
        for (int c = 0; c < N; ++c) {
            hi[c].x = fma((double)lo[c].x, inv, hi[c].x);
            hi[c].y = fma((double)lo[c].y, inv, hi[c].y);
            lo[c].x = (R)0;
            lo[c].y = (R)0;
        }
        store64<N>(x_hi, off + i, hi);
        X::store(x_lo, off + i, lo);
    }
}

// |b|^2 per rhs -> bb, active, unit scale
__global__ void __launch_bounds__(kThreads) norm_bb_kernel(BlasArgs a, const double2* b) {
    const int k = blockIdx.y;
    const long long off = (long long)k * a.len;
    double val[1] = {0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.len;
         i += (long long)gridDim.x * blockDim.x) {
        const double2 v = __ldg(b + off + i);
        val[0] = fma(v.x, v.x, fma(v.y, v.y, val[0]));
    }
    __shared__ double s_vals[kMaxRedVals];
    const bool mx[1] = {false};
    if (block_reduce_arrive<double, 1>(a.red, val, a.n, mx, s_vals)) {
        const int t = threadIdx.x;
        if (t < a.n) {
            const double bb = s_vals[t];
            a.cg->bb[t] = bb;
            a.cg->active[t] = (bb > 0.0 && isfinite(bb)) ? 1 : 0;
            if (!isfinite(bb)) atomicOr(&a.cg->flags, kFlagNaN);
            a.cg->scale[t] = 1.0;
            a.cg->scale_old[t] = 1.0;
            a.cg->rr[t] = 0.0;
            a.cg->alpha[t] = 0.0;
            a.cg->beta[t] = 0.0;
        }
        if (t == 0) {
            a.cg->freeze2 = a.freeze2;
            a.cg->alpha_max = a.alpha_max;
        }
        if (t == 0) a.cg->flags = isfinite(s_vals[0]) ? a.cg->flags : (a.cg->flags | kFlagNaN);
    }
}

// r_hi = b (start from x0 = 0): |r|^2 and max|r_i| -> reliable finish
__global__ void __launch_bounds__(kThreads) copy_residual_kernel(BlasArgs a, const double2* b,
                                                                 double2* r_hi, double tol2) {
    const int k = blockIdx.y;
    const long long off = (long long)k * a.len;
    double val[2] = {0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.len;
         i += (long long)gridDim.x * blockDim.x) {
        const double2 v = __ldg(b + off + i);
        r_hi[off + i] = v;
        const double n2 = v.x * v.x + v.y * v.y;
        val[0] += n2;
        val[1] = fmax(val[1], sqrt(n2));
    }
    __shared__ double s_vals[kMaxRedVals];
    const bool mx[2] = {false, true};
    if (block_reduce_arrive<double, 2>(a.red, val, a.n, mx, s_vals))
        finish_reliable(a.cg, s_vals, a.n, tol2);
}

// r_lo = scale r_hi ; p_lo = reset ? r_lo : p_lo * scale/scale_old ; rr = |r_lo|^2
template <typename S>
__global__ void __launch_bounds__(kThreads) rescale_kernel(BlasArgs a, const double2* r_hi,
                                                           void* r_lo, void* p_lo, int reset_p) {
    using V = Vec<S>;
    using R = typename V::R;
    using RC = typename CxOf<R>::T;
    constexpr int N = V::N;
    const int k = blockIdx.y;
    const long long nch = a.len / N;
    const long long off = (long long)k * nch;
    R val[1] = {(R)0};
    if (a.cg->active[k]) {
        const bool reset = reset_p != 0 || a.cg->reset_p[k] != 0;
        const double sc = a.cg->scale[k];
        const R ratio = (R)(a.cg->scale[k] / a.cg->scale_old[k]);
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nch;
             i += (long long)gridDim.x * blockDim.x) {
            double2 hi[N];
            RC lo[N];
            load64<N>(r_hi, off + i, hi);
#pragma unroll
            for (int c = 0; c < N; ++c) {
                lo[c].x = (R)(hi[c].x * sc);
                lo[c].y = (R)(hi[c].y * sc);
            }
            V::store(r_lo, off + i, lo);
            V::round(lo);   // the stored values define rr
#pragma unroll
            for (int c = 0; c < N; ++c) val[0] = fma(lo[c].x, lo[c].x, fma(lo[c].y, lo[c].y, val[0]));
            if (reset) {
                V::store(p_lo, off + i, lo);
            } else {
                RC pv[N];
                V::load(p_lo, off + i, pv);
#pragma unroll
                for (int c = 0; c < N; ++c) {
                    pv[c].x *= ratio;
                    pv[c].y *= ratio;
                }
                V::store(p_lo, off + i, pv);
            }
        }
    }
    __shared__ double s_vals[kMaxRedVals];
    const bool mx[1] = {false};
    if (block_reduce_arrive<R, 1>(a.red, val, a.n, mx, s_vals)) {
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

// pAp = Re <p, Ap> -> alpha = rr / pAp (full-lattice operator)
template <typename S>
__global__ void __launch_bounds__(kThreads) dot_alpha_kernel(BlasArgs a, const void* p, const void* Ap) {
    using V = Vec<S>;
    using R = typename V::R;
    using RC = typename CxOf<R>::T;
    constexpr int N = V::N;
    const int k = blockIdx.y;
    const long long nch = a.len / N;
    const long long off = (long long)k * nch;
    R val[1] = {(R)0};
    if (moving(a.cg, k)) {
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nch;
             i += (long long)gridDim.x * blockDim.x) {
            RC pv[N], av[N];
            V::load(p, off + i, pv);
            V::load(Ap, off + i, av);
#pragma unroll
            for (int c = 0; c < N; ++c) val[0] = fma(pv[c].x, av[c].x, fma(pv[c].y, av[c].y, val[0]));
        }
    }
    __shared__ double s_vals[kMaxRedVals];
    const bool mx[1] = {false};
    if (block_reduce_arrive<R, 1>(a.red, val, a.n, mx, s_vals)) finish_cg_alpha(a.cg, s_vals, a.n);
}

// |r_hi|^2 and max |r_i| -> reliable finish (full-lattice residual)
__global__ void __launch_bounds__(kThreads) residual_norm_kernel(BlasArgs a, const double2* r_hi,
                                                                 double tol2) {
    const int k = blockIdx.y;
    const long long off = (long long)k * a.len;
    double val[2] = {0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.len;
         i += (long long)gridDim.x * blockDim.x) {
        const double2 v = __ldg(r_hi + off + i);
        const double n2 = v.x * v.x + v.y * v.y;
        val[0] += n2;
        val[1] = fmax(val[1], sqrt(n2));
    }
    __shared__ double s_vals[kMaxRedVals];
    const bool mx[2] = {false, true};
    if (block_reduce_arrive<double, 2>(a.red, val, a.n, mx, s_vals))
        finish_reliable(a.cg, s_vals, a.n, tol2);
}

// [h][V_h][3] <-> [h][3][V_h] per rhs (FP64 complex)
__global__ void transpose_spinor_kernel(const double2* __restrict__ in, double2* __restrict__ out,
                                        int halves, int vh, int to_soa) {
    const int k = blockIdx.y;
    const long long per = (long long)halves * vh;
    const double2* src = in + (size_t)k * per * 3;
    double2* dst = out + (size_t)k * per * 3;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < per;
         i += (long long)gridDim.x * blockDim.x) {
        const long long hb = i / vh, h = i - hb * vh;
        const size_t base = (size_t)hb * vh * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t aos = base + 3 * (size_t)h + c, soa = base + (size_t)c * vh + h;
            if (to_soa)
                dst[soa] = src[aos];
            else
                dst[aos] = src[soa];
        }
    }
}

dim3 blas_grid(long long chunks, int n) {
    long long b = (chunks + kThreads - 1) / kThreads;
    // about 8 resident blocks per SM in total, shared by the n rhs
    long long cap = (8ll * device_sm_count() + n - 1) / n;
    if (cap < 1) cap = 1;
    if (b > cap) b = cap;
    if (b > kMaxRedBlocks) b = kMaxRedBlocks;
    if (b < 1) b = 1;
    return dim3((unsigned)b, (unsigned)n);
}

template <typename S>
constexpr int vec_n() {
    return Vec<S>::N;
}

}  // namespace

#define HISQ_PREC_SWITCH(prec, CALL)                  \
    switch (prec) {                                   \
        case HISQ_F64: { using S = double; CALL; break; } \
        case HISQ_F32: { using S = float; CALL; break; }  \
        case HISQ_F16: { using S = __half; CALL; break; } \
        default: return cudaErrorInvalidValue;        \
    }

cudaError_t launch_cg_update_r(const BlasArgs& a, int prec, void* r, const void* Ap, cudaStream_t s) {
    HISQ_PREC_SWITCH(prec, (update_r_kernel<S><<<blas_grid(a.len / vec_n<S>(), a.n), kThreads, 0, s>>>(
                                a, r, Ap)));
    return cudaGetLastError();
}

cudaError_t launch_cg_update_px(const BlasArgs& a, int prec, void* x, const void* r, void* p,
                                cudaStream_t s) {
    HISQ_PREC_SWITCH(prec, (update_px_kernel<S><<<blas_grid(a.len / vec_n<S>(), a.n), kThreads, 0, s>>>(
                                a, x, r, p)));
    return cudaGetLastError();
}

cudaError_t launch_accum_solution(const BlasArgs& a, int prec, double2* x_hi, void* x_lo,
                                  cudaStream_t s) {
    HISQ_PREC_SWITCH(prec, (accum_kernel<S><<<blas_grid(a.len / vec_n<S>(), a.n), kThreads, 0, s>>>(
                                a, x_hi, x_lo)));
    return cudaGetLastError();
}

cudaError_t launch_dot_alpha(const BlasArgs& a, int prec, const void* p, const void* Ap,
                             cudaStream_t s) {
    HISQ_PREC_SWITCH(prec, (dot_alpha_kernel<S><<<blas_grid(a.len / vec_n<S>(), a.n), kThreads, 0, s>>>(
                                a, p, Ap)));
    return cudaGetLastError();
}

cudaError_t launch_residual_norm(const BlasArgs& a, const double2* r_hi, double tol2, cudaStream_t s) {
    residual_norm_kernel<<<blas_grid(a.len, a.n), kThreads, 0, s>>>(a, r_hi, tol2);
    return cudaGetLastError();
}

cudaError_t launch_transpose_spinor(const double2* in, double2* out, int n, int halves, int vh,
                                    int to_soa, cudaStream_t s) {
    transpose_spinor_kernel<<<blas_grid((long long)halves * vh, n), kThreads, 0, s>>>(in, out, halves, vh,
                                                                                     to_soa);
    return cudaGetLastError();
}

cudaError_t launch_norm_bb(const BlasArgs& a, const double2* b, cudaStream_t s) {
    norm_bb_kernel<<<blas_grid(a.len, a.n), kThreads, 0, s>>>(a, b);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kThreads) keep_best_kernel(BlasArgs a, const double2* x, double2* xb) {
    const int k = blockIdx.y;
    if (!a.cg->keep[k]) return;
    const long long off = (long long)k * a.len;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.len;
         i += (long long)gridDim.x * blockDim.x)
        xb[off + i] = x[off + i];
}

cudaError_t launch_keep_best(const BlasArgs& a, const double2* x, double2* x_best, cudaStream_t s) {
    keep_best_kernel<<<blas_grid(a.len, a.n), kThreads, 0, s>>>(a, x, x_best);
    return cudaGetLastError();
}

cudaError_t launch_copy_residual(const BlasArgs& a, const double2* b, double2* r_hi, double tol2,
                                 cudaStream_t s) {
    copy_residual_kernel<<<blas_grid(a.len, a.n), kThreads, 0, s>>>(a, b, r_hi, tol2);
    return cudaGetLastError();
}

cudaError_t launch_reliable_rescale(const BlasArgs& a, int prec, const double2* r_hi, void* r_lo,
                                    void* p_lo, int reset_p, cudaStream_t s) {
    HISQ_PREC_SWITCH(prec, (rescale_kernel<S><<<blas_grid(a.len / vec_n<S>(), a.n), kThreads, 0, s>>>(
                                a, r_hi, r_lo, p_lo, reset_p)));
    return cudaGetLastError();
}

}  // namespace hisq
