// Link force (outer products) and FP64 complex dot products for the
// gradient of a solve with respect to the links, the mass and mu.
//
// For a loss L(x) with x = (M^dag M)^-1 b, lambda = (M^dag M)^-1 dL/dx*,
// y = M x and z = M lambda, the change of L under dM is
//   dL = -Re[ y^dag dM lambda + z^dag dM x ].
// The link U_mu(x) enters D through f U_mu(x) v(x+mu) and
// -(1/f) U_mu(x)^dag v(x) (at site x+mu), with f = e^{h mu_chem} on temporal
// links (h = 1 for U, 3 for N). The gradient of Re[a^dag dD b] with respect to
// the entries of that link (d/dRe + i d/dIm) is
//   F(a, b) = f a(x) b(x+h mu)^dag - (1/f) b(x) a(x+h mu)^dag .
#include "hisq_internal.cuh"
#include "reduce.cuh"

namespace hisq {

namespace {

__global__ void link_force_kernel(Geom g, int hop, double mu_chem, double coef, int n,
                                  ForcePtrs ptrs, double2* __restrict__ out) {
    const long long V = 2ll * g.vh;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < 4 * V;
         w += (long long)gridDim.x * blockDim.x) {
        const int mu = (int)(w / V);
        const long long i = w - mu * V;
        int c[4];
        long long r = i;
        c[0] = (int)(r % g.L[0]);
        r /= g.L[0];
        c[1] = (int)(r % g.L[1]);
        r /= g.L[1];
        c[2] = (int)(r % g.L[2]);
        c[3] = (int)(r / g.L[2]);
        const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
        c[mu] = (c[mu] + hop) % g.L[mu];
        const long long j = c[0] + (long long)g.L[0] * (c[1] + (long long)g.L[1] * (c[2] + (long long)g.L[2] * c[3]));
        const int parj = par ^ (hop & 1);
        const long long si = ((long long)par * g.vh + (i >> 1)) * 3;
        const long long sj = ((long long)parj * g.vh + (j >> 1)) * 3;
        double ff = 1.0, fb = 1.0;
        if (mu == 3) {
            ff = exp(hop * mu_chem);
            fb = exp(-hop * mu_chem);
        }
        double2 F[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) F[e] = make_double2(0.0, 0.0);
        for (int k = 0; k < n; ++k) {
            const double2* a = ptrs.a[k];
            const double2* b = ptrs.b[k];
            double2 ai[3], bj[3], bi[3], aj[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                ai[q] = a[si + q];
                bj[q] = b[sj + q];
                bi[q] = b[si + q];
                aj[q] = a[sj + q];
            }
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    // ff * a_p(x) conj(b_q(x+h mu)) - fb * b_p(x) conj(a_q(x+h mu))
                    const double re1 = ai[p].x * bj[q].x + ai[p].y * bj[q].y;
                    const double im1 = ai[p].y * bj[q].x - ai[p].x * bj[q].y;
                    const double re2 = bi[p].x * aj[q].x + bi[p].y * aj[q].y;
                    const double im2 = bi[p].y * aj[q].x - bi[p].x * aj[q].y;
                    F[3 * p + q].x += ff * re1 - fb * re2;
                    F[3 * p + q].y += ff * im1 - fb * im2;
                }
        }
        double2* o = out + w * 9;
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            double2 v = o[e];
            v.x += coef * F[e].x;
            v.y += coef * F[e].y;
            o[e] = v;
        }
    }
}

constexpr int kDotThreads = 256;

// out[2k] + i out[2k+1] = <v_k, w_k> = sum conj(v) w, FP64, fixed order
__global__ void __launch_bounds__(kDotThreads) cdot_kernel(ForcePtrs vw, long long len, int n,
                                                           RedScratch red, double* out) {
    const int k = blockIdx.y;
    double val[2] = {0.0, 0.0};
    const double2* vk = vw.a[k];
    const double2* wk = vw.b[k];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
         i += (long long)gridDim.x * blockDim.x) {
        const double2 a = vk[i], b = wk[i];
        val[0] = fma(a.x, b.x, fma(a.y, b.y, val[0]));
        val[1] = fma(a.x, b.y, fma(-a.y, b.x, val[1]));
    }
    __shared__ double s_w[2][kDotThreads / 32];
    __shared__ double s_vals[kMaxRedVals];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = 0; j < 2; ++j) {
        const double t = warp_sum(val[j]);
        if (lane == 0) s_w[j][warp] = t;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double acc = 0.0;
        for (int q = 0; q < kDotThreads / 32; ++q) acc += s_w[threadIdx.x][q];
        red.partials[(size_t)(k * 2 + threadIdx.x) * kMaxRedBlocks + blockIdx.x] = acc;
    }
    if (!last_block_arrive(red.counter, gridDim.x * gridDim.y)) return;
    finish_values(red, 2 * n, gridDim.x, [](int) { return false; }, s_vals);
    if (threadIdx.x < 2 * n) out[threadIdx.x] = s_vals[threadIdx.x];
}

}  // namespace

cudaError_t launch_link_force(const Geom& g, int hop, double mu_chem, double coef, int n,
                              const ForcePtrs& ptrs, double2* out, cudaStream_t s) {
    long long blocks = (8ll * g.vh + 255) / 256;
    const long long cap = 16ll * device_sm_count();
    if (blocks > cap) blocks = cap;
    link_force_kernel<<<(unsigned)blocks, 256, 0, s>>>(g, hop, mu_chem, coef, n, ptrs, out);
    return cudaGetLastError();
}

cudaError_t launch_cdot(const ForcePtrs& vw, long long len, int n, RedScratch red, double* out,
                        cudaStream_t s) {
    long long b = (len + kDotThreads - 1) / kDotThreads;
    long long cap = (8ll * device_sm_count() + n - 1) / n;
    if (b > cap) b = cap;
    if (b > kMaxRedBlocks) b = kMaxRedBlocks;
    if (b < 1) b = 1;
    cdot_kernel<<<dim3((unsigned)b, (unsigned)n), kDotThreads, 0, s>>>(vw, len, n, red, out);
    return cudaGetLastError();
}

}  // namespace hisq
