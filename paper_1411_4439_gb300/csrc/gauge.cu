// Link packing and reconstruction (Sec. 1: links stored in fewer reals).
//
// Canonical input: complex128 [4][V][3][3], lexicographic site order.
// Internal output: per (parity, mu) block the stored components of V_h
// sites in the storage precision (FP64, FP32, or 16-bit fixed point with one
// scale per stored component): FP64 as [component][V_h]; FP32 and 16-bit as
// [component pair][V_h] (two components of a site in one 16- or 8-byte word)
// and the odd last component as [V_h] (link_offset). A warp's 32 consecutive
// sites read each word with one coalesced access.
//   R18: 9 components; R14: rows 1-2 and z with row3 = z conj(row1 x row2);
//   R12: rows 1-2 with row3 = (sigma/s) conj(row1 x row2).
// Every packed link is reconstructed here in FP64 and compared with the
// input; the largest deviation is returned so the loader can reject links
// that the chosen compression cannot represent.
#include "hisq_internal.cuh"

namespace hisq {

namespace {

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zsub(double2 a, double2 b) {
    return make_double2(a.x - b.x, a.y - b.y);
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double zabs(double2 a) { return sqrt(a.x * a.x + a.y * a.y); }

// conj(a x b) for rows a = m[0..2], b = m[3..5]
__device__ __forceinline__ void cross_conj(const double2* m, double2* c) {
    c[0] = zconj(zsub(zmul(m[1], m[5]), zmul(m[2], m[4])));
    c[1] = zconj(zsub(zmul(m[2], m[3]), zmul(m[0], m[5])));
    c[2] = zconj(zsub(zmul(m[0], m[4]), zmul(m[1], m[3])));
}

struct Site {
    int x, y, z, t, parity, h;
};

__device__ __forceinline__ Site site_of(const Geom& g, long long i) {
    Site s;
    long long r = i;
    s.x = (int)(r % g.L[0]);
    r /= g.L[0];
    s.y = (int)(r % g.L[1]);
    r /= g.L[1];
    s.z = (int)(r % g.L[2]);
    s.t = (int)(r / g.L[2]);
    s.parity = (s.x + s.y + s.z + s.t) & 1;
    s.h = (int)(i >> 1);
    return s;
}

// staggered sign eta_mu(x) * bc(x, mu) of the link x -> x + hop mu (antiperiodic t)
__device__ __forceinline__ int staggered_sign(const Geom& g, const Site& s, int mu, int hop) {
    int e = 0;
    if (mu >= 1) e += s.x;
    if (mu >= 2) e += s.y;
    if (mu >= 3) e += s.z;
    int sg = (e & 1) ? -1 : 1;
    if (mu == 3 && s.t + hop >= g.L[3]) sg = -sg;
    return sg;
}

// Compute the `ncomp` stored complex numbers of one link and its reconstruct error.
__device__ __forceinline__ double encode(const double2* m, int recon, int sign, double inv_s,
                                         double2* enc) {
#pragma unroll
    for (int c = 0; c < 6; ++c) enc[c] = m[c];
    double err = 0.0;
    if (recon == 18) {
        enc[6] = m[6];
        enc[7] = m[7];
        enc[8] = m[8];
        return 0.0;
    }
    double2 cc[3];
    cross_conj(m, cc);
    double2 f;
    if (recon == 14) {
        int k = 0;
        double best = zabs(cc[0]);
        if (zabs(cc[1]) > best) { k = 1; best = zabs(cc[1]); }
        if (zabs(cc[2]) > best) { k = 2; best = zabs(cc[2]); }
        if (best > 0.0) {
            // z = row3_k / cc_k
            const double d = cc[k].x * cc[k].x + cc[k].y * cc[k].y;
            f = make_double2((m[6 + k].x * cc[k].x + m[6 + k].y * cc[k].y) / d,
                             (m[6 + k].y * cc[k].x - m[6 + k].x * cc[k].y) / d);
        } else {
            f = make_double2(0.0, 0.0);
        }
        enc[6] = f;
    } else {
        f = make_double2(sign > 0 ? inv_s : -inv_s, 0.0);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double2 r3 = zmul(f, cc[c]);
        err = fmax(err, zabs(zsub(r3, m[6 + c])));
    }
    return err;
}

template <typename C> __device__ __forceinline__ C narrow(double2 v);
template <> __device__ __forceinline__ double2 narrow<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 narrow<float2>(double2 v) {
    return make_float2((float)v.x, (float)v.y);
}
template <> __device__ __forceinline__ __half2 narrow<__half2>(double2 v) {
    return __floats2half2_rn((float)v.x, (float)v.y);
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* bits, double v) {
    if (!(v >= 0.0)) v = __longlong_as_double(0x7ff0000000000000ll);   // NaN -> +inf
    atomicMax(bits, (unsigned long long)__double_as_longlong(v));
}

// 16-bit fixed point: round to nearest of v / scale, clamped to +-32767
__device__ __forceinline__ short quantize(double v, double inv_scale) {
    double q = rint(v * inv_scale);
    q = fmin(fmax(q, -32767.0), 32767.0);
    return (short)q;
}

template <typename C>
__device__ __forceinline__ C store_comp(double2 v, const double* comp_scale, int c) {
    return narrow<C>(v);
}
template <>
__device__ __forceinline__ short2 store_comp<short2>(double2 v, const double* comp_scale, int c) {
    const double sc = comp_scale[c];
    const double inv = sc > 0.0 ? 1.0 / sc : 0.0;
    return make_short2(quantize(v.x, inv), quantize(v.y, inv));
}

template <typename C>
__global__ void pack_kernel(Geom g, const double2* __restrict__ canon, int recon, int hop,
                            double inv_s, C* __restrict__ out, unsigned long long* err_bits,
                            const double* __restrict__ comp_scale) {
    const int nc = recon / 2;
    const long long V = 2ll * g.vh;
    double worst = 0.0;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < 4 * V;
         w += (long long)gridDim.x * blockDim.x) {
        const int mu = (int)(w / V);
        const long long i = w - mu * V;
        const Site s = site_of(g, i);
        double2 m[9], enc[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) m[c] = canon[w * 9 + c];
        const int sg = (recon == 12) ? staggered_sign(g, s, mu, hop) : 1;
        worst = fmax(worst, encode(m, recon, sg, inv_s, enc));
        C* block = out + ((size_t)(s.parity * 4 + mu) * nc) * g.vh;
        for (int c = 0; c < nc; ++c) block[link_offset<C>(c, nc, g.vh, s.h)] = store_comp<C>(enc[c], comp_scale, c);
    }
    if (err_bits != nullptr) atomic_max_nonneg(err_bits, worst);
}

__global__ void absmax_kernel(Geom g, const double2* __restrict__ canon, int recon, int hop,
                              double inv_s, unsigned long long* maxbits) {
    const int nc = recon / 2;
    const long long V = 2ll * g.vh;
    double mx[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) mx[c] = 0.0;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < 4 * V;
         w += (long long)gridDim.x * blockDim.x) {
        const int mu = (int)(w / V);
        const Site s = site_of(g, w - mu * V);
        double2 m[9], enc[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) m[c] = canon[w * 9 + c];
        const int sg = (recon == 12) ? staggered_sign(g, s, mu, hop) : 1;
        encode(m, recon, sg, inv_s, enc);
#pragma unroll
        for (int c = 0; c < 9; ++c)
            if (c < nc) mx[c] = fmax(mx[c], fmax(fabs(enc[c].x), fabs(enc[c].y)));
    }
    for (int c = 0; c < nc; ++c) atomic_max_nonneg(maxbits + c, mx[c]);
}

__global__ void compress_kernel(Geom g, const double2* __restrict__ canon, int recon, int hop,
                                double inv_s, double* __restrict__ packed,
                                unsigned long long* err_bits) {
    const int nc = recon / 2;
    const long long V = 2ll * g.vh;
    double worst = 0.0;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < 4 * V;
         w += (long long)gridDim.x * blockDim.x) {
        const int mu = (int)(w / V);
        const Site s = site_of(g, w - mu * V);
        double2 m[9], enc[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) m[c] = canon[w * 9 + c];
        const int sg = (recon == 12) ? staggered_sign(g, s, mu, hop) : 1;
        worst = fmax(worst, encode(m, recon, sg, inv_s, enc));
        for (int c = 0; c < nc; ++c) {
            packed[w * recon + 2 * c] = enc[c].x;
            packed[w * recon + 2 * c + 1] = enc[c].y;
        }
    }
    if (err_bits != nullptr) atomic_max_nonneg(err_bits, worst);
}

__global__ void reconstruct_kernel(Geom g, const double* __restrict__ packed, int recon, int hop,
                                   double inv_s, double2* __restrict__ canon) {
    const int nc = recon / 2;
    const long long V = 2ll * g.vh;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < 4 * V;
         w += (long long)gridDim.x * blockDim.x) {
        const int mu = (int)(w / V);
        const Site s = site_of(g, w - mu * V);
        double2 m[9];
        for (int c = 0; c < nc; ++c)
            m[c] = make_double2(packed[w * recon + 2 * c], packed[w * recon + 2 * c + 1]);
        if (recon != 18) {
            double2 cc[3], f;
            cross_conj(m, cc);
            if (recon == 14) {
                f = m[6];
            } else {
                const int sg = staggered_sign(g, s, mu, hop);
                f = make_double2(sg > 0 ? inv_s : -inv_s, 0.0);
            }
            for (int c = 0; c < 3; ++c) m[6 + c] = zmul(f, cc[c]);
        }
        for (int c = 0; c < 9; ++c) canon[w * 9 + c] = m[c];
    }
}

unsigned grid_for(long long work) {
    long long b = (work + 255) / 256;
    const long long cap = 32ll * device_sm_count();
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace

cudaError_t launch_pack_links(const Geom& g, const double2* canon, int prec, int recon, int hop,
                              double r12_inv_scale, void* out, unsigned long long* err_bits,
                              const double* comp_scale, cudaStream_t s) {
    const unsigned grid = grid_for(8ll * g.vh);
    switch (prec) {
        case HISQ_F64:
            pack_kernel<double2><<<grid, 256, 0, s>>>(g, canon, recon, hop, r12_inv_scale,
                                                      (double2*)out, err_bits, comp_scale);
            break;
        case HISQ_F32:
            pack_kernel<float2><<<grid, 256, 0, s>>>(g, canon, recon, hop, r12_inv_scale,
                                                     (float2*)out, err_bits, comp_scale);
            break;
        case HISQ_F16:
            if (comp_scale == nullptr) return cudaErrorInvalidValue;
            pack_kernel<short2><<<grid, 256, 0, s>>>(g, canon, recon, hop, r12_inv_scale,
                                                     (short2*)out, err_bits, comp_scale);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_link_absmax(const Geom& g, const double2* canon, int recon, int hop,
                               double r12_inv_scale, unsigned long long* maxbits, cudaStream_t s) {
    absmax_kernel<<<grid_for(8ll * g.vh), 256, 0, s>>>(g, canon, recon, hop, r12_inv_scale, maxbits);
    return cudaGetLastError();
}

cudaError_t launch_compress_links(const Geom& g, const double2* canon, int recon, int hop,
                                  double r12_inv_scale, double* packed,
                                  unsigned long long* err_bits, cudaStream_t s) {
    compress_kernel<<<grid_for(8ll * g.vh), 256, 0, s>>>(g, canon, recon, hop, r12_inv_scale,
                                                         packed, err_bits);
    return cudaGetLastError();
}

cudaError_t launch_reconstruct_links(const Geom& g, const double* packed, int recon, int hop,
                                     double r12_inv_scale, double2* canon, cudaStream_t s) {
    reconstruct_kernel<<<grid_for(8ll * g.vh), 256, 0, s>>>(g, packed, recon, hop,
                                                            r12_inv_scale, canon);
    return cudaGetLastError();
}

}  // namespace hisq
