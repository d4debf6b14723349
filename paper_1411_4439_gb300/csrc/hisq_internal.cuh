// Internal declarations shared by the CUDA translation units of libhisq.
//
// Data layout in HBM (all site-major, so consecutive threads touch
// consecutive addresses):
//   links   [parity][mu][complex component c][V_h]  of double2 / float2 / half2
//           c < 9 (R18), 6 (R12: rows 1-2) or 7 (R14: rows 1-2 and z)
//   spinors [V_h][3] complex per rhs (the ABI layout), one pointer per rhs
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "hisq.h"

namespace hisq {

constexpr int kMaxRhs = 16;
constexpr int kMaxRedVals = 2 * kMaxRhs;   // per-rhs norm and max
constexpr int kMaxRedBlocks = 4096;         // partial-sum slots per reduction

// ---------------------------------------------------------------------------
// Geometry of the checkerboarded lattice
// ---------------------------------------------------------------------------
struct Geom {
    int L[4];     // Lx, Ly, Lz, Lt
    int hx;       // Lx / 2 : half sites per x row
    int vh;       // V / 2
    int sy;       // half-index stride of y: hx
    int sz;       // half-index stride of z: hx * Ly
    int st;       // half-index stride of t: hx * Ly * Lz
};

// ---------------------------------------------------------------------------
// Storage precision traits
// ---------------------------------------------------------------------------
template <typename S> struct Traits;
template <> struct Traits<double> {
    using C = double2;     // stored complex
    using R = double;      // arithmetic
    using RC = double2;    // arithmetic complex
    static constexpr int prec = HISQ_F64;
};
template <> struct Traits<float> {
    using C = float2;
    using R = float;
    using RC = float2;
    static constexpr int prec = HISQ_F32;
};
template <> struct Traits<__half> {
    using C = __half2;
    using R = float;
    using RC = float2;
    static constexpr int prec = HISQ_F16;
};

// 16-bit link storage: each real is a signed 16-bit integer q with value
// q * scale_c, one scale per stored complex component c of a field (the
// largest |Re|, |Im| of that component over the field / 32767). Links have a
// known bounded range, so this keeps 2^-15 of the range where IEEE half keeps
// 2^-11 of each value.
struct Fx16 {};
template <> struct Traits<Fx16> {
    using C = short2;
    using R = float;
    using RC = float2;
    static constexpr int prec = HISQ_F16;
};

// One stored link component in arithmetic precision; sc is the component's
// scale (used by the 16-bit fixed-point storage only).
__device__ __forceinline__ double2 link_elem(double2 v, float) { return v; }
__device__ __forceinline__ float2 link_elem(float2 v, float) { return v; }
__device__ __forceinline__ float2 link_elem(__half2 v, float) { return __half22float2(v); }
__device__ __forceinline__ float2 link_elem(short2 v, float sc) {
    return make_float2((float)v.x * sc, (float)v.y * sc);
}

// Link slab layout of one (parity, mu) block of nc stored components. FP32
// and 16-bit storage keep components (2p, 2p+1) of a site side by side, so a
// thread reads two of them with one 16- or 8-byte load: [nc/2 pairs][V_h]
// then [V_h] of the last component when nc is odd. FP64 keeps [nc][V_h]
// (one double2 is already 16 bytes).
template <typename LC> struct LinkPair { static constexpr bool paired = false; };
template <> struct LinkPair<float2> {
    static constexpr bool paired = true;
    using V = float4;
};
template <> struct LinkPair<short2> {
    static constexpr bool paired = true;
    using V = short4;
};

__device__ __forceinline__ void split_pair(const float4& w, float2& a, float2& b) {
    a = make_float2(w.x, w.y);
    b = make_float2(w.z, w.w);
}
__device__ __forceinline__ void split_pair(const short4& w, short2& a, short2& b) {
    a = make_short2(w.x, w.y);
    b = make_short2(w.z, w.w);
}

// Offset (in stored complex numbers) of component c of site idx in a block.
template <typename LC>
__host__ __device__ __forceinline__ size_t link_offset(int c, int nc, long long vh, long long idx) {
    if (!LinkPair<LC>::paired) return (size_t)c * vh + idx;
    const int np = nc & ~1;
    return c < np ? ((size_t)(c >> 1) * vh + idx) * 2 + (c & 1) : (size_t)np * vh + idx;
}

// Components [0, NC) of the link of site idx from a block, streaming loads.
template <typename LC, int NC, int NL>
__device__ __forceinline__ void load_link_raw(LC (&l)[NL], const LC* __restrict__ block, int vh, int idx) {
    static_assert(NC <= NL, "link buffer too small");
    if constexpr (LinkPair<LC>::paired) {
        using V = typename LinkPair<LC>::V;
        const V* pb = reinterpret_cast<const V*>(block);
#pragma unroll
        for (int p = 0; p < NC / 2; ++p) split_pair(__ldcs(pb + (size_t)p * vh + idx), l[2 * p], l[2 * p + 1]);
        if constexpr (NC & 1) l[NC - 1] = __ldcs(block + (size_t)(NC - 1) * vh + idx);
    } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) l[c] = __ldcs(block + (size_t)c * vh + idx);
    }
}

__device__ __forceinline__ double2 ld_c(const double2* p) { return __ldg(p); }
__device__ __forceinline__ float2 ld_c(const float2* p) { return __ldg(p); }
__device__ __forceinline__ float2 ld_c(const __half2* p) { return __half22float2(__ldg(p)); }

// The value a store of v through p leaves in memory, in arithmetic precision.
__device__ __forceinline__ double2 stored_value(double2 v, const double2*) { return v; }
__device__ __forceinline__ float2 stored_value(float2 v, const float2*) { return v; }
__device__ __forceinline__ float2 stored_value(float2 v, const __half2*) {
    return __half22float2(__float22half2_rn(v));
}


__device__ __forceinline__ void st_c(double2* p, double2 v) { *p = v; }
__device__ __forceinline__ void st_c(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void st_c(__half2* p, float2 v) { *p = __float22half2_rn(v); }

// ---------------------------------------------------------------------------
// Reductions: per-block partials and a last-block finish in fixed order
// ---------------------------------------------------------------------------
struct RedScratch {
    double* partials;        // [kMaxRedVals][kMaxRedBlocks]
    unsigned int* counter;   // zero between launches; the last block resets it
};

// CG scalars live on the device so that no iteration needs the host.
struct CgScalars {
    double rr[kMaxRhs];        // iterated |r|^2 in the scaled low-precision units
    double pAp[kMaxRhs];
    double alpha[kMaxRhs];
    double beta[kMaxRhs];
    double rr_rel[kMaxRhs];    // |r|^2 right after the last reliable update (scaled)
    double bb[kMaxRhs];        // |b|^2, FP64
    double rr_true[kMaxRhs];   // |b - A x|^2 at the last reliable update, FP64
    double rmax[kMaxRhs];      // max |component| of that residual
    double scale[kMaxRhs];     // low-precision vectors hold scale * true vector
    double scale_old[kMaxRhs];
    int active[kMaxRhs];       // 1 while rhs k is iterating
    int frozen[kMaxRhs];       // 1: residual fell below freeze2 * rr_rel; skip until the next reliable update
    int stall[kMaxRhs];        // 1: <p,Ap> <= 0 in low precision; this iteration restarts p = r
    int restarts[kMaxRhs];     // number of such restarts in this solve
    int reset_p[kMaxRhs];      // 1: the reliable update restarts p = r (true and iterated residual disagree)
    double freeze2;            // squared residual drop that freezes an rhs (precision safety net)
    double alpha_max;          // alpha above this bound (1/lambda_min) means lost precision: restart
    int flags;                 // kFlagBreakdown | kFlagNaN
    // state of the device-driven iteration loop (one graph launch per solve)
    int iter;                  // iterations run
    int since_rel;             // iterations since the last reliable update
    int reliable;              // reliable updates done
    int need;                  // the last decision asked for a reliable update
    int result;                // HISQ_OK, or HISQ_ENOCONV / HISQ_EBREAKDOWN decided on the device
    int seen_restarts[kMaxRhs];
    int restarted[kMaxRhs];    // restarts counted since the previous decision
    int was[kMaxRhs];          // active before the pending reliable update
    int bad_updates[kMaxRhs];  // consecutive restarted updates without FP64 progress
    int iters_k[kMaxRhs];      // iteration at which rhs k converged
    double before[kMaxRhs];    // rr_true before the pending reliable update
    // the lowest FP64 residual seen and whether the last one set it (the
    // solution at that point is kept for a solve that ends without converging)
    double rr_best[kMaxRhs];
    int have_best[kMaxRhs];
    int keep[kMaxRhs];
};
constexpr int kFlagBreakdown = 1;
constexpr int kFlagNaN = 2;
constexpr int kFlagTimeout = 4;   // a bounded device-side wait gave up

enum RedMode : int {
    RED_NONE = 0,
    RED_DOT_XW = 1,      // Re <x, w> per rhs (x = epilogue input, w = output)
    RED_NORM_MAX_W = 2   // |w|^2 and max |w_i| per rhs
};

enum Finish : int {
    FIN_STORE = 0,       // write the reduced values to red_out
    FIN_CG_ALPHA = 1,    // pAp -> alpha = rr / pAp (masked)
    FIN_RELIABLE = 2,    // FP64 true residual -> convergence, next scale
    FIN_CG_BETA = 3,     // rr' -> beta = rr' / rr (masked)
    FIN_BB = 4,          // |b|^2 -> bb, active = (bb > 0), scale = 1
    FIN_RR = 5,          // |r_lo|^2 after a reliable update -> rr, rr_rel
};

// ---------------------------------------------------------------------------
// Dslash launch arguments
// ---------------------------------------------------------------------------
struct DslashArgs {
    Geom g;
    int parity;                         // output parity
    int nrhs;                           // rhs in this launch
    const void* U;                      // packed links, [2][4][ncomp][vh]
    const void* N;
    const void* in[kMaxRhs];            // opposite-parity inputs
    void* out[kMaxRhs];                 // outputs
    const void* x[kMaxRhs];             // epilogue x (output parity), or null
    const void* y[kMaxRhs];             // epilogue y (output parity), or null
    double cx, cd;                      // out = [y] + cx * x + cd * (D in)
    double ft1, bt1, ft3, bt3;          // temporal hop factors e^{+mu}, e^{-mu}, e^{3mu}, e^{-3mu}
    int has_mu;                         // 1 if any factor differs from 1
    int t_only;                         // 1: temporal hops only (d D / d mu)
    int l2_prefetch;                    // 1: bulk-prefetch each tile's links into L2
    int* status;                        // bounded waits that give up OR kFlagTimeout here (or null)
    double r12_inv_scale;               // 1 / s for R12 fat links
    float lscale_u[9];                  // per-component scales of 16-bit fat links
    float lscale_n[9];                  // per-component scales of 16-bit Naik links
    int red_mode;
    int finish;
    double tol2;                        // FIN_RELIABLE: tol^2
    RedScratch red;
    double* red_out;                    // [vals] for FIN_STORE
    CgScalars* cg;                      // for FIN_CG_ALPHA / FIN_RELIABLE
};

// Epilogue kinds (template parameter of the Dslash kernel)
enum Epi : int { EPI_NONE = 0, EPI_X = 1, EPI_XY = 2 };

// Thread mapping and spinor layout of one launch: rpt rhs per thread,
// compiled for at least minb resident 256-thread blocks per SM; kind 0 is
// the register kernel, 1 the register kernel with packed f32x2 complex
// arithmetic (FP32 arithmetic only), 2 the kernel with links staged in shared
// memory by bulk copies (FP32 arithmetic only).
// Kinds 5, 6 and 9 to 12 run on the bundle spinor layout (dslash_bundle.cuh),
// with packed f32x2 arithmetic and the next hop's link in flight: the fully
// unrolled hop loop (5), also the next hop's neighbours in flight (6), the
// compact hop loop (9), compact with the neighbours in flight (10), and the
// neighbour chunks copied into shared memory one (11) or two (12) hops ahead,
// the compact loop with the chunks staged one (13) or three (14) ahead, and
// the unrolled loop with the x/y neighbours from a shared-memory tile (15).
enum DslashKind : int {
    KIND_REG = 0, KIND_PACKED = 1, KIND_STAGED = 2, KIND_PIPE1 = 3, KIND_PIPE2 = 4,
    KIND_BUNDLE = 5, KIND_BUNDLE_SPIN = 6, KIND_BUNDLE_COMPACT = 9, KIND_BUNDLE_COMPACT_SPIN = 10,
    KIND_BUNDLE_SMEM1 = 11, KIND_BUNDLE_SMEM2 = 12, KIND_BUNDLE_CSMEM1 = 13, KIND_BUNDLE_CSMEM3 = 14,
    KIND_BUNDLE_XY = 15
};
struct DslashTune {
    int rpt;
    int minb;
    int kind;
    int layout;     // HISQ_AOS, HISQ_SOA or HISQ_BUNDLE
    int prefetch;   // bulk L2 prefetch of each tile's links
};

// Dispatch into the instantiated kernels. prec is the spinor and link storage
// precision; nrhs must be a multiple of t.rpt with nrhs / t.rpt <= 8.
cudaError_t launch_dslash(const DslashArgs& a, int prec, int ru, int rn, int epi,
                          const DslashTune& t, cudaStream_t s);
bool dslash_variant_supported(int prec, int ru, int rn, int epi);
// Built (rpt, minb, kind) mappings of a precision, and the default one for an rpt.
bool dslash_mapping_built(int prec, int rpt, int minb, int kind);
DslashTune dslash_default_tune(int prec, int rpt, int layout);
DslashTune dslash_register_tune(int prec, int rpt, int layout);
// Whether the staged-link kernel can run this lattice with `groups` groups of rpt rhs.
bool dslash_staged_ok(const Geom& g, int prec, int rpt, int groups);
// Largest rhs-per-thread value instantiated for a precision.
int dslash_max_rpt(int prec);
// Bundle layout: rhs per 16-byte chunk of a storage precision (F32: 2,
// F16: 4; 0 where there is no bundle kernel), whether a bundle mapping is
// built for a link compression pair, and the default bundle mapping for n
// rhs (rpt 0 when n does not fit the layout).
int bundle_width(int prec);
bool bundle_mapping_built(int prec, int ru, int rn, int rpt, int minb, int kind);
DslashTune dslash_bundle_tune(int prec, int n);

// Spinor layout conversion of FP64 vectors: n rhs, `halves` parity blocks of
// vh sites each; to_soa: [h][V_h][3] -> [h][3][V_h], else the reverse.
cudaError_t launch_transpose_spinor(const double2* in, double2* out, int n, int halves, int vh,
                                    int to_soa, cudaStream_t s);

// ---------------------------------------------------------------------------
// Link packing (gauge.cu)
// ---------------------------------------------------------------------------
// Pack canonical complex128 [4][V][3][3] into [2][4][ncomp][vh] of `prec`,
// with reconstruct residual max written (as ordered bits) to *err_bits.
// F16 links are 16-bit fixed point: comp_scale[c] (device, FP64) is the
// scale of stored component c (see launch_link_absmax); ignored otherwise.
cudaError_t launch_pack_links(const Geom& g, const double2* canon, int prec, int recon,
                              int hop, double r12_inv_scale, void* out,
                              unsigned long long* err_bits, const double* comp_scale,
                              cudaStream_t s);
// Largest |Re| or |Im| of every stored component (recon / 2 of them) over the
// field, as the bits of non-negative doubles OR-maximised into maxbits[c].
cudaError_t launch_link_absmax(const Geom& g, const double2* canon, int recon, int hop,
                               double r12_inv_scale, unsigned long long* maxbits, cudaStream_t s);
// Compress to double [4][V][r] and back (ABI helpers).
cudaError_t launch_compress_links(const Geom& g, const double2* canon, int recon, int hop,
                                  double r12_inv_scale, double* packed,
                                  unsigned long long* err_bits, cudaStream_t s);
cudaError_t launch_reconstruct_links(const Geom& g, const double* packed, int recon,
                                     int hop, double r12_inv_scale, double2* canon,
                                     cudaStream_t s);

// ---------------------------------------------------------------------------
// CG vector kernels (blas.cu). Vectors: one contiguous [n][vh*3] complex block.
// ---------------------------------------------------------------------------
struct BlasArgs {
    int n;               // rhs
    long long len;       // complex elements per rhs (vh * 3)
    RedScratch red;
    CgScalars* cg;
    double freeze2;      // norm_bb stores it into cg->freeze2
    double alpha_max;    // norm_bb stores it into cg->alpha_max
};
// r -= alpha Ap; rr' = |r|^2 -> beta = rr'/rr, rr = rr'
cudaError_t launch_cg_update_r(const BlasArgs& a, int prec, void* r, const void* Ap, cudaStream_t s);
// x_lo += alpha p; p = r + beta p (one pass over the old p)
cudaError_t launch_cg_update_px(const BlasArgs& a, int prec, void* x, const void* r, void* p,
                                cudaStream_t s);
// x_hi (FP64) += x_lo / scale ; x_lo = 0
cudaError_t launch_accum_solution(const BlasArgs& a, int prec, double2* x_hi, void* x_lo,
                                  cudaStream_t s);
// pAp = Re <p, Ap> -> alpha (full-lattice operator, where the Dslash epilogue
// does not see p)
cudaError_t launch_dot_alpha(const BlasArgs& a, int prec, const void* p, const void* Ap,
                             cudaStream_t s);
// |r_hi|^2 and max|r_i| with the reliable-update finish
cudaError_t launch_residual_norm(const BlasArgs& a, const double2* r_hi, double tol2,
                                 cudaStream_t s);
// |b|^2 -> bb; active = (bb > 0); scale = 1
cudaError_t launch_norm_bb(const BlasArgs& a, const double2* b, cudaStream_t s);
// r_hi = b (x0 = 0) with the reliable-update finish (rr_true, rmax, scale)
// x_best[k] = x[k] for the rhs whose last FP64 residual is their lowest (cg->keep)
cudaError_t launch_keep_best(const BlasArgs& a, const double2* x, double2* x_best, cudaStream_t s);
cudaError_t launch_copy_residual(const BlasArgs& a, const double2* b, double2* r_hi,
                                 double tol2, cudaStream_t s);
// r_lo = scale * r_hi; p_lo = reset_p ? r_lo : p_lo * scale / scale_old;
// rr = rr_rel = |r_lo|^2 (active rhs only)
cudaError_t launch_reliable_rescale(const BlasArgs& a, int prec, const double2* r_hi,
                                    void* r_lo, void* p_lo, int reset_p, cudaStream_t s);

// Bundle-layout versions (blas_bundle.cu): vectors [n / W][3][V_h] chunks of
// 16 bytes (W rhs each); a.len = 3 V_h; x_lo is FP32 [n / W][3][V_h] chunks of
// W complex numbers (real parts, then imaginary parts).
cudaError_t launch_cg_update_r_bundle(const BlasArgs& a, int prec, void* r, const void* Ap, cudaStream_t s);
cudaError_t launch_cg_update_px_bundle(const BlasArgs& a, int prec, void* x, const void* r, void* p,
                                       cudaStream_t s);
cudaError_t launch_accum_solution_bundle(const BlasArgs& a, int prec, double2* x_hi, void* x_lo, int vh,
                                         cudaStream_t s);
cudaError_t launch_reliable_rescale_bundle(const BlasArgs& a, int prec, const double2* r_hi, void* r_lo,
                                           void* p_lo, int reset_p, int vh, cudaStream_t s);
struct BundlePtrs {
    const double2* p[kMaxRhs];
};
// n FP64 [V_h][3] vectors <-> one bundle of storage prec (pack rounds to it).
cudaError_t launch_bundle_pack(const BundlePtrs& ptrs, int n, int prec, long long vh, void* bundle,
                               cudaStream_t s);
cudaError_t launch_bundle_unpack(const void* bundle, const BundlePtrs& ptrs, int n, int prec, long long vh,
                                 cudaStream_t s);

// ---------------------------------------------------------------------------
// Gradients (force.cu)
// ---------------------------------------------------------------------------
struct ForcePtrs {
    const double2* a[kMaxRhs];   // full-lattice parity-blocked FP64 vectors [2][vh][3]
    const double2* b[kMaxRhs];
};
// out[mu][i] += coef * sum_k [f a_k(i) b_k(i+hop mu)^dag - (1/f) b_k(i) a_k(i+hop mu)^dag]
// with f = e^{hop mu_chem} on temporal links; out canonical complex128 [4][V][3][3].
cudaError_t launch_link_force(const Geom& g, int hop, double mu_chem, double coef, int n,
                              const ForcePtrs& ptrs, double2* out, cudaStream_t s);
// out[2k] + i out[2k+1] = <a_k, b_k> over len complex numbers, FP64, deterministic
cudaError_t launch_cdot(const ForcePtrs& vw, long long len, int n, RedScratch red, double* out,
                        cudaStream_t s);

int device_sm_count();
void record_error(const char* msg);

}  // namespace hisq
