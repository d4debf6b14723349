// Multi-rhs Dslash on the rhs-interleaved bundle layout (Eq. 3 on a bundle,
// Eq. 4), the kernel of the mixed-precision CG.
//
// Bundle layout: 16-byte chunks, each holding one colour of W consecutive rhs
// at one site, real parts first:
//   FP32 storage (W = 2): float4  (re_k, re_k+1, im_k, im_k+1)
//   FP16 storage (W = 4): 8 halves (re_k .. re_k+3, im_k .. im_k+3)
// Chunk (group g = k / W, colour c, site h) is element (3 g + c) V_h + h of
// the buffer. A warp of 32 consecutive sites reads 512 contiguous bytes per
// chunk row, for the neighbours of every hop (the y, z, t hops shift the row
// by a constant; the x hops stay inside it).
//
// Thread mapping: one output site and R rhs per thread (R / W chunks per
// colour), blockDim.y groups of R rhs sharing the sites of a block. Per hop
// the thread loads one link (reconstructed in registers) and 3 R / W chunks.
//
// Arithmetic: with PK the rhs are processed in pairs by packed FP32
// instructions (fma.rn.f32x2): for a link element m = (mr, mi) and the pair
// vectors VR = (re_k, re_k+1), VI = (im_k, im_k+1)
//   forward  acc += m v      : AR += (mr,mr) VR + (-mi,-mi) VI ; AI += (mr,mr) VI + (mi,mi) VR
//   backward acc -= m^dag v  : AR += (-mr,-mr) VR + (-mi,-mi) VI ; AI += (-mr,-mr) VI + (mi,mi) VR
// so one link element serves R / 2 pairs with 3 packed operands. Without PK
// every rhs takes scalar FMAs. Accumulation is FP32 in both.
//
// Hop loops (one per kernel variant):
//   BundleHops                all 16 hops unrolled; the link of hop e + LD and
//                             the neighbour chunks of hop e + SD (LD, SD in
//                             {0, 1}) are loaded before hop e is multiplied;
//   BundleHopsCompact         the direction as a runtime loop (a quarter of
//                             the code: no instruction-fetch stalls);
//   BundleHopsStaged          unrolled, the neighbour chunks copied into
//                             shared memory D hops ahead by per-thread cp.async;
//   BundleHopsCompactStaged   the compact loop with that staging (D = 1 or 3),
//                             the default for FP16 storage.
// Sites are visited plane by plane with the longer of z and t slow
// (visit_site), so the neighbour chunks stay in L2 between their readers.
#pragma once

#include "dslash_impl.cuh"

namespace hisq {

template <typename S> struct Bundle;
template <> struct Bundle<float> {
    static constexpr int W = 2;
};
template <> struct Bundle<__half> {
    static constexpr int W = 4;
};

// Pair j of a chunk as packed (re, re') and (im, im').
__device__ __forceinline__ void chunk_pair(const uint4& c, int j, f2x& vr, f2x& vi, float) {
    // FP32: one pair per chunk
    vr = pk2(__uint_as_float(c.x), __uint_as_float(c.y));
    vi = pk2(__uint_as_float(c.z), __uint_as_float(c.w));
}
__device__ __forceinline__ float2 h2f(unsigned u) {
    __half2 h;
    memcpy(&h, &u, 4);
    return __half22float2(h);
}
__device__ __forceinline__ void chunk_pair(const uint4& c, int j, f2x& vr, f2x& vi, __half) {
    const float2 r = h2f(j ? c.y : c.x);
    const float2 i = h2f(j ? c.w : c.z);
    vr = pk2(r.x, r.y);
    vi = pk2(i.x, i.y);
}

// rhs l of a chunk as a complex number (scalar arithmetic path).
__device__ __forceinline__ float2 chunk_rhs(const uint4& c, int l, float) {
    return l == 0 ? make_float2(__uint_as_float(c.x), __uint_as_float(c.z))
                  : make_float2(__uint_as_float(c.y), __uint_as_float(c.w));
}
__device__ __forceinline__ float2 chunk_rhs(const uint4& c, int l, __half) {
    const float2 r = h2f(l < 2 ? c.x : c.y);
    const float2 i = h2f(l < 2 ? c.z : c.w);
    return (l & 1) ? make_float2(r.y, i.y) : make_float2(r.x, i.x);
}

// Chunk holding rhs values w[0 .. W) of one colour.
__device__ __forceinline__ uint4 make_chunk(const float2 (&w)[2], float) {
    return make_uint4(__float_as_uint(w[0].x), __float_as_uint(w[1].x), __float_as_uint(w[0].y),
                      __float_as_uint(w[1].y));
}
__device__ __forceinline__ unsigned f2h(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    unsigned u;
    memcpy(&u, &h, 4);
    return u;
}
__device__ __forceinline__ uint4 make_chunk(const float2 (&w)[4], __half) {
    return make_uint4(f2h(w[0].x, w[1].x), f2h(w[2].x, w[3].x), f2h(w[0].y, w[1].y), f2h(w[2].y, w[3].y));
}
// The values a chunk store leaves in memory (FP16 rounds).
__device__ __forceinline__ float2 stored_rhs(float2 v, float) { return v; }
__device__ __forceinline__ float2 stored_rhs(float2 v, __half) {
    return __half22float2(__floats2half2_rn(v.x, v.y));
}

// Asynchronous 16-byte copies global -> shared (L1 bypassed).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Rows of the x/y neighbour tile of a block: the x-rows its 128 sites span
// (at most 127 / hx + 2) and three more on each side for the y hops.
__host__ __device__ constexpr int xy_tile_rows(int hx) { return 127 / hx + 8; }

// XY: the neighbour chunks of the x and y hops come from a shared-memory tile
// of whole x-rows of the block's (z, t) plane (set by set_tile), the z and t
// hops are taken first, from global memory, while the tile arrives.
template <typename S, typename LS, int RU, int RN, int R, bool PK, int LD, int SD, bool XY = false>
struct BundleHops {
    using LC = typename Traits<LS>::C;
    static constexpr int W = Bundle<S>::W;
    static constexpr int NG = R / W;   // chunks per colour
    static constexpr int P = R / 2;    // rhs pairs
    static constexpr int NCU = (RU == 18) ? 9 : (RU == 14 ? 7 : 6);
    static constexpr int NCN = (RN == 18) ? 9 : (RN == 14 ? 7 : 6);
    static constexpr int NCMAX = NCU > NCN ? NCU : NCN;
    static_assert(R % W == 0 && R % 2 == 0, "rhs per thread must fill whole chunks and pairs");

    struct Raw {
        LC l[NCMAX];
        uint4 v[3][NG];
    };

    const DslashArgs& a;
    const LC* __restrict__ Ub;
    const LC* __restrict__ Nb;
    const uint4* __restrict__ in;   // this thread's first chunk row: group k0 / W
    int vh, p, q, h, hrow, x, y, z, t;
    uint32_t tile = 0;              // XY: shared address of the tile
    int tile_stride = 0;            // XY: sites per chunk plane of the tile
    int tile_y0 = 0;                // XY: global y of tile row 0
    f2x (&ar)[P][3];
    f2x (&ai)[P][3];
    float2 (&acc)[R][3];

    __device__ __forceinline__ void set_tile(uint32_t base, int stride, int y0) {
        tile = base;
        tile_stride = stride;
        tile_y0 = y0;
    }

    // hop e of the S-th step: the natural order, or z, t, x, y with XY
    template <int ST>
    __host__ __device__ static constexpr int hop_of() {
        if constexpr (!XY) {
            return ST;
        } else {
            constexpr int D = ST >> 2;
            constexpr int MU = D == 0 ? 2 : D == 1 ? 3 : D == 2 ? 0 : 1;
            return (MU << 2) | (ST & 3);
        }
    }

    __device__ __forceinline__ BundleHops(const DslashArgs& args, int h_, int k0, f2x (&ar_)[P][3],
                                          f2x (&ai_)[P][3], float2 (&acc_)[R][3])
        : a(args), ar(ar_), ai(ai_), acc(acc_) {
        Ub = reinterpret_cast<const LC*>(a.U);
        Nb = reinterpret_cast<const LC*>(a.N);
        vh = a.g.vh;
        in = reinterpret_cast<const uint4*>(a.in[0]) + (size_t)(k0 / W) * 3 * vh;
        p = a.parity;
        q = 1 - p;
        h = h_;
        const int xh = h % a.g.hx;
        int r = h / a.g.hx;
        y = r % a.g.L[1];
        r /= a.g.L[1];
        z = r % a.g.L[2];
        t = r / a.g.L[2];
        x = 2 * xh + ((p + y + z + t) & 1);
        hrow = h - xh;
    }

    template <int MU>
    __device__ __forceinline__ int coord() const {
        return MU == 0 ? x : MU == 1 ? y : MU == 2 ? z : t;
    }

    template <int E>
    __device__ __forceinline__ int neighbour() const {
        constexpr int MU = E >> 2, HOP = E & 3;
        constexpr int D = HOP == 0 ? 1 : HOP == 1 ? -1 : HOP == 2 ? 3 : -3;
        const int c = coord<MU>();
        const int cn = wrap(c + D, a.g.L[MU]);
        if (MU == 0) return hrow + (cn >> 1);
        const int stride = MU == 1 ? a.g.sy : MU == 2 ? a.g.sz : a.g.st;
        return h + (cn - c) * stride;
    }

    template <int E>
    __device__ __forceinline__ void issue_link(Raw& b) const {
        constexpr int MU = E >> 2, HOP = E & 3;
        constexpr bool NAIK = HOP >= 2;
        constexpr bool BACK = HOP & 1;
        constexpr int NC = NAIK ? NCN : NCU;
        const LC* base = (NAIK ? Nb : Ub) + (size_t)((BACK ? q : p) * 4 + MU) * NC * vh;
        const int li = BACK ? neighbour<E>() : h;
        load_link_raw<LC, NC>(b.l, base, vh, li);
    }

    template <int E>
    __device__ __forceinline__ void issue_spin(Raw& b) const {
        constexpr int MU = E >> 2;
        if constexpr (XY && MU <= 1) {
            // tile site of the neighbour: its row relative to tile row 0, and
            // its half-index column (x hops move along the row, y hops keep it)
            constexpr int HOP = E & 3;
            constexpr int D = HOP == 0 ? 1 : HOP == 1 ? -1 : HOP == 2 ? 3 : -3;
            const int Ly = a.g.L[1];
            int row, col;
            if constexpr (MU == 0) {
                row = y;
                col = wrap(x + D, a.g.L[0]) >> 1;
            } else {
                row = wrap(y + D, Ly);
                col = h - hrow;
            }
            const int ts = wrap(row - tile_y0, Ly) * a.g.hx + col;
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int g = 0; g < NG; ++g) {
                    const uint32_t ad = tile + (uint32_t)((c * NG + g) * tile_stride + ts) * 16u;
                    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                                 : "=r"(b.v[c][g].x), "=r"(b.v[c][g].y), "=r"(b.v[c][g].z), "=r"(b.v[c][g].w)
                                 : "r"(ad));
                }
        } else {
            const int hn = neighbour<E>();
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int g = 0; g < NG; ++g) b.v[c][g] = __ldg(in + (size_t)(g * 3 + c) * vh + hn);
        }
    }

    template <int E>
    __device__ __forceinline__ void compute(const Raw& b) {
        constexpr int MU = E >> 2, HOP = E & 3;
        constexpr bool NAIK = HOP >= 2;
        constexpr bool BACK = HOP & 1;
        constexpr int REC = NAIK ? RN : RU;
        constexpr int NC = NAIK ? NCN : NCU;
        const float* sc = NAIK ? a.lscale_n : a.lscale_u;
        Link<float2> m;
#pragma unroll
        for (int c = 0; c < 6; ++c) m.e[c] = link_elem(b.l[c], sc[c]);
        if constexpr (REC == 18) {
#pragma unroll
            for (int c = 6; c < 9; ++c) m.e[c] = link_elem(b.l[c], sc[c]);
        } else if constexpr (REC == 14) {
            third_row(m, link_elem(b.l[NC - 1], sc[NC - 1]));
        } else {
            const int e = MU == 0 ? 0 : MU == 1 ? x : MU == 2 ? (x + y) : (x + y + z);
            int sgn = (e & 1) ? -1 : 1;
            if (MU == 3 && ((HOP == 0 && t == a.g.L[3] - 1) || (HOP == 1 && t == 0))) sgn = -sgn;
            const float inv_s = (float)a.r12_inv_scale;
            third_row(m, make_float2(sgn > 0 ? inv_s : -inv_s, 0.f));
        }
        if (MU == 3 && a.has_mu) {
            const double f = HOP == 0 ? a.ft1 : HOP == 1 ? a.bt1 : HOP == 2 ? a.ft3 : a.bt3;
            scale_link(m, (float)f);
        }
        if constexpr (PK) {
            f2x vr[P][3], vi[P][3];
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int pp = 0; pp < P; ++pp)
                    chunk_pair(b.v[j][(2 * pp) / W], ((2 * pp) % W) / 2, vr[pp][j], vi[pp][j], S{});
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const float2 e = BACK ? m.e[3 * j + i] : m.e[3 * i + j];
                    const f2x A = BACK ? pk2(-e.x, -e.x) : pk2(e.x, e.x);
                    const f2x B = pk2(-e.y, -e.y);
                    const f2x C = pk2(e.y, e.y);
                    // four passes over the pairs, so that an accumulator's
                    // next update is 2 P instructions after its last one
#pragma unroll
                    for (int pp = 0; pp < P; ++pp) ar[pp][i] = fma2(A, vr[pp][j], ar[pp][i]);
#pragma unroll
                    for (int pp = 0; pp < P; ++pp) ai[pp][i] = fma2(A, vi[pp][j], ai[pp][i]);
#pragma unroll
                    for (int pp = 0; pp < P; ++pp) ar[pp][i] = fma2(B, vi[pp][j], ar[pp][i]);
#pragma unroll
                    for (int pp = 0; pp < P; ++pp) ai[pp][i] = fma2(C, vr[pp][j], ai[pp][i]);
                }
        } else {
#pragma unroll
            for (int k = 0; k < R; ++k) {
                float2 v[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) v[c] = chunk_rhs(b.v[c][k / W], k % W, S{});
                if (BACK)
                    mv_sub_dag(acc[k], m, v);
                else
                    mv_add(acc[k], m, v);
            }
        }
    }

    template <int ST>
    __device__ __forceinline__ void step(Raw (&buf)[2]) {
        if constexpr (ST + LD < 16) issue_link<hop_of<ST + LD>()>(buf[(ST + LD) & 1]);
        if constexpr (XY && ST + SD == 8) {
            // the first x hop: the tile copies have landed for every thread
            cp_async_wait<0>();
            __syncthreads();
        }
        if constexpr (ST + SD < 16) issue_spin<hop_of<ST + SD>()>(buf[(ST + SD) & 1]);
        compute<hop_of<ST>()>(buf[ST & 1]);
        if constexpr (ST + 1 < 16) step<ST + 1>(buf);
    }

    __device__ __forceinline__ void run() {
        Raw buf[2];
        if constexpr (LD == 1) issue_link<hop_of<0>()>(buf[0]);
        if constexpr (SD == 1) issue_spin<hop_of<0>()>(buf[0]);
        step<0>(buf);
    }
};

// Compact form of the same hop loop: the direction mu is a runtime loop (the
// four hops of a direction are unrolled), which keeps the kernel's code a
// quarter of the fully unrolled size, and each hop converts and multiplies
// one colour j of the neighbour bundle at a time, so only that colour's
// packed pairs are live beside the accumulators. The link of the next hop
// (and with SD = 1 the next hop's neighbour chunks) is loaded before the
// current hop is multiplied, across direction boundaries too.
template <typename S, typename LS, int RU, int RN, int R, int SD>
struct BundleHopsCompact {
    using LC = typename Traits<LS>::C;
    static constexpr int W = Bundle<S>::W;
    static constexpr int NG = R / W;
    static constexpr int P = R / 2;
    static constexpr int NCU = (RU == 18) ? 9 : (RU == 14 ? 7 : 6);
    static constexpr int NCN = (RN == 18) ? 9 : (RN == 14 ? 7 : 6);
    static constexpr int NCMAX = NCU > NCN ? NCU : NCN;

    struct Raw {
        LC l[NCMAX];
        uint4 v[3][NG];
    };

    const DslashArgs& a;
    const LC* __restrict__ Ub;
    const LC* __restrict__ Nb;
    const uint4* __restrict__ in;
    int vh, p, q, h, hrow, x, y, z, t;
    f2x (&ar)[P][3];
    f2x (&ai)[P][3];

    __device__ __forceinline__ BundleHopsCompact(const DslashArgs& args, int h_, int k0, f2x (&ar_)[P][3],
                                                 f2x (&ai_)[P][3])
        : a(args), ar(ar_), ai(ai_) {
        Ub = reinterpret_cast<const LC*>(a.U);
        Nb = reinterpret_cast<const LC*>(a.N);
        vh = a.g.vh;
        in = reinterpret_cast<const uint4*>(a.in[0]) + (size_t)(k0 / W) * 3 * vh;
        p = a.parity;
        q = 1 - p;
        h = h_;
        const int xh = h % a.g.hx;
        int r = h / a.g.hx;
        y = r % a.g.L[1];
        r /= a.g.L[1];
        z = r % a.g.L[2];
        t = r / a.g.L[2];
        x = 2 * xh + ((p + y + z + t) & 1);
        hrow = h - xh;
    }

    __device__ __forceinline__ int coord(int mu) const { return mu == 0 ? x : mu == 1 ? y : mu == 2 ? z : t; }

    template <int HOP>
    __device__ __forceinline__ int neighbour(int mu) const {
        constexpr int D = HOP == 0 ? 1 : HOP == 1 ? -1 : HOP == 2 ? 3 : -3;
        const int c = coord(mu);
        const int cn = wrap(c + D, a.g.L[mu]);
        if (mu == 0) return hrow + (cn >> 1);
        const int stride = mu == 1 ? a.g.sy : mu == 2 ? a.g.sz : a.g.st;
        return h + (cn - c) * stride;
    }

    template <int HOP>
    __device__ __forceinline__ void issue_link(int mu, Raw& b) const {
        constexpr bool NAIK = HOP >= 2;
        constexpr bool BACK = HOP & 1;
        constexpr int NC = NAIK ? NCN : NCU;
        const LC* base = (NAIK ? Nb : Ub) + (size_t)((BACK ? q : p) * 4 + mu) * NC * vh;
        const int li = BACK ? neighbour<HOP>(mu) : h;
        load_link_raw<LC, NC>(b.l, base, vh, li);
    }

    template <int HOP>
    __device__ __forceinline__ void issue_spin(int mu, Raw& b) const {
        const int hn = neighbour<HOP>(mu);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int g = 0; g < NG; ++g) b.v[c][g] = __ldg(in + (size_t)(g * 3 + c) * vh + hn);
    }

    template <int HOP>
    __device__ __forceinline__ void compute(int mu, const Raw& b) {
        constexpr bool NAIK = HOP >= 2;
        constexpr bool BACK = HOP & 1;
        constexpr int REC = NAIK ? RN : RU;
        constexpr int NC = NAIK ? NCN : NCU;
        const float* sc = NAIK ? a.lscale_n : a.lscale_u;
        Link<float2> m;
#pragma unroll
        for (int c = 0; c < 6; ++c) m.e[c] = link_elem(b.l[c], sc[c]);
        if constexpr (REC == 18) {
#pragma unroll
            for (int c = 6; c < 9; ++c) m.e[c] = link_elem(b.l[c], sc[c]);
        } else if constexpr (REC == 14) {
            third_row(m, link_elem(b.l[NC - 1], sc[NC - 1]));
        } else {
            const int e = mu == 0 ? 0 : mu == 1 ? x : mu == 2 ? (x + y) : (x + y + z);
            int sgn = (e & 1) ? -1 : 1;
            if (mu == 3 && ((HOP == 0 && t == a.g.L[3] - 1) || (HOP == 1 && t == 0))) sgn = -sgn;
            const float inv_s = (float)a.r12_inv_scale;
            third_row(m, make_float2(sgn > 0 ? inv_s : -inv_s, 0.f));
        }
        if (mu == 3 && a.has_mu) {
            const double f = HOP == 0 ? a.ft1 : HOP == 1 ? a.bt1 : HOP == 2 ? a.ft3 : a.bt3;
            scale_link(m, (float)f);
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            f2x vr[P], vi[P];
#pragma unroll
            for (int pp = 0; pp < P; ++pp) chunk_pair(b.v[j][(2 * pp) / W], ((2 * pp) % W) / 2, vr[pp], vi[pp], S{});
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float2 e = BACK ? m.e[3 * j + i] : m.e[3 * i + j];
                const f2x A = BACK ? pk2(-e.x, -e.x) : pk2(e.x, e.x);
                const f2x B = pk2(-e.y, -e.y);
                const f2x C = pk2(e.y, e.y);
#pragma unroll
                for (int pp = 0; pp < P; ++pp) ar[pp][i] = fma2(A, vr[pp], ar[pp][i]);
#pragma unroll
                for (int pp = 0; pp < P; ++pp) ai[pp][i] = fma2(A, vi[pp], ai[pp][i]);
#pragma unroll
                for (int pp = 0; pp < P; ++pp) ar[pp][i] = fma2(B, vi[pp], ar[pp][i]);
#pragma unroll
                for (int pp = 0; pp < P; ++pp) ai[pp][i] = fma2(C, vr[pp], ai[pp][i]);
            }
        }
    }

    // hop HOP of direction mu: first the look-ahead loads (the next hop's
    // link, and with SD its neighbour chunks), then this hop's
    template <int HOP>
    __device__ __forceinline__ void step(int mu, Raw (&buf)[2]) {
        constexpr int NEXT = (HOP + 1) & 3;
        const int nmu = HOP == 3 ? mu + 1 : mu;
        if (nmu < 4) {
            issue_link<NEXT>(nmu, buf[NEXT & 1]);
            if constexpr (SD == 1) issue_spin<NEXT>(nmu, buf[NEXT & 1]);
        }
        if constexpr (SD == 0) issue_spin<HOP>(mu, buf[HOP & 1]);
        compute<HOP>(mu, buf[HOP & 1]);
    }

    __device__ __forceinline__ void run() {
        Raw buf[2];
        issue_link<0>(0, buf[0]);
        if constexpr (SD == 1) issue_spin<0>(0, buf[0]);
#pragma unroll 1
        for (int mu = 0; mu < 4; ++mu) {
            step<0>(mu, buf);
            step<1>(mu, buf);
            step<2>(mu, buf);
            step<3>(mu, buf);
        }
    }
};

// Hop loop with the neighbour chunks staged through shared memory: every
// thread copies the chunks of hop e + D into its own slots of a ring of
// D + 1 stages with per-thread asynchronous 16-byte copies (cp.async, L1
// bypassed), so the copies in flight hold no registers; hop e then reads its
// chunks back one colour at a time. Slot (stage s, chunk c) of thread t sits
// at ((s * 3 NG + c) * T + t) * 16 bytes, T the block's thread count:
// consecutive threads touch consecutive 16-byte words (no bank conflicts).
// The link of the next hop is loaded into registers one hop ahead.

template <typename S, typename LS, int RU, int RN, int R, int D>
struct BundleHopsStaged {
    using LC = typename Traits<LS>::C;
    static constexpr int W = Bundle<S>::W;
    static constexpr int NG = R / W;
    static constexpr int P = R / 2;
    static constexpr int NCU = (RU == 18) ? 9 : (RU == 14 ? 7 : 6);
    static constexpr int NCN = (RN == 18) ? 9 : (RN == 14 ? 7 : 6);
    static constexpr int NCMAX = NCU > NCN ? NCU : NCN;
    static constexpr int NS = D + 1;   // stages in the ring

    struct Lk {
        LC l[NCMAX];
    };

    const DslashArgs& a;
    const LC* __restrict__ Ub;
    const LC* __restrict__ Nb;
    const uint4* __restrict__ in;
    uint32_t slot0;   // shared address of this thread's chunk (stage 0, chunk 0)
    uint32_t tstride; // bytes between consecutive chunks of one thread: 16 T
    int vh, p, q, h, hrow, x, y, z, t;
    f2x (&ar)[P][3];
    f2x (&ai)[P][3];

    __device__ __forceinline__ BundleHopsStaged(const DslashArgs& args, int h_, int k0, uint32_t slot0_,
                                                uint32_t tstride_, f2x (&ar_)[P][3], f2x (&ai_)[P][3])
        : a(args), slot0(slot0_), tstride(tstride_), ar(ar_), ai(ai_) {
        Ub = reinterpret_cast<const LC*>(a.U);
        Nb = reinterpret_cast<const LC*>(a.N);
        vh = a.g.vh;
        in = reinterpret_cast<const uint4*>(a.in[0]) + (size_t)(k0 / W) * 3 * vh;
        p = a.parity;
        q = 1 - p;
        h = h_;
        const int xh = h % a.g.hx;
        int r = h / a.g.hx;
        y = r % a.g.L[1];
        r /= a.g.L[1];
        z = r % a.g.L[2];
        t = r / a.g.L[2];
        x = 2 * xh + ((p + y + z + t) & 1);
        hrow = h - xh;
    }

    template <int MU>
    __device__ __forceinline__ int coord() const {
        return MU == 0 ? x : MU == 1 ? y : MU == 2 ? z : t;
    }

    template <int E>
    __device__ __forceinline__ int neighbour() const {
        constexpr int MU = E >> 2, HOP = E & 3;
        constexpr int DD = HOP == 0 ? 1 : HOP == 1 ? -1 : HOP == 2 ? 3 : -3;
        const int c = coord<MU>();
        const int cn = wrap(c + DD, a.g.L[MU]);
        if (MU == 0) return hrow + (cn >> 1);
        const int stride = MU == 1 ? a.g.sy : MU == 2 ? a.g.sz : a.g.st;
        return h + (cn - c) * stride;
    }

    template <int E>
    __device__ __forceinline__ void issue_link(Lk& b) const {
        constexpr int MU = E >> 2, HOP = E & 3;
        constexpr bool NAIK = HOP >= 2;
        constexpr bool BACK = HOP & 1;
        constexpr int NC = NAIK ? NCN : NCU;
        const LC* base = (NAIK ? Nb : Ub) + (size_t)((BACK ? q : p) * 4 + MU) * NC * vh;
        const int li = BACK ? neighbour<E>() : h;
        load_link_raw<LC, NC>(b.l, base, vh, li);
    }

    // asynchronous copies of hop E's neighbour chunks into stage E % NS, one group
    template <int E>
    __device__ __forceinline__ void stage(int) const {
        const int hn = neighbour<E>();
        const uint32_t st = slot0 + (uint32_t)((E % NS) * 3 * NG) * tstride;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int g = 0; g < NG; ++g)
                cp_async16(st + (uint32_t)(c * NG + g) * tstride, in + (size_t)(g * 3 + c) * vh + hn);
        cp_async_commit();
    }

    template <int E>
    __device__ __forceinline__ void compute(const Lk& b) {
        constexpr int MU = E >> 2, HOP = E & 3;
        constexpr bool NAIK = HOP >= 2;
        constexpr bool BACK = HOP & 1;
        constexpr int REC = NAIK ? RN : RU;
        constexpr int NC = NAIK ? NCN : NCU;
        const float* sc = NAIK ? a.lscale_n : a.lscale_u;
        Link<float2> m;
#pragma unroll
        for (int c = 0; c < 6; ++c) m.e[c] = link_elem(b.l[c], sc[c]);
        if constexpr (REC == 18) {
#pragma unroll
            for (int c = 6; c < 9; ++c) m.e[c] = link_elem(b.l[c], sc[c]);
        } else if constexpr (REC == 14) {
            third_row(m, link_elem(b.l[NC - 1], sc[NC - 1]));
        } else {
            const int e = MU == 0 ? 0 : MU == 1 ? x : MU == 2 ? (x + y) : (x + y + z);
            int sgn = (e & 1) ? -1 : 1;
            if (MU == 3 && ((HOP == 0 && t == a.g.L[3] - 1) || (HOP == 1 && t == 0))) sgn = -sgn;
            const float inv_s = (float)a.r12_inv_scale;
            third_row(m, make_float2(sgn > 0 ? inv_s : -inv_s, 0.f));
        }
        if (MU == 3 && a.has_mu) {
            const double f = HOP == 0 ? a.ft1 : HOP == 1 ? a.bt1 : HOP == 2 ? a.ft3 : a.bt3;
            scale_link(m, (float)f);
        }
        const uint32_t st = slot0 + (uint32_t)((E % NS) * 3 * NG) * tstride;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            uint4 ch[NG];
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                const uint32_t ad = st + (uint32_t)(j * NG + g) * tstride;
                asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                             : "=r"(ch[g].x), "=r"(ch[g].y), "=r"(ch[g].z), "=r"(ch[g].w)
                             : "r"(ad));
            }
            f2x vr[P], vi[P];
#pragma unroll
            for (int pp = 0; pp < P; ++pp) chunk_pair(ch[(2 * pp) / W], ((2 * pp) % W) / 2, vr[pp], vi[pp], S{});
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float2 e = BACK ? m.e[3 * j + i] : m.e[3 * i + j];
                const f2x A = BACK ? pk2(-e.x, -e.x) : pk2(e.x, e.x);
                const f2x B = pk2(-e.y, -e.y);
                const f2x C = pk2(e.y, e.y);
#pragma unroll
                for (int pp = 0; pp < P; ++pp) ar[pp][i] = fma2(A, vr[pp], ar[pp][i]);
#pragma unroll
                for (int pp = 0; pp < P; ++pp) ai[pp][i] = fma2(A, vi[pp], ai[pp][i]);
#pragma unroll
                for (int pp = 0; pp < P; ++pp) ar[pp][i] = fma2(B, vi[pp], ar[pp][i]);
#pragma unroll
                for (int pp = 0; pp < P; ++pp) ai[pp][i] = fma2(C, vr[pp], ai[pp][i]);
            }
        }
    }

    template <int E>
    __device__ __forceinline__ void step(Lk (&lk)[2]) {
        if constexpr (E + 1 < 16) issue_link<E + 1>(lk[(E + 1) & 1]);
        if constexpr (E + D < 16) stage<E + D>(0);
        // the groups committed after hop E's: min(D, 15 - E) of them may stay in flight
        constexpr int AFTER = (15 - E) < D ? (15 - E) : D;
        cp_async_wait<AFTER>();
        compute<E>(lk[E & 1]);
        if constexpr (E + 1 < 16) step<E + 1>(lk);
    }

    template <int I>
    __device__ __forceinline__ void prologue() const {
        if constexpr (I < D) {
            stage<I>(0);
            prologue<I + 1>();
        }
    }

    __device__ __forceinline__ void run() {
        Lk lk[2];
        issue_link<0>(lk[0]);
        prologue<0>();
        step<0>(lk);
    }
};

// Compact hop loop (direction as a runtime loop, a quarter of the code, so
// the warps of an SM share a small instruction footprint) with the
// neighbour chunks staged in shared memory D hops ahead as in
// BundleHopsStaged; D = 1 or 3, so the stage of hop 4 mu + HOP is fixed by
// HOP alone (NS = D + 1 divides 4).
template <typename S, typename LS, int RU, int RN, int R, int D>
struct BundleHopsCompactStaged {
    using LC = typename Traits<LS>::C;
    static constexpr int W = Bundle<S>::W;
    static constexpr int NG = R / W;
    static constexpr int P = R / 2;
    static constexpr int NCU = (RU == 18) ? 9 : (RU == 14 ? 7 : 6);
    static constexpr int NCN = (RN == 18) ? 9 : (RN == 14 ? 7 : 6);
    static constexpr int NCMAX = NCU > NCN ? NCU : NCN;
    static constexpr int NS = D + 1;
    static_assert(4 % NS == 0, "the stage of a hop must not depend on its direction");

    struct Lk {
        LC l[NCMAX];
    };

    const DslashArgs& a;
    const LC* __restrict__ Ub;
    const LC* __restrict__ Nb;
    const uint4* __restrict__ in;
    uint32_t slot0;
    uint32_t tstride;
    int vh, p, q, h, hrow, x, y, z, t;
    f2x (&ar)[P][3];
    f2x (&ai)[P][3];

    __device__ __forceinline__ BundleHopsCompactStaged(const DslashArgs& args, int h_, int k0, uint32_t slot0_,
                                                       uint32_t tstride_, f2x (&ar_)[P][3], f2x (&ai_)[P][3])
        : a(args), slot0(slot0_), tstride(tstride_), ar(ar_), ai(ai_) {
        Ub = reinterpret_cast<const LC*>(a.U);
        Nb = reinterpret_cast<const LC*>(a.N);
        vh = a.g.vh;
        in = reinterpret_cast<const uint4*>(a.in[0]) + (size_t)(k0 / W) * 3 * vh;
        p = a.parity;
        q = 1 - p;
        h = h_;
        const int xh = h % a.g.hx;
        int r = h / a.g.hx;
        y = r % a.g.L[1];
        r /= a.g.L[1];
        z = r % a.g.L[2];
        t = r / a.g.L[2];
        x = 2 * xh + ((p + y + z + t) & 1);
        hrow = h - xh;
    }

    __device__ __forceinline__ int coord(int mu) const { return mu == 0 ? x : mu == 1 ? y : mu == 2 ? z : t; }

    template <int HOP>
    __device__ __forceinline__ int neighbour(int mu) const {
        constexpr int DD = HOP == 0 ? 1 : HOP == 1 ? -1 : HOP == 2 ? 3 : -3;
        const int c = coord(mu);
        const int cn = wrap(c + DD, a.g.L[mu]);
        if (mu == 0) return hrow + (cn >> 1);
        const int stride = mu == 1 ? a.g.sy : mu == 2 ? a.g.sz : a.g.st;
        return h + (cn - c) * stride;
    }

    template <int HOP>
    __device__ __forceinline__ void issue_link(int mu, Lk& b) const {
        constexpr bool NAIK = HOP >= 2;
        constexpr bool BACK = HOP & 1;
        constexpr int NC = NAIK ? NCN : NCU;
        const LC* base = (NAIK ? Nb : Ub) + (size_t)((BACK ? q : p) * 4 + mu) * NC * vh;
        const int li = BACK ? neighbour<HOP>(mu) : h;
        load_link_raw<LC, NC>(b.l, base, vh, li);
    }

    template <int HOP>
    __device__ __forceinline__ void stage(int mu) const {
        const int hn = neighbour<HOP>(mu);
        const uint32_t st = slot0 + (uint32_t)((HOP % NS) * 3 * NG) * tstride;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int g = 0; g < NG; ++g)
                cp_async16(st + (uint32_t)(c * NG + g) * tstride, in + (size_t)(g * 3 + c) * vh + hn);
        cp_async_commit();
    }

    template <int HOP>
    __device__ __forceinline__ void compute(int mu, const Lk& b) {
        constexpr bool NAIK = HOP >= 2;
        constexpr bool BACK = HOP & 1;
        constexpr int REC = NAIK ? RN : RU;
        constexpr int NC = NAIK ? NCN : NCU;
        const float* sc = NAIK ? a.lscale_n : a.lscale_u;
        Link<float2> m;
#pragma unroll
        for (int c = 0; c < 6; ++c) m.e[c] = link_elem(b.l[c], sc[c]);
        if constexpr (REC == 18) {
#pragma unroll
            for (int c = 6; c < 9; ++c) m.e[c] = link_elem(b.l[c], sc[c]);
        } else if constexpr (REC == 14) {
            third_row(m, link_elem(b.l[NC - 1], sc[NC - 1]));
        } else {
            const int e = mu == 0 ? 0 : mu == 1 ? x : mu == 2 ? (x + y) : (x + y + z);
            int sgn = (e & 1) ? -1 : 1;
            if (mu == 3 && ((HOP == 0 && t == a.g.L[3] - 1) || (HOP == 1 && t == 0))) sgn = -sgn;
            const float inv_s = (float)a.r12_inv_scale;
            third_row(m, make_float2(sgn > 0 ? inv_s : -inv_s, 0.f));
        }
        if (mu == 3 && a.has_mu) {
            const double f = HOP == 0 ? a.ft1 : HOP == 1 ? a.bt1 : HOP == 2 ? a.ft3 : a.bt3;
            scale_link(m, (float)f);
        }
        const uint32_t st = slot0 + (uint32_t)((HOP % NS) * 3 * NG) * tstride;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            uint4 ch[NG];
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                const uint32_t ad = st + (uint32_t)(j * NG + g) * tstride;
                asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                             : "=r"(ch[g].x), "=r"(ch[g].y), "=r"(ch[g].z), "=r"(ch[g].w)
                             : "r"(ad));
            }
            f2x vr[P], vi[P];
#pragma unroll
            for (int pp = 0; pp < P; ++pp) chunk_pair(ch[(2 * pp) / W], ((2 * pp) % W) / 2, vr[pp], vi[pp], S{});
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float2 e = BACK ? m.e[3 * j + i] : m.e[3 * i + j];
                const f2x A = BACK ? pk2(-e.x, -e.x) : pk2(e.x, e.x);
                const f2x B = pk2(-e.y, -e.y);
                const f2x C = pk2(e.y, e.y);
#pragma unroll
                for (int pp = 0; pp < P; ++pp) ar[pp][i] = fma2(A, vr[pp], ar[pp][i]);
#pragma unroll
                for (int pp = 0; pp < P; ++pp) ai[pp][i] = fma2(A, vi[pp], ai[pp][i]);
#pragma unroll
                for (int pp = 0; pp < P; ++pp) ar[pp][i] = fma2(B, vi[pp], ar[pp][i]);
#pragma unroll
                for (int pp = 0; pp < P; ++pp) ai[pp][i] = fma2(C, vr[pp], ai[pp][i]);
            }
        }
    }

    // stage hop e + D (direction mu + (HOP + D) / 4), load the next link,
    // wait for hop e's chunks, multiply
    template <int HOP>
    __device__ __forceinline__ void step(int mu, Lk (&lk)[2]) {
        constexpr int SH = (HOP + D) & 3;                 // hop index of e + D within its direction
        const int smu = mu + (HOP + D) / 4;               // its direction
        const bool staged_more = smu < 4;
        if (staged_more) stage<SH>(smu);
        constexpr int NEXT = (HOP + 1) & 3;
        const int nmu = HOP == 3 ? mu + 1 : mu;
        if (nmu < 4) issue_link<NEXT>(nmu, lk[NEXT & 1]);
        // groups committed after hop e's: D while later hops were staged, fewer at the end
        const int remaining = 15 - (4 * mu + HOP);
        if (remaining >= D)
            cp_async_wait<D>();
        else if (D >= 3 && remaining == 2)
            cp_async_wait<(D >= 3 ? 2 : 0)>();
        else if (D >= 2 && remaining == 1)
            cp_async_wait<(D >= 2 ? 1 : 0)>();
        else
            cp_async_wait<0>();
        compute<HOP>(mu, lk[HOP & 1]);
    }

    __device__ __forceinline__ void run() {
        Lk lk[2];
        issue_link<0>(0, lk[0]);
        // prologue: hops 0 .. D-1 of direction 0
        stage<0>(0);
        if constexpr (D >= 2) stage<1>(0);
        if constexpr (D >= 3) stage<2>(0);
#pragma unroll 1
        for (int mu = 0; mu < 4; ++mu) {
            step<0>(mu, lk);
            step<1>(mu, lk);
            step<2>(mu, lk);
            step<3>(mu, lk);
        }
    }
};

// One Dslash of parity a.parity on the bundle layout: out = D in (EPI_NONE)
// or out = cx x + cd (D in) with optionally Re<x, out> per rhs (EPI_X), for
// the rhs of every thread group. a.in[0], a.out[0], a.x[0] are bundle bases.
template <typename S, typename LS, int RU, int RN, int R, int MINB, bool PK, int LD, int SD, int EPI,
          bool COMPACT, int STAGE = 0>
__global__ void __launch_bounds__(128, MINB) dslash_bundle_kernel(const DslashArgs a) {
    constexpr int W = Bundle<S>::W;
    constexpr int NG = R / W;
    constexpr int P = R / 2;
    const int vh = a.g.vh;
    const int k0 = threadIdx.y * R;
    const size_t gofs = (size_t)(k0 / W) * 3 * vh;

    float red0[R], red1[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        red0[j] = 0.f;
        red1[j] = 0.f;
    }
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v - (int)threadIdx.x < vh;
         v += gridDim.x * blockDim.x) {
        if (v >= vh) continue;
        const int h = visit_site(v, a.g);
        if constexpr (EPI == EPI_X) {
            // the epilogue's x is read after the hops; start it towards L2 now
            const uint4* xb = reinterpret_cast<const uint4*>(a.x[0]) + gofs + h;
#pragma unroll
            for (int c = 0; c < 3 * NG; ++c)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(xb + (size_t)c * vh));
        }
        f2x ar[P][3], ai[P][3];
        float2 acc[R][3];
#pragma unroll
        for (int pp = 0; pp < P; ++pp)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                ar[pp][c] = 0ull;
                ai[pp][c] = 0ull;
            }
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[k][c] = make_float2(0.f, 0.f);
        if constexpr (STAGE == 30) {
            // x/y neighbour tile (one rhs group, (z, t) planes of whole
            // 128-site runs; checked by the launcher): whole x-rows of this
            // block's plane, three rows beyond its own on each side
            extern __shared__ __align__(16) unsigned char bundle_smem[];
            const uint32_t base = static_cast<uint32_t>(__cvta_generic_to_shared(bundle_smem));
            const int hx = a.g.hx, Ly = a.g.L[1], plane = a.g.sz;
            const int tsmax = xy_tile_rows(hx) * hx;
            const int v0 = v - (int)threadIdx.x;
            const int h0 = visit_site(v0, a.g), h1 = visit_site(v0 + (int)blockDim.x - 1, a.g);
            const int pbase = h0 - h0 % plane;
            const int y0 = (h0 - pbase) / hx, y1 = (h1 - pbase) / hx;
            const int ya = wrap(y0 - 3, Ly);
            const int ts = (y1 - y0 + 7) * hx;
            const uint4* src = reinterpret_cast<const uint4*>(a.in[0]);
            __syncthreads();   // every thread is done with the previous tile
            for (int st = threadIdx.x; st < ts; st += blockDim.x) {
                const int tr = st / hx, col = st - tr * hx;
                const int hg = pbase + ((ya + tr) % Ly) * hx + col;
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int g = 0; g < NG; ++g)
                        cp_async16(base + (uint32_t)((c * NG + g) * tsmax + st) * 16u,
                                   src + (size_t)(g * 3 + c) * vh + hg);
            }
            cp_async_commit();
            BundleHops<S, LS, RU, RN, R, PK, LD, SD, true> hops(a, h, k0, ar, ai, acc);
            hops.set_tile(base, tsmax, ya);
            hops.run();
        } else if constexpr (STAGE > 10) {
            // compact hop loop with staged neighbours, D = STAGE - 10
            extern __shared__ __align__(16) unsigned char bundle_smem[];
            const int tid = threadIdx.x + threadIdx.y * blockDim.x;
            const uint32_t base = static_cast<uint32_t>(__cvta_generic_to_shared(bundle_smem));
            BundleHopsCompactStaged<S, LS, RU, RN, R, STAGE - 10> hops(a, h, k0, base + 16u * tid,
                                                                       16u * blockDim.x * blockDim.y, ar, ai);
            hops.run();
        } else if constexpr (STAGE > 0 && STAGE < 10) {
            extern __shared__ __align__(16) unsigned char bundle_smem[];
            const int tid = threadIdx.x + threadIdx.y * blockDim.x;
            const uint32_t base = static_cast<uint32_t>(__cvta_generic_to_shared(bundle_smem));
            BundleHopsStaged<S, LS, RU, RN, R, STAGE> hops(a, h, k0, base + 16u * tid,
                                                           16u * blockDim.x * blockDim.y, ar, ai);
            hops.run();
        } else if constexpr (COMPACT) {
            static_assert(PK, "the compact hop loop uses packed arithmetic");
            BundleHopsCompact<S, LS, RU, RN, R, SD> hops(a, h, k0, ar, ai);
            hops.run();
        } else {
            BundleHops<S, LS, RU, RN, R, PK, LD, SD> hops(a, h, k0, ar, ai, acc);
            hops.run();
        }
        if constexpr (PK) {
#pragma unroll
            for (int pp = 0; pp < P; ++pp)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float2 re = up2(ar[pp][c]), im = up2(ai[pp][c]);
                    acc[2 * pp][c] = make_float2(re.x, im.x);
                    acc[2 * pp + 1][c] = make_float2(re.y, im.y);
                }
        }
        // epilogue: out = [cx x +] cd acc, stored as chunks
        const float cx = (float)a.cx, cd = (float)a.cd;
        const uint4* xb = EPI == EPI_X ? reinterpret_cast<const uint4*>(a.x[0]) + gofs + h : nullptr;
        uint4* ob = reinterpret_cast<uint4*>(a.out[0]) + gofs + h;
#pragma unroll
        for (int g = 0; g < NG; ++g)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float2 w[W];
                if constexpr (EPI == EPI_X) {
                    const uint4 xc = __ldg(xb + (size_t)(g * 3 + c) * vh);
#pragma unroll
                    for (int l = 0; l < W; ++l) {
                        const float2 xv = chunk_rhs(xc, l, S{});
                        const float2 av = acc[g * W + l][c];
                        w[l] = make_float2(fmaf(cd, av.x, cx * xv.x), fmaf(cd, av.y, cx * xv.y));
                        if (a.red_mode == RED_DOT_XW) {
                            const float2 sv = stored_rhs(w[l], S{});
                            red0[g * W + l] = fmaf(xv.x, sv.x, fmaf(xv.y, sv.y, red0[g * W + l]));
                        }
                    }
                } else {
#pragma unroll
                    for (int l = 0; l < W; ++l) w[l] = acc[g * W + l][c];
                }
                ob[(size_t)(g * 3 + c) * vh] = make_chunk(w, S{});
            }
    }
    if (a.red_mode == RED_NONE) return;
    block_reduce_finish<R>(a, k0, red0, red1);
}

// Whether (n, rhs per thread) fits the bundle kernel of storage S.
template <typename S>
__host__ __device__ constexpr bool bundle_shape_ok(int n, int rpt) {
    return rpt % Bundle<S>::W == 0 && rpt % 2 == 0 && n % rpt == 0 && n / rpt >= 1 && n / rpt <= 4;
}

template <typename S, typename LS, int RU, int RN, int R, int MINB, bool PK, int LD, int SD, int EPI,
          bool COMPACT, int STAGE = 0>
cudaError_t launch_dslash_bundle(const DslashArgs& a, cudaStream_t s) {
    if (a.t_only || !bundle_shape_ok<S>(a.nrhs, R)) return cudaErrorInvalidValue;
    if (EPI == EPI_NONE && a.red_mode != RED_NONE) return cudaErrorInvalidValue;
    const int G = a.nrhs / R;
    if (G > 4) return cudaErrorInvalidValue;
    const int bx = 128 / G;   // 128 threads: 128 / G sites x G rhs groups
    const dim3 block(bx, G);
    auto* kern = dslash_bundle_kernel<S, LS, RU, RN, R, MINB, PK, LD, SD, EPI, COMPACT, STAGE>;
    int occ = 0;
    cudaError_t e = cudaSuccess;
    size_t smem = 0;
    if constexpr (STAGE == 30) {
        // the x/y tile needs one rhs group and (z, t) planes made of whole
        // 128-site runs; otherwise the same loop without the tile
        smem = (size_t)3 * (R / Bundle<S>::W) * xy_tile_rows(a.g.hx) * a.g.hx * 16;
        if (G != 1 || a.g.sz % 128 != 0 || smem > 100 * 1024)
            return launch_dslash_bundle<S, LS, RU, RN, R, MINB, PK, LD, SD, EPI, COMPACT, 0>(a, s);
        // the tile's size follows the lattice: occupancy per call
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, bx * G, smem);
        if (e != cudaSuccess) return e;
        if (occ < 1) return cudaErrorInvalidConfiguration;
    } else {
        // staged: (D + 1) stages x 3 R / W chunks of 16 bytes per thread, D = STAGE
        // (unrolled loop) or STAGE - 10 (compact loop)
        constexpr int DEPTH = STAGE > 10 ? STAGE - 10 : STAGE;
        smem = DEPTH > 0 ? (size_t)(DEPTH + 1) * 3 * (R / Bundle<S>::W) * 16 * 128 : 0;
        static OccCache cache;   // this kernel instance's occupancy per device
        e = cached_occupancy(cache, kern, bx * G, smem, G, &occ);
        if (e != cudaSuccess) return e;
    }
    long long nblk = ((long long)a.g.vh + bx - 1) / bx;
    const long long cap = (long long)occ * device_sm_count();
    if (nblk > cap) nblk = cap;
    if (nblk > kMaxRedBlocks) nblk = kMaxRedBlocks;
    kern<<<(unsigned)nblk, block, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace hisq
