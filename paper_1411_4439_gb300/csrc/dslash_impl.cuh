// Multi-rhs HISQ Dslash kernel, Eq. 3 applied to a bundle of rhs as in Eq. 4.
//
// One thread owns one output site and RPT right-hand sides; blockDim.y groups
// split the bundle (nrhs = blockDim.y * RPT), so all groups of a block share
// the same sites and re-read the same links from L1. Per output site the 16
// hops (4 directions x {+1, -1, +3, -3}) each load one link once for all RPT
// rhs and gather RPT neighbour vectors. Links are reconstructed in registers
// (R12 / R14), temporal links are rescaled by the chemical-potential factors,
// and the epilogue forms out = [y] + cx * x + cd * (D in) and, optionally, the
// per-rhs reductions the CG needs (Re<x,out> or |out|^2 and max|out_i|).
#pragma once

#include <atomic>

#include "hisq_internal.cuh"
#include "reduce.cuh"

namespace hisq {

template <typename RC>
struct Link {
    RC e[9];
};

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

// acc += a * b
template <typename RC>
__device__ __forceinline__ void cmadd(RC& acc, const RC a, const RC b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}

// acc -= conj(a) * b
template <typename RC>
__device__ __forceinline__ void cmsub_conj(RC& acc, const RC a, const RC b) {
    acc.x = fma(-a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}

template <typename RC>
__device__ __forceinline__ RC cmul(const RC a, const RC b) {
    RC c;
    c.x = a.x * b.x - a.y * b.y;
    c.y = a.x * b.y + a.y * b.x;
    return c;
}

// row3 = f * conj(row1 x row2), f complex
template <typename RC>
__device__ __forceinline__ void third_row(Link<RC>& m, const RC f) {
    RC c0, c1, c2;
    c0 = cmul(m.e[1], m.e[5]);
    c0.x -= m.e[2].x * m.e[4].x - m.e[2].y * m.e[4].y;
    c0.y -= m.e[2].x * m.e[4].y + m.e[2].y * m.e[4].x;
    c1 = cmul(m.e[2], m.e[3]);
    c1.x -= m.e[0].x * m.e[5].x - m.e[0].y * m.e[5].y;
    c1.y -= m.e[0].x * m.e[5].y + m.e[0].y * m.e[5].x;
    c2 = cmul(m.e[0], m.e[4]);
    c2.x -= m.e[1].x * m.e[3].x - m.e[1].y * m.e[3].y;
    c2.y -= m.e[1].x * m.e[3].y + m.e[1].y * m.e[3].x;
    c0.y = -c0.y;
    c1.y = -c1.y;
    c2.y = -c2.y;
    m.e[6] = cmul(f, c0);
    m.e[7] = cmul(f, c1);
    m.e[8] = cmul(f, c2);
}

// Load one link of `recon` reals from `base` (the (parity, mu) block, laid
// out as link_offset describes), site index `idx`, with streaming
// (evict-first) loads: every link is read once per launch. `sign` is the
// staggered sign used by R12 (ignored otherwise); sc holds the component
// scales of 16-bit links.
template <typename LC, int RECON, typename RC>
__device__ __forceinline__ void load_link(Link<RC>& m, const LC* __restrict__ base, int vh,
                                          int idx, typename Traits<float>::R inv_s_f,
                                          double inv_s_d, int sign, const float* sc) {
    using R = decltype(RC{}.x);
    constexpr int NC = (RECON == 18) ? 9 : (RECON == 14 ? 7 : 6);
    auto put = [&](int c, LC raw) {
        const auto v = link_elem(raw, sc[c]);
        m.e[c].x = (R)v.x;
        m.e[c].y = (R)v.y;
    };
    // stored components, converted as they arrive (no raw copy of the link)
    if constexpr (LinkPair<LC>::paired) {
        using V = typename LinkPair<LC>::V;
        const V* pb = reinterpret_cast<const V*>(base);
#pragma unroll
        for (int p = 0; p < NC / 2; ++p) {
            LC a, b;
            split_pair(__ldcs(pb + (size_t)p * vh + idx), a, b);
            put(2 * p, a);
            put(2 * p + 1, b);
        }
        if constexpr (NC & 1) put(NC - 1, __ldcs(base + (size_t)(NC - 1) * vh + idx));
    } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) put(c, __ldcs(base + (size_t)c * vh + idx));
    }
    if constexpr (RECON == 14) {
        third_row(m, m.e[6]);
    } else if constexpr (RECON == 12) {
        RC f;
        const R inv_s = (sizeof(R) == 8) ? (R)inv_s_d : (R)inv_s_f;
        f.x = sign > 0 ? inv_s : -inv_s;
        f.y = (R)0;
        third_row(m, f);
    }
}

template <typename RC, typename R>
__device__ __forceinline__ void scale_link(Link<RC>& m, const R f) {
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        m.e[c].x *= f;
        m.e[c].y *= f;
    }
}

// Spinor element (site idx, colour c) of one rhs: AoS [V_h][3] or SoA [3][V_h].
template <int LAYOUT>
__device__ __forceinline__ size_t spinor_index(int idx, int c, int vh) {
    return LAYOUT == HISQ_SOA ? (size_t)c * vh + idx : 3 * (size_t)idx + c;
}

template <typename SC, int LAYOUT, typename RC>
__device__ __forceinline__ void load_spinor(RC (&v)[3], const void* p, int idx, int vh) {
    using R = decltype(RC{}.x);
    const SC* s = reinterpret_cast<const SC*>(p);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const auto t = ld_c(s + spinor_index<LAYOUT>(idx, c, vh));
        v[c].x = (R)t.x;
        v[c].y = (R)t.y;
    }
}

// acc[i] += sum_j m_ij v_j
template <typename RC>
__device__ __forceinline__ void mv_add(RC (&acc)[3], const Link<RC>& m, const RC (&v)[3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) cmadd(acc[i], m.e[3 * i + j], v[j]);
}

// acc[i] -= sum_j conj(m_ji) v_j
template <typename RC>
__device__ __forceinline__ void mv_sub_dag(RC (&acc)[3], const Link<RC>& m, const RC (&v)[3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) cmsub_conj(acc[i], m.e[3 * j + i], v[j]);
}

// ---------------------------------------------------------------------------
// Packed FP32 (f32x2) complex arithmetic: a complex multiply-add is two
// fma.rn.f32x2 on (re, im) pairs instead of four scalar FMAs.
//   a*b   = (a.x, a.x) * (b.x, b.y) + (-a.y, a.y) * (b.y, b.x)
//  -a^* b = (-a.x, -a.x) * (b.x, b.y) + (-a.y, a.y) * (b.y, b.x)
// ---------------------------------------------------------------------------
typedef unsigned long long f2x;

__device__ __forceinline__ f2x pk2(float lo, float hi) {
    f2x r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ float2 up2(f2x v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}

__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c) {
    f2x d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Link elements as the two packed factors above; sgn = +1 forward, -1 for
// the daggered backward hop (which also reads element (j, i)).
struct PLink {
    f2x p1[9];
    f2x p2[9];
};

__device__ __forceinline__ void pack_link(PLink& pl, const Link<float2>& m, float sgn) {
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        pl.p1[e] = pk2(sgn * m.e[e].x, sgn * m.e[e].x);
        pl.p2[e] = pk2(-m.e[e].y, m.e[e].y);
    }
}

// acc[i] += sum_j m_ij v_j (fwd) or acc[i] -= sum_j conj(m_ji) v_j (bwd)
template <bool DAG>
__device__ __forceinline__ void mv_packed(f2x (&acc)[3], const PLink& pl, const float2 (&v)[3]) {
    f2x b1[3], b2[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        b1[j] = pk2(v[j].x, v[j].y);
        b2[j] = pk2(v[j].y, v[j].x);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int e = DAG ? 3 * j + i : 3 * i + j;
            acc[i] = fma2(pl.p1[e], b1[j], acc[i]);
            acc[i] = fma2(pl.p2[e], b2[j], acc[i]);
        }
}

// Asynchronous bulk prefetch of elements [elem0, elem1) of a run of `len`
// link elements into L2 (no registers, no completion to wait for). The range
// is clamped to the run and widened to 16-byte boundaries.
template <typename LC>
__device__ __forceinline__ void prefetch_slab(const LC* slab, long long len, long long elem0, long long elem1) {
    if (elem0 < 0) elem0 = 0;
    if (elem1 > len) elem1 = len;
    if (elem1 <= elem0) return;
    uintptr_t b0 = reinterpret_cast<uintptr_t>(slab + elem0) & ~(uintptr_t)15;
    uintptr_t b1 = (reinterpret_cast<uintptr_t>(slab + elem1) + 15) & ~(uintptr_t)15;
    const uintptr_t lim = reinterpret_cast<uintptr_t>(slab + len) & ~(uintptr_t)15;
    if (b1 > lim) b1 = lim;
    if (b1 <= b0) return;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(b0), "r"((unsigned)(b1 - b0))
                 : "memory");
}

// Site range [e0, e1) of every stored component of one (parity, mu) block.
template <typename LC>
__device__ __forceinline__ void prefetch_block(const LC* block, int nc, int vh, long long e0, long long e1) {
    if constexpr (LinkPair<LC>::paired) {
        const int np = nc & ~1;
        for (int p = 0; p < np / 2; ++p) prefetch_slab(block + (size_t)2 * p * vh, 2ll * vh, 2 * e0, 2 * e1);
        if (nc & 1) prefetch_slab(block + (size_t)np * vh, (long long)vh, e0, e1);
    } else {
        for (int c = 0; c < nc; ++c) prefetch_slab(block + (size_t)c * vh, (long long)vh, e0, e1);
    }
}

// Lanes of the first warp prefetch into L2 the links that the block's sites
// [hb, hb + nb) read: forward links of those sites and backward links of
// their neighbours (shifted ranges; wrapped neighbours are not covered).
template <typename LC, int NCU, int NCN>
__device__ __forceinline__ void prefetch_tile_links(const LC* Ub, const LC* Nb, const Geom& g, int p,
                                                    int hb, int nb) {
    if (threadIdx.y != 0 || threadIdx.x >= 32) return;
    const int q = 1 - p;
    const int vh = g.vh;
    // 16 jobs: direction mu, field (fat, Naik), forward or backward
    for (int job = threadIdx.x; job < 16; job += 32) {
        const int mu = job >> 2;
        const bool naik = (job >> 1) & 1;
        const bool back = job & 1;
        const int nc = naik ? NCN : NCU;
        const LC* base = naik ? Nb : Ub;
        const int par = back ? q : p;
        const LC* block = base + (size_t)(par * 4 + mu) * nc * vh;
        long long e0 = hb, e1 = (long long)hb + nb;
        if (back) {
            const int d = naik ? 3 : 1;
            if (mu == 0) {
                e0 -= g.hx;
                e1 += g.hx;
            } else {
                const int s = (mu == 1) ? g.sy : (mu == 2) ? g.sz : g.st;
                e0 -= (long long)d * s;
                e1 -= (long long)d * s;
            }
        }
        prefetch_block(block, nc, vh, e0, e1);
    }
}

__device__ __forceinline__ int wrap(int c, int L) {
    c = (c >= L) ? c - L : c;
    return (c < 0) ? c + L : c;
}

template <typename SC, int RPT, int EPI, int LAYOUT, typename R, typename RC>
__device__ __forceinline__ void epilogue_site(const DslashArgs& a, int h, int k0, const RC (&acc)[RPT][3],
                                              R (&red0)[RPT], R (&red1)[RPT]);
template <int RPT, typename R>
__device__ __forceinline__ void block_reduce_finish(const DslashArgs& a, int k0, R (&red0)[RPT],
                                                    R (&red1)[RPT]);

template <typename S, typename LS, int RU, int RN, int RPT, int MINB, int EPI, int LAYOUT, bool PACK>
__global__ void __launch_bounds__(256, MINB) dslash_kernel(const DslashArgs a) {
    using R = typename Traits<S>::R;
    static_assert(!PACK || sizeof(R) == 4, "packed f32x2 arithmetic needs FP32 accumulation");
    using RC = typename Cx<R>::T;
    using SC = typename Traits<S>::C;
    using LC = typename Traits<LS>::C;
    constexpr int NCU = (RU == 18) ? 9 : (RU == 14 ? 7 : 6);
    constexpr int NCN = (RN == 18) ? 9 : (RN == 14 ? 7 : 6);

    const Geom& g = a.g;
    const int vh = g.vh;
    const int p = a.parity, q = 1 - p;
    const int k0 = threadIdx.y * RPT;
    const LC* __restrict__ Ub = reinterpret_cast<const LC*>(a.U);
    const LC* __restrict__ Nb = reinterpret_cast<const LC*>(a.N);
    const float inv_s_f = (float)a.r12_inv_scale;

    R red0[RPT], red1[RPT];
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        red0[j] = (R)0;
        red1[j] = (R)0;
    }

    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h - (int)threadIdx.x < vh;
         h += gridDim.x * blockDim.x) {
        if (a.l2_prefetch) {
            // pull this tile's links into L2 at full bandwidth while the first
            // hops wait on their own loads; later hops then hit in L2
            prefetch_tile_links<LC, NCU, NCN>(Ub, Nb, g, p, h - (int)threadIdx.x, blockDim.x);
        }
        if (h >= vh) continue;
        // coordinates of output site h of parity p
        const int xh = h % g.hx;
        int r = h / g.hx;
        const int y = r % g.L[1];
        r /= g.L[1];
        const int z = r % g.L[2];
        const int t = r / g.L[2];
        const int x = 2 * xh + ((p + y + z + t) & 1);
        const int hrow = h - xh;

        RC acc[RPT][3];
        f2x accp[PACK ? RPT : 1][3];
#pragma unroll
        for (int j = 0; j < RPT; ++j)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                acc[j][c].x = (R)0;
                acc[j][c].y = (R)0;
                if constexpr (PACK) accp[j][c] = pk2(0.f, 0.f);
            }

#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            if (mu < 3 && a.t_only) continue;
            const int coord = (mu == 0) ? x : (mu == 1) ? y : (mu == 2) ? z : t;
            const int ext = g.L[mu];
            const int stride = (mu == 1) ? g.sy : (mu == 2) ? g.sz : g.st;
            // staggered sign of this site's mu links (R12 only); eta_mu(x - mu) = eta_mu(x)
            int eta = 1;
            if (RU == 12) {
                const int e = (mu == 0) ? 0 : (mu == 1) ? x : (mu == 2) ? (x + y) : (x + y + z);
                eta = (e & 1) ? -1 : 1;
            }
            const LC* Uf = Ub + (size_t)(p * 4 + mu) * NCU * vh;
            const LC* Ubk = Ub + (size_t)(q * 4 + mu) * NCU * vh;
            const LC* Nf = Nb + (size_t)(p * 4 + mu) * NCN * vh;
            const LC* Nbk = Nb + (size_t)(q * 4 + mu) * NCN * vh;

#pragma unroll
            for (int hop = 0; hop < 4; ++hop) {
                const int d = (hop == 0) ? 1 : (hop == 1) ? -1 : (hop == 2) ? 3 : -3;
                const int cn = wrap(coord + d, ext);
                const int hn = (mu == 0) ? hrow + (cn >> 1) : h + (cn - coord) * stride;
                Link<RC> m;
                if (hop == 0) {
                    const int sgn = (RU == 12 && mu == 3 && t == ext - 1) ? -eta : eta;
                    load_link<LC, RU, RC>(m, Uf, vh, h, inv_s_f, a.r12_inv_scale, sgn, a.lscale_u);
                } else if (hop == 1) {
                    const int sgn = (RU == 12 && mu == 3 && t == 0) ? -eta : eta;
                    load_link<LC, RU, RC>(m, Ubk, vh, hn, inv_s_f, a.r12_inv_scale, sgn, a.lscale_u);
                } else if (hop == 2) {
                    load_link<LC, RN, RC>(m, Nf, vh, h, inv_s_f, a.r12_inv_scale, 1, a.lscale_n);
                } else {
                    load_link<LC, RN, RC>(m, Nbk, vh, hn, inv_s_f, a.r12_inv_scale, 1, a.lscale_n);
                }
                if (mu == 3 && a.has_mu) {
                    const double f = (hop == 0) ? a.ft1 : (hop == 1) ? a.bt1 : (hop == 2) ? a.ft3 : a.bt3;
                    scale_link(m, (R)f);
                }
                if constexpr (PACK) {
                    PLink pl;
                    pack_link(pl, m, (hop == 0 || hop == 2) ? 1.f : -1.f);
#pragma unroll
                    for (int j = 0; j < RPT; ++j) {
                        float2 v[3];
                        load_spinor<SC, LAYOUT, float2>(v, a.in[k0 + j], hn, vh);
                        if (hop == 0 || hop == 2)
                            mv_packed<false>(accp[j], pl, v);
                        else
                            mv_packed<true>(accp[j], pl, v);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < RPT; ++j) {
                        RC v[3];
                        load_spinor<SC, LAYOUT, RC>(v, a.in[k0 + j], hn, vh);
                        if (hop == 0 || hop == 2)
                            mv_add(acc[j], m, v);
                        else
                            mv_sub_dag(acc[j], m, v);
                    }
                }
            }
        }
        if constexpr (PACK) {
#pragma unroll
            for (int j = 0; j < RPT; ++j)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float2 u = up2(accp[j][c]);
                    acc[j][c].x = u.x;
                    acc[j][c].y = u.y;
                }
        }

        epilogue_site<SC, RPT, EPI, LAYOUT>(a, h, k0, acc, red0, red1);
    }

    if (a.red_mode == RED_NONE) return;
    block_reduce_finish<RPT>(a, k0, red0, red1);
}

// Epilogue of one output site: out = [y] + cx x + cd (D in) for the thread's
// RPT rhs, stored in the spinor layout, with the per-thread reduction terms.
template <typename SC, int RPT, int EPI, int LAYOUT, typename R, typename RC>
__device__ __forceinline__ void epilogue_site(const DslashArgs& a, int h, int k0, const RC (&acc)[RPT][3],
                                              R (&red0)[RPT], R (&red1)[RPT]) {
    const int vh = a.g.vh;
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const int k = k0 + j;
        RC w[3];
        if (EPI == EPI_NONE) {
#pragma unroll
            for (int c = 0; c < 3; ++c) w[c] = acc[j][c];
        } else {
            RC xv[3];
            load_spinor<SC, LAYOUT, RC>(xv, a.x[k], h, vh);
            const R cx = (R)a.cx, cd = (R)a.cd;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                w[c].x = fma(cd, acc[j][c].x, cx * xv[c].x);
                w[c].y = fma(cd, acc[j][c].y, cx * xv[c].y);
            }
            if (EPI == EPI_XY) {
                RC yv[3];
                load_spinor<SC, LAYOUT, RC>(yv, a.y[k], h, vh);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    w[c].x += yv[c].x;
                    w[c].y += yv[c].y;
                }
            }
            if (a.red_mode == RED_DOT_XW) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    red0[j] = fma(xv[c].x, w[c].x, red0[j]);
                    red0[j] = fma(xv[c].y, w[c].y, red0[j]);
                }
            }
        }
        SC* o = reinterpret_cast<SC*>(a.out[k]);
#pragma unroll
        for (int c = 0; c < 3; ++c) st_c(o + spinor_index<LAYOUT>(h, c, vh), w[c]);
        if (a.red_mode == RED_NORM_MAX_W) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                // reduce what was stored, so the norm matches the stored vector
                const RC sv = stored_value(w[c], (const SC*)o);
                const R n2 = sv.x * sv.x + sv.y * sv.y;
                red0[j] += n2;
                red1[j] = fmax(red1[j], sqrt(n2));
            }
        }
    }
}

// Per-rhs block reduction (warp tree -> shared -> partial slot) and the
// last-block finish. Called by every thread of the block.
template <int RPT, typename R>
__device__ __forceinline__ void block_reduce_finish(const DslashArgs& a, int k0, R (&red0)[RPT],
                                                    R (&red1)[RPT]) {
    // per-rhs block reduction: warp (fixed tree) -> shared -> partial slot
    __shared__ double s_part[kMaxRedVals][8];
    __shared__ double s_vals[kMaxRedVals];
    const int nv = (a.red_mode == RED_NORM_MAX_W) ? 2 : 1;
    const int lane = threadIdx.x & 31;
    const int wig = threadIdx.x >> 5;            // warp index within the group
    const int wpg = blockDim.x >> 5;             // warps per group
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const double s0 = (double)warp_sum(red0[j]);
        const double s1 = (double)warp_max(red1[j]);
        if (lane == 0) {
            s_part[(k0 + j) * nv][wig] = s0;
            if (nv == 2) s_part[(k0 + j) * nv + 1][wig] = s1;
        }
    }
    __syncthreads();
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nvals = a.nrhs * nv;
    if (tid < nvals) {
        const bool is_max = (nv == 2) && (tid & 1);
        double acc = 0.0;
        for (int w = 0; w < wpg; ++w) acc = is_max ? fmax(acc, s_part[tid][w]) : acc + s_part[tid][w];
        a.red.partials[(size_t)tid * kMaxRedBlocks + blockIdx.x] = acc;
    }
    if (!last_block_arrive(a.red.counter, gridDim.x)) return;
    finish_values(a.red, nvals, gridDim.x, [nv](int v) { return nv == 2 && (v & 1); }, s_vals);
    if (a.finish == FIN_CG_ALPHA) {
        finish_cg_alpha(a.cg, s_vals, a.nrhs);
    } else if (a.finish == FIN_RELIABLE) {
        finish_reliable(a.cg, s_vals, a.nrhs, a.tol2);
    } else if (a.red_out != nullptr && tid < nvals) {
        a.red_out[tid] = s_vals[tid];
    }
}

// Resident blocks per SM of one kernel, cached per device: every launcher
// (one per kernel instance) owns its cache and passes it in; the first call
// on a device measures the occupancy and sets the kernel's shared-memory
// attribute there. Kernels without dynamic shared memory (smem == 0) gather
// their neighbour vectors through L1, so they get the smallest shared-memory
// carveout that still holds as many blocks as their registers allow (the
// few KB of static reduction buffers per block would otherwise cap a
// zero carveout at two blocks); the rest of the SRAM is L1.
struct OccCache {
    std::atomic<int> v[64][16];
};

template <typename K>
cudaError_t cached_occupancy(OccCache& cache, K* kern, int threads, size_t smem, int slot, int* occ) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || slot < 0 || slot >= 16) return cudaErrorInvalidValue;
    int v = cache.v[dev][slot].load(std::memory_order_relaxed);
    if (v == 0) {
        if (smem == 0) {
            // the largest occupancy any carveout reaches, then the smallest
            // carveout (percent of the maximum shared memory) that reaches it
            const int carveouts[] = {0, 4, 8, 12, 16, 25, 50, 100};
            int occ_at[8] = {0};
            int best = 0;
            for (int i = 0; i < 8; ++i) {
                e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, carveouts[i]);
                if (e != cudaSuccess) return e;
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_at[i], kern, threads, 0);
                if (e != cudaSuccess) return e;
                if (occ_at[i] > best) best = occ_at[i];
            }
            int pick = 7;
            for (int i = 0; i < 8; ++i)
                if (occ_at[i] == best) {
                    pick = i;
                    break;
                }
            e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, carveouts[pick]);
            if (e != cudaSuccess) return e;
            v = best;
        } else {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, threads, smem);
            if (e != cudaSuccess) return e;
        }
        if (v < 1) v = 1;
        cache.v[dev][slot].store(v, std::memory_order_relaxed);
    }
    *occ = v;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Host-side launcher for one instance
// ---------------------------------------------------------------------------
template <typename S, typename LS, int RU, int RN, int RPT, int MINB, int EPI, int LAYOUT, bool PACK>
cudaError_t launch_dslash_instance(const DslashArgs& a, cudaStream_t s) {
    const int G = a.nrhs / RPT;
    if (G < 1 || G * RPT != a.nrhs || G > 8) return cudaErrorInvalidValue;
    int bx = 256 / G;
    bx &= ~31;
    const dim3 block(bx, G);
    auto* kern = dslash_kernel<S, LS, RU, RN, RPT, MINB, EPI, LAYOUT, PACK>;
    static OccCache cache;   // this kernel instance's occupancy per device
    int occ = 0;
    cudaError_t e = cached_occupancy(cache, kern, bx * G, 0, G, &occ);
    if (e != cudaSuccess) return e;
    long long nblk = ((long long)a.g.vh + bx - 1) / bx;
    long long cap = (long long)occ * device_sm_count();
    if (nblk > cap) nblk = cap;
    if (nblk > kMaxRedBlocks) nblk = kMaxRedBlocks;
    kern<<<(unsigned)nblk, block, 0, s>>>(a);
    return cudaGetLastError();
}

// Output site of the v-th visit. The sites of one (z, t) plane (an x-y block
// of hx Ly half sites, contiguous in memory) are visited together; the planes
// are visited with the longer of the z and t extents as the slow index. A
// site's neighbour chunks are read again by the sites up to three planes away
// along z and t, and the chunks must stay in L2 meanwhile: with the slow index
// running over the longer extent the visits in between cover 6 / max(Lz, Lt)
// of the lattice (1/8 at 48^3x12 instead of 1/2 with t slow), so the input
// spinors are read from DRAM about once.
__device__ __forceinline__ int visit_site(int v, const Geom& g) {
    if (g.L[2] <= g.L[3]) return v;    // t slow: memory order
    const int plane = g.sz;
    const int k = v / plane;
    const int z = k / g.L[3], t = k - z * g.L[3];
    return (t * g.L[2] + z) * plane + (v - k * plane);
}

}  // namespace hisq
