// Multi-rhs Dslash with the links staged through shared memory by bulk
// asynchronous copies (cp.async.bulk + mbarrier), one direction mu ahead.
//
// A block owns a tile of TS consecutive output sites of one parity (whole
// x-rows inside one y-z plane of constant z and t) and blockDim.y rhs groups.
// For every direction the tile needs four link runs per component: forward U
// and N of its own sites, and backward U and N of its neighbours. With the
// tile made of whole rows inside one plane, every run is one contiguous slice
// of a (parity, mu) link block, per component or component pair (the backward y runs split
// in two where y wraps). One thread issues the copies of direction mu+1 into
// the second buffer while all threads compute direction mu from the first,
// so link loads neither wait in registers nor occupy them. The neighbour
// spinors are gathered from L1/L2 as in the register kernel.
//
// Waits on the mbarrier are bounded; a wait that gives up records
// kFlagTimeout in *a.status and the block returns.
#pragma once

#include "dslash_impl.cuh"

namespace hisq {

constexpr int kStagedTile = 128;                 // output sites per tile
// Block size the kernel is compiled for: one group of 8 rhs per thread, or
// up to two groups of fewer rhs (the register budget follows from it).
__host__ __device__ constexpr int staged_max_threads(int rpt) { return rpt >= 8 ? 128 : 256; }
constexpr long long kWaitCycles = 4ll << 30;      // ~2 s of SM clock before a wait gives up

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Bounded wait for phase `parity` of `bar`: gives up (false) after about
// kWaitCycles SM clocks. Each try_wait returns after a bounded suspension.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
    const long long start = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - start > kWaitCycles) return false;
    return true;
}

// Runs per component of each link type lt (0 Ufwd, 1 Ubwd, 2 Nfwd, 3 Nbwd)
// and where they start in a stage buffer, in units of one tile run.
template <int NCU, int NCN>
__device__ __forceinline__ int NC_of(int lt) { return lt < 2 ? NCU : NCN; }
template <int NCU, int NCN>
__device__ __forceinline__ int staged_offset(int lt) {
    return lt == 0 ? 0 : lt == 1 ? NCU : lt == 2 ? 2 * NCU : 2 * NCU + NCN;
}

// Link of `recon` reals from a shared stage region laid out as a global block
// with V_h = ts: component c of tile site idx at base[link_offset(c, nc, ts, idx)].
template <typename LC, int RECON, typename RC>
__device__ __forceinline__ void load_link_shared(Link<RC>& m, const LC* base, int ts, int idx, float inv_s_f,
                                                 double inv_s_d, int sign, const float* sc) {
    using R = decltype(RC{}.x);
    constexpr int NC = (RECON == 18) ? 9 : (RECON == 14 ? 7 : 6);
#pragma unroll
    for (int c = 0; c < (RECON == 18 ? 9 : 6); ++c) {
        const auto v = link_elem(base[link_offset<LC>(c, NC, ts, idx)], sc[c]);
        m.e[c].x = (R)v.x;
        m.e[c].y = (R)v.y;
    }
    if (RECON == 14) {
        const auto zv = link_elem(base[link_offset<LC>(NC - 1, NC, ts, idx)], sc[NC - 1]);
        RC zz;
        zz.x = (R)zv.x;
        zz.y = (R)zv.y;
        third_row(m, zz);
    } else if (RECON == 12) {
        RC f;
        const R inv_s = (sizeof(R) == 8) ? (R)inv_s_d : (R)inv_s_f;
        f.x = sign > 0 ? inv_s : -inv_s;
        f.y = (R)0;
        third_row(m, f);
    }
}

// Link runs of one direction: component c of type lt (0 Ufwd, 1 Ubwd, 2 Nfwd,
// 3 Nbwd) lands at buf + (off[lt] + c) * TS, in output-site order for the
// forward runs and the backward runs of mu >= 1, and in neighbour order
// (index hn - h0) for the backward runs of mu = 0.
template <typename LC, int NCU, int NCN>
__device__ __forceinline__ unsigned issue_direction(LC* buf, const LC* Ub, const LC* Nb, const Geom& g,
                                                    int p, int h0, int mu, uint64_t* bar) {
    const int q = 1 - p, vh = g.vh, TS = kStagedTile;
    // coordinates shared by the whole tile: first row's y, the plane's z, t
    int r = h0 / g.hx;
    const int y0 = r % g.L[1];
    r /= g.L[1];
    const int z0 = r % g.L[2];
    const int t0 = r / g.L[2];
    const int rows = TS / g.hx;
    unsigned bytes = 0;
    // runs: (dst element, src element, count) per link type, up to two each
    long long src[4][2];
    int dst[4][2], cnt[4][2], nrun[4];
    for (int lt = 0; lt < 4; ++lt) {
        const bool back = lt & 1;
        const int d = (lt >= 2) ? 3 : 1;
        nrun[lt] = 1;
        dst[lt][0] = 0;
        cnt[lt][0] = TS;
        src[lt][0] = h0;
        if (!back || mu == 0) continue;
        if (mu == 1) {
            // rows with y < d wrap to y + Ly - d
            const int wrap_rows = (y0 < d) ? min(d - y0, rows) : 0;
            const int sy = g.sy;
            if (wrap_rows > 0) {
                src[lt][0] = h0 + (long long)(g.L[1] - d) * sy;
                cnt[lt][0] = wrap_rows * g.hx;
                if (wrap_rows < rows) {
                    nrun[lt] = 2;
                    dst[lt][1] = wrap_rows * g.hx;
                    src[lt][1] = h0 + (long long)wrap_rows * g.hx - (long long)d * sy;
                    cnt[lt][1] = TS - wrap_rows * g.hx;
                }
            } else {
                src[lt][0] = h0 - (long long)d * sy;
            }
        } else {
            const int c = (mu == 2) ? z0 : t0;
            const int L = g.L[mu];
            const int s = (mu == 2) ? g.sz : g.st;
            src[lt][0] = h0 + (long long)((c >= d) ? -d : L - d) * s;
        }
    }
    for (int lt = 0; lt < 4; ++lt)
        for (int k = 0; k < nrun[lt]; ++k) bytes += (unsigned)cnt[lt][k] * NC_of<NCU, NCN>(lt) * sizeof(LC);
    mbar_arrive_expect_tx(bar, bytes);
    for (int lt = 0; lt < 4; ++lt) {
        const bool back = lt & 1;
        const int nc = NC_of<NCU, NCN>(lt);
        const LC* base = (lt >= 2) ? Nb : Ub;
        const int par = back ? q : p;
        // the stage region of this link type mirrors the global block layout
        // (link_offset) with V_h replaced by the tile size
        LC* region = buf + (size_t)staged_offset<NCU, NCN>(lt) * TS;
        const LC* block = base + (size_t)(par * 4 + mu) * nc * vh;
        const int words = LinkPair<LC>::paired ? (nc + 1) / 2 : nc;
        for (int w = 0; w < words; ++w) {
            // a word is a component pair, or a single component (FP64, odd last)
            const bool pair = LinkPair<LC>::paired && 2 * w + 1 < nc;
            const int c0 = LinkPair<LC>::paired ? 2 * w : w;
            const int per = pair ? 2 : 1;
            for (int k = 0; k < nrun[lt]; ++k)
                bulk_copy_g2s(region + link_offset<LC>(c0, nc, TS, dst[lt][k]),
                              block + link_offset<LC>(c0, nc, vh, src[lt][k]),
                              (unsigned)cnt[lt][k] * per * sizeof(LC), bar);
        }
    }
    return bytes;
}

template <typename S, typename LS, int RU, int RN, int RPT, int MINB, int EPI, int LAYOUT>
__global__ void __launch_bounds__(staged_max_threads(RPT), MINB) dslash_staged_kernel(const DslashArgs a) {
    using R = typename Traits<S>::R;
    using RC = typename Cx<R>::T;
    using SC = typename Traits<S>::C;
    using LC = typename Traits<LS>::C;
    constexpr int NCU = (RU == 18) ? 9 : (RU == 14 ? 7 : 6);
    constexpr int NCN = (RN == 18) ? 9 : (RN == 14 ? 7 : 6);
    constexpr int NSTAGE = 2 * (NCU + NCN);   // component runs per direction
    constexpr int TS = kStagedTile;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    LC* bufs = reinterpret_cast<LC*>(smem_raw);                       // [2][NSTAGE][TS]
    __shared__ __align__(8) uint64_t bars[2];

    const Geom& g = a.g;
    const int vh = g.vh;
    const int p = a.parity;
    const int k0 = threadIdx.y * RPT;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const LC* __restrict__ Ub = reinterpret_cast<const LC*>(a.U);
    const LC* __restrict__ Nb = reinterpret_cast<const LC*>(a.N);
    const float inv_s_f = (float)a.r12_inv_scale;
    const int ntiles = vh / TS;

    R red0[RPT], red1[RPT];
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        red0[j] = (R)0;
        red1[j] = (R)0;
    }

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // steps are (tile, mu) in order; step s uses buffer s & 1, phase (s >> 1) & 1
    const int first = blockIdx.x;
    int step = 0;
    bool ok = true;
    bool next_issued = false;   // the copies of step + 1 were issued during step
    if (tid == 0 && first < ntiles)
        issue_direction<LC, NCU, NCN>(bufs, Ub, Nb, g, p, first * TS, 0, &bars[0]);

    for (int tile = first; tile < ntiles; tile += gridDim.x) {
        const int h0 = tile * TS;
        const int h = h0 + threadIdx.x;
        const int xh = h % g.hx;
        int r = h / g.hx;
        const int y = r % g.L[1];
        r /= g.L[1];
        const int z = r % g.L[2];
        const int t = r / g.L[2];
        const int x = 2 * xh + ((p + y + z + t) & 1);
        const int hrow = h - xh;

        RC acc[RPT][3];
#pragma unroll
        for (int j = 0; j < RPT; ++j)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                acc[j][c].x = (R)0;
                acc[j][c].y = (R)0;
            }

#pragma unroll 1
        for (int mu = 0; mu < 4; ++mu, ++step) {
            const int b = step & 1;
            // the buffer of the next step was last read in the previous step
            __syncthreads();
            const int ntile = (mu == 3) ? tile + gridDim.x : tile;
            next_issued = ntile < ntiles;
            if (tid == 0) {
                const int nmu = (mu + 1) & 3;
                if (ntile < ntiles) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    issue_direction<LC, NCU, NCN>(bufs + (size_t)(b ^ 1) * NSTAGE * TS, Ub, Nb, g, p,
                                                  ntile * TS, nmu, &bars[b ^ 1]);
                }
            }
            // one decision for the whole block, so no thread leaves a barrier
            // that the others still wait at
            const bool waited = mbar_wait_bounded(&bars[b], (step >> 1) & 1);
            if (__syncthreads_or(!waited)) {
                ok = false;
                break;
            }
            if (mu < 3 && a.t_only) continue;
            const LC* buf = bufs + (size_t)b * NSTAGE * TS;
            const int coord = (mu == 0) ? x : (mu == 1) ? y : (mu == 2) ? z : t;
            const int ext = g.L[mu];
            const int stride = (mu == 1) ? g.sy : (mu == 2) ? g.sz : g.st;
            int eta = 1;
            if (RU == 12) {
                const int e = (mu == 0) ? 0 : (mu == 1) ? x : (mu == 2) ? (x + y) : (x + y + z);
                eta = (e & 1) ? -1 : 1;
            }
#pragma unroll
            for (int hop = 0; hop < 4; ++hop) {
                const int d = (hop == 0) ? 1 : (hop == 1) ? -1 : (hop == 2) ? 3 : -3;
                const int cn = wrap(coord + d, ext);
                int hn;
                if (mu == 0)
                    hn = hrow + (cn >> 1);
                else if (mu == 1)
                    hn = h + (cn - coord) * stride;
                else
                    hn = h + (cn - coord) * stride;
                const int lt = hop == 0 ? 0 : hop == 1 ? 1 : hop == 2 ? 2 : 3;
                const int sidx = (mu == 0 && (hop & 1)) ? hn - h0 : threadIdx.x;
                const LC* base = buf + (size_t)staged_offset<NCU, NCN>(lt) * TS;
                Link<RC> m;
                if (hop < 2) {
                    int sgn = eta;
                    if (RU == 12 && mu == 3) {
                        if (hop == 0 && t == ext - 1) sgn = -eta;
                        if (hop == 1 && t == 0) sgn = -eta;
                    }
                    load_link_shared<LC, RU, RC>(m, base, TS, sidx, inv_s_f, a.r12_inv_scale, sgn, a.lscale_u);
                } else {
                    load_link_shared<LC, RN, RC>(m, base, TS, sidx, inv_s_f, a.r12_inv_scale, 1, a.lscale_n);
                }
                if (mu == 3 && a.has_mu) {
                    const double f = (hop == 0) ? a.ft1 : (hop == 1) ? a.bt1 : (hop == 2) ? a.ft3 : a.bt3;
                    scale_link(m, (R)f);
                }
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
        if (!ok) break;
        epilogue_site<SC, RPT, EPI, LAYOUT>(a, h, k0, acc, red0, red1);
    }
    if (!ok) {
        // Record the failure. No bulk copy may still be writing into this
        // block's shared memory when it exits, so both buffers' outstanding
        // copies get a bounded chance to land: those of the step whose wait
        // gave up, and those of the next step if they were issued.
        if (tid == 0 && a.status != nullptr) atomicOr(a.status, kFlagTimeout);
        mbar_wait_bounded(&bars[step & 1], (step >> 1) & 1);
        if (next_issued) mbar_wait_bounded(&bars[(step + 1) & 1], ((step + 1) >> 1) & 1);
        return;
    }
    if (a.red_mode == RED_NONE) return;
    block_reduce_finish<RPT>(a, k0, red0, red1);
}

// True when the tile of kStagedTile whole rows lies inside one y-z plane and
// every bulk copy is 16-byte aligned for link elements of `elem` bytes.
inline bool staged_geometry_ok(const Geom& g, size_t elem) {
    const int TS = kStagedTile;
    if (TS % g.hx != 0) return false;
    if ((g.hx * g.L[1]) % TS != 0) return false;
    if ((g.hx * elem) % 16 != 0) return false;     // row-sized runs and row shifts
    if (((size_t)g.vh * elem) % 16 != 0) return false;
    return true;
}

template <typename S, typename LS, int RU, int RN, int RPT, int MINB, int EPI, int LAYOUT>
cudaError_t launch_dslash_staged(const DslashArgs& a, cudaStream_t s) {
    using LC = typename Traits<LS>::C;
    constexpr int NCU = (RU == 18) ? 9 : (RU == 14 ? 7 : 6);
    constexpr int NCN = (RN == 18) ? 9 : (RN == 14 ? 7 : 6);
    const int G = a.nrhs / RPT;
    if (G < 1 || G * RPT != a.nrhs || G * kStagedTile > staged_max_threads(RPT)) return cudaErrorInvalidValue;
    if (!staged_geometry_ok(a.g, sizeof(LC))) return cudaErrorInvalidValue;
    const dim3 block(kStagedTile, G);
    const size_t smem = 2ull * 2 * (NCU + NCN) * kStagedTile * sizeof(LC);
    auto* kern = dslash_staged_kernel<S, LS, RU, RN, RPT, MINB, EPI, LAYOUT>;
    static OccCache cache;   // this kernel instance's occupancy per device
    int occ = 0;
    cudaError_t e = cached_occupancy(cache, kern, kStagedTile * G, smem, G, &occ);
    if (e != cudaSuccess) return e;
    long long nblk = a.g.vh / kStagedTile;
    const long long cap = (long long)occ * device_sm_count();
    if (nblk > cap) nblk = cap;
    if (nblk > kMaxRedBlocks) nblk = kMaxRedBlocks;
    kern<<<(unsigned)nblk, block, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace hisq
