// Software-pipelined multi-rhs Dslash (Eq. 3 on a bundle, Eq. 4).
//
// Same thread mapping and arithmetic as dslash_kernel (one output site and
// RPT rhs per thread, blockDim.y rhs groups), but the 16 hops are a pipeline:
// the raw link components and the RPT neighbour vectors of hop e + DEPTH are
// loaded, in storage precision, into a rotating register buffer before hop e
// is multiplied. The gathers of a 32^3x8 bundle are L2 hits of several
// hundred cycles; with the loads of the next hop in flight during the
// 36 * RPT fused multiply-adds of the current one, a thread keeps about
// (9 + 3 RPT) loads outstanding all the time instead of only between hops.
// Temporal-only operators (d^n D / d mu^n) are not routed here.
#pragma once

#include "dslash_impl.cuh"

namespace hisq {

template <typename LC, typename SC, int NCMAX, int RPT>
struct HopRaw {
    LC l[NCMAX];
    SC v[RPT][3];
};

__device__ __forceinline__ float2 to_rc(float2 v) { return v; }
__device__ __forceinline__ double2 to_rc(double2 v) { return v; }
__device__ __forceinline__ float2 to_rc(__half2 v) { return __half22float2(v); }

template <typename S, typename LS, int RU, int RN, int RPT, int DEPTH, int LAYOUT>
struct DslashPipe {
    using R = typename Traits<S>::R;
    using RC = typename Cx<R>::T;
    using SC = typename Traits<S>::C;
    using LC = typename Traits<LS>::C;
    static constexpr int NCU = (RU == 18) ? 9 : (RU == 14 ? 7 : 6);
    static constexpr int NCN = (RN == 18) ? 9 : (RN == 14 ? 7 : 6);
    static constexpr int NCMAX = NCU > NCN ? NCU : NCN;
    static constexpr int NB = DEPTH + 1;
    using Raw = HopRaw<LC, SC, NCMAX, RPT>;

    const DslashArgs& a;
    const LC* __restrict__ Ub;
    const LC* __restrict__ Nb;
    int vh, p, q, k0, h, hrow, x, y, z, t;
    RC (&acc)[RPT][3];

    __device__ __forceinline__ DslashPipe(const DslashArgs& args, int h_, int k0_, RC (&acc_)[RPT][3])
        : a(args), acc(acc_) {
        Ub = reinterpret_cast<const LC*>(a.U);
        Nb = reinterpret_cast<const LC*>(a.N);
        vh = a.g.vh;
        p = a.parity;
        q = 1 - p;
        k0 = k0_;
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

    // neighbour (other parity) of the output site for hop E = 4 mu + hop
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
    __device__ __forceinline__ void issue(Raw& b) const {
        constexpr int MU = E >> 2, HOP = E & 3;
        constexpr bool NAIK = HOP >= 2;
        constexpr bool BACK = HOP & 1;
        constexpr int NC = NAIK ? NCN : NCU;
        const int hn = neighbour<E>();
        const LC* base = (NAIK ? Nb : Ub) + (size_t)((BACK ? q : p) * 4 + MU) * NC * vh;
        const int li = BACK ? hn : h;
        load_link_raw<LC, NC>(b.l, base, vh, li);
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            const SC* s = reinterpret_cast<const SC*>(a.in[k0 + j]);
#pragma unroll
            for (int c = 0; c < 3; ++c) b.v[j][c] = __ldg(s + spinor_index<LAYOUT>(hn, c, vh));
        }
    }

    template <int E>
    __device__ __forceinline__ void compute(const Raw& b) {
        constexpr int MU = E >> 2, HOP = E & 3;
        constexpr bool NAIK = HOP >= 2;
        constexpr int REC = NAIK ? RN : RU;
        constexpr int NC = NAIK ? NCN : NCU;
        const float* sc = NAIK ? a.lscale_n : a.lscale_u;
        Link<RC> m;
#pragma unroll
        for (int c = 0; c < 6; ++c) m.e[c] = link_elem(b.l[c], sc[c]);
        if constexpr (REC == 18) {
#pragma unroll
            for (int c = 6; c < 9; ++c) m.e[c] = link_elem(b.l[c], sc[c]);
        } else if constexpr (REC == 14) {
            third_row(m, link_elem(b.l[NC - 1], sc[NC - 1]));
        } else {
            // staggered sign of this site's mu links; eta_mu(x - mu) = eta_mu(x),
            // and the antiperiodic t boundary flips the wrapped link
            const int e = MU == 0 ? 0 : MU == 1 ? x : MU == 2 ? (x + y) : (x + y + z);
            int sgn = (e & 1) ? -1 : 1;
            if (MU == 3 && ((HOP == 0 && t == a.g.L[3] - 1) || (HOP == 1 && t == 0))) sgn = -sgn;
            const R inv_s = (sizeof(R) == 8) ? (R)a.r12_inv_scale : (R)(float)a.r12_inv_scale;
            RC f;
            f.x = sgn > 0 ? inv_s : -inv_s;
            f.y = (R)0;
            third_row(m, f);
        }
        if (MU == 3 && a.has_mu) {
            const double f = HOP == 0 ? a.ft1 : HOP == 1 ? a.bt1 : HOP == 2 ? a.ft3 : a.bt3;
            scale_link(m, (R)f);
        }
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            RC v[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) v[c] = to_rc(b.v[j][c]);
            if (HOP == 0 || HOP == 2)
                mv_add(acc[j], m, v);
            else
                mv_sub_dag(acc[j], m, v);
        }
    }

    template <int E>
    __device__ __forceinline__ void step(Raw (&buf)[NB]) {
        if constexpr (E + DEPTH < 16) issue<E + DEPTH>(buf[(E + DEPTH) % NB]);
        compute<E>(buf[E % NB]);
        if constexpr (E + 1 < 16) step<E + 1>(buf);
    }

    template <int I>
    __device__ __forceinline__ void prologue(Raw (&buf)[NB]) {
        if constexpr (I < DEPTH) {
            issue<I>(buf[I]);
            prologue<I + 1>(buf);
        }
    }

    __device__ __forceinline__ void run() {
        Raw buf[NB];
        prologue<0>(buf);
        step<0>(buf);
    }
};

// Epilogue with x read before the hops (xr, storage precision): the load is
// long done when the hops finish, where reading x after them measured 8 % of
// the launch at 32^3x8, n = 8. out = cx x + cd (D in), optional Re<x, out>.
template <typename SC, int RPT, int EPI, int LAYOUT, typename R, typename RC>
__device__ __forceinline__ void epilogue_site_px(const DslashArgs& a, int h, int k0, const RC (&acc)[RPT][3],
                                                 const SC (&xr)[RPT][3], R (&red0)[RPT], R (&red1)[RPT]) {
    static_assert(EPI == EPI_X, "the pipelined kernel's early-x epilogue serves EPI_X only");
    const int vh = a.g.vh;
    const R cx = (R)a.cx, cd = (R)a.cd;
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        RC w[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const RC xv = to_rc(xr[j][c]);
            w[c].x = fma(cd, acc[j][c].x, cx * xv.x);
            w[c].y = fma(cd, acc[j][c].y, cx * xv.y);
            if (a.red_mode == RED_DOT_XW) {
                red0[j] = fma(xv.x, w[c].x, red0[j]);
                red0[j] = fma(xv.y, w[c].y, red0[j]);
            }
        }
        SC* o = reinterpret_cast<SC*>(a.out[k0 + j]);
#pragma unroll
        for (int c = 0; c < 3; ++c) st_c(o + spinor_index<LAYOUT>(h, c, vh), w[c]);
        if (a.red_mode == RED_NORM_MAX_W) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const RC sv = stored_value(w[c], (const SC*)o);
                const R n2 = sv.x * sv.x + sv.y * sv.y;
                red0[j] += n2;
                red1[j] = fmax(red1[j], sqrt(n2));
            }
        }
    }
}

template <typename S, typename LS, int RU, int RN, int RPT, int MINB, int DEPTH, int EPI, int LAYOUT>
__global__ void __launch_bounds__(256, MINB) dslash_pipe_kernel(const DslashArgs a) {
    using R = typename Traits<S>::R;
    using RC = typename Cx<R>::T;
    using SC = typename Traits<S>::C;
    const int vh = a.g.vh;
    const int k0 = threadIdx.y * RPT;

    R red0[RPT], red1[RPT];
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        red0[j] = (R)0;
        red1[j] = (R)0;
    }
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v - (int)threadIdx.x < vh;
         v += gridDim.x * blockDim.x) {
        if (v >= vh) continue;
        const int h = visit_site(v, a.g);
        RC acc[RPT][3];
#pragma unroll
        for (int j = 0; j < RPT; ++j)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                acc[j][c].x = (R)0;
                acc[j][c].y = (R)0;
            }
        if constexpr (EPI == EPI_X) {
            SC xr[RPT][3];
#pragma unroll
            for (int j = 0; j < RPT; ++j)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    xr[j][c] = __ldg(reinterpret_cast<const SC*>(a.x[k0 + j]) + spinor_index<LAYOUT>(h, c, vh));
            DslashPipe<S, LS, RU, RN, RPT, DEPTH, LAYOUT> pipe(a, h, k0, acc);
            pipe.run();
            epilogue_site_px<SC, RPT, EPI, LAYOUT>(a, h, k0, acc, xr, red0, red1);
        } else {
            DslashPipe<S, LS, RU, RN, RPT, DEPTH, LAYOUT> pipe(a, h, k0, acc);
            pipe.run();
            epilogue_site<SC, RPT, EPI, LAYOUT>(a, h, k0, acc, red0, red1);
        }
    }
    if (a.red_mode == RED_NONE) return;
    block_reduce_finish<RPT>(a, k0, red0, red1);
}

template <typename S, typename LS, int RU, int RN, int RPT, int MINB, int DEPTH, int EPI, int LAYOUT>
cudaError_t launch_dslash_pipe(const DslashArgs& a, cudaStream_t s) {
    if (a.t_only) return cudaErrorInvalidValue;
    const int G = a.nrhs / RPT;
    if (G < 1 || G * RPT != a.nrhs || G > 8) return cudaErrorInvalidValue;
    int bx = 256 / G;
    bx &= ~31;
    const dim3 block(bx, G);
    auto* kern = dslash_pipe_kernel<S, LS, RU, RN, RPT, MINB, DEPTH, EPI, LAYOUT>;
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

}  // namespace hisq
