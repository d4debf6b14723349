// Block partials plus a last-block finish, in a fixed order (deterministic).
//
// Every block writes one partial per reduced value to
// partials[value * kMaxRedBlocks + blockIdx.x], fences, and bumps a counter;
// the block that arrives last sums the partials of every value in a fixed
// order (one warp per value, lane-strided, then a fixed shuffle tree), resets
// the counter for the next launch and runs the finish logic.
#pragma once

#include "hisq_internal.cuh"

namespace hisq {

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename R>
__device__ __forceinline__ R warp_max(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Signals arrival of this block; true in the block that arrived last.
__device__ __forceinline__ bool last_block_arrive(unsigned int* counter, unsigned int nblocks) {
    __shared__ unsigned int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const unsigned int prev = atomicAdd(counter, 1u);
        s_last = (prev == nblocks - 1u) ? 1u : 0u;
    }
    __syncthreads();
    return s_last != 0u;
}

// In the last block: out[v] = sum (or max, when is_max(v)) over slots of
// partials[v][0 .. nslots). Must be called by all threads of the block.
template <typename IsMax>
__device__ __forceinline__ void finish_values(const RedScratch& red, int nvals, int nslots,
                                              IsMax is_max, double* out_smem) {
    __threadfence();
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nthreads = blockDim.x * blockDim.y;
    const int warp = tid >> 5, lane = tid & 31, nwarps = nthreads >> 5;
    for (int v = warp; v < nvals; v += nwarps) {
        const double* src = red.partials + (size_t)v * kMaxRedBlocks;
        const bool mx = is_max(v);
        double acc = 0.0;
        for (int i = lane; i < nslots; i += 32) {
            const double t = __ldcg(src + i);
            acc = mx ? fmax(acc, t) : acc + t;
        }
        acc = mx ? warp_max(acc) : warp_sum(acc);
        if (lane == 0) out_smem[v] = acc;
    }
    if (tid == 0) *red.counter = 0u;
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Finish logic shared by the Dslash and vector kernels
// ---------------------------------------------------------------------------

// An rhs moves (takes part in alpha/beta updates) while active and not frozen.
__device__ __forceinline__ bool moving(const CgScalars* cg, int k) {
    return cg->active[k] && !cg->frozen[k];
}

// pAp -> alpha_k = rr_k / pAp_k for moving rhs. A non-finite pAp is an error;
// pAp <= 0 means the low-precision iteration lost A-conjugacy: alpha = 0 and
// this iteration restarts the rhs from p = r (beta = 0).
__device__ __forceinline__ void finish_cg_alpha(CgScalars* cg, const double* vals, int n) {
    const int k = threadIdx.x + threadIdx.y * blockDim.x;
    if (k < n) {
        const double pAp = vals[k];
        double alpha = 0.0;
        if (moving(cg, k)) {
            if (!isfinite(pAp)) {
                atomicOr(&cg->flags, kFlagNaN);
            } else if (!(pAp > 0.0) || !(cg->rr[k] <= cg->alpha_max * pAp)) {
                // pAp <= 0, or alpha above 1/lambda_min: the low-precision
                // iteration lost conjugacy; restart this rhs from p = r
                cg->stall[k] = 1;
            } else {
                alpha = cg->rr[k] / pAp;
            }
        }
        cg->pAp[k] = pAp;
        cg->alpha[k] = alpha;
    }
}

// rr' -> beta_k = rr'_k / rr_k, rr_k = rr'_k for moving rhs; freezes an rhs
// whose residual fell by more than freeze2 since the last reliable update.
__device__ __forceinline__ void finish_cg_beta(CgScalars* cg, const double* vals, int n) {
    const int k = threadIdx.x + threadIdx.y * blockDim.x;
    if (k < n) {
        double beta = 0.0;
        if (moving(cg, k)) {
            const double rr_new = vals[k];
            if (!isfinite(rr_new)) {
                atomicOr(&cg->flags, kFlagNaN);
            } else {
                if (cg->stall[k]) {
                    cg->stall[k] = 0;
                    cg->restarts[k] += 1;
                } else if (cg->rr[k] > 0.0) {
                    beta = rr_new / cg->rr[k];
                }
                cg->rr[k] = rr_new;
                if (rr_new <= cg->freeze2 * cg->rr_rel[k]) cg->frozen[k] = 1;
            }
        }
        cg->beta[k] = beta;
    }
}

// FP64 true residual (|r|^2 at vals[2k], max|r_i| at vals[2k+1]): record it,
// retire rhs whose residual meets tol2 * |b|^2, pick the next scale.
__device__ __forceinline__ void finish_reliable(CgScalars* cg, const double* vals, int n,
                                                double tol2) {
    const int k = threadIdx.x + threadIdx.y * blockDim.x;
    if (k < n) {
        const double nrm = vals[2 * k], mx = vals[2 * k + 1];
        // The search direction p is kept across the update while the
        // iterated residual still describes the true one. Once the true
        // residual is 10x (in norm) above the iterated one, the iteration has
        // run into its rounding floor and p no longer belongs to this
        // residual; a frozen rhs skipped its last p update. Both restart
        // from p = r.
        const double sc = cg->scale[k];
        const double iterated = cg->rr[k] / (sc * sc);
        cg->reset_p[k] = (nrm > 100.0 * iterated || cg->frozen[k]) ? 1 : 0;
        cg->rr_true[k] = nrm;
        cg->rmax[k] = mx;
        const int better = isfinite(nrm) && (!cg->have_best[k] || nrm < cg->rr_best[k]);
        cg->keep[k] = better;
        if (better) {
            cg->rr_best[k] = nrm;
            cg->have_best[k] = 1;
        }
        if (!isfinite(nrm)) {
            atomicOr(&cg->flags, kFlagNaN);
            cg->active[k] = 0;
        } else if (cg->active[k] && nrm <= tol2 * cg->bb[k]) {
            cg->active[k] = 0;
        }
        cg->scale_old[k] = cg->scale[k];
        cg->scale[k] = (mx > 0.0 && isfinite(mx)) ? 1.0 / mx : 1.0;
    }
}

}  // namespace hisq
