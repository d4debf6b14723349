// One (storage precision, fat recon, Naik recon) family of Dslash kernels.
//
// This file is compiled once per family with
//   -DHISQ_STORE=<double|float|__half> -DHISQ_LSTORE=<double|float|hisq::Fx16>
//   -DHISQ_RU=<18|12|14> -DHISQ_RN=<18|14>
//   -DHISQ_FAMILY=<function name> -DHISQ_MAX_RPT=<4|8> -DHISQ_WITH_XY=<0|1>
//   -DHISQ_LAYOUT=<0 (AoS)|1 (SoA)>
// so the families build in parallel translation units. Each family holds the
// thread mappings (rhs per thread, minimum resident blocks, kernel kind)
// listed in dslash_dispatch.cu, for one spinor layout. Kinds: 0 register
// kernel, 1 register kernel with packed f32x2 arithmetic, 2 links staged in
// shared memory by bulk copies, 3 and 4 register kernel with the loads of
// the next one or two hops in flight (software pipeline).
#include "dslash_pipe.cuh"
#include "dslash_staged.cuh"

#if !defined(HISQ_STORE) || !defined(HISQ_LSTORE) || !defined(HISQ_RU) || !defined(HISQ_RN) || !defined(HISQ_FAMILY) || \
    !defined(HISQ_LAYOUT)
#error "dslash_inst.cu needs HISQ_STORE, HISQ_RU, HISQ_RN, HISQ_FAMILY and HISQ_LAYOUT"
#endif

namespace hisq {

#define HISQ_INST(R, B, P) \
    launch_dslash_instance<S, LS, HISQ_RU, HISQ_RN, R, B, EPI, LAYOUT, P>(a, s)
#define HISQ_STAGED(R, B) launch_dslash_staged<S, LS, HISQ_RU, HISQ_RN, R, B, EPI, LAYOUT>(a, s)
#define HISQ_PIPE(R, B, D) launch_dslash_pipe<S, LS, HISQ_RU, HISQ_RN, R, B, D, EPI, LAYOUT>(a, s)

template <int EPI, int LAYOUT>
static cudaError_t family_by_variant(const DslashArgs& a, int rpt, int minb, int kind,
                                     cudaStream_t s) {
    using S = HISQ_STORE;       // spinor storage
    using LS = HISQ_LSTORE;     // link storage
    const int key = rpt * 100 + minb * 10 + kind;
    switch (key) {
#if HISQ_MAX_RPT >= 8
        // FP32 / FP16 storage, FP32 arithmetic
        case 140: return HISQ_INST(1, 4, false);
        case 230: return HISQ_INST(2, 3, false);
        case 231: return HISQ_INST(2, 3, true);
        case 420: return HISQ_INST(4, 2, false);
        case 421: return HISQ_INST(4, 2, true);
        case 430: return HISQ_INST(4, 3, false);
        case 820: return HISQ_INST(8, 2, false);
        case 821: return HISQ_INST(8, 2, true);
        case 422: return HISQ_STAGED(4, 2);
        case 432: return HISQ_STAGED(4, 3);
        case 822: return HISQ_STAGED(8, 2);
        case 832: return HISQ_STAGED(8, 3);
        case 423: return HISQ_PIPE(4, 2, 1);
        case 414: return HISQ_PIPE(4, 1, 2);
        case 424: return HISQ_PIPE(4, 2, 2);
        case 813: return HISQ_PIPE(8, 1, 1);
#else
        // FP64 storage and arithmetic
        case 120: return HISQ_INST(1, 2, false);
        case 220: return HISQ_INST(2, 2, false);
        case 410: return HISQ_INST(4, 1, false);
#endif
        default: return cudaErrorInvalidValue;
    }
}

#undef HISQ_INST
#undef HISQ_STAGED
#undef HISQ_PIPE

template <int LAYOUT>
static cudaError_t family_by_epi(const DslashArgs& a, int epi, int rpt, int minb, int kind,
                                 cudaStream_t s) {
    switch (epi) {
        case EPI_NONE: return family_by_variant<EPI_NONE, LAYOUT>(a, rpt, minb, kind, s);
        case EPI_X: return family_by_variant<EPI_X, LAYOUT>(a, rpt, minb, kind, s);
#if HISQ_WITH_XY
        case EPI_XY: return family_by_variant<EPI_XY, LAYOUT>(a, rpt, minb, kind, s);
#endif
        default: return cudaErrorInvalidValue;
    }
}

// One translation unit per (family, spinor layout): HISQ_LAYOUT selects it.
cudaError_t HISQ_FAMILY(const DslashArgs& a, int epi, int rpt, int minb, int kind, cudaStream_t s) {
    return family_by_epi<HISQ_LAYOUT>(a, epi, rpt, minb, kind, s);
}

}  // namespace hisq
