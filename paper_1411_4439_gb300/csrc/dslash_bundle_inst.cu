// One (storage precision, fat recon, Naik recon) family of bundle-layout
// Dslash kernels (dslash_bundle.cuh).
//
// Compiled once per FP32 / FP16 family with
//   -DHISQ_STORE=<float|__half> -DHISQ_LSTORE=<float|hisq::Fx16>
//   -DHISQ_RU=<18|12|14> -DHISQ_RN=<18|14> -DHISQ_FAMILY=<function name>
//   -DHISQ_BUNDLE_FULL=<0|1>
// HISQ_BUNDLE_FULL builds every (rhs per thread, min blocks, kind) mapping the
// autotuner can choose from; otherwise the default mappings only.
#include "dslash_bundle.cuh"

#if !defined(HISQ_STORE) || !defined(HISQ_LSTORE) || !defined(HISQ_RU) || !defined(HISQ_RN) || !defined(HISQ_FAMILY)
#error "dslash_bundle_inst.cu needs HISQ_STORE, HISQ_LSTORE, HISQ_RU, HISQ_RN and HISQ_FAMILY"
#endif

namespace hisq {

// kind -> (packed arithmetic, link look-ahead, neighbour look-ahead)
#define HISQ_B(R, B, PK, LD, SD) \
    launch_dslash_bundle<S, LS, HISQ_RU, HISQ_RN, R, B, PK, LD, SD, EPI>(a, s)

template <int EPI>
static cudaError_t bundle_by_variant(const DslashArgs& a, int rpt, int minb, int kind, cudaStream_t s) {
    using S = HISQ_STORE;
    using LS = HISQ_LSTORE;
    const int key = rpt * 100 + minb * 10 + kind;
    switch (key) {
        case 825: return HISQ_B(8, 2, true, 1, 0);
        case 435: return HISQ_B(4, 3, true, 1, 0);
#if HISQ_BUNDLE_FULL
        case 815: return HISQ_B(8, 1, true, 1, 0);
        case 835: return HISQ_B(8, 3, true, 1, 0);
        case 445: return HISQ_B(4, 4, true, 1, 0);
        case 816: return HISQ_B(8, 1, true, 1, 1);
        case 826: return HISQ_B(8, 2, true, 1, 1);
        case 436: return HISQ_B(4, 3, true, 1, 1);
        case 827: return HISQ_B(8, 2, false, 1, 0);
        case 837: return HISQ_B(8, 3, false, 1, 0);
        case 437: return HISQ_B(4, 3, false, 1, 0);
        case 447: return HISQ_B(4, 4, false, 1, 0);
        case 828: return HISQ_B(8, 2, true, 0, 0);
        case 838: return HISQ_B(8, 3, true, 0, 0);
        case 448: return HISQ_B(4, 4, true, 0, 0);
#endif
        default: return cudaErrorInvalidValue;
    }
}

#undef HISQ_B

cudaError_t HISQ_FAMILY(const DslashArgs& a, int epi, int rpt, int minb, int kind, cudaStream_t s) {
    switch (epi) {
        case EPI_NONE: return bundle_by_variant<EPI_NONE>(a, rpt, minb, kind, s);
        case EPI_X: return bundle_by_variant<EPI_X>(a, rpt, minb, kind, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hisq
