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

// kind -> hop loop: 5 unrolled, next link ahead; 6 unrolled, next link and
// neighbours ahead; 9 compact, next link ahead; 10 compact, next link and
// neighbours ahead
#define HISQ_B(R, B, SD, COMPACT) \
    launch_dslash_bundle<S, LS, HISQ_RU, HISQ_RN, R, B, true, 1, SD, EPI, COMPACT>(a, s)
#define HISQ_BS(R, B, D) launch_dslash_bundle<S, LS, HISQ_RU, HISQ_RN, R, B, true, 1, 0, EPI, false, D>(a, s)

template <int EPI>
static cudaError_t bundle_by_variant(const DslashArgs& a, int rpt, int minb, int kind, cudaStream_t s) {
    using S = HISQ_STORE;
    using LS = HISQ_LSTORE;
    const int key = rpt * 1000 + minb * 100 + kind;
    switch (key) {
        case 8305: return HISQ_B(8, 3, 0, false);
        case 4405: return HISQ_B(4, 4, 0, false);
        case 8309: return HISQ_B(8, 3, 0, true);
        case 8413: return HISQ_BS(8, 4, 11);
#if HISQ_BUNDLE_FULL
        case 8205: return HISQ_B(8, 2, 0, false);
        case 4305: return HISQ_B(4, 3, 0, false);
        case 4409: return HISQ_B(4, 4, 0, true);
        case 8105: return HISQ_B(8, 1, 0, false);
        case 8106: return HISQ_B(8, 1, 1, false);
        case 8206: return HISQ_B(8, 2, 1, false);
        case 4306: return HISQ_B(4, 3, 1, false);
        case 8209: return HISQ_B(8, 2, 0, true);
        case 8409: return HISQ_B(8, 4, 0, true);
        case 4309: return HISQ_B(4, 3, 0, true);
        case 8210: return HISQ_B(8, 2, 1, true);
        case 8310: return HISQ_B(8, 3, 1, true);
        case 4310: return HISQ_B(4, 3, 1, true);
        case 4410: return HISQ_B(4, 4, 1, true);
        // neighbour chunks staged in shared memory D hops ahead: kind 11 (D = 1), 12 (D = 2)
        case 8211: return HISQ_BS(8, 2, 1);
        case 8311: return HISQ_BS(8, 3, 1);
        case 8411: return HISQ_BS(8, 4, 1);
        case 8212: return HISQ_BS(8, 2, 2);
        case 8312: return HISQ_BS(8, 3, 2);
        case 4411: return HISQ_BS(4, 4, 1);
        // compact loop with neighbours staged in shared memory: kind 13 (D = 1), 14 (D = 3)
        case 8313: return HISQ_BS(8, 3, 11);
        case 8314: return HISQ_BS(8, 3, 13);
        case 8414: return HISQ_BS(8, 4, 13);
        case 4414: return HISQ_BS(4, 4, 13);
        // unrolled loop with the x/y neighbour tile in shared memory: kind 15
        case 8315: return HISQ_BS(8, 3, 30);
        case 8215: return HISQ_BS(8, 2, 30);
#endif
        default: return cudaErrorInvalidValue;
    }
}

#undef HISQ_B
#undef HISQ_BS

cudaError_t HISQ_FAMILY(const DslashArgs& a, int epi, int rpt, int minb, int kind, cudaStream_t s) {
    switch (epi) {
        case EPI_NONE: return bundle_by_variant<EPI_NONE>(a, rpt, minb, kind, s);
        case EPI_X: return bundle_by_variant<EPI_X>(a, rpt, minb, kind, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hisq
