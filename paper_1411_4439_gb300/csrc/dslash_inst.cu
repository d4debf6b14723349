// One (storage precision, fat recon, Naik recon) family of Dslash kernels.
//
// This file is compiled once per family with
//   -DHISQ_STORE=<double|float|__half> -DHISQ_RU=<18|12|14> -DHISQ_RN=<18|14>
//   -DHISQ_FAMILY=<function name>
// so the families build in parallel translation units.
#include "dslash_impl.cuh"

#if !defined(HISQ_STORE) || !defined(HISQ_RU) || !defined(HISQ_RN) || !defined(HISQ_FAMILY)
#error "dslash_inst.cu needs HISQ_STORE, HISQ_RU, HISQ_RN and HISQ_FAMILY"
#endif

namespace hisq {

template <int EPI, int LAYOUT>
static cudaError_t family_by_variant(const DslashArgs& a, int rpt, int minb, cudaStream_t s) {
    using S = HISQ_STORE;
    const int key = rpt * 10 + minb;
    switch (key) {
#if HISQ_MAX_RPT >= 8
        // FP32 / FP16 storage
        case 14: return launch_dslash_instance<S, S, HISQ_RU, HISQ_RN, 1, 4, EPI, LAYOUT>(a, s);
        case 23: return launch_dslash_instance<S, S, HISQ_RU, HISQ_RN, 2, 3, EPI, LAYOUT>(a, s);
        case 42: return launch_dslash_instance<S, S, HISQ_RU, HISQ_RN, 4, 2, EPI, LAYOUT>(a, s);
        case 43: return launch_dslash_instance<S, S, HISQ_RU, HISQ_RN, 4, 3, EPI, LAYOUT>(a, s);
        case 82: return launch_dslash_instance<S, S, HISQ_RU, HISQ_RN, 8, 2, EPI, LAYOUT>(a, s);
#else
        // FP64 storage
        case 12: return launch_dslash_instance<S, S, HISQ_RU, HISQ_RN, 1, 2, EPI, LAYOUT>(a, s);
        case 22: return launch_dslash_instance<S, S, HISQ_RU, HISQ_RN, 2, 2, EPI, LAYOUT>(a, s);
        case 41: return launch_dslash_instance<S, S, HISQ_RU, HISQ_RN, 4, 1, EPI, LAYOUT>(a, s);
#endif
        default: return cudaErrorInvalidValue;
    }
}

template <int LAYOUT>
static cudaError_t family_by_epi(const DslashArgs& a, int epi, int rpt, int minb, cudaStream_t s) {
    switch (epi) {
        case EPI_NONE: return family_by_variant<EPI_NONE, LAYOUT>(a, rpt, minb, s);
        case EPI_X: return family_by_variant<EPI_X, LAYOUT>(a, rpt, minb, s);
#if HISQ_WITH_XY
        case EPI_XY: return family_by_variant<EPI_XY, LAYOUT>(a, rpt, minb, s);
#endif
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t HISQ_FAMILY(const DslashArgs& a, int epi, int rpt, int minb, int layout, cudaStream_t s) {
    return layout == HISQ_SOA ? family_by_epi<HISQ_SOA>(a, epi, rpt, minb, s)
                              : family_by_epi<HISQ_AOS>(a, epi, rpt, minb, s);
}

}  // namespace hisq
