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

template <int EPI>
static cudaError_t family_by_rpt(const DslashArgs& a, int rpt, cudaStream_t s) {
    using S = HISQ_STORE;
    switch (rpt) {
        case 1: return launch_dslash_instance<S, S, HISQ_RU, HISQ_RN, 1, EPI>(a, s);
        case 2: return launch_dslash_instance<S, S, HISQ_RU, HISQ_RN, 2, EPI>(a, s);
        case 4: return launch_dslash_instance<S, S, HISQ_RU, HISQ_RN, 4, EPI>(a, s);
#if HISQ_MAX_RPT >= 8
        case 8: return launch_dslash_instance<S, S, HISQ_RU, HISQ_RN, 8, EPI>(a, s);
#endif
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t HISQ_FAMILY(const DslashArgs& a, int epi, int rpt, cudaStream_t s) {
    switch (epi) {
        case EPI_NONE: return family_by_rpt<EPI_NONE>(a, rpt, s);
        case EPI_X: return family_by_rpt<EPI_X>(a, rpt, s);
#if HISQ_WITH_XY
        case EPI_XY: return family_by_rpt<EPI_XY>(a, rpt, s);
#endif
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hisq
