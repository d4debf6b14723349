// Routes a Dslash request to the kernel family built for its storage
// precision and link compression (see dslash_inst.cu).
#include "hisq_internal.cuh"

namespace hisq {

cudaError_t dslash_f64_18_18(const DslashArgs&, int, int, cudaStream_t);
cudaError_t dslash_f32_18_18(const DslashArgs&, int, int, cudaStream_t);
cudaError_t dslash_f32_18_14(const DslashArgs&, int, int, cudaStream_t);
cudaError_t dslash_f32_12_14(const DslashArgs&, int, int, cudaStream_t);
cudaError_t dslash_f32_14_14(const DslashArgs&, int, int, cudaStream_t);
cudaError_t dslash_f16_18_18(const DslashArgs&, int, int, cudaStream_t);
cudaError_t dslash_f16_18_14(const DslashArgs&, int, int, cudaStream_t);
cudaError_t dslash_f16_12_14(const DslashArgs&, int, int, cudaStream_t);
cudaError_t dslash_f16_14_14(const DslashArgs&, int, int, cudaStream_t);

int dslash_max_rpt(int prec) { return prec == HISQ_F64 ? 4 : 8; }

bool dslash_variant_supported(int prec, int ru, int rn, int epi) {
    if (prec == HISQ_F64) return ru == 18 && rn == 18 && epi >= EPI_NONE && epi <= EPI_XY;
    if (prec != HISQ_F32 && prec != HISQ_F16) return false;
    if (epi != EPI_NONE && epi != EPI_X) return false;
    return (ru == 18 && rn == 18) || (ru == 18 && rn == 14) || (ru == 12 && rn == 14) ||
           (ru == 14 && rn == 14);
}

cudaError_t launch_dslash(const DslashArgs& a, int prec, int ru, int rn, int epi, int rpt,
                          cudaStream_t s) {
    if (!dslash_variant_supported(prec, ru, rn, epi)) return cudaErrorInvalidValue;
    if (prec == HISQ_F64) return dslash_f64_18_18(a, epi, rpt, s);
    const int key = ru * 100 + rn;
    if (prec == HISQ_F32) {
        switch (key) {
            case 1818: return dslash_f32_18_18(a, epi, rpt, s);
            case 1814: return dslash_f32_18_14(a, epi, rpt, s);
            case 1214: return dslash_f32_12_14(a, epi, rpt, s);
            case 1414: return dslash_f32_14_14(a, epi, rpt, s);
        }
    } else {
        switch (key) {
            case 1818: return dslash_f16_18_18(a, epi, rpt, s);
            case 1814: return dslash_f16_18_14(a, epi, rpt, s);
            case 1214: return dslash_f16_12_14(a, epi, rpt, s);
            case 1414: return dslash_f16_14_14(a, epi, rpt, s);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace hisq
