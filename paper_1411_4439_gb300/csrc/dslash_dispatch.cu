// Routes a Dslash request to the kernel family built for its storage
// precision and link compression (see dslash_inst.cu).
#include "hisq_internal.cuh"

namespace hisq {

cudaError_t dslash_f64_18_18(const DslashArgs&, int, int, int, int, cudaStream_t);
cudaError_t dslash_f32_18_18(const DslashArgs&, int, int, int, int, cudaStream_t);
cudaError_t dslash_f32_18_14(const DslashArgs&, int, int, int, int, cudaStream_t);
cudaError_t dslash_f32_12_14(const DslashArgs&, int, int, int, int, cudaStream_t);
cudaError_t dslash_f32_14_14(const DslashArgs&, int, int, int, int, cudaStream_t);
cudaError_t dslash_f16_18_18(const DslashArgs&, int, int, int, int, cudaStream_t);
cudaError_t dslash_f16_18_14(const DslashArgs&, int, int, int, int, cudaStream_t);
cudaError_t dslash_f16_12_14(const DslashArgs&, int, int, int, int, cudaStream_t);
cudaError_t dslash_f16_14_14(const DslashArgs&, int, int, int, int, cudaStream_t);

int dslash_max_rpt(int prec) { return prec == HISQ_F64 ? 4 : 8; }

// (rpt, minb) pairs compiled in dslash_inst.cu, default first
bool dslash_mapping_built(int prec, int rpt, int minb) {
    const int key = rpt * 10 + minb;
    if (prec == HISQ_F64) return key == 12 || key == 22 || key == 41;
    return key == 14 || key == 23 || key == 42 || key == 43 || key == 82;
}

int dslash_default_minb(int prec, int rpt) {
    if (prec == HISQ_F64) return rpt == 1 ? 2 : rpt == 2 ? 2 : rpt == 4 ? 1 : 0;
    return rpt == 1 ? 4 : rpt == 2 ? 3 : rpt == 4 ? 2 : rpt == 8 ? 2 : 0;
}

bool dslash_variant_supported(int prec, int ru, int rn, int epi) {
    if (prec == HISQ_F64) return ru == 18 && rn == 18 && epi >= EPI_NONE && epi <= EPI_XY;
    if (prec != HISQ_F32 && prec != HISQ_F16) return false;
    if (epi != EPI_NONE && epi != EPI_X) return false;
    return (ru == 18 && rn == 18) || (ru == 18 && rn == 14) || (ru == 12 && rn == 14) ||
           (ru == 14 && rn == 14);
}

cudaError_t launch_dslash(const DslashArgs& a, int prec, int ru, int rn, int epi,
                          const DslashTune& t, cudaStream_t s) {
    if (!dslash_variant_supported(prec, ru, rn, epi)) return cudaErrorInvalidValue;
    if (!dslash_mapping_built(prec, t.rpt, t.minb)) return cudaErrorInvalidValue;
    const int r = t.rpt, b = t.minb, l = t.layout;
    if (prec == HISQ_F64) return dslash_f64_18_18(a, epi, r, b, l, s);
    const int key = ru * 100 + rn;
    if (prec == HISQ_F32) {
        switch (key) {
            case 1818: return dslash_f32_18_18(a, epi, r, b, l, s);
            case 1814: return dslash_f32_18_14(a, epi, r, b, l, s);
            case 1214: return dslash_f32_12_14(a, epi, r, b, l, s);
            case 1414: return dslash_f32_14_14(a, epi, r, b, l, s);
        }
    } else {
        switch (key) {
            case 1818: return dslash_f16_18_18(a, epi, r, b, l, s);
            case 1814: return dslash_f16_18_14(a, epi, r, b, l, s);
            case 1214: return dslash_f16_12_14(a, epi, r, b, l, s);
            case 1414: return dslash_f16_14_14(a, epi, r, b, l, s);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace hisq
