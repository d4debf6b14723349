// Routes a Dslash request to the kernel family built for its storage
// precision and link compression (see dslash_inst.cu), and owns the table of
// thread mappings those families contain.
#include "hisq_internal.cuh"

namespace hisq {

#define HISQ_FAMILY_DECL(name)                                                                     \
    cudaError_t name##_aos(const DslashArgs&, int epi, int rpt, int minb, int kind, cudaStream_t); \
    cudaError_t name##_soa(const DslashArgs&, int epi, int rpt, int minb, int kind, cudaStream_t);   \
    static cudaError_t name(const DslashArgs& a, int epi, int rpt, int minb, int kind, int layout,  \
                            cudaStream_t s) {                                                       \
        return layout == HISQ_SOA ? name##_soa(a, epi, rpt, minb, kind, s)                          \
                                  : name##_aos(a, epi, rpt, minb, kind, s);                         \
    }
HISQ_FAMILY_DECL(dslash_f64_18_18);
HISQ_FAMILY_DECL(dslash_f32_18_18);
HISQ_FAMILY_DECL(dslash_f32_18_14);
HISQ_FAMILY_DECL(dslash_f32_12_14);
HISQ_FAMILY_DECL(dslash_f32_14_14);
HISQ_FAMILY_DECL(dslash_f16_18_18);
HISQ_FAMILY_DECL(dslash_f16_18_14);
HISQ_FAMILY_DECL(dslash_f16_12_14);
HISQ_FAMILY_DECL(dslash_f16_14_14);
#undef HISQ_FAMILY_DECL

// bundle-layout families (dslash_bundle_inst.cu)
cudaError_t dslash_f32_18_18_bundle(const DslashArgs&, int, int, int, int, cudaStream_t);
cudaError_t dslash_f32_18_14_bundle(const DslashArgs&, int, int, int, int, cudaStream_t);
cudaError_t dslash_f32_12_14_bundle(const DslashArgs&, int, int, int, int, cudaStream_t);
cudaError_t dslash_f32_14_14_bundle(const DslashArgs&, int, int, int, int, cudaStream_t);
cudaError_t dslash_f16_18_18_bundle(const DslashArgs&, int, int, int, int, cudaStream_t);
cudaError_t dslash_f16_18_14_bundle(const DslashArgs&, int, int, int, int, cudaStream_t);
cudaError_t dslash_f16_12_14_bundle(const DslashArgs&, int, int, int, int, cudaStream_t);
cudaError_t dslash_f16_14_14_bundle(const DslashArgs&, int, int, int, int, cudaStream_t);

int dslash_max_rpt(int prec) { return prec == HISQ_F64 ? 4 : 8; }

// (rpt, minb, kind) of the bundle kernels: every family has the default
// mappings; the U r18 / N r14 families (the configurations' compression) also
// the variants the autotuner chooses from.
bool bundle_mapping_built(int prec, int ru, int rn, int rpt, int minb, int kind) {
    if (prec != HISQ_F32 && prec != HISQ_F16) return false;
    const int key = rpt * 1000 + minb * 100 + kind;
    if (key == 8305 || key == 4405 || key == 8309 || key == 8413) return true;
    if (!(ru == 18 && rn == 14)) return false;
    switch (key) {
        case 8205: case 4305: case 4409: case 8105: case 8106: case 8206: case 4306: case 8209: case 8409: case 4309:
        case 8210: case 8310: case 4310: case 4410: case 8211: case 8311: case 8411: case 8212: case 8312:
        case 4411: case 8313: case 8314: case 8414: case 4414: case 8315: case 8215:
            return true;
        default:
            return false;
    }
}

// Default bundle mapping for n rhs: eight rhs per thread when n allows
// (every link element then serves four rhs pairs), else four. Measured at
// 48^3x12, n = 8: FP16 storage runs fastest with the compact hop loop and
// the neighbour chunks staged in shared memory (16 warps per SM, 201 us),
// FP32 with the unrolled loop at 12 warps per SM (215 us).
DslashTune dslash_bundle_tune(int prec, int n) {
    DslashTune t;
    t.layout = HISQ_BUNDLE;
    t.kind = KIND_BUNDLE;
    t.prefetch = 0;
    t.rpt = 0;
    t.minb = 0;
    const int W = bundle_width(prec);
    if (W == 0 || n % W != 0) return t;
    if (n % 8 == 0 && n / 8 <= 4) {
        t.rpt = 8;
        t.minb = prec == HISQ_F16 ? 4 : 3;
        if (prec == HISQ_F16) t.kind = KIND_BUNDLE_CSMEM1;
    } else if (n % 4 == 0 && n / 4 <= 4) {
        t.rpt = 4;
        t.minb = 4;
    }
    return t;
}

// (rpt, minb, kind) triples compiled in dslash_inst.cu
bool dslash_mapping_built(int prec, int rpt, int minb, int kind) {
    const int key = rpt * 100 + minb * 10 + kind;
    if (prec == HISQ_F64) return key == 120 || key == 220 || key == 410;
    switch (key) {
        case 140: case 230: case 231: case 420: case 421: case 430: case 820: case 821:
        case 422: case 432: case 822: case 832:
        case 423: case 414: case 424: case 813:
            return true;
        default:
            return false;
    }
}

// Register kernel with the register budget measured best for an rpt (GB300,
// 32^3x8 and 48^3x12, n = 8, FP32).
DslashTune dslash_register_tune(int prec, int rpt, int layout) {
    DslashTune t;
    t.rpt = rpt;
    t.layout = layout;
    t.kind = KIND_REG;
    t.prefetch = 0;
    if (prec == HISQ_F64) {
        t.minb = rpt == 4 ? 1 : 2;
    } else {
        t.minb = rpt == 1 ? 4 : rpt == 2 ? 3 : 2;
    }
    return t;
}

// Default mapping for an rpt: with FP32/FP16 storage and four rhs per thread
// the kernel with the loads of the next two hops in flight (measured 6 % to
// 17 % faster than the register kernel at n = 4 and 8), else the register
// kernel.
DslashTune dslash_default_tune(int prec, int rpt, int layout) {
    DslashTune t = dslash_register_tune(prec, rpt, layout);
    if (prec != HISQ_F64 && rpt == 4) {
        t.minb = 2;
        t.kind = KIND_PIPE2;
    }
    return t;
}

// Tiles of 128 sites must be whole x-rows inside one y-z plane, and every
// row-sized bulk copy 16-byte aligned (see dslash_staged.cuh).
bool dslash_staged_ok(const Geom& g, int prec, int rpt, int groups) {
    if (prec != HISQ_F32 && prec != HISQ_F16) return false;
    if (groups < 1 || groups > (rpt >= 8 ? 1 : 2)) return false;
    const long long elem = prec == HISQ_F32 ? 8 : 4;
    const int ts = 128;
    return ts % g.hx == 0 && (g.hx * g.L[1]) % ts == 0 && (g.hx * elem) % 16 == 0 &&
           ((long long)g.vh * elem) % 16 == 0;
}

bool dslash_variant_supported(int prec, int ru, int rn, int epi) {
    if (prec == HISQ_F64) return ru == 18 && rn == 18 && epi >= EPI_NONE && epi <= EPI_XY;
    if (prec != HISQ_F32 && prec != HISQ_F16) return false;
    if (epi != EPI_NONE && epi != EPI_X) return false;
    return (ru == 18 && rn == 18) || (ru == 18 && rn == 14) || (ru == 12 && rn == 14) ||
           (ru == 14 && rn == 14);
}

static cudaError_t launch_bundle(const DslashArgs& a, int prec, int ru, int rn, int epi,
                                 const DslashTune& t, cudaStream_t s) {
    if (!bundle_mapping_built(prec, ru, rn, t.rpt, t.minb, t.kind)) return cudaErrorInvalidValue;
    if (epi != EPI_NONE && epi != EPI_X) return cudaErrorInvalidValue;
    const int r = t.rpt, b = t.minb, k = t.kind;
    const int key = ru * 100 + rn;
    if (prec == HISQ_F32) {
        switch (key) {
            case 1818: return dslash_f32_18_18_bundle(a, epi, r, b, k, s);
            case 1814: return dslash_f32_18_14_bundle(a, epi, r, b, k, s);
            case 1214: return dslash_f32_12_14_bundle(a, epi, r, b, k, s);
            case 1414: return dslash_f32_14_14_bundle(a, epi, r, b, k, s);
        }
    } else if (prec == HISQ_F16) {
        switch (key) {
            case 1818: return dslash_f16_18_18_bundle(a, epi, r, b, k, s);
            case 1814: return dslash_f16_18_14_bundle(a, epi, r, b, k, s);
            case 1214: return dslash_f16_12_14_bundle(a, epi, r, b, k, s);
            case 1414: return dslash_f16_14_14_bundle(a, epi, r, b, k, s);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_dslash(const DslashArgs& a, int prec, int ru, int rn, int epi,
                          const DslashTune& t, cudaStream_t s) {
    if (!dslash_variant_supported(prec, ru, rn, epi)) return cudaErrorInvalidValue;
    if (t.layout == HISQ_BUNDLE) return launch_bundle(a, prec, ru, rn, epi, t, s);
    if (!dslash_mapping_built(prec, t.rpt, t.minb, t.kind)) return cudaErrorInvalidValue;
    if (a.t_only && (t.kind == KIND_PIPE1 || t.kind == KIND_PIPE2)) {
        // the pipelined kernels run all 16 hops; temporal-only operators take
        // the register kernel of the same rhs count
        return launch_dslash(a, prec, ru, rn, epi, dslash_register_tune(prec, t.rpt, t.layout), s);
    }
    if (t.prefetch != a.l2_prefetch) {
        DslashArgs c = a;
        c.l2_prefetch = t.prefetch;
        return launch_dslash(c, prec, ru, rn, epi, t, s);
    }
    const int r = t.rpt, b = t.minb, k = t.kind, l = t.layout;
    if (prec == HISQ_F64) return dslash_f64_18_18(a, epi, r, b, k, l, s);
    const int key = ru * 100 + rn;
    if (prec == HISQ_F32) {
        switch (key) {
            case 1818: return dslash_f32_18_18(a, epi, r, b, k, l, s);
            case 1814: return dslash_f32_18_14(a, epi, r, b, k, l, s);
            case 1214: return dslash_f32_12_14(a, epi, r, b, k, l, s);
            case 1414: return dslash_f32_14_14(a, epi, r, b, k, l, s);
        }
    } else {
        switch (key) {
            case 1818: return dslash_f16_18_18(a, epi, r, b, k, l, s);
            case 1814: return dslash_f16_18_14(a, epi, r, b, k, l, s);
            case 1214: return dslash_f16_12_14(a, epi, r, b, k, l, s);
            case 1414: return dslash_f16_14_14(a, epi, r, b, k, l, s);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace hisq
