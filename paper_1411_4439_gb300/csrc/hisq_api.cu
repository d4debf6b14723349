// C ABI of libhisq: gauge handles, Dslash and normal-operator entry points,
// and the mixed-precision multi-rhs CG driver.
//
// The CG (Hestenes-Stiefel, one independent CG per rhs sharing each Dslash)
// keeps all of its scalars on the device: alpha and beta are formed by the
// last block of the reduction that produces their numerators/denominators,
// so an iteration is four kernel launches with no host round trip. The host
// polls the scalars every `check_every` iterations to decide on FP64
// reliable updates (every `reliable_every` iterations, or when a residual
// fell by `reliable_delta`, or when an iterated residual claims
// convergence), and replays the iterations from a captured CUDA graph.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "hisq_internal.cuh"

using namespace hisq;

namespace {

thread_local std::string g_last_error;

hisq_status fail(hisq_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define HISQ_CUDA(call)                                                                   \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? HISQ_ENOMEM : HISQ_ECUDA,       \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                        \
    } while (0)

size_t prec_complex_bytes(int prec) {
    return prec == HISQ_F64 ? 16 : prec == HISQ_F32 ? 8 : 4;
}

bool valid_prec(int p) { return p == HISQ_F64 || p == HISQ_F32 || p == HISQ_F16; }

// Storage of the CG's low-precision solution increment: FP16 iterations keep
// it in FP32 (see XType in blas.cu).
int solution_prec(int prec) { return prec == HISQ_F16 ? HISQ_F32 : prec; }

hisq_status make_geom(const int L[4], Geom* g) {
    if (L == nullptr) return fail(HISQ_EINVAL, "lattice extents pointer is NULL");
    long long V = 1;
    for (int m = 0; m < 4; ++m) {
        if (L[m] < 4 || (L[m] & 1))
            return fail(HISQ_EINVAL, "extent L[%d] = %d must be even and >= 4", m, L[m]);
        V *= L[m];
    }
    // internal link slabs index up to 2 * 4 * 9 * V_h elements with 32-bit site math
    if (V / 2 > (1ll << 26)) return fail(HISQ_EINVAL, "lattice too large (V = %lld)", V);
    for (int m = 0; m < 4; ++m) g->L[m] = L[m];
    g->hx = L[0] / 2;
    g->vh = (int)(V / 2);
    g->sy = g->hx;
    g->sz = g->hx * L[1];
    g->st = g->hx * L[1] * L[2];
    return HISQ_OK;
}

// Device pointer test: memory the GPU can address directly (device or managed).
bool is_device_pointer(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

namespace hisq {
// Message for hisq_last_error() from entry points in other translation units.
void record_error(const char* msg) { g_last_error = msg; }

int device_sm_count() {
    // per device; atomic so that host threads launching concurrently read
    // either 0 (and query) or the stored count
    static std::atomic<int> cached[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    int v = cached[dev].load(std::memory_order_relaxed);
    if (v == 0) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        v = n > 0 ? n : 1;
        cached[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}
}  // namespace hisq

// ---------------------------------------------------------------------------
// Workspaces
// ---------------------------------------------------------------------------
namespace {

struct GraphKey {
    int chunk;
    double mass, mu;
    int rpt;   // the mapping and variant of the captured kernels, encoded
    bool operator<(const GraphKey& o) const {
        return std::tie(chunk, mass, mu, rpt) < std::tie(o.chunk, o.mass, o.mu, o.rpt);
    }
};

struct Workspace {
    int n = 0, prec = 0, full = 0;
    long long len = 0;           // complex numbers per rhs of one CG vector
    long long len_half = 0;      // complex numbers per rhs of one parity (3 V_h)
    void* r_lo = nullptr;
    void* p_lo = nullptr;
    void* Ap_lo = nullptr;
    void* x_lo = nullptr;
    void* t_lo = nullptr;        // operator temporary
    double2* b_hi = nullptr;
    double2* x_hi = nullptr;
    double2* r_hi = nullptr;
    double2* t_hi = nullptr;
    double2* x_best = nullptr;   // the solution at the lowest FP64 residual so far
    CgScalars* cg = nullptr;
    CgScalars* cg_host = nullptr;
    double* partials = nullptr;
    unsigned int* counter = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t cap_body = nullptr;   // captures the device loop's body
    cudaStream_t cap_if = nullptr;     // captures its reliable-update branch
    std::map<GraphKey, cudaGraphExec_t> graphs;
    std::map<std::tuple<int, double, double, int, int, int, double, double>, cudaGraphExec_t> loops;
    std::vector<cudaEvent_t> prof_ev;  // profile_kernels: 5 events per iteration of a chunk
    double prof_us[4] = {0, 0, 0, 0};  // summed kernel times of the profiled iterations
    int prof_iters = 0;
    size_t bytes = 0;
};

void free_workspace(Workspace* w) {
    if (!w) return;
    for (auto& kv : w->graphs) cudaGraphExecDestroy(kv.second);
    for (auto& kv : w->loops) cudaGraphExecDestroy(kv.second);
    void* ptrs[] = {w->r_lo, w->p_lo, w->Ap_lo, w->x_lo, w->t_lo, w->b_hi, w->x_hi,
                    w->r_hi, w->t_hi, w->x_best, w->cg, w->partials, w->counter};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (w->cg_host) cudaFreeHost(w->cg_host);
    if (w->cap_stream) cudaStreamDestroy(w->cap_stream);
    if (w->cap_body) cudaStreamDestroy(w->cap_body);
    if (w->cap_if) cudaStreamDestroy(w->cap_if);
    for (cudaEvent_t e : w->prof_ev) cudaEventDestroy(e);
    delete w;
}

}  // namespace

struct hisq_gauge_s {
    Geom g;
    int device = 0;
    int prec = HISQ_F32, recon_U = 18, recon_N = 18;
    double r12_inv_scale = 1.0;
    float lscale_u[9] = {1, 1, 1, 1, 1, 1, 1, 1, 1};   // 16-bit link component scales
    float lscale_n[9] = {1, 1, 1, 1, 1, 1, 1, 1, 1};
    void* U_lo = nullptr;        // storage copy (prec, recon)
    void* N_lo = nullptr;
    double2* U64 = nullptr;      // FP64 R18 copy
    double2* N64 = nullptr;
    size_t link_bytes = 0;
    int tune_rpt = 0;            // 0 = automatic
    int tune_minb = 0;
    int tune_flags = 0;          // HISQ_MAP_* bits
    std::map<int, DslashTune> tuned;   // autotuned mappings by tuned_key(n, prec, layout)
    void* mdagm_tmp = nullptr;
    size_t mdagm_tmp_bytes = 0;
    double* dot_partials = nullptr;     // reduction scratch of hisq_cdot
    unsigned int* dot_counter = nullptr;
    double* dot_out = nullptr;
    std::vector<Workspace*> ws;
    std::mutex mtx;
};

extern "C" int hisq_version(void) { return 1 * 10000 + 0 * 100 + 0; }

extern "C" const char* hisq_last_error(void) { return g_last_error.c_str(); }

// ---------------------------------------------------------------------------
// Gauge handles
// ---------------------------------------------------------------------------
namespace {

hisq_status pack_field(hisq_gauge g, const double2* canon, int prec, int recon, int hop,
                       double recon_tol, void** out, size_t* bytes, const char* name,
                       cudaStream_t s) {
    const size_t nc = (size_t)recon / 2;
    const size_t sz = 2 * 4 * nc * (size_t)g->g.vh * prec_complex_bytes(prec);
    HISQ_CUDA(cudaMalloc(out, sz));
    *bytes += sz;
    // scratch: [0] reconstruct error bits, [1..9] component maxima (16-bit
    // storage), then the 9 component scales as doubles
    unsigned long long* scratch = nullptr;
    HISQ_CUDA(cudaMalloc(&scratch, 19 * sizeof(unsigned long long)));
    unsigned long long* err_bits = scratch;
    double* comp_scale = reinterpret_cast<double*>(scratch + 10);
    cudaError_t e = cudaMemsetAsync(scratch, 0, 19 * sizeof(unsigned long long), s);
    if (e == cudaSuccess && prec == HISQ_F16) {
        // one scale per stored component: its largest |Re|, |Im| / 32767
        e = launch_link_absmax(g->g, canon, recon, hop, g->r12_inv_scale, scratch + 1, s);
        unsigned long long mb[9] = {0};
        if (e == cudaSuccess) e = cudaMemcpyAsync(mb, scratch + 1, sizeof(mb), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        double sc[9];
        float* keep = (hop == 1) ? g->lscale_u : g->lscale_n;
        for (size_t c = 0; c < 9; ++c) {
            double mx;
            memcpy(&mx, &mb[c], sizeof(mx));
            sc[c] = (c < nc && mx > 0.0 && std::isfinite(mx)) ? mx / 32767.0 : 1.0;
            // the kernels dequantise with the FP32 scale: quantise with the same value
            keep[c] = (float)sc[c];
            sc[c] = (double)keep[c];
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(comp_scale, sc, sizeof(sc), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e == cudaSuccess)
        e = launch_pack_links(g->g, canon, prec, recon, hop, g->r12_inv_scale, *out, err_bits,
                              prec == HISQ_F16 ? comp_scale : nullptr, s);
    unsigned long long bits = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, err_bits, sizeof(bits), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(scratch);
    HISQ_CUDA(e);
    double err;
    memcpy(&err, &bits, sizeof(err));
    if (!(err <= recon_tol))
        return fail(HISQ_ERECON, "%s links are not representable with %d reals: max reconstruct error %.3e > tol %.3e",
                    name, recon, err, recon_tol);
    return HISQ_OK;
}

void destroy_gauge(hisq_gauge g) {
    if (!g) return;
    for (Workspace* w : g->ws) free_workspace(w);
    if (g->U_lo && g->U_lo != g->U64) cudaFree(g->U_lo);
    if (g->N_lo && g->N_lo != g->N64) cudaFree(g->N_lo);
    if (g->U64) cudaFree(g->U64);
    if (g->N64) cudaFree(g->N64);
    if (g->mdagm_tmp) cudaFree(g->mdagm_tmp);
    if (g->dot_partials) cudaFree(g->dot_partials);
    if (g->dot_counter) cudaFree(g->dot_counter);
    if (g->dot_out) cudaFree(g->dot_out);
    delete g;
}

}  // namespace

extern "C" hisq_status hisq_gauge_load(const int L[4], const void* U, const void* N, int on_device,
                                       hisq_prec prec, hisq_recon recon_U, hisq_recon recon_N,
                                       double recon_tol, void* stream, hisq_gauge* out) {
    if (out == nullptr) return fail(HISQ_EINVAL, "out handle pointer is NULL");
    *out = nullptr;
    if (U == nullptr || N == nullptr) return fail(HISQ_EINVAL, "link pointer is NULL");
    if (!valid_prec(prec)) return fail(HISQ_EINVAL, "unknown precision %d", prec);
    if (recon_U != 18 && recon_U != 12 && recon_U != 14)
        return fail(HISQ_EINVAL, "recon_U must be 18, 12 or 14 (got %d)", recon_U);
    if (recon_N != 18 && recon_N != 14)
        return fail(HISQ_EINVAL, "recon_N must be 18 or 14 (got %d)", recon_N);
    if (prec == HISQ_F64 && (recon_U != 18 || recon_N != 18))
        return fail(HISQ_EINVAL, "F64 storage requires R18 for both fields");
    if (!dslash_variant_supported(prec, recon_U, recon_N, EPI_NONE))
        return fail(HISQ_EINVAL, "no Dslash kernel for recon (%d, %d)", recon_U, recon_N);
    if (!(recon_tol >= 0.0)) return fail(HISQ_EINVAL, "recon_tol must be >= 0");
    Geom geom;
    hisq_status st = make_geom(L, &geom);
    if (st != HISQ_OK) return st;
    if (on_device && (!is_device_pointer(U) || !is_device_pointer(N)))
        return fail(HISQ_EINVAL, "on_device = 1 but a link pointer is not device memory");

    cudaStream_t s = (cudaStream_t)stream;
    hisq_gauge g = new hisq_gauge_s();
    g->g = geom;
    cudaGetDevice(&g->device);
    g->prec = prec;
    g->recon_U = recon_U;
    g->recon_N = recon_N;
    const size_t canon_bytes = (size_t)4 * 2 * geom.vh * 9 * sizeof(double2);
    const double2* cu = (const double2*)U;
    const double2* cn = (const double2*)N;
    double2* stage = nullptr;
    auto cleanup = [&](hisq_status code) {
        if (stage) cudaFree(stage);
        if (code != HISQ_OK) destroy_gauge(g);
        return code;
    };
    if (!on_device) {
        if (cudaMalloc(&stage, 2 * canon_bytes) != cudaSuccess)
            return cleanup(fail(HISQ_ENOMEM, "cannot allocate %zu bytes to stage links", 2 * canon_bytes));
        if (cudaMemcpyAsync(stage, U, canon_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(stage + canon_bytes / sizeof(double2), N, canon_bytes,
                            cudaMemcpyHostToDevice, s) != cudaSuccess)
            return cleanup(fail(HISQ_ECUDA, "link upload failed: %s", cudaGetErrorString(cudaGetLastError())));
        cu = stage;
        cn = stage + canon_bytes / sizeof(double2);
    }
    if (recon_U == 12) {
        // s = |row 1| of U_0 at site 0
        double2 row[3];
        if (cudaMemcpyAsync(row, cu, sizeof(row), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return cleanup(fail(HISQ_ECUDA, "reading U[0][0] failed"));
        const double sc = std::sqrt(row[0].x * row[0].x + row[0].y * row[0].y + row[1].x * row[1].x +
                                    row[1].y * row[1].y + row[2].x * row[2].x + row[2].y * row[2].y);
        if (!(sc > 0.0)) return cleanup(fail(HISQ_ERECON, "R12 needs a nonzero first row in U[0][0]"));
        g->r12_inv_scale = 1.0 / sc;
    }
    size_t bytes = 0;
    st = pack_field(g, cu, HISQ_F64, 18, 1, recon_tol, (void**)&g->U64, &bytes, "fat", s);
    if (st == HISQ_OK) st = pack_field(g, cn, HISQ_F64, 18, 3, recon_tol, (void**)&g->N64, &bytes, "Naik", s);
    if (st == HISQ_OK) {
        if (prec == HISQ_F64) {
            g->U_lo = g->U64;
            g->N_lo = g->N64;
        } else {
            st = pack_field(g, cu, prec, recon_U, 1, recon_tol, &g->U_lo, &bytes, "fat", s);
            if (st == HISQ_OK) st = pack_field(g, cn, prec, recon_N, 3, recon_tol, &g->N_lo, &bytes, "Naik", s);
        }
    }
    if (st != HISQ_OK) return cleanup(st);
    g->link_bytes = bytes;
    *out = g;
    return cleanup(HISQ_OK);
}

extern "C" hisq_status hisq_gauge_free(hisq_gauge g) {
    if (!g) return HISQ_OK;
    destroy_gauge(g);
    return HISQ_OK;
}

extern "C" hisq_status hisq_gauge_info(hisq_gauge g, int L[4], hisq_prec* prec, hisq_recon* recon_U,
                                       hisq_recon* recon_N, size_t* device_bytes) {
    if (!g) return fail(HISQ_EINVAL, "NULL handle");
    if (L)
        for (int m = 0; m < 4; ++m) L[m] = g->g.L[m];
    if (prec) *prec = g->prec;
    if (recon_U) *recon_U = g->recon_U;
    if (recon_N) *recon_N = g->recon_N;
    if (device_bytes) {
        size_t b = g->link_bytes + g->mdagm_tmp_bytes;
        for (Workspace* w : g->ws) b += w->bytes;
        *device_bytes = b;
    }
    return HISQ_OK;
}

extern "C" hisq_status hisq_set_dslash_mapping(hisq_gauge g, int rpt, int minb, int flags) {
    if (!g) return fail(HISQ_EINVAL, "NULL handle");
    if (rpt != 0 && rpt != 1 && rpt != 2 && rpt != 4 && rpt != 8)
        return fail(HISQ_EINVAL, "rhs per thread must be 0 (auto), 1, 2, 4 or 8");
    if (minb < 0 || minb > 8) return fail(HISQ_EINVAL, "min blocks per SM must be 0 (auto) .. 8");
    if (flags & ~(HISQ_MAP_PACKED | HISQ_MAP_L2_PREFETCH | HISQ_MAP_STAGED | HISQ_MAP_PIPELINED |
                  HISQ_MAP_PIPELINED2 | HISQ_MAP_COMPACT | HISQ_MAP_TILE_XY))
        return fail(HISQ_EINVAL, "unknown mapping flags %d", flags);
    // STAGED with PIPELINED2 selects the bundle kernel staging two hops ahead
    const int kinds = !!(flags & HISQ_MAP_PACKED) + !!(flags & HISQ_MAP_STAGED) +
                      !!(flags & HISQ_MAP_PIPELINED) + !!(flags & HISQ_MAP_PIPELINED2) +
                      !!(flags & HISQ_MAP_TILE_XY) -
                      ((flags & HISQ_MAP_STAGED) && (flags & HISQ_MAP_PIPELINED2) ? 1 : 0);
    if (kinds > 1) return fail(HISQ_EINVAL, "mapping flags %d name more than one kernel kind", flags);
    g->tune_rpt = rpt;
    g->tune_minb = minb;
    g->tune_flags = flags;
    return HISQ_OK;
}

// ---------------------------------------------------------------------------
// Link compression helpers
// ---------------------------------------------------------------------------
extern "C" hisq_status hisq_link_compress(const int L[4], const void* links, hisq_recon r,
                                          void* packed, double* max_err, void* stream) {
    Geom g;
    hisq_status st = make_geom(L, &g);
    if (st != HISQ_OK) return st;
    if (r != 18 && r != 14 && r != 12) return fail(HISQ_EINVAL, "recon must be 18, 14 or 12");
    if (!links || !packed) return fail(HISQ_EINVAL, "NULL pointer");
    if (!is_device_pointer(links) || !is_device_pointer(packed))
        return fail(HISQ_EINVAL, "link_compress takes device pointers");
    cudaStream_t s = (cudaStream_t)stream;
    double inv_s = 1.0;
    if (r == 12) {
        double2 row[3];
        HISQ_CUDA(cudaMemcpyAsync(row, links, sizeof(row), cudaMemcpyDeviceToHost, s));
        HISQ_CUDA(cudaStreamSynchronize(s));
        const double sc = std::sqrt(row[0].x * row[0].x + row[0].y * row[0].y + row[1].x * row[1].x +
                                    row[1].y * row[1].y + row[2].x * row[2].x + row[2].y * row[2].y);
        if (!(sc > 0.0)) return fail(HISQ_ERECON, "R12 needs a nonzero first row in link 0");
        inv_s = 1.0 / sc;
    }
    unsigned long long* bits_d = nullptr;
    HISQ_CUDA(cudaMalloc(&bits_d, sizeof(unsigned long long)));
    cudaError_t e = cudaMemsetAsync(bits_d, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess)
        e = launch_compress_links(g, (const double2*)links, r, 1, inv_s, (double*)packed, bits_d, s);
    unsigned long long bits = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, bits_d, sizeof(bits), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(bits_d);
    HISQ_CUDA(e);
    if (max_err) memcpy(max_err, &bits, sizeof(double));
    return HISQ_OK;
}

extern "C" hisq_status hisq_link_reconstruct(const int L[4], const void* packed, hisq_recon r,
                                             void* links, void* stream) {
    Geom g;
    hisq_status st = make_geom(L, &g);
    if (st != HISQ_OK) return st;
    if (r != 18 && r != 14 && r != 12) return fail(HISQ_EINVAL, "recon must be 18, 14 or 12");
    if (!links || !packed) return fail(HISQ_EINVAL, "NULL pointer");
    if (!is_device_pointer(links) || !is_device_pointer(packed))
        return fail(HISQ_EINVAL, "link_reconstruct takes device pointers");
    cudaStream_t s = (cudaStream_t)stream;
    double inv_s = 1.0;
    if (r == 12) {
        // row 1 of link 0 is stored verbatim: its norm is s
        double v[6];
        HISQ_CUDA(cudaMemcpyAsync(v, packed, sizeof(v), cudaMemcpyDeviceToHost, s));
        HISQ_CUDA(cudaStreamSynchronize(s));
        double n2 = 0;
        for (double a : v) n2 += a * a;
        if (!(n2 > 0.0)) return fail(HISQ_ERECON, "R12 needs a nonzero first row in link 0");
        inv_s = 1.0 / std::sqrt(n2);
    }
    HISQ_CUDA(launch_reconstruct_links(g, (const double*)packed, r, 1, inv_s, (double2*)links, s));
    HISQ_CUDA(cudaStreamSynchronize(s));
    return HISQ_OK;
}

// ---------------------------------------------------------------------------
// Dslash and normal operator
// ---------------------------------------------------------------------------
namespace {

int link_recon_u(hisq_gauge g, int prec) { return prec == HISQ_F64 ? 18 : g->recon_U; }
int link_recon_n(hisq_gauge g, int prec) { return prec == HISQ_F64 ? 18 : g->recon_N; }

int auto_rpt(int n, int prec) {
    const int mx = dslash_max_rpt(prec);
    int r = 1;
    while (r * 2 <= mx && n % (r * 2) == 0) r *= 2;
    // FP32/FP16 storage below 16 rhs: two groups of four rhs per thread with
    // the pipelined kernel beat one group of eight
    if (prec != HISQ_F64 && r == 8 && n < 16) r = 4;
    while (n / r > 8 && r < mx) r *= 2;   // at most 8 rhs groups per block
    return r;
}

int tuned_key(int n, int prec, int layout) { return n * 100 + prec * 10 + layout; }

int kind_of_flags(int flags) {
    if (flags & HISQ_MAP_PACKED) return KIND_PACKED;
    if (flags & HISQ_MAP_STAGED) return KIND_STAGED;
    if (flags & HISQ_MAP_PIPELINED) return KIND_PIPE1;
    if (flags & HISQ_MAP_PIPELINED2) return KIND_PIPE2;
    return KIND_REG;
}

int bundle_kind_of_flags(int flags) {
    if (flags & HISQ_MAP_TILE_XY) return KIND_BUNDLE_XY;
    if ((flags & HISQ_MAP_STAGED) && (flags & HISQ_MAP_COMPACT))
        return (flags & HISQ_MAP_PIPELINED2) ? KIND_BUNDLE_CSMEM3 : KIND_BUNDLE_CSMEM1;
    if (flags & HISQ_MAP_STAGED) return (flags & HISQ_MAP_PIPELINED2) ? KIND_BUNDLE_SMEM2 : KIND_BUNDLE_SMEM1;
    const bool spin = flags & (HISQ_MAP_PIPELINED | HISQ_MAP_PIPELINED2);
    if (flags & HISQ_MAP_COMPACT) return spin ? KIND_BUNDLE_COMPACT_SPIN : KIND_BUNDLE_COMPACT;
    return spin ? KIND_BUNDLE_SPIN : KIND_BUNDLE;
}

int flags_of_tune(const DslashTune& t) {
    if (t.layout == HISQ_BUNDLE && t.kind == KIND_BUNDLE_XY) return HISQ_MAP_TILE_XY;
    if (t.layout == HISQ_BUNDLE && (t.kind == KIND_BUNDLE_SMEM1 || t.kind == KIND_BUNDLE_SMEM2))
        return HISQ_MAP_STAGED | (t.kind == KIND_BUNDLE_SMEM2 ? HISQ_MAP_PIPELINED2 : 0);
    if (t.layout == HISQ_BUNDLE && (t.kind == KIND_BUNDLE_CSMEM1 || t.kind == KIND_BUNDLE_CSMEM3))
        return HISQ_MAP_STAGED | HISQ_MAP_COMPACT | (t.kind == KIND_BUNDLE_CSMEM3 ? HISQ_MAP_PIPELINED2 : 0);
    if (t.layout == HISQ_BUNDLE)
        return (t.kind == KIND_BUNDLE_COMPACT || t.kind == KIND_BUNDLE_COMPACT_SPIN ? HISQ_MAP_COMPACT : 0) |
               (t.kind == KIND_BUNDLE_SPIN || t.kind == KIND_BUNDLE_COMPACT_SPIN ? HISQ_MAP_PIPELINED : 0);
    const int k = t.kind == KIND_PACKED   ? HISQ_MAP_PACKED
                  : t.kind == KIND_STAGED ? HISQ_MAP_STAGED
                  : t.kind == KIND_PIPE1  ? HISQ_MAP_PIPELINED
                  : t.kind == KIND_PIPE2  ? HISQ_MAP_PIPELINED2
                                          : 0;
    return k | (t.prefetch ? HISQ_MAP_L2_PREFETCH : 0);
}

// Thread mapping for n rhs: the requested rpt, else the handle's explicit
// setting, else the autotuned mapping for (n, prec, layout), else the
// largest power of two dividing n (at most 8 rhs groups per block).
DslashTune pick_tune(hisq_gauge g, int n, int prec, int requested, int layout) {
    if (layout == HISQ_BUNDLE) {
        // the bundle kernel (rpt 0 when n does not fit the layout)
        if (!requested && g->tune_rpt == 0 && g->tune_flags == 0) {
            auto it = g->tuned.find(tuned_key(n, prec, layout));
            if (it != g->tuned.end()) return it->second;
        }
        DslashTune t = dslash_bundle_tune(prec, n);
        if (t.rpt == 0) return t;
        const int ru = link_recon_u(g, prec), rn = link_recon_n(g, prec);
        const int r = requested ? requested : g->tune_rpt;
        if (r && n % r == 0 && n / r <= 4) {
            const int b = (!requested && g->tune_minb) ? g->tune_minb : (r == 8 && prec != HISQ_F16 ? 3 : 4);
            const int k = requested ? (r == 8 && prec == HISQ_F16 ? KIND_BUNDLE_CSMEM1 : KIND_BUNDLE)
                                    : bundle_kind_of_flags(g->tune_flags);
            if (bundle_mapping_built(prec, ru, rn, r, b, k)) {
                t.rpt = r;
                t.minb = b;
                t.kind = k;
            }
        } else if (!requested && g->tune_flags) {
            const int k = bundle_kind_of_flags(g->tune_flags);
            if (bundle_mapping_built(prec, ru, rn, t.rpt, t.minb, k)) t.kind = k;
        }
        return t;
    }
    if (!requested && g->tune_rpt == 0 && g->tune_flags == 0) {
        auto it = g->tuned.find(tuned_key(n, prec, layout));
        if (it != g->tuned.end()) return it->second;
    }
    int r = requested ? requested : g->tune_rpt;
    if (r == 0 || r > dslash_max_rpt(prec) || n % r != 0 || n / r > 8) r = auto_rpt(n, prec);
    DslashTune t = dslash_default_tune(prec, r, layout);
    const int kind = kind_of_flags(g->tune_flags);
    if (!requested && g->tune_minb && r == g->tune_rpt && dslash_mapping_built(prec, r, g->tune_minb, kind) &&
        (kind != KIND_STAGED || dslash_staged_ok(g->g, prec, r, n / r))) {
        t.minb = g->tune_minb;
        t.kind = kind;
    }
    if (g->tune_flags & HISQ_MAP_L2_PREFETCH) t.prefetch = 1;
    return t;
}

}  // namespace

extern "C" hisq_status hisq_get_dslash_mapping_ex(hisq_gauge g, int n, hisq_prec prec, hisq_layout layout,
                                                 int* rpt, int* minb, int* flags) {
    if (!g) return fail(HISQ_EINVAL, "NULL handle");
    if (n < 1 || n > kMaxRhs) return fail(HISQ_EINVAL, "n = %d outside 1..%d", n, kMaxRhs);
    if (!valid_prec(prec)) return fail(HISQ_EINVAL, "unknown precision %d", prec);
    if (layout != HISQ_AOS && layout != HISQ_SOA && layout != HISQ_BUNDLE)
        return fail(HISQ_EINVAL, "unknown layout %d", layout);
    const DslashTune t = pick_tune(g, n, prec, 0, layout);
    if (layout == HISQ_BUNDLE && t.rpt == 0) return fail(HISQ_EINVAL, "no bundle kernel for n = %d", n);
    if (rpt) *rpt = t.rpt;
    if (minb) *minb = t.minb;
    if (flags) *flags = flags_of_tune(t);
    return HISQ_OK;
}

extern "C" hisq_status hisq_get_dslash_mapping(hisq_gauge g, int n, hisq_prec prec, int* rpt, int* minb,
                                              int* flags) {
    return hisq_get_dslash_mapping_ex(g, n, prec, HISQ_AOS, rpt, minb, flags);
}

namespace {

bool aligned_for(const void* p, int prec) {
    return ((uintptr_t)p % prec_complex_bytes(prec)) == 0;
}

void fill_common(DslashArgs& a, hisq_gauge g, int prec, int parity, int n) {
    memset(&a, 0, sizeof(a));
    a.g = g->g;
    a.parity = parity;
    a.nrhs = n;
    a.U = (prec == HISQ_F64) ? (const void*)g->U64 : g->U_lo;
    a.N = (prec == HISQ_F64) ? (const void*)g->N64 : g->N_lo;
    a.cx = 0.0;
    a.cd = 1.0;
    a.ft1 = a.bt1 = a.ft3 = a.bt3 = 1.0;
    a.has_mu = 0;
    a.r12_inv_scale = g->r12_inv_scale;
    for (int c = 0; c < 9; ++c) {
        a.lscale_u[c] = g->lscale_u[c];
        a.lscale_n[c] = g->lscale_n[c];
    }
    a.red_mode = RED_NONE;
    a.finish = FIN_STORE;
}

void set_mu(DslashArgs& a, double mu) {
    a.ft1 = std::exp(mu);
    a.bt1 = std::exp(-mu);
    a.ft3 = std::exp(3.0 * mu);
    a.bt3 = std::exp(-3.0 * mu);
    a.has_mu = (mu != 0.0) ? 1 : 0;
}

hisq_status check_spinors(hisq_gauge g, const void* const v[], void* const w[], int n, int prec) {
    if (!g) return fail(HISQ_EINVAL, "NULL handle");
    if (n < 1 || n > kMaxRhs) return fail(HISQ_EINVAL, "n = %d outside 1..%d", n, kMaxRhs);
    if (!valid_prec(prec)) return fail(HISQ_EINVAL, "unknown spinor precision %d", prec);
    if (prec != HISQ_F64 && prec != g->prec)
        return fail(HISQ_EINVAL, "spinor precision %d needs links stored in the same precision (handle has %d)",
                    prec, g->prec);
    if (!v || !w) return fail(HISQ_EINVAL, "NULL pointer array");
    for (int k = 0; k < n; ++k) {
        if (!v[k] || !w[k]) return fail(HISQ_EINVAL, "NULL spinor pointer for rhs %d", k);
        if (!aligned_for(v[k], prec) || !aligned_for(w[k], prec))
            return fail(HISQ_EINVAL, "spinor pointer for rhs %d is not %zu-byte aligned", k,
                        prec_complex_bytes(prec));
    }
    return HISQ_OK;
}

// Bundle buffers: n fits the chunk width of prec, one 16-byte-aligned pointer each.
hisq_status check_bundle(hisq_gauge g, const void* v, const void* w, int n, int prec) {
    if (!g) return fail(HISQ_EINVAL, "NULL handle");
    const int W = bundle_width(prec);
    if (W == 0) return fail(HISQ_EINVAL, "the bundle layout needs F32 or F16 storage");
    if (prec != g->prec)
        return fail(HISQ_EINVAL, "spinor precision %d needs links stored in the same precision (handle has %d)",
                    prec, g->prec);
    if (n < W || n > kMaxRhs || n % W != 0)
        return fail(HISQ_EINVAL, "n = %d: the bundle layout of this precision needs a multiple of %d up to %d", n,
                    W, kMaxRhs);
    if (!v || !w) return fail(HISQ_EINVAL, "NULL bundle pointer");
    if ((uintptr_t)v % 16 || (uintptr_t)w % 16) return fail(HISQ_EINVAL, "bundle pointers must be 16-byte aligned");
    return HISQ_OK;
}

}  // namespace

extern "C" hisq_status hisq_dslash_ex(hisq_gauge g, double mu, const void* const v[], void* const w[],
                                      int n, int parity, hisq_prec spinor_prec, hisq_layout layout,
                                      void* stream) {
    if (layout == HISQ_BUNDLE) {
        if (!v || !w) return fail(HISQ_EINVAL, "NULL pointer array");
        hisq_status st = check_bundle(g, v[0], w[0], n, spinor_prec);
        if (st != HISQ_OK) return st;
    } else {
        hisq_status st = check_spinors(g, v, w, n, spinor_prec);
        if (st != HISQ_OK) return st;
    }
    if (parity != 0 && parity != 1) return fail(HISQ_EINVAL, "parity must be 0 or 1");
    if (layout != HISQ_AOS && layout != HISQ_SOA && layout != HISQ_BUNDLE)
        return fail(HISQ_EINVAL, "unknown layout %d", layout);
    if (!std::isfinite(mu)) return fail(HISQ_EINVAL, "mu must be finite");
    DslashArgs a;
    fill_common(a, g, spinor_prec, parity, n);
    set_mu(a, mu);
    if (layout == HISQ_BUNDLE) {
        a.in[0] = v[0];
        a.out[0] = w[0];
        const DslashTune t = pick_tune(g, n, spinor_prec, 0, layout);
        if (t.rpt == 0) return fail(HISQ_EINVAL, "no bundle kernel for n = %d", n);
        HISQ_CUDA(launch_dslash(a, spinor_prec, link_recon_u(g, spinor_prec), link_recon_n(g, spinor_prec),
                                EPI_NONE, t, (cudaStream_t)stream));
        return HISQ_OK;
    }
    for (int k = 0; k < n; ++k) {
        a.in[k] = v[k];
        a.out[k] = w[k];
    }
    const DslashTune t = pick_tune(g, n, spinor_prec, 0, layout);
    HISQ_CUDA(launch_dslash(a, spinor_prec, link_recon_u(g, spinor_prec), link_recon_n(g, spinor_prec),
                            EPI_NONE, t, (cudaStream_t)stream));
    return HISQ_OK;
}

extern "C" hisq_status hisq_dslash(hisq_gauge g, const void* const v[], void* const w[], int n,
                                   int parity, hisq_prec spinor_prec, void* stream) {
    return hisq_dslash_ex(g, 0.0, v, w, n, parity, spinor_prec, HISQ_AOS, stream);
}

extern "C" hisq_status hisq_bundle_pack(hisq_gauge g, const void* const src[], int n, hisq_prec prec,
                                        void* bundle, void* stream) {
    hisq_status st = check_bundle(g, bundle, bundle, n, prec);
    if (st != HISQ_OK) return st;
    if (!src) return fail(HISQ_EINVAL, "NULL pointer array");
    BundlePtrs p;
    memset(&p, 0, sizeof(p));
    for (int k = 0; k < n; ++k) {
        if (!src[k] || (uintptr_t)src[k] % 16) return fail(HISQ_EINVAL, "source %d is NULL or not 16-byte aligned", k);
        p.p[k] = (const double2*)src[k];
    }
    HISQ_CUDA(launch_bundle_pack(p, n, prec, g->g.vh, bundle, (cudaStream_t)stream));
    return HISQ_OK;
}

extern "C" hisq_status hisq_bundle_unpack(hisq_gauge g, const void* bundle, int n, hisq_prec prec,
                                          void* const dst[], void* stream) {
    hisq_status st = check_bundle(g, bundle, bundle, n, prec);
    if (st != HISQ_OK) return st;
    if (!dst) return fail(HISQ_EINVAL, "NULL pointer array");
    BundlePtrs p;
    memset(&p, 0, sizeof(p));
    for (int k = 0; k < n; ++k) {
        if (!dst[k] || (uintptr_t)dst[k] % 16)
            return fail(HISQ_EINVAL, "destination %d is NULL or not 16-byte aligned", k);
        p.p[k] = (const double2*)dst[k];
    }
    HISQ_CUDA(launch_bundle_unpack(bundle, p, n, prec, g->g.vh, (cudaStream_t)stream));
    return HISQ_OK;
}

extern "C" hisq_status hisq_mdagm(hisq_gauge g, double mass, const void* const v[], void* const w[],
                                  int n, hisq_prec spinor_prec, void* stream) {
    hisq_status st = check_spinors(g, v, w, n, spinor_prec);
    if (st != HISQ_OK) return st;
    if (!std::isfinite(mass)) return fail(HISQ_EINVAL, "mass must be finite");
    const size_t per = (size_t)g->g.vh * 3 * prec_complex_bytes(spinor_prec);
    std::lock_guard<std::mutex> lock(g->mtx);
    if (g->mdagm_tmp_bytes < per * n) {
        if (g->mdagm_tmp) cudaFree(g->mdagm_tmp);
        g->mdagm_tmp = nullptr;
        g->mdagm_tmp_bytes = 0;
        HISQ_CUDA(cudaMalloc(&g->mdagm_tmp, per * kMaxRhs));
        g->mdagm_tmp_bytes = per * kMaxRhs;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const DslashTune t = pick_tune(g, n, spinor_prec, 0, HISQ_AOS);
    const int ru = link_recon_u(g, spinor_prec), rn = link_recon_n(g, spinor_prec);
    DslashArgs a;
    fill_common(a, g, spinor_prec, 1, n);
    for (int k = 0; k < n; ++k) {
        a.in[k] = v[k];
        a.out[k] = (char*)g->mdagm_tmp + per * k;
    }
    HISQ_CUDA(launch_dslash(a, spinor_prec, ru, rn, EPI_NONE, t, s));
    DslashArgs b;
    fill_common(b, g, spinor_prec, 0, n);
    b.cx = 4.0 * mass * mass;
    b.cd = -1.0;
    for (int k = 0; k < n; ++k) {
        b.in[k] = (char*)g->mdagm_tmp + per * k;
        b.out[k] = w[k];
        b.x[k] = v[k];
    }
    HISQ_CUDA(launch_dslash(b, spinor_prec, ru, rn, EPI_X, t, s));
    return HISQ_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: times every built Dslash mapping that fits (n, prec, layout) on
// this handle and keeps the fastest for later calls of that shape.
// ---------------------------------------------------------------------------
namespace {

std::vector<DslashTune> candidate_tunes(hisq_gauge g, int n, int prec, int layout) {
    std::vector<DslashTune> out;
    if (layout == HISQ_BUNDLE) {
        const int ru = link_recon_u(g, prec), rn = link_recon_n(g, prec);
        const int kinds[] = {KIND_BUNDLE, KIND_BUNDLE_SPIN, KIND_BUNDLE_COMPACT, KIND_BUNDLE_COMPACT_SPIN,
                             KIND_BUNDLE_SMEM1, KIND_BUNDLE_SMEM2, KIND_BUNDLE_CSMEM1, KIND_BUNDLE_CSMEM3,
                             KIND_BUNDLE_XY};
        for (int r : {4, 8}) {
            if (n % r != 0 || n / r > 4) continue;
            for (int b = 1; b <= 4; ++b)
                for (int k : kinds) {
                    if (!bundle_mapping_built(prec, ru, rn, r, b, k)) continue;
                    DslashTune t = dslash_bundle_tune(prec, n);
                    if (t.rpt == 0) continue;
                    t.rpt = r;
                    t.minb = b;
                    t.kind = k;
                    out.push_back(t);
                }
        }
        return out;
    }
    const int rpts[] = {1, 2, 4, 8};
    const int minbs[] = {1, 2, 3, 4};
    const int kinds[] = {KIND_REG, KIND_PACKED, KIND_STAGED, KIND_PIPE1, KIND_PIPE2};
    for (int r : rpts) {
        if (r > dslash_max_rpt(prec) || n % r != 0 || n / r > 8) continue;
        for (int b : minbs)
            for (int k : kinds) {
                if (!dslash_mapping_built(prec, r, b, k)) continue;
                if (k == KIND_STAGED && !dslash_staged_ok(g->g, prec, r, n / r)) continue;
                DslashTune t = dslash_default_tune(prec, r, layout);
                t.minb = b;
                t.kind = k;
                out.push_back(t);
            }
    }
    return out;
}

}  // namespace

extern "C" hisq_status hisq_autotune_dslash(hisq_gauge g, int n, hisq_prec prec, hisq_layout layout, int reps,
                                           int* rpt, int* minb, int* flags, double* seconds) {
    if (!g) return fail(HISQ_EINVAL, "NULL handle");
    if (n < 1 || n > kMaxRhs) return fail(HISQ_EINVAL, "n = %d outside 1..%d", n, kMaxRhs);
    if (!valid_prec(prec) || (prec != HISQ_F64 && prec != g->prec))
        return fail(HISQ_EINVAL, "precision %d not available on this handle", prec);
    if (layout != HISQ_AOS && layout != HISQ_SOA && layout != HISQ_BUNDLE)
        return fail(HISQ_EINVAL, "unknown layout %d", layout);
    if (layout == HISQ_BUNDLE && dslash_bundle_tune(prec, n).rpt == 0)
        return fail(HISQ_EINVAL, "no bundle kernel for n = %d in precision %d", n, prec);
    if (reps < 1) reps = 5;
    std::lock_guard<std::mutex> lock(g->mtx);
    const size_t per = (size_t)g->g.vh * 3 * prec_complex_bytes(prec);
    void* buf = nullptr;
    HISQ_CUDA(cudaMalloc(&buf, 2 * per * n));
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s) cudaStreamDestroy(s);
        cudaFree(buf);
    };
    cudaError_t e = cudaMemset(buf, 0, 2 * per * n);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cleanup();
        HISQ_CUDA(e);
    }
    DslashArgs a;
    fill_common(a, g, prec, 0, n);
    for (int k = 0; k < n; ++k) {
        a.in[k] = (char*)buf + per * k;
        a.out[k] = (char*)buf + per * (n + k);
    }
    if (layout == HISQ_BUNDLE) a.out[0] = (char*)buf + per * n;   // one bundle in, one out
    const int ru = link_recon_u(g, prec), rn = link_recon_n(g, prec);
    double best = HUGE_VAL;
    DslashTune best_t = layout == HISQ_BUNDLE ? dslash_bundle_tune(prec, n)
                                              : dslash_default_tune(prec, auto_rpt(n, prec), layout);
    for (const DslashTune& t : candidate_tunes(g, n, prec, layout)) {
        e = launch_dslash(a, prec, ru, rn, EPI_NONE, t, s);   // warm-up (and first-use set-up)
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        for (int i = 0; i < reps && e == cudaSuccess; ++i) e = launch_dslash(a, prec, ru, rn, EPI_NONE, t, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            cleanup();
            HISQ_CUDA(e);
        }
        const double sec = ms * 1e-3 / reps;
        if (sec < best) {
            best = sec;
            best_t = t;
        }
    }
    cleanup();
    g->tuned[tuned_key(n, prec, layout)] = best_t;
    if (rpt) *rpt = best_t.rpt;
    if (minb) *minb = best_t.minb;
    if (flags) *flags = flags_of_tune(best_t);
    if (seconds) *seconds = best;
    return HISQ_OK;
}

// Gauge load that also chooses the link compression: every (recon_U, recon_N)
// pair with a kernel for the storage precision and exact for these links is
// loaded and autotuned for n rhs; the fastest handle is kept. Choices are
// cached per (L, n, prec) for the process.
namespace {

struct TunedShape {
    int ru, rn;
    std::map<int, DslashTune> tuned;
};
std::mutex g_shape_mtx;
std::map<std::tuple<int, int, int, int, int, int>, TunedShape> g_shape_cache;

}  // namespace

extern "C" hisq_status hisq_gauge_load_tuned(const int L[4], const void* U, const void* N, int on_device,
                                            hisq_prec prec, int n, double recon_tol, void* stream,
                                            hisq_gauge* out) {
    if (out == nullptr) return fail(HISQ_EINVAL, "out handle pointer is NULL");
    *out = nullptr;
    if (L == nullptr) return fail(HISQ_EINVAL, "L is NULL");
    if (n < 1 || n > kMaxRhs) return fail(HISQ_EINVAL, "n = %d outside 1..%d", n, kMaxRhs);
    if (!valid_prec(prec)) return fail(HISQ_EINVAL, "unknown precision %d", prec);
    const auto key = std::make_tuple(L[0], L[1], L[2], L[3], n, (int)prec);
    {
        std::lock_guard<std::mutex> lk(g_shape_mtx);
        auto it = g_shape_cache.find(key);
        if (it != g_shape_cache.end()) {
            hisq_status st = hisq_gauge_load(L, U, N, on_device, prec, (hisq_recon)it->second.ru,
                                             (hisq_recon)it->second.rn, recon_tol, stream, out);
            if (st == HISQ_OK) (*out)->tuned = it->second.tuned;
            // links of the same shape that the cached pair cannot hold: search again
            if (st != HISQ_ERECON) return st;
        }
    }
    std::vector<std::pair<int, int>> pairs;
    if (prec == HISQ_F64)
        pairs = {{18, 18}};
    else
        pairs = {{18, 18}, {18, 14}, {12, 14}, {14, 14}};
    hisq_gauge best = nullptr;
    double best_s = HUGE_VAL;
    hisq_status last = HISQ_OK;
    for (const auto& pr : pairs) {
        hisq_gauge g = nullptr;
        hisq_status st = hisq_gauge_load(L, U, N, on_device, prec, (hisq_recon)pr.first, (hisq_recon)pr.second,
                                         recon_tol, stream, &g);
        if (st == HISQ_ERECON) continue;        // not exact for these links
        if (st != HISQ_OK) {
            last = st;
            break;
        }
        // the layout the CG runs on (the bundle where n fits it) decides; the
        // ABI layouts are tuned too for direct Dslash calls
        const bool bundle = prec != HISQ_F64 && dslash_bundle_tune(prec, n).rpt != 0;
        double sec_cg = 0.0, sec_soa = 0.0, sec_aos = 0.0;
        st = hisq_autotune_dslash(g, n, prec, HISQ_SOA, 5, nullptr, nullptr, nullptr, &sec_soa);
        if (st == HISQ_OK) st = hisq_autotune_dslash(g, n, prec, HISQ_AOS, 5, nullptr, nullptr, nullptr, &sec_aos);
        if (st == HISQ_OK && bundle)
            st = hisq_autotune_dslash(g, n, prec, HISQ_BUNDLE, 5, nullptr, nullptr, nullptr, &sec_cg);
        if (!bundle) sec_cg = sec_aos;
        if (st != HISQ_OK) {
            hisq_gauge_free(g);
            last = st;
            break;
        }
        if (sec_cg < best_s) {
            if (best) hisq_gauge_free(best);
            best = g;
            best_s = sec_cg;
        } else {
            hisq_gauge_free(g);
        }
    }
    if (last != HISQ_OK) {
        if (best) hisq_gauge_free(best);
        return last;
    }
    if (!best) return fail(HISQ_ERECON, "no link compression holds these links within recon_tol");
    {
        std::lock_guard<std::mutex> lk(g_shape_mtx);
        g_shape_cache[key] = TunedShape{best->recon_U, best->recon_N, best->tuned};
    }
    *out = best;
    return HISQ_OK;
}

// Bundle size: seconds per rhs of the tuned Dslash for every power-of-two
// bundle up to n_max; the smallest wins.
extern "C" hisq_status hisq_autotune_bundle(hisq_gauge g, int n_max, hisq_prec prec, hisq_layout layout,
                                           int reps, int* best_n, double* seconds_per_rhs) {
    if (!g) return fail(HISQ_EINVAL, "NULL handle");
    if (n_max < 1 || n_max > kMaxRhs) return fail(HISQ_EINVAL, "n_max = %d outside 1..%d", n_max, kMaxRhs);
    int bn = 0;
    double bs = HUGE_VAL;
    for (int n = 1; n <= n_max; n *= 2) {
        if (layout == HISQ_BUNDLE && dslash_bundle_tune(prec, n).rpt == 0) continue;   // n does not fill a chunk
        double sec = 0.0;
        hisq_status st = hisq_autotune_dslash(g, n, prec, layout, reps, nullptr, nullptr, nullptr, &sec);
        if (st != HISQ_OK) return st;
        if (sec / n < bs) {
            bs = sec / n;
            bn = n;
        }
    }
    if (best_n) *best_n = bn;
    if (seconds_per_rhs) *seconds_per_rhs = bs;
    return HISQ_OK;
}

// ---------------------------------------------------------------------------
// Full-lattice fermion matrix, its mu derivative, link force, dot products
// ---------------------------------------------------------------------------
extern "C" hisq_status hisq_apply_m(hisq_gauge g, double mass, double mu, int op,
                                   const void* const v[], void* const w[], int n,
                                   hisq_prec spinor_prec, void* stream) {
    hisq_status st = check_spinors(g, v, w, n, spinor_prec);
    if (st != HISQ_OK) return st;
    if (op < HISQ_OP_M || op > HISQ_OP_D4M_DMU4) return fail(HISQ_EINVAL, "unknown operator %d", op);
    if (!std::isfinite(mass) || !std::isfinite(mu)) return fail(HISQ_EINVAL, "mass and mu must be finite");
    const size_t half = (size_t)g->g.vh * 3 * prec_complex_bytes(spinor_prec);
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j) {
            const char* a = (const char*)v[k];
            const char* b = (const char*)w[j];
            if (a < b + 2 * half && b < a + 2 * half)
                return fail(HISQ_EINVAL, "output %d overlaps input %d", j, k);
        }
    cudaStream_t s = (cudaStream_t)stream;
    const DslashTune t = pick_tune(g, n, spinor_prec, 0, HISQ_AOS);
    const int ru = link_recon_u(g, spinor_prec), rn = link_recon_n(g, spinor_prec);
    for (int par = 0; par < 2; ++par) {
        DslashArgs a;
        fill_common(a, g, spinor_prec, par, n);
        for (int k = 0; k < n; ++k) {
            a.in[k] = (const char*)v[k] + (1 - par) * half;
            a.out[k] = (char*)w[k] + par * half;
            a.x[k] = (const char*)v[k] + par * half;
        }
        int epi = EPI_X;
        if (op == HISQ_OP_M) {
            set_mu(a, mu);
            a.cx = 2.0 * mass;
            a.cd = 1.0;
        } else if (op == HISQ_OP_MDAG) {
            set_mu(a, -mu);
            a.cx = 2.0 * mass;
            a.cd = -1.0;
        } else {
            // k-th mu-derivative of the temporal hops: e^{mu} U v(x+t),
            // -(-1)^k e^{-mu} U^dag v(x-t), 3^k e^{3mu} N v(x+3t),
            // -(-3)^k e^{-3mu} N^dag v(x-3t). The kernel subtracts the
            // backward terms, so bt1 = (-1)^k e^{-mu} and bt3 = (-3)^k e^{-3mu}.
            const int k = op - HISQ_OP_DM_DMU + 1;
            a.ft1 = std::exp(mu);
            a.bt1 = std::pow(-1.0, k) * std::exp(-mu);
            a.ft3 = std::pow(3.0, k) * std::exp(3.0 * mu);
            a.bt3 = std::pow(-3.0, k) * std::exp(-3.0 * mu);
            a.has_mu = 1;
            a.t_only = 1;
            epi = EPI_NONE;
        }
        HISQ_CUDA(launch_dslash(a, spinor_prec, ru, rn, epi, t, s));
    }
    return HISQ_OK;
}

extern "C" hisq_status hisq_link_force(hisq_gauge g, double mu, int hop, const void* const a[],
                                      const void* const b[], int n, double coef, void* out,
                                      void* stream) {
    if (!g) return fail(HISQ_EINVAL, "NULL handle");
    if (n < 1 || n > kMaxRhs) return fail(HISQ_EINVAL, "n = %d outside 1..%d", n, kMaxRhs);
    if (hop != 1 && hop != 3) return fail(HISQ_EINVAL, "hop must be 1 (fat) or 3 (Naik)");
    if (!a || !b || !out) return fail(HISQ_EINVAL, "NULL pointer");
    ForcePtrs fp;
    memset(&fp, 0, sizeof(fp));
    for (int k = 0; k < n; ++k) {
        if (!a[k] || !b[k]) return fail(HISQ_EINVAL, "NULL vector pointer for rhs %d", k);
        if (!aligned_for(a[k], HISQ_F64) || !aligned_for(b[k], HISQ_F64))
            return fail(HISQ_EINVAL, "vector pointer for rhs %d is not 16-byte aligned", k);
        fp.a[k] = (const double2*)a[k];
        fp.b[k] = (const double2*)b[k];
    }
    if (!aligned_for(out, HISQ_F64)) return fail(HISQ_EINVAL, "force output is not 16-byte aligned");
    HISQ_CUDA(launch_link_force(g->g, hop, mu, coef, n, fp, (double2*)out, (cudaStream_t)stream));
    return HISQ_OK;
}

extern "C" hisq_status hisq_cdot(hisq_gauge g, const void* const a[], const void* const b[], int n,
                                long long len, double* out, void* stream) {
    if (!g) return fail(HISQ_EINVAL, "NULL handle");
    if (n < 1 || n > kMaxRhs) return fail(HISQ_EINVAL, "n = %d outside 1..%d", n, kMaxRhs);
    if (len < 1) return fail(HISQ_EINVAL, "len must be >= 1");
    if (!a || !b || !out) return fail(HISQ_EINVAL, "NULL pointer");
    ForcePtrs fp;
    memset(&fp, 0, sizeof(fp));
    for (int k = 0; k < n; ++k) {
        if (!a[k] || !b[k]) return fail(HISQ_EINVAL, "NULL vector pointer for rhs %d", k);
        if (!aligned_for(a[k], HISQ_F64) || !aligned_for(b[k], HISQ_F64))
            return fail(HISQ_EINVAL, "vector pointer for rhs %d is not 16-byte aligned", k);
        fp.a[k] = (const double2*)a[k];
        fp.b[k] = (const double2*)b[k];
    }
    std::lock_guard<std::mutex> lock(g->mtx);
    if (!g->dot_partials) {
        HISQ_CUDA(cudaMalloc(&g->dot_partials, sizeof(double) * kMaxRedVals * kMaxRedBlocks));
        HISQ_CUDA(cudaMalloc(&g->dot_counter, sizeof(unsigned int)));
        HISQ_CUDA(cudaMemset(g->dot_counter, 0, sizeof(unsigned int)));
        HISQ_CUDA(cudaMalloc(&g->dot_out, sizeof(double) * kMaxRedVals));
    }
    cudaStream_t s = (cudaStream_t)stream;
    RedScratch red{g->dot_partials, g->dot_counter};
    HISQ_CUDA(launch_cdot(fp, len, n, red, g->dot_out, s));
    HISQ_CUDA(cudaMemcpyAsync(out, g->dot_out, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, s));
    HISQ_CUDA(cudaStreamSynchronize(s));
    return HISQ_OK;
}

// ---------------------------------------------------------------------------
// Conjugate gradient
// ---------------------------------------------------------------------------
extern "C" void hisq_cg_default_params(hisq_cg_params* p) {
    if (!p) return;
    p->maxiter = 100000;
    p->reliable_every = 50;
    p->reliable_delta = 0.1;
    p->inner_prec = HISQ_F32;
    p->use_x0 = 0;
    p->even_odd = 1;
    p->check_every = 10;
    p->use_graphs = 1;
    p->rhs_per_thread = 0;
    // the bundle layout where n fits it (F32 / F16 even-odd solves), else AoS
    p->spinor_layout = HISQ_BUNDLE;
    p->device_loop = 1;
    p->profile_kernels = 0;
}

namespace {

hisq_status get_workspace(hisq_gauge g, int n, int prec, int full, Workspace** out) {
    for (Workspace* w : g->ws)
        if (w->n == n && w->prec == prec && w->full == full) {
            *out = w;
            return HISQ_OK;
        }
    Workspace* w = new Workspace();
    w->n = n;
    w->prec = prec;
    w->full = full;
    w->len_half = 3ll * g->g.vh;
    w->len = full ? 2 * w->len_half : w->len_half;
    const size_t lo = (size_t)n * w->len * prec_complex_bytes(prec);
    const size_t xlo = (size_t)n * w->len * prec_complex_bytes(solution_prec(prec));
    const size_t hi = (size_t)n * w->len * sizeof(double2);
    const size_t tlo = (size_t)n * w->len * prec_complex_bytes(prec);
    const size_t thi = (size_t)n * w->len * sizeof(double2);
    cudaError_t e = cudaSuccess;
    auto al = [&](void** p, size_t sz) {
        if (e == cudaSuccess) {
            e = cudaMalloc(p, sz);
            if (e == cudaSuccess) w->bytes += sz;
        }
    };
    al(&w->r_lo, lo);
    al(&w->p_lo, lo);
    al(&w->Ap_lo, lo);
    al(&w->x_lo, xlo);
    al(&w->t_lo, tlo);
    al((void**)&w->b_hi, hi);
    al((void**)&w->x_hi, hi);
    al((void**)&w->r_hi, hi);
    al((void**)&w->t_hi, thi);
    al((void**)&w->x_best, hi);
    al((void**)&w->cg, sizeof(CgScalars));
    al((void**)&w->partials, sizeof(double) * kMaxRedVals * kMaxRedBlocks);
    al((void**)&w->counter, sizeof(unsigned int) * 4);
    if (e == cudaSuccess) e = cudaMemset(w->counter, 0, sizeof(unsigned int) * 4);
    // vectors of rhs that never iterate must still hold finite numbers
    void* zero_lo[] = {w->r_lo, w->p_lo, w->Ap_lo, w->t_lo};
    for (void* z : zero_lo)
        if (e == cudaSuccess) e = cudaMemset(z, 0, lo);
    if (e == cudaSuccess) e = cudaMemset(w->x_lo, 0, xlo);
    double2* zero_hi[] = {w->b_hi, w->x_hi, w->r_hi, w->t_hi, w->x_best};
    for (double2* z : zero_hi)
        if (e == cudaSuccess) e = cudaMemset(z, 0, hi);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&w->cg_host, sizeof(CgScalars));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w->cap_body, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w->cap_if, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        free_workspace(w);
        return fail(e == cudaErrorMemoryAllocation ? HISQ_ENOMEM : HISQ_ECUDA,
                    "CG workspace allocation failed: %s", cudaGetErrorString(e));
    }
    g->ws.push_back(w);
    *out = w;
    return HISQ_OK;
}

// ---------------------------------------------------------------------------
// Device-driven iteration loop: after every chunk of iterations a one-warp
// kernel takes the decisions the host would take (reliable update or not),
// sets the condition of an IF node holding the reliable update, and a second
// one-warp kernel after it books the update, detects convergence, the
// iteration cap and breakdowns, and sets the condition of the WHILE node
// that repeats the chunk. The host launches one graph per solve.
// ---------------------------------------------------------------------------
struct LoopArgs {
    CgScalars* cg;
    int n;
    int chunk;
    int maxiter;
    int reliable_every;
    double delta2;                        // reliable_delta^2
    double tol2;
    cudaGraphConditionalHandle h_if;      // runs the reliable update
    cudaGraphConditionalHandle h_loop;    // repeats the chunk
};

__global__ void loop_decide_kernel(LoopArgs a) {
    CgScalars* cg = a.cg;
    const int k = threadIdx.x;
    const int iter = cg->iter + a.chunk;
    const int since = cg->since_rel + a.chunk;
    int need = 0;
    if (k < a.n) {
        const int act = cg->active[k];
        const int restarted = act && cg->restarts[k] != cg->seen_restarts[k];
        cg->seen_restarts[k] = cg->restarts[k];
        cg->restarted[k] = restarted;
        if (act) {
            const double sc = cg->scale[k];
            need = cg->frozen[k] || restarted || cg->rr[k] <= a.delta2 * cg->rr_rel[k] ||
                   cg->rr[k] <= a.tol2 * cg->bb[k] * sc * sc;
        }
        cg->was[k] = act;
        cg->before[k] = cg->rr_true[k];
    }
    need = __any_sync(0xffffffffu, need) || since >= a.reliable_every || iter >= a.maxiter;
    if (cg->flags) need = 0;   // the post step stops the loop
    if (k == 0) {
        cg->iter = iter;
        cg->since_rel = since;
        cg->need = need;
        cudaGraphSetConditional(a.h_if, need ? 1u : 0u);
    }
}

__global__ void loop_post_kernel(LoopArgs a) {
    CgScalars* cg = a.cg;
    const int k = threadIdx.x;
    const int need = cg->need;
    const int iter = cg->iter;
    int broke = 0;
    if (need && k < a.n) {
        if (cg->was[k] && !cg->active[k]) cg->iters_k[k] = iter;
        // restarts that bring no progress of the FP64 residual are a breakdown
        const int bad = (cg->was[k] && cg->active[k] && cg->restarted[k] && !(cg->rr_true[k] < cg->before[k]))
                            ? cg->bad_updates[k] + 1
                            : 0;
        cg->bad_updates[k] = bad;
        broke = bad >= 3;
    }
    broke = __any_sync(0xffffffffu, broke);
    const int any_active = __any_sync(0xffffffffu, k < a.n && cg->active[k]);
    if (k == 0) {
        int result = cg->result;
        if (need) {
            cg->reliable += 1;
            cg->since_rel = 0;
        }
        if (broke) result = HISQ_EBREAKDOWN;
        int done = !any_active || cg->flags || result != HISQ_OK;
        if (!done && iter >= a.maxiter) {
            result = HISQ_ENOCONV;
            done = 1;
        }
        cg->result = result;
        cudaGraphSetConditional(a.h_loop, done ? 0u : 1u);
    }
}

struct Solver {
    hisq_gauge g;
    Workspace* w;
    int n, prec, full;
    bool bundle = false;       // low-precision vectors in the bundle layout
    bool profile = false;      // time the launches of each iteration (profile_kernels)
    DslashTune tune, tune64;   // inner (low precision) and FP64 Dslash mappings
    double mass, mu;
    double tol2;

    BlasArgs blas() const {
        BlasArgs b;
        b.n = n;
        b.len = w->len;
        b.red.partials = w->partials;
        b.red.counter = w->counter;
        b.cg = w->cg;
        // freeze an rhs when its low-precision residual fell far enough to
        // risk underflow / stagnation before the host schedules an update
        b.freeze2 = prec == HISQ_F16 ? 1e-6 : prec == HISQ_F32 ? 1e-10 : 0.0;
        // A >= 4m^2 for the even-odd operator and for M^dag M at mu = 0, and
        // alpha = rr / pAp <= rr / (4m^2 |p|^2) <= 1 / (4m^2); twice that
        // bound leaves room for rounding. No bound is used at mu != 0.
        b.alpha_max = (mu == 0.0 && mass != 0.0) ? 2.0 / (4.0 * mass * mass) : HUGE_VAL;
        return b;
    }

    void* lo_ptr(void* base, int k, long long off = 0) const {
        return (char*)base + ((size_t)k * w->len + off) * prec_complex_bytes(prec);
    }
    double2* hi_ptr(double2* base, int k, long long off = 0) const {
        return base + (size_t)k * w->len + off;
    }

    DslashArgs args(int p, int lp) const {
        DslashArgs a;
        fill_common(a, g, lp, p, n);
        a.red.partials = w->partials;
        a.red.counter = w->counter;
        a.cg = w->cg;
        a.status = &w->cg->flags;
        a.tol2 = tol2;
        return a;
    }

    // Low-precision A p -> Ap; the last reduction block forms alpha. `mid`
    // (profiling) is recorded between the first and the second operator half.
    cudaError_t apply_lo(cudaStream_t s, cudaEvent_t mid = nullptr) const {
        const int ru = g->recon_U, rn = g->recon_N;
        cudaError_t e;
        if (bundle) {
            DslashArgs a = args(1, prec);   // t = D_oe p
            a.in[0] = w->p_lo;
            a.out[0] = w->t_lo;
            e = launch_dslash(a, prec, ru, rn, EPI_NONE, tune, s);
            if (e == cudaSuccess && mid) e = cudaEventRecord(mid, s);
            if (e != cudaSuccess) return e;
            DslashArgs b = args(0, prec);   // Ap = 4m^2 p - D_eo t, pAp = Re<p, Ap>
            b.cx = 4.0 * mass * mass;
            b.cd = -1.0;
            b.red_mode = RED_DOT_XW;
            b.finish = FIN_CG_ALPHA;
            b.in[0] = w->t_lo;
            b.out[0] = w->Ap_lo;
            b.x[0] = w->p_lo;
            return launch_dslash(b, prec, ru, rn, EPI_X, tune, s);
        }
        if (!full) {
            DslashArgs a = args(1, prec);   // t = D_oe p
            for (int k = 0; k < n; ++k) {
                a.in[k] = lo_ptr(w->p_lo, k);
                a.out[k] = lo_ptr(w->t_lo, k);
            }
            e = launch_dslash(a, prec, ru, rn, EPI_NONE, tune, s);
            if (e == cudaSuccess && mid) e = cudaEventRecord(mid, s);
            if (e != cudaSuccess) return e;
            DslashArgs b = args(0, prec);   // Ap = 4m^2 p - D_eo t, pAp = Re<p, Ap>
            b.cx = 4.0 * mass * mass;
            b.cd = -1.0;
            b.red_mode = RED_DOT_XW;
            b.finish = FIN_CG_ALPHA;
            for (int k = 0; k < n; ++k) {
                b.in[k] = lo_ptr(w->t_lo, k);
                b.out[k] = lo_ptr(w->Ap_lo, k);
                b.x[k] = lo_ptr(w->p_lo, k);
            }
            return launch_dslash(b, prec, ru, rn, EPI_X, tune, s);
        }
        // full lattice: y = M(mu) p into t, Ap = M(mu)^dag y, then alpha from Re<p, Ap>
        const long long hl = w->len_half;
        for (int par = 0; par < 2; ++par) {
            DslashArgs a = args(par, prec);
            set_mu(a, mu);
            a.cx = 2.0 * mass;
            a.cd = 1.0;
            for (int k = 0; k < n; ++k) {
                a.in[k] = lo_ptr(w->p_lo, k, (1 - par) * hl);
                a.out[k] = lo_ptr(w->t_lo, k, par * hl);
                a.x[k] = lo_ptr(w->p_lo, k, par * hl);
            }
            e = launch_dslash(a, prec, ru, rn, EPI_X, tune, s);
            if (e != cudaSuccess) return e;
        }
        if (mid) {
            e = cudaEventRecord(mid, s);
            if (e != cudaSuccess) return e;
        }
        for (int par = 0; par < 2; ++par) {
            DslashArgs a = args(par, prec);
            set_mu(a, -mu);
            a.cx = 2.0 * mass;
            a.cd = -1.0;
            for (int k = 0; k < n; ++k) {
                a.in[k] = lo_ptr(w->t_lo, k, (1 - par) * hl);
                a.out[k] = lo_ptr(w->Ap_lo, k, par * hl);
                a.x[k] = lo_ptr(w->t_lo, k, par * hl);
            }
            e = launch_dslash(a, prec, ru, rn, EPI_X, tune, s);
            if (e != cudaSuccess) return e;
        }
        return launch_dot_alpha(blas(), prec, w->p_lo, w->Ap_lo, s);
    }

    // One CG iteration on every active rhs; ev (profiling) gets 5 events
    // around its four launches.
    cudaError_t iterate(cudaStream_t s, const cudaEvent_t* ev = nullptr) const {
        cudaError_t e = ev ? cudaEventRecord(ev[0], s) : cudaSuccess;
        if (e == cudaSuccess) e = apply_lo(s, ev ? ev[1] : nullptr);
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], s);
        if (bundle) {
            if (e == cudaSuccess) e = launch_cg_update_r_bundle(blas(), prec, w->r_lo, w->Ap_lo, s);
            if (e == cudaSuccess && ev) e = cudaEventRecord(ev[3], s);
            if (e == cudaSuccess) e = launch_cg_update_px_bundle(blas(), prec, w->x_lo, w->r_lo, w->p_lo, s);
        } else {
            if (e == cudaSuccess) e = launch_cg_update_r(blas(), prec, w->r_lo, w->Ap_lo, s);
            if (e == cudaSuccess && ev) e = cudaEventRecord(ev[3], s);
            if (e == cudaSuccess) e = launch_cg_update_px(blas(), prec, w->x_lo, w->r_lo, w->p_lo, s);
        }
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[4], s);
        return e;
    }

    // r_hi = b - A x_hi in FP64 with the reliable finish (convergence, scale).
    cudaError_t true_residual(cudaStream_t s) const {
        const int f = HISQ_F64;
        cudaError_t e;
        if (!full) {
            DslashArgs a = args(1, f);   // t = D_oe x
            for (int k = 0; k < n; ++k) {
                a.in[k] = hi_ptr(w->x_hi, k);
                a.out[k] = hi_ptr(w->t_hi, k);
            }
            e = launch_dslash(a, f, 18, 18, EPI_NONE, tune64, s);
            if (e != cudaSuccess) return e;
            DslashArgs b = args(0, f);   // r = b - 4m^2 x + D_eo t
            b.cx = -4.0 * mass * mass;
            b.cd = 1.0;
            b.red_mode = RED_NORM_MAX_W;
            b.finish = FIN_RELIABLE;
            for (int k = 0; k < n; ++k) {
                b.in[k] = hi_ptr(w->t_hi, k);
                b.out[k] = hi_ptr(w->r_hi, k);
                b.x[k] = hi_ptr(w->x_hi, k);
                b.y[k] = hi_ptr(w->b_hi, k);
            }
            return launch_dslash(b, f, 18, 18, EPI_XY, tune64, s);
        }
        const long long hl = w->len_half;
        for (int par = 0; par < 2; ++par) {   // y = M(mu) x
            DslashArgs a = args(par, f);
            set_mu(a, mu);
            a.cx = 2.0 * mass;
            a.cd = 1.0;
            for (int k = 0; k < n; ++k) {
                a.in[k] = hi_ptr(w->x_hi, k, (1 - par) * hl);
                a.out[k] = hi_ptr(w->t_hi, k, par * hl);
                a.x[k] = hi_ptr(w->x_hi, k, par * hl);
            }
            e = launch_dslash(a, f, 18, 18, EPI_X, tune64, s);
            if (e != cudaSuccess) return e;
        }
        for (int par = 0; par < 2; ++par) {   // r = b - 2m y + D(-mu) y
            DslashArgs a = args(par, f);
            set_mu(a, -mu);
            a.cx = -2.0 * mass;
            a.cd = 1.0;
            for (int k = 0; k < n; ++k) {
                a.in[k] = hi_ptr(w->t_hi, k, (1 - par) * hl);
                a.out[k] = hi_ptr(w->r_hi, k, par * hl);
                a.x[k] = hi_ptr(w->t_hi, k, par * hl);
                a.y[k] = hi_ptr(w->b_hi, k, par * hl);
            }
            e = launch_dslash(a, f, 18, 18, EPI_XY, tune64, s);
            if (e != cudaSuccess) return e;
        }
        return launch_residual_norm(blas(), w->r_hi, tol2, s);
    }

    cudaError_t accum(cudaStream_t s) const {
        return bundle ? launch_accum_solution_bundle(blas(), prec, w->x_hi, w->x_lo, g->g.vh, s)
                      : launch_accum_solution(blas(), prec, w->x_hi, w->x_lo, s);
    }

    cudaError_t rescale(int reset_p, cudaStream_t s) const {
        return bundle ? launch_reliable_rescale_bundle(blas(), prec, w->r_hi, w->r_lo, w->p_lo, reset_p, g->g.vh, s)
                      : launch_reliable_rescale(blas(), prec, w->r_hi, w->r_lo, w->p_lo, reset_p, s);
    }

    cudaError_t reliable_update(cudaStream_t s) const {
        cudaError_t e = accum(s);
        if (e == cudaSuccess) e = true_residual(s);
        if (e == cudaSuccess) e = launch_keep_best(blas(), w->x_hi, w->x_best, s);
        if (e == cudaSuccess) e = rescale(0, s);
        return e;
    }

    cudaError_t poll(cudaStream_t s) const {
        cudaError_t e = cudaMemcpyAsync(w->cg_host, w->cg, sizeof(CgScalars), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return e;
    }

    // Adds to the graph being captured on stream s a WHILE node whose body runs
    // la.chunk iterations, the decision kernel, an IF node holding the
    // reliable update, and the booking kernel (see loop_decide_kernel).
    cudaError_t capture_loop(cudaStream_t s, LoopArgs la) const {
        cudaStreamCaptureStatus cs;
        cudaGraph_t graph = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &graph, &deps, nullptr, &nd);
        if (e != cudaSuccess) return e;
        cudaGraphConditionalHandle h_loop;
        e = cudaGraphConditionalHandleCreate(&h_loop, graph, 1, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) return e;
        // node parameters in zeroed raw storage (the struct has no default constructor)
        alignas(cudaGraphNodeParams) unsigned char wbuf[sizeof(cudaGraphNodeParams)] = {};
        cudaGraphNodeParams& wp = *reinterpret_cast<cudaGraphNodeParams*>(wbuf);
        wp.type = cudaGraphNodeTypeConditional;
        wp.conditional.handle = h_loop;
        wp.conditional.type = cudaGraphCondTypeWhile;
        wp.conditional.size = 1;
        cudaGraphNode_t wnode;
        e = cudaGraphAddNode(&wnode, graph, deps, nullptr, nd, &wp);
        if (e != cudaSuccess) return e;
        e = cudaStreamUpdateCaptureDependencies(s, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies);
        if (e != cudaSuccess) return e;
        cudaGraph_t body = wp.conditional.phGraph_out[0];
        cudaGraphConditionalHandle h_if;
        e = cudaGraphConditionalHandleCreate(&h_if, body, 0, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) return e;
        la.h_if = h_if;
        la.h_loop = h_loop;
        cudaStream_t sb = w->cap_body, si = w->cap_if;
        e = cudaStreamBeginCaptureToGraph(sb, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        for (int i = 0; i < la.chunk && e == cudaSuccess; ++i) e = iterate(sb);
        if (e == cudaSuccess) {
            loop_decide_kernel<<<1, 32, 0, sb>>>(la);
            e = cudaGetLastError();
        }
        cudaGraph_t g2 = nullptr;
        if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(sb, &cs, nullptr, &g2, &deps, nullptr, &nd);
        alignas(cudaGraphNodeParams) unsigned char ibuf[sizeof(cudaGraphNodeParams)] = {};
        cudaGraphNodeParams& ip = *reinterpret_cast<cudaGraphNodeParams*>(ibuf);
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = h_if;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        cudaGraphNode_t inode;
        if (e == cudaSuccess) e = cudaGraphAddNode(&inode, g2, deps, nullptr, nd, &ip);
        if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(sb, &inode, nullptr, 1, cudaStreamSetCaptureDependencies);
        if (e == cudaSuccess) {
            e = cudaStreamBeginCaptureToGraph(si, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e1 = reliable_update(si);
                cudaGraph_t gi = nullptr;
                cudaError_t e2 = cudaStreamEndCapture(si, &gi);
                e = e1 != cudaSuccess ? e1 : e2;
            }
        }
        if (e == cudaSuccess) {
            loop_post_kernel<<<1, 32, 0, sb>>>(la);
            e = cudaGetLastError();
        }
        cudaGraph_t gb = nullptr;
        cudaError_t e3 = cudaStreamEndCapture(sb, &gb);
        return e != cudaSuccess ? e : e3;
    }

    // Run `chunk` iterations, from a captured graph when enabled.
    hisq_status run_chunk(int chunk, bool graphs, cudaStream_t s) {
        if (profile) {
            // every iteration but the chunk's first (which follows the host's
            // poll, so the GPU may wait for its launch) is timed
            const size_t need = 5 * (size_t)chunk;
            while (w->prof_ev.size() < need) {
                cudaEvent_t e;
                HISQ_CUDA(cudaEventCreate(&e));
                w->prof_ev.push_back(e);
            }
            for (int i = 0; i < chunk; ++i) HISQ_CUDA(iterate(s, i > 0 ? &w->prof_ev[5 * i] : nullptr));
            if (chunk > 1) {
                HISQ_CUDA(cudaEventSynchronize(w->prof_ev[5 * (chunk - 1) + 4]));
                for (int i = 1; i < chunk; ++i) {
                    for (int k = 0; k < 4; ++k) {
                        float ms = 0.f;
                        HISQ_CUDA(cudaEventElapsedTime(&ms, w->prof_ev[5 * i + k], w->prof_ev[5 * i + k + 1]));
                        w->prof_us[k] += 1e3 * ms;
                    }
                    ++w->prof_iters;
                }
            }
            return HISQ_OK;
        }
        if (!graphs) {
            for (int i = 0; i < chunk; ++i) HISQ_CUDA(iterate(s));
            return HISQ_OK;
        }
        GraphKey key{chunk, mass, mu, tune.kind * 1000 + tune.rpt * 100 + tune.minb * 10 + tune.layout};
        auto it = w->graphs.find(key);
        if (it == w->graphs.end()) {
            if (w->graphs.size() >= 8) {
                for (auto& kv : w->graphs) cudaGraphExecDestroy(kv.second);
                w->graphs.clear();
            }
            cudaGraph_t graph = nullptr;
            HISQ_CUDA(cudaStreamBeginCapture(w->cap_stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            for (int i = 0; i < chunk && e == cudaSuccess; ++i) e = iterate(w->cap_stream);
            cudaError_t e2 = cudaStreamEndCapture(w->cap_stream, &graph);
            HISQ_CUDA(e);
            HISQ_CUDA(e2);
            cudaGraphExec_t exec = nullptr;
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            HISQ_CUDA(e);
            it = w->graphs.emplace(key, exec).first;
        }
        HISQ_CUDA(cudaGraphLaunch(it->second, s));
        return HISQ_OK;
    }
};

}  // namespace

// One solve in progress: setup, host-side decisions after every chunk of
// iterations, and the final copy-out. hisq_cg_solve drives one of these;
// hisq_cg_solve_batched drives several through one CUDA graph per chunk.
namespace {

struct CgRun {
    hisq_gauge g = nullptr;
    Workspace* w = nullptr;
    Solver sv;
    hisq_cg_params prm;
    void* const* x = nullptr;
    int n = 0, halves = 1;
    bool soa = true;
    size_t vec_bytes = 0;
    int iters_k[kMaxRhs], seen_restarts[kMaxRhs], bad_updates[kMaxRhs];
    int iter = 0, since_rel = 0, reliable = 0;
    hisq_status result = HISQ_OK;
    bool stop = false;
    std::chrono::steady_clock::time_point t0;

    static bool debug() {
        static const bool d = [] {
            const char* e = getenv("HISQ_DEBUG_CG");
            return e != nullptr && e[0] != '\0' && e[0] != '0';
        }();
        return d;
    }

    // Validates the request (handle lock held by the caller).
    static hisq_status check(hisq_gauge g, double mass, double mu, const void* const b[], void* const x[],
                             int n, double tol, const hisq_cg_params* p, hisq_cg_params* out) {
        if (!g) return fail(HISQ_EINVAL, "NULL handle");
        if (n < 1 || n > kMaxRhs) return fail(HISQ_EINVAL, "n = %d outside 1..%d", n, kMaxRhs);
        if (!(tol > 0.0) || !std::isfinite(tol)) return fail(HISQ_EINVAL, "tol must be positive and finite");
        if (!std::isfinite(mass) || !std::isfinite(mu)) return fail(HISQ_EINVAL, "mass and mu must be finite");
        if (!b || !x) return fail(HISQ_EINVAL, "NULL pointer array");
        for (int k = 0; k < n; ++k)
            if (!b[k] || !x[k]) return fail(HISQ_EINVAL, "NULL source or solution pointer for rhs %d", k);
        hisq_cg_params prm;
        hisq_cg_default_params(&prm);
        if (p) prm = *p;
        if (!valid_prec(prm.inner_prec)) return fail(HISQ_EINVAL, "unknown inner precision %d", prm.inner_prec);
        if (prm.inner_prec != HISQ_F64 && prm.inner_prec != g->prec)
            return fail(HISQ_EINVAL, "inner precision %d needs links stored in that precision (handle has %d)",
                        prm.inner_prec, g->prec);
        if (prm.even_odd && mu != 0.0)
            return fail(HISQ_EINVAL, "mu != 0 needs the full-lattice solve (even_odd = 0)");
        if (prm.maxiter < 1) return fail(HISQ_EINVAL, "maxiter must be >= 1");
        if (prm.check_every < 1) prm.check_every = 1;
        if (prm.reliable_every < 1) prm.reliable_every = 1 << 30;
        if (prm.spinor_layout != HISQ_AOS && prm.spinor_layout != HISQ_SOA && prm.spinor_layout != HISQ_BUNDLE)
            return fail(HISQ_EINVAL, "unknown spinor layout %d", prm.spinor_layout);
        if (!(prm.reliable_delta >= 0.0 && prm.reliable_delta < 1.0))
            return fail(HISQ_EINVAL, "reliable_delta must be in [0, 1)");
        if (prm.profile_kernels) {   // the timed launches come from the host
            prm.use_graphs = 0;
            prm.device_loop = 0;
        }
        *out = prm;
        return HISQ_OK;
    }

    hisq_status start(hisq_gauge gg, double mass, double mu, const void* const b[], void* const xx[], int nn,
                      double tol, const hisq_cg_params& p, cudaStream_t s) {
        t0 = std::chrono::steady_clock::now();
        g = gg;
        prm = p;
        x = xx;
        n = nn;
        const int full = prm.even_odd ? 0 : 1;
        hisq_status st = get_workspace(g, n, prm.inner_prec, full, &w);
        if (st != HISQ_OK) return st;
        sv.g = g;
        sv.w = w;
        sv.n = n;
        sv.prec = prm.inner_prec;
        sv.full = full;
        // the bundle layout where it fits, else the ABI layout
        if (prm.spinor_layout == HISQ_BUNDLE) {
            const DslashTune tb = full ? DslashTune{} : pick_tune(g, n, sv.prec, prm.rhs_per_thread, HISQ_BUNDLE);
            sv.bundle = !full && bundle_width(sv.prec) != 0 && tb.rpt != 0;
            if (!sv.bundle) prm.spinor_layout = HISQ_AOS;
        }
        sv.tune = pick_tune(g, n, sv.prec, prm.rhs_per_thread, prm.spinor_layout);
        sv.tune64 = pick_tune(g, n, HISQ_F64, 0, sv.bundle ? HISQ_AOS : prm.spinor_layout);
        sv.mass = mass;
        sv.mu = mu;
        sv.tol2 = tol * tol;
        sv.profile = prm.profile_kernels != 0;
        for (int k = 0; k < 4; ++k) w->prof_us[k] = 0.0;
        w->prof_iters = 0;
        for (int k = 0; k < n; ++k) iters_k[k] = seen_restarts[k] = bad_updates[k] = 0;

        // sources and initial guess into the FP64 blocks; the caller's vectors
        // are AoS, an SoA solve transposes them through r_hi
        vec_bytes = (size_t)w->len * sizeof(double2);
        soa = prm.spinor_layout == HISQ_SOA;
        halves = full ? 2 : 1;
        double2* bdst = soa ? w->r_hi : w->b_hi;
        for (int k = 0; k < n; ++k)
            HISQ_CUDA(cudaMemcpyAsync(sv.hi_ptr(bdst, k), b[k], vec_bytes, cudaMemcpyDefault, s));
        if (soa) HISQ_CUDA(launch_transpose_spinor(w->r_hi, w->b_hi, n, halves, g->g.vh, 1, s));
        if (prm.use_x0) {
            double2* xdst = soa ? w->r_hi : w->x_hi;
            for (int k = 0; k < n; ++k)
                HISQ_CUDA(cudaMemcpyAsync(sv.hi_ptr(xdst, k), x[k], vec_bytes, cudaMemcpyDefault, s));
            if (soa) HISQ_CUDA(launch_transpose_spinor(w->r_hi, w->x_hi, n, halves, g->g.vh, 1, s));
        } else {
            HISQ_CUDA(cudaMemsetAsync(w->x_hi, 0, vec_bytes * n, s));
        }
        HISQ_CUDA(cudaMemsetAsync(w->cg, 0, sizeof(CgScalars), s));
        HISQ_CUDA(cudaMemsetAsync(w->x_lo, 0, (size_t)n * w->len * prec_complex_bytes(solution_prec(sv.prec)), s));
        HISQ_CUDA(launch_norm_bb(sv.blas(), w->b_hi, s));
        if (prm.use_x0) {
            HISQ_CUDA(sv.true_residual(s));
        } else {
            HISQ_CUDA(launch_copy_residual(sv.blas(), w->b_hi, w->r_hi, sv.tol2, s));
        }
        HISQ_CUDA(launch_keep_best(sv.blas(), w->x_hi, w->x_best, s));
        HISQ_CUDA(sv.rescale(1, s));
        HISQ_CUDA(sv.poll(s));
        update_stop();
        return HISQ_OK;
    }

    void update_stop() {
        const CgScalars& h = *w->cg_host;
        bool any = false;
        for (int k = 0; k < n; ++k) any = any || h.active[k];
        if (!any || h.flags || result != HISQ_OK) stop = true;
        if (!stop && iter >= prm.maxiter) {
            result = HISQ_ENOCONV;
            stop = true;
        }
    }

    // Iterations to run before the next host decision.
    int next_chunk() const {
        int chunk = prm.check_every;
        if (chunk > prm.reliable_every - since_rel) chunk = prm.reliable_every - since_rel;
        if (chunk > prm.maxiter - iter) chunk = prm.maxiter - iter;
        return chunk < 1 ? 1 : chunk;
    }

    // After `chunk` iterations ran on stream s: poll, decide on a reliable update.
    hisq_status after_chunk(int chunk, cudaStream_t s) {
        iter += chunk;
        since_rel += chunk;
        HISQ_CUDA(sv.poll(s));
        const CgScalars& h = *w->cg_host;
        if (debug()) {
            fprintf(stderr, "[hisq cg] iter %d flags %d\n", iter, h.flags);
            for (int k = 0; k < n; ++k)
                fprintf(stderr, "  rhs %d active %d frozen %d restarts %d rr %.3e rr_rel %.3e pAp %.3e alpha %.3e "
                        "beta %.3e rr_true %.3e bb %.3e scale %.3e\n", k, h.active[k], h.frozen[k],
                        h.restarts[k], h.rr[k], h.rr_rel[k], h.pAp[k], h.alpha[k], h.beta[k], h.rr_true[k],
                        h.bb[k], h.scale[k]);
        }
        if (h.flags) {
            stop = true;
            return HISQ_OK;
        }
        const double d2 = prm.reliable_delta * prm.reliable_delta;
        bool need = since_rel >= prm.reliable_every || iter >= prm.maxiter;
        bool restarted[kMaxRhs];
        for (int k = 0; k < n; ++k) {
            restarted[k] = h.active[k] && h.restarts[k] != seen_restarts[k];
            seen_restarts[k] = h.restarts[k];
            if (!h.active[k]) continue;
            if (h.frozen[k] || restarted[k]) need = true;
            if (h.rr[k] <= d2 * h.rr_rel[k]) need = true;
            if (h.rr[k] <= sv.tol2 * h.bb[k] * h.scale[k] * h.scale[k]) need = true;
        }
        if (need) {
            int was[kMaxRhs];
            double before[kMaxRhs];
            for (int k = 0; k < n; ++k) {
                was[k] = h.active[k];
                before[k] = h.rr_true[k];
            }
            HISQ_CUDA(sv.reliable_update(s));
            HISQ_CUDA(sv.poll(s));
            ++reliable;
            since_rel = 0;
            const CgScalars& a = *w->cg_host;
            for (int k = 0; k < n; ++k) {
                if (was[k] && !a.active[k]) iters_k[k] = iter;
                // restarts that bring no progress of the FP64 residual are a breakdown
                if (was[k] && a.active[k] && restarted[k] && !(a.rr_true[k] < before[k]))
                    ++bad_updates[k];
                else
                    bad_updates[k] = 0;
                if (bad_updates[k] >= 3) result = HISQ_EBREAKDOWN;
            }
        }
        update_stop();
        return HISQ_OK;
    }

    // Whether the whole solve can run as one graph launch (the chunk of the
    // loop body divides the iteration cap and the reliable-update period).
    bool device_loop_ok() const {
        const int c = prm.check_every;
        return prm.use_graphs && prm.device_loop && prm.maxiter % c == 0 &&
               (prm.reliable_every % c == 0 || prm.reliable_every >= prm.maxiter);
    }

    LoopArgs loop_args() const {
        LoopArgs la;
        la.cg = w->cg;
        la.n = n;
        la.chunk = prm.check_every;
        la.maxiter = prm.maxiter;
        la.reliable_every = prm.reliable_every;
        la.delta2 = prm.reliable_delta * prm.reliable_delta;
        la.tol2 = sv.tol2;
        la.h_if = la.h_loop = 0;
        return la;
    }

    // After the device loop ended: read its book-keeping into the host state.
    hisq_status after_device_loop(cudaStream_t s) {
        HISQ_CUDA(sv.poll(s));
        const CgScalars& h = *w->cg_host;
        iter = h.iter;
        reliable = h.reliable;
        for (int k = 0; k < n; ++k) iters_k[k] = h.iters_k[k];
        if (h.result != HISQ_OK && result == HISQ_OK) result = (hisq_status)h.result;
        stop = true;
        return HISQ_OK;
    }

    // The solve as one launch of a cached graph holding the device loop.
    hisq_status run_device_loop(cudaStream_t s) {
        const auto key = std::make_tuple(prm.check_every, sv.mass, sv.mu,
                                         sv.tune.kind * 10000 + sv.tune.rpt * 100 + sv.tune.minb * 10 + sv.tune.layout,
                                         prm.maxiter, prm.reliable_every, prm.reliable_delta, sv.tol2);
        auto it = w->loops.find(key);
        if (it == w->loops.end()) {
            if (w->loops.size() >= 4) {
                for (auto& kv : w->loops) cudaGraphExecDestroy(kv.second);
                w->loops.clear();
            }
            cudaGraph_t graph = nullptr;
            HISQ_CUDA(cudaStreamBeginCapture(w->cap_stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = sv.capture_loop(w->cap_stream, loop_args());
            cudaError_t e2 = cudaStreamEndCapture(w->cap_stream, &graph);
            HISQ_CUDA(e);
            HISQ_CUDA(e2);
            cudaGraphExec_t exec = nullptr;
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            HISQ_CUDA(e);
            it = w->loops.emplace(key, exec).first;
        }
        HISQ_CUDA(cudaGraphLaunch(it->second, s));
        return after_device_loop(s);
    }

    // Copy the solution out, fill stats and return the status of the solve.
    hisq_status finish(hisq_cg_stats* stats, cudaStream_t s) {
        if (result == HISQ_ENOCONV) {
            for (int k = 0; k < n; ++k)
                if (w->cg_host->active[k]) iters_k[k] = iter;
        }
        if (w->cg_host->flags) {
            // fold what the low-precision solution gathered so far into x
            HISQ_CUDA(sv.accum(s));
            HISQ_CUDA(sv.poll(s));
        }
        const CgScalars& h = *w->cg_host;
        hisq_status res = result;
        if (h.flags & kFlagTimeout)
            res = fail(HISQ_ETIMEOUT, "a bounded device-side wait gave up");
        else if (h.flags & kFlagNaN)
            res = fail(HISQ_ENAN, "non-finite value in the CG (source or residual)");
        else if ((h.flags & kFlagBreakdown) || res == HISQ_EBREAKDOWN)
            res = fail(HISQ_EBREAKDOWN, "CG breakdown: <p, A p> <= 0 repeatedly with no FP64 progress");
        else if (res == HISQ_ENOCONV)
            fail(HISQ_ENOCONV, "CG did not converge in %d iterations", prm.maxiter);
        // a solve that ends without converging returns, per rhs, the solution
        // at the lowest FP64 residual it reached
        double rr_out[kMaxRhs];
        for (int k = 0; k < n; ++k) {
            rr_out[k] = h.rr_true[k];
            if (res != HISQ_OK && h.have_best[k] && !(h.rr_true[k] <= h.rr_best[k])) {
                HISQ_CUDA(cudaMemcpyAsync(sv.hi_ptr(w->x_hi, k), sv.hi_ptr(w->x_best, k), vec_bytes,
                                          cudaMemcpyDeviceToDevice, s));
                rr_out[k] = h.rr_best[k];
            }
        }
        double2* xsrc = w->x_hi;
        if (soa) {
            HISQ_CUDA(launch_transpose_spinor(w->x_hi, w->t_hi, n, halves, g->g.vh, 0, s));
            xsrc = w->t_hi;
        }
        for (int k = 0; k < n; ++k)
            HISQ_CUDA(cudaMemcpyAsync(x[k], sv.hi_ptr(xsrc, k), vec_bytes, cudaMemcpyDefault, s));
        HISQ_CUDA(cudaStreamSynchronize(s));
        if (stats) {
            memset(stats, 0, sizeof(*stats));
            for (int k = 0; k < n; ++k) {
                stats->iters[k] = iters_k[k];
                stats->true_rel_res[k] = h.bb[k] > 0 ? std::sqrt(rr_out[k] / h.bb[k]) : 0.0;
            }
            stats->total_iters = iter;
            stats->reliable_updates = reliable;
            stats->profiled_iters = w->prof_iters;
            for (int k = 0; k < 4; ++k)
                stats->kernel_us[k] = w->prof_iters > 0 ? w->prof_us[k] / w->prof_iters : 0.0;
            stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        }
        return res;
    }
};

}  // namespace

extern "C" hisq_status hisq_cg_solve(hisq_gauge g, double mass, double mu, const void* const b[],
                                     void* const x[], int n, double tol, const hisq_cg_params* p,
                                     hisq_cg_stats* stats, void* stream) {
    hisq_cg_params prm;
    hisq_status st = CgRun::check(g, mass, mu, b, x, n, tol, p, &prm);
    if (st != HISQ_OK) return st;
    std::lock_guard<std::mutex> lock(g->mtx);
    cudaStream_t s = (cudaStream_t)stream;
    CgRun run;
    st = run.start(g, mass, mu, b, x, n, tol, prm, s);
    if (st != HISQ_OK) return st;
    if (!run.stop && run.device_loop_ok()) {
        st = run.run_device_loop(s);
        if (st != HISQ_OK) return st;
    }
    while (!run.stop) {
        const int chunk = run.next_chunk();
        st = run.sv.run_chunk(chunk, prm.use_graphs != 0, s);
        if (st != HISQ_OK) return st;
        st = run.after_chunk(chunk, s);
        if (st != HISQ_OK) return st;
    }
    return run.finish(stats, s);
}

// Several independent solves (distinct handles, e.g. lattices of uneven
// volume) advanced together: every chunk of iterations of all unfinished
// solves is one CUDA graph whose branches run the solves concurrently.
extern "C" hisq_status hisq_cg_solve_batched(const hisq_cg_problem* probs, int nprob,
                                             const hisq_cg_params* p, hisq_cg_stats* stats,
                                             void* stream) {
    if (!probs || nprob < 1 || nprob > 64) return fail(HISQ_EINVAL, "nprob must be 1..64");
    std::vector<hisq_cg_params> prm(nprob);
    for (int i = 0; i < nprob; ++i) {
        const hisq_cg_problem& q = probs[i];
        hisq_status st = CgRun::check(q.g, q.mass, q.mu, q.b, q.x, q.n, q.tol, p, &prm[i]);
        if (st != HISQ_OK) return st;
        for (int j = 0; j < i; ++j)
            if (probs[j].g == q.g) return fail(HISQ_EINVAL, "problems %d and %d share a handle", j, i);
    }
    // lock the handles in address order
    std::vector<hisq_gauge> order;
    for (int i = 0; i < nprob; ++i) order.push_back(probs[i].g);
    std::sort(order.begin(), order.end());
    std::vector<std::unique_lock<std::mutex>> locks;
    for (hisq_gauge h : order) locks.emplace_back(h->mtx);

    cudaStream_t s = (cudaStream_t)stream;
    std::vector<CgRun> runs(nprob);
    for (int i = 0; i < nprob; ++i) {
        const hisq_cg_problem& q = probs[i];
        hisq_status st = runs[i].start(q.g, q.mass, q.mu, q.b, q.x, q.n, q.tol, prm[i], s);
        if (st != HISQ_OK) return st;
    }
    const bool graphs = (p ? p->use_graphs : 1) != 0;
    cudaStream_t cap = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join(nprob, nullptr);
    std::map<std::pair<unsigned long long, int>, cudaGraphExec_t> cache;
    auto cleanup = [&]() {
        for (auto& kv : cache) cudaGraphExecDestroy(kv.second);
        for (cudaEvent_t e : join)
            if (e) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        if (cap) cudaStreamDestroy(cap);
    };
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int i = 0; i < nprob && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cleanup();
        return fail(HISQ_ECUDA, "batched solve set-up failed: %s", cudaGetErrorString(e));
    }
    hisq_status st = HISQ_OK;
    // every unfinished problem as one device loop, all in one graph launch
    bool dev_loop = graphs;
    for (int i = 0; i < nprob; ++i) dev_loop = dev_loop && (runs[i].stop || runs[i].device_loop_ok());
    if (dev_loop) {
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = cudaEventRecord(fork, cap);
        for (int i = 0; i < nprob && e == cudaSuccess; ++i) {
            if (runs[i].stop) continue;
            cudaStream_t si = runs[i].w->cap_stream;
            e = cudaStreamWaitEvent(si, fork, 0);
            if (e == cudaSuccess) e = runs[i].sv.capture_loop(si, runs[i].loop_args());
            if (e == cudaSuccess) e = cudaEventRecord(join[i], si);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, join[i], 0);
        }
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (e == cudaSuccess) e = e2;
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e == cudaSuccess) {
            cache.emplace(std::make_pair(~0ull, 0), exec);
            e = cudaGraphLaunch(exec, s);
        }
        if (e != cudaSuccess) st = fail(HISQ_ECUDA, "batched device loop failed: %s", cudaGetErrorString(e));
        for (int i = 0; i < nprob && st == HISQ_OK; ++i)
            if (!runs[i].stop) st = runs[i].after_device_loop(s);
    }
    while (st == HISQ_OK) {
        unsigned long long mask = 0;
        int chunk = 1 << 30;
        for (int i = 0; i < nprob; ++i)
            if (!runs[i].stop) {
                mask |= 1ull << i;
                chunk = std::min(chunk, runs[i].next_chunk());
            }
        if (mask == 0) break;
        if (graphs) {
            auto key = std::make_pair(mask, chunk);
            auto it = cache.find(key);
            if (it == cache.end()) {
                cudaGraph_t graph = nullptr;
                e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) e = cudaEventRecord(fork, cap);
                for (int i = 0; i < nprob && e == cudaSuccess; ++i) {
                    if (!(mask >> i & 1)) continue;
                    cudaStream_t si = runs[i].w->cap_stream;
                    e = cudaStreamWaitEvent(si, fork, 0);
                    for (int c = 0; c < chunk && e == cudaSuccess; ++c) e = runs[i].sv.iterate(si);
                    if (e == cudaSuccess) e = cudaEventRecord(join[i], si);
                    if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, join[i], 0);
                }
                cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
                if (e == cudaSuccess) e = e2;
                cudaGraphExec_t exec = nullptr;
                if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
                if (graph) cudaGraphDestroy(graph);
                if (e != cudaSuccess) {
                    st = fail(HISQ_ECUDA, "batched graph capture failed: %s", cudaGetErrorString(e));
                    break;
                }
                it = cache.emplace(key, exec).first;
            }
            e = cudaGraphLaunch(it->second, s);
        } else {
            for (int i = 0; i < nprob && e == cudaSuccess; ++i)
                if (mask >> i & 1)
                    for (int c = 0; c < chunk && e == cudaSuccess; ++c) e = runs[i].sv.iterate(s);
        }
        if (e != cudaSuccess) {
            st = fail(HISQ_ECUDA, "batched iteration launch failed: %s", cudaGetErrorString(e));
            break;
        }
        for (int i = 0; i < nprob && st == HISQ_OK; ++i)
            if (mask >> i & 1) st = runs[i].after_chunk(chunk, s);
    }
    cleanup();
    if (st != HISQ_OK) return st;
    hisq_status result = HISQ_OK;
    for (int i = 0; i < nprob; ++i) {
        hisq_status r = runs[i].finish(stats ? &stats[i] : nullptr, s);
        if (result == HISQ_OK && r != HISQ_OK) result = r;
    }
    return result;
}
