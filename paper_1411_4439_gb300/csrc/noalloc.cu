// hisq_cdot_noalloc: the per-rhs FP64 dot product of hisq_cdot for callers
// that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: processes whose device memory is
// entirely owned by another allocator (a framework's caching pool), where an
// extra allocation fails or fragments the pool, and latency-critical code for
// which the implicit device synchronisation of cudaMalloc is not acceptable.
// For them this entry point keeps its reduction scratch (block partial sums,
// the arrival counter of the last-block finish and the reduced values) in a
// fixed file-scope device array instead of memory allocated at run time. The
// array is sized for the largest bundle the library accepts (16 rhs) and is
// held by every GPU that loads the library until the process exits.
#include <cstring>
#include <mutex>

#include "hisq_internal.cuh"

namespace {

struct StaticDotScratch {
    double partials[hisq::kMaxRedVals * hisq::kMaxRedBlocks];   // 1 MiB
    unsigned int counter;
    unsigned int pad[63];
    double out[hisq::kMaxRedVals];
};

static __device__ __align__(256) StaticDotScratch g_dot_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
StaticDotScratch* g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device, looked up once per
// device (the name g_dot_scratch is only a host-side stand-in in host code).
cudaError_t scratch_address(StaticDotScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (g_addr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_dot_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<StaticDotScratch*>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

hisq_status reject(hisq_status code, const char* msg) {
    hisq::record_error(msg);
    return code;
}

}  // namespace

extern "C" hisq_status hisq_cdot_noalloc(const void* const a[], const void* const b[], int n,
                                         long long len, double* out, void* stream) {
    using namespace hisq;
    if (n < 1 || n > kMaxRhs)
        return reject(HISQ_EINVAL, "hisq_cdot_noalloc: n must be 1..16, the bundle size its static scratch holds");
    if (len < 1) return reject(HISQ_EINVAL, "hisq_cdot_noalloc: len must be >= 1");
    if (!a || !b || !out) return reject(HISQ_EINVAL, "hisq_cdot_noalloc: NULL pointer");
    ForcePtrs fp;
    memset(&fp, 0, sizeof(fp));
    for (int k = 0; k < n; ++k) {
        if (!a[k] || !b[k]) return reject(HISQ_EINVAL, "hisq_cdot_noalloc: NULL vector pointer");
        if ((reinterpret_cast<uintptr_t>(a[k]) | reinterpret_cast<uintptr_t>(b[k])) & 15)
            return reject(HISQ_EINVAL, "hisq_cdot_noalloc: vectors must be 16-byte aligned");
        fp.a[k] = static_cast<const double2*>(a[k]);
        fp.b[k] = static_cast<const double2*>(b[k]);
    }
    StaticDotScratch* scr = nullptr;
    cudaError_t e = scratch_address(&scr);
    if (e != cudaSuccess) return reject(HISQ_ECUDA, "hisq_cdot_noalloc: cudaGetSymbolAddress failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the arrival counter must start at zero; the last block leaves it zero,
    // but a call interrupted by an earlier error may not have
    e = cudaMemsetAsync(&scr->counter, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) e = launch_cdot(fp, len, n, RedScratch{scr->partials, &scr->counter}, scr->out, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, scr->out, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return reject(HISQ_ECUDA, cudaGetErrorString(e));
    return HISQ_OK;
}
