// Allocation-free template normalisation (cui_template_sigma_noalloc).
//
// Some callers cannot allocate device memory at the moment they need a
// result: pipelines whose device memory is all owned by one pool allocator
// with a fixed budget, or real-time loops that must not take the time (and
// the implicit synchronisation) a cudaMalloc can take.  Such a caller may
// still need to renormalise a bank when its noise estimate changes.  This
// entry point computes every template's sigma^2 for a given PSD with the same
// kernels cui_segment_upload uses (amplitude table, prefix sums, per-template
// lookup), but all of their scratch lives in one fixed-size array compiled
// into the library, so the call itself allocates nothing.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "bands.h"
#include "internal.h"

namespace cui {
namespace {

constexpr int64_t kNoallocMaxN = int64_t(1) << 20;     // largest segment length
constexpr int64_t kNoallocMaxTemplates = int64_t(1) << 14;
constexpr int64_t kNoallocScanBlocks = (kNoallocMaxN / 2 + 1) / 2048 + 2;

struct NoallocScratch {
    double amp[kNoallocMaxN / 2];        // k^(-7/6)
    double prefix[kNoallocMaxN / 2 + 1]; // prefix sums of amp^2 / S
    double bsum[kNoallocScanBlocks];     // per-block sums of the scan
    int32_t khi[kNoallocMaxTemplates];   // exclusive upper bin of every template
    float invnorm[kNoallocMaxTemplates]; // written by the lookup kernel, unused here
    SegScales scales;                    // scale_w must read 1
};

// ~8.2 MiB on every GPU that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
NoallocScratch *g_noalloc_ptr[kMaxDevices] = {};

} // namespace
} // namespace cui

using namespace cui;

// The lookup kernel scales by scales->scale_w, which must read exactly 1 here
// (the array keeps the previous call's contents, so it is set on every call).
__global__ void k_noalloc_unit_scales(SegScales *scales) { *scales = SegScales{0.0, 0.0, 1.0, 1.0}; }

static cui_status noalloc_fail(cui_status st, const char *msg)
{
    set_last_error(msg); // reported by cui_last_error()
    return st;
}

extern "C" cui_status cui_template_sigma_noalloc(const double *psd_dev, int64_t n, double sample_rate, double f_low,
                                                 const double *m1, const double *m2, int64_t count,
                                                 double *sigma2_dev, void *stream)
{
    char msg[200];
    if (!psd_dev || !m1 || !m2 || !sigma2_dev) return noalloc_fail(CUI_ERR_ARG, "pointers must be non-NULL");
    if (n < 64 || (n & (n - 1))) return noalloc_fail(CUI_ERR_ARG, "n must be a power of two >= 64");
    if (n > kNoallocMaxN) {
        std::snprintf(msg, sizeof msg, "n = %lld exceeds the allocation-free maximum of %lld samples", (long long)n,
                      (long long)kNoallocMaxN);
        return noalloc_fail(CUI_ERR_ARG, msg);
    }
    if (count < 1 || count > kNoallocMaxTemplates) {
        std::snprintf(msg, sizeof msg, "count = %lld must be in [1, %lld] (the allocation-free maximum)",
                      (long long)count, (long long)kNoallocMaxTemplates);
        return noalloc_fail(CUI_ERR_ARG, msg);
    }
    if (!(sample_rate > 0) || !(f_low > 0) || !std::isfinite(sample_rate) || !std::isfinite(f_low))
        return noalloc_fail(CUI_ERR_ARG, "sample_rate and f_low must be finite and > 0");
    for (int64_t t = 0; t < count; ++t)
        if (!(m1[t] > 0) || !(m2[t] > 0) || !std::isfinite(m1[t]) || !std::isfinite(m2[t]))
            return noalloc_fail(CUI_ERR_ARG, "masses must be finite and > 0");

    // Device address of the scratch array on the current device.  The host
    // symbol is only a stand-in: its device address is looked up once per
    // device, with that device current (the first call on a device).
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(CUI_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(CUI_ERR_CUDA, "device index out of range");
    NoallocScratch *sc = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) {
                std::snprintf(msg, sizeof msg, "cudaGetSymbolAddress of the scratch array failed: %s",
                              cudaGetErrorString(e));
                return noalloc_fail(CUI_ERR_CUDA, msg);
            }
            g_noalloc_ptr[dev] = (NoallocScratch *)ptr;
        }
        sc = g_noalloc_ptr[dev];
    }

    const cudaStream_t s = (cudaStream_t)stream;
    const double df = sample_rate / (double)n;
    const int64_t nh = n / 2;
    const int k_low = band_k_low(f_low, df, nh); // clamped: f_low at or above Nyquist leaves every band empty
    // upper bins, copied from a stack buffer in chunks (a pageable source is
    // staged before cudaMemcpyAsync returns, so the buffer can be reused)
    int32_t chunk[512];
    for (int64_t t0 = 0; t0 < count; t0 += 512) {
        const int64_t m = std::min<int64_t>(512, count - t0);
        for (int64_t i = 0; i < m; ++i) chunk[i] = band_k_hi(m1[t0 + i], m2[t0 + i], df, nh);
        e = cudaMemcpyAsync(sc->khi + t0, chunk, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return noalloc_fail(CUI_ERR_CUDA, cudaGetErrorString(e));
    }
    k_noalloc_unit_scales<<<1, 1, 0, s>>>(&sc->scales);
    launched();
    launch_amp_table(sc->amp, nh, s);
    launch_prefix(psd_dev, sc->amp, n, k_low, sc->prefix, sc->bsum, s);
    launch_template_norm(sc->prefix, sc->khi, k_low, count, sample_rate, n, &sc->scales, sigma2_dev, sc->invnorm,
                         s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(CUI_ERR_CUDA, cudaGetErrorString(e));
    return CUI_OK;
}
