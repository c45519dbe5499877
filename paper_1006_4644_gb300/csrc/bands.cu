// Template band edges (one rule for the whole library) and the coherent
// two-band combination of the multi-band search.
#include <algorithm>
#include <cmath>

#include "bands.h"
#include "internal.h"

namespace cui {

constexpr double kMsunSec = 4.925490947e-6; // G M_sun / c^3 (s)

int band_k_low(double f_low, double df, int64_t nh)
{
    return std::max<int>(1, (int)std::min<double>(std::ceil(f_low / df), (double)nh));
}

int32_t band_k_hi(double m1, double m2, double df, int64_t nh)
{
    const double M = (m1 + m2) * kMsunSec;
    const double f_isco = 1.0 / (std::pow(6.0, 1.5) * kPi * M);
    return (int32_t)std::min<double>(std::ceil(f_isco / df), (double)nh);
}

// One thread per candidate: the two bands' correlators add coherently.
__global__ void k_band_combine(const double *__restrict__ zh, const double *__restrict__ zl, int n,
                               double *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double re = zh[3 * i] + zl[3 * i], im = zh[3 * i + 1] + zl[3 * i + 1];
    const double s2 = zh[3 * i + 2] + zl[3 * i + 2];
    out[2 * i] = s2 > 0.0 ? sqrt(re * re + im * im) / sqrt(s2) : 0.0;
    out[2 * i + 1] = atan2(im, re);
}

cudaError_t launch_band_combine(const double *zh, const double *zl, int n, double *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_band_combine<<<(n + 127) / 128, 128, 0, s>>>(zh, zl, n, out);
    launched();
    return cudaGetLastError();
}

} // namespace cui

using namespace cui;

extern "C" cui_status cui_template_bands(const double *m1, const double *m2, int64_t n_templates, int64_t n,
                                         double sample_rate, double f_low, int32_t *k_low_out, int32_t *k_hi_out)
{
    if (!m1 || !m2 || (n_templates > 0 && !k_hi_out) || n_templates < 0) {
        set_last_error("m1, m2 and k_hi_out must be non-NULL and n_templates >= 0");
        return CUI_ERR_ARG;
    }
    if (n < 2 || (n & (n - 1))) {
        set_last_error("n must be a power of two >= 2");
        return CUI_ERR_ARG;
    }
    if (!(sample_rate > 0) || !std::isfinite(sample_rate) || !(f_low > 0) || !std::isfinite(f_low)) {
        set_last_error("sample_rate and f_low must be finite and > 0");
        return CUI_ERR_ARG;
    }
    const double df = sample_rate / (double)n;
    for (int64_t t = 0; t < n_templates; ++t) {
        if (!(m1[t] > 0) || !(m2[t] > 0) || !std::isfinite(m1[t]) || !std::isfinite(m2[t])) {
            set_last_error("masses must be finite and > 0");
            return CUI_ERR_ARG;
        }
        k_hi_out[t] = band_k_hi(m1[t], m2[t], df, n / 2);
    }
    if (k_low_out) *k_low_out = band_k_low(f_low, df, n / 2);
    return CUI_OK;
}
