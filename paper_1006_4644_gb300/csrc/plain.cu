// Plain per-template path: the paper's pipeline structure, one kernel per
// step (Sec. "Pipeline main details": device_template_proc, its normalisation
// reduction, device_complex_mf, the inverse transform, then the detection
// that device_madd2 / device_maxfind perform).  For each template:
//   1. generate h~_k with the TaylorF2 phase evaluated per bin in FP64,
//   2. sigma^2 by a reduction of |h~|^2 / S over the band,
//   3. q_k = (d~_k / S_k) conj(h~_k),
//   4. inverse FFT of q by radix-16 Stockham passes through global memory,
//   5. rho^2 = |z|^2 / sigma^2 reduced to the peak and window maxima.
// Precision: FP32 storage, products and FFT (phase still in FP64 per bin), or
// FP64 throughout.  It is the per-template baseline the fused path is
// measured against, and a second GPU implementation to cross-check it.
#include "internal.h"

namespace cui {

// TaylorF2 phase Psi(f) (t_c = 0, phi_c = 0), PN terms alpha_i with i <= pn_x2.
__device__ double taylorf2_phase(double M, double eta, int pn_x2, double f)
{
    const double pi = kPi;
    const double v = cbrt(pi * M * f);
    const double v2 = v * v, v5 = v2 * v2 * v;
    const double eta2 = eta * eta;
    double sum = 1.0;
    double vp = v2;
    if (pn_x2 >= 2) sum += (3715.0 / 756.0 + 55.0 / 9.0 * eta) * vp;
    vp *= v;
    if (pn_x2 >= 3) sum += -16.0 * pi * vp;
    vp *= v;
    if (pn_x2 >= 4) sum += (15293365.0 / 508032.0 + 27145.0 / 504.0 * eta + 3085.0 / 72.0 * eta2) * vp;
    vp *= v;
    if (pn_x2 >= 5) sum += pi * (38645.0 / 756.0 - 65.0 / 9.0 * eta) * (1.0 + 3.0 * log(v * sqrt(6.0))) * vp;
    vp *= v;
    if (pn_x2 >= 6)
        sum += (11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * pi * pi - 6848.0 / 21.0 * 0.57721566490153286061 +
                eta * (-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * pi * pi) + 76055.0 / 1728.0 * eta2 -
                127825.0 / 1296.0 * eta2 * eta - 6848.0 / 21.0 * log(4.0 * v)) *
               vp;
    vp *= v;
    if (pn_x2 >= 7) sum += pi * (77096675.0 / 254016.0 + 378515.0 / 1512.0 * eta - 74045.0 / 756.0 * eta2) * vp;
    return -pi / 4.0 + 3.0 / (128.0 * eta * v5) * sum;
}

template <typename Rl> __global__ void k_plain_gen(const PlainArgs a, int t, cpx_t<Rl> *h)
{
    const int64_t nh = a.n / 2;
    const double M = a.mass[2 * t], eta = a.mass[2 * t + 1];
    const int khi = a.khi[t];
    const double df = a.fs / (double)a.n;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nh; k += (int64_t)gridDim.x * blockDim.x) {
        cpx_t<Rl> out = mk(Rl(0), Rl(0));
        if (k >= a.k_low && k < khi) {
            const double psi = taylorf2_phase(M, eta, a.pn_x2, (double)k * df);
            const double amp = a.amp[k];
            if constexpr (sizeof(Rl) == 8) {
                double s, c;
                sincos(psi, &s, &c);
                out = mk(Rl(amp * c), Rl(-amp * s));
            } else {
                const double red = psi - 2.0 * kPi * rint(psi / (2.0 * kPi));
                float s, c;
                sincosf((float)red, &s, &c);
                const float fa = (float)amp;
                out = mk(Rl(fa * c), Rl(-fa * s));
            }
        }
        h[k] = out;
    }
}

template <typename Rl> __global__ void k_plain_sigma(const PlainArgs a, int t, const cpx_t<Rl> *h)
{
    __shared__ double sh[32];
    const int khi = a.khi[t];
    double s = 0.0;
    for (int64_t k = a.k_low + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < khi;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double x = (double)h[k].x, y = (double)h[k].y;
        s += (x * x + y * y) / a.psd[k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) atomicAdd(a.acc, s);
    }
}

template <typename Rl> __global__ void k_plain_mul(const PlainArgs a, int t, const cpx_t<Rl> *h, cpx_t<Rl> *q)
{
    const int khi = a.khi[t];
    const cpx_t<Rl> *dS = (const cpx_t<Rl> *)a.dS;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.n; k += (int64_t)gridDim.x * blockDim.x)
        q[k] = (k >= a.k_low && k < khi) ? cmulc(dS[k], h[k]) : mk(Rl(0), Rl(0));
}

template <typename Rl> __global__ void k_plain_detect(const PlainArgs a, int t, const cpx_t<Rl> *z)
{
    __shared__ unsigned long long s_key[32];
    __shared__ float s_zr[32], s_zi[32];
    const double sd = a.scales->scale_d;
    const double acc = *a.acc;
    const double df = a.fs / (double)a.n;
    const Rl inv = acc > 0.0 ? Rl(4.0 * df / (sd * sd * acc)) : Rl(0);
    unsigned long long best = 0ull;
    float bzr = 0.f, bzi = 0.f;
    for (int64_t j = a.lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.hi;
         j += (int64_t)gridDim.x * blockDim.x) {
        const cpx_t<Rl> v = z[j];
        const Rl r2 = (v.x * v.x + v.y * v.y) * inv;
        const unsigned long long key = make_key((float)r2, (uint32_t)j);
        if (key > best) {
            best = key;
            bzr = (float)v.x;
            bzi = (float)v.y;
        }
        if ((float)r2 > a.thr2) {
            const int m = (int)((j - a.lo) / a.window);
            slot_max(a.win + m, key, (float)atan2((double)v.y, (double)v.x), a.err, a.cas_rounds);
        }
    }
    warp_max_key(best, bzr, bzi);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        s_key[wid] = best;
        s_zr[wid] = bzr;
        s_zi[wid] = bzi;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        best = lane < nw ? s_key[lane] : 0ull;
        bzr = lane < nw ? s_zr[lane] : 0.f;
        bzi = lane < nw ? s_zi[lane] : 0.f;
        warp_max_key(best, bzr, bzi);
        if (lane == 0 && best != 0ull) slot_max(a.peak + t, best, atan2f(bzi, bzr), a.err, a.cas_rounds);
    }
}

template <typename Rl> static cudaError_t plain_template(const PlainArgs &a, int t, cudaStream_t s)
{
    using C = cpx_t<Rl>;
    C *h = (C *)a.h, *qa = (C *)a.qa, *qb = (C *)a.qb;
    cudaMemsetAsync(a.acc, 0, sizeof(double), s);
    k_plain_gen<Rl><<<1216, 256, 0, s>>>(a, t, h);
    k_plain_sigma<Rl><<<608, 256, 0, s>>>(a, t, h);
    k_plain_mul<Rl><<<1216, 256, 0, s>>>(a, t, h, qa);
    C *z = nullptr;
    if constexpr (sizeof(Rl) == 8) launch_fft_passes_f64(qa, qb, a.log2n, +1, a.tw, s, &z);
    else launch_fft_passes_f32(qa, qb, a.log2n, +1, a.tw, s, &z);
    k_plain_detect<Rl><<<608, 256, 0, s>>>(a, t, z);
    launched(4);
    return cudaGetLastError();
}

cudaError_t launch_plain_template(const PlainArgs &a, int t, cudaStream_t s)
{
    return a.fp64 ? plain_template<double>(a, t, s) : plain_template<float>(a, t, s);
}

} // namespace cui
