// Segment preparation: the FP64 data spectrum d~ (eq:matchedfilter's X(f)),
// the noise-weighted data the filters read, per-template sigma^2 from prefix
// sums, and the template-independent tables (amplitude law, anchor basis).
// Also the generic multi-pass Stockham FFT over global memory that the
// segment transform and the per-template plain path use.
#include <cfloat>
#include <cstdio>

#include "internal.h"

namespace cui {

// ------------------------------------------------ Stockham global passes ---
// exp(SIGN 2 pi i m / 2^log2n) = hi[m >> shift] * lo[m & (2^shift - 1)]: two
// small tables, built once per bank (k_twiddle_tables), replace a
// transcendental call per twiddle.
template <typename Rl> struct TwTab {
    const cpx_t<Rl> *lo, *hi;
    int shift, log2n;
};

template <typename Rl, int SIGN> __device__ __forceinline__ cpx_t<Rl> tab_turn(const TwTab<Rl> &t, int64_t m)
{
    const cpx_t<Rl> a = t.hi[m >> t.shift], b = t.lo[m & ((int64_t(1) << t.shift) - 1)];
    const cpx_t<Rl> w = cmul(a, b);
    return SIGN > 0 ? w : mk(w.x, -w.y);
}

// One radix-R Stockham stage over a length-L transform whose sub-transforms
// of size Ns are done: task j reads in[j + r L/R], applies the twiddles
// exp(SIGN 2 pi i (j mod Ns) r / (Ns R)), an R-point DFT, and writes
// out[(j / Ns) Ns R + j mod Ns + r Ns].
template <typename Rl, int R, int SIGN>
__global__ void __launch_bounds__(256) k_stockham(const cpx_t<Rl> *__restrict__ in, cpx_t<Rl> *__restrict__ out,
                                                  int64_t L, int64_t Ns, int lshift, const TwTab<Rl> tw)
{
    using C = cpx_t<Rl>;
    const int64_t q = L / R;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= q) return;
    in += (int64_t)blockIdx.y * L; // one transform per grid row
    out += (int64_t)blockIdx.y * L;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[j + r * q];
    const int64_t jm = j & (Ns - 1);
    if (Ns > 1) {
        // (jm r) / (Ns R) in units of the table's 2^log2n
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tab_turn<Rl, SIGN>(tw, (jm * r) << lshift));
    }
    dft<R, SIGN>(v);
    const int64_t idx = (j / Ns) * Ns * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) out[idx + r * Ns] = v[r];
}

template <typename Rl, int SIGN>
static void stage(const cpx_t<Rl> *in, cpx_t<Rl> *out, int64_t L, int64_t Ns, int R, const TwTab<Rl> &tw,
                  cudaStream_t s, int batch)
{
    const int64_t q = L / R;
    const dim3 blocks((unsigned)((q + 255) / 256), (unsigned)batch);
    int lg = 0;
    while ((int64_t(1) << lg) < Ns * R) ++lg;
    const int lshift = tw.log2n - lg;
    switch (R) {
    case 2: k_stockham<Rl, 2, SIGN><<<blocks, 256, 0, s>>>(in, out, L, Ns, lshift, tw); break;
    case 4: k_stockham<Rl, 4, SIGN><<<blocks, 256, 0, s>>>(in, out, L, Ns, lshift, tw); break;
    case 8: k_stockham<Rl, 8, SIGN><<<blocks, 256, 0, s>>>(in, out, L, Ns, lshift, tw); break;
    default: k_stockham<Rl, 16, SIGN><<<blocks, 256, 0, s>>>(in, out, L, Ns, lshift, tw); break;
    }
    launched();
}

// Full transform of length 2^log2n: one small-radix stage (if log2n is not a
// multiple of 4) then radix-16 stages, ping-ponging between a and b.
template <typename Rl>
static void fft_passes(cpx_t<Rl> *a, cpx_t<Rl> *b, int log2n, int sign, const TwTab<Rl> &tw, cudaStream_t s,
                       cpx_t<Rl> **result, int batch = 1, int max_lr = 4)
{
    const int64_t L = int64_t(1) << log2n;
    int64_t Ns = 1;
    cpx_t<Rl> *src = a, *dst = b;
    int rem = log2n % max_lr;
    int left = log2n;
    while (left > 0) {
        int lr = rem ? rem : max_lr;
        rem = 0;
        int R = 1 << lr;
        if (sign > 0) stage<Rl, +1>(src, dst, L, Ns, R, tw, s, batch);
        else stage<Rl, -1>(src, dst, L, Ns, R, tw, s, batch);
        Ns *= R;
        left -= lr;
        cpx_t<Rl> *t = src;
        src = dst;
        dst = t;
    }
    *result = src;
}

void launch_fft_passes_f64(double2 *a, double2 *b, int log2n, int sign, const Twiddles &tw, cudaStream_t s,
                           double2 **result)
{
    fft_passes<double>(a, b, log2n, sign, TwTab<double>{tw.lo64, tw.hi64, tw.shift, tw.log2n}, s, result);
}
void launch_fft_passes_f32(float2 *a, float2 *b, int log2n, int sign, const Twiddles &tw, cudaStream_t s,
                           float2 **result, int batch)
{
    fft_passes<float>(a, b, log2n, sign, TwTab<float>{tw.lo32, tw.hi32, tw.shift, tw.log2n}, s, result, batch);
}

// Segment transform in double-float.  FP64 runs at a small fraction of the
// FP32 rate on this GPU, while a double-float value (hi + lo, 48 significant
// bits) costs a handful of FP32 operations, so the once-per-segment transform
// keeps near-FP64 accuracy at FP32 speed.  The input is scaled by 2^kDfShift
// (exact) so that strain of ~1e-21 and its spectrum sit far from the FP32
// range limits; the output is scaled back.
constexpr int kDfShift = 64;
// radix of the double-float passes: small radices give the long double-float
// dependency chains enough threads to hide their latency
constexpr int kDfLog2Radix = 4;

// x 2^kDfShift as hi + lo from the bits of x alone (integer and FP32 operations;
// FP64 arithmetic is the slow path on this GPU): hi carries the top 24
// significant bits (truncated), lo the remaining 29 rounded to 24.  Zero and
// subnormal inputs give zero.
__device__ __forceinline__ df split_double(double x)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((u >> 52) & 0x7FF);
    if (e == 0) return {0.f, 0.f};
    const unsigned sign = (unsigned)(u >> 63) << 31;
    const float hi1 = __uint_as_float(sign | (127u << 23) | (unsigned)((u >> 29) & 0x7FFFFF)); // +-1.m
    const float lo1 = __uint_as_float(__float_as_uint((float)(unsigned)(u & 0x1FFFFFFF)) | sign);
    return {ldexpf(hi1, e - 1023 + kDfShift), ldexpf(lo1, e - 1075 + kDfShift)};
}

// z_m = d_2m + i d_2m+1 (x 2^kDfShift), m < M = N/2: the real segment as M
// complex values, so that one M-point transform serves it
__global__ void k_real_pairs_to_dfc(const double *__restrict__ d, dfc *__restrict__ out, int64_t m)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        out[j] = dfc{split_double(d[2 * j]), split_double(d[2 * j + 1])};
}

// X_k, k = 0 .. M, from Z = DFT_M(z), in place (Z_k becomes X_k; slot M is
// written too).  With E and O the transforms of the even and odd samples,
// Z_k = E_k + i O_k and conj(Z_{M-k}) = E_k - i O_k, so E_k = (Z_k +
// conj(Z_{M-k}))/2, O_k = -i (Z_k - conj(Z_{M-k}))/2, X_k = E_k + W^k O_k and
// X_{M-k} = conj(E_k - W^k O_k), W = e^(-2 pi i / N).  Thread k does k and M-k.
__global__ void k_real_post(dfc *io, int64_t m, const TwTab<df> tw)
{
    const df half = {0.5f, 0.0f};
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= m / 2;
         k += (int64_t)gridDim.x * blockDim.x) {
        const dfc a = io[k];
        const dfc zc = io[k == 0 ? 0 : m - k];
        const dfc b = {zc.x, -zc.y}; // conj(Z_{M-k})
        const dfc e = {(a.x + b.x) * half, (a.y + b.y) * half};
        const dfc o = {(a.y - b.y) * half, (b.x - a.x) * half}; // -i (a - b) / 2
        const dfc t = cmul(o, tab_turn<df, -1>(tw, k));
        const dfc lo = e + t, hi = e - t;
        double2 *out = reinterpret_cast<double2 *>(io);
        out[k] = make_double2(ldexp((double)lo.x.hi + (double)lo.x.lo, -kDfShift),
                              ldexp((double)lo.y.hi + (double)lo.y.lo, -kDfShift));
        if (k != m - k)
            out[m - k] = make_double2(ldexp((double)hi.x.hi + (double)hi.x.lo, -kDfShift),
                                      -ldexp((double)hi.y.hi + (double)hi.y.lo, -kDfShift));
    }
}

// X_k = sum_j d_j e^(-2 pi i jk/N) for k = 0 .. N/2, as FP64, in a or b: an
// N/2-point double-float transform of the sample pairs, then the split above.
void launch_segment_transform_df(const double *d, double2 *a, double2 *b, int log2n, const Twiddles &tw,
                                 cudaStream_t s, double2 **result)
{
    const int64_t m = int64_t(1) << (log2n - 1);
    dfc *da = reinterpret_cast<dfc *>(a), *db = reinterpret_cast<dfc *>(b), *r = nullptr;
    const TwTab<df> tt{tw.lodf, tw.hidf, tw.shift, tw.log2n};
    k_real_pairs_to_dfc<<<1216, 256, 0, s>>>(d, da, m);
    launched();
    fft_passes<df>(da, db, log2n - 1, -1, tt, s, &r, 1, kDfLog2Radix);
    k_real_post<<<1216, 256, 0, s>>>(r, m, tt);
    launched();
    *result = reinterpret_cast<double2 *>(r);
}

// ------------------------------------------------- band-limited series ---
// Y_k' (k' < m = N / decim) = X_k' on the band, its Hermitian mirror above
// m / 2, zero elsewhere (and at m / 2), as double-float scaled by 2^kDfShift.
__global__ void k_band_spectrum(const double2 *__restrict__ X, dfc *__restrict__ Y, int64_t m, int64_t ka,
                                int64_t kb)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = j <= m / 2 ? j : m - j;
        dfc y = {df{0.f, 0.f}, df{0.f, 0.f}};
        if (k >= ka && k < kb && k < m / 2) {
            const double2 x = X[k];
            y = dfc{split_double(x.x), split_double(j <= m / 2 ? x.y : -x.y)};
        }
        Y[j] = y;
    }
}

// out_j = Re(Y_j) 2^-kDfShift / n, j < m
__global__ void k_dfc_real_out(const dfc *__restrict__ Y, double *__restrict__ out, int64_t m, double inv_n)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        out[j] = ldexp((double)Y[j].x.hi + (double)Y[j].x.lo, -kDfShift) * inv_n;
}

// x'_j = (1/N) sum over the band's bins k (and mirrors) of X_k e^(2 pi i k j / m),
// j < m = N / decim: the segment restricted to bins [ka, kb) below m / 2 at
// the sample rate fs / decim.  a and b hold m double-float values each.  The
// Stockham twiddles depend only on the sub-transform sizes, so the bank's
// tables (built for N) serve the shorter transform.
void launch_band_series(const double2 *X, int64_t n, int log2m, int64_t ka, int64_t kb, const Twiddles &tw,
                        dfc *a, dfc *b, double *out, cudaStream_t s)
{
    const int64_t m = int64_t(1) << log2m;
    k_band_spectrum<<<1216, 256, 0, s>>>(X, a, m, ka, kb);
    launched();
    dfc *r = nullptr;
    fft_passes<df>(a, b, log2m, +1, TwTab<df>{tw.lodf, tw.hidf, tw.shift, tw.log2n}, s, &r, 1, kDfLog2Radix);
    k_dfc_real_out<<<1216, 256, 0, s>>>(r, out, m, 1.0 / (double)n);
    launched();
}

// lo[i] = exp(2 pi i i / 2^log2n), hi[i] = exp(2 pi i (i << shift) / 2^log2n), in FP64 and FP32
__global__ void k_twiddle_tables(Twiddles t)
{
    const int nlo = 1 << t.shift, nhi = 1 << (t.log2n - t.shift);
    const double n = (double)(int64_t(1) << t.log2n);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nlo + nhi; i += gridDim.x * blockDim.x) {
        const int64_t m = i < nlo ? (int64_t)i : ((int64_t)(i - nlo) << t.shift);
        double s, c;
        sincospi(2.0 * (double)m / n, &s, &c);
        double2 *d = i < nlo ? t.lo64 + i : t.hi64 + (i - nlo);
        float2 *f = i < nlo ? t.lo32 + i : t.hi32 + (i - nlo);
        *d = make_double2(c, s);
        *f = make_float2((float)c, (float)s);
        if (t.lodf) {
            dfc *q = i < nlo ? t.lodf + i : t.hidf + (i - nlo);
            const float ch = __double2float_rn(c), sh = __double2float_rn(s);
            *q = dfc{df{ch, __double2float_rn(c - (double)ch)}, df{sh, __double2float_rn(s - (double)sh)}};
        }
    }
}

void launch_twiddle_tables(const Twiddles &t, cudaStream_t s)
{
    k_twiddle_tables<<<16, 256, 0, s>>>(t);
    launched();
}

// -------------------------------------------------------- segment inputs ---

// amp_k = k^(-7/6) for k >= 1 (the Newtonian amplitude law without its
// df^(-7/6) factor), amp_0 = 0.
__global__ void k_amp(double *amp, int64_t nh)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nh; k += (int64_t)gridDim.x * blockDim.x)
        amp[k] = k == 0 ? 0.0 : pow((double)k, -7.0 / 6.0);
}
void launch_amp_table(double *amp, int64_t nh, cudaStream_t s)
{
    k_amp<<<1216, 256, 0, s>>>(amp, nh);
    launched();
}

// The lowest k in [k_lo, k_hi) whose psd[k] is not finite and > 0, into
// *bad (preset to all ones by the caller), by atomicMin.
__global__ void k_psd_check(const double *__restrict__ psd, int64_t k_lo, int64_t k_hi, unsigned long long *bad)
{
    for (int64_t k = k_lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < k_hi;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double v = psd[k];
        if (!(v > 0.0 && v <= DBL_MAX)) atomicMin(bad, (unsigned long long)k);
    }
}
void launch_psd_check(const double *psd, int64_t k_lo, int64_t k_hi, unsigned long long *bad, cudaStream_t s)
{
    k_psd_check<<<1216, 256, 0, s>>>(psd, k_lo, k_hi, bad);
    launched();
}

// Band maxima of |d~ amp / S| and |d~ / S|, to a power of two: only the
// scale below is taken from them, so integer operations on the exponent
// fields replace the FP64 arithmetic (the slow path on this GPU).  With e(v)
// the exponent of v, the estimate 2^(e(max(|Re X|, |Im X|)) - e(S) [+ e(amp)]
// + e(1/fs)) lies within a factor 2^-1 .. 2^3.5 of the true maximum.
// Non-negative doubles compare as unsigned integers, so atomicMax on their
// bits is a floating-point max.
__device__ __forceinline__ int exp_field(double v) { return (int)((__double_as_longlong(v) >> 52) & 0x7FF); }
constexpr int kNoExp = -(1 << 20);

// raise the exponent maxima (ew: weighted data, ed: plain data) by bin k of the band
__device__ __forceinline__ void exp_max_bin(const double2 *__restrict__ X, const double *__restrict__ psd,
                                            const double *__restrict__ amp, int64_t k, int &ew, int &ed)
{
    const double2 x = X[k];
    const long long bx = __double_as_longlong(x.x) & 0x7FFFFFFFFFFFFFFFll;
    const long long by = __double_as_longlong(x.y) & 0x7FFFFFFFFFFFFFFFll;
    const int ex = (int)((bx > by ? bx : by) >> 52); // 0 for zero (and subnormal) bins
    if (ex == 0) return;
    const int d = ex - exp_field(psd[k]);
    ed = max(ed, d);
    ew = max(ew, d + exp_field(amp[k]) - 1023);
}

// the block's exponent maxima, then one atomic pair per block on the two
// shared addresses
__device__ __forceinline__ void block_exp_max(int ew, int ed, int e_fs, SegScales *sc)
{
    __shared__ int s_ew[32], s_ed[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ew = max(ew, __shfl_xor_sync(0xffffffffu, ew, o));
        ed = max(ed, __shfl_xor_sync(0xffffffffu, ed, o));
    }
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_ew[wid] = ew;
        s_ed[wid] = ed;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            ew = max(ew, s_ew[w]);
            ed = max(ed, s_ed[w]);
        }
        if (ed != kNoExp) {
            const double mw = ldexp(1.0, ew + e_fs), md = ldexp(1.0, ed + e_fs);
            atomicMax((unsigned long long *)&sc->max_w, (unsigned long long)__double_as_longlong(mw));
            atomicMax((unsigned long long *)&sc->max_d, (unsigned long long)__double_as_longlong(md));
        }
    }
}

__device__ __forceinline__ double pow2_scale(double m)
{
    // a power of two that brings m into [1, 2); exact, so rho is unchanged
    return m > 0.0 ? ldexp(1.0, -ilogb(m)) : 1.0;
}

// wbar_k = scale_w d~_k amp_k / S_k and dS_k = scale_d d~_k / S_k on the band
// [k_low, N/2), zero below it.
__device__ __forceinline__ void weighted_bin(const double2 *__restrict__ X, const double *__restrict__ psd,
                                             const double *__restrict__ amp, int64_t k, int k_low, double inv_fs,
                                             double sw, double sd, float2 *__restrict__ wbar, void *dS,
                                             bool dS_fp64)
{
    double2 w = make_double2(0.0, 0.0);
    if (k >= k_low) {
        double f = inv_fs / psd[k];
        w = make_double2(X[k].x * f, X[k].y * f);
    }
    wbar[k] = make_float2((float)(w.x * amp[k] * sw), (float)(w.y * amp[k] * sw));
    if (dS) {
        if (dS_fp64) ((double2 *)dS)[k] = make_double2(w.x * sd, w.y * sd);
        else ((float2 *)dS)[k] = make_float2((float)(w.x * sd), (float)(w.y * sd));
    }
}

// ------------------------------------------------------------ prefix sums ---
// P[k] = sum_{k_low <= k' < k} amp_k'^2 / S_k', k = 0 .. N/2, in FP64.
constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanBlock = kScanThreads * kScanPer;

__device__ __forceinline__ double g_term(const double *psd, const double *amp, int64_t k, int64_t nh, int k_low)
{
    if (k < k_low || k >= nh) return 0.0;
    double a = amp[k];
    return a * a / psd[k];
}

__device__ __forceinline__ double block_exclusive_scan(double v, double *sh, double *total)
{
    // inclusive warp scan, then scan of warp totals
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        double y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        double w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            double y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;
    }
    __syncthreads();
    double warp_off = wid ? sh[wid - 1] : 0.0;
    *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_off + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(const double *psd, const double *amp, int64_t nh,
                                                            int k_low, double *bsum)
{
    __shared__ double sh[32];
    const int64_t k0 = (int64_t)blockIdx.x * kScanBlock + threadIdx.x * kScanPer;
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) s += g_term(psd, amp, k0 + i, nh, k_low);
    double tot;
    block_exclusive_scan(s, sh, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_offsets(double *bsum, int nb)
{
    __shared__ double sh[32];
    double carry = 0.0;
    for (int base = 0; base < nb; base += 1024) {
        int i = base + threadIdx.x;
        double v = i < nb ? bsum[i] : 0.0;
        double tot;
        double ex = block_exclusive_scan(v, sh, &tot);
        if (i < nb) bsum[i] = carry + ex;
        carry += tot;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_write(const double *psd, const double *amp, int64_t nh,
                                                             int k_low, const double *boff, double *prefix)
{
    __shared__ double sh[32];
    const int64_t k0 = (int64_t)blockIdx.x * kScanBlock + threadIdx.x * kScanPer;
    double g[kScanPer];
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        g[i] = g_term(psd, amp, k0 + i, nh, k_low);
        s += g[i];
    }
    double tot;
    double run = boff[blockIdx.x] + block_exclusive_scan(s, sh, &tot);
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        if (k0 + i <= nh) prefix[k0 + i] = run;
        run += g[i];
    }
}

void launch_prefix(const double *psd, const double *amp, int64_t n, int k_low, double *prefix, double *work,
                   cudaStream_t s)
{
    const int64_t nh = n / 2;
    // nh + 1 outputs (P[nh] is the total)
    const int nb = (int)((nh + 1 + kScanBlock - 1) / kScanBlock);
    k_scan_sums<<<nb, kScanThreads, 0, s>>>(psd, amp, nh, k_low, work);
    k_scan_offsets<<<1, 1024, 0, s>>>(work, nb);
    k_scan_write<<<nb, kScanThreads, 0, s>>>(psd, amp, nh, k_low, work, prefix);
    launched(3);
}

// The weighted data and the prefix sums in two passes over the spectrum, for
// the bank's upload.  Pass 1 (one block per kScanBlock bins, kScanPer
// consecutive bins per thread, as k_scan_sums) takes the block sums of P's
// terms and the exponent maxima; k_scan_offsets scans the block sums; pass 2
// (the same blocks) writes wbar and dS (coalesced: bin base + t + r blockDim)
// and the prefix sums (the per-thread grouping of pass 1, so the offsets
// match the sums bit for bit).
__global__ void __launch_bounds__(kScanThreads) k_seg_reduce(const double2 *__restrict__ X,
                                                             const double *__restrict__ psd,
                                                             const double *__restrict__ amp, int64_t nh, int k_low,
                                                             int e_fs, SegScales *sc, double *bsum)
{
    __shared__ double sh[32];
    const int64_t k0 = (int64_t)blockIdx.x * kScanBlock + threadIdx.x * kScanPer;
    double s = 0.0;
    int ew = kNoExp, ed = kNoExp;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        const int64_t k = k0 + i;
        s += g_term(psd, amp, k, nh, k_low);
        if (k >= k_low && k < nh) exp_max_bin(X, psd, amp, k, ew, ed);
    }
    double tot;
    block_exclusive_scan(s, sh, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
    block_exp_max(ew, ed, e_fs, sc);
}

__global__ void __launch_bounds__(kScanThreads) k_seg_write(const double2 *__restrict__ X,
                                                            const double *__restrict__ psd,
                                                            const double *__restrict__ amp, int64_t nh, int k_low,
                                                            double inv_fs, SegScales *sc, float2 *__restrict__ wbar,
                                                            void *dS, bool dS_fp64, const double *boff,
                                                            double *prefix)
{
    __shared__ double sh[32];
    const double sw = pow2_scale(sc->max_w), sd = pow2_scale(sc->max_d);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->scale_w = sw;
        sc->scale_d = sd;
    }
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        const int64_t k = base + threadIdx.x + i * kScanThreads;
        if (k < nh) weighted_bin(X, psd, amp, k, k_low, inv_fs, sw, sd, wbar, dS, dS_fp64);
    }
    const int64_t k0 = base + threadIdx.x * kScanPer;
    double g[kScanPer];
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        g[i] = g_term(psd, amp, k0 + i, nh, k_low);
        s += g[i];
    }
    double tot;
    double run = boff[blockIdx.x] + block_exclusive_scan(s, sh, &tot);
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        if (k0 + i <= nh) prefix[k0 + i] = run;
        run += g[i];
    }
}

void launch_segment_weights(const double2 *X, const double *psd, const double *amp, int64_t n, int k_low, double fs,
                            SegScales *scales, float2 *wbar, void *dS, bool dS_fp64, double *prefix, double *work,
                            cudaStream_t s)
{
    const int64_t nh = n / 2;
    const int nb = (int)((nh + 1 + kScanBlock - 1) / kScanBlock); // nh + 1 prefix values
    cudaMemsetAsync(scales, 0, sizeof(SegScales), s);
    k_seg_reduce<<<nb, kScanThreads, 0, s>>>(X, psd, amp, nh, k_low, ilogb(1.0 / fs), scales, work);
    k_scan_offsets<<<1, 1024, 0, s>>>(work, nb);
    k_seg_write<<<nb, kScanThreads, 0, s>>>(X, psd, amp, nh, k_low, 1.0 / fs, scales, wbar, dS, dS_fp64, work, prefix);
    launched(3);
}

// sigma^2_t = 4 df df^(-7/3) (P[k_hi(t)] - P[klo]) (the amplitude law's
// df^(-7/6) factor squared) and the fused path's normaliser
// 4 df / (scale_w^2 (P[k_hi] - P[klo])); klo >= the segment's k_low.
__global__ void k_tnorm(const double *prefix, const int32_t *khi, int klo, int64_t nt, int64_t nh, double df,
                        double dfp, const SegScales *sc, double *sigma2, float *invnorm)
{
    const double sw = sc->scale_w;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t kh = khi[t];
        kh = kh < 0 ? 0 : (kh > nh ? nh : kh);
        double P = kh > klo ? prefix[kh] - prefix[klo] : 0.0;
        sigma2[t] = 4.0 * df * dfp * P;
        invnorm[t] = P > 0.0 ? (float)(4.0 * df / (sw * sw * P)) : 0.0f;
    }
}

void launch_template_norm(const double *prefix, const int32_t *khi, int klo, int64_t nt, double fs, int64_t n,
                          const SegScales *scales, double *sigma2, float *invnorm, cudaStream_t s)
{
    const double df = fs / (double)n;
    const double dfp = pow(df, -7.0 / 3.0);
    const int blocks = (int)((nt + 255) / 256);
    k_tnorm<<<blocks < 1216 ? blocks : 1216, 256, 0, s>>>(prefix, khi, klo, nt, n / 2, df, dfp, scales, sigma2, invnorm);
    launched();
}

// ------------------------------------------------------ anchor basis table --
// Anchor (a, cb) sits at bin k_a = n2 a + cb C + C/2 for rows a < n1/2 and
// column blocks cb < n2/C.  The phase of every template is a fixed linear
// combination of nine template-independent functions of k (see bank
// creation), tabulated here at every anchor:
//   k^-5/3, k^-1, k^-2/3, k^-1/3, 1, ln k, k^1/3, k^1/3 ln k, k^2/3.
__device__ __forceinline__ void basis_values(double k, double *v)
{
    const double q = cbrt(k), lk = log(k);
    v[0] = 1.0 / (k * q * q);
    v[1] = 1.0 / k;
    v[2] = 1.0 / (q * q);
    v[3] = 1.0 / q;
    v[4] = 1.0;
    v[5] = lk;
    v[6] = q;
    v[7] = q * lk;
    v[8] = q * q;
}

// The same nine functions at every bin k < kx (k = 0 is never read).
__global__ void k_exact_table(float2 *g, int kx)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kx; k += gridDim.x * blockDim.x) {
        double v[kNB];
        basis_values(k > 0 ? (double)k : 1.0, v);
#pragma unroll
        for (int i = 0; i < kNB; ++i) {
            float hi = (float)v[i];
            g[(int64_t)k * kNB + i] = make_float2(hi, (float)(v[i] - (double)hi));
        }
    }
}

void launch_exact_table(float2 *g, int kx, cudaStream_t s)
{
    if (kx > 0) {
        k_exact_table<<<(kx + 255) / 256, 256, 0, s>>>(g, kx);
        launched();
    }
}

__global__ void k_basis(double *g, float2 *gdf, int n1, int n2, int ccols)
{
    const int nb = n2 / ccols;
    const int na = (n1 / 2) * nb;
    for (int ai = blockIdx.x * blockDim.x + threadIdx.x; ai < na; ai += gridDim.x * blockDim.x) {
        const int a = ai / nb, cb = ai % nb;
        const double k = (double)n2 * a + (double)cb * ccols + ccols / 2;
        double v[kNB];
        basis_values(k, v);
#pragma unroll
        for (int i = 0; i < kNB; ++i) {
            g[(int64_t)ai * kNB + i] = v[i];
            float hi = (float)v[i];
            gdf[(int64_t)ai * kNB + i] = make_float2(hi, (float)(v[i] - (double)hi));
        }
    }
}

void launch_basis_table(double *g, float2 *g_df, int n1, int n2, int ccols, cudaStream_t s)
{
    const int na = (n1 / 2) * (n2 / ccols);
    const int blocks = (na + 255) / 256;
    k_basis<<<blocks, 256, 0, s>>>(g, g_df, n1, n2, ccols);
    launched();
}

} // namespace cui
