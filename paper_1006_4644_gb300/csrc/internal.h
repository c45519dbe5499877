// Host-side declarations shared by the library's translation units: the
// device-side parameter blocks and the kernel launchers each .cu exports.
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "cui.h"
#include "common.cuh"

namespace cui {

constexpr double kPi = 3.141592653589793238462643383279502884;

// Message returned by cui_last_error() on this thread.
void set_last_error(const char *msg);

// Kernel launches issued by this library (read by the tracing calls).
extern std::atomic<long long> g_launches;
inline void launched(int n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }
constexpr int kNB = 9; // phase basis functions of the anchor expansion

// Segment-level scalars written on the device by cui_segment_upload.
struct SegScales {
    double max_w;   // max |d~ k^(-7/6) / S| over the band
    double max_d;   // max |d~ / S| over the band
    double scale_w; // power of two applied to the fused path's weighted data
    double scale_d; // power of two applied to the plain path's weighted data
};

// Taylor-coefficient factors of the anchor expansion (filled at bank creation).
struct DerivConsts {
    float B[4][kNB]; // B[n][i] = binom(p_i, n) for the power-law basis functions
    float gam[4];    // cross terms of k^(1/3) ln k
    float lam[4];    // ln k terms, (-1)^(n+1) / n
};

// ------------------------------------------------------------- segment.cu --
// Two-level twiddle tables of a length-2^log2n transform:
// exp(2 pi i m / 2^log2n) = hi[m >> shift] * lo[m & (2^shift - 1)].
struct Twiddles {
    double2 *lo64, *hi64;
    float2 *lo32, *hi32;
    int shift, log2n;
    dfc *lodf = nullptr, *hidf = nullptr; // the same in double-float, when allocated
};
void launch_twiddle_tables(const Twiddles &t, cudaStream_t s);
void launch_fft_passes_f64(double2 *a, double2 *b, int log2n, int sign, const Twiddles &tw, cudaStream_t s,
                           double2 **result);
// batch transforms of length 2^log2n stored back to back (grid rows)
void launch_fft_passes_f32(float2 *a, float2 *b, int log2n, int sign, const Twiddles &tw, cudaStream_t s,
                           float2 **result, int batch = 1);
// d~ = DFT(d) (sign -1) of a real series in double-float arithmetic, returned
// as FP64 complex bins 0 .. N/2 in one of the two N-element buffers (a or b)
void launch_segment_transform_df(const double *d, double2 *a, double2 *b, int log2n, const Twiddles &tw,
                                 cudaStream_t s, double2 **result);
void launch_amp_table(double *amp, int64_t nhalf, cudaStream_t s);
// lowest k in [k_lo, k_hi) with psd[k] not finite and > 0 into *bad (atomicMin; preset to ~0)
void launch_psd_check(const double *psd, int64_t k_lo, int64_t k_hi, unsigned long long *bad, cudaStream_t s);
// the segment restricted to bins [ka, kb) below m/2, m = 2^log2m <= n samples
// at the rate fs n / m; X the segment's bins 0 .. n/2, a and b m elements each
void launch_band_series(const double2 *X, int64_t n, int log2m, int64_t ka, int64_t kb, const Twiddles &tw,
                        dfc *a, dfc *b, double *out, cudaStream_t s);
// wbar, dS (plain path), the segment scales and the prefix sums P of the
// upload in two passes over the spectrum (work: one double per 2048 bins)
void launch_segment_weights(const double2 *X, const double *psd, const double *amp, int64_t n, int k_low, double fs,
                            SegScales *scales, float2 *wbar, void *dS, bool dS_fp64, double *prefix, double *work,
                            cudaStream_t s);
void launch_prefix(const double *psd, const double *amp, int64_t n, int k_low, double *prefix, double *work,
                   cudaStream_t s);
// sigma^2 and the fused normaliser of every template over [klo, khi[t])
void launch_template_norm(const double *prefix, const int32_t *khi, int klo, int64_t nt, double fs, int64_t n,
                          const SegScales *scales, double *sigma2, float *invnorm, cudaStream_t s);
void launch_basis_table(double *g, float2 *g_df, int n1, int n2, int ccols, cudaStream_t s);
void launch_exact_table(float2 *g, int kx, cudaStream_t s);

// --------------------------------------------------------------- fused.cu --
struct FusedArgs {
    const float2 *wbar;     // [N/2] weighted data with k^(-7/6) folded in
    const double *coef;     // [T][9] phase coefficients (cycles), FP64
    const float2 *coef_df;  // [T][9] the same as double-float pairs
    const double *basis;    // [A][9] anchor basis values, FP64
    const float2 *basis_df; // [A][9] the same as double-float pairs
    const int32_t *khi;     // [T] exclusive upper bin
    const int32_t *kex;     // [T] bins below this use the exact per-bin phase
    const float2 *gexact;   // [KX][9] basis values at every bin k < KX, double-float
    const float *invnorm;   // [T] 4 df / (scale^2 P[khi])
    const int32_t *order;   // device template order of this call
    int64_t base;           // first position of this batch in `order`
    void *ywork;            // [B][N] spectrum between the two passes
    Slot *peak;             // [T] peak slots
    Slot *prec;             // [B][nrec] per-row-pair peak records of the streamed pass 2 (else unused)
    int nrec;               // records per template (fused_records_per_template)
    Slot *win;              // [B][nwin] window slots
    int *err;               // device error word
    int cas_rounds;         // bound of the compare-and-swap loops (kCasRounds)
    unsigned long long copy_wait_ns; // bound of a streamed pass-2 wait for its row pair
    int64_t n;
    int log2n, n1, n2, ccols, rpc;
    int k_low;
    int64_t lo, hi, window;
    int nwin;
    float thr2;
    bool fp64; // anchor phases in FP64 instead of double-float
    bool bf16;
};
void fused_set_consts(const DerivConsts &dc, cudaStream_t s);
bool fused_supported(int log2n);
bool fused_tiling_ok(int log2n, int n1, int ccols, int rpc);
void fused_default_tiling(int log2n, int *n1, int *ccols, int *rpc);
size_t fused_pass1_smem(int n1, int ccols);
size_t fused_pass2_smem(int n2, int rpc);
// peak records per template of the streamed pass 2 (rpc 0): its row pairs, or its rows when unpaired
int fused_records_per_template(int n1, int n2);
cudaError_t launch_pass1(const FusedArgs &a, int count, cudaStream_t s);
cudaError_t launch_pass2(const FusedArgs &a, int count, cudaStream_t s);
constexpr int kChisqMaxBands = 64;
// chi^2 (and rho) of n triggers (tmpl, sample) with `bands` sub-bands
cudaError_t launch_chisq(const FusedArgs &a, const double *prefix, const int2 *trig, int n, int bands, float *chisq,
                         float *rho, cudaStream_t s);
cudaError_t launch_template_out(const FusedArgs &a, int t, const double *amp, double dfac, float2 *out,
                                cudaStream_t s);
// band correlator of n queries (tmpl[i], time u[i] as a 64-bit fraction of the
// segment) over [ka, min(kb, khi0[t])): out[3 i ..] = (Re z, Im z, sigma_B^2)
cudaError_t launch_band(const FusedArgs &a, const double *prefix, const int32_t *khi0, const int32_t *tmpl,
                        const uint64_t *u, int n, int ka, int kb, const SegScales *sc, double zfac, double sfac,
                        double *out, cudaStream_t s);

struct FinalizeArgs {
    const int32_t *order;    // device template order
    int64_t base;            // first position in `order`
    int count;               // templates in this batch
    Slot *peak;              // [T]
    const Slot *prec;        // [count][nrec] peak records (streamed pass 2), or NULL: the peak slots hold the peaks
    int nrec;
    Slot *win;               // [count][nwin]
    int nwin;
    int64_t lo, window;
    cui_peak *peaks_out;     // [T]
    cui_trigger *trig;       // [cap]
    int64_t trig_cap;
    unsigned long long *trig_count;
    Slot *cluster;           // [nwin] loudest trigger of each window over the bank
    int *err;
    int cas_rounds;          // bound of the compare-and-swap loops
};
cudaError_t launch_finalize(const FinalizeArgs &a, cudaStream_t s);

// ---------------------------------------------------------------- plain.cu --
struct PlainArgs {
    const double *mass;      // [T][2]: total mass (s), symmetric mass ratio
    const int32_t *khi;      // [T]
    const double *amp;       // [N/2] k^(-7/6)
    const double *psd;       // [N/2+1]
    const void *dS;          // [N/2] scaled d~/S (float2 or double2)
    const SegScales *scales;
    Twiddles tw;             // FFT twiddle tables
    void *h, *qa, *qb;       // work buffers, N complex each (h: N/2)
    double *acc;             // sigma sum, one double
    Slot *peak, *win;
    int *err;
    int cas_rounds; // bound of the compare-and-swap loops
    int64_t n;
    int log2n, pn_x2, k_low;
    double fs;
    int64_t lo, hi, window;
    int nwin;
    float thr2;
    bool fp64;
};
cudaError_t launch_plain_template(const PlainArgs &a, int t, cudaStream_t s);

// ------------------------------------------------------------------ api.cu --
// The uploaded segment's unnormalised FP64 transform X_k (k < N), its PSD,
// N and the sample rate; false if no segment has been uploaded.
bool bank_segment_spectrum(cui_bank b, const double2 **X, const double **psd, int64_t *n, double *fs);

} // namespace cui
