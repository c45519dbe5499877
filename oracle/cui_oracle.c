/*
 * FP64 CPU oracle of the bank matched filter -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg load
 * this file's library.  It shares no code, header, table or constant with the
 * CUDA library and is written for a reader to check against the paper by eye:
 * no blocking, no fusion, no reordering beyond what each definition states.
 *
 * What it computes (paper: Sec. "Matched filtering", eq:matchedfilter and the
 * per-chunk loop that follows it):
 *   d~_k   = dt * sum_j d_j exp(-2 pi i j k / N)                (data spectrum)
 *   h~_k   = f_k^(-7/6) exp(-i Psi(f_k)), k_lo <= k < k_hi       (SPA template)
 *   sigma2 = 4 df sum_k |h~_k|^2 / S_k                          (normalisation)
 *   z_j    = 4 df sum_k d~_k conj(h~_k) / S_k exp(+2 pi i j k / N)   (correlator)
 *   rho_j  = |z_j| / sigma ;  phase_j = arg z_j
 *   peak   = argmax over [lo, hi) of rho_j^2, ties to the lowest j
 *   triggers: per window [lo + mW, lo + (m+1)W) the maximum (lowest j on ties),
 *             kept if rho > threshold.
 * The two-polarisation form (steps 2-3 of the per-chunk loop) is provided as a
 * separate function built from two real inverse transforms.
 *
 * Psi(f) is the stationary-phase (TaylorF2) phase of the post-Newtonian
 * inspiral the paper's generator section refers to (Sec. "template
 * generation"), with t_c = 0 and phi_c = 0.  The paper prints no formula for
 * it; the coefficients below are the published TaylorF2 ones (e.g. Buonanno,
 * Iyer, Ochsner, Pan & Sathyaprakash, PRD 80, 084043 (2009), Eq. 3.18).
 * Convention: the time-domain template coalesces at t = 0, so with
 * exp(-i Psi) the chirp occupies the end of the circular buffer.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.141592653589793238462643383279502884
#define OR_MSUN_S 4.925490947e-6 /* G M_sun / c^3 in seconds */
#define OR_EULER 0.5772156649015328606065120900824024310

static int is_pow2(long n) { return n > 0 && (n & (n - 1)) == 0; }

/* ------------------------------------------------------------------------ */
/* Discrete Fourier transforms                                               */
/* ------------------------------------------------------------------------ */

/* Naive DFT, O(n^2): y_k = sum_j x_j exp(sign * 2 pi i j k / n). */
void or_dft(long n, int sign, const double *xr, const double *xi, double *yr, double *yi)
{
    for (long k = 0; k < n; ++k) {
        double sr = 0.0, si = 0.0;
        for (long j = 0; j < n; ++j) {
            /* (j k) mod n is exact in integers, so the angle stays small */
            double a = sign * 2.0 * OR_PI * (double)((j * k) % n) / (double)n;
            double c = cos(a), s = sin(a);
            sr += xr[j] * c - xi[j] * s;
            si += xr[j] * s + xi[j] * c;
        }
        yr[k] = sr;
        yi[k] = si;
    }
}

/* Textbook iterative radix-2 Cooley-Tukey FFT, in place, unnormalised:
 * bit-reversal permutation followed by log2(n) butterfly stages.
 * Returns 0, or -1 if n is not a power of two or memory is short. */
int or_fft(long n, int sign, double *xr, double *xi)
{
    if (!is_pow2(n)) return -1;
    for (long i = 1, j = 0; i < n; ++i) {
        long bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = xr[i]; xr[i] = xr[j]; xr[j] = t;
            t = xi[i]; xi[i] = xi[j]; xi[j] = t;
        }
    }
    double *wr = (double *)malloc(sizeof(double) * (size_t)(n / 2 + 1));
    double *wi = (double *)malloc(sizeof(double) * (size_t)(n / 2 + 1));
    if (!wr || !wi) { free(wr); free(wi); return -1; }
    for (long len = 2; len <= n; len <<= 1) {
        long half = len >> 1;
        for (long m = 0; m < half; ++m) {
            double a = sign * 2.0 * OR_PI * (double)m / (double)len;
            wr[m] = cos(a);
            wi[m] = sin(a);
        }
        for (long i = 0; i < n; i += len) {
            for (long m = 0; m < half; ++m) {
                long p = i + m, q = i + m + half;
                double vr = xr[q] * wr[m] - xi[q] * wi[m];
                double vi = xr[q] * wi[m] + xi[q] * wr[m];
                xr[q] = xr[p] - vr; xi[q] = xi[p] - vi;
                xr[p] += vr;        xi[p] += vi;
            }
        }
    }
    free(wr);
    free(wi);
    return 0;
}

/* Data spectrum d~_k = dt * sum_j d_j exp(-2 pi i j k / n), k = 0..n/2
 * (eq:matchedfilter's X(f), sampled at f_k = k fs / n). */
int or_segment_spectrum(long n, double fs, const double *d, double *dr, double *di)
{
    double *xr = (double *)malloc(sizeof(double) * (size_t)n);
    double *xi = (double *)calloc((size_t)n, sizeof(double));
    if (!xr || !xi) { free(xr); free(xi); return -1; }
    memcpy(xr, d, sizeof(double) * (size_t)n);
    int rc = or_fft(n, -1, xr, xi);
    if (rc == 0) {
        double dt = 1.0 / fs;
        for (long k = 0; k <= n / 2; ++k) { dr[k] = dt * xr[k]; di[k] = dt * xi[k]; }
    }
    free(xr);
    free(xi);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Stationary-phase template                                                 */
/* ------------------------------------------------------------------------ */

/* TaylorF2 phase Psi(f) (radians) for masses m1, m2 (solar masses), keeping
 * the PN terms alpha_i with i <= pn_x2 (twice the PN order: 0 = Newtonian,
 * 4 = 2.0PN, 7 = 3.5PN).  t_c = 0, phi_c = 0.
 *   Psi = -pi/4 + 3 / (128 eta v^5) * sum_i alpha_i v^i,  v = (pi M f)^(1/3). */
void or_spa_phase(double m1, double m2, int pn_x2, long nf, const double *f, double *psi)
{
    const double M = (m1 + m2) * OR_MSUN_S;
    const double eta = m1 * m2 / ((m1 + m2) * (m1 + m2));
    const double pi = OR_PI;
    const double v_lso = 1.0 / sqrt(6.0);
    for (long i = 0; i < nf; ++i) {
        double v = cbrt(pi * M * f[i]);
        double a[8];
        a[0] = 1.0;
        a[1] = 0.0;
        a[2] = 3715.0 / 756.0 + 55.0 * eta / 9.0;
        a[3] = -16.0 * pi;
        a[4] = 15293365.0 / 508032.0 + 27145.0 * eta / 504.0 + 3085.0 * eta * eta / 72.0;
        a[5] = pi * (38645.0 / 756.0 - 65.0 * eta / 9.0) * (1.0 + 3.0 * log(v / v_lso));
        a[6] = 11583231236531.0 / 4694215680.0 - 640.0 * pi * pi / 3.0 - 6848.0 * OR_EULER / 21.0
             + eta * (-15737765635.0 / 3048192.0 + 2255.0 * pi * pi / 12.0)
             + 76055.0 * eta * eta / 1728.0 - 127825.0 * eta * eta * eta / 1296.0
             - 6848.0 / 21.0 * log(4.0 * v);
        a[7] = pi * (77096675.0 / 254016.0 + 378515.0 * eta / 1512.0 - 74045.0 * eta * eta / 756.0);
        double sum = 0.0, vi = 1.0;
        for (int p = 0; p <= pn_x2 && p < 8; ++p) {
            sum += a[p] * vi;
            vi *= v;
        }
        double v5 = v * v * v * v * v;
        psi[i] = -pi / 4.0 + 3.0 / (128.0 * eta * v5) * sum;
    }
}

/* Band of a template: first bin at or above f_low, and the first bin at or
 * above f_ISCO = 1 / (6^(3/2) pi M), capped at n/2 (Nyquist excluded). */
void or_template_band(double m1, double m2, double f_low, double fs, long n, long *k_lo, long *k_hi)
{
    const double M = (m1 + m2) * OR_MSUN_S;
    const double df = fs / (double)n;
    double f_isco = 1.0 / (pow(6.0, 1.5) * OR_PI * M);
    long lo = (long)ceil(f_low / df);
    long hi = (long)ceil(f_isco / df);
    if (lo < 1) lo = 1;
    if (hi > n / 2) hi = n / 2;
    *k_lo = lo;
    *k_hi = hi;
}

/* h~_k = f_k^(-7/6) exp(-i Psi(f_k)) for k_lo <= k < k_hi, zero for the other
 * one-sided bins k = 0..n/2 (Newtonian amplitude; its constant factor does
 * not change rho). */
int or_spa_template(double m1, double m2, int pn_x2, double f_low, double fs, long n,
                    double *hr, double *hi, long *k_lo, long *k_hi)
{
    long lo, hi_;
    or_template_band(m1, m2, f_low, fs, n, &lo, &hi_);
    *k_lo = lo;
    *k_hi = hi_;
    for (long k = 0; k <= n / 2; ++k) { hr[k] = 0.0; hi[k] = 0.0; }
    if (hi_ <= lo) return 0;
    long nb = hi_ - lo;
    double *f = (double *)malloc(sizeof(double) * (size_t)nb);
    double *psi = (double *)malloc(sizeof(double) * (size_t)nb);
    if (!f || !psi) { free(f); free(psi); return -1; }
    const double df = fs / (double)n;
    for (long k = lo; k < hi_; ++k) f[k - lo] = (double)k * df;
    or_spa_phase(m1, m2, pn_x2, nb, f, psi);
    for (long k = lo; k < hi_; ++k) {
        double amp = pow(f[k - lo], -7.0 / 6.0);
        hr[k] = amp * cos(psi[k - lo]);
        hi[k] = -amp * sin(psi[k - lo]);
    }
    free(f);
    free(psi);
    return 0;
}

/* sigma^2 = <h, h> = 4 df sum_{k_lo <= k < k_hi} |h~_k|^2 / S_k  (the template
 * normalisation of the per-chunk loop's step 1). */
double or_sigma2(long n, double fs, const double *hr, const double *hi, const double *psd,
                 long k_lo, long k_hi)
{
    const double df = fs / (double)n;
    double s = 0.0;
    for (long k = k_lo; k < k_hi; ++k) s += (hr[k] * hr[k] + hi[k] * hi[k]) / psd[k];
    return 4.0 * df * s;
}

/* ------------------------------------------------------------------------ */
/* Correlator                                                                */
/* ------------------------------------------------------------------------ */

/* z_j = 4 df sum_{k_lo <= k < k_hi} d~_k conj(h~_k) / S_k exp(+2 pi i j k / n),
 * j = 0..n-1 (eq:matchedfilter on the sampled one-sided band; circular). */
int or_correlate(long n, double fs, const double *dr, const double *di, const double *hr,
                 const double *hi, const double *psd, long k_lo, long k_hi, double *zr, double *zi)
{
    const double df = fs / (double)n;
    for (long j = 0; j < n; ++j) { zr[j] = 0.0; zi[j] = 0.0; }
    for (long k = k_lo; k < k_hi; ++k) {
        /* d~ * conj(h~) / S */
        zr[k] = (dr[k] * hr[k] + di[k] * hi[k]) / psd[k];
        zi[k] = (di[k] * hr[k] - dr[k] * hi[k]) / psd[k];
    }
    if (or_fft(n, +1, zr, zi) != 0) return -1;
    for (long j = 0; j < n; ++j) { zr[j] *= 4.0 * df; zi[j] *= 4.0 * df; }
    return 0;
}

/* The paper's two-polarisation correlators (per-chunk loop, steps 2-3):
 * theta_+ has spectrum h~ and theta_x has spectrum i h~ on positive
 * frequencies; each real correlator c(t) = <x, theta>(t) is the inverse
 * transform of the two-sided Hermitian spectrum 2 df X Theta* / S, whose
 * negative-frequency half is the complex conjugate of the positive half. */
int or_correlate_polarisations(long n, double fs, const double *dr, const double *di,
                               const double *hr, const double *hi, const double *psd,
                               long k_lo, long k_hi, double *cplus, double *ccross)
{
    const double df = fs / (double)n;
    double *ar = (double *)calloc((size_t)n, sizeof(double));
    double *ai = (double *)calloc((size_t)n, sizeof(double));
    if (!ar || !ai) { free(ar); free(ai); return -1; }
    for (int pol = 0; pol < 2; ++pol) {
        memset(ar, 0, sizeof(double) * (size_t)n);
        memset(ai, 0, sizeof(double) * (size_t)n);
        for (long k = k_lo; k < k_hi; ++k) {
            /* Theta~ = h~ (plus) or i h~ (cross) */
            double tr = pol == 0 ? hr[k] : -hi[k];
            double ti = pol == 0 ? hi[k] : hr[k];
            double pr = (dr[k] * tr + di[k] * ti) / psd[k];
            double pi_ = (di[k] * tr - dr[k] * ti) / psd[k];
            ar[k] = 2.0 * df * pr;
            ai[k] = 2.0 * df * pi_;
            ar[n - k] = 2.0 * df * pr;   /* Hermitian mirror at -f_k */
            ai[n - k] = -2.0 * df * pi_;
        }
        if (or_fft(n, +1, ar, ai) != 0) { free(ar); free(ai); return -1; }
        double *out = pol == 0 ? cplus : ccross;
        for (long j = 0; j < n; ++j) out[j] = ar[j];
    }
    free(ar);
    free(ai);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Peak and threshold triggers                                               */
/* ------------------------------------------------------------------------ */

/* rho_j^2 = |z_j|^2 / sigma2 (defined as 0 when sigma2 == 0).  Peak: maximum
 * of rho^2 over [lo, hi), the lowest j on ties.  Triggers: for each window
 * [lo + m W, min(lo + (m+1) W, hi)) its maximum (lowest j on ties), kept if
 * rho > thr.  Writes at most `cap` triggers and returns how many there are. */
long or_peak_triggers(long n, const double *zr, const double *zi, double sigma2, long lo, long hi,
                      long window, double thr, long *peak_j, double *peak_rho, double *peak_phase,
                      long *trig_j, double *trig_rho, double *trig_phase, long cap)
{
    (void)n;
    long best_j = lo;
    double best = -1.0;
    long count = 0;
    for (long w0 = lo; w0 < hi; w0 += window) {
        long w1 = w0 + window < hi ? w0 + window : hi;
        long wj = w0;
        double wbest = -1.0;
        for (long j = w0; j < w1; ++j) {
            double r2 = sigma2 > 0.0 ? (zr[j] * zr[j] + zi[j] * zi[j]) / sigma2 : 0.0;
            if (r2 > wbest) { wbest = r2; wj = j; }
        }
        if (wbest > best) { best = wbest; best_j = wj; }
        if (sqrt(wbest) > thr) {
            if (count < cap) {
                trig_j[count] = wj;
                trig_rho[count] = sqrt(wbest);
                trig_phase[count] = atan2(zi[wj], zr[wj]);
            }
            ++count;
        }
    }
    *peak_j = best_j;
    *peak_rho = best >= 0.0 ? sqrt(best) : 0.0;
    *peak_phase = hi > lo ? atan2(zi[best_j], zr[best_j]) : 0.0;
    return count;
}

/* One template through the whole per-chunk loop: template, sigma^2,
 * correlator, peak and triggers.  Returns the trigger count or -1. */
long or_filter_template(long n, double fs, const double *dr, const double *di, const double *psd,
                        double m1, double m2, int pn_x2, double f_low, long lo, long hi,
                        long window, double thr, double *sigma2_out, long *peak_j,
                        double *peak_rho, double *peak_phase, long *trig_j, double *trig_rho,
                        double *trig_phase, long cap)
{
    double *hr = (double *)malloc(sizeof(double) * (size_t)(n / 2 + 1));
    double *hi_ = (double *)malloc(sizeof(double) * (size_t)(n / 2 + 1));
    double *zr = (double *)malloc(sizeof(double) * (size_t)n);
    double *zi = (double *)malloc(sizeof(double) * (size_t)n);
    long count = -1;
    if (hr && hi_ && zr && zi) {
        long k_lo, k_hi;
        if (or_spa_template(m1, m2, pn_x2, f_low, fs, n, hr, hi_, &k_lo, &k_hi) == 0) {
            double s2 = or_sigma2(n, fs, hr, hi_, psd, k_lo, k_hi);
            *sigma2_out = s2;
            if (or_correlate(n, fs, dr, di, hr, hi_, psd, k_lo, k_hi, zr, zi) == 0)
                count = or_peak_triggers(n, zr, zi, s2, lo, hi, window, thr, peak_j, peak_rho,
                                         peak_phase, trig_j, trig_rho, trig_phase, cap);
        }
    }
    free(hr);
    free(hi_);
    free(zr);
    free(zi);
    return count;
}
