/*
 * cui.h -- C ABI of the GB300 bank matched filter.
 *
 * The library matched-filters one detector segment against a bank of
 * stationary-phase post-Newtonian inspiral templates and reduces the
 * normalised correlator |z|^2 / sigma^2 to a peak and threshold triggers per
 * template.  It follows the paper's problem statement (Bosi,
 * arXiv:1006.4644, Sec. "Matched filtering"): a bank of (m1, m2) points, a
 * data chunk with its noise power spectrum, the correlator of
 * eq:matchedfilter for each template, normalised so that <theta, theta> = 1,
 * its maximum above a threshold, and a reduction of those maxima.
 *
 * Conventions shared by every call:
 *  - Every call returns a cui_status; nothing throws across the ABI.  A
 *    failing call leaves a message for cui_last_error() (thread-local).
 *  - Work is enqueued asynchronously on desc.stream (a cudaStream_t; NULL is
 *    the legacy default stream).  cui_triggers, cui_peaks and cui_bank_sigma
 *    synchronise that stream before they return.
 *  - Input pointers are not retained: the library copies what it needs into
 *    memory it owns.  Pointers documented as "device" must be device (or
 *    managed) memory of the current device; all others are host memory.
 *  - A handle is used by one host thread at a time; calls on one handle are
 *    not re-entrant.  Distinct handles are independent.
 *  - Units: masses in solar masses, frequencies in Hz, the PSD in 1/Hz
 *    (one-sided), the strain dimensionless, samples at desc.sample_rate.
 *
 * Definitions (k = one-sided frequency bin, f_k = k fs / N, df = fs / N):
 *   d~_k   = (1/fs) sum_j d_j exp(-2 pi i j k / N)
 *   h~_k   = f_k^(-7/6) exp(-i Psi(f_k)) for k_lo <= k < k_hi, else 0, where
 *            Psi is the TaylorF2 phase (t_c = 0, phi_c = 0) truncated at
 *            twice-PN-order pn_order_x2, k_lo = ceil(f_low / df) and
 *            k_hi = min(ceil(f_ISCO / df), N/2), f_ISCO = 1 / (6^1.5 pi M)
 *   sigma^2 = 4 df sum_k |h~_k|^2 / S_k
 *   z_j    = 4 df sum_k d~_k conj(h~_k) / S_k exp(+2 pi i j k / N), j in [0, N)
 *   rho_j  = |z_j| / sigma,  phase_j = arg z_j
 *   peak   = argmax of rho over [valid_lo, valid_hi), lowest sample on ties
 *   triggers: one per window [valid_lo + m W, valid_lo + (m+1) W) (clipped to
 *            valid_hi) whose maximum rho exceeds snr_threshold (strictly).
 */
#ifndef CUI_H
#define CUI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CUI_OK = 0,
    CUI_ERR_ARG = 1,      /* invalid argument (message says which)             */
    CUI_ERR_CUDA = 2,     /* a CUDA runtime call failed                         */
    CUI_ERR_OOM = 3,      /* device memory allocation failed                    */
    CUI_ERR_STATE = 4,    /* call out of order (e.g. filter before upload)      */
    CUI_ERR_OVERFLOW = 5, /* more triggers than the buffer holds; n_total exact */
    CUI_ERR_TIMEOUT = 6   /* a bounded device wait gave up; handle stays usable */
} cui_status;

/* desc.flags */
#define CUI_PSI_FP64    0x1u /* fused path: anchor phases in native FP64 (default: double-float FP32 pairs) */
#define CUI_STORE_BF16  0x2u /* fused path: store the spectrum between FFT passes as bf16 pairs */
#define CUI_PLAIN       0x4u /* per-template unfused path: generate, multiply, multi-pass FFT, detect */
#define CUI_PLAIN_FP64  0x8u /* with CUI_PLAIN: template, product and FFT in FP64 (else FP32) */
#define CUI_NO_GRAPH    0x10u /* fused path: launch kernels directly instead of replaying a captured CUDA graph */

typedef struct cui_bank_s *cui_bank; /* opaque; owns every device buffer it allocates */

typedef struct {
    int32_t pn_order_x2;      /* twice the PN order of the phase, 0..7 (4 = 2.0PN, 7 = 3.5PN) */
    int32_t reserved0;        /* must be 0 */
    double f_low;             /* lower cut-off (Hz), > 0 */
    double sample_rate;       /* fs (Hz), > 0 */
    int64_t n;                /* segment length N: a power of two, 2^6 .. 2^22 */
    uint32_t flags;           /* CUI_* flags above */
    uint32_t reserved1;       /* must be 0 */
    double snr_threshold;     /* trigger threshold on rho (default reading: 6) */
    int64_t window;           /* trigger window W in samples, >= 1 */
    int64_t valid_lo;         /* samples considered: [valid_lo, valid_hi), 0 <= lo <= hi <= N */
    int64_t valid_hi;
    int64_t trigger_capacity; /* device trigger records; 0 selects 1 << 20 */
    void *stream;             /* cudaStream_t for all work of this handle */
} cui_bank_desc;

typedef struct {
    int64_t sample; /* argmax j of rho over the valid range */
    float snr;      /* rho at that sample */
    float phase;    /* arg z at that sample (radians) */
} cui_peak;

typedef struct {
    int32_t tmpl;   /* template index in the bank */
    int32_t pad;
    int64_t sample; /* sample of the window maximum */
    float snr;      /* rho there, > snr_threshold */
    float phase;    /* arg z there */
} cui_trigger;

/* Build a bank of n_templates templates (m1[i], m2[i]), host arrays that are
 * copied.  Allocates the handle's device memory and per-template constants on
 * the current device; enqueues set-up work on desc->stream.
 * Errors: CUI_ERR_ARG (bad desc field, n_templates < 1, masses <= 0 or not
 * finite), CUI_ERR_OOM, CUI_ERR_CUDA.  *out is NULL on failure.
 * Paper: the bank of (m1, m2) points (Sec. "Matched filtering") and
 * host_template_init / device_template_init (Sec. "Pipeline main details"). */
cui_status cui_bank_create(const cui_bank_desc *desc, const double *m1, const double *m2,
                           int64_t n_templates, cui_bank *out);

/* Upload one segment: strain d_j (n = desc.n FP64 samples) and its one-sided
 * PSD S_k (n_psd = N/2 + 1 FP64 values, 1/Hz; only bins in [k_lo, N/2) are
 * read and must be finite and > 0).  on_device = 1 means both pointers are
 * device memory, 0 host memory (pinned host memory makes the copies
 * asynchronous).  Computes d~ (double-float transform, FP64 result), the
 * noise-weighted data and every template's sigma^2 on the device.  A host PSD
 * is checked on the device: the call queues all of its work, then waits until
 * the GPU has checked the PSD (the work queued behind the check goes on).
 * Device PSDs are not checked and the call does not wait.
 * Errors: CUI_ERR_ARG (n != desc.n, n_psd != N/2 + 1, NULL pointers; a host
 * PSD bin in the band that is not finite and > 0, which leaves the bank
 * without a segment until the next successful upload), CUI_ERR_CUDA.  Paper: the data chunk X(f) and S_n(f) of
 * eq:matchedfilter. */
cui_status cui_segment_upload(cui_bank bank, const double *strain, int64_t n, const double *psd,
                              int64_t n_psd, int on_device);

/* Filter `count` templates of the bank against the uploaded segment.  order:
 * host array of distinct template indices in [0, n_templates), or NULL for all
 * templates in bank order (count must then equal n_templates).  peaks_dev:
 * device array of n_templates records (caller-owned) receiving the peak of
 * every filtered template at its template index, or NULL to keep peaks in the
 * handle (read them with cui_peaks).  Triggers of this call replace those of
 * the previous call.  Asynchronous.
 * Errors: CUI_ERR_STATE (no segment uploaded), CUI_ERR_ARG, CUI_ERR_CUDA.
 * Paper: the per-chunk loop of Sec. "Matched filtering", steps 1-4. */
cui_status cui_filter_bank(cui_bank bank, const int32_t *order, int64_t count, cui_peak *peaks_dev);

/* Copy the peaks of the last filter call that kept them in the handle to
 * host_out[0 .. count), indexed by template (count <= n_templates).
 * Synchronises.  Errors: CUI_ERR_ARG, CUI_ERR_STATE, CUI_ERR_CUDA,
 * CUI_ERR_TIMEOUT.  Paper: each template's maximum of the SNR over the data
 * chunk, step 4 of Sec. "Matched filtering". */
cui_status cui_peaks(cui_bank bank, cui_peak *host_out, int64_t count);

/* Copy the triggers of the last filter call to host_out and their exact total
 * number to *n_total.  min(*n_total, capacity, desc.trigger_capacity) records
 * are written, sorted by (tmpl, sample).  When the device buffer
 * (desc.trigger_capacity) overflowed, the records kept are an arbitrary
 * subset; peaks are unaffected.  Synchronises.  Returns CUI_ERR_OVERFLOW when
 * *n_total exceeds `capacity` or the device buffer, CUI_ERR_TIMEOUT if a
 * bounded device wait gave up during the call.
 * Paper: the candidate set {t_0^i} of step 4 and its reduction. */
cui_status cui_triggers(cui_bank bank, cui_trigger *host_out, int64_t capacity, int64_t *n_total);

/* cui_peaks and cui_triggers in one call: host_peaks[0 .. n_peaks) and up to
 * `capacity` trigger records with their total in *n_total, as those two calls
 * give them, read back with one synchronisation: the copy of the peaks and the
 * count goes with a copy of the first max(1024, 2 c) device trigger records
 * (at most the device capacity), c the count of the handle's previous read-out
 * (1024 before the first); a larger count costs a second copy of all records.
 * Synchronises.  Errors: as cui_peaks and cui_triggers.
 * Paper: the per-template maxima and candidate set of step 4, read back to the
 * host as the pipeline's result. */
cui_status cui_results(cui_bank bank, cui_peak *host_peaks, int64_t n_peaks, cui_trigger *host_trig,
                       int64_t capacity, int64_t *n_total);

/* Cross-template clustering of the last filter call's triggers: for each
 * trigger window [valid_lo + m W, valid_lo + (m+1) W) (the same windows as
 * the per-template triggers), the loudest trigger over all filtered
 * templates; among equal rho the lowest sample, then the lowest template.
 * Computed on the device while the triggers are compacted (one 128-bit
 * compare-and-swap per trigger), so it is exact even when the trigger buffer
 * overflowed.  Writes min(*n_total, capacity) records in increasing sample
 * order (one per window that has a trigger) and the exact count to *n_total.
 * Synchronises.  Errors: CUI_ERR_ARG, CUI_ERR_STATE (no filter call since the
 * last upload), CUI_ERR_OVERFLOW (*n_total > capacity), CUI_ERR_TIMEOUT,
 * CUI_ERR_CUDA.  Paper: the reduction of the per-template candidates to local
 * maxima (Sec. "Matched filtering", final step) and the clustering it leaves
 * to the CPU (Sec. "Pipeline main details"). */
cui_status cui_cluster_triggers(cui_bank bank, cui_trigger *host_out, int64_t capacity, int64_t *n_total);

/* Signal-consistency (chi^2) test at n triggers (host records, e.g. from
 * cui_triggers; only tmpl and sample are read) against the uploaded segment.
 * The template's band [k_lo, k_hi) is split into `bands` sub-bands of equal
 * template power, edges k_l = min{k : Pw(k) >= (l/bands) Pw(k_hi)} with
 * Pw(k) = sum_{k_lo <= j < k} |h~_j|^2 / S_j; with the sub-band correlators
 * z_l (z restricted to band l, at the trigger's sample) and z = sum_l z_l,
 *   chi^2 = bands sum_l |z_l - z / bands|^2 / sigma^2,
 * about 2 bands - 2 in Gaussian noise and ~0 for the exact template.
 * host_chisq[i] receives chi^2 of trigger i; host_rho (nullable) the rho
 * recomputed from the same sums.  Fused banks only.  Synchronises.
 * Errors: CUI_ERR_ARG (bands outside [1, 64], a template or sample out of
 * range, NULL pointers), CUI_ERR_STATE (plain bank, no segment),
 * CUI_ERR_CUDA, CUI_ERR_TIMEOUT.  Paper: the chi^2 discrimination against
 * non-Gaussian noise listed among the pipeline's future work (Sec.
 * "Conclusions"), in the equal-power sub-band form of the matched-filter
 * literature it builds on. */
cui_status cui_trigger_chisq(cui_bank bank, int32_t bands, const cui_trigger *trig, int64_t n, float *host_chisq,
                             float *host_rho);

/* Multi-band search (Sec. "Online analysis considerations": the frequency
 * range divided into bands, the matched filter run first on the upper band,
 * where the chirp is shortest and carries most of the SNR, and the lower bands
 * added afterwards for the candidates).
 *
 * cui_bank_set_band restricts every later filter call, and the sigma, chi^2
 * and clustering results that follow from it, to each template's bins in
 * [f_lo, f_hi): bins k_lo' <= k < min(k_hi(t), k_hi') with
 * k_lo' = max(k_low, ceil(f_lo / df)) and k_hi' = ceil(f_hi / df), capped at
 * N/2; f_hi <= 0 sets no upper limit, and f_lo <= f_low with f_hi <= 0 gives
 * back the full band.  sigma^2 is the template's power inside the band, so rho
 * is the band's own SNR.  With f_lo well above f_low the band's chirp lasts
 * only tau(f_lo), and the band can be searched on segments much shorter than
 * the whole template.  The band stays in force across uploads until it is set
 * again.  Asynchronous; the host waits once, for earlier calls on the stream.
 * Errors: CUI_ERR_ARG (NULL bank, edges not finite), CUI_ERR_CUDA. */
cui_status cui_bank_set_band(cui_bank bank, double f_lo, double f_hi);

/* Band correlators at arbitrary times, by direct sums over the band's bins (no
 * FFT).  Query i is template tmpl[i] at time t_sec[i] (seconds after the
 * segment's first sample, taken modulo T = N / fs):
 *   z_i = 4 df sum_{k in B_i} d~_k conj(h~_k) / S_k exp(+2 pi i k df t_i),
 *   sigma_i^2 = 4 df sum_{k in B_i} |h~_k|^2 / S_k,
 * h~_k = f_k^(-7/6) exp(-i Psi(f_k)) generated by the filter's method
 * (double-float phase anchors, one per block of 32 bins, or of the tiling's
 * ccols where N / n1 < 32, FP32 per bin; the
 * phase within 1e-6 cycles of the FP64 value), B_i = [max(f_lo, f_low), f_hi)
 * cut to the template's own band [f_low,
 * f_isco) (f_hi <= 0: no upper limit), whatever cui_bank_set_band holds.  At a
 * sample time j / fs over the filter's band, z_i / sigma is the filter's rho
 * with its phase.  Both are in physical units (strain and PSD as uploaded,
 * frequencies in Hz), so that the results of banks holding the same data at
 * other lengths or sample rates add up: over disjoint bands b of one template
 * at one time, rho = |sum_b z_b| / sqrt(sum_b sigma_b^2).  host_z receives 2n
 * doubles (Re z_i, Im z_i), host_sigma2 (nullable) n doubles.  Fused banks
 * only.  Synchronises.  Errors: CUI_ERR_ARG (template out of range, time or
 * edges not finite, NULL pointers), CUI_ERR_STATE (plain bank, no segment),
 * CUI_ERR_CUDA, CUI_ERR_TIMEOUT. */
cui_status cui_band_correlate(cui_bank bank, const int32_t *tmpl, const double *t_sec, int64_t n, double f_lo,
                              double f_hi, double *host_z, double *host_sigma2);

/* The last step of the multi-band search: n candidates completed by the
 * lower band and combined coherently.  Candidate i is template tmpl[i] of
 * both banks (the same bank points, checked), detected by `high` (usually a
 * short segment, band set to [f_split, ...)) at time t_high[i] seconds after
 * high's first sample; `low` holds the data to complete it (the whole
 * segment, or a decimated copy of its lower band) and the same instant is
 * t_low[i] seconds after low's first sample.  With the band correlators of
 * cui_band_correlate, z_h over [f_split, ...) on `high` and z_l over
 * [..., f_split) on `low`:
 *   rho_i = |z_h + z_l| / sqrt(sigma_h^2 + sigma_l^2),  phase_i = arg(z_h + z_l)
 * written to host_rho and host_phase (n doubles each); host_sums (nullable)
 * receives 6 n doubles (Re z_h, Im z_h, sigma_h^2, Re z_l, Im z_l,
 * sigma_l^2).  The sums run on each bank's stream, the combination on low's
 * after high's; synchronises both.  Paper: Sec. "Online analysis
 * considerations" (the bands are analysed separately, the high one first,
 * then the lower bands added for the candidates).  Errors: CUI_ERR_ARG (NULL
 * pointers, different bank points, f_split not finite and > 0, a template
 * out of range, a time not finite), CUI_ERR_STATE (plain bank, no segment),
 * CUI_ERR_CUDA, CUI_ERR_TIMEOUT. */
cui_status cui_band_combine(cui_bank high, const double *t_high, cui_bank low, const double *t_low,
                            const int32_t *tmpl, int64_t n, double f_split, double *host_rho, double *host_phase,
                            double *host_sums);

/* The band of every template as the banks use it, on host arrays, without a
 * GPU: *k_low_out (nullable) = max(1, ceil(f_low / df)) clamped to N/2,
 * k_hi_out[t] = min(ceil(f_isco / df), N/2) with f_isco = 1 / (6^(3/2) pi M),
 * M = (m1[t] + m2[t]) G Msun / c^3, df = sample_rate / n.  For callers that
 * plan work by band (the sharding of a bank across GPUs weighs templates by
 * k_hi - k_low), so that they use the library's own rule.  Paper: the
 * low-frequency cut-off sets a template's length (Sec. "Online analysis
 * considerations" and its footnote); the upper end at the innermost stable
 * circular orbit is not in the paper (this library's reading).  Errors:
 * CUI_ERR_ARG (NULL pointers, n not a power of two >= 2, non-finite or
 * non-positive rate, f_low or masses). */
cui_status cui_template_bands(const double *m1, const double *m2, int64_t n_templates, int64_t n,
                              double sample_rate, double f_low, int32_t *k_low_out, int32_t *k_hi_out);

/* The uploaded segment restricted to one band and resampled, for the
 * multi-band search: the series that the upper band is searched on (short
 * segments cut from it, at the full rate) and the decimated series that
 * carries a lower band to a bank at a lower sample rate.
 *   x'_j = (1/N) sum_{k in B} X_k e^(+2 pi i k j / m) + c.c., j < m = N / decim,
 * X_k = sum_j d_j e^(-2 pi i jk/N) the segment's DFT (computed at upload in
 * double-float, near-FP64 accuracy) and B the bins ceil(f_lo/df) <= k <
 * ceil(f_hi/df) below m/2 (f_hi <= 0: up to m/2; the bin at m/2 is dropped).
 * With decim = 1 it is the band-passed segment at the full rate; a band below
 * the new Nyquist frequency fs / (2 decim) loses nothing by the decimation.
 * out_dev: m doubles of device memory, caller-owned.  decim: a power of two,
 * N / decim >= 16.  Asynchronous on the bank's stream.  Errors: CUI_ERR_ARG,
 * CUI_ERR_STATE (no segment), CUI_ERR_CUDA. */
cui_status cui_segment_band_series(cui_bank bank, double f_lo, double f_hi, int32_t decim, double *out_dev);

/* The paper's own template form: the two polarisations of template `tmpl` in
 * the time domain at the bank's sample rate, post-Newtonian order pn_x2 / 2
 * (<= 2.5) in phase and Newtonian in amplitude (Sec. "template
 * generation").  Orbital evolution in the TaylorT2 form from the binding
 * energy and flux of circular orbits: t(v) and phi(v) as series in
 * v = (M omega)^(1/3) (t_c = phi_c = 0); sample j is at
 * t_j = -((N - j) mod N) / fs, so the chirp coalesces at sample 0 and runs
 * backwards through the end of the buffer, as the SPA templates do.
 * hp_dev[j] = v^2 cos 2 phi, hx_dev[j] = v^2 sin 2 phi between f_low and the
 * innermost stable orbit (v = 6^-1/2), 0 elsewhere and for t < -N / fs.
 * Device FP64 arrays of N samples, caller-owned.  Asynchronous.
 * Uploaded as strain and filtered with the bank, it gives the match with the
 * stationary-phase templates (the mismatch of eq:mismatch).
 * Errors: CUI_ERR_ARG (template or order out of range, NULL pointers),
 * CUI_ERR_CUDA. */
cui_status cui_td_template(cui_bank bank, int64_t tmpl, int32_t pn_x2, double *hp_dev, double *hx_dev);

/* sigma_t = sqrt(4 df sum_k |h~_k|^2 / S_k) of every template for the
 * uploaded PSD, to host_sigma[0 .. n_templates).  Synchronises.
 * Errors: CUI_ERR_STATE (no segment), CUI_ERR_CUDA.
 * Paper: the template normalisation of step 1 (Sec. "template generation
 * and normalization"). */
cui_status cui_bank_sigma(cui_bank bank, double *host_sigma);

/* Write template t as the fused path generates it: h~_k for k = 0 .. N/2 as
 * N/2 + 1 interleaved FP32 (re, im) pairs to device memory out_dev, zero
 * outside [k_lo, k_hi).  Asynchronous.  Errors: CUI_ERR_ARG, CUI_ERR_CUDA.
 * Paper: device_template_proc (Sec. "Pipeline main details"). */
cui_status cui_bank_template(cui_bank bank, int64_t t, float *out_dev);

/* Tiling of the fused path.  The correlator of length N is computed as
 * N = n1 * n2: pass 1 runs n1-point transforms over `ccols` columns per CTA
 * (fused with template generation), pass 2 runs n2-point transforms over
 * `rpc` rows per CTA (fused with the peak / threshold reduction), and
 * `batch` templates share one pass-1 / pass-2 launch pair (their spectra,
 * batch * N complex values, live in a workspace between the passes). */
typedef struct {
    int32_t n1;    /* 64, 128 or 256 (subject to the kernels built for N) */
    int32_t ccols; /* 16, 32 or 64 */
    int32_t rpc;   /* rows per pass-2 CTA; 0: the streamed persistent pass 2
                      (one CTA per SM, rows copied into shared memory by the
                      bulk-copy engine), for n2 = N / n1 = 4096 (row pairs)
                      and 16384 (rows split four ways in frequency) */
    int32_t batch; /* templates per launch pair, >= 1 */
} cui_tuning;

/* Current tiling.  Errors: CUI_ERR_ARG, CUI_ERR_STATE (per-template path).
 * Not in the paper (this library's kernel tiling), as the two calls below. */
cui_status cui_bank_get_tuning(cui_bank bank, cui_tuning *out);

/* Select a tiling; reallocates the workspace (synchronises the stream).
 * Errors: CUI_ERR_ARG (no kernel for that tiling at this N), CUI_ERR_STATE
 * (per-template path), CUI_ERR_OOM, CUI_ERR_CUDA.  Results do not depend on
 * the tiling beyond floating-point rounding. */
cui_status cui_bank_set_tuning(cui_bank bank, const cui_tuning *tuning);

/* Autotuner: time cui_filter_bank on the uploaded segment (`reps` calls per
 * candidate, CUDA events on desc.stream) for every tiling that has kernels at
 * this N, keep the fastest selected, and return it and its time per call.
 * Overwrites the peaks and triggers of earlier calls.  Errors:
 * CUI_ERR_STATE (no segment, or per-template path), CUI_ERR_ARG, CUI_ERR_CUDA.
 * Not in the paper: its kernels had no tunable tiling. */
cui_status cui_bank_autotune(cui_bank bank, int32_t reps, cui_tuning *best, double *best_ms);

/* Bounds of the handle's device waits, for tests of the error path.  The
 * only spins in the library are the compare-and-swap loops that raise the
 * peak, window and cluster slots (at most cas_rounds rounds, default 2^20)
 * and, in the streamed pass 2 (tiling rpc 0), each wait for a row (pair) to
 * land in shared memory (at most copy_wait_ns ns on the GPU's global
 * timer, default 10^9; 0 makes every such wait give up at once).  A wait
 * that runs out sets the device error word and
 * its kernel skips the rest of its work (the streamed pass 2 still waits up to
 * 10^9 ns for a copy in flight before its CTA exits); the next synchronising
 * call returns CUI_ERR_TIMEOUT and clears the word, and the handle stays
 * usable: the next cui_segment_upload and filter call give full results
 * again.  Negative values restore the defaults; values above them return
 * CUI_ERR_ARG.  Synchronises the stream.  Paper: the final reduction of the
 * per-template maxima (Sec. "Matched filtering"), whose device-side form here
 * needs these waits; the bounds themselves are not in the paper. */
cui_status cui_bank_set_wait_bounds(cui_bank bank, int64_t cas_rounds, int64_t copy_wait_ns);

/* Tracing.  cui_trace_enable(bank, level): 0 off; 1 records CUDA events on
 * desc.stream around each call's groups of kernels ("segment", "plain", and
 * "graph" for the captured fused filter); 2 also times every fused kernel
 * group ("pass1", "pass2", "finalize"), for which the fused filter launches
 * its kernels directly instead of replaying its graph.  cui_trace_read
 * synchronises, writes up to `capacity` per-group totals (launches of this
 * library's kernels, summed event time) to host_out, the number of groups to
 * *n, and clears the record.
 * Errors: CUI_ERR_ARG, CUI_ERR_CUDA.  Paper: the per-step timing information
 * of Sec. "GPU based detection pipeline performances and profiling". */
typedef struct {
    char name[24];
    int64_t launches; /* kernel launches in this group */
    int64_t calls;    /* timed intervals */
    double ms;        /* total event time */
} cui_trace_stat;

cui_status cui_trace_enable(cui_bank bank, int on);
cui_status cui_trace_read(cui_bank bank, cui_trace_stat *host_out, int64_t capacity, int64_t *n);

/* ------------------------------------------------------------------------
 * Learned prescreen.  Ranks regions of the bank (groups of templates sorted
 * by chirp mass) from whitened band powers of a segment, so that likely
 * regions are filtered first.  The paper motivates it only in passing: for
 * banks of ~10^6 templates it doubts that exhaustive filtering is the right
 * approach (introduction, footnote).  Features: u_k = d~_k sqrt(4 df / S_k) on [f_low, fs/2) split
 * into `bands` log-spaced bands; per band X_b(j) = sum_{k in band} u_k
 * exp(+2 pi i j k / N); F[b][m] = log(mean_{frame m} |X_b|^2 / (2 n_b)) over
 * N / frame frames.  Network: 4 conv1d layers of 32 channels (kernel 5,
 * stride 1 then 2, zero padding 2, ReLU), per-channel mean and max over time,
 * linear 64 -> 128 (ReLU) -> regions; BF16 weights, FP32 accumulation; soft
 * label cross-entropy; Adam.  Training is deterministic for a given seed.
 * Device arrays: features [count][bands][N/frame] float, targets and scores
 * [count][regions] float.  Asynchronous on desc.stream unless stated.
 * Errors of every call below: CUI_ERR_ARG (NULL handle or pointer, a size
 * out of the ranges stated, a count above max_batch), CUI_ERR_OOM (create),
 * CUI_ERR_CUDA; cui_prescreen_bank_features also CUI_ERR_STATE (the bank
 * holds no segment).
 * ------------------------------------------------------------------------ */
typedef struct cui_prescreen_s *cui_prescreen;

typedef struct {
    int64_t n;          /* segment length of the features: power of two in [2^10, 2^22] */
    double sample_rate; /* Hz */
    double f_low;       /* Hz, lower edge of the lowest band */
    int32_t bands;      /* 1 .. 16 */
    int32_t frame;      /* samples per frame: a multiple of 32 dividing n, n / frame in [8, 256] */
    int32_t regions;    /* outputs, 2 .. 256 */
    int32_t max_batch;  /* largest training / gradient batch, 1 .. 4096 */
    float lr, beta1, beta2, eps; /* Adam */
    uint64_t seed;      /* parameter initialisation */
    void *stream;       /* cudaStream_t */
} cui_prescreen_desc;

cui_status cui_prescreen_create(const cui_prescreen_desc *desc, cui_prescreen *out);
void cui_prescreen_destroy(cui_prescreen p);
/* number of parameters and of frames per feature row */
cui_status cui_prescreen_info(cui_prescreen p, int64_t *n_params, int32_t *frames);
/* features of `count` segments: dtilde_dev = [count][N/2 + 1] complex FP64
 * (interleaved) data spectra d~_k, psd_dev = [N/2 + 1] FP64 */
cui_status cui_prescreen_features(cui_prescreen p, const double *dtilde_dev, const double *psd_dev, int64_t count,
                                  float *feat_dev);
/* features of the segment last uploaded to `bank` (same N and sample rate) */
cui_status cui_prescreen_bank_features(cui_prescreen p, cui_bank bank, float *feat_dev);
/* region scores (logits) of `count` feature rows */
cui_status cui_prescreen_scores(cui_prescreen p, const float *feat_dev, int64_t count, float *scores_dev);
/* one Adam step on a batch; loss_host (nullable) receives the mean loss and
 * then the call synchronises */
cui_status cui_prescreen_train_step(cui_prescreen p, const float *feat_dev, const float *target_dev, int64_t count,
                                    float *loss_host);
/* mean gradient of the batch loss w.r.t. the parameters (n_params floats,
 * device), without updating them */
cui_status cui_prescreen_gradient(cui_prescreen p, const float *feat_dev, const float *target_dev, int64_t count,
                                  float *grad_dev, float *loss_host);
/* checkpoint / resume: FP32 parameters, Adam moments (host arrays of
 * n_params floats, each nullable on get; m, v nullable on set = zero) and the
 * step counter.  Synchronise. */
cui_status cui_prescreen_get_state(cui_prescreen p, float *theta, float *m, float *v, int64_t *step);
cui_status cui_prescreen_set_state(cui_prescreen p, const float *theta, const float *m, const float *v,
                                   int64_t step);
/* Feature standardisation, part of the network's state: every forward pass
 * (scores, training, gradients) reads x' = (x - mean_b) / std_b for the
 * features x of band b.  A new handle has mean 0 and std 1.  fit_norm sets
 * them from `count` feature rows on the device (FP64 sums of x and x^2 over
 * the count * frames values of each band; std is the population standard
 * deviation, 1 where it is zero or not finite), asynchronously; set_norm and
 * get_norm take and return host arrays of `bands` floats and synchronise
 * (set_norm: mean finite, std finite and > 0).  Not in the paper. */
cui_status cui_prescreen_fit_norm(cui_prescreen p, const float *feat_dev, int64_t count);
cui_status cui_prescreen_set_norm(cui_prescreen p, const float *mean, const float *stddev);
cui_status cui_prescreen_get_norm(cui_prescreen p, float *mean, float *stddev);
/* Ensemble scores: prob_dev[s][c] = (1/k) sum_e softmax(z_e(s))[c], the mean
 * over the k networks nets[0 .. k) (same bands, frames and regions; each with
 * its own standardisation) of their region probabilities for `count` feature
 * rows, device arrays as for cui_prescreen_scores.  Runs on nets[0]'s stream
 * in chunks of its max_batch, networks added in index order (deterministic);
 * waits for the other networks' streams first when they differ.  Not in the
 * paper. */
cui_status cui_prescreen_ensemble_scores(const cui_prescreen *nets, int32_t k, const float *feat_dev, int64_t count,
                                         float *prob_dev);
/* Filtering order from region scores, on host arrays: the n_templates bank
 * points (m1[t], m2[t] in solar masses, finite and > 0) sorted by chirp mass
 * Mc = (m1 m2)^(3/5) / (m1 + m2)^(1/5) (equal Mc: lower index first) and cut
 * into `regions` equal-count groups in increasing Mc (the first
 * n_templates mod regions groups one template longer); then the groups by
 * descending scores[0 .. regions) (finite; equal scores: lower region first),
 * the first min(top_k, regions) of them, each in increasing Mc.  Writes those
 * template indices to order_out (room for n_templates, caller-owned) and
 * their number to *n_out: the `order` argument of cui_filter_bank.  Does not
 * touch the GPU.  Errors: CUI_ERR_ARG.  Paper: the introduction's remark that
 * at the ET scale of 1-2 million templates a search should be smarter than
 * brute force; the regions and scores are this library's prescreen. */
cui_status cui_prescreen_rank(const double *m1, const double *m2, int64_t n_templates, const float *scores,
                              int32_t regions, int32_t top_k, int32_t *order_out, int64_t *n_out);

/* The same ranking with the bank's chirp-mass order computed once: create
 * keeps the bank points sorted and cut into `regions` groups (the rules of
 * cui_prescreen_rank; host arrays, copied), order writes the template order
 * of the top_k best-scored regions exactly as cui_prescreen_rank would, in
 * O(regions log regions + templates written) per call, destroy frees the plan
 * (NULL allowed).  Host only, no GPU.  Errors: CUI_ERR_ARG.  Paper: as
 * cui_prescreen_rank; the plan itself is not in the paper. */
typedef struct cui_regions_s *cui_regions;
cui_status cui_regions_create(const double *m1, const double *m2, int64_t n_templates, int32_t regions,
                              cui_regions *out);
cui_status cui_regions_order(cui_regions plan, const float *scores, int32_t top_k, int32_t *order_out,
                             int64_t *n_out);
void cui_regions_destroy(cui_regions plan);

/* Allocation-free normalisation: sigma_t^2 = 4 df sum_k |h~_k|^2 / S_k of
 * `count` templates (m1[t], m2[t], host arrays, read during the call) for the
 * one-sided PSD psd_dev (N/2 + 1 FP64 values in device memory, read on
 * [k_lo, N/2)), written to sigma2_dev[0 .. count) (device, caller-owned),
 * asynchronously on `stream`.  No counterpart in the paper: it serves callers
 * that cannot allocate device memory when they need the result -- pipelines
 * whose device memory belongs to one pool allocator with a fixed budget,
 * real-time loops that cannot wait for an allocation -- for instance to
 * renormalise a bank after a new PSD estimate.  It allocates nothing: its
 * scratch is one array of about 8.2 MiB compiled into the library, which
 * every GPU that loads the library holds until the process exits.  The first
 * call on a device looks up that array's device address (with the device
 * current); make that first call before any stream capture.  The upper bins
 * are computed on the host and copied from pageable host memory (staged
 * before the call returns).  psd_dev is not validated: it must be finite and
 * > 0 on [k_lo, N/2), or sigma^2 comes out inf or NaN with CUI_OK.  Limits: N
 * a power of two in [64, 2^20], 1 <= count <= 16384; larger values return
 * CUI_ERR_ARG.  All calls share the array: calls that overlap on the GPU
 * (other streams, other host threads) race and must be serialised by the
 * caller.  Same conventions and units as cui_bank_create;
 * k_lo = ceil(f_low / df) (capped at N/2), k_hi as there.
 * Errors: CUI_ERR_ARG, CUI_ERR_CUDA. */
cui_status cui_template_sigma_noalloc(const double *psd_dev, int64_t n, double sample_rate, double f_low,
                                      const double *m1, const double *m2, int64_t count, double *sigma2_dev,
                                      void *stream);

/* Release every resource of the handle (synchronises its stream first).
 * NULL is allowed. */
void cui_bank_destroy(cui_bank bank);

/* Message of the last failing call on this thread ("" if none); the string
 * belongs to the library and stays valid until the thread's next failing
 * call.  Not in the paper. */
const char *cui_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CUI_H */
