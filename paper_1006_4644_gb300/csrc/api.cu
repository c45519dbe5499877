// C ABI of the bank matched filter (include/cui.h): argument checking, the
// per-template constants, device buffers and the order of kernel launches.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "bands.h"
#include "internal.h"
#include "td.h"

using namespace cui;

namespace {

thread_local std::string g_err;

cui_status fail(cui_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

cui_status cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(CUI_ERR_OOM, "%s: out of device memory", what);
    }
    return fail(CUI_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CUI_TRY(call, what)                                                                                          \
    do {                                                                                                             \
        cudaError_t e_ = (call);                                                                                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);                                                           \
    } while (0)

constexpr double kMsunS = 4.925490947e-6; // G M_sun / c^3 (s)
constexpr double kEuler = 0.57721566490153286061;

bool is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }
int ilog2(int64_t n)
{
    int l = 0;
    while ((int64_t(1) << l) < n) ++l;
    return l;
}

// binom(p, n) for real p
double binom(double p, int n)
{
    double r = 1.0;
    for (int m = 0; m < n; ++m) r *= (p - m) / (m + 1);
    return r;
}

DerivConsts make_deriv_consts()
{
    const double pw[kNB] = {-5.0 / 3, -1.0, -2.0 / 3, -1.0 / 3, 0.0, 0.0, 1.0 / 3, 0.0, 2.0 / 3};
    DerivConsts dc;
    std::memset(&dc, 0, sizeof dc);
    for (int n = 1; n < 4; ++n) {
        for (int i = 0; i < kNB; ++i) {
            if (i == 4 || i == 5) dc.B[n][i] = 0.f; // constant; ln k handled by lam
            else if (i == 7) dc.B[n][i] = (float)binom(1.0 / 3, n);
            else dc.B[n][i] = (float)binom(pw[i], n);
        }
        dc.lam[n] = (float)((n % 2 ? 1.0 : -1.0) / n);
        double g = 0.0;
        for (int m = 0; m < n; ++m) g += binom(1.0 / 3, m) * (((n - m) % 2 ? 1.0 : -1.0) / (n - m));
        dc.gam[n] = (float)g;
    }
    return dc;
}

// Phase of template (m1, m2) as Phi(k) = sum_i c_i g_i(k) in cycles, with
// g = {k^-5/3, k^-1, k^-2/3, k^-1/3, 1, ln k, k^1/3, k^1/3 ln k, k^2/3}: the
// TaylorF2 phase Psi(f) = -pi/4 + 3/(128 eta v^5) sum_i alpha_i v^i at
// f = k df, v = u k^(1/3), u = (pi M df)^(1/3), with ln v expanded.
void phase_coefficients(double m1, double m2, int pn, double df, double *c)
{
    const double pi = kPi;
    const double M = (m1 + m2) * kMsunS;
    const double eta = m1 * m2 / ((m1 + m2) * (m1 + m2));
    const double P = 3.0 / (128.0 * eta);
    const double u = std::cbrt(pi * M * df);
    const double a2 = 3715.0 / 756.0 + 55.0 / 9.0 * eta;
    const double a3 = -16.0 * pi;
    const double a4 = 15293365.0 / 508032.0 + 27145.0 / 504.0 * eta + 3085.0 / 72.0 * eta * eta;
    const double A5 = pi * (38645.0 / 756.0 - 65.0 / 9.0 * eta);
    const double A6 = 11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * pi * pi - 6848.0 / 21.0 * kEuler +
                      eta * (-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * pi * pi) + 76055.0 / 1728.0 * eta * eta -
                      127825.0 / 1296.0 * eta * eta * eta;
    const double a7 = pi * (77096675.0 / 254016.0 + 378515.0 / 1512.0 * eta - 74045.0 / 756.0 * eta * eta);
    double r[kNB] = {0};
    r[0] = P * std::pow(u, -5.0);
    if (pn >= 2) r[1] = P * a2 * std::pow(u, -3.0);
    if (pn >= 3) r[2] = P * a3 * std::pow(u, -2.0);
    if (pn >= 4) r[3] = P * a4 / u;
    r[4] = -pi / 4.0;
    if (pn >= 5) {
        r[4] += P * A5 * (1.0 + 3.0 * std::log(u * std::sqrt(6.0)));
        r[5] = P * A5;
    }
    if (pn >= 6) {
        r[6] = P * u * (A6 - 6848.0 / 21.0 * std::log(4.0 * u));
        r[7] = -P * u * 6848.0 / 63.0;
    }
    if (pn >= 7) r[8] = P * a7 * u * u;
    for (int i = 0; i < kNB; ++i) c[i] = r[i] / (2.0 * pi);
}

// First bin from which the per-row cubic of the fused path is accurate: its
// remainder is dominated by the leading k^(-5/3) term,
// |binom(-5/3, 4)| |c_0| k^(-5/3) (C/2 / k)^4, kept below kExactTol cycles
// with a safety factor of 4.  Bins below it get the exact per-bin phase.
constexpr double kExactTol = 1e-6;
constexpr int kExactMax = 1 << 16;
int exact_bound(double c0, int ccols, int64_t nh)
{
    const double h = ccols / 2.0;
    const double k = std::pow(4.0 * 3.1701 * std::fabs(c0) * h * h * h * h / kExactTol, 3.0 / 17.0);
    return (int)std::min<double>(std::ceil(k), (double)std::min<int64_t>(nh, kExactMax));
}

// What a captured filter call depends on besides the buffers' contents.
struct GraphKey {
    int64_t count;
    const int32_t *order;
    const cui_peak *peaks;
    int n1, ccols, rpc, batch;
    bool operator==(const GraphKey &o) const
    {
        return count == o.count && order == o.order && peaks == o.peaks && n1 == o.n1 && ccols == o.ccols &&
               rpc == o.rpc && batch == o.batch;
    }
};

template <typename T> cudaError_t dalloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    return cudaMalloc((void **)p, count * sizeof(T));
}

} // namespace

struct cui_bank_s {
    cui_bank_desc desc;
    cudaStream_t stream = nullptr;
    int log2n = 0;
    int64_t n = 0, nh = 0, nt = 0;
    int k_low = 0;
    int band_lo = 0, band_hi = 0; // band of the filter calls: [band_lo, min(band_hi, k_hi(t)))
    double df = 0;
    bool fused = false, plain_fp64 = false;
    int nwin = 0;
    // per template
    std::vector<int32_t> h_khi;     // k_hi(t): first bin at or above f_isco, capped at N/2
    std::vector<int32_t> h_khi_eff; // min(k_hi(t), band_hi), the copy behind d_khi
    int32_t *d_khi0 = nullptr;      // k_hi(t)
    double *d_coef = nullptr;
    float2 *d_coef_df = nullptr;
    double *d_mass = nullptr;
    int32_t *d_khi = nullptr;
    double *d_sigma2 = nullptr;
    float *d_invnorm = nullptr;
    Slot *d_peak = nullptr;
    cui_peak *d_peaks = nullptr;
    int32_t *d_iota = nullptr;
    // segment
    double *d_strain = nullptr, *d_psd = nullptr, *d_amp = nullptr, *d_prefix = nullptr, *d_scan = nullptr;
    double2 *d_fa = nullptr, *d_fb = nullptr;
    const double2 *d_X = nullptr; // which of d_fa / d_fb holds the segment transform
    float2 *d_wbar = nullptr;
    void *d_dS = nullptr;
    SegScales *d_scales = nullptr;
    Twiddles tw = {nullptr, nullptr, nullptr, nullptr, 0, 0};
    // fused
    int n1 = 0, n2 = 0, ccols = 0, rpc = 0, batch = 0;
    double *d_basis = nullptr;
    float2 *d_basis_df = nullptr;
    int32_t *d_kex = nullptr;
    float2 *d_gexact = nullptr;
    std::vector<int32_t> h_kex;
    // anchors and exact-phase bounds of the chi^2 and band-sum kernels: blocks
    // of pf_ccols bins (the filter's own tables when its ccols is that width)
    double *d_basis_pf = nullptr;
    float2 *d_basis_df_pf = nullptr;
    int32_t *d_kex_pf = nullptr;
    int pf_ccols = 0;
    std::vector<int32_t> h_kex_pf;
    std::vector<double> h_c0;   // leading phase coefficient of every template
    std::vector<double> h_mass; // (M in seconds, eta) of every template
    int kx = 0;
    void *d_y = nullptr;
    Slot *d_win = nullptr;
    Slot *d_prec = nullptr; // [batch][n1 / 2] peak records of the streamed pass 2 (tiling rpc 0)
    // plain
    void *d_h = nullptr, *d_qa = nullptr, *d_qb = nullptr;
    double *d_acc = nullptr;
    Slot *d_pwin = nullptr;
    Slot *d_cluster = nullptr; // [nwin] loudest trigger of each window over the bank (last filter call)
    bool filtered = false;     // a filter call ran since the last upload
    int cas_rounds = kCasRounds;                // bounds of the device waits
    unsigned long long copy_wait_ns = kCopyWaitNs;
    // outputs
    cui_trigger *d_trig = nullptr;
    int64_t trig_cap = 0;
    unsigned long long *d_trig_count = nullptr;
    int *d_err = nullptr;
    struct Stage {
        int err, pad;
        unsigned long long trig_count;
        unsigned long long psd_bad; // first bad PSD bin of the last host upload, ~0 if none
    } *h_stage = nullptr;           // pinned: read back with one synchronisation
    unsigned long long *d_psd_bad = nullptr;
    cudaEvent_t ev_psd = nullptr;
    // pinned read-out staging: the peaks, and a prefix of the trigger records
    // sized from the previous count, copied in the same synchronisation
    cui_peak *h_peaks = nullptr;
    cui_trigger *h_trig = nullptr;
    int64_t h_trig_cap = 0, trig_hint = 1024;
    int32_t *d_order = nullptr;
    int64_t order_cap = 0;
    bool have_segment = false, have_peaks = false;
    // CUDA graph of the last fused filter call and its signature; the capture
    // forks onto a second stream so that pass 1 of a batch overlaps pass 2 of
    // the previous one (two Y buffers, events fork / p1[2] / p2[2] / join)
    cudaStream_t cap_stream = nullptr, cap_stream2 = nullptr;
    cudaEvent_t gev[6] = {};
    int ny = 1; // Y buffers: 2 when a call can hold more than one batch
    GraphKey gkey = {};
    cudaGraphExec_t gexec = nullptr;
    long long glaunches = 0;
    // tracing: (group, start, stop, launches) per recorded interval
    int trace = 0; // 0 off, 1 call groups, 2 every kernel group
    struct Mark {
        int group;
        cudaEvent_t a, b;
        long long launches;
    };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> pool;
};

namespace cui {
std::atomic<long long> g_launches{0};
void set_last_error(const char *msg) { g_err = msg; }

bool bank_segment_spectrum(cui_bank b, const double2 **X, const double **psd, int64_t *n, double *fs)
{
    if (!b || !b->have_segment || !b->d_X) return false;
    *X = b->d_X;
    *psd = b->d_psd;
    *n = b->n;
    *fs = b->desc.sample_rate;
    return true;
}
} // namespace cui

namespace {
const char *const kGroups[] = {"segment", "pass1", "pass2", "finalize", "plain", "graph"};
constexpr int kNGroups = 6;

cudaEvent_t take_event(cui_bank b)
{
    if (!b->pool.empty()) {
        cudaEvent_t e = b->pool.back();
        b->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Opens a traced interval of `group` on the bank's stream when the tracing
// level is at least `level`; close() ends it.  Per-kernel groups use level 2,
// at which the fused path launches directly (a graph could not hold events
// of the bank's own stream).
struct Span {
    cui_bank b;
    int group;
    cudaEvent_t a = nullptr;
    long long l0 = 0;
    Span(cui_bank b_, int g, int level = 1) : b(b_), group(g)
    {
        if (b->trace < level) return;
        a = take_event(b);
        l0 = g_launches.load();
        cudaEventRecord(a, b->stream);
    }
    void close()
    {
        if (!a) return;
        cudaEvent_t e = take_event(b);
        cudaEventRecord(e, b->stream);
        b->marks.push_back({group, a, e, g_launches.load() - l0});
        a = nullptr;
    }
    ~Span() { close(); }
};
} // namespace

static void release(cui_bank b)
{
    void *ptrs[] = {b->d_coef, b->d_coef_df, b->d_mass, b->d_khi, b->d_khi0, b->d_sigma2, b->d_invnorm, b->d_peak, b->d_peaks,
                    b->d_iota, b->d_strain, b->d_psd, b->d_amp, b->d_prefix, b->d_scan, b->d_fa, b->d_fb,
                    b->tw.lo64, b->tw.hi64, b->tw.lo32, b->tw.hi32, b->tw.lodf, b->tw.hidf,
                    b->d_wbar, b->d_dS, b->d_scales, b->d_basis, b->d_basis_df, b->d_kex, b->d_gexact, b->d_y,
                    b->d_win, b->d_prec, b->d_h, b->d_qa, b->d_qb, b->d_acc, b->d_pwin, b->d_cluster, b->d_trig, b->d_trig_count, b->d_err,
                    b->d_order, b->d_psd_bad};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (b->d_basis_pf != b->d_basis) cudaFree(b->d_basis_pf);
    if (b->d_basis_df_pf != b->d_basis_df) cudaFree(b->d_basis_df_pf);
    if (b->d_kex_pf != b->d_kex) cudaFree(b->d_kex_pf);
    for (auto &m : b->marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    for (cudaEvent_t e : b->pool) cudaEventDestroy(e);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->cap_stream2) cudaStreamDestroy(b->cap_stream2);
    for (cudaEvent_t ev : b->gev)
        if (ev) cudaEventDestroy(ev);
    if (b->h_stage) cudaFreeHost(b->h_stage);
    if (b->h_peaks) cudaFreeHost(b->h_peaks);
    if (b->h_trig) cudaFreeHost(b->h_trig);
    if (b->ev_psd) cudaEventDestroy(b->ev_psd);
}

extern "C" const char *cui_last_error(void) { return g_err.c_str(); }

constexpr int kPostCols = 32; // anchor block of the chi^2 and band-sum kernels

// One anchor table (blocks of ccols bins below N/2) and its exact-phase bounds.
static cudaError_t build_anchor_set(cui_bank b, int n1, int n2, int ccols, const std::vector<int32_t> &kex,
                                    double **basis, float2 **basis_df, int32_t **d_kex)
{
    const int64_t na = (int64_t)(n1 / 2) * (n2 / ccols);
    cudaError_t e;
    if ((e = dalloc(basis, na * kNB)) != cudaSuccess) return e;
    if ((e = dalloc(basis_df, na * kNB)) != cudaSuccess) return e;
    if ((e = dalloc(d_kex, b->nt)) != cudaSuccess) return e;
    launch_basis_table(*basis, *basis_df, n1, n2, ccols, b->stream);
    return cudaMemcpyAsync(*d_kex, kex.data(), sizeof(int32_t) * b->nt, cudaMemcpyHostToDevice, b->stream);
}

// Anchor basis table, per-template exact-phase bounds and the per-bin exact
// table for a tiling (n1 rows, ccols columns per pass-1 CTA), and the tables
// of the chi^2 and band-sum kernels.  Synchronous.
static cudaError_t build_phase_tables(cui_bank b, int n1, int ccols)
{
    const cudaStream_t s = b->stream;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (b->gexec) { // the captured graph refers to the buffers replaced here
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    if (b->d_basis_pf != b->d_basis) cudaFree(b->d_basis_pf);
    if (b->d_basis_df_pf != b->d_basis_df) cudaFree(b->d_basis_df_pf);
    if (b->d_kex_pf != b->d_kex) cudaFree(b->d_kex_pf);
    b->d_basis_pf = nullptr;
    b->d_basis_df_pf = nullptr;
    b->d_kex_pf = nullptr;
    for (void *p : {(void *)b->d_basis, (void *)b->d_basis_df, (void *)b->d_kex, (void *)b->d_gexact})
        if (p) cudaFree(p);
    b->d_basis = nullptr;
    b->d_basis_df = nullptr;
    b->d_kex = nullptr;
    b->d_gexact = nullptr;
    const int n2 = (int)(b->n / n1);
    // the chi^2 and band-sum kernels evaluate one anchor per block of bins, a
    // larger share of their work than of pass 1's: they use blocks of
    // kPostCols bins whatever the filter's tiling
    const int pf = (ccols != kPostCols && n2 % kPostCols == 0) ? kPostCols : ccols;
    b->pf_ccols = pf;
    b->h_kex.resize(b->nt);
    b->h_kex_pf.resize(b->nt);
    b->kx = 0;
    for (int64_t t = 0; t < b->nt; ++t) {
        b->h_kex[t] = exact_bound(b->h_c0[t], ccols, b->nh);
        b->h_kex_pf[t] = exact_bound(b->h_c0[t], pf, b->nh);
        b->kx = std::max(b->kx, std::max(b->h_kex[t], b->h_kex_pf[t])); // one exact table serves both
    }
    if ((e = build_anchor_set(b, n1, n2, ccols, b->h_kex, &b->d_basis, &b->d_basis_df, &b->d_kex)) != cudaSuccess)
        return e;
    if (pf == ccols) {
        b->d_basis_pf = b->d_basis;
        b->d_basis_df_pf = b->d_basis_df;
        b->d_kex_pf = b->d_kex;
    } else if ((e = build_anchor_set(b, n1, n2, pf, b->h_kex_pf, &b->d_basis_pf, &b->d_basis_df_pf, &b->d_kex_pf)) !=
               cudaSuccess) {
        return e;
    }
    if ((e = dalloc(&b->d_gexact, (int64_t)std::max(1, b->kx) * kNB)) != cudaSuccess) return e;
    launch_exact_table(b->d_gexact, b->kx, s);
    fused_set_consts(make_deriv_consts(), s);
    return cudaStreamSynchronize(s);
}

// Select a tiling of the fused path and (re)allocate what depends on it.
static cudaError_t configure_fused(cui_bank b, const cui_tuning &tu)
{
    if (!fused_tiling_ok(b->log2n, tu.n1, tu.ccols, tu.rpc) || tu.batch < 1) return cudaErrorInvalidValue;
    const cudaStream_t s = b->stream;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    if (b->d_y) cudaFree(b->d_y);
    if (b->d_win) cudaFree(b->d_win);
    if (b->d_prec) cudaFree(b->d_prec);
    b->d_y = nullptr;
    b->d_win = nullptr;
    b->d_prec = nullptr;
    b->n1 = tu.n1;
    b->n2 = (int)(b->n / tu.n1);
    b->ccols = tu.ccols;
    b->rpc = tu.rpc;
    b->batch = (int)std::min<int64_t>(tu.batch, b->nt);
    const size_t per = (size_t)b->n * ((b->desc.flags & CUI_STORE_BF16) ? 4 : 8);
    b->ny = b->nt > b->batch ? 2 : 1;
    if ((e = cudaMalloc(&b->d_y, per * (size_t)b->batch * b->ny)) != cudaSuccess) return e;
    if ((e = dalloc(&b->d_win, (int64_t)b->batch * std::max(1, b->nwin))) != cudaSuccess) return e;
    if (tu.rpc == 0 &&
        (e = dalloc(&b->d_prec, (int64_t)b->batch * fused_records_per_template(tu.n1, b->n2))) != cudaSuccess)
        return e;
    e = cudaMemsetAsync(b->d_win, 0, sizeof(Slot) * (size_t)b->batch * std::max(1, b->nwin), s);
    if (e != cudaSuccess) return e;
    return build_phase_tables(b, tu.n1, tu.ccols);
}

extern "C" cui_status cui_bank_create(const cui_bank_desc *desc, const double *m1, const double *m2,
                                      int64_t n_templates, cui_bank *out)
{
    if (!out) return fail(CUI_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!desc || !m1 || !m2) return fail(CUI_ERR_ARG, "desc, m1 and m2 must be non-NULL");
    const cui_bank_desc &d = *desc;
    if (!is_pow2(d.n) || d.n < 64 || d.n > (int64_t(1) << 22))
        return fail(CUI_ERR_ARG, "n = %lld must be a power of two in [2^6, 2^22]", (long long)d.n);
    if (d.pn_order_x2 < 0 || d.pn_order_x2 > 7) return fail(CUI_ERR_ARG, "pn_order_x2 must be in 0..7");
    if (d.reserved0 != 0 || d.reserved1 != 0) return fail(CUI_ERR_ARG, "reserved fields must be 0");
    if (!(d.sample_rate > 0) || !std::isfinite(d.sample_rate)) return fail(CUI_ERR_ARG, "sample_rate must be > 0");
    if (!(d.f_low > 0) || !std::isfinite(d.f_low)) return fail(CUI_ERR_ARG, "f_low must be > 0");
    if (d.window < 1) return fail(CUI_ERR_ARG, "window must be >= 1");
    if (d.valid_lo < 0 || d.valid_hi < d.valid_lo || d.valid_hi > d.n)
        return fail(CUI_ERR_ARG, "need 0 <= valid_lo <= valid_hi <= n");
    if (!std::isfinite(d.snr_threshold) || d.snr_threshold < 0) return fail(CUI_ERR_ARG, "snr_threshold must be >= 0");
    if (d.trigger_capacity < 0) return fail(CUI_ERR_ARG, "trigger_capacity must be >= 0");
    if (d.flags & ~(CUI_PSI_FP64 | CUI_STORE_BF16 | CUI_PLAIN | CUI_PLAIN_FP64 | CUI_NO_GRAPH))
        return fail(CUI_ERR_ARG, "unknown flags");
    if (n_templates < 1 || n_templates > (int64_t(1) << 31) - 1) return fail(CUI_ERR_ARG, "n_templates out of range");
    for (int64_t i = 0; i < n_templates; ++i)
        if (!(m1[i] > 0) || !(m2[i] > 0) || !std::isfinite(m1[i]) || !std::isfinite(m2[i]))
            return fail(CUI_ERR_ARG, "template %lld: masses must be finite and > 0", (long long)i);

    cui_bank b = new cui_bank_s();
    b->desc = d;
    b->stream = (cudaStream_t)d.stream;
    b->n = d.n;
    b->nh = d.n / 2;
    b->log2n = ilog2(d.n);
    b->nt = n_templates;
    b->df = d.sample_rate / (double)d.n;
    // clamped before the conversion: an f_low at or above Nyquist leaves every band empty
    b->k_low = band_k_low(d.f_low, b->df, b->nh);
    b->band_lo = b->k_low;
    b->band_hi = (int)(d.n / 2);
    b->fused = !(d.flags & CUI_PLAIN) && fused_supported(b->log2n);
    b->plain_fp64 = (d.flags & CUI_PLAIN) && (d.flags & CUI_PLAIN_FP64);
    b->nwin = (int)((d.valid_hi - d.valid_lo + d.window - 1) / d.window);
    b->trig_cap = d.trigger_capacity ? d.trigger_capacity : (int64_t(1) << 20);
    const int64_t nt = n_templates;
    const int pn = d.pn_order_x2;

    // per-template constants on the host
    std::vector<double> coef(nt * kNB), mass(2 * nt);
    std::vector<float2> coef_df(nt * kNB);
    std::vector<int32_t> iota(nt);
    b->h_khi.resize(nt);
    for (int64_t t = 0; t < nt; ++t) {
        const double M = (m1[t] + m2[t]) * kMsunS;
        b->h_khi[t] = band_k_hi(m1[t], m2[t], b->df, b->nh);
        phase_coefficients(m1[t], m2[t], pn, b->df, &coef[t * kNB]);
        for (int i = 0; i < kNB; ++i) {
            const double c = coef[t * kNB + i];
            const float hi = (float)c;
            coef_df[t * kNB + i] = make_float2(hi, (float)(c - (double)hi));
        }
        mass[2 * t] = M;
        mass[2 * t + 1] = m1[t] * m2[t] / ((m1[t] + m2[t]) * (m1[t] + m2[t]));
        iota[t] = (int32_t)t;
    }

    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) {
        if (e == cudaSuccess && x != cudaSuccess) e = x;
    };
    const cudaStream_t s = b->stream;
    chk(dalloc(&b->d_coef, nt * kNB));
    chk(dalloc(&b->d_coef_df, nt * kNB));
    chk(dalloc(&b->d_mass, 2 * nt));
    chk(dalloc(&b->d_khi, nt));
    chk(dalloc(&b->d_khi0, nt));
    chk(dalloc(&b->d_sigma2, nt));
    chk(dalloc(&b->d_invnorm, nt));
    chk(dalloc(&b->d_peak, nt));
    chk(dalloc(&b->d_peaks, nt));
    chk(dalloc(&b->d_iota, nt));
    chk(dalloc(&b->d_strain, b->n));
    chk(dalloc(&b->d_psd, b->nh + 1));
    chk(dalloc(&b->d_amp, b->nh));
    chk(dalloc(&b->d_prefix, b->nh + 1));
    chk(dalloc(&b->d_scan, (b->nh + 1) / 2048 + 2));
    chk(dalloc(&b->d_fa, b->n));
    chk(dalloc(&b->d_fb, b->n));
    chk(dalloc(&b->d_wbar, b->nh));
    chk(dalloc(&b->d_scales, 1));
    b->tw.log2n = b->log2n;
    b->tw.shift = (b->log2n + 1) / 2;
    chk(dalloc(&b->tw.lo64, int64_t(1) << b->tw.shift));
    chk(dalloc(&b->tw.hi64, int64_t(1) << (b->log2n - b->tw.shift)));
    chk(dalloc(&b->tw.lo32, int64_t(1) << b->tw.shift));
    chk(dalloc(&b->tw.hi32, int64_t(1) << (b->log2n - b->tw.shift)));
    chk(dalloc(&b->tw.lodf, int64_t(1) << b->tw.shift));
    chk(dalloc(&b->tw.hidf, int64_t(1) << (b->log2n - b->tw.shift)));
    chk(dalloc(&b->d_trig, b->trig_cap));
    chk(dalloc(&b->d_trig_count, 1));
    chk(dalloc(&b->d_cluster, std::max(1, b->nwin)));
    chk(dalloc(&b->d_err, 1));
    chk(cudaMallocHost(&b->h_stage, sizeof(*b->h_stage)));
    chk(cudaMallocHost(&b->h_peaks, sizeof(cui_peak) * nt));
    chk(dalloc(&b->d_psd_bad, 1));
    chk(cudaEventCreateWithFlags(&b->ev_psd, cudaEventDisableTiming));
    chk(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    chk(cudaStreamCreateWithFlags(&b->cap_stream2, cudaStreamNonBlocking));
    for (cudaEvent_t &ev : b->gev) chk(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    b->h_c0.resize(nt);
    for (int64_t t = 0; t < nt; ++t) b->h_c0[t] = coef[t * kNB];
    if (b->fused) {
        // tiling and its buffers are set up after the constants are on the device
    } else {
        const size_t rs = b->plain_fp64 ? sizeof(double2) : sizeof(float2);
        chk(cudaMalloc(&b->d_dS, rs * b->nh));
        chk(cudaMalloc(&b->d_h, rs * b->nh));
        chk(cudaMalloc(&b->d_qa, rs * b->n));
        chk(cudaMalloc(&b->d_qb, rs * b->n));
        chk(dalloc(&b->d_acc, 1));
        chk(dalloc(&b->d_pwin, std::max(1, b->nwin)));
    }
    if (e != cudaSuccess) {
        release(b);
        delete b;
        return cuda_fail(e, "cui_bank_create");
    }
    chk(cudaMemcpyAsync(b->d_coef, coef.data(), sizeof(double) * nt * kNB, cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(b->d_coef_df, coef_df.data(), sizeof(float2) * nt * kNB, cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(b->d_mass, mass.data(), sizeof(double) * 2 * nt, cudaMemcpyHostToDevice, s));
    b->h_mass = mass;
    chk(cudaMemcpyAsync(b->d_khi, b->h_khi.data(), sizeof(int32_t) * nt, cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(b->d_khi0, b->h_khi.data(), sizeof(int32_t) * nt, cudaMemcpyHostToDevice, s));
    b->h_khi_eff = b->h_khi;
    chk(cudaMemcpyAsync(b->d_iota, iota.data(), sizeof(int32_t) * nt, cudaMemcpyHostToDevice, s));
    chk(cudaMemsetAsync(b->d_peak, 0, sizeof(Slot) * nt, s));
    chk(cudaMemsetAsync(b->d_err, 0, sizeof(int), s));
    chk(cudaMemsetAsync(b->d_trig_count, 0, sizeof(unsigned long long), s));
    launch_amp_table(b->d_amp, b->nh, s);
    launch_twiddle_tables(b->tw, s);
    if (b->fused) {
        cui_tuning tu;
        fused_default_tiling(b->log2n, &tu.n1, &tu.ccols, &tu.rpc);
        const int64_t per = b->n * ((d.flags & CUI_STORE_BF16) ? 4 : 8);
        tu.batch = (int32_t)std::min<int64_t>(nt, std::max<int64_t>(1, std::min<int64_t>(4096, (1ll << 31) / per)));
        chk(configure_fused(b, tu));
    } else {
        chk(cudaMemsetAsync(b->d_pwin, 0, sizeof(Slot) * std::max(1, b->nwin), s));
    }
    chk(cudaGetLastError());
    // the host vectors above are pageable: wait for their copies before they go
    chk(cudaStreamSynchronize(s));
    if (e != cudaSuccess) {
        release(b);
        delete b;
        return cuda_fail(e, "cui_bank_create");
    }
    *out = b;
    return CUI_OK;
}

extern "C" void cui_bank_destroy(cui_bank b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    release(b);
    delete b;
}

extern "C" cui_status cui_segment_upload(cui_bank b, const double *strain, int64_t n, const double *psd,
                                         int64_t n_psd, int on_device)
{
    if (!b) return fail(CUI_ERR_ARG, "bank is NULL");
    if (!strain || !psd) return fail(CUI_ERR_ARG, "strain and psd must be non-NULL");
    if (n != b->n) return fail(CUI_ERR_ARG, "n = %lld differs from the bank's %lld", (long long)n, (long long)b->n);
    if (n_psd != b->nh + 1) return fail(CUI_ERR_ARG, "n_psd must be N/2 + 1 = %lld", (long long)(b->nh + 1));
    const cudaStream_t s = b->stream;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    // Everything is queued before the host waits: a host PSD is checked on the
    // device (one pass over the band) and the host waits for that check only,
    // while the GPU goes on with the weighting queued behind it.
    CUI_TRY(cudaMemcpyAsync(b->d_strain, strain, sizeof(double) * b->n, kind, s), "strain copy");
    Span span(b, 0);
    double2 *X = nullptr;
    launch_segment_transform_df(b->d_strain, b->d_fa, b->d_fb, b->log2n, b->tw, s, &X);
    CUI_TRY(cudaMemcpyAsync(b->d_psd, psd, sizeof(double) * (b->nh + 1), kind, s), "psd copy");
    if (!on_device) {
        CUI_TRY(cudaMemsetAsync(b->d_psd_bad, 0xFF, sizeof(unsigned long long), s), "psd check");
        launch_psd_check(b->d_psd, b->k_low, b->nh, b->d_psd_bad, s);
        CUI_TRY(cudaMemcpyAsync(&b->h_stage->psd_bad, b->d_psd_bad, sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, s),
                "psd check");
        CUI_TRY(cudaEventRecord(b->ev_psd, s), "psd check");
    }
    b->d_X = X;
    launch_segment_weights(X, b->d_psd, b->d_amp, b->n, b->k_low, b->desc.sample_rate, b->d_scales, b->d_wbar,
                           b->d_dS, b->plain_fp64, b->d_prefix, b->d_scan, s);
    launch_template_norm(b->d_prefix, b->d_khi, b->band_lo, b->nt, b->desc.sample_rate, b->n, b->d_scales,
                         b->d_sigma2, b->d_invnorm, s);
    CUI_TRY(cudaGetLastError(), "cui_segment_upload");
    if (!on_device) {
        CUI_TRY(cudaEventSynchronize(b->ev_psd), "psd check");
        const unsigned long long k = b->h_stage->psd_bad;
        if (k != ~0ull) {
            b->have_segment = false; // the data queued above replaced the previous segment's
            return fail(CUI_ERR_ARG, "psd[%llu] must be finite and > 0 in the band", k);
        }
    }
    b->have_segment = true;
    b->filtered = false;
    return CUI_OK;
}

static FusedArgs fused_args(cui_bank b, const int32_t *order, int64_t base)
{
    FusedArgs a;
    a.wbar = b->d_wbar;
    a.coef = b->d_coef;
    a.coef_df = b->d_coef_df;
    a.basis = b->d_basis;
    a.basis_df = b->d_basis_df;
    a.khi = b->d_khi;
    a.kex = b->d_kex;
    a.gexact = b->d_gexact;
    a.invnorm = b->d_invnorm;
    a.k_low = b->band_lo;
    a.order = order;
    a.base = base;
    a.ywork = b->d_y;
    a.peak = b->d_peak;
    a.prec = b->d_prec;
    a.nrec = b->n1 > 0 ? fused_records_per_template(b->n1, b->n2) : 0;
    a.win = b->d_win;
    a.err = b->d_err;
    a.cas_rounds = b->cas_rounds;
    a.copy_wait_ns = b->copy_wait_ns;
    a.n = b->n;
    a.log2n = b->log2n;
    a.n1 = b->n1;
    a.n2 = b->n2;
    a.ccols = b->ccols;
    a.rpc = b->rpc;
    a.lo = b->desc.valid_lo;
    a.hi = b->desc.valid_hi;
    a.window = b->desc.window;
    a.nwin = b->nwin;
    a.thr2 = (float)(b->desc.snr_threshold * b->desc.snr_threshold);
    a.fp64 = (b->desc.flags & CUI_PSI_FP64) != 0;
    a.bf16 = (b->desc.flags & CUI_STORE_BF16) != 0;
    return a;
}

// The arguments of the chi^2 and band-sum kernels: the filter's, with the
// anchors of their own block width.
static FusedArgs fused_args_post(cui_bank b)
{
    FusedArgs a = fused_args(b, b->d_iota, 0);
    a.basis = b->d_basis_pf;
    a.basis_df = b->d_basis_df_pf;
    a.kex = b->d_kex_pf;
    a.ccols = b->pf_ccols;
    return a;
}

// Zero the outputs that one filter call accumulates: the trigger count and the
// bank-wide window slots.
static cudaError_t reset_call_outputs(cui_bank b, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(b->d_trig_count, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_cluster, 0, sizeof(Slot) * std::max(1, b->nwin), s);
    return e;
}

static FinalizeArgs finalize_args(cui_bank b, const int32_t *d_ord, cui_peak *pout)
{
    FinalizeArgs fa;
    fa.order = d_ord;
    fa.peak = b->d_peak;
    fa.prec = b->fused && b->rpc == 0 ? b->d_prec : nullptr; // the streamed pass 2 writes records
    fa.nrec = b->n1 > 0 ? fused_records_per_template(b->n1, b->n2) : 0;
    fa.win = b->d_win;
    fa.nwin = b->nwin;
    fa.lo = b->desc.valid_lo;
    fa.window = b->desc.window;
    fa.peaks_out = pout;
    fa.trig = b->d_trig;
    fa.trig_cap = b->trig_cap;
    fa.trig_count = b->d_trig_count;
    fa.cluster = b->d_cluster;
    fa.err = b->d_err;
    fa.cas_rounds = b->cas_rounds;
    fa.base = 0;
    fa.count = 0;
    return fa;
}

// The fused path's launches for `count` templates: per batch, pass 1,
// pass 2 and the finalize kernels.
static cudaError_t enqueue_fused(cui_bank b, const int32_t *d_ord, int64_t count, cui_peak *pout, cudaStream_t s)
{
    FinalizeArgs fa = finalize_args(b, d_ord, pout);
    for (int64_t base = 0; base < count; base += b->batch) {
        const int bc = (int)std::min<int64_t>(b->batch, count - base);
        FusedArgs a = fused_args(b, d_ord, base);
        cudaError_t e;
        {
            Span sp(b, 1, 2);
            if ((e = launch_pass1(a, bc, s)) != cudaSuccess) return e;
        }
        {
            Span sp(b, 2, 2);
            if ((e = launch_pass2(a, bc, s)) != cudaSuccess) return e;
        }
        fa.base = base;
        fa.count = bc;
        Span sp(b, 3, 2);
        if ((e = launch_finalize(fa, s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The same with pass 1 of batch i on stream sa and pass 2 + finalize on sb:
// pass 1 of batch i + 1 runs while pass 2 of batch i reads the other Y
// buffer.  Only under graph capture (the events order the two streams).
static cudaError_t enqueue_fused_overlap(cui_bank b, const int32_t *d_ord, int64_t count, cui_peak *pout,
                                         cudaStream_t sa, cudaStream_t sb)
{
    FinalizeArgs fa = finalize_args(b, d_ord, pout);
    cudaEvent_t fork = b->gev[0], join = b->gev[1], *p1 = b->gev + 2, *p2 = b->gev + 4;
    const size_t slice = (size_t)b->n * ((b->desc.flags & CUI_STORE_BF16) ? 4 : 8) * (size_t)b->batch;
    cudaError_t e;
    if ((e = cudaEventRecord(fork, sa)) != cudaSuccess || (e = cudaStreamWaitEvent(sb, fork, 0)) != cudaSuccess)
        return e;
    int i = 0;
    for (int64_t base = 0; base < count; base += b->batch, ++i) {
        const int bc = (int)std::min<int64_t>(b->batch, count - base);
        FusedArgs a = fused_args(b, d_ord, base);
        a.ywork = (char *)b->d_y + (size_t)(i & 1) * slice;
        if (i >= 2 && (e = cudaStreamWaitEvent(sa, p2[i & 1], 0)) != cudaSuccess) return e; // batch i-2 has read it
        if ((e = launch_pass1(a, bc, sa)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(p1[i & 1], sa)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(sb, p1[i & 1], 0)) != cudaSuccess) return e;
        if ((e = launch_pass2(a, bc, sb)) != cudaSuccess) return e;
        fa.base = base;
        fa.count = bc;
        if ((e = launch_finalize(fa, sb)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(p2[i & 1], sb)) != cudaSuccess) return e;
    }
    if ((e = cudaEventRecord(join, sb)) != cudaSuccess) return e;
    return cudaStreamWaitEvent(sa, join, 0);
}

extern "C" cui_status cui_filter_bank(cui_bank b, const int32_t *order, int64_t count, cui_peak *peaks_dev)
{
    if (!b) return fail(CUI_ERR_ARG, "bank is NULL");
    if (!b->have_segment) return fail(CUI_ERR_STATE, "no segment uploaded");
    if (count < 0 || count > b->nt) return fail(CUI_ERR_ARG, "count must be in [0, n_templates]");
    if (!order && count != b->nt) return fail(CUI_ERR_ARG, "order == NULL requires count == n_templates");
    const cudaStream_t s = b->stream;
    const int32_t *d_ord = b->d_iota;
    if (order) {
        std::vector<uint8_t> seen(b->nt, 0);
        for (int64_t i = 0; i < count; ++i) {
            if (order[i] < 0 || order[i] >= b->nt)
                return fail(CUI_ERR_ARG, "order[%lld] = %d out of range", (long long)i, order[i]);
            if (seen[order[i]]++) return fail(CUI_ERR_ARG, "order lists template %d twice", order[i]);
        }
        if (count > b->order_cap) {
            if (b->d_order) cudaFree(b->d_order);
            b->d_order = nullptr;
            b->order_cap = 0;
            CUI_TRY(dalloc(&b->d_order, count), "order buffer");
            b->order_cap = count;
        }
        if (count) CUI_TRY(cudaMemcpyAsync(b->d_order, order, sizeof(int32_t) * count, cudaMemcpyHostToDevice, s),
                           "order copy");
        d_ord = b->d_order;
    }
    cui_peak *pout = peaks_dev ? peaks_dev : b->d_peaks;
    if (b->fused && b->trace < 2 && !(b->desc.flags & CUI_NO_GRAPH) && count > 0) {
        // The whole call as one CUDA graph: captured once per signature on the
        // bank's private stream, replayed on the caller's stream.
        const GraphKey key = {count, d_ord, pout, b->n1, b->ccols, b->rpc, b->batch};
        if (!b->gexec || !(b->gkey == key)) {
            if (b->gexec) cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
            const long long l0 = g_launches.load();
            CUI_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal), "graph capture");
            cudaError_t e1 = reset_call_outputs(b, b->cap_stream);
            cudaError_t e2 = e1;
            if (e1 == cudaSuccess)
                e2 = b->ny > 1 && count > b->batch
                         ? enqueue_fused_overlap(b, d_ord, count, pout, b->cap_stream, b->cap_stream2)
                         : enqueue_fused(b, d_ord, count, pout, b->cap_stream);
            cudaGraph_t graph = nullptr;
            cudaError_t e3 = cudaStreamEndCapture(b->cap_stream, &graph);
            if (e2 != cudaSuccess || e3 != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return cuda_fail(e2 != cudaSuccess ? e2 : e3, "graph capture");
            }
            cudaError_t e4 = cudaGraphInstantiate(&b->gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (e4 != cudaSuccess) {
                b->gexec = nullptr;
                return cuda_fail(e4, "graph instantiate");
            }
            b->gkey = key;
            b->glaunches = g_launches.load() - l0;
            g_launches.fetch_sub(b->glaunches); // counted when replayed
        }
        Span sp(b, 5);
        CUI_TRY(cudaGraphLaunch(b->gexec, s), "graph launch");
        launched((int)b->glaunches);
    } else if (b->fused) {
        CUI_TRY(reset_call_outputs(b, s), "trigger reset");
        CUI_TRY(enqueue_fused(b, d_ord, count, pout, s), "fused filter");
    } else {
        CUI_TRY(reset_call_outputs(b, s), "trigger reset");
        FinalizeArgs fa = finalize_args(b, d_ord, pout);
        PlainArgs a;
        a.mass = b->d_mass;
        a.khi = b->d_khi;
        a.amp = b->d_amp;
        a.psd = b->d_psd;
        a.dS = b->d_dS;
        a.scales = b->d_scales;
        a.tw = b->tw;
        a.h = b->d_h;
        a.qa = b->d_qa;
        a.qb = b->d_qb;
        a.acc = b->d_acc;
        a.peak = b->d_peak;
        a.win = b->d_pwin;
        a.err = b->d_err;
        a.cas_rounds = b->cas_rounds;
        a.n = b->n;
        a.log2n = b->log2n;
        a.pn_x2 = b->desc.pn_order_x2;
        a.k_low = b->band_lo;
        a.fs = b->desc.sample_rate;
        a.lo = b->desc.valid_lo;
        a.hi = b->desc.valid_hi;
        a.window = b->desc.window;
        a.nwin = b->nwin;
        a.thr2 = (float)(b->desc.snr_threshold * b->desc.snr_threshold);
        a.fp64 = b->plain_fp64;
        fa.win = b->d_pwin;
        fa.count = 1;
        for (int64_t pos = 0; pos < count; ++pos) {
            const int t = order ? order[pos] : (int)pos;
            Span sp(b, 4);
            CUI_TRY(launch_plain_template(a, t, s), "plain filter");
            fa.base = pos;
            CUI_TRY(launch_finalize(fa, s), "finalize");
        }
    }
    b->have_peaks = peaks_dev == nullptr;
    b->filtered = true;
    return CUI_OK;
}

extern "C" cui_status cui_bank_set_wait_bounds(cui_bank b, int64_t cas_rounds, int64_t copy_wait_ns)
{
    if (!b) return fail(CUI_ERR_ARG, "bank is NULL");
    if (cas_rounds > kCasRounds || copy_wait_ns > (int64_t)kCopyWaitNs)
        return fail(CUI_ERR_ARG, "bounds above the defaults (%d rounds, %llu ns) are not allowed", kCasRounds,
                    (unsigned long long)kCopyWaitNs);
    CUI_TRY(cudaStreamSynchronize(b->stream), "stream synchronize");
    b->cas_rounds = cas_rounds < 0 ? kCasRounds : (int)cas_rounds;
    b->copy_wait_ns = copy_wait_ns < 0 ? kCopyWaitNs : (unsigned long long)copy_wait_ns;
    if (b->gexec) { // the captured graph holds the previous bounds
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    return CUI_OK;
}

extern "C" cui_status cui_bank_get_tuning(cui_bank b, cui_tuning *out)
{
    if (!b || !out) return fail(CUI_ERR_ARG, "bank and out must be non-NULL");
    if (!b->fused) return fail(CUI_ERR_STATE, "the bank runs the per-template path, which has no tiling");
    *out = cui_tuning{b->n1, b->ccols, b->rpc, b->batch};
    return CUI_OK;
}

extern "C" cui_status cui_bank_set_tuning(cui_bank b, const cui_tuning *tu)
{
    if (!b || !tu) return fail(CUI_ERR_ARG, "bank and tuning must be non-NULL");
    if (!b->fused) return fail(CUI_ERR_STATE, "the bank runs the per-template path, which has no tiling");
    if (tu->n1 <= 0 || b->n % tu->n1 || !fused_tiling_ok(b->log2n, tu->n1, tu->ccols, tu->rpc) || tu->batch < 1)
        return fail(CUI_ERR_ARG, "no kernels for n1 = %d, ccols = %d, rpc = %d, batch = %d at N = %lld", tu->n1,
                    tu->ccols, tu->rpc, tu->batch, (long long)b->n);
    CUI_TRY(configure_fused(b, *tu), "cui_bank_set_tuning");
    return CUI_OK;
}

extern "C" cui_status cui_bank_autotune(cui_bank b, int32_t reps, cui_tuning *best, double *best_ms)
{
    if (!b || reps < 1) return fail(CUI_ERR_ARG, "bank must be non-NULL and reps >= 1");
    if (!b->fused) return fail(CUI_ERR_STATE, "the bank runs the per-template path, which has no tiling");
    if (!b->have_segment) return fail(CUI_ERR_STATE, "autotuning times the uploaded segment: upload one first");
    const cudaStream_t s = b->stream;
    const int trace = b->trace;
    b->trace = 0;
    cudaEvent_t e0, e1;
    CUI_TRY(cudaEventCreate(&e0), "autotune events");
    CUI_TRY(cudaEventCreate(&e1), "autotune events");
    cui_tuning cur = {b->n1, b->ccols, b->rpc, b->batch}, top = cur;
    double top_ms = 1e300;
    const int n1s[] = {64, 128, 256}, ccs[] = {16, 32, 64}, rpcs[] = {0, 1, 2, 4, 8, 16, 32};
    const int64_t per = b->n * ((b->desc.flags & CUI_STORE_BF16) ? 4 : 8);
    std::vector<int> batches;
    for (int64_t bt = 16; bt <= 4096; bt *= 4)
        if (bt * per <= (4ll << 30)) batches.push_back((int)bt);
    for (int n1 : n1s)
        for (int cc : ccs)
            for (int rp : rpcs) {
                if (!fused_tiling_ok(b->log2n, n1, cc, rp)) continue;
                for (int bt : batches) {
                    cui_tuning tu = {n1, cc, rp, bt};
                    if (configure_fused(b, tu) != cudaSuccess) {
                        cudaGetLastError();
                        continue;
                    }
                    cui_status st = cui_filter_bank(b, nullptr, b->nt, nullptr);
                    if (st != CUI_OK) continue;
                    cudaEventRecord(e0, s);
                    for (int r = 0; r < reps; ++r) cui_filter_bank(b, nullptr, b->nt, nullptr);
                    cudaEventRecord(e1, s);
                    if (cudaEventSynchronize(e1) != cudaSuccess) continue;
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms / reps < top_ms) {
                        top_ms = ms / reps;
                        top = tu;
                    }
                    if (bt >= b->nt) break; // larger batches change nothing
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->trace = trace;
    CUI_TRY(configure_fused(b, top_ms < 1e300 ? top : cur), "autotune: selecting the best tiling");
    if (best) *best = cui_tuning{b->n1, b->ccols, b->rpc, b->batch};
    if (best_ms) *best_ms = top_ms;
    return CUI_OK;
}

extern "C" cui_status cui_trace_enable(cui_bank b, int on)
{
    if (!b) return fail(CUI_ERR_ARG, "bank is NULL");
    b->trace = on < 0 ? 0 : (on > 2 ? 2 : on);
    return CUI_OK;
}

extern "C" cui_status cui_trace_read(cui_bank b, cui_trace_stat *host_out, int64_t capacity, int64_t *n)
{
    if (!b || !n || capacity < 0 || (capacity > 0 && !host_out)) return fail(CUI_ERR_ARG, "bad arguments");
    CUI_TRY(cudaStreamSynchronize(b->stream), "stream synchronize");
    cui_trace_stat st[kNGroups];
    std::memset(st, 0, sizeof st);
    for (int g = 0; g < kNGroups; ++g) std::snprintf(st[g].name, sizeof st[g].name, "%s", kGroups[g]);
    cudaError_t e = cudaSuccess;
    for (auto &m : b->marks) {
        float ms = 0.f;
        cudaError_t x = cudaEventElapsedTime(&ms, m.a, m.b);
        if (x != cudaSuccess && e == cudaSuccess) e = x;
        st[m.group].ms += ms;
        st[m.group].calls += 1;
        st[m.group].launches += m.launches;
        b->pool.push_back(m.a);
        b->pool.push_back(m.b);
    }
    b->marks.clear();
    if (e != cudaSuccess) return cuda_fail(e, "trace events");
    int64_t k = 0;
    for (int g = 0; g < kNGroups; ++g)
        if (st[g].calls) {
            if (k < capacity) host_out[k] = st[g];
            ++k;
        }
    *n = k;
    return CUI_OK;
}

// Wait for the bank's stream and read the device error word (and the trigger
// count when asked) through the pinned staging area: one synchronisation.
static cui_status sync_and_check(cui_bank b, unsigned long long *trig_count = nullptr)
{
    CUI_TRY(cudaMemcpyAsync(&b->h_stage->err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream),
            "error word");
    if (trig_count)
        CUI_TRY(cudaMemcpyAsync(&b->h_stage->trig_count, b->d_trig_count, sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, b->stream),
                "trigger count");
    CUI_TRY(cudaStreamSynchronize(b->stream), "stream synchronize");
    if (trig_count) *trig_count = b->h_stage->trig_count;
    const int err = b->h_stage->err;
    if (err) {
        cudaMemset(b->d_err, 0, sizeof(int));
        return fail(CUI_ERR_TIMEOUT, "a bounded device wait gave up (code %d)", err);
    }
    return CUI_OK;
}

// Peaks and/or triggers of the last filter call with one synchronisation in
// the common case: the error word, the trigger count, the peaks and the first
// records (as many as the previous call had, doubled) are copied into pinned
// staging together; only a larger count needs a second copy.
static cui_status read_results(cui_bank b, cui_peak *peaks_out, int64_t n_peaks, cui_trigger *trig_out,
                               int64_t capacity, int64_t *n_total)
{
    const cudaStream_t s = b->stream;
    const bool want_trig = n_total != nullptr;
    int64_t pre = 0;
    if (want_trig) {
        pre = std::min<int64_t>(b->trig_cap, std::max<int64_t>(1024, 2 * b->trig_hint));
        if (pre > b->h_trig_cap) {
            if (b->h_trig) cudaFreeHost(b->h_trig);
            b->h_trig = nullptr;
            b->h_trig_cap = 0;
            CUI_TRY(cudaMallocHost(&b->h_trig, sizeof(cui_trigger) * pre), "trigger staging");
            b->h_trig_cap = pre;
        }
        CUI_TRY(cudaMemcpyAsync(b->h_trig, b->d_trig, sizeof(cui_trigger) * pre, cudaMemcpyDeviceToHost, s),
                "trigger copy");
    }
    if (n_peaks > 0)
        CUI_TRY(cudaMemcpyAsync(b->h_peaks, b->d_peaks, sizeof(cui_peak) * n_peaks, cudaMemcpyDeviceToHost, s),
                "peaks copy");
    unsigned long long cnt = 0;
    cui_status st = sync_and_check(b, want_trig ? &cnt : nullptr);
    if (want_trig) *n_total = (int64_t)cnt;
    if (st != CUI_OK) return st;
    if (n_peaks > 0) std::memcpy(peaks_out, b->h_peaks, sizeof(cui_peak) * n_peaks);
    if (!want_trig) return CUI_OK;
    const int64_t have = std::min<int64_t>((int64_t)cnt, b->trig_cap);
    b->trig_hint = have;
    std::vector<cui_trigger> tmp(have);
    if (have <= pre) {
        if (have) std::memcpy(tmp.data(), b->h_trig, sizeof(cui_trigger) * have);
    } else {
        CUI_TRY(cudaMemcpy(tmp.data(), b->d_trig, sizeof(cui_trigger) * have, cudaMemcpyDeviceToHost), "trigger copy");
    }
    std::sort(tmp.begin(), tmp.end(), [](const cui_trigger &x, const cui_trigger &y) {
        return x.tmpl != y.tmpl ? x.tmpl < y.tmpl : x.sample < y.sample;
    });
    const int64_t nout = std::min<int64_t>(have, capacity);
    if (nout) std::memcpy(trig_out, tmp.data(), sizeof(cui_trigger) * nout);
    if ((int64_t)cnt > b->trig_cap)
        return fail(CUI_ERR_OVERFLOW, "%llu triggers exceed the device buffer of %lld (only those were kept)", cnt,
                    (long long)b->trig_cap);
    if ((int64_t)cnt > capacity)
        return fail(CUI_ERR_OVERFLOW, "%llu triggers exceed capacity %lld", cnt, (long long)capacity);
    return CUI_OK;
}

extern "C" cui_status cui_peaks(cui_bank b, cui_peak *host_out, int64_t count)
{
    if (!b || !host_out) return fail(CUI_ERR_ARG, "bank and host_out must be non-NULL");
    if (count < 0 || count > b->nt) return fail(CUI_ERR_ARG, "count must be in [0, n_templates]");
    if (!b->have_peaks) return fail(CUI_ERR_STATE, "no filter call kept its peaks in the handle");
    return read_results(b, host_out, count, nullptr, 0, nullptr);
}

extern "C" cui_status cui_triggers(cui_bank b, cui_trigger *host_out, int64_t capacity, int64_t *n_total)
{
    if (!b || !n_total) return fail(CUI_ERR_ARG, "bank and n_total must be non-NULL");
    if (capacity < 0 || (capacity > 0 && !host_out)) return fail(CUI_ERR_ARG, "bad capacity / host_out");
    return read_results(b, nullptr, 0, host_out, capacity, n_total);
}

extern "C" cui_status cui_results(cui_bank b, cui_peak *host_peaks, int64_t n_peaks, cui_trigger *host_trig,
                                  int64_t capacity, int64_t *n_total)
{
    if (!b || !host_peaks || !n_total) return fail(CUI_ERR_ARG, "bank, host_peaks and n_total must be non-NULL");
    if (n_peaks < 0 || n_peaks > b->nt) return fail(CUI_ERR_ARG, "n_peaks must be in [0, n_templates]");
    if (capacity < 0 || (capacity > 0 && !host_trig)) return fail(CUI_ERR_ARG, "bad capacity / host_trig");
    if (!b->have_peaks) return fail(CUI_ERR_STATE, "no filter call kept its peaks in the handle");
    return read_results(b, host_peaks, n_peaks, host_trig, capacity, n_total);
}

extern "C" cui_status cui_cluster_triggers(cui_bank b, cui_trigger *host_out, int64_t capacity, int64_t *n_total)
{
    if (!b || !n_total) return fail(CUI_ERR_ARG, "bank and n_total must be non-NULL");
    if (capacity < 0 || (capacity > 0 && !host_out)) return fail(CUI_ERR_ARG, "bad capacity / host_out");
    if (!b->filtered) return fail(CUI_ERR_STATE, "no filter call since the last upload");
    const int nw = std::max(1, b->nwin);
    std::vector<Slot> h(nw);
    CUI_TRY(cudaMemcpyAsync(h.data(), b->d_cluster, sizeof(Slot) * nw, cudaMemcpyDeviceToHost, b->stream),
            "cluster copy");
    cui_status st = sync_and_check(b);
    if (st != CUI_OK) return st;
    int64_t n = 0;
    for (int w = 0; w < nw; ++w) {
        const Slot &sl = h[w];
        if (sl.key == 0ull) continue;
        if (n < capacity) {
            cui_trigger tr;
            const uint32_t r2 = (uint32_t)(sl.key >> 32);
            float rho2, ph;
            std::memcpy(&rho2, &r2, 4);
            std::memcpy(&ph, &sl.phase_bits, 4);
            tr.tmpl = (int32_t)(0xFFFFFFFFu - sl.pad);
            tr.pad = 0;
            tr.sample = (int64_t)(0xFFFFFFFFu - (uint32_t)(sl.key & 0xFFFFFFFFull));
            tr.snr = std::sqrt(rho2);
            tr.phase = ph;
            host_out[n] = tr;
        }
        ++n;
    }
    *n_total = n;
    if (n > capacity) return fail(CUI_ERR_OVERFLOW, "%lld clustered triggers exceed capacity %lld", (long long)n,
                                  (long long)capacity);
    return CUI_OK;
}

extern "C" cui_status cui_trigger_chisq(cui_bank b, int32_t bands, const cui_trigger *trig, int64_t n,
                                        float *host_chisq, float *host_rho)
{
    if (!b) return fail(CUI_ERR_ARG, "bank is NULL");
    if (bands < 1 || bands > kChisqMaxBands) return fail(CUI_ERR_ARG, "bands must be in [1, %d]", kChisqMaxBands);
    if (n < 0 || n > (int64_t(1) << 30) || (n > 0 && (!trig || !host_chisq)))
        return fail(CUI_ERR_ARG, "bad trigger count or NULL pointers");
    if (!b->fused) return fail(CUI_ERR_STATE, "the chi^2 test needs the fused path (N >= 2^12, no CUI_PLAIN)");
    if (!b->have_segment) return fail(CUI_ERR_STATE, "no segment uploaded");
    if (n == 0) return CUI_OK;
    std::vector<int2> h(n);
    for (int64_t i = 0; i < n; ++i) {
        if (trig[i].tmpl < 0 || trig[i].tmpl >= b->nt || trig[i].sample < 0 || trig[i].sample >= b->n)
            return fail(CUI_ERR_ARG, "trigger %lld: template or sample out of range", (long long)i);
        h[i] = make_int2(trig[i].tmpl, (int)trig[i].sample);
    }
    const cudaStream_t s = b->stream;
    int2 *d_trig = nullptr;
    float *d_out = nullptr;
    cudaError_t e = cudaMalloc(&d_trig, sizeof(int2) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(float) * 2 * n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_trig, h.data(), sizeof(int2) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = launch_chisq(fused_args_post(b), b->d_prefix, d_trig, (int)n, bands, d_out, d_out + n, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_chisq, d_out, sizeof(float) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && host_rho)
        e = cudaMemcpyAsync(host_rho, d_out + n, sizeof(float) * n, cudaMemcpyDeviceToHost, s);
    cui_status st = e == cudaSuccess ? sync_and_check(b) : cuda_fail(e, "chi^2");
    cudaFree(d_trig);
    cudaFree(d_out);
    return st;
}

extern "C" cui_status cui_bank_set_band(cui_bank b, double f_lo, double f_hi)
{
    if (!b) return fail(CUI_ERR_ARG, "bank is NULL");
    if (!std::isfinite(f_lo) || !std::isfinite(f_hi)) return fail(CUI_ERR_ARG, "band edges must be finite");
    const double klo = std::ceil(f_lo / b->df), khi = std::ceil(f_hi / b->df);
    const int lo = (int)std::max<double>(b->k_low, std::min<double>(klo, (double)b->nh));
    const int hi = f_hi <= 0.0 ? (int)b->nh : (int)std::max<double>(lo, std::min<double>(khi, (double)b->nh));
    if (lo == b->band_lo && hi == b->band_hi) return CUI_OK;
    const cudaStream_t s = b->stream;
    // the pageable copy source below is reused: wait for any earlier copy of it
    CUI_TRY(cudaStreamSynchronize(s), "stream synchronize");
    b->band_lo = lo;
    b->band_hi = hi;
    for (int64_t t = 0; t < b->nt; ++t) b->h_khi_eff[t] = std::min<int32_t>(b->h_khi[t], hi);
    CUI_TRY(cudaMemcpyAsync(b->d_khi, b->h_khi_eff.data(), sizeof(int32_t) * b->nt, cudaMemcpyHostToDevice, s),
            "band copy");
    if (b->gexec) { // the captured call holds the old lower edge
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    if (b->have_segment)
        launch_template_norm(b->d_prefix, b->d_khi, b->band_lo, b->nt, b->desc.sample_rate, b->n, b->d_scales,
                             b->d_sigma2, b->d_invnorm, s);
    b->filtered = false;
    CUI_TRY(cudaGetLastError(), "cui_bank_set_band");
    return CUI_OK;
}

extern "C" cui_status cui_segment_band_series(cui_bank b, double f_lo, double f_hi, int32_t decim, double *out_dev)
{
    if (!b || !out_dev) return fail(CUI_ERR_ARG, "bank and out_dev must be non-NULL");
    if (!std::isfinite(f_lo) || !std::isfinite(f_hi)) return fail(CUI_ERR_ARG, "band edges must be finite");
    if (decim < 1 || (decim & (decim - 1)) || (int64_t)decim > b->n / 16)
        return fail(CUI_ERR_ARG, "decim must be a power of two with N / decim >= 16");
    if (!b->have_segment || !b->d_X) return fail(CUI_ERR_STATE, "no segment uploaded");
    const int64_t m = b->n / decim;
    const double klo = std::ceil(f_lo / b->df), khi = std::ceil(f_hi / b->df);
    const int64_t ka = (int64_t)std::max<double>(0.0, std::min<double>(klo, (double)(m / 2)));
    const int64_t kb = f_hi <= 0.0 ? m / 2 : (int64_t)std::max<double>(ka, std::min<double>(khi, (double)(m / 2)));
    const cudaStream_t s = b->stream;
    dfc *a = nullptr;
    CUI_TRY(cudaMallocAsync(&a, sizeof(dfc) * 2 * m, s), "band series buffers");
    launch_band_series(b->d_X, b->n, ilog2(m), ka, kb, b->tw, a, a + m, out_dev, s);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(a, s);
    CUI_TRY(e, "cui_segment_band_series");
    return CUI_OK;
}

// Validated band-sum queries of one bank: template ids, times as 64-bit
// fractions of the segment, the band's bins and the physical-unit factors.
struct BandQuery {
    std::vector<int32_t> t;
    std::vector<uint64_t> u;
    int ka = 0, kb = 0;
    double zfac = 0, sfac = 0;
};

static cui_status band_query(cui_bank b, const int32_t *tmpl, const double *t_sec, int64_t n, double f_lo,
                             double f_hi, BandQuery &q)
{
    if (!std::isfinite(f_lo) || !std::isfinite(f_hi)) return fail(CUI_ERR_ARG, "band edges must be finite");
    if (!b->fused) return fail(CUI_ERR_STATE, "band sums need the fused path (N >= 2^12, no CUI_PLAIN)");
    if (!b->have_segment) return fail(CUI_ERR_STATE, "no segment uploaded");
    const double T = (double)b->n / b->desc.sample_rate;
    q.t.resize(n);
    q.u.resize(n);
    for (int64_t i = 0; i < n; ++i) {
        if (tmpl[i] < 0 || tmpl[i] >= b->nt) return fail(CUI_ERR_ARG, "query %lld: template out of range", (long long)i);
        if (!std::isfinite(t_sec[i])) return fail(CUI_ERR_ARG, "query %lld: time must be finite", (long long)i);
        q.t[i] = tmpl[i];
        // t / T mod 1 as a 64-bit fraction (exact for sample times j / fs)
        double fr = t_sec[i] / T;
        fr -= std::floor(fr);
        const double x = std::ldexp(fr, 64);
        q.u[i] = x >= 18446744073709551616.0 ? 0ull : (uint64_t)x;
    }
    const double klo = std::ceil(f_lo / b->df), khi = std::ceil(f_hi / b->df);
    q.ka = (int)std::max<double>(b->k_low, std::min<double>(klo, (double)b->nh));
    q.kb = f_hi <= 0.0 ? (int)b->nh : (int)std::max<double>(q.ka, std::min<double>(khi, (double)b->nh));
    const double df = b->df;
    q.zfac = 4.0 * df * std::pow(df, -7.0 / 6.0);
    q.sfac = 4.0 * df * std::pow(df, -7.0 / 3.0);
    return CUI_OK;
}

// Device buffers of one batch of band sums, freed by the destructor (after the
// caller's synchronisation).
struct BandBufs {
    int32_t *t = nullptr;
    uint64_t *u = nullptr;
    double *out = nullptr;
    ~BandBufs()
    {
        cudaFree(t);
        cudaFree(u);
        cudaFree(out);
    }
};

// Queue the sums of q on the bank's stream into bufs.out[3 i ..] = (Re z, Im z, sigma^2).
static cudaError_t band_queue(cui_bank b, const BandQuery &q, BandBufs &bufs)
{
    const int64_t n = (int64_t)q.t.size();
    const cudaStream_t s = b->stream;
    cudaError_t e = cudaMalloc(&bufs.t, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&bufs.u, sizeof(uint64_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&bufs.out, sizeof(double) * 3 * n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bufs.t, q.t.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bufs.u, q.u.data(), sizeof(uint64_t) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = launch_band(fused_args_post(b), b->d_prefix, b->d_khi0, bufs.t, bufs.u, (int)n, q.ka, q.kb,
                        b->d_scales, q.zfac, q.sfac, bufs.out, s);
    return e;
}

extern "C" cui_status cui_band_correlate(cui_bank b, const int32_t *tmpl, const double *t_sec, int64_t n,
                                         double f_lo, double f_hi, double *host_z, double *host_sigma2)
{
    if (!b) return fail(CUI_ERR_ARG, "bank is NULL");
    if (n < 0 || n > (int64_t(1) << 30) || (n > 0 && (!tmpl || !t_sec || !host_z)))
        return fail(CUI_ERR_ARG, "bad query count or NULL pointers");
    BandQuery q;
    cui_status st = band_query(b, tmpl, t_sec, n, f_lo, f_hi, q);
    if (st != CUI_OK || n == 0) return st;
    std::vector<double> out(3 * n);
    BandBufs bufs;
    cudaError_t e = band_queue(b, q, bufs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out.data(), bufs.out, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, b->stream);
    st = e == cudaSuccess ? sync_and_check(b) : cuda_fail(e, "band sums");
    if (st != CUI_OK) return st;
    for (int64_t i = 0; i < n; ++i) {
        host_z[2 * i] = out[3 * i];
        host_z[2 * i + 1] = out[3 * i + 1];
        if (host_sigma2) host_sigma2[i] = out[3 * i + 2];
    }
    return CUI_OK;
}

extern "C" cui_status cui_band_combine(cui_bank high, const double *t_high, cui_bank low, const double *t_low,
                                       const int32_t *tmpl, int64_t n, double f_split, double *host_rho,
                                       double *host_phase, double *host_sums)
{
    if (!high || !low) return fail(CUI_ERR_ARG, "both banks must be non-NULL");
    if (n < 0 || n > (int64_t(1) << 30) || (n > 0 && (!tmpl || !t_high || !t_low || !host_rho || !host_phase)))
        return fail(CUI_ERR_ARG, "bad candidate count or NULL pointers");
    if (high->nt != low->nt) return fail(CUI_ERR_ARG, "the two banks hold different numbers of templates");
    for (int64_t t = 0; t < high->nt; ++t)
        if (high->h_mass[2 * t] != low->h_mass[2 * t] || high->h_mass[2 * t + 1] != low->h_mass[2 * t + 1])
            return fail(CUI_ERR_ARG, "template %lld differs between the two banks", (long long)t);
    if (!std::isfinite(f_split) || !(f_split > 0)) return fail(CUI_ERR_ARG, "f_split must be finite and > 0");
    BandQuery qh, ql;
    cui_status st = band_query(high, tmpl, t_high, n, f_split, 0.0, qh);
    if (st == CUI_OK) st = band_query(low, tmpl, t_low, n, 0.0, f_split, ql);
    if (st != CUI_OK || n == 0) return st;
    BandBufs bh, bl;
    double *d_res = nullptr;
    std::vector<double> res(2 * n), sums(host_sums ? 6 * n : 0);
    cudaEvent_t ev = nullptr;
    cudaError_t e = band_queue(high, qh, bh);
    if (e == cudaSuccess) e = band_queue(low, ql, bl);
    if (e == cudaSuccess) e = cudaMalloc(&d_res, sizeof(double) * 2 * n);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, high->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(low->stream, ev, 0);
    if (e == cudaSuccess) e = launch_band_combine(bh.out, bl.out, (int)n, d_res, low->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(res.data(), d_res, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, low->stream);
    if (e == cudaSuccess && host_sums) {
        e = cudaMemcpyAsync(sums.data(), bh.out, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, low->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sums.data() + 3 * n, bl.out, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost,
                                low->stream);
    }
    st = e == cudaSuccess ? sync_and_check(high) : cuda_fail(e, "band combination");
    if (st == CUI_OK) st = sync_and_check(low);
    if (ev) cudaEventDestroy(ev);
    cudaFree(d_res);
    if (st != CUI_OK) return st;
    for (int64_t i = 0; i < n; ++i) {
        host_rho[i] = res[2 * i];
        host_phase[i] = res[2 * i + 1];
        if (host_sums) {
            for (int c = 0; c < 3; ++c) {
                host_sums[6 * i + c] = sums[3 * i + c];
                host_sums[6 * i + 3 + c] = sums[3 * n + 3 * i + c];
            }
        }
    }
    return CUI_OK;
}

extern "C" cui_status cui_td_template(cui_bank b, int64_t t, int32_t pn_x2, double *hp_dev, double *hx_dev)
{
    if (!b || !hp_dev || !hx_dev) return fail(CUI_ERR_ARG, "bank and output pointers must be non-NULL");
    if (t < 0 || t >= b->nt) return fail(CUI_ERR_ARG, "template %lld out of range", (long long)t);
    if (pn_x2 < 0 || pn_x2 > 5) return fail(CUI_ERR_ARG, "the time-domain generator keeps up to 2.5PN (pn_x2 <= 5)");
    TdArgs a;
    td_coefficients(b->h_mass[2 * t], b->h_mass[2 * t + 1], pn_x2, a);
    a.v_lo = std::cbrt(3.14159265358979323846 * a.M * b->desc.f_low);
    a.v_hi = 1.0 / std::sqrt(6.0);
    a.t_lo = td_time(a, a.v_lo);
    a.t_hi = a.v_lo < a.v_hi ? td_time(a, a.v_hi) : a.t_lo - 1.0; // empty band: all zeros
    a.fs = b->desc.sample_rate;
    a.n = b->n;
    CUI_TRY(launch_td_template(a, hp_dev, hx_dev, b->stream), "time-domain template");
    launched();
    return CUI_OK;
}

extern "C" cui_status cui_bank_sigma(cui_bank b, double *host_sigma)
{
    if (!b || !host_sigma) return fail(CUI_ERR_ARG, "bank and host_sigma must be non-NULL");
    if (!b->have_segment) return fail(CUI_ERR_STATE, "no segment uploaded");
    CUI_TRY(cudaStreamSynchronize(b->stream), "stream synchronize");
    CUI_TRY(cudaMemcpy(host_sigma, b->d_sigma2, sizeof(double) * b->nt, cudaMemcpyDeviceToHost), "sigma copy");
    for (int64_t t = 0; t < b->nt; ++t) host_sigma[t] = std::sqrt(host_sigma[t]);
    return CUI_OK;
}

extern "C" cui_status cui_bank_template(cui_bank b, int64_t t, float *out_dev)
{
    if (!b || !out_dev) return fail(CUI_ERR_ARG, "bank and out_dev must be non-NULL");
    if (t < 0 || t >= b->nt) return fail(CUI_ERR_ARG, "template index out of range");
    if (!fused_supported(b->log2n))
        return fail(CUI_ERR_ARG, "template read-out needs the fused path's sizes (2^12 <= N <= 2^22)");
    if (!b->fused) {
        // anchors for the read-out are built on first use for plain-path banks
        if (!b->d_basis) {
            fused_default_tiling(b->log2n, &b->n1, &b->ccols, &b->rpc);
            b->n2 = (int)(b->n / b->n1);
            CUI_TRY(build_phase_tables(b, b->n1, b->ccols), "template read-out tables");
        }
    }
    FusedArgs a = fused_args(b, b->d_iota, 0);
    const double dfac = std::pow(b->df, -7.0 / 6.0);
    CUI_TRY(launch_template_out(a, (int)t, b->d_amp, dfac, (float2 *)out_dev, b->stream), "template read-out");
    return CUI_OK;
}
