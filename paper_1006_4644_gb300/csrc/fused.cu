// Fused batched bank filter (the per-chunk loop of Sec. "Matched filtering",
// steps 1-4, for many templates at once).
//
// The correlator z_j = sum_k q_k exp(+2 pi i j k / N), with
// q_k = wbar_k exp(+2 pi i Phi_t(k)) on the template's band, is computed as a
// four-step transform N = n1 * n2, k = n2 a + b, j = c + n1 d:
//   pass 1 (per column b): Y[c][b] = exp(2 pi i b c / N) sum_a q[n2 a + b] exp(2 pi i a c / n1)
//   pass 2 (per row c):    z[c + n1 d] = sum_b Y[c][b] exp(2 pi i b d / n2)
// Pass 1 generates q on the fly (template generation fused into the
// correlation product); pass 2 never writes z: its epilogue reduces
// rho^2 = |z|^2 / sigma^2 to the template's peak and to per-window maxima above
// the threshold.  Y is the only spectrum that touches global memory: one
// write and one read of N complex values per template.
//
// Template phase.  Phi_t(k) = Psi_t(k df) / (2 pi) is a fixed linear
// combination of nine template-independent functions of k.  Each pass-1 CTA
// owns C consecutive bins of every row, so per row it evaluates Phi and its
// first three derivatives at the centre bin k_a in FP64 (or double-float),
// reduces Phi(k_a) and Phi'(k_a) modulo 1 (exact for integer offsets), and
// every bin k_a + x of the row then costs one FP32 cubic in x, one fast
// sincos of an argument already in [-pi, pi) and one complex product.
#include <cuda_bf16.h>

#include <algorithm>

#include <type_traits>

#include "internal.h"

namespace cui {

__constant__ DerivConsts c_dc;

void fused_set_consts(const DerivConsts &dc, cudaStream_t s)
{
    cudaMemcpyToSymbolAsync(c_dc, &dc, sizeof(dc), 0, cudaMemcpyHostToDevice, s);
}

// ------------------------------------------------------------ storage ----
// Y is written once by pass 1 and read once by pass 2 after the whole batch:
// streaming accesses (evict first) keep it from displacing the weighted data
// and the tables that every CTA reads from L2.
template <typename ST> __device__ __forceinline__ void st_c(ST *p, float2 v);
template <> __device__ __forceinline__ void st_c<float2>(float2 *p, float2 v) { __stcs(p, v); }
template <> __device__ __forceinline__ void st_c<__nv_bfloat162>(__nv_bfloat162 *p, float2 v)
{
    const __nv_bfloat162 b = __float22bfloat162_rn(v);
    __stcs((unsigned *)p, *(const unsigned *)&b);
}
template <typename ST> __device__ __forceinline__ float2 ld_c(const ST *p);
template <> __device__ __forceinline__ float2 ld_c<float2>(const float2 *p) { return __ldcs(p); }
template <> __device__ __forceinline__ float2 ld_c<__nv_bfloat162>(const __nv_bfloat162 *p)
{
    const unsigned u = __ldcs((const unsigned *)p);
    return __bfloat1622float2(*(const __nv_bfloat162 *)&u);
}

// Paired layout of Y: rows c and c + n1/2 of one template interleaved at each
// column b as (re_c, re_c', im_c, im_c'), which pass 2 loads straight into a
// c2 (the two rows are its two lanes).  Row pair c holds n2 such entries.
template <typename ST> struct pair_of;
template <> struct pair_of<float2> { using T = float4; };
template <> struct pair_of<__nv_bfloat162> { using T = uint2; };
template <typename ST> using pair_t = typename pair_of<ST>::T;

template <typename ST> __device__ __forceinline__ void st_pair(pair_t<ST> *p, float2 lo, float2 hi);
template <> __device__ __forceinline__ void st_pair<float2>(float4 *p, float2 lo, float2 hi)
{
    __stcs(p, make_float4(lo.x, hi.x, lo.y, hi.y));
}
template <> __device__ __forceinline__ void st_pair<__nv_bfloat162>(uint2 *p, float2 lo, float2 hi)
{
    const __nv_bfloat162 re = __floats2bfloat162_rn(lo.x, hi.x), im = __floats2bfloat162_rn(lo.y, hi.y);
    __stcs(p, make_uint2(*(const unsigned *)&re, *(const unsigned *)&im));
}
template <typename ST> __device__ __forceinline__ c2 ld_pair(const pair_t<ST> *p);
template <> __device__ __forceinline__ c2 ld_pair<float2>(const float4 *p)
{
    const float4 q = __ldcs(p);
    return {make_float2(q.x, q.y), make_float2(q.z, q.w)};
}
template <> __device__ __forceinline__ c2 ld_pair<__nv_bfloat162>(const uint2 *p)
{
    const uint2 q = __ldcs(p);
    return {__bfloat1622float2(*(const __nv_bfloat162 *)&q.x), __bfloat1622float2(*(const __nv_bfloat162 *)&q.y)};
}

// element idx of template-slice `base`, as one complex (unpaired) or one row pair
template <typename ST, bool PAIR> __device__ __forceinline__ auto ld_y(const char *base, size_t idx)
{
    if constexpr (PAIR) return ld_pair<ST>((const pair_t<ST> *)base + idx);
    else return ld_c<ST>((const ST *)base + idx);
}

// exp(2 pi i m / d) for 0 <= m < d, accurate to ~1 ulp.
__device__ __forceinline__ float2 turn(unsigned m, unsigned d)
{
    float s, c;
    sincospif(2.0f * ((float)m / (float)d), &s, &c);
    return make_float2(c, s);
}

// ------------------------------------------------------------- anchors ----
__device__ __forceinline__ float4 anchor_derivs(float phi0, const float *tf, float u7, float c5, float x)
{
    float s1 = c_dc.gam[1] * u7 + c_dc.lam[1] * c5;
    float s2 = c_dc.gam[2] * u7 + c_dc.lam[2] * c5;
    float s3 = c_dc.gam[3] * u7 + c_dc.lam[3] * c5;
#pragma unroll
    for (int i = 0; i < kNB; ++i) {
        s1 = fmaf(c_dc.B[1][i], tf[i], s1);
        s2 = fmaf(c_dc.B[2][i], tf[i], s2);
        s3 = fmaf(c_dc.B[3][i], tf[i], s3);
    }
    float p1 = s1 * x;
    p1 -= rintf(p1); // only integer offsets multiply Phi', so Phi' mod 1 suffices
    const float x2 = x * x;
    return make_float4(phi0, p1, s2 * x2, s3 * x2 * x);
}

// (Phi(k_a) mod 1, Phi'(k_a) mod 1, Phi''(k_a)/2, Phi'''(k_a)/6) in cycles.
// Default: the nine products c_i g_i(k_a) in double-float (FMA two-products,
// two-sum accumulation of the high parts, plain accumulation of the low
// parts); p.fp64 selects native FP64 instead.
__device__ __forceinline__ float4 anchor_eval(const FusedArgs &p, int t, int64_t ai, float ka)
{
    float tf[kNB];
    float phi0, u7, c5;
    if (p.fp64) {
        const double *c = p.coef + (int64_t)t * kNB;
        const double *g = p.basis + ai * kNB;
        double T[kNB];
#pragma unroll
        for (int i = 0; i < kNB; ++i) T[i] = c[i] * g[i];
        double s = T[0];
#pragma unroll
        for (int i = 1; i < kNB; ++i) s += T[i];
        s -= rint(s);
        phi0 = (float)s;
#pragma unroll
        for (int i = 0; i < kNB; ++i) tf[i] = (float)T[i];
        u7 = (float)(c[7] * g[6]);
        c5 = (float)c[5];
    } else {
        const float2 *c = p.coef_df + (int64_t)t * kNB;
        const float2 *g = p.basis_df + ai * kNB;
        float s = 0.f, e = 0.f;
#pragma unroll
        for (int i = 0; i < kNB; ++i) {
            const float2 ci = c[i], gi = g[i];
            const float ph = __fmul_rn(ci.x, gi.x);
            float pe = __fmaf_rn(ci.x, gi.x, -ph);
            pe = __fmaf_rn(ci.x, gi.y, pe);
            pe = __fmaf_rn(ci.y, gi.x, pe);
            const float sn = __fadd_rn(s, ph);
            const float bb = __fsub_rn(sn, s);
            const float er = __fadd_rn(__fsub_rn(s, __fsub_rn(sn, bb)), __fsub_rn(ph, bb));
            s = sn;
            e = __fadd_rn(e, __fadd_rn(er, pe));
            tf[i] = ph;
        }
        phi0 = __fadd_rn(__fsub_rn(s, rintf(s)), e);
        u7 = c[7].x * g[6].x;
        c5 = c[5].x;
    }
    return anchor_derivs(phi0, tf, u7, c5, 1.0f / ka);
}

// Phi(k) mod 1 evaluated exactly (double-float) from the per-bin basis table;
// used below k_ex(t), where a cubic over C bins would not be accurate enough.
__device__ __forceinline__ float phase_exact(const float2 *c, const float2 *g)
{
    df s = {0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < kNB; ++i) {
        const float2 gi = g[i];
        s = df_add(s, df_mul(df{c[i].x, c[i].y}, df{gi.x, gi.y}));
    }
    return __fsub_rn(s.hi, rintf(s.hi)) + s.lo;
}

__device__ __forceinline__ float2 rotate(float ph, float2 w)
{
    ph -= rintf(ph);
    float s, c;
    __sincosf(6.283185307179586f * ph, &s, &c);
    return make_float2(w.x * c - w.y * s, w.x * s + w.y * c);
}

// q = w exp(2 pi i Phi) with Phi = a.x + x (a.y + x (a.z + x a.w)).
__device__ __forceinline__ float2 gen_bin(float4 a, float x, float2 w)
{
    return rotate(fmaf(x, fmaf(x, fmaf(x, a.w, a.z), a.y), a.x), w);
}

__device__ __forceinline__ int ceil_div_pos(int num, int den) { return num <= 0 ? 0 : (num + den - 1) / den; }

// ---------------------------------------------------------------- pass 1 ---
// Stage 0 of a column block for one template: generate q on rows
// a = j + r N1/R0 (only r < NZ can fall inside the band, because the band
// ends below N/2, i.e. below row N1/2) and take the input-pruned R0-point DFT.
template <int N1, int R0, int C, int NZ>
__device__ __forceinline__ void p1_stage0(float2 *v, const FusedArgs &p, const float4 *anc, const float2 *cdf, int jt,
                                          int col, int b0, int a_lo, int a_hi, int klo, int khi, int kex)
{
    constexpr int T0 = 16 / R0;
    const float x = (float)(col - C / 2);
    const int bcol = b0 + col;
    const int n2 = p.n2;
#pragma unroll
    for (int i = 0; i < T0; ++i) {
        const int j = jt + i * (N1 / 16);
#pragma unroll
        for (int r = 0; r < NZ; ++r) {
            const int a = j + r * (N1 / R0);
            float2 q = make_float2(0.f, 0.f);
            if (a >= a_lo && a < a_hi) {
                const int k = n2 * a + bcol;
                if (k >= klo && k < khi)
                    q = k < kex ? rotate(phase_exact(cdf, p.gexact + (int64_t)k * kNB), p.wbar[k])
                                : gen_bin(anc[a], x, p.wbar[k]);
            }
            v[i * R0 + r] = q;
        }
        dft_nz<R0, NZ, +1>(v + i * R0);
    }
}

// Grid (n2 / C, ceil(B / G)).  A CTA owns C columns of n1 = R0 * R1 rows and
// runs G templates through them, so the twiddles that depend only on the
// position (the stage-1 table and the inter-pass factors exp(2 pi i b c / N),
// kept in registers) are computed once per CTA.  PAIR selects the paired
// layout of Y (rows c and c + n1/2 interleaved), else rows are stored whole.
constexpr int p1_min_blocks(int nt) { return nt == 256 ? 3 : (nt <= 512 ? 2 : 1); }

template <int N1, int R0, int R1, int C, int G, typename ST, bool PAIR>
__global__ void __launch_bounds__(C *N1 / 16, p1_min_blocks(C *N1 / 16)) k_pass1(const FusedArgs p, int count)
{
    constexpr int NT = C * N1 / 16;
    constexpr int NROW = N1 / 2;
    constexpr int T1 = 16 / R1;
    __shared__ float4 anc[G][NROW];
    __shared__ float2 tw[N1];
    __shared__ float2 cdf[G][kNB];
    extern __shared__ float2 sm[]; // [N1][C]
    const int tid = threadIdx.x;
    const int col = tid % C;
    const int jt = tid / C;
    const int cb = blockIdx.x;
    const int n2 = p.n2;
    const int b0 = cb * C;
    const int bcol = b0 + col;
    const int klo = p.k_low;
    const int64_t N = p.n;

    for (int m = tid; m < N1; m += NT) tw[m] = turn(m, N1);
    // exp(2 pi i b c / N) for this thread's stage-1 outputs c = j + r N1/R1 is
    // ipb[i] * ips^r: one accurate root per task and one step, per CTA
    float2 ipb[T1];
#pragma unroll
    for (int i = 0; i < T1; ++i)
        ipb[i] = turn(((unsigned)bcol * (unsigned)(jt + i * (N1 / 16))) & (unsigned)(N - 1), (unsigned)N);
    const float2 ips = turn(((unsigned)bcol * (unsigned)(N1 / R1)) & (unsigned)(N - 1), (unsigned)N);

    // anchors of all the CTA's templates in one balanced phase
    const int y0 = blockIdx.y * G;
    const int ng = min(G, count - y0);
    const int a_lo = ceil_div_pos(klo - b0 - (C - 1), n2);
    for (int m = tid; m < G * NROW; m += NT) {
        const int g = m / NROW, a = m % NROW;
        if (g >= ng || a < a_lo) continue;
        const int t = p.order[p.base + y0 + g];
        if (a < min(NROW, ceil_div_pos(p.khi[t] - b0, n2))) {
            const int64_t ai = (int64_t)a * (n2 / C) + cb;
            anc[g][a] = anchor_eval(p, t, ai, (float)((int64_t)n2 * a + b0 + C / 2));
        }
    }
    for (int m = tid; m < ng * kNB; m += NT) // a CTA can have fewer threads than G kNB
        cdf[m / kNB][m % kNB] = p.coef_df[(int64_t)p.order[p.base + y0 + m / kNB] * kNB + m % kNB];
    // band edges of the CTA's templates, read once
    __shared__ int2 tk[G];
    for (int g = tid; g < ng; g += NT) {
        const int t = p.order[p.base + y0 + g];
        tk[g] = make_int2(p.khi[t], p.kex[t]);
    }
    __syncthreads();

    for (int g = 0; g < ng; ++g) {
        const int y = y0 + g;
        const int khi = tk[g].x;
        const int kex = tk[g].y;
        const int a_hi = min(NROW, ceil_div_pos(khi - b0, n2));

        float2 v[16];
        // number of stage-0 inputs per task that can be nonzero, rounded up to a power of two
        const int nzr = ceil_div_pos(a_hi, N1 / R0);
        if (nzr <= 1) p1_stage0<N1, R0, C, 1>(v, p, anc[g], cdf[g], jt, col, b0, a_lo, a_hi, klo, khi, kex);
        else if (nzr <= 2) p1_stage0<N1, R0, C, 2>(v, p, anc[g], cdf[g], jt, col, b0, a_lo, a_hi, klo, khi, kex);
        else if (nzr <= 4 || R0 <= 8) p1_stage0<N1, R0, C, (R0 > 8 ? 4 : R0 / 2)>(v, p, anc[g], cdf[g], jt, col, b0,
                                                                                    a_lo, a_hi, klo, khi, kex);
        else p1_stage0<N1, R0, C, R0 / 2>(v, p, anc[g], cdf[g], jt, col, b0, a_lo, a_hi, klo, khi, kex);
        if (g > 0) __syncthreads(); // every thread has read the previous template's sm
#pragma unroll
        for (int i = 0; i < 16 / R0; ++i) {
            const int j = jt + i * (N1 / 16);
#pragma unroll
            for (int r = 0; r < R0; ++r) sm[(j * R0 + r) * C + col] = v[i * R0 + r];
        }
        __syncthreads();

        // stage 1 (last): radix R1 over sub-transforms of size R0; times exp(2 pi i b c / N)
        char *yslice = (char *)p.ywork + (size_t)y * (size_t)N * sizeof(ST);
#pragma unroll
        for (int i = 0; i < T1; ++i) {
            const int j = jt + i * (N1 / 16);
            float2 *u = v + i * R1;
#pragma unroll
            for (int r = 0; r < R1; ++r) u[r] = sm[(j + r * (N1 / R1)) * C + col];
            const int jm = j % R0;
#pragma unroll
            for (int r = 1; r < R1; ++r) u[r] = cmul(u[r], tw[jm * r]);
            dft<R1, +1>(u);
            float2 w = ipb[i];
            if constexpr (PAIR) {
#pragma unroll
                for (int r = 0; r < R1; ++r) {
                    u[r] = cmul(u[r], w);
                    w = cmul(w, ips);
                }
                // output c = j + r N1/R1 and its partner c + N1/2 (r + R1/2) form one row pair
#pragma unroll
                for (int r = 0; r < R1 / 2; ++r) {
                    const int c = j + r * (N1 / R1);
                    st_pair<ST>((pair_t<ST> *)yslice + (size_t)c * n2 + bcol, u[r], u[r + R1 / 2]);
                }
            } else {
#pragma unroll
                for (int r = 0; r < R1; ++r) {
                    const int c = j + r * (N1 / R1);
                    st_c<ST>((ST *)yslice + (size_t)c * n2 + bcol, cmul(u[r], w));
                    w = cmul(w, ips);
                }
            }
        }
    }
}

// ---------------------------------------------------------------- pass 2 ---
// One spare slot every 16 keeps the stride-16 stores conflict-free.  Rows of
// 4096 and 16384 points run their last two stages on half-warp groups (see
// k_pass2), whose accesses step by 256 or 1024 elements; extra slots every
// 256 (and 4096) keep those conflict-free too.  For a power of two Q and
// 0 <= j < Q, padi(j + r Q) = padi(j) + padi(r Q): the strided accesses below
// add a compile-time offset to one computed base.
template <int L> constexpr bool kGroupRows = L == 4096 || L == 16384;
template <int L> __host__ __device__ constexpr int padi(int i)
{
    return i + (i >> 4) + (kGroupRows<L> ? (i >> 8) : 0) + (L == 16384 ? (i >> 12) : 0);
}
template <int L> constexpr int padded() { return kGroupRows<L> ? padi<L>(L - 1) + 1 : L + L / 16; }

// Elements of pass 2 are one complex value (float2) or, in the paired layout,
// the same position of two rows (c2, one row per lane).
template <typename E> constexpr int lanes_of = 1;
template <> constexpr int lanes_of<c2> = 2;
// |z|^2 of each lane
__device__ __forceinline__ float2 abs2(float2 z) { return make_float2(fmaf(z.x, z.x, z.y * z.y), 0.f); }
__device__ __forceinline__ float2 abs2(c2 z) { return __ffma2_rn(z.re, z.re, __fmul2_rn(z.im, z.im)); }
// z of lane l
__device__ __forceinline__ float2 lane(float2 z, int) { return z; }
__device__ __forceinline__ float2 lane(c2 z, int l) { return l ? make_float2(z.re.y, z.im.y) : make_float2(z.re.x, z.im.x); }

// load v[i R + r] = row[j + r L/R] for this thread's tasks j = lt + i L/PPT
template <int L, int R, int PPT, typename E> __device__ __forceinline__ void p2_load(E *v, const E *row, int lt)
{
    constexpr int TPR = L / PPT, T = PPT / R, Q = L / R;
#pragma unroll
    for (int i = 0; i < T; ++i) {
        const E *b = row + padi<L>(lt + i * TPR); // task j = lt + i L/PPT < Q
#pragma unroll
        for (int r = 0; r < R; ++r) v[i * R + r] = b[padi<L>(r * Q)];
    }
}

// Stockham output positions (j / NS) NS R + j mod NS + r NS
template <int L, int R, int NS, int PPT, typename E>
__device__ __forceinline__ void p2_store(const E *v, E *row, int lt)
{
    constexpr int TPR = L / PPT, T = PPT / R;
#pragma unroll
    for (int i = 0; i < T; ++i) {
        const int j = lt + i * TPR;
        // idx is a multiple of NS R plus j mod NS < NS, so the padding splits as above
        E *b = row + padi<L>((j / NS) * NS * R + (j & (NS - 1)));
#pragma unroll
        for (int r = 0; r < R; ++r) b[padi<L>(r * NS)] = v[i * R + r];
    }
}

// twiddles exp(2 pi i (j mod NS) r / (NS R)) from a table laid out r-major,
// tw[r NS + jm], so that consecutive lanes read consecutive words
template <int R, typename E> __device__ __forceinline__ void p2_tw_table(E *u, int j, int NS, const float2 *tw)
{
    const float2 *t = tw + (j & (NS - 1));
#pragma unroll
    for (int r = 1; r < R; ++r) u[r] = cmul(u[r], t[r * NS]);
}

// the same by powers of one accurately computed root w = exp(2 pi i jm / (NS R))
template <int R, typename E> __device__ __forceinline__ void p2_tw_root(E *u, float2 w)
{
    float2 wr = w;
#pragma unroll
    for (int r = 1; r < R; ++r) {
        u[r] = cmul(u[r], wr);
        wr = cmul(wr, w);
    }
}

template <int R> __device__ __forceinline__ float2 p2_root(int j, int NS)
{
    return turn((unsigned)(j & (NS - 1)), (unsigned)(NS * R));
}

// One stage: twiddles from the table `tw` (TABLE), else by powers of the
// roots w[i] that the caller computed ahead (p2_root).
template <int L, int R, int NS, bool TABLE, int PPT, typename E>
__device__ __forceinline__ void p2_stage(E *v, E *row, int lt, const float2 *tw, const float2 *w = nullptr)
{
    constexpr int TPR = L / PPT, T = PPT / R;
    p2_load<L, R, PPT>(v, row, lt);
#pragma unroll
    for (int i = 0; i < T; ++i) {
        const int j = lt + i * TPR;
        if constexpr (TABLE) p2_tw_table<R>(v + i * R, j, NS, tw);
        else p2_tw_root<R>(v + i * R, w[i]);
        dft<R, +1>(v + i * R);
    }
}

// Rare path of the epilogue: one sample above threshold raises its window's
// maximum.  Out of line and with scalar arguments, so that the common path
// keeps every value in registers.
__device__ __noinline__ void p2_emit(Slot *win, int64_t s, int64_t lo, int64_t window, float r2, float zr, float zi,
                                     int *err, int rounds)
{
    slot_max(win + (int)((s - lo) / window), make_key(r2, (uint32_t)s), atan2f(zi, zr), err, rounds);
}

// Each lane's maximum of |z|^2 over this thread's outputs d = j + r L/RL of
// its row; CHECK limits d to [dlo, dhi) (rows that leave the valid range).
template <int L, int RL, bool CHECK, int PPT, typename E>
__device__ __forceinline__ void p2_max(const E *v, int lt, float *m, const int *dlo, const int *dhi)
{
    constexpr int TPR = L / PPT, TL = PPT / RL, NL = lanes_of<E>;
#pragma unroll
    for (int r = 0; r < RL; ++r)
#pragma unroll
        for (int i = 0; i < TL; ++i) {
            const int d = lt + i * TPR + r * (L / RL);
            const float2 a = abs2(v[i * RL + r]);
#pragma unroll
            for (int l = 0; l < NL; ++l)
                if (!CHECK || (d >= dlo[l] && d < dhi[l])) m[l] = fmaxf(m[l], l ? a.y : a.x);
        }
}

// The lowest sample (and its z) among this thread's in-range outputs whose
// |z|^2 equals M; run only by threads that hold the CTA's maximum.
template <int L, int RL, int PPT, typename E>
__device__ __forceinline__ int64_t p2_find(const E *v, int lt, float M, const int64_t *cl, int n1, const int *dlo,
                                           const int *dhi, float2 &zb)
{
    constexpr int TPR = L / PPT, TL = PPT / RL, NL = lanes_of<E>;
    int64_t best = INT64_MAX;
#pragma unroll
    for (int r = 0; r < RL; ++r)
#pragma unroll
        for (int i = 0; i < TL; ++i) {
            const int d = lt + i * TPR + r * (L / RL);
            const float2 a = abs2(v[i * RL + r]);
#pragma unroll
            for (int l = 0; l < NL; ++l) {
                const int64_t s = cl[l] + (int64_t)n1 * d;
                if ((l ? a.y : a.x) == M && d >= dlo[l] && d < dhi[l] && s < best) {
                    best = s;
                    zb = lane(v[i * RL + r], l);
                }
            }
        }
    return best;
}

// Epilogue of a row (pair) whose last stage left output d = lg + i L/PPT +
// r L/RL in v[i RL + r].  Output d of lane l is sample s = c_l + n1 d with
// c_l = c + l n1/2; SPLIT (a row split four ways in frequency) puts 4 n1 in
// place of n1, so s = c + 2 l n1 + 4 n1 d.  |z|^2 is compared before the
// (positive) scaling.  The
// maximum of |z|^2 over the NW warps that share `s_max` is reduced first
// (`bar` is their barrier); only the threads that hold it then look for their
// lowest sample with it and raise a peak slot: the template's global slot, or
// with a shared `local` slot that one (so that no thread waits on an L2 round
// trip here; the caller stores it to global memory later).
template <int L, int RL, int PPT, int NW, bool SPLIT = false, typename E, typename Bar>
__device__ __forceinline__ void p2_epilogue(const E *v, int lg, int c, int y, int t, const FusedArgs &p, float *s_max,
                                            Bar bar, Slot *local = nullptr)
{
    constexpr int NL = lanes_of<E>;
    constexpr int TPR = L / PPT;
    const float inv = p.invnorm[t];
    const int n1 = SPLIT ? 4 * p.n1 : p.n1; // sample step between consecutive outputs d
    const int64_t lo = p.lo, hi = p.hi;
    int64_t cl[NL];
    int dlo[NL], dhi[NL];
    bool full = true;
    float m[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        cl[l] = c + (int64_t)l * (n1 / 2);
        dlo[l] = 0;
        dhi[l] = L;
        if (!(lo <= cl[l] && cl[l] + (int64_t)n1 * (L - 1) < hi)) {
            full = false;
            dlo[l] = (int)max((int64_t)0, (lo - cl[l] + n1 - 1) / n1);
            dhi[l] = (int)min((int64_t)L, hi > cl[l] ? (hi - cl[l] + n1 - 1) / n1 : (int64_t)0);
        }
        m[l] = -1.f;
    }
    if (full) p2_max<L, RL, false, PPT>(v, lg, m, dlo, dhi);
    else p2_max<L, RL, true, PPT>(v, lg, m, dlo, dhi);

    float mx = m[0];
#pragma unroll
    for (int l = 1; l < NL; ++l) mx = fmaxf(mx, m[l]);
    if (mx * inv > p.thr2) {
        constexpr int TL = PPT / RL;
        Slot *win = p.win + (size_t)y * p.nwin;
#pragma unroll
        for (int r = 0; r < RL; ++r)
#pragma unroll
            for (int i = 0; i < TL; ++i) {
                const int d = lg + i * TPR + r * (L / RL);
                const float2 a = abs2(v[i * RL + r]);
#pragma unroll
                for (int l = 0; l < NL; ++l) {
                    const float r2 = (l ? a.y : a.x) * inv;
                    if (r2 > p.thr2 && d >= dlo[l] && d < dhi[l]) {
                        const float2 z = lane(v[i * RL + r], l);
                        p2_emit(win, cl[l] + (int64_t)n1 * d, lo, p.window, r2, z.x, z.y, p.err, p.cas_rounds);
                    }
                }
            }
    }
    float wm = mx;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) wm = fmaxf(wm, __shfl_xor_sync(0xffffffffu, wm, off));
    const int lane_id = threadIdx.x & 31, wid = (threadIdx.x >> 5) % NW;
    if (lane_id == 0) s_max[wid] = wm;
    bar();
    float M = s_max[0];
#pragma unroll
    for (int w = 1; w < NW; ++w) M = fmaxf(M, s_max[w]);
    if (M >= 0.f && mx == M) {
        float2 zb = make_float2(0.f, 0.f);
        const int64_t sb = p2_find<L, RL, PPT>(v, lg, M, cl, n1, dlo, dhi, zb);
        if (local) slot_max_shared(local, make_key(M * inv, (uint32_t)sb), atan2f(zb.y, zb.x), p.err, p.cas_rounds);
        else slot_max(p.peak + t, make_key(M * inv, (uint32_t)sb), atan2f(zb.y, zb.x), p.err, p.cas_rounds);
    }
}

// Grid (rows / RPC, B), rows = n1 (or n1 / 2 row pairs when PAIR).  RPC rows
// (row pairs) of length L, L/PPT threads per row, PPT points per thread.  In the paired layout lane l
// of every element belongs to row c + l n1/2, and each packed FP32x2
// instruction of the transform serves both rows.
template <int L, int RPC, typename ST, int R0, int R1, int R2, int R3, bool PAIR, int PPT>
__global__ void __launch_bounds__(RPC *L / PPT) k_pass2(const FusedArgs p)
{
    using E = std::conditional_t<PAIR, c2, float2>;
    constexpr int NL = lanes_of<E>;
    constexpr int TPR = L / PPT;
    constexpr int NT = RPC * TPR;
    constexpr int LP = padded<L>();
    constexpr int NW = NT / 32;
    constexpr int RL = R3 > 1 ? R3 : (R2 > 1 ? R2 : R1);
    constexpr int NSL = L / RL;
    constexpr size_t ROWB = (size_t)L * NL * sizeof(ST); // bytes of one row (pair) of Y
    extern __shared__ float4 sm4[];
    E *sm = reinterpret_cast<E *>(sm4);
    __shared__ float2 tw1[R0 * R1]; // stage-1 twiddles (sub-transform size R0)
    __shared__ float2 tw2[R3 > 1 ? R0 * R1 * R2 : 1]; // stage-2 twiddles of four-stage rows
    __shared__ float s_max[NW];
    const int tid = threadIdx.x;
    const int rr = tid / TPR, lt = tid % TPR;
    // When the last two radices are 16, the row splits before them into
    // G = L / 256 independent 256-point transforms, transform g touching only
    // the positions = g (mod G).  Thread lt = 16 g + q takes task j = G q + g
    // of those two stages, so each transform lives in one half-warp and the
    // exchange between them needs warp barriers only.
    constexpr bool GROUP = kGroupRows<L> && PPT == 16 && RL == 16 && (R3 > 1 ? R2 : R1) == 16;
    const int lg = GROUP ? (lt & 15) * (L / 256) + (lt >> 4) : lt;
    const int y = blockIdx.y;
    const int t = p.order[p.base + y];
    const int c = blockIdx.x * RPC + rr;
    E *row = sm + rr * LP;
    const char *yslice = (const char *)p.ywork + (size_t)y * (size_t)p.n * sizeof(ST);
    // roots of the last stage's twiddles, when they are not taken from tw1
    float2 wl[R2 == 1 ? 1 : PPT / RL];
    if constexpr (R2 != 1)
#pragma unroll
        for (int i = 0; i < PPT / RL; ++i) wl[i] = p2_root<RL>(lg + i * TPR, NSL);
    E v[PPT];
    {
        constexpr int T = PPT / R0;
        // every load of Y is issued before the twiddle tables are filled, so
        // that their latency overlaps the table arithmetic
#pragma unroll
        for (int i = 0; i < T; ++i)
#pragma unroll
            for (int r = 0; r < R0; ++r)
                v[i * R0 + r] = ld_y<ST, PAIR>(yslice, (size_t)c * L + lt + i * TPR + r * (L / R0));
        // tw1[r R0 + jm] = exp(2 pi i jm r / (R0 R1))
        for (int m = tid; m < R0 * R1; m += NT) tw1[m] = turn((m % R0) * (m / R0), R0 * R1);
        if constexpr (R3 > 1)
            for (int m = tid; m < R0 * R1 * R2; m += NT)
                tw2[m] = turn((m % (R0 * R1)) * (m / (R0 * R1)), R0 * R1 * R2);
#pragma unroll
        for (int i = 0; i < T; ++i) dft<R0, +1>(v + i * R0);
        p2_store<L, R0, 1, PPT>(v, row, lt);
        __syncthreads();
    }
    {
        // Y is read exactly once: invalidate its L2 lines so that, when a batch
        // stays resident in L2 between the passes, they are never written back
        constexpr int LINES = (int)(RPC * ROWB / 128);
        const char *yb = yslice + (size_t)blockIdx.x * RPC * ROWB;
        for (int m = tid; m < LINES; m += NT)
            asm volatile("discard.global.L2 [%0], 128;" ::"l"(yb + (size_t)m * 128) : "memory");
    }
    if constexpr (GROUP && R3 == 1) {
        p2_stage<L, R1, R0, true, PPT>(v, row, lg, tw1);
        __syncwarp();
        p2_store<L, R1, R0, PPT>(v, row, lg);
        __syncwarp();
    } else if constexpr (R2 > 1) {
        p2_stage<L, R1, R0, true, PPT>(v, row, lt, tw1);
        __syncthreads();
        p2_store<L, R1, R0, PPT>(v, row, lt);
        __syncthreads();
        if constexpr (R3 > 1 && GROUP) {
            p2_stage<L, R2, R0 * R1, true, PPT>(v, row, lg, tw2);
            __syncwarp();
            p2_store<L, R2, R0 * R1, PPT>(v, row, lg);
            __syncwarp();
        } else if constexpr (R3 > 1) {
            p2_stage<L, R2, R0 * R1, true, PPT>(v, row, lt, tw2);
            __syncthreads();
            p2_store<L, R2, R0 * R1, PPT>(v, row, lt);
            __syncthreads();
        }
    }
    p2_stage<L, RL, NSL, R2 == 1, PPT>(v, row, lg, tw1, wl);

    p2_epilogue<L, RL, PPT, NW>(v, lg, c, y, t, p, s_max, [] { __syncthreads(); });
}

// ------------------------------------------------------ streamed pass 2 ---
// Pass 2 with its input streamed into shared memory by the bulk-copy (TMA)
// engine, for paired rows of 4096 points (n2 = 4096: N = 2^18, 2^19, 2^20).
// One persistent CTA per SM holds two teams of 256 threads, each with its own
// padded exchange buffer, and one staging buffer S of a row pair.  The CTA's
// row pairs i = blockIdx.x + k gridDim.x alternate between the teams (even k
// team 0, odd k team 1).  A team waits for its row pair to land in S, reads
// its stage-0 inputs from S, and as soon as all of its threads have read S
// one of them issues the bulk copy of the CTA's next row pair (the other
// team's) into S.  The copy then runs while both teams transform, so every SM
// keeps a 64 KB load in flight without holding registers for it, which the
// one-row-pair-per-CTA kernel could not do at two CTAs per SM.  Each team has
// its own mbarrier, so a wait can never be satisfied by the other team's copy.
//
// Every wait is bounded on the global timer (p.copy_wait_ns, one second by
// default).  A team whose wait gives up sets bit 4 of the error word
// (CUI_ERR_TIMEOUT on the host), skips the rest of its work and stops issuing
// copies, so the other team's wait gives up too; before the CTA exits, a copy
// still in flight is waited for (always up to one second), so no copy lands in
// a finished CTA's shared memory.
constexpr int kStreamL = 4096;     // row length of the streamed pass 2
constexpr int kStreamTeam = 256;   // threads per team: L / 16 points per thread
constexpr int kStreamCopies = 4;   // bulk copies per row pair (one mbarrier transaction)

__device__ __forceinline__ uint32_t smem_u32(const void *ptr) { return (uint32_t)__cvta_generic_to_shared(ptr); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// global -> shared bulk copy completing `bytes` transactions on *bar
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until the phase of *bar with parity `parity` has completed; false when
// `limit_ns` pass first (at once for a limit of 0, which only tests use).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned long long limit_ns)
{
    if (limit_ns == 0) return false;
    const uint32_t a = smem_u32(bar);
    unsigned long long t0 = 0;
    for (unsigned it = 0;; ++it) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (ok) return true;
        const unsigned long long now = global_ns();
        if (it == 0) t0 = now;
        else if (now - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void named_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int nthreads)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <typename ST> __device__ __forceinline__ c2 pair_from(pair_t<ST> q);
template <> __device__ __forceinline__ c2 pair_from<float2>(float4 q)
{
    return {make_float2(q.x, q.y), make_float2(q.z, q.w)};
}
template <> __device__ __forceinline__ c2 pair_from<__nv_bfloat162>(uint2 q)
{
    return {__bfloat1622float2(*(const __nv_bfloat162 *)&q.x), __bfloat1622float2(*(const __nv_bfloat162 *)&q.y)};
}

template <typename ST> constexpr size_t stream_stage_bytes() { return (size_t)kStreamL * sizeof(pair_t<ST>); }
template <typename ST> constexpr size_t stream_smem()
{
    return stream_stage_bytes<ST>() + 2 * (size_t)padded<kStreamL>() * sizeof(c2);
}

// Issue the bulk copies of row pair `item` (ROWB bytes at ywork + item ROWB)
// into S on *bar.  One thread.
template <typename ST>
__device__ __forceinline__ void stream_issue(const FusedArgs &p, int item, void *S, uint64_t *bar)
{
    constexpr unsigned ROWB = (unsigned)stream_stage_bytes<ST>();
    constexpr unsigned PART = ROWB / kStreamCopies;
    const char *src = (const char *)p.ywork + (size_t)item * ROWB;
    // the team's generic-proxy reads of S are ordered before the copy's writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, ROWB);
#pragma unroll
    for (int q = 0; q < kStreamCopies; ++q) bulk_load((char *)S + q * PART, src + q * PART, PART, bar);
}

// Grid min(SMs, rows pairs of the batch), 2 teams of 256 threads; row pair
// i of the batch is template y = i / (n1/2), row pair c = i mod (n1/2).
template <typename ST> __global__ void __launch_bounds__(2 * kStreamTeam, 1) k_pass2_stream(const FusedArgs p, int count)
{
    constexpr int L = kStreamL, PPT = 16, R = 16, TPR = kStreamTeam, NW = TPR / 32;
    constexpr int LP = padded<L>();
    constexpr size_t ROWB = stream_stage_bytes<ST>();
    extern __shared__ __align__(128) float4 sm4[];
    pair_t<ST> *S = reinterpret_cast<pair_t<ST> *>(sm4);
    __shared__ float2 tw1[R * R];
    __shared__ float s_max[2][NW];
    __shared__ __align__(8) uint64_t full[2];
    __shared__ int abort_flag[2], issued[2], consumed[2];
    __shared__ Slot s_peak[2]; // each team's peak of its current row pair
    const int tid = threadIdx.x;
    const int team = tid / TPR, lt = tid % TPR;
    // last two stages on half-warp groups (as in k_pass2 for 4096-point rows)
    const int lg = (lt & 15) * (L / 256) + (lt >> 4);
    c2 *row = reinterpret_cast<c2 *>((char *)sm4 + ROWB) + team * LP;
    const int npairs = p.n1 / 2;
    const int total = count * npairs; // <= 4096 templates x 128 row pairs
    const int G = gridDim.x;
    const int bar_release = 1 + 2 * team, bar_team = 2 + 2 * team;

    for (int m = tid; m < R * R; m += 2 * TPR) tw1[m] = turn((m % R) * (m / R), R * R);
    if (tid == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag[0] = abort_flag[1] = 0;
        issued[0] = issued[1] = 0;
        consumed[0] = consumed[1] = 0;
        s_peak[0] = s_peak[1] = Slot{0ull, 0u, 0u};
    }
    __syncthreads();
    if (tid == 0 && (int)blockIdx.x < total) {
        issued[0] = 1;
        stream_issue<ST>(p, blockIdx.x, S, &full[0]);
    }
    // root of the last stage's twiddles: the same for every row pair
    const float2 wl = p2_root<R>(lg, L / R);

    int j = 0;     // row pairs this team has taken
    int prev = -1; // the team's previous row pair, whose peak record is still in s_peak
    for (int i = blockIdx.x + team * G; i < total; i += 2 * G, ++j) {
        if (!mbar_wait(&full[team], j & 1, p.copy_wait_ns)) {
            abort_flag[team] = 1;
            atomicOr(p.err, 4);
        }
        c2 v[PPT];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = pair_from<ST>(S[lt + r * (L / R)]);
        // S is free once every thread of the team has read it: the team's
        // first warp waits for the others and issues the next row pair
        if (lt < 32) {
            named_sync(bar_release, TPR);
            if (lt == 0 && !abort_flag[team] && i + G < total) {
                issued[team ^ 1] += 1;
                stream_issue<ST>(p, i + G, S, &full[team ^ 1]);
            }
        } else {
            named_arrive(bar_release, TPR);
        }
        dft<R, +1>(v);
        p2_store<L, R, 1, PPT>(v, row, lt);
        named_sync(bar_team, TPR);
        if (abort_flag[team]) break; // the same in every thread of the team after the barrier
        if (lt == 0 && prev >= 0) { // the previous row pair's peak (its CAS came before this barrier)
            p.prec[prev] = s_peak[team];
            s_peak[team] = Slot{0ull, 0u, 0u};
        }
        prev = i;
        const int y = i / npairs, c = i % npairs;
        {
            // Y is read exactly once: drop its L2 lines so that they are never written back
            const char *yb = (const char *)p.ywork + (size_t)i * ROWB;
            for (int m = lt; m < (int)(ROWB / 128); m += TPR)
                asm volatile("discard.global.L2 [%0], 128;" ::"l"(yb + (size_t)m * 128) : "memory");
        }
        p2_stage<L, R, R, true, PPT>(v, row, lg, tw1);
        __syncwarp();
        p2_store<L, R, R, PPT>(v, row, lg);
        __syncwarp();
        p2_stage<L, R, L / R, false, PPT>(v, row, lg, tw1, &wl);
        const int t = p.order[p.base + y];
        p2_epilogue<L, R, PPT, NW>(v, lg, c, y, t, p, s_max[team], [bar_team] { named_sync(bar_team, TPR); },
                                   &s_peak[team]);
    }
    if (lt == 0) consumed[team] = j;
    __syncthreads();
    if (lt == 0 && prev >= 0) p.prec[prev] = s_peak[team]; // the team's last row pair
    // a team that gave up can leave one copy in flight: let it land first
    if (tid == 0)
        for (int q = 0; q < 2; ++q)
            if (issued[q] > consumed[q] && !mbar_wait(&full[q], consumed[q] & 1, kCopyWaitNs)) atomicOr(p.err, 4);
}

// Streamed pass 2 for rows of 16384 points (N = 2^22 with n1 = 256), on the
// paired arithmetic of the 4096-point rows.  Split in frequency four ways,
// b = b' + 4096 m and d = 4 k + q (b', k < 4096; m, q < 4):
//   z[4 k + q] = sum_b' exp(2 pi i b' k / 4096) u_q[b'],
//   u_q[b'] = exp(2 pi i q b' / 16384) sum_m i^(m q) x[b' + 4096 m],
// a row is four independent 4096-point transforms.  Team 0 runs q = 0 and 2,
// team 1 q = 1 and 3, each pair as the two lanes of one packed transform, the
// transform of k_pass2_stream.  Each team computes its u from the row in
// shared memory: the first half (b < 8192) in the staging buffer S, the second
// half in the first bytes of team 0's exchange buffer.  One persistent CTA of
// two teams per SM, one row at a time: once both teams have read the row, the
// next row's first half is copied into S (it lands while the row is
// transformed) and, once team 0's last stage has read its exchange buffer, the
// next row's second half into that buffer (it lands during team 0's epilogue
// and the rest of team 1's transform).  Waits and the error path as in
// k_pass2_stream.
constexpr int kStream16L = 16384;
template <typename ST> constexpr size_t s16_half_bytes() { return (size_t)(kStream16L / 2) * sizeof(ST); }
template <typename ST> constexpr size_t s16_smem()
{
    return s16_half_bytes<ST>() + 2 * (size_t)padded<kStreamL>() * sizeof(c2);
}

template <typename ST> __device__ __forceinline__ float2 elem_from(ST q);
template <> __device__ __forceinline__ float2 elem_from<float2>(float2 q) { return q; }
template <> __device__ __forceinline__ float2 elem_from<__nv_bfloat162>(__nv_bfloat162 q) { return __bfloat1622float2(q); }

// Copy half `h` (0 or 1) of row `item` (ROWB = 2 HALF bytes at ywork + item ROWB)
// into dst, completing its bytes on *bar.  One thread.
template <typename ST>
__device__ __forceinline__ void s16_issue_half(const FusedArgs &p, int item, int h, void *dst, uint64_t *bar)
{
    constexpr unsigned HALF = (unsigned)s16_half_bytes<ST>();
    const char *src = (const char *)p.ywork + (size_t)item * 2 * HALF + (size_t)h * HALF;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 2; ++q) bulk_load((char *)dst + q * (HALF / 2), src + q * (HALF / 2), HALF / 2, bar);
}

__device__ __forceinline__ Slot larger_slot(Slot a, Slot b) { return b.key > a.key ? b : a; }

// Grid min(SMs, rows of the batch), 2 teams of 256 threads; row i of the batch
// is template y = i / n1, row c = i mod n1.
template <typename ST> __global__ void __launch_bounds__(2 * kStreamTeam, 1) k_pass2_split16k(const FusedArgs p, int count)
{
    constexpr int L = kStreamL, PPT = 16, R = 16, TPR = kStreamTeam, NW = TPR / 32;
    constexpr int LP = padded<L>();
    constexpr unsigned HALF = (unsigned)s16_half_bytes<ST>();
    extern __shared__ __align__(128) float4 sm4[];
    const ST *S = reinterpret_cast<const ST *>(sm4);
    c2 *xb = reinterpret_cast<c2 *>((char *)sm4 + HALF);  // the teams' exchange buffers
    const ST *W = reinterpret_cast<const ST *>(xb);       // the row's second half, in team 0's buffer
    __shared__ float2 tw1[R * R];
    __shared__ float s_max[2][NW];
    __shared__ __align__(8) uint64_t full;
    __shared__ int abort_flag, issued;
    __shared__ Slot s_peak[2][2]; // [row parity][team]: each team's peak of the row
    // exp(2 pi i q b' / 16384) at b' = lt + 256 r is rt[q][lt] st[q]^r (q = 1, 2, 3)
    __shared__ float2 rt[3][kStreamTeam], st[3];
    const int tid = threadIdx.x;
    const int team = tid / TPR, lt = tid % TPR;
    const int lg = (lt & 15) * (L / 256) + (lt >> 4); // the last two stages on half-warp groups
    c2 *row = xb + team * LP;
    const int n1 = p.n1;
    const int total = count * n1; // <= 64 templates x 256 rows in practice (4 GiB of Y at most)
    const int G = gridDim.x;
    const int bar_team = 1 + team;

    for (int m = tid; m < R * R; m += 2 * TPR) tw1[m] = turn((m % R) * (m / R), R * R);
    for (int m = tid; m < 3 * TPR; m += 2 * TPR) rt[m / TPR][m % TPR] = turn((unsigned)((m / TPR + 1) * (m % TPR)), 4 * L);
    if (tid < 3) st[tid] = turn((unsigned)(tid + 1), 64u);
    if (tid == 0) {
        mbar_init(&full, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
        issued = 0;
        s_peak[0][0] = s_peak[0][1] = s_peak[1][0] = s_peak[1][1] = Slot{0ull, 0u, 0u};
    }
    __syncthreads();
    if (tid == 0 && (int)blockIdx.x < total) {
        issued = 1;
        mbar_expect_tx(&full, 2 * HALF);
        s16_issue_half<ST>(p, blockIdx.x, 0, (void *)S, &full);
        s16_issue_half<ST>(p, blockIdx.x, 1, (void *)W, &full);
    }
    const float2 wl = p2_root<R>(lg, L / R);

    int j = 0, prev = -1;
    for (int i = blockIdx.x; i < total; i += G, ++j) {
        if (!mbar_wait(&full, j & 1, p.copy_wait_ns)) {
            abort_flag = 1;
            atomicOr(p.err, 4);
        }
        c2 v[PPT];
        // the twiddled lanes: team 0 q = 2, team 1 q = 1 and 3
        const int qa = team ? 0 : 1;
        const float2 st_a = st[qa];
        float2 wa = rt[qa][lt];
        if (team == 0) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int b = lt + r * (L / R);
                const float2 x0 = elem_from<ST>(S[b]), x1 = elem_from<ST>(S[b + L]);
                const float2 x2 = elem_from<ST>(W[b]), x3 = elem_from<ST>(W[b + L]);
                const float2 s0 = make_float2(x0.x + x2.x, x0.y + x2.y), s1 = make_float2(x1.x + x3.x, x1.y + x3.y);
                const float2 u2 = cmul(make_float2(s0.x - s1.x, s0.y - s1.y), wa);
                v[r] = c2{make_float2(s0.x + s1.x, u2.x), make_float2(s0.y + s1.y, u2.y)};
                wa = cmul(wa, st_a);
            }
        } else {
            // both lanes twiddled: the twiddle pair (q = 1, 3) is a c2, stepped and
            // applied with packed products
            const float2 ta = rt[0][lt], tb = rt[2][lt], sa = st[0], sb = st[2];
            c2 T = {make_float2(ta.x, tb.x), make_float2(ta.y, tb.y)};
            const float2 sre = make_float2(sa.x, sb.x), sim = make_float2(sa.y, sb.y);
            const float2 nsim = make_float2(-sa.y, -sb.y);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int b = lt + r * (L / R);
                const float2 x0 = elem_from<ST>(S[b]), x1 = elem_from<ST>(S[b + L]);
                const float2 x2 = elem_from<ST>(W[b]), x3 = elem_from<ST>(W[b + L]);
                const float2 d0 = make_float2(x0.x - x2.x, x0.y - x2.y), d1 = make_float2(x1.x - x3.x, x1.y - x3.y);
                // q = 1: d0 + i d1; q = 3: d0 - i d1 (and the negated imaginary parts)
                const float2 pre = make_float2(d0.x - d1.y, d0.x + d1.y), pim = make_float2(d0.y + d1.x, d0.y - d1.x);
                const float2 npim = make_float2(-d0.y - d1.x, d1.x - d0.y);
                v[r] = c2{__ffma2_rn(T.im, npim, __fmul2_rn(T.re, pre)), __ffma2_rn(T.im, pre, __fmul2_rn(T.re, pim))};
                T = c2{__ffma2_rn(T.im, nsim, __fmul2_rn(T.re, sre)), __ffma2_rn(T.im, sre, __fmul2_rn(T.re, sim))};
            }
        }
        __syncthreads(); // both teams have read the row; abort_flag settled
        if (abort_flag) break;
        const bool has_next = i + G < total;
        if (tid == 0) {
            if (prev >= 0) { // the previous row's peak (both teams raised their slots before this barrier)
                Slot *q = s_peak[(j + 1) & 1];
                p.prec[prev] = larger_slot(q[0], q[1]);
                q[0] = q[1] = Slot{0ull, 0u, 0u};
            }
            if (has_next) { // the next row's first half lands while this row is transformed
                issued += 1;
                mbar_expect_tx(&full, 2 * HALF);
                s16_issue_half<ST>(p, i + G, 0, (void *)S, &full);
            }
        }
        prev = i;
        {
            // Y is read exactly once: drop its L2 lines so that they are never written back
            const char *yb = (const char *)p.ywork + (size_t)i * 2 * HALF;
            for (int m = tid; m < (int)(2 * HALF / 128); m += 2 * TPR)
                asm volatile("discard.global.L2 [%0], 128;" ::"l"(yb + (size_t)m * 128) : "memory");
        }
        dft<R, +1>(v);
        p2_store<L, R, 1, PPT>(v, row, lt);
        named_sync(bar_team, TPR);
        p2_stage<L, R, R, true, PPT>(v, row, lg, tw1);
        __syncwarp();
        p2_store<L, R, R, PPT>(v, row, lg);
        __syncwarp();
        p2_stage<L, R, L / R, false, PPT>(v, row, lg, tw1, &wl);
        const int y = i / n1, c = i % n1;
        const int t = p.order[p.base + y];
        // the epilogue's team barrier follows every thread's last read of the
        // team's exchange buffer: then team 0's may take the next row's second half
        p2_epilogue<L, R, PPT, NW, true>(
            v, lg, c + team * n1, y, t, p, s_max[team],
            [&] {
                named_sync(bar_team, TPR);
                if (tid == 0 && has_next) s16_issue_half<ST>(p, i + G, 1, (void *)W, &full);
            },
            &s_peak[j & 1][team]);
    }
    __syncthreads();
    if (tid == 0) {
        if (prev >= 0) p.prec[prev] = larger_slot(s_peak[(j + 1) & 1][0], s_peak[(j + 1) & 1][1]); // the last row's peak
        // a wait that gave up leaves that row's copies in flight: let them land first
        if (issued > j && !mbar_wait(&full, j & 1, kCopyWaitNs)) atomicOr(p.err, 4);
    }
}

// ------------------------------------------------------------ dispatch ----
// Opt the kernel in to `bytes` of dynamic shared memory.  Always set: the
// 48 KB default covers static plus dynamic memory, so a dynamic size below
// 48 KB can still need the opt-in.
template <typename K> static cudaError_t allow_smem(K kernel, size_t bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

constexpr int kPass1Group = 8;    // templates per pass-1 CTA (2 -> 2.24, 4 -> 2.07, 8 -> 2.02, 16 -> 2.12 us at 2^20)
constexpr int kPairMaxL = 8192;   // pass 2 runs on row pairs up to this row length

static bool paired(int n2) { return n2 <= kPairMaxL; }

size_t fused_pass1_smem(int n1, int ccols) { return (size_t)n1 * ccols * sizeof(float2); }
int fused_records_per_template(int n1, int n2) { return n2 <= kPairMaxL ? n1 / 2 : n1; }

size_t fused_pass2_smem(int n2, int rpc)
{
    if (rpc == 0) return n2 == kStream16L ? s16_smem<float2>() : stream_smem<float2>();
    int lp = n2 + n2 / 16; // padded<L>() of the kernel
    if (n2 == 4096) lp = padded<4096>();
    if (n2 == 16384) lp = padded<16384>();
    return (size_t)rpc * lp * (paired(n2) ? sizeof(c2) : sizeof(float2));
}

bool fused_supported(int log2n) { return log2n >= 12 && log2n <= 22; }

// A tiling has kernels when pass 1 exists for (n1, ccols) and pass 2 for (n2, rpc).
bool fused_tiling_ok(int log2n, int n1, int ccols, int rpc)
{
    if (!fused_supported(log2n) || (n1 != 64 && n1 != 128 && n1 != 256) || (ccols != 16 && ccols != 32 && ccols != 64)) return false;
    const int64_t n2 = (int64_t(1) << log2n) / n1;
    if (n2 % ccols) return false;
    // rpc 0: the streamed persistent pass 2 (k_pass2_stream)
    static const int pass2[][2] = {{64, 32},  {128, 16}, {256, 8},  {512, 4},  {1024, 4},  {2048, 2},
                                   {4096, 2}, {4096, 1}, {4096, 0}, {8192, 1}, {16384, 1}, {16384, 0}};
    for (auto &q : pass2)
        if (q[0] == n2 && q[1] == rpc) return true;
    return false;
}

void fused_default_tiling(int log2n, int *n1, int *ccols, int *rpc)
{
    static const int tab[23][2] = {{0, 0},  {0, 0},  {0, 0},  {0, 0},  {0, 0},  {0, 0},  {0, 0},  {0, 0},
                                   {0, 0},  {0, 0},  {0, 0},  {0, 0},  {64, 32}, {64, 16}, {64, 8}, {64, 4},
                                   {64, 4}, {128, 4}, {256, 4}, {256, 2}, {256, 0}, {256, 1}, {256, 0}};
    *n1 = tab[log2n][0];
    *rpc = tab[log2n][1];
    // N = 2^20: the tiling the autotuner picks on GB300 (streamed pass 2, 16 columns per pass-1 CTA)
    *ccols = log2n == 20 ? 16 : 32;
}

template <int N1, int R0, int R1, int C, typename ST>
static cudaError_t run_pass1(const FusedArgs &a, int count, cudaStream_t s)
{
    auto k = paired(a.n2) ? k_pass1<N1, R0, R1, C, kPass1Group, ST, true> : k_pass1<N1, R0, R1, C, kPass1Group, ST, false>;
    const size_t smem = fused_pass1_smem(N1, C);
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(a.n2 / C), (unsigned)((count + kPass1Group - 1) / kPass1Group));
    k<<<grid, C * N1 / 16, smem, s>>>(a, count);
    return cudaGetLastError();
}

template <typename ST> static cudaError_t pass1_dispatch(const FusedArgs &a, int count, cudaStream_t s)
{
    if (a.ccols == 16) {
        if (a.n1 == 64) return run_pass1<64, 8, 8, 16, ST>(a, count, s);
        if (a.n1 == 128) return run_pass1<128, 8, 16, 16, ST>(a, count, s);
        if (a.n1 == 256) return run_pass1<256, 16, 16, 16, ST>(a, count, s);
    } else if (a.ccols == 32) {
        if (a.n1 == 64) return run_pass1<64, 8, 8, 32, ST>(a, count, s);
        if (a.n1 == 128) return run_pass1<128, 8, 16, 32, ST>(a, count, s);
        if (a.n1 == 256) return run_pass1<256, 16, 16, 32, ST>(a, count, s);
    } else if (a.ccols == 64) {
        if (a.n1 == 64) return run_pass1<64, 8, 8, 64, ST>(a, count, s);
        if (a.n1 == 128) return run_pass1<128, 8, 16, 64, ST>(a, count, s);
        if (a.n1 == 256) return run_pass1<256, 16, 16, 64, ST>(a, count, s);
    }
    return cudaErrorInvalidValue;
}

template <int L, int RPC, typename ST, int R0, int R1, int R2, int R3, int PPT = 16>
static cudaError_t run_pass2(const FusedArgs &a, int count, cudaStream_t s)
{
    constexpr bool PAIR = L <= kPairMaxL;
    auto k = k_pass2<L, RPC, ST, R0, R1, R2, R3, PAIR, PPT>;
    const size_t smem = fused_pass2_smem(L, RPC);
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(a.n1 / (PAIR ? 2 : 1) / RPC), (unsigned)count);
    k<<<grid, RPC * L / PPT, smem, s>>>(a);
    return cudaGetLastError();
}

static int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return n;
}

template <typename ST> static cudaError_t run_pass2_stream(const FusedArgs &a, int count, cudaStream_t s)
{
    auto k = k_pass2_stream<ST>;
    const size_t smem = stream_smem<ST>();
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess) return e;
    const int64_t total = (int64_t)count * (a.n1 / 2);
    const int sms = sm_count();
    if (sms <= 0) return cudaErrorInvalidDevice;
    if (total <= 0) return cudaSuccess;
    k<<<(unsigned)std::min<int64_t>(sms, total), 2 * kStreamTeam, smem, s>>>(a, count);
    return cudaGetLastError();
}

template <typename ST> static cudaError_t run_pass2_split16k(const FusedArgs &a, int count, cudaStream_t s)
{
    auto k = k_pass2_split16k<ST>;
    const size_t smem = s16_smem<ST>();
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess) return e;
    const int64_t total = (int64_t)count * a.n1;
    const int sms = sm_count();
    if (sms <= 0) return cudaErrorInvalidDevice;
    if (total <= 0) return cudaSuccess;
    k<<<(unsigned)std::min<int64_t>(sms, total), 2 * kStreamTeam, smem, s>>>(a, count);
    return cudaGetLastError();
}

template <typename ST> static cudaError_t pass2_dispatch(const FusedArgs &a, int count, cudaStream_t s)
{
    const int L = a.n2, R = a.rpc;
    if (L == kStreamL && R == 0) return run_pass2_stream<ST>(a, count, s);
    if (L == kStream16L && R == 0) return run_pass2_split16k<ST>(a, count, s);
    if (L == 64 && R == 32) return run_pass2<64, 32, ST, 4, 16, 1, 1>(a, count, s);
    if (L == 128 && R == 16) return run_pass2<128, 16, ST, 8, 16, 1, 1>(a, count, s);
    if (L == 256 && R == 8) return run_pass2<256, 8, ST, 16, 16, 1, 1>(a, count, s);
    if (L == 512 && R == 4) return run_pass2<512, 4, ST, 2, 16, 16, 1>(a, count, s);
    if (L == 1024 && R == 4) return run_pass2<1024, 4, ST, 4, 16, 16, 1>(a, count, s);
    if (L == 2048 && R == 2) return run_pass2<2048, 2, ST, 8, 16, 16, 1>(a, count, s);
    if (L == 4096 && R == 2) return run_pass2<4096, 2, ST, 16, 16, 16, 1>(a, count, s);
    if (L == 4096 && R == 1) return run_pass2<4096, 1, ST, 16, 16, 16, 1>(a, count, s);
    if (L == 8192 && R == 1) return run_pass2<8192, 1, ST, 2, 16, 16, 16>(a, count, s);
    if (L == 16384 && R == 1) return run_pass2<16384, 1, ST, 4, 16, 16, 16>(a, count, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_pass1(const FusedArgs &a, int count, cudaStream_t s)
{
    launched();
    return a.bf16 ? pass1_dispatch<__nv_bfloat162>(a, count, s) : pass1_dispatch<float2>(a, count, s);
}

cudaError_t launch_pass2(const FusedArgs &a, int count, cudaStream_t s)
{
    launched();
    return a.bf16 ? pass2_dispatch<__nv_bfloat162>(a, count, s) : pass2_dispatch<float2>(a, count, s);
}

// ---------------------------------------------------- template read-out ---
// h~_k = df^(-7/6) amp_k exp(-2 pi i Phi(k)) for k = 0 .. N/2 exactly as pass 1
// generates exp(+2 pi i Phi) (same anchors, same cubic), for tests.
__global__ void k_template_out(const FusedArgs p, int t, const double *amp, double dfac, float2 *out)
{
    const int64_t nh = p.n / 2;
    const int n2 = p.n2, C = p.ccols;
    const int khi = p.khi[t];
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= nh; k += (int64_t)gridDim.x * blockDim.x) {
        float2 h = make_float2(0.f, 0.f);
        if (k >= p.k_low && k < khi) {
            const int a = (int)(k / n2), b = (int)(k % n2), cb = b / C;
            const int64_t ai = (int64_t)a * (n2 / C) + cb;
            const float4 an = anchor_eval(p, t, ai, (float)((int64_t)n2 * a + cb * C + C / 2));
            const float2 one = make_float2(1.f, 0.f);
            const float2 e = k < p.kex[t] ? rotate(phase_exact(p.coef_df + (int64_t)t * kNB, p.gexact + k * kNB), one)
                                          : gen_bin(an, (float)(b - cb * C - C / 2), one);
            const float m = (float)(amp[k] * dfac);
            h = make_float2(m * e.x, -m * e.y);
        }
        out[k] = h;
    }
}

cudaError_t launch_template_out(const FusedArgs &a, int t, const double *amp, double dfac, float2 *out,
                                cudaStream_t s)
{
    k_template_out<<<1216, 256, 0, s>>>(a, t, amp, dfac, out);
    launched();
    return cudaGetLastError();
}

// ------------------------------------------------- direct band sums ----
constexpr int kSumWarps = 8;    // warps of a band-correlator CTA (one query each)
constexpr int kChisqWarps = 32; // warps of a chi^2 CTA (one trigger each: fewer, longer CTAs)

// This thread's share of sum_{ka <= k < kb} q_k exp(2 pi i k u / 2^64), with
// q_k generated exactly as pass 1 generates it (same anchors, cubic and
// exact-phase table) and the time u a 64-bit fraction of the segment (sample
// s is u = s 2^64 / N).  Lane j of a warp evaluates the anchor of block
// base + j; the warp then sweeps those blocks of C bins.
// q_k exp(2 pi i k u / 2^64) for one bin k of block anchor a (offset x in the block)
__device__ __forceinline__ float2 band_term(const FusedArgs &p, const float2 *cdf, int kex, float4 a, int k, int x,
                                            uint64_t u)
{
    const float2 w = p.wbar[k];
    const float2 q = k < kex ? rotate(phase_exact(cdf, p.gexact + (int64_t)k * kNB), w)
                             : gen_bin(a, (float)(x - p.ccols / 2), w);
    // the turn k u / 2^64 mod 1, from the top 32 bits of k u mod 2^64, in [-1/2, 1/2)
    const float fr = (float)(int32_t)(uint32_t)(((uint64_t)k * u) >> 32) * 2.3283064365386963e-10f;
    float sn, cs;
    __sincosf(6.283185307179586f * fr, &sn, &cs);
    return cmul(q, make_float2(cs, sn));
}

template <int NW> __device__ float2 band_sum(const FusedArgs &p, int t, const float2 *cdf, int ka, int kb, uint64_t u)
{
    float2 acc = make_float2(0.f, 0.f);
    if (kb <= ka) return acc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int C = p.ccols, kex = p.kex[t];
    const int B0 = ka / C, B1 = (kb - 1) / C;
    for (int base = B0 + warp * 32; base <= B1; base += NW * 32) {
        float4 anc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (base + lane <= B1) anc = anchor_eval(p, t, base + lane, (float)((int64_t)(base + lane) * C + C / 2));
        const int nb = min(32, B1 - base + 1);
        // blocks of fewer than 32 bins: the warp sweeps 32 / C blocks at a time
        const int per = C < 32 ? 32 / C : 1;
        for (int j0 = 0; j0 < nb; j0 += per) {
            const int j = j0 + (per > 1 ? lane / C : 0); // this lane's block (< 32)
            const float4 a = make_float4(__shfl_sync(0xffffffffu, anc.x, j), __shfl_sync(0xffffffffu, anc.y, j),
                                         __shfl_sync(0xffffffffu, anc.z, j), __shfl_sync(0xffffffffu, anc.w, j));
            const int B = base + j;
            for (int x = per > 1 ? lane % C : lane; x < C; x += 32) {
                const int k = B * C + x;
                if (j >= nb || k < ka || k >= kb) continue;
                const float2 v = band_term(p, cdf, kex, a, k, x, u);
                acc.x += v.x;
                acc.y += v.y;
            }
        }
    }
    return acc;
}

// All P sub-band sums of one trigger in one sweep over the band
// [bnd[0], bnd[P]): warp w takes the chunks of 32 blocks w, w + NW, ... in
// order and adds its partial sum of sub-band l into part[l][w] (lane 0 only,
// in the warp's order) whenever its sweep leaves l, so every warp does an
// equal share of the bins and the result does not depend on scheduling.
template <int NW>
__device__ void chisq_sweep(const FusedArgs &p, int t, const float2 *cdf, const int *bnd, int P, uint64_t u,
                            float2 (*part)[NW])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ka = bnd[0], kb = bnd[P];
    if (kb <= ka) return;
    const int C = p.ccols, kex = p.kex[t];
    const int B0 = ka / C, B1 = (kb - 1) / C;
    const int per = C < 32 ? 32 / C : 1; // blocks per warp step (C <= 64: at most two bins per lane)
    auto flush = [&](int m, float2 v) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
            v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
        }
        if (lane == 0) part[m][warp] = part[m][warp] + v;
    };
    int l = 0; // the sub-band acc belongs to (the same in every lane)
    float2 acc = make_float2(0.f, 0.f);
    for (int base = B0 + warp * 32; base <= B1; base += NW * 32) {
        float4 anc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (base + lane <= B1) anc = anchor_eval(p, t, base + lane, (float)((int64_t)(base + lane) * C + C / 2));
        const int nb = min(32, B1 - base + 1);
        for (int j0 = 0; j0 < nb; j0 += per) {
            const int j = j0 + (per > 1 ? lane / C : 0);
            const float4 a = make_float4(__shfl_sync(0xffffffffu, anc.x, j), __shfl_sync(0xffffffffu, anc.y, j),
                                         __shfl_sync(0xffffffffu, anc.z, j), __shfl_sync(0xffffffffu, anc.w, j));
            // this step's bins [k0, k1), and the sub-bands l .. le they fall in
            const int k0 = max((base + j0) * C, ka), k1 = min((base + j0 + min(per, nb - j0)) * C, kb);
            while (l < P - 1 && k0 >= bnd[l + 1]) {
                flush(l, acc);
                acc = make_float2(0.f, 0.f);
                ++l;
            }
            int le = l;
            while (le < P - 1 && k1 - 1 >= bnd[le + 1]) ++le;
            // this lane's bins: x0 and, for 64-bin blocks, x0 + 32
            const int x0 = per > 1 ? lane % C : lane;
            const int B = base + j;
            int kk0 = -1, kk1 = -1;
            float2 v0 = make_float2(0.f, 0.f), v1 = make_float2(0.f, 0.f);
            if (j < nb) {
                const int k = B * C + x0;
                if (k >= ka && k < kb) {
                    kk0 = k;
                    v0 = band_term(p, cdf, kex, a, k, x0, u);
                }
                if (x0 + 32 < C && B * C + x0 + 32 >= ka && B * C + x0 + 32 < kb) {
                    kk1 = B * C + x0 + 32;
                    v1 = band_term(p, cdf, kex, a, kk1, x0 + 32, u);
                }
            }
            if (le == l) {
                acc = acc + v0 + v1;
            } else { // an edge inside this step: split the lane's bins by sub-band
                for (int m = l; m <= le; ++m) {
                    float2 s = m == l ? acc : make_float2(0.f, 0.f);
                    if (kk0 >= bnd[m] && kk0 < bnd[m + 1]) s = s + v0;
                    if (kk1 >= bnd[m] && kk1 < bnd[m + 1]) s = s + v1;
                    if (m < le) flush(m, s);
                    else acc = s;
                }
                l = le;
            }
        }
    }
    flush(l, acc);
}

// The CTA's sum of every thread's value, in a fixed order; valid in thread 0.
__device__ float2 cta_sum(float2 acc, float2 *part)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    float2 z = make_float2(0.f, 0.f);
    if (threadIdx.x == 0)
        for (int w = 0; w < kSumWarps; ++w) z = z + part[w];
    __syncthreads();
    return z;
}

// Band correlator at arbitrary times (multi-band search): query i is template
// tmpl[i] at time u[i]; the band is [ka, min(kb, k_hi(t))) with k_hi(t) the
// template's own upper edge (khi0, whatever band the filter calls use).
// out[3 i .. 3 i + 2] = (Re z, Im z, sigma_B^2) in physical units:
// z = zfac sum q_k e^(2 pi i k u) / scale_w and sigma_B^2 = sfac (Pw[kb'] - Pw[ka]).
__global__ void __launch_bounds__(kSumWarps * 32) k_band(const FusedArgs p, const double *prefix,
                                                        const int32_t *khi0, const int32_t *tmpl, const uint64_t *u,
                                                        int ka, int kb, const SegScales *sc, double zfac, double sfac,
                                                        double *out)
{
    __shared__ float2 cdf[kNB];
    __shared__ float2 part[kSumWarps];
    const int i = blockIdx.x;
    const int t = tmpl[i];
    const int kh = min(kb, khi0[t]);
    if (threadIdx.x < kNB) cdf[threadIdx.x] = p.coef_df[(int64_t)t * kNB + threadIdx.x];
    __syncthreads();
    const float2 z = cta_sum(band_sum<kSumWarps>(p, t, cdf, ka, kh, u[i]), part);
    if (threadIdx.x == 0) {
        const double f = zfac / sc->scale_w;
        out[3 * (int64_t)i] = f * (double)z.x;
        out[3 * (int64_t)i + 1] = f * (double)z.y;
        out[3 * (int64_t)i + 2] = kh > ka ? sfac * (prefix[kh] - prefix[ka]) : 0.0;
    }
}

cudaError_t launch_band(const FusedArgs &a, const double *prefix, const int32_t *khi0, const int32_t *tmpl,
                        const uint64_t *u, int n, int ka, int kb, const SegScales *sc, double zfac, double sfac,
                        double *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_band<<<n, kSumWarps * 32, 0, s>>>(a, prefix, khi0, tmpl, u, ka, kb, sc, zfac, sfac, out);
    launched();
    return cudaGetLastError();
}

// --------------------------------------------------------- chi^2 veto ----
// Signal-consistency test at a trigger (template t, sample s): the template's
// band [k_low, k_hi) (as the filter calls use it) is split into P sub-bands of
// equal template power, edges k_l = min{k : Pw[k] - Pw[k_low] >= (l/P)
// (Pw[k_hi] - Pw[k_low])} from the prefix sums Pw of |h~_k|^2 / S_k; the
// sub-band correlators z_l(s) = sum_{k in band l} q_k exp(2 pi i k s / N) are
// summed directly at s; then chi^2 = P sum_l |z_l - z/P|^2 / sigma^2 with
// z = sum_l z_l.
__global__ void __launch_bounds__(kChisqWarps * 32) k_chisq(const FusedArgs p, const double *prefix, const int2 *trig,
                                                           int P, float *chisq, float *rho)
{
    __shared__ int bnd[kChisqMaxBands + 1];
    __shared__ float2 cdf[kNB];
    __shared__ float2 part[kChisqMaxBands][kChisqWarps];
    __shared__ float2 zl[kChisqMaxBands];
    const int i = blockIdx.x;
    const int t = trig[i].x;
    const uint64_t u = (uint64_t)(uint32_t)trig[i].y << (64 - p.log2n);
    const int klo = p.k_low, khi = max(p.khi[t], klo);
    if (threadIdx.x < kNB) cdf[threadIdx.x] = p.coef_df[(int64_t)t * kNB + threadIdx.x];
    if (threadIdx.x <= P) {
        const int l = threadIdx.x;
        int e = l == 0 ? klo : khi;
        if (l > 0 && l < P) {
            // smallest k in [klo, khi] with Pw[k] - Pw[klo] >= (l/P) (Pw[khi] - Pw[klo])
            const double target = prefix[klo] + (prefix[khi] - prefix[klo]) * (double)l / (double)P;
            int lo = klo, hi = khi;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (prefix[mid] >= target) hi = mid;
                else lo = mid + 1;
            }
            e = lo;
        }
        bnd[l] = e;
    }
    __syncthreads();
    // each warp owns part[*][warp]: no barrier between its zeroing and its sums
    for (int l = threadIdx.x & 31; l < P; l += 32) part[l][threadIdx.x >> 5] = make_float2(0.f, 0.f);
    __syncwarp();
    chisq_sweep<kChisqWarps>(p, t, cdf, bnd, P, u, part);
    __syncthreads();
    if (threadIdx.x < P) {
        float2 z = make_float2(0.f, 0.f);
        for (int w = 0; w < kChisqWarps; ++w) z = z + part[threadIdx.x][w];
        zl[threadIdx.x] = z;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float2 z = make_float2(0.f, 0.f);
        for (int l = 0; l < P; ++l) z = z + zl[l];
        const float inv = p.invnorm[t];
        float c2 = 0.f;
        for (int l = 0; l < P; ++l) {
            const float dx = zl[l].x - z.x / P, dy = zl[l].y - z.y / P;
            c2 += dx * dx + dy * dy;
        }
        chisq[i] = P * c2 * inv;
        if (rho) rho[i] = sqrtf((z.x * z.x + z.y * z.y) * inv);
    }
}

cudaError_t launch_chisq(const FusedArgs &a, const double *prefix, const int2 *trig, int n, int bands, float *chisq,
                         float *rho, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_chisq<<<n, kChisqWarps * 32, 0, s>>>(a, prefix, trig, bands, chisq, rho);
    launched();
    return cudaGetLastError();
}

// -------------------------------------------------------------- finalize ---
__device__ __forceinline__ void decode(const Slot &sl, int64_t &sample, float &snr, float &phase)
{
    sample = (int64_t)(0xFFFFFFFFu - (uint32_t)(sl.key & 0xFFFFFFFFull));
    snr = sqrtf(__uint_as_float((uint32_t)(sl.key >> 32)));
    phase = __uint_as_float(sl.phase_bits);
}

// The largest record of template y (key order: rho^2, then the lower sample);
// one warp per template.
__device__ __forceinline__ Slot best_record(const Slot *rec, int nrec)
{
    const int lane = threadIdx.x & 31;
    unsigned long long key = 0ull;
    unsigned int ph = 0u;
    for (int r = lane; r < nrec; r += 32) {
        const Slot q = rec[r];
        if (q.key > key) {
            key = q.key;
            ph = q.phase_bits;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, off);
        const unsigned int p2 = __shfl_xor_sync(0xffffffffu, ph, off);
        if (k2 > key) {
            key = k2;
            ph = p2;
        }
    }
    return Slot{key, ph, 0u};
}

__global__ void k_finalize_records(const FinalizeArgs a)
{
    const int lane = threadIdx.x & 31;
    for (int y = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; y < a.count; y += (gridDim.x * blockDim.x) >> 5) {
        const Slot sl = best_record(a.prec + (size_t)y * a.nrec, a.nrec);
        if (lane != 0) continue;
        const int t = a.order[a.base + y];
        cui_peak o;
        if (sl.key == 0ull) {
            o.sample = a.lo;
            o.snr = 0.f;
            o.phase = 0.f;
        } else {
            decode(sl, o.sample, o.snr, o.phase);
        }
        a.peaks_out[t] = o;
    }
}

__global__ void k_finalize_peaks(const FinalizeArgs a)
{
    for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < a.count; y += gridDim.x * blockDim.x) {
        const int t = a.order[a.base + y];
        Slot sl = a.peak[t];
        cui_peak o;
        if (sl.key == 0ull) {
            o.sample = a.lo;
            o.snr = 0.f;
            o.phase = 0.f;
        } else {
            decode(sl, o.sample, o.snr, o.phase);
        }
        a.peaks_out[t] = o;
        Slot zero = {0ull, 0u, 0u};
        a.peak[t] = zero;
    }
}

__global__ void k_finalize_windows(const FinalizeArgs a)
{
    const int64_t total = (int64_t)a.count * a.nwin;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        Slot sl = a.win[i];
        if (sl.key == 0ull) continue;
        const int y = (int)(i / a.nwin);
        cui_trigger tr;
        tr.tmpl = a.order[a.base + y];
        tr.pad = 0;
        decode(sl, tr.sample, tr.snr, tr.phase);
        const unsigned long long pos = atomicAdd(a.trig_count, 1ull);
        if (pos < (unsigned long long)a.trig_cap) a.trig[pos] = tr;
        cluster_max(a.cluster + (i % a.nwin), sl.key, (uint32_t)tr.tmpl, sl.phase_bits, a.err, a.cas_rounds);
        Slot zero = {0ull, 0u, 0u};
        a.win[i] = zero;
    }
}

cudaError_t launch_finalize(const FinalizeArgs &a, cudaStream_t s)
{
    if (a.prec) {
        const int wb = (a.count + 7) / 8; // 8 warps per CTA, one per template
        k_finalize_records<<<wb < 1216 ? wb : 1216, 256, 0, s>>>(a);
    } else {
        const int pb = (a.count + 255) / 256;
        k_finalize_peaks<<<pb < 1216 ? pb : 1216, 256, 0, s>>>(a);
    }
    const int64_t total = (int64_t)a.count * a.nwin;
    const int64_t wb = (total + 255) / 256;
    k_finalize_windows<<<(unsigned)(wb < 4864 ? (wb > 0 ? wb : 1) : 4864), 256, 0, s>>>(a);
    launched(2);
    return cudaGetLastError();
}

} // namespace cui
