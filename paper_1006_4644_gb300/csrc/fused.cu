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

#include "internal.h"

namespace cui {

__constant__ DerivConsts c_dc;

void fused_set_consts(const DerivConsts &dc, cudaStream_t s)
{
    cudaMemcpyToSymbolAsync(c_dc, &dc, sizeof(dc), 0, cudaMemcpyHostToDevice, s);
}

// ------------------------------------------------------------ storage ----
template <typename ST> __device__ __forceinline__ void st_c(ST *p, float2 v);
template <> __device__ __forceinline__ void st_c<float2>(float2 *p, float2 v) { *p = v; }
template <> __device__ __forceinline__ void st_c<__nv_bfloat162>(__nv_bfloat162 *p, float2 v)
{
    *p = __float22bfloat162_rn(v);
}
template <typename ST> __device__ __forceinline__ float2 ld_c(const ST *p);
template <> __device__ __forceinline__ float2 ld_c<float2>(const float2 *p) { return *p; }
template <> __device__ __forceinline__ float2 ld_c<__nv_bfloat162>(const __nv_bfloat162 *p)
{
    return __bfloat1622float2(*p);
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
__device__ __forceinline__ float4 anchor_eval(const FusedArgs &p, int t, int64_t ai, float ka)
{
    float tf[kNB];
    float phi0, u7, c5;
    if (!p.df) {
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
        df s = {0.0f, 0.0f};
#pragma unroll
        for (int i = 0; i < kNB; ++i) {
            float2 ci = c[i], gi = g[i];
            df T = df_mul(df{ci.x, ci.y}, df{gi.x, gi.y});
            s = df_add(s, T);
            tf[i] = T.hi;
        }
        float h = __fsub_rn(s.hi, rintf(s.hi));
        phi0 = h + s.lo;
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
// Grid (n2 / C, B).  C columns, n1 = R0 * R1 rows; thread = (column, j).
template <int N1, int R0, int R1, int C, typename ST>
__global__ void __launch_bounds__(C *N1 / 16) k_pass1(const FusedArgs p)
{
    constexpr int NT = C * N1 / 16;
    constexpr int NROW = N1 / 2;
    __shared__ float4 anc[NROW];
    __shared__ float2 tw[N1];
    __shared__ float2 cdf[kNB];
    extern __shared__ float2 sm[]; // [N1][C]
    const int tid = threadIdx.x;
    const int col = tid % C;
    const int jt = tid / C;
    const int y = blockIdx.y;
    const int t = p.order[p.base + y];
    const int cb = blockIdx.x;
    const int n2 = p.n2;
    const int b0 = cb * C;
    const int khi = p.khi[t];
    const int klo = p.k_low;
    const int kex = p.kex[t];
    const int a_lo = ceil_div_pos(klo - b0 - (C - 1), n2);
    const int a_hi = min(NROW, ceil_div_pos(khi - b0, n2));

    for (int m = tid; m < N1; m += NT) tw[m] = turn(m, N1);
    if (tid < kNB) cdf[tid] = p.coef_df[(int64_t)t * kNB + tid];
    for (int a = a_lo + tid; a < a_hi; a += NT) {
        const int64_t ai = (int64_t)a * (n2 / C) + cb;
        anc[a] = anchor_eval(p, t, ai, (float)((int64_t)n2 * a + b0 + C / 2));
    }
    __syncthreads();

    // stage 0: generate q for rows a = j + r N1/R0 of column b0 + col, DFT over r
    constexpr int T0 = 16 / R0;
    float2 v[16];
    const float x = (float)(col - C / 2);
    const int bcol = b0 + col;
#pragma unroll
    for (int i = 0; i < T0; ++i) {
        const int j = jt + i * (N1 / 16);
#pragma unroll
        for (int r = 0; r < R0; ++r) {
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
        dft<R0, +1>(v + i * R0);
    }
#pragma unroll
    for (int i = 0; i < T0; ++i) {
        const int j = jt + i * (N1 / 16);
#pragma unroll
        for (int r = 0; r < R0; ++r) sm[(j * R0 + r) * C + col] = v[i * R0 + r];
    }
    __syncthreads();

    // stage 1 (last): radix R1 with sub-transforms of size R0 done
    constexpr int T1 = 16 / R1;
    const int64_t N = p.n;
    ST *yout = (ST *)p.ywork + (size_t)y * (size_t)N;
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
        // outputs c = j + r N1/R1, times exp(2 pi i b c / N)
        const unsigned mask = (unsigned)(N - 1);
        float2 w = turn(((unsigned)bcol * (unsigned)j) & mask, (unsigned)N);
        const float2 step = turn(((unsigned)bcol * (unsigned)(N1 / R1)) & mask, (unsigned)N);
#pragma unroll
        for (int r = 0; r < R1; ++r) {
            const int c = j + r * (N1 / R1);
            st_c<ST>(yout + (size_t)c * n2 + bcol, cmul(u[r], w));
            w = cmul(w, step);
        }
    }
}

// ---------------------------------------------------------------- pass 2 ---
__device__ __forceinline__ int padi(int i) { return i + (i >> 4); }

template <int L, int R> __device__ __forceinline__ void p2_twiddle(float2 *u, int j, int Ns)
{
    const int jm = j & (Ns - 1);
    float2 w = turn((unsigned)jm, (unsigned)(Ns * R));
    float2 wr = w;
#pragma unroll
    for (int r = 1; r < R; ++r) {
        u[r] = cmul(u[r], wr);
        wr = cmul(wr, w);
    }
}

// middle stage: smem -> registers -> smem (in place, synchronised)
template <int L, int R, int NS> __device__ __forceinline__ void p2_mid(float2 *v, float2 *row, int lt)
{
    constexpr int TPR = L / 16;
    constexpr int T = 16 / R;
#pragma unroll
    for (int i = 0; i < T; ++i) {
        const int j = lt + i * TPR;
        float2 *u = v + i * R;
#pragma unroll
        for (int r = 0; r < R; ++r) u[r] = row[padi(j + r * (L / R))];
        if (NS > 1) p2_twiddle<L, R>(u, j, NS);
        dft<R, +1>(u);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < T; ++i) {
        const int j = lt + i * TPR;
        const int idx = (j / NS) * NS * R + (j & (NS - 1));
#pragma unroll
        for (int r = 0; r < R; ++r) row[padi(idx + r * NS)] = v[i * R + r];
    }
    __syncthreads();
}

// Grid (n1 / RPC, B).  RPC rows of length L, L/16 threads per row.
template <int L, int RPC, typename ST, int R0, int R1, int R2, int R3>
__global__ void __launch_bounds__(RPC *L / 16) k_pass2(const FusedArgs p)
{
    constexpr int TPR = L / 16;
    constexpr int NT = RPC * TPR;
    constexpr int LP = L + L / 16;
    constexpr int NW = (NT + 31) / 32;
    extern __shared__ float2 sm[];
    __shared__ unsigned long long s_key[NW];
    __shared__ float s_zr[NW], s_zi[NW];
    const int tid = threadIdx.x;
    const int rr = tid / TPR, lt = tid % TPR;
    const int y = blockIdx.y;
    const int t = p.order[p.base + y];
    const int c = blockIdx.x * RPC + rr;
    float2 *row = sm + rr * LP;
    const ST *src = (const ST *)p.ywork + (size_t)y * (size_t)p.n + (size_t)c * L;

    float2 v[16];
    // stage 0 straight from global memory (no twiddle)
    {
        constexpr int T = 16 / R0;
#pragma unroll
        for (int i = 0; i < T; ++i) {
            const int j = lt + i * TPR;
#pragma unroll
            for (int r = 0; r < R0; ++r) v[i * R0 + r] = ld_c<ST>(src + j + r * (L / R0));
            dft<R0, +1>(v + i * R0);
        }
#pragma unroll
        for (int i = 0; i < T; ++i) {
            const int j = lt + i * TPR;
#pragma unroll
            for (int r = 0; r < R0; ++r) row[padi(j * R0 + r)] = v[i * R0 + r];
        }
        __syncthreads();
    }
    // middle stages, then the last stage's radix and sub-transform size
    constexpr int RL = R3 > 1 ? R3 : (R2 > 1 ? R2 : R1);
    constexpr int NSL = L / RL;
    if constexpr (R2 > 1) p2_mid<L, R1, R0>(v, row, lt);
    if constexpr (R3 > 1) p2_mid<L, R2, R0 * R1>(v, row, lt);
    // last stage into registers
    constexpr int TL = 16 / RL;
#pragma unroll
    for (int i = 0; i < TL; ++i) {
        const int j = lt + i * TPR;
        float2 *u = v + i * RL;
#pragma unroll
        for (int r = 0; r < RL; ++r) u[r] = row[padi(j + r * (L / RL))];
        p2_twiddle<L, RL>(u, j, NSL);
        dft<RL, +1>(u);
    }

    // epilogue: rho^2 at samples s = c + n1 (j + r L/RL)
    const float inv = p.invnorm[t];
    const int64_t lo = p.lo, hi = p.hi;
    unsigned long long best = 0ull;
    float bzr = 0.f, bzi = 0.f;
#pragma unroll
    for (int i = 0; i < TL; ++i) {
        const int j = lt + i * TPR;
#pragma unroll
        for (int r = 0; r < RL; ++r) {
            const float2 z = v[i * RL + r];
            const int64_t s = (int64_t)c + (int64_t)p.n1 * (j + r * (L / RL));
            if (s >= lo && s < hi) {
                const float r2 = (z.x * z.x + z.y * z.y) * inv;
                const unsigned long long key = make_key(r2, (uint32_t)s);
                if (key > best) {
                    best = key;
                    bzr = z.x;
                    bzi = z.y;
                }
                if (r2 > p.thr2) {
                    const int m = (int)((s - lo) / p.window);
                    slot_max(p.win + (size_t)y * p.nwin + m, key, atan2f(z.y, z.x), p.err);
                }
            }
        }
    }
    warp_max_key(best, bzr, bzi);
    const int lane = tid & 31, wid = tid >> 5;
    if (lane == 0) {
        s_key[wid] = best;
        s_zr[wid] = bzr;
        s_zi[wid] = bzi;
    }
    __syncthreads();
    if (wid == 0) {
        best = lane < NW ? s_key[lane] : 0ull;
        bzr = lane < NW ? s_zr[lane] : 0.f;
        bzi = lane < NW ? s_zi[lane] : 0.f;
        warp_max_key(best, bzr, bzi);
        if (lane == 0 && best != 0ull) slot_max(p.peak + t, best, atan2f(bzi, bzr), p.err);
    }
}

// ------------------------------------------------------------ dispatch ----
template <typename K> static cudaError_t allow_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

size_t fused_pass1_smem(int n1, int ccols) { return (size_t)n1 * ccols * sizeof(float2); }
size_t fused_pass2_smem(int n2, int rpc) { return (size_t)rpc * (n2 + n2 / 16) * sizeof(float2); }

bool fused_supported(int log2n) { return log2n >= 12 && log2n <= 22; }

void fused_default_tiling(int log2n, int *n1, int *ccols, int *rpc)
{
    static const int tab[23][2] = {{0, 0},  {0, 0},  {0, 0},  {0, 0},  {0, 0},  {0, 0},  {0, 0},  {0, 0},
                                   {0, 0},  {0, 0},  {0, 0},  {0, 0},  {64, 32}, {64, 16}, {64, 8}, {64, 4},
                                   {64, 4}, {128, 4}, {256, 4}, {256, 2}, {256, 2}, {256, 1}, {256, 1}};
    *n1 = tab[log2n][0];
    *rpc = tab[log2n][1];
    *ccols = 32;
}

template <int N1, int R0, int R1, int C, typename ST>
static cudaError_t run_pass1(const FusedArgs &a, int count, cudaStream_t s)
{
    auto k = k_pass1<N1, R0, R1, C, ST>;
    const size_t smem = fused_pass1_smem(N1, C);
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(a.n2 / C), (unsigned)count);
    k<<<grid, C * N1 / 16, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename ST> static cudaError_t pass1_dispatch(const FusedArgs &a, int count, cudaStream_t s)
{
    if (a.ccols == 32) {
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

template <int L, int RPC, typename ST, int R0, int R1, int R2, int R3>
static cudaError_t run_pass2(const FusedArgs &a, int count, cudaStream_t s)
{
    auto k = k_pass2<L, RPC, ST, R0, R1, R2, R3>;
    const size_t smem = fused_pass2_smem(L, RPC);
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(a.n1 / RPC), (unsigned)count);
    k<<<grid, RPC * L / 16, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename ST> static cudaError_t pass2_dispatch(const FusedArgs &a, int count, cudaStream_t s)
{
    const int L = a.n2, R = a.rpc;
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

// -------------------------------------------------------------- finalize ---
__device__ __forceinline__ void decode(const Slot &sl, int64_t &sample, float &snr, float &phase)
{
    sample = (int64_t)(0xFFFFFFFFu - (uint32_t)(sl.key & 0xFFFFFFFFull));
    snr = sqrtf(__uint_as_float((uint32_t)(sl.key >> 32)));
    phase = __uint_as_float(sl.phase_bits);
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
        Slot zero = {0ull, 0u, 0u};
        a.win[i] = zero;
    }
}

cudaError_t launch_finalize(const FinalizeArgs &a, cudaStream_t s)
{
    const int pb = (a.count + 255) / 256;
    k_finalize_peaks<<<pb < 1216 ? pb : 1216, 256, 0, s>>>(a);
    const int64_t total = (int64_t)a.count * a.nwin;
    const int64_t wb = (total + 255) / 256;
    k_finalize_windows<<<(unsigned)(wb < 4864 ? (wb > 0 ? wb : 1) : 4864), 256, 0, s>>>(a);
    launched(2);
    return cudaGetLastError();
}

} // namespace cui
