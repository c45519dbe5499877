// Device helpers shared by the library's kernels: complex arithmetic,
// in-register DFTs of radix 2/4/8/16, double-float (FP32 pair) arithmetic and
// the 16-byte "best sample" slot updated with a 128-bit compare-and-swap.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#define CUI_HD __host__ __device__ __forceinline__

namespace cui {

// ---------------------------------------------------------------- complex ---
template <typename R> struct cpx;
template <> struct cpx<float> { using T = float2; };
template <> struct cpx<double> { using T = double2; };
template <typename R> using cpx_t = typename cpx<R>::T;

CUI_HD float2 mk(float x, float y) { return make_float2(x, y); }
CUI_HD double2 mk(double x, double y) { return make_double2(x, y); }
CUI_HD float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
CUI_HD float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
CUI_HD double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
CUI_HD double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
template <typename C> CUI_HD C cmul(C a, C b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename C> CUI_HD C cmulc(C a, C b) { return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); } // a * conj(b)
template <typename C, typename R> CUI_HD C cscale(C a, R s) { return mk(a.x * s, a.y * s); }
// multiply by sign * i  (i for SIGN = +1, -i for SIGN = -1)
template <int SIGN, typename C> CUI_HD C mul_si(C a) { return SIGN > 0 ? mk(-a.y, a.x) : mk(a.y, -a.x); }
// a + sign * i * d and a - sign * i * d
template <int SIGN, typename C> CUI_HD C add_si(C a, C d)
{
    return SIGN > 0 ? mk(a.x - d.y, a.y + d.x) : mk(a.x + d.y, a.y - d.x);
}
template <int SIGN, typename C> CUI_HD C sub_si(C a, C d)
{
    return SIGN > 0 ? mk(a.x + d.y, a.y - d.x) : mk(a.x - d.y, a.y + d.x);
}

// ------------------------------------------------- paired complex (f32x2) ---
// Two independent complex numbers (lanes 0 and 1, e.g. two rows of one
// transform) kept as a real pair and an imaginary pair, so that every add,
// subtract and multiply of a transform is one packed FP32x2 instruction for
// both lanes (sm_100 family).  Multiplying by +-i only exchanges the pairs.
struct c2 {
    float2 re, im;
};

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as one fused multiply-add by -1 (exact product, one rounding)
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 f2neg(float2 a) { return __fmul2_rn(a, make_float2(-1.f, -1.f)); }
__device__ __forceinline__ c2 operator+(c2 a, c2 b) { return {f2add(a.re, b.re), f2add(a.im, b.im)}; }
__device__ __forceinline__ c2 operator-(c2 a, c2 b) { return {f2sub(a.re, b.re), f2sub(a.im, b.im)}; }
// both lanes times the same complex w
__device__ __forceinline__ c2 cmul(c2 a, float2 w)
{
    const float2 wx = make_float2(w.x, w.x), wy = make_float2(w.y, w.y), nwy = make_float2(-w.y, -w.y);
    return {__ffma2_rn(a.im, nwy, __fmul2_rn(a.re, wx)), __ffma2_rn(a.im, wx, __fmul2_rn(a.re, wy))};
}
template <int SIGN> __device__ __forceinline__ c2 mul_si(c2 a)
{
    return SIGN > 0 ? c2{f2neg(a.im), a.re} : c2{a.im, f2neg(a.re)};
}
template <int SIGN> __device__ __forceinline__ c2 add_si(c2 a, c2 d)
{
    return SIGN > 0 ? c2{f2sub(a.re, d.im), f2add(a.im, d.re)} : c2{f2add(a.re, d.im), f2sub(a.im, d.re)};
}
template <int SIGN> __device__ __forceinline__ c2 sub_si(c2 a, c2 d)
{
    return SIGN > 0 ? c2{f2add(a.re, d.im), f2sub(a.im, d.re)} : c2{f2sub(a.re, d.im), f2add(a.im, d.re)};
}

// real type of a complex type
template <typename C> struct real_of { using T = decltype(C{}.x); };
template <> struct real_of<c2> { using T = float; };
template <typename C> using real_t = typename real_of<C>::T;

// ------------------------------------------------------ in-register DFTs ---
// y_k = sum_r v_r exp(SIGN 2 pi i r k / R), in place, natural order.
template <int SIGN, typename C> CUI_HD void dft2(C &a, C &b)
{
    C t = a - b;
    a = a + b;
    b = t;
}

template <int SIGN, typename C> CUI_HD void dft4(C &v0, C &v1, C &v2, C &v3)
{
    const C a0 = v0 + v2, a1 = v0 - v2, a2 = v1 + v3, d = v1 - v3;
    v0 = a0 + a2;
    v2 = a0 - a2;
    v1 = add_si<SIGN>(a1, d);
    v3 = sub_si<SIGN>(a1, d);
}

template <typename R> struct k16 {
    static constexpr R c1 = R(0.92387953251128675613); // cos(pi/8)
    static constexpr R s1 = R(0.38268343236508977173); // sin(pi/8)
    static constexpr R r2 = R(0.70710678118654752440); // cos(pi/4)
};

// omega_8^m for m = 1, 2, 3 applied to a (SIGN-dependent direction)
template <int SIGN, typename C, typename R> CUI_HD C w8(C a, int m)
{
    const R h = k16<R>::r2;
    if (m == 1) return cmul(a, mk(h, SIGN * h));
    if (m == 2) return mul_si<SIGN>(a);
    return cmul(a, mk(-h, SIGN * h));
}

template <int SIGN, typename C> CUI_HD void dft8(C *v)
{
    using R = real_t<C>;
    // r = r1 + 2 r2: DFT4 over r2 for r1 = 0, 1; twiddle w8^(r1 k2); DFT2 over r1.
    dft4<SIGN>(v[0], v[2], v[4], v[6]);
    dft4<SIGN>(v[1], v[3], v[5], v[7]);
    v[3] = w8<SIGN, C, R>(v[3], 1);
    v[5] = w8<SIGN, C, R>(v[5], 2);
    v[7] = w8<SIGN, C, R>(v[7], 3);
    // now a[r1][k2] sits at v[r1 + 2 k2]; output y[k2 + 4 k1] = a[0][k2] +/- a[1][k2]
    C y[8];
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
        y[k2] = v[2 * k2] + v[2 * k2 + 1];
        y[k2 + 4] = v[2 * k2] - v[2 * k2 + 1];
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = y[i];
}

template <int SIGN, typename C> CUI_HD void dft16(C *v)
{
    using R = real_t<C>;
    // r = r1 + 4 r2: DFT4 over r2 for each r1, twiddle w16^(r1 k2), DFT4 over r1.
#pragma unroll
    for (int r1 = 0; r1 < 4; ++r1) dft4<SIGN>(v[r1], v[r1 + 4], v[r1 + 8], v[r1 + 12]);
    // a[r1][k2] at v[r1 + 4 k2]
    const R c1 = k16<R>::c1, s1 = k16<R>::s1, h = k16<R>::r2;
    // w16^m, m = r1 * k2 in {1,2,3,4,6,9}
    v[5] = cmul(v[5], mk(c1, SIGN * s1));          // r1=1,k2=1: m=1
    v[9] = cmul(v[9], mk(h, SIGN * h));            // r1=1,k2=2: m=2
    v[13] = cmul(v[13], mk(s1, SIGN * c1));        // r1=1,k2=3: m=3
    v[6] = cmul(v[6], mk(h, SIGN * h));            // r1=2,k2=1: m=2
    v[10] = mul_si<SIGN>(v[10]);                   // r1=2,k2=2: m=4
    v[14] = cmul(v[14], mk(-h, SIGN * h));         // r1=2,k2=3: m=6
    v[7] = cmul(v[7], mk(s1, SIGN * c1));          // r1=3,k2=1: m=3
    v[11] = cmul(v[11], mk(-h, SIGN * h));         // r1=3,k2=2: m=6
    v[15] = cmul(v[15], mk(-c1, -SIGN * s1));      // r1=3,k2=3: m=9
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) dft4<SIGN>(v[4 * k2], v[4 * k2 + 1], v[4 * k2 + 2], v[4 * k2 + 3]);
    // y[k2 + 4 k1] now at v[4 k2 + k1]: transpose 4x4
    C y[16];
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2)
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) y[k2 + 4 * k1] = v[4 * k2 + k1];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = y[i];
}

template <int R, int SIGN, typename C> CUI_HD void dft(C *v)
{
    if constexpr (R == 2) dft2<SIGN>(v[0], v[1]);
    else if constexpr (R == 4) dft4<SIGN>(v[0], v[1], v[2], v[3]);
    else if constexpr (R == 8) dft8<SIGN>(v);
    else dft16<SIGN>(v);
}

// --------------------------------------------- input-pruned DFTs --------
// DFT4 of (a, b, 0, 0): inputs v2, v3 are not read.
template <int SIGN, typename C> CUI_HD void dft4_lo2(C &v0, C &v1, C &v2, C &v3)
{
    const C a = v0, b = v1;
    v0 = a + b;
    v1 = add_si<SIGN>(a, b);
    v2 = a - b;
    v3 = sub_si<SIGN>(a, b);
}

// DFT_R of v when only v[0 .. NZ) can be nonzero (NZ a power of two <= R):
// the butterflies that would only combine known zeros are skipped, and the
// inputs v[NZ ..) are never read.  Same decompositions as dft8 / dft16.
template <int NZ, int SIGN, typename C> CUI_HD void dft8_nz(C *v)
{
    using R = real_t<C>;
    if constexpr (NZ >= 8) {
        dft8<SIGN>(v);
    } else if constexpr (NZ == 1) {
#pragma unroll
        for (int i = 1; i < 8; ++i) v[i] = v[0];
    } else {
        // r = r1 + 2 r2: first layer over r2
        if constexpr (NZ == 4) {
            dft4_lo2<SIGN>(v[0], v[2], v[4], v[6]);
            dft4_lo2<SIGN>(v[1], v[3], v[5], v[7]);
        } else { // NZ == 2: r2 = 0 only
            v[2] = v[4] = v[6] = v[0];
            v[3] = v[5] = v[7] = v[1];
        }
        v[3] = w8<SIGN, C, R>(v[3], 1);
        v[5] = w8<SIGN, C, R>(v[5], 2);
        v[7] = w8<SIGN, C, R>(v[7], 3);
        C y[8];
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
            y[k2] = v[2 * k2] + v[2 * k2 + 1];
            y[k2 + 4] = v[2 * k2] - v[2 * k2 + 1];
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = y[i];
    }
}

template <int NZ, int SIGN, typename C> CUI_HD void dft16_nz(C *v)
{
    using R = real_t<C>;
    if constexpr (NZ >= 16) {
        dft16<SIGN>(v);
    } else if constexpr (NZ == 1) {
#pragma unroll
        for (int i = 1; i < 16; ++i) v[i] = v[0];
    } else {
        // r = r1 + 4 r2: first layer over r2 gives a[r1][k2] at v[r1 + 4 k2]
        if constexpr (NZ == 8) {
#pragma unroll
            for (int r1 = 0; r1 < 4; ++r1) dft4_lo2<SIGN>(v[r1], v[r1 + 4], v[r1 + 8], v[r1 + 12]);
        } else { // NZ == 2 or 4: r2 = 0 only
#pragma unroll
            for (int r1 = 0; r1 < NZ; ++r1) v[r1 + 4] = v[r1 + 8] = v[r1 + 12] = v[r1];
        }
        const R c1 = k16<R>::c1, s1 = k16<R>::s1, h = k16<R>::r2;
        v[5] = cmul(v[5], mk(c1, SIGN * s1));
        v[9] = cmul(v[9], mk(h, SIGN * h));
        v[13] = cmul(v[13], mk(s1, SIGN * c1));
        if constexpr (NZ >= 4) {
            v[6] = cmul(v[6], mk(h, SIGN * h));
            v[10] = mul_si<SIGN>(v[10]);
            v[14] = cmul(v[14], mk(-h, SIGN * h));
            v[7] = cmul(v[7], mk(s1, SIGN * c1));
            v[11] = cmul(v[11], mk(-h, SIGN * h));
            v[15] = cmul(v[15], mk(-c1, -SIGN * s1));
        }
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
            if constexpr (NZ >= 4) dft4<SIGN>(v[4 * k2], v[4 * k2 + 1], v[4 * k2 + 2], v[4 * k2 + 3]);
            else dft4_lo2<SIGN>(v[4 * k2], v[4 * k2 + 1], v[4 * k2 + 2], v[4 * k2 + 3]);
        }
        C y[16];
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2)
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) y[k2 + 4 * k1] = v[4 * k2 + k1];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = y[i];
    }
}

template <int R, int NZ, int SIGN, typename C> CUI_HD void dft_nz(C *v)
{
    if constexpr (NZ >= R) dft<R, SIGN>(v);
    else if constexpr (R == 8) dft8_nz<NZ, SIGN>(v);
    else if constexpr (R == 16) dft16_nz<NZ, SIGN>(v);
    else dft<R, SIGN>(v); // radix 2 and 4 are not pruned (their inputs are zero-filled by the caller)
}

// ---------------------------------------------- double-float arithmetic ---
// Error-free transformations (Knuth's two-sum, FMA two-product; Dekker 1971)
// on FP32 pairs hi + lo, with intrinsics so no operation is contracted or
// reassociated.
struct df { float hi, lo; };

__device__ __forceinline__ df two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ df quick_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df a, df b)
{
    df s = two_sum(a.hi, b.hi);
    df t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = quick_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_mul(df a, df b)
{
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return quick_two_sum(p, e);
}

// Transform arithmetic on double-float values: the sum keeps the exact
// two-sum of the high parts and adds the low parts once (error ~2^-47 of the
// larger operand, which is what a transform's error is measured against).
// With these operators and `dfc`, the generic DFTs above run in double-float.
__device__ __forceinline__ df operator+(df a, df b)
{
    const df s = two_sum(a.hi, b.hi);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df operator-(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) { return df_mul(a, b); }
__device__ __forceinline__ df operator*(int sign, df a) { return sign > 0 ? a : -a; }

struct dfc {
    df x, y;
};
template <> struct cpx<df> { using T = dfc; };
__device__ __forceinline__ dfc mk(df x, df y) { return {x, y}; }
__device__ __forceinline__ dfc operator+(dfc a, dfc b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ dfc operator-(dfc a, dfc b) { return {a.x - b.x, a.y - b.y}; }

// the radix-16 constants split into high and low floats
constexpr df df_const(double v) { return {(float)v, (float)(v - (double)(float)v)}; }
template <> struct k16<df> {
    static constexpr df c1 = df_const(0.92387953251128675613); // cos(pi/8)
    static constexpr df s1 = df_const(0.38268343236508977173); // sin(pi/8)
    static constexpr df r2 = df_const(0.70710678118654752440); // cos(pi/4)
};

// ------------------------------------------------------ best-sample slot ---
// 16 bytes: key = (float bits of rho^2) << 32 | (0xFFFFFFFF - sample), so the
// largest key is the largest rho^2 and, among equal rho^2, the lowest sample;
// then the phase of z at that sample.  key == 0 means empty.
struct __align__(16) Slot {
    unsigned long long key;
    unsigned int phase_bits;
    unsigned int pad;
};

__device__ __forceinline__ unsigned long long make_key(float rho2, uint32_t sample)
{
    return ((unsigned long long)__float_as_uint(rho2) << 32) | (unsigned long long)(0xFFFFFFFFu - sample);
}

// Rounds of the compare-and-swap loops below before they give up (the
// library's default; a bank can lower it to test the error path).
constexpr int kCasRounds = 1 << 20;
// Time limit of a device wait for a bulk copy (global timer, ns).
constexpr unsigned long long kCopyWaitNs = 1000000000ull;

// Raise the slot to (key, phase) if key is larger.  Lock-free: each failed
// CAS means another thread stored a larger key, so the loop ends after at most
// as many rounds as there are competing writers; the bound (`rounds`) only
// guards against a logic error and is reported through *err.
__device__ __forceinline__ void slot_max(Slot *s, unsigned long long key, float phase, int *err, int rounds)
{
    unsigned long long cur_lo = *(volatile unsigned long long *)&s->key;
    unsigned long long cur_hi = *(volatile unsigned long long *)&s->phase_bits;
    const unsigned long long new_hi = (unsigned long long)__float_as_uint(phase);
    for (int it = 0; it < rounds; ++it) {
        if (cur_lo >= key) return;
        unsigned long long old_lo, old_hi;
        asm volatile("{\n\t.reg .b128 d, c, n;\n\t"
                     "mov.b128 c, {%2, %3};\n\t"
                     "mov.b128 n, {%4, %5};\n\t"
                     "atom.global.cas.b128 d, [%6], c, n;\n\t"
                     "mov.b128 {%0, %1}, d;\n\t}"
                     : "=l"(old_lo), "=l"(old_hi)
                     : "l"(cur_lo), "l"(cur_hi), "l"(key), "l"(new_hi), "l"(s)
                     : "memory");
        if (old_lo == cur_lo && old_hi == cur_hi) return;
        cur_lo = old_lo;
        cur_hi = old_hi;
    }
    atomicOr(err, 2);
}

// slot_max on a slot in shared memory (the same bounded loop, 128-bit CAS in
// the shared state space): for a CTA that reduces its own maximum before one
// plain store of the slot to global memory.
__device__ __forceinline__ void slot_max_shared(Slot *s, unsigned long long key, float phase, int *err, int rounds)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(s);
    unsigned long long cur_lo = *(volatile unsigned long long *)&s->key;
    unsigned long long cur_hi = *(volatile unsigned long long *)&s->phase_bits;
    const unsigned long long new_hi = (unsigned long long)__float_as_uint(phase);
    for (int it = 0; it < rounds; ++it) {
        if (cur_lo >= key) return;
        unsigned long long old_lo, old_hi;
        asm volatile("{\n\t.reg .b128 d, c, n;\n\t"
                     "mov.b128 c, {%2, %3};\n\t"
                     "mov.b128 n, {%4, %5};\n\t"
                     "atom.shared.cas.b128 d, [%6], c, n;\n\t"
                     "mov.b128 {%0, %1}, d;\n\t}"
                     : "=l"(old_lo), "=l"(old_hi)
                     : "l"(cur_lo), "l"(cur_hi), "l"(key), "l"(new_hi), "r"(a)
                     : "memory");
        if (old_lo == cur_lo && old_hi == cur_hi) return;
        cur_lo = old_lo;
        cur_hi = old_hi;
    }
    atomicOr(err, 2);
}

// Bank-wide window slot: raise it to (key, template, phase) if (key, lower
// template) is larger; the template is kept as 0xFFFFFFFF - tmpl in `pad`, so
// among equal keys the lowest template wins.  Same bounded CAS as slot_max.
__device__ __forceinline__ void cluster_max(Slot *s, unsigned long long key, uint32_t tmpl, uint32_t phase_bits,
                                            int *err, int rounds)
{
    const unsigned long long tinv = (unsigned long long)(0xFFFFFFFFu - tmpl);
    const unsigned long long new_hi = (tinv << 32) | (unsigned long long)phase_bits;
    unsigned long long cur_lo = *(volatile unsigned long long *)&s->key;
    unsigned long long cur_hi = *(volatile unsigned long long *)&s->phase_bits;
    for (int it = 0; it < rounds; ++it) {
        if (cur_lo > key || (cur_lo == key && (cur_hi >> 32) >= tinv)) return;
        unsigned long long old_lo, old_hi;
        asm volatile("{\n\t.reg .b128 d, c, n;\n\t"
                     "mov.b128 c, {%2, %3};\n\t"
                     "mov.b128 n, {%4, %5};\n\t"
                     "atom.global.cas.b128 d, [%6], c, n;\n\t"
                     "mov.b128 {%0, %1}, d;\n\t}"
                     : "=l"(old_lo), "=l"(old_hi)
                     : "l"(cur_lo), "l"(cur_hi), "l"(key), "l"(new_hi), "l"(s)
                     : "memory");
        if (old_lo == cur_lo && old_hi == cur_hi) return;
        cur_lo = old_lo;
        cur_hi = old_hi;
    }
    atomicOr(err, 2);
}

// Warp-wide maximum of (key, zr, zi) by key.
__device__ __forceinline__ void warp_max_key(unsigned long long &key, float &zr, float &zi)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, off);
        float r2 = __shfl_xor_sync(0xffffffffu, zr, off);
        float i2 = __shfl_xor_sync(0xffffffffu, zi, off);
        if (k2 > key) { key = k2; zr = r2; zi = i2; }
    }
}

} // namespace cui
