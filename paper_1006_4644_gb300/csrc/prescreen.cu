// Learned prescreen: whitened band-power features of a segment, a small
// 1D-conv + MLP network that scores bank regions, and its training (forward,
// backward, deterministic gradient reduction, Adam), all in hand-written
// kernels.  The paper motivates it only in passing (for ~10^6 templates it
// doubts exhaustive filtering, introduction footnote); its shape follows the
// stated configuration: 4 conv1d layers of 32 channels (kernel 5,
// stride 1 then 2, zero padding 2, ReLU), per-channel mean and max pooling,
// MLP 64 -> 128 -> regions, BF16 weights with FP32 accumulation.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace cui {

constexpr int PS_CH = 32, PS_KS = 5, PS_HID = 128, PS_NT = 256;

struct PsLayout {
    int bands, frames, regions;
    int64_t off[12]; // W1 b1 W2 b2 W3 b3 W4 b4 F1 c1 F2 c2 offsets in the flat parameter vector
    int64_t total;
};

PsLayout ps_layout(int bands, int frames, int regions)
{
    PsLayout L;
    L.bands = bands;
    L.frames = frames;
    L.regions = regions;
    int64_t sizes[12];
    int cin = bands;
    for (int l = 0; l < 4; ++l) {
        sizes[2 * l] = (int64_t)PS_CH * cin * PS_KS;
        sizes[2 * l + 1] = PS_CH;
        cin = PS_CH;
    }
    sizes[8] = (int64_t)PS_HID * 2 * PS_CH;
    sizes[9] = PS_HID;
    sizes[10] = (int64_t)regions * PS_HID;
    sizes[11] = regions;
    int64_t o = 0;
    for (int i = 0; i < 12; ++i) {
        L.off[i] = o;
        o += sizes[i];
    }
    L.total = o;
    return L;
}

// ------------------------------------------------------------- features ---
// buf[(s B + b) N + k] = u_k = d~_k sqrt(4 df / S_k) for k in band b, else 0.
__global__ void k_ps_band_fill(const double2 *__restrict__ spec, int64_t spec_stride, double spec_scale,
                               const double *__restrict__ psd, const int2 *__restrict__ band, int bands, int64_t n,
                               double df, int count, float2 *__restrict__ buf)
{
    const int64_t total = (int64_t)count * bands * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = i % n;
        const int64_t sb = i / n;
        const int b = (int)(sb % bands);
        const int64_t s = sb / bands;
        float2 v = make_float2(0.f, 0.f);
        if (k >= band[b].x && k < band[b].y) {
            const double2 d = spec[s * spec_stride + k];
            const double w = spec_scale * sqrt(4.0 * df / psd[k]);
            v = make_float2((float)(d.x * w), (float)(d.y * w));
        }
        buf[i] = v;
    }
}

// feat[s][b][m] = log( mean_{j in frame m} |x_{s,b}(j)|^2 / (2 n_b) ); one warp per frame
__global__ void k_ps_frames(const float2 *__restrict__ x, const int2 *__restrict__ band, int bands, int64_t n,
                            int frame, int count, float *__restrict__ feat)
{
    const int frames = (int)(n / frame);
    const int64_t total = (int64_t)count * bands * frames;
    const int lane = threadIdx.x & 31;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total;
         w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int m = (int)(w % frames);
        const int64_t sb = w / frames;
        const int b = (int)(sb % bands);
        const float2 *p = x + sb * n + (int64_t)m * frame;
        float acc = 0.f;
        for (int j = lane; j < frame; j += 32) acc = fmaf(p[j].x, p[j].x, fmaf(p[j].y, p[j].y, acc));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const int nb = band[b].y - band[b].x;
            feat[w] = nb > 0 ? logf(acc / ((float)frame * 2.0f * (float)nb)) : 0.f;
        }
    }
}

// ------------------------------------------------------------- network ----
struct PsArgs {
    const __nv_bfloat16 *w; // BF16 parameters
    const float *norm;      // [2 B]: per-band mean, then 1 / standard deviation
    PsLayout L;
};

// stage parameters [o0, o0 + n) (BF16) into shared memory as FP32
__device__ __forceinline__ void ps_stage(float *dst, const __nv_bfloat16 *src, int64_t n)
{
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) dst[i] = __bfloat162float(src[i]);
}

// out[o][t] = relu(b[o] + sum_{i,k} W[o][i][k] in[i][s t + k - 2])
__device__ void ps_conv_fwd(const float *W, const float *bias, const float *in, int cin, int lin, int stride,
                            float *out, int lout)
{
    for (int idx = threadIdx.x; idx < PS_CH * lout; idx += blockDim.x) {
        const int o = idx / lout, t = idx % lout;
        float acc = bias[o];
        for (int i = 0; i < cin; ++i) {
            const float *wr = W + (o * cin + i) * PS_KS;
            const float *xr = in + i * lin;
#pragma unroll
            for (int k = 0; k < PS_KS; ++k) {
                const int u = stride * t + k - 2;
                if (u >= 0 && u < lin) acc = fmaf(wr[k], xr[u], acc);
            }
        }
        out[idx] = fmaxf(acc, 0.f);
    }
}

// gradients of one conv layer: dW, db into g (FP32, this sample), din = W^T dout
__device__ void ps_conv_bwd(const float *W, const float *in, int cin, int lin, int stride, const float *dout,
                            int lout, float *gW, float *gb, float *din)
{
    for (int idx = threadIdx.x; idx < PS_CH * cin * PS_KS; idx += blockDim.x) {
        const int k = idx % PS_KS, i = (idx / PS_KS) % cin, o = idx / (PS_KS * cin);
        float acc = 0.f;
        for (int t = 0; t < lout; ++t) {
            const int u = stride * t + k - 2;
            if (u >= 0 && u < lin) acc = fmaf(dout[o * lout + t], in[i * lin + u], acc);
        }
        gW[idx] = acc;
    }
    for (int o = threadIdx.x; o < PS_CH; o += blockDim.x) {
        float acc = 0.f;
        for (int t = 0; t < lout; ++t) acc += dout[o * lout + t];
        gb[o] = acc;
    }
    if (!din) return;
    for (int idx = threadIdx.x; idx < cin * lin; idx += blockDim.x) {
        const int i = idx / lin, u = idx % lin;
        float acc = 0.f;
        for (int o = 0; o < PS_CH; ++o)
#pragma unroll
            for (int k = 0; k < PS_KS; ++k) {
                const int v = u + 2 - k;
                if (v >= 0 && v % stride == 0 && v / stride < lout)
                    acc = fmaf(W[(o * cin + i) * PS_KS + k], dout[o * lout + v / stride], acc);
            }
        din[idx] = acc;
    }
}

// One sample per CTA.  Forward always; with targets, the loss and the
// per-sample gradient (written to grads[s][...], reduced later in a fixed
// order so training is deterministic).
__global__ void __launch_bounds__(PS_NT) k_ps_net(const PsArgs a, const float *__restrict__ feat,
                                                  const float *__restrict__ target, float *__restrict__ logits,
                                                  float *__restrict__ loss, float *__restrict__ grads)
{
    extern __shared__ float sm[];
    const PsLayout &L = a.L;
    const int B = L.bands, T = L.frames, R = L.regions;
    const int s = blockIdx.x;
    const int l1 = T, l2 = (T - 1) / 2 + 1, l3 = (l2 - 1) / 2 + 1, l4 = (l3 - 1) / 2 + 1;
    const int lens[5] = {T, l1, l2, l3, l4};
    // shared memory: weights of the current layer, activations and their gradients
    float *wst = sm;                                             // up to max(R, 2 CH) * HID floats
    float *act[5];
    act[0] = wst + max(R, 2 * PS_CH) * PS_HID + PS_HID + R; // x [B][T]
    act[1] = act[0] + B * T;
    act[2] = act[1] + PS_CH * l1;
    act[3] = act[2] + PS_CH * l2;
    act[4] = act[3] + PS_CH * l3;
    float *pool = act[4] + PS_CH * l4; // [2 CH]
    float *hid = pool + 2 * PS_CH;     // [HID]
    float *z = hid + PS_HID;           // [R]
    float *dz = z + R;                 // [R]
    float *dh = dz + R;                // [HID]
    float *dp = dh + PS_HID;           // [2 CH]
    float *dA = dp + 2 * PS_CH;        // two ping-pong gradient buffers of CH * T floats
    float *dB = dA + PS_CH * T;
    float *red = dB + PS_CH * T;       // [32] reduction scratch
    const int NT = blockDim.x;

    // standardised features (x - mean_b) / std_b
    for (int i = threadIdx.x; i < B * T; i += NT)
        act[0][i] = (feat[(int64_t)s * B * T + i] - a.norm[i / T]) * a.norm[B + i / T];
    // ---- forward
    for (int l = 0; l < 4; ++l) {
        const int cin = l == 0 ? B : PS_CH;
        __syncthreads();
        ps_stage(wst, a.w + L.off[2 * l], (int64_t)PS_CH * cin * PS_KS);
        ps_stage(wst + PS_CH * cin * PS_KS, a.w + L.off[2 * l + 1], PS_CH);
        __syncthreads();
        ps_conv_fwd(wst, wst + PS_CH * cin * PS_KS, act[l], cin, lens[l], l == 0 ? 1 : 2, act[l + 1], lens[l + 1]);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < PS_CH; c += NT) {
        float sum = 0.f, mx = -INFINITY;
        for (int t = 0; t < l4; ++t) {
            const float v = act[4][c * l4 + t];
            sum += v;
            mx = fmaxf(mx, v);
        }
        pool[c] = sum / (float)l4;
        pool[PS_CH + c] = mx;
    }
    ps_stage(wst, a.w + L.off[8], (int64_t)PS_HID * 2 * PS_CH);
    ps_stage(wst + PS_HID * 2 * PS_CH, a.w + L.off[9], PS_HID);
    __syncthreads();
    for (int j = threadIdx.x; j < PS_HID; j += NT) {
        float acc = wst[PS_HID * 2 * PS_CH + j];
        for (int i = 0; i < 2 * PS_CH; ++i) acc = fmaf(wst[j * 2 * PS_CH + i], pool[i], acc);
        hid[j] = fmaxf(acc, 0.f);
    }
    __syncthreads();
    ps_stage(wst, a.w + L.off[10], (int64_t)R * PS_HID);
    ps_stage(wst + R * PS_HID, a.w + L.off[11], R);
    __syncthreads();
    for (int c = threadIdx.x; c < R; c += NT) {
        float acc = wst[R * PS_HID + c];
        for (int j = 0; j < PS_HID; ++j) acc = fmaf(wst[c * PS_HID + j], hid[j], acc);
        z[c] = acc;
        if (logits) logits[(int64_t)s * R + c] = acc;
    }
    __syncthreads();
    if (!target) return;

    // ---- loss = -sum_c y_c log softmax(z)_c, and dz = softmax(z) sum(y) - y
    if (threadIdx.x < 32) {
        float mx = -INFINITY;
        for (int c = threadIdx.x; c < R; c += 32) mx = fmaxf(mx, z[c]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        float se = 0.f, ys = 0.f, yz = 0.f;
        const float *y = target + (int64_t)s * R;
        for (int c = threadIdx.x; c < R; c += 32) {
            se += expf(z[c] - mx);
            ys += y[c];
            yz += y[c] * z[c];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            se += __shfl_xor_sync(0xffffffffu, se, o);
            ys += __shfl_xor_sync(0xffffffffu, ys, o);
            yz += __shfl_xor_sync(0xffffffffu, yz, o);
        }
        const float lse = mx + logf(se);
        if (threadIdx.x == 0) {
            red[0] = lse;
            red[1] = ys;
            if (loss) loss[s] = ys * lse - yz;
        }
    }
    __syncthreads();
    {
        const float lse = red[0], ys = red[1];
        const float *y = target + (int64_t)s * R;
        for (int c = threadIdx.x; c < R; c += NT) dz[c] = expf(z[c] - lse) * ys - y[c];
    }
    __syncthreads();
    float *g = grads + (int64_t)s * L.total;
    // fc2 (weights still staged)
    for (int idx = threadIdx.x; idx < R * PS_HID; idx += NT) g[L.off[10] + idx] = dz[idx / PS_HID] * hid[idx % PS_HID];
    for (int c = threadIdx.x; c < R; c += NT) g[L.off[11] + c] = dz[c];
    for (int j = threadIdx.x; j < PS_HID; j += NT) {
        float acc = 0.f;
        for (int c = 0; c < R; ++c) acc = fmaf(wst[c * PS_HID + j], dz[c], acc);
        dh[j] = hid[j] > 0.f ? acc : 0.f;
    }
    __syncthreads();
    ps_stage(wst, a.w + L.off[8], (int64_t)PS_HID * 2 * PS_CH);
    __syncthreads();
    for (int idx = threadIdx.x; idx < PS_HID * 2 * PS_CH; idx += NT)
        g[L.off[8] + idx] = dh[idx / (2 * PS_CH)] * pool[idx % (2 * PS_CH)];
    for (int j = threadIdx.x; j < PS_HID; j += NT) g[L.off[9] + j] = dh[j];
    for (int i = threadIdx.x; i < 2 * PS_CH; i += NT) {
        float acc = 0.f;
        for (int j = 0; j < PS_HID; ++j) acc = fmaf(wst[j * 2 * PS_CH + i], dh[j], acc);
        dp[i] = acc;
    }
    __syncthreads();
    // pooling: mean spreads dp/T, max routes to the first maximum; then relu'
    float *dcur = dA, *dnext = dB;
    for (int c = threadIdx.x; c < PS_CH; c += NT) {
        int am = 0;
        float mx = act[4][c * l4];
        for (int t = 1; t < l4; ++t)
            if (act[4][c * l4 + t] > mx) {
                mx = act[4][c * l4 + t];
                am = t;
            }
        for (int t = 0; t < l4; ++t) {
            float d = dp[c] / (float)l4 + (t == am ? dp[PS_CH + c] : 0.f);
            dcur[c * l4 + t] = act[4][c * l4 + t] > 0.f ? d : 0.f;
        }
    }
    for (int l = 3; l >= 0; --l) {
        const int cin = l == 0 ? B : PS_CH;
        __syncthreads();
        ps_stage(wst, a.w + L.off[2 * l], (int64_t)PS_CH * cin * PS_KS);
        __syncthreads();
        ps_conv_bwd(wst, act[l], cin, lens[l], l == 0 ? 1 : 2, dcur, lens[l + 1], g + L.off[2 * l],
                    g + L.off[2 * l + 1], l > 0 ? dnext : nullptr);
        __syncthreads();
        if (l > 0) {
            for (int i = threadIdx.x; i < PS_CH * lens[l]; i += NT)
                if (!(act[l][i] > 0.f)) dnext[i] = 0.f;
            float *t = dcur;
            dcur = dnext;
            dnext = t;
        }
    }
}

size_t ps_net_smem(const PsLayout &L)
{
    const int T = L.frames, R = L.regions;
    const int l2 = (T - 1) / 2 + 1, l3 = (l2 - 1) / 2 + 1, l4 = (l3 - 1) / 2 + 1;
    size_t f = (size_t)std::max(R, 2 * PS_CH) * PS_HID + PS_HID + R; // weights + biases
    f += (size_t)L.bands * T + PS_CH * (T + l2 + l3 + l4);          // activations
    f += 2 * PS_CH + PS_HID + 2 * R + PS_HID + 2 * PS_CH;           // pool, hid, z, dz, dh, dp
    f += 2 * (size_t)PS_CH * T + 32;                                // gradient ping-pong, scratch
    return f * sizeof(float);
}

// Per-band standardisation of `count` feature rows [count][B][T]: one CTA per
// band sums x and x^2 in FP64 over the count * T values, each thread a fixed
// strided share and the block a fixed-order reduction (deterministic).
// norm[b] = mean, norm[B + b] = 1 / std (population), 1 where the spread is
// zero or not finite.
__global__ void k_ps_fit_norm(const float *__restrict__ feat, int64_t count, int B, int T, float *__restrict__ norm)
{
    __shared__ double s1[256], s2[256];
    const int b = blockIdx.x;
    double a1 = 0.0, a2 = 0.0;
    const int64_t tot = count * T;
    for (int64_t i = threadIdx.x; i < tot; i += blockDim.x) {
        const double x = feat[(i / T) * B * T + (int64_t)b * T + i % T];
        a1 += x;
        a2 += x * x;
    }
    s1[threadIdx.x] = a1;
    s2[threadIdx.x] = a2;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            s1[threadIdx.x] += s1[threadIdx.x + h];
            s2[threadIdx.x] += s2[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mean = s1[0] / (double)tot;
        const double var = s2[0] / (double)tot - mean * mean;
        const double sd = var > 0.0 ? sqrt(var) : 0.0;
        norm[b] = (float)mean;
        norm[B + b] = sd > 0.0 && isfinite(sd) ? (float)(1.0 / sd) : 1.f;
    }
}

// probs[s][c] (+)= softmax(logits[s])[c] / k for `count` rows of R logits;
// one warp per row.  `first` overwrites, else accumulates (networks are added
// in a fixed order, so the mean is deterministic).
__global__ void k_ps_softmax_mean(const float *__restrict__ logits, int count, int R, float inv_k, int first,
                                  float *__restrict__ probs)
{
    const int lane = threadIdx.x & 31;
    for (int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < count; s += (gridDim.x * blockDim.x) >> 5) {
        const float *z = logits + (int64_t)s * R;
        float mx = -INFINITY;
        for (int c = lane; c < R; c += 32) mx = fmaxf(mx, z[c]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        float se = 0.f;
        for (int c = lane; c < R; c += 32) se += expf(z[c] - mx);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
        const float sc = inv_k / se;
        float *out = probs + (int64_t)s * R;
        for (int c = lane; c < R; c += 32) {
            const float q = expf(z[c] - mx) * sc;
            out[c] = first ? q : out[c] + q;
        }
    }
}

// g[p] = (1/count) sum_s grads[s][p], summed in sample order (deterministic)
__global__ void k_ps_reduce(const float *__restrict__ grads, int64_t P, int count, float *__restrict__ g)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int s = 0; s < count; ++s) acc += grads[(int64_t)s * P + p];
        g[p] = acc / (float)count;
    }
}

// Adam with bias correction; refreshes the BF16 copy used by the network.
__global__ void k_ps_adam(float *__restrict__ theta, float *__restrict__ m, float *__restrict__ v,
                          const float *__restrict__ g, __nv_bfloat16 *__restrict__ w, int64_t P, float lr, float b1,
                          float b2, float eps, float c1, float c2)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
        const float gp = g[p];
        const float mp = b1 * m[p] + (1.f - b1) * gp;
        const float vp = b2 * v[p] + (1.f - b2) * gp * gp;
        m[p] = mp;
        v[p] = vp;
        const float th = theta[p] - lr * (mp / c1) / (sqrtf(vp / c2) + eps);
        theta[p] = th;
        w[p] = __float2bfloat16_rn(th);
    }
}

__global__ void k_ps_to_bf16(const float *__restrict__ theta, __nv_bfloat16 *__restrict__ w, int64_t P)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x)
        w[p] = __float2bfloat16_rn(theta[p]);
}

// Deterministic initialisation from a counter-based hash (SplitMix64 output
// function on seed + index): weights uniform in +-sqrt(6 / fan_in) (+-sqrt(3 /
// fan_in) for the output layer), biases zero.
__device__ __forceinline__ unsigned long long ps_mix(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_ps_init(float *__restrict__ theta, const PsLayout L, unsigned long long seed)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < L.total; p += (int64_t)gridDim.x * blockDim.x) {
        int blk = 11;
        while (blk > 0 && p < L.off[blk]) --blk;
        float val = 0.f;
        if (blk % 2 == 0) {
            const int fan_in = blk < 8 ? (blk == 0 ? L.bands : PS_CH) * PS_KS : (blk == 8 ? 2 * PS_CH : PS_HID);
            const float a = sqrtf((blk == 10 ? 3.f : 6.f) / (float)fan_in);
            const unsigned long long h = ps_mix(seed + (unsigned long long)(p + 1) * 0x9E3779B97F4A7C15ull);
            const float u = (float)(h >> 40) * (1.0f / 16777216.0f); // [0, 1)
            val = (2.f * u - 1.f) * a;
        }
        theta[p] = val;
    }
}

} // namespace cui

// ===================================================================== ABI ==
using namespace cui;

struct cui_prescreen_s {
    cui_prescreen_desc desc;
    cudaStream_t stream = nullptr;
    PsLayout L;
    int log2n = 0;
    int frames = 0;
    std::vector<int2> h_band;
    int2 *d_band = nullptr;
    Twiddles tw = {nullptr, nullptr, nullptr, nullptr, 0, 0};
    float2 *d_fa = nullptr, *d_fb = nullptr; // feature FFT buffers
    int chunk = 0;                            // segments per feature chunk
    float *d_theta = nullptr, *d_m = nullptr, *d_v = nullptr, *d_g = nullptr, *d_grads = nullptr;
    __nv_bfloat16 *d_w = nullptr;
    float *d_loss = nullptr;
    float *d_norm = nullptr;   // [2 B] feature standardisation (mean, 1 / std)
    float *d_logits = nullptr; // [max_batch][regions] scratch of the ensemble scores
    int64_t step = 0;
};

static cui_status ps_fail(cui_status st, const char *msg)
{
    set_last_error(msg);
    return st;
}

#define PS_TRY(call)                                                                                                 \
    do {                                                                                                             \
        cudaError_t e_ = (call);                                                                                     \
        if (e_ != cudaSuccess)                                                                                       \
            return ps_fail(e_ == cudaErrorMemoryAllocation ? CUI_ERR_OOM : CUI_ERR_CUDA, cudaGetErrorString(e_));   \
    } while (0)

static void ps_release(cui_prescreen p)
{
    void *ptrs[] = {p->d_band, p->tw.lo64, p->tw.hi64, p->tw.lo32, p->tw.hi32, p->d_fa, p->d_fb, p->d_theta,
                    p->d_m, p->d_v, p->d_g, p->d_grads, p->d_w, p->d_loss, p->d_norm, p->d_logits};
    for (void *q : ptrs)
        if (q) cudaFree(q);
}

extern "C" cui_status cui_prescreen_create(const cui_prescreen_desc *d, cui_prescreen *out)
{
    if (!d || !out) return ps_fail(CUI_ERR_ARG, "desc and out must be non-NULL");
    *out = nullptr;
    if (d->n < 1024 || (d->n & (d->n - 1)) || d->n > (int64_t(1) << 22))
        return ps_fail(CUI_ERR_ARG, "n must be a power of two in [2^10, 2^22]");
    if (d->bands < 1 || d->bands > 16) return ps_fail(CUI_ERR_ARG, "bands must be in [1, 16]");
    if (d->frame < 32 || (d->frame & 31) || d->n % d->frame) return ps_fail(CUI_ERR_ARG, "frame must be a multiple of 32 dividing n");
    if (d->n / d->frame < 8 || d->n / d->frame > 256) return ps_fail(CUI_ERR_ARG, "n / frame must be in [8, 256]");
    if (d->regions < 2 || d->regions > 256) return ps_fail(CUI_ERR_ARG, "regions must be in [2, 256]");
    if (d->max_batch < 1 || d->max_batch > 4096) return ps_fail(CUI_ERR_ARG, "max_batch must be in [1, 4096]");
    if (!(d->sample_rate > 0) || !std::isfinite(d->sample_rate) || !(d->f_low > 0) || d->f_low >= d->sample_rate / 2)
        return ps_fail(CUI_ERR_ARG, "need a finite sample_rate and 0 < f_low < sample_rate / 2");
    cui_prescreen p = new cui_prescreen_s();
    p->desc = *d;
    p->stream = (cudaStream_t)d->stream;
    p->frames = (int)(d->n / d->frame);
    p->L = ps_layout(d->bands, p->frames, d->regions);
    while ((int64_t(1) << p->log2n) < d->n) ++p->log2n;
    // log-spaced band edges between f_low and fs/2 (bins [k0, k1))
    const double df = d->sample_rate / (double)d->n;
    std::vector<int64_t> k(d->bands + 1);
    for (int b = 0; b <= d->bands; ++b)
        k[b] = (int64_t)std::ceil(d->f_low * std::pow(d->sample_rate / 2 / d->f_low, (double)b / d->bands) / df);
    k[0] = std::max<int64_t>(k[0], 1);
    k[d->bands] = d->n / 2;
    for (int b = 0; b < d->bands; ++b) p->h_band.push_back(make_int2((int)k[b], (int)std::max(k[b], k[b + 1])));
    p->chunk = (int)std::max<int64_t>(1, std::min<int64_t>(64, (int64_t(1) << 27) / (d->n * d->bands)));
    const int64_t P = p->L.total;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
    };
    chk(cudaMalloc(&p->d_band, sizeof(int2) * d->bands));
    p->tw.log2n = p->log2n;
    p->tw.shift = (p->log2n + 1) / 2;
    chk(cudaMalloc(&p->tw.lo64, sizeof(double2) << p->tw.shift));
    chk(cudaMalloc(&p->tw.hi64, sizeof(double2) << (p->log2n - p->tw.shift)));
    chk(cudaMalloc(&p->tw.lo32, sizeof(float2) << p->tw.shift));
    chk(cudaMalloc(&p->tw.hi32, sizeof(float2) << (p->log2n - p->tw.shift)));
    chk(cudaMalloc(&p->d_fa, sizeof(float2) * d->n * d->bands * p->chunk));
    chk(cudaMalloc(&p->d_fb, sizeof(float2) * d->n * d->bands * p->chunk));
    chk(cudaMalloc(&p->d_theta, sizeof(float) * P));
    chk(cudaMalloc(&p->d_m, sizeof(float) * P));
    chk(cudaMalloc(&p->d_v, sizeof(float) * P));
    chk(cudaMalloc(&p->d_g, sizeof(float) * P));
    chk(cudaMalloc(&p->d_grads, sizeof(float) * P * d->max_batch));
    chk(cudaMalloc(&p->d_w, sizeof(__nv_bfloat16) * P));
    chk(cudaMalloc(&p->d_loss, sizeof(float) * d->max_batch));
    chk(cudaMalloc(&p->d_norm, sizeof(float) * 2 * d->bands));
    chk(cudaMalloc(&p->d_logits, sizeof(float) * d->max_batch * d->regions));
    if (e != cudaSuccess) {
        ps_release(p);
        delete p;
        return ps_fail(e == cudaErrorMemoryAllocation ? CUI_ERR_OOM : CUI_ERR_CUDA, cudaGetErrorString(e));
    }
    const cudaStream_t s = p->stream;
    chk(cudaMemcpyAsync(p->d_band, p->h_band.data(), sizeof(int2) * d->bands, cudaMemcpyHostToDevice, s));
    launch_twiddle_tables(p->tw, s);
    k_ps_init<<<256, 256, 0, s>>>(p->d_theta, p->L, (unsigned long long)d->seed);
    k_ps_to_bf16<<<256, 256, 0, s>>>(p->d_theta, p->d_w, P);
    launched(2);
    chk(cudaMemsetAsync(p->d_m, 0, sizeof(float) * P, s));
    chk(cudaMemsetAsync(p->d_v, 0, sizeof(float) * P, s));
    {
        // no standardisation until one is fitted or set: mean 0, 1 / std = 1
        std::vector<float> unit(2 * d->bands, 0.f);
        std::fill(unit.begin() + d->bands, unit.end(), 1.f);
        chk(cudaMemcpyAsync(p->d_norm, unit.data(), sizeof(float) * unit.size(), cudaMemcpyHostToDevice, s));
        chk(cudaStreamSynchronize(s)); // the host vector is pageable and goes out of scope
    }
    chk(cudaFuncSetAttribute(k_ps_net, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ps_net_smem(p->L)));
    chk(cudaGetLastError());
    chk(cudaStreamSynchronize(s));
    if (e != cudaSuccess) {
        ps_release(p);
        delete p;
        return ps_fail(CUI_ERR_CUDA, cudaGetErrorString(e));
    }
    *out = p;
    return CUI_OK;
}

extern "C" void cui_prescreen_destroy(cui_prescreen p)
{
    if (!p) return;
    cudaStreamSynchronize(p->stream);
    ps_release(p);
    delete p;
}

extern "C" cui_status cui_prescreen_info(cui_prescreen p, int64_t *n_params, int32_t *frames)
{
    if (!p) return ps_fail(CUI_ERR_ARG, "prescreen is NULL");
    if (n_params) *n_params = p->L.total;
    if (frames) *frames = p->frames;
    return CUI_OK;
}

static cui_status ps_features_impl(cui_prescreen p, const double2 *spec, int64_t stride, double scale,
                                   const double *psd_dev, int64_t count, float *feat)
{
    const cudaStream_t s = p->stream;
    const int B = p->desc.bands;
    const double df = p->desc.sample_rate / (double)p->desc.n;
    for (int64_t s0 = 0; s0 < count; s0 += p->chunk) {
        const int c = (int)std::min<int64_t>(p->chunk, count - s0);
        k_ps_band_fill<<<1216, 256, 0, s>>>(spec + s0 * stride, stride, scale, psd_dev, p->d_band, B, p->desc.n, df,
                                              c, p->d_fa);
        float2 *x = nullptr;
        launch_fft_passes_f32(p->d_fa, p->d_fb, p->log2n, +1, p->tw, s, &x, c * B);
        k_ps_frames<<<1216, 256, 0, s>>>(x, p->d_band, B, p->desc.n, p->desc.frame, c,
                                           feat + s0 * (int64_t)B * p->frames);
        launched(2);
    }
    PS_TRY(cudaGetLastError());
    return CUI_OK;
}

extern "C" cui_status cui_prescreen_features(cui_prescreen p, const double *dtilde_dev, const double *psd_dev,
                                             int64_t count, float *feat_dev)
{
    if (!p || !dtilde_dev || !psd_dev || !feat_dev || count < 0) return ps_fail(CUI_ERR_ARG, "bad arguments");
    return ps_features_impl(p, (const double2 *)dtilde_dev, p->desc.n / 2 + 1, 1.0, psd_dev, count, feat_dev);
}

extern "C" cui_status cui_prescreen_bank_features(cui_prescreen p, cui_bank bank, float *feat_dev)
{
    if (!p || !bank || !feat_dev) return ps_fail(CUI_ERR_ARG, "bad arguments");
    const double2 *X = nullptr;
    const double *psd = nullptr;
    int64_t n = 0;
    double fs = 0;
    if (!bank_segment_spectrum(bank, &X, &psd, &n, &fs)) return ps_fail(CUI_ERR_STATE, "the bank has no segment");
    if (n != p->desc.n || fs != p->desc.sample_rate)
        return ps_fail(CUI_ERR_ARG, "the bank's segment length or sample rate differs from the prescreen's");
    // the bank holds the unnormalised transform; d~ = X / fs
    return ps_features_impl(p, X, n, 1.0 / fs, psd, 1, feat_dev);
}

static cui_status ps_check_batch(cui_prescreen p, const float *feat, int64_t count)
{
    if (!p || !feat) return ps_fail(CUI_ERR_ARG, "bad arguments");
    if (count < 1 || count > p->desc.max_batch) return ps_fail(CUI_ERR_ARG, "count must be in [1, max_batch]");
    return CUI_OK;
}

extern "C" cui_status cui_prescreen_scores(cui_prescreen p, const float *feat_dev, int64_t count, float *scores_dev)
{
    if (!scores_dev) return ps_fail(CUI_ERR_ARG, "scores_dev is NULL");
    if (!p || !feat_dev || count < 0) return ps_fail(CUI_ERR_ARG, "bad arguments");
    PsArgs a = {p->d_w, p->d_norm, p->L};
    // the attribute is per kernel, shared by prescreens of other sizes: set it per call
    PS_TRY(cudaFuncSetAttribute(k_ps_net, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ps_net_smem(p->L)));
    for (int64_t s0 = 0; s0 < count; s0 += 65535) {
        const int c = (int)std::min<int64_t>(65535, count - s0);
        k_ps_net<<<c, PS_NT, ps_net_smem(p->L), p->stream>>>(a, feat_dev + s0 * p->L.bands * p->frames, nullptr,
                                                            scores_dev + s0 * p->L.regions, nullptr, nullptr);
        launched();
    }
    PS_TRY(cudaGetLastError());
    return CUI_OK;
}

static cui_status ps_grad(cui_prescreen p, const float *feat, const float *target, int64_t count)
{
    PsArgs a = {p->d_w, p->d_norm, p->L};
    PS_TRY(cudaFuncSetAttribute(k_ps_net, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ps_net_smem(p->L)));
    k_ps_net<<<(unsigned)count, PS_NT, ps_net_smem(p->L), p->stream>>>(a, feat, target, nullptr, p->d_loss,
                                                                       p->d_grads);
    k_ps_reduce<<<(unsigned)((p->L.total + 255) / 256), 256, 0, p->stream>>>(p->d_grads, p->L.total, (int)count,
                                                                            p->d_g);
    launched(2);
    PS_TRY(cudaGetLastError());
    return CUI_OK;
}

static cui_status ps_loss(cui_prescreen p, int64_t count, float *loss_host)
{
    if (!loss_host) return CUI_OK;
    std::vector<float> l(count);
    PS_TRY(cudaMemcpyAsync(l.data(), p->d_loss, sizeof(float) * count, cudaMemcpyDeviceToHost, p->stream));
    PS_TRY(cudaStreamSynchronize(p->stream));
    double acc = 0;
    for (float x : l) acc += x;
    *loss_host = (float)(acc / count);
    return CUI_OK;
}

extern "C" cui_status cui_prescreen_gradient(cui_prescreen p, const float *feat_dev, const float *target_dev,
                                             int64_t count, float *grad_dev, float *loss_host)
{
    cui_status st = ps_check_batch(p, feat_dev, count);
    if (st != CUI_OK) return st;
    if (!target_dev || !grad_dev) return ps_fail(CUI_ERR_ARG, "target_dev and grad_dev must be non-NULL");
    if ((st = ps_grad(p, feat_dev, target_dev, count)) != CUI_OK) return st;
    PS_TRY(cudaMemcpyAsync(grad_dev, p->d_g, sizeof(float) * p->L.total, cudaMemcpyDeviceToDevice, p->stream));
    return ps_loss(p, count, loss_host);
}

extern "C" cui_status cui_prescreen_train_step(cui_prescreen p, const float *feat_dev, const float *target_dev,
                                               int64_t count, float *loss_host)
{
    cui_status st = ps_check_batch(p, feat_dev, count);
    if (st != CUI_OK) return st;
    if (!target_dev) return ps_fail(CUI_ERR_ARG, "target_dev must be non-NULL");
    if ((st = ps_grad(p, feat_dev, target_dev, count)) != CUI_OK) return st;
    p->step += 1;
    const cui_prescreen_desc &d = p->desc;
    // bias corrections 1 - beta^t in FP64 (in FP32, 1 - 0.999^t loses four digits to cancellation)
    const float c1 = (float)(1.0 - std::pow((double)d.beta1, (double)p->step));
    const float c2 = (float)(1.0 - std::pow((double)d.beta2, (double)p->step));
    k_ps_adam<<<(unsigned)((p->L.total + 255) / 256), 256, 0, p->stream>>>(p->d_theta, p->d_m, p->d_v, p->d_g,
                                                                          p->d_w, p->L.total, d.lr, d.beta1,
                                                                          d.beta2, d.eps, c1, c2);
    launched();
    PS_TRY(cudaGetLastError());
    return ps_loss(p, count, loss_host);
}

extern "C" cui_status cui_prescreen_get_state(cui_prescreen p, float *theta, float *m, float *v, int64_t *step)
{
    if (!p) return ps_fail(CUI_ERR_ARG, "prescreen is NULL");
    PS_TRY(cudaStreamSynchronize(p->stream));
    const size_t b = sizeof(float) * p->L.total;
    if (theta) PS_TRY(cudaMemcpy(theta, p->d_theta, b, cudaMemcpyDeviceToHost));
    if (m) PS_TRY(cudaMemcpy(m, p->d_m, b, cudaMemcpyDeviceToHost));
    if (v) PS_TRY(cudaMemcpy(v, p->d_v, b, cudaMemcpyDeviceToHost));
    if (step) *step = p->step;
    return CUI_OK;
}

extern "C" cui_status cui_prescreen_set_state(cui_prescreen p, const float *theta, const float *m, const float *v,
                                              int64_t step)
{
    if (!p || !theta || step < 0) return ps_fail(CUI_ERR_ARG, "bad arguments");
    const size_t b = sizeof(float) * p->L.total;
    PS_TRY(cudaStreamSynchronize(p->stream));
    PS_TRY(cudaMemcpy(p->d_theta, theta, b, cudaMemcpyHostToDevice));
    if (m) PS_TRY(cudaMemcpy(p->d_m, m, b, cudaMemcpyHostToDevice));
    else PS_TRY(cudaMemset(p->d_m, 0, b));
    if (v) PS_TRY(cudaMemcpy(p->d_v, v, b, cudaMemcpyHostToDevice));
    else PS_TRY(cudaMemset(p->d_v, 0, b));
    p->step = step;
    k_ps_to_bf16<<<256, 256, 0, p->stream>>>(p->d_theta, p->d_w, p->L.total);
    launched();
    PS_TRY(cudaGetLastError());
    PS_TRY(cudaStreamSynchronize(p->stream));
    return CUI_OK;
}

extern "C" cui_status cui_prescreen_fit_norm(cui_prescreen p, const float *feat_dev, int64_t count)
{
    if (!p || !feat_dev || count < 1) return ps_fail(CUI_ERR_ARG, "bad arguments");
    k_ps_fit_norm<<<p->desc.bands, 256, 0, p->stream>>>(feat_dev, count, p->desc.bands, p->frames, p->d_norm);
    launched();
    PS_TRY(cudaGetLastError());
    return CUI_OK;
}

extern "C" cui_status cui_prescreen_set_norm(cui_prescreen p, const float *mean, const float *stddev)
{
    if (!p || !mean || !stddev) return ps_fail(CUI_ERR_ARG, "bad arguments");
    const int B = p->desc.bands;
    std::vector<float> h(2 * B);
    for (int b = 0; b < B; ++b) {
        if (!std::isfinite(mean[b]) || !(stddev[b] > 0.f) || !std::isfinite(stddev[b]))
            return ps_fail(CUI_ERR_ARG, "mean must be finite and stddev finite and > 0");
        h[b] = mean[b];
        h[B + b] = 1.f / stddev[b];
    }
    PS_TRY(cudaMemcpyAsync(p->d_norm, h.data(), sizeof(float) * 2 * B, cudaMemcpyHostToDevice, p->stream));
    PS_TRY(cudaStreamSynchronize(p->stream));
    return CUI_OK;
}

extern "C" cui_status cui_prescreen_get_norm(cui_prescreen p, float *mean, float *stddev)
{
    if (!p || !mean || !stddev) return ps_fail(CUI_ERR_ARG, "bad arguments");
    const int B = p->desc.bands;
    std::vector<float> h(2 * B);
    PS_TRY(cudaMemcpyAsync(h.data(), p->d_norm, sizeof(float) * 2 * B, cudaMemcpyDeviceToHost, p->stream));
    PS_TRY(cudaStreamSynchronize(p->stream));
    for (int b = 0; b < B; ++b) {
        mean[b] = h[b];
        stddev[b] = 1.f / h[B + b];
    }
    return CUI_OK;
}

extern "C" cui_status cui_prescreen_ensemble_scores(const cui_prescreen *nets, int32_t k, const float *feat_dev,
                                                    int64_t count, float *prob_dev)
{
    if (!nets || k < 1 || !feat_dev || !prob_dev || count < 0) return ps_fail(CUI_ERR_ARG, "bad arguments");
    for (int32_t e = 0; e < k; ++e) {
        if (!nets[e]) return ps_fail(CUI_ERR_ARG, "a network handle is NULL");
        const cui_prescreen_desc &d = nets[e]->desc;
        if (d.bands != nets[0]->desc.bands || nets[e]->frames != nets[0]->frames || d.regions != nets[0]->desc.regions)
            return ps_fail(CUI_ERR_ARG, "the networks differ in bands, frames or regions");
    }
    cui_prescreen p0 = nets[0];
    const int R = p0->desc.regions;
    const int64_t row = (int64_t)p0->desc.bands * p0->frames;
    // every network runs on the first one's stream, into its scratch, in chunks of its max_batch
    for (int64_t s0 = 0; s0 < count; s0 += p0->desc.max_batch) {
        const int c = (int)std::min<int64_t>(p0->desc.max_batch, count - s0);
        for (int32_t e = 0; e < k; ++e) {
            cui_prescreen p = nets[e];
            PsArgs a = {p->d_w, p->d_norm, p->L};
            PS_TRY(cudaFuncSetAttribute(k_ps_net, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ps_net_smem(p->L)));
            if (e > 0 && p->stream != p0->stream) PS_TRY(cudaStreamSynchronize(p->stream)); // its own pending work
            k_ps_net<<<c, PS_NT, ps_net_smem(p->L), p0->stream>>>(a, feat_dev + s0 * row, nullptr, p0->d_logits,
                                                                  nullptr, nullptr);
            k_ps_softmax_mean<<<(c + 7) / 8, 256, 0, p0->stream>>>(p0->d_logits, c, R, 1.f / (float)k, e == 0,
                                                                 prob_dev + s0 * R);
            launched(2);
        }
    }
    PS_TRY(cudaGetLastError());
    return CUI_OK;
}

// ------------------------------------------------------------ ranking ---
// Host work on O(templates) values: the bank in increasing chirp mass
// (stable, so equal masses keep bank order), cut into `regions` equal-count
// groups (the first n mod regions one template longer), the groups taken by
// descending score (equal scores: lower region first).  A region plan keeps
// the sorted bank, so that ranking one segment's scores only sorts the
// region scores.
struct cui_regions_s {
    std::vector<int32_t> by_mc; // template indices in increasing chirp mass
    int32_t regions = 0;
    int64_t start(int64_t r) const
    {
        const int64_t n = (int64_t)by_mc.size(), q = n / regions, rem = n % regions;
        return r * q + std::min<int64_t>(r, rem);
    }
};

static cui_status regions_build(const double *m1, const double *m2, int64_t n, int32_t regions, cui_regions_s &g)
{
    if (!m1 || !m2) return ps_fail(CUI_ERR_ARG, "m1 and m2 must be non-NULL");
    if (n < 0 || n > INT32_MAX) return ps_fail(CUI_ERR_ARG, "n_templates must be in [0, 2^31)");
    if (regions < 1) return ps_fail(CUI_ERR_ARG, "regions must be >= 1");
    std::vector<double> mc((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        if (!(m1[i] > 0.0 && m2[i] > 0.0 && std::isfinite(m1[i]) && std::isfinite(m2[i])))
            return ps_fail(CUI_ERR_ARG, "masses must be finite and > 0");
        mc[(size_t)i] = std::pow(m1[i] * m2[i], 0.6) / std::pow(m1[i] + m2[i], 0.2);
    }
    g.by_mc.resize((size_t)n);
    for (int64_t i = 0; i < n; ++i) g.by_mc[(size_t)i] = (int32_t)i;
    std::stable_sort(g.by_mc.begin(), g.by_mc.end(),
                     [&](int32_t a, int32_t b) { return mc[(size_t)a] < mc[(size_t)b]; });
    g.regions = regions;
    return CUI_OK;
}

static cui_status regions_order(const cui_regions_s &g, const float *scores, int32_t top_k, int32_t *order_out,
                                int64_t *n_out)
{
    if (!scores || !n_out) return ps_fail(CUI_ERR_ARG, "scores and n_out must be non-NULL");
    if (!g.by_mc.empty() && !order_out) return ps_fail(CUI_ERR_ARG, "order_out must be non-NULL");
    if (top_k < 0) return ps_fail(CUI_ERR_ARG, "top_k must be >= 0");
    for (int32_t r = 0; r < g.regions; ++r)
        if (!std::isfinite(scores[r])) return ps_fail(CUI_ERR_ARG, "scores must be finite");
    std::vector<int32_t> ranked((size_t)g.regions);
    for (int32_t r = 0; r < g.regions; ++r) ranked[(size_t)r] = r;
    std::stable_sort(ranked.begin(), ranked.end(), [&](int32_t a, int32_t b) { return scores[a] > scores[b]; });
    int64_t w = 0;
    for (int32_t k = 0; k < std::min(top_k, g.regions); ++k) {
        const int64_t r = ranked[(size_t)k];
        for (int64_t p = g.start(r); p < g.start(r + 1); ++p) order_out[w++] = g.by_mc[(size_t)p];
    }
    *n_out = w;
    return CUI_OK;
}

extern "C" cui_status cui_prescreen_rank(const double *m1, const double *m2, int64_t n_templates, const float *scores,
                                         int32_t regions, int32_t top_k, int32_t *order_out, int64_t *n_out)
{
    if (!scores || !n_out) return ps_fail(CUI_ERR_ARG, "m1, m2, scores and n_out must be non-NULL");
    cui_regions_s g;
    cui_status st = regions_build(m1, m2, n_templates, regions, g);
    if (st != CUI_OK) return st;
    return regions_order(g, scores, top_k, order_out, n_out);
}

extern "C" cui_status cui_regions_create(const double *m1, const double *m2, int64_t n_templates, int32_t regions,
                                         cui_regions *out)
{
    if (!out) return ps_fail(CUI_ERR_ARG, "out must be non-NULL");
    *out = nullptr;
    cui_regions g = new cui_regions_s();
    cui_status st = regions_build(m1, m2, n_templates, regions, *g);
    if (st != CUI_OK) {
        delete g;
        return st;
    }
    *out = g;
    return CUI_OK;
}

extern "C" cui_status cui_regions_order(cui_regions g, const float *scores, int32_t top_k, int32_t *order_out,
                                        int64_t *n_out)
{
    if (!g) return ps_fail(CUI_ERR_ARG, "region plan is NULL");
    return regions_order(*g, scores, top_k, order_out, n_out);
}

extern "C" void cui_regions_destroy(cui_regions g) { delete g; }
