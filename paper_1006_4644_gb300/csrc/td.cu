// Time-domain template generator: the paper's own form of the templates
// (Sec. "template generation": the two polarisations of a circular inspiral
// in the time domain, post-Newtonian order 2.5 in phase and 0 in amplitude),
// which the paper then Fourier transforms and normalises.  The orbital
// evolution is the TaylorT2 form of the PN literature it cites: from the
// binding energy E(v) = -(1/2) eta M v^2 [1 + e1 v^2 + e2 v^4] and the flux
// F(v) = (32/5) eta^2 v^10 [1 + f2 v^2 + f3 v^3 + f4 v^4 + f5 v^5] of circular
// orbits, dt/dv = -E'/F = (5 M / (32 eta)) v^-9 sum_k a_k v^k and
// dphi/dv = (v^3 / M) dt/dv, integrated term by term (t_c = phi_c = 0).  Each
// sample solves t(v) = t_j by Newton in FP64 and writes
// h_+ = v^2 cos 2 phi, h_x = v^2 sin 2 phi.
#include <cmath>

#include "td.h"

namespace cui {

void td_coefficients(double M, double eta, int pn_x2, TdArgs &a)
{
    const double pi = 3.14159265358979323846;
    const double e[6] = {1.0, 0.0, -0.75 - eta / 12.0, 0.0, -27.0 / 8.0 + 19.0 * eta / 8.0 - eta * eta / 24.0, 0.0};
    const double f[6] = {1.0,
                         0.0,
                         -1247.0 / 336.0 - 35.0 * eta / 12.0,
                         4.0 * pi,
                         -44711.0 / 9072.0 + 9271.0 * eta / 504.0 + 65.0 * eta * eta / 18.0,
                         -(8191.0 / 672.0 + 583.0 * eta / 24.0) * pi};
    double num[6], ak[6] = {0, 0, 0, 0, 0, 0};
    for (int k = 0; k < 6; ++k) num[k] = (k + 2) / 2.0 * e[k]; // -E'(v) / (eta M v)
    for (int k = 0; k <= pn_x2; ++k) {
        double s = num[k];
        for (int i = 0; i < k; ++i) s -= ak[i] * f[k - i];
        ak[k] = s;
    }
    const double pre_t = 5.0 * M / (32.0 * eta), pre_p = 5.0 / (32.0 * eta);
    a.kmax = pn_x2;
    a.clog = 0.0;
    for (int k = 0; k < 6; ++k) {
        a.ct[k] = pre_t * ak[k] / (k - 8);
        a.cd[k] = pre_t * ak[k];
        a.cp[k] = k == 5 ? 0.0 : pre_p * ak[k] / (k - 5);
    }
    a.clog = pre_p * ak[5];
    a.M = M;
    a.eta = eta;
}

__host__ __device__ inline double poly(const double *c, int kmax, double v)
{
    double s = 0.0;
    for (int k = kmax; k >= 0; --k) s = s * v + c[k];
    return s;
}

double td_time(const TdArgs &a, double v) { return poly(a.ct, a.kmax, v) / std::pow(v, 8); }

__global__ void k_td_template(const TdArgs a, double *hp, double *hx)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.n; j += (int64_t)gridDim.x * blockDim.x) {
        const double t = -(double)((a.n - j) % a.n) / a.fs;
        double p = 0.0, x = 0.0;
        if (j != 0 && t >= a.t_lo && t <= a.t_hi) {
            // Newton on t(v) = t from the Newtonian inverse (integer powers by
            // products: FP64 pow is the slow path on this GPU)
            double v = sqrt(sqrt(sqrt(5.0 * a.M / (256.0 * a.eta * -t))));
            v = fmin(fmax(v, a.v_lo), a.v_hi);
            for (int it = 0; it < 12; ++it) {
                const double v2 = v * v, v4 = v2 * v2, v8 = v4 * v4;
                const double g = poly(a.ct, a.kmax, v) / v8 - t;
                const double dv = g / (poly(a.cd, a.kmax, v) / (v8 * v));
                v = fmin(fmax(v - dv, a.v_lo), a.v_hi);
                if (fabs(dv) <= 1e-15 * v) break;
            }
            const double v2 = v * v;
            const double phi = poly(a.cp, a.kmax, v) / (v2 * v2 * v) + a.clog * log(v);
            double s, c;
            sincos(2.0 * phi, &s, &c);
            p = v2 * c;
            x = v2 * s;
        }
        hp[j] = p;
        hx[j] = x;
    }
}

cudaError_t launch_td_template(const TdArgs &a, double *hp, double *hx, cudaStream_t s)
{
    k_td_template<<<1216, 256, 0, s>>>(a, hp, hx);
    return cudaGetLastError();
}

} // namespace cui
