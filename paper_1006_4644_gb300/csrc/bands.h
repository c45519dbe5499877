// Band edges of the templates and the coherent sum of two bands' correlators
// (the last step of the multi-band search, Sec. "Online analysis
// considerations").  Host functions shared by every translation unit that
// needs a template's bins, so that one rule defines them.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cui {

// k_low = ceil(f_low / df), at least 1 and clamped to N/2 before the integer
// conversion (an f_low at or above Nyquist leaves every band empty).
int band_k_low(double f_low, double df, int64_t nh);

// k_hi = min(ceil(f_isco / df), N/2) with f_isco = 1 / (6^(3/2) pi M), the
// innermost stable circular orbit of the total mass M = (m1 + m2) G Msun / c^3.
int32_t band_k_hi(double m1, double m2, double df, int64_t nh);

// out[2 i .. 2 i + 1] = (rho, phase) of z = z_h + z_l with
// rho = |z| / sqrt(s2_h + s2_l), phase = arg z, from the band sums
// zh[3 i ..] = (Re z_h, Im z_h, s2_h) and zl[3 i ..] likewise.
cudaError_t launch_band_combine(const double *zh, const double *zl, int n, double *out, cudaStream_t s);

} // namespace cui
