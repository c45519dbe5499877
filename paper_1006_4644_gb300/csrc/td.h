// Time-domain template generator (the paper's own: post-Newtonian order 2.5 in
// phase, 0 in amplitude, two polarisations), TaylorT2 form.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cui {

struct TdArgs {
    double ct[6];   // t(v) = v^-8 sum_k ct[k] v^k  (ct[k] = pre_t a_k / (k - 8))
    double cd[6];   // dt/dv = v^-9 sum_k cd[k] v^k
    double cp[6];   // phi(v) = v^-5 sum_{k != 5} cp[k] v^k + clog ln v
    double clog;
    int kmax;       // highest power kept (twice the PN order)
    double M;       // total mass (s)
    double eta;
    double v_lo, v_hi, t_lo, t_hi;
    double fs;
    int64_t n;
};

// TaylorT2 coefficients of a template (host): the series division of the
// binding-energy and flux brackets, integrated term by term
void td_coefficients(double M, double eta, int pn_x2, TdArgs &a);
double td_time(const TdArgs &a, double v);
cudaError_t launch_td_template(const TdArgs &a, double *hp, double *hx, cudaStream_t s);

} // namespace cui
