// Device evaluation of the Matern covariance of Eq. 1, shared by tile
// generation and kriging.  See matern.cu for the method.
#pragma once
#include "geo_internal.cuh"

namespace geo {

// Parameters of Eq. 1 prepared for the entry functions below (device side, so
// that a batched launch can read theta from device memory and a single launch
// computes exactly the same values): kind selects a closed form for nu in
// {1/2, 3/2, 5/2}; log_c = (nu - 1) log 2 + log Gamma(nu).
__device__ __forceinline__ MaternP make_matern_dev(const geo_theta& th) {
    MaternP m;
    m.sigma2 = th.sigma2;
    m.inv_beta = 1.0 / th.beta;
    m.nu = th.nu;
    m.nugget = th.nugget;
    m.log_c = (th.nu - 1.0) * 0.69314718055994530942 + lgamma(th.nu);
    m.kind = 0;
    if (th.nu == 0.5) m.kind = 1;
    else if (th.nu == 1.5) m.kind = 2;
    else if (th.nu == 2.5) m.kind = 3;
    return m;
}

// e^x K_nu(x), FP64, x > 0.
__device__ __forceinline__ double ekv_fp64(double nu, double x) {
    const double h = fmin(0.2, 0.45 * rsqrt(x));
    const double u1 = expm1(0.5 * h);       // e^{h/2} - 1
    const double m1 = -expm1(-0.5 * h);     // 1 - e^{-h/2}
    const double r1 = exp(nu * h), ri1 = exp(-nu * h);
    double u = 0.0, mm = 0.0, r = 1.0, ri = 1.0;
    double acc = 0.5;                       // t = 0: exp(0) * cosh(0) with weight 1/2
    for (int k = 1; k < 400; ++k) {
        if ((k & 15) == 0) {                // re-anchor the recurrences
            const double t = k * h;
            u = expm1(0.5 * t);
            mm = -expm1(-0.5 * t);
            r = exp(nu * t);
            ri = exp(-nu * t);
        } else {
            u = fma(u, u1, u) + u1;
            mm = fma(-mm, m1, mm) + m1;
            r *= r1;
            ri *= ri1;
        }
        const double s = u + mm;            // 2 sinh(t/2)
        const double a = 0.5 * x * s * s;   // x (cosh t - 1)
        const double term = exp(-a) * 0.5 * (r + ri);
        acc += term;
        // past the peak of the integrand and negligible
        if (a > 40.0 && x * 0.5 * s * ((1.0 + u) + (1.0 - mm)) > nu) break;  // x sinh t > nu
    }
    return acc * h;
}

// e^x K_nu(x), FP32, x > 0.  The positive terms are summed with a running
// compensation (Kahan), so the sum adds O(u) instead of O(terms * u).
__device__ __forceinline__ float ekv_fp32(float nu, float x) {
    const float h = fminf(0.35f, 0.7f * rsqrtf(x));
    float acc = 0.5f, comp = 0.0f;
    for (int k = 1; k < 128; ++k) {
        const float t = k * h;
        const float u = expm1f(0.5f * t);
        const float mm = -expm1f(-0.5f * t);
        const float s = u + mm;
        const float a = 0.5f * x * s * s;
        const float r = expf(nu * t);
        const float term = expf(-a) * 0.5f * (r + 1.0f / r);
        const float yk = __fsub_rn(term, comp);
        const float tk = __fadd_rn(acc, yk);
        comp = __fsub_rn(__fsub_rn(tk, acc), yk);
        acc = tk;
        if (a > 20.0f && x * sinhf(t) > nu) break;
    }
    return acc * h;
}

__device__ __forceinline__ double matern_fp64(double x, const MaternP& m) {
    switch (m.kind) {
        case 1: return m.sigma2 * exp(-x);
        case 2: return m.sigma2 * (1.0 + x) * exp(-x);
        case 3: return m.sigma2 * (1.0 + x + x * x * (1.0 / 3.0)) * exp(-x);
        default:
            if (x > 745.0) return 0.0;
            return m.sigma2 * exp(m.nu * log(x) - x - m.log_c) * ekv_fp64(m.nu, x);
    }
}

// Exact sum of two floats: s + e = a + b (Knuth's TwoSum).
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
    const float s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
    return s;
}

// FP32 entry from x = xh + xl (xl the low part of r/beta): the closed forms use
// e^{-x} = e^{-xh} (1 - xl), so the error of the argument does not grow with x.
// The general-nu form sigma2 x^nu e^-x / (2^(nu-1) Gamma(nu)) * [e^x K_nu(x)]
// takes its first factor as exp(A) (1 + dA): A = nu log xh - xh - log_c in
// float, dA the exact rounding errors of that sum (two-product, TwoSum) plus
// the first-order effect of xl and of log_c's low part, so the exponent's
// rounding (~x u) does not enter the entry's error.  sigma2 enters as
// s2 + s2_lo (its float rounding would otherwise scale every entry alike).
__device__ __forceinline__ float matern_fp32(float xh, float xl, const MaternP& m, float s2, float s2_lo,
                                             float nu, float log_c, float log_c_lo) {
    float q;
    switch (m.kind) {
        case 1: q = expf(-xh) * (1.0f - xl); break;
        case 2: q = ((1.0f + xh) + xl) * (expf(-xh) * (1.0f - xl)); break;
        case 3: {
            const float x = xh + xl;
            q = (1.0f + x + x * x * (1.0f / 3.0f)) * (expf(-xh) * (1.0f - xl));
            break;
        }
        default: {
            if (xh > 110.0f) return 0.0f;
            const float lg = logf(xh);
            const float pr = __fmul_rn(nu, lg), pe = fmaf(nu, lg, -pr);   // pr + pe = nu * lg exactly
            float e1, e2;
            const float a1 = two_sum(pr, -xh, e1);
            const float a2 = two_sum(a1, -log_c, e2);
            const float dA = ((pe + e1) + e2) - log_c_lo - xl + nu * xl / xh;
            q = expf(a2) * (1.0f + dA) * ekv_fp32(nu, xh);
        }
    }
    return fmaf(s2, q, s2_lo * q);
}

}  // namespace geo
