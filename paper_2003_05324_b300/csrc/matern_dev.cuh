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

// Tables and constants of the FP32 exponential and logarithm below, prepared
// on the host in double: 2^(-j/32) = hi[j] + lo[j] (j = 0..31); c = ln2/32 =
// c_hi + c_lo with c_hi holding 11 significant bits (n c_hi is exact in FP32
// for |n| < 2^13), inv_c = 32/ln2 rounded; ln(1 + j/64) = lnc_hi[j] +
// lnc_lo[j] and inv_cj[j] = 1/(1 + j/64) rounded (j = 0..63); ln2 = ln2_hi +
// ln2_lo with ln2_hi holding 16 significant bits.
struct ExpTab {
    float hi[32], lo[32];
    float lnc_hi[64], lnc_lo[64], inv_cj[64];
    float c_hi, c_lo, inv_c, ln2_hi, ln2_lo;
};

// Exact sum of two floats: s + e = a + b (Knuth's TwoSum).
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
    const float s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
    return s;
}

// e^y for y = yh + yl, |y| <= 103, as an unnormalised float pair (eh + el) 2^k
// with relative error below 2^-29, in FP32 arithmetic only (Tang's
// table-driven method, 1989): y = n c + r with n = rint(y / c), c = ln2/32,
// |r| <= c/2 (+ rounding); e^y = 2^(n >> 5) 2^((n & 31)/32) e^r, the middle
// factor from the table (2^(j/32) = 2 * 2^(-(32-j)/32)), e^r = 1 + q with
// q = r + r^2/2 + r^3/6 + r^4/24 (the next term is below 2^-39).  yh - n c_hi
// is exact (Sterbenz), so r carries y's low part and c's second word.
__device__ __forceinline__ void exp_pair(float yh, float yl, const ExpTab& T, float& eh, float& el, int& k) {
    const float nf = rintf(yh * T.inv_c);
    const int n = (int)nf;
    const float r = fmaf(-nf, T.c_lo, __fsub_rn(yh, __fmul_rn(nf, T.c_hi))) + yl;
    const float q = r * fmaf(r, fmaf(r, fmaf(r, 1.0f / 24.0f, 1.0f / 6.0f), 0.5f), 1.0f);
    const int j = n & 31;
    k = n >> 5;
    const float th = j ? 2.0f * T.hi[32 - j] : 1.0f, tl = j ? 2.0f * T.lo[32 - j] : 0.0f;
    eh = th;
    el = fmaf(th, q, fmaf(tl, q, tl));
}

// ln x for x = xh + xl > 0 (xh normal) as a float pair, absolute error below
// 2^-29: xh = m 2^(e-1) with m in [1, 2), m = c_j (1 + d) with c_j = 1 + j/64
// (m - c_j exact, |d| < 1/64), ln x = (e-1) ln2 + ln c_j + ln(1 + d) + xl/xh,
// ln(1 + d) by its series to d^5 (the next term is below 2^-38).
__device__ __forceinline__ void log_pair(float xh, float xl, const ExpTab& T, float& lh, float& ll) {
    int e;
    const float m = 2.0f * frexpf(xh, &e);
    const int j = min(63, (int)((m - 1.0f) * 64.0f));
    const float d = (m - (1.0f + (float)j * (1.0f / 64.0f))) * T.inv_cj[j];
    const float p = d * fmaf(d, fmaf(d, fmaf(d, fmaf(d, 0.2f, -0.25f), 1.0f / 3.0f), -0.5f), 1.0f);
    const float ef = (float)(e - 1);
    float e1, e2;
    const float s1 = two_sum(__fmul_rn(ef, T.ln2_hi), T.lnc_hi[j], e1);
    const float s2 = two_sum(s1, p, e2);
    const float low = (e1 + e2) + fmaf(ef, T.ln2_lo, T.lnc_lo[j]) + xl / xh;
    lh = __fadd_rn(s2, low);
    ll = __fsub_rn(low, __fsub_rn(lh, s2));
}

// 2^e for e <= 127 (exact), 0 below 2^-126: a quadrature term that small is far
// beneath the FP32 resolution of the sum it joins.
__device__ __forceinline__ float pow2i(int e) { return e < -126 ? 0.0f : __int_as_float((e + 127) << 23); }

// e^-x for x = xh + xl >= 0 (see exp_pair).
__device__ __forceinline__ void exp_neg_pair(float xh, float xl, const ExpTab& T, float& eh, float& el, int& k) {
    exp_pair(-xh, -xl, T, eh, el, k);
}

// sigma2 (s2 + s2_lo) times the pair (ph + pl) times 2^-k, rounded once at the end.
__device__ __forceinline__ float scale_pair(float s2, float s2_lo, float ph, float pl, int k) {
    const float p = __fmul_rn(s2, ph);
    const float pe = fmaf(s2, ph, -p);
    const float tail = fmaf(s2, pl, fmaf(s2_lo, ph, pe));
    return ldexpf(__fadd_rn(p, tail), -k);
}

// (ah + al)(bh + bl) as an unnormalised pair (exact leading product; the
// pairs here are not normalised, so al bl is kept too).
__device__ __forceinline__ void mul_pair(float ah, float al, float bh, float bl, float& ph, float& pl) {
    ph = __fmul_rn(ah, bh);
    pl = fmaf(ah, bl, fmaf(al, bh, fmaf(al, bl, fmaf(ah, bh, -ph))));
}

// e^x K_nu(x) for x = xh > 0 and nu = nuh + nul (both words, so that the float
// rounding of nu does not bias the entries), in FP32 arithmetic, as a float
// pair (Kh + Kl), with d = d/dx log(e^x K_nu(x)) for the first-order effect of
// x's low word.  The trapezoid rule of ekv_fp64 on the same integrand: each
// term (1/2)(e^(-a + nu t) + e^(-a - nu t)), a = x (cosh t - 1) = 2 x sinh^2(t/2),
// with both exponentials from exp_pair (no overflow of cosh(nu t) alone), the
// terms added in pair arithmetic (TwoSum).  Step h = min(0.35, 0.7/sqrt(x)).
__device__ __forceinline__ void ekv_pair(float nuh, float nul, float x, const ExpTab& T, float& Kh, float& Kl,
                                         float& d) {
    const float h = fminf(0.35f, 0.7f * rsqrtf(x));
    float sh = 0.5f, sl = 0.0f, s1 = 0.0f;   // t = 0: weight 1/2, cosh t - 1 = 0
    for (int k = 1; k < 128; ++k) {
        const float t = (float)k * h;
        const float u = expm1f(0.5f * t), mm = -expm1f(-0.5f * t);
        const float s = u + mm;                 // 2 sinh(t/2)
        const float c1 = 0.5f * s * s;          // cosh t - 1
        const float a = x * c1;
        const float yh = __fmul_rn(nuh, t), yl = fmaf(nuh, t, -yh) + nul * t;
        float e0, pe0, ph0 = two_sum(-a, yh, e0);
        const float pl0 = e0 + yl;
        float e1h, e1l, e2h, e2l;
        int k1, k2;
        exp_pair(ph0, pl0, T, e1h, e1l, k1);
        ph0 = two_sum(-a, -yh, pe0);
        exp_pair(ph0, pe0 - yl, T, e2h, e2l, k2);
        const float w1 = pow2i(k1 - 1), w2 = pow2i(k2 - 1);
        e1h *= w1;
        e1l *= w1;
        e2h *= w2;
        e2l *= w2;
        float te;
        const float th = two_sum(e1h, e2h, te);
        const float tl = te + e1l + e2l;
        float se;
        const float ns = two_sum(sh, th, se);
        sl += se + tl;
        sh = ns;
        s1 = fmaf(c1, th, s1);
        if (a > 20.0f && x * sinhf(t) > nuh) break;
    }
    Kh = __fmul_rn(sh, h);
    Kl = fmaf(sh, h, -Kh) + sl * h;
    d = -s1 / sh;   // d/dx log(e^x K_nu(x)) = -(int (cosh t - 1) f) / (int f)
}

// FP32 entry from x = xh + xl (xl the low part of r/beta).  The closed forms
// (nu = 1/2, 3/2, 5/2) carry e^-x and the polynomial factor as float pairs and
// round once: the entry is within ~0.5 ulp (+2^-28 relative) of the exact value,
// as if computed in FP64 and rounded, with no FP64 operation.
// The general-nu form sigma2 x^nu e^-x / (2^(nu-1) Gamma(nu)) * [e^x K_nu(x)]
// takes its first factor as exp(A) (1 + dA): A = nu log xh - xh - log_c in
// float, dA the exact rounding errors of that sum (two-product, TwoSum) plus
// the first-order effect of xl and of log_c's low part, so the exponent's
// rounding (~x u) does not enter the entry's error.  sigma2 enters as
// s2 + s2_lo (its float rounding would otherwise scale every entry alike).
__device__ __forceinline__ float matern_fp32(float xh, float xl, const MaternP& m, float s2, float s2_lo,
                                             float nu, float nu_lo, float log_c, float log_c_lo, const ExpTab& T) {
    switch (m.kind) {
        case 1:
        case 2:
        case 3: {
            if (xh > 103.0f) return 0.0f;
            float eh, el;
            int k;
            exp_neg_pair(xh, xl, T, eh, el, k);
            if (m.kind == 1) return scale_pair(s2, s2_lo, eh, el, -k);
            // P = 1 + x (+ x^2/3) as a pair
            float e0;
            float ph = two_sum(1.0f, xh, e0);
            float pl = e0 + xl;
            if (m.kind == 3) {
                const float sh = __fmul_rn(xh, xh);
                const float sl = fmaf(xh, xh, -sh) + 2.0f * xh * xl;
                const float th = __fmul_rn(sh, 1.0f / 3.0f);                    // x^2/3 as th + tl
                const float tl = (fmaf(-3.0f, th, sh) + sl) * (1.0f / 3.0f);
                float e1;
                const float uh = two_sum(ph, th, e1);
                pl = pl + tl + e1;
                ph = uh;
            }
            float mh, ml;
            mul_pair(ph, pl, eh, el, mh, ml);
            return scale_pair(s2, s2_lo, mh, ml, -k);
        }
        default: {
            // sigma2 x^nu e^-x / (2^(nu-1) Gamma(nu)) * [e^x K_nu(x)]: the first
            // factor is e^A with A = nu ln x - x - log_c as a pair (log_pair,
            // both words of nu and of log_c), the second from ekv_pair at xh
            // with the first-order correction for xl; one rounding at the end.
            if (xh > 110.0f) return 0.0f;
            float lh, ll;
            log_pair(xh, xl, T, lh, ll);
            const float ph = __fmul_rn(nu, lh);
            const float pe = fmaf(nu, lh, -ph) + fmaf(nu, ll, nu_lo * lh);
            float e1, e2;
            const float a1 = two_sum(ph, -xh, e1);
            const float a2 = two_sum(a1, -log_c, e2);
            const float al = ((pe + e1) + e2) - xl - log_c_lo;
            float eh, el;
            int k;
            exp_pair(a2, al, T, eh, el, k);
            float kh, kl, dk;
            ekv_pair(nu, nu_lo, xh, T, kh, kl, dk);
            kl = fmaf(kh, dk * xl, kl);   // e^x K_nu(x) at x = xh + xl, to first order
            float mh, ml;
            mul_pair(eh, el, kh, kl, mh, ml);
            return scale_pair(s2, s2_lo, mh, ml, -k);
        }
    }
}

}  // namespace geo
