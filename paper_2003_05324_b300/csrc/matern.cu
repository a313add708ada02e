// A2: Matern covariance tile generation (Eq. 1) with an in-kernel Bessel K_nu.
//
// C(r) = theta1 / (2^(theta3-1) Gamma(theta3)) (r/theta2)^theta3 K_theta3(r/theta2).
//
// K_nu is evaluated from the integral representation
//     K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt,
// scaled by e^x: e^x K_nu(x) = int_0^inf exp(-x (cosh t - 1)) cosh(nu t) dt,
// with the trapezoid rule.  The integrand is analytic and bounded in a strip
// around the real axis, so the rule converges geometrically in 1/h; for large x
// the integrand narrows like 1/sqrt(x), so the step is h = min(h0, c/sqrt(x)).
// Constants (h0, c, cut-off) were fixed against scipy's kve: FP64 error below
// ~1e-13, FP32 variant below ~2e-9 before rounding.  cosh t - 1 is formed as
// (u + m)^2 / 2 with u = e^{t/2} - 1 and m = 1 - e^{-t/2}, each advanced by an
// exact-sign recurrence (no cancellation) and re-anchored every 16 steps.
// Half-integer nu (1/2, 3/2, 5/2) use the elementary closed forms of K_nu.
//
// Each tile is written directly in its own precision (Algorithm 1's initial
// FP64 -> FP32 conversion of off-band tiles is fused away).  Off-band entries
// are computed in FP32 arithmetic from FP64 coordinate differences.
#include <math.h>

#include "dag.cuh"
#include "geo_internal.cuh"
#include "matern_dev.cuh"

namespace geo {

static double host_lgamma(double v) { return lgamma(v); }

// The table of the FP32 exponential (matern_dev.cuh), from the double exp2.
static const ExpTab& exp_table() {
    static const ExpTab tab = [] {
        ExpTab t;
        for (int j = 0; j < 32; ++j) {
            const double e = exp2(-j / 32.0);
            t.hi[j] = (float)e;
            t.lo[j] = (float)(e - (double)t.hi[j]);
        }
        const double c = log(2.0) / 32.0;
        const double c_hi = rint(c * 65536.0) / 65536.0;   // c in [2^-6, 2^-5): 11 significant bits
        t.c_hi = (float)c_hi;
        t.c_lo = (float)(c - c_hi);
        t.inv_c = (float)(1.0 / c);
        for (int j = 0; j < 64; ++j) {
            const double cj = 1.0 + j / 64.0, l = log(cj);
            t.lnc_hi[j] = (float)l;
            t.lnc_lo[j] = (float)(l - (double)t.lnc_hi[j]);
            t.inv_cj[j] = (float)(1.0 / cj);
        }
        const double ln2 = log(2.0), ln2_hi = rint(ln2 * 65536.0) / 65536.0;   // 16 significant bits
        t.ln2_hi = (float)ln2_hi;
        t.ln2_lo = (float)(ln2 - ln2_hi);
        return t;
    }();
    return tab;
}

MaternP make_matern(const geo_theta& th) {
    MaternP m;
    m.sigma2 = th.sigma2;
    m.inv_beta = 1.0 / th.beta;
    m.nu = th.nu;
    m.nugget = th.nugget;
    m.log_c = (th.nu - 1.0) * log(2.0) + host_lgamma(th.nu);
    m.kind = 0;
    if (th.nu == 0.5) m.kind = 1;
    else if (th.nu == 1.5) m.kind = 2;
    else if (th.nu == 2.5) m.kind = 3;
    return m;
}

// One CTA per (lower tile, chunk of 32 columns); threads run down the rows so
// that the column-major stores coalesce.  FP32 (off-band) entries: coordinates
// are scaled by 1/beta in FP64 once per point and split into float hi + lo, so
// the scaled difference (hi_a - hi_b) + (lo_a - lo_b) is within ~1 ulp of the
// FP64 difference without any FP64 operation per entry.
constexpr int GEN_THREADS = 256;
constexpr int GEN_COLS = 32;

// Tile of grid row t.  The in-band (FP64) tiles, whose entries take the slow
// FP64 pipe, are spread evenly over the grid instead of following the
// column-major order, in which the last diagonal tiles crowd the end of the
// launch onto a few SMs: in-band tile q (diagonal by diagonal) sits at grid
// row floor(q T / n_dp) of the T rows, and the off-band tiles fill the other
// rows in column-major order.
__device__ void gen_tile_of(int t, int p, int band, int& i, int& j) {
    const long long b = min(band, p);
    const long long n_dp = b * p - b * (b - 1) / 2, T = (long long)p * (p + 1) / 2;
    const long long q = ((long long)t * n_dp + T - 1) / T;   // in-band tiles at rows < t
    if (q < n_dp && (q * T) / n_dp == t) {                     // row t holds in-band tile q
        long long r = q;
        int d = 0;
        while (r >= p - d) { r -= p - d; ++d; }
        j = (int)r;
        i = j + d;
        return;
    }
    long long o = t - q;                                       // off-band tile o, column-major
    j = 0;
    while (o >= p - j - b) { o -= p - j - b; ++j; }
    i = j + (int)b + (int)o;
}

// The entries of columns c0 .. c0 + 31 of tile (i, j), one CTA.
__device__ __forceinline__ void gen_block(const Layout& L, const double* __restrict__ x,
                                          const double* __restrict__ y, const MaternP& smp, const ExpTab& stab,
                                          int i, int j, int c0) {
    const MaternP mp = smp;
    const int nb = L.nb;
    if (c0 >= nb) return;
    const int cols = min(GEN_COLS, nb - c0);
    __shared__ double cx[GEN_COLS], cy[GEN_COLS];
    __shared__ float cxh[GEN_COLS], cxl[GEN_COLS], cyh[GEN_COLS], cyl[GEN_COLS];
    if (threadIdx.x < cols) {
        const int g = j * nb + c0 + threadIdx.x;
        const double gx = g < L.n ? x[g] : 0.0, gy = g < L.n ? y[g] : 0.0;
        cx[threadIdx.x] = gx;
        cy[threadIdx.x] = gy;
        const double sx = gx * mp.inv_beta, sy = gy * mp.inv_beta;
        const float hx = (float)sx, hy = (float)sy;
        cxh[threadIdx.x] = hx;
        cxl[threadIdx.x] = (float)(sx - (double)hx);
        cyh[threadIdx.x] = hy;
        cyl[threadIdx.x] = (float)(sy - (double)hy);
    }
    __syncthreads();
    const bool dp = is_dp(i, j, L.band);
    const float s2f = (float)mp.sigma2, nuf = (float)mp.nu, lcf = (float)mp.log_c;
    const float nul = (float)(mp.nu - (double)nuf);
    const float lcl = (float)(mp.log_c - (double)lcf), s2l = (float)(mp.sigma2 - (double)s2f);
    for (int a = threadIdx.x; a < nb; a += GEN_THREADS) {
        const int ga = i * nb + a;
        const bool va = ga < L.n;
        const double xa = va ? x[ga] : 0.0, ya = va ? y[ga] : 0.0;
        if (dp) {
            double* T = dp_tile(L, i, j);
            for (int c = 0; c < cols; ++c) {
                const int gb = j * nb + c0 + c;
                const bool vb = gb < L.n;
                double v;
                if (!va || !vb) v = (ga == gb) ? 1.0 : 0.0;          // decoupled padding rows
                else if (ga == gb) v = mp.sigma2 + mp.nugget;
                else if (i == j && a < c0 + c) v = 0.0;   // upper triangle of a diagonal tile: never read
                else {
                    const double dx = xa - cx[c], dy = ya - cy[c];
                    const double r = sqrt(dx * dx + dy * dy);
                    v = (r == 0.0) ? mp.sigma2 : matern_fp64(r * mp.inv_beta, mp);
                }
                T[(size_t)(c0 + c) * nb + a] = v;
            }
        } else if (L.flags & GEO_FLAG_DST) {   // the DST approximation: tiles beyond the band are zero
            float* T = sp_tile(L, i, j);
            for (int c = 0; c < cols; ++c) T[(size_t)(c0 + c) * nb + a] = 0.0f;
        } else if (L.flags & GEO_FLAG_FP64_OFFBAND_GEN) {
            float* T = sp_tile(L, i, j);
            for (int c = 0; c < cols; ++c) {
                const int gb = j * nb + c0 + c;
                float v = 0.0f;
                if (va && gb < L.n) {
                    const double dx = xa - cx[c], dy = ya - cy[c];
                    const double r = sqrt(dx * dx + dy * dy);
                    v = (float)((r == 0.0) ? mp.sigma2 : matern_fp64(r * mp.inv_beta, mp));
                }
                T[(size_t)(c0 + c) * nb + a] = v;
            }
        } else {
            float* T = sp_tile(L, i, j);
            const double sx = xa * mp.inv_beta, sy = ya * mp.inv_beta;
            const float hx = (float)sx, hy = (float)sy;
            const float lx = (float)(sx - (double)hx), ly = (float)(sy - (double)hy);
            for (int c = 0; c < cols; ++c) {
                const int gb = j * nb + c0 + c;
                float v = 0.0f;                                       // off-band: never on the diagonal
                if (va && gb < L.n) {
                    // scaled differences as normalized float pairs: two-sum of the high
                    // parts, add the low parts, then renormalize (fast two-sum) so that
                    // the low part is below half an ulp of the high part even when the
                    // points nearly coincide.  The _rn intrinsics keep the compiler from
                    // contracting these steps.
                    float dxh, dxl, dyh, dyl;
                    {
                        const float s = __fsub_rn(hx, cxh[c]), bv = __fsub_rn(s, hx);
                        const float e = __fadd_rn(__fsub_rn(__fsub_rn(hx, __fsub_rn(s, bv)), __fadd_rn(cxh[c], bv)),
                                                  __fsub_rn(lx, cxl[c]));
                        dxh = __fadd_rn(s, e);
                        dxl = __fsub_rn(e, __fsub_rn(dxh, s));
                    }
                    {
                        const float s = __fsub_rn(hy, cyh[c]), bv = __fsub_rn(s, hy);
                        const float e = __fadd_rn(__fsub_rn(__fsub_rn(hy, __fsub_rn(s, bv)), __fadd_rn(cyh[c], bv)),
                                                  __fsub_rn(ly, cyl[c]));
                        dyh = __fadd_rn(s, e);
                        dyl = __fsub_rn(e, __fsub_rn(dyh, s));
                    }
                    // r^2 = (dxh + dxl)^2 + (dyh + dyl)^2 as hi + lo (two-product via fma)
                    const float px = __fmul_rn(dxh, dxh), qx = fmaf(dxh, dxh, -px);
                    const float py = __fmul_rn(dyh, dyh), qy = fmaf(dyh, dyh, -py);
                    const float r2h = __fadd_rn(px, py);
                    const float bb = __fsub_rn(r2h, px);
                    const float r2l = ((px - (r2h - bb)) + (py - bb)) + qx + qy + 2.0f * (dxh * dxl + dyh * dyl);
                    const float xh = sqrtf(r2h);
                    if (xh == 0.0f) v = s2f;
                    else {
                        const float xl = (fmaf(-xh, xh, r2h) + r2l) / (2.0f * xh);
                        v = matern_fp32(xh, xl, mp, s2f, s2l, nuf, nul, lcf, lcl, stab);
                    }
                }
                T[(size_t)(c0 + c) * nb + a] = v;
            }
        }
    }
}

// Prologue of both generator kernels: theta (from `dth` when given: device
// memory, for batched evaluations and graph replays; else `th`) and the
// exponential tables in shared memory; with reset_status the problem's first
// CTA also clears its status words (the batched path has no separate reset).
__device__ __forceinline__ void gen_prologue(const Layout& L, const geo_theta& th, const geo_theta* dth,
                                             bool reset, const ExpTab& etab, MaternP& smp, ExpTab& stab) {
    if (threadIdx.x == 0) smp = make_matern_dev(dth ? *dth : th);
    static_assert(sizeof(ExpTab) % sizeof(float) == 0, "ExpTab words");
    for (int w = threadIdx.x; w < (int)(sizeof(ExpTab) / sizeof(float)); w += GEN_THREADS)
        reinterpret_cast<float*>(&stab)[w] = reinterpret_cast<const float*>(&etab)[w];
    if (reset && threadIdx.x < ST_WORDS) L.status[threadIdx.x] = 0;
    __syncthreads();
}

__global__ void __launch_bounds__(GEN_THREADS) matern_tiles_kernel(Layout L, const double* __restrict__ x,
                                                                   const double* __restrict__ y, geo_theta th,
                                                                   const geo_theta* __restrict__ dth,
                                                                   int reset_status, ExpTab etab) {
    __shared__ MaternP smp;
    __shared__ ExpTab stab;
    gen_prologue(L, th, dth, reset_status && blockIdx.x == 0 && blockIdx.y == 0, etab, smp, stab);
    int i, j;
    gen_tile_of(blockIdx.y, L.p, L.band, i, j);
    gen_block(L, x, y, smp, stab, i, j, blockIdx.x * GEN_COLS);
}

// Every problem of a batch in one launch: the CTAs of problem b are
// jobs[b].block0 .. jobs[b + 1].block0 - 1 (each problem's grid of the single
// launch, flattened column chunk fastest), so the slow blocks of one problem
// run beside the others' instead of one launch after another; theta of
// problem b from dth[b].
__global__ void __launch_bounds__(GEN_THREADS) matern_batch_kernel(const ProbDev* __restrict__ probs,
                                                                   const GenJob* __restrict__ jobs, int nprob,
                                                                   const geo_theta* __restrict__ dth,
                                                                   ExpTab etab) {
    __shared__ MaternP smp;
    __shared__ ExpTab stab;
    __shared__ int sb;
    const long long blk = blockIdx.x;
    if (threadIdx.x == 0) {   // the job holding this CTA: the last b with block0 <= blk
        int lo = 0, hi = nprob - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (jobs[mid].block0 <= blk) lo = mid;
            else hi = mid - 1;
        }
        sb = lo;
    }
    __syncthreads();
    const int b = sb;
    const Layout& L = probs[b].L;
    const long long local = blk - jobs[b].block0;
    const int ncx = (L.nb + GEN_COLS - 1) / GEN_COLS;
    gen_prologue(L, geo_theta{}, dth + b, local == 0, etab, smp, stab);
    int i, j;
    gen_tile_of((int)(local / ncx), L.p, L.band, i, j);
    gen_block(L, jobs[b].x, jobs[b].y, smp, stab, i, j, (int)(local % ncx) * GEN_COLS);
}

cudaError_t launch_matern_tiles(const Layout& L, const double* x, const double* y, const geo_theta& th,
                                const geo_theta* dth, int reset_status, cudaStream_t s) {
    dim3 grid((L.nb + GEN_COLS - 1) / GEN_COLS, L.p * (L.p + 1) / 2);
    matern_tiles_kernel<<<grid, GEN_THREADS, 0, s>>>(L, x, y, th, dth, reset_status, exp_table());
    count_launch();
    return cudaGetLastError();
}

long long gen_blocks(const Layout& L) {
    return (long long)((L.nb + GEN_COLS - 1) / GEN_COLS) * ((long long)L.p * (L.p + 1) / 2);
}

cudaError_t launch_matern_batch(const ProbDev* d_probs, const GenJob* d_jobs, int nprob, long long total_blocks,
                                const geo_theta* dth, cudaStream_t s) {
    if (total_blocks < 1 || total_blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    matern_batch_kernel<<<(unsigned)total_blocks, GEN_THREADS, 0, s>>>(d_probs, d_jobs, nprob, dth, exp_table());
    count_launch();
    return cudaGetLastError();
}

// ---- dense <-> tile store (test utilities) --------------------------------
__global__ void load_dense_kernel(Layout L, const double* __restrict__ a) {
    const int nb = L.nb, p = L.p, n = L.n;
    int t = blockIdx.y, j = 0;
    while (t >= p - j) { t -= p - j; ++j; }
    const int i = j + t;
    const int c = blockIdx.x;
    if (c >= nb) return;
    const bool dp = is_dp(i, j, L.band);
    for (int r = threadIdx.x; r < nb; r += blockDim.x) {
        const int gr = i * nb + r, gc = j * nb + c;
        double v;
        if (gr < n && gc < n) v = (gr >= gc) ? a[(size_t)gc * n + gr] : a[(size_t)gr * n + gc];
        else v = (gr == gc) ? 1.0 : 0.0;
        const size_t e = (size_t)c * nb + r;
        if (dp) dp_tile(L, i, j)[e] = v;
        else sp_tile(L, i, j)[e] = (float)v;
    }
}

__global__ void to_dense_kernel(Layout L, double* __restrict__ out) {
    const int nb = L.nb, n = L.n;
    const int gc = blockIdx.x;
    for (int gr = threadIdx.x; gr < n; gr += blockDim.x) {
        double v = 0.0;
        if (gr >= gc) {
            const int i = gr / nb, j = gc / nb, r = gr % nb, c = gc % nb;
            const size_t e = (size_t)c * nb + r;
            v = is_dp(i, j, L.band) ? dp_tile(L, i, j)[e] : (double)sp_tile(L, i, j)[e];
        }
        out[(size_t)gc * n + gr] = v;
    }
}

cudaError_t launch_load_dense(const Layout& L, const double* a, cudaStream_t s) {
    dim3 grid(L.nb, L.p * (L.p + 1) / 2);
    load_dense_kernel<<<grid, 128, 0, s>>>(L, a);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_to_dense(const Layout& L, double* out, cudaStream_t s) {
    to_dense_kernel<<<L.n, 256, 0, s>>>(L, out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace geo
