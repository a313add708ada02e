// A10-A11 and A13: log-determinant, forward solve and quadratic form of Eq. 2,
// and the kriging predictor, from the factored tile store.
//
// Forward solve y = L^-1 Z by tile rows: for i = 0..p-1, solve the diagonal
// tile (FP64, one CTA) and subtract L(l,i) y_i from every later block row
// (one CTA per 128 rows of each tile; FP32 tiles promoted, FP64 accumulation).
// The per-tile partial sums of log L_aa and y_a^2 are reduced in a fixed order,
// so the result is bitwise reproducible.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "geo_internal.cuh"
#include "matern_dev.cuh"
#include "ysolve.cuh"

namespace geo {

constexpr int SV_THREADS = 256;

struct BlockSync {
    __device__ void operator()() const { __syncthreads(); }
};

// Solve L_ii y_i = r_i in place (r_i already holds Z_i minus the earlier block
// rows' contributions); record 2 sum log L_aa and sum y_a^2 of this tile.  One
// CTA of SV_THREADS threads.
__device__ void trsv_diag_tile(const Layout& L, int i, double* __restrict__ yv, double* __restrict__ part) {
    __shared__ YSolveSmem S;
    ysolve_diag_tile(L, i, yv, part, (int)threadIdx.x, SV_THREADS, S, BlockSync());
}

__global__ void __launch_bounds__(SV_THREADS) trsv_diag_kernel(Layout L, int i, double* __restrict__ yv,
                                                               double* __restrict__ part) {
    if (failed(L)) return;
    trsv_diag_tile(L, i, yv, part);
}

constexpr int GV_ROWS = 128;

// y_l -= L(l,i) y_i for every block row l > i.
__global__ void __launch_bounds__(GV_ROWS) trsv_update_kernel(Layout L, int i, double* __restrict__ yv) {
    if (failed(L)) return;
    const int nb = L.nb;
    const int l = i + 1 + blockIdx.y;
    const int r = blockIdx.x * GV_ROWS + threadIdx.x;
    extern __shared__ double yi[];
    for (int c = threadIdx.x; c < nb; c += GV_ROWS) yi[c] = yv[(size_t)i * nb + c];
    __syncthreads();
    if (r >= nb) return;
    yv[(size_t)l * nb + r] -= yrow_update(L, l, i, r, yi);
}

__global__ void trsv_load_kernel(Layout L, const double* __restrict__ z, double* __restrict__ yv) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < L.p * L.nb) yv[g] = g < L.n ? z[g] : 0.0;
}

// The per-tile partials exist only when every diagonal solve ran: after a
// failed factorization (the solves return early) the outputs are NaN, never
// partials left over from an earlier solve in the same scratch.
__global__ void trsv_finish_kernel(Layout L, const double* __restrict__ part, double* logdet, double* quad,
                                   double* loglik) {
    if (threadIdx.x != 0) return;
    if (failed(L)) {
        *logdet = *quad = nan("");
        if (loglik) *loglik = nan("");
        return;
    }
    ysolve_finish(L, part, logdet, quad, loglik);
}

static cudaError_t forward_solve(const Layout& L, double* yv, double* part, cudaStream_t s) {
    const int p = L.p, nb = L.nb;
    for (int i = 0; i < p; ++i) {
        trsv_diag_kernel<<<1, SV_THREADS, 0, s>>>(L, i, yv, part);
        count_launch();
        if (i + 1 < p) {
            trsv_update_kernel<<<dim3((nb + GV_ROWS - 1) / GV_ROWS, p - i - 1), GV_ROWS, nb * sizeof(double), s>>>(
                L, i, yv);
            count_launch();
        }
    }
    return cudaGetLastError();
}

cudaError_t run_logdet_trsv(const Layout& L, const double* z, double* logdet, double* quad, double* y,
                            cudaStream_t s, double* loglik) {
    double* yv = y ? y : L.scal + 2 * L.p + 8;
    double* part = L.scal;
    const int np = L.p * L.nb;
    trsv_load_kernel<<<(np + 255) / 256, 256, 0, s>>>(L, z, yv);
    count_launch();
    cudaError_t e = forward_solve(L, yv, part, s);
    if (e) return e;
    trsv_finish_kernel<<<1, 32, 0, s>>>(L, part, logdet, quad, loglik);
    count_launch();
    return cudaGetLastError();
}

// ------------------------------------------ allocation-free forward solve ---
// Scratch of geo_logdet_trsv_noalloc: y (padded length) followed by the per-tile
// partial sums.  On a store whose factorization succeeded every entry the
// solve reads is written first in the same call (the load kernel fills all of
// y, each tile writes its own partials), so nothing needs clearing between
// calls; on a failed one the diagonal solves write nothing and the finish
// kernel returns NaN instead of reading the partials.  The array is
// process-wide and shared by all calls: calls that overlap on the GPU race on it.
static __device__ __align__(256) double g_noalloc_scratch[GEO_NOALLOC_MAX_N + 2 * GEO_NOALLOC_MAX_P];

// Device address of the array, looked up once per device (with that device
// current); the host-side symbol is only a stand-in and never a device address.
static double* noalloc_scratch_ptr(cudaError_t* err) {
    static double* ptrs[64] = {nullptr};
    static std::mutex mu;
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess || dev < 0 || dev >= 64) {
        if (*err == cudaSuccess) *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!ptrs[dev]) {
        void* p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (*err != cudaSuccess) return nullptr;
        ptrs[dev] = (double*)p;
    }
    return ptrs[dev];
}

cudaError_t run_logdet_trsv_noalloc(const Layout& L, const double* z, double* logdet, double* quad,
                                    cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    double* base = noalloc_scratch_ptr(&e);
    if (!base) return e;
    double* yv = base;
    double* part = base + GEO_NOALLOC_MAX_N;
    const int np = L.p * L.nb;
    trsv_load_kernel<<<(np + 255) / 256, 256, 0, s>>>(L, z, yv);
    count_launch();
    e = forward_solve(L, yv, part, s);
    if (e) return e;
    trsv_finish_kernel<<<1, 32, 0, s>>>(L, part, logdet, quad, nullptr);
    count_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------- kriging ---
// Back solve L' alpha = y, tile row by tile row from the bottom.
__global__ void __launch_bounds__(256) trsv_t_diag_kernel(Layout L, int i, double* __restrict__ w) {
    if (failed(L)) return;
    const int nb = L.nb, tid = threadIdx.x;
    const double* A = dp_tile(L, i, i);
    double* v = w + (size_t)i * nb;
    __shared__ double red[8];
    // alpha_a = (v_a - sum_{b>a} L[b][a] alpha_b) / L[a][a], a from nb-1 down
    for (int a = nb - 1; a >= 0; --a) {
        double acc = 0.0;
        for (int b = a + 1 + tid; b < nb; b += 256) acc = fma(A[(size_t)a * nb + b], v[b], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if ((tid & 31) == 0) red[tid >> 5] = acc;
        __syncthreads();
        if (tid == 0) {
            double sacc = 0.0;
            for (int q = 0; q < 8; ++q) sacc += red[q];
            v[a] = (v[a] - sacc) / A[(size_t)a * nb + a];
        }
        __syncthreads();
    }
}

// w_j -= L(i,j)' alpha_i for every block row j < i; one warp per column.
__global__ void __launch_bounds__(256) trsv_t_update_kernel(Layout L, int i, double* __restrict__ w) {
    if (failed(L)) return;
    const int nb = L.nb;
    const int j = blockIdx.y;
    const int c = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (c >= nb) return;
    const double* al = w + (size_t)i * nb;
    double acc = 0.0;
    if (is_dp(i, j, L.band)) {
        const double* A = dp_tile(L, i, j) + (size_t)c * nb;
        for (int a = lane; a < nb; a += 32) acc = fma(A[a], al[a], acc);
    } else {
        const float* A = sp_tile(L, i, j) + (size_t)c * nb;
        for (int a = lane; a < nb; a += 32) acc = fma((double)A[a], al[a], acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) w[(size_t)j * nb + c] -= acc;
}

// zhat_q = sum_a C(||s_new_q - s_a||) alpha_a, one CTA per new point.  Under
// the DST approximation (Section V-B) the sum runs over the observed points
// whose tile is within `band` tiles of the new point's tile -- the tile of its
// nearest observed point, the lowest index on a tie -- as the truncated
// covariance does for the observed points themselves.
__global__ void __launch_bounds__(256) krige_cross_kernel(Layout L, const double* __restrict__ x,
                                                          const double* __restrict__ y,
                                                          const double* __restrict__ alpha, MaternP mp,
                                                          const double* __restrict__ xn,
                                                          const double* __restrict__ yn, double* __restrict__ zhat) {
    const int q = blockIdx.x, tid = threadIdx.x;
    const double xq = xn[q], yq = yn[q];
    int lo = 0, hi = L.n;
    if (L.flags & GEO_FLAG_DST) {
        double best = INFINITY;
        int bi = 0x7fffffff;
        for (int a = tid; a < L.n; a += 256) {   // squares and sum rounded separately (no contraction)
            const double dx = __dsub_rn(xq, x[a]), dy = __dsub_rn(yq, y[a]);
            const double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
            if (r2 < best) {   // a increases: the first minimum is the lowest index
                best = r2;
                bi = a;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double b2 = __shfl_down_sync(0xffffffffu, best, o);
            const int i2 = __shfl_down_sync(0xffffffffu, bi, o);
            if (b2 < best || (b2 == best && i2 < bi)) {
                best = b2;
                bi = i2;
            }
        }
        __shared__ double sb[8];
        __shared__ int si[8], home;
        if ((tid & 31) == 0) {
            sb[tid >> 5] = best;
            si[tid >> 5] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            double b = sb[0];
            int i = si[0];
            for (int w2 = 1; w2 < 8; ++w2)
                if (sb[w2] < b || (sb[w2] == b && si[w2] < i)) {
                    b = sb[w2];
                    i = si[w2];
                }
            home = i / L.nb;
        }
        __syncthreads();
        const int b = min(L.band, L.p);   // (a band past p keeps every tile)
        lo = max(0, home - b + 1) * L.nb;
        hi = min(L.n, (home + b) * L.nb);
    }
    double acc = 0.0;
    for (int a = lo + tid; a < hi; a += 256) {
        const double dx = xq - x[a], dy = yq - y[a];
        const double r = sqrt(dx * dx + dy * dy);
        const double c = (r == 0.0) ? mp.sigma2 : matern_fp64(r * mp.inv_beta, mp);
        acc = fma(c, alpha[a], acc);
    }
    __shared__ double red[8];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w2 = 0; w2 < 8; ++w2) s += red[w2];
        zhat[q] = s;
    }
}

cudaError_t run_krige(const Layout& L, const double* x, const double* y, const double* z, const MaternP& mp,
                      const double* xn, const double* yn, int m, double* zhat, double* work, cudaStream_t s) {
    const int p = L.p, nb = L.nb, np = p * nb;
    double* w = work;             // y, then alpha, in place
    double* part = work + np;     // per-tile partials (unused here)
    trsv_load_kernel<<<(np + 255) / 256, 256, 0, s>>>(L, z, w);
    count_launch();
    cudaError_t e = forward_solve(L, w, part, s);
    if (e) return e;
    for (int i = p - 1; i >= 0; --i) {
        trsv_t_diag_kernel<<<1, 256, 0, s>>>(L, i, w);
        count_launch();
        if (i > 0) {
            trsv_t_update_kernel<<<dim3((nb + 7) / 8, i), 256, 0, s>>>(L, i, w);
            count_launch();
        }
    }
    if (m > 0) {
        krige_cross_kernel<<<m, 256, 0, s>>>(L, x, y, w, mp, xn, yn, zhat);
        count_launch();
    }
    return cudaGetLastError();
}

}  // namespace geo
