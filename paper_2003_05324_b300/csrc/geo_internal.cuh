// Internal device-side view of one problem's tile store and shared helpers.
//
// Tile (i, j), i >= j, of the p x p tile grid is an nb x nb column-major block
// stored contiguously: in the FP64 store when i - j < band (Algorithm 1's
// diag_thick), otherwise in the FP32 store.  `off[i*p + j]` is its element
// offset inside the store of its precision (-1 for the upper triangle).
// Panel tiles (i > j) also own a slot of planes: NPL = 7 BF16 planes
// (fixed-point slices of their value, scaled per row: 8 bits each, 56 bits in
// all) read by the in-band (FP64-accurate) products, and -- when the store has
// off-band tiles -- NPLH = 4 FP16 planes of an 8/12/12-bit split of the same
// row-scaled value read by the off-band (FP32-accurate) products.  Each plane is
// pp x pp row-major with the column (the contraction index of the updates)
// contiguous and zero padding beyond nb; one scale exponent per row.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/geo.h"

namespace geo {

// status words in the workspace
enum { ST_CODE = 0, ST_INFO = 1, ST_TIMEOUT_WHERE = 2, ST_BAR_COUNT = 4, ST_BAR_GEN = 5, ST_WORDS = 16 };

struct Layout {
    int n, nb, p, band, pp, lp_mode, flags;
    int npl;        // planes per panel-tile slot: NPL, or NPL + NPLH with off-band tiles
    double* dp;
    float* sp;
    const long long* off;
    const int* slot;
    __nv_bfloat16* planes;
    int* rexp;      // per panel-tile row: scale exponent of its fixed-point slices [slot][pp]
    int* status;
    int* tickets;   // [2p] work counters of the persistent update kernels (FP64: k, off-band: p + k)
    double* scal;   // scalar scratch: per-tile log-det and quad partials [2*p], results [2]
    const unsigned char* far;   // [p*p] far-tier map of the tiles (nullptr: no far tier)
    int far_products;           // products of a far update (1 or 3)
};

constexpr int NPL = 7;    // BF16 8-bit slice planes (in-band products)
constexpr int NPLH = 4;   // FP16 planes a0, a1, a2 2^-12, a1 2^-12 of the 8/12/12 split (off-band products)
// planes per slot of a store with band b and p tiles per side
__host__ __device__ inline int planes_per_slot(int band, int p) { return band < p ? NPL + NPLH : NPL; }

__host__ __device__ inline bool is_dp(int i, int j, int band) { return (i - j) < band; }

__device__ __forceinline__ double* dp_tile(const Layout& L, int i, int j) { return L.dp + L.off[i * L.p + j]; }
__device__ __forceinline__ float* sp_tile(const Layout& L, int i, int j) { return L.sp + L.off[i * L.p + j]; }
__device__ __forceinline__ __nv_bfloat16* plane(const Layout& L, int i, int j, int s) {
    return L.planes + ((size_t)L.slot[i * L.p + j] * L.npl + s) * (size_t)L.pp * L.pp;
}
__device__ __forceinline__ bool failed(const Layout& L) {
    return *((volatile int*)L.status + ST_CODE) != 0;
}

__device__ __forceinline__ long long gtimer() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Record a device-side timeout (first writer wins) with a code for where it happened.
__device__ __forceinline__ void set_timeout(const Layout& L, int where) {
    atomicCAS(L.status + ST_CODE, 0, GEO_ERR_TIMEOUT);
    atomicCAS(L.status + ST_TIMEOUT_WHERE, 0, where);
}

// Matern parameters prepared on the host (Eq. 1): kind selects a closed form
// for nu in {1/2, 3/2, 5/2}; log_c = (nu - 1) log 2 + log Gamma(nu).
struct MaternP {
    double sigma2, inv_beta, nu, nugget, log_c;
    int kind;   // 0 general nu, 1: nu = 1/2, 2: nu = 3/2, 3: nu = 5/2
};

MaternP make_matern(const geo_theta& th);

// Eq. 2 from the log-determinant and the quadratic form (one expression for the
// host and the device, so both give the same bits).
constexpr double GEO_LOG_2PI = 1.8378770664093454835606594728112;
__host__ __device__ inline double assemble_loglik(int n, double logdet, double quad) {
#ifdef __CUDA_ARCH__
    // no contraction into FMAs: the same roundings as the host's
    const double a = __dmul_rn(__dmul_rn(-0.5, (double)n), GEO_LOG_2PI);
    return __dsub_rn(__dsub_rn(a, __dmul_rn(0.5, logdet)), __dmul_rn(0.5, quad));
#else
    return -0.5 * (double)n * GEO_LOG_2PI - 0.5 * logdet - 0.5 * quad;
#endif
}

Layout make_layout(const geo_tiles* t);

// Instrumentation (api.cu): a launch counter and optional event timing of
// selected kernels (kinds: 0 FP64 update, 1 off-band update, 2 potrf, 3 trsm).
void count_launch(int n = 1);
bool prof_on();
void prof_begin(int kind, cudaStream_t s);
void prof_end(int kind, cudaStream_t s);

// Launchers (defined in their own .cu files; all asynchronous on `s`).
// far-tier map of the store's tiles (geo_tiles_set_far): far[i*p + j] = 1 for
// off-band tiles (i, j) with i - j >= far_band (if > 0) or whose bounding
// boxes of locations lie far_dist or more apart (if > 0); scratch: 4p doubles
cudaError_t launch_far_map(const Layout& L, unsigned char* far, int far_band, const double* x, const double* y,
                           double far_dist, double* scratch, cudaStream_t s);
cudaError_t launch_matern_tiles(const Layout& L, const double* x, const double* y, const geo_theta& th,
                                const geo_theta* dth, int reset_status, cudaStream_t s);
cudaError_t launch_load_dense(const Layout& L, const double* a, cudaStream_t s);
cudaError_t launch_to_dense(const Layout& L, double* out, cudaStream_t s);
cudaError_t run_potrf_mp(const geo_tiles* t, const Layout& L, cudaStream_t s);
// loglik (optional): also Eq. 2 assembled on the device
cudaError_t run_logdet_trsv(const Layout& L, const double* z, double* logdet, double* quad, double* y,
                            cudaStream_t s, double* loglik = nullptr);
cudaError_t run_logdet_trsv_noalloc(const Layout& L, const double* z, double* logdet, double* quad,
                                    cudaStream_t s);
cudaError_t run_krige(const Layout& L, const double* x, const double* y, const double* z, const MaternP& mp,
                      const double* xn, const double* yn, int m, double* zhat, double* work, cudaStream_t s);

}  // namespace geo
