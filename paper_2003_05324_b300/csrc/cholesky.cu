// A3-A9: Algorithm 1, the mixed-precision tile Cholesky factorization, on one GPU.
//
// Per outer step k (Algorithm 1's loop over k):
//   potrf   FP64 Cholesky of the diagonal tile (k,k)                     (dpotrf)
//   trsm    every panel tile (i,k), i > k: X <- X L_kk^-T; FP64 for tiles
//           within the band, FP32 arithmetic against the FP32 copy of L_kk
//           (tmp_0k) for the others                                      (dtrsm / strsm)
//   split   each solved panel tile -> its fixed-point slice planes (row scale
//           exponent, 8-bit slices held in BF16) for the tensor-core updates;
//           this step-by-step path's off-band update reads four of them (the
//           SP copy of in-band panel tiles, Algorithm 1's dconv2s, is the
//           FP32-level value these slices carry)
//   update  trailing tiles (i,j), k < j <= i: FP64 for the diagonal (dsyrk,
//           always FP64) and the band (dgemm), FP32-accurate for the rest
//           (sgemm).  The FP64 and off-band updates run concurrently on two
//           streams: they use different pipes (FP64 vs tensor / FP32).
// Off-band tiles live only in FP32: in Algorithm 1 their FP64 copy is the exact
// promotion of the FP32 result (sconv2d), so FP64 consumers promote on load.
#include <math.h>

#include <algorithm>

#include "geo_internal.cuh"
#include "lp_gemm.cuh"

namespace geo {

// ---------------------------------------------------------------- potrf ---
// FP64 Cholesky of the diagonal tile (k,k), right-looking over 32-column blocks,
// spread over a cooperative grid (one CTA per SM, each with its own FP64 pipe):
//   every CTA factors the 32 x 32 diagonal block redundantly in shared memory
//   (so all CTAs see a failing pivot at the same point and stop together);
//   each warp solves a 32-row group of the panel below it;  grid barrier;
//   CTAs split the trailing lower triangle into 32 x 32 blocks;  grid barrier.
// Barriers spin on a generation word with a 2 s bound (GEO_ERR_TIMEOUT).
constexpr int PO_THREADS = 256;
constexpr int PO_BS = 32;
constexpr int PO_LD = PO_BS + 1;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier of a cooperative launch; false (in every thread of the CTA)
// once any CTA has recorded an error.
__device__ bool grid_sync(const Layout& L) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned* cnt = (unsigned*)(L.status + ST_BAR_COUNT);
        unsigned* gen = (unsigned*)(L.status + ST_BAR_GEN);
        const unsigned g = ld_acquire_u32(gen);
        __threadfence();
        if (atomicAdd(cnt, 1u) == gridDim.x - 1) {
            atomicExch(cnt, 0u);
            __threadfence();
            st_release_u32(gen, g + 1);
        } else {
            const long long deadline = gtimer() + 2000000000LL;
            unsigned it = 0;
            while (ld_acquire_u32(gen) == g) {
                if ((++it & 1023u) == 0 && gtimer() > deadline) {
                    set_timeout(L, 4);
                    break;
                }
            }
        }
        ok_s = (*((volatile int*)L.status + ST_CODE) == 0);
    }
    __syncthreads();
    return ok_s != 0;
}

__global__ void __launch_bounds__(PO_THREADS) potrf_tile_kernel(Layout L, int k) {
    if (failed(L)) return;
    double* A = dp_tile(L, k, k);
    const int nb = L.nb, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, cta = blockIdx.x;
    __shared__ double D[PO_BS * PO_LD];
    __shared__ double Pr[PO_BS * PO_LD], Ps[PO_BS * PO_LD];
    __shared__ int bad;
    for (int c0 = 0; c0 < nb; c0 += PO_BS) {
        const int w = min(PO_BS, nb - c0);
        if (tid == 0) bad = 0;
        for (int idx = tid; idx < w * w; idx += PO_THREADS) {
            const int r = idx % w, c = idx / w;
            D[r * PO_LD + c] = A[(size_t)(c0 + c) * nb + c0 + r];
        }
        __syncthreads();
        if (warp == 0) {
            for (int c = 0; c < w; ++c) {
                double d = D[c * PO_LD + c];
                if (!(d > 0.0)) {   // also catches NaN
                    if (lane == 0) {
                        bad = 1;
                        if (cta == 0 && atomicCAS(L.status + ST_CODE, 0, GEO_ERR_NOT_SPD) == 0)
                            L.status[ST_INFO] = k * nb + c0 + c + 1;
                    }
                    break;
                }
                d = sqrt(d);
                __syncwarp();
                if (lane == c) D[c * PO_LD + c] = d;
                if (lane > c && lane < w) D[lane * PO_LD + c] /= d;
                __syncwarp();
                if (lane > c && lane < w) {
                    const double lc = D[lane * PO_LD + c];
                    for (int j = c + 1; j <= lane; ++j) D[lane * PO_LD + j] -= lc * D[j * PO_LD + c];
                }
                __syncwarp();
            }
        }
        __syncthreads();
        if (bad) return;
        if (cta == 0)
            for (int idx = tid; idx < w * w; idx += PO_THREADS) {
                const int r = idx % w, c = idx / w;
                if (r >= c) A[(size_t)(c0 + c) * nb + c0 + r] = D[r * PO_LD + c];
            }
        // panel: rows below the block, X <- X D^-T, one warp per 32-row group
        const int m = nb - c0 - w;
        const int ngroups = (m + 31) / 32;
        for (int g = cta * (PO_THREADS / 32) + warp; g < ngroups; g += G * (PO_THREADS / 32)) {
            const int r = c0 + w + g * 32 + lane;
            if (r < nb) {
                double v[PO_BS];
#pragma unroll
                for (int c = 0; c < PO_BS; ++c) v[c] = (c < w) ? A[(size_t)(c0 + c) * nb + r] : 0.0;
#pragma unroll
                for (int c = 0; c < PO_BS; ++c) {
                    if (c < w) {
                        double s = v[c];
#pragma unroll
                        for (int t = 0; t < c; ++t) s -= v[t] * D[c * PO_LD + t];
                        v[c] = s / D[c * PO_LD + c];
                    }
                }
#pragma unroll
                for (int c = 0; c < PO_BS; ++c)
                    if (c < w) A[(size_t)(c0 + c) * nb + r] = v[c];
            }
        }
        if (!grid_sync(L)) return;
        // trailing update of the lower m x m block in 32 x 32 pieces
        const int mb = (m + 31) / 32;
        const int npieces = mb * (mb + 1) / 2;
        for (int q = cta; q < npieces; q += G) {
            int bi = (int)((sqrtf(8.0f * q + 1.0f) - 1.0f) * 0.5f);
            while (bi * (bi + 1) / 2 > q) --bi;
            while ((bi + 1) * (bi + 2) / 2 <= q) ++bi;
            const int bj = q - bi * (bi + 1) / 2;
            const int r0 = c0 + w + 32 * bi, s0 = c0 + w + 32 * bj;
            for (int idx = tid; idx < 32 * PO_BS; idx += PO_THREADS) {
                const int rr = idx % 32, t = idx / 32;
                Pr[rr * PO_LD + t] = (r0 + rr < nb && t < w) ? A[(size_t)(c0 + t) * nb + r0 + rr] : 0.0;
                Ps[rr * PO_LD + t] = (s0 + rr < nb && t < w) ? A[(size_t)(c0 + t) * nb + s0 + rr] : 0.0;
            }
            __syncthreads();
            const int rr = tid % 32, cb = (tid / 32) * 4;
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
            for (int t = 0; t < w; ++t) {
                const double a = Pr[rr * PO_LD + t];
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[e] = fma(a, Ps[(cb + e) * PO_LD + t], acc[e]);
            }
            const int r = r0 + rr;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int s = s0 + cb + e;
                if (r < nb && s < nb && (bi != bj || rr >= cb + e)) A[(size_t)s * nb + r] -= acc[e];
            }
            __syncthreads();
        }
        if (!grid_sync(L)) return;
    }
}

// ----------------------------------------------------------------- trsm ---
constexpr int TR_THREADS = 128;
constexpr int TR_CB = 16;

template <typename T>
__device__ __forceinline__ void trsm_rows(const double* __restrict__ Lkk, T* __restrict__ X, int nb, int r0,
                                          T* Ls) {
    const int tid = threadIdx.x, r = r0 + tid;
    const bool valid = r < nb;
    for (int cb = 0; cb < nb; cb += TR_CB) {
        const int w = min(TR_CB, nb - cb);
        for (int idx = tid; idx < (cb + w) * TR_CB; idx += blockDim.x) {
            const int t = idx / TR_CB, jj = idx % TR_CB;
            // Ls[t][jj] = L[cb+jj][t]; only entries with t <= cb+jj are ever read
            Ls[idx] = (jj < w && t <= cb + jj) ? (T)Lkk[(size_t)t * nb + cb + jj] : (T)0;
        }
        __syncthreads();
        if (valid) {
            T acc[TR_CB];
#pragma unroll
            for (int jj = 0; jj < TR_CB; ++jj) acc[jj] = (jj < w) ? X[(size_t)(cb + jj) * nb + r] : (T)0;
            // sum_t x_t L[cb+jj][t] in partial sums of TR_CB terms (cb is a multiple
            // of TR_CB): the rounding error grows with cb/16 + 16, not with cb
            for (int t0 = 0; t0 < cb; t0 += TR_CB) {
                T part[TR_CB];
#pragma unroll
                for (int jj = 0; jj < TR_CB; ++jj) part[jj] = (T)0;
#pragma unroll 4
                for (int t = t0; t < t0 + TR_CB; ++t) {
                    const T xt = X[(size_t)t * nb + r];
                    const T* lrow = Ls + t * TR_CB;
#pragma unroll
                    for (int jj = 0; jj < TR_CB; ++jj) part[jj] = fma(xt, lrow[jj], part[jj]);
                }
#pragma unroll
                for (int jj = 0; jj < TR_CB; ++jj) acc[jj] -= part[jj];
            }
#pragma unroll
            for (int jj = 0; jj < TR_CB; ++jj) {
                if (jj < w) {
                    const T* lrow = Ls + (cb + jj) * TR_CB;
                    const T xv = acc[jj] / lrow[jj];
                    acc[jj] = xv;
#pragma unroll
                    for (int j2 = jj + 1; j2 < TR_CB; ++j2) acc[j2] -= xv * lrow[j2];
                }
            }
#pragma unroll
            for (int jj = 0; jj < TR_CB; ++jj)
                if (jj < w) X[(size_t)(cb + jj) * nb + r] = acc[jj];
        }
        __syncthreads();
    }
}

// FP64 triangular solves of the in-band panel tiles (i - k < band): one warp
// per 32 rows, so a tile spreads over nb/32 SMs (FP64 throughput is per SM).
__global__ void __launch_bounds__(32) trsm_panel_dp_kernel(Layout L, int k) {
    if (failed(L)) return;
    const int i = k + 1 + blockIdx.y;
    extern __shared__ double trsm_sm[];
    trsm_rows<double>(dp_tile(L, k, k), dp_tile(L, i, k), L.nb, blockIdx.x * 32, trsm_sm);
}

// FP32 triangular solves of the off-band panel tiles against the FP32 copy of
// L_kk (Algorithm 1's tmp_0k, rounded on load), 128 rows per CTA.
__global__ void __launch_bounds__(TR_THREADS) trsm_panel_sp_kernel(Layout L, int k) {
    if (failed(L)) return;
    const int i = k + L.band + blockIdx.y;
    extern __shared__ double trsm_sm[];
    trsm_rows<float>(dp_tile(L, k, k), sp_tile(L, i, k), L.nb, blockIdx.x * TR_THREADS, (float*)trsm_sm);
}

// ------------------------------------------------ FP64 update (DMMA f64) ---
// C(i,j) -= A(i,k) A(j,k)' for the diagonal (dsyrk) and in-band (dgemm) targets
// of step k.  One CTA per 64 x 64 sub-block; 4 warps of 32 x 32, each a 4 x 4
// grid of m8n8k4 FP64 MMAs.  Sources in FP32 storage are promoted exactly.
constexpr int U64_THREADS = 128;
constexpr int U64_BM = 64;
constexpr int U64_BK = 8;                 // K chunk per smem buffer (two buffers)
constexpr int U64_LD = U64_BK + 4;
constexpr int U64_PER_T = U64_BM * U64_BK / U64_THREADS;   // staged values per thread and operand

__device__ __forceinline__ void dmma_884(double& c0, double& c1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c0), "+d"(c1)
                 : "d"(a), "d"(b));
}

// target t of step k among tiles with i - j = d in [d_lo, d_hi): diagonal-major order
__device__ __forceinline__ bool decode_target(int t, int k, int p, int d_lo, int d_hi, int& i, int& j) {
    const int m = p - k - 1;
    for (int d = d_lo; d < min(d_hi, m); ++d) {
        const int cnt = m - d;
        if (t < cnt) {
            j = k + 1 + t;
            i = j + d;
            return true;
        }
        t -= cnt;
    }
    return false;
}

// Register-staged loads of one K chunk (rows row0..row0+63, columns kc..kc+BK-1)
// of a column-major tile, promoted to FP64; then stored to shared memory.
template <typename T>
__device__ __forceinline__ void load_chunk(double (&v)[U64_PER_T], const T* __restrict__ src, int nb, int row0,
                                           int kc) {
#pragma unroll
    for (int q = 0; q < U64_PER_T; ++q) {
        const int idx = threadIdx.x + q * U64_THREADS;
        const int rr = idx % U64_BM, tt = idx / U64_BM;
        const int r = row0 + rr, t = kc + tt;
        v[q] = (r < nb && t < nb) ? (double)src[(size_t)t * nb + r] : 0.0;
    }
}
__device__ __forceinline__ void store_chunk(double* S, const double (&v)[U64_PER_T]) {
#pragma unroll
    for (int q = 0; q < U64_PER_T; ++q) {
        const int idx = threadIdx.x + q * U64_THREADS;
        S[(idx % U64_BM) * U64_LD + idx / U64_BM] = v[q];
    }
}

// Persistent: CTAs take (target, sub-block) items from a per-step ticket counter,
// so late-starting CTAs (sharing SMs with the tensor-core update) just take fewer.
__global__ void __launch_bounds__(U64_THREADS) update_fp64_kernel(Layout L, int k, int n_items) {
    const int nb = L.nb, nsb = (nb + U64_BM - 1) / U64_BM;
    __shared__ double As[2][U64_BM * U64_LD], Bs[2][U64_BM * U64_LD];
    __shared__ int item_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tq = lane & 3;
    const int wr = (warp >> 1) * 32, wc = (warp & 1) * 32;
    for (;;) {
        if (threadIdx.x == 0) item_s = failed(L) ? n_items : atomicAdd(L.tickets + k, 1);
        __syncthreads();
        const int item = item_s;
        __syncthreads();
        if (item >= n_items) return;
        int i, j;
        decode_target(item / (nsb * nsb), k, L.p, 0, L.band, i, j);
        const int sb = item % (nsb * nsb);
        const int sbr = sb / nsb, sbc = sb % nsb;
        const bool syrk = (i == j);
        if (syrk && sbr < sbc) continue;
        const int R0 = sbr * U64_BM, C0 = sbc * U64_BM;
        double acc[4][4][2];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b][0] = acc[a][b][1] = 0.0;
        const bool a_dp = is_dp(i, k, L.band), b_dp = is_dp(j, k, L.band);
        const double* Ad = a_dp ? dp_tile(L, i, k) : nullptr;
        const float* As32 = a_dp ? nullptr : sp_tile(L, i, k);
        const double* Bd = b_dp ? dp_tile(L, j, k) : nullptr;
        const float* Bs32 = b_dp ? nullptr : sp_tile(L, j, k);
        double va[U64_PER_T], vb[U64_PER_T];
        auto fetch = [&](int kc) {
            if (a_dp) load_chunk(va, Ad, nb, R0, kc);
            else load_chunk(va, As32, nb, R0, kc);
            if (b_dp) load_chunk(vb, Bd, nb, C0, kc);
            else load_chunk(vb, Bs32, nb, C0, kc);
        };
        fetch(0);
        store_chunk(As[0], va);
        store_chunk(Bs[0], vb);
        __syncthreads();
        int buf = 0;
        for (int kc = 0; kc < nb; kc += U64_BK, buf ^= 1) {
            const bool more = kc + U64_BK < nb;
            if (more) fetch(kc + U64_BK);   // global loads in flight during the MMAs below
#pragma unroll
            for (int kk = 0; kk < U64_BK; kk += 4) {
                double af[4], bf[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) af[a] = As[buf][(wr + a * 8 + g) * U64_LD + kk + tq];
#pragma unroll
                for (int b = 0; b < 4; ++b) bf[b] = Bs[buf][(wc + b * 8 + g) * U64_LD + kk + tq];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) dmma_884(acc[a][b][0], acc[a][b][1], af[a], bf[b]);
            }
            if (more) {
                store_chunk(As[buf ^ 1], va);
                store_chunk(Bs[buf ^ 1], vb);
            }
            __syncthreads();
        }
        double* C = dp_tile(L, i, j);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int r = R0 + wr + a * 8 + g, c = C0 + wc + b * 8 + 2 * tq + e;
                    if (r < nb && c < nb && (!syrk || r >= c)) C[(size_t)c * nb + r] -= acc[a][b][e];
                }
    }
}

// ------------------------------------------- off-band update, FP32 SIMT ---
// C(i,j) -= A(i,k) A(j,k)' in FP32 for off-band targets (sgemm); the B source
// may be an in-band FP64 panel tile, rounded to FP32 on load (dconv2s).
constexpr int U32_THREADS = 256;
constexpr int U32_BM = 64;
constexpr int U32_BK = 32;
constexpr int U32_LD = U32_BM + 4;

template <typename T>
__device__ __forceinline__ void stage_kmajor32(float* S, const T* __restrict__ src, int nb, int row0, int kc) {
    for (int idx = threadIdx.x; idx < U32_BM * U32_BK; idx += U32_THREADS) {
        const int rr = idx % U32_BM, tt = idx / U32_BM;
        const int r = row0 + rr, t = kc + tt;
        S[tt * U32_LD + rr] = (r < nb && t < nb) ? (float)src[(size_t)t * nb + r] : 0.0f;
    }
}

__global__ void __launch_bounds__(U32_THREADS) update_lp_simt_kernel(Layout L, int k) {
    if (failed(L)) return;
    int i, j;
    if (!decode_target(blockIdx.y, k, L.p, L.band, L.p, i, j)) return;
    const int nb = L.nb, nsb = (nb + U32_BM - 1) / U32_BM;
    const int R0 = (blockIdx.x / nsb) * U32_BM, C0 = (blockIdx.x % nsb) * U32_BM;
    __shared__ __align__(16) float As[U32_BK * U32_LD], Bs[U32_BK * U32_LD];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
    const bool b_dp = is_dp(j, k, L.band);
    for (int kc = 0; kc < nb; kc += U32_BK) {
        stage_kmajor32(As, sp_tile(L, i, k), nb, R0, kc);
        if (b_dp) stage_kmajor32(Bs, dp_tile(L, j, k), nb, C0, kc);
        else stage_kmajor32(Bs, sp_tile(L, j, k), nb, C0, kc);
        __syncthreads();
        float part[4][4];   // per-chunk partial sums, then one add per chunk
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) part[a][b] = 0.0f;
#pragma unroll 8
        for (int tt = 0; tt < U32_BK; ++tt) {
            const float4 av = *reinterpret_cast<const float4*>(As + tt * U32_LD + ty * 4);
            const float4 bv = *reinterpret_cast<const float4*>(Bs + tt * U32_LD + tx * 4);
            const float a4[4] = {av.x, av.y, av.z, av.w}, b4[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) part[a][b] = fmaf(a4[a], b4[b], part[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += part[a][b];
        __syncthreads();
    }
    float* C = sp_tile(L, i, j);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int r = R0 + ty * 4 + a, c = C0 + tx * 4 + b;
            if (r < nb && c < nb) C[(size_t)c * nb + r] -= acc[a][b];
        }
}

// ------------------------------------------------------------ driver ---
static int count_targets(int k, int p, int d_lo, int d_hi) {
    const int m = p - k - 1;
    int cnt = 0;
    for (int d = d_lo; d < d_hi && d < m; ++d) cnt += m - d;
    return cnt;
}

cudaError_t run_potrf_mp(const geo_tiles* t, const Layout& L, cudaStream_t s) {
    const int p = L.p, nb = L.nb;
    cudaStream_t aux = (cudaStream_t)t->aux_stream;
    cudaEvent_t ev_fork = (cudaEvent_t)t->ev_fork, ev_join = (cudaEvent_t)t->ev_join;
    const size_t tr_smem = (size_t)nb * TR_CB * sizeof(double);
    cudaError_t e;
    // cooperative grid for the diagonal-tile factorization: as many CTAs as the
    // first trailing update has 32 x 32 pieces, at most one per SM
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, potrf_tile_kernel, PO_THREADS, 0))) return e;
    const int mb0 = (nb - std::min(nb, PO_BS) + 31) / 32;
    const int po_grid = std::max(1, std::min({mb0 * (mb0 + 1) / 2, nsm, nsm * per_sm}));
    if ((e = cudaFuncSetAttribute(trsm_panel_dp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tr_smem)))
        return e;
    if ((e = cudaFuncSetAttribute(trsm_panel_sp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(tr_smem / 2))))
        return e;
    const int nsb64 = (nb + U64_BM - 1) / U64_BM, nsb32 = (nb + U32_BM - 1) / U32_BM;
    for (int k = 0; k < p; ++k) {
        {
            Layout La = L;
            int ka = k;
            void* args[] = {&La, &ka};
            prof_begin(2, s);
            if ((e = cudaLaunchCooperativeKernel((const void*)potrf_tile_kernel, dim3(po_grid), dim3(PO_THREADS), args,
                                                 0, s)))
                return e;
            prof_end(2, s);
            count_launch();
        }
        if (k == p - 1) break;
        const int m = p - k - 1;
        const int n_in = std::min(L.band - 1, m), n_off = m - n_in;
        prof_begin(3, s);
        if (n_in > 0) trsm_panel_dp_kernel<<<dim3((nb + 31) / 32, n_in), 32, tr_smem, s>>>(L, k);
        if (n_off > 0)
            trsm_panel_sp_kernel<<<dim3((nb + TR_THREADS - 1) / TR_THREADS, n_off), TR_THREADS, tr_smem / 2, s>>>(L, k);
        prof_end(3, s);
        count_launch((n_in > 0) + (n_off > 0));
        const int n64 = count_targets(k, p, 0, L.band);
        const int nlp = count_targets(k, p, L.band, p);
        if (nlp > 0) {
            if (L.lp_mode == GEO_LP_SPLIT_BF16) {
                if ((e = launch_split_panel(L, k, s))) return e;
            }
            if ((e = cudaEventRecord(ev_fork, s))) return e;
            if ((e = cudaStreamWaitEvent(aux, ev_fork, 0))) return e;
            prof_begin(1, aux);
            if (L.lp_mode == GEO_LP_SPLIT_BF16) {
                if ((e = launch_lp_gemm_tc(t, L, k, nlp, aux))) return e;
            } else {
                update_lp_simt_kernel<<<dim3(nsb32 * nsb32, nlp), U32_THREADS, 0, aux>>>(L, k);
                count_launch();
            }
            prof_end(1, aux);
            if ((e = cudaEventRecord(ev_join, aux))) return e;
        }
        if (n64 > 0) {
            prof_begin(0, s);
            const int items = nsb64 * nsb64 * n64;
            // one CTA per SM while the tensor-core update shares the SMs (both fit on
            // every SM side by side), two when the FP64 update runs alone
            update_fp64_kernel<<<std::min(items, (nlp > 0 ? 1 : 2) * nsm), U64_THREADS, 0, s>>>(L, k, items);
            prof_end(0, s);
            count_launch();
        }
        if (nlp > 0) {
            if ((e = cudaStreamWaitEvent(s, ev_join, 0))) return e;
        }
        if ((e = cudaGetLastError())) return e;
    }
    return cudaGetLastError();
}

}  // namespace geo
