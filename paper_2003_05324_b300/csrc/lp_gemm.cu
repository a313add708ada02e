// BF16 plane split of panel tiles and the tcgen05 off-band update (see lp_gemm.cuh).
//
// Off-band update kernel (one launch per outer step k, persistent, one CTA per SM):
//   work item = (off-band target (i,j), 128-row block mb, 128-column block nc)
//   warp 0      TMA producer: per K chunk of 32, the four slice planes of A(i,k)
//               rows [mb*128, +128) and of A(j,k) rows [nc*128, +128) -> one stage
//   warp 1      TMEM allocation and a single issuing thread: 10 slice pairs x 2
//               UMMA (M=128, N=128, K=16, BF16 in, FP32 accumulate) per stage
//   warps 2..5  epilogue: tcgen05.ld of both accumulators, C -= scaled sum in place
// Three smem stages (64 KB each, two loads in flight while one computes) and two
// sets of TMEM accumulators (all 512 columns) let the epilogue of one item
// overlap the main loop of the next.  Every mbarrier wait is
// bounded by a %globaltimer deadline; on expiry the CTA records GEO_ERR_TIMEOUT,
// drains its outstanding copies and MMAs (also bounded), frees TMEM and exits.
#include <cuda.h>
#include <string.h>

#include <algorithm>

#include "lp_gemm.cuh"
#include "tc_common.cuh"

namespace geo {

// ------------------------------------------------------------ split ---
// One CTA per 32 rows of a panel tile (i,k), all columns.  Phase 1: the row
// maxima give each row a power-of-two scale 2^E (|v| 2^-E < 1/2).  Phase 2:
// each value is cut into NPL rounded 8-bit slices (slice_value), exactly, from
// its stored precision: the FP32 value of an off-band tile, the FP64 value of
// an in-band one.  Writes go through a 32 x 32 shared transpose so both sides
// coalesce.
__global__ void __launch_bounds__(256) split_panel_kernel(Layout L, int k) {
    if (failed(L)) return;
    const int i = k + 1 + blockIdx.y;
    const int nb = L.nb, pp = L.pp;
    const int r0 = blockIdx.x * 32;
    __shared__ double t[32][33];
    __shared__ float pmax[8][32];
    __shared__ int es[32];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const bool dp = is_dp(i, k, L.band);
    const double* Ad = dp ? dp_tile(L, i, k) : nullptr;
    const float* As = dp ? nullptr : sp_tile(L, i, k);
    auto val = [&](int r, int c) -> double {
        if (r >= nb || c >= nb) return 0.0;
        return dp ? Ad[(size_t)c * nb + r] : (double)As[(size_t)c * nb + r];
    };
    float mx = 0.0f;
    for (int c = ty; c < nb; c += 8) mx = fmaxf(mx, fabsf((float)val(r0 + tx, c)));
    pmax[ty][tx] = mx;
    __syncthreads();
    if (ty == 0) {
        float m = pmax[0][tx];
#pragma unroll
        for (int w = 1; w < 8; ++w) m = fmaxf(m, pmax[w][tx]);
        const int e = row_exponent(m);
        es[tx] = e;
        L.rexp[(size_t)L.slot[i * L.p + k] * pp + r0 + tx] = e;
    }
    __syncthreads();
    __nv_bfloat16* P0 = plane(L, i, k, 0);
    const size_t pstride = (size_t)pp * pp;
    for (int cb = 0; cb < pp; cb += 32) {
        for (int q = ty; q < 32; q += 8) t[tx][q] = val(r0 + tx, cb + q);
        __syncthreads();
        for (int q = ty; q < 32; q += 8) {
            const int r = r0 + q, c = cb + tx;
            __nv_bfloat16 sl[NPL];
            slice_value<double>(t[q][tx], es[q], sl);
            const size_t e = (size_t)r * pp + c;
#pragma unroll
            for (int s = 0; s < NPL; ++s) P0[s * pstride + e] = sl[s];
        }
        __syncthreads();
    }
}

cudaError_t launch_split_panel(const Layout& L, int k, cudaStream_t s) {
    const int m = L.p - k - 1;
    dim3 grid(L.pp / 32, m);
    split_panel_kernel<<<grid, 256, 0, s>>>(L, k);
    count_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------- tcgen05 GEMM ---
__device__ __forceinline__ void decode_lp_target(int t, int k, int p, int band, int& i, int& j) {
    const int m = p - k - 1;
    for (int d = band; d < m; ++d) {
        const int cnt = m - d;
        if (t < cnt) {
            j = k + 1 + t;
            i = j + d;
            return;
        }
        t -= cnt;
    }
    i = j = -1;
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    lp_gemm_tc_kernel(Layout L, const __grid_constant__ CUtensorMap tmap_a,
                      const __grid_constant__ CUtensorMap tmap_b, int k, int nlp) {
    extern __shared__ uint8_t tc_smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = (uint64_t*)(smem + TC_STAGES * TC_STAGE_BYTES);
    // bars: full[S], empty[S], tfull[2], tempty[2]; then tmem base + flags
    volatile uint32_t* tmem_slot = (volatile uint32_t*)(bars + 2 * TC_STAGES + 4);
    volatile int* abort_flag = (volatile int*)(bars + 2 * TC_STAGES + 5);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t bar0 = smem_u32(bars);
    auto FULL = [&](int s) { return bar0 + 8u * s; };
    auto EMPTY = [&](int s) { return bar0 + 8u * (TC_STAGES + s); };
    auto TFULL = [&](int a) { return bar0 + 8u * (2 * TC_STAGES + a); };
    auto TEMPTY = [&](int a) { return bar0 + 8u * (2 * TC_STAGES + 2 + a); };

    if (threadIdx.x == 0) {
        *abort_flag = failed(L) ? 1 : 0;
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(FULL(s), 1);
            mbar_init(EMPTY(s), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(TFULL(a), 1);
            mbar_init(TEMPTY(a), 128);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (*abort_flag) return;   // uniform: decided before any allocation
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32((const void*)tmem_slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    const int nb = L.nb, pp = L.pp, p = L.p;
    const int nmb = (pp + TC_BM - 1) / TC_BM, nnc = (pp + TC_BN - 1) / TC_BN;
    const int per_target = nmb * nnc;
    const int total = nlp * per_target;
    const int nk = pp / TC_BK;
    const long long t_start = gtimer();

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int w = blockIdx.x; w < total && ok; w += gridDim.x) {
                int i, j;
                decode_lp_target(w / per_target, k, p, L.band, i, j);
                const int rem = w % per_target, mb = rem / nnc, nc = rem % nnc;
                const int sa = L.slot[i * p + k] * L.npl, sb = L.slot[j * p + k] * L.npl;
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int st = it % TC_STAGES;
                    const uint32_t ph = (it / TC_STAGES) & 1;
                    if (*abort_flag || !mbar_wait(EMPTY(st), ph ^ 1, gtimer() + TC_WAIT_NS)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(FULL(st), TC_STAGE_BYTES);
                    uint8_t* sbase = smem + st * TC_STAGE_BYTES;
#pragma unroll
                    for (int s = 0; s < TC_NS; ++s)
                        tma_load_3d(smem_u32(sbase + s * TC_A_BYTES), &tmap_a, kc * TC_BK, mb * TC_BM, sa + s,
                                    FULL(st));
#pragma unroll
                    for (int s = 0; s < TC_NS; ++s)
                        tma_load_3d(smem_u32(sbase + TC_NS * TC_A_BYTES + s * TC_B_BYTES), &tmap_b, kc * TC_BK,
                                    nc * TC_BN, sb + s, FULL(st));
                }
            }
            if (!ok) {
                *abort_flag = 1;
                set_timeout(L, 1);
            }
            // drain: the copies of the last stages issued must land before exit
            for (int q = max(0, it - TC_STAGES); q < it; ++q)
                mbar_wait(FULL(q % TC_STAGES), (q / TC_STAGES) & 1, gtimer() + TC_WAIT_NS);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0, tc = 0;
            bool ok = true;
            for (int w = blockIdx.x; w < total && ok; w += gridDim.x, ++tc) {
                const int acc = tc & 1;
                const uint32_t aph = (tc >> 1) & 1;
                if (*abort_flag || !mbar_wait(TEMPTY(acc), aph ^ 1, gtimer() + TC_WAIT_NS)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dst0 = tmem_base + acc * (2 * TC_BN), dst1 = dst0 + TC_BN;
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int st = it % TC_STAGES;
                    const uint32_t ph = (it / TC_STAGES) & 1;
                    if (*abort_flag || !mbar_wait(FULL(st), ph, gtimer() + TC_WAIT_NS)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sbase = smem_u32(smem + st * TC_STAGE_BYTES);
#pragma unroll
                    for (int q = 0; q < TC_NPAIRS; ++q) {
                        const uint32_t a_addr = sbase + c_pair_a[q] * TC_A_BYTES;
                        const uint32_t b_addr = sbase + TC_NS * TC_A_BYTES + c_pair_b[q] * TC_B_BYTES;
#pragma unroll
                        for (int kk = 0; kk < TC_BK / 16; ++kk) {
                            if (q == 0)
                                umma_bf16(dst0, sw64_desc(a_addr + kk * 32), sw64_desc(b_addr + kk * 32),
                                          (kc | kk) != 0);
                            else
                                umma_bf16(dst1, sw64_desc(a_addr + kk * 32), sw64_desc(b_addr + kk * 32),
                                          (kc | (q - 1) | kk) != 0);
                        }
                    }
                    umma_commit(EMPTY(st));   // stage reusable once these MMAs complete
                }
                if (!ok) break;
                umma_commit(TFULL(acc));     // accumulator ready for the epilogue
            }
            if (!ok) {
                *abort_flag = 1;
                set_timeout(L, 2);
            }
            // drain: all issued MMAs retire before TMEM is released
            if (it > 0) {
                const int q = it - 1;
                mbar_wait(EMPTY(q % TC_STAGES), (q / TC_STAGES) & 1, gtimer() + TC_WAIT_NS);
            }
        }
    } else {
        // epilogue warps 2..5 -> TMEM lane quadrant warp % 4.  Each thread owns one
        // row of the 128 x 128 block; its 128 C values are loaded into registers
        // before waiting for the accumulator, so the loads overlap the main loop.
        const int quad = warp & 3;
        const int row_in = quad * 32 + lane;
        int tc = 0;
        for (int w = blockIdx.x; w < total; w += gridDim.x, ++tc) {
            const int acc = tc & 1;
            const uint32_t aph = (tc >> 1) & 1;
            int i, j;
            decode_lp_target(w / per_target, k, p, L.band, i, j);
            const int rem = w % per_target, mb = rem / nnc, nc = rem % nnc;
            float* C = sp_tile(L, i, j);
            const int r = mb * TC_BM + row_in;
            const bool rv = r < nb;
            // columns [c_begin, c_begin + ncol) of this block exist in the tile
            const int c_begin = nc * TC_BN;
            const int ncol = rv ? max(0, min(TC_BN, nb - c_begin)) : 0;
            float* Crow = C + (size_t)c_begin * nb + (rv ? r : 0);
            constexpr int BATCH = 32;   // columns per register batch
            float cpre[BATCH];
#pragma unroll
            for (int e = 0; e < BATCH; ++e) cpre[e] = (e < ncol) ? Crow[(size_t)e * nb] : 0.0f;
            if (*abort_flag || !mbar_wait(TFULL(acc), aph, gtimer() + TC_WAIT_NS)) {
                if (!*abort_flag) {
                    *abort_flag = 1;
                    set_timeout(L, 3);
                }
                break;
            }
            tc_fence_after();
            const uint32_t taddr = tmem_base + ((uint32_t)(quad * 32) << 16) + acc * (2 * TC_BN);
            // C -= 2^(E_r + E_c - 16) (acc0 + acc12): one FP32 rounding of the sum, an
            // exact power-of-two scaling, one rounding of the update
            const int* eb = L.rexp + (size_t)L.slot[j * p + k] * pp;
            const int er = (r < pp) ? L.rexp[(size_t)L.slot[i * p + k] * pp + r] : 0;
#pragma unroll 1
            for (int h = 0; h < TC_BN / BATCH; ++h) {
                if (h > 0) {
#pragma unroll
                    for (int e = 0; e < BATCH; ++e)
                        cpre[e] = (h * BATCH + e < ncol) ? Crow[(size_t)(h * BATCH + e) * nb] : 0.0f;
                }
#pragma unroll
                for (int cc = 0; cc < BATCH; cc += 16) {
                    float v0[16], v1[16];
                    tmem_ld16(taddr + h * BATCH + cc, v0);
                    tmem_ld16(taddr + TC_BN + h * BATCH + cc, v1);
                    // the 16 column exponents: uniform across the warp (broadcast loads);
                    // rows >= pp of the B tile do not exist, their exponent reads as 0
                    int ec[16];
                    const int cl0 = c_begin + h * BATCH + cc;
                    if (cl0 + 16 <= pp) {
                        const int4* e4 = reinterpret_cast<const int4*>(eb + cl0);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int4 w4 = __ldg(e4 + q);
                            ec[4 * q] = w4.x;
                            ec[4 * q + 1] = w4.y;
                            ec[4 * q + 2] = w4.z;
                            ec[4 * q + 3] = w4.w;
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < 16; ++e) ec[e] = 0;
                    }
#pragma unroll
                    for (int e = 0; e < 16; ++e) cpre[cc + e] -= (v0[e] + v1[e]) * pow2f(er + ec[e] - 16);
                }
#pragma unroll
                for (int e = 0; e < BATCH; ++e)
                    if (h * BATCH + e < ncol) Crow[(size_t)(h * BATCH + e) * nb] = cpre[e];
            }
            tc_fence_before();
            mbar_arrive(TEMPTY(acc));
        }
    }
    (void)t_start;
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------- host side ---
typedef CUresult (*PFN_encodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PFN_encodeTiled get_encode() {
    static PFN_encodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_encodeTiled)p;
    }
    return fn;
}

// 3D map over all planes: (K = pp, rows = pp, plane index = npl * n_slots); the
// box is 32 columns (64 bytes, the swizzle width) by `rows` rows.
static int make_plane_map(const Layout& L, long long nslots, int rows, CUtensorMap* map) {
    PFN_encodeTiled enc = get_encode();
    if (!enc) return 1;
    cuuint64_t dims[3] = {(cuuint64_t)L.pp, (cuuint64_t)L.pp, (cuuint64_t)(L.npl * nslots)};
    cuuint64_t strides[2] = {(cuuint64_t)L.pp * 2, (cuuint64_t)L.pp * L.pp * 2};
    cuuint32_t box[3] = {TC_BK, (cuuint32_t)rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)L.planes, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : 2;
}

// maps[0]: A operand boxes (128 rows), maps[1]: off-band B boxes (128 rows),
// maps[2]: in-band B boxes (64 rows)
int prepare_lp_gemm(geo_tiles* t, const Layout& L) {
    static_assert(3 * sizeof(CUtensorMap) <= sizeof(((geo_tiles*)0)->tmap), "tensor map storage");
    if (!L.planes || t->lay.n_slots == 0) return 0;
    CUtensorMap maps[3];
    int rc = make_plane_map(L, t->lay.n_slots, TC_BM, &maps[0]);
    if (!rc) rc = make_plane_map(L, t->lay.n_slots, TC_BN, &maps[1]);
    if (!rc) rc = make_plane_map(L, t->lay.n_slots, EX_BN, &maps[2]);
    if (rc) return rc;
    memcpy(t->tmap, maps, sizeof(maps));
    return 0;
}

static int g_num_sms = 0;

cudaError_t launch_lp_gemm_tc(const geo_tiles* t, const Layout& L, int k, int nlp, cudaStream_t s) {
    static bool attr_set = false;
    cudaError_t e;
    if (!attr_set) {
        if ((e = cudaFuncSetAttribute(lp_gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)TC_SMEM)))
            return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        attr_set = true;
    }
    const int per_target = ((L.pp + TC_BM - 1) / TC_BM) * ((L.pp + TC_BN - 1) / TC_BN);
    const long long total = (long long)nlp * per_target;
    const int grid = (int)std::min<long long>(total, g_num_sms > 0 ? g_num_sms : 148);
    CUtensorMap maps[2];
    memcpy(maps, t->tmap, sizeof(maps));
    lp_gemm_tc_kernel<<<grid, TC_THREADS, TC_SMEM, s>>>(L, maps[0], maps[1], k, nlp);
    count_launch();
    return cudaGetLastError();
}

}  // namespace geo
