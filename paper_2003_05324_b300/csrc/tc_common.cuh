// Shared pieces of the tcgen05 off-band update: tile shapes, the fixed-point
// slice pairs, and thin wrappers over the PTX it needs (mbarrier, TMA, UMMA
// descriptors, tcgen05 MMA / commit / load, release-acquire counters).
#pragma once
#include <cuda.h>

#include "geo_internal.cuh"

namespace geo {

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 32;  // K chunk of 32 BF16 = one 64-byte swizzle row
constexpr int TC_NS = 4;                             // slices per operand
constexpr int TC_NPAIRS = 10;                        // slice pairs (a, b) with a + b <= 3
constexpr int TC_STAGES = 3;
constexpr int TC_A_BYTES = TC_BM * TC_BK * 2;        // 8 KB, one A slice chunk
constexpr int TC_B_BYTES = TC_BN * TC_BK * 2;        // 8 KB, one B slice chunk
constexpr int TC_STAGE_BYTES = TC_NS * (TC_A_BYTES + TC_B_BYTES);
constexpr int TC_THREADS = 192;
constexpr int TC_TMEM_COLS = 4 * TC_BN;             // 2 buffers x (level-0, levels 1-3) accumulators
constexpr size_t TC_SMEM = (size_t)TC_STAGES * TC_STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
constexpr long long TC_WAIT_NS = 2000000000LL;      // 2 s per wait

// slice pairs (a, b) kept: (0,0) -> exact level-0 accumulator; the others,
// smallest weight first, -> the second accumulator
__constant__ int c_pair_a[TC_NPAIRS] = {0, 0, 1, 2, 3, 0, 1, 2, 0, 1};
__constant__ int c_pair_b[TC_NPAIRS] = {0, 3, 2, 1, 0, 2, 1, 0, 1, 0};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: false after the deadline
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long deadline) {
    for (uint32_t it = 0;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255u) == 255u && gtimer() > deadline) return false;
    }
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}
// UMMA shared-memory descriptor: K-major operand, 64-byte swizzle (rows of 64
// bytes as written by TMA with SWIZZLE_64B), 8-row groups 512 bytes apart (SBO),
// descriptor version 1.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}
// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, N, M
constexpr uint32_t TC_IDESC =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(r[e]);
}

// 2^e as a float for e >= -126 (exact), 0 below: contributions that small are
// beneath the FP32 resolution of any covariance entry they update.
__device__ __forceinline__ float pow2f(int e) {
    return e < -126 ? 0.0f : __int_as_float((min(e, 127) + 127) << 23);
}

__device__ __forceinline__ int ld_acquire_s32(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(int* p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// order this thread's generic-proxy global writes before later async-proxy (TMA) reads
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

}  // namespace geo
