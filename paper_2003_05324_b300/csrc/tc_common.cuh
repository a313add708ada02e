// Shared pieces of the tcgen05 off-band update: tile shapes, the fixed-point
// slice pairs, and thin wrappers over the PTX it needs (mbarrier, TMA, UMMA
// descriptors, tcgen05 MMA / commit / load, release-acquire counters).
#pragma once
#include <cuda.h>
#include <cuda_fp16.h>

#include "geo_internal.cuh"

namespace geo {

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 32;  // K chunk of 32 BF16 = one 64-byte swizzle row
constexpr int TC_NS = 4;                             // slices per operand of an off-band (FP32-accurate) product
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

// ---- FP32-accurate products of the persistent scheduler's off-band items:
// FP16 planes of an 8/12/12-bit split (slice_value_h).  A stage holds the A
// planes h0 = a0, h1 = a1, h2 = a2 2^-12 and the B planes h0..h2 and h3 = b1
// 2^-12.  With t = a0 + e a1 + e^2 a2 (e = 2^-12) for each operand,
//   t_A t_B = a0 b0 + e [a0 b1 + a1 b0 + a0 (b2 e) + (a2 e) b0 + a1 (b1 e)] + O(e^3):
// six products instead of the ten of the 8-bit BF16 split (fewer shared-memory
// operand reads per flop, which bound the 8-bit split's MMA rate).  a0 b0
// (|a0|, |b0| <= 128) sums exactly in FP32 for K <= 1024 (below 2^24); the
// bracket, 2^-12 below it, goes to the second accumulator, smallest weights
// first.  The epilogue forms acc0 + 2^-12 acc1.
// The six (A plane, B plane) pairs, in issue order: (0,0) -> acc0; (1,3),
// (0,2), (2,0), (0,1), (1,0) -> acc1 (the MMA thread spells them out with
// compile-time shared-memory offsets).
constexpr int TC_HA = 3, TC_HB = 4, TC_HPAIRS = 6;
constexpr uint32_t TC_H_STAGE_BYTES = TC_HA * TC_A_BYTES + TC_HB * TC_B_BYTES;
static_assert(TC_H_STAGE_BYTES <= (uint32_t)TC_STAGE_BYTES, "FP16 stage");

// ---- FP64-accurate products for in-band (FP64) targets ("EX" items).
// Seven slices a_0..a_6 per operand (|a_s| <= 128, 56 bits below the row
// scale) and every pair with a + b <= 6 (28 pairs).  A 128 x 64 output block
// is accumulated over K parts of EX_KP = 256: one product of two slices sums
// at most 256 * 2^14 = 2^22 in integer units, so an accumulator holding up to
// four pairs of one level a + b stays at or below 2^24 and the tensor core's
// FP32 accumulation is exact.  Each level L has its own TMEM slot at column
// 64 L (L = 0..6), except the fifth pair of level 4, (4, 0), which goes to slot
// X at column 448: levels 0..4 are exact, levels 5 and 6 (2^-40 below level 0)
// are FP32-accumulated.  Each K part is drained into the FP64 target, so the
// error of the whole update is that of FP64 accumulation.
// The pairs that share an A slice are one MMA whose B operand is the run of
// consecutive B slices (64 rows each, adjacent in shared memory) and whose
// accumulator is the run of consecutive level slots: pass 1 stages A slices
// 0..3 and B slices 0..6 and issues 7 MMAs of N = 64..256 (22 pairs); pass 2
// stages A slices 4..6 and B slices 0..2 and issues 4 MMAs (6 pairs).
constexpr int EX_BN = 64;
constexpr int EX_KP = 256;
constexpr int EX_NSLOT = 8;                          // levels 0..6 and X
constexpr int EX_X = 7;                              // slot of the pair (4, 0)
constexpr int EX_B_BYTES = EX_BN * TC_BK * 2;        // 4 KB
constexpr int EX_P1_MMAS = 7, EX_P2_MMAS = 4;
constexpr uint32_t EX_P1_BYTES = 4 * TC_A_BYTES + 7 * EX_B_BYTES;
constexpr uint32_t EX_P2_BYTES = 3 * TC_A_BYTES + 3 * EX_B_BYTES;
static_assert(EX_P1_BYTES <= (uint32_t)TC_STAGE_BYTES, "EX stage");
static_assert(EX_NSLOT * EX_BN <= 4 * TC_BN, "EX accumulators");
// (A slice, first B slice, number of B slices, first slot); pass 2's A slice
// index counts from slice 4
__constant__ signed char c_ex1[EX_P1_MMAS][4] = {
    {0, 0, 4, 0}, {0, 4, 3, 4},                                      // (0,0..3) (0,4..6)
    {1, 0, 4, 1}, {1, 4, 2, 5},                                      // (1,0..3) (1,4..5)
    {2, 0, 4, 2}, {2, 4, 1, 6},                                      // (2,0..3) (2,4)
    {3, 0, 4, 3}};                                                   // (3,0..3)
__constant__ signed char c_ex2[EX_P2_MMAS][4] = {
    {0, 0, 1, EX_X},                                                 // (4,0): slot X
    {0, 1, 2, 5},                                                    // (4,1..2)
    {1, 0, 2, 5},                                                    // (5,0..1)
    {2, 0, 1, 6}};                                                   // (6,0)

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

// kind::f16 with FP16 A and B (the FP16 off-band planes), D = F32
constexpr uint32_t TC_IDESC_F16 = (1u << 4) | ((uint32_t)(TC_BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);

// kind::f16, D = F32, A = B = BF16, K-major, M = 128 and N = nrows (a multiple of 16, <= 256)
__host__ __device__ constexpr uint32_t ex_idesc(int nrows) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(nrows >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc,
                                          uint32_t idesc = TC_IDESC) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
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

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = __uint_as_float(r[e]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 8 columns of each of the eight in-band slots (64 columns apart) for this
// warp's 32 lanes, loads and the wait in one statement so that no use of the
// registers can be scheduled before the wait
__device__ __forceinline__ void tmem_ld8x8(uint32_t taddr, float (&v)[EX_NSLOT][8]) {
    uint32_t r[EX_NSLOT][8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%64];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%65];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%66];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24,%25,%26,%27,%28,%29,%30,%31}, [%67];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%32,%33,%34,%35,%36,%37,%38,%39}, [%68];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%40,%41,%42,%43,%44,%45,%46,%47}, [%69];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%48,%49,%50,%51,%52,%53,%54,%55}, [%70];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%56,%57,%58,%59,%60,%61,%62,%63}, [%71];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0][0]), "=r"(r[0][1]), "=r"(r[0][2]), "=r"(r[0][3]), "=r"(r[0][4]), "=r"(r[0][5]),
          "=r"(r[0][6]), "=r"(r[0][7]), "=r"(r[1][0]), "=r"(r[1][1]), "=r"(r[1][2]), "=r"(r[1][3]),
          "=r"(r[1][4]), "=r"(r[1][5]), "=r"(r[1][6]), "=r"(r[1][7]), "=r"(r[2][0]), "=r"(r[2][1]),
          "=r"(r[2][2]), "=r"(r[2][3]), "=r"(r[2][4]), "=r"(r[2][5]), "=r"(r[2][6]), "=r"(r[2][7]),
          "=r"(r[3][0]), "=r"(r[3][1]), "=r"(r[3][2]), "=r"(r[3][3]), "=r"(r[3][4]), "=r"(r[3][5]),
          "=r"(r[3][6]), "=r"(r[3][7]), "=r"(r[4][0]), "=r"(r[4][1]), "=r"(r[4][2]), "=r"(r[4][3]),
          "=r"(r[4][4]), "=r"(r[4][5]), "=r"(r[4][6]), "=r"(r[4][7]), "=r"(r[5][0]), "=r"(r[5][1]),
          "=r"(r[5][2]), "=r"(r[5][3]), "=r"(r[5][4]), "=r"(r[5][5]), "=r"(r[5][6]), "=r"(r[5][7]),
          "=r"(r[6][0]), "=r"(r[6][1]), "=r"(r[6][2]), "=r"(r[6][3]), "=r"(r[6][4]), "=r"(r[6][5]),
          "=r"(r[6][6]), "=r"(r[6][7]), "=r"(r[7][0]), "=r"(r[7][1]), "=r"(r[7][2]), "=r"(r[7][3]),
          "=r"(r[7][4]), "=r"(r[7][5]), "=r"(r[7][6]), "=r"(r[7][7])
        : "r"(taddr), "r"(taddr + EX_BN), "r"(taddr + 2 * EX_BN), "r"(taddr + 3 * EX_BN), "r"(taddr + 4 * EX_BN),
          "r"(taddr + 5 * EX_BN), "r"(taddr + 6 * EX_BN), "r"(taddr + 7 * EX_BN)
        : "memory");
#pragma unroll
    for (int a = 0; a < EX_NSLOT; ++a)
#pragma unroll
        for (int e = 0; e < 8; ++e) v[a][e] = __uint_as_float(r[a][e]);
}

// Fixed-point slicing of one value v of a row with scale exponent e
// (|v| 2^-e < 1/2): t = v 2^(8-e), a_s = rint(t), t = 256 (t - a_s), s = 0..NPL-1,
// so |a_s| <= 128 and v = 2^(e-8) sum_s a_s 2^-8s + O(2^(e-65)).  Every step is
// exact in T (float for an FP32 value, double for an FP64 one); slice s is
// stored as the BF16 a_s 2^-8s (exact: |a_s| has at most 8 significant bits).
template <typename T>
__device__ __forceinline__ void slice_value(T v, int e, __nv_bfloat16* out) {
    T t = (sizeof(T) == 8) ? (T)ldexp((double)v, 8 - e) : (T)ldexpf((float)v, 8 - e);
    float w = 1.0f;
#pragma unroll
    for (int s = 0; s < NPL; ++s) {
        const T a = rint(t);
        out[s] = __float2bfloat16_rn((float)a * w);
        t = (t - a) * (T)256;
        w *= (1.0f / 256.0f);
    }
}

// The eight in-band slots of one output as one exact fixed-point sum, in units
// of 2^-40 of the level-0 unit.  Slot L <= 4 (and X, level 4) holds integers
// times 2^-8L of magnitude at most 2^24 (exact), so I_L = s_L 2^8L is an exact
// float-to-int conversion; the FP32-accumulated level-5 and level-6 slots are
// each rounded to the nearest unit (2^-40, below their own accumulation error).
// |level 0| <= 2^22 bounds the total by 2^62 (1 + 2^-7 + ...) < 2^63.  Integer
// arithmetic replaces the FP64 additions: on this part the FP64 pipe runs at
// 1/71 of the FP32 rate, and one conversion of the total to FP64 is left.
__device__ __forceinline__ long long ex_fixed_total(float s0, float s1, float s2, float s3, float s4, float s5,
                                                    float s6, float sx) {
    const long long i0 = __float2int_rn(s0);
    const long long i1 = __float2int_rn(s1 * 256.0f);
    const long long i2 = __float2int_rn(s2 * 65536.0f);
    const long long i3 = __float2int_rn(s3 * 16777216.0f);
    const long long i4 = (long long)__float2int_rn(s4 * 4294967296.0f) + (long long)__float2int_rn(sx * 4294967296.0f);
    const long long i56 =
        (long long)__float2int_rn(s5 * 1099511627776.0f) + (long long)__float2int_rn(s6 * 1099511627776.0f);
    return (i0 << 40) + (i1 << 32) + (i2 << 24) + (i3 << 16) + (i4 << 8) + i56;
}

// The FP16 planes of one value for the off-band products: with t = v 2^(8-e)
// (|t| < 128), a0 = rint(t), a1 = rint(2^12 (t - a0)), a2 = rint(2^12 (2^12 (t -
// a0) - a1)), so |a0| <= 128, |a1|, |a2| <= 2048 and t = a0 + a1 2^-12 + a2
// 2^-24 + O(2^-25) (32 bits below the row scale, as the four 8-bit slices).
// Stored: a0, a1, a2 2^-12, a1 2^-12 -- integers up to 2048 and those integers
// times 2^-12 (normal FP16 numbers), all exact.  Every step is exact in T.
template <typename T>
__device__ __forceinline__ void slice_value_h(T v, int e, __half* out) {
    const T t = (sizeof(T) == 8) ? (T)ldexp((double)v, 8 - e) : (T)ldexpf((float)v, 8 - e);
    const T a0 = rint(t);
    const T r1 = (t - a0) * (T)4096;
    const T a1 = rint(r1);
    const T a2 = rint((r1 - a1) * (T)4096);
    out[0] = __float2half_rn((float)a0);
    out[1] = __float2half_rn((float)a1);
    out[2] = __float2half_rn((float)a2 * (1.0f / 4096.0f));
    out[3] = __float2half_rn((float)a1 * (1.0f / 4096.0f));
}

// row scale exponent of a row whose largest magnitude (rounded to float) is m
__device__ __forceinline__ int row_exponent(float m) {
    int e = 0;
    if (m > 0.0f) {
        frexpf(m, &e);   // m < 2^e
        e += 1;          // |v| 2^-e < 1/2
    }
    return e;
}

// 2^e as a double, exact for -1022 <= e <= 1023 (the range of two row scales)
__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }

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
