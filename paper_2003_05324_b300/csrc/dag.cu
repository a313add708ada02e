// A9: a persistent device-side tile-DAG scheduler for Algorithm 1 (replaces the
// paper's StarPU runtime).
//
// One cooperative launch, one CTA per SM, runs the whole factorization.  Each
// CTA hosts two worker groups that take tasks from two global queues:
//   tensor group (warps 0..5)  trailing updates on the tensor cores: TMA warp,
//                              single-thread MMA issue, 4 epilogue warps, items
//                              (128 x 128 output blocks) taken one at a time from
//                              the tensor queue.  Off-band targets: FP32-accurate
//                              products of FP16 slice planes (six MMAs per K
//                              step, tc_common.cuh); in-band (FP64)
//                              targets, by default: the FP64-accurate dsyrk /
//                              dgemm of the seven-slice products (tc_common.cuh);
//   CUDA-core group (warps 6..9) everything else, from the CUDA-core queue:
//       PC(k)        critical chain of dpotrf(k): for each 32 x 32 sub-block
//                    step s, the factor of (s,s), the solve of (s+1,s) and
//                    the update of (s+1,s+1)
//       PC2(k)       the chain below it: solve of (s+2,s), update of (s+2,s+1)
//       PT(k,r,s)    solve of sub-block (r,s) against L(s,s)
//       PU(k,r,c,s)  sub-block update (r,c) -= (r,s)(c,s)'      (DMMA f64)
//       TRSM(k,i,q)  rows of panel tile (i,k): dtrsm (band) or strsm (off band),
//                    followed, for tensor-core mode, by the fixed-point slicing
//                    of the solved rows (row exponent + slice planes)
//       UPD(k,i,j,q) 64 x 64 sub-block of a dsyrk / in-band dgemm    (DMMA f64;
//                    only with GEO_FLAG_FP64_DMMA, otherwise these updates
//                    are tensor items)
// Dependencies are integer counters in global memory, raised with release
// atomics and awaited with acquire loads (bounded by %globaltimer):
//   upd[i][j]   update items applied to tile (i,j) (all steps)
//   sub[i][j][q] steps applied to update sub-block q of tile (i,j) (an update
//               of step k waits only for step k-1 on its own sub-block)
//   tcnt[i][k]  solved row chunks of panel tile (i,k)
//   pot[k][r][c] operations applied to sub-block (r,c) of diagonal tile k, in
//               order: PU for s = 0..min(r,c)-1, then PT (r > c) or the
//               factor (r == c), whichever task (PT, PU, PC, PC2) runs them
// The queues are ordered topologically:
//   priority:  A(0) C(0) A(1) C(1) ...     A(k) = PC(k) PC2(k), the other
//                                          potrf(k) sub-tasks, trsm(k),
//                                          C(k) = FP64 items of step k on column k+1
//   bulk:      B(0) B(1) ...               B(k) = FP64 items of step k on columns >= k+2
//   tensor:    C'(0) B'(0) C'(1) B'(1) ... (tensor items, same split by column)
//   solve:     YD(0) YG(0;..) YD(1) ...    forward solve L y = Z fused into the
//                                          factorization; its head is claimed
//                                          only once its inputs are final
// (with the in-band updates on the tensor cores, C(k) and B(k) are empty).
// While a bulk queue exists at most a third of the CUDA-core groups (at least
// three, at most PRIO_LIMIT) work in the priority queue at once (its tasks form
// narrow dependency chains; the others keep the FP64 pipes busy with bulk
// items), and a bulk item of step k is claimed only after the priority head has
// passed A(k)'s solves.  Every wait is then on a task a running worker holds or
// can take: PC(k) and PC2(k) wait on sub-tasks queued after them, which a third
// priority worker takes in order; a priority task of step k+1 may wait on bulk
// items of step k, which the groups kept out of the priority queue take; tensor
// items and bulk items wait only on solves already claimed.  With at least
// GEO_MIN_CTAS = 4 CTAs, co-resident or not, the schedule cannot deadlock (with
// two, both CUDA-core groups can sit in PC(k) and PC2(k) waiting for sub-tasks
// no one is left to take).  Failure (non-SPD pivot, timeout) sets the status words; all
// workers poll them and leave, the tensor group draining its copies and MMAs
// and freeing tensor memory first.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "dag.cuh"
#include "tc_common.cuh"
#include "ysolve.cuh"

namespace geo {

// ------------------------------------------------------------- host side ---
static int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Rows per panel-solve task: FP64 (in-band) tiles of at least DP_SPLIT_MIN_NB
// rows in chunks of 32 rows, each row's contraction split over the group's four
// warps (FP64 is per warp instruction and slow on this part, so one warp per 32
// rows would set the pace of the whole step); smaller FP64 tiles, and FP32
// tiles, in chunks of 128, one thread per row.  (On tiles of 128 the split's
// per-column-block diagonal solves cost more SM time than they save, and the
// many-problem launches that use such tiles have parallelism to spare: the
// all-FP64 batch of 256 problems took 3.69 s with the split and 3.13 s
// without; on tiles of 500 the split halves the step.)  The row-per-thread
// FP64 solve lives only in the kernel instantiation of launches that hold such
// tiles (dag_kernel<true>): in the other one its code would cost the FP32 and
// tensor paths registers.
constexpr int DP_TRSM_ROWS = 32;
constexpr int SP_TRSM_ROWS = 128;
__host__ __device__ inline int dp_trsm_rows(int nb) { return nb >= DP_SPLIT_MIN_NB ? DP_TRSM_ROWS : SP_TRSM_ROWS; }

SchedGeom sched_geom(int p, int nb, int band, int pp, bool ex, bool dst) {
    SchedGeom g;
    g.p = p;
    g.ex = ex ? 1 : 0;
    g.dst = dst ? 1 : 0;
    g.ns = ceil_div(nb, 32);
    g.nsb64 = ceil_div(nb, 64);
    g.items64 = g.nsb64 * g.nsb64;
    g.items_tc = ceil_div(pp, TC_BM) * ceil_div(pp, TC_BN);
    g.chunks_dp = ceil_div(nb, dp_trsm_rows(nb));
    g.chunks_sp = ceil_div(nb, SP_TRSM_ROWS);
    g.chunks_y = ceil_div(nb, 128);
    // counters: grab counters, upd[p*p], tcnt[p*p], pot[p*ns*ns], sub[p*p*maxitems],
    // ycnt[p*chunks_y], ydone[p] + the number of finished YD tasks + the head of
    // the problem's own solve queue
    g.max_items = std::max(g.items64, g.items_tc);
    g.n_counters = 16 + 2 * (long long)p * p + (long long)p * g.ns * g.ns + (long long)p * p * g.max_items +
                   (long long)p * g.chunks_y + p + 2;
    long long n_prio = 0, n_bulk = 0, n_tct = 0, n_y = 0;
    // with DST, panel tiles (i,k) at i - k >= band are zero: no solve, no
    // update reads them, no forward-solve contribution
    const int reach = dst ? band : p;   // rows i < k + reach of panel k are nonzero
    for (int k = 0; k < p; ++k) {
        const int iend = (int)std::min<long long>(p, (long long)k + reach);
        n_y += 1 + (long long)(iend - k - 1) * g.chunks_y;   // YD(k), YG(i > k, chunks)
        const int ns = g.ns;
        // PC, PC2, then PT and PU without the chains' PT(s+1, s), PU(s+1, s+1, s),
        // PT(s+2, s) and PU(s+2, s+1, s)
        const long long n2 = std::max(0, ns - 2);
        n_prio += 2 + ns * (ns - 1) / 2 - (ns - 1) - n2 + (long long)ns * (ns - 1) * (ns + 1) / 6 - (ns - 1) - n2;
        for (int i = k + 1; i < iend; ++i) n_prio += is_dp(i, k, band) ? g.chunks_dp : g.chunks_sp;
        for (int j = k + 1; j < iend; ++j)
            for (int i = j; i < iend; ++i) {
                if (is_dp(i, j, band) && !ex) (j == k + 1 ? n_prio : n_bulk) += g.items64;
                else n_tct += 1;
            }
    }
    g.n_prio = n_prio;
    g.n_bulk = n_bulk;
    g.n_g2 = n_prio + n_bulk;
    g.n_tct = n_tct;
    g.n_y = n_y;
    return g;
}

// Fill the CUDA-core queues and the tensor-queue targets in their queue order.
// Priority queue: A(k) C(k) for k = 0, 1, ...; bulk queue: B(0) B(1) ...;
// trsm_end[k] = priority-queue index just past A(k)'s triangular solves.  With
// in-band updates on the tensor cores (g.ex) every update is a tensor target
// and the CUDA-core queues hold only the A(k).  Forward-solve queue: Y(0) Y(1)
// ..., Y(k) = YD(k) then YG(k; i, q) for i = k+1..p-1 -- the forward solve of
// Eq. 2 fused into the factorization (used only by a launch given Z).  With
// the DST approximation (g.dst) only rows i < k + band of each step exist.
void sched_build(const SchedGeom& g, int band, std::vector<G2Task>& prio, std::vector<G2Task>& bulk,
                 std::vector<int>& trsm_end, std::vector<G2Task>& yq, std::vector<int4>& tct) {
    const int p = g.p, ns = g.ns;
    const bool ex = g.ex != 0;
    auto iend = [&](int k) { return g.dst ? std::min(p, k + band) : p; };
    prio.clear();
    bulk.clear();
    tct.clear();
    yq.clear();
    trsm_end.assign((size_t)p, 0);
    for (int k = 0; k < p; ++k) {
        yq.push_back({T_YD, k, 0, 0, 0});
        for (int i = k + 1; i < iend(k); ++i)
            for (int q = 0; q < g.chunks_y; ++q) yq.push_back({T_YG, k, i, q, 0});
    }
    auto A = [&](int k) {
        prio.push_back({T_PC, k, 0, 0, 0});
        prio.push_back({T_PC2, k, 0, 0, 0});
        for (int s = 0; s < ns; ++s) {
            for (int r = s + 3; r < ns; ++r) prio.push_back({T_PT, k, r, s, 0});
            for (int c = s + 1; c < ns; ++c)
                for (int r = c; r < ns; ++r)
                    if (!(r == s + 1 && c == s + 1) && !(r == s + 2 && c == s + 1))
                        prio.push_back({T_PU, k, r, c, s});
        }
        for (int i = k + 1; i < iend(k); ++i) {
            const int nq = is_dp(i, k, band) ? g.chunks_dp : g.chunks_sp;
            for (int q = 0; q < nq; ++q) prio.push_back({T_TRSM, k, i, q, 0});
        }
        trsm_end[(size_t)k] = (int)prio.size();
    };
    auto fp64_items = [&](std::vector<G2Task>& out, int k, int jlo, int jhi) {
        for (int j = jlo; j < jhi; ++j)
            for (int i = j; i < p; ++i)
                if (is_dp(i, j, band))
                    for (int q = 0; q < g.items64; ++q) out.push_back({T_UPD, k, i, j, q});
    };
    for (int k = 0; k < p; ++k) {
        A(k);
        if (ex) continue;
        if (k + 1 < p) fp64_items(prio, k, k + 1, k + 2);   // C(k): column k+1
        fp64_items(bulk, k, k + 2, p);                      // B(k): columns >= k+2
    }
    // tensor queue in right-looking order, C'(k) B'(k) per step.  (A
    // left-looking order -- all updates of column j before column j+1 -- was
    // measured 2x slower: it chains the j updates of each block of the next
    // panel into the critical path.)  B'(k) takes column k+2 (the next step's
    // look-ahead column) first, then the other columns in groups of SWEEP_W,
    // row by row: the items in flight then read the panel blocks of one row
    // and of SWEEP_W columns instead of sweeping the whole panel once per
    // column, which keeps more of the panel's slice planes in L2.
    constexpr int SWEEP_W = 8;
    for (int k = 0; k < p; ++k) {
        const int ie = iend(k);
        for (int i = k + 1; i < ie; ++i)                 // C'(k): column k+1
            if (ex || !is_dp(i, k + 1, band)) tct.push_back(make_int4(i, k + 1, k, 0));
        for (int j = k + 2; j < std::min(ie, k + 3); ++j)  // B'(k): column k+2
            for (int i = j; i < ie; ++i)
                if (ex || !is_dp(i, j, band)) tct.push_back(make_int4(i, j, k, 0));
        for (int j0 = k + 3; j0 < ie; j0 += SWEEP_W)      // columns >= k+3
            for (int i = j0; i < ie; ++i)
                for (int j = j0; j < std::min(j0 + SWEEP_W, i + 1); ++j)
                    if (ex || !is_dp(i, j, band)) tct.push_back(make_int4(i, j, k, 0));
    }
}

// ----------------------------------------------------------- device side ---
constexpr int G2_THREADS = 128;
constexpr int DAG_THREADS = TC_THREADS + G2_THREADS;
constexpr int RING = 8;
constexpr size_t DAG_DYN_SMEM = (size_t)TC_STAGES * TC_STAGE_BYTES + 1024 /*align*/ + 512 /*barriers, ring*/;

constexpr int Y_SCAN = 2;       // problems whose solve-queue head a claim attempt looks at
constexpr int PRIO_LIMIT = 48;   // workers allowed inside priority tasks at once when a bulk queue exists

struct DagArgs {
    ProbDev one;             // the problem of a single-problem launch
    const ProbDev* probs;    // batched launch: the problems' views in global memory (nullptr: single)
    const G2Task* prio;
    const G2Task* bulk;
    long long n_prio, n_bulk;
    const int4* tct;         // tensor targets (i, j, k, problem)
    long long n_tc_items;
    const G2Task* yq;        // forward-solve queue of a single-problem launch given Z (else n_y = 0)
    long long n_y;
    int per;                 // tensor items per target
    int* ctr;    // [0] priority head, [1] tensor head, [2] bulk head, [3] workers in priority tasks,
                 // [4] abort: a wait timed out somewhere, [5] forward-solve head
    unsigned long long* trace_ctr;   // optional task trace (nullptr: off)
    geo_trace_rec* trace;
    long long trace_cap;
    long long wait_ns;       // bound of every wait of the launch (geo_tiles_set_timeout_ns)
    int nprob;               // batched launch: number of problems
    double* out;             // batched launch: problem b's (l, log|Sigma|, Z' Sigma^-1 Z) at out[3b]
    long long* done_ns;      // optional: [0] launch start, [1 + pid] when that problem's result was written
};

__device__ __forceinline__ const ProbDev& prob_of(const DagArgs& A, int pid) {
    return A.probs ? A.probs[pid] : A.one;
}
__device__ __forceinline__ bool aborted(const DagArgs& A) { return *((volatile const int*)A.ctr + 4) != 0; }

__device__ __forceinline__ int smid() {
    int s;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
    return s;
}

__device__ __forceinline__ void trace_put(const DagArgs& A, int type, int k, int a, int b, int c, long long t0,
                                          long long t1, long long t2) {
    if (!A.trace) return;
    const unsigned long long q = atomicAdd(A.trace_ctr, 1ull);
    if ((long long)q >= A.trace_cap) return;
    geo_trace_rec r;
    r.type = type;
    r.sm = smid();
    r.k = k;
    r.a = a;
    r.b = b;
    r.c = c;
    r.t_claim = t0;
    r.t_ready = t1;
    r.t_end = t2;
    A.trace[q] = r;
}

__device__ __forceinline__ void g2_sync() { asm volatile("bar.sync 2, 128;" ::: "memory"); }
struct G2Sync {
    __device__ void operator()() const { g2_sync(); }
};
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Wait until *p >= v (acquire).  False once the problem's status records a
// failure, the launch is aborted, or the wait exceeds its bound (the launch's,
// or `bound` ns if > 0; then it records GEO_ERR_TIMEOUT with `where` in the
// problem's status and aborts the launch: a timeout means the schedule itself
// went wrong).
__device__ bool wait_ge(const DagArgs& A, const Layout& L, const int* p, int v, int where, long long bound = 0) {
    if (ld_acquire_s32(p) >= v) return true;
    const long long dl = gtimer() + (bound > 0 ? bound : A.wait_ns);
    for (unsigned it = 1;; ++it) {
        __nanosleep(64);
        if (ld_acquire_s32(p) >= v) return true;
        if ((it & 31u) == 0) {
            if (failed(L) || aborted(A)) return false;
            if (gtimer() > dl) {
                set_timeout(L, where);
                atomicExch(A.ctr + 4, 1);
                return false;
            }
        }
    }
}

// first step whose update reaches block row i (0, or with DST the first step
// k' whose panel tile (i,k') is nonzero), and the number of such steps before k
__device__ __forceinline__ int first_step(const ProbDev& P, int i) {
    return P.g.dst ? max(0, i - P.L.band + 1) : 0;
}
__device__ __forceinline__ int steps_before(const ProbDev& P, int i, int k) { return k - first_step(P, i); }
// update items applied to tile (i,j) per step
__device__ __forceinline__ int items_of(const ProbDev& P, int i, int j) {
    return (is_dp(i, j, P.L.band) && !P.g.ex) ? P.g.items64 : P.g.items_tc;
}
__device__ __forceinline__ int chunks_of(const ProbDev& P, int i, int k) {
    return is_dp(i, k, P.L.band) ? P.g.chunks_dp : P.g.chunks_sp;
}
__device__ __forceinline__ int* sub_at(const ProbDev& P, int i, int j, int q) {
    return P.sub + ((size_t)i * P.L.p + j) * P.g.max_items + q;
}
__device__ __forceinline__ int* pot_at(const ProbDev& P, int k, int r, int c) {
    return P.pot + ((size_t)k * P.g.ns + r) * P.g.ns + c;
}

// ---- CUDA-core group: shared memory of one task at a time
struct G2Smem {
    union {
        struct {
            double As[2][64 * 12], Bs[2][64 * 12];   // UPD: double-buffered K chunks of 8
        } upd;
        struct {
            double D[32 * 33], X[32 * 33];           // PC / PT / PU operands
        } pot;
        struct {
            double Lb[(16 * 32 + 32 * 33) / 2 + 8];  // TRSM: 16 x SB stage + SB x SB diagonal block
        } tr;
        struct {                                     // FP64 TRSM (g2_trsm_dp)
            double Ls[4][16 * 8];                    // per-warp 16 x 8 stage of L_kk
            double part[3][32][9];                   // warps 1..3: partial sums per row
            double Ld[8 * 17];                       // diagonal 8 x 8 block
            float rmax[32];                          // row maxima for the slicing
        } trd;
        YSolveSmem yd;                               // YD: diagonal forward solve
        double yk[YS_MAX_NB];                        // YG: y_k
    };
    int task, kind, ok, rows_ok;
};

// PT(k,r,s): X(r,s) <- X(r,s) L(s,s)^-T, right-looking over the 32 columns:
// lane i scales row i of column c by 1/L_cc, then row i of the later columns
// j > c is updated, the four warps taking the columns j = c+1.. in turn.
__device__ void g2_pt(const ProbDev& P, G2Smem& S, int k, int r, int s, int g) {
    const Layout& L = P.L;
    const int nb = L.nb, c0 = s * 32, r0 = r * 32, w = min(32, nb - c0), h = min(32, nb - r0);
    const int lane = g & 31, wp = g >> 5;
    double* T = dp_tile(L, k, k);
    double* D = S.pot.D;
    double* X = S.pot.X;
    for (int idx = g; idx < 32 * 32; idx += G2_THREADS) {
        const int a = idx % 32, b = idx / 32;
        D[a * 33 + b] = (a < w && b < w && a >= b) ? T[(size_t)(c0 + b) * nb + c0 + a] : 0.0;
        X[a * 33 + b] = (a < h && b < w) ? T[(size_t)(c0 + b) * nb + r0 + a] : 0.0;
    }
    g2_sync();
    // reciprocal pivots in the (unused) upper triangle's first row slot: D[c*33 + 32]
    if (g < w) D[g * 33 + 32] = 1.0 / D[g * 33 + g];
    g2_sync();
    for (int c = 0; c < w; ++c) {
        if (g < h) X[g * 33 + c] *= D[c * 33 + 32];
        g2_sync();
        if (lane < h) {
            const double xc = X[lane * 33 + c];
            for (int j = c + 1 + ((wp - (c + 1)) & 3); j < w; j += 4)
                X[lane * 33 + j] = fma(-xc, D[j * 33 + c], X[lane * 33 + j]);
        }
        g2_sync();
    }
    for (int idx = g; idx < 32 * 32; idx += G2_THREADS) {
        const int a = idx % 32, b = idx / 32;
        if (a < h && b < w) T[(size_t)(c0 + b) * nb + r0 + a] = X[a * 33 + b];
    }
}

__device__ __forceinline__ void dmma884(double& c0, double& c1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c0), "+d"(c1)
                 : "d"(a), "d"(b));
}

// PU(k,r,c,s): sub-block (r,c) -= (r,s)(c,s)'; 4 warps x 16 x 16, DMMA.
__device__ void g2_pu(const ProbDev& P, G2Smem& S, int k, int r, int c, int s, int g) {
    const Layout& L = P.L;
    const int nb = L.nb, s0 = s * 32, r0 = r * 32, q0 = c * 32;
    double* T = dp_tile(L, k, k);
    double* Ar = S.pot.D;
    double* Bc = S.pot.X;
    for (int idx = g; idx < 32 * 32; idx += G2_THREADS) {
        const int a = idx % 32, t = idx / 32;
        const bool tv = s0 + t < nb;
        Ar[a * 33 + t] = (tv && r0 + a < nb) ? T[(size_t)(s0 + t) * nb + r0 + a] : 0.0;
        Bc[a * 33 + t] = (tv && q0 + a < nb) ? T[(size_t)(s0 + t) * nb + q0 + a] : 0.0;
    }
    g2_sync();
    const int lane = g & 31, wp = g >> 5, gi = lane >> 2, tq = lane & 3;
    const int wr = (wp >> 1) * 16, wc = (wp & 1) * 16;
    double acc[2][2][2] = {{{0.0, 0.0}, {0.0, 0.0}}, {{0.0, 0.0}, {0.0, 0.0}}};
#pragma unroll
    for (int kk = 0; kk < 32; kk += 4) {
        double af[2], bf[2];
#pragma unroll
        for (int a = 0; a < 2; ++a) af[a] = Ar[(wr + a * 8 + gi) * 33 + kk + tq];
#pragma unroll
        for (int b = 0; b < 2; ++b) bf[b] = Bc[(wc + b * 8 + gi) * 33 + kk + tq];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) dmma884(acc[a][b][0], acc[a][b][1], af[a], bf[b]);
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int rr = r0 + wr + a * 8 + gi, cc = q0 + wc + b * 8 + 2 * tq + e;
                if (rr < nb && cc < nb && (r != c || rr >= cc)) T[(size_t)cc * nb + rr] -= acc[a][b][e];
            }
}

// ---- PC(k): the critical chain of dpotrf(k), one task.
// In the right-looking sub-block Cholesky of diagonal tile k the chain
// PF(s) -> PT(s+1, s) -> PU(s+1, s+1, s) -> PF(s+1) -> ... decides how long the
// factorization of the tile takes.  Run as separate tasks, every link pays a
// claim, a dependency wait, a reload of its operands from L2 and a release;
// with FP64 at 1/64 of the FP32 rate on this part those handoffs cost more than
// the arithmetic.  PC(k) runs the whole chain in one CUDA-core group with the
// two blocks it carries (L(s,s) and L(s+1,s)) kept in shared memory; the other
// PT and PU tasks of the tile (off the chain) stay in the queue, and the
// counters pot(k, r, c) keep their meaning: PC raises pot(s,s) by 2 (the last
// update PU(s,s,s-1) and PF(s); 1 for s = 0) and pot(s+1,s) by 1 (PT(s+1,s)).

// D (w x w lower, 32 x 33 row-major in shared memory) <- its Cholesky factor;
// false if a pivot is not positive (status set, the same in every thread).
__device__ bool pc_factor(const Layout& L, double* D, int w, int row0, int g) {
    const int lane = g & 31, wp = g >> 5;
    for (int c = 0; c < w; ++c) {
        const double d = D[c * 33 + c];
        if (!(d > 0.0)) {
            if (g == 0 && atomicCAS(L.status + ST_CODE, 0, GEO_ERR_NOT_SPD) == 0) L.status[ST_INFO] = row0 + c + 1;
            return false;
        }
        const double rs = rsqrt(d);
        g2_sync();
        if (g < w - c) D[(c + g) * 33 + c] = (g == 0) ? d * rs : D[(c + g) * 33 + c] * rs;
        g2_sync();
        const int i = c + 1 + lane;
        if (i < w) {
            const double li = D[i * 33 + c];
            for (int j = c + 1 + ((wp - (c + 1)) & 3); j <= i; j += 4) D[i * 33 + j] = fma(-li, D[j * 33 + c], D[i * 33 + j]);
        }
        g2_sync();
    }
    return true;
}

// X (h x w, 32 x 33) <- X D^-T with D the factored block (reciprocal pivots in
// D's padding column 32).
__device__ void pc_solve(double* D, double* X, int h, int w, int g) {
    const int lane = g & 31, wp = g >> 5;
    if (g < w) D[g * 33 + 32] = 1.0 / D[g * 33 + g];
    g2_sync();
    for (int c = 0; c < w; ++c) {
        if (g < h) X[g * 33 + c] *= D[c * 33 + 32];
        g2_sync();
        if (lane < h) {
            const double xc = X[lane * 33 + c];
            for (int j = c + 1 + ((wp - (c + 1)) & 3); j < w; j += 4)
                X[lane * 33 + j] = fma(-xc, D[j * 33 + c], X[lane * 33 + j]);
        }
        g2_sync();
    }
}

// D (lower 32 x 32) -= X X' with X 32 x 32 (zero beyond its rows), DMMA, the
// contraction in steps of 4 as in PU.  The ten 8 x 8 tiles on and below the
// diagonal are spread over the four warps (3, 3, 2, 2): DMMA throughput per
// SM sub-partition, not latency, bounds this product on the chain.
__device__ void pc_syrk(double* D, const double* X, int g) {
    const int lane = g & 31, wp = g >> 5, gi = lane >> 2, tq = lane & 3;
    for (int t = wp; t < 10; t += 4) {
        const int tr = t < 1 ? 0 : t < 3 ? 1 : t < 6 ? 2 : 3;   // lower tiles in row order
        const int tc = t - tr * (tr + 1) / 2;
        double c0 = 0.0, c1 = 0.0;
#pragma unroll
        for (int kk = 0; kk < 32; kk += 4)
            dmma884(c0, c1, X[(tr * 8 + gi) * 33 + kk + tq], X[(tc * 8 + gi) * 33 + kk + tq]);
        const int rr = tr * 8 + gi, cc = tc * 8 + 2 * tq;
        if (rr >= cc) D[rr * 33 + cc] -= c0;
        if (rr >= cc + 1) D[rr * 33 + cc + 1] -= c1;
    }
}

__device__ bool g2_pchain(const DagArgs& A, const ProbDev& P, G2Smem& S, int k, int g) {
    const Layout& L = P.L;
    const int nb = L.nb, ns = P.g.ns;
    double* T = dp_tile(L, k, k);
    double* D = S.pot.D;
    double* X = S.pot.X;
    long long t0 = 0, t1 = 0, t2 = 0;   // sub-step times for the optional task trace (thread 0)
    for (int s = 0; s < ns; ++s) {
        const int c0 = s * 32, w = min(32, nb - c0);
        // (s,s) after the other workers' updates t <= s-2; the last one, from
        // the block solved in the previous step, is applied here
        if (g == 0 && A.trace) t0 = gtimer();
        if (g == 0) S.rows_ok = (s < 2 || wait_ge(A, L, pot_at(P, k, s, s), s - 1, 46)) ? 1 : 0;
        if (g == 0 && A.trace) t1 = gtimer();
        g2_sync();
        if (!S.rows_ok) return false;
#pragma unroll
        for (int u = 0; u < 32 * 32 / G2_THREADS; ++u) {   // all loads in flight at once
            const int idx = g + u * G2_THREADS, r = idx % 32, c = idx / 32;
            D[r * 33 + c] = (r < w && c < w && r >= c) ? T[(size_t)(c0 + c) * nb + c0 + r] : 0.0;
        }
        g2_sync();
        if (s > 0) {
            pc_syrk(D, X, g);
            g2_sync();
        }
        if (!pc_factor(L, D, w, k * nb + c0, g)) return false;
        for (int idx = g; idx < w * w; idx += G2_THREADS) {
            const int r = idx % w, c = idx / w;
            if (r >= c) T[(size_t)(c0 + c) * nb + c0 + r] = D[r * 33 + c];
        }
        __threadfence();
        g2_sync();
        if (g == 0) red_release_add(pot_at(P, k, s, s), s == 0 ? 1 : 2);
        if (g == 0 && A.trace) {
            t2 = gtimer();
            trace_put(A, 12, k, s, 0, 0, t0, t1, t2);   // wait, then update + factor of (s,s)
        }
        if (s + 1 == ns) break;
        // PT(s+1, s) after the other workers' updates t < s of that block
        const int r0 = c0 + 32, h = min(32, nb - r0);
        if (g == 0) S.rows_ok = (s == 0 || wait_ge(A, L, pot_at(P, k, s + 1, s), s, 47)) ? 1 : 0;
        if (g == 0 && A.trace) t1 = gtimer();
        g2_sync();
        if (!S.rows_ok) return false;
#pragma unroll
        for (int u = 0; u < 32 * 32 / G2_THREADS; ++u) {
            const int idx = g + u * G2_THREADS, a = idx % 32, b = idx / 32;
            X[a * 33 + b] = (a < h && b < w) ? T[(size_t)(c0 + b) * nb + r0 + a] : 0.0;
        }
        g2_sync();
        pc_solve(D, X, h, w, g);
        for (int idx = g; idx < 32 * 32; idx += G2_THREADS) {
            const int a = idx % 32, b = idx / 32;
            if (a < h && b < w) T[(size_t)(c0 + b) * nb + r0 + a] = X[a * 33 + b];
        }
        __threadfence();
        g2_sync();
        if (g == 0) red_release_add(pot_at(P, k, s + 1, s), 1);
        if (g == 0 && A.trace) trace_put(A, 13, k, s, 0, 0, t2, t1, gtimer());   // wait, then solve of (s+1,s)
    }
    return true;
}

// ---- PC2(k): the chain one sub-block below PC(k).  For each s it solves
// (s+2, s) against L(s,s) as soon as PF(s) is done, then applies (s+2, s+1) -=
// L(s+2, s) L(s+1, s)', the update PT(s+2, s+1) of PC's next step waits for.
// Run as separate tasks these two links, each paying a claim, a dependency
// wait and reloads, set the pace of PC; here they overlap PC's own work.
// Raises pot(s+2, s) and pot(s+2, s+1) by 1 each.
__device__ bool g2_pchain2(const DagArgs& A, const ProbDev& P, G2Smem& S, int k, int g) {
    const Layout& L = P.L;
    const int nb = L.nb, ns = P.g.ns;
    const int lane = g & 31, wp = g >> 5, gi = lane >> 2, tq = lane & 3;
    double* T = dp_tile(L, k, k);
    double* D = S.pot.D;
    double* X = S.pot.X;
    for (int s = 0; s + 2 < ns; ++s) {
        const int c0 = s * 32, r0 = c0 + 64, q0 = c0 + 32;
        const int w = 32, h = min(32, nb - r0);
        // PT(s+2, s): L(s,s) final, and the other workers' updates t < s of (s+2, s)
        if (g == 0)
            S.rows_ok = (wait_ge(A, L, pot_at(P, k, s, s), s + 1, 48) &&
                         (s == 0 || wait_ge(A, L, pot_at(P, k, s + 2, s), s, 49)))
                            ? 1
                            : 0;
        g2_sync();
        if (!S.rows_ok) return false;
#pragma unroll
        for (int u = 0; u < 32 * 32 / G2_THREADS; ++u) {
            const int idx = g + u * G2_THREADS, a = idx % 32, b = idx / 32;
            D[a * 33 + b] = (a >= b) ? T[(size_t)(c0 + b) * nb + c0 + a] : 0.0;
            X[a * 33 + b] = (a < h) ? T[(size_t)(c0 + b) * nb + r0 + a] : 0.0;
        }
        g2_sync();
        pc_solve(D, X, h, w, g);
        for (int idx = g; idx < 32 * 32; idx += G2_THREADS) {
            const int a = idx % 32, b = idx / 32;
            if (a < h) T[(size_t)(c0 + b) * nb + r0 + a] = X[a * 33 + b];
        }
        __threadfence();
        g2_sync();
        if (g == 0) red_release_add(pot_at(P, k, s + 2, s), 1);
        // PU(s+2, s+1, s): L(s+1, s) from PC, and the updates t < s of (s+2, s+1)
        if (g == 0)
            S.rows_ok = (wait_ge(A, L, pot_at(P, k, s + 1, s), s + 1, 57) &&
                         (s == 0 || wait_ge(A, L, pot_at(P, k, s + 2, s + 1), s, 58)))
                            ? 1
                            : 0;
        g2_sync();
        if (!S.rows_ok) return false;
#pragma unroll
        for (int u = 0; u < 32 * 32 / G2_THREADS; ++u) {
            const int idx = g + u * G2_THREADS, a = idx % 32, b = idx / 32;
            D[a * 33 + b] = T[(size_t)(c0 + b) * nb + q0 + a];   // L(s+1, s): 32 full rows
        }
        g2_sync();
        {
            const int wr = (wp >> 1) * 16, wc = (wp & 1) * 16;
            double acc[2][2][2] = {{{0.0, 0.0}, {0.0, 0.0}}, {{0.0, 0.0}, {0.0, 0.0}}};
#pragma unroll
            for (int kk = 0; kk < 32; kk += 4) {
                double af[2], bf[2];
#pragma unroll
                for (int a = 0; a < 2; ++a) af[a] = X[(wr + a * 8 + gi) * 33 + kk + tq];
#pragma unroll
                for (int b = 0; b < 2; ++b) bf[b] = D[(wc + b * 8 + gi) * 33 + kk + tq];
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int b = 0; b < 2; ++b) dmma884(acc[a][b][0], acc[a][b][1], af[a], bf[b]);
            }
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b)
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int rr = wr + a * 8 + gi, cc = wc + b * 8 + 2 * tq + e;
                        if (rr < h) T[(size_t)(q0 + cc) * nb + r0 + rr] -= acc[a][b][e];
                    }
        }
        __threadfence();
        g2_sync();
        if (g == 0) red_release_add(pot_at(P, k, s + 2, s + 1), 1);
    }
    return true;
}

// TRSM rows [r0, r0 + nrows) of panel tile (i,k) against L_kk (T = double for a
// band tile, float against FP32(L_kk) otherwise); thread g owns row r0 + g.
// Left-looking over super-blocks of SB columns held in registers: each earlier
// solved value of the row is read once per super-block and feeds SB FMAs, 16
// reads in flight at a time; the earlier columns' contributions are summed 16
// terms at a time before entering the accumulator.  L is staged through shared
// memory 16 x SB (and SB x SB for the diagonal block).  Returns max |x| of the row.
// ready(hi): called by the whole group before rows [0, hi) of L_kk are first
// read; false (the same in every thread) abandons the solve, returning -1.
template <typename T, int SB, typename Ready>
__device__ float g2_trsm_rows(const double* __restrict__ Lkk, T* __restrict__ X, int nb, int r0, int nrows, int g,
                              G2Smem& S, Ready& ready) {
    const int r = r0 + g;
    const bool valid = g < nrows && r < nb;
    T* Lst = reinterpret_cast<T*>(S.tr.Lb);            // [16][SB]
    T* Ld = reinterpret_cast<T*>(S.tr.Lb) + 16 * SB;   // [SB][SB + 1]
    float rowmax = 0.0f;
    for (int sb0 = 0; sb0 < nb; sb0 += SB) {
        const int w = min(SB, nb - sb0);
        if (!ready(sb0 + w)) return -1.0f;
        T acc[SB];
#pragma unroll
        for (int jj = 0; jj < SB; ++jj) acc[jj] = (valid && jj < w) ? X[(size_t)(sb0 + jj) * nb + r] : (T)0;
        // software pipeline over the stages of 16 earlier columns: the loads of
        // stage t0 + 16 are issued before the FMAs of stage t0
        constexpr int LPT = 16 * SB / G2_THREADS;   // staged L values per thread
        T lreg[LPT], xs[16];
        auto load_stage = [&](int t0) {
#pragma unroll
            for (int u = 0; u < LPT; ++u) {
                const int idx = g + u * G2_THREADS, tt = idx / SB, jj = idx % SB;
                lreg[u] = (jj < w) ? (T)Lkk[(size_t)(t0 + tt) * nb + sb0 + jj] : (T)0;
            }
            if (valid) {
#pragma unroll
                for (int tt = 0; tt < 16; ++tt) xs[tt] = X[(size_t)(t0 + tt) * nb + r];
            }
        };
        if (sb0 > 0) load_stage(0);
        for (int t0 = 0; t0 < sb0; t0 += 16) {
#pragma unroll
            for (int u = 0; u < LPT; ++u) Lst[g + u * G2_THREADS] = lreg[u];
            T xcur[16];
#pragma unroll
            for (int tt = 0; tt < 16; ++tt) xcur[tt] = xs[tt];
            g2_sync();
            if (t0 + 16 < sb0) load_stage(t0 + 16);
            if (valid) {
                T part[SB];
#pragma unroll
                for (int jj = 0; jj < SB; ++jj) part[jj] = (T)0;
#pragma unroll
                for (int tt = 0; tt < 16; ++tt)
#pragma unroll
                    for (int jj = 0; jj < SB; ++jj) part[jj] = fma(xcur[tt], Lst[tt * SB + jj], part[jj]);
#pragma unroll
                for (int jj = 0; jj < SB; ++jj) acc[jj] -= part[jj];
            }
            g2_sync();
        }
        // diagonal block: Ld[jj][ii] = L[sb0 + jj][sb0 + ii]
        for (int idx = g; idx < SB * SB; idx += G2_THREADS) {
            const int jj = idx / SB, ii = idx % SB;
            Ld[jj * (SB + 1) + ii] = (jj < w && ii <= jj) ? (T)Lkk[(size_t)(sb0 + ii) * nb + sb0 + jj] : (T)0;
        }
        g2_sync();
        if (valid) {
#pragma unroll
            for (int jj = 0; jj < SB; ++jj) {
                if (jj < w) {
                    const T xv = acc[jj] / Ld[jj * (SB + 1) + jj];
                    acc[jj] = xv;
#pragma unroll
                    for (int j2 = jj + 1; j2 < SB; ++j2) acc[j2] -= xv * Ld[j2 * (SB + 1) + jj];
                }
            }
#pragma unroll
            for (int jj = 0; jj < SB; ++jj)
                if (jj < w) {
                    X[(size_t)(sb0 + jj) * nb + r] = acc[jj];
                    rowmax = fmaxf(rowmax, fabsf((float)acc[jj]));
                }
        }
        g2_sync();
    }
    return rowmax;
}

// Fixed-point slicing of one solved row: row exponent, the NPL BF16 planes
// (slice_value) and, in a store with off-band tiles, the NPLH FP16 planes
// (slice_value_h) of the whole padded row, from the row's stored precision.
template <typename T>
__device__ void g2_slice_row(const Layout& L, const T* __restrict__ X, int i, int k, int r, float m) {
    const int nb = L.nb, pp = L.pp;
    const int e = row_exponent(m);
    const int slot = L.slot[i * L.p + k];
    L.rexp[(size_t)slot * pp + r] = e;
    __nv_bfloat16* P0 = plane(L, i, k, 0) + (size_t)r * pp;
    const size_t pstride = (size_t)pp * pp;
    for (int c0 = 0; c0 < pp; c0 += 8) {
        __align__(16) __nv_bfloat16 sl[NPL][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int c = c0 + q;
            const T v = (c < nb) ? X[(size_t)c * nb + r] : (T)0;
            __nv_bfloat16 d[NPL];
            slice_value<T>(v, e, d);
#pragma unroll
            for (int s = 0; s < NPL; ++s) sl[s][q] = d[s];
        }
#pragma unroll
        for (int s = 0; s < NPL; ++s)
            *reinterpret_cast<uint4*>(P0 + s * pstride + c0) = *reinterpret_cast<const uint4*>(sl[s]);
        if (L.npl > NPL) {
            __align__(16) __half sh[NPLH][8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int c = c0 + q;
                const T v = (c < nb) ? X[(size_t)c * nb + r] : (T)0;
                __half d[NPLH];
                slice_value_h<T>(v, e, d);
#pragma unroll
                for (int s = 0; s < NPLH; ++s) sh[s][q] = d[s];
            }
#pragma unroll
            for (int s = 0; s < NPLH; ++s)
                *reinterpret_cast<uint4*>(P0 + (NPL + s) * pstride + c0) = *reinterpret_cast<const uint4*>(sh[s]);
        }
    }
}

// FP64 panel solve of rows [r0, r0 + 32) of tile (i,k) against L_kk: lane l
// owns row r0 + l; for each 8-column super-block the contraction over the
// earlier columns is split over the four warps (16-column stages dealt in
// turn, each stage summed in registers), the partials are added in a fixed
// order, and warp 0 finishes the diagonal block.  ready(hi) as in
// g2_trsm_rows.  Leaves each row's max |x| in S.trd.rmax; false if abandoned.
// (8 columns at a time keep the registers of this path below those of the
// tensor group's epilogue, which shares the kernel's register budget.)
template <typename Ready>
__device__ bool g2_trsm_dp(const double* __restrict__ Lkk, double* __restrict__ X, int nb, int r0, int g,
                           G2Smem& S, Ready& ready) {
    constexpr int SB = 8, TS = 16;
    const int lane = g & 31, wp = g >> 5, r = r0 + lane;
    const bool valid = r < nb;
    double* Ls = S.trd.Ls[wp];
    float rowmax = 0.0f;
    for (int sb0 = 0; sb0 < nb; sb0 += SB) {
        const int w = min(SB, nb - sb0);
        if (!ready(sb0 + w)) return false;
        double part[SB];
#pragma unroll
        for (int jj = 0; jj < SB; ++jj) part[jj] = 0.0;
        const int tend = sb0 & ~(TS - 1);   // whole stages of TS earlier columns; the rest below
        for (int t0 = TS * wp; t0 < tend; t0 += 4 * TS) {
#pragma unroll
            for (int u = 0; u < TS * SB / 32; ++u) {
                const int idx = lane + 32 * u, tt = idx / SB, jj = idx % SB;
                Ls[idx] = (jj < w) ? Lkk[(size_t)(t0 + tt) * nb + sb0 + jj] : 0.0;
            }
            __syncwarp();
#pragma unroll
            for (int tt = 0; tt < TS; ++tt) {
                const double xv = valid ? X[(size_t)(t0 + tt) * nb + r] : 0.0;
#pragma unroll
                for (int jj = 0; jj < SB; ++jj) part[jj] = fma(xv, Ls[tt * SB + jj], part[jj]);
            }
            __syncwarp();
        }
        if (wp == 0) {
            // the columns [tend, sb0) (a partial stage) and the diagonal block
            for (int idx = lane; idx < SB * SB; idx += 32) {
                const int jj = idx / SB, ii = idx % SB;
                S.trd.Ld[jj * 17 + ii] = (jj < w && ii <= jj) ? Lkk[(size_t)(sb0 + ii) * nb + sb0 + jj] : 0.0;
            }
            for (int t = tend; t < sb0; ++t) {
                const double xv = valid ? X[(size_t)t * nb + r] : 0.0;
#pragma unroll
                for (int jj = 0; jj < SB; ++jj)
                    part[jj] = fma(xv, (jj < w) ? Lkk[(size_t)t * nb + sb0 + jj] : 0.0, part[jj]);
            }
        } else {
#pragma unroll
            for (int jj = 0; jj < SB; ++jj) S.trd.part[wp - 1][lane][jj] = part[jj];
        }
        g2_sync();
        if (wp == 0 && valid) {
            double acc[SB];
#pragma unroll
            for (int jj = 0; jj < SB; ++jj) {
                const double s4 = (part[jj] + S.trd.part[0][lane][jj]) + (S.trd.part[1][lane][jj] + S.trd.part[2][lane][jj]);
                acc[jj] = (jj < w) ? X[(size_t)(sb0 + jj) * nb + r] - s4 : 0.0;
            }
#pragma unroll
            for (int jj = 0; jj < SB; ++jj) {
                if (jj < w) {
                    const double xv = acc[jj] / S.trd.Ld[jj * 17 + jj];
                    acc[jj] = xv;
#pragma unroll
                    for (int j2 = jj + 1; j2 < SB; ++j2) acc[j2] = fma(-xv, S.trd.Ld[j2 * 17 + jj], acc[j2]);
                }
            }
#pragma unroll
            for (int jj = 0; jj < SB; ++jj)
                if (jj < w) {
                    X[(size_t)(sb0 + jj) * nb + r] = acc[jj];
                    rowmax = fmaxf(rowmax, fabsf((float)acc[jj]));
                }
        }
        g2_sync();
    }
    if (wp == 0) S.trd.rmax[lane] = rowmax;
    g2_sync();
    return true;
}

// Fixed-point slicing of the 32 rows solved by g2_trsm_dp: each warp slices a
// quarter of the padded columns of every row (lane = row), FP64 values.
__device__ void g2_slice_rows_dp(const Layout& L, const double* __restrict__ X, int i, int k, int r0, int g,
                                 G2Smem& S) {
    const int nb = L.nb, pp = L.pp, lane = g & 31, wp = g >> 5, r = r0 + lane;
    if (r >= nb) return;
    const int e = row_exponent(S.trd.rmax[lane]);
    const int slot = L.slot[i * L.p + k];
    if (wp == 0) L.rexp[(size_t)slot * pp + r] = e;
    __nv_bfloat16* P0 = plane(L, i, k, 0) + (size_t)r * pp;
    const size_t pstride = (size_t)pp * pp;
    const int q4 = pp / 4;   // pp is a multiple of 64: quarters of 16 columns or more
    for (int c0 = wp * q4; c0 < (wp + 1) * q4; c0 += 8) {
        __align__(16) __nv_bfloat16 sl[NPL][8];
        __align__(16) __half sh[NPLH][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int c = c0 + q;
            const double v = (c < nb) ? X[(size_t)c * nb + r] : 0.0;
            __nv_bfloat16 d[NPL];
            slice_value<double>(v, e, d);
#pragma unroll
            for (int s2 = 0; s2 < NPL; ++s2) sl[s2][q] = d[s2];
            if (L.npl > NPL) {
                __half dh[NPLH];
                slice_value_h<double>(v, e, dh);
#pragma unroll
                for (int s2 = 0; s2 < NPLH; ++s2) sh[s2][q] = dh[s2];
            }
        }
#pragma unroll
        for (int s2 = 0; s2 < NPL; ++s2)
            *reinterpret_cast<uint4*>(P0 + s2 * pstride + c0) = *reinterpret_cast<const uint4*>(sl[s2]);
        if (L.npl > NPL) {
#pragma unroll
            for (int s2 = 0; s2 < NPLH; ++s2)
                *reinterpret_cast<uint4*>(P0 + (NPL + s2) * pstride + c0) = *reinterpret_cast<const uint4*>(sh[s2]);
        }
    }
}

// UPD(k,i,j,q): 64 x 64 sub-block q of target (i,j) -= A(i,k) A(j,k)' in FP64.
__device__ void g2_upd(const ProbDev& P, G2Smem& S, int k, int i, int j, int q, int g) {
    const Layout& L = P.L;
    const int nb = L.nb, nsb = P.g.nsb64;
    const int sbr = q / nsb, sbc = q % nsb;
    const bool syrk = (i == j);
    if (syrk && sbr < sbc) return;
    const int R0 = sbr * 64, C0 = sbc * 64;
    const int lane = g & 31, wp = g >> 5, gi = lane >> 2, tq = lane & 3;
    const int wr = (wp >> 1) * 32, wc = (wp & 1) * 32;
    double acc[4][4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b][0] = acc[a][b][1] = 0.0;
    const bool a_dp = is_dp(i, k, L.band), b_dp = is_dp(j, k, L.band);
    // on a diagonal sub-block of a dsyrk, the warp owning the upper-right 32 x 32
    // quadrant has nothing below the diagonal: it only helps with the loads
    const bool idle = syrk && sbr == sbc && wr == 0 && wc == 32;
    const double* Ad = a_dp ? dp_tile(L, i, k) : nullptr;
    const float* Af = a_dp ? nullptr : sp_tile(L, i, k);
    const double* Bd = b_dp ? dp_tile(L, j, k) : nullptr;
    const float* Bf = b_dp ? nullptr : sp_tile(L, j, k);
    double va[4], vb[4];   // 64 x 8 chunk / 128 threads
    auto fetch = [&](int kc) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int idx = g + u * G2_THREADS, rr = idx % 64, tt = idx / 64, t = kc + tt;
            va[u] = (R0 + rr < nb && t < nb) ? (a_dp ? Ad[(size_t)t * nb + R0 + rr] : (double)Af[(size_t)t * nb + R0 + rr]) : 0.0;
            vb[u] = (C0 + rr < nb && t < nb) ? (b_dp ? Bd[(size_t)t * nb + C0 + rr] : (double)Bf[(size_t)t * nb + C0 + rr]) : 0.0;
        }
    };
    auto store = [&](int b) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int idx = g + u * G2_THREADS;
            S.upd.As[b][(idx % 64) * 12 + idx / 64] = va[u];
            S.upd.Bs[b][(idx % 64) * 12 + idx / 64] = vb[u];
        }
    };
    fetch(0);
    store(0);
    g2_sync();
    int buf = 0;
    for (int kc = 0; kc < nb; kc += 8, buf ^= 1) {
        const bool more = kc + 8 < nb;
        if (more) fetch(kc + 8);
#pragma unroll
        for (int kk = 0; kk < 8; kk += 4) {
            if (idle) break;
            double af[4], bf[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) af[a] = S.upd.As[buf][(wr + a * 8 + gi) * 12 + kk + tq];
#pragma unroll
            for (int b = 0; b < 4; ++b) bf[b] = S.upd.Bs[buf][(wc + b * 8 + gi) * 12 + kk + tq];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) dmma884(acc[a][b][0], acc[a][b][1], af[a], bf[b]);
        }
        if (more) store(buf ^ 1);
        g2_sync();
    }
    double* C = dp_tile(L, i, j);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int rr = R0 + wr + a * 8 + gi, cc = C0 + wc + b * 8 + 2 * tq + e;
                if (rr < nb && cc < nb && (!syrk || rr >= cc)) C[(size_t)cc * nb + rr] -= acc[a][b][e];
            }
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *(volatile const int*)p; }

// Dependencies of a forward-solve task, checked without waiting (acquire loads):
// YD(k) needs L_kk final and every earlier block row's contribution to block
// row k; YG(k; i, q) needs y_k, the solved tile (i,k) and the contributions of
// the steps before k to its rows.
__device__ bool y_ready(const ProbDev& P, const G2Task& t) {
    const int k = t.k, cy = P.g.chunks_y;
    if (t.type == T_YD) {
        if (ld_acquire_s32(pot_at(P, k, P.g.ns - 1, P.g.ns - 1)) < P.g.ns) return false;
        for (int q = 0; q < cy; ++q)
            if (ld_acquire_s32(P.ycnt + k * cy + q) < steps_before(P, k, k)) return false;
        // the last one sums every block row's partials: all other YD done
        return k < P.L.p - 1 || ld_acquire_s32(P.ydone + P.L.p) >= P.L.p - 1;
    }
    return ld_acquire_s32(P.ydone + k) >= 1 && ld_acquire_s32(P.tcnt + t.a * P.L.p + k) >= chunks_of(P, t.a, k) &&
           ld_acquire_s32(P.ycnt + t.a * cy + t.b) >= steps_before(P, t.a, k);
}

// Stop the whole launch (a wait timed out): the flag every wait polls, and in a
// single-problem launch that problem's status.
__device__ void abort_launch(const DagArgs& A, int where) {
    atomicExch(A.ctr + 4, 1);
    if (!A.probs) set_timeout(A.one.L, where);
}

template <bool kSmallDP>
__device__ void g2_worker(const DagArgs& A, G2Smem& S) {
    const int g = threadIdx.x - TC_THREADS;
    int* prio_head = A.ctr + 0;
    int* bulk_head = A.ctr + 2;
    int* inflight = A.ctr + 3;
    int* y_taken = A.ctr + 5;   // forward-solve tasks taken, all problems
    const int nq = A.probs ? A.nprob : 1;
    int yrot = (int)blockIdx.x % nq;   // (thread 0) next problem whose solve queue to look at
    __shared__ long long t_claim, t_ready;
    // groups allowed in the priority queue at once while bulk items exist
    const int prio_cap = A.n_bulk > 0 ? max(3, min(PRIO_LIMIT, (int)gridDim.x / 3)) : DAG_THREADS * 4096;
    for (;;) {
        // ---- claim: the forward-solve queue's head when its dependencies are
        // met (so it never holds a worker waiting), else the priority queue while
        // fewer than PRIO_LIMIT workers are in it, otherwise the bulk queue once
        // the priority head has passed the solves its next items need; sleep
        // when none is available.
        if (g == 0) {
            int kind = -1, idx = -1;
            const long long dl = gtimer() + A.wait_ns;
            for (unsigned spin = 0; kind < 0; ++spin) {
                if (aborted(A) || (!A.probs && failed(A.one.L))) break;
                // each problem has its own solve queue (a segment of yq, taken in
                // order, its head only when ready); look at Y_SCAN problems per
                // attempt, in a rotation that starts at this CTA's index, so that
                // no problem's head waits behind another's.  (A solve task of a
                // failed problem is taken at once and dropped below.)
                int yt = 0;   // solve tasks taken so far, all problems
                if (A.n_y > 0 && nq == 1) {   // one problem: its head is that count (one load)
                    const ProbDev& P = prob_of(A, 0);
                    const int h = ld_volatile(P.yhead);
                    yt = h;
                    if (h < A.n_y && (failed(P.L) || y_ready(P, A.yq[h])) && atomicCAS(P.yhead, h, h + 1) == h) {
                        idx = h;
                        kind = 2;
                        break;
                    }
                } else if (A.n_y > 0 && (yt = ld_volatile(y_taken)) < A.n_y) {
                    for (int q = 0; q < min(Y_SCAN, nq) && kind < 0; ++q) {
                        const int pid = yrot;
                        yrot = yrot + 1 == nq ? 0 : yrot + 1;
                        const ProbDev& P = prob_of(A, pid);
                        const int h = ld_volatile(P.yhead);
                        if (P.y0 + h >= P.y1) continue;
                        const G2Task& ty = A.yq[P.y0 + h];
                        if ((failed(P.L) || y_ready(P, ty)) && atomicCAS(P.yhead, h, h + 1) == h) {
                            atomicAdd(y_taken, 1);
                            idx = P.y0 + h;
                            kind = 2;
                        }
                    }
                    if (kind >= 0) break;
                }
                const int ph = ld_volatile(prio_head);
                if (ph < A.n_prio) {
                    if (atomicAdd(inflight, 1) < prio_cap) {
                        idx = atomicAdd(prio_head, 1);
                        if (idx < A.n_prio) {
                            kind = 0;
                            break;
                        }
                    }
                    atomicSub(inflight, 1);
                }
                const int bh = ld_volatile(bulk_head);
                if (bh < A.n_bulk) {
                    const G2Task& tb = A.bulk[bh];
                    if (ld_volatile(prio_head) >= prob_of(A, tb.pid).trsm_end[tb.k]) {
                        idx = atomicAdd(bulk_head, 1);
                        if (idx < A.n_bulk) {
                            kind = 1;
                            break;
                        }
                    }
                } else if (ph >= A.n_prio && yt >= A.n_y) {
                    break;   // every queue exhausted
                }
                __nanosleep(256);
                if ((spin & 63u) == 63u && gtimer() > dl) {
                    abort_launch(A, 10);
                    break;
                }
            }
            S.task = kind < 0 ? -1 : idx;
            S.kind = kind;
            t_claim = gtimer();
        }
        g2_sync();
        if (S.task < 0) return;
        const int kind = S.kind, tix = S.task;
        const G2Task t = kind == 0 ? A.prio[tix] : kind == 1 ? A.bulk[tix] : A.yq[tix];
        const ProbDev& P = prob_of(A, t.pid);
        const Layout& L = P.L;
        const int nb = L.nb, ns = P.g.ns;
        // ---- dependencies (thread 0 waits, the group follows); a task of a
        // problem that has failed (not positive definite) is skipped
        if (g == 0) {
            bool ok = !failed(L);
            const int k = t.k;
            if (ok && kind == 1 && ld_volatile(prio_head) < P.trsm_end[k])
                ok = wait_ge(A, L, prio_head, P.trsm_end[k], 25);
            if (ok) switch (t.type) {
                case T_PC:   // the tile's trailing updates; the chain waits for the rest as it goes
                case T_PC2:
                    ok = wait_ge(A, L, P.upd + k * L.p + k, steps_before(P, k, k) * items_of(P, k, k), 11);
                    break;
                case T_PT:
                    if (t.b == 0) ok = wait_ge(A, L, P.upd + k * L.p + k, steps_before(P, k, k) * items_of(P, k, k), 13);
                    ok = ok && wait_ge(A, L, pot_at(P, k, t.b, t.b), t.b + 1, 14) &&
                         wait_ge(A, L, pot_at(P, k, t.a, t.b), t.b, 15);
                    break;
                case T_PU:
                    if (t.c == 0) ok = wait_ge(A, L, P.upd + k * L.p + k, steps_before(P, k, k) * items_of(P, k, k), 16);
                    ok = ok && wait_ge(A, L, pot_at(P, k, t.a, t.c), t.c + 1, 17) &&
                         wait_ge(A, L, pot_at(P, k, t.b, t.c), t.c + 1, 18) &&
                         wait_ge(A, L, pot_at(P, k, t.a, t.b), t.c, 19);
                    break;
                case T_TRSM:   // the first sub-block of L_kk; the solve waits for later ones as it goes
                    ok = wait_ge(A, L, pot_at(P, k, 0, 0), 1, 20) &&
                         wait_ge(A, L, P.upd + t.a * L.p + k, steps_before(P, t.a, k) * items_of(P, t.a, k), 21);
                    break;
                case T_YD:   // L_kk final and every earlier block row's contribution applied; the
                             // last one also every other YD (with DST nothing else orders them)
                    if (P.z) {
                        ok = wait_ge(A, L, pot_at(P, k, ns - 1, ns - 1), ns, 40);
                        for (int q = 0; ok && q < P.g.chunks_y; ++q)
                            ok = wait_ge(A, L, P.ycnt + k * P.g.chunks_y + q, steps_before(P, k, k), 41);
                        if (ok && k == L.p - 1) ok = wait_ge(A, L, P.ydone + L.p, L.p - 1, 50);
                    }
                    break;
                case T_YG:   // y_k solved, tile (i,k) solved, contributions of steps < k applied
                    if (P.z)
                        ok = wait_ge(A, L, P.ydone + k, 1, 42) &&
                             wait_ge(A, L, P.tcnt + t.a * L.p + k, chunks_of(P, t.a, k), 43) &&
                             wait_ge(A, L, P.ycnt + t.a * P.g.chunks_y + t.b, steps_before(P, t.a, k), 44);
                    break;
                default:   // T_UPD: own sub-block's previous step only
                    ok = wait_ge(A, L, P.tcnt + t.a * L.p + k, chunks_of(P, t.a, k), 22) &&
                         wait_ge(A, L, P.tcnt + t.b * L.p + k, chunks_of(P, t.b, k), 23) &&
                         wait_ge(A, L, sub_at(P, t.a, t.b, t.c), steps_before(P, t.a, k), 24);
                    break;
            }
            S.ok = ok ? 1 : 0;
            t_ready = gtimer();
        }
        g2_sync();
        if (!S.ok) {   // failed problem or aborted launch: drop the task
            if (g == 0 && kind == 0) atomicSub(inflight, 1);
            continue;
        }
        // ---- the task
        int* done = nullptr;
        bool ran = true;
        switch (t.type) {
            case T_PC:   // signals its own sub-blocks as it goes
                ran = g2_pchain(A, P, S, t.k, g);
                break;
            case T_PC2:
                ran = g2_pchain2(A, P, S, t.k, g);
                break;
            case T_PT:
                g2_pt(P, S, t.k, t.a, t.b, g);
                done = pot_at(P, t.k, t.a, t.b);
                break;
            case T_PU:
                g2_pu(P, S, t.k, t.a, t.b, t.c, g);
                done = pot_at(P, t.k, t.a, t.b);
                break;
            case T_TRSM: {
                const int i = t.a, k = t.k, q = t.b;
                const double* Lkk = dp_tile(L, k, k);
                const int r = q * SP_TRSM_ROWS + g;
                // POTRF(k) finishes L_kk's 32-row sub-blocks in order (sub-block
                // row s is final once (s,s) is factored): the solve of this tile
                // runs alongside it, waiting only before rows not yet final
                int s_done = 0;
                auto ready = [&](int hi) -> bool {
                    const int s = (hi - 1) / 32;
                    if (s < s_done) return true;
                    if (g == 0) S.rows_ok = wait_ge(A, L, pot_at(P, k, s, s), s + 1, 45) ? 1 : 0;
                    g2_sync();
                    s_done = s + 1;
                    return S.rows_ok != 0;
                };
                if (is_dp(i, k, L.band) && nb >= DP_SPLIT_MIN_NB) {
                    double* X = dp_tile(L, i, k);
                    ran = g2_trsm_dp(Lkk, X, nb, q * DP_TRSM_ROWS, g, S, ready);
                    if (ran && L.planes) g2_slice_rows_dp(L, X, i, k, q * DP_TRSM_ROWS, g, S);
                } else if (is_dp(i, k, L.band)) {
                    if constexpr (kSmallDP) {
                        double* X = dp_tile(L, i, k);
                        const float m =
                            g2_trsm_rows<double, 16>(Lkk, X, nb, q * SP_TRSM_ROWS, SP_TRSM_ROWS, g, S, ready);
                        ran = m >= 0.0f;
                        if (ran && L.planes && r < nb) g2_slice_row<double>(L, X, i, k, r, m);
                    } else {   // the host launches dag_kernel<true> for such tiles
                        if (g == 0) abort_launch(A, 59);
                        ran = false;
                    }
                } else {
                    float* X = sp_tile(L, i, k);
                    const float m = g2_trsm_rows<float, 32>(Lkk, X, nb, q * SP_TRSM_ROWS, SP_TRSM_ROWS, g, S, ready);
                    ran = m >= 0.0f;
                    if (ran && L.planes && r < nb) g2_slice_row<float>(L, X, i, k, r, m);
                }
                fence_proxy_async_global();   // the planes are read by TMA
                done = P.tcnt + i * L.p + k;
                break;
            }
            case T_YD: {   // y_k = L_kk^-1 r_k (r_k = Z_k when no step reaches block row k); the last
                           // one sums the partials
                if (!P.z) break;
                const int k = t.k;
                double* yv = L.scal + 2 * L.p + 8;
                if (first_step(P, k) == k)
                    for (int r = g; r < nb; r += G2_THREADS) {
                        const size_t gi = (size_t)k * nb + r;
                        yv[gi] = gi < (size_t)L.n ? P.z[gi] : 0.0;
                    }
                g2_sync();
                ysolve_diag_tile(L, k, yv, L.scal, g, G2_THREADS, S.yd, G2Sync());
                if (k == L.p - 1 && g == 0) {
                    if (A.probs) {   // batched: (l, log|Sigma|, Z' Sigma^-1 Z) of problem pid
                        double* o = A.out + 3 * (size_t)t.pid;
                        ysolve_finish(L, L.scal, o + 1, o + 2, o);
                    } else {
                        ysolve_finish(L, L.scal, P.res, P.res + 1, P.res + 2);
                    }
                    if (A.done_ns) {
                        __threadfence();
                        A.done_ns[1 + t.pid] = gtimer();
                    }
                }
                done = P.ydone + k;
                break;
            }
            case T_YG: {   // rows of r_i -= L(i,k) y_k (the first step reaching row i starts from Z_i)
                if (!P.z) break;
                const int i = t.a, k = t.k;
                double* yv = L.scal + 2 * L.p + 8;
                for (int c = g; c < nb; c += G2_THREADS) S.yk[c] = yv[(size_t)k * nb + c];
                g2_sync();
                const int r = t.b * G2_THREADS + g;
                if (r < nb) {
                    const double acc = yrow_update(L, i, k, r, S.yk);
                    const size_t gi = (size_t)i * nb + r;
                    const double base = (k == first_step(P, i)) ? (gi < (size_t)L.n ? P.z[gi] : 0.0) : yv[gi];
                    yv[gi] = base - acc;
                }
                done = P.ycnt + i * P.g.chunks_y + t.b;
                break;
            }
            default:
                g2_upd(P, S, t.k, t.a, t.b, t.c, g);
                done = P.upd + t.a * L.p + t.b;
                break;
        }
        __threadfence();
        g2_sync();
        if (g == 0) {
            if (ran && done) {   // (no counter: a solve task of a launch without Z)
                if (t.type == T_UPD) red_release_add(sub_at(P, t.a, t.b, t.c), 1);
                if (t.type == T_YD) red_release_add(P.ydone + L.p, 1);
                red_release_add(done, 1);
            }
            if (kind == 0) atomicSub(inflight, 1);
            trace_put(A, t.type, t.k, t.a, t.b, t.c, t_claim, t_ready, gtimer());
        }
    }
}

// ---- tensor group: the split-BF16 update with dynamic items and dependencies
// bounded mbarrier wait for the scheduler: gives up when the launch is aborted
// (or a single problem has failed), on an abort of this CTA, or after the launch's wait bound
__device__ bool dwait(const DagArgs& A, uint32_t bar, uint32_t parity, volatile int* abort_flag) {
    if (mbar_try(bar, parity)) return true;
    const long long dl = gtimer() + A.wait_ns;
    for (unsigned it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255u) == 0) {
            if (*abort_flag || aborted(A) || (!A.probs && failed(A.one.L))) return false;
            if (gtimer() > dl) return false;
        }
    }
}

// Tensor-queue item w: target (i,j) of step k, output block (mb, nc) of
// TC_BM x TC_BN.  An off-band target's block is one FP32-accurate product (one
// TMEM buffer, 10 slice pairs over the whole contraction); an in-band target's
// block (with in-band updates on the tensor cores) is FP64-accurate: for each of its one or two 64-column halves
// and each 256-long part of the contraction, the 28 slice pairs of two passes
// into seven accumulators spanning both TMEM buffers, drained into the FP64
// tile before the next part.  Blocks of a diagonal target wholly above its
// diagonal are not computed.
struct TcItem {
    int i, j, k, mb, nc, rem, pid;
    bool ex, skip, pad;
    int nh;   // in-band: 64-column halves holding columns < nb
    int fp;   // off-band target of the far tier: its products (1 or 3); 0 = the six of the FP32-accurate tier
};

__device__ __forceinline__ TcItem tc_decode(const DagArgs& A, long long w) {
    const int4 tg = A.tct[w / A.per];
    TcItem t;
    t.i = tg.x;
    t.j = tg.y;
    t.k = tg.z;
    t.pid = tg.w;
    const ProbDev& P = prob_of(A, t.pid);
    const int nnc = (P.L.pp + TC_BN - 1) / TC_BN;
    t.rem = (int)(w % A.per);
    t.pad = t.rem >= P.g.items_tc;   // a smaller problem of a batch: no such block
    t.mb = t.rem / nnc;
    t.nc = t.rem % nnc;
    t.ex = P.g.ex && is_dp(t.i, t.j, P.L.band);
    t.skip = t.ex && t.i == t.j && t.mb < t.nc;
    t.nh = (t.nc * TC_BN + EX_BN < P.L.nb) ? 2 : 1;
    t.fp = (!t.ex && P.L.far && P.L.far[t.i * P.L.p + t.j]) ? P.L.far_products : 0;
    return t;
}

__device__ void tc_worker(const DagArgs& A, const CUtensorMap* tmap_a, const CUtensorMap* tmap_b,
                          const CUtensorMap* tmap_b64, uint8_t* smem, uint64_t* bars, uint32_t tmem_base,
                          volatile int* abort_flag, volatile int* ring) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ int s_epi_skip;
    const uint32_t bar0 = smem_u32(bars);
    auto FULL = [&](int s) { return bar0 + 8u * s; };
    auto EMPTY = [&](int s) { return bar0 + 8u * (TC_STAGES + s); };
    auto TFULL = [&](int a) { return bar0 + 8u * (2 * TC_STAGES + a); };
    auto TEMPTY = [&](int a) { return bar0 + 8u * (2 * TC_STAGES + 2 + a); };
    auto RFULL = [&](int q) { return bar0 + 8u * (2 * TC_STAGES + 4 + q); };
    constexpr int KPC = EX_KP / TC_BK;   // K chunks per part of an in-band item
    const bool single = A.probs == nullptr;
    if (warp == 0) {
        if (lane != 0) return;
        int it = 0;
        for (int t = 0;;) {
            const long long tq0 = A.trace ? gtimer() : 0;   // trace: claim, dependencies met, first copies issued
            long long tq1 = 0;
            long long w = (*abort_flag || aborted(A) || (single && failed(A.one.L))) ? -1 : atomicAdd(A.ctr + 1, 1);
            if (w >= A.n_tc_items) w = -1;
            TcItem m;
            if (w >= 0) {
                m = tc_decode(A, w);
                const ProbDev& P = prob_of(A, m.pid);
                if (m.pad || (!single && failed(P.L))) continue;   // no such block / problem failed
                if (m.skip) {   // nothing below the diagonal: count the item as applied
                    red_release_add(P.upd + m.i * P.L.p + m.j, 1);
                    continue;
                }
                // (the test hook GEO_FLAG_TEST_STALL asks the items of step 0
                // for one solved row chunk more than the panel tile has: that
                // wait can never be met and ends by half the launch's bound, so
                // it gives up before any wait downstream of it and its location
                // is the one recorded)
                const int stall = (P.L.flags & GEO_FLAG_TEST_STALL) && m.k == 0;
                const bool ok = wait_ge(A, P.L, P.tcnt + m.i * P.L.p + m.k, chunks_of(P, m.i, m.k) + stall, 31,
                                        stall ? A.wait_ns / 2 : 0) &&
                                wait_ge(A, P.L, P.tcnt + m.j * P.L.p + m.k, chunks_of(P, m.j, m.k), 32);
                if (!ok) {
                    if (!single && !aborted(A)) continue;   // its problem failed meanwhile
                    w = -1;
                } else {
                    fence_proxy_async_global();
                }
                if (A.trace) tq1 = gtimer();
            }
            ring[t % RING] = (int)w;
            mbar_arrive(RFULL(t % RING));
            ++t;
            const int st0 = it % TC_STAGES;
            if (w < 0) {
                // hand the end marker to the MMA thread through the next stage
                if (dwait(A, EMPTY(st0), ((it / TC_STAGES) & 1) ^ 1, abort_flag)) mbar_arrive(FULL(st0));
                ++it;
                break;
            }
            const ProbDev& P = prob_of(A, m.pid);
            const int p = P.L.p, nk = P.L.pp / TC_BK, nkp = (nk + KPC - 1) / KPC;
            const int sa = P.L.slot[m.i * p + m.k] * P.L.npl, sb = P.L.slot[m.j * p + m.k] * P.L.npl;
            const CUtensorMap* map_a = single ? tmap_a : P.tmap;
            const CUtensorMap* map_b = single ? tmap_b : P.tmap + 1;
            const CUtensorMap* map_b64 = single ? tmap_b64 : P.tmap + 2;
            bool ok = true;
            auto next_stage = [&](uint32_t bytes) -> uint8_t* {
                const int st = it % TC_STAGES;
                const uint32_t ph = (it / TC_STAGES) & 1;
                if (!dwait(A, EMPTY(st), ph ^ 1, abort_flag)) return nullptr;
                mbar_expect_tx(FULL(st), bytes);
                return smem + st * TC_STAGE_BYTES;
            };
            if (!m.ex) {   // FP16 planes NPL.. of the 8/12/12 split (a far item: the first one or two of each)
                const int na = m.fp == 1 ? 1 : m.fp == 3 ? 2 : TC_HA;
                const int nbq = m.fp == 1 ? 1 : m.fp == 3 ? 2 : TC_HB;
                const uint32_t bytes = (uint32_t)(na * TC_A_BYTES + nbq * TC_B_BYTES);
                for (int kc = 0; kc < nk && ok; ++kc, ++it) {
                    uint8_t* sbase = next_stage(bytes);
                    if (!sbase) {
                        ok = false;
                        break;
                    }
                    const uint32_t full = FULL(it % TC_STAGES);
                    for (int s = 0; s < na; ++s)
                        tma_load_3d(smem_u32(sbase + s * TC_A_BYTES), map_a, kc * TC_BK, m.mb * TC_BM, sa + NPL + s,
                                    full);
                    for (int s = 0; s < nbq; ++s)
                        tma_load_3d(smem_u32(sbase + TC_HA * TC_A_BYTES + s * TC_B_BYTES), map_b, kc * TC_BK,
                                    m.nc * TC_BN, sb + NPL + s, full);
                    if (A.trace && kc == 0) trace_put(A, 16, m.k, m.i, m.j, m.rem, tq0, tq1, gtimer());
                }
            } else {
                for (int h = 0; h < m.nh && ok; ++h) {
                    const int brow = m.nc * TC_BN + h * EX_BN;
                    for (int kp = 0; kp < nkp && ok; ++kp) {
                        const int kc0 = kp * KPC, kc1 = min(nk, kc0 + KPC);
                        for (int pass = 0; pass < 2 && ok; ++pass)
                            for (int kc = kc0; kc < kc1; ++kc, ++it) {
                                uint8_t* sbase = next_stage(pass == 0 ? EX_P1_BYTES : EX_P2_BYTES);
                                if (!sbase) {
                                    ok = false;
                                    break;
                                }
                                const uint32_t full = FULL(it % TC_STAGES);
                                if (pass == 0) {
#pragma unroll
                                    for (int s = 0; s < 4; ++s)
                                        tma_load_3d(smem_u32(sbase + s * TC_A_BYTES), map_a, kc * TC_BK,
                                                    m.mb * TC_BM, sa + s, full);
#pragma unroll
                                    for (int s = 0; s < NPL; ++s)
                                        tma_load_3d(smem_u32(sbase + 4 * TC_A_BYTES + s * EX_B_BYTES), map_b64,
                                                    kc * TC_BK, brow, sb + s, full);
                                } else {
#pragma unroll
                                    for (int u = 0; u < 3; ++u)
                                        tma_load_3d(smem_u32(sbase + u * TC_A_BYTES), map_a, kc * TC_BK,
                                                    m.mb * TC_BM, sa + 4 + u, full);
#pragma unroll
                                    for (int s = 0; s < 3; ++s)
                                        tma_load_3d(smem_u32(sbase + 3 * TC_A_BYTES + s * EX_B_BYTES), map_b64,
                                                    kc * TC_BK, brow, sb + s, full);
                                }
                            }
                    }
                }
            }
            if (!ok) {
                abort_launch(A, 33);
                *abort_flag = 1;
                break;
            }
        }
        for (int q = max(0, it - TC_STAGES); q < it; ++q)
            mbar_wait(FULL(q % TC_STAGES), (q / TC_STAGES) & 1, gtimer() + min(A.wait_ns, TC_WAIT_NS));
    } else if (warp == 1) {
        if (lane != 0) return;
        int it = 0;
        int use0 = 0, use1 = 0, nxt = 0;   // completed uses of each TMEM buffer; buffer of the next off-band item
        auto bail = [&](int where) {
            abort_launch(A, where);
            *abort_flag = 1;
            mbar_arrive(TFULL(0));
            mbar_arrive(TFULL(1));
        };
        for (int tc = 0;; ++tc) {
            // the first stage of the item carries the item id (or the end marker)
            const int st0 = it % TC_STAGES;
            const long long tm0 = A.trace ? gtimer() : 0;   // trace: waiting for the item, first stage in
            if (!dwait(A, FULL(st0), (it / TC_STAGES) & 1, abort_flag)) {
                bail(34);
                break;
            }
            const long long tm1 = A.trace ? gtimer() : 0;
            const int w = ring[tc % RING];
            if (w < 0) break;   // end marker (the epilogue reads it from the ring)
            const TcItem m = tc_decode(A, w);
            const ProbDev& P = prob_of(A, m.pid);
            const int nk = P.L.pp / TC_BK, nkp = (nk + KPC - 1) / KPC;
            bool ok = true;
            bool first = true;   // FULL(it) of the item's first stage already observed
            auto stage = [&]() -> uint32_t {
                const int st = it % TC_STAGES;
                if (!first && !dwait(A, FULL(st), (it / TC_STAGES) & 1, abort_flag)) return 0;
                first = false;
                tc_fence_after();
                return smem_u32(smem + st * TC_STAGE_BYTES);
            };
            if (!m.ex) {
                const int b = nxt;
                if (!dwait(A, TEMPTY(b), ((b ? use1 : use0) & 1) ^ 1, abort_flag)) {
                    bail(35);
                    break;
                }
                tc_fence_after();
                const uint32_t dst0 = tmem_base + b * (2 * TC_BN), dst1 = dst0 + TC_BN;
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const uint32_t sbase = stage();
                    if (!sbase) {
                        ok = false;
                        break;
                    }
                    if (m.fp == 0) {
                        // descriptors from the stage's one: a shared-memory offset of
                        // o bytes adds o / 16 to it (addresses stay below 2^18 bytes)
                        constexpr int PA[TC_HPAIRS] = {0, 1, 0, 2, 0, 1};   // the six pairs (tc_common.cuh)
                        constexpr int PB[TC_HPAIRS] = {0, 3, 2, 0, 1, 0};
                        const uint64_t da = sw64_desc(sbase);
                        const uint64_t db = da + (uint64_t)((TC_HA * TC_A_BYTES) >> 4);
                        const uint32_t later = kc != 0;
#pragma unroll
                        for (int q = 0; q < TC_HPAIRS; ++q)
#pragma unroll
                            for (int kk = 0; kk < TC_BK / 16; ++kk)
                                umma_bf16(q == 0 ? dst0 : dst1,
                                          da + (uint64_t)((PA[q] * TC_A_BYTES + kk * 32) >> 4),
                                          db + (uint64_t)((PB[q] * TC_B_BYTES + kk * 32) >> 4),
                                          later | (uint32_t)((q > 1) | (kk > 0)), TC_IDESC_F16);
                    } else {
                        // far tier: a0 b0 -> acc0; with three products a0 b1 + a1 b0 -> acc1
                        const uint32_t a0 = sbase, a1 = sbase + TC_A_BYTES;
                        const uint32_t b0 = sbase + TC_HA * TC_A_BYTES, b1 = b0 + TC_B_BYTES;
#pragma unroll
                        for (int kk = 0; kk < TC_BK / 16; ++kk)
                            umma_bf16(dst0, sw64_desc(a0 + kk * 32), sw64_desc(b0 + kk * 32), (kc | kk) != 0,
                                      TC_IDESC_F16);
                        if (m.fp == 3) {
#pragma unroll
                            for (int kk = 0; kk < TC_BK / 16; ++kk)
                                umma_bf16(dst1, sw64_desc(a0 + kk * 32), sw64_desc(b1 + kk * 32), (kc | kk) != 0,
                                          TC_IDESC_F16);
#pragma unroll
                            for (int kk = 0; kk < TC_BK / 16; ++kk)
                                umma_bf16(dst1, sw64_desc(a1 + kk * 32), sw64_desc(b0 + kk * 32), 1u, TC_IDESC_F16);
                        }
                    }
                    umma_commit(EMPTY(it % TC_STAGES));
                }
                if (!ok) {
                    bail(36);
                    break;
                }
                umma_commit(TFULL(b));
                if (b) ++use1;
                else ++use0;
                nxt ^= 1;
                if (A.trace) trace_put(A, 15, m.k, m.i, m.j, m.rem, tm0, tm1, gtimer());
            } else {
                for (int h = 0; h < m.nh && ok; ++h)
                    for (int kp = 0; kp < nkp && ok; ++kp) {
                        if (!dwait(A, TEMPTY(0), (use0 & 1) ^ 1, abort_flag) ||
                            !dwait(A, TEMPTY(1), (use1 & 1) ^ 1, abort_flag)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        uint32_t touched = 0;
                        const int kc0 = kp * KPC, kc1 = min(nk, kc0 + KPC);
                        for (int pass = 0; pass < 2 && ok; ++pass)
                            for (int kc = kc0; kc < kc1; ++kc, ++it) {
                                const uint32_t sbase = stage();
                                if (!sbase) {
                                    ok = false;
                                    break;
                                }
                                // one MMA per (A slice, run of B slices): N = 64 x the run,
                                // the accumulator the run of level slots; each slot's
                                // first product of the part overwrites it
                                const int nq = pass == 0 ? EX_P1_MMAS : EX_P2_MMAS;
                                const uint32_t b_base = sbase + (pass == 0 ? 4 : 3) * TC_A_BYTES;
#pragma unroll 1
                                for (int q = 0; q < nq; ++q) {
                                    const signed char* e = pass == 0 ? c_ex1[q] : c_ex2[q];
                                    const int slot = e[3], cnt = e[2];
                                    const uint32_t a_addr = sbase + e[0] * TC_A_BYTES;
                                    const uint32_t b_addr = b_base + e[1] * EX_B_BYTES;
                                    const uint32_t idesc = ex_idesc(EX_BN * cnt);
#pragma unroll
                                    for (int kk = 0; kk < TC_BK / 16; ++kk) {
                                        umma_bf16(tmem_base + slot * EX_BN, sw64_desc(a_addr + kk * 32),
                                                  sw64_desc(b_addr + kk * 32), (touched >> slot) & 1u, idesc);
                                        touched |= ((1u << cnt) - 1u) << slot;
                                    }
                                }
                                umma_commit(EMPTY(it % TC_STAGES));
                            }
                        if (!ok) break;
                        umma_commit(TFULL(0));
                        umma_commit(TFULL(1));
                        ++use0;
                        ++use1;
                    }
                if (!ok) {
                    bail(36);
                    break;
                }
            }
        }
        if (it > 0) {
            const int q = it - 1;
            mbar_wait(EMPTY(q % TC_STAGES), (q / TC_STAGES) & 1, gtimer() + min(A.wait_ns, TC_WAIT_NS));
        }
    } else {
        // epilogue warps 2..5: TMEM lane quadrant warp % 4
        const int quad = warp & 3;
        const int row_in = quad * 32 + lane;
        int use0 = 0, use1 = 0, nxt = 0;
        for (int tc = 0;; ++tc) {
            if (!dwait(A, RFULL(tc % RING), (tc / RING) & 1, abort_flag)) {
                abort_launch(A, 37);
                *abort_flag = 1;
                break;
            }
            const int w = ring[tc % RING];
            if (w < 0) break;
            const TcItem m = tc_decode(A, w);
            const int i = m.i, j = m.j, k = m.k;
            const ProbDev& P = prob_of(A, m.pid);
            const Layout& L = P.L;
            const int nb = L.nb, pp = L.pp, p = L.p;
            const int nk = pp / TC_BK, nkp = (nk + KPC - 1) / KPC;
            // read-modify-write of C(i,j) only after the previous step's items on
            // it; when its problem has failed (batched launch) the item's TMEM is
            // still consumed, but nothing is written
            const long long te0 = gtimer();
            long long te1 = te0;   // products done (off-band), for the trace
            if (threadIdx.x == 64) {
                s_epi_skip = 0;
                if (!wait_ge(A, L, sub_at(P, i, j, m.rem), steps_before(P, i, k), 38)) {
                    if (single || aborted(A)) *abort_flag = 1;
                    else s_epi_skip = 1;
                }
            }
            epi_sync();
            if (*abort_flag) break;
            const bool write = s_epi_skip == 0;
            const int r = m.mb * TC_BM + row_in;
            const bool rv = write && r < nb;
            const int* eb = L.rexp + (size_t)L.slot[j * p + k] * pp;
            const int er = (r < pp) ? L.rexp[(size_t)L.slot[i * p + k] * pp + r] : 0;
            const uint32_t tlane = (uint32_t)(quad * 32) << 16;
            bool ok = true;
            if (!m.ex) {
                const int b = nxt;
                float* C = sp_tile(L, i, j);
                const int c_begin = m.nc * TC_BN;
                const int ncol = rv ? max(0, min(TC_BN, nb - c_begin)) : 0;
                float* Crow = C + (size_t)c_begin * nb + (rv ? r : 0);
                constexpr int BATCH = 32;
                float cpre[BATCH];
#pragma unroll
                for (int e = 0; e < BATCH; ++e) cpre[e] = (e < ncol) ? Crow[(size_t)e * nb] : 0.0f;
                if (!dwait(A, TFULL(b), (b ? use1 : use0) & 1, abort_flag) || *abort_flag) {
                    abort_launch(A, 39);
                    *abort_flag = 1;
                    break;
                }
                if (A.trace) te1 = gtimer();
                tc_fence_after();
                const uint32_t taddr = tmem_base + tlane + b * (2 * TC_BN);
#pragma unroll 1
                for (int hb = 0; hb < TC_BN / BATCH; ++hb) {
                    if (hb > 0) {
#pragma unroll
                        for (int e = 0; e < BATCH; ++e)
                            cpre[e] = (hb * BATCH + e < ncol) ? Crow[(size_t)(hb * BATCH + e) * nb] : 0.0f;
                    }
#pragma unroll
                    for (int cc = 0; cc < BATCH; cc += 16) {
                        float v0[16], v1[16];
                        tmem_ld16(taddr + hb * BATCH + cc, v0);
                        if (m.fp != 1) {
                            tmem_ld16(taddr + TC_BN + hb * BATCH + cc, v1);
                        } else {   // the one-product far tier writes no second accumulator
#pragma unroll
                            for (int e = 0; e < 16; ++e) v1[e] = 0.0f;
                        }
                        int ec[16];
                        const int cl0 = c_begin + hb * BATCH + cc;
                        if (cl0 + 16 <= pp) {
                            const int4* e4 = reinterpret_cast<const int4*>(eb + cl0);
#pragma unroll
                            for (int qq = 0; qq < 4; ++qq) {
                                const int4 w4 = e4[qq];
                                ec[4 * qq] = w4.x;
                                ec[4 * qq + 1] = w4.y;
                                ec[4 * qq + 2] = w4.z;
                                ec[4 * qq + 3] = w4.w;
                            }
                        } else {
#pragma unroll
                            for (int e = 0; e < 16; ++e) ec[e] = 0;
                        }
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            cpre[cc + e] -= fmaf(v1[e], 1.0f / 4096.0f, v0[e]) * pow2f(er + ec[e] - 16);
                    }
#pragma unroll
                    for (int e = 0; e < BATCH; ++e)
                        if (hb * BATCH + e < ncol) Crow[(size_t)(hb * BATCH + e) * nb] = cpre[e];
                }
                tc_fence_before();
                mbar_arrive(TEMPTY(b));
                if (b) ++use1;
                else ++use0;
                nxt ^= 1;
            } else {
                double* C = dp_tile(L, i, j);
                const bool diag = (i == j);
                for (int h = 0; h < m.nh && ok; ++h) {
                    const int c_begin = m.nc * TC_BN + h * EX_BN;
                    int ncol = rv ? max(0, min(EX_BN, nb - c_begin)) : 0;
                    if (diag) ncol = min(ncol, max(0, r - c_begin + 1));   // lower triangle only
                    double* Crow = C + (size_t)c_begin * nb + (rv ? r : 0);
                    for (int kp = 0; kp < nkp; ++kp) {
                        const long long tp0 = (A.trace && threadIdx.x == 64) ? gtimer() : 0;
                        double cpre[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) cpre[e] = (e < ncol) ? Crow[(size_t)e * nb] : 0.0;
                        if (!dwait(A, TFULL(0), use0 & 1, abort_flag) ||
                            !dwait(A, TFULL(1), use1 & 1, abort_flag) || *abort_flag) {
                            ok = false;
                            break;
                        }
                        const long long tp1 = (A.trace && threadIdx.x == 64) ? gtimer() : 0;
                        tc_fence_after();
#pragma unroll 1
                        for (int cc = 0; cc < EX_BN; cc += 8) {
                            float v[EX_NSLOT][8];
                            tmem_ld8x8(tmem_base + tlane + cc, v);
                            const int4 ea = *reinterpret_cast<const int4*>(eb + c_begin + cc);
                            const int4 ebb = *reinterpret_cast<const int4*>(eb + c_begin + cc + 4);
                            const int ec[8] = {ea.x, ea.y, ea.z, ea.w, ebb.x, ebb.y, ebb.z, ebb.w};
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                const long long tot = ex_fixed_total(v[0][e], v[1][e], v[2][e], v[3][e], v[4][e],
                                                                     v[5][e], v[6][e], v[EX_X][e]);
                                cpre[e] = fma(-(double)tot, pow2d(er + ec[e] - 56), cpre[e]);
                            }
#pragma unroll
                            for (int e = 0; e < 8; ++e)
                                if (cc + e < ncol) Crow[(size_t)(cc + e) * nb] = cpre[e];
                            if (cc + 8 < EX_BN) {
#pragma unroll
                                for (int e = 0; e < 8; ++e)
                                    cpre[e] = (cc + 8 + e < ncol) ? Crow[(size_t)(cc + 8 + e) * nb] : 0.0;
                            }
                        }
                        tc_fence_before();
                        mbar_arrive(TEMPTY(0));
                        mbar_arrive(TEMPTY(1));
                        ++use0;
                        ++use1;
                        if (A.trace && threadIdx.x == 64)   // one (slice, part): products done, drained
                            trace_put(A, 14, k, i, j, h * nkp + kp, tp0, tp1, gtimer());
                    }
                }
                if (!ok) {
                    abort_launch(A, 39);
                    *abort_flag = 1;
                    break;
                }
            }
            __threadfence();
            epi_sync();
            if (threadIdx.x == 64 && write) {
                red_release_add(sub_at(P, i, j, m.rem), 1);
                red_release_add(P.upd + i * p + j, 1);
                trace_put(A, m.ex ? 11 : 10, k, i, j, m.rem, te0, te1, gtimer());
            }
        }
    }
}

template <bool kSmallDP>
__global__ void __launch_bounds__(DAG_THREADS, 1)
    dag_kernel(DagArgs A, const __grid_constant__ CUtensorMap tmap_a, const __grid_constant__ CUtensorMap tmap_b,
               const __grid_constant__ CUtensorMap tmap_b64) {
    extern __shared__ uint8_t dag_smem_raw[];
    __shared__ G2Smem g2s;
    uint8_t* smem = (uint8_t*)(((uintptr_t)dag_smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = (uint64_t*)(smem + TC_STAGES * TC_STAGE_BYTES);
    // bars: FULL[S], EMPTY[S], TFULL[2], TEMPTY[2], RFULL[RING]; then tmem slot, abort flag, ring
    volatile uint32_t* tmem_slot = (volatile uint32_t*)(bars + 2 * TC_STAGES + 4 + RING);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    volatile int* ring = abort_flag + 1;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0 && blockIdx.x == 0 && A.done_ns) A.done_ns[0] = gtimer();
    if (threadIdx.x == 0) {
        *abort_flag = 0;
        const uint32_t b0 = smem_u32(bars);
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(b0 + 8u * s, 1);
            mbar_init(b0 + 8u * (TC_STAGES + s), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(b0 + 8u * (2 * TC_STAGES + a), 1);
            mbar_init(b0 + 8u * (2 * TC_STAGES + 2 + a), 128);
        }
        for (int q = 0; q < RING; ++q) mbar_init(b0 + 8u * (2 * TC_STAGES + 4 + q), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
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
    if (threadIdx.x < TC_THREADS) tc_worker(A, &tmap_a, &tmap_b, &tmap_b64, smem, bars, tmem_base, abort_flag, ring);
    else g2_worker<kSmallDP>(A, g2s);
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TC_TMEM_COLS)
                     : "memory");
    }
    // an aborted batched launch: every problem whose last solve task did not
    // run is marked as timed out (its result stays NaN)
    if (A.probs && blockIdx.x == 0 && threadIdx.x == 0 && aborted(A))
        for (int b = 0; b < A.nprob; ++b) {
            const ProbDev& P = A.probs[b];
            if (ld_acquire_s32(P.ydone + P.L.p - 1) < 1) set_timeout(P.L, 9);
        }
}

template <bool kSmallDP>
static cudaError_t dag_prepare(int& nsm) {
    static int attr_done = 0, nsm_cached = 0;
    cudaError_t e;
    if (!attr_done) {
        if ((e = cudaFuncSetAttribute(dag_kernel<kSmallDP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)DAG_DYN_SMEM)))
            return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm_cached, cudaDevAttrMultiProcessorCount, dev);
        attr_done = 1;
    }
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dag_kernel<kSmallDP>, DAG_THREADS, DAG_DYN_SMEM)))
        return e;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    nsm = nsm_cached;
    return cudaSuccess;
}

// counters of one problem inside its block (after the 16 launch-wide words)
void bind_counters(ProbDev& P, int* base) {
    const int p = P.L.p;
    P.upd = base;
    P.tcnt = P.upd + (size_t)p * p;
    P.pot = P.tcnt + (size_t)p * p;
    P.sub = P.pot + (size_t)p * P.g.ns * P.g.ns;
    P.ycnt = P.sub + (size_t)p * p * P.g.max_items;
    P.ydone = P.ycnt + (size_t)p * P.g.chunks_y;
    P.yhead = P.ydone + p + 1;   // the problem's own forward-solve queue: tasks taken
}

cudaError_t run_potrf_dag(const geo_tiles* t, const Layout& L, const SchedView& sv, const double* z, double* res,
                          cudaStream_t s) {
    int nsm = 0;
    const bool small_dp = dag_small_dp(L.nb, L.band);
    cudaError_t e = small_dp ? dag_prepare<true>(nsm) : dag_prepare<false>(nsm);
    if (e) return e;
    if ((e = cudaMemsetAsync(sv.counters, 0, sizeof(int) * (size_t)sv.geom.n_counters, s))) return e;
    DagArgs A;
    memset(&A, 0, sizeof(A));
    A.one.L = L;
    A.one.g = sv.geom;
    A.one.trsm_end = sv.trsm_end;
    A.one.tmap = nullptr;
    A.one.z = z;
    A.one.res = res;
    A.yq = z ? sv.yq : nullptr;
    A.n_y = z ? sv.geom.n_y : 0;
    bind_counters(A.one, sv.counters + 16);
    A.one.yhead = sv.counters + 5;   // one problem: the solve head beside the launch's other queue heads
    A.one.y0 = 0;
    A.one.y1 = (int)A.n_y;
    A.probs = nullptr;
    A.prio = sv.prio;
    A.bulk = sv.bulk;
    A.n_prio = sv.geom.n_prio;
    A.n_bulk = sv.geom.n_bulk;
    A.tct = sv.tct;
    A.per = sv.geom.items_tc;
    A.n_tc_items = sv.geom.n_tct * (long long)A.per;
    A.ctr = sv.counters;
    A.trace_ctr = (unsigned long long*)t->trace;
    A.trace = t->trace ? (geo_trace_rec*)((char*)t->trace + 64) : nullptr;
    A.trace_cap = t->trace_cap;
    A.wait_ns = t->timeout_ns > 0 ? t->timeout_ns : GEO_DEFAULT_TIMEOUT_NS;
    CUtensorMap maps[3];
    memcpy(maps, t->tmap, sizeof(maps));
    void* args[] = {&A, &maps[0], &maps[1], &maps[2]};
    prof_begin(4, s);
    e = cudaLaunchCooperativeKernel(small_dp ? (const void*)dag_kernel<true> : (const void*)dag_kernel<false>,
                                    dim3(nsm), dim3(DAG_THREADS), args, DAG_DYN_SMEM, s);
    prof_end(4, s);
    count_launch();
    return e;
}

void sched_merge(const std::vector<SchedGeom>& g, const std::vector<int>& band, BatchPlan& out) {
    const int nprob = (int)g.size();
    out.prio.clear();
    out.bulk.clear();
    out.tct.clear();
    out.trsm_end.assign((size_t)nprob, std::vector<int>());
    out.per = 1;
    std::vector<std::vector<G2Task>> prio((size_t)nprob), bulk((size_t)nprob);
    std::vector<std::vector<int>> tend((size_t)nprob);
    std::vector<std::vector<G2Task>> yq((size_t)nprob);
    std::vector<std::vector<int4>> tct((size_t)nprob);
    int pmax = 0;
    for (int b = 0; b < nprob; ++b) {
        sched_build(g[(size_t)b], band[(size_t)b], prio[(size_t)b], bulk[(size_t)b], tend[(size_t)b], yq[(size_t)b],
                    tct[(size_t)b]);
        out.trsm_end[(size_t)b].assign((size_t)g[(size_t)b].p, 0);
        out.per = std::max(out.per, g[(size_t)b].items_tc);
        pmax = std::max(pmax, g[(size_t)b].p);
    }
    // every queue of a problem is ordered by step; step k of all problems
    // precedes step k+1 of any (staggering the problems' steps against each
    // other was measured to make no difference).  Each problem's solve runs
    // inside the launch from its own queue, and its result is written as soon
    // as its own last block row is solved.
    out.yq.clear();
    std::vector<size_t> ip((size_t)nprob, 0), ib((size_t)nprob, 0), it((size_t)nprob, 0);
    for (int k = 0; k < pmax; ++k) {
        for (int b = 0; b < nprob; ++b) {
            const std::vector<G2Task>& q = prio[(size_t)b];
            const size_t seg0 = ip[(size_t)b];
            const size_t base = out.prio.size();
            while (ip[(size_t)b] < q.size() && q[ip[(size_t)b]].k == k) {
                G2Task tk = q[ip[(size_t)b]++];
                tk.pid = b;
                out.prio.push_back(tk);
            }
            if (k < g[(size_t)b].p)
                out.trsm_end[(size_t)b][(size_t)k] = (int)(base + ((size_t)tend[(size_t)b][(size_t)k] - seg0));
        }
        for (int b = 0; b < nprob; ++b) {
            const std::vector<G2Task>& q = bulk[(size_t)b];
            while (ib[(size_t)b] < q.size() && q[ib[(size_t)b]].k == k) {
                G2Task tk = q[ib[(size_t)b]++];
                tk.pid = b;
                out.bulk.push_back(tk);
            }
        }
        for (int b = 0; b < nprob; ++b) {
            const std::vector<int4>& q = tct[(size_t)b];
            while (it[(size_t)b] < q.size() && q[it[(size_t)b]].z == k) {
                int4 v = q[it[(size_t)b]++];
                v.w = b;
                out.tct.push_back(v);
            }
        }
    }
    // the forward-solve queues stay one segment per problem, each taken by its
    // own head (ybeg[b] .. ybeg[b + 1])
    out.ybeg.assign((size_t)nprob + 1, 0);
    for (int b = 0; b < nprob; ++b) {
        out.ybeg[(size_t)b] = (int)out.yq.size();
        for (G2Task tk : yq[(size_t)b]) {
            tk.pid = b;
            out.yq.push_back(tk);
        }
    }
    out.ybeg[(size_t)nprob] = (int)out.yq.size();
}

cudaError_t run_potrf_dag_batch(const ProbDev* d_probs, int nprob, const G2Task* prio, long long n_prio,
                                const G2Task* bulk, long long n_bulk, const int4* tct, long long n_tct, int per,
                                const G2Task* yq, long long n_y, double* out, long long* done_ns,
                                int* counters, size_t counter_bytes, void* trace, long long trace_cap,
                                bool small_dp, long long wait_ns, int ctas, cudaStream_t s) {
    int nsm = 0;
    cudaError_t e = small_dp ? dag_prepare<true>(nsm) : dag_prepare<false>(nsm);
    if (e) return e;
    if ((e = cudaMemsetAsync(counters, 0, counter_bytes, s))) return e;
    // results start as NaN (every byte 0xFF): a problem whose factorization
    // fails never reaches its last solve task and keeps them
    if ((e = cudaMemsetAsync(out, 0xFF, 3 * sizeof(double) * (size_t)nprob, s))) return e;
    if (done_ns && (e = cudaMemsetAsync(done_ns, 0, sizeof(long long) * ((size_t)nprob + 1), s))) return e;
    DagArgs A;
    memset(&A, 0, sizeof(A));
    A.probs = d_probs;
    A.prio = prio;
    A.bulk = bulk;
    A.n_prio = n_prio;
    A.n_bulk = n_bulk;
    A.tct = tct;
    A.per = per;
    A.n_tc_items = n_tct * (long long)per;
    A.ctr = counters;
    A.trace_ctr = (unsigned long long*)trace;
    A.trace = trace ? (geo_trace_rec*)((char*)trace + 64) : nullptr;
    A.trace_cap = trace_cap;
    A.wait_ns = wait_ns > 0 ? wait_ns : GEO_DEFAULT_TIMEOUT_NS;
    A.yq = yq;
    A.n_y = n_y;
    A.nprob = nprob;
    A.out = out;
    A.done_ns = done_ns;
    CUtensorMap maps[3];
    memset(maps, 0, sizeof(maps));   // unused: each problem's maps are in its view
    void* args[] = {&A, &maps[0], &maps[1], &maps[2]};
    const void* fn = small_dp ? (const void*)dag_kernel<true> : (const void*)dag_kernel<false>;
    prof_begin(4, s);
    if (ctas > 0 && ctas < nsm) {
        // a share of the SMs: a plain launch, so that launches on other streams
        // run beside it.  The schedule needs no co-residency: with at least
        // GEO_MIN_CTAS workers (the caller's check) every wait is on a task a
        // running worker holds or can take.
        e = cudaLaunchKernel(fn, dim3(ctas), dim3(DAG_THREADS), args, DAG_DYN_SMEM, s);
    } else {
        e = cudaLaunchCooperativeKernel(fn, dim3(nsm), dim3(DAG_THREADS), args, DAG_DYN_SMEM, s);
    }
    prof_end(4, s);
    count_launch();
    return e;
}

}  // namespace geo
