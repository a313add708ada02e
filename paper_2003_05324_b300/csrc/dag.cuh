// Persistent tile-DAG scheduler of Algorithm 1 (see dag.cu): task records,
// queue geometry and the host entry point.
#pragma once
#include <cuda.h>

#include <vector>

#include "geo_internal.cuh"

namespace geo {

// (type 0 is unused: the sub-block factors run inside PC)
enum TaskType : int { T_PT = 1, T_PU = 2, T_TRSM = 3, T_UPD = 4, T_YD = 5, T_YG = 6, T_PC = 7, T_PC2 = 8 };

// One CUDA-core task: PT(k; a = r, b = s), PU(k; a = r, b = c, c = s),
// TRSM(k; a = i, b = row chunk), UPD(k; a = i, b = j, c = 64 x 64 sub-block),
// YD(k) diagonal forward solve of block row k, YG(k; a = i, b = row chunk)
// r_i -= L(i,k) y_k, PC(k) the critical chain of dpotrf(k) and PC2(k) the
// chain one sub-block below it (see dag.cu);
// pid: the problem it belongs to (0 in a single-problem launch).
struct G2Task {
    int type, k, a, b, c, pid;
};

// FP64 panel tiles of at least this many rows are solved in 32-row tasks with
// the contraction split over the group's warps, smaller ones one row per thread
constexpr int DP_SPLIT_MIN_NB = 256;
inline bool dag_small_dp(int nb, int band) { return nb < DP_SPLIT_MIN_NB && band > 1; }

struct SchedGeom {
    int p, ex, dst, ns, nsb64, items64, items_tc, max_items, chunks_dp, chunks_sp, chunks_y;
    long long n_counters, n_g2, n_prio, n_bulk, n_tct, n_y;
};

// Device view of the scheduler's tables inside the meta buffer.
struct SchedView {
    SchedGeom geom;
    int* counters;       // zeroed before each factorization
    const G2Task* prio;  // CUDA-core priority queue, in order
    const G2Task* bulk;  // CUDA-core bulk queue, in order
    const int* trsm_end; // [p] priority index past A(k)'s solves
    const int4* tct;     // tensor queue targets (i, j, k), in order
    const G2Task* yq;    // forward-solve queue Y(0) Y(1) ..., in order
};

// Device view of one problem of a launch: its layout, queue geometry, its
// dependency counters, the priority-queue index past each step's solves,
// (batched launches) its three tensor maps in global memory, and Z for the
// forward solve fused into the factorization (nullptr: factor only).
struct ProbDev {
    Layout L;
    SchedGeom g;
    int *upd, *tcnt, *pot, *sub, *ycnt, *ydone, *yhead;
    int y0, y1;    // its forward-solve tasks: yq[y0 .. y1)
    const double* z;
    double* res;   // (log|Sigma|, Z' Sigma^-1 Z, Eq. 2) of the fused solve
    const int* trsm_end;
    const CUtensorMap* tmap;
};

// ex: in-band (FP64) updates as FP64-accurate tensor-core items instead of
// CUDA-core DMMA items
// ex: in-band updates on the tensor cores; dst: the DST approximation (tiles
// at i - j >= band are zero and get no tasks)
SchedGeom sched_geom(int p, int nb, int band, int pp, bool ex, bool dst = false);
// yq: the forward-solve queue (claimed only when its head is ready)
void sched_build(const SchedGeom& g, int band, std::vector<G2Task>& prio, std::vector<G2Task>& bulk,
                 std::vector<int>& trsm_end, std::vector<G2Task>& yq, std::vector<int4>& tct);
// z: Z for the fused forward solve (log-det, quadratic form and Eq. 2 into
// res[0..2]), or nullptr to factor only
cudaError_t run_potrf_dag(const geo_tiles* t, const Layout& L, const SchedView& sv, const double* z, double* res,
                          cudaStream_t s);

// Batched generation: problem b's coordinates and the index of its first CTA
// in the one generator launch of a batch (block0 increasing, from 0).
struct GenJob {
    const double* x;
    const double* y;
    long long block0;
};
// CTAs of one problem's generation (column chunks x lower tiles).
long long gen_blocks(const Layout& L);
// Generate every problem's tiles (theta of problem b from dth[b], device
// memory) in one launch of total_blocks CTAs; also clears each problem's
// status words.
cudaError_t launch_matern_batch(const ProbDev* d_probs, const GenJob* d_jobs, int nprob, long long total_blocks,
                                const geo_theta* dth, cudaStream_t s);

// Batched launch: every problem's tasks in one persistent kernel.  The host
// merges the problems' queues step by step (each problem keeps its own
// topological order, so the merge is one too).
struct BatchPlan {
    std::vector<G2Task> prio, bulk, yq;   // yq: the problems' forward-solve queues, one segment each
    std::vector<int> ybeg;                // problem b's segment: yq[ybeg[b] .. ybeg[b + 1])
    std::vector<int4> tct;            // (i, j, k, problem)
    std::vector<std::vector<int>> trsm_end;
    int per = 1;                      // tensor items per target (largest over the problems)
};
void sched_merge(const std::vector<SchedGeom>& g, const std::vector<int>& band, BatchPlan& out);
// point P's counters into a block of P.g.n_counters - 16 ints
void bind_counters(ProbDev& P, int* base);
// probs: nprob device views in global memory (their counters inside `counters`,
// zeroed by this call), queues in device memory as laid out by the caller; the
// forward solve of every problem runs inside the launch (yq) and writes its
// (l, log|Sigma|, Z' Sigma^-1 Z) to out[3b] (NaN if it fails) and, with
// done_ns, [0] the launch start and [1 + b] its completion (%globaltimer).
// small_dp: some problem has FP64 panel tiles (band > 1) of fewer than
// DP_SPLIT_MIN_NB rows (dag_small_dp), solved one row per thread.
// ctas: 0 = one CTA per SM (cooperative launch), else a plain launch of that
// many CTAs (a share of the SMs; launches on other streams run beside it).
cudaError_t run_potrf_dag_batch(const ProbDev* d_probs, int nprob, const G2Task* prio, long long n_prio,
                                const G2Task* bulk, long long n_bulk, const int4* tct, long long n_tct, int per,
                                const G2Task* yq, long long n_y, double* out, long long* done_ns,
                                int* counters, size_t counter_bytes, void* trace, long long trace_cap,
                                bool small_dp, long long wait_ns, int ctas, cudaStream_t s);

}  // namespace geo
