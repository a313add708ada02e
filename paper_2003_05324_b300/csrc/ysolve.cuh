// A10-A11 building blocks shared by the standalone forward-solve kernels
// (solve.cu) and the solve tasks of the persistent factorization (dag.cu).
//
// The forward solve y = L^-1 Z of Eq. 2 runs by tile rows: the diagonal tile
// solve L_ii y_i = r_i, and the updates r_l -= L(l,i) y_i of the later block
// rows.  Per element the arithmetic and its order are fixed here and do not
// depend on the number of threads that run them, so the standalone kernels,
// the batched solve and the tasks fused into the factorization all give the
// same bits.
#pragma once
#include "geo_internal.cuh"

namespace geo {

constexpr int YS_BS = 32;      // column block of the diagonal solve
constexpr int YS_MAX_NB = 768; // largest tile the layout accepts

struct YSolveSmem {
    double Db[YS_BS * (YS_BS + 1)];   // 32 x 32 diagonal block of L_ii
    double ys[YS_BS];                 // its solved values
    double rinv[YS_BS];               // reciprocal pivots
    double lg[YS_MAX_NB];             // log L_aa of the tile
};

// Solve L_ii y_i = r_i in place (y_i holds r_i on entry) with threads
// tid = 0..nt-1 (nt a multiple of 32, at least 32) synchronised by sync(); write
// part[2i] = 2 sum_a log L_aa and part[2i+1] = sum_a y_a^2 of the tile.
//   * column blocks of 32: warp 0 solves the block by substitution (one column
//     at a time, shuffles), then each later row r subtracts its 32 products in
//     column order (one thread per row);
//   * the two sums: lane l of warp 0 adds the terms a = l, l + 32, ... in
//     order, then a fixed shuffle tree.
template <typename Sync>
__device__ void ysolve_diag_tile(const Layout& L, int i, double* __restrict__ yv, double* __restrict__ part,
                                 int tid, int nt, YSolveSmem& S, Sync sync) {
    const int nb = L.nb, lane = tid & 31, warp = tid >> 5;
    const double* A = dp_tile(L, i, i);
    double* y = yv + (size_t)i * nb;
    for (int c0 = 0; c0 < nb; c0 += YS_BS) {
        const int w = min(YS_BS, nb - c0);
        for (int idx = tid; idx < w * w; idx += nt) {
            const int r = idx % w, c = idx / w;
            S.Db[r * (YS_BS + 1) + c] = A[(size_t)(c0 + c) * nb + c0 + r];
        }
        sync();
        if (tid < w) S.rinv[tid] = 1.0 / S.Db[tid * (YS_BS + 1) + tid];
        sync();
        if (warp == 0) {
            double v = lane < w ? y[c0 + lane] : 0.0;
            for (int c = 0; c < w; ++c) {
                const double xc = __shfl_sync(0xffffffffu, v, c) * S.rinv[c];
                if (lane == c) v = xc;
                if (lane > c && lane < w) v = fma(-S.Db[lane * (YS_BS + 1) + c], xc, v);
            }
            if (lane < w) {
                S.ys[lane] = v;
                y[c0 + lane] = v;
            }
        }
        sync();
        for (int r = c0 + w + tid; r < nb; r += nt) {
            double acc = 0.0;
            for (int c = 0; c < w; ++c) acc = fma(A[(size_t)(c0 + c) * nb + r], S.ys[c], acc);
            y[r] -= acc;
        }
        sync();
    }
    for (int a = tid; a < nb; a += nt) S.lg[a] = log(A[(size_t)a * nb + a]);
    sync();
    if (warp == 0) {
        double ld = 0.0, q = 0.0;
        for (int a = lane; a < nb; a += 32) {
            ld += S.lg[a];
            q = fma(y[a], y[a], q);
        }
        for (int o = 16; o > 0; o >>= 1) {
            ld += __shfl_down_sync(0xffffffffu, ld, o);
            q += __shfl_down_sync(0xffffffffu, q, o);
        }
        if (lane == 0) {
            part[2 * i] = 2.0 * ld;
            part[2 * i + 1] = q;
        }
    }
}

// Row r of L(l,i) y_i (yi: y_i), FP64 accumulation in column order; an FP32
// (off-band) tile is promoted exactly.
__device__ __forceinline__ double yrow_update(const Layout& L, int l, int i, int r, const double* yi) {
    const int nb = L.nb;
    double acc = 0.0;
    if (is_dp(l, i, L.band)) {
        const double* A = dp_tile(L, l, i);
        for (int c = 0; c < nb; ++c) acc = fma(A[(size_t)c * nb + r], yi[c], acc);
    } else {
        const float* A = sp_tile(L, l, i);
        for (int c = 0; c < nb; ++c) acc = fma((double)A[(size_t)c * nb + r], yi[c], acc);
    }
    return acc;
}

// log|Sigma| and Z' Sigma^-1 Z from the per-tile partials, summed in tile
// order, and (loglik != nullptr) Eq. 2 assembled from them.
__device__ __forceinline__ void ysolve_finish(const Layout& L, const double* part, double* logdet, double* quad,
                                              double* loglik = nullptr) {
    double s0 = 0.0, s1 = 0.0;
    for (int i = 0; i < L.p; ++i) {
        s0 += part[2 * i];
        s1 += part[2 * i + 1];
    }
    *logdet = s0;
    *quad = s1;
    if (loglik) *loglik = assemble_loglik(L.n, s0, s1);
}

}  // namespace geo
