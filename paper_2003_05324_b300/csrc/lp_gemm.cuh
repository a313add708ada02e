// Off-band (FP32-accurate) update of Algorithm 1 (sgemm) on the tcgen05 tensor
// cores, step-by-step path (GEO_FLAG_STEPWISE).  Each panel row is scaled by a
// power of two 2^E (|v| 2^-E < 1/2) and cut into rounded 8-bit integer slices
// a0, a1, ... (|a_s| <= 128; the split writes seven, this update reads the
// first four), stored exactly in BF16 as P_s = a_s 2^-8s, so that
// v = 2^(E-8) (P0 + P1 + P2 + P3) to 2^-33 of the row's scale.  Then
//   C <- C - 2^(E_r+E_c-16) [ P0 P0' + sum over the nine pairs (a, b), 1 <= a + b <= 3, of Pa Pb' ].
// P0 P0' is a sum of integers below 2^23 for K <= 1024, so the tensor cores
// accumulate it exactly (their FP32 accumulation truncates; exact sums make that
// moot); the other pairs, 2^-8 and more smaller, go to a second accumulator.
// The dropped pairs weigh 2^-32 of the leading one: the update is FP32-accurate
// and free of the accumulation bias a single truncating accumulator would add.
#pragma once
#include "geo_internal.cuh"

namespace geo {

// Write the BF16 slice planes of every panel tile (i, k), i > k.
cudaError_t launch_split_panel(const Layout& L, int k, cudaStream_t s);

// Encode the TMA descriptor of the bound planes buffer into t->tmap (host).
// Returns 0 on success.
int prepare_lp_gemm(geo_tiles* t, const Layout& L);

// C(i,j) -= A(i,k) A(j,k)' for the nlp off-band targets of step k.
cudaError_t launch_lp_gemm_tc(const geo_tiles* t, const Layout& L, int k, int nlp, cudaStream_t s);

}  // namespace geo
