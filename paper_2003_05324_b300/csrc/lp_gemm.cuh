// Off-band (FP32-accurate) update of Algorithm 1 (sgemm) on the tcgen05 tensor
// cores.  Each FP32 panel row is scaled by a power of two 2^E (|v| 2^-E < 1/2)
// and cut into three rounded 8-bit integer slices a0, a1, a2 (|a_s| <= 128),
// stored exactly in BF16 as P0 = a0, P1 = a1 2^-8, P2 = a2 2^-16, so that
// v = 2^(E-8) (P0 + P1 + P2) to 2^-25 of the row's scale.  Then
//   C <- C - 2^(E_r+E_c-16) [ sum P0 P0'  +  sum (P1P1' + P0P2' + P2P0' + P0P1' + P1P0') ].
// The first sum is of integers below 2^23 for K <= 1024, so the tensor cores
// accumulate it exactly (their FP32 accumulation truncates; exact sums make that
// moot); the second, 2^-8 smaller, goes to its own accumulator.  The dropped
// pairs weigh 2^-24 of the leading one: the update is FP32-accurate and free of
// the accumulation bias a single truncating accumulator would add.
#pragma once
#include "geo_internal.cuh"

namespace geo {

// Write the three BF16 planes of every panel tile (i, k), i > k.
cudaError_t launch_split_panel(const Layout& L, int k, cudaStream_t s);

// Encode the TMA descriptor of the bound planes buffer into t->tmap (host).
// Returns 0 on success.
int prepare_lp_gemm(geo_tiles* t, const Layout& L);

// C(i,j) -= A(i,k) A(j,k)' for the nlp off-band targets of step k.
cudaError_t launch_lp_gemm_tc(const geo_tiles* t, const Layout& L, int k, int nlp, cudaStream_t s);

}  // namespace geo
