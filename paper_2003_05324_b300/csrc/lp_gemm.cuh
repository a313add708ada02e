// Off-band (FP32-accurate) update of Algorithm 1 (sgemm) on the tcgen05 tensor
// cores: the FP32 panel tiles are split into three BF16 planes
// (hi = bf16(v), mid = bf16(v - hi), lo = bf16(v - hi - mid)) and
// C <- C - sum over the six pairs (hi,hi) (hi,mid) (mid,hi) (hi,lo) (lo,hi) (mid,mid)
// of A_s B_t', accumulated in FP32 in tensor memory.  The dropped pairs are of
// relative size 2^-24 and below, i.e. the result is FP32-accurate.
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
