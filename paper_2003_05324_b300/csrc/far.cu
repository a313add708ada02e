// Tile map of the far tier (three-precision extension, Section IX): which
// off-band tiles take the reduced-product updates.  A tile (i, j) is far when
// i - j >= far_band or when the bounding boxes of the two tiles' locations are
// at least far_dist apart.
#include <math.h>

#include "geo_internal.cuh"

namespace geo {

// box[4i..4i+3] = (min x, max x, min y, max y) of tile i's locations (the
// last tile may be short); one CTA per tile
__global__ void __launch_bounds__(256) far_box_kernel(Layout L, const double* __restrict__ x,
                                                      const double* __restrict__ y, double* __restrict__ box) {
    const int i = blockIdx.x, tid = threadIdx.x;
    const int r0 = i * L.nb, r1 = min(L.n, r0 + L.nb);
    double v[4] = {INFINITY, -INFINITY, INFINITY, -INFINITY};
    for (int r = r0 + tid; r < r1; r += 256) {
        v[0] = fmin(v[0], x[r]);
        v[1] = fmax(v[1], x[r]);
        v[2] = fmin(v[2], y[r]);
        v[3] = fmax(v[3], y[r]);
    }
    __shared__ double red[4][8];
    for (int o = 16; o > 0; o >>= 1) {
        v[0] = fmin(v[0], __shfl_down_sync(0xffffffffu, v[0], o));
        v[1] = fmax(v[1], __shfl_down_sync(0xffffffffu, v[1], o));
        v[2] = fmin(v[2], __shfl_down_sync(0xffffffffu, v[2], o));
        v[3] = fmax(v[3], __shfl_down_sync(0xffffffffu, v[3], o));
    }
    if ((tid & 31) == 0)
        for (int q = 0; q < 4; ++q) red[q][tid >> 5] = v[q];
    __syncthreads();
    if (tid < 4) {
        double a = red[tid][0];
        for (int w = 1; w < 8; ++w) a = (tid & 1) ? fmax(a, red[tid][w]) : fmin(a, red[tid][w]);
        box[4 * i + tid] = a;
    }
}

// one thread per tile pair (i, j) of the p x p map
__global__ void far_map_kernel(Layout L, unsigned char* __restrict__ far, int far_band, double far_dist,
                               const double* __restrict__ box) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = L.p;
    if (q >= p * p) return;
    const int i = q / p, j = q % p;
    unsigned char f = 0;
    if (i > j && !is_dp(i, j, L.band)) {
        if (far_band > 0 && i - j >= far_band) f = 1;
        if (box && far_dist > 0.0) {
            const double* bi = box + 4 * i;
            const double* bj = box + 4 * j;
            const double gx = fmax(0.0, fmax(bj[0] - bi[1], bi[0] - bj[1]));
            const double gy = fmax(0.0, fmax(bj[2] - bi[3], bi[2] - bj[3]));
            if (sqrt(gx * gx + gy * gy) >= far_dist) f = 1;
        }
    }
    far[q] = f;
}

cudaError_t launch_far_map(const Layout& L, unsigned char* far, int far_band, const double* x, const double* y,
                           double far_dist, double* scratch, cudaStream_t s) {
    const bool dist = far_dist > 0.0 && x && y;
    if (dist) {
        far_box_kernel<<<L.p, 256, 0, s>>>(L, x, y, scratch);
        count_launch();
    }
    const int np = L.p * L.p;
    far_map_kernel<<<(np + 255) / 256, 256, 0, s>>>(L, far, far_band, far_dist, dist ? scratch : nullptr);
    count_launch();
    return cudaGetLastError();
}

}  // namespace geo
