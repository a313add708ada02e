// Throughput probe for the roofline denominators this library reports against:
// FP64 DFMA, FP64 DMMA (mma.sync m8n8k4) and FP32 FFMA, each a bounded loop of
// independent FMA chains; and the latency of dependent chains of FP64 FMA,
// rsqrt, division, log and FP64 -> FP32 conversion in one warp (clock64), the
// costs that bound a factorization's critical path when FP64 is slow.
// Build: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o probe fp64_peak_probe.cu
#include <cstdio>
#include <cuda_runtime.h>
#define ITERS 4096
__global__ void dfma_k(double* out, double a, double b) {
  double x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3, x4=x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for (int i = 0; i < ITERS; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0+x1+x2+x3+x4+x5+x6+x7;
}
__global__ void ffma_k(float* out, float a, float b) {
  float x[16];
#pragma unroll
  for (int u = 0; u < 16; ++u) x[u] = threadIdx.x + u;
  for (int i = 0; i < ITERS; ++i) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int u = 0; u < 16; ++u) x[u] = fmaf(x[u], a, b);
  }
  float s = 0; for (int u = 0; u < 16; ++u) s += x[u];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void dmma_k(double* out, double a) {
  double acc[4][2];
  for (int c = 0; c < 4; ++c) { acc[c][0] = 0; acc[c][1] = 0; }
  double fa = a + threadIdx.x, fb = a - threadIdx.x;
  for (int i = 0; i < ITERS / 4; ++i) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(acc[c][0]), "+d"(acc[c][1]) : "d"(fa), "d"(fb));
  }
  double s = 0; for (int c = 0; c < 4; ++c) s += acc[c][0] + acc[c][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
// one warp, `active` lanes, a dependent chain of n operations of one kind
__global__ void chain_k(double* out, long long* cyc, int n, int active, int mode) {
  const int lane = threadIdx.x;
  double a = 1.0 + lane * 1e-3;
  const double b = 0.999999, c = 1e-7;
  float fa = 1.0f + lane * 1e-3f;
  __syncwarp();
  const long long t0 = clock64();
  if (lane < active) {
    if (mode == 0) { for (int i = 0; i < n; ++i) a = fma(a, b, c); }
    else if (mode == 1) { for (int i = 0; i < n; ++i) a = rsqrt(a) + 0.5; }
    else if (mode == 2) { for (int i = 0; i < n; ++i) fa = fmaf(fa, 0.999999f, 1e-7f); a = fa; }
    else if (mode == 3) { for (int i = 0; i < n; ++i) a = 1.0 / a + 0.25; }
    else if (mode == 4) { for (int i = 0; i < n; ++i) a = (double)(float)a * b; }
    else { for (int i = 0; i < n; ++i) a = log(a) + 1.5; }
  }
  __syncwarp();
  const long long t1 = clock64();
  out[lane] = a;
  if (lane == 0) *cyc = t1 - t0;
}

int main() {
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  int clk; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  printf("SMs %d clock(kHz) %d\n", sms, clk);
  double* d; float* f; cudaMalloc(&d, sizeof(double) * sms * 8 * 1024); cudaMalloc(&f, sizeof(float) * sms * 8 * 1024);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1); float ms;
  for (int blocksPerSM : {2, 4, 8}) {
    int grid = sms * blocksPerSM, thr = 256;
    dfma_k<<<grid, thr>>>(d, 1.0000001, 1e-9);
    cudaEventRecord(e0); dfma_k<<<grid, thr>>>(d, 1.0000001, 1e-9); cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    double flops = 2.0 * 8 * 4 * (double)ITERS * grid * thr;
    printf("DFMA bps=%d: %.3f ms  %.3f TFLOP/s\n", blocksPerSM, ms, flops / ms / 1e9);
    dmma_k<<<grid, thr>>>(d, 1.0);
    cudaEventRecord(e0); dmma_k<<<grid, thr>>>(d, 1.0); cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    flops = 2.0 * 8 * 8 * 4 * 4 * (double)(ITERS / 4) * grid * (thr / 32);
    printf("DMMA bps=%d: %.3f ms  %.3f TFLOP/s\n", blocksPerSM, ms, flops / ms / 1e9);
    ffma_k<<<grid, thr>>>(f, 1.0000001f, 1e-9f);
    cudaEventRecord(e0); ffma_k<<<grid, thr>>>(f, 1.0000001f, 1e-9f); cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    flops = 2.0 * 16 * 4 * (double)ITERS * grid * thr;
    printf("FFMA bps=%d: %.3f ms  %.3f TFLOP/s\n", blocksPerSM, ms, flops / ms / 1e9);
  }
  long long* cyc; cudaMalloc(&cyc, sizeof(long long));
  const char* names[] = {"dfma", "drsqrt + dadd", "ffma", "ddiv + dadd", "f2f.f32.f64 + dmul", "dlog + dadd"};
  for (int mode = 0; mode < 6; ++mode)
    for (int active : {32, 1}) {
      chain_k<<<1, 32>>>(d, cyc, 256, active, mode);
      chain_k<<<1, 32>>>(d, cyc, 256, active, mode);
      long long h = 0; cudaMemcpy(&h, cyc, sizeof(h), cudaMemcpyDeviceToHost);
      printf("latency %-20s lanes=%2d: %.1f cycles per step\n", names[mode], active, (double)h / 256);
    }
  cudaError_t err = cudaDeviceSynchronize();
  printf("status %s\n", cudaGetErrorString(err));
  return err != cudaSuccess;
}
