// Measurement helper of the benchmark, not part of the library's C ABI:
// arithmetic throughput of this GPU, for the rooflines of the ALU-bound
// kernels -- packed FP32x2 fused multiply-adds (FFMA2, the FP32 step's
// arithmetic) and FP64 fused multiply-adds, each thread running eight
// independent chains so that the pipes stay full.  Built into its own
// library (libpclb_bench.so), loaded only by the benchmark and its test.
// Returns 0 on success, 1 for a NULL output, 3 on a CUDA error; the call
// synchronizes its stream and allocates nothing.
#include <cuda_runtime.h>

#include "f32x2.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kIters = 4096;
__device__ double g_alu_sink[2];

__global__ void __launch_bounds__(kThreads) ffma2_chains(float seed) {
  using namespace pclb;
  f2 acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = make_float2(seed + c, seed - c);
  const f2 m = make_float2(0.999f, 1.001f), a = make_float2(1e-3f, -1e-3f);
#pragma unroll 1
  for (int i = 0; i < kIters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = fma2(acc[c], m, a);
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c].x + acc[c].y;
  if (s == 12345.678f) g_alu_sink[0] = s;   // never true: keeps the chains live
}

__global__ void __launch_bounds__(kThreads) dfma_chains(double seed) {
  double acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = seed + c;
#pragma unroll 1
  for (int i = 0; i < kIters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], 0.999999, 1e-6);
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  if (s == 12345.678) g_alu_sink[1] = s;
}

}  // namespace

extern "C" int bench_alu_peaks(void* stream, double* out) {
  if (!out) return 1;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 3;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return 3;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return 3;
  }
  const int blocks = 8 * n_sm;   // 8 CTAs of 256 threads per SM
  const double threads = (double)blocks * kThreads;
  int st = 0;
  for (int k = 0; k < 2 && st == 0; ++k) {
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {   // the first launch warms up
      cudaEventRecord(e0, s);
      if (k == 0)
        ffma2_chains<<<blocks, kThreads, 0, s>>>(1.0f + rep);
      else
        dfma_chains<<<blocks, kThreads, 0, s>>>(1.0 + rep);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        st = 3;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < best) best = ms;
    }
    // FP32x2: two multiply-adds (4 flops) per instruction; FP64: one (2 flops)
    const double flops = threads * kIters * kChains * (k == 0 ? 4.0 : 2.0);
    out[k] = flops / (best * 1e-3) / 1e12;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}
