// FP32 FMA throughput microbenchmark: the denominator of the ALU roofline the
// render kernels are measured against (the FP32 pipe binds them; no dense
// contraction is involved).  Built as a library of its own
// (_build/libocrpeak.so), never linked into the renderer.
//
// Every thread runs kChains independent FFMA chains x <- x a + b (a just
// below one, so the values stay bounded and finite), kUnroll steps per loop
// trip; enough warps per SM and independent chains per warp cover the FMA
// latency, so the pipe issues one FFMA per lane per cycle at best.  The
// chains' sums are stored so that nothing is dead code.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fma_chains_kernel(float a, float b, int trips,
                                                              float *out) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int t = 0; t < trips; ++t) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[(size_t)blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

// Runs the kernel `reps` times (after one warm-up) on an internal stream with
// `blocks_per_sm` CTAs of 256 threads per SM and `trips` loop trips, and
// returns through *best_fma_per_s the highest FFMA instruction rate of one
// launch (lane-FMAs per second, one FMA = 2 flops), through *median_fma_per_s
// the median, and through *ms_best the duration of the fastest launch.
// Returns 0 on success, a negative CUDA error code otherwise.
extern "C" int ocr_fp32_fma_peak(int blocks_per_sm, int trips, int reps, double *best_fma_per_s,
                                 double *median_fma_per_s, float *ms_best) {
  if (blocks_per_sm < 1 || trips < 1 || reps < 1 || reps > 64 || !best_fma_per_s ||
      !median_fma_per_s || !ms_best)
    return -1;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return -(int)e;
  const int blocks = nsm * blocks_per_sm;
  float *out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms[64];
  e = cudaMalloc((void **)&out, sizeof(float) * (size_t)blocks * kThreads);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int r = -1; r < reps && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, st);
    if (e != cudaSuccess) break;
    fma_chains_kernel<<<blocks, kThreads, 0, st>>>(0.99999994f, 1e-7f, trips, out);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (r >= 0) ms[r] = t;
  }
  if (out) cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (e != cudaSuccess) return -(int)e;
  // insertion sort of the launch times
  for (int i = 1; i < reps; ++i)
    for (int j = i; j > 0 && ms[j] < ms[j - 1]; --j) {
      const float t = ms[j];
      ms[j] = ms[j - 1];
      ms[j - 1] = t;
    }
  const double fmas = (double)blocks * kThreads * (double)trips * kUnroll * kChains;
  *ms_best = ms[0];
  *best_fma_per_s = fmas / (ms[0] * 1e-3);
  *median_fma_per_s = fmas / (ms[reps / 2] * 1e-3);
  return 0;
}
