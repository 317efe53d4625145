// Measurement aid: the GPU's FP32 and FP64 fused multiply-add rates, measured
// with a kernel of independent FMA chains timed by CUDA events.  The
// benchmark reports each ALU-bound kernel as a fraction of these measured
// rates instead of a rate derived from unit counts and clocks.
#include <cuda_runtime.h>

#include <algorithm>

#include "pavg.h"

namespace {

constexpr int kChains = 8;     // independent accumulators per thread
constexpr int kUnroll = 16;

// Every thread runs kChains independent chains a <- a * x + y, `iters` x
// kUnroll steps each; x and y come from the arguments so nothing folds at
// compile time, and the chains' sum is stored so nothing is eliminated.
template <typename T>
__global__ void k_fma_chains(T x, T y, int iters, T* sink) {
  T a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == (T)-1.2345) sink[blockIdx.x] = s;  // practically never true; keeps the chains alive
}

template <typename T>
int measure(double* tflops, cudaStream_t st) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PAVG_ERR_CUDA;
  const int threads = 512;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<T>, threads, 0) != cudaSuccess ||
      per_sm < 1)
    return PAVG_ERR_CUDA;
  const int blocks = sms * per_sm;
  const int iters = sizeof(T) == 8 ? 64 : 256;  // a few ms per launch either way
  T* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = PAVG_OK;
  if (cudaMalloc(&sink, sizeof(T) * blocks) != cudaSuccess) return PAVG_ERR_NOMEM;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = PAVG_ERR_CUDA;
  double best = 0.0;
  for (int rep = 0; rep < 6 && rc == PAVG_OK; ++rep) {  // the first launch warms up
    cudaEventRecord(e0, st);
    k_fma_chains<T><<<blocks, threads, 0, st>>>((T)0.999999, (T)1e-7, iters, sink);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) { rc = PAVG_ERR_CUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flop = 2.0 * (double)blocks * threads * kChains * kUnroll * (double)iters;
    if (rep > 0 && ms > 0.f) best = std::max(best, flop / (ms * 1e-3) / 1e12);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (rc == PAVG_OK) *tflops = best;
  return rc;
}

}  // namespace

extern "C" int pavg_measure_fma_peak(int fp64, double* tflops, void* stream) {
  if (!tflops) return PAVG_ERR_INVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return fp64 ? measure<double>(tflops, st) : measure<float>(tflops, st);
}
