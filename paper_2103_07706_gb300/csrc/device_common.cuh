// Device helpers shared by the kernel translation units: DOF gathering,
// element SpMV, deterministic block reductions and the bounded grid barrier.
#pragma once

#include <cuda_runtime.h>

#include "device.h"

namespace pavg {
namespace {

constexpr long long kBarrierTimeoutCycles = 4000000000LL;  // ~2 s at 2 GHz

__host__ __device__ constexpr int psym(int i, int j) { return i * 12 - i * (i - 1) / 2 + (j - i); }
__host__ __device__ constexpr int pasym(int i, int j) { return i * 11 - i * (i - 1) / 2 + (j - i - 1); }

// Global DOF indices and orientation signs of the 12 velocity DOFs of cell c.
__device__ __forceinline__ unsigned cell_dofs(const DeviceMesh& m, int64_t c, int dof[12], double sg[12]) {
  unsigned al = m.cell_aligned[c];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    int e = m.cell_edges[i * m.F + c];
    bool a = (al >> i) & 1u;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      dof[3 * i + j] = 3 * e + j;
      sg[3 * i + j] = (a || j == 1) ? 1.0 : -1.0;
    }
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    dof[9 + j] = (int)(3 * m.E + 3 * c + j);
    sg[9 + j] = 1.0;
  }
  return al;
}

// w = A_K u for the cell's packed symmetric 12x12 element matrix.
__device__ __forceinline__ void spmv_cell(const double* __restrict__ M1, int64_t F, int64_t c,
                                          const double u[12], double w[12]) {
#pragma unroll
  for (int i = 0; i < 12; ++i) w[i] = 0.0;
#pragma unroll
  for (int i = 0; i < 12; ++i) {
#pragma unroll
    for (int j = i; j < 12; ++j) {
      double a = __ldg(&M1[psym(i, j) * F + c]);
      w[i] = fma(a, u[j], w[i]);
      if (j != i) w[j] = fma(a, u[i], w[j]);
    }
  }
}

template <int THREADS>
__device__ __forceinline__ void block_sum3(double a, double b, double c, double out[3]) {
  __shared__ double sh[3][THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  if (lane == 0) { sh[0][warp] = a; sh[1][warp] = b; sh[2][warp] = c; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0, s2 = 0;
    for (int k = 0; k < THREADS / 32; ++k) { s0 += sh[0][k]; s1 += sh[1][k]; s2 += sh[2][k]; }
    out[0] = s0; out[1] = s1; out[2] = s2;
  }
  __syncthreads();
}

// Sense-reversing grid barrier with a bounded wait.  Returns false (and latches
// kFlagTimeout) when the wait gives up or another block already timed out.
__device__ bool grid_barrier(unsigned* bar, int* flags) {
  __shared__ int s_ok;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    unsigned gen = *vgen;
    __threadfence();
    unsigned arrived = atomicAdd(bar, 1u);
    int ok = 1;
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long t0 = clock64();
      while (*vgen == gen) {
        if (clock64() - t0 > kBarrierTimeoutCycles) {
          atomicOr(flags, kFlagTimeout);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    if (*((volatile int*)flags) & kFlagTimeout) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Deterministic sum of the per-block partials [3][nb] by every block.
template <int THREADS>
__device__ __forceinline__ void reduce_partials(const double* part, int nb, double out[3]) {
  double a = 0, b = 0, c = 0;
  for (int k = threadIdx.x; k < nb; k += THREADS) {
    a += __ldcg(&part[k]);
    b += __ldcg(&part[nb + k]);
    c += __ldcg(&part[2 * nb + k]);
  }
  block_sum3<THREADS>(a, b, c, out);
}
}  // namespace
}  // namespace pavg
