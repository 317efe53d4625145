// Host-side helpers of the C-ABI shared by its translation units (api.cu,
// batch_api.cu): error reporting, allocation, plans and the building blocks
// that enqueue kernels on a context.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "context.h"
#include "device.h"

using namespace pavg;
using pavg_detail::AvgPlan;
using pavg_detail::EventPair;
using pavg_detail::SharedMesh;

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return set_err(ctx, PAVG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Counts one of this library's kernels and checks its launch.
#define KL(call)          \
  do {                    \
    ++ctx->launches;      \
    CK(call);             \
  } while (0)

namespace pavg_api {

int set_err(pavg_ctx* c, int code, const std::string& msg);

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
}

template <class T>
cudaError_t upload(T** p, const std::vector<T>& v) {
  cudaError_t e = dalloc(p, v.size());
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
}

// out = N(U) (weak form, mass solves), with scratch for the right-hand side.
int enq_nonlinear(pavg_ctx* ctx, const double* U, double* out, double* scratch, cudaStream_t st);
// Workspace of the shared-basis average for degree K and M shifts.
int ensure_avg_workspace(pavg_ctx* ctx, int K, int M);
// Shifts, weights, coefficient tables of (T, M), cached on the context; with
// 0 <= m0 < m1 <= M only the shifts m0 .. m1-1 of the M-point rule (their
// weights normalised over all M), m1 < 0 meaning M.
int get_plan(pavg_ctx* ctx, double T, int M, AvgPlan** out, int m0 = 0, int m1 = -1);
// Middle of the shared-basis average: U_m = sum_k A[m][k] Q_k, r_m = N(U_m)
// (weak form), y_k = sum_m B[k][m] r_m written over Q_k.
int enq_avg_shifts(pavg_ctx* ctx, const AvgPlan& pl, cudaStream_t st);
// The whole shared-basis average on `st` (no graph): U -> out.
int enq_avg(pavg_ctx* ctx, const AvgPlan& pl, const double* U, double* out, cudaStream_t st);
// Energy inner product <U, V>_W = H u^T M1 v + g eta^T M2 zeta (synchronous, legacy stream).
double host_winner(pavg_ctx* ctx, const double* U, const double* V);
// The shared-basis average through the context's cached graph.
int run_avg(pavg_ctx* ctx, double T, int M, const double* U, double* out, cudaStream_t st, int m0 = 0,
            int m1 = -1);
// Error flags latched on the device, as a return code.
int check_flags(pavg_ctx* ctx);

}  // namespace pavg_api
