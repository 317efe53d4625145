// Device-side data of one context and the host wrappers that launch kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "pavg_internal.h"

namespace pavg {

enum : int { kFlagNoConv = 1, kFlagTimeout = 2, kFlagNonFinite = 4 };

struct DeviceMesh {
  int64_t F = 0, E = 0, n_u = 0, n_eta = 0, n = 0;
  int32_t* cell_edges = nullptr;    // [3][F]
  uint8_t* cell_aligned = nullptr;  // [F]
  int32_t* edge_plus = nullptr;     // [E]
  int32_t* edge_minus = nullptr;    // [E]
  uint8_t* edge_lpos = nullptr;     // [E]
  double* M1 = nullptr;             // [78][F]
  double* C = nullptr;              // [66][F]
  double* det = nullptr;            // [F]
  double* G = nullptr;              // [3][F]
  double* dinv = nullptr;           // [n_u]
  double* topo = nullptr;           // [n_eta] topography b
};

// Scratch of the persistent CG solver.
struct CgWork {
  double* x = nullptr;        // [n_u]
  double* r[2] = {nullptr, nullptr};
  double* s[2] = {nullptr, nullptr};
  double* w[3] = {nullptr, nullptr, nullptr};
  double* p = nullptr;
  double* partial = nullptr;  // [2][3][nblocks] (double-buffered)
  unsigned* bar = nullptr;    // [2]: arrival counter, generation
  int* flags = nullptr;       // latched error flags
  unsigned long long* stats = nullptr;  // [0] solves, [1] iterations, [2] max iterations
  int nblocks = 0;
  int threads = 0;
};

struct CgParams {
  double rtol;
  int maxit;
};

// Upload constant tables (reference element data) to the current device.
cudaError_t upload_tables(const ConstTables& t);

// Grid size for the persistent CG kernel (all blocks co-resident).
cudaError_t cg_configure(int64_t F, CgWork* w);

// out_u = scale_x * M1^{-1} b + add (add may be null); all [n_u].
cudaError_t launch_cg(const DeviceMesh& m, const CgWork& w, const CgParams& cp, const double* b,
                      double* out, double scale_x, const double* add, cudaStream_t st);

// Linear-operator application of the recurrences (Sec. 2.5 weak forms):
//   ru  = y_u + s (-C u + g D^T eta)          (assembled weak-form velocity rhs)
//   eta_out = M2^{-1} (y_eta + s (-H D u)) + z_eta
// y_u, y_eta, z_eta may be null (zero).  ru must be zeroed on the edge DOFs
// (the first 3E entries) before the call.
cudaError_t launch_apply_K(const DeviceMesh& m, const double* U, double s, double g, double H,
                           const double* y_u, const double* y_eta, const double* z_eta,
                           double* ru, double* eta_out, cudaStream_t st);

// Weak-form right-hand side of N for B states [B][n] -> r [B][n]
// (r's velocity edge DOFs must be zeroed first).
cudaError_t launch_nonlinear_rhs(const DeviceMesh& m, const double* U, double* r, int B,
                                 int upwind, cudaStream_t st);

// eta_out = M2^{-1} r_eta (+ add) for B blocks of n_eta with strides.
cudaError_t launch_m2inv(const DeviceMesh& m, const double* r, int64_t rstride, double* out,
                         int64_t ostride, int B, cudaStream_t st);

// out[m][j] = sum_k A[m][k] in[k][j] (+ beta out[m][j] when accumulate), j < len.
// A is [Mo][Ki] in device memory.
cudaError_t launch_combine(const double* A, int Mo, int Ki, const double* in, int64_t in_stride,
                           double* out, int64_t out_stride, int64_t len, cudaStream_t st);

// out = a x + b y (+ c z); any of y, z may be null.
cudaError_t launch_lincomb(double* out, double a, const double* x, double b, const double* y,
                           double c, const double* z, int64_t len, cudaStream_t st);

// Energy inner products <U, V>_W = H u^T M1 v + g eta^T M2 zeta, per block partials
// written to part (size >= nblocks returned).  Host sums them.
cudaError_t launch_winner(const DeviceMesh& m, const double* U, const double* V, double g, double H,
                          double* part, int* nblocks, cudaStream_t st);

// Sets kFlagNonFinite when any entry of x is not finite.
cudaError_t launch_check_finite(const double* x, int64_t len, int* flags, cudaStream_t st);

}  // namespace pavg
