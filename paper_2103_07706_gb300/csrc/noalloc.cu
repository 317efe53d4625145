// pavg_linear_noalloc: L U for one state with no device allocation at all.
//
// Who needs it: callers that must not (or cannot) call cudaMalloc at the point
// where they apply L - code running between cudaStreamBeginCapture and
// cudaStreamEndCapture in the global capture mode (where cudaMalloc is an
// illegal, capture-invalidating call), real-time or signal-driven loops whose
// latency budget forbids the allocator, and hosts whose device memory is
// handed out by another framework's pool with a hard cap.  pavg_linear itself
// does not allocate either, but its scratch belongs to the context; this entry
// point takes all of its scratch (the assembled velocity right-hand side and
// every conjugate-gradient work vector) from one file-scope device array that
// exists from the moment the library is loaded.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "context.h"

namespace {

// Largest velocity space served: refinement 5, the paper's 20480-cell mesh
// (E = 30720 edges, n_u = 3E + 3F = 153600 DOFs).
constexpr int64_t kMaxNu = 153600;
// Per-block partial sums of the CG reductions: 2 buffers x 3 sums x blocks.
constexpr int64_t kMaxPartials = 6 * 4096;
// Layout in doubles: ru | x | r0 | r1 | s0 | s1 | w0 | w1 | w2 | p | partials | barrier words.
constexpr int64_t kScratchDoubles = 10 * kMaxNu + kMaxPartials + 8;  // about 12.5 MB

// Every GPU that loads the library holds this array until the process exits.
// In host code its name is only a host-side stand-in; the device address comes
// from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Set-up, once per device, with that device current: look the array's device
// address up.  Runs inside the first call on each device.
int scratch_for_current_device(double** out, std::string* msg) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *msg = std::string("pavg_linear_noalloc: no usable current device: ") + cudaGetErrorString(e);
    return PAVG_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      *msg = std::string("pavg_linear_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
      return PAVG_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return PAVG_OK;
}

}  // namespace

extern "C" int pavg_linear_noalloc(pavg_ctx* ctx, const double* U, double* LU, void* stream) {
  if (!ctx || !U || !LU || LU == U) return PAVG_ERR_INVAL;
  const pavg::DeviceMesh& m = ctx->dm;
  if (m.n_u > kMaxNu) {
    ctx->err = "pavg_linear_noalloc: " + std::to_string(m.n_u) + " velocity DOFs exceed the static scratch (at most " +
               std::to_string(kMaxNu) + ", refinement <= 5)";
    return PAVG_ERR_INVAL;
  }
  if (6 * (int64_t)ctx->cg.nblocks > kMaxPartials) {
    ctx->err = "pavg_linear_noalloc: CG grid larger than the static partial-sum buffer";
    return PAVG_ERR_INVAL;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != ctx->device) {
    ctx->err = "pavg_linear_noalloc: the context's device must be current";
    return PAVG_ERR_INVAL;
  }
  double* base = nullptr;
  int rc = scratch_for_current_device(&base, &ctx->err);
  if (rc) return rc;
  const int64_t nu = m.n_u;
  double* ru = base;
  pavg::CgWork w = ctx->cg;  // grid size, error flags and counters of the context
  w.x = base + 1 * nu;
  w.r[0] = base + 2 * nu;
  w.r[1] = base + 3 * nu;
  w.s[0] = base + 4 * nu;
  w.s[1] = base + 5 * nu;
  w.w[0] = base + 6 * nu;
  w.w[1] = base + 7 * nu;
  w.w[2] = base + 8 * nu;
  w.p = base + 9 * nu;
  w.partial = base + 10 * nu;
  w.bar = reinterpret_cast<unsigned*>(base + 10 * nu + kMaxPartials);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // What must start at zero is cleared on every call: the shared-edge part of
  // the assembled right-hand side here, the first accumulation buffer and the
  // barrier counter inside launch_cg.  Everything else is written before it is
  // read.  Calls that overlap on the GPU share this scratch and race.
  cudaError_t e = cudaMemsetAsync(ru, 0, sizeof(double) * 3 * m.E, st);
  if (e == cudaSuccess)
    e = pavg::launch_apply_K(m, U, 1.0, ctx->p.g, ctx->p.H, nullptr, nullptr, nullptr, ru, LU + nu, st);
  if (e == cudaSuccess) e = pavg::launch_cg(m, w, ctx->cgp, ru, LU, 1.0, nullptr, st);
  if (e != cudaSuccess) {
    ctx->err = std::string("pavg_linear_noalloc: ") + cudaGetErrorString(e);
    return PAVG_ERR_CUDA;
  }
  return PAVG_OK;
}
