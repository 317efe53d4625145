// Mixed-precision solver for the velocity mass matrix M1 (FP64-accurate),
// one problem per launch: the persistent cooperative kernel k_cg_ir runs every
// refinement sweep of one solve.  The solver itself (FP32 block-Jacobi CG
// inside FP64 residual refinement) is in cg_ir.cuh.  When the mesh allows,
// the block's FP32 element matrices stay in shared memory for the whole
// solve (up to about 540 cells per SM: the refinement-6 mesh).
#include <cuda_runtime.h>

#include "cg_ir.cuh"
#include "device.h"

namespace pavg {
namespace {

constexpr int kIrThreads = 256;  // 64 cells x 4 triples
constexpr int kIrCells = kIrThreads / 4;

template <bool RES>
__global__ void __launch_bounds__(kIrThreads, 3) k_cg_ir(DeviceMesh m, CgIrWork w, CgIrParams cp,
                                                         const double* __restrict__ b, double* out, double scale_x,
                                                         const double* __restrict__ add) {
  extern __shared__ float s_mat[];  // [passes][64][kMatStride] when RES, then [passes][256] triples
  int* s_tri = reinterpret_cast<int*>(s_mat + (size_t)w.passes * kIrCells * kMatStride);
  const int nb = gridDim.x, bid = blockIdx.x;
  if (RES) cg_load_resident<kIrThreads>(m, nb, bid, s_mat, s_tri);
  const GridSync gs = {w.partial, w.partial_f, w.scal, w.tag, w.bar, w.flags};
  unsigned epoch = 0;
  cg_solve<kIrThreads, RES>(m, w, gs, cp, b, out, scale_x, add, nb, bid, s_mat, s_tri, epoch);
}

}  // namespace

cudaError_t cg_ir_configure(int64_t F, CgIrWork* w) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t need = (F + kIrCells - 1) / kIrCells;
  // resident matrices: try 3, then 2 blocks per SM
  e = cudaFuncSetAttribute(k_cg_ir<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  for (int bps = 3; bps >= 2; --bps) {
    const int64_t nb = need < (int64_t)bps * sms ? need : (int64_t)bps * sms;
    const int64_t passes = (need + nb - 1) / nb;
    const size_t smem = sizeof(float) * (size_t)passes * kIrCells * kMatStride + sizeof(int) * (size_t)passes * kIrThreads;
    if (smem > 200 * 1024) continue;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_ir<true>, kIrThreads, smem);
    if (e != cudaSuccess) return e;
    if ((int64_t)per_sm * sms >= nb) {
      w->nblocks = (int)nb;
      w->passes = (int)passes;
      w->smem = smem;
      return cudaSuccess;
    }
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_ir<false>, kIrThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t maxb = (int64_t)per_sm * sms;
  w->nblocks = (int)(need < maxb ? need : maxb);
  w->passes = (int)((need + w->nblocks - 1) / w->nblocks);
  w->smem = 0;
  return cudaSuccess;
}

cudaError_t launch_cg_ir(const DeviceMesh& m, const CgIrWork& w, const CgIrParams& cp, const double* b,
                         double* out, double scale_x, const double* add, cudaStream_t st) {
  // zero on entry: the FP32 accumulation slots and the FP64 product on the
  // shared (edge) DOFs, and the barrier's arrival counter
  cudaError_t e = cudaSuccess;
  for (int s = 5; s <= 7 && e == cudaSuccess; ++s)
    e = cudaMemsetAsync(w.fbuf + (size_t)s * 4 * (m.E + m.F), 0, sizeof(float) * 4 * m.E, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.ax, 0, sizeof(double) * 3 * m.E, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.bar, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.tag, 0, 4 * sizeof(unsigned long long), st);  // epochs start at 1
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(w.nblocks);
  cfg.blockDim = dim3(kIrThreads);
  cfg.dynamicSmemBytes = w.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (w.smem > 0) return cudaLaunchKernelEx(&cfg, k_cg_ir<true>, m, w, cp, b, out, scale_x, add);
  return cudaLaunchKernelEx(&cfg, k_cg_ir<false>, m, w, cp, b, out, scale_x, add);
}

}  // namespace pavg
