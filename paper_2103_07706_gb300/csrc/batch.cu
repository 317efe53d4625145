// Batched persistent recurrence kernel: many instances (meshes of different
// refinement, different T and M) advance their Chebyshev chains (forward
// phase shifts, Sec. 2.4) or their Clenshaw sums (backward phase shifts and
// weighted sum, Sec. 2.2) in ONE cooperative launch.  Each instance is a
// problem with its own range of blocks; a step of a problem is
//   1. the element-local application of Khat = [[-C, g D^T], [-H D, 0]]
//      (velocity part assembled by atomics into ru, elevation part through
//      the 3x3 DG1 mass inverse straight to the output),
//   2. the mixed-precision M1 solve of cg_ir.cuh on ru,
//   3. a barrier among the problem's blocks.
// A problem's blocks never wait on another problem's, so instances with short
// chains finish early and instances of different size share the GPU; the
// single-vector recurrences of all instances run concurrently.
#include <cuda_runtime.h>

#include "cg_ir.cuh"
#include "device.h"

namespace pavg {
namespace {

struct ChainTables {
  double D[3][12];
  double M2inv_ref[3][3];
};
__constant__ ChainTables c_ktab;

// Entry (k, l) of cell c's M2^{-1} on the cubic surface (packed 00, 01, 02, 11, 12, 22; [6][F]).
__device__ __forceinline__ double m2i(const DeviceMesh& m, int64_t c, int k, int l) {
  const int a = k < l ? k : l, b = k < l ? l : k;
  const int idx = a == 0 ? b : (a == 1 ? 2 + b : 5);
  return __ldg(&m.M2i[idx * m.F + c]);
}

// Step 1 on the solver's thread layout (four threads per cell, thread q of
// cell c holds DOF triple t = tri(c, q), edges q < 3, interior q = 3):
//   ru[3t+j] += y_u (owner only) + s (-C u + g D^T eta)   rows 3q+j of the cell,
//   eta_out[3c+q] = M2^{-1}(y_eta + s (-H D u)) + z_eta    (q < 3),
// or with U null only the second line without the D u term.  C is stored
// with the global orientation signs, D is the reference matrix and takes the
// signs of the cell's local-to-global map.
template <int NT, bool RES>
__device__ __forceinline__ void apply_K_phase(const DeviceMesh& m, const double* __restrict__ U, double s, double g,
                                              double H, const double* __restrict__ y_u,
                                              const double* __restrict__ y_eta, const double* __restrict__ z_eta,
                                              double* ru, double* eta_out, int nb, int bid, const int* s_tri) {
  constexpr int kCells = NT / 4;
  const int64_t F = m.F;
  const int q = threadIdx.x & 3, cl = threadIdx.x >> 2;
  int p = 0;
  for (int64_t cb = (int64_t)bid * kCells; cb < F; cb += (int64_t)nb * kCells, ++p) {
    const int64_t c = cb + cl;
    const bool active = c < F;
    bool own = false;
    int t = 0;
    unsigned al = 0;
    double uq[3] = {0.0, 0.0, 0.0}, eta[3] = {0.0, 0.0, 0.0};
    if (active) {
      t = triple<NT, RES>(m.tri, s_tri, p, c, q, own);
      al = m.cell_aligned[c];
      if (U) {
#pragma unroll
        for (int j = 0; j < 3; ++j) uq[j] = __ldcg(&U[3 * t + j]);
#pragma unroll
        for (int k = 0; k < 3; ++k) eta[k] = __ldcg(&U[m.n_u + 3 * c + k]);
      }
    }
    double ua[12];
    gather12(uq, ua);
    if (!active) continue;
    if (U) {
      // sign of local DOF i: reversed edges flip moments 0 and 2
      auto sg = [al](int i) { return (i >= 9 || ((al >> (i / 3)) & 1u) || i % 3 == 1) ? 1.0 : -1.0; };
#pragma unroll
      for (int jj = 0; jj < 3; ++jj) {
        const int i = 3 * q + jj;
        double r = 0.0;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          if (k == i) continue;
          const double a = __ldg(&m.C[(int64_t)(k > i ? pasym(i, k) : pasym(k, i)) * F + c]);
          r = k > i ? fma(-a, ua[k], r) : fma(a, ua[k], r);
        }
        double dt = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) dt = fma(c_ktab.D[k][i], eta[k], dt);
        double v = s * fma(g * sg(i), dt, r);
        if (own && y_u) v += __ldcg(&y_u[3 * t + jj]);
        if (q < 3) atomicAdd(&ru[3 * t + jj], v);
        else ru[3 * t + jj] = v;
      }
      if (q < 3) {
        double rl[3];
#pragma unroll
        for (int l = 0; l < 3; ++l) {
          double du = 0.0;
#pragma unroll
          for (int i = 0; i < 12; ++i) du = fma(c_ktab.D[l][i] * sg(i), ua[i], du);
          rl[l] = s * (-H * du);
          if (y_eta) rl[l] += __ldcg(&y_eta[3 * c + l]);
        }
        double v = 0.0;
        if (m.M2i) {  // cubic cells: the cell's own M2^{-1}
#pragma unroll
          for (int l = 0; l < 3; ++l) v = fma(m2i(m, c, q, l), rl[l], v);
        } else {
#pragma unroll
          for (int l = 0; l < 3; ++l) v = fma(c_ktab.M2inv_ref[q][l], rl[l], v);
          v *= 1.0 / m.det[c];
        }
        if (z_eta) v += __ldcg(&z_eta[3 * c + q]);
        eta_out[3 * c + q] = v;
      }
    } else if (q < 3) {
      double v = 0.0;
      if (m.M2i) {
#pragma unroll
        for (int l = 0; l < 3; ++l) v = fma(m2i(m, c, q, l), __ldcg(&y_eta[3 * c + l]), v);
      } else {
#pragma unroll
        for (int l = 0; l < 3; ++l) v = fma(c_ktab.M2inv_ref[q][l], __ldcg(&y_eta[3 * c + l]), v);
        v *= 1.0 / m.det[c];
      }
      if (z_eta) v += __ldcg(&z_eta[3 * c + q]);
      eta_out[3 * c + q] = v;
    }
  }
}

// Zeroes, on the edge triples this block owns: ru (when not null) and, when
// `solver` is set, the solver's accumulation slots 5-7 and its FP64 product.
template <int NT, bool RES>
__device__ __forceinline__ void zero_owned_edges(const DeviceMesh& m, const CgIrWork& w, double* ru, bool solver,
                                                 int nb, int bid, const int* s_tri) {
  constexpr int kCells = NT / 4;
  const int64_t F = m.F, S4 = 4 * (m.E + m.F);
  const int q = threadIdx.x & 3, cl = threadIdx.x >> 2;
  if (q == 3) return;  // interior triples are written, never accumulated
  int p = 0;
  for (int64_t cb = (int64_t)bid * kCells; cb < F; cb += (int64_t)nb * kCells, ++p) {
    const int64_t c = cb + cl;
    if (c >= F) continue;
    bool own = false;
    const int t = triple<NT, RES>(m.tri, s_tri, p, c, q, own);
    if (!own) continue;
#pragma unroll
    for (int j = 0; j < 3; ++j)
      if (ru) ru[3 * t + j] = 0.0;
    if (solver) {
      const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int sl = 5; sl <= 7; ++sl) reinterpret_cast<float4*>(w.fbuf + sl * S4)[t] = z;
#pragma unroll
      for (int j = 0; j < 3; ++j) w.ax[3 * t + j] = 0.0;
    }
  }
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <int NT>
struct ChainBounds;
template <>
struct ChainBounds<128> { static constexpr int kMinBlocks = 6; };
template <>
struct ChainBounds<256> { static constexpr int kMinBlocks = 3; };

template <int NT, bool RES>
__global__ void __launch_bounds__(NT, ChainBounds<NT>::kMinBlocks)
    k_chain(const ChainProblem* __restrict__ probs, int P, int max_steps) {
  constexpr int kCells = NT / 4;
  extern __shared__ float s_mat[];
  __shared__ __align__(16) unsigned long long s_raw[(sizeof(ChainProblem) + 7) / 8];
  __shared__ int s_p;
  if (threadIdx.x == 0) {  // the problem whose block range holds this block
    int lo = 0, hi = P - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (probs[mid].block0 <= (int)blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
    s_p = lo;
  }
  __syncthreads();
  {
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(probs + s_p);
    for (int i = threadIdx.x; i < (int)((sizeof(ChainProblem) + 7) / 8); i += NT) s_raw[i] = __ldg(&src[i]);
  }
  __syncthreads();
  const ChainProblem& pr = *reinterpret_cast<const ChainProblem*>(s_raw);
  const DeviceMesh& m = pr.m;
  const int nb = pr.nblocks, bid = (int)blockIdx.x - pr.block0;
  if (bid < 0 || bid >= nb) return;  // not reached: the host covers the grid exactly
  const int64_t F = m.F, n = m.n, nu = m.n_u;
  const int passes = (int)(((F + kCells - 1) / kCells + nb - 1) / nb);
  int* s_tri = reinterpret_cast<int*>(s_mat + (size_t)passes * kCells * kMatStride);
  if (RES) cg_load_resident<NT>(m, nb, bid, s_mat, s_tri);
  const GridSync gs = {pr.partial, pr.partial_f, pr.scal, pr.sync + 1, reinterpret_cast<unsigned*>(pr.sync),
                       pr.w.flags};
  unsigned epoch = 0;
  double red[3];
  zero_owned_edges<NT, RES>(m, pr.w, pr.ru, true, nb, bid, s_tri);
  bool ok = grid_sum3<NT, double>(gs, nb, bid, epoch, 0.0, 0.0, 0.0, red);
  if (pr.timer && bid == 0 && threadIdx.x == 0) pr.timer[0] = global_ns();
  const int K = pr.K;
  int nsteps = pr.mode == 0 ? K : K + 1;
  if (max_steps >= 0 && max_steps < nsteps) nsteps = max_steps;
  for (int j = 0; ok && j < nsteps; ++j) {
    const double* in;
    const double* y;
    const double* z;
    double* outv;
    double s;
    if (pr.mode == 0) {
      in = pr.Q + (int64_t)j * n;
      y = nullptr;
      z = j > 0 ? pr.Q + (int64_t)(j - 1) * n : nullptr;
      outv = pr.Q + (int64_t)(j + 1) * n;
      s = (j == 0 ? 1.0 : 2.0) / pr.lam;
    } else {
      const int k = K - j;
      in = k + 1 <= K ? pr.bufs[(k + 1) % 3] : nullptr;
      y = pr.Q + (int64_t)k * n;
      z = k + 2 <= K ? pr.bufs[(k + 2) % 3] : nullptr;
      outv = k == 0 ? pr.out : pr.bufs[k % 3];
      s = (k == 0 ? 1.0 : 2.0) / pr.lam;
    }
    apply_K_phase<NT, RES>(m, in, s, pr.g, pr.H, y, y ? y + nu : nullptr, z ? z + nu : nullptr, pr.ru, outv + nu, nb,
                           bid, s_tri);
    if (in) {
      ok = grid_sum3<NT, double>(gs, nb, bid, epoch, 0.0, 0.0, 0.0, red);
      if (!ok) break;
    }
    ok = cg_solve<NT, RES>(m, pr.w, gs, pr.cp, in ? pr.ru : y, outv, 1.0, z, nb, bid, s_mat, s_tri, epoch);
    if (!ok) break;
    if (in) zero_owned_edges<NT, RES>(m, pr.w, pr.ru, false, nb, bid, s_tri);
    ok = grid_sum3<NT, double>(gs, nb, bid, epoch, 0.0, 0.0, 0.0, red);
  }
  if (pr.timer && bid == 0 && threadIdx.x == 0) pr.timer[1] = global_ns();
}

template <int NT, bool RES>
cudaError_t launch_t(const ChainProblem* d_probs, int P, int nblocks, size_t smem, int max_steps, cudaStream_t st) {
  static bool attr = false;
  if (RES && !attr) {
    cudaError_t e = cudaFuncSetAttribute(k_chain<NT, RES>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nblocks);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_chain<NT, RES>, d_probs, P, max_steps);
}

template <int NT, bool RES>
cudaError_t occupancy_t(size_t smem, int* per_sm) {
  if (RES) {
    cudaError_t e = cudaFuncSetAttribute(k_chain<NT, RES>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_chain<NT, RES>, NT, smem);
}

}  // namespace

cudaError_t upload_chain_tables(const ConstTables& t) {
  ChainTables k;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 12; ++b) k.D[a][b] = t.D[a][b];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) k.M2inv_ref[a][b] = t.M2inv_ref[a][b];
  return cudaMemcpyToSymbol(c_ktab, &k, sizeof(k));
}

size_t chain_res_smem(int64_t F, int nb, int nt) {
  const int64_t cells = nt / 4;
  const int64_t passes = ((F + cells - 1) / cells + nb - 1) / nb;
  return sizeof(float) * (size_t)(passes * cells * kMatStride) + sizeof(int) * (size_t)(passes * nt);
}

cudaError_t chain_occupancy(int nt, bool res, size_t smem, int* per_sm) {
  if (nt == 128) return res ? occupancy_t<128, true>(smem, per_sm) : occupancy_t<128, false>(smem, per_sm);
  if (nt == 256) return res ? occupancy_t<256, true>(smem, per_sm) : occupancy_t<256, false>(smem, per_sm);
  return cudaErrorInvalidValue;
}

cudaError_t launch_chain(const ChainProblem* d_probs, int P, int nblocks_total, int nt, bool res, size_t smem,
                         int max_steps, cudaStream_t st) {
  if (P <= 0 || nblocks_total <= 0) return cudaErrorInvalidValue;
  if (nt == 128)
    return res ? launch_t<128, true>(d_probs, P, nblocks_total, smem, max_steps, st)
               : launch_t<128, false>(d_probs, P, nblocks_total, smem, max_steps, st);
  if (nt == 256)
    return res ? launch_t<256, true>(d_probs, P, nblocks_total, smem, max_steps, st)
               : launch_t<256, false>(d_probs, P, nblocks_total, smem, max_steps, st);
  return cudaErrorInvalidValue;
}

}  // namespace pavg
