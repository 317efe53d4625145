// Subdomain mass solver: M1 x = b to FP64 accuracy with no grid-wide wait per
// inner iteration.
//
// Iterative refinement as in the mixed solver (FP32 inner solves on the FP64
// residual r / ||r||, FP64 residual b - M1 x after each sweep), but the inner
// solve is a Chebyshev semi-iteration on the block-Jacobi preconditioned M1
// over a fixed interval [a, b] that contains its spectrum (Lanczos estimate
// from the set-up, widened 5 % each way): it needs no inner products, so an
// inner iteration only has to wait for the neighbouring parts' contributions
// to the DOF triples they share, never for the whole grid.  With centre
// theta = (a + b) / 2, half-width delta = (b - a) / 2, sigma = theta / delta:
//   d_0 = P r_0 / theta,  rho_0 = 1 / sigma,  and for k = 0, 1, ...
//   x_{k+1} = x_k + d_k,  r_{k+1} = r_k - M1 d_k,  rho_{k+1} = 1 / (2 sigma - rho_k),
//   d_{k+1} = rho_{k+1} rho_k d_k + (2 rho_{k+1} / delta) P r_{k+1}.
// The iteration count per sweep is fixed in advance by the polynomial's error
// bound; the FP64 residual of each sweep (one grid-wide sum) decides whether
// another sweep follows.
//
// Layout.  Block p owns the contiguous cells cell0[p] .. cell0[p+1]-1 and the
// local DOF triples they touch.  Its cells' FP32 packed element matrices stay
// in shared memory for the whole solve; thread i serves local cell i (the
// 12 x 12 product into per-(cell, q) slots) and local triples i and i + NT
// (preconditioner block, r, d, x in registers).  A triple shared with another
// part is held by both: each part adds its own cell's slot and the partner's
// contribution, published as tagged 64-bit words (32-bit tag, 32-bit payload;
// FP64 values as two halves) in a double-buffered slot, so both copies are
// bitwise equal (a + b = b + a) and evolve identically.
//
// Every wait is bounded (sp.wait_cycles of clock64); a block whose wait runs
// out latches PAVG_ERR_TIMEOUT and leaves, and its neighbours' waits then run
// out too.  Tags and the arrival counter run on from launch to launch (the
// epoch base is stored back by block 0 at the end), so no buffer is cleared
// per launch; after a failed launch sd_reset_work clears them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "device.h"
#include "device_common.cuh"

namespace pavg {
namespace {

constexpr int kSdThreads = 768;   // one thread per local cell (up to 768) and two triples each
constexpr int kSdRounds = 2;      // local triples per thread at most
constexpr int kSdMatStride = 79;  // floats per cell's packed matrix (78, padded: conflict-free columns)
constexpr int kSdMaxIters = 256;  // Chebyshev iterations per sweep at most (the set-up caps it)

__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long atom_add_acq_rel_u64(unsigned long long* p, unsigned long long v) {
  unsigned long long r;
  asm volatile("atom.add.acq_rel.gpu.u64 %0, [%1], %2;" : "=l"(r) : "l"(p), "l"(v) : "memory");
  return r;
}

__device__ __forceinline__ unsigned long long tagged(unsigned tag, unsigned payload) {
  return ((unsigned long long)tag << 32) | payload;
}

// Waits until the N tagged words at p carry `tag` (bounded, one budget for
// all N); returns their payloads.
template <int N>
__device__ __forceinline__ bool poll_tagged(const unsigned long long* p, unsigned tag, unsigned out[N],
                                            long long limit) {
  const long long t0 = clock64();
  bool ok = true;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    unsigned long long v = ld_relaxed64(p + k);
    while (ok && (unsigned)(v >> 32) != tag) {
      if (clock64() - t0 > limit) ok = false;
      v = ld_relaxed64(p + k);
    }
    out[k] = (unsigned)v;
  }
  return ok;
}

// Deterministic sum of one double per thread over all nb blocks, one wait:
// each block publishes its partial, the last to arrive (the arrival counter
// runs on monotonically, so the last arrival of sum j is the one that makes it
// a multiple of nb) adds the partials in block order and publishes the total
// with the tag; the others wait for the tag.
template <int NT>
__device__ bool sd_grid_sum(const SdWork& w, int nb, int bid, unsigned long long tag, double v, double* out,
                            long long limit) {
  __shared__ double s_w[NT / 32];
  __shared__ double s_res;
  __shared__ int s_last, s_ok;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) s_w[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < NT / 32; ++k) s += s_w[k];
    __stcg(&w.part[bid], s);
    const unsigned long long old = atom_add_acq_rel_u64(&w.sync[0], 1ull);  // releases the partial
    s_last = (old + 1ull) % (unsigned long long)nb == 0ull;
    s_ok = 1;
  }
  __syncthreads();
  if (s_last) {
    if (warp == 0) {
      __threadfence();
      double t = 0.0;
      for (int k = lane; k < nb; k += 32) t += __ldcg(&w.part[k]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (lane == 0) {
        s_res = t;
        __stcg(w.pub, t);
        st_release_u64(&w.sync[1], tag);
      }
    }
  } else if (threadIdx.x == 0) {
    const long long t0 = clock64();
    while (ld_acquire_u64(&w.sync[1]) != tag) {
      if (clock64() - t0 > limit) {
        atomicOr(w.flags, kFlagTimeout);
        s_ok = 0;
        break;
      }
    }
    if (s_ok) s_res = __ldcg(w.pub);
  }
  __syncthreads();
  *out = s_res;
  const bool ok = s_ok != 0;
  __syncthreads();
  return ok;
}

// y = A v for one cell's packed symmetric 12 x 12 matrix (A(i, j) = Ap[psym(i, j) * stride]).
template <typename T, typename Load>
__device__ __forceinline__ void sym12(Load A, const T v[12], T y[12]) {
#pragma unroll
  for (int i = 0; i < 12; ++i) y[i] = T(0);
#pragma unroll
  for (int i = 0; i < 12; ++i)
#pragma unroll
    for (int j = i; j < 12; ++j) {
      const T a = A(psym(i, j));
      y[i] = fma(a, v[j], y[i]);
      if (j != i) y[j] = fma(a, v[i], y[j]);
    }
}

__device__ __forceinline__ void apply_p(const float p[6], const float r[3], float u[3]) {
  u[0] = fmaf(p[0], r[0], fmaf(p[1], r[1], p[2] * r[2]));
  u[1] = fmaf(p[1], r[0], fmaf(p[3], r[1], p[4] * r[2]));
  u[2] = fmaf(p[2], r[0], fmaf(p[4], r[1], p[5] * r[2]));
}

// Dynamic shared memory of a block: the packed FP32 matrices, then a region
// used as d (float4 per local triple) + cell slots (float4 per (cell, q)) in
// the FP32 phases and as the staged FP64 iterate (3 doubles per triple) in the
// FP64 product.
__host__ __device__ inline size_t sd_mat_floats(int max_cells) {
  return ((size_t)max_cells * kSdMatStride + 3) & ~(size_t)3;
}
inline size_t sd_smem_bytes(int max_cells, int max_lt) {
  const size_t region = std::max((size_t)max_lt * 16 + (size_t)max_cells * 64, (size_t)max_lt * 24);
  return sd_mat_floats(max_cells) * 4 + region;
}

template <int NT>
__global__ void __launch_bounds__(NT, 1)
    k_cheb_sd(DeviceMesh m, SdMesh sd, SdWork w, SdParams sp, const double* __restrict__ b, double* out,
              double scale_x, const double* __restrict__ add) {
  extern __shared__ float4 smem4[];
  float* s_mat = reinterpret_cast<float*>(smem4);
  float4* s_d = reinterpret_cast<float4*>(s_mat + sd_mat_floats(sd.max_cells));
  float4* s_slot = s_d + sd.max_lt;
  double* s_x64 = reinterpret_cast<double*>(s_d);
  __shared__ unsigned long long s_base;
  // the recurrence's scalars, the same in every sweep: d_{k+1} = c1[k] d_k + c2[k] P r_{k+1}
  __shared__ float s_c1[kSdMaxIters], s_c2[kSdMaxIters];

  const int nb = gridDim.x, bid = blockIdx.x, tid = threadIdx.x;
  if (sp.stall_mode == 1 && bid == sp.stall_part) return;  // test hook: never arrives
  const int64_t F = m.F;
  const int c0 = sd.cell0[bid], nc = sd.cell0[bid + 1] - c0;
  const int l0 = sd.lt0[bid], nl = sd.lt0[bid + 1] - l0;
  const long long limit = sp.wait_cycles;
  const int ns = sd.nslots;

  // ---- resident data: FP32 matrices of the block's cells (coalesced over cells)
  for (int t = tid; t < 78 * nc; t += NT) {
    const int idx = t / nc, k = t - idx * nc;
    s_mat[k * kSdMatStride + idx] = __ldg(&m.M1p[(int64_t)idx * F + c0 + k]);
  }
  if (tid == 0) {
    s_base = ld_relaxed64(&w.sync[2]);
    const double sigma = sp.theta / sp.delta;
    double rho = 1.0 / sigma;
    for (int k = 0; k < sp.iters && k < kSdMaxIters; ++k) {
      const double rho_n = 1.0 / (2.0 * sigma - rho);
      s_c1[k] = (float)(rho_n * rho);
      s_c2[k] = (float)(2.0 * rho_n / sp.delta);
      rho = rho_n;
    }
  }
  // ---- per-triple registers
  // d lives in shared memory only (s_d[lt], written and read by the thread that owns lt)
  float P[kSdRounds][6], r[kSdRounds][3], x[kSdRounds][3];
  uint32_t gt[kSdRounds], slot[kSdRounds];
  int recv[kSdRounds];
  double rr_loc = 0.0;
#pragma unroll
  for (int j = 0; j < kSdRounds; ++j) {
    const int lt = tid + j * NT;
    gt[j] = 0; slot[j] = 0xffffffffu; recv[j] = -1;
#pragma unroll
    for (int k = 0; k < 6; ++k) P[j][k] = 0.f;
    if (lt < nl) {
      gt[j] = __ldg(&sd.lt_gtri[l0 + lt]);
      slot[j] = __ldg(&sd.lt_slot[l0 + lt]);
      recv[j] = __ldg(&sd.lt_recv[l0 + lt]);
      const int64_t t = gt[j] & 0x7fffffffu;
      const float4 pa = __ldg(reinterpret_cast<const float4*>(m.Pinv) + 2 * t);
      const float4 pb = __ldg(reinterpret_cast<const float4*>(m.Pinv) + 2 * t + 1);
      P[j][0] = pa.x; P[j][1] = pa.y; P[j][2] = pa.z; P[j][3] = pa.w; P[j][4] = pb.x; P[j][5] = pb.y;
      const bool own = gt[j] >> 31;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double v = __ldg(&b[3 * t + k]);
        __stcg(&w.r64[3 * (int64_t)(l0 + lt) + k], v);
        __stcg(&w.x64[3 * (int64_t)(l0 + lt) + k], 0.0);
        if (own) rr_loc = fma(v, v, rr_loc);
      }
    }
  }
  __syncthreads();
  const unsigned long long base = s_base;
  unsigned long long ep = 0;
  double bb = 0.0;
  bool alive = sd_grid_sum<NT>(w, nb, bid, base + (++ep), rr_loc, &bb, limit);
  bool bad = !isfinite(bb), conv = !(bb > 0.0), have_x = false;
  const double tol2 = sp.rtol * sp.rtol * bb;
  double rr = bb;
  int sweeps = 0;
  const float inv_theta = (float)(1.0 / sp.theta);

  while (alive && !bad && !conv && sweeps < sp.max_sweeps) {
    // ---- sweep start: r_0 = r / ||r|| in FP32, x_0 = 0, d_0 = P r_0 / theta
    const double scale = 1.0 / sqrt(rr);
#pragma unroll
    for (int j = 0; j < kSdRounds; ++j) {
      const int lt = tid + j * NT;
#pragma unroll
      for (int k = 0; k < 3; ++k) { r[j][k] = 0.f; x[j][k] = 0.f; }
      if (lt < nl) {
#pragma unroll
        for (int k = 0; k < 3; ++k) r[j][k] = (float)(__ldcg(&w.r64[3 * (int64_t)(l0 + lt) + k]) * scale);
        float u[3];
        apply_p(P[j], r[j], u);
        s_d[lt] = make_float4(u[0] * inv_theta, u[1] * inv_theta, u[2] * inv_theta, 0.f);
      }
    }
    __syncthreads();
    for (int it = 0; it < sp.iters; ++it) {
      ++ep;
      const unsigned tag = (unsigned)(base + ep);
      unsigned long long* xbuf = w.xch32 + (size_t)((base + ep) & 1ull) * ns * 4;
      // ---- cell phase: each local cell's product with d into its four slots;
      //      contributions to shared triples also go to the partner
      if (sp.stall_mode == 2 && bid == sp.stall_part) return;  // test hook: never publishes
      for (int kc = tid; kc < nc; kc += NT) {
        const ushort4 L = __ldg(&sd.cell_lt[c0 + kc]);
        float v[12];
        const unsigned short li[4] = {L.x, L.y, L.z, L.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 a = s_d[li[q]];
          v[3 * q] = a.x; v[3 * q + 1] = a.y; v[3 * q + 2] = a.z;
        }
        const float* A = s_mat + kc * kSdMatStride;
        float y[12];
        sym12<float>([&](int i) { return A[i]; }, v, y);
#pragma unroll
        for (int q = 0; q < 4; ++q) s_slot[4 * kc + q] = make_float4(y[3 * q], y[3 * q + 1], y[3 * q + 2], 0.f);
        const int4 S = __ldg(&sd.cell_send[c0 + kc]);
        const int sq[3] = {S.x, S.y, S.z};
#pragma unroll
        for (int q = 0; q < 3; ++q)
          if (sq[q] >= 0) {
            unsigned long long* p = xbuf + (size_t)sq[q] * 4;
#pragma unroll
            for (int k = 0; k < 3; ++k) st_relaxed64(p + k, tagged(tag, __float_as_uint(y[3 * q + k])));
          }
      }
      __syncthreads();
      // ---- triple phase: M1 d on every local triple, then the recurrence
      const float c1 = s_c1[it], c2 = s_c2[it];
      const bool more = it + 1 < sp.iters;
      bool fail = false;
      // the partition numbers shared triples first: the second round (no
      // partner) before the first, which may wait for one
#pragma unroll
      for (int j = kSdRounds - 1; j >= 0; --j) {
        const int lt = tid + j * NT;
        if (lt >= nl) continue;
        const unsigned s0 = slot[j] & 0xffffu, s1 = slot[j] >> 16;
        const float4 a = s_slot[s0];
        float ad[3] = {a.x, a.y, a.z};
        if (s1 != 0xffffu) {
          const float4 c = s_slot[s1];
          ad[0] += c.x; ad[1] += c.y; ad[2] += c.z;
        } else if (recv[j] >= 0) {
          unsigned u[3];
          if (poll_tagged<3>(w.xch32 + (size_t)((base + ep) & 1ull) * ns * 4 + (size_t)recv[j] * 4, tag, u, limit)) {
            ad[0] += __uint_as_float(u[0]); ad[1] += __uint_as_float(u[1]); ad[2] += __uint_as_float(u[2]);
          } else {
            fail = true;
          }
        }
        const float4 dv = s_d[lt];
        const float dk[3] = {dv.x, dv.y, dv.z};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          x[j][k] += dk[k];
          r[j][k] -= ad[k];
        }
        if (more) {
          float u[3];
          apply_p(P[j], r[j], u);
          s_d[lt] = make_float4(fmaf(c1, dk[0], c2 * u[0]), fmaf(c1, dk[1], c2 * u[1]), fmaf(c1, dk[2], c2 * u[2]), 0.f);
        }
      }
      if (fail) atomicOr(w.flags, kFlagTimeout);
      if (__syncthreads_or(fail)) return;
    }
    // ---- FP64 refinement: x += x_32 ||r||, staged in shared memory for the product
    const double inv = 1.0 / scale;
#pragma unroll
    for (int j = 0; j < kSdRounds; ++j) {
      const int lt = tid + j * NT;
      if (lt >= nl) continue;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        double* px = &w.x64[3 * (int64_t)(l0 + lt) + k];
        const double xn = fma((double)x[j][k], inv, __ldcg(px));
        __stcg(px, xn);
        s_x64[3 * lt + k] = xn;
      }
    }
    have_x = true;
    __syncthreads();
    ++ep;
    const unsigned tag64 = (unsigned)(base + ep);
    unsigned long long* xb64 = w.xch64 + (size_t)((base + ep) & 1ull) * ns * 6;
    // ---- cell phase: FP64 products with the FP64 element matrices (global memory)
    for (int kc = tid; kc < nc; kc += NT) {
      const ushort4 L = __ldg(&sd.cell_lt[c0 + kc]);
      const unsigned short li[4] = {L.x, L.y, L.z, L.w};
      double v[12];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < 3; ++k) v[3 * q + k] = s_x64[3 * li[q] + k];
      // row by row with a rolled loop (one running sum; the symmetric form's
      // twelve sums next to the twelve values would not fit the registers of
      // 768 threads), then the shared triples' rows go to the partners
      const double* A = m.M1 + c0 + kc;
      double* ys = w.y64 + 12 * (int64_t)(c0 + kc);
#pragma unroll 1
      for (int i = 0; i < 12; ++i) {
        double acc = 0.0;
#pragma unroll
        for (int jj = 0; jj < 12; ++jj)
          acc = fma(__ldg(A + (int64_t)(i <= jj ? psym(i, jj) : psym(jj, i)) * F), v[jj], acc);
        __stcg(ys + i, acc);
      }
      const int4 S = __ldg(&sd.cell_send[c0 + kc]);
      const int sq[3] = {S.x, S.y, S.z};
#pragma unroll
      for (int q = 0; q < 3; ++q)
        if (sq[q] >= 0) {
          unsigned long long* p = xb64 + (size_t)sq[q] * 6;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const unsigned long long bits = (unsigned long long)__double_as_longlong(__ldcg(ys + 3 * q + k));
            st_relaxed64(p + 2 * k, tagged(tag64, (unsigned)(bits >> 32)));
            st_relaxed64(p + 2 * k + 1, tagged(tag64, (unsigned)bits));
          }
        }
    }
    __syncthreads();
    // ---- triple phase: r = b - M1 x on every local triple; norm over owned ones
    rr_loc = 0.0;
    bool fail = false;
#pragma unroll
    for (int j = kSdRounds - 1; j >= 0; --j) {  // as in the FP32 phase: the round that may wait last
      const int lt = tid + j * NT;
      if (lt >= nl) continue;
      const unsigned s0 = slot[j] & 0xffffu, s1 = slot[j] >> 16;
      const double* y0 = w.y64 + 12 * (int64_t)(c0 + (s0 >> 2)) + 3 * (s0 & 3);
      double ad[3] = {__ldcg(y0), __ldcg(y0 + 1), __ldcg(y0 + 2)};
      if (s1 != 0xffffu) {
        const double* y1 = w.y64 + 12 * (int64_t)(c0 + (s1 >> 2)) + 3 * (s1 & 3);
        ad[0] += __ldcg(y1); ad[1] += __ldcg(y1 + 1); ad[2] += __ldcg(y1 + 2);
      } else if (recv[j] >= 0) {
        unsigned u[6];
        if (poll_tagged<6>(w.xch64 + (size_t)((base + ep) & 1ull) * ns * 6 + (size_t)recv[j] * 6, tag64, u, limit)) {
#pragma unroll
          for (int k = 0; k < 3; ++k)
            ad[k] += __longlong_as_double((long long)(((unsigned long long)u[2 * k] << 32) | u[2 * k + 1]));
        } else {
          fail = true;
        }
      }
      const int64_t t = gt[j] & 0x7fffffffu;
      const bool own = gt[j] >> 31;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double rk = __ldg(&b[3 * t + k]) - ad[k];
        __stcg(&w.r64[3 * (int64_t)(l0 + lt) + k], rk);
        if (own) rr_loc = fma(rk, rk, rr_loc);
      }
    }
    if (fail) atomicOr(w.flags, kFlagTimeout);
    if (__syncthreads_or(fail)) return;
    alive = sd_grid_sum<NT>(w, nb, bid, base + (++ep), rr_loc, &rr, limit);
    ++sweeps;
    if (!isfinite(rr)) bad = true;
    conv = rr <= tol2;
  }
  if (!alive) return;
  // ---- out = scale_x x + add on the owned triples
#pragma unroll
  for (int j = 0; j < kSdRounds; ++j) {
    const int lt = tid + j * NT;
    if (lt >= nl || !(gt[j] >> 31)) continue;
    const int64_t t = gt[j] & 0x7fffffffu;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double v = have_x ? scale_x * __ldcg(&w.x64[3 * (int64_t)(l0 + lt) + k]) : 0.0;
      if (add) v += __ldg(&add[3 * t + k]);
      out[3 * t + k] = v;
    }
  }
  if (bid == 0 && tid == 0) {
    if (bad) atomicOr(w.flags, kFlagNonFinite);
    else if (!conv) atomicOr(w.flags, kFlagNoConv);
    const unsigned long long inner = (unsigned long long)sweeps * sp.iters;
    atomicAdd(&w.stats[0], 1ull);
    atomicAdd(&w.stats[1], inner);
    atomicMax(&w.stats[2], inner);
    atomicAdd(&w.stats[3], (unsigned long long)sweeps);
    // every block read the base before it arrived at the first grid sum, and
    // every block has arrived at the last one: the next launch continues here
    st_relaxed64(&w.sync[2], base + ep);
  }
}

}  // namespace

template <class T>
static cudaError_t upload_vec(T** dst, const std::vector<T>& v) {
  cudaError_t e = cudaMalloc((void**)dst, sizeof(T) * std::max<size_t>(v.size(), 1));
  if (e != cudaSuccess) return e;
  return v.empty() ? cudaSuccess : cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
}

cudaError_t sd_configure(int64_t F, int64_t E, const std::vector<int32_t>& tri, double lmin, double lmax, int P,
                         SdMesh* sd) {
  *sd = SdMesh();
  int dev = 0, sms = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if (P < 1 || P > sms || P > F || !(lmin > 0.0) || !(lmax > lmin)) return cudaSuccess;
  SdPartition part;
  try {
    build_sd_partition(F, E, tri, P, &part);
  } catch (const std::exception&) {
    return cudaSuccess;  // not available: the context uses the global solver
  }
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, k_cheb_sd<kSdThreads>);
  if (e != cudaSuccess) return e;
  const size_t smem = sd_smem_bytes(part.max_cells, part.max_lt);
  if (part.max_lt > kSdRounds * kSdThreads || smem + fa.sharedSizeBytes > (size_t)optin) return cudaSuccess;
  // the attribute belongs to the kernel (per device), not to this mesh: allow
  // the largest block any mesh may need, so that configuring a small mesh
  // after a large one does not make the large one's launches invalid
  e = cudaFuncSetAttribute(k_cheb_sd<kSdThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - (int)fa.sharedSizeBytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cheb_sd<kSdThreads>, kSdThreads, smem);
  if (e != cudaSuccess) return e;
  if ((int64_t)per_sm * sms < P) return cudaSuccess;
  std::vector<ushort4> cl(F);
  std::vector<int4> cs(F);
  for (int64_t c = 0; c < F; ++c) {
    cl[c] = make_ushort4((unsigned short)part.cell_lt[4 * c], (unsigned short)part.cell_lt[4 * c + 1],
                         (unsigned short)part.cell_lt[4 * c + 2], (unsigned short)part.cell_lt[4 * c + 3]);
    cs[c] = make_int4(part.cell_send[4 * c], part.cell_send[4 * c + 1], part.cell_send[4 * c + 2], -1);
  }
  SdMesh s;
  s.max_cells = part.max_cells;
  s.max_lt = part.max_lt;
  s.nslots = part.nslots;
  s.total_lt = part.lt0[P];
  s.smem = smem;
  s.lmin = lmin;
  s.lmax = lmax;
  if ((e = upload_vec(&s.cell0, part.cell0)) != cudaSuccess || (e = upload_vec(&s.lt0, part.lt0)) != cudaSuccess ||
      (e = upload_vec(&s.lt_gtri, part.lt_gtri)) != cudaSuccess ||
      (e = upload_vec(&s.lt_slot, part.lt_slot)) != cudaSuccess ||
      (e = upload_vec(&s.lt_recv, part.lt_recv)) != cudaSuccess || (e = upload_vec(&s.cell_lt, cl)) != cudaSuccess ||
      (e = upload_vec(&s.cell_send, cs)) != cudaSuccess) {
    sd_free(&s);
    return e;
  }
  s.P = P;
  *sd = s;
  return cudaSuccess;
}

void sd_free(SdMesh* sd) {
  cudaFree(sd->cell0); cudaFree(sd->lt0); cudaFree(sd->lt_gtri); cudaFree(sd->lt_slot); cudaFree(sd->lt_recv);
  cudaFree(sd->cell_lt); cudaFree(sd->cell_send);
  *sd = SdMesh();
}

cudaError_t sd_reset_work(const SdMesh& sd, int64_t F, SdWork* w) {
  (void)F;
  const size_t ns = (size_t)std::max(sd.nslots, 1);
  cudaError_t e = cudaMemset(w->xch32, 0, sizeof(unsigned long long) * 2 * ns * 4);
  if (e == cudaSuccess) e = cudaMemset(w->xch64, 0, sizeof(unsigned long long) * 2 * ns * 6);
  if (e == cudaSuccess) e = cudaMemset(w->sync, 0, sizeof(unsigned long long) * 4);
  return e;
}

cudaError_t sd_alloc_work(const SdMesh& sd, int64_t F, SdWork* w) {
  const size_t ns = (size_t)std::max(sd.nslots, 1), lt = (size_t)std::max(sd.total_lt, 1);
  cudaError_t e = cudaMalloc((void**)&w->xch32, sizeof(unsigned long long) * 2 * ns * 4);
  if (e == cudaSuccess) e = cudaMalloc((void**)&w->xch64, sizeof(unsigned long long) * 2 * ns * 6);
  if (e == cudaSuccess) e = cudaMalloc((void**)&w->y64, sizeof(double) * 12 * (size_t)F);
  if (e == cudaSuccess) e = cudaMalloc((void**)&w->x64, sizeof(double) * 3 * lt);
  if (e == cudaSuccess) e = cudaMalloc((void**)&w->r64, sizeof(double) * 3 * lt);
  if (e == cudaSuccess) e = cudaMalloc((void**)&w->part, sizeof(double) * std::max(sd.P, 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&w->pub, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&w->sync, sizeof(unsigned long long) * 4);
  if (e == cudaSuccess) e = sd_reset_work(sd, F, w);
  return e;
}

void sd_free_work(SdWork* w) {
  cudaFree(w->xch32); cudaFree(w->xch64); cudaFree(w->y64); cudaFree(w->x64); cudaFree(w->r64);
  cudaFree(w->part); cudaFree(w->pub); cudaFree(w->sync);
  w->xch32 = w->xch64 = nullptr;
  w->y64 = w->x64 = w->r64 = w->part = w->pub = nullptr;
  w->sync = nullptr;
}

cudaError_t launch_cheb_sd(const DeviceMesh& m, const SdMesh& sd, const SdWork& w, const SdParams& sp,
                           const double* b, double* out, double scale_x, const double* add, cudaStream_t st) {
  if (sd.P < 1) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sd.P);
  cfg.blockDim = dim3(kSdThreads);
  cfg.dynamicSmemBytes = sd.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_cheb_sd<kSdThreads>, m, sd, w, sp, b, out, scale_x, add);
}

}  // namespace pavg
