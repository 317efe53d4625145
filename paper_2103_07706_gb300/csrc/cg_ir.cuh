// Device code of the mixed-precision M1 solver, shared by the single-problem
// kernel (cg_mixed.cu) and the batched persistent kernel (batch.cu).
//
// M1 x = b is solved by iterative refinement: each sweep solves
// M1 d = r / ||r|| in FP32 by conjugate gradients (single-reduction form, one
// bounded barrier per iteration, 3x3 block-Jacobi preconditioner on the
// triples of DOFs that share an edge or a cell interior), adds d ||r|| to the
// FP64 iterate and recomputes the FP64 residual r = b - M1 x with the FP64
// element matrices.  The FP64 residual makes the result FP64-accurate; the
// FP32 iterations run at the FP32 rate, 64x the FP64 rate of GB300.
//
// Thread layout: four threads per cell, one per DOF triple (the three moments
// of an edge, or the three interior moments).  Each thread applies its
// triple's 3x3 preconditioner block; the four threads of a cell exchange their
// values by warp shuffles and each computes three rows of the cell's element
// matrix.  A block of NT threads handles NT/4 cells per pass; the nb blocks
// of one problem take cells (bid + j nb) NT/4 ... in passes j.  With RES the
// block's FP32 element matrices sit in shared memory for the whole solve;
// otherwise they stream from L2 ([36][F][4] row blocks).
// Sums over a problem's blocks take one barrier: each block publishes a
// partial, the last block to arrive adds all partials in block order (so the
// result does not depend on arrival order) and releases the others by a
// tagged publication.  FP32 phases reduce in FP32, FP64 phases in FP64.
// Several problems can share one cooperative launch: their blocks never wait
// on one another.
#pragma once

#include <cuda_runtime.h>

#include "device.h"
#include "device_common.cuh"

namespace pavg {
namespace {

constexpr int kMatStride = 79;   // packed 78 entries per cell, padded to spread shared-memory banks

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned r;
  asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "r"(v) : "memory");
  return r;
}
__device__ __forceinline__ void red_add_release(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned r;
  asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(r) : "l"(p) : "memory");
  return r;
}

struct GridSync {
  double* partial;
  float* partial_f;
  double* scal;
  unsigned long long* tag;
  unsigned* bar;
  int* flags;
};

__device__ __forceinline__ float* part_of(const GridSync& g, float) { return g.partial_f; }
__device__ __forceinline__ double* part_of(const GridSync& g, double) { return g.partial; }

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
  unsigned long long r;
  asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(r) : "l"(p) : "memory");
  return r;
}

// Sum of three per-thread values over the nb blocks that work on one problem
// (bid = this block's index among them), deterministic, one barrier.
// `epoch` counts the sums of this launch (identical in every block).
// The last block to arrive publishes each sum as a 64-bit word tagged with
// the epoch (FP32 sums: tag in the high half, value in the low half; FP64
// sums: the values first, then a tag word), so waiting blocks learn that the
// barrier is open and read the sums with the same loads.
template <int NT, typename Tv>
__device__ __forceinline__ bool grid_sum3(const GridSync& g, int nb, int bid, unsigned& epoch, Tv a, Tv b, Tv c,
                                          double out[3]) {
  __shared__ Tv sh[3][NT / 32];
  __shared__ double s_out[3];
  __shared__ int s_last, s_ok;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool fp32 = sizeof(Tv) == 4;
  Tv* part = part_of(g, Tv(0));
  ++epoch;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  if (lane == 0) { sh[0][warp] = a; sh[1][warp] = b; sh[2][warp] = c; }
  __syncthreads();
  if (threadIdx.x == 0) {
    Tv s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
    for (int k = 0; k < NT / 32; ++k) { s0 += sh[0][k]; s1 += sh[1][k]; s2 += sh[2][k]; }
    part[bid] = s0;
    part[nb + bid] = s1;
    part[2 * nb + bid] = s2;
    const unsigned arrived = atom_add_acq_rel(g.bar, 1u);  // releases this block's writes
    s_last = arrived == (unsigned)(nb - 1);
    s_ok = 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    Tv t0 = 0, t1 = 0, t2 = 0;
    for (int k = threadIdx.x; k < nb; k += NT) {
      t0 += __ldcg(&part[k]);
      t1 += __ldcg(&part[nb + k]);
      t2 += __ldcg(&part[2 * nb + k]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      t0 += __shfl_down_sync(0xffffffffu, t0, o);
      t1 += __shfl_down_sync(0xffffffffu, t1, o);
      t2 += __shfl_down_sync(0xffffffffu, t2, o);
    }
    __syncthreads();
    if (lane == 0) { sh[0][warp] = t0; sh[1][warp] = t1; sh[2][warp] = t2; }
    __syncthreads();
    if (threadIdx.x == 0) {
      Tv s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
      for (int k = 0; k < NT / 32; ++k) { s0 += sh[0][k]; s1 += sh[1][k]; s2 += sh[2][k]; }
      s_out[0] = (double)s0;
      s_out[1] = (double)s1;
      s_out[2] = (double)s2;
      *((volatile unsigned*)g.bar) = 0u;
      const unsigned long long hi = (unsigned long long)epoch << 32;
      if (fp32) {
        __threadfence();
        volatile unsigned long long* t = g.tag;
        t[0] = hi | __float_as_uint((float)s0);
        t[1] = hi | __float_as_uint((float)s1);
        t[2] = hi | __float_as_uint((float)s2);
      } else {
        g.scal[0] = (double)s0;
        g.scal[1] = (double)s1;
        g.scal[2] = (double)s2;
        __threadfence();
        *((volatile unsigned long long*)&g.tag[3]) = hi;
      }
    }
  } else if (threadIdx.x == 0) {
    const long long t_start = clock64();
    const int k0 = fp32 ? 0 : 3, k1 = fp32 ? 2 : 3;
    for (int k = k0; k <= k1 && s_ok; ++k) {
      unsigned long long v;
      while (((v = ld_acquire64(&g.tag[k])) >> 32) != epoch) {
        if (clock64() - t_start > kBarrierTimeoutCycles) {
          atomicOr(g.flags, kFlagTimeout);
          s_ok = 0;
          break;
        }
        __nanosleep(16);
      }
      if (fp32) s_out[k] = (double)__uint_as_float((unsigned)(v & 0xffffffffu));
    }
    if (!fp32) {
      s_out[0] = __ldcg(&g.scal[0]);
      s_out[1] = __ldcg(&g.scal[1]);
      s_out[2] = __ldcg(&g.scal[2]);
    }
    if (*((volatile int*)g.flags) & kFlagTimeout) s_ok = 0;
  }
  __syncthreads();
  out[0] = s_out[0];
  out[1] = s_out[1];
  out[2] = s_out[2];
  const bool ok = s_ok != 0;
  __syncthreads();
  return ok;
}

__device__ __forceinline__ void load_P(const float* __restrict__ P, int t, float p[6]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(P) + 2 * t);
  const float4 b = __ldg(reinterpret_cast<const float4*>(P) + 2 * t + 1);
  p[0] = a.x; p[1] = a.y; p[2] = a.z; p[3] = a.w; p[4] = b.x; p[5] = b.y;
}

// FP32 vectors hold each DOF triple in one 16-byte slot (the 4th float unused).
__device__ __forceinline__ void ld3(const float* base, int t, float v[3]) {
  const float4 a = __ldcg(reinterpret_cast<const float4*>(base) + t);
  v[0] = a.x; v[1] = a.y; v[2] = a.z;
}
__device__ __forceinline__ void st3(float* base, int t, const float v[3]) {
  reinterpret_cast<float4*>(base)[t] = make_float4(v[0], v[1], v[2], 0.f);
}
// Vector reduction into a triple slot: one L2 request for the three values.
__device__ __forceinline__ void red3(float* base, int t, const float v[3]) {
  asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(base + 4 * t), "f"(v[0]),
               "f"(v[1]), "f"(v[2]), "f"(0.f)
               : "memory");
}

// u = P r for one symmetric 3x3 block p = (00, 01, 02, 11, 12, 22).
__device__ __forceinline__ void apply3(const float p[6], const float r[3], float u[3]) {
  u[0] = fmaf(p[0], r[0], fmaf(p[1], r[1], p[2] * r[2]));
  u[1] = fmaf(p[1], r[0], fmaf(p[3], r[1], p[4] * r[2]));
  u[2] = fmaf(p[2], r[0], fmaf(p[4], r[1], p[5] * r[2]));
}

__device__ __forceinline__ int packed_index(int i, int k) {
  const int a = i < k ? i : k, b = i < k ? k : i;
  return a * 12 - a * (a - 1) / 2 + (b - a);
}

// The cell's 12 values, gathered from its four threads.
template <typename T>
__device__ __forceinline__ void gather12(const T v[3], T va[12]) {
  const int base = (threadIdx.x & 31) & ~3;
#pragma unroll
  for (int src = 0; src < 4; ++src)
#pragma unroll
    for (int j = 0; j < 3; ++j) va[3 * src + j] = __shfl_sync(0xffffffffu, v[j], base + src);
}

// Rows 3q .. 3q+2 of the cell's FP32 element matrix times its 12 values.
// RES: the matrix sits in shared memory, packed, at sm + cell_slot * kMatStride.
// Otherwise it streams from the [36][F][4] row-block layout in global memory.
template <bool RES>
__device__ __forceinline__ void rows3(const float* __restrict__ A, const float* sm, int64_t F, int64_t c, int q,
                                      bool active, const float u[3], float wl[3]) {
  float ua[12];
  gather12(u, ua);
  wl[0] = wl[1] = wl[2] = 0.f;
  if (!active) return;
  if (RES) {
#pragma unroll 1
    for (int j = 0; j < 3; ++j) {
      const int i = 3 * q + j;
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < 12; ++k) acc = fmaf(sm[packed_index(i, k)], ua[k], acc);
      if (j == 0) wl[0] = acc;
      else if (j == 1) wl[1] = acc;
      else wl[2] = acc;
    }
  } else {
    const int64_t stride = 4 * F, off = 4 * c + q;
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 12; ++k) wl[j] = fmaf(__ldg(&A[(j * 12 + k) * stride + off]), ua[k], wl[j]);
  }
}

// Same with the FP64 packed element matrix ([78][F]) in global memory.
__device__ __forceinline__ void rows3_d(const double* __restrict__ M1, int64_t F, int64_t c, int q, bool active,
                                        const double x[3], double wl[3]) {
  double xa[12];
  gather12(x, xa);
  wl[0] = wl[1] = wl[2] = 0.0;
  if (!active) return;
#pragma unroll 1
  for (int j = 0; j < 3; ++j) {
    const int i = 3 * q + j;
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < 12; ++k) acc = fma(__ldg(&M1[(int64_t)packed_index(i, k) * F + c]), xa[k], acc);
    if (j == 0) wl[0] = acc;
    else if (j == 1) wl[1] = acc;
    else wl[2] = acc;
  }
}

// DOF triple of thread (c, q) in pass p: DOFs 3t .. 3t+2, and whether the
// cell owns it (from shared memory on the resident path).
template <int NT, bool RES>
__device__ __forceinline__ int triple(const int32_t* __restrict__ tri, const int* s_tri, int p, int64_t c, int q,
                                      bool& own) {
  const int v = RES ? s_tri[p * NT + threadIdx.x] : __ldg(&tri[4 * c + q]);
  own = v < 0;
  return v & 0x7fffffff;
}


// Copies this block's FP32 element matrices and DOF triples into shared memory
// (the RES path): s_mat [passes][NT/4][kMatStride], s_tri [passes][NT].
template <int NT>
__device__ __forceinline__ void cg_load_resident(const DeviceMesh& m, int nb, int bid, float* s_mat, int* s_tri) {
  constexpr int kCells = NT / 4;
  const int64_t F = m.F;
  const int q = threadIdx.x & 3, cl = threadIdx.x >> 2;
  int pp = 0;
  for (int64_t cb = (int64_t)bid * kCells; cb < F; cb += (int64_t)nb * kCells, ++pp) {
    for (int t = threadIdx.x; t < 78 * kCells; t += NT) {
      const int idx = t / kCells, k = t % kCells;
      const int64_t c = cb + k;
      s_mat[(pp * kCells + k) * kMatStride + idx] = c < F ? __ldg(&m.M1p[(int64_t)idx * F + c]) : 0.f;
    }
    const int64_t c = cb + cl;
    s_tri[pp * NT + threadIdx.x] = c < F ? __ldg(&m.tri[4 * c + q]) : 0;
  }
  __syncthreads();
}

// out_u = scale_x * M1^{-1} b + add on the velocity DOFs, by the nb blocks of
// one problem.  Returns false when a wait timed out or a value was not finite
// (the problem's flags are set).  On a normal return the edge parts of the
// accumulation slots 5-7 of w.fbuf and of w.ax are zero again, as on entry.
template <int NT, bool RES>
__device__ bool cg_solve(const DeviceMesh& m, const CgIrWork& w, const GridSync& gs, const CgIrParams& cp,
                         const double* __restrict__ b, double* out, double scale_x, const double* __restrict__ add,
                         int nb, int bid, const float* s_mat, const int* s_tri, unsigned& epoch) {
  constexpr int kCells = NT / 4;
  __shared__ double s_alpha, s_gamma, s_rr0;
  __shared__ float s_f[2];  // alpha, beta of the current FP32 iteration
  __shared__ int s_state;   // 0 continue, 1 converged, 2 non-finite
  const int64_t F = m.F, T = m.E + m.F;
  const int q = threadIdx.x & 3, cl = threadIdx.x >> 2;
  const int64_t cbase0 = (int64_t)bid * kCells, cstride = (int64_t)nb * kCells;
  const int S4 = 4 * (int)T;  // floats per FP32 vector slot
  float* __restrict__ FB = w.fbuf;
  double red[3];

  // ---- ||b||^2 (owners of each triple)
  double pb = 0.0;
  int p = 0;
  for (int64_t cb = cbase0; cb < F; cb += cstride, ++p) {
    const int64_t c = cb + cl;
    if (c >= F) continue;
    bool own = false;
    const int t = triple<NT, RES>(m.tri, s_tri, p, c, q, own);
    if (own)
#pragma unroll
      for (int j = 0; j < 3; ++j) { const double v = __ldg(&b[3 * t + j]); pb = fma(v, v, pb); }
  }
  bool alive = grid_sum3<NT, double>(gs, nb, bid, epoch, pb, 0.0, 0.0, red);
  const double bb = red[0];
  const double tol2 = cp.rtol * cp.rtol * bb;
  bool bad = !isfinite(bb);
  bool conv = !(bb > 0.0);
  double rr64 = bb;
  const double* rsrc = b;
  int xcur = 0;
  bool have_x = false;
  int sweeps = 0, inner_total = 0;

  for (; alive && !conv && !bad && sweeps < cp.max_sweeps; ++sweeps) {
    const double scale = 1.0 / sqrt(rr64);
    // ---- FP32 start: r0 = r / ||r||, u0 = P r0, w0 = A u0 (into slot 5, zero on entry)
    float pg = 0.f, pd = 0.f, pr = 0.f;
    {
      p = 0;
      for (int64_t cb = cbase0; cb < F; cb += cstride, ++p) {
        const int64_t c = cb + cl;
        const bool active = c < F;
        bool own = false;
        int t = 0;
        float r0[3] = {0.f, 0.f, 0.f}, u[3] = {0.f, 0.f, 0.f}, wl[3], pb3[6];
        if (active) {
          t = triple<NT, RES>(m.tri, s_tri, p, c, q, own);
          load_P(m.Pinv, t, pb3);
#pragma unroll
          for (int j = 0; j < 3; ++j) r0[j] = (float)(__ldcg(&rsrc[3 * t + j]) * scale);
          apply3(pb3, r0, u);
        }
        rows3<RES>(m.M1f, s_mat + (p * kCells + cl) * kMatStride, F, c, q, active, u, wl);
        if (active) {
#pragma unroll
          for (int j = 0; j < 3; ++j) pd = fmaf(u[j], wl[j], pd);
          if (q < 3) red3(FB + 5 * S4, t, wl);
          else st3(FB + 5 * S4, t, wl);
          if (own) {
            st3(FB + 1 * S4, t, r0);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
              pg = fmaf(r0[j], u[j], pg);
              pr = fmaf(r0[j], r0[j], pr);
            }
          }
        }
      }
    }
    alive = grid_sum3<NT, float>(gs, nb, bid, epoch, pg, pd, pr, red);
    if (threadIdx.x == 0) {
      s_gamma = red[0];
      s_rr0 = red[2];
      s_alpha = red[0] / red[1];
      s_f[0] = (float)s_alpha;
      s_f[1] = 0.f;
      s_state = isfinite(s_alpha) ? 0 : 2;
    }
    __syncthreads();
    if (s_state == 2) { bad = true; break; }
    int it = 0;
    for (; alive && it < cp.max_inner; ++it) {
      const int i = it;
      const int o_rin = (1 + (i & 1)) * S4, o_rout = (2 - (i & 1)) * S4;
      const int o_sin = (3 + ((i + 1) & 1)) * S4, o_sout = (3 + (i & 1)) * S4;
      const int i3 = i % 3;
      const int o_win = (5 + i3) * S4, o_wacc = (5 + (i3 + 1) % 3) * S4, o_wz = (5 + (i3 + 2) % 3) * S4;
      const int o_p = 8 * S4;
      const float fa = s_f[0], fb = s_f[1];
      pg = pd = pr = 0.f;
      p = 0;
      for (int64_t cb = cbase0; cb < F; cb += cstride, ++p) {
        const int64_t c = cb + cl;
        const bool active = c < F;
        bool own = false;
        int t = 0;
        float rold[3] = {0.f, 0.f, 0.f}, rn[3] = {0.f, 0.f, 0.f}, sv[3] = {0.f, 0.f, 0.f};
        float u[3] = {0.f, 0.f, 0.f}, wl[3], pb3[6], pold[3] = {0.f, 0.f, 0.f}, xold[3] = {0.f, 0.f, 0.f};
        if (active) {
          t = triple<NT, RES>(m.tri, s_tri, p, c, q, own);
          // every load of this pass first, then arithmetic, then every store
          load_P(m.Pinv, t, pb3);
          float wv[3], sp[3] = {0.f, 0.f, 0.f};
          ld3(FB + o_rin, t, rold);
          ld3(FB + o_win, t, wv);
          if (i > 0) ld3(FB + o_sin, t, sp);
          if (own && i > 0) { ld3(FB + o_p, t, pold); ld3(FB, t, xold); }
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            sv[j] = i > 0 ? fmaf(fb, sp[j], wv[j]) : wv[j];
            rn[j] = fmaf(-fa, sv[j], rold[j]);
          }
          apply3(pb3, rn, u);
        }
        rows3<RES>(m.M1f, s_mat + (p * kCells + cl) * kMatStride, F, c, q, active, u, wl);
        if (active) {
#pragma unroll
          for (int j = 0; j < 3; ++j) pd = fmaf(u[j], wl[j], pd);
          if (q < 3) red3(FB + o_wacc, t, wl);
          else st3(FB + o_wacc, t, wl);
          if (own) {
            float ui[3], pv[3], xv[3];
            apply3(pb3, rold, ui);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
              pv[j] = i > 0 ? fmaf(fb, pold[j], ui[j]) : ui[j];
              xv[j] = i > 0 ? fmaf(fa, pv[j], xold[j]) : fa * pv[j];
              pg = fmaf(rn[j], u[j], pg);
              pr = fmaf(rn[j], rn[j], pr);
            }
            st3(FB + o_sout, t, sv);
            st3(FB + o_rout, t, rn);
            st3(FB + o_p, t, pv);
            st3(FB, t, xv);
            if (q < 3) {
              const float z[3] = {0.f, 0.f, 0.f};
              st3(FB + o_wz, t, z);
            }
          }
        }
      }
      alive = grid_sum3<NT, float>(gs, nb, bid, epoch, pg, pd, pr, red);
      // the recurrence scalars live in shared memory, updated by thread 0
      if (threadIdx.x == 0) {
        const double gnew = red[0], dnew = red[1], rrf = red[2];
        if (!(isfinite(gnew) && isfinite(dnew) && isfinite(rrf))) {
          s_state = 2;
        } else if (rrf <= (double)cp.inner_rtol * (double)cp.inner_rtol * s_rr0) {
          s_state = 1;
        } else {
          const double bnew = gnew / s_gamma;
          s_alpha = gnew / (dnew - bnew * gnew / s_alpha);
          s_gamma = gnew;
          s_f[0] = (float)s_alpha;
          s_f[1] = (float)bnew;
          s_state = 0;
        }
      }
      __syncthreads();
      const int state = s_state;
      __syncthreads();
      if (state == 2) { bad = true; ++it; break; }
      if (state == 1) { ++it; break; }
    }
    inner_total += it;
    if (!alive || bad) break;
    // ---- x_new = x_old + d / scale and A x_new (FP64) into ax; clear slots 5-7 for the next sweep
    const double* xold = xcur ? w.x[1] : w.x[0];
    double* xnew = xcur ? w.x[0] : w.x[1];
    const double inv = 1.0 / scale;
    p = 0;
    for (int64_t cb = cbase0; cb < F; cb += cstride, ++p) {
      const int64_t c = cb + cl;
      const bool active = c < F;
      bool own = false;
      int t = 0;
      double xn[3] = {0.0, 0.0, 0.0}, ax[3];
      if (active) {
        t = triple<NT, RES>(m.tri, s_tri, p, c, q, own);
        double xo[3] = {0.0, 0.0, 0.0};
        float dxf[3];
        ld3(FB, t, dxf);
#pragma unroll
        for (int j = 0; j < 3; ++j)
          if (have_x) xo[j] = __ldcg(&xold[3 * t + j]);
#pragma unroll
        for (int j = 0; j < 3; ++j) xn[j] = fma((double)dxf[j], inv, xo[j]);
      }
      rows3_d(m.M1, F, c, q, active, xn, ax);
      if (active) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const int d = 3 * t + j;
          if (q < 3) atomicAdd(&w.ax[d], ax[j]);
          else w.ax[d] = ax[j];
          if (own) {
            xnew[d] = xn[j];
            if (q < 3 && j == 0) {
              const float z[3] = {0.f, 0.f, 0.f};
              st3(FB + 5 * S4, t, z);
              st3(FB + 6 * S4, t, z);
              st3(FB + 7 * S4, t, z);
            }
          }
        }
      }
    }
    alive = grid_sum3<NT, double>(gs, nb, bid, epoch, 0.0, 0.0, 0.0, red);
    if (!alive) break;
    // ---- r = b - A x (FP64) by the owners; clear ax for the next sweep
    double prr = 0.0;
    p = 0;
    for (int64_t cb = cbase0; cb < F; cb += cstride, ++p) {
      const int64_t c = cb + cl;
      if (c >= F) continue;
      bool own = false;
      const int t = triple<NT, RES>(m.tri, s_tri, p, c, q, own);
      if (!own) continue;
      double bv[3], av[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) { bv[j] = __ldg(&b[3 * t + j]); av[j] = __ldcg(&w.ax[3 * t + j]); }
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int d = 3 * t + j;
        const double r = bv[j] - av[j];
        w.r64[d] = r;
        if (q < 3) w.ax[d] = 0.0;
        prr = fma(r, r, prr);
      }
    }
    alive = grid_sum3<NT, double>(gs, nb, bid, epoch, prr, 0.0, 0.0, red);
    rr64 = red[0];
    xcur ^= 1;
    have_x = true;
    rsrc = w.r64;
    if (!isfinite(rr64)) { bad = true; break; }
    conv = rr64 <= tol2;
  }
  if (threadIdx.x == 0 && bid == 0) {
    if (bad) atomicOr(w.flags, kFlagNonFinite);
    else if (alive && !conv) atomicOr(w.flags, kFlagNoConv);
  }
  // ---- out = scale_x x + add on owned DOFs
  const double* xfin = xcur ? w.x[1] : w.x[0];
  p = 0;
  for (int64_t cb = cbase0; cb < F; cb += cstride, ++p) {
    const int64_t c = cb + cl;
    if (c >= F) continue;
    bool own = false;
    const int t = triple<NT, RES>(m.tri, s_tri, p, c, q, own);
    if (!own) continue;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int d = 3 * t + j;
      double v = scale_x * (have_x ? __ldcg(&xfin[d]) : 0.0);
      if (add) v += __ldg(&add[d]);
      out[d] = v;
    }
  }
  if (threadIdx.x == 0 && bid == 0) {
    atomicAdd(&w.stats[0], 1ull);
    atomicAdd(&w.stats[1], (unsigned long long)inner_total);
    atomicMax(&w.stats[2], (unsigned long long)inner_total);
    atomicAdd(&w.stats[3], (unsigned long long)sweeps);
  }
  return alive && !bad;
}

}  // namespace
}  // namespace pavg
