// CUDA kernels of libpavg for sm_103a: the operators K-hat and N (FP64, and
// the FP32 variants of the mixed-precision mode), the shift/coefficient
// contractions, small vector kernels, and the FP64 Jacobi CG.
//
// Layout: per-cell data in structure-of-arrays form ([k][F]) so that a warp of
// consecutive cells reads consecutive addresses; element matrices carry the
// orientation signs, so gathered global DOF values are used as they are.
// Assembly of edge DOFs (shared by exactly two cells) uses atomicAdd into a
// zeroed buffer: with exactly two contributions, 0 + a + b == 0 + b + a in IEEE
// arithmetic, so the result does not depend on the order of arrival.
#include <cuda_runtime.h>

#include <type_traits>

#include "device.h"
#include "device_common.cuh"

namespace pavg {

__constant__ ConstTables c_tab;
__constant__ TablesT<float> c_tabf;

__constant__ TablesP3<double> c_tab3;
__constant__ TablesP3<float> c_tab3f;

cudaError_t upload_tables(const ConstTables& t) {
  cudaError_t e = cudaMemcpyToSymbol(c_tab, &t, sizeof(t));
  if (e != cudaSuccess) return e;
  const TablesT<float> f = tables_to_float(t);
  return cudaMemcpyToSymbol(c_tabf, &f, sizeof(f));
}

// The reference tables in the arithmetic type R (FP64, or the FP32 copy).
template <typename R>
__device__ __forceinline__ const TablesT<R>& tab();
template <>
__device__ __forceinline__ const TablesT<double>& tab<double>() { return c_tab; }
template <>
__device__ __forceinline__ const TablesT<float>& tab<float>() { return c_tabf; }

cudaError_t upload_tables3(const TablesP3<double>& t) {
  cudaError_t e = cudaMemcpyToSymbol(c_tab3, &t, sizeof(t));
  if (e != cudaSuccess) return e;
  const TablesP3<float> f = tables_to_float(t);
  return cudaMemcpyToSymbol(c_tab3f, &f, sizeof(f));
}

namespace {


constexpr int kCgThreads = 256;

// Persistent conjugate gradients on M1 (Jacobi preconditioner), in the
// single-reduction form of Chronopoulos and Gear: one grid barrier per
// iteration.  M1 is applied cell by cell from the element matrices; the
// inner products use u^T A u = sum_K u_K^T A_K u_K, so no assembled product is
// needed before the reduction.  Every DOF has one owner cell (interior DOFs:
// their cell; edge DOFs: the cell that runs the edge low -> high), which alone
// writes its per-DOF vectors; shared values are recomputed identically by both
// cells from double-buffered inputs.
__global__ void __launch_bounds__(kCgThreads) k_cg(DeviceMesh m, CgWork w, CgParams cp,
                                                   const double* __restrict__ b, double* out,
                                                   double scale_x, const double* __restrict__ add) {
  __shared__ double sc[3];
  const int64_t F = m.F;
  const int64_t nE = 3 * m.E;
  const int nb = gridDim.x;
  const int64_t g0 = (int64_t)blockIdx.x * kCgThreads + threadIdx.x;
  const int64_t gs = (int64_t)nb * kCgThreads;
  double pg = 0, pd = 0, pr = 0;

  // ---- initial residual r0 = b (x0 = 0), u0 = P r0, w0 = A u0 into w[0]
  for (int64_t c = g0; c < F; c += gs) {
    int dof[12];
    double sg[12];
    unsigned al = cell_dofs(m, c, dof, sg);
    double u[12], wl[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) u[k] = __ldg(&m.dinv[dof[k]]) * __ldg(&b[dof[k]]);
    spmv_cell(m.M1, F, c, u, wl);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      pd = fma(u[k], wl[k], pd);
      if (k < 9) atomicAdd(&w.w[0][dof[k]], wl[k]);
      else w.w[0][dof[k]] = wl[k];
      bool own = k >= 9 || ((al >> (k / 3)) & 1u);
      if (own) {
        double r0 = __ldg(&b[dof[k]]);
        w.r[0][dof[k]] = r0;
        pg = fma(r0, u[k], pg);
        pr = fma(r0, r0, pr);
        if (k < 9) w.w[1][dof[k]] = 0.0;
      }
    }
  }
  // The partials are double-buffered: a block may write the next round's
  // partial before a slower block has finished reading this round's.
  {
    double s3[3];
    block_sum3<kCgThreads>(pg, pd, pr, s3);
    if (threadIdx.x == 0) {
      w.partial[blockIdx.x] = s3[0];
      w.partial[nb + blockIdx.x] = s3[1];
      w.partial[2 * nb + blockIdx.x] = s3[2];
    }
  }
  bool alive = grid_barrier(w.bar, w.flags);
  {
    double t[3];
    reduce_partials<kCgThreads>(w.partial, nb, t);
    if (threadIdx.x == 0) { sc[0] = t[0]; sc[1] = t[1]; sc[2] = t[2]; }
    __syncthreads();
  }
  double gamma = sc[0], delta = sc[1];
  const double bb = sc[2];
  const double tol2 = cp.rtol * cp.rtol * bb;
  double alpha = gamma / delta, beta = 0.0;
  int it = 0;
  bool done = !(bb > 0.0);
  bool have_x = false;
  if (!isfinite(bb) || (!done && !isfinite(alpha))) {
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(w.flags, kFlagNonFinite);
    done = true;
  }
  for (; alive && !done && it < cp.maxit; ++it) {
    const int i = it;
    const double* rin = (i & 1) ? w.r[1] : w.r[0];
    double* rout = (i & 1) ? w.r[0] : w.r[1];
    const double* sin_ = (i & 1) ? w.s[0] : w.s[1];
    double* sout = (i & 1) ? w.s[1] : w.s[0];
    const int i3 = i % 3;
    const double* win = i3 == 0 ? w.w[0] : (i3 == 1 ? w.w[1] : w.w[2]);
    double* wacc = i3 == 0 ? w.w[1] : (i3 == 1 ? w.w[2] : w.w[0]);
    double* wzero = i3 == 0 ? w.w[2] : (i3 == 1 ? w.w[0] : w.w[1]);
    pg = pd = pr = 0.0;
    for (int64_t c = g0; c < F; c += gs) {
      int dof[12];
      double sg[12];
      unsigned al = cell_dofs(m, c, dof, sg);
      double u[12], wl[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const int d = dof[k];
        const double rold = __ldcg(&rin[d]);
        const double winv = __ldcg(&win[d]);
        const double s_i = i > 0 ? fma(beta, __ldcg(&sin_[d]), winv) : winv;
        const double rn = fma(-alpha, s_i, rold);
        const double dv = __ldg(&m.dinv[d]);
        u[k] = dv * rn;
        const bool own = k >= 9 || ((al >> (k / 3)) & 1u);
        if (own) {
          sout[d] = s_i;
          rout[d] = rn;
          const double ui = dv * rold;
          const double pv = i > 0 ? fma(beta, __ldcg(&w.p[d]), ui) : ui;
          w.p[d] = pv;
          w.x[d] = i > 0 ? fma(alpha, pv, __ldcg(&w.x[d])) : alpha * pv;
          if (k < 9) wzero[d] = 0.0;
          pg = fma(rn, u[k], pg);
          pr = fma(rn, rn, pr);
        }
      }
      spmv_cell(m.M1, F, c, u, wl);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        pd = fma(u[k], wl[k], pd);
        if (k < 9) atomicAdd(&wacc[dof[k]], wl[k]);
        else wacc[dof[k]] = wl[k];
      }
    }
    have_x = true;
    double s3[3];
    double* part = w.partial + ((i + 1) & 1) * 3 * nb;
    block_sum3<kCgThreads>(pg, pd, pr, s3);
    if (threadIdx.x == 0) {
      part[blockIdx.x] = s3[0];
      part[nb + blockIdx.x] = s3[1];
      part[2 * nb + blockIdx.x] = s3[2];
    }
    alive = grid_barrier(w.bar, w.flags);
    double t[3];
    reduce_partials<kCgThreads>(part, nb, t);
    if (threadIdx.x == 0) { sc[0] = t[0]; sc[1] = t[1]; sc[2] = t[2]; }
    __syncthreads();
    const double gnew = sc[0], dnew = sc[1], rr = sc[2];
    if (!(isfinite(gnew) && isfinite(dnew) && isfinite(rr))) {
      if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(w.flags, kFlagNonFinite);
      ++it;
      break;
    }
    if (rr <= tol2) { ++it; done = true; break; }
    double bnew = gnew / gamma;
    alpha = gnew / (dnew - bnew * gnew / alpha);
    beta = bnew;
    gamma = gnew;
  }
  if (alive && !done && it >= cp.maxit && threadIdx.x == 0 && blockIdx.x == 0) atomicOr(w.flags, kFlagNoConv);
  // ---- out = scale_x x + add on owned DOFs
  for (int64_t c = g0; c < F; c += gs) {
    int dof[12];
    double sg[12];
    unsigned al = cell_dofs(m, c, dof, sg);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      bool own = k >= 9 || ((al >> (k / 3)) & 1u);
      if (!own) continue;
      const int d = dof[k];
      double xv = have_x ? __ldcg(&w.x[d]) : 0.0;
      double v = scale_x * xv;
      if (add) v += __ldg(&add[d]);
      out[d] = v;
    }
  }
  (void)nE;
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    atomicAdd(&w.stats[0], 1ull);
    atomicAdd(&w.stats[1], (unsigned long long)it);
    atomicMax(&w.stats[2], (unsigned long long)it);
  }
}

// Entry (k, l) of a cell's symmetric 3 x 3 matrix stored packed 00, 01, 02,
// 11, 12, 22 in structure-of-arrays form [6][F] (k, l compile-time constants
// in unrolled loops).
__device__ __forceinline__ double sym3(const double* __restrict__ P, int64_t F, int64_t c, int k, int l) {
  const int a = k < l ? k : l, b = k < l ? l : k;
  const int idx = a == 0 ? b : (a == 1 ? 2 + b : 5);
  return __ldg(&P[idx * F + c]);
}

// ru = y_u + s (-C u + g D^T eta);  eta_out = M2^{-1}(y_eta + s (-H D u)) + z_eta.
// T: the arithmetic of the K-hat products (double; float in the mixed mode,
// with the FP32 copy of C): the additions of y and z, the M2 inverse and the
// outputs stay FP64 (they are the recurrences' own terms).
template <typename T>
__global__ void __launch_bounds__(128) k_apply_K(DeviceMesh m, const double* __restrict__ U, double s,
                                                 double g, double H, const double* __restrict__ y_u,
                                                 const double* __restrict__ y_eta,
                                                 const double* __restrict__ z_eta, double* ru,
                                                 double* eta_out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m.F) return;
  const int64_t F = m.F;
  const TablesT<T>& TT = tab<T>();
  int dof[12];
  double sg[12];
  unsigned al = cell_dofs(m, c, dof, sg);
  T u[12], r[12], eta[3];
#pragma unroll
  for (int k = 0; k < 12; ++k) { u[k] = (T)__ldg(&U[dof[k]]); r[k] = T(0); }
#pragma unroll
  for (int k = 0; k < 3; ++k) eta[k] = (T)__ldg(&U[m.n_u + 3 * c + k]);
#pragma unroll
  for (int i = 0; i < 12; ++i) {
#pragma unroll
    for (int j = i + 1; j < 12; ++j) {
      T a;
      if constexpr (std::is_same<T, double>::value) a = __ldg(&m.C[pasym(i, j) * F + c]);
      else a = __ldg(&m.Cf[pasym(i, j) * F + c]);
      r[i] = fma(-a, u[j], r[i]);
      r[j] = fma(a, u[i], r[j]);
    }
  }
  // the orientation signs are +-1: applied as sign flips of the operands
  // (exact, and no multiplications), the same numbers as D_ki sg_i u_i
  T us[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) us[i] = sg[i] < 0.0 ? -u[i] : u[i];
  T Du[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    T t = T(0);
#pragma unroll
    for (int i = 0; i < 12; ++i) t = fma(TT.D[k][i], us[i], t);
    Du[k] = t;
  }
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    T t = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) t = fma(TT.D[k][i], eta[k], t);
    double v = (double)((T)s * fma((T)g, sg[i] < 0.0 ? -t : t, r[i]));
    bool own = i >= 9 || ((al >> (i / 3)) & 1u);
    if (own && y_u) v += __ldg(&y_u[dof[i]]);
    if (i < 9) atomicAdd(&ru[dof[i]], v);
    else ru[dof[i]] = v;
  }
  double rl[3];
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    rl[l] = (double)((T)s * (-(T)H * Du[l]));
    if (y_eta) rl[l] += __ldg(&y_eta[3 * c + l]);
  }
  if (m.M2i) {  // cubic cells: the cell's own M2^{-1}
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double v = 0.0;
#pragma unroll
      for (int l = 0; l < 3; ++l) v = fma(sym3(m.M2i, F, c, k, l), rl[l], v);
      if (z_eta) v += __ldg(&z_eta[3 * c + k]);
      eta_out[3 * c + k] = v;
    }
    return;
  }
  const double idet = 1.0 / m.det[c];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double v = 0.0;
#pragma unroll
    for (int l = 0; l < 3; ++l) v = fma(c_tab.M2inv_ref[k][l], rl[l], v);
    v *= idet;
    if (z_eta) v += __ldg(&z_eta[3 * c + k]);
    eta_out[3 * c + k] = v;
  }
}

// ------------------------------------------------------------------ nonlinear operator
// Arithmetic type R: double (FP64 path) or float (mixed precision, where each
// quadrature point's contribution is formed in FP32 and the sums over the
// quadrature points are accumulated in FP64).
template <typename R>
__device__ __forceinline__ const TablesP3<R>& tab3();
template <>
__device__ __forceinline__ const TablesP3<double>& tab3<double>() { return c_tab3; }
template <>
__device__ __forceinline__ const TablesP3<float>& tab3<float>() { return c_tab3f; }
// the nonlinear kernels' tables for geometry degree GEO
template <typename R, int GEO>
__device__ __forceinline__ const auto& ntab() {
  if constexpr (GEO == 3) return tab3<R>();
  else return tab<R>();
}

// Explicitly rounded operations (never contracted or reordered by the compiler).
template <typename R>
struct Rn;
template <>
struct Rn<double> {
  static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
};
template <>
struct Rn<float> {
  static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
};

template <typename R>
struct Side {
  R c[12];   // signed local coefficients
  R h[3];    // eta - b at the local vertices
  R det, G00, G01, G11;
  R dv[3];   // div_hat u_hat at the local vertices, formed in FP64 (strong form of the elevation terms)
};

template <typename R>
__device__ __forceinline__ void load_side(const DeviceMesh& m, const double* __restrict__ U, int64_t cell,
                                          Side<R>& S) {
  int dof[12];
  double sg[12];
  cell_dofs(m, cell, dof, sg);
  double cd[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const double v = __ldg(&U[dof[k]]);
    cd[k] = sg[k] < 0.0 ? -v : v;  // orientation sign (+-1) as a sign flip
    S.c[k] = (R)cd[k];
  }
  {
    // the divergence of a nearly divergence-free field is a cancelling sum of
    // edge fluxes: form it from the FP64 coefficients
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      double d = 0.0;
#pragma unroll
      for (int k = 0; k < 12; ++k) d = fma(cd[k], c_tab.div_vert[k][v], d);
      S.dv[v] = (R)d;
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) S.h[k] = (R)(__ldg(&U[m.n_u + 3 * cell + k]) - __ldg(&m.topo[3 * cell + k]));
  S.det = (R)__ldg(&m.det[cell]);
  S.G00 = (R)__ldg(&m.G[cell]);
  S.G01 = (R)__ldg(&m.G[m.F + cell]);
  S.G11 = (R)__ldg(&m.G[2 * m.F + cell]);
}

// One side's metric at a facet point: the cell's constant one on flat cells,
// the cubic map's at the point otherwise.
template <typename R>
struct SideGeom {
  R G00, G01, G11, inv_det;  // J^T J and 1 / det
};

template <typename R>
struct FacetValues {
  R flux;     // u+ . n+ ds / dtau
  R tan;      // |e| (t . u~)
  R hup;      // (eta - b)~
  R hp, hm;   // eta - b on each side
  R up0, up1, um0, um1;
};

// Values shared by the two cells of a facet at point p (formed once per edge
// and point, for both cells).  Upwind: the side the flow leaves (flux > 0:
// plus); the printed rule of Sec. 2.5 (u~ = u+ when u . n+ < 0) is the
// alternative for the velocity.
template <typename R, typename TT>
__device__ __forceinline__ FacetValues<R> facet_point(const TT& T, const Side<R>& P, const SideGeom<R>& gP, int lp,
                                                      const Side<R>& Mn, const SideGeom<R>& gM, int lm, int p,
                                                      int upwind) {
  using O = Rn<R>;
  FacetValues<R> f;
  R a0 = 0, a1 = 0, b0 = 0, b1 = 0, hp = 0, hm = 0;
#pragma unroll
  for (int j = 0; j < 12; ++j) {
    a0 = O::fma(P.c[j], T.fq_psi[0][lp][p][j][0], a0);
    a1 = O::fma(P.c[j], T.fq_psi[0][lp][p][j][1], a1);
    b0 = O::fma(Mn.c[j], T.fq_psi[1][lm][p][j][0], b0);
    b1 = O::fma(Mn.c[j], T.fq_psi[1][lm][p][j][1], b1);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    hp = O::fma(P.h[k], T.fq_phi[0][lp][p][k], hp);
    hm = O::fma(Mn.h[k], T.fq_phi[1][lm][p][k], hm);
  }
  const R dp0 = T.edge_dir[lp][0], dp1 = T.edge_dir[lp][1];
  const R dm0 = T.edge_dir[lm][0], dm1 = T.edge_dir[lm][1];
  const R flux = O::sub(O::mul(a0, dp1), O::mul(a1, dp0));
  const bool plus_up = flux > R(0);
  const bool plus_up_vel = upwind == PAVG_UPWIND_STANDARD ? plus_up : (flux < R(0));
  R tan;
  if (plus_up_vel) {
    R g0 = O::fma(gP.G00, a0, O::mul(gP.G01, a1));
    R g1 = O::fma(gP.G01, a0, O::mul(gP.G11, a1));
    tan = O::mul(O::fma(dp0, g0, O::mul(dp1, g1)), gP.inv_det);
  } else {
    R g0 = O::fma(gM.G00, b0, O::mul(gM.G01, b1));
    R g1 = O::fma(gM.G01, b0, O::mul(gM.G11, b1));
    tan = -O::mul(O::fma(dm0, g0, O::mul(dm1, g1)), gM.inv_det);
  }
  f.flux = flux;
  f.tan = tan;
  f.hup = plus_up ? hp : hm;
  f.hp = hp;
  f.hm = hm;
  f.up0 = a0; f.up1 = a1; f.um0 = b0; f.um1 = b1;
  return f;
}

// Facet terms of N (Sec. 2.5) for one edge and one state, for both of its
// cells at once: at each of the edge's quadrature points the upwinded values
// are formed once (facet_point), and each side's contributions
//   r_j  -= / += w (u_perp . w_j) (t . u~)      (velocity tests of that side)
//   re_k -/+ w phi_k (u . n+) ((eta - b)_side - (eta - b)~)   (elevation tests, strong form)
// are summed over the points in FP64 and stored in the side's slot
// FR[cell][local edge][15] (each slot written by exactly one edge).
// GEO = 1: flat cells (4 points, each cell's constant metric); GEO = 3: the
// piecewise cubic surface (5 points, each side's metric at the point, from
// m.geo_f), where the scale factor of the velocity term is 1 / det of the
// side at the point.
template <typename R, int GEO>
__global__ void __launch_bounds__(128) k_facets(DeviceMesh m, const double* __restrict__ Uall, double* FRall,
                                                int upwind) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.E) return;
  constexpr int NQ = GEO == 3 ? kFacetQ3 : kFacetQ;
  const auto& T = ntab<R, GEO>();
  constexpr bool kStrongDG = true;  // both precisions: see k_nonlinear
  const double* U = Uall + (int64_t)blockIdx.y * m.n;
  double* FR = FRall + (int64_t)blockIdx.y * m.F * 45;
  const int64_t cp = m.edge_plus[e], cm = m.edge_minus[e];
  const unsigned lpos = m.edge_lpos[e];
  const int lp = (int)(lpos & 3u), lm = (int)(lpos >> 2);
  Side<R> P, Mn;
  load_side(m, U, cp, P);
  load_side(m, U, cm, Mn);
  double rp[12], rm[12], ep[3] = {0.0, 0.0, 0.0}, em[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int j = 0; j < 12; ++j) rp[j] = rm[j] = 0.0;
  R inv_p = R(0), inv_m = R(0);  // flat cells: one reciprocal per side and edge
  if constexpr (GEO != 3) {
    inv_p = R(1) / P.det;
    inv_m = R(1) / Mn.det;
  }
#pragma unroll 1
  for (int p = 0; p < NQ; ++p) {
    const R wp = T.fq_w[p];
    SideGeom<R> gP, gM;
    if constexpr (GEO == 3) {
      const int64_t PE = (int64_t)NQ * m.E, o = (int64_t)p * m.E + e;
      gP = {(R)__ldg(&m.geo_f[0 * PE + o]), (R)__ldg(&m.geo_f[1 * PE + o]), (R)__ldg(&m.geo_f[2 * PE + o]),
            (R)__ldg(&m.geo_f[3 * PE + o])};
      gM = {(R)__ldg(&m.geo_f[4 * PE + o]), (R)__ldg(&m.geo_f[5 * PE + o]), (R)__ldg(&m.geo_f[6 * PE + o]),
            (R)__ldg(&m.geo_f[7 * PE + o])};
    } else {
      gP = {P.G00, P.G01, P.G11, inv_p};
      gM = {Mn.G00, Mn.G01, Mn.G11, inv_m};
    }
    const FacetValues<R> f = facet_point(T, P, gP, lp, Mn, gM, lm, p, upwind);
    // u_perp . w_j = cross2(u_hat, psi_j) / det on each side, times w (t . u~)
    const R tw = wp * f.tan;
    const R scp = -tw * gP.inv_det, scm = tw * gM.inv_det;
    const R Ap = scp * f.up0, Bp = scp * f.up1, Am = scm * f.um0, Bm = scm * f.um1;
#pragma unroll
    for (int j = 0; j < 12; ++j) {
      const R* qp = T.fq_psi[0][lp][p][j];
      const R* qm = T.fq_psi[1][lm][p][j];
      if constexpr (std::is_same<R, double>::value) {
        rp[j] = fma(Ap, qp[1], fma(-Bp, qp[0], rp[j]));
        rm[j] = fma(Am, qm[1], fma(-Bm, qm[0], rm[j]));
      } else {  // FP32 contributions, FP64 sums over the points
        rp[j] += (double)fmaf(Ap, qp[1], -Bp * qp[0]);
        rm[j] += (double)fmaf(Am, qm[1], -Bm * qm[0]);
      }
    }
    const R fhp = kStrongDG ? wp * f.flux * (f.hp - f.hup) : -wp * f.flux * f.hup;
    const R fhm = kStrongDG ? wp * f.flux * (f.hup - f.hm) : wp * f.flux * f.hup;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      ep[k] += (double)(fhp * T.fq_phi[0][lp][p][k]);
      em[k] += (double)(fhm * T.fq_phi[1][lm][p][k]);
    }
  }
  double* sp = FR + (cp * 3 + lp) * 15;
  double* sm = FR + (cm * 3 + lm) * 15;
#pragma unroll
  for (int j = 0; j < 12; ++j) { sp[j] = rp[j]; sm[j] = rm[j]; }
#pragma unroll
  for (int k = 0; k < 3; ++k) { sp[12 + k] = ep[k]; sm[12 + k] = em[k]; }
}

// Weak-form right-hand side of N (Sec. 2.5) for one cell and one state:
//   r_i  = int_K [u . grad_perp(u_perp . w_i) + div w_i |u|^2/2]
//          - int_dK (+/-) (u_perp . w_i) (t . u~)          (velocity test w_i)
//   re_k = int_K grad phi_k . u (eta - b) -/+ int_dK phi_k (u . n+) (eta - b)~
// The cell integrand in reference form is, with v = G u_hat and the
// derivative d_tau = v1 d/dx - v0 d/dy:
//   [d_tau cross2(u_hat, psi_i) + div psi_i (u_hat . v) / 2] / det^2.
// This kernel forms the cell integrals and adds the facet integrals that
// k_facets stored for the cell's three edges.  Sums over quadrature points
// are accumulated in FP64.
// The elevation terms use the equivalent strong form
//   re_k = -int_K phi_k div(u (eta - b)) + int_dK phi_k (u . n) ((eta - b)_own - (eta - b)~),
// identical under exact integration (the divergence theorem on each cell;
// the integrands are polynomials, of degree 3 in the cell and 4 on a facet,
// integrated exactly), which avoids the cancellation between the cell and
// facet terms of the weak form (both grow like 1 / h while their sum does
// not).  In FP64 that cancellation cost about two decimal digits of the
// elevation part of N on balanced states at refinement 6; in FP32 all of
// them.
//
// GEO = 3, the piecewise cubic surface: J, det and G vary over the cell and
// the integrand gains the term of d_tau det (the derivative of 1 / det in
// u_perp . w_i = cross2(u_hat, psi_i) / det):
//   w / det^2 [d_tau cross2(u_hat, psi_i) - cross2(u_hat, psi_i) d_tau det / det
//              + div psi_i (u_hat . v) / 2],
// with G, w / det^2 and grad_hat det / det per point from m.geo_c and the
// 25-point Stroud rule.  The elevation terms do not involve the geometry.
template <typename R, int GEO>
__global__ void __launch_bounds__(128) k_nonlinear(DeviceMesh m, const double* __restrict__ Uall, double* Rall,
                                                   const double* __restrict__ FRall) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m.F) return;
  constexpr int NQ = GEO == 3 ? kCellQ3 : kCellQ;
  const auto& T = ntab<R, GEO>();
  constexpr bool kStrongDG = true;  // both precisions: see k_nonlinear
  const int64_t n = m.n;
  const double* U = Uall + (int64_t)blockIdx.y * n;
  double* Rout = Rall + (int64_t)blockIdx.y * n;
  Side<R> own;
  load_side(m, U, c, own);
  double r[12], re[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int i = 0; i < 12; ++i) r[i] = 0.0;
  // ---- cell terms
#pragma unroll 1
  for (int q = 0; q < NQ; ++q) {
    R u0 = 0, u1 = 0, d00 = 0, d01 = 0, d10 = 0, d11 = 0;  // d_ca = d u_c / d x_a
#pragma unroll
    for (int j = 0; j < 12; ++j) {
      const R cj = own.c[j];
      u0 = fma(cj, T.cq_psi[q][j][0], u0);
      u1 = fma(cj, T.cq_psi[q][j][1], u1);
      d00 = fma(cj, T.cq_dpsi[q][j][0][0], d00);
      d01 = fma(cj, T.cq_dpsi[q][j][0][1], d01);
      d10 = fma(cj, T.cq_dpsi[q][j][1][0], d10);
      d11 = fma(cj, T.cq_dpsi[q][j][1][1], d11);
    }
    const R h = own.h[0] * T.cq_phi[q][0] + own.h[1] * T.cq_phi[q][1] + own.h[2] * T.cq_phi[q][2];
    R G00, G01, G11, W;
    R tx = 0, ty = 0;  // grad_hat det / det (cubic cells)
    if constexpr (GEO == 3) {
      const int64_t QF = (int64_t)NQ * m.F, o = (int64_t)q * m.F + c;
      G00 = (R)__ldg(&m.geo_c[0 * QF + o]);
      G01 = (R)__ldg(&m.geo_c[1 * QF + o]);
      G11 = (R)__ldg(&m.geo_c[2 * QF + o]);
      W = (R)__ldg(&m.geo_c[3 * QF + o]);
      tx = (R)__ldg(&m.geo_c[4 * QF + o]);
      ty = (R)__ldg(&m.geo_c[5 * QF + o]);
    } else {
      G00 = own.G00;
      G01 = own.G01;
      G11 = own.G11;
      W = T.cq_w[q];
    }
    const R v0 = G00 * u0 + G01 * u1;
    const R v1 = G01 * u0 + G11 * u1;
    const R wq = T.cq_w[q];
    const R half_ke = R(0.5) * (u0 * v0 + u1 * v1);
    R t0 = v1 * d00 - v0 * d01;  // d_tau u_hat
    R t1 = v1 * d10 - v0 * d11;
    if constexpr (GEO == 3) {  // - cross2(u_hat, psi_i) d_tau det / det
      const R tau = v1 * tx - v0 * ty;
      t0 -= u0 * tau;
      t1 -= u1 * tau;
    }
    // coefficients of psi_i0, psi_i1, d0 psi_i0, d1 psi_i0, d0 psi_i1, d1 psi_i1
    const R k0 = -t1 * W, k1 = t0 * W;
    const R k2 = (-u1 * v1 + half_ke) * W, k3 = (u1 * v0) * W;
    const R k4 = (u0 * v1) * W, k5 = (-u0 * v0 + half_ke) * W;
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      if constexpr (std::is_same<R, double>::value) {  // straight into the point sum
        double t = fma(k0, T.cq_psi[q][i][0], r[i]);
        t = fma(k1, T.cq_psi[q][i][1], t);
        t = fma(k2, T.cq_dpsi[q][i][0][0], t);
        t = fma(k3, T.cq_dpsi[q][i][0][1], t);
        t = fma(k4, T.cq_dpsi[q][i][1][0], t);
        r[i] = fma(k5, T.cq_dpsi[q][i][1][1], t);
      } else {  // FP32 contribution of the point, FP64 sum over the points
        R t = k0 * T.cq_psi[q][i][0];
        t = fma(k1, T.cq_psi[q][i][1], t);
        t = fma(k2, T.cq_dpsi[q][i][0][0], t);
        t = fma(k3, T.cq_dpsi[q][i][0][1], t);
        t = fma(k4, T.cq_dpsi[q][i][1][0], t);
        t = fma(k5, T.cq_dpsi[q][i][1][1], t);
        r[i] += (double)t;
      }
    }
    if (kStrongDG) {
      // div_hat(u_hat h_hat) = h_hat (d00 + d11) + u_hat . grad_hat h_hat (DG1: constant gradient)
      const R divu = own.dv[0] * T.cq_phi[q][0] + own.dv[1] * T.cq_phi[q][1] + own.dv[2] * T.cq_phi[q][2];
      const R g = h * divu + u0 * (own.h[1] - own.h[0]) + u1 * (own.h[2] - own.h[0]);
      const R gw = g * wq;
#pragma unroll
      for (int k = 0; k < 3; ++k) re[k] -= (double)(gw * T.cq_phi[q][k]);
    } else {
      const R hw = h * wq;
      re[0] -= (double)((u0 + u1) * hw);
      re[1] += (double)(u0 * hw);
      re[2] += (double)(u1 * hw);
    }
  }
  if constexpr (GEO != 3) {  // flat cells: the constant 1 / det^2 (per point on cubic cells)
    const double idet2 = 1.0 / ((double)own.det * (double)own.det);
#pragma unroll
    for (int i = 0; i < 12; ++i) r[i] *= idet2;
  }
  // ---- facet terms, evaluated once per edge by k_facets (slots [c][local edge][15])
  const double* FR = FRall + ((int64_t)blockIdx.y * m.F + c) * 45;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 12; ++j) r[j] += __ldcg(&FR[15 * i + j]);
#pragma unroll
    for (int k = 0; k < 3; ++k) re[k] += __ldcg(&FR[15 * i + 12 + k]);
  }
  // ---- to global numbering
  int dof[12];
  double sg[12];
  cell_dofs(m, c, dof, sg);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    double v = sg[k] < 0.0 ? -r[k] : r[k];  // orientation sign as a sign flip
    if (k < 9) atomicAdd(&Rout[dof[k]], v);
    else Rout[dof[k]] = v;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) Rout[m.n_u + 3 * c + k] = re[k];
}

__global__ void k_m2inv(DeviceMesh m, const double* __restrict__ r, int64_t rstride, double* out,
                        int64_t ostride) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m.F) return;
  const double* rb = r + blockIdx.y * rstride;
  double* ob = out + blockIdx.y * ostride;
  double v[3];
#pragma unroll
  for (int l = 0; l < 3; ++l) v[l] = rb[3 * c + l];
  if (m.M2i) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double t = 0.0;
#pragma unroll
      for (int l = 0; l < 3; ++l) t = fma(sym3(m.M2i, m.F, c, k, l), v[l], t);
      ob[3 * c + k] = t;
    }
    return;
  }
  const double idet = 1.0 / m.det[c];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double t = 0.0;
#pragma unroll
    for (int l = 0; l < 3; ++l) t = fma(c_tab.M2inv_ref[k][l], v[l], t);
    ob[3 * c + k] = t * idet;
  }
}

// out[m][j] = sum_k A[m][k] in[k][j]; MT output rows per block row, whose
// nonzero k range is k < lim[tile] when lim is given.  TA: accumulation type
// (double on the FP64 path, float in mixed precision).
template <int MT, typename TA>
__global__ void __launch_bounds__(256) k_combine(const double* __restrict__ A, int Mo, int Ki,
                                                 const int* __restrict__ lim, const double* __restrict__ in,
                                                 int64_t in_stride, double* out, int64_t out_stride, int64_t len) {
  extern __shared__ __align__(16) unsigned char sA_raw[];
  TA* sA = reinterpret_cast<TA*>(sA_raw);  // [MT][Ki]
  const int m0 = blockIdx.y * MT;
  const int kn = lim ? lim[blockIdx.y] : Ki;
  for (int t = threadIdx.x; t < MT * Ki; t += blockDim.x) {
    int mm = m0 + t / Ki, k = t % Ki;
    sA[t] = mm < Mo ? (TA)A[(int64_t)mm * Ki + k] : TA(0);
  }
  __syncthreads();
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < len; j += (int64_t)gridDim.x * blockDim.x) {
    TA acc[MT];
#pragma unroll
    for (int t = 0; t < MT; ++t) acc[t] = TA(0);
    for (int k = 0; k < kn; ++k) {
      const TA v = (TA)__ldg(&in[(int64_t)k * in_stride + j]);
#pragma unroll
      for (int t = 0; t < MT; ++t) acc[t] = fma(sA[t * Ki + k], v, acc[t]);
    }
#pragma unroll
    for (int t = 0; t < MT; ++t)
      if (m0 + t < Mo) out[(int64_t)(m0 + t) * out_stride + j] = (double)acc[t];
  }
}

// The same contractions when the shifts come in pairs +s, -s with equal
// coefficients c_k(lam |s|) and weights (a symmetric rule): for pair p,
//   E_p = sum_{k even} c_pk Q_k,  O_p = sum_{k odd} c_pk Q_k,
//   U_{2p} = E_p + O_p (s > 0),  U_{2p+1} = E_p - O_p (s < 0),
// one multiply-add per pair and k instead of one per shift and k.  A is
// [P][Ki] (c_pk), lim[t] the k range of pair tile t.
template <int MT, typename TA>
__global__ void __launch_bounds__(256) k_combine_pairs_fwd(const double* __restrict__ A, int P, int Ki,
                                                           const int* __restrict__ lim, const double* __restrict__ in,
                                                           int64_t in_stride, double* out, int64_t out_stride,
                                                           int64_t len) {
  extern __shared__ __align__(16) unsigned char sA_raw[];
  TA* sA = reinterpret_cast<TA*>(sA_raw);  // [MT][Ki]
  const int p0 = blockIdx.y * MT;
  const int kn = lim ? lim[blockIdx.y] : Ki;
  for (int t = threadIdx.x; t < MT * Ki; t += blockDim.x) {
    int pp = p0 + t / Ki, k = t % Ki;
    sA[t] = pp < P ? (TA)A[(int64_t)pp * Ki + k] : TA(0);
  }
  __syncthreads();
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < len; j += (int64_t)gridDim.x * blockDim.x) {
    TA e[MT], o[MT];
#pragma unroll
    for (int t = 0; t < MT; ++t) { e[t] = TA(0); o[t] = TA(0); }
    int k = 0;
    for (; k + 1 < kn; k += 2) {
      const TA v0 = (TA)__ldg(&in[(int64_t)k * in_stride + j]);
      const TA v1 = (TA)__ldg(&in[(int64_t)(k + 1) * in_stride + j]);
#pragma unroll
      for (int t = 0; t < MT; ++t) {
        e[t] = fma(sA[t * Ki + k], v0, e[t]);
        o[t] = fma(sA[t * Ki + k + 1], v1, o[t]);
      }
    }
    if (k < kn) {
      const TA v0 = (TA)__ldg(&in[(int64_t)k * in_stride + j]);
#pragma unroll
      for (int t = 0; t < MT; ++t) e[t] = fma(sA[t * Ki + k], v0, e[t]);
    }
#pragma unroll
    for (int t = 0; t < MT; ++t)
      if (p0 + t < P) {
        out[(int64_t)(2 * (p0 + t)) * out_stride + j] = (double)(e[t] + o[t]);
        out[(int64_t)(2 * (p0 + t) + 1) * out_stride + j] = (double)(e[t] - o[t]);
      }
  }
}

// Backward contraction over pairs: y_k = sum_p B_kp (k even ? S_p : D_p) with
// S_p = r_{2p+1} + r_{2p}, D_p = r_{2p+1} - r_{2p} (B_kp = w_p c_pk; the
// pair's +s member carries (-1)^k, its -s member 1).  B is [Ko][P], lim[t]
// the number of pairs of row tile t with a nonzero entry; MT is even, so the
// parity of row k0 + t is that of t.
template <int MT>
__global__ void __launch_bounds__(256) k_combine_pairs_bwd(const double* __restrict__ B, int Ko, int P,
                                                           const int* __restrict__ lim, const double* __restrict__ R,
                                                           int64_t r_stride, double* out, int64_t out_stride,
                                                           int64_t len) {
  static_assert(MT % 2 == 0, "row tiles start at even k");
  extern __shared__ __align__(16) unsigned char sB_raw[];
  double* sB = reinterpret_cast<double*>(sB_raw);  // [MT][P]
  const int k0 = blockIdx.y * MT;
  const int pn = lim ? lim[blockIdx.y] : P;
  for (int t = threadIdx.x; t < MT * P; t += blockDim.x) {
    int kk = k0 + t / P, pp = t % P;
    sB[t] = kk < Ko ? B[(int64_t)kk * P + pp] : 0.0;
  }
  __syncthreads();
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < len; j += (int64_t)gridDim.x * blockDim.x) {
    double acc[MT];
#pragma unroll
    for (int t = 0; t < MT; ++t) acc[t] = 0.0;
    for (int pp = 0; pp < pn; ++pp) {
      const double rp = __ldg(&R[(int64_t)(2 * pp) * r_stride + j]);
      const double rm = __ldg(&R[(int64_t)(2 * pp + 1) * r_stride + j]);
      const double S = rm + rp, D = rm - rp;
#pragma unroll
      for (int t = 0; t < MT; ++t) acc[t] = fma(sB[t * P + pp], (t & 1) ? D : S, acc[t]);
    }
#pragma unroll
    for (int t = 0; t < MT; ++t)
      if (k0 + t < Ko) out[(int64_t)(k0 + t) * out_stride + j] = acc[t];
  }
}

__global__ void k_lincomb(double* out, double a, const double* __restrict__ x, double b,
                          const double* __restrict__ y, double c, const double* __restrict__ z, int64_t len) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < len; j += (int64_t)gridDim.x * blockDim.x) {
    double v = a * x[j];
    if (y) v = fma(b, y[j], v);
    if (z) v = fma(c, z[j], v);
    out[j] = v;
  }
}

__global__ void __launch_bounds__(256) k_winner(DeviceMesh m, const double* __restrict__ U,
                                                const double* __restrict__ V, double g, double H,
                                                double* part) {
  double acc = 0.0;
  for (int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x; c < m.F; c += (int64_t)gridDim.x * 256) {
    int dof[12];
    double sg[12];
    cell_dofs(m, c, dof, sg);
    double u[12], v[12], w[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) { u[k] = U[dof[k]]; v[k] = V[dof[k]]; }
    spmv_cell(m.M1, m.F, c, v, w);
    double su = 0.0;
#pragma unroll
    for (int k = 0; k < 12; ++k) su = fma(u[k], w[k], su);
    double se = 0.0;
    const double det = m.det[c];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        const double a = m.M2e ? U[m.n_u + 3 * c + k] * sym3(m.M2e, m.F, c, k, l)
                               : U[m.n_u + 3 * c + k] * c_tab.M2_ref[k][l] * det;
        se = fma(a, V[m.n_u + 3 * c + l], se);
      }
    acc += H * su + g * se;
  }
  double s3[3];
  block_sum3<256>(acc, 0.0, 0.0, s3);
  if (threadIdx.x == 0) part[blockIdx.x] = s3[0];
}

// The paper's error norms (Sec. 3) per cell, summed over the block:
// u^T M1 u, the L2 norm squared of div u (the DG1 field D u / M2, so
// (D_K u)^T M2_K^{-1} (D_K u) on the cell) and eta^T M2 eta.
__global__ void __launch_bounds__(256) k_norms(DeviceMesh m, const double* __restrict__ U, double* part) {
  double a = 0.0, dv = 0.0, e = 0.0;
  for (int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x; c < m.F; c += (int64_t)gridDim.x * 256) {
    int dof[12];
    double sg[12], u[12], w[12];
    cell_dofs(m, c, dof, sg);
#pragma unroll
    for (int k = 0; k < 12; ++k) u[k] = U[dof[k]];
    spmv_cell(m.M1, m.F, c, u, w);
#pragma unroll
    for (int k = 0; k < 12; ++k) a = fma(u[k], w[k], a);
    const double det = m.det[c];
    double d[3], h[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double t = 0.0;
#pragma unroll
      for (int i = 0; i < 12; ++i) t = fma(c_tab.D[k][i] * sg[i], u[i], t);
      d[k] = t;
      h[k] = U[m.n_u + 3 * c + k];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        if (m.M2i) {  // cubic cells: the cell's own M2 and M2^{-1}
          dv = fma(d[k] * sym3(m.M2i, m.F, c, k, l), d[l], dv);
          e = fma(h[k] * sym3(m.M2e, m.F, c, k, l), h[l], e);
        } else {
          dv = fma(d[k] * c_tab.M2inv_ref[k][l] / det, d[l], dv);
          e = fma(h[k] * c_tab.M2_ref[k][l] * det, h[l], e);
        }
      }
  }
  double s3[3];
  block_sum3<256>(a, dv, e, s3);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = s3[0];
    part[3 * blockIdx.x + 1] = s3[1];
    part[3 * blockIdx.x + 2] = s3[2];
  }
}

__global__ void k_check_finite(const double* __restrict__ x, int64_t len, int* flags) {
  bool bad = false;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < len; j += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(x[j])) bad = true;
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, kFlagNonFinite);
}

int grid_for(int64_t len, int threads, int cap = 152 * 16) {
  int64_t g = (len + threads - 1) / threads;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

cudaError_t cg_configure(int64_t F, CgWork* w) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg, kCgThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t need = (F + kCgThreads - 1) / kCgThreads;
  int64_t maxb = (int64_t)per_sm * sms;
  w->nblocks = (int)(need < maxb ? need : maxb);
  if (w->nblocks < 1) w->nblocks = 1;
  w->threads = kCgThreads;
  return cudaSuccess;
}

cudaError_t launch_cg(const DeviceMesh& m, const CgWork& w, const CgParams& cp, const double* b,
                      double* out, double scale_x, const double* add, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(w.w[0], 0, sizeof(double) * 3 * m.E, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(w.bar, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(w.nblocks);
  cfg.blockDim = dim3(kCgThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_cg, m, w, cp, b, out, scale_x, add);
}

cudaError_t launch_apply_K(const DeviceMesh& m, const double* U, double s, double g, double H,
                           const double* y_u, const double* y_eta, const double* z_eta, double* ru,
                           double* eta_out, cudaStream_t st, bool fp32) {
  int g_ = (int)((m.F + 127) / 128);
  if (fp32 && m.Cf) k_apply_K<float><<<g_, 128, 0, st>>>(m, U, s, g, H, y_u, y_eta, z_eta, ru, eta_out);
  else k_apply_K<double><<<g_, 128, 0, st>>>(m, U, s, g, H, y_u, y_eta, z_eta, ru, eta_out);
  return cudaGetLastError();
}

cudaError_t launch_nonlinear_rhs(const DeviceMesh& m, const double* U, double* r, int B, int upwind,
                                 cudaStream_t st, bool fp32, double* facets, int chunk) {
  if (!facets || chunk < 1) return cudaErrorInvalidValue;
  for (int b0 = 0; b0 < B; b0 += chunk) {
    const int nb = B - b0 < chunk ? B - b0 : chunk;
    const double* Ub = U + (int64_t)b0 * m.n;
    double* rb = r + (int64_t)b0 * m.n;
    dim3 ge((unsigned)((m.E + 127) / 128), (unsigned)nb), gc((unsigned)((m.F + 127) / 128), (unsigned)nb);
    const bool cubic = m.geo_c != nullptr;
    if (fp32 && cubic) {
      k_facets<float, 3><<<ge, 128, 0, st>>>(m, Ub, facets, upwind);
      k_nonlinear<float, 3><<<gc, 128, 0, st>>>(m, Ub, rb, facets);
    } else if (fp32) {
      k_facets<float, 1><<<ge, 128, 0, st>>>(m, Ub, facets, upwind);
      k_nonlinear<float, 1><<<gc, 128, 0, st>>>(m, Ub, rb, facets);
    } else if (cubic) {
      k_facets<double, 3><<<ge, 128, 0, st>>>(m, Ub, facets, upwind);
      k_nonlinear<double, 3><<<gc, 128, 0, st>>>(m, Ub, rb, facets);
    } else {
      k_facets<double, 1><<<ge, 128, 0, st>>>(m, Ub, facets, upwind);
      k_nonlinear<double, 1><<<gc, 128, 0, st>>>(m, Ub, rb, facets);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_m2inv(const DeviceMesh& m, const double* r, int64_t rstride, double* out,
                         int64_t ostride, int B, cudaStream_t st) {
  dim3 grid((unsigned)((m.F + 255) / 256), (unsigned)B);
  k_m2inv<<<grid, 256, 0, st>>>(m, r, rstride, out, ostride);
  return cudaGetLastError();
}

int combine_tile() { return 8; }

cudaError_t launch_combine(const double* A, int Mo, int Ki, const int* lim, const double* in, int64_t in_stride,
                           double* out, int64_t out_stride, int64_t len, cudaStream_t st, bool fp32) {
  constexpr int MT = 8;
  const size_t smem = (fp32 ? sizeof(float) : sizeof(double)) * MT * Ki;
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_combine<MT, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_combine<MT, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  dim3 grid((unsigned)grid_for(len, 256, 152 * 4), (unsigned)((Mo + MT - 1) / MT));
  if (fp32) k_combine<MT, float><<<grid, 256, smem, st>>>(A, Mo, Ki, lim, in, in_stride, out, out_stride, len);
  else k_combine<MT, double><<<grid, 256, smem, st>>>(A, Mo, Ki, lim, in, in_stride, out, out_stride, len);
  return cudaGetLastError();
}

cudaError_t launch_combine_pairs_fwd(const double* A, int P, int Ki, const int* lim, const double* in,
                                     int64_t in_stride, double* out, int64_t out_stride, int64_t len,
                                     cudaStream_t st, bool fp32) {
  constexpr int MT = 8;
  const size_t smem = (fp32 ? sizeof(float) : sizeof(double)) * MT * Ki;
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_combine_pairs_fwd<MT, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_combine_pairs_fwd<MT, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  dim3 grid((unsigned)grid_for(len, 256, 152 * 4), (unsigned)((P + MT - 1) / MT));
  if (fp32)
    k_combine_pairs_fwd<MT, float><<<grid, 256, smem, st>>>(A, P, Ki, lim, in, in_stride, out, out_stride, len);
  else
    k_combine_pairs_fwd<MT, double><<<grid, 256, smem, st>>>(A, P, Ki, lim, in, in_stride, out, out_stride, len);
  return cudaGetLastError();
}

cudaError_t launch_combine_pairs_bwd(const double* B, int Ko, int P, const int* lim, const double* R,
                                     int64_t r_stride, double* out, int64_t out_stride, int64_t len,
                                     cudaStream_t st) {
  constexpr int MT = 8;
  const size_t smem = sizeof(double) * MT * P;
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_combine_pairs_bwd<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  dim3 grid((unsigned)grid_for(len, 256, 152 * 4), (unsigned)((Ko + MT - 1) / MT));
  k_combine_pairs_bwd<MT><<<grid, 256, smem, st>>>(B, Ko, P, lim, R, r_stride, out, out_stride, len);
  return cudaGetLastError();
}

cudaError_t launch_lincomb(double* out, double a, const double* x, double b, const double* y, double c,
                           const double* z, int64_t len, cudaStream_t st) {
  k_lincomb<<<grid_for(len, 256), 256, 0, st>>>(out, a, x, b, y, c, z, len);
  return cudaGetLastError();
}

cudaError_t launch_winner(const DeviceMesh& m, const double* U, const double* V, double g, double H,
                          double* part, int* nblocks, cudaStream_t st) {
  int nb = grid_for(m.F, 256, 304);
  k_winner<<<nb, 256, 0, st>>>(m, U, V, g, H, part);
  *nblocks = nb;
  return cudaGetLastError();
}

cudaError_t launch_norms(const DeviceMesh& m, const double* U, double* part, int* nblocks, cudaStream_t st) {
  int nb = grid_for(m.F, 256, 304);
  k_norms<<<nb, 256, 0, st>>>(m, U, part);
  *nblocks = nb;
  return cudaGetLastError();
}

cudaError_t launch_check_finite(const double* x, int64_t len, int* flags, cudaStream_t st) {
  k_check_finite<<<grid_for(len, 256, 304), 256, 0, st>>>(x, len, flags);
  return cudaGetLastError();
}

}  // namespace pavg
