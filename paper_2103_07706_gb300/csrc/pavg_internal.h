// Internal declarations of libpavg: host setup (setup.cpp) and device side (*.cu).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "pavg.h"

namespace pavg {

// Number of cell quadrature points used by the nonlinear kernels (degree-5
// symmetric rule), facet points per edge (Gauss-Legendre, part of the method's
// definition because the upwind choice is taken per point).
constexpr int kCellQ = 7;
constexpr int kFacetQ = 4;
// On the piecewise cubic surface (Sec. 3) the integrands carry 1/det and are
// not polynomials, so the rules are part of the discretisation: the 5 x 5
// Stroud conical product rule in cells, 5-point Gauss-Legendre on facets.
constexpr int kCellQ3 = 25;
constexpr int kFacetQ3 = 5;

// Canonical icosahedral mesh (paper Sec. 3).
struct Mesh {
  int refinement = 0;
  double radius = 0;
  std::vector<double> verts;          // [V][3]
  std::vector<int32_t> cells;         // [F][3] counter-clockwise from outside
  std::vector<int32_t> edges;         // [E][2] low, high
  std::vector<int32_t> cell_edges;    // [F][3] local edge i is opposite local vertex i
  std::vector<uint8_t> cell_aligned;  // [F] bit i: cell runs local edge i low -> high
  std::vector<int32_t> edge_plus;     // [E] cell running the edge low -> high
  std::vector<int32_t> edge_minus;    // [E]
  std::vector<uint8_t> edge_lpos;     // [E] local index in plus | (local index in minus) << 2
  int64_t F() const { return (int64_t)cells.size() / 3; }
  int64_t E() const { return (int64_t)edges.size() / 2; }
  int64_t V() const { return (int64_t)verts.size() / 3; }
};

void build_mesh(int refinement, double radius, Mesh* m);

// Reference BDM2 element: psi_i = sum_l coef[l][i] mono_l, 12 vector monomials.
struct RefElement {
  double coef[12][12];
  void eval(double x, double y, double val[12][2]) const;
  void eval_grad(double x, double y, double grad[12][2][2]) const;  // [i][component][d/dx, d/dy]
};
void build_reference_element(RefElement* el);

// Gauss-Legendre on [0, 1].
void gauss_legendre01(int n, double* x, double* w);

// Tables copied to __constant__ memory for the kernels (one copy in FP64 and
// one in FP32; every member is an array of R, so the two layouts correspond
// element by element).
template <typename R>
struct TablesT {
  R D[3][12];             // int_ref phi_i div psi_j
  R M2inv_ref[3][3];      // inverse of int_ref phi_i phi_j (M2^{-1} = M2inv_ref / det)
  R M2_ref[3][3];         // int_ref phi_i phi_j (M2 = det * M2_ref)
  // cell rule for N: points, weights and basis data
  R cq_w[kCellQ];
  R cq_psi[kCellQ][12][2];
  R cq_dpsi[kCellQ][12][2][2];
  R cq_phi[kCellQ][3];
  // facet rule: for each local edge (3) and each point, the reference basis at
  // tau (plus side: counter-clockwise parameter tau) and at 1 - tau (minus side)
  R fq_w[kFacetQ];
  R fq_psi[2][3][kFacetQ][12][2];   // [side][local edge][point]
  R fq_phi[2][3][kFacetQ][3];
  R edge_dir[3][2];
  R div_vert[12][3];      // div_hat psi_j at the reference vertices (a P1 function)
};
using ConstTables = TablesT<double>;

// Reference tables of the cubic-geometry nonlinear kernels (same layout
// conventions as TablesT, for the rules of kCellQ3 and kFacetQ3 points).
template <typename R>
struct TablesP3 {
  R cq_w[kCellQ3];
  R cq_psi[kCellQ3][12][2];
  R cq_dpsi[kCellQ3][12][2][2];
  R cq_phi[kCellQ3][3];
  R fq_w[kFacetQ3];
  R fq_psi[2][3][kFacetQ3][12][2];
  R fq_phi[2][3][kFacetQ3][3];
  R edge_dir[3][2];
};

inline TablesP3<float> tables_to_float(const TablesP3<double>& t) {
  static_assert(sizeof(TablesP3<double>) == 2 * sizeof(TablesP3<float>), "tables must be plain arrays");
  TablesP3<float> f;
  const double* src = reinterpret_cast<const double*>(&t);
  float* dst = reinterpret_cast<float*>(&f);
  for (size_t i = 0; i < sizeof(TablesP3<double>) / sizeof(double); ++i) dst[i] = (float)src[i];
  return f;
}

inline TablesT<float> tables_to_float(const ConstTables& t) {
  static_assert(sizeof(ConstTables) == 2 * sizeof(TablesT<float>), "tables must be plain arrays");
  TablesT<float> f;
  const double* src = reinterpret_cast<const double*>(&t);
  float* dst = reinterpret_cast<float*>(&f);
  for (size_t i = 0; i < sizeof(ConstTables) / sizeof(double); ++i) dst[i] = (float)src[i];
  return f;
}

// Per-cell data in structure-of-arrays form.
struct HostCellData {
  std::vector<double> M1;      // [78][F] signed element mass matrices, packed upper triangle
  std::vector<double> C;       // [66][F] signed Coriolis element matrices, packed strict upper
  std::vector<double> det;     // [F]
  std::vector<double> G;       // [3][F] metric J^T J: G00, G01, G11
  std::vector<double> dinv;    // [n_u] 1 / diag(M1)
  std::vector<float> M1f;      // [36][F][4] M1 rounded to FP32, row blocks: entry (e, c, q) is
                               // row 3q + e / 12, column e % 12 of cell c's signed 12 x 12 matrix
  std::vector<float> Pinv;     // [E + F][8] inverses of the 3x3 diagonal blocks of M1 (00,01,02,11,12,22,-,-)
  std::vector<float> M1p;      // [78][F] M1 rounded to FP32, packed upper triangle (shared-memory path)
  std::vector<int32_t> tri;    // [F][4] DOF triple of (cell, q) | owner bit 31 (q = 0..2 edges, 3 interior)
  // cubic geometry only (empty on flat cells, where M2 = det * M2_ref)
  std::vector<double> M2e;     // [6][F] DG1 element mass matrices, packed 00, 01, 02, 11, 12, 22
  std::vector<double> M2i;     // [6][F] their inverses, same packing
  std::vector<double> geo_c;   // [6][kCellQ3][F] per cell point: G00, G01, G11, w / det^2,
                               // (d det / d xi0) / det, (d det / d xi1) / det
  std::vector<double> geo_f;   // [8][kFacetQ3][E] per edge point: the plus cell's G00, G01, G11, 1 / det,
                               // then the minus cell's, each at its own parameter of the point
};
// Element data on the flat (geometry_degree 1) or piecewise cubic (3) surface.
// `tab3` receives the cubic kernels' tables (filled for degree 3 only).
void build_cell_data(const Mesh& m, const RefElement& el, double omega, int geometry_degree, HostCellData* out,
                     ConstTables* tab, TablesP3<double>* tab3);

// The cubic cell map (Sec. 3) of cell c at reference point (x, y).
struct PointGeometry {
  double x[3];                  // the point
  double J[3][2];               // dx / dxi
  double det, G00, G01, G11;    // |J0 x J1|, J^T J
  double ddet[2];               // d det / d xi_a
};
void p3_geometry(const Mesh& m, int64_t c, double x, double y, PointGeometry* g);
// 5 x 5 Stroud conical product rule on the reference triangle (area 1/2).
void stroud_rule(int n, std::vector<double>* px, std::vector<double>* py, std::vector<double>* pw);

// Partition of the cells for the subdomain mass solver: part p owns the
// contiguous cells cell0[p] .. cell0[p+1]-1 and numbers the DOF triples its
// cells touch locally (lt0[p] .. lt0[p+1]-1 in the arrays below).
struct SdPartition {
  int P = 0;
  std::vector<int32_t> cell0;     // [P+1]
  std::vector<int32_t> lt0;       // [P+1]
  std::vector<uint32_t> lt_gtri;  // [lt] global triple | bit 31: this part owns it (writes it, counts it in norms)
  std::vector<uint32_t> lt_slot;  // [lt] the local (cell - cell0) * 4 + q positions of the triple's local
                                  //      cells: low 16 bits, high 16 bits; 0xffff = none
  std::vector<int32_t> lt_recv;   // [lt] send slot of the other part for a triple shared with it, else -1
  std::vector<int32_t> cell_lt;   // [F][4] local triple of (cell, q)
  std::vector<int32_t> cell_send; // [F][4] send slot of (cell, q) when its triple is shared, else -1
  int32_t nslots = 0;             // send slots (two per shared triple)
  int32_t max_cells = 0, max_lt = 0, max_shared = 0;
};
void build_sd_partition(int64_t F, int64_t E, const std::vector<int32_t>& tri, int P, SdPartition* out);
// Extreme eigenvalues of the block-Jacobi preconditioned M1 (preconditioned Lanczos, `iters` steps).
void sd_spectrum(int64_t F, int64_t E, const std::vector<double>& M1, const std::vector<int32_t>& tri,
                 const std::vector<float>& Pinv, int iters, double* lmin, double* lmax);
// Chebyshev iterations on [a, b] that reduce the error by inner_rtol.
int sd_iterations(double a, double b, double inner_rtol);

// Largest lambda_max |t| accepted for one exponential.  The coefficients
// are a direct O(N^2) transform with N >= Lb + 64, and the series has about
// Lb terms, each one mass solve; 16384 is 50 times the widest benchmark
// window (refinement 7, T = 4 h: 336).
constexpr double kMaxChebArg = PAVG_MAX_CHEB_ARG;

// Chebyshev coefficients c_k of e^{tL} in the real recurrence (Sec. 2.4):
// returns the truncated list (degree K = size - 1) for Lb = lambda_max |t|,
// or an empty list when Lb is negative, not finite or above kMaxChebArg.
std::vector<double> cheb_coefficients(double Lb, double tol);
inline std::string cheb_limit_msg(double Lb) {
  return "lambda_max |t| = " + std::to_string(Lb) + " is not finite or above " + std::to_string(kMaxChebArg) +
         " (the widest exponential accepted)";
}

// Riemann-sum shifts and weights (Sec. 2.2).
int shifts_weights(double T, int M, int rule, std::vector<double>* s, std::vector<double>* w);

inline int packed_sym(int i, int j) {  // i <= j, row-major upper triangle of 12x12
  return i * 12 - i * (i - 1) / 2 + (j - i);
}
inline int packed_asym(int i, int j) {  // i < j
  return i * 11 - i * (i - 1) / 2 + (j - i - 1);
}

}  // namespace pavg
