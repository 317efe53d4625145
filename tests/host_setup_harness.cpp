// Command-line access to the library's host-side set-up (csrc/setup.cpp) for
// the CPU tests, with no GPU and no CUDA runtime:
//   mesh R RADIUS PREFIX  the canonical icosahedral mesh (Sec. 3): writes
//                         PREFIX.verts (float64 [V][3]) and PREFIX.cells
//                         (int32 [F][3]); prints "V F E"
//   cheb LB TOL           the truncated Chebyshev coefficients of e^{tL} for
//                         LB = lambda_max |t| (Sec. 2.4): prints the count,
//                         then one coefficient per line (count 0: refused)
//   shifts T M RULE       the Riemann-sum shifts and weights (Sec. 2.2):
//                         prints the status, then "s w" per line
//   cells R RADIUS OMEGA PREFIX [DEGREE]
//                         the per-cell element matrices of M1 and C (Sec. 2.5)
//                         as the kernels store them (signed, packed), expanded
//                         and placed at their global DOFs: writes
//                         PREFIX.{m1,c}.{row,col} (int64) and .val (float64)
//                         triplets, PREFIX.det and PREFIX.g (float64 [3][F]:
//                         G00, G01, G11 of G = J^T J); prints "n_u F".  With
//                         DEGREE 3 (the piecewise cubic surface of Sec. 3) also
//                         PREFIX.m2e, .m2i (float64 [6][F]), .geoc (float64
//                         [6][25][F]) and .geof (float64 [8][5][E]; G00, G01, G11,
//                         1 / det per side)
//   stroud N              the N x N Stroud conical product rule: "x y w" lines
//   tables                the reference tables the kernels read from constant
//                         memory: prints D (3 x 12), then M2 and M2^{-1} (3 x 3)
//                         of the reference cell, one row per line
//   solver R RADIUS PREFIX
//                         the mixed solver's and the facet kernels' set-up
//                         data, raw: PREFIX.tri (int32 [F][4]), .pinv (float32
//                         [E + F][8]), .dinv (float64 [n_u]), .m1 (float64
//                         [78][F]), .m1p (float32 [78][F]), .m1f (float32
//                         [36][F][4]), .eplus / .eminus (int32 [E]), .elpos
//                         (uint8 [E]); prints "E F"
//   partition R RADIUS P PREFIX
//                         the subdomain solver's partition of the cells into P
//                         parts (csrc/sd_setup.cpp): writes PREFIX.cell0,
//                         .lt0 (int32 [P+1]), .gtri, .slot (uint32 [lt]), .recv
//                         (int32 [lt]), .celllt, .cellsend (int32 [F][4]);
//                         prints "nslots max_cells max_lt max_shared"
//   spectrum R RADIUS ITERS
//                         Lanczos estimate of the extreme eigenvalues of the
//                         block-Jacobi preconditioned M1: prints "lmin lmax"
//   chebits A B TOL       Chebyshev iterations on [A, B] that reduce the error
//                         by TOL
//   element X1 Y1 X2 Y2 ...
//                         the reference BDM2 basis at each point: one line of
//                         24 values psi_i[c], then one of 48 derivatives
//                         d psi_i[c] / d xi_a (order i, c, a)
//   gauss N               the N-point Gauss-Legendre rule on [0, 1]: "x w" lines
//   cellrule              the cell rule of the nonlinear kernels: "w phi0 phi1
//                         phi2" per point (phi = the DG1 basis at the point)
//   ntables               the remaining constant tables of the nonlinear
//                         kernels, one per line, flattened in C order:
//                         cq_psi, cq_dpsi, fq_w, fq_psi, fq_phi, edge_dir,
//                         div_vert
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "pavg_internal.h"

namespace {

bool write_all(const std::string& path, const void* data, size_t bytes) {
  FILE* f = std::fopen(path.c_str(), "wb");
  if (!f) return false;
  const bool ok = std::fwrite(data, 1, bytes, f) == bytes;
  return std::fclose(f) == 0 && ok;
}

}  // namespace

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  const std::string cmd = argv[1];
  if (cmd == "mesh" && argc == 5) {
    pavg::Mesh m;
    pavg::build_mesh(std::atoi(argv[2]), std::strtod(argv[3], nullptr), &m);
    const std::string prefix = argv[4];
    if (!write_all(prefix + ".verts", m.verts.data(), sizeof(double) * m.verts.size()) ||
        !write_all(prefix + ".cells", m.cells.data(), sizeof(int32_t) * m.cells.size()))
      return 3;
    std::printf("%lld %lld %lld\n", (long long)m.V(), (long long)m.F(), (long long)m.E());
    return 0;
  }
  if (cmd == "cheb" && argc == 4) {
    const std::vector<double> c = pavg::cheb_coefficients(std::strtod(argv[2], nullptr), std::strtod(argv[3], nullptr));
    std::printf("%zu\n", c.size());
    for (double x : c) std::printf("%.17g\n", x);
    return 0;
  }
  if (cmd == "shifts" && argc == 5) {
    std::vector<double> s, w;
    const int rc = pavg::shifts_weights(std::strtod(argv[2], nullptr), std::atoi(argv[3]), std::atoi(argv[4]), &s, &w);
    std::printf("%d\n", rc);
    for (size_t i = 0; i < s.size(); ++i) std::printf("%.17g %.17g\n", s[i], w[i]);
    return 0;
  }
  if (cmd == "stroud" && argc == 3) {
    std::vector<double> x, y, w;
    pavg::stroud_rule(std::atoi(argv[2]), &x, &y, &w);
    for (size_t k = 0; k < w.size(); ++k) std::printf("%.17g %.17g %.17g\n", x[k], y[k], w[k]);
    return 0;
  }
  if (cmd == "cells" && (argc == 6 || argc == 7)) {
    pavg::Mesh m;
    pavg::build_mesh(std::atoi(argv[2]), std::strtod(argv[3], nullptr), &m);
    pavg::RefElement el;
    pavg::build_reference_element(&el);
    pavg::HostCellData cd;
    pavg::ConstTables tab;
    pavg::TablesP3<double> tab3;
    const int degree = argc == 7 ? std::atoi(argv[6]) : 1;
    pavg::build_cell_data(m, el, std::strtod(argv[4], nullptr), degree, &cd, &tab, &tab3);
    const int64_t F = m.F();
    std::vector<int64_t> r1, c1, rc, cc;
    std::vector<double> v1, vc;
    for (int64_t c = 0; c < F; ++c) {
      int64_t g[12];
      for (int l = 0; l < 12; ++l) g[l] = 3 * (int64_t)(cd.tri[4 * c + l / 3] & 0x7fffffff) + l % 3;
      for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j) {
          const int a = i < j ? i : j, b = i < j ? j : i;
          r1.push_back(g[i]);
          c1.push_back(g[j]);
          v1.push_back(cd.M1[(int64_t)pavg::packed_sym(a, b) * F + c]);
          if (i != j) {
            const double x = cd.C[(int64_t)pavg::packed_asym(a, b) * F + c];
            rc.push_back(g[i]);
            cc.push_back(g[j]);
            vc.push_back(i < j ? x : -x);
          }
        }
    }
    const std::string p = argv[5];
    if (!write_all(p + ".m1.row", r1.data(), 8 * r1.size()) || !write_all(p + ".m1.col", c1.data(), 8 * c1.size()) ||
        !write_all(p + ".m1.val", v1.data(), 8 * v1.size()) || !write_all(p + ".c.row", rc.data(), 8 * rc.size()) ||
        !write_all(p + ".c.col", cc.data(), 8 * cc.size()) || !write_all(p + ".c.val", vc.data(), 8 * vc.size()) ||
        !write_all(p + ".det", cd.det.data(), 8 * cd.det.size()) || !write_all(p + ".g", cd.G.data(), 8 * cd.G.size()))
      return 3;
    if (degree == 3 &&
        (!write_all(p + ".m2e", cd.M2e.data(), 8 * cd.M2e.size()) ||
         !write_all(p + ".m2i", cd.M2i.data(), 8 * cd.M2i.size()) ||
         !write_all(p + ".geoc", cd.geo_c.data(), 8 * cd.geo_c.size()) ||
         !write_all(p + ".geof", cd.geo_f.data(), 8 * cd.geo_f.size())))
      return 3;
    std::printf("%lld %lld\n", (long long)(3 * m.E() + 3 * F), (long long)F);
    return 0;
  }
  if (cmd == "tables" && argc == 2) {
    pavg::Mesh m;
    pavg::build_mesh(0, 1.0, &m);
    pavg::RefElement el;
    pavg::build_reference_element(&el);
    pavg::HostCellData cd;
    pavg::ConstTables tab;
    pavg::build_cell_data(m, el, 0.0, 1, &cd, &tab, nullptr);
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 12; ++j) std::printf("%.17g ", tab.D[i][j]);
      std::printf("\n");
    }
    for (int i = 0; i < 3; ++i) std::printf("%.17g %.17g %.17g\n", tab.M2_ref[i][0], tab.M2_ref[i][1], tab.M2_ref[i][2]);
    for (int i = 0; i < 3; ++i)
      std::printf("%.17g %.17g %.17g\n", tab.M2inv_ref[i][0], tab.M2inv_ref[i][1], tab.M2inv_ref[i][2]);
    return 0;
  }
  if (cmd == "solver" && argc == 5) {
    pavg::Mesh m;
    pavg::build_mesh(std::atoi(argv[2]), std::strtod(argv[3], nullptr), &m);
    pavg::RefElement el;
    pavg::build_reference_element(&el);
    pavg::HostCellData cd;
    pavg::ConstTables tab;
    pavg::build_cell_data(m, el, 7.292e-5, 1, &cd, &tab, nullptr);
    const std::string p = argv[4];
    if (!write_all(p + ".tri", cd.tri.data(), 4 * cd.tri.size()) ||
        !write_all(p + ".pinv", cd.Pinv.data(), 4 * cd.Pinv.size()) ||
        !write_all(p + ".dinv", cd.dinv.data(), 8 * cd.dinv.size()) ||
        !write_all(p + ".m1", cd.M1.data(), 8 * cd.M1.size()) || !write_all(p + ".m1p", cd.M1p.data(), 4 * cd.M1p.size()) ||
        !write_all(p + ".m1f", cd.M1f.data(), 4 * cd.M1f.size()) ||
        !write_all(p + ".eplus", m.edge_plus.data(), 4 * m.edge_plus.size()) ||
        !write_all(p + ".eminus", m.edge_minus.data(), 4 * m.edge_minus.size()) ||
        !write_all(p + ".elpos", m.edge_lpos.data(), m.edge_lpos.size()))
      return 3;
    std::printf("%lld %lld\n", (long long)m.E(), (long long)m.F());
    return 0;
  }
  if ((cmd == "partition" && argc == 6) || (cmd == "spectrum" && argc == 5)) {
    pavg::Mesh m;
    pavg::build_mesh(std::atoi(argv[2]), std::strtod(argv[3], nullptr), &m);
    pavg::RefElement el;
    pavg::build_reference_element(&el);
    pavg::HostCellData cd;
    pavg::ConstTables tab;
    pavg::build_cell_data(m, el, 7.292e-5, 1, &cd, &tab, nullptr);
    if (cmd == "spectrum") {
      double lo = 0, hi = 0;
      pavg::sd_spectrum(m.F(), m.E(), cd.M1, cd.tri, cd.Pinv, std::atoi(argv[4]), &lo, &hi);
      std::printf("%.17g %.17g\n", lo, hi);
      return 0;
    }
    pavg::SdPartition sp;
    pavg::build_sd_partition(m.F(), m.E(), cd.tri, std::atoi(argv[4]), &sp);
    const std::string p = argv[5];
    if (!write_all(p + ".cell0", sp.cell0.data(), 4 * sp.cell0.size()) ||
        !write_all(p + ".lt0", sp.lt0.data(), 4 * sp.lt0.size()) ||
        !write_all(p + ".gtri", sp.lt_gtri.data(), 4 * sp.lt_gtri.size()) ||
        !write_all(p + ".slot", sp.lt_slot.data(), 4 * sp.lt_slot.size()) ||
        !write_all(p + ".recv", sp.lt_recv.data(), 4 * sp.lt_recv.size()) ||
        !write_all(p + ".celllt", sp.cell_lt.data(), 4 * sp.cell_lt.size()) ||
        !write_all(p + ".cellsend", sp.cell_send.data(), 4 * sp.cell_send.size()))
      return 3;
    std::printf("%d %d %d %d\n", sp.nslots, sp.max_cells, sp.max_lt, sp.max_shared);
    return 0;
  }
  if (cmd == "chebits" && argc == 5) {
    std::printf("%d\n", pavg::sd_iterations(std::strtod(argv[2], nullptr), std::strtod(argv[3], nullptr),
                                             std::strtod(argv[4], nullptr)));
    return 0;
  }
  if (cmd == "element" && argc >= 4 && argc % 2 == 0) {
    pavg::RefElement el;
    pavg::build_reference_element(&el);
    for (int a = 2; a + 1 < argc; a += 2) {
      const double x = std::strtod(argv[a], nullptr), y = std::strtod(argv[a + 1], nullptr);
      double v[12][2], g[12][2][2];
      el.eval(x, y, v);
      el.eval_grad(x, y, g);
      for (int i = 0; i < 12; ++i) std::printf("%.17g %.17g ", v[i][0], v[i][1]);
      std::printf("\n");
      for (int i = 0; i < 12; ++i)
        for (int c = 0; c < 2; ++c) std::printf("%.17g %.17g ", g[i][c][0], g[i][c][1]);
      std::printf("\n");
    }
    return 0;
  }
  if (cmd == "gauss" && argc == 3) {
    const int n = std::atoi(argv[2]);
    if (n < 1 || n > 64) return 2;
    std::vector<double> x(n), w(n);
    pavg::gauss_legendre01(n, x.data(), w.data());
    for (int i = 0; i < n; ++i) std::printf("%.17g %.17g\n", x[i], w[i]);
    return 0;
  }
  if (cmd == "cellrule" && argc == 2) {
    pavg::Mesh m;
    pavg::build_mesh(0, 1.0, &m);
    pavg::RefElement el;
    pavg::build_reference_element(&el);
    pavg::HostCellData cd;
    pavg::ConstTables tab;
    pavg::build_cell_data(m, el, 0.0, 1, &cd, &tab, nullptr);
    for (int q = 0; q < pavg::kCellQ; ++q)
      std::printf("%.17g %.17g %.17g %.17g\n", tab.cq_w[q], tab.cq_phi[q][0], tab.cq_phi[q][1], tab.cq_phi[q][2]);
    return 0;
  }
  if (cmd == "ntables" && argc == 2) {
    pavg::Mesh m;
    pavg::build_mesh(0, 1.0, &m);
    pavg::RefElement el;
    pavg::build_reference_element(&el);
    pavg::HostCellData cd;
    pavg::ConstTables tab;
    pavg::build_cell_data(m, el, 0.0, 1, &cd, &tab, nullptr);
    auto line = [](const double* p, size_t n) {
      for (size_t i = 0; i < n; ++i) std::printf("%.17g ", p[i]);
      std::printf("\n");
    };
    line(&tab.cq_psi[0][0][0], sizeof(tab.cq_psi) / sizeof(double));
    line(&tab.cq_dpsi[0][0][0][0], sizeof(tab.cq_dpsi) / sizeof(double));
    line(&tab.fq_w[0], sizeof(tab.fq_w) / sizeof(double));
    line(&tab.fq_psi[0][0][0][0][0], sizeof(tab.fq_psi) / sizeof(double));
    line(&tab.fq_phi[0][0][0][0], sizeof(tab.fq_phi) / sizeof(double));
    line(&tab.edge_dir[0][0], sizeof(tab.edge_dir) / sizeof(double));
    line(&tab.div_vert[0][0], sizeof(tab.div_vert) / sizeof(double));
    return 0;
  }
  return 2;
}
