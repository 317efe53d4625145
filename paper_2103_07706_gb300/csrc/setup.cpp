// Host-side setup of libpavg: canonical mesh, Gauss rules, reference BDM2/DG1
// element, per-cell geometry and element matrices, Chebyshev coefficients and
// Riemann-sum weights.  Compiled with -ffp-contract=off so that vertex
// coordinates are rounded identically on every host.
#include <algorithm>
#include <numeric>
#include <array>
#include <cmath>
#include <complex>
#include <map>
#include <stdexcept>
#include <tuple>

#include "pavg_internal.h"

namespace pavg {

// ---------------------------------------------------------------- mesh
namespace {

void scale_to(const double p[3], double radius, double out[3]) {
  double nrm = std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  double s = radius / nrm;
  out[0] = p[0] * s;
  out[1] = p[1] * s;
  out[2] = p[2] * s;
}

}  // namespace

// Paper Sec. 3: icosahedral grid.  Construction (the numbering both the
// library and its tests rely on): the 12 icosahedron vertices sorted by
// (x, y, z); faces = mutually adjacent triples, counter-clockwise from
// outside, smallest index first, sorted; refinement splits face (a, b, c) into
// (a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca) with midpoints projected
// to the sphere and numbered on first visit (edges visited ab, bc, ca).
void build_mesh(int refinement, double radius, Mesh* m) {
  const double phi = (1.0 + std::sqrt(5.0)) / 2.0;
  std::vector<std::array<double, 3>> raw;
  for (double a : {-1.0, 1.0})
    for (double b : {-1.0, 1.0}) {
      raw.push_back({0.0, a, b * phi});
      raw.push_back({a, b * phi, 0.0});
      raw.push_back({a * phi, 0.0, b});
    }
  std::sort(raw.begin(), raw.end());
  std::vector<std::array<int, 3>> faces;
  auto d2 = [&](int i, int j) {
    double s = 0;
    for (int k = 0; k < 3; ++k) s += (raw[i][k] - raw[j][k]) * (raw[i][k] - raw[j][k]);
    return s;
  };
  for (int i = 0; i < 12; ++i)
    for (int j = i + 1; j < 12; ++j)
      for (int k = j + 1; k < 12; ++k) {
        if (std::fabs(d2(i, j) - 4) > 1e-9 || std::fabs(d2(j, k) - 4) > 1e-9 ||
            std::fabs(d2(i, k) - 4) > 1e-9)
          continue;
        const auto &a = raw[i], &b = raw[j], &c = raw[k];
        double cx = b[1] * c[2] - b[2] * c[1], cy = b[2] * c[0] - b[0] * c[2],
               cz = b[0] * c[1] - b[1] * c[0];
        double triple = a[0] * cx + a[1] * cy + a[2] * cz;
        std::array<int, 3> f = triple > 0 ? std::array<int, 3>{i, j, k} : std::array<int, 3>{i, k, j};
        int r = (int)(std::min_element(f.begin(), f.end()) - f.begin());
        std::rotate(f.begin(), f.begin() + r, f.end());
        faces.push_back(f);
      }
  std::sort(faces.begin(), faces.end());
  if (faces.size() != 20) throw std::runtime_error("icosahedron construction failed");
  std::vector<std::array<double, 3>> verts(12);
  for (int i = 0; i < 12; ++i) scale_to(raw[i].data(), radius, verts[i].data());

  for (int level = 0; level < refinement; ++level) {
    std::map<std::pair<int, int>, int> mid;
    auto midpoint = [&](int a, int b) {
      auto key = std::make_pair(std::min(a, b), std::max(a, b));
      auto it = mid.find(key);
      if (it != mid.end()) return it->second;
      double s[3] = {verts[a][0] + verts[b][0], verts[a][1] + verts[b][1], verts[a][2] + verts[b][2]};
      std::array<double, 3> v;
      scale_to(s, radius, v.data());
      verts.push_back(v);
      int id = (int)verts.size() - 1;
      mid[key] = id;
      return id;
    };
    std::vector<std::array<int, 3>> next;
    next.reserve(faces.size() * 4);
    for (const auto& f : faces) {
      int a = f[0], b = f[1], c = f[2];
      int ab = midpoint(a, b), bc = midpoint(b, c), ca = midpoint(c, a);
      next.push_back({a, ab, ca});
      next.push_back({ab, b, bc});
      next.push_back({ca, bc, c});
      next.push_back({ab, bc, ca});
    }
    faces.swap(next);
  }

  m->refinement = refinement;
  m->radius = radius;
  m->verts.resize(verts.size() * 3);
  for (size_t i = 0; i < verts.size(); ++i)
    for (int k = 0; k < 3; ++k) m->verts[3 * i + k] = verts[i][k];
  const int64_t F = (int64_t)faces.size();
  m->cells.resize(3 * F);
  for (int64_t c = 0; c < F; ++c)
    for (int k = 0; k < 3; ++k) m->cells[3 * c + k] = faces[c][k];

  // edges: sorted (low, high) pairs
  std::vector<std::pair<int, int>> ev;
  ev.reserve(3 * F);
  for (int64_t c = 0; c < F; ++c) {
    int v[3] = {faces[c][0], faces[c][1], faces[c][2]};
    for (int i = 0; i < 3; ++i) {
      int p = v[(i + 1) % 3], q = v[(i + 2) % 3];
      ev.emplace_back(std::min(p, q), std::max(p, q));
    }
  }
  std::sort(ev.begin(), ev.end());
  ev.erase(std::unique(ev.begin(), ev.end()), ev.end());
  const int64_t E = (int64_t)ev.size();
  m->edges.resize(2 * E);
  for (int64_t e = 0; e < E; ++e) {
    m->edges[2 * e] = ev[e].first;
    m->edges[2 * e + 1] = ev[e].second;
  }
  m->cell_edges.assign(3 * F, -1);
  m->cell_aligned.assign(F, 0);
  m->edge_plus.assign(E, -1);
  m->edge_minus.assign(E, -1);
  m->edge_lpos.assign(E, 0);
  for (int64_t c = 0; c < F; ++c) {
    int v[3] = {faces[c][0], faces[c][1], faces[c][2]};
    for (int i = 0; i < 3; ++i) {
      // local edge i runs v[i+1] -> v[i+2] counter-clockwise
      int p = v[(i + 1) % 3], q = v[(i + 2) % 3];
      auto key = std::make_pair(std::min(p, q), std::max(p, q));
      int64_t e = std::lower_bound(ev.begin(), ev.end(), key) - ev.begin();
      m->cell_edges[3 * c + i] = (int32_t)e;
      if (p < q) {
        m->cell_aligned[c] |= (uint8_t)(1u << i);
        if (m->edge_plus[e] >= 0) throw std::runtime_error("edge traversed twice low->high");
        m->edge_plus[e] = (int32_t)c;
        m->edge_lpos[e] |= (uint8_t)i;
      } else {
        if (m->edge_minus[e] >= 0) throw std::runtime_error("edge traversed twice high->low");
        m->edge_minus[e] = (int32_t)c;
        m->edge_lpos[e] |= (uint8_t)(i << 2);
      }
    }
  }
  for (int64_t e = 0; e < E; ++e)
    if (m->edge_plus[e] < 0 || m->edge_minus[e] < 0) throw std::runtime_error("open edge in mesh");
}

// ---------------------------------------------------------------- quadrature
void gauss_legendre01(int n, double* x, double* w) {
  // Newton iteration on P_n from the Chebyshev-like initial guesses.
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double pn = p1, pnm1 = p0;  // P_n, P_{n-1} (n >= 2)
      dp = n * (z * pn - pnm1) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    x[n - 1 - i] = 0.5 * (z + 1.0);
    w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);  // (2 / ((1-z^2) P'^2)) / 2
  }
}

namespace {

// Jacobi polynomial P_n^{(a,b)}(x) by its three-term recurrence in n.
double jacobi(int n, double a, double b, double x) {
  if (n == 0) return 1.0;
  double p0 = 1.0, p1 = 0.5 * (2.0 * (a + 1.0) + (a + b + 2.0) * (x - 1.0));
  for (int k = 2; k <= n; ++k) {
    const double s = 2.0 * k + a + b;
    const double c1 = 2.0 * k * (k + a + b) * (s - 2.0);
    const double c2 = (s - 1.0) * (s * (s - 2.0) * x + a * a - b * b);
    const double c3 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * s;
    const double p2 = (c2 * p1 - c3 * p0) / c1;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

}  // namespace

// Gauss-Jacobi rule for the weight (1 - x) on [-1, 1] (a = 1, b = 0): the
// nodes are the zeros of P_n^{(1,0)}, bracketed by sign changes on a fine grid
// and bisected to the last bit; the weights are
// 4 / ((1 - x^2) P_n'(x)^2), with P_n' = (n + 2)/2 P_{n-1}^{(2,1)}.
void gauss_jacobi10(int n, double* x, double* w) {
  const int grid = 4096;
  int found = 0;
  double xa = -1.0, fa = jacobi(n, 1.0, 0.0, xa);
  for (int k = 1; k <= grid && found < n; ++k) {
    const double xb = -1.0 + 2.0 * k / grid, fb = jacobi(n, 1.0, 0.0, xb);
    if (fa == 0.0 || (fa < 0.0) != (fb < 0.0)) {
      double lo = xa, hi = xb, flo = fa;
      for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        const double fm = jacobi(n, 1.0, 0.0, mid);
        if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else hi = mid;
      }
      x[found++] = 0.5 * (lo + hi);
    }
    xa = xb;
    fa = fb;
  }
  if (found != n) throw std::runtime_error("Gauss-Jacobi: roots not bracketed");
  for (int i = 0; i < n; ++i) {
    const double d = 0.5 * (n + 2.0) * jacobi(n - 1, 2.0, 1.0, x[i]);
    w[i] = 4.0 / ((1.0 - x[i] * x[i]) * d * d);
  }
}

// Stroud conical product rule on the reference triangle: x = s, y = t (1 - s)
// with s from Gauss-Jacobi (its weight absorbs the Jacobian 1 - s, mapped to
// [0, 1]) and t from Gauss-Legendre; n x n points, exact to degree 2n - 1.
// Checked against int x^a y^b = a! b! / (a + b + 2)! for a + b <= 2n - 1.
void stroud_rule(int n, std::vector<double>* px, std::vector<double>* py, std::vector<double>* pw) {
  std::vector<double> xs(n), ws(n), t(n), wt(n);
  gauss_jacobi10(n, xs.data(), ws.data());
  gauss_legendre01(n, t.data(), wt.data());
  px->clear(); py->clear(); pw->clear();
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double s = 0.5 * (xs[i] + 1.0);
      px->push_back(s);
      py->push_back(t[j] * (1.0 - s));
      pw->push_back(0.25 * ws[i] * wt[j]);
    }
  for (int a = 0; a <= 2 * n - 1; ++a)
    for (int b = 0; a + b <= 2 * n - 1; ++b) {
      double sum = 0.0;
      for (size_t k = 0; k < pw->size(); ++k) sum += (*pw)[k] * std::pow((*px)[k], a) * std::pow((*py)[k], b);
      const double want = std::tgamma(a + 1.0) * std::tgamma(b + 1.0) / std::tgamma(a + b + 3.0);
      if (std::fabs(sum - want) > 1e-15) throw std::runtime_error("Stroud rule check failed");
    }
}

// ---------------------------------------------------------------- cubic geometry (Sec. 3)
// The piecewise cubic surface: each cell's map is the cubic Lagrange
// interpolant, in barycentric coordinates (l0, l1, l2) = (1 - x - y, x, y),
// of ten nodes: the vertices, the points (2/3, 1/3) of each edge and the
// centroid of the flat triangle, each projected radially onto the sphere.
// Basis: vertex i  l_i (3 l_i - 1)(3 l_i - 2) / 2,
//        edge (i,j) 9/2 l_i l_j (3 l_i - 1)   (the node with l_i = 2/3, l_j = 1/3),
//        centroid  27 l0 l1 l2.
namespace {

struct P3Nodes {
  double X[10][3];
};

const int kP3Pair[6][2] = {{0, 1}, {1, 0}, {1, 2}, {2, 1}, {2, 0}, {0, 2}};

void p3_nodes(const Mesh& m, int64_t c, double radius, P3Nodes* n) {
  const double* v[3] = {&m.verts[3 * m.cells[3 * c + 0]], &m.verts[3 * m.cells[3 * c + 1]],
                        &m.verts[3 * m.cells[3 * c + 2]]};
  for (int k = 0; k < 10; ++k) {
    double lam[3] = {0.0, 0.0, 0.0};
    if (k < 3) lam[k] = 1.0;
    else if (k < 9) { lam[kP3Pair[k - 3][0]] = 2.0 / 3.0; lam[kP3Pair[k - 3][1]] = 1.0 / 3.0; }
    else lam[0] = lam[1] = lam[2] = 1.0 / 3.0;
    double p[3];
    for (int d = 0; d < 3; ++d) p[d] = lam[0] * v[0][d] + lam[1] * v[1][d] + lam[2] * v[2][d];
    if (k < 3) {
      for (int d = 0; d < 3; ++d) n->X[k][d] = v[k][d];
    } else {
      const double s = radius / std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
      for (int d = 0; d < 3; ++d) n->X[k][d] = p[d] * s;
    }
  }
}

// Value, lambda-gradient and lambda-Hessian of cubic basis function k.
void p3_basis(int k, const double l[3], double* N, double dN[3], double d2N[3][3]) {
  for (int a = 0; a < 3; ++a) {
    dN[a] = 0.0;
    for (int b = 0; b < 3; ++b) d2N[a][b] = 0.0;
  }
  if (k < 3) {
    const double t = l[k];
    *N = 0.5 * t * (3.0 * t - 1.0) * (3.0 * t - 2.0);
    dN[k] = 0.5 * (27.0 * t * t - 18.0 * t + 2.0);
    d2N[k][k] = 27.0 * t - 9.0;
  } else if (k < 9) {
    const int i = kP3Pair[k - 3][0], j = kP3Pair[k - 3][1];
    *N = 4.5 * l[i] * l[j] * (3.0 * l[i] - 1.0);
    dN[i] = 4.5 * l[j] * (6.0 * l[i] - 1.0);
    dN[j] = 4.5 * l[i] * (3.0 * l[i] - 1.0);
    d2N[i][i] = 27.0 * l[j];
    d2N[i][j] = d2N[j][i] = 4.5 * (6.0 * l[i] - 1.0);
  } else {
    *N = 27.0 * l[0] * l[1] * l[2];
    dN[0] = 27.0 * l[1] * l[2];
    dN[1] = 27.0 * l[0] * l[2];
    dN[2] = 27.0 * l[0] * l[1];
    d2N[0][1] = d2N[1][0] = 27.0 * l[2];
    d2N[0][2] = d2N[2][0] = 27.0 * l[1];
    d2N[1][2] = d2N[2][1] = 27.0 * l[0];
  }
}

void cross3(const double a[3], const double b[3], double out[3]) {
  out[0] = a[1] * b[2] - a[2] * b[1];
  out[1] = a[2] * b[0] - a[0] * b[2];
  out[2] = a[0] * b[1] - a[1] * b[0];
}

void p3_eval(const P3Nodes& n, double x, double y, PointGeometry* g) {
  const double l[3] = {1.0 - x - y, x, y};
  const double dl[2][3] = {{-1.0, 1.0, 0.0}, {-1.0, 0.0, 1.0}};  // d lambda / d xi_a
  double H[2][2][3] = {};
  for (int d = 0; d < 3; ++d) { g->x[d] = 0.0; g->J[d][0] = g->J[d][1] = 0.0; }
  for (int k = 0; k < 10; ++k) {
    double N, dN[3], d2N[3][3];
    p3_basis(k, l, &N, dN, d2N);
    double da[2], dab[2][2];
    for (int a = 0; a < 2; ++a) {
      da[a] = dN[0] * dl[a][0] + dN[1] * dl[a][1] + dN[2] * dl[a][2];
      for (int b = 0; b < 2; ++b) {
        double t = 0.0;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) t += d2N[i][j] * dl[a][i] * dl[b][j];
        dab[a][b] = t;
      }
    }
    for (int d = 0; d < 3; ++d) {
      g->x[d] += N * n.X[k][d];
      for (int a = 0; a < 2; ++a) {
        g->J[d][a] += da[a] * n.X[k][d];
        for (int b = 0; b < 2; ++b) H[a][b][d] += dab[a][b] * n.X[k][d];
      }
    }
  }
  const double J0[3] = {g->J[0][0], g->J[1][0], g->J[2][0]};
  const double J1[3] = {g->J[0][1], g->J[1][1], g->J[2][1]};
  double cr[3];
  cross3(J0, J1, cr);
  g->det = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
  g->G00 = J0[0] * J0[0] + J0[1] * J0[1] + J0[2] * J0[2];
  g->G01 = J0[0] * J1[0] + J0[1] * J1[1] + J0[2] * J1[2];
  g->G11 = J1[0] * J1[0] + J1[1] * J1[1] + J1[2] * J1[2];
  // d det / d xi_a = k . (d_a J0 x J1 + J0 x d_a J1),  d_a J_b = H[a][b]
  for (int a = 0; a < 2; ++a) {
    double u[3], v[3];
    cross3(H[a][0], J1, u);
    cross3(J0, H[a][1], v);
    g->ddet[a] = (cr[0] * (u[0] + v[0]) + cr[1] * (u[1] + v[1]) + cr[2] * (u[2] + v[2])) / g->det;
  }
}

}  // namespace

void p3_geometry(const Mesh& m, int64_t c, double x, double y, PointGeometry* g) {
  P3Nodes n;
  p3_nodes(m, c, m.radius, &n);
  p3_eval(n, x, y, g);
}

namespace {

// Collapsed Gauss-Legendre rule on the reference triangle:
// x = s, y = t (1 - s), weight w_s w_t (1 - s); exact to degree 2n - 2.
void triangle_gl(int n, std::vector<double>* px, std::vector<double>* py, std::vector<double>* pw) {
  std::vector<double> x(n), w(n);
  gauss_legendre01(n, x.data(), w.data());
  px->clear(); py->clear(); pw->clear();
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      px->push_back(x[i]);
      py->push_back(x[j] * (1.0 - x[i]));
      pw->push_back(w[i] * w[j] * (1.0 - x[i]));
    }
}

// Symmetric 7-point rule of degree 5 on the reference triangle (area 1/2).
void triangle_deg5(double px[7], double py[7], double pw[7]) {
  const double r = std::sqrt(15.0);
  const double a1 = (6.0 - r) / 21.0, b1 = (9.0 + 2.0 * r) / 21.0;
  const double a2 = (6.0 + r) / 21.0, b2 = (9.0 - 2.0 * r) / 21.0;
  const double w1 = (155.0 - r) / 2400.0, w2 = (155.0 + r) / 2400.0;
  double x[7] = {1.0 / 3.0, a1, a1, b1, a2, a2, b2};
  double y[7] = {1.0 / 3.0, a1, b1, a1, a2, b2, a2};
  double w[7] = {9.0 / 80.0, w1, w1, w1, w2, w2, w2};
  for (int i = 0; i < 7; ++i) { px[i] = x[i]; py[i] = y[i]; pw[i] = w[i]; }
}

const double kEdgeStart[3][2] = {{1.0, 0.0}, {0.0, 1.0}, {0.0, 0.0}};
const double kEdgeDir[3][2] = {{-1.0, 1.0}, {0.0, -1.0}, {1.0, 0.0}};

// scalar P2 monomials ordered 1, x, y, xx, xy, yy and their gradients
void mono(double x, double y, double m[6]) {
  m[0] = 1.0; m[1] = x; m[2] = y; m[3] = x * x; m[4] = x * y; m[5] = y * y;
}
void mono_grad(double x, double y, double g[6][2]) {
  g[0][0] = 0; g[0][1] = 0;
  g[1][0] = 1; g[1][1] = 0;
  g[2][0] = 0; g[2][1] = 1;
  g[3][0] = 2 * x; g[3][1] = 0;
  g[4][0] = y; g[4][1] = x;
  g[5][0] = 0; g[5][1] = 2 * y;
}
// vector monomial l (0..11): component l / 6 carries scalar monomial l % 6
void vmono(double x, double y, double v[12][2]) {
  double m[6];
  mono(x, y, m);
  for (int l = 0; l < 12; ++l) {
    v[l][0] = l < 6 ? m[l] : 0.0;
    v[l][1] = l < 6 ? 0.0 : m[l - 6];
  }
}

bool invert(int n, const double* A, double* out) {
  std::vector<double> a(A, A + n * n), inv(n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(a[r * n + col]) > std::fabs(a[piv * n + col])) piv = r;
    if (std::fabs(a[piv * n + col]) < 1e-300) return false;
    if (piv != col)
      for (int k = 0; k < n; ++k) {
        std::swap(a[piv * n + k], a[col * n + k]);
        std::swap(inv[piv * n + k], inv[col * n + k]);
      }
    double d = a[col * n + col];
    for (int k = 0; k < n; ++k) { a[col * n + k] /= d; inv[col * n + k] /= d; }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = a[r * n + col];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) { a[r * n + k] -= f * a[col * n + k]; inv[r * n + k] -= f * inv[col * n + k]; }
    }
  }
  std::copy(inv.begin(), inv.end(), out);
  return true;
}

}  // namespace

// ---------------------------------------------------------------- reference element
// Degrees of freedom of BDM2 (paper Sec. 2.5: V1 = BDM2): Legendre moments of
// the outward flux on each edge (counter-clockwise parameter), and interior
// moments against (1,0), (0,1), (-y,x).  The basis is dual to them.
// Exact rational numbers with small numerators and denominators: the BDM2
// Vandermonde matrix and its inverse have entries of at most a few hundred.
struct Rat {
  int64_t n = 0, d = 1;
  Rat() = default;
  Rat(int64_t num, int64_t den = 1) : n(num), d(den) {
    if (d < 0) { n = -n; d = -d; }
    int64_t g = std::gcd(n < 0 ? -n : n, d);
    if (g > 1) { n /= g; d /= g; }
  }
};
Rat operator+(Rat a, Rat b) { return Rat(a.n * b.d + b.n * a.d, a.d * b.d); }
Rat operator-(Rat a, Rat b) { return Rat(a.n * b.d - b.n * a.d, a.d * b.d); }
Rat operator*(Rat a, Rat b) { return Rat(a.n * b.n, a.d * b.d); }
Rat operator/(Rat a, Rat b) { return Rat(a.n * b.d, a.d * b.n); }

// Product of two polynomials in one variable (integer coefficients, lowest first).
std::vector<int64_t> pmul(const std::vector<int64_t>& a, const std::vector<int64_t>& b) {
  std::vector<int64_t> r(a.size() + b.size() - 1, 0);
  for (size_t i = 0; i < a.size(); ++i)
    for (size_t j = 0; j < b.size(); ++j) r[i + j] += a[i] * b[j];
  return r;
}

// The reference BDM2 basis is dual to the DOF functionals, l_k(psi_i) =
// delta_ki: its coefficients over the vector monomials are the inverse of
// V[k][l] = l_k(m_l).  Every entry of V is rational (along edge i,
// x = sx + tau dx and y = sy + tau dy have integer start and direction, so a
// monomial is an integer polynomial in tau and int_0^1 tau^k = 1/(k+1); over
// the triangle int x^a y^b = a! b! / (a+b+2)!), and so is the inverse (its
// entries are integers), so both are computed exactly and the basis carries
// no rounding from inverting V (cond(V) is about 530).
void build_reference_element(RefElement* el) {
  const int pa[6] = {0, 1, 0, 2, 1, 0}, pb[6] = {0, 0, 1, 0, 1, 2};  // monomial 1, x, y, xx, xy, yy
  const std::vector<int64_t> leg[3] = {{1}, {-1, 2}, {1, -6, 6}};
  const int64_t es[3][2] = {{1, 0}, {0, 1}, {0, 0}}, ed[3][2] = {{-1, 1}, {0, -1}, {1, 0}};
  Rat V[12][24];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int l = 0; l < 12; ++l) {
        std::vector<int64_t> m = {1};
        for (int k = 0; k < pa[l % 6]; ++k) m = pmul(m, {es[i][0], ed[i][0]});
        for (int k = 0; k < pb[l % 6]; ++k) m = pmul(m, {es[i][1], ed[i][1]});
        const int64_t fx = l < 6 ? ed[i][1] : -ed[i][0];  // cross2(m_l, d_i)
        std::vector<int64_t> p = pmul(m, leg[j]);
        Rat s(0);
        for (size_t k = 0; k < p.size(); ++k) s = s + Rat(p[k] * fx, (int64_t)k + 1);
        V[3 * i + j][l] = s;
      }
  auto fact = [](int n) { int64_t f = 1; for (int k = 2; k <= n; ++k) f *= k; return f; };
  auto tri = [&](int a, int b) { return Rat(fact(a) * fact(b), fact(a + b + 2)); };
  for (int l = 0; l < 12; ++l) {
    const int a = pa[l % 6], b = pb[l % 6];
    V[9][l] = l < 6 ? tri(a, b) : Rat(0);                      // q_0 = (1, 0)
    V[10][l] = l < 6 ? Rat(0) : tri(a, b);                     // q_1 = (0, 1)
    V[11][l] = l < 6 ? Rat(0) - tri(a, b + 1) : tri(a + 1, b); // q_2 = (-y, x)
  }
  for (int r = 0; r < 12; ++r)
    for (int c = 0; c < 12; ++c) V[r][12 + c] = Rat(r == c ? 1 : 0);
  for (int col = 0; col < 12; ++col) {  // Gauss-Jordan, exact
    int piv = col;
    while (piv < 12 && V[piv][col].n == 0) ++piv;
    if (piv == 12) throw std::runtime_error("BDM2 Vandermonde is singular");
    for (int c = 0; c < 24; ++c) std::swap(V[col][c], V[piv][c]);
    const Rat pv = V[col][col];
    for (int c = 0; c < 24; ++c) V[col][c] = V[col][c] / pv;
    for (int r = 0; r < 12; ++r) {
      if (r == col || V[r][col].n == 0) continue;
      const Rat f = V[r][col];
      for (int c = 0; c < 24; ++c) V[r][c] = V[r][c] - f * V[col][c];
    }
  }
  for (int l = 0; l < 12; ++l)
    for (int i = 0; i < 12; ++i) el->coef[l][i] = (double)V[l][12 + i].n / (double)V[l][12 + i].d;
}

void RefElement::eval(double x, double y, double val[12][2]) const {
  double v[12][2];
  vmono(x, y, v);
  for (int i = 0; i < 12; ++i) {
    double a = 0, b = 0;
    for (int l = 0; l < 12; ++l) { a += coef[l][i] * v[l][0]; b += coef[l][i] * v[l][1]; }
    val[i][0] = a;
    val[i][1] = b;
  }
}

void RefElement::eval_grad(double x, double y, double grad[12][2][2]) const {
  double g[6][2];
  mono_grad(x, y, g);
  for (int i = 0; i < 12; ++i)
    for (int c = 0; c < 2; ++c)
      for (int d = 0; d < 2; ++d) {
        double s = 0;
        for (int p = 0; p < 6; ++p) s += coef[6 * c + p][i] * g[p][d];
        grad[i][c][d] = s;
      }
}

// ---------------------------------------------------------------- cell data
// Element matrices of Sec. 2.5 on flat cells with the contravariant Piola map:
//   M1_ij = int psi_i^T G psi_j / det,  C_ij = int f cross2(psi_j, psi_i)
// (C_ij = int w_i . f (k x w_j) dx), f = 2 Omega z / R at the cell point;
// D_ij = int phi_i div psi_j is the same on every cell.  Signs map the cell's
// counter-clockwise edge DOFs to the global ones: (-1)^(j+1) for moment j on an
// edge the cell runs high -> low.
void build_cell_data(const Mesh& m, const RefElement& el, double omega, int geometry_degree, HostCellData* out,
                     ConstTables* tab, TablesP3<double>* tab3) {
  const int64_t F = m.F(), E = m.E();
  const bool cubic = geometry_degree == 3;
  const int64_t n_u = 3 * E + 3 * F;
  std::vector<double> qx, qy, qw;
  triangle_gl(4, &qx, &qy, &qw);
  const int Q = (int)qx.size();
  std::vector<double> psi(Q * 24), dpsi(Q * 48), phi(Q * 3);
  for (int q = 0; q < Q; ++q) {
    el.eval(qx[q], qy[q], reinterpret_cast<double(*)[2]>(&psi[q * 24]));
    el.eval_grad(qx[q], qy[q], reinterpret_cast<double(*)[2][2]>(&dpsi[q * 48]));
    phi[q * 3 + 0] = 1.0 - qx[q] - qy[q];
    phi[q * 3 + 1] = qx[q];
    phi[q * 3 + 2] = qy[q];
  }
  // D (reference) and DG1 reference mass
  double M2r[9] = {0};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 12; ++j) {
      double s = 0;
      for (int q = 0; q < Q; ++q) s += qw[q] * phi[q * 3 + i] * (dpsi[q * 48 + j * 4 + 0] + dpsi[q * 48 + j * 4 + 3]);
      tab->D[i][j] = s;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int q = 0; q < Q; ++q) s += qw[q] * phi[q * 3 + i] * phi[q * 3 + j];
      M2r[i * 3 + j] = s;
    }
  double M2i[9];
  if (!invert(3, M2r, M2i)) throw std::runtime_error("DG1 mass singular");
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      tab->M2inv_ref[i][j] = M2i[i * 3 + j];
      tab->M2_ref[i][j] = M2r[i * 3 + j];
    }

  out->M1.assign(78 * F, 0.0);
  out->C.assign(66 * F, 0.0);
  out->det.assign(F, 0.0);
  out->G.assign(3 * F, 0.0);
  std::vector<double> diag(n_u, 0.0);
  // cubic surface: the 5 x 5 Stroud rule and the reference data at its points
  std::vector<double> sx, sy, sw, spsi, sphi;
  if (cubic) {
    stroud_rule(5, &sx, &sy, &sw);
    spsi.resize(kCellQ3 * 24);
    sphi.resize(kCellQ3 * 3);
    for (int q = 0; q < kCellQ3; ++q) {
      el.eval(sx[q], sy[q], reinterpret_cast<double(*)[2]>(&spsi[q * 24]));
      sphi[q * 3 + 0] = 1.0 - sx[q] - sy[q];
      sphi[q * 3 + 1] = sx[q];
      sphi[q * 3 + 2] = sy[q];
    }
    out->M2e.assign(6 * F, 0.0);
    out->M2i.assign(6 * F, 0.0);
    out->geo_c.assign((size_t)6 * kCellQ3 * F, 0.0);
  }
  for (int64_t c = 0; c < F; ++c) {
    const double* a = &m.verts[3 * m.cells[3 * c + 0]];
    const double* b = &m.verts[3 * m.cells[3 * c + 1]];
    const double* d = &m.verts[3 * m.cells[3 * c + 2]];
    double J0[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double J1[3] = {d[0] - a[0], d[1] - a[1], d[2] - a[2]};
    double cr[3] = {J0[1] * J1[2] - J0[2] * J1[1], J0[2] * J1[0] - J0[0] * J1[2], J0[0] * J1[1] - J0[1] * J1[0]};
    double det = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    double G00 = J0[0] * J0[0] + J0[1] * J0[1] + J0[2] * J0[2];
    double G01 = J0[0] * J1[0] + J0[1] * J1[1] + J0[2] * J1[2];
    double G11 = J1[0] * J1[0] + J1[1] * J1[1] + J1[2] * J1[2];
    out->det[c] = det;  // the flat triangle's (cell-size features on either surface)
    out->G[0 * F + c] = G00;
    out->G[1 * F + c] = G01;
    out->G[2 * F + c] = G11;
    double sgn[12];
    int dof[12];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        bool al = (m.cell_aligned[c] >> i) & 1;
        sgn[3 * i + j] = al ? 1.0 : (j == 1 ? 1.0 : -1.0);
        dof[3 * i + j] = 3 * m.cell_edges[3 * c + i] + j;
      }
    for (int j = 0; j < 3; ++j) { sgn[9 + j] = 1.0; dof[9 + j] = (int)(3 * E + 3 * c + j); }
    double m1[12][12], cc[12][12];  // unsigned element matrices (upper triangles used)
    if (cubic) {
      // M1_ij = sum_q w psi_i . G psi_j / det,  C_ij = sum_q w f cross2(psi_j, psi_i),
      // M2_kl = sum_q w det phi_k phi_l, with J, det, G and f = 2 Omega z / R at each point
      P3Nodes nodes;
      p3_nodes(m, c, m.radius, &nodes);
      double m2[3][3] = {};
      for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j) m1[i][j] = cc[i][j] = 0.0;
      for (int q = 0; q < kCellQ3; ++q) {
        PointGeometry g;
        p3_eval(nodes, sx[q], sy[q], &g);
        const double f = 2.0 * omega * g.x[2] / m.radius;
        const double wq = sw[q];
        const double* ps = &spsi[q * 24];
        for (int i = 0; i < 12; ++i)
          for (int j = i; j < 12; ++j) {
            const double* pi = ps + 2 * i;
            const double* pj = ps + 2 * j;
            m1[i][j] += wq * (pi[0] * (g.G00 * pj[0] + g.G01 * pj[1]) + pi[1] * (g.G01 * pj[0] + g.G11 * pj[1])) / g.det;
            cc[i][j] += wq * f * (pj[0] * pi[1] - pj[1] * pi[0]);
          }
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) m2[k][l] += wq * g.det * sphi[q * 3 + k] * sphi[q * 3 + l];
        double* gc = &out->geo_c[0];
        const int64_t QF = (int64_t)kCellQ3 * F;
        gc[0 * QF + q * F + c] = g.G00;
        gc[1 * QF + q * F + c] = g.G01;
        gc[2 * QF + q * F + c] = g.G11;
        gc[3 * QF + q * F + c] = wq / (g.det * g.det);
        gc[4 * QF + q * F + c] = g.ddet[0] / g.det;
        gc[5 * QF + q * F + c] = g.ddet[1] / g.det;
      }
      double inv[9], mm[9];
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) mm[3 * k + l] = 0.5 * (m2[k][l] + m2[l][k]);
      if (!invert(3, mm, inv)) throw std::runtime_error("singular DG1 element mass");
      const int pk[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
      for (int k = 0; k < 6; ++k) {
        out->M2e[(int64_t)k * F + c] = mm[3 * pk[k][0] + pk[k][1]];
        out->M2i[(int64_t)k * F + c] = 0.5 * (inv[3 * pk[k][0] + pk[k][1]] + inv[3 * pk[k][1] + pk[k][0]]);
      }
    } else {
      double fz[64];
      for (int q = 0; q < Q; ++q) {
        double z = a[2] + J0[2] * qx[q] + J1[2] * qy[q];
        fz[q] = 2.0 * omega * z / m.radius;
      }
      for (int i = 0; i < 12; ++i)
        for (int j = i; j < 12; ++j) {
          double sm = 0, sc = 0;
          for (int q = 0; q < Q; ++q) {
            const double* pi = &psi[q * 24 + 2 * i];
            const double* pj = &psi[q * 24 + 2 * j];
            sm += qw[q] * (pi[0] * (G00 * pj[0] + G01 * pj[1]) + pi[1] * (G01 * pj[0] + G11 * pj[1]));
            sc += qw[q] * fz[q] * (pj[0] * pi[1] - pj[1] * pi[0]);
          }
          m1[i][j] = sm / det;
          cc[i][j] = sc;
        }
    }
    for (int i = 0; i < 12; ++i)
      for (int j = i; j < 12; ++j) {
        double ss = sgn[i] * sgn[j];
        out->M1[(int64_t)packed_sym(i, j) * F + c] = ss * m1[i][j];
        if (j > i) out->C[(int64_t)packed_asym(i, j) * F + c] = ss * cc[i][j];
        if (i == j) diag[dof[i]] += m1[i][j];
      }
  }
  out->dinv.resize(n_u);
  for (int64_t k = 0; k < n_u; ++k) out->dinv[k] = 1.0 / diag[k];

  // FP32 copy of the element matrices and the 3x3 diagonal blocks of the
  // assembled M1 (each edge's three moments, each cell's three interior
  // DOFs: triple t = dof / 3), inverted in FP64 and stored in FP32.
  out->M1f.resize((size_t)144 * F);
  for (int64_t c = 0; c < F; ++c)
    for (int q = 0; q < 4; ++q)
      for (int e = 0; e < 36; ++e) {
        int i = 3 * q + e / 12, j = e % 12;
        int pk = i <= j ? packed_sym(i, j) : packed_sym(j, i);
        out->M1f[((size_t)e * F + c) * 4 + q] = (float)out->M1[(int64_t)pk * F + c];
      }
  out->M1p.resize(out->M1.size());
  for (size_t k = 0; k < out->M1.size(); ++k) out->M1p[k] = (float)out->M1[k];
  out->tri.resize((size_t)4 * F);
  for (int64_t c = 0; c < F; ++c) {
    for (int q = 0; q < 3; ++q) {
      uint32_t t = (uint32_t)m.cell_edges[3 * c + q];
      if ((m.cell_aligned[c] >> q) & 1u) t |= 0x80000000u;
      out->tri[4 * c + q] = (int32_t)t;
    }
    out->tri[4 * c + 3] = (int32_t)((uint32_t)(E + c) | 0x80000000u);
  }
  const int64_t T = E + F;
  std::vector<double> blk(9 * T, 0.0);
  for (int64_t c = 0; c < F; ++c)
    for (int q = 0; q < 4; ++q) {
      int64_t t = q < 3 ? m.cell_edges[3 * c + q] : E + c;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          int i = 3 * q + a, j = 3 * q + b;
          int pk = i <= j ? packed_sym(i, j) : packed_sym(j, i);
          blk[9 * t + 3 * a + b] += out->M1[(int64_t)pk * F + c];
        }
    }
  out->Pinv.assign(8 * T, 0.0f);
  for (int64_t t = 0; t < T; ++t) {
    double inv[9];
    if (!invert(3, &blk[9 * t], inv)) throw std::runtime_error("singular diagonal block of M1");
    const int idx[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    for (int k = 0; k < 6; ++k) {
      double v = 0.5 * (inv[3 * idx[k][0] + idx[k][1]] + inv[3 * idx[k][1] + idx[k][0]]);
      out->Pinv[8 * t + k] = (float)v;
    }
  }

  // tables for the nonlinear kernels
  double cx[7], cy[7], cw[7];
  triangle_deg5(cx, cy, cw);
  for (int q = 0; q < kCellQ; ++q) {
    tab->cq_w[q] = cw[q];
    el.eval(cx[q], cy[q], tab->cq_psi[q]);
    el.eval_grad(cx[q], cy[q], tab->cq_dpsi[q]);
    tab->cq_phi[q][0] = 1.0 - cx[q] - cy[q];
    tab->cq_phi[q][1] = cx[q];
    tab->cq_phi[q][2] = cy[q];
  }
  double fx[kFacetQ], fw[kFacetQ];
  gauss_legendre01(kFacetQ, fx, fw);
  for (int p = 0; p < kFacetQ; ++p) tab->fq_w[p] = fw[p];
  for (int side = 0; side < 2; ++side)
    for (int i = 0; i < 3; ++i)
      for (int p = 0; p < kFacetQ; ++p) {
        double t = side == 0 ? fx[p] : 1.0 - fx[p];
        double x = kEdgeStart[i][0] + t * kEdgeDir[i][0];
        double y = kEdgeStart[i][1] + t * kEdgeDir[i][1];
        el.eval(x, y, tab->fq_psi[side][i][p]);
        tab->fq_phi[side][i][p][0] = 1.0 - x - y;
        tab->fq_phi[side][i][p][1] = x;
        tab->fq_phi[side][i][p][2] = y;
      }
  for (int i = 0; i < 3; ++i) { tab->edge_dir[i][0] = kEdgeDir[i][0]; tab->edge_dir[i][1] = kEdgeDir[i][1]; }
  const double vx[3] = {0.0, 1.0, 0.0}, vy[3] = {0.0, 0.0, 1.0};
  for (int v = 0; v < 3; ++v) {
    double g[12][2][2];
    el.eval_grad(vx[v], vy[v], g);
    for (int j = 0; j < 12; ++j) tab->div_vert[j][v] = g[j][0][0] + g[j][1][1];
  }

  // self-check of the degree-5 rule
  for (int p = 0; p <= 5; ++p)
    for (int q = 0; q + p <= 5; ++q) {
      double s = 0;
      for (int k = 0; k < 7; ++k) s += cw[k] * std::pow(cx[k], p) * std::pow(cy[k], q);
      double fp = std::tgamma(p + 1.0), fq = std::tgamma(q + 1.0), fpq = std::tgamma(p + q + 3.0);
      if (std::fabs(s - fp * fq / fpq) > 1e-15) throw std::runtime_error("degree-5 rule check failed");
    }

  if (!cubic) return;
  // cubic surface: the kernels' rules (the Stroud cell rule, 5-point facets),
  // and each edge's two cells' metric at every facet point, each at its own
  // parameter of the point (tau on the plus side, 1 - tau on the minus side)
  for (int q = 0; q < kCellQ3; ++q) {
    tab3->cq_w[q] = sw[q];
    el.eval(sx[q], sy[q], tab3->cq_psi[q]);
    el.eval_grad(sx[q], sy[q], tab3->cq_dpsi[q]);
    tab3->cq_phi[q][0] = 1.0 - sx[q] - sy[q];
    tab3->cq_phi[q][1] = sx[q];
    tab3->cq_phi[q][2] = sy[q];
  }
  double gx[kFacetQ3], gw[kFacetQ3];
  gauss_legendre01(kFacetQ3, gx, gw);
  for (int p = 0; p < kFacetQ3; ++p) tab3->fq_w[p] = gw[p];
  for (int side = 0; side < 2; ++side)
    for (int i = 0; i < 3; ++i)
      for (int p = 0; p < kFacetQ3; ++p) {
        double t = side == 0 ? gx[p] : 1.0 - gx[p];
        double x = kEdgeStart[i][0] + t * kEdgeDir[i][0];
        double y = kEdgeStart[i][1] + t * kEdgeDir[i][1];
        el.eval(x, y, tab3->fq_psi[side][i][p]);
        tab3->fq_phi[side][i][p][0] = 1.0 - x - y;
        tab3->fq_phi[side][i][p][1] = x;
        tab3->fq_phi[side][i][p][2] = y;
      }
  for (int i = 0; i < 3; ++i) { tab3->edge_dir[i][0] = kEdgeDir[i][0]; tab3->edge_dir[i][1] = kEdgeDir[i][1]; }
  out->geo_f.assign((size_t)8 * kFacetQ3 * E, 0.0);
  const int64_t PE = (int64_t)kFacetQ3 * E;
  for (int64_t e = 0; e < E; ++e) {
    const int64_t cell[2] = {m.edge_plus[e], m.edge_minus[e]};
    const int loc[2] = {m.edge_lpos[e] & 3, m.edge_lpos[e] >> 2};
    for (int side = 0; side < 2; ++side) {
      P3Nodes nodes;
      p3_nodes(m, cell[side], m.radius, &nodes);
      for (int p = 0; p < kFacetQ3; ++p) {
        const double t = side == 0 ? gx[p] : 1.0 - gx[p];
        PointGeometry g;
        p3_eval(nodes, kEdgeStart[loc[side]][0] + t * kEdgeDir[loc[side]][0],
                kEdgeStart[loc[side]][1] + t * kEdgeDir[loc[side]][1], &g);
        const double v[4] = {g.G00, g.G01, g.G11, 1.0 / g.det};
        for (int k = 0; k < 4; ++k) out->geo_f[(4 * side + k) * PE + p * E + e] = v[k];
      }
    }
  }
}

// ---------------------------------------------------------------- Chebyshev coefficients
// Sec. 2.4: coefficients of e^{i Lb y} = sum_k a_k T_k(y) from samples at the
// Chebyshev-Lobatto points (a discrete cosine transform, evaluated directly),
// then c_k = a_k i^{-k} for the real recurrence Q_{k+1} = 2 X Q_k + Q_{k-1};
// truncation: the smallest K with sum_{j > K} |c_j| <= tol.
std::vector<double> cheb_coefficients(double Lb, double tol) {
  if (!(Lb >= 0.0) || !(Lb <= kMaxChebArg)) return {};
  if (Lb == 0.0) return {1.0};
  int N = 1;
  while (N < Lb + 64.0) N <<= 1;
  std::vector<double> cg(N + 1), sg(N + 1), ctab(2 * N);
  for (int j = 0; j <= N; ++j) {
    double y = std::cos(M_PI * j / N);
    cg[j] = std::cos(Lb * y);
    sg[j] = std::sin(Lb * y);
  }
  for (int k = 0; k < 2 * N; ++k) ctab[k] = std::cos(M_PI * k / N);
  std::vector<double> c(N + 1);
  for (int k = 0; k <= N; ++k) {
    const std::vector<double>& g = (k % 2 == 0) ? cg : sg;
    double s = 0.5 * (g[0] + g[N] * ctab[(int64_t)N * k % (2 * N)]);
    for (int j = 1; j < N; ++j) s += g[j] * ctab[(int64_t)j * k % (2 * N)];
    s *= 2.0 / N;
    if (k == 0 || k == N) s *= 0.5;
    int m = k / 2;
    c[k] = (m % 2 == 0) ? s : -s;
  }
  int K = N;
  double tail = 0.0;
  while (K > 0 && tail + std::fabs(c[K]) <= tol) {
    tail += std::fabs(c[K]);
    --K;
  }
  c.resize(K + 1);
  return c;
}

// Sec. 2.2: weights w_m = rho(s_m / T) / sum_j rho(s_j / T) with the C-infinity
// bump rho(x) = exp(-1 / (1/4 - x^2)) on |x| < 1/2.
int shifts_weights(double T, int M, int rule, std::vector<double>* s, std::vector<double>* w) {
  if (M < 1 || !(T >= 0) || !std::isfinite(T)) return PAVG_ERR_INVAL;
  s->assign(M, 0.0);
  w->assign(M, 0.0);
  if (rule == PAVG_QUAD_MIDPOINT) {
    // exactly antisymmetric: s_{M-1-m} = -s_m (and s = 0 in the middle of an odd M)
    for (int m = 0; m < M / 2; ++m) {
      (*s)[m] = -0.5 * T + (m + 0.5) * T / M;
      (*s)[M - 1 - m] = -(*s)[m];
    }
  } else if (rule == PAVG_QUAD_CLOSED) {
    if (M < 3 || M % 2 == 0) return PAVG_ERR_INVAL;
    int Nh = (M - 1) / 2;
    for (int m = 0; m < M; ++m) (*s)[m] = (m - Nh) * (0.5 * T) / Nh;
  } else {
    return PAVG_ERR_INVAL;
  }
  if (T == 0.0) {
    for (int m = 0; m < M; ++m) { (*s)[m] = 0.0; (*w)[m] = 1.0 / M; }
    return PAVG_OK;
  }
  double tot = 0;
  for (int m = 0; m < M; ++m) {
    double x = (*s)[m] / T;
    double r = std::fabs(x) < 0.5 ? std::exp(-1.0 / (0.25 - x * x)) : 0.0;
    (*w)[m] = r;
    tot += r;
  }
  for (int m = 0; m < M; ++m) (*w)[m] /= tot;
  return PAVG_OK;
}

}  // namespace pavg
