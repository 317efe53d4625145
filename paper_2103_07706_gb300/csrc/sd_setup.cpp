// Host set-up of the subdomain mass solver (cheb_sd.cu): the partition of the
// cells into parts, each part's local numbering of the DOF triples it touches,
// the pairing of the triples two parts share, and the interval of the
// Chebyshev iteration (the spectrum of the block-Jacobi preconditioned M1).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <stdexcept>
#include <vector>

#include "pavg_internal.h"

namespace pavg {

// Parts are contiguous ranges of the canonical cell order.  That order is
// hierarchical (the four children of a cell are consecutive at every level of
// refinement), so a contiguous range is a union of a few compact patches and
// its boundary is short: at refinement 6 in 152 parts, about 140 of the ~1420
// triples a part touches are shared with one of its (at most 9) neighbours.
void build_sd_partition(int64_t F, int64_t E, const std::vector<int32_t>& tri, int P, SdPartition* out) {
  if (P < 1 || F < P || (int64_t)tri.size() != 4 * F) throw std::invalid_argument("bad subdomain partition");
  SdPartition& sp = *out;
  sp = SdPartition();
  sp.P = P;
  const int64_t T = E + F;
  std::vector<int32_t> part_of_cell(F);
  sp.cell0.resize(P + 1);
  for (int p = 0; p <= P; ++p) sp.cell0[p] = (int32_t)((int64_t)p * F / P);
  for (int p = 0; p < P; ++p)
    for (int64_t c = sp.cell0[p]; c < sp.cell0[p + 1]; ++c) part_of_cell[c] = p;
  // the two cells of every triple (interior triples: one)
  std::vector<int32_t> tcell(2 * T, -1);
  std::vector<int8_t> tq(2 * T, -1);
  for (int64_t c = 0; c < F; ++c)
    for (int q = 0; q < 4; ++q) {
      const int64_t t = tri[4 * c + q] & 0x7fffffff;
      const int k = tcell[2 * t] < 0 ? 0 : 1;
      if (k == 1 && tcell[2 * t + 1] >= 0) throw std::runtime_error("a triple touched by three cells");
      tcell[2 * t + k] = (int32_t)c;
      tq[2 * t + k] = (int8_t)q;
    }
  sp.lt0.assign(P + 1, 0);
  sp.cell_lt.assign(4 * F, 0);
  sp.cell_send.assign(4 * F, -1);
  std::vector<int32_t> local(T, -1), seen_by(T, -1);
  // send slot of (part, shared triple): numbered part by part; the partner's
  // slot of the same triple is where this part receives from
  std::vector<int64_t> send_slot(2 * T, -1);  // [t][k]: slot written by the part of tcell[2t + k]
  int32_t nslots = 0;
  for (int p = 0; p < P; ++p) {
    const int32_t c0 = sp.cell0[p], c1 = sp.cell0[p + 1];
    int32_t nl = 0;
    std::vector<int64_t> order;
    for (int32_t c = c0; c < c1; ++c)
      for (int q = 0; q < 4; ++q) {
        const int64_t t = tri[4 * c + q] & 0x7fffffff;
        if (seen_by[t] != p) {
          seen_by[t] = p;
          order.push_back(t);
        }
      }
    // triples shared with another part first: the kernel's thread i serves
    // local triples i and i + NT and handles the second before the first, so
    // a shared triple's partner contribution has the longest time to arrive
    auto shared = [&](int64_t t) {
      return tcell[2 * t + 1] >= 0 && (part_of_cell[tcell[2 * t]] != p || part_of_cell[tcell[2 * t + 1]] != p);
    };
    std::stable_partition(order.begin(), order.end(), shared);
    for (int64_t t : order) local[t] = nl++;
    for (int32_t c = c0; c < c1; ++c)
      for (int q = 0; q < 4; ++q) sp.cell_lt[4 * c + q] = local[tri[4 * c + q] & 0x7fffffff];
    if (nl > 0xfffe || c1 - c0 > 0x3fff) throw std::runtime_error("subdomain too large for 16-bit local indices");
    sp.lt0[p + 1] = sp.lt0[p] + nl;
    sp.max_cells = std::max<int32_t>(sp.max_cells, c1 - c0);
    sp.max_lt = std::max<int32_t>(sp.max_lt, nl);
    for (int64_t t : order) {
      uint32_t gt = (uint32_t)t;
      uint32_t slot = 0xffffffffu;
      int nloc = 0;
      for (int k = 0; k < 2; ++k) {
        const int32_t c = tcell[2 * t + k];
        if (c < 0 || part_of_cell[c] != p) continue;
        const uint32_t s = (uint32_t)((c - c0) * 4 + tq[2 * t + k]);
        slot = nloc == 0 ? (slot & 0xffff0000u) | s : (slot & 0x0000ffffu) | (s << 16);
        ++nloc;
        if (tri[4 * c + tq[2 * t + k]] < 0) gt |= 0x80000000u;  // the owning cell is in this part
      }
      if (nloc == 1) slot |= 0xffff0000u;
      int32_t recv = -1;
      if (tcell[2 * t + 1] >= 0 && nloc == 1) {  // shared with another part: one local cell, one remote
        const int kl = part_of_cell[tcell[2 * t]] == p ? 0 : 1;
        send_slot[2 * t + kl] = nslots++;
        const int32_t c = tcell[2 * t + kl];
        sp.cell_send[4 * c + tq[2 * t + kl]] = (int32_t)send_slot[2 * t + kl];
        recv = -2 - kl;  // resolved below, once the partner's slot exists
      }
      sp.lt_gtri.push_back(gt);
      sp.lt_slot.push_back(slot);
      sp.lt_recv.push_back(recv);
    }
  }
  // resolve receive slots: the partner's send slot of the same triple
  for (int p = 0; p < P; ++p)
    for (int32_t i = sp.lt0[p]; i < sp.lt0[p + 1]; ++i) {
      if (sp.lt_recv[i] >= -1) continue;
      const int kl = -2 - sp.lt_recv[i];
      const int64_t t = sp.lt_gtri[i] & 0x7fffffff;
      const int64_t s = send_slot[2 * t + (1 - kl)];
      if (s < 0) throw std::runtime_error("unpaired shared triple");
      sp.lt_recv[i] = (int32_t)s;
    }
  sp.nslots = nslots;
  // shared triples per part (for the statistics)
  for (int p = 0; p < P; ++p) {
    int32_t ns = 0;
    for (int32_t i = sp.lt0[p]; i < sp.lt0[p + 1]; ++i) ns += sp.lt_recv[i] >= 0 ? 1 : 0;
    sp.max_shared = std::max(sp.max_shared, ns);
  }
}

namespace {

// y = M1 x with the signed packed FP64 element matrices ([78][F]).
void m1_apply(int64_t F, const std::vector<double>& M1, const std::vector<int32_t>& tri, const double* x, double* y,
              int64_t n_u) {
  std::fill(y, y + n_u, 0.0);
  for (int64_t c = 0; c < F; ++c) {
    int64_t dof[12];
    for (int q = 0; q < 4; ++q) {
      const int64_t t = tri[4 * c + q] & 0x7fffffff;
      for (int j = 0; j < 3; ++j) dof[3 * q + j] = 3 * t + j;
    }
    double xl[12];
    for (int i = 0; i < 12; ++i) xl[i] = x[dof[i]];
    for (int i = 0; i < 12; ++i) {
      double s = 0.0;
      for (int j = 0; j < 12; ++j) s += M1[(int64_t)(i <= j ? packed_sym(i, j) : packed_sym(j, i)) * F + c] * xl[j];
      y[dof[i]] += s;
    }
  }
}

// Eigenvalues of the symmetric tridiagonal matrix (diag a, off-diagonal b) below
// x: Sturm sequence count.
int sturm_count(const std::vector<double>& a, const std::vector<double>& b, double x) {
  int cnt = 0;
  double d = 1.0;
  for (size_t i = 0; i < a.size(); ++i) {
    const double bb = i ? b[i - 1] * b[i - 1] : 0.0;
    d = a[i] - x - (i ? bb / d : 0.0);
    if (d == 0.0) d = 1e-300;
    if (d < 0) ++cnt;
  }
  return cnt;
}

double tridiag_eig(const std::vector<double>& a, const std::vector<double>& b, int k, double lo, double hi) {
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_count(a, b, mid) > k) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

}  // namespace

// Extreme eigenvalues of P M1 (P: the inverses of the 3x3 diagonal blocks, as
// the kernels apply them) by preconditioned Lanczos: `iters` steps of
// preconditioned conjugate gradients on M1 x = v from a seeded vector give the
// Lanczos tridiagonal matrix (diagonal 1/alpha_k + beta_{k-1}/alpha_{k-1},
// off-diagonal sqrt(beta_k)/alpha_k), whose extreme eigenvalues approach those
// of P M1 from inside.
void sd_spectrum(int64_t F, int64_t E, const std::vector<double>& M1, const std::vector<int32_t>& tri,
                 const std::vector<float>& Pinv, int iters, double* lmin, double* lmax) {
  const int64_t n_u = 3 * (E + F), T = E + F;
  std::vector<double> x(n_u, 0.0), r(n_u), z(n_u), p(n_u), q(n_u);
  uint64_t s = 7706;
  for (auto& v : r) {  // seeded uniform(-1, 1) start (xorshift)
    s ^= s << 13; s ^= s >> 7; s ^= s << 17;
    v = (double)(s >> 11) / 9007199254740992.0 * 2.0 - 1.0;
  }
  auto precond = [&](const std::vector<double>& in, std::vector<double>& out) {
    for (int64_t t = 0; t < T; ++t) {
      const float* P = &Pinv[8 * t];
      const double a = in[3 * t], b = in[3 * t + 1], c = in[3 * t + 2];
      out[3 * t] = P[0] * a + P[1] * b + P[2] * c;
      out[3 * t + 1] = P[1] * a + P[3] * b + P[4] * c;
      out[3 * t + 2] = P[2] * a + P[4] * b + P[5] * c;
    }
  };
  precond(r, z);
  p = z;
  double rz = 0.0;
  for (int64_t i = 0; i < n_u; ++i) rz += r[i] * z[i];
  std::vector<double> al, be, diag, off;
  for (int k = 0; k < iters; ++k) {
    m1_apply(F, M1, tri, p.data(), q.data(), n_u);
    double pq = 0.0;
    for (int64_t i = 0; i < n_u; ++i) pq += p[i] * q[i];
    const double alpha = rz / pq;
    for (int64_t i = 0; i < n_u; ++i) r[i] -= alpha * q[i];
    precond(r, z);
    double rz1 = 0.0;
    for (int64_t i = 0; i < n_u; ++i) rz1 += r[i] * z[i];
    const double beta = rz1 / rz;
    al.push_back(alpha);
    be.push_back(beta);
    for (int64_t i = 0; i < n_u; ++i) p[i] = z[i] + beta * p[i];
    rz = rz1;
    if (!(rz > 0.0)) break;
  }
  const size_t m = al.size();
  if (m < 2) throw std::runtime_error("Lanczos estimate of the preconditioned spectrum failed");
  for (size_t k = 0; k < m; ++k) {
    diag.push_back(1.0 / al[k] + (k ? be[k - 1] / al[k - 1] : 0.0));
    if (k + 1 < m) off.push_back(std::sqrt(be[k]) / al[k]);
  }
  double lo = 1e300, hi = -1e300;
  for (size_t k = 0; k < m; ++k) {
    const double rad = std::fabs(k ? off[k - 1] : 0.0) + std::fabs(k + 1 < m ? off[k] : 0.0);
    lo = std::min(lo, diag[k] - rad);
    hi = std::max(hi, diag[k] + rad);
  }
  *lmin = tridiag_eig(diag, off, 0, lo, hi);
  *lmax = tridiag_eig(diag, off, (int)m - 1, lo, hi);
}

// Inner iterations per refinement sweep: the smallest k for which the
// Chebyshev polynomial on [a, b] reduces the error by inner_rtol,
// 2 / (c^k + c^-k) <= inner_rtol with c = (sqrt(b/a) + 1) / (sqrt(b/a) - 1).
int sd_iterations(double a, double b, double inner_rtol) {
  const double sk = std::sqrt(b / a), c = (sk + 1.0) / (sk - 1.0);
  int k = 1;
  while (k < 1000 && 2.0 / (std::pow(c, k) + std::pow(c, -k)) > inner_rtol) ++k;
  return k;
}

}  // namespace pavg
