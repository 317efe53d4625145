// C-ABI of libpavg (declared in include/pavg.h): context lifetime, buffers and
// the host-side sequencing of the kernels in device.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <random>
#include <string>
#include <vector>

#include "device.h"

using namespace pavg;

#include "api_internal.h"

namespace pavg_api {

#ifndef PAVG_MIXED_SOLVE_RTOL
#define PAVG_MIXED_SOLVE_RTOL 1e-5
#endif
// Relative residual at which mass solves stop in mixed precision.
constexpr double kMixedSolveRtol = PAVG_MIXED_SOLVE_RTOL;
// Bound of every wait of the subdomain solver on another block: about 2 s of
// the SM clock (2.07 GHz).
constexpr long long kSdWaitCycles = 4000000000LL;

int set_err(pavg_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

void begin_call(pavg_ctx* ctx) {
  ctx->launches = 0;
  ctx->cur_pairs.clear();
  ctx->ev_used = 0;
}

void end_call(pavg_ctx* ctx) {
  ctx->last_launches = ctx->launches;
  ctx->last_pairs = ctx->cur_pairs;
}

struct CallScope {
  pavg_ctx* ctx;
  explicit CallScope(pavg_ctx* c) : ctx(c) { begin_call(c); }
  ~CallScope() { end_call(ctx); }
};

cudaEvent_t next_event(pavg_ctx* ctx) {
  cudaEvent_t e = nullptr;
  if (ctx->capturing) {  // owned by the plan: replays re-record it
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  if (ctx->ev_used < ctx->ev_pool.size()) return ctx->ev_pool[ctx->ev_used++];
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  ctx->ev_pool.push_back(e);
  ctx->ev_used = ctx->ev_pool.size();
  return e;
}

// ---------------------------------------------------------------- building blocks
// velocity part out_u = M1^{-1} b (scaled, plus add); eta part by the caller.
int enq_cg(pavg_ctx* ctx, const double* b, double* out, double scale, const double* add, cudaStream_t st) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ctx->timing) {
    e0 = next_event(ctx);
    e1 = next_event(ctx);
    if (!e0 || !e1) return set_err(ctx, PAVG_ERR_CUDA, "event creation failed");
    // inside a stream capture an event becomes a graph record node only with
    // cudaEventRecordExternal (a plain record is a capture dependency)
    CK(cudaEventRecordWithFlags(e0, st, ctx->capturing ? cudaEventRecordExternal : cudaEventRecordDefault));
  }
  if (ctx->use_sd)
    KL(launch_cheb_sd(ctx->dm, ctx->sd, ctx->sdw, ctx->sdp, b, out, scale, add, st));
  else if (ctx->p.solver == PAVG_SOLVER_FP64)
    KL(launch_cg(ctx->dm, ctx->cg, ctx->cgp, b, out, scale, add, st));
  else
    KL(launch_cg_ir(ctx->dm, ctx->cgi, ctx->cgip, b, out, scale, add, st));
  if (ctx->timing) {
    CK(cudaEventRecordWithFlags(e1, st, ctx->capturing ? cudaEventRecordExternal : cudaEventRecordDefault));
    ctx->cur_pairs.emplace_back(e0, e1);
    if (ctx->capturing) ctx->capturing->pairs.emplace_back(e0, e1);
  }
  return PAVG_OK;
}

// out = M^{-1} R (both parts).
int enq_mass_solve(pavg_ctx* ctx, const double* R, double* out, cudaStream_t st) {
  const DeviceMesh& m = ctx->dm;
  int rc = enq_cg(ctx, R, out, 1.0, nullptr, st);
  if (rc) return rc;
  KL(launch_m2inv(m, R + m.n_u, 0, out + m.n_u, 0, 1, st));
  return PAVG_OK;
}

// One step of the Chebyshev / Clenshaw recurrences:
//   out = M^{-1}(y + s Khat in) + z,   Khat = [[-C, g D^T], [-H D, 0]]
// with in, y, z optional (null = 0).  L = M^{-1} Khat (Sec. 2.5).
int enq_step(pavg_ctx* ctx, const double* in, double s, const double* y, const double* z, double* out,
             cudaStream_t st) {
  const DeviceMesh& m = ctx->dm;
  const int64_t nu = m.n_u;
  if (in) {
    CK(cudaMemsetAsync(ctx->ru, 0, sizeof(double) * 3 * m.E, st));
    KL(launch_apply_K(m, in, s, ctx->p.g, ctx->p.H, y, y ? y + nu : nullptr, z ? z + nu : nullptr, ctx->ru,
                      out + nu, st, ctx->p.precision == PAVG_PRECISION_MIXED));
    return enq_cg(ctx, ctx->ru, out, 1.0, z, st);
  }
  // in == 0: out = M^{-1} y + z
  if (!y) return set_err(ctx, PAVG_ERR_INVAL, "internal: empty recurrence step");
  int rc = enq_cg(ctx, y, out, 1.0, z, st);
  if (rc) return rc;
  KL(launch_m2inv(m, y + nu, 0, out + nu, 0, 1, st));
  if (z) KL(launch_lincomb(out + nu, 1.0, out + nu, 1.0, z + nu, 0.0, nullptr, m.n_eta, st));
  return PAVG_OK;
}

int enq_linear(pavg_ctx* ctx, const double* U, double* out, cudaStream_t st) {
  return enq_step(ctx, U, 1.0, nullptr, nullptr, out, st);
}

int enq_nonlinear(pavg_ctx* ctx, const double* U, double* out, double* scratch, cudaStream_t st) {
  const DeviceMesh& m = ctx->dm;
  CK(cudaMemsetAsync(scratch, 0, sizeof(double) * 3 * m.E, st));
  KL(launch_nonlinear_rhs(m, U, scratch, 1, ctx->p.upwind_convention, st,
                          ctx->p.precision == PAVG_PRECISION_MIXED, ctx->facets, ctx->facet_chunk));
  return enq_mass_solve(ctx, scratch, out, st);
}

// out = e^{tL} U (Sec. 2.4): X = sgn(t) L / lambda_max, Q_0 = U, Q_1 = X U,
// Q_{k+1} = 2 X Q_k + Q_{k-1}; out = sum_k c_k(lambda |t|) Q_k.
int enq_expL(pavg_ctx* ctx, double t, const double* U, double* out, cudaStream_t st) {
  const int64_t n = ctx->dm.n;
  if (t == 0.0) {
    CK(cudaMemcpyAsync(out, U, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    ctx->last_degree = 0;
    return PAVG_OK;
  }
  std::vector<double> c = cheb_coefficients(ctx->lam * std::fabs(t), ctx->p.cheb_tol);
  if (c.empty()) return set_err(ctx, PAVG_ERR_INVAL, cheb_limit_msg(ctx->lam * std::fabs(t)));
  const int K = (int)c.size() - 1;
  ctx->last_degree = K;
  const double sgn = t > 0 ? 1.0 : -1.0;
  double* acc = ctx->vec[3];
  KL(launch_lincomb(acc, c[0], U, 0.0, nullptr, 0.0, nullptr, n, st));
  const double* qm1 = nullptr;
  const double* qk = U;
  double* bufs[3] = {ctx->vec[0], ctx->vec[1], ctx->vec[2]};
  for (int k = 0; k < K; ++k) {
    double* qn = bufs[k % 3];
    int rc = enq_step(ctx, qk, (k == 0 ? 1.0 : 2.0) * sgn / ctx->lam, nullptr, qm1, qn, st);
    if (rc) return rc;
    KL(launch_lincomb(acc, 1.0, acc, c[k + 1], qn, 0.0, nullptr, n, st));
    qm1 = qk;
    qk = qn;
  }
  CK(cudaMemcpyAsync(out, acc, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  return PAVG_OK;
}

void drop_graph(AvgPlan* pl) {
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  pl->exec = nullptr;
  for (auto& pr : pl->pairs) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
  pl->pairs.clear();
  pl->launches = 0;
}

int ensure_avg_workspace(pavg_ctx* ctx, int K, int M) {
  const int64_t n = ctx->dm.n;
  if (K <= ctx->Kcap && M <= ctx->Mcap) return PAVG_OK;
  // buffers move: drop every captured graph that refers to them
  cudaDeviceSynchronize();
  for (auto& kv : ctx->plans) drop_graph(&kv.second);
  int nk = std::max(K, ctx->Kcap), nm = std::max(M, ctx->Mcap);
  cudaFree(ctx->Q); cudaFree(ctx->Um); cudaFree(ctx->Rm);
  ctx->Q = ctx->Um = ctx->Rm = nullptr;
  ctx->Kcap = -1; ctx->Mcap = 0;
  if (dalloc(&ctx->Q, (size_t)(nk + 1) * n) != cudaSuccess || dalloc(&ctx->Um, (size_t)nm * n) != cudaSuccess ||
      dalloc(&ctx->Rm, (size_t)nm * n) != cudaSuccess)
    return set_err(ctx, PAVG_ERR_NOMEM, "averaged_rhs workspace allocation failed");
  ctx->Kcap = nk;
  ctx->Mcap = nm;
  return PAVG_OK;
}

int get_plan(pavg_ctx* ctx, double T, int M, AvgPlan** out, int m0, int m1) {
  if (m1 < 0) m1 = M;
  if (M < 1 || m0 < 0 || m1 > M || m0 >= m1) return set_err(ctx, PAVG_ERR_INVAL, "invalid shift group");
  auto key = std::make_tuple(T, M, m0, m1);
  auto it = ctx->plans.find(key);
  if (it != ctx->plans.end()) { *out = &it->second; return PAVG_OK; }
  std::vector<double> s_all, w_all;
  int rc = shifts_weights(T, M, ctx->p.quad_rule, &s_all, &w_all);
  if (rc) return set_err(ctx, rc, "invalid T / M / quadrature rule");
  const std::vector<double> s(s_all.begin() + m0, s_all.begin() + m1), w(w_all.begin() + m0, w_all.begin() + m1);
  const int Mrule = M;
  M = m1 - m0;
  std::vector<std::vector<double>> cs(M);
  int K = 0;
  for (int m = 0; m < M; ++m) {
    cs[m] = cheb_coefficients(ctx->lam * std::fabs(s[m]), ctx->p.cheb_tol);
    if (cs[m].empty()) return set_err(ctx, PAVG_ERR_INVAL, cheb_limit_msg(ctx->lam * std::fabs(s[m])));
    K = std::max(K, (int)cs[m].size() - 1);
  }
  AvgPlan pl;
  pl.T = T; pl.M = M; pl.K = K; pl.M_rule = Mrule; pl.m0 = m0;
  const int tile = combine_tile();
  // Pairs: every shift s > 0 with a partner -s of the same coefficients and
  // weight (the midpoint rule with even M, and symmetric groups of it); the
  // contractions then run once per pair (E +/- O).  Pairs ordered by
  // decreasing degree, rows 2p (s > 0) and 2p + 1 (s < 0) of U_m and r_m.
  {
    std::vector<int> pos, used(M, 0);
    std::vector<std::pair<int, int>> pairs;
    for (int m = 0; m < M; ++m)
      if (s[m] > 0.0) pos.push_back(m);
    bool ok = 2 * (int)pos.size() == M;
    for (int a : pos) {
      if (!ok) break;
      int b = -1;
      for (int m = 0; m < M && b < 0; ++m)
        if (!used[m] && s[m] == -s[a] && w[m] == w[a] && cs[m] == cs[a]) b = m;
      if (b < 0) ok = false;
      else { used[b] = 1; pairs.emplace_back(a, b); }
    }
    if (ok && !pairs.empty()) {
      std::stable_sort(pairs.begin(), pairs.end(),
                       [&](const std::pair<int, int>& x, const std::pair<int, int>& y) {
                         return cs[x.first].size() > cs[y.first].size();
                       });
      const int P = (int)pairs.size();
      std::vector<double> Ap((size_t)P * (K + 1), 0.0), Bp((size_t)(K + 1) * P, 0.0);
      for (int p = 0; p < P; ++p) {
        const int m = pairs[p].first;
        for (int k = 0; k < (int)cs[m].size(); ++k) {
          Ap[(size_t)p * (K + 1) + k] = cs[m][k];
          Bp[(size_t)k * P + p] = w[m] * cs[m][k];
        }
      }
      std::vector<int> la((P + tile - 1) / tile), lb((K + 1 + tile - 1) / tile);
      for (size_t j = 0; j < la.size(); ++j) la[j] = (int)cs[pairs[j * tile].first].size();
      for (size_t j = 0; j < lb.size(); ++j) {
        int cnt = 0;
        for (int p = 0; p < P; ++p) cnt += (int)cs[pairs[p].first].size() > (int)(j * tile) ? 1 : 0;
        lb[j] = cnt;
      }
      if (upload(&pl.dAp, Ap) != cudaSuccess || upload(&pl.dBp, Bp) != cudaSuccess ||
          upload(&pl.dlimAp, la) != cudaSuccess || upload(&pl.dlimBp, lb) != cudaSuccess) {
        cudaFree(pl.dAp); cudaFree(pl.dBp); cudaFree(pl.dlimAp); cudaFree(pl.dlimBp);
        return set_err(ctx, PAVG_ERR_NOMEM, "plan upload failed");
      }
      pl.P = P;
      auto res = ctx->plans.emplace(key, pl);
      *out = &res.first->second;
      return PAVG_OK;
    }
  }
  // Shifts ordered by decreasing degree K_m: each 8-row tile of the forward
  // table then uses a prefix of the k range, and each 8-row tile of the
  // backward table a prefix of the shifts; the contractions skip the zeros.
  std::vector<int> ord(M);
  for (int m = 0; m < M; ++m) ord[m] = m;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return cs[a].size() > cs[b].size(); });
  std::vector<double> A((size_t)M * (K + 1), 0.0), B((size_t)(K + 1) * M, 0.0);
  for (int r = 0; r < M; ++r) {
    const int m = ord[r];
    double sg = s[m] >= 0 ? 1.0 : -1.0;
    double fw = 1.0, bw = 1.0;  // sgn^k and (-sgn)^k
    for (int k = 0; k <= K; ++k) {
      double ck = k < (int)cs[m].size() ? cs[m][k] : 0.0;
      A[(size_t)r * (K + 1) + k] = ck * fw;
      B[(size_t)k * M + r] = w[m] * ck * bw;
      fw *= sg;
      bw *= -sg;
    }
  }
  std::vector<int> limA((M + tile - 1) / tile), limB((K + 1 + tile - 1) / tile);
  for (size_t j = 0; j < limA.size(); ++j) limA[j] = (int)cs[ord[j * tile]].size();
  for (size_t j = 0; j < limB.size(); ++j) {
    int cnt = 0;
    for (int r = 0; r < M; ++r) cnt += (int)cs[ord[r]].size() > (int)(j * tile) ? 1 : 0;
    limB[j] = cnt;
  }
  if (upload(&pl.dA, A) != cudaSuccess || upload(&pl.dB, B) != cudaSuccess || upload(&pl.dlimA, limA) != cudaSuccess ||
      upload(&pl.dlimB, limB) != cudaSuccess)
    return set_err(ctx, PAVG_ERR_NOMEM, "plan upload failed");
  auto res = ctx->plans.emplace(key, pl);
  *out = &res.first->second;
  return PAVG_OK;
}

int enq_avg_shifts(pavg_ctx* ctx, const AvgPlan& pl, cudaStream_t st) {
  const DeviceMesh& m = ctx->dm;
  const int64_t n = m.n;
  const int K = pl.K, M = pl.M;
  double* Q = ctx->Q;
  const bool fp32 = ctx->p.precision == PAVG_PRECISION_MIXED;
  if (pl.P > 0) KL(launch_combine_pairs_fwd(pl.dAp, pl.P, K + 1, pl.dlimAp, Q, n, ctx->Um, n, n, st, fp32));
  else KL(launch_combine(pl.dA, M, K + 1, pl.dlimA, Q, n, ctx->Um, n, n, st, fp32));
  CK(cudaMemset2DAsync(ctx->Rm, sizeof(double) * n, 0, sizeof(double) * 3 * m.E, M, st));
  KL(launch_nonlinear_rhs(m, ctx->Um, ctx->Rm, M, ctx->p.upwind_convention, st, fp32, ctx->facets, ctx->facet_chunk));
  // the weighted sum over shifts stays FP64 in every precision: the average
  // cancels most of the oscillating terms, so rounding here is amplified
  if (pl.P > 0) KL(launch_combine_pairs_bwd(pl.dBp, K + 1, pl.P, pl.dlimBp, ctx->Rm, n, Q, n, n, st));
  else KL(launch_combine(pl.dB, K + 1, M, pl.dlimB, ctx->Rm, n, Q, n, n, st));  // y_k overwrite Q_k
  return PAVG_OK;
}

// Shared-basis averaged nonlinearity (Sec. 2.2, Eq. vt_discretised):
//   U_m = sum_k c_k(lam|s_m|) sgn(s_m)^k Q_k,  Q_k = Q_k(L/lam) U      (forward)
//   r_m = weak-form N(U_m)                                             (Sec. 2.5)
//   y_k = sum_m w_m c_k(lam|s_m|) (-sgn s_m)^k r_m
//   S   = sum_k Q_k(L/lam) M^{-1} y_k by Clenshaw:
//         b_k = M^{-1}(y_k + (2/lam) Khat b_{k+1}) + b_{k+2},
//         S   = M^{-1}(y_0 + Khat b_1 / lam) + b_2.
// Equal to sum_m w_m e^{-s_m L} M^{-1} r_m term by term because every factor is
// a polynomial in the one operator L.
int enq_avg(pavg_ctx* ctx, const AvgPlan& pl, const double* U, double* out, cudaStream_t st) {
  const DeviceMesh& m = ctx->dm;
  const int64_t n = m.n;
  const int K = pl.K;
  if (pl.T == 0.0) {  // every weight is 1/M: the group's share of N(U)
    int rc = enq_nonlinear(ctx, U, out, ctx->Rm, st);
    if (rc || pl.M == pl.M_rule) return rc;
    KL(launch_lincomb(out, (double)pl.M / pl.M_rule, out, 0.0, nullptr, 0.0, nullptr, n, st));
    return PAVG_OK;
  }
  double* Q = ctx->Q;
  if (U != Q) CK(cudaMemcpyAsync(Q, U, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  for (int k = 0; k < K; ++k) {
    int rc = enq_step(ctx, Q + (int64_t)k * n, (k == 0 ? 1.0 : 2.0) / ctx->lam, nullptr,
                      k == 0 ? nullptr : Q + (int64_t)(k - 1) * n, Q + (int64_t)(k + 1) * n, st);
    if (rc) return rc;
  }
  int rc0 = enq_avg_shifts(ctx, pl, st);
  if (rc0) return rc0;
  double* b[3] = {ctx->vec[0], ctx->vec[1], ctx->vec[2]};
  const double* b1 = nullptr;  // b_{k+1}
  const double* b2 = nullptr;  // b_{k+2}
  for (int k = K; k >= 1; --k) {
    double* bk = b[k % 3];
    int rc = enq_step(ctx, b1, 2.0 / ctx->lam, Q + (int64_t)k * n, b2, bk, st);
    if (rc) return rc;
    b2 = b1;
    b1 = bk;
  }
  int rc = enq_step(ctx, b1, 1.0 / ctx->lam, Q, b2, out, st);
  if (rc) return rc;
  ctx->last_degree = K;
  return PAVG_OK;
}

int run_avg(pavg_ctx* ctx, double T, int M, const double* U, double* out, cudaStream_t st, int m0, int m1) {
  AvgPlan* pl = nullptr;
  int rc = get_plan(ctx, T, M, &pl, m0, m1);
  if (rc) return rc;
  rc = ensure_avg_workspace(ctx, pl->K, pl->M);
  if (rc) return rc;
  const int64_t n = ctx->dm.n;
  if (!ctx->use_graphs) return enq_avg(ctx, *pl, U, out, st);
  if (pl->exec && pl->timed != ctx->timing) drop_graph(pl);
  if (!pl->exec) {
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    ctx->capturing = pl;
    ctx->launches = 0;
    int rc2 = enq_avg(ctx, *pl, ctx->io_in, ctx->io_out, ctx->cap_stream);
    ctx->capturing = nullptr;
    pl->launches = ctx->launches;
    pl->timed = ctx->timing;
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
    if (rc2) { if (graph) cudaGraphDestroy(graph); return rc2; }
    if (e != cudaSuccess) return set_err(ctx, PAVG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&pl->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { pl->exec = nullptr; return set_err(ctx, PAVG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e)); }
  }
  CK(cudaMemcpyAsync(ctx->io_in, U, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  CK(cudaGraphLaunch(pl->exec, st));
  CK(cudaMemcpyAsync(out, ctx->io_out, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  ctx->last_degree = pl->K;
  ctx->launches += pl->launches;
  ctx->cur_pairs.insert(ctx->cur_pairs.end(), pl->pairs.begin(), pl->pairs.end());
  return PAVG_OK;
}

double host_winner(pavg_ctx* ctx, const double* U, const double* V) {
  int nb = 0;
  if (launch_winner(ctx->dm, U, V, ctx->p.g, ctx->p.H, ctx->dpart, &nb, 0) != cudaSuccess) return NAN;
  if (cudaMemcpy(ctx->host_part, ctx->dpart, sizeof(double) * nb, cudaMemcpyDeviceToHost) != cudaSuccess) return NAN;
  double s = 0;
  for (int i = 0; i < nb; ++i) s += ctx->host_part[i];
  return s;
}

// Sec. 2.4 needs |lambda_max|; the paper does not say how it is found.  Power
// iteration on -L^2 (self-adjoint, positive semi-definite in the energy inner
// product) from a seeded random start; the Rayleigh quotient approaches
// lambda_max^2 from below, so the estimate is widened by 2 %.
int estimate_lambda(pavg_ctx* ctx) {
  const int64_t n = ctx->dm.n;
  std::mt19937_64 rng(7706);
  std::normal_distribution<double> nd;
  std::vector<double> h(n);
  for (auto& x : h) x = nd(rng);
  double *v = ctx->vec[4], *Lv = ctx->vec[5], *w = ctx->vec[3];
  if (cudaMemcpy(v, h.data(), sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess)
    return set_err(ctx, PAVG_ERR_CUDA, "lambda_max: upload failed");
  double nv = std::sqrt(host_winner(ctx, v, v));
  if (!(nv > 0) || launch_lincomb(v, 1.0 / nv, v, 0, nullptr, 0, nullptr, n, 0) != cudaSuccess)
    return set_err(ctx, PAVG_ERR_CUDA, "lambda_max: normalisation failed");
  double est = 0;
  for (int it = 0; it < 400; ++it) {
    int rc = enq_linear(ctx, v, Lv, 0);
    if (rc) return rc;
    double rq = host_winner(ctx, Lv, Lv);
    rc = enq_linear(ctx, Lv, w, 0);
    if (rc) return rc;
    double nw = std::sqrt(host_winner(ctx, w, w));
    if (!(nw > 0) || !std::isfinite(rq)) return set_err(ctx, PAVG_ERR_NONFINITE, "lambda_max: iteration failed");
    if (launch_lincomb(v, -1.0 / nw, w, 0, nullptr, 0, nullptr, n, 0) != cudaSuccess)
      return set_err(ctx, PAVG_ERR_CUDA, "lambda_max: update failed");
    double nest = std::sqrt(rq);
    if (est > 0 && std::fabs(nest - est) <= 1e-9 * nest) { est = nest; break; }
    est = nest;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return set_err(ctx, PAVG_ERR_CUDA, "lambda_max: sync failed");
  ctx->lam = 1.02 * est;
  return PAVG_OK;
}

int check_flags(pavg_ctx* ctx) {
  int f = 0;
  if (cudaMemcpy(&f, ctx->cg.flags, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return set_err(ctx, PAVG_ERR_CUDA, "reading device flags failed");
  if (f & kFlagTimeout) return set_err(ctx, PAVG_ERR_TIMEOUT, "a bounded device-side wait timed out");
  if (f & kFlagNonFinite) return set_err(ctx, PAVG_ERR_NONFINITE, "non-finite value detected");
  if (f & kFlagNoConv) return set_err(ctx, PAVG_ERR_NOCONV, "M1 CG did not converge within cg_maxit");
  return PAVG_OK;
}

// Meshes and their operator data are shared by every context with the same
// refinement, radius, rotation rate and geometry on one device: they are
// read-only after set-up, and instances that share them also share their L2
// footprint.
std::mutex g_mesh_mu;
std::map<pavg_detail::MeshKey, SharedMesh*> g_meshes;

void free_device_mesh(DeviceMesh& m) {
  cudaFree(m.cell_edges); cudaFree(m.cell_aligned); cudaFree(m.edge_plus); cudaFree(m.edge_minus);
  cudaFree(m.edge_lpos); cudaFree(m.M1); cudaFree(m.C); cudaFree(m.det); cudaFree(m.G); cudaFree(m.dinv);
  cudaFree(m.M1f); cudaFree(m.Pinv); cudaFree(m.M1p); cudaFree(m.tri);
  cudaFree(m.M2e); cudaFree(m.M2i); cudaFree(m.geo_c); cudaFree(m.geo_f); cudaFree(m.Cf);
  m = DeviceMesh();
}

int build_shared_mesh(const pavg_params* p, SharedMesh* sh, std::string* why) {
  build_mesh(p->refinement, p->radius, &sh->mesh);
  RefElement el;
  build_reference_element(&el);
  HostCellData hc;
  ConstTables tab;
  TablesP3<double> tab3;
  const bool cubic = p->geometry_degree == 3;
  build_cell_data(sh->mesh, el, p->omega, p->geometry_degree, &hc, &tab, &tab3);
  if (upload_tables(tab) != cudaSuccess || upload_chain_tables(tab) != cudaSuccess ||
      (cubic && upload_tables3(tab3) != cudaSuccess)) {
    *why = "constant upload failed";
    return PAVG_ERR_CUDA;
  }
  const Mesh& ms = sh->mesh;
  DeviceMesh& m = sh->dm;
  m.F = ms.F(); m.E = ms.E(); m.n_u = 3 * m.E + 3 * m.F; m.n_eta = 3 * m.F; m.n = m.n_u + m.n_eta;
  std::vector<int32_t> ce(3 * m.F);
  for (int64_t c = 0; c < m.F; ++c)
    for (int i = 0; i < 3; ++i) ce[i * m.F + c] = ms.cell_edges[3 * c + i];
  // FP32 element matrices both packed (shared-memory residency) and in row
  // blocks (streamed): either solver path may run on any mesh
  const bool ok = upload(&m.cell_edges, ce) == cudaSuccess && upload(&m.cell_aligned, ms.cell_aligned) == cudaSuccess &&
                  upload(&m.edge_plus, ms.edge_plus) == cudaSuccess && upload(&m.edge_minus, ms.edge_minus) == cudaSuccess &&
                  upload(&m.edge_lpos, ms.edge_lpos) == cudaSuccess && upload(&m.M1, hc.M1) == cudaSuccess &&
                  upload(&m.C, hc.C) == cudaSuccess && upload(&m.det, hc.det) == cudaSuccess &&
                  upload(&m.G, hc.G) == cudaSuccess && upload(&m.dinv, hc.dinv) == cudaSuccess &&
                  upload(&m.Pinv, hc.Pinv) == cudaSuccess && upload(&m.tri, hc.tri) == cudaSuccess &&
                  upload(&m.M1p, hc.M1p) == cudaSuccess && upload(&m.M1f, hc.M1f) == cudaSuccess &&
                  upload(&m.Cf, std::vector<float>(hc.C.begin(), hc.C.end())) == cudaSuccess &&
                  (!cubic || (upload(&m.M2e, hc.M2e) == cudaSuccess && upload(&m.M2i, hc.M2i) == cudaSuccess &&
                              upload(&m.geo_c, hc.geo_c) == cudaSuccess && upload(&m.geo_f, hc.geo_f) == cudaSuccess));
  if (!ok) {
    free_device_mesh(m);
    *why = "device upload failed";
    return PAVG_ERR_NOMEM;
  }
  // the subdomain solver's Chebyshev interval (the partitions are built per
  // part count when a context asks for one)
  try {
    sd_spectrum(m.F, m.E, hc.M1, hc.tri, hc.Pinv, 40, &sh->sd_lmin, &sh->sd_lmax);
  } catch (const std::exception&) {
    sh->sd_lmin = sh->sd_lmax = 0.0;
  }
  sh->tri = hc.tri;
  return PAVG_OK;
}

// The subdomain partition of a shared mesh into P parts (built on first use;
// P = 0 in the result when it does not fit).  Called under g_mesh_mu.
int sd_partition_for(SharedMesh* sh, int P, SdMesh* out, std::string* why) {
  auto it = sh->sds.find(P);
  if (it == sh->sds.end()) {
    SdMesh sd;
    if (sd_configure(sh->dm.F, sh->dm.E, sh->tri, sh->sd_lmin, sh->sd_lmax, P, &sd) != cudaSuccess) {
      *why = "subdomain solver set-up failed";
      return PAVG_ERR_CUDA;
    }
    it = sh->sds.emplace(P, sd).first;
  }
  *out = it->second;
  return PAVG_OK;
}

int acquire_mesh(const pavg_params* p, int device, SharedMesh** out, std::string* why) {
  std::lock_guard<std::mutex> lock(g_mesh_mu);
  const pavg_detail::MeshKey key = std::make_tuple(p->refinement, p->radius, p->omega, device, p->geometry_degree);
  auto it = g_meshes.find(key);
  if (it != g_meshes.end()) {
    ++it->second->refs;
    *out = it->second;
    return PAVG_OK;
  }
  std::unique_ptr<SharedMesh> sh(new SharedMesh());
  int rc = build_shared_mesh(p, sh.get(), why);
  if (rc) return rc;
  sh->refs = 1;
  sh->key = key;
  g_meshes.emplace(key, sh.get());
  *out = sh.release();
  return PAVG_OK;
}

void release_mesh(SharedMesh* sh) {
  if (!sh) return;
  std::lock_guard<std::mutex> lock(g_mesh_mu);
  if (--sh->refs > 0) return;
  g_meshes.erase(sh->key);
  free_device_mesh(sh->dm);
  for (auto& kv : sh->sds) sd_free(&kv.second);
  delete sh;
}

void free_ctx(pavg_ctx* c) {
  if (!c) return;
  for (auto& kv : c->plans) {
    drop_graph(&kv.second);
    cudaFree(kv.second.dlimA);
    cudaFree(kv.second.dlimB);
    cudaFree(kv.second.dA);
    cudaFree(kv.second.dB);
    cudaFree(kv.second.dAp);
    cudaFree(kv.second.dBp);
    cudaFree(kv.second.dlimAp);
    cudaFree(kv.second.dlimBp);
  }
  DeviceMesh& m = c->dm;
  cudaFree(m.topo);
  release_mesh(c->shared);
  CgWork& w = c->cg;
  cudaFree(w.x); cudaFree(w.r[0]); cudaFree(w.r[1]); cudaFree(w.s[0]); cudaFree(w.s[1]);
  cudaFree(w.w[0]); cudaFree(w.w[1]); cudaFree(w.w[2]); cudaFree(w.p); cudaFree(w.partial);
  cudaFree(w.bar); cudaFree(w.flags); cudaFree(w.stats);
  CgIrWork& wi = c->cgi;
  cudaFree(wi.x[0]); cudaFree(wi.x[1]); cudaFree(wi.ax); cudaFree(wi.r64); cudaFree(wi.fbuf);
  cudaFree(wi.partial); cudaFree(wi.partial_f);
  cudaFree(wi.bar); cudaFree(wi.scal); cudaFree(wi.tag);
  sd_free_work(&c->sdw);
  cudaFree(c->ru);
  cudaFree(c->facets);
  for (auto* v : c->vec) cudaFree(v);
  cudaFree(c->io_in); cudaFree(c->io_out); cudaFree(c->Q); cudaFree(c->Um); cudaFree(c->Rm);
  cudaFree(c->ts);
  cudaFree(c->dpart);
  if (c->host_part) cudaFreeHost(c->host_part);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  delete c;
}

bool valid_params(const pavg_params* p) {
  return p && p->refinement >= 0 && p->refinement <= 8 && p->radius > 0 && p->g > 0 && p->H > 0 &&
         p->cheb_tol > 0 && p->cg_rtol > 0 && p->cg_maxit > 0 && p->lambda_max >= 0 && std::isfinite(p->omega) &&
         (p->quad_rule == PAVG_QUAD_MIDPOINT || p->quad_rule == PAVG_QUAD_CLOSED) &&
         (p->upwind_convention == PAVG_UPWIND_STANDARD || p->upwind_convention == PAVG_UPWIND_AS_PRINTED) &&
         (p->solver == PAVG_SOLVER_MIXED || p->solver == PAVG_SOLVER_FP64 || p->solver == PAVG_SOLVER_SUBDOMAIN) &&
         (p->precision == PAVG_PRECISION_FP64 || p->precision == PAVG_PRECISION_MIXED) && p->sd_part_cells >= 0 &&
         (p->geometry_degree == 1 || p->geometry_degree == 3);
}

}  // namespace pavg_api

using namespace pavg_api;

extern "C" {

int pavg_default_params(pavg_params* p) {
  if (!p) return PAVG_ERR_INVAL;
  p->refinement = 3;
  p->radius = 6.37122e6;
  p->omega = 7.292e-5;
  p->g = 9.80616;
  p->H = 5000.0;
  p->cheb_tol = 1e-6;
  p->cg_rtol = 1e-14;
  p->cg_maxit = 400;
  p->lambda_max = 0.0;
  p->quad_rule = PAVG_QUAD_MIDPOINT;
  p->upwind_convention = PAVG_UPWIND_STANDARD;
  p->solver = PAVG_SOLVER_SUBDOMAIN;
  p->precision = PAVG_PRECISION_FP64;
  p->sd_part_cells = 0;
  p->geometry_degree = 1;
  return PAVG_OK;
}

int pavg_create(const pavg_params* p, pavg_ctx** out) {
  if (!out) return PAVG_ERR_INVAL;
  *out = nullptr;
  if (!valid_params(p)) return PAVG_ERR_INVAL;
  pavg_ctx* ctx = new pavg_ctx();
  static std::atomic<uint64_t> next_uid{1};
  ctx->uid = next_uid++;
  ctx->p = *p;
  ctx->cgp.rtol = p->cg_rtol;
  ctx->cgp.maxit = p->cg_maxit;
  const bool mixed = p->precision == PAVG_PRECISION_MIXED;
  if (mixed) ctx->cgp.rtol = std::max(p->cg_rtol, kMixedSolveRtol);
  ctx->cgip.rtol = mixed ? std::max(p->cg_rtol, kMixedSolveRtol) : p->cg_rtol;
  ctx->cgip.max_sweeps = 8;
  ctx->cgip.inner_rtol = mixed ? 1e-6f : 1e-5f;
  ctx->cgip.max_inner = p->cg_maxit < 200 ? p->cg_maxit : 200;
  int rc = PAVG_OK;
  try {
    cudaGetDevice(&ctx->device);
    SharedMesh* sh = nullptr;
    std::string why;
    if ((rc = acquire_mesh(p, ctx->device, &sh, &why))) { set_err(ctx, rc, why); throw 0; }
    ctx->shared = sh;
    ctx->mesh = sh->mesh;
    ctx->dm = sh->dm;
    if (p->solver == PAVG_SOLVER_SUBDOMAIN) {
      int sms = 0;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
      const int64_t F = sh->dm.F;
      const int64_t want = p->sd_part_cells > 0 ? (F + p->sd_part_cells - 1) / p->sd_part_cells : F / 32;
      const int P = (int)std::max<int64_t>(1, std::min<int64_t>(sms, want));
      std::lock_guard<std::mutex> lock(g_mesh_mu);
      if ((rc = sd_partition_for(sh, P, &ctx->sd, &why))) { set_err(ctx, rc, why); throw 0; }
    }
    DeviceMesh& m = ctx->dm;
    bool ok = dalloc(&m.topo, m.n_eta) == cudaSuccess;
    if (!ok) { rc = set_err(ctx, PAVG_ERR_NOMEM, "device upload failed"); throw 0; }
    if (cudaMemset(m.topo, 0, sizeof(double) * m.n_eta) != cudaSuccess) {
      rc = set_err(ctx, PAVG_ERR_CUDA, "topography initialisation failed");
      throw 0;
    }
    // facet scratch of N: up to kFacetChunk states per launch, at most ~512 MB
    ctx->facet_chunk = (int)std::max<int64_t>(
        1, std::min<int64_t>(kFacetChunk, ((int64_t)512 << 20) / ((int64_t)45 * sizeof(double) * m.F)));
    CgWork& w = ctx->cg;
    if (cg_configure(m.F, &w) != cudaSuccess) { rc = set_err(ctx, PAVG_ERR_CUDA, "CG configuration failed"); throw 0; }
    ok = dalloc(&w.x, m.n_u) == cudaSuccess && dalloc(&w.r[0], m.n_u) == cudaSuccess &&
         dalloc(&w.r[1], m.n_u) == cudaSuccess && dalloc(&w.s[0], m.n_u) == cudaSuccess &&
         dalloc(&w.s[1], m.n_u) == cudaSuccess && dalloc(&w.w[0], m.n_u) == cudaSuccess &&
         dalloc(&w.w[1], m.n_u) == cudaSuccess && dalloc(&w.w[2], m.n_u) == cudaSuccess &&
         dalloc(&w.p, m.n_u) == cudaSuccess && dalloc(&w.partial, 6 * (size_t)w.nblocks) == cudaSuccess &&
         dalloc(&w.bar, 2) == cudaSuccess && dalloc(&w.flags, 1) == cudaSuccess && dalloc(&w.stats, 4) == cudaSuccess &&
         dalloc(&ctx->ru, m.n_u) == cudaSuccess && dalloc(&ctx->io_in, m.n) == cudaSuccess &&
         dalloc(&ctx->facets, (size_t)ctx->facet_chunk * 45 * m.F) == cudaSuccess &&
         dalloc(&ctx->io_out, m.n) == cudaSuccess && dalloc(&ctx->dpart, 4096) == cudaSuccess &&
         cudaMallocHost((void**)&ctx->host_part, sizeof(double) * 4096) == cudaSuccess;
    for (auto*& v : ctx->vec) ok = ok && dalloc(&v, m.n) == cudaSuccess;
    CgIrWork& wi = ctx->cgi;
    ok = ok && cg_ir_configure(m.F, &wi) == cudaSuccess;
    ok = ok && dalloc(&wi.x[0], m.n_u) == cudaSuccess && dalloc(&wi.x[1], m.n_u) == cudaSuccess &&
         dalloc(&wi.ax, m.n_u) == cudaSuccess && dalloc(&wi.r64, m.n_u) == cudaSuccess &&
         dalloc(&wi.fbuf, 9 * 4 * (size_t)(m.E + m.F)) == cudaSuccess &&
         dalloc(&wi.partial, 3 * (size_t)wi.nblocks) == cudaSuccess &&
         dalloc(&wi.partial_f, 3 * (size_t)wi.nblocks) == cudaSuccess &&
         dalloc(&wi.scal, 8) == cudaSuccess && dalloc(&wi.tag, 4) == cudaSuccess &&
         dalloc(&wi.bar, 2) == cudaSuccess;
    wi.flags = w.flags;
    wi.stats = w.stats;
    if (ok && p->solver == PAVG_SOLVER_SUBDOMAIN && ctx->sd.P > 0) {
      ok = sd_alloc_work(ctx->sd, m.F, &ctx->sdw) == cudaSuccess;
      ctx->sdw.flags = w.flags;
      ctx->sdw.stats = w.stats;
      const double a = 0.95 * ctx->sd.lmin, bnd = 1.05 * ctx->sd.lmax;  // Lanczos estimates lie inside
      SdParams& sp = ctx->sdp;
      sp.rtol = ctx->cgip.rtol;
      sp.max_sweeps = 8;
      // cg_maxit caps the inner iterations of one refinement sweep, as for the mixed solver
      sp.iters = std::min(std::min(sd_iterations(a, bnd, mixed ? 1e-6 : 1e-5), p->cg_maxit), 256);
      sp.theta = 0.5 * (bnd + a);
      sp.delta = 0.5 * (bnd - a);
      sp.wait_cycles = kSdWaitCycles;
      sp.stall_mode = 0;
      sp.stall_part = -1;
      ctx->use_sd = ok;
    }
    if (ok) {
      float* fb = wi.fbuf;
      const int64_t s4 = 4 * (m.E + m.F);
      wi.xf = fb;
      wi.rf[0] = fb + 1 * s4; wi.rf[1] = fb + 2 * s4;
      wi.sf[0] = fb + 3 * s4; wi.sf[1] = fb + 4 * s4;
      wi.wf[0] = fb + 5 * s4; wi.wf[1] = fb + 6 * s4; wi.wf[2] = fb + 7 * s4;
      wi.pf = fb + 8 * s4;
    }
    if (!ok) { rc = set_err(ctx, PAVG_ERR_NOMEM, "workspace allocation failed"); throw 0; }
    if (cudaMemset(w.bar, 0, 2 * sizeof(unsigned)) != cudaSuccess || cudaMemset(w.flags, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(w.stats, 0, 4 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(ctx->cgi.bar, 0, 2 * sizeof(unsigned)) != cudaSuccess) {
      rc = set_err(ctx, PAVG_ERR_CUDA, "solver state initialisation failed");
      throw 0;
    }
    if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      rc = set_err(ctx, PAVG_ERR_CUDA, "stream creation failed");
      throw 0;
    }
    if (p->lambda_max > 0) {
      ctx->lam = p->lambda_max;
    } else {
      rc = estimate_lambda(ctx);
      if (rc) throw 0;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) { rc = set_err(ctx, PAVG_ERR_CUDA, "setup failed"); throw 0; }
    rc = check_flags(ctx);
    if (rc) throw 0;
  } catch (const std::exception& e) {
    std::fprintf(stderr, "pavg_create: %s\n", e.what());
    free_ctx(ctx);
    return PAVG_ERR_INVAL;
  } catch (int) {
    std::fprintf(stderr, "pavg_create: %s\n", ctx->err.c_str());
    free_ctx(ctx);
    return rc ? rc : PAVG_ERR_CUDA;
  }
  *out = ctx;
  return PAVG_OK;
}

int pavg_destroy(pavg_ctx* ctx) {
  if (!ctx) return PAVG_ERR_INVAL;
  cudaDeviceSynchronize();
  free_ctx(ctx);
  return PAVG_OK;
}

int pavg_sizes(const pavg_ctx* ctx, int64_t* n_u, int64_t* n_eta, int64_t* n_cells, int64_t* n_edges,
               int64_t* n_verts) {
  if (!ctx) return PAVG_ERR_INVAL;
  if (n_u) *n_u = ctx->dm.n_u;
  if (n_eta) *n_eta = ctx->dm.n_eta;
  if (n_cells) *n_cells = ctx->dm.F;
  if (n_edges) *n_edges = ctx->dm.E;
  if (n_verts) *n_verts = ctx->mesh.V();
  return PAVG_OK;
}

int pavg_mesh_export(const pavg_ctx* ctx, double* vert_xyz, int32_t* cell_verts) {
  if (!ctx) return PAVG_ERR_INVAL;
  if (vert_xyz) std::memcpy(vert_xyz, ctx->mesh.verts.data(), sizeof(double) * ctx->mesh.verts.size());
  if (cell_verts) std::memcpy(cell_verts, ctx->mesh.cells.data(), sizeof(int32_t) * ctx->mesh.cells.size());
  return PAVG_OK;
}

int pavg_set_topography(pavg_ctx* ctx, const double* b) {
  if (!ctx || !b) return PAVG_ERR_INVAL;
  CK(cudaMemcpy(ctx->dm.topo, b, sizeof(double) * ctx->dm.n_eta, cudaMemcpyDeviceToDevice));
  return PAVG_OK;
}

int pavg_lambda_max(const pavg_ctx* ctx, double* out) {
  if (!ctx || !out) return PAVG_ERR_INVAL;
  *out = ctx->lam;
  return PAVG_OK;
}

int pavg_linear(pavg_ctx* ctx, const double* U, double* LU, int B, void* stream) {
  if (!ctx || B < 0 || (B > 0 && (!U || !LU))) return PAVG_ERR_INVAL;
  if (B > 0 && LU == U) return set_err(ctx, PAVG_ERR_INVAL, "pavg_linear: the output aliases the input");
  CallScope scope_(ctx);
  const int64_t n = ctx->dm.n;
  for (int b = 0; b < B; ++b) {
    int rc = enq_linear(ctx, U + b * n, LU + b * n, S(stream));
    if (rc) return rc;
  }
  return PAVG_OK;
}

int pavg_nonlinear(pavg_ctx* ctx, const double* U, double* NU, int B, void* stream) {
  if (!ctx || B < 0 || (B > 0 && (!U || !NU))) return PAVG_ERR_INVAL;
  if (B > 0 && NU == U) return set_err(ctx, PAVG_ERR_INVAL, "pavg_nonlinear: the output aliases the input");
  CallScope scope_(ctx);
  const int64_t n = ctx->dm.n;
  for (int b = 0; b < B; ++b) {
    int rc = enq_nonlinear(ctx, U + b * n, NU + b * n, ctx->vec[5], S(stream));
    if (rc) return rc;
  }
  return PAVG_OK;
}

int pavg_expL_apply(pavg_ctx* ctx, double t, const double* U, double* out, int B, void* stream) {
  if (!ctx || B < 0 || (B > 0 && (!U || !out)) || !std::isfinite(t)) return PAVG_ERR_INVAL;
  if (B > 0 && out == U) return set_err(ctx, PAVG_ERR_INVAL, "pavg_expL_apply: the output aliases the input");
  CallScope scope_(ctx);
  const int64_t n = ctx->dm.n;
  for (int b = 0; b < B; ++b) {
    int rc = enq_expL(ctx, t, U + b * n, out + b * n, S(stream));
    if (rc) return rc;
  }
  return PAVG_OK;
}

int pavg_averaged_rhs(pavg_ctx* ctx, double T, int M, const double* U, double* out, void* stream) {
  if (!ctx || !U || !out || M < 1 || !(T >= 0) || !std::isfinite(T)) return PAVG_ERR_INVAL;
  if (out == U) return set_err(ctx, PAVG_ERR_INVAL, "pavg_averaged_rhs: the output aliases the input");
  CallScope scope_(ctx);
  return run_avg(ctx, T, M, U, out, S(stream));
}

int pavg_averaged_rhs_group(pavg_ctx* ctx, double T, int M, int m0, int m1, const double* U, double* out,
                            void* stream) {
  if (!ctx || !U || !out || M < 1 || !(T >= 0) || !std::isfinite(T)) return PAVG_ERR_INVAL;
  if (m0 < 0 || m1 > M || m0 >= m1) return set_err(ctx, PAVG_ERR_INVAL, "pavg_averaged_rhs_group: need 0 <= m0 < m1 <= M");
  if (out == U) return set_err(ctx, PAVG_ERR_INVAL, "pavg_averaged_rhs_group: the output aliases the input");
  CallScope scope_(ctx);
  return run_avg(ctx, T, M, U, out, S(stream), m0, m1);
}

int pavg_averaged_rhs_literal(pavg_ctx* ctx, double T, int M, const double* U, double* out, void* stream) {
  if (!ctx || !U || !out || M < 1 || !(T >= 0) || !std::isfinite(T)) return PAVG_ERR_INVAL;
  if (out == U) return set_err(ctx, PAVG_ERR_INVAL, "pavg_averaged_rhs_literal: the output aliases the input");
  CallScope scope_(ctx);
  cudaStream_t st = S(stream);
  const int64_t n = ctx->dm.n;
  if (T == 0.0) return enq_nonlinear(ctx, U, out, ctx->vec[5], st);
  std::vector<double> s, w;
  int rc = shifts_weights(T, M, ctx->p.quad_rule, &s, &w);
  if (rc) return set_err(ctx, rc, "invalid T / M / quadrature rule");
  double* acc = ctx->io_out;
  double* V = ctx->io_in;
  double* term = ctx->vec[4];
  CK(cudaMemsetAsync(acc, 0, sizeof(double) * n, st));
  for (int m = 0; m < M; ++m) {
    if (w[m] == 0.0) continue;
    rc = enq_expL(ctx, s[m], U, V, st);
    if (rc) return rc;
    rc = enq_nonlinear(ctx, V, term, ctx->vec[5], st);
    if (rc) return rc;
    rc = enq_expL(ctx, -s[m], term, V, st);
    if (rc) return rc;
    KL(launch_lincomb(acc, 1.0, acc, w[m], V, 0.0, nullptr, n, st));
  }
  CK(cudaMemcpyAsync(out, acc, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  return PAVG_OK;
}

// Shift marching (an alternative to the shared basis): the shifts of both
// point rules are equally spaced, so V_0 = e^{s_0 L} U, V_{m+1} = e^{ds L} V_m,
// and the backward sum nests (Horner): H_{M-1} = M^{-1} w_{M-1} r_{M-1},
// H_m = M^{-1} w_m r_m + e^{-ds L} H_{m+1}, out = e^{-s_0 L} H_0, with r_m the
// weak form of N(V_m).  Every short exponential is truncated by the tail rule
// of Sec. 2.4, so the result differs from pavg_averaged_rhs by those extra
// truncations.
int pavg_averaged_rhs_marching(pavg_ctx* ctx, double T, int M, const double* U, double* out, void* stream) {
  if (!ctx || !U || !out || M < 1 || !(T >= 0) || !std::isfinite(T)) return PAVG_ERR_INVAL;
  if (out == U) return set_err(ctx, PAVG_ERR_INVAL, "pavg_averaged_rhs_marching: the output aliases the input");
  CallScope scope_(ctx);
  cudaStream_t st = S(stream);
  const DeviceMesh& m = ctx->dm;
  const int64_t n = m.n;
  if (T == 0.0) return enq_nonlinear(ctx, U, out, ctx->vec[5], st);
  std::vector<double> s, w;
  int rc = shifts_weights(T, M, ctx->p.quad_rule, &s, &w);
  if (rc) return set_err(ctx, rc, "invalid T / M / quadrature rule");
  for (int k = 0; k < M; ++k)
    if (cheb_coefficients(ctx->lam * std::fabs(s[k]), ctx->p.cheb_tol).empty())
      return set_err(ctx, PAVG_ERR_INVAL, cheb_limit_msg(ctx->lam * std::fabs(s[k])));
  rc = ensure_avg_workspace(ctx, std::max(ctx->Kcap, 0), M);
  if (rc) return rc;
  double* V = ctx->Um;  // [M][n] shifted states
  double* R = ctx->Rm;  // [M][n] weak forms of N
  if ((rc = enq_expL(ctx, s[0], U, V, st))) return rc;
  for (int k = 1; k < M; ++k)
    if ((rc = enq_expL(ctx, s[k] - s[k - 1], V + (int64_t)(k - 1) * n, V + (int64_t)k * n, st))) return rc;
  const bool fp32 = ctx->p.precision == PAVG_PRECISION_MIXED;
  CK(cudaMemset2DAsync(R, sizeof(double) * n, 0, sizeof(double) * 3 * m.E, M, st));
  KL(launch_nonlinear_rhs(m, V, R, M, ctx->p.upwind_convention, st, fp32, ctx->facets, ctx->facet_chunk));
  double* H = ctx->io_out;
  double* wr = ctx->io_in;
  double* tn = ctx->vec[4];
  double* te = ctx->vec[5];
  bool started = false;
  for (int k = M - 1; k >= 0; --k) {
    if (started) {
      if ((rc = enq_expL(ctx, -(s[k + 1] - s[k]), H, te, st))) return rc;
    }
    if (w[k] != 0.0) {
      KL(launch_lincomb(wr, w[k], R + (int64_t)k * n, 0.0, nullptr, 0.0, nullptr, n, st));
      if ((rc = enq_mass_solve(ctx, wr, tn, st))) return rc;
      if (started) KL(launch_lincomb(H, 1.0, tn, 1.0, te, 0.0, nullptr, n, st));
      else CK(cudaMemcpyAsync(H, tn, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    } else if (started) {
      CK(cudaMemcpyAsync(H, te, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    } else {
      CK(cudaMemsetAsync(H, 0, sizeof(double) * n, st));
    }
    started = true;
  }
  return enq_expL(ctx, -s[0], H, out, st);
}

// Sec. 2.3 (Eqs. stage1_c to stage4), with E(t) = e^{tL} and N-bar the average:
//   k1 = N-bar(U);  U1 = U + dt/2 k1;  k2 = N-bar(E(dt/2) U1);  U2 = E(dt/2) U + dt/2 k2
//   k3 = N-bar(U2); U3 = E(dt/2) U + dt k3;  k4 = N-bar(E(dt/2) U3)
//   U+ = E(dt) U + dt/6 [E(dt) k1 + 2 E(dt/2) k2 + 2 E(dt/2) k3 + k4]
// evaluated as E(dt)(U + dt/6 k1) + dt/6 [2 E(dt/2)(k2 + k3) + k4] (E is linear).
int pavg_timestep(pavg_ctx* ctx, double dt, double T, int M, double* U, int nsteps, void* stream) {
  if (!ctx || !U || M < 1 || nsteps < 0 || !(T >= 0) || !std::isfinite(T) || !std::isfinite(dt)) return PAVG_ERR_INVAL;
  CallScope scope_(ctx);
  cudaStream_t st = S(stream);
  const int64_t n = ctx->dm.n;
  AvgPlan* pl = nullptr;
  int rc = get_plan(ctx, T, M, &pl);
  if (rc) return rc;
  rc = ensure_avg_workspace(ctx, pl->K, M);
  if (rc) return rc;
  // stage vectors: context workspace, allocated once by the first call
  if (!ctx->ts && dalloc(&ctx->ts, (size_t)7 * n) != cudaSuccess) {
    ctx->ts = nullptr;
    return set_err(ctx, PAVG_ERR_NOMEM, "timestep workspace allocation failed");
  }
  double* k1 = ctx->ts;
  double *k2 = k1 + n, *k3 = k2 + n, *k4 = k3 + n, *EhU = k4 + n, *tmp = EhU + n, *tmp2 = tmp + n;
  for (int step = 0; step < nsteps; ++step) {
    if ((rc = run_avg(ctx, T, M, U, k1, st))) return rc;
    if ((rc = enq_expL(ctx, 0.5 * dt, U, EhU, st))) return rc;
    if (launch_lincomb(tmp, 1.0, U, 0.5 * dt, k1, 0, nullptr, n, st) != cudaSuccess) return PAVG_ERR_CUDA;
    if ((rc = enq_expL(ctx, 0.5 * dt, tmp, tmp2, st))) return rc;
    if ((rc = run_avg(ctx, T, M, tmp2, k2, st))) return rc;
    if (launch_lincomb(tmp, 1.0, EhU, 0.5 * dt, k2, 0, nullptr, n, st) != cudaSuccess) return PAVG_ERR_CUDA;
    if ((rc = run_avg(ctx, T, M, tmp, k3, st))) return rc;
    if (launch_lincomb(tmp, 1.0, EhU, dt, k3, 0, nullptr, n, st) != cudaSuccess) return PAVG_ERR_CUDA;
    if ((rc = enq_expL(ctx, 0.5 * dt, tmp, tmp2, st))) return rc;
    if ((rc = run_avg(ctx, T, M, tmp2, k4, st))) return rc;
    // U+ = E(dt)(U + dt/6 k1) + dt/6 [2 E(dt/2)(k2 + k3) + k4]
    if (launch_lincomb(tmp, 1.0, k2, 1.0, k3, 0, nullptr, n, st) != cudaSuccess) return PAVG_ERR_CUDA;
    if ((rc = enq_expL(ctx, 0.5 * dt, tmp, tmp2, st))) return rc;
    if (launch_lincomb(tmp, 1.0, U, dt / 6.0, k1, 0, nullptr, n, st) != cudaSuccess) return PAVG_ERR_CUDA;
    if ((rc = enq_expL(ctx, dt, tmp, EhU, st))) return rc;
    if (launch_lincomb(U, 1.0, EhU, dt / 3.0, tmp2, dt / 6.0, k4, n, st) != cudaSuccess) return PAVG_ERR_CUDA;
  }
  return PAVG_OK;
}

int pavg_norms(pavg_ctx* ctx, const double* U, double* out, void* stream) {
  if (!ctx || !U || !out) return PAVG_ERR_INVAL;
  int nb = 0;
  cudaStream_t st = S(stream);
  KL(launch_norms(ctx->dm, U, ctx->dpart, &nb, st));
  CK(cudaMemcpyAsync(ctx->host_part, ctx->dpart, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  double a = 0.0, d = 0.0, e = 0.0;
  for (int i = 0; i < nb; ++i) {
    a += ctx->host_part[3 * i];
    d += ctx->host_part[3 * i + 1];
    e += ctx->host_part[3 * i + 2];
  }
  out[0] = std::sqrt(a);
  out[1] = std::sqrt(a + d);
  out[2] = std::sqrt(e);
  return PAVG_OK;
}

int pavg_sync(pavg_ctx* ctx, void* stream) {
  if (!ctx) return PAVG_ERR_INVAL;
  CK(cudaStreamSynchronize(S(stream)));
  return check_flags(ctx);
}

int pavg_get_stats(pavg_ctx* ctx, pavg_stats* out) {
  if (!ctx || !out) return PAVG_ERR_INVAL;
  CK(cudaDeviceSynchronize());
  unsigned long long st[4];
  int f = 0;
  CK(cudaMemcpy(st, ctx->cg.stats, sizeof(st), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&f, ctx->cg.flags, sizeof(int), cudaMemcpyDeviceToHost));
  out->lambda_max = ctx->lam;
  out->last_degree = ctx->last_degree;
  out->cg_solves = (int)st[0];
  out->cg_iters_max = (int)st[2];
  out->cg_iters_mean = st[0] ? (double)st[1] / (double)st[0] : 0.0;
  out->cg_sweeps_mean = st[0] ? (double)st[3] / (double)st[0] : 0.0;
  out->error_flags = f;
  out->kernel_launches = ctx->last_launches;
  out->solver_in_use = ctx->use_sd ? PAVG_SOLVER_SUBDOMAIN
                                   : (ctx->p.solver == PAVG_SOLVER_FP64 ? PAVG_SOLVER_FP64 : PAVG_SOLVER_MIXED);
  return PAVG_OK;
}

int pavg_kernel_timing(pavg_ctx* ctx, int enable) {
  if (!ctx) return PAVG_ERR_INVAL;
  ctx->timing = enable != 0;
  return PAVG_OK;
}

int pavg_kernel_time(pavg_ctx* ctx, double* total_ms, int* launches) {
  if (!ctx || !total_ms || !launches) return PAVG_ERR_INVAL;
  double tot = 0.0;
  for (auto& pr : ctx->last_pairs) {
    CK(cudaEventSynchronize(pr.second));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, pr.first, pr.second));
    tot += ms;
  }
  *total_ms = tot;
  *launches = (int)ctx->last_pairs.size();
  return PAVG_OK;
}

int pavg_reset_stats(pavg_ctx* ctx) {
  if (!ctx) return PAVG_ERR_INVAL;
  CK(cudaDeviceSynchronize());
  CK(cudaMemset(ctx->cg.stats, 0, 4 * sizeof(unsigned long long)));
  CK(cudaMemset(ctx->cg.flags, 0, sizeof(int)));
  if (ctx->use_sd) CK(sd_reset_work(ctx->sd, ctx->dm.F, &ctx->sdw));
  return PAVG_OK;
}

int pavg_test_stall(pavg_ctx* ctx, int mode, int part, double wait_us) {
  if (!ctx || mode < 0 || mode > 2 || !(wait_us >= 0) || !std::isfinite(wait_us)) return PAVG_ERR_INVAL;
  if (!ctx->use_sd) return set_err(ctx, PAVG_ERR_INVAL, "pavg_test_stall: the context does not use the subdomain solver");
  if (mode != 0 && (part < 0 || part >= ctx->sd.P)) return set_err(ctx, PAVG_ERR_INVAL, "pavg_test_stall: no such block");
  CK(cudaDeviceSynchronize());
  for (auto& kv : ctx->plans) drop_graph(&kv.second);  // graphs hold the old kernel parameters
  ctx->sdp.stall_mode = mode;
  ctx->sdp.stall_part = mode ? part : -1;
  ctx->sdp.wait_cycles = wait_us > 0 ? (long long)(wait_us * 2070.0) : kSdWaitCycles;
  return PAVG_OK;
}

const char* pavg_last_error(const pavg_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

}  // extern "C"
