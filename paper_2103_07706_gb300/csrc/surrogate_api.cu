// C-ABI of the learned surrogate (declared in include/pavg.h): parameters,
// training store, training loop, inference and the Riemann-sum fallback.
// The host sequences the kernels of surrogate.cu; every arithmetic step runs
// on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <random>
#include <string>
#include <vector>

#include "api_internal.h"

using namespace pavg_api;

namespace {

constexpr int kIn = kSurInputs, kOut = kSurOutputs;
constexpr int kMseBlocks = 64;

#define SCK(call)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return sset_err(s, PAVG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Device scratch for one context the surrogate runs on.
struct CtxData {
  uint64_t uid = 0;        // the context these buffers were made for
  float* geo = nullptr;    // [F][4]
  float* X = nullptr;      // [F][124]
  float* H1 = nullptr;     // [F][hidden]
  float* H2 = nullptr;
  float* Y = nullptr;      // [F][15]
  double* corr = nullptr;  // [n]
  double* vc = nullptr;    // [n] cheap average
  double* vf = nullptr;    // [n] large-M average
  double* diff = nullptr;  // [n]
};

}  // namespace

struct pavg_surrogate {
  int hidden = 128;
  int64_t nparams = 0;
  int64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  int64_t t = 0;  // Adam steps taken
  float *mu_x = nullptr, *sd_x = nullptr, *mu_y = nullptr, *sd_y = nullptr;
  bool scaled = false;
  // training store
  float *Xtr = nullptr, *Ztr = nullptr;
  int64_t rows = 0, cap = 0;
  // minibatch workspace
  int bcap = 0;
  float *Xb = nullptr, *Zb = nullptr, *H1 = nullptr, *H2 = nullptr, *Y = nullptr, *dY = nullptr, *dA2 = nullptr,
        *dA1 = nullptr, *split = nullptr;
  int* perm = nullptr;
  int64_t perm_cap = 0;
  double *part = nullptr, *loss = nullptr;
  std::map<pavg_ctx*, CtxData> ctx;
  std::string err;
};

namespace {

int sset_err(pavg_surrogate* s, int code, const std::string& msg) {
  if (s) s->err = msg;
  return code;
}

constexpr int kSplits = 16;  // K splits of the weight-gradient products

void free_ctxdata(CtxData& d) {
  cudaFree(d.geo); cudaFree(d.X); cudaFree(d.H1); cudaFree(d.H2); cudaFree(d.Y);
  cudaFree(d.corr); cudaFree(d.vc); cudaFree(d.vf); cudaFree(d.diff);
  d = CtxData();
}

void free_sur(pavg_surrogate* s) {
  if (!s) return;
  cudaFree(s->p); cudaFree(s->g); cudaFree(s->m); cudaFree(s->v);
  cudaFree(s->mu_x); cudaFree(s->sd_x); cudaFree(s->mu_y); cudaFree(s->sd_y);
  cudaFree(s->Xtr); cudaFree(s->Ztr);
  cudaFree(s->Xb); cudaFree(s->Zb); cudaFree(s->H1); cudaFree(s->H2); cudaFree(s->Y); cudaFree(s->dY);
  cudaFree(s->dA2); cudaFree(s->dA1); cudaFree(s->split); cudaFree(s->perm); cudaFree(s->part); cudaFree(s->loss);
  for (auto& kv : s->ctx) free_ctxdata(kv.second);
  delete s;
}

// z_c / R, G00 / det, G01 / det, G11 / det of every cell of the context's mesh (setup data).
std::vector<float> cell_geometry(const pavg_ctx* ctx) {
  const Mesh& ms = ctx->mesh;
  const int64_t F = ms.F();
  std::vector<float> g(4 * F);
  for (int64_t c = 0; c < F; ++c) {
    const double* a = &ms.verts[3 * (size_t)ms.cells[3 * c]];
    const double* b = &ms.verts[3 * (size_t)ms.cells[3 * c + 1]];
    const double* d = &ms.verts[3 * (size_t)ms.cells[3 * c + 2]];
    double j0[3], j1[3];
    for (int k = 0; k < 3; ++k) { j0[k] = b[k] - a[k]; j1[k] = d[k] - a[k]; }
    const double cx = j0[1] * j1[2] - j0[2] * j1[1], cy = j0[2] * j1[0] - j0[0] * j1[2],
                 cz = j0[0] * j1[1] - j0[1] * j1[0];
    const double det = std::sqrt(cx * cx + cy * cy + cz * cz);
    const double g00 = j0[0] * j0[0] + j0[1] * j0[1] + j0[2] * j0[2];
    const double g01 = j0[0] * j1[0] + j0[1] * j1[1] + j0[2] * j1[2];
    const double g11 = j1[0] * j1[0] + j1[1] * j1[1] + j1[2] * j1[2];
    const double zc = a[2] + (j0[2] + j1[2]) / 3.0;
    g[4 * c] = (float)(zc / ms.radius);
    g[4 * c + 1] = (float)(g00 / det);
    g[4 * c + 2] = (float)(g01 / det);
    g[4 * c + 3] = (float)(g11 / det);
  }
  return g;
}

int ctx_data(pavg_surrogate* s, pavg_ctx* ctx, CtxData** out) {
  auto it = s->ctx.find(ctx);
  if (it != s->ctx.end()) {
    if (it->second.uid == ctx->uid) { *out = &it->second; return PAVG_OK; }
    free_ctxdata(it->second);  // a new context at a destroyed one's address
    s->ctx.erase(it);
  }
  CtxData d;
  d.uid = ctx->uid;
  const int64_t F = ctx->dm.F, n = ctx->dm.n;
  bool ok = upload(&d.geo, cell_geometry(ctx)) == cudaSuccess && dalloc(&d.X, (size_t)F * kIn) == cudaSuccess &&
            dalloc(&d.H1, (size_t)F * s->hidden) == cudaSuccess && dalloc(&d.H2, (size_t)F * s->hidden) == cudaSuccess &&
            dalloc(&d.Y, (size_t)F * kOut) == cudaSuccess && dalloc(&d.corr, n) == cudaSuccess &&
            dalloc(&d.vc, n) == cudaSuccess && dalloc(&d.vf, n) == cudaSuccess && dalloc(&d.diff, n) == cudaSuccess;
  if (!ok) {
    free_ctxdata(d);
    return sset_err(s, PAVG_ERR_NOMEM, "surrogate: context scratch allocation failed");
  }
  auto res = s->ctx.emplace(ctx, d);
  *out = &res.first->second;
  return PAVG_OK;
}

int ensure_batch(pavg_surrogate* s, int B) {
  if (B <= s->bcap) return PAVG_OK;
  cudaFree(s->Xb); cudaFree(s->Zb); cudaFree(s->H1); cudaFree(s->H2); cudaFree(s->Y); cudaFree(s->dY);
  cudaFree(s->dA2); cudaFree(s->dA1);
  s->bcap = 0;
  const size_t H = (size_t)s->hidden;
  bool ok = dalloc(&s->Xb, (size_t)B * kIn) == cudaSuccess && dalloc(&s->Zb, (size_t)B * kOut) == cudaSuccess &&
            dalloc(&s->H1, (size_t)B * H) == cudaSuccess && dalloc(&s->H2, (size_t)B * H) == cudaSuccess &&
            dalloc(&s->Y, (size_t)B * kOut) == cudaSuccess && dalloc(&s->dY, (size_t)B * kOut) == cudaSuccess &&
            dalloc(&s->dA2, (size_t)B * H) == cudaSuccess && dalloc(&s->dA1, (size_t)B * H) == cudaSuccess;
  if (!ok) return sset_err(s, PAVG_ERR_NOMEM, "surrogate: minibatch allocation failed");
  s->bcap = B;
  return PAVG_OK;
}

// Forward pass of rows X [B][124] into H1, H2, Y (bf16: operands rounded).
int forward(pavg_surrogate* s, const float* X, int B, float* H1, float* H2, float* Y, bool bf16, cudaStream_t st) {
  const int H = s->hidden;
  SCK(sur_gemm(SurGemm::kForwardTanh, B, H, kIn, X, kIn, s->p + s->oW1, kIn, H1, H, s->p + s->ob1, nullptr, 0, 1,
               bf16, st));
  SCK(sur_gemm(SurGemm::kForwardTanh, B, H, H, H1, H, s->p + s->oW2, H, H2, H, s->p + s->ob2, nullptr, 0, 1, bf16,
               st));
  SCK(sur_gemm(SurGemm::kForwardLinear, B, kOut, H, H2, H, s->p + s->oW3, H, Y, kOut, s->p + s->ob3, nullptr, 0, 1,
               bf16, st));
  return PAVG_OK;
}

// Loss (added to s->loss) and gradient (into s->g) of rows Xb/Zb [B].
int backward(pavg_surrogate* s, const float* X, const float* Z, int B, cudaStream_t st) {
  const int H = s->hidden;
  int rc = forward(s, X, B, s->H1, s->H2, s->Y, false, st);
  if (rc) return rc;
  const int64_t cnt = (int64_t)B * kOut;
  SCK(sur_mse(s->Y, Z, cnt, (float)(2.0 / (double)cnt), s->dY, s->part, kMseBlocks, (double)cnt, s->loss, st));
  // dW3 [15][H] = dY^T H2, db3 = column sums of dY
  SCK(sur_gemm(SurGemm::kWeightGrad, kOut, H, B, s->dY, kOut, s->H2, H, s->split, H, nullptr, nullptr, 0, kSplits,
               false, st));
  SCK(sur_reduce_splits(s->split, kSplits, (int64_t)kOut * H, s->g + s->oW3, st));
  SCK(sur_colsum(s->dY, B, kOut, kOut, s->g + s->ob3, st));
  // dA2 = (dY W3) (1 - H2^2)
  SCK(sur_gemm(SurGemm::kBackwardData, B, H, kOut, s->dY, kOut, s->p + s->oW3, H, s->dA2, H, nullptr, s->H2, H, 1,
               false, st));
  SCK(sur_gemm(SurGemm::kWeightGrad, H, H, B, s->dA2, H, s->H1, H, s->split, H, nullptr, nullptr, 0, kSplits, false,
               st));
  SCK(sur_reduce_splits(s->split, kSplits, (int64_t)H * H, s->g + s->oW2, st));
  SCK(sur_colsum(s->dA2, B, H, H, s->g + s->ob2, st));
  // dA1 = (dA2 W2) (1 - H1^2)
  SCK(sur_gemm(SurGemm::kBackwardData, B, H, H, s->dA2, H, s->p + s->oW2, H, s->dA1, H, nullptr, s->H1, H, 1, false,
               st));
  SCK(sur_gemm(SurGemm::kWeightGrad, H, kIn, B, s->dA1, H, X, kIn, s->split, kIn, nullptr, nullptr, 0, kSplits, false,
               st));
  SCK(sur_reduce_splits(s->split, kSplits, (int64_t)H * kIn, s->g + s->oW1, st));
  SCK(sur_colsum(s->dA1, B, H, H, s->g + s->ob1, st));
  return PAVG_OK;
}

int adam(pavg_surrogate* s, const float* g, double lr, cudaStream_t st) {
  const double b1 = 0.9, b2 = 0.999;
  ++s->t;
  const double c1 = 1.0 / (1.0 - std::pow(b1, (double)s->t)), c2 = 1.0 / (1.0 - std::pow(b2, (double)s->t));
  SCK(sur_adam(s->p, g, s->m, s->v, s->nparams, (float)lr, (float)b1, (float)b2, 1e-8f, (float)c1, (float)c2, st));
  return PAVG_OK;
}

}  // namespace

extern "C" {

int pavg_surrogate_create(int hidden, uint64_t seed, pavg_surrogate** out) {
  if (!out) return PAVG_ERR_INVAL;
  *out = nullptr;
  if (hidden < 1 || hidden > 4096) return PAVG_ERR_INVAL;
  pavg_surrogate* s = new pavg_surrogate();
  const int64_t H = hidden;
  s->hidden = hidden;
  s->oW1 = 0;
  s->ob1 = s->oW1 + H * kIn;
  s->oW2 = s->ob1 + H;
  s->ob2 = s->oW2 + H * H;
  s->oW3 = s->ob2 + H;
  s->ob3 = s->oW3 + (int64_t)kOut * H;
  s->nparams = s->ob3 + kOut;
  // Glorot-uniform weights, zero biases
  std::vector<float> p(s->nparams, 0.f);
  std::mt19937_64 rng(seed);
  auto glorot = [&](int64_t off, int64_t rows, int64_t cols) {
    const double lim = std::sqrt(6.0 / (double)(rows + cols));
    std::uniform_real_distribution<double> u(-lim, lim);
    for (int64_t i = 0; i < rows * cols; ++i) p[off + i] = (float)u(rng);
  };
  glorot(s->oW1, H, kIn);
  glorot(s->oW2, H, H);
  glorot(s->oW3, kOut, H);
  std::vector<float> zero(kIn, 0.f), one(kIn, 1.f);
  bool ok = upload(&s->p, p) == cudaSuccess && dalloc(&s->g, s->nparams) == cudaSuccess &&
            dalloc(&s->m, s->nparams) == cudaSuccess && dalloc(&s->v, s->nparams) == cudaSuccess &&
            upload(&s->mu_x, zero) == cudaSuccess && upload(&s->sd_x, one) == cudaSuccess &&
            dalloc(&s->mu_y, kOut) == cudaSuccess && dalloc(&s->sd_y, kOut) == cudaSuccess &&
            dalloc(&s->split, (size_t)kSplits * H * std::max<int64_t>(H, kIn)) == cudaSuccess &&
            dalloc(&s->part, kMseBlocks) == cudaSuccess && dalloc(&s->loss, 1) == cudaSuccess;
  ok = ok && cudaMemset(s->m, 0, sizeof(float) * s->nparams) == cudaSuccess &&
       cudaMemset(s->v, 0, sizeof(float) * s->nparams) == cudaSuccess &&
       cudaMemcpy(s->mu_y, zero.data(), sizeof(float) * kOut, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(s->sd_y, one.data(), sizeof(float) * kOut, cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    free_sur(s);
    return PAVG_ERR_NOMEM;
  }
  *out = s;
  return PAVG_OK;
}

int pavg_surrogate_destroy(pavg_surrogate* s) {
  if (!s) return PAVG_ERR_INVAL;
  cudaDeviceSynchronize();
  free_sur(s);
  return PAVG_OK;
}

int pavg_surrogate_nparams(const pavg_surrogate* s, int64_t* n) {
  if (!s || !n) return PAVG_ERR_INVAL;
  *n = s->nparams;
  return PAVG_OK;
}

int pavg_surrogate_get_params(const pavg_surrogate* s, float* host) {
  if (!s || !host) return PAVG_ERR_INVAL;
  if (cudaMemcpy(host, s->p, sizeof(float) * s->nparams, cudaMemcpyDeviceToHost) != cudaSuccess) return PAVG_ERR_CUDA;
  return PAVG_OK;
}

int pavg_surrogate_set_params(pavg_surrogate* s, const float* host) {
  if (!s || !host) return PAVG_ERR_INVAL;
  SCK(cudaMemcpy(s->p, host, sizeof(float) * s->nparams, cudaMemcpyHostToDevice));
  return PAVG_OK;
}

int pavg_surrogate_get_scaling(const pavg_surrogate* s, float* mu_x, float* sd_x, float* mu_y, float* sd_y) {
  if (!s || !mu_x || !sd_x || !mu_y || !sd_y) return PAVG_ERR_INVAL;
  bool ok = cudaMemcpy(mu_x, s->mu_x, sizeof(float) * kIn, cudaMemcpyDeviceToHost) == cudaSuccess &&
            cudaMemcpy(sd_x, s->sd_x, sizeof(float) * kIn, cudaMemcpyDeviceToHost) == cudaSuccess &&
            cudaMemcpy(mu_y, s->mu_y, sizeof(float) * kOut, cudaMemcpyDeviceToHost) == cudaSuccess &&
            cudaMemcpy(sd_y, s->sd_y, sizeof(float) * kOut, cudaMemcpyDeviceToHost) == cudaSuccess;
  return ok ? PAVG_OK : PAVG_ERR_CUDA;
}

int pavg_surrogate_set_scaling(pavg_surrogate* s, const float* mu_x, const float* sd_x, const float* mu_y,
                               const float* sd_y) {
  if (!s || !mu_x || !sd_x || !mu_y || !sd_y) return PAVG_ERR_INVAL;
  for (int j = 0; j < kIn; ++j)
    if (!(sd_x[j] > 0.f)) return sset_err(s, PAVG_ERR_INVAL, "non-positive scale");
  for (int j = 0; j < kOut; ++j)
    if (!(sd_y[j] > 0.f)) return sset_err(s, PAVG_ERR_INVAL, "non-positive scale");
  SCK(cudaMemcpy(s->mu_x, mu_x, sizeof(float) * kIn, cudaMemcpyHostToDevice));
  SCK(cudaMemcpy(s->sd_x, sd_x, sizeof(float) * kIn, cudaMemcpyHostToDevice));
  SCK(cudaMemcpy(s->mu_y, mu_y, sizeof(float) * kOut, cudaMemcpyHostToDevice));
  SCK(cudaMemcpy(s->sd_y, sd_y, sizeof(float) * kOut, cudaMemcpyHostToDevice));
  s->scaled = true;
  return PAVG_OK;
}

int pavg_surrogate_add_pairs(pavg_surrogate* s, pavg_ctx* ctx, int n, const double* const* U,
                             const double* const* Vc, const double* const* Vf, void* stream) {
  if (!s || !ctx || n < 0 || (n > 0 && (!U || !Vc || !Vf))) return PAVG_ERR_INVAL;
  if (s->scaled) return sset_err(s, PAVG_ERR_INVAL, "pairs must be added before the scaling is fitted");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  CtxData* d = nullptr;
  int rc = ctx_data(s, ctx, &d);
  if (rc) return rc;
  const int64_t F = ctx->dm.F;
  const int64_t need = s->rows + (int64_t)n * F;
  if (need > s->cap) {  // grow the store (keeps the rows so far)
    const int64_t cap = std::max(need, 2 * s->cap);
    float *X = nullptr, *Z = nullptr;
    if (dalloc(&X, (size_t)cap * kIn) != cudaSuccess || dalloc(&Z, (size_t)cap * kOut) != cudaSuccess) {
      cudaFree(X);
      return sset_err(s, PAVG_ERR_NOMEM, "surrogate: training store allocation failed");
    }
    SCK(cudaStreamSynchronize(st));
    if (s->rows) {
      SCK(cudaMemcpy(X, s->Xtr, sizeof(float) * s->rows * kIn, cudaMemcpyDeviceToDevice));
      SCK(cudaMemcpy(Z, s->Ztr, sizeof(float) * s->rows * kOut, cudaMemcpyDeviceToDevice));
    }
    cudaFree(s->Xtr);
    cudaFree(s->Ztr);
    s->Xtr = X;
    s->Ztr = Z;
    s->cap = cap;
  }
  for (int i = 0; i < n; ++i) {
    if (!U[i] || !Vc[i] || !Vf[i]) return sset_err(s, PAVG_ERR_INVAL, "null pair pointer");
    SCK(sur_features(ctx->dm, U[i], Vc[i], d->geo, nullptr, nullptr, s->Xtr + (size_t)s->rows * kIn, st));
    SCK(sur_targets(ctx->dm, Vf[i], Vc[i], nullptr, nullptr, s->Ztr + (size_t)s->rows * kOut, st));
    s->rows += F;
  }
  return PAVG_OK;
}

int pavg_surrogate_rows(const pavg_surrogate* s, int64_t* rows) {
  if (!s || !rows) return PAVG_ERR_INVAL;
  *rows = s->rows;
  return PAVG_OK;
}

int pavg_surrogate_fit_scaling(pavg_surrogate* s, void* stream) {
  if (!s) return PAVG_ERR_INVAL;
  if (s->scaled) return sset_err(s, PAVG_ERR_INVAL, "scaling already fitted");
  if (s->rows < 2) return sset_err(s, PAVG_ERR_INVAL, "no training rows");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  SCK(sur_colstats(s->Xtr, s->rows, kIn, s->mu_x, s->sd_x, st));
  SCK(sur_colstats(s->Ztr, s->rows, kOut, s->mu_y, s->sd_y, st));
  SCK(sur_standardize(s->Xtr, s->rows, kIn, s->mu_x, s->sd_x, st));
  SCK(sur_standardize(s->Ztr, s->rows, kOut, s->mu_y, s->sd_y, st));
  s->scaled = true;
  return PAVG_OK;
}

int pavg_surrogate_train(pavg_surrogate* s, int epochs, int batch, double lr, uint64_t seed,
                         double* loss_per_epoch, void* stream) {
  if (!s || epochs < 0 || batch < 1 || !(lr > 0)) return PAVG_ERR_INVAL;
  if (!s->scaled) return sset_err(s, PAVG_ERR_INVAL, "fit the scaling before training");
  if (s->rows < 1) return sset_err(s, PAVG_ERR_INVAL, "no training rows");
  if (s->rows > 0x7fffffff) return sset_err(s, PAVG_ERR_INVAL, "too many training rows");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int B = (int)std::min<int64_t>(batch, s->rows);
  int rc = ensure_batch(s, B);
  if (rc) return rc;
  if (s->perm_cap < s->rows) {
    cudaFree(s->perm);
    s->perm = nullptr;
    s->perm_cap = 0;
    if (dalloc(&s->perm, (size_t)s->rows) != cudaSuccess) return sset_err(s, PAVG_ERR_NOMEM, "permutation");
    s->perm_cap = s->rows;
  }
  std::vector<int> perm(s->rows);
  std::mt19937_64 rng(seed);
  const int64_t nb = s->rows / B;  // whole minibatches per epoch
  for (int ep = 0; ep < epochs; ++ep) {
    std::iota(perm.begin(), perm.end(), 0);
    std::shuffle(perm.begin(), perm.end(), rng);
    SCK(cudaStreamSynchronize(st));
    SCK(cudaMemcpy(s->perm, perm.data(), sizeof(int) * s->rows, cudaMemcpyHostToDevice));
    SCK(cudaMemsetAsync(s->loss, 0, sizeof(double), st));
    for (int64_t k = 0; k < nb; ++k) {
      SCK(sur_gather_rows(s->Xtr, s->perm + k * B, B, kIn, s->Xb, st));
      SCK(sur_gather_rows(s->Ztr, s->perm + k * B, B, kOut, s->Zb, st));
      if ((rc = backward(s, s->Xb, s->Zb, B, st))) return rc;
      if ((rc = adam(s, s->g, lr, st))) return rc;
    }
    double l = 0.0;
    SCK(cudaMemcpyAsync(&l, s->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    if (loss_per_epoch) loss_per_epoch[ep] = l / (double)nb;
    if (!std::isfinite(l)) return sset_err(s, PAVG_ERR_NONFINITE, "training loss is not finite");
  }
  return PAVG_OK;
}

int pavg_surrogate_gradient(pavg_surrogate* s, const float* X, const float* Z, int B, float* grad, double* loss,
                            void* stream) {
  if (!s || !X || !Z || B < 1 || !grad || !loss) return PAVG_ERR_INVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int rc = ensure_batch(s, B);
  if (rc) return rc;
  SCK(cudaMemsetAsync(s->loss, 0, sizeof(double), st));
  if ((rc = backward(s, X, Z, B, st))) return rc;
  SCK(cudaMemcpyAsync(grad, s->g, sizeof(float) * s->nparams, cudaMemcpyDeviceToDevice, st));
  SCK(cudaMemcpyAsync(loss, s->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
  SCK(cudaStreamSynchronize(st));
  return PAVG_OK;
}

int pavg_surrogate_adam_step(pavg_surrogate* s, const float* grad, double lr, void* stream) {
  if (!s || !grad || !(lr > 0)) return PAVG_ERR_INVAL;
  return adam(s, grad, lr, reinterpret_cast<cudaStream_t>(stream));
}

int pavg_surrogate_features(pavg_surrogate* s, pavg_ctx* ctx, const double* U, const double* V, float* X,
                            int standardised, void* stream) {
  if (!s || !ctx || !U || !V || !X) return PAVG_ERR_INVAL;
  CtxData* d = nullptr;
  int rc = ctx_data(s, ctx, &d);
  if (rc) return rc;
  SCK(sur_features(ctx->dm, U, V, d->geo, standardised ? s->mu_x : nullptr, standardised ? s->sd_x : nullptr, X,
                   reinterpret_cast<cudaStream_t>(stream)));
  return PAVG_OK;
}

int pavg_surrogate_apply(pavg_surrogate* s, pavg_ctx* ctx, const double* U, const double* V, double* out, int bf16,
                         void* stream) {
  if (!s || !ctx || !U || !V || !out || out == U || out == V) return PAVG_ERR_INVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  CtxData* d = nullptr;
  int rc = ctx_data(s, ctx, &d);
  if (rc) return rc;
  const DeviceMesh& m = ctx->dm;
  const int F = (int)m.F;
  SCK(sur_features(m, U, V, d->geo, s->mu_x, s->sd_x, d->X, st));
  if ((rc = forward(s, d->X, F, d->H1, d->H2, d->Y, bf16 != 0, st))) return rc;
  SCK(sur_scatter(m, d->Y, s->mu_y, s->sd_y, d->corr, st));
  SCK(launch_lincomb(out, 1.0, V, 1.0, d->corr, 0.0, nullptr, m.n, st));
  return PAVG_OK;
}

int pavg_surrogate_averaged_rhs(pavg_surrogate* s, pavg_ctx* ctx, double T, int Mc, int Mf, double threshold,
                                int check, int bf16, const double* U, double* out, int* used_fallback,
                                double* rel_err, void* stream) {
  if (!s || !ctx || !U || !out || out == U || Mc < 1 || Mf < 1 || !(T >= 0) || !std::isfinite(T))
    return PAVG_ERR_INVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  CtxData* d = nullptr;
  int rc = ctx_data(s, ctx, &d);
  if (rc) return rc;
  if (used_fallback) *used_fallback = 0;
  if (rel_err) *rel_err = -1.0;
  if ((rc = run_avg(ctx, T, Mc, U, d->vc, st))) return sset_err(s, rc, "cheap average: " + ctx->err);
  if ((rc = pavg_surrogate_apply(s, ctx, U, d->vc, out, bf16, stream))) return rc;
  if (!check) return PAVG_OK;
  if ((rc = run_avg(ctx, T, Mf, U, d->vf, st))) return sset_err(s, rc, "full average: " + ctx->err);
  SCK(launch_lincomb(d->diff, 1.0, out, -1.0, d->vf, 0.0, nullptr, ctx->dm.n, st));
  SCK(cudaStreamSynchronize(st));
  const double num = host_winner(ctx, d->diff, d->diff), den = host_winner(ctx, d->vf, d->vf);
  if (!std::isfinite(num) || !std::isfinite(den)) return sset_err(s, PAVG_ERR_NONFINITE, "error estimate");
  const double err = den > 0 ? std::sqrt(num / den) : (num > 0 ? INFINITY : 0.0);
  if (rel_err) *rel_err = err;
  if (!(err <= threshold)) {
    SCK(cudaMemcpyAsync(out, d->vf, sizeof(double) * ctx->dm.n, cudaMemcpyDeviceToDevice, st));
    if (used_fallback) *used_fallback = 1;
  }
  return PAVG_OK;
}

const char* pavg_surrogate_last_error(const pavg_surrogate* s) {
  if (!s) return "null surrogate";
  return s->err.c_str();
}

}  // extern "C"
