// Kernels of the learned mesh-local surrogate: cell features, the MLP's
// forward and backward passes as tiled GEMMs with fused epilogues, the loss,
// bias gradients, Adam, and the scatter of per-cell outputs to DOFs.
//
// The MLP (124 inputs, two hidden tanh layers, 15 outputs per cell) is small:
// a training step over 8192 cells is about 1.6 GFLOP, an inference over the
// 327680 cells of refinement 7 about 22 GFLOP.  Both are far from any
// roofline of their own next to the averages they replace, so the GEMMs are
// plain shared-memory tiled FP32 kernels (64 x 64 output tile, 16-deep k
// slices, 4 x 4 outputs per thread).  BF16 inference runs on the tensor
// cores (mma.sync, BF16 operands, FP32 accumulation).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "device.h"
#include "device_common.cuh"

namespace pavg {
namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16, kGemmThreads = 256;

__device__ __forceinline__ float round_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// C = op(A) op(B) (+ epilogue), op(A) is M x K, op(B) is K x N.
// TA: A stored K x M (element (m, k) at A[k lda + m]); else M x K (A[m lda + k]).
// TB: B stored N x K (element (k, n) at B[n ldb + k]); else K x N (B[k ldb + n]).
// EPI 0: store; 1: tanh(v + bias[n]); 2: v + bias[n]; 3: v (1 - aux[m][n]^2).
// gridDim.z > 1 splits K into gridDim.z chunks of kchunk, chunk z stored at C + z M ldc.
template <bool TA, bool TB, int EPI, bool BF16>
__global__ void __launch_bounds__(kGemmThreads) k_gemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                                      const float* __restrict__ B, int ldb, float* C, int ldc,
                                                      const float* __restrict__ bias, const float* __restrict__ aux,
                                                      int ldaux, int kchunk) {
  __shared__ float As[kBK][kBM + 4];
  __shared__ float Bs[kBK][kBN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = kb; k0 < ke; k0 += kBK) {
#pragma unroll
    for (int r = 0; r < (kBM * kBK) / kGemmThreads; ++r) {
      const int idx = tid + r * kGemmThreads;
      int mm, kk;
      if (TA) { mm = idx % kBM; kk = idx / kBM; }
      else { kk = idx % kBK; mm = idx / kBK; }
      const int gm = m0 + mm, gk = k0 + kk;
      float v = 0.f;
      if (gm < M && gk < ke) v = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
      As[kk][mm] = BF16 ? round_bf16(v) : v;
    }
#pragma unroll
    for (int r = 0; r < (kBN * kBK) / kGemmThreads; ++r) {
      const int idx = tid + r * kGemmThreads;
      int nn, kk;
      if (TB) { kk = idx % kBK; nn = idx / kBK; }
      else { nn = idx % kBN; kk = idx / kBN; }
      const int gn = n0 + nn, gk = k0 + kk;
      float v = 0.f;
      if (gn < N && gk < ke) v = TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
      Bs[kk][nn] = BF16 ? round_bf16(v) : v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kBK; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  float* Cz = C + (size_t)blockIdx.z * M * ldc;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= N) continue;
      float v = acc[i][j];
      if (EPI == 1) v = tanhf(v + bias[n]);
      else if (EPI == 2) v += bias[n];
      else if (EPI == 3) {
        const float h = aux[(size_t)m * ldaux + n];
        v *= 1.f - h * h;
      }
      Cz[(size_t)m * ldc + n] = v;
    }
  }
}

// BF16 inference on the tensor cores: C [M][N] = A [M][K] W^T + bias (tanh
// when EPI = 1), W stored [N][K], both rounded to BF16, FP32 accumulation,
// by mma.sync m16n8k16 (row.col, bf16 x bf16 -> f32).  Block tile 64 x 64,
// four warps of 32 x 32 (2 x 4 tiles of 16 x 8), K in slices of 16 staged in
// shared memory as BF16.
constexpr int kTcBM = 64, kTcBN = 64, kTcBK = 16;

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x (low half) = lo
  return *reinterpret_cast<const unsigned*>(&v);
}

template <int EPI>
__global__ void __launch_bounds__(128) k_gemm_bf16_tc(int M, int N, int K, const float* __restrict__ A, int lda,
                                                     const float* __restrict__ W, int ldw, float* C, int ldc,
                                                     const float* __restrict__ bias) {
  // BF16 pairs along k: As[m][k/2], Ws[n][k/2] (one 32-bit word = two k values)
  __shared__ unsigned As[kTcBM][kTcBK / 2 + 1];
  __shared__ unsigned Ws[kTcBN][kTcBK / 2 + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m0 = blockIdx.y * kTcBM, n0 = blockIdx.x * kTcBN;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;  // warp tile origin in the block tile
  const int g = lane >> 2, tg = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
  for (int k0 = 0; k0 < K; k0 += kTcBK) {
    // stage: 64 rows x 8 pairs for A and for W, 128 threads x 4 pairs each
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int idx = tid + 128 * r, row = idx >> 3, kp = idx & 7, k = k0 + 2 * kp;
      const int gm = m0 + row, gn = n0 + row;
      float a0 = 0.f, a1 = 0.f, w0 = 0.f, w1 = 0.f;
      if (gm < M) {
        if (k < K) a0 = A[(size_t)gm * lda + k];
        if (k + 1 < K) a1 = A[(size_t)gm * lda + k + 1];
      }
      if (gn < N) {
        if (k < K) w0 = W[(size_t)gn * ldw + k];
        if (k + 1 < K) w1 = W[(size_t)gn * ldw + k + 1];
      }
      As[row][kp] = pack_bf16(a0, a1);
      Ws[row][kp] = pack_bf16(w0, w1);
    }
    __syncthreads();
    unsigned af[2][4], bf[4][2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int r0 = wm + 16 * i + g;
      af[i][0] = As[r0][tg];          // rows g,   k 2tg..2tg+1
      af[i][1] = As[r0 + 8][tg];      // rows g+8, k 2tg..2tg+1
      af[i][2] = As[r0][tg + 4];      // rows g,   k 2tg+8..
      af[i][3] = As[r0 + 8][tg + 4];  // rows g+8, k 2tg+8..
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = wn + 8 * j + g;
      bf[j][0] = Ws[n][tg];      // k 2tg..2tg+1, column n
      bf[j][1] = Ws[n][tg + 4];  // k 2tg+8..,    column n
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
            "{%0, %1, %2, %3};"
            : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
            : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bf[j][0]), "r"(bf[j][1]));
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = m0 + wm + 16 * i + g + (r >= 2 ? 8 : 0);
        const int n = n0 + wn + 8 * j + 2 * tg + (r & 1);
        if (m < M && n < N) {
          float v = acc[i][j][r] + bias[n];
          if (EPI == 1) v = tanhf(v);
          C[(size_t)m * ldc + n] = v;
        }
      }
}

// out[i] = sum over z of part[z count + i], in z order.
__global__ void k_reduce_splits(const float* __restrict__ part, int splits, int64_t count, float* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  float s = 0.f;
  for (int z = 0; z < splits; ++z) s += part[(size_t)z * count + i];
  out[i] = s;
}

// out[j] = sum over rows of A[r][j] (one block per column, fixed-order tree).
__global__ void k_colsum(const float* __restrict__ A, int rows, int ld, float* out) {
  __shared__ float sh[256];
  const int j = blockIdx.x;
  float s = 0.f;
  for (int r = threadIdx.x; r < rows; r += 256) s += A[(size_t)r * ld + j];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = sh[0];
}

// dY = scale (Y - Z) and per-block sums of (Y - Z)^2 (FP64).
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ Z, int64_t count, float scale,
                      float* dY, double* part) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < count; i += (int64_t)gridDim.x * 256) {
    const float r = Y[i] - Z[i];
    dY[i] = scale * r;
    s += (double)r * (double)r;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// acc += sum of part[0 .. n) / denom, by one thread (fixed order).
__global__ void k_accumulate(const double* __restrict__ part, int n, double denom, double* acc) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += part[i];
  *acc += s / denom;
}

__global__ void k_adam(float* p, const float* __restrict__ g, float* m, float* v, int64_t n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// The 15 local values of cell c of state X: signed velocity coefficients, elevation values.
__device__ __forceinline__ void cell_local(const DeviceMesh& m, int64_t c, const double* __restrict__ X,
                                           double out[15]) {
  int dof[12];
  double sg[12];
  cell_dofs(m, c, dof, sg);
#pragma unroll
  for (int k = 0; k < 12; ++k) out[k] = sg[k] * __ldg(&X[dof[k]]);
#pragma unroll
  for (int j = 0; j < 3; ++j) out[12 + j] = __ldg(&X[m.n_u + 3 * c + j]);
}

__device__ __forceinline__ int64_t across(const DeviceMesh& m, int64_t c, int i) {
  const int e = m.cell_edges[i * m.F + c];
  const int p = m.edge_plus[e];
  return p == c ? m.edge_minus[e] : p;
}

// Row c of the feature matrix: own U, own V, then (U, V) of the cells across
// local edges 0, 1, 2, then the 4 geometric values; velocity values over the
// row cell's length scale sqrt(det_c); (x - mu) / sd when mu is given.
__global__ void k_sur_features(DeviceMesh m, const double* __restrict__ U, const double* __restrict__ V,
                               const float* __restrict__ geo, const float* __restrict__ mu,
                               const float* __restrict__ sd, float* X) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m.F) return;
  float* row = X + (size_t)c * kSurInputs;
  const double inv_ell = 1.0 / sqrt(m.det[c]);
  double v[15];
  auto put = [&](int base) {
#pragma unroll
    for (int k = 0; k < 15; ++k) {
      float x = (float)(k < 12 ? v[k] * inv_ell : v[k]);
      if (mu) x = (x - mu[base + k]) / sd[base + k];
      row[base + k] = x;
    }
  };
  cell_local(m, c, U, v);
  put(0);
  cell_local(m, c, V, v);
  put(15);
  for (int i = 0; i < 3; ++i) {
    const int64_t nb = across(m, c, i);
    cell_local(m, nb, U, v);
    put(30 + 30 * i);
    cell_local(m, nb, V, v);
    put(45 + 30 * i);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float x = geo[4 * c + k];
    if (mu) x = (x - mu[120 + k]) / sd[120 + k];
    row[120 + k] = x;
  }
}

// Row c of the targets: local values of Vf - Vc, velocity values over
// sqrt(det_c), (z - mu) / sd when mu is given.
__global__ void k_sur_targets(DeviceMesh m, const double* __restrict__ Vf, const double* __restrict__ Vc,
                              const float* __restrict__ mu, const float* __restrict__ sd, float* Z) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m.F) return;
  double a[15], b[15];
  cell_local(m, c, Vf, a);
  cell_local(m, c, Vc, b);
  const double inv_ell = 1.0 / sqrt(m.det[c]);
#pragma unroll
  for (int k = 0; k < 15; ++k) {
    float z = (float)(k < 12 ? (a[k] - b[k]) * inv_ell : a[k] - b[k]);
    if (mu) z = (z - mu[k]) / sd[k];
    Z[(size_t)c * kSurOutputs + k] = z;
  }
}

// corr += scatter of the de-standardised outputs (velocity values times
// sqrt(det_c)): interior velocity and
// elevation values stored, edge values half from each of the two cells
// (corr's edge DOFs zero on entry; two additions into zero are exact in
// either order).
__global__ void k_sur_scatter(DeviceMesh m, const float* __restrict__ Y, const float* __restrict__ mu,
                              const float* __restrict__ sd, double* corr) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m.F) return;
  int dof[12];
  double sg[12];
  cell_dofs(m, c, dof, sg);
  double y[15];
  const double ell = sqrt(m.det[c]);
#pragma unroll
  for (int k = 0; k < 15; ++k) {
    y[k] = (double)Y[(size_t)c * kSurOutputs + k] * (double)sd[k] + (double)mu[k];
    if (k < 12) y[k] *= ell;
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) atomicAdd(&corr[dof[k]], 0.5 * sg[k] * y[k]);
#pragma unroll
  for (int k = 9; k < 12; ++k) corr[dof[k]] = y[k];
#pragma unroll
  for (int j = 0; j < 3; ++j) corr[m.n_u + 3 * c + j] = y[12 + j];
}

// Column means and standard deviations of X [rows][cols] (FP64 sums, two passes).
__global__ void k_colstats(const float* __restrict__ X, int64_t rows, int cols, float* mu, float* sd) {
  __shared__ double sh[256];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < rows; r += 256) s += X[(size_t)r * cols + j];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double mean = sh[0] / (double)rows;
  __syncthreads();
  s = 0.0;
  for (int64_t r = threadIdx.x; r < rows; r += 256) {
    const double d = X[(size_t)r * cols + j] - mean;
    s += d * d;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double var = sh[0] / (double)rows;
    mu[j] = (float)mean;
    sd[j] = var > 0.0 ? (float)sqrt(var) : 1.f;
  }
}

__global__ void k_standardize(float* X, int64_t rows, int cols, const float* __restrict__ mu,
                              const float* __restrict__ sd) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  const int j = (int)(i % cols);
  X[i] = (X[i] - mu[j]) / sd[j];
}

// dst[r][:] = src[idx[r]][:] for r < rows.
__global__ void k_gather_rows(const float* __restrict__ src, const int* __restrict__ idx, int rows, int cols,
                              float* dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)rows * cols) return;
  const int r = (int)(i / cols), j = (int)(i % cols);
  dst[i] = src[(size_t)idx[r] * cols + j];
}

template <bool TA, bool TB, int EPI, bool BF16>
cudaError_t gemm_t(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                   const float* bias, const float* aux, int ldaux, int splits, cudaStream_t st) {
  const int kchunk = splits > 1 ? ((K + splits - 1) / splits + kBK - 1) / kBK * kBK : K;
  dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM, splits > 1 ? splits : 1);
  k_gemm<TA, TB, EPI, BF16><<<grid, kGemmThreads, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, aux, ldaux,
                                                          kchunk);
  return cudaGetLastError();
}

template <int EPI>
cudaError_t gemm_bf16_tc(int M, int N, int K, const float* A, int lda, const float* W, int ldw, float* C, int ldc,
                         const float* bias, cudaStream_t st) {
  dim3 grid((N + kTcBN - 1) / kTcBN, (M + kTcBM - 1) / kTcBM);
  k_gemm_bf16_tc<EPI><<<grid, 128, 0, st>>>(M, N, K, A, lda, W, ldw, C, ldc, bias);
  return cudaGetLastError();
}

}  // namespace

cudaError_t sur_gemm(SurGemm kind, int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C,
                     int ldc, const float* bias, const float* aux, int ldaux, int splits, bool bf16,
                     cudaStream_t st) {
  switch (kind) {
    case SurGemm::kForwardTanh:  // A [M][K], B = W [N][K]
      if (bf16) return gemm_bf16_tc<1>(M, N, K, A, lda, B, ldb, C, ldc, bias, st);
      return gemm_t<false, true, 1, false>(M, N, K, A, lda, B, ldb, C, ldc, bias, aux, ldaux, 1, st);
    case SurGemm::kForwardLinear:
      if (bf16) return gemm_bf16_tc<2>(M, N, K, A, lda, B, ldb, C, ldc, bias, st);
      return gemm_t<false, true, 2, false>(M, N, K, A, lda, B, ldb, C, ldc, bias, aux, ldaux, 1, st);
    case SurGemm::kBackwardData:  // dA = (dY [M][K] W [K][N]) (1 - H^2)
      return gemm_t<false, false, 3, false>(M, N, K, A, lda, B, ldb, C, ldc, bias, aux, ldaux, 1, st);
    case SurGemm::kWeightGrad:  // dW [M][N] = dY^T (dY stored [K][M]) X [K][N], split over K
      return gemm_t<true, false, 0, false>(M, N, K, A, lda, B, ldb, C, ldc, bias, aux, ldaux, splits, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t sur_reduce_splits(const float* part, int splits, int64_t count, float* out, cudaStream_t st) {
  k_reduce_splits<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(part, splits, count, out);
  return cudaGetLastError();
}

cudaError_t sur_colsum(const float* A, int rows, int cols, int ld, float* out, cudaStream_t st) {
  k_colsum<<<cols, 256, 0, st>>>(A, rows, ld, out);
  return cudaGetLastError();
}

cudaError_t sur_mse(const float* Y, const float* Z, int64_t count, float scale, float* dY, double* part, int nblocks,
                    double denom, double* acc, cudaStream_t st) {
  k_mse<<<nblocks, 256, 0, st>>>(Y, Z, count, scale, dY, part);
  k_accumulate<<<1, 1, 0, st>>>(part, nblocks, denom, acc);
  return cudaGetLastError();
}

cudaError_t sur_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2, float eps,
                     float c1, float c2, cudaStream_t st) {
  k_adam<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t sur_features(const DeviceMesh& m, const double* U, const double* V, const float* geo, const float* mu,
                         const float* sd, float* X, cudaStream_t st) {
  k_sur_features<<<(unsigned)((m.F + 127) / 128), 128, 0, st>>>(m, U, V, geo, mu, sd, X);
  return cudaGetLastError();
}

cudaError_t sur_targets(const DeviceMesh& m, const double* Vf, const double* Vc, const float* mu, const float* sd,
                        float* Z, cudaStream_t st) {
  k_sur_targets<<<(unsigned)((m.F + 127) / 128), 128, 0, st>>>(m, Vf, Vc, mu, sd, Z);
  return cudaGetLastError();
}

cudaError_t sur_scatter(const DeviceMesh& m, const float* Y, const float* mu, const float* sd, double* corr,
                        cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(corr, 0, sizeof(double) * 3 * m.E, st);
  if (e != cudaSuccess) return e;
  k_sur_scatter<<<(unsigned)((m.F + 127) / 128), 128, 0, st>>>(m, Y, mu, sd, corr);
  return cudaGetLastError();
}

cudaError_t sur_colstats(const float* X, int64_t rows, int cols, float* mu, float* sd, cudaStream_t st) {
  k_colstats<<<cols, 256, 0, st>>>(X, rows, cols, mu, sd);
  return cudaGetLastError();
}

cudaError_t sur_standardize(float* X, int64_t rows, int cols, const float* mu, const float* sd, cudaStream_t st) {
  const int64_t n = rows * cols;
  k_standardize<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(X, rows, cols, mu, sd);
  return cudaGetLastError();
}

cudaError_t sur_gather_rows(const float* src, const int* idx, int rows, int cols, float* dst, cudaStream_t st) {
  const int64_t n = (int64_t)rows * cols;
  k_gather_rows<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, idx, rows, cols, dst);
  return cudaGetLastError();
}

}  // namespace pavg
