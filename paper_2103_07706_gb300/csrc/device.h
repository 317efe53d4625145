// Device-side data of one context and the host wrappers that launch kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "pavg_internal.h"

namespace pavg {

enum : int { kFlagNoConv = 1, kFlagTimeout = 2, kFlagNonFinite = 4 };

struct DeviceMesh {
  int64_t F = 0, E = 0, n_u = 0, n_eta = 0, n = 0;
  int32_t* cell_edges = nullptr;    // [3][F]
  uint8_t* cell_aligned = nullptr;  // [F]
  int32_t* edge_plus = nullptr;     // [E]
  int32_t* edge_minus = nullptr;    // [E]
  uint8_t* edge_lpos = nullptr;     // [E]
  double* M1 = nullptr;             // [78][F]
  double* C = nullptr;              // [66][F]
  float* Cf = nullptr;              // [66][F] C rounded to FP32 (the mixed mode's K-hat products)
  double* det = nullptr;            // [F]
  double* G = nullptr;              // [3][F]
  double* dinv = nullptr;           // [n_u]
  double* topo = nullptr;           // [n_eta] topography b
  float* M1f = nullptr;             // [36][F][4] M1 element matrices in FP32, row blocks of 3 rows per triple
  float* Pinv = nullptr;            // [E + F][8] inverses of the 3x3 diagonal blocks of M1, FP32, padded
  float* M1p = nullptr;             // [78][F] packed M1 in FP32 (loaded into shared memory), or null
  int32_t* tri = nullptr;           // [F][4] DOF triple of (cell, q) with the owner flag in bit 31
  // piecewise cubic surface only (null on flat cells, where M2 = det * M2_ref)
  double* M2e = nullptr;            // [6][F] DG1 element mass matrices, packed 00, 01, 02, 11, 12, 22
  double* M2i = nullptr;            // [6][F] their inverses
  double* geo_c = nullptr;          // [6][kCellQ3][F] G00, G01, G11, w / det^2, d0 det / det, d1 det / det
  double* geo_f = nullptr;          // [8][kFacetQ3][E] plus side G00, G01, G11, 1 / det; then minus side
};

// Scratch of the persistent CG solver.
struct CgWork {
  double* x = nullptr;        // [n_u]
  double* r[2] = {nullptr, nullptr};
  double* s[2] = {nullptr, nullptr};
  double* w[3] = {nullptr, nullptr, nullptr};
  double* p = nullptr;
  double* partial = nullptr;  // [2][3][nblocks] (double-buffered)
  unsigned* bar = nullptr;    // [2]: arrival counter, generation
  int* flags = nullptr;       // latched error flags
  unsigned long long* stats = nullptr;  // [0] solves, [1] iterations, [2] max iterations
  int nblocks = 0;
  int threads = 0;
};

struct CgParams {
  double rtol;
  int maxit;
};

// Scratch of the mixed-precision solver: FP32 conjugate gradients on M1 with a
// 3x3 block-Jacobi preconditioner, refined by FP64 residuals b - M1 x.
struct CgIrWork {
  double* x[2] = {nullptr, nullptr};   // FP64 iterate (ping-pong between sweeps)
  double* ax = nullptr;                // FP64 M1 x (assembled; edge part zero between uses)
  double* r64 = nullptr;               // FP64 residual
  // FP32 vectors, one allocation of 9 slots of T = E + F triples x 4 floats
  // (each DOF triple padded to 16 bytes), addressed by 32-bit offsets:
  // slot 0 correction x, 1-2 residual r, 3-4 s, 5-7 w (three rotating), 8 p
  float* fbuf = nullptr;
  float* xf = nullptr;                 // views into fbuf
  float* rf[2] = {nullptr, nullptr};
  float* sf[2] = {nullptr, nullptr};
  float* wf[3] = {nullptr, nullptr, nullptr};
  float* pf = nullptr;
  double* partial = nullptr;           // [3][nblocks] per-block partial sums (FP64 phases)
  float* partial_f = nullptr;          // [3][nblocks] per-block partial sums (FP32 phases)
  double* scal = nullptr;              // [4] published global sums (FP64 phases)
  unsigned long long* tag = nullptr;   // [4] published sums tagged with their barrier epoch
  unsigned* bar = nullptr;             // [2]
  int* flags = nullptr;
  unsigned long long* stats = nullptr; // [0] solves, [1] inner iterations, [2] max per solve, [3] sweeps
  int nblocks = 0;
  int passes = 0;        // cells per block / 64, rounded up
  size_t smem = 0;       // dynamic shared memory: resident FP32 element matrices (0: streamed)
};

struct CgIrParams {
  double rtol;        // FP64 relative residual target
  int max_sweeps;     // FP64 refinement sweeps
  float inner_rtol;   // FP32 inner reduction per sweep
  int max_inner;      // FP32 iterations per sweep
};

// Chooses the grid and whether the FP32 element matrices stay resident in
// shared memory for the whole solve (fills w->nblocks, passes, smem).
cudaError_t cg_ir_configure(int64_t F, CgIrWork* w);

// out_u = scale_x * M1^{-1} b + add, mixed precision, FP64-accurate.
cudaError_t launch_cg_ir(const DeviceMesh& m, const CgIrWork& w, const CgIrParams& cp, const double* b,
                         double* out, double scale_x, const double* add, cudaStream_t st);

// Subdomain mass solver (cheb_sd.cu).  One block per part of a contiguous
// partition of the cells; each part keeps its cells' FP32 element matrices
// in shared memory and its DOF triples' FP32 vectors in registers, and
// exchanges only the contributions to the triples it shares with a
// neighbouring part (tagged words, no grid-wide wait per inner iteration).
// Read-only partition data, shared by the contexts of one mesh:
struct SdMesh {
  int P = 0;                     // parts = blocks of the cooperative launch (0: not available)
  int max_cells = 0, max_lt = 0, nslots = 0, total_lt = 0;
  size_t smem = 0;               // dynamic shared memory per block
  double lmin = 0, lmax = 0;     // Lanczos estimates of the spectrum of P M1
  int32_t* cell0 = nullptr;      // [P+1]
  int32_t* lt0 = nullptr;        // [P+1]
  uint32_t* lt_gtri = nullptr;   // [lt] global triple | owner bit 31
  uint32_t* lt_slot = nullptr;   // [lt] two 16-bit local (cell, q) positions, 0xffff = none
  int32_t* lt_recv = nullptr;    // [lt] partner's send slot of a shared triple, -1 otherwise
  ushort4* cell_lt = nullptr;    // [F] local triples of the cell's four (cell, q)
  int4* cell_send = nullptr;     // [F] send slot of (cell, q), q < 3, -1 when not shared
};

// Per-context scratch of the subdomain solver.
struct SdWork {
  unsigned long long* xch32 = nullptr;  // [2][nslots][4] tagged FP32 words (3 used)
  unsigned long long* xch64 = nullptr;  // [2][nslots][6] tagged 32-bit halves of FP64 values
  double* y64 = nullptr;                // [F][12] FP64 cell contributions of a refinement product
  double* x64 = nullptr;                // [lt][3] FP64 iterate, each part's own copy of its triples
  double* r64 = nullptr;                // [lt][3] FP64 residual of the last sweep, likewise
  double* part = nullptr;               // [P] block partial sums
  double* pub = nullptr;                // [1] published grid sum
  unsigned long long* sync = nullptr;   // [4]: arrivals (monotonic), published tag, epoch base, spare
  int* flags = nullptr;
  unsigned long long* stats = nullptr;
};

struct SdParams {
  double rtol;          // FP64 relative residual target
  int max_sweeps;       // FP64 refinement sweeps
  int iters;            // Chebyshev iterations per sweep
  double theta, delta;  // centre and half-width of the Chebyshev interval
  long long wait_cycles;  // bound of every wait on another block (clock64 cycles)
  int stall_mode;       // test hook, 0 = off; 1: block stall_part never arrives at the first grid sum;
  int stall_part;       //            2: block stall_part never publishes its shared contributions
};

// Builds the partition of F cells into P parts on the current device when its
// blocks fit in shared memory and are co-resident; sd->P = 0 otherwise.
// [lmin, lmax]: the spectrum estimate of the preconditioned M1 (sd_spectrum).
cudaError_t sd_configure(int64_t F, int64_t E, const std::vector<int32_t>& tri, double lmin, double lmax, int P,
                         SdMesh* sd);
void sd_free(SdMesh* sd);
cudaError_t sd_alloc_work(const SdMesh& sd, int64_t F, SdWork* w);
void sd_free_work(SdWork* w);
// Clears the exchange words and synchronisation counters (after a failed launch).
cudaError_t sd_reset_work(const SdMesh& sd, int64_t F, SdWork* w);
// out_u = scale_x * M1^{-1} b + add, FP64-accurate.
cudaError_t launch_cheb_sd(const DeviceMesh& m, const SdMesh& sd, const SdWork& w, const SdParams& sp,
                           const double* b, double* out, double scale_x, const double* add, cudaStream_t st);

// One problem of the batched persistent recurrence kernel (k_chain): one
// instance's whole forward Chebyshev chain (mode 0, K steps)
//   Q_{k+1} = M^{-1}(s_k Khat Q_k) + Q_{k-1},  s_0 = 1/lam, s_k = 2/lam,
// or its Clenshaw recurrence (mode 1, K + 1 steps, k = K .. 0)
//   b_k = M^{-1}(y_k + s_k Khat b_{k+1}) + b_{k+2}   (b_0 is the result),
// run by the blocks block0 .. block0 + nblocks - 1 of the launch, which
// synchronise only among themselves.
struct ChainProblem {
  DeviceMesh m;
  CgIrWork w;                   // solver scratch of the instance's context
  CgIrParams cp;
  double g, H, lam;
  double* ru;                   // [n_u] assembled velocity right-hand side
  double* Q;                    // mode 0: Q_0 .. Q_K; mode 1: y_0 .. y_K  ([K+1][n])
  double* bufs[3];              // mode 1: b_k in bufs[k % 3]
  double* out;                  // mode 1: result b_0
  double* partial;              // [3][nblocks] per-block sums, FP64 phases
  float* partial_f;             // [3][nblocks] per-block sums, FP32 phases
  double* scal;                 // [8]
  unsigned long long* sync;     // [8]: arrival counter (word 0), tagged sums (words 1-4); zero at launch
  unsigned long long* timer;    // [2] or null: global timer (ns) when the problem's steps start and end
  int mode, K;
  int block0, nblocks;
};

// Launch of k_chain over P problems and nblocks_total co-resident blocks of
// nt threads (128 or 256).  res: FP32 element matrices resident in shared
// memory (smem bytes per block).  max_steps >= 0 stops every problem after
// that many steps (autotuning runs).  Cooperative launch: all blocks are
// co-resident.
cudaError_t launch_chain(const ChainProblem* d_probs, int P, int nblocks_total, int nt, bool res, size_t smem,
                         int max_steps, cudaStream_t st);
// Blocks of k_chain<nt, res> that fit on one SM with smem dynamic bytes.
cudaError_t chain_occupancy(int nt, bool res, size_t smem, int* per_sm);
// Dynamic shared memory of the resident path for a problem of F cells on nb blocks.
size_t chain_res_smem(int64_t F, int nb, int nt);
// Upload of the reference-element tables used by k_chain.
cudaError_t upload_chain_tables(const ConstTables& t);

// ---- learned surrogate (surrogate.cu)
constexpr int kSurInputs = 124;   // 8 x 15 local values + 4 geometric values
constexpr int kSurOutputs = 15;

enum class SurGemm {
  kForwardTanh,    // C [M][N] = tanh(A [M][K] W^T + bias), W stored [N][K]
  kForwardLinear,  // C = A W^T + bias
  kBackwardData,   // C [M][N] = (A [M][K] W [K][N]) (1 - aux^2)
  kWeightGrad,     // C [M][N] = A^T B, A stored [K][M], B [K][N]; split over K into `splits` partials
};
cudaError_t sur_gemm(SurGemm kind, int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C,
                     int ldc, const float* bias, const float* aux, int ldaux, int splits, bool bf16,
                     cudaStream_t st);
cudaError_t sur_reduce_splits(const float* part, int splits, int64_t count, float* out, cudaStream_t st);
cudaError_t sur_colsum(const float* A, int rows, int cols, int ld, float* out, cudaStream_t st);
// dY = scale (Y - Z); *acc += sum (Y - Z)^2 / denom (part: nblocks doubles of scratch).
cudaError_t sur_mse(const float* Y, const float* Z, int64_t count, float scale, float* dY, double* part, int nblocks,
                    double denom, double* acc, cudaStream_t st);
cudaError_t sur_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2, float eps,
                     float c1, float c2, cudaStream_t st);
// Feature rows [F][124] of (U, V); geo [F][4]; standardised when mu is not null.
cudaError_t sur_features(const DeviceMesh& m, const double* U, const double* V, const float* geo, const float* mu,
                         const float* sd, float* X, cudaStream_t st);
// Target rows [F][15] = local values of Vf - Vc; standardised when mu is not null.
cudaError_t sur_targets(const DeviceMesh& m, const double* Vf, const double* Vc, const float* mu, const float* sd,
                        float* Z, cudaStream_t st);
// corr (n) = scatter of Y [F][15] * sd + mu (edge DOFs: mean of the two cells).
cudaError_t sur_scatter(const DeviceMesh& m, const float* Y, const float* mu, const float* sd, double* corr,
                        cudaStream_t st);
cudaError_t sur_colstats(const float* X, int64_t rows, int cols, float* mu, float* sd, cudaStream_t st);
cudaError_t sur_standardize(float* X, int64_t rows, int cols, const float* mu, const float* sd, cudaStream_t st);
cudaError_t sur_gather_rows(const float* src, const int* idx, int rows, int cols, float* dst, cudaStream_t st);

// Upload constant tables (reference element data) to the current device.
cudaError_t upload_tables(const ConstTables& t);
cudaError_t upload_tables3(const TablesP3<double>& t);  // the cubic-geometry nonlinear kernels' tables

// Grid size for the persistent CG kernel (all blocks co-resident).
cudaError_t cg_configure(int64_t F, CgWork* w);

// out_u = scale_x * M1^{-1} b + add (add may be null); all [n_u].
cudaError_t launch_cg(const DeviceMesh& m, const CgWork& w, const CgParams& cp, const double* b,
                      double* out, double scale_x, const double* add, cudaStream_t st);

// Linear-operator application of the recurrences (Sec. 2.5 weak forms):
//   ru  = y_u + s (-C u + g D^T eta)          (assembled weak-form velocity rhs)
//   eta_out = M2^{-1} (y_eta + s (-H D u)) + z_eta
// y_u, y_eta, z_eta may be null (zero).  ru must be zeroed on the edge DOFs
// (the first 3E entries) before the call.
cudaError_t launch_apply_K(const DeviceMesh& m, const double* U, double s, double g, double H,
                           const double* y_u, const double* y_eta, const double* z_eta,
                           double* ru, double* eta_out, cudaStream_t st, bool fp32 = false);

// Weak-form right-hand side of N for B states [B][n] -> r [B][n]
// (r's velocity edge DOFs must be zeroed first), in chunks of `chunk` states:
// per chunk one launch over the edges (facet terms of both cells, into
// `facets`, chunk x F x 3 x 15 doubles of scratch) and one over the cells.
// kFacetChunk is the largest chunk (contexts use fewer on large meshes).
// fp32: FP32 arithmetic per quadrature point, FP64 sums over the points.
constexpr int kFacetChunk = 16;
cudaError_t launch_nonlinear_rhs(const DeviceMesh& m, const double* U, double* r, int B,
                                 int upwind, cudaStream_t st, bool fp32, double* facets, int chunk);

// eta_out = M2^{-1} r_eta (+ add) for B blocks of n_eta with strides.
cudaError_t launch_m2inv(const DeviceMesh& m, const double* r, int64_t rstride, double* out,
                         int64_t ostride, int B, cudaStream_t st);

// out[m][j] = sum_k A[m][k] in[k][j], j < len.  A is [Mo][Ki] in device
// memory; rows are processed in tiles of combine_tile(), and when lim is not
// null tile t only uses k < lim[t] (the rest of its rows being zero).
int combine_tile();
cudaError_t launch_combine(const double* A, int Mo, int Ki, const int* lim, const double* in, int64_t in_stride,
                           double* out, int64_t out_stride, int64_t len, cudaStream_t st, bool fp32 = false);

// The contractions for shifts in +/- pairs (equal coefficients and weights):
// forward out[2p] = E_p + O_p, out[2p+1] = E_p - O_p from A [P][Ki] (even and
// odd k of row p), lim per tile of combine_tile() pairs; backward out[k] =
// sum_p B[k][p] (k even ? R[2p+1] + R[2p] : R[2p+1] - R[2p]), lim per tile of
// combine_tile() rows (pairs with a nonzero entry).
cudaError_t launch_combine_pairs_fwd(const double* A, int P, int Ki, const int* lim, const double* in,
                                     int64_t in_stride, double* out, int64_t out_stride, int64_t len,
                                     cudaStream_t st, bool fp32 = false);
cudaError_t launch_combine_pairs_bwd(const double* B, int Ko, int P, const int* lim, const double* R,
                                     int64_t r_stride, double* out, int64_t out_stride, int64_t len,
                                     cudaStream_t st);

// out = a x + b y (+ c z); any of y, z may be null.
cudaError_t launch_lincomb(double* out, double a, const double* x, double b, const double* y,
                           double c, const double* z, int64_t len, cudaStream_t st);

// Energy inner products <U, V>_W = H u^T M1 v + g eta^T M2 zeta, per block partials
// written to part (size >= nblocks returned).  Host sums them.
cudaError_t launch_winner(const DeviceMesh& m, const double* U, const double* V, double g, double H,
                          double* part, int* nblocks, cudaStream_t st);

// Per-block partial sums [nblocks][3] of u^T M1 u, ||div u||^2 and eta^T M2 eta.
cudaError_t launch_norms(const DeviceMesh& m, const double* U, double* part, int* nblocks, cudaStream_t st);

// Sets kFlagNonFinite when any entry of x is not finite.
cudaError_t launch_check_finite(const double* x, int64_t len, int* flags, cudaStream_t st);

}  // namespace pavg
