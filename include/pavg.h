/*
 * pavg.h - phase-averaged rotating shallow water on the sphere, GB300 (sm_103a).
 *
 * C-ABI of libpavg.so.  The method is that of Yamazaki, Cotter & Wingate,
 * "Time parallel integration and phase averaging for the nonlinear shallow
 * water equations on the sphere" (arXiv 2103.07706):
 *   U_t = L U + N(U)                                   (Sec. 2.1, Eq. split_eqs)
 *   N-bar(U) = sum_m w_m e^{-s_m L} N(e^{s_m L} U)      (Sec. 2.2, Eq. vt_discretised)
 *   e^{tL} by a truncated Chebyshev series               (Sec. 2.4, Eq. cheby)
 *   averaged Lawson RK4                                  (Sec. 2.3, Eqs. stage1_c-stage4)
 * with L and N the compatible finite element operators of Sec. 2.5
 * (BDM2 velocity, DG1 elevation) on an icosahedral mesh (Sec. 3).
 *
 * Conventions shared by every call
 * --------------------------------
 * State vectors are FP64, contiguous, u first then eta:
 *   U = [u (n_u = 3E + 3F) | eta (n_eta = 3F)],  n = n_u + n_eta,
 * F = 20 * 4^r cells, E = 30 * 4^r edges.  Velocity DOF 3e + j is the j-th
 * Legendre moment (j = 0, 1, 2 on [0, 1], low -> high vertex) of the flux
 * across edge e towards the side of t x k (t the low->high tangent, k the
 * cell's outward normal); DOF 3E + 3c + j is the j-th interior moment of cell c
 * against (1,0), (0,1), (-y,x) on the reference triangle.  Elevation DOF
 * 3c + i is the value at local vertex i of cell c.  Cells, vertices and edges
 * are numbered by the canonical icosahedral construction exported by
 * pavg_mesh_export.  A batch of B states is laid out [B][n]; B = 0 is a
 * valid empty batch (no work; its state pointers may then be NULL).
 *
 * Pointers marked "device" are caller-owned CUDA device memory (e.g. a torch
 * tensor's data_ptr()); the library never frees them.  Calls that take a
 * `stream` enqueue their work on that cudaStream_t (NULL = legacy default
 * stream) and return without synchronising unless stated; the caller keeps
 * inputs alive until the work completes.  One context must not be used from
 * two streams at the same time: it owns one set of scratch buffers.
 *
 * Every function returns PAVG_OK (0) or a negative error code and never throws.
 * Errors raised on the device (a CG solve that did not converge, a bounded
 * device-side wait that timed out, a non-finite value) are latched in the
 * context and reported by pavg_get_stats / pavg_sync.  pavg_last_error gives a
 * readable message for the last failure of a context.
 */
#ifndef PAVG_H
#define PAVG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PAVG_OK 0
#define PAVG_ERR_INVAL (-1)     /* bad argument (null pointer, size, range) */
#define PAVG_ERR_NOMEM (-2)     /* device allocation failed */
#define PAVG_ERR_CUDA (-3)      /* a CUDA runtime call failed */
#define PAVG_ERR_NOCONV (-4)    /* mass-matrix CG reached cg_maxit */
#define PAVG_ERR_NONFINITE (-5) /* NaN or Inf detected */
#define PAVG_ERR_TIMEOUT (-6)   /* a bounded device-side wait gave up */

/* Widest exponential accepted: lambda_max |t| of one e^{tL} (Sec. 2.4).  The
 * series then has about that many terms, each one mass solve. */
#define PAVG_MAX_CHEB_ARG 16384.0

#define PAVG_QUAD_MIDPOINT 0     /* s_m = -T/2 + (m + 1/2) T / M            */
#define PAVG_QUAD_CLOSED 1       /* odd M = 2N+1, s_k = k (T/2) / N, k=-N..N */
#define PAVG_UPWIND_STANDARD 0   /* u~, (eta-b)~ from the side the flow leaves */
#define PAVG_UPWIND_AS_PRINTED 1 /* u~ = u+ when u.n+ < 0, as printed in Sec. 2.5 */
#define PAVG_SOLVER_MIXED 0      /* M1 solves: FP32 block-Jacobi CG refined by FP64 residuals */
#define PAVG_SOLVER_FP64 1       /* M1 solves: FP64 Jacobi CG */
#define PAVG_SOLVER_SUBDOMAIN 2  /* M1 solves: FP32 block-Jacobi Chebyshev iterations on one part of
                                    the mesh per SM (neighbour-only exchange), refined by FP64
                                    residuals; falls back to PAVG_SOLVER_MIXED where the parts do not
                                    fit in shared memory (refinement 7 and above on 152 SMs) */
#define PAVG_PRECISION_FP64 0    /* every result FP64-accurate (mass solves to cg_rtol) */
#define PAVG_PRECISION_MIXED 1   /* N, the forward shift contraction and the K-hat products of L in
                                    FP32 arithmetic (FP64 sums over quadrature points), mass solves to
                                    max(cg_rtol, 1e-5) (one FP32 sweep, FP64 residual); the weighted sum
                                    over shifts, state vectors, recurrences and timestep updates stay
                                    FP64 */

typedef struct pavg_ctx pavg_ctx; /* opaque, library-owned */

/* Model parameters (SI units).  Sec. 2.1 (R, Omega, g, H), Sec. 2.4 (cheb_tol). */
typedef struct {
  int refinement;         /* r >= 0: F = 20 * 4^r cells (r = 5 is the paper's N_C = 20480) */
  double radius;          /* R, sphere radius [m] */
  double omega;           /* Omega, rotation rate [1/s]; f = 2 Omega z / R */
  double g;               /* gravity [m/s^2] */
  double H;               /* mean depth [m] */
  double cheb_tol;        /* Chebyshev tail threshold (1e-6 in Sec. 2.4); > 0 */
  double cg_rtol;         /* relative residual target of the M1 CG solves; > 0 */
  int cg_maxit;           /* iteration cap of each M1 CG solve; > 0 */
  double lambda_max;      /* |lambda_max| of L [1/s]; 0 -> estimate by power iteration at create */
  int quad_rule;          /* PAVG_QUAD_MIDPOINT or PAVG_QUAD_CLOSED */
  int upwind_convention;  /* PAVG_UPWIND_STANDARD or PAVG_UPWIND_AS_PRINTED */
  int solver;             /* PAVG_SOLVER_SUBDOMAIN (default), PAVG_SOLVER_MIXED or PAVG_SOLVER_FP64;
                             all reach cg_rtol in FP64; cg_maxit caps the iterations of one solve
                             (FP64) or of one refinement sweep (mixed, at most 8 sweeps); the
                             subdomain solver runs a fixed number of Chebyshev iterations per
                             sweep (at most 8 sweeps) */
  int precision;          /* PAVG_PRECISION_FP64 (default) or PAVG_PRECISION_MIXED */
  int sd_part_cells;      /* subdomain solver: 0 (default) splits the mesh over every SM (parts of
                             F / SMs cells, at least 32); > 0 asks for parts of at least this many
                             cells, so a small mesh's solve occupies fewer SMs and solves of other
                             contexts can run beside it (batches, concurrent streams) */
  int geometry_degree;    /* 1 (default): flat triangles through the mesh vertices; 3: the piecewise
                             cubic approximation of the sphere of Sec. 3 (each cell the cubic
                             interpolant of ten points projected onto the sphere), with the 5 x 5
                             Stroud cell rule and 5-point facet rule that its non-polynomial
                             integrands require; the same mesh, DOFs and state layout either way */
} pavg_params;

/* Fill `p` with the defaults: r = 3, R = 6.37122e6, Omega = 7.292e-5,
 * g = 9.80616, H = 5000, cheb_tol = 1e-6, cg_rtol = 1e-14, cg_maxit = 400,
 * lambda_max = 0, midpoint rule, standard upwinding, subdomain solver, FP64 precision,
 * sd_part_cells = 0, geometry_degree = 1. */
int pavg_default_params(pavg_params* p);

/* Build the mesh and FE data (Sec. 2.5, Sec. 3) on the current CUDA device and
 * upload them.  *out receives a new context; free it with pavg_destroy.
 * Errors: INVAL (bad params, r > 8), NOMEM, CUDA. */
int pavg_create(const pavg_params* p, pavg_ctx** out);
int pavg_destroy(pavg_ctx* ctx);

/* Sizes of the discretisation.  Any output pointer may be NULL. */
int pavg_sizes(const pavg_ctx* ctx, int64_t* n_u, int64_t* n_eta, int64_t* n_cells,
               int64_t* n_edges, int64_t* n_verts);

/* Copy the canonical mesh to HOST buffers: vert_xyz [V][3] (metres) and
 * cell_verts [F][3] (counter-clockwise seen from outside).  Either may be NULL. */
int pavg_mesh_export(const pavg_ctx* ctx, double* vert_xyz, int32_t* cell_verts);

/* Topography b as a DG1 field (device, n_eta doubles, copied).  Default 0. */
int pavg_set_topography(pavg_ctx* ctx, const double* b_dg1);

/* The lambda_max in use (given, or estimated at create).  Host output. */
int pavg_lambda_max(const pavg_ctx* ctx, double* out);

/* LU = L U for B states (device [B][n] in, device [B][n] out; may not alias).
 * Sec. 2.5, Eq. ueq_int and the eta equation after it. */
int pavg_linear(pavg_ctx* ctx, const double* U, double* LU, int B, void* stream);

/* NU = N(U) for B states (device [B][n]; may not alias).  Sec. 2.5, the two
 * weak forms after Eq. ueq_int, with upwinded facet terms. */
int pavg_nonlinear(pavg_ctx* ctx, const double* U, double* NU, int B, void* stream);

/* out = e^{tL} U for B states by the truncated Chebyshev series (Sec. 2.4,
 * Eq. cheby, truncation at cheb_tol).  t in seconds, any sign; t = 0 copies.
 * U and out are device [B][n] and may not alias.  INVAL when t is not
 * finite or lambda_max |t| > PAVG_MAX_CHEB_ARG. */
int pavg_expL_apply(pavg_ctx* ctx, double t, const double* U, double* out, int B, void* stream);

/* out = N-bar(U) = sum_m w_m e^{-s_m L} N(e^{s_m L} U) (Sec. 2.2, Eq. vt_discretised),
 * window T >= 0 seconds, M >= 1 shifts; T = 0 gives N(U).  Shared-basis
 * evaluation: one Chebyshev chain of L / lambda_max serves every shift and the
 * backward maps are summed by a Clenshaw recurrence.  This is an exact
 * rewriting of the sum: every term is a polynomial in the one operator L, so
 * the terms commute.  U, out: device, n doubles, may not alias.
 * The work for each (T, M) is captured once in a CUDA graph and replayed.
 * INVAL when T is negative or not finite, M < 1, or lambda_max T / 2 >
 * PAVG_MAX_CHEB_ARG (the widest shift's exponential). */
int pavg_averaged_rhs(pavg_ctx* ctx, double T, int M, const double* U, double* out, void* stream);

/* Part of N-bar(U): the terms of the shifts m0 <= m < m1 of the M-point rule,
 *   out = sum_{m0 <= m < m1} w_m e^{-s_m L} N(e^{s_m L} U),
 * with the weights w_m of the whole rule (normalised over all M shifts), so
 * that the partial sums of any partition of 0..M-1 into groups add up to
 * pavg_averaged_rhs(T, M).  This is the paper's parallel decomposition: the
 * Riemann terms are independent and are distributed over groups of processes
 * whose partial sums are reduced once (Sec. 2.5, last paragraph; Sec. 2.2).
 * Evaluated in the shared-basis form restricted to the group: one Chebyshev
 * chain of degree max_{m in group} K_m, so a group of small |s_m| has a
 * short chain.  With T = 0 every weight is 1/M and out = (m1 - m0)/M N(U).
 * INVAL unless 0 <= m0 < m1 <= M, and under pavg_averaged_rhs's limits. */
int pavg_averaged_rhs_group(pavg_ctx* ctx, double T, int M, int m0, int m1, const double* U, double* out,
                            void* stream);

/* The same sum in its literal form: for each shift its own forward exponential,
 * N with its mass solves and backward exponential, summed in shift order. */
int pavg_averaged_rhs_literal(pavg_ctx* ctx, double T, int M, const double* U, double* out,
                              void* stream);

/* The same average by shift marching: the shifts of both point rules are
 * equally spaced (spacing ds), so the shifted states follow one another,
 * V_0 = e^{s_0 L} U, V_{m+1} = e^{ds L} V_m, and the backward maps nest
 * (Horner): H_{M-1} = w_{M-1} N(V_{M-1}), H_m = w_m N(V_m) + e^{-ds L} H_{m+1},
 * out = e^{-s_0 L} H_0 (Sec. 2.2's sum with e^{s_{m+1} L} = e^{ds L} e^{s_m L}).
 * It needs K(|s_0|) + (M-1) K(ds) chain steps each way (K(t) the degree of
 * e^{tL}) against 2 K_max + 1 for the shared basis, and each short
 * exponential is truncated by the tail rule of Sec. 2.4, so the result
 * differs from pavg_averaged_rhs by those extra truncations (it equals the
 * direct sum as cheb_tol -> 0).  Not graph-captured.  Same limits as
 * pavg_averaged_rhs. */
int pavg_averaged_rhs_marching(pavg_ctx* ctx, double T, int M, const double* U, double* out,
                               void* stream);

/* nsteps averaged Lawson RK4 steps of size dt (Sec. 2.3, Eqs. stage1_c to stage4),
 * in place on the device state U_inout (n doubles).  INVAL for a
 * non-finite dt or T, for lambda_max |dt| > PAVG_MAX_CHEB_ARG (each step
 * applies e^{dt L}), and under pavg_averaged_rhs's limits on T and M.
 * Asynchronous on `stream` like the other state calls (no synchronisation,
 * no allocation per step): the seven stage vectors of a step are context
 * workspace, allocated by the first call (NOMEM if that fails). */
int pavg_timestep(pavg_ctx* ctx, double dt, double T, int M, double* U_inout, int nsteps,
                  void* stream);

/* LU = L U for ONE state (device, n doubles each; may not alias), computed
 * without any device allocation: all scratch (assembled right-hand side,
 * conjugate-gradient work vectors) comes from a file-scope device array of the
 * library sized for at most 153600 velocity DOFs (refinement <= 5, about
 * 12.5 MB, held by every GPU that loads the library until the process exits).
 * It is for callers that cannot call cudaMalloc where they apply L (inside a
 * global-mode stream capture, real-time loops, capped external memory pools).
 * The paper has no counterpart: this is an interface convenience.
 * Solver: always the FP64 Jacobi CG on M1 to the context's mass-solve
 * tolerance, whatever the context's `solver` setting.  With PAVG_PRECISION_FP64
 * that tolerance is cg_rtol (1e-14 by default) and the result equals
 * pavg_linear's to about 1e-13; with PAVG_PRECISION_MIXED both solves stop at
 * a relative residual of 1e-5 and the two results agree to about that level.
 * Errors: INVAL for a null argument, a mesh larger than the limit or when the
 * context's device is not current; CUDA when the set-up lookup fails.  The
 * first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it for the life of the process; make that
 * first call before any stream capture.  The cached address dies with the
 * device's primary context: after cudaDeviceReset no pavg call may be made
 * (contexts must be destroyed before a reset in any case).
 * Every call shares the one array, so calls that overlap on the GPU race;
 * serialise them (one stream, or events).  As for the other state calls, a
 * device-side failure (iteration cap, non-finite value, a bounded wait that
 * gave up, or a failure latched by an earlier call on the context) is reported
 * by the next pavg_sync: LU is valid only once pavg_sync returns PAVG_OK. */
int pavg_linear_noalloc(pavg_ctx* ctx, const double* U, double* LU, void* stream);

/* The paper's error norms of a state U (device, n doubles; Sec. 3):
 * out[0] = ||u||_{L2} = sqrt(u^T M1 u), out[1] = ||u||_{H(div)} =
 * sqrt(||u||^2 + ||div u||^2) with div u the DG1 field M2^{-1} D u, and
 * out[2] = ||eta||_{L2} = sqrt(eta^T M2 eta) (host array of 3).  Runs on
 * `stream` and synchronises it. */
int pavg_norms(pavg_ctx* ctx, const double* U, double* out, void* stream);

/* Wait for the context's work on `stream` and report latched device errors. */
int pavg_sync(pavg_ctx* ctx, void* stream);

typedef struct {
  double lambda_max;      /* in use */
  int last_degree;        /* Chebyshev degree K of the last exponential / K_max of the last average */
  int cg_solves;          /* M1 solves since create (or the last reset) */
  int cg_iters_max;       /* largest iteration count of one solve */
  double cg_iters_mean;   /* mean CG iterations per solve (mixed solver: FP32 iterations, all sweeps) */
  int error_flags;        /* bit 0 NOCONV, bit 1 TIMEOUT, bit 2 NONFINITE */
  int kernel_launches;    /* kernels enqueued by the last API call (graph replays: kernels in the graph) */
  double cg_sweeps_mean;  /* FP64 refinement sweeps per solve (mixed solver; 0 for FP64 CG) */
  int solver_in_use;      /* PAVG_SOLVER_* of the context's M1 solves (SUBDOMAIN falls back to MIXED
                             where its parts do not fit in shared memory) */
} pavg_stats;

/* Synchronises the device, then fills *out. */
int pavg_get_stats(pavg_ctx* ctx, pavg_stats* out);

/* Clear the latched device error flags and the CG counters, and the subdomain
 * solver's exchange and synchronisation words (after a timed-out launch they
 * are inconsistent; the context is usable again once this returns). */
int pavg_reset_stats(pavg_ctx* ctx);

/* Test aid for the bounded waits of the subdomain solver (no counterpart in
 * the paper).  mode 1: block `part` leaves the next solves before it arrives
 * at their first grid-wide sum; mode 2: block `part` never publishes its
 * contributions to the triples it shares; mode 0: off.  wait_us bounds every
 * wait on another block (microseconds of the SM clock, at 2.07 GHz; 0 keeps
 * the default of about 2 s).  With a stall on, the other blocks' waits run
 * out, PAVG_ERR_TIMEOUT is latched and reported by pavg_sync; every block
 * leaves within a few wait bounds.  INVAL when the context does not use the
 * subdomain solver or `part` is not one of its blocks. */
int pavg_test_stall(pavg_ctx* ctx, int mode, int part, double wait_us);

/* Measurement aid: the current device's fused multiply-add rate in TFLOP/s
 * (fp64 != 0: FP64, else FP32), from a kernel of independent FMA chains on
 * every SM timed with CUDA events on `stream` (best of five launches after a
 * warm-up; synchronises; allocates a few KB).  The paper has no counterpart:
 * the benchmark uses it as the peak of ALU-bound kernels. */
int pavg_measure_fma_peak(int fp64, double* tflops, void* stream);

/* Measurement aid: when enabled, every M1 CG launch (the dominant kernel) is
 * bracketed by CUDA events on its stream, also inside captured graphs (plans
 * captured with the other setting are re-captured).  Off by default. */
int pavg_kernel_timing(pavg_ctx* ctx, int enable);

/* Sum of the bracketed CG durations of the most recent API call and their
 * count (host outputs; synchronises on the last event).  0 / 0 when timing
 * was off. */
int pavg_kernel_time(pavg_ctx* ctx, double* total_ms, int* launches);

/* Readable message of the last failure (static storage owned by the context). */
const char* pavg_last_error(const pavg_ctx* ctx);

/* ------------------------------------------------------------------------
 * Batches: many independent instances evaluated together.
 *
 * A batch groups n contexts (any refinements and parameters, each with the
 * mixed M1 solver, the default).  pavg_batch_averaged_rhs computes, for every
 * instance i, out_i = N-bar(U_i) with its own window T_i and shift count M_i
 * (Sec. 2.2, Eq. vt_discretised, evaluated as pavg_averaged_rhs does).  The
 * single-vector Chebyshev chains of all instances (Sec. 2.4) run in ONE
 * persistent cooperative launch, each instance on its own range of blocks
 * that synchronise only among themselves; likewise every instance's Clenshaw
 * sum.  The shift contractions and N run per instance between the two
 * launches.  Everything between the input and output copies is captured once
 * per (T_i, M_i) list in a CUDA graph and replayed.
 *
 * The grid of the persistent launches is chosen by an autotuner: threads per
 * block (128 or 256, i.e. 32 or 64 cells per block-pass), co-resident blocks
 * per SM, whether the FP32 element matrices stay in shared memory, and how
 * blocks are shared among instances.  It times each candidate on a few steps
 * of the real forward chains (per-instance device timers) and keeps the one
 * with the smallest predicted launch time.  Results of different
 * configurations differ only by rounding; a fixed configuration gives
 * bit-identical results on every call.
 *
 * A context may belong to one batch at a time and must not be used by other
 * calls while a batch call on it is in flight.  The contexts must outlive the
 * batch.  Per-instance errors are latched in each context (pavg_sync,
 * pavg_get_stats on the context); pavg_batch_sync reports the first.
 * ------------------------------------------------------------------------ */
typedef struct pavg_batch pavg_batch; /* opaque, library-owned */

typedef struct {
  int threads;        /* 128 or 256 */
  int blocks_per_sm;  /* co-resident blocks of the persistent launch per SM */
  int resident;       /* 1: FP32 element matrices in shared memory; 0: streamed from L2 */
  int weighting;      /* blocks per instance proportional to 0: cells x chain steps, 1: cells */
  double predicted_ms;/* autotuner's measured time of one evaluation of the batch (0 when set by hand) */
  int strategy;       /* 0: every instance's chains in persistent launches (the fields above);
                         1: one graph branch per instance, each evaluated with its own context's
                         solver, the branches running concurrently where the GPU has room */
} pavg_batch_config;

/* ctxs: host array of n distinct contexts on the current device, n >= 1.
 * The persistent chains run their own mass solves (FP32 conjugate gradients
 * refined by FP64 residuals, as PAVG_SOLVER_MIXED) whichever of the two
 * mixed solvers the contexts use.
 * Errors: INVAL (null, n < 1, a repeated context, a context with the FP64
 * solver or on another device), NOMEM. */
int pavg_batch_create(pavg_ctx* const* ctxs, int n, pavg_batch** out);
int pavg_batch_destroy(pavg_batch* b);

/* T, M: host arrays of n windows (seconds, >= 0) and shift counts (>= 1).
 * U, out: host arrays of n device pointers, instance i's state and result
 * (n_i doubles each, not aliasing).  Autotunes on the first call when no
 * configuration is set.  INVAL (pavg_batch_last_error says why) for a
 * null or aliasing pointer, a negative or
 * non-finite T_i, M_i < 1, or lambda_max_i T_i / 2 > PAVG_MAX_CHEB_ARG. */
int pavg_batch_averaged_rhs(pavg_batch* b, const double* T, const int* M, const double* const* U,
                            double* const* out, void* stream);

/* nsteps averaged Lawson RK4 steps (Sec. 2.3, Eqs. stage1_c to stage4) of
 * every instance, in place on U[i] (host array of device pointers), with its
 * own dt[i], T[i], M[i] (host arrays).  The four averaged right-hand sides of
 * a step run as batched evaluations; the six exponentials of a step run as
 * one persistent launch of all instances' Chebyshev chains each, followed by
 * a one-row contraction per instance.  Results equal pavg_timestep on each
 * context up to rounding.  INVAL for a null pointer, a non-finite dt_i, the
 * limits of pavg_batch_averaged_rhs, or lambda_max_i |dt_i| >
 * PAVG_MAX_CHEB_ARG. */
int pavg_batch_timestep(pavg_batch* b, const double* dt, const double* T, const int* M, double* const* U,
                        int nsteps, void* stream);

/* Runs the autotuner on these inputs (the work of one call's forward chains,
 * truncated to a few steps per candidate), keeps the best configuration and
 * returns it.  Synchronises `stream`. */
int pavg_batch_autotune(pavg_batch* b, const double* T, const int* M, const double* const* U, void* stream,
                        pavg_batch_config* best);
/* Sets or reads the configuration used by later calls (captured graphs of
 * another configuration are dropped).  Set: INVAL when the configuration
 * cannot be launched co-resident for some (T, M) list at call time, reported
 * then by pavg_batch_averaged_rhs. */
int pavg_batch_set_config(pavg_batch* b, const pavg_batch_config* cfg);
int pavg_batch_get_config(const pavg_batch* b, pavg_batch_config* cfg);

/* Durations of the two persistent launches of the last pavg_batch_averaged_rhs
 * (forward chains, Clenshaw sums), from events inside the graph; host
 * outputs, synchronises on the last event. */
int pavg_batch_kernel_time(pavg_batch* b, double* forward_ms, double* backward_ms);

/* Wait for the batch's work on `stream`; the first latched instance error. */
int pavg_batch_sync(pavg_batch* b, void* stream);

/* Readable message of the batch's last failure. */
const char* pavg_batch_last_error(const pavg_batch* b);

/* ------------------------------------------------------------------------
 * Learned surrogate of the large-M average.
 *
 * Wide windows T need many shifts M for the Riemann sum of Sec. 2.2 to
 * resolve the fast oscillations.  The surrogate keeps a cheap average with
 * few shifts, V = N-bar_Mc(U), and adds a learned correction towards the
 * large-M average:
 *   S(U) = V + scatter(sd_y * MLP((features(U, V) - mu_x) / sd_x) + mu_y).
 * features: per cell, its 15 local values (12 velocity coefficients times the
 * local-to-global signs of Sec. 2.5, 3 elevation values) of U and of V, the
 * same for the 3 cells across its edges (their own frames, local edge order),
 * and z_c / R, G00 / det, G01 / det, G11 / det of the cell: 124 FP32 inputs;
 * velocity values (moments of a flux) are divided by the row cell's length
 * scale sqrt(det), so that meshes of different refinement give rows of the
 * same size (targets likewise; outputs are multiplied back).
 * MLP: 124 -> hidden -> hidden -> 15, tanh hidden units, FP32 weights, in
 * flat order W1 [hidden][124], b1, W2 [hidden][hidden], b2, W3 [15][hidden], b3.
 * scatter: elevation and interior velocity values to their DOFs; an edge DOF
 * takes the mean of its two cells' values (times their signs).
 * Training: targets are the cell's 15 local values of N-bar_Mf(U) - V;
 * standardised mean squared error; Adam (beta1 0.9, beta2 0.999, eps 1e-8).
 * Every step (features, GEMMs, activations, loss, gradients, Adam, scatter)
 * runs in the library's kernels.  The Riemann sum with Mf shifts judges the
 * surrogate's error and replaces it above a threshold.
 *
 * A surrogate is independent of any mesh: its weights are trained on pairs
 * from one context and applied on any other (another refinement).  Scratch
 * for each context it is used with is allocated on first use.
 * ------------------------------------------------------------------------ */
typedef struct pavg_surrogate pavg_surrogate; /* opaque, library-owned */

/* hidden >= 1 units per layer; weights Glorot-uniform from `seed` (host
 * 64-bit Mersenne twister), biases zero, standardisation identity. */
int pavg_surrogate_create(int hidden, uint64_t seed, pavg_surrogate** out);
int pavg_surrogate_destroy(pavg_surrogate* s);
int pavg_surrogate_nparams(const pavg_surrogate* s, int64_t* n);
/* Host copies of the flat FP32 parameter vector (nparams floats). */
int pavg_surrogate_get_params(const pavg_surrogate* s, float* host);
int pavg_surrogate_set_params(pavg_surrogate* s, const float* host);
/* Host copies of the standardisation: mu_x, sd_x (124 each), mu_y, sd_y (15 each). */
int pavg_surrogate_get_scaling(const pavg_surrogate* s, float* mu_x, float* sd_x, float* mu_y, float* sd_y);
int pavg_surrogate_set_scaling(pavg_surrogate* s, const float* mu_x, const float* sd_x, const float* mu_y,
                               const float* sd_y);

/* Appends the F raw feature rows and raw target rows of n training pairs:
 * states U[i], cheap averages Vc[i], large-M averages Vf[i] (host arrays of
 * device pointers to n_ctx doubles each). */
int pavg_surrogate_add_pairs(pavg_surrogate* s, pavg_ctx* ctx, int n, const double* const* U,
                             const double* const* Vc, const double* const* Vf, void* stream);
/* Rows stored so far. */
int pavg_surrogate_rows(const pavg_surrogate* s, int64_t* rows);
/* Column means / standard deviations over the stored rows become the
 * standardisation; the stored rows are standardised in place.  Once. */
int pavg_surrogate_fit_scaling(pavg_surrogate* s, void* stream);
/* epochs passes of Adam over the stored rows in minibatches of `batch` rows
 * (a fresh permutation per epoch from `seed`), learning rate lr.
 * loss_per_epoch: host array of epochs doubles (mean standardised squared
 * error over each epoch's minibatches) or NULL.  Synchronises `stream`. */
int pavg_surrogate_train(pavg_surrogate* s, int epochs, int batch, double lr, uint64_t seed,
                         double* loss_per_epoch, void* stream);
/* Loss and gradient of the current parameters on rows X [B][124]
 * (standardised) against Z [B][15] (device FP32); grad: device, nparams
 * floats; *loss: host.  Synchronises `stream`. */
int pavg_surrogate_gradient(pavg_surrogate* s, const float* X, const float* Z, int B, float* grad, double* loss,
                            void* stream);
/* One Adam update of the parameters with the given gradient (device). */
int pavg_surrogate_adam_step(pavg_surrogate* s, const float* grad, double lr, void* stream);

/* Feature rows X [F][124] (device FP32) of state U and cheap average V on
 * the context's mesh; standardised with the surrogate's scaling when
 * `standardised` is set, raw otherwise. */
int pavg_surrogate_features(pavg_surrogate* s, pavg_ctx* ctx, const double* U, const double* V, float* X,
                            int standardised, void* stream);

/* out = V + correction for state U and its cheap average V (device, n doubles
 * each; out may not alias them).  bf16: the MLP's GEMMs on the tensor cores
 * with BF16 operands and FP32 accumulation. */
int pavg_surrogate_apply(pavg_surrogate* s, pavg_ctx* ctx, const double* U, const double* V, double* out, int bf16,
                         void* stream);
/* The surrogate form of N-bar(U) with its fallback: V = N-bar_Mc(U), out =
 * V + correction.  When check is set, also computes N-bar_Mf(U); if the
 * relative error of the surrogate in the energy norm (H u^T M1 u + g eta^T M2 eta)
 * exceeds threshold, out is replaced by N-bar_Mf(U) and *used_fallback = 1.
 * *rel_err: the measured error (-1 when check is 0).  Synchronises `stream`
 * when check is set. */
int pavg_surrogate_averaged_rhs(pavg_surrogate* s, pavg_ctx* ctx, double T, int Mc, int Mf, double threshold,
                                int check, int bf16, const double* U, double* out, int* used_fallback,
                                double* rel_err, void* stream);

const char* pavg_surrogate_last_error(const pavg_surrogate* s);

#ifdef __cplusplus
}
#endif

#endif /* PAVG_H */
