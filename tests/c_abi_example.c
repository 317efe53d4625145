/* A C program on the library's C-ABI alone (include/pavg.h, libpavg.so):
 * refinement 2, one averaged right-hand side and one time step of a state
 * that is at rest (u = 0, eta = const): N(rest) = 0, so N-bar(rest) = 0, and
 * the step returns the state up to the truncation of the Chebyshev series
 * (its value at L = 0 is 1 to within cheb_tol = 1e-6 per exponential).
 * Exit status 0 when every call succeeds and both checks hold. */
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "pavg.h"

#define CHECK(call)                                                          \
  do {                                                                       \
    int rc_ = (call);                                                        \
    if (rc_ != PAVG_OK) {                                                    \
      fprintf(stderr, "%s failed: %d (%s)\n", #call, rc_, pavg_last_error(ctx)); \
      return 1;                                                              \
    }                                                                        \
  } while (0)

int main(void) {
  pavg_params p;
  pavg_ctx* ctx = NULL;
  if (pavg_default_params(&p) != PAVG_OK) return 1;
  p.refinement = 2;
  p.lambda_max = 0.00142;
  CHECK(pavg_create(&p, &ctx));
  int64_t n_u = 0, n_eta = 0;
  CHECK(pavg_sizes(ctx, &n_u, &n_eta, NULL, NULL, NULL));
  const int64_t n = n_u + n_eta;
  double* h = (double*)calloc((size_t)n, sizeof(double));
  for (int64_t i = n_u; i < n; ++i) h[i] = 3.0;  /* eta = 3 m everywhere, u = 0 */
  double *U = NULL, *S = NULL;
  if (cudaMalloc((void**)&U, sizeof(double) * n) != cudaSuccess ||
      cudaMalloc((void**)&S, sizeof(double) * n) != cudaSuccess)
    return 1;
  cudaMemcpy(U, h, sizeof(double) * n, cudaMemcpyHostToDevice);
  CHECK(pavg_averaged_rhs(ctx, 3600.0, 8, U, S, NULL));
  CHECK(pavg_timestep(ctx, 900.0, 3600.0, 8, U, 1, NULL));
  CHECK(pavg_sync(ctx, NULL));
  double* s = (double*)malloc(sizeof(double) * n);
  cudaMemcpy(s, S, sizeof(double) * n, cudaMemcpyDeviceToHost);
  double smax = 0.0, dmax = 0.0;
  for (int64_t i = 0; i < n; ++i) smax = fmax(smax, fabs(s[i]));
  cudaMemcpy(s, U, sizeof(double) * n, cudaMemcpyDeviceToHost);
  for (int64_t i = 0; i < n; ++i) dmax = fmax(dmax, fabs(s[i] - h[i]));
  printf("rest state: |N-bar| max %.3e, |step - U| max %.3e\n", smax, dmax);
  cudaFree(U);
  cudaFree(S);
  free(h);
  free(s);
  CHECK(pavg_destroy(ctx));
  ctx = NULL;
  return (smax < 1e-12 && dmax < 3e-5) ? 0 : 2;  /* 1e-5 of the 3 m elevation */
}
