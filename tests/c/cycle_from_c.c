/* One CheFSI cycle driven from plain C through include/dgchefsi.h: device
 * memory from the CUDA runtime, every step a library call (Alg. 1 steps 1-5,
 * occupations, diagonal density blocks). Reads the problem from a binary file
 * written by tests/test_c_abi.py and prints the Ritz values, mu and sum_K tr P.
 *
 * File layout (native endianness): int64 M, nnzb, n_values, N, Ns, m;
 * int32 nb[M]; int64 row_ptr[M+1]; int32 col[nnzb]; int64 blk_off[nnzb];
 * double values[n_values]; double X[Ns*N] (state-major); double v0[N];
 * double Ne, kT. */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "dgchefsi.h"

#define CHECK_ST(call)                                                               \
  do {                                                                               \
    dgchefsi_status st_ = (call);                                                    \
    if (st_ != DGCHEFSI_OK) {                                                        \
      fprintf(stderr, "%s failed (%d): %s\n", #call, (int)st_, dgchefsi_last_error()); \
      return 1;                                                                      \
    }                                                                                \
  } while (0)
#define CHECK_CUDA(call)                                                             \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      fprintf(stderr, "%s failed: %s\n", #call, cudaGetErrorString(e_));             \
      return 1;                                                                      \
    }                                                                                \
  } while (0)

static void* read_n(FILE* fh, size_t bytes) {
  void* p = malloc(bytes ? bytes : 1);
  if (p && bytes && fread(p, 1, bytes, fh) != bytes) {
    free(p);
    return NULL;
  }
  return p;
}

int main(int argc, char** argv) {
  if (argc != 2) {
    fprintf(stderr, "usage: %s problem.bin\n", argv[0]);
    return 2;
  }
  FILE* fh = fopen(argv[1], "rb");
  if (!fh) return 2;
  int64_t hdr[6];
  if (fread(hdr, sizeof(int64_t), 6, fh) != 6) return 2;
  const int64_t M = hdr[0], nnzb = hdr[1], nv = hdr[2], N = hdr[3], Ns = hdr[4];
  const int m = (int)hdr[5];
  int32_t* nb = read_n(fh, sizeof(int32_t) * M);
  int64_t* row_ptr = read_n(fh, sizeof(int64_t) * (M + 1));
  int32_t* col = read_n(fh, sizeof(int32_t) * nnzb);
  int64_t* blk_off = read_n(fh, sizeof(int64_t) * nnzb);
  double* values = read_n(fh, sizeof(double) * nv);
  double* X = read_n(fh, sizeof(double) * Ns * N);
  double* v0 = read_n(fh, sizeof(double) * N);
  double sc[2];
  if (!nb || !row_ptr || !col || !blk_off || !values || !X || !v0 || fread(sc, sizeof(double), 2, fh) != 2) return 2;
  fclose(fh);

  dgchefsi_ctx* ctx = NULL;
  CHECK_ST(dgchefsi_create((int32_t)M, nb, row_ptr, col, blk_off, values, nv, NULL, &ctx));
  double *dX, *dY, *dv, *dritz, *df, *dmu, *dP;
  int64_t np = 0;
  for (int64_t K = 0; K < M; ++K) np += (int64_t)nb[K] * nb[K];
  CHECK_CUDA(cudaMalloc((void**)&dX, sizeof(double) * Ns * N));
  CHECK_CUDA(cudaMalloc((void**)&dY, sizeof(double) * Ns * N));
  CHECK_CUDA(cudaMalloc((void**)&dv, sizeof(double) * N));
  CHECK_CUDA(cudaMalloc((void**)&dritz, sizeof(double) * Ns));
  CHECK_CUDA(cudaMalloc((void**)&df, sizeof(double) * Ns));
  CHECK_CUDA(cudaMalloc((void**)&dmu, sizeof(double)));
  CHECK_CUDA(cudaMalloc((void**)&dP, sizeof(double) * np));
  CHECK_CUDA(cudaMemcpy(dX, X, sizeof(double) * Ns * N, cudaMemcpyHostToDevice));
  CHECK_CUDA(cudaMemcpy(dv, v0, sizeof(double) * N, cudaMemcpyHostToDevice));

  double b = 0.0, tmin = 0.0;
  CHECK_ST(dgchefsi_bounds(ctx, dv, 10, &b, &tmin));            /* step 1 */
  const double a0 = tmin, a = tmin + (b - tmin) * (double)Ns / (double)N;
  CHECK_ST(dgchefsi_filter(ctx, DGCHEFSI_F64, dX, dY, Ns, N, m, a, b, a0));   /* step 2 */
  CHECK_ST(dgchefsi_rayleigh_ritz(ctx, dY, Ns, N, dritz));       /* steps 3-5 */
  CHECK_ST(dgchefsi_occupations(ctx, dritz, Ns, sc[0], sc[1], df, dmu));
  CHECK_ST(dgchefsi_density_blocks(ctx, dY, Ns, N, df, dP));
  CHECK_CUDA(cudaDeviceSynchronize());

  double* ritz = malloc(sizeof(double) * Ns);
  double* P = malloc(sizeof(double) * np);
  double mu = 0.0;
  if (!ritz || !P) return 2;
  CHECK_CUDA(cudaMemcpy(ritz, dritz, sizeof(double) * Ns, cudaMemcpyDeviceToHost));
  CHECK_CUDA(cudaMemcpy(&mu, dmu, sizeof(double), cudaMemcpyDeviceToHost));
  CHECK_CUDA(cudaMemcpy(P, dP, sizeof(double) * np, cudaMemcpyDeviceToHost));
  double tr = 0.0;
  int64_t o = 0;
  for (int64_t K = 0; K < M; ++K) {
    for (int32_t j = 0; j < nb[K]; ++j) tr += P[o + (int64_t)j * nb[K] + j];
    o += (int64_t)nb[K] * nb[K];
  }
  printf("BOUNDS %.17g %.17g %.17g\n", a, b, a0);
  printf("RITZ");
  for (int64_t i = 0; i < Ns; ++i) printf(" %.17g", ritz[i]);
  printf("\nMU %.17g\nTRACE_P %.17g\n", mu, tr);
  dgchefsi_destroy(ctx);
  cudaFree(dX); cudaFree(dY); cudaFree(dv); cudaFree(dritz); cudaFree(df); cudaFree(dmu); cudaFree(dP);
  free(nb); free(row_ptr); free(col); free(blk_off); free(values); free(X); free(v0); free(ritz); free(P);
  return 0;
}
