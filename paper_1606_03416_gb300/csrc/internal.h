// Internal launchers shared by the library's translation units (not part of the ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dg {

// Device view of the block-sparse H (block-CSR over elements, FP64 blocks).
struct HView {
  int32_t M;
  int64_t N;
  const int32_t* nb;       // [M]
  const int64_t* off;      // [M+1] natural row offsets
  const int64_t* row_ptr;  // [M+1]
  const int32_t* col;      // [nnzb]
  const int64_t* blk_off;  // [nnzb] offsets into vals (doubles)
  const double* vals;
  int32_t max_nb;
  int32_t tj = 64;  // FP64 filter: output columns per tile (64 if every n_K is a multiple of 64, else 32)
};

void count_launch(int n = 1);

// out = alpha * ((H - cI) in) - beta * prev   (prev may be null when beta == 0;
// out may alias prev, never in). in: (Ns x ld_in), prev/out: (Ns x ld_out),
// state-major FP64.
cudaError_t filter_step_f64(const HView& h, const double* in, int64_t ld_in, const double* prev, double* out,
                            int64_t ld_out, int64_t Ns, double alpha, double c, double beta, cudaStream_t s);

// The same step with c, alpha_k = coef[1 + 2 step], beta_k = coef[2 + 2 step]
// read from device memory (coef[0] = c), so a captured graph can be replayed
// with new filter bounds.
cudaError_t filter_step_f64_dev(const HView& h, const double* in, int64_t ld_in, const double* prev, double* out,
                                int64_t ld_out, int64_t Ns, const double* coef, int step, cudaStream_t s);

// Launches `blocks` x 256 threads, each running 8 independent chains of
// `iters` DFMAs (16 iters flops per thread); `sink` (device, one double) is
// written only in a case that does not occur.
cudaError_t dfma_rate(int64_t iters, int blocks, double* sink, cudaStream_t s);

// Loads the modules of the Lanczos kernels below (no launch), so that a later
// first launch allocates nothing (used when a context is created).
cudaError_t preload_lanczos_kernels();

// y = H x for one vector (Lanczos).
cudaError_t spmv_f64(const HView& h, const double* x, double* y, cudaStream_t s);

// out[l] = V_l . w for l < nv, V_l = V + l*ldv (deterministic block reductions).
cudaError_t dots_f64(const double* V, int64_t ldv, int nv, const double* w, int64_t n, double* out, cudaStream_t s);
// w -= sum_l coef[l] V_l   (coef on the device)
cudaError_t sub_combination_f64(double* w, const double* V, int64_t ldv, const double* coef, int nv, int64_t n, cudaStream_t s);
// y = a*x + b*y  (host scalars); if y_out != y, y_out = a*x + b*y
cudaError_t axpby_f64(double a, const double* x, double b, const double* y, double* y_out, int64_t n, cudaStream_t s);

// C[i,j] = sum_r A[i,r] B[j,r]  (A: rows x K, B: cols x K, row-major, K contiguous).
// lower_only: compute tiles with i-tile >= j-tile and mirror to the upper triangle
// (for a symmetric result, A == B).  symmetrise: C <- (C + C^T)/2 afterwards.
cudaError_t gemm_nt_f64(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                        int64_t rows, int64_t cols, int64_t K, bool lower_only, bool symmetrise, cudaStream_t s);

// C[i,r] = sum_l A[i,l] B[l,r]  (A: rows x K row-major, B: K x cols row-major).
// a_lower: A is lower triangular (entries l > i are treated as zero, not read).
cudaError_t gemm_nn_f64(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                        int64_t rows, int64_t cols, int64_t K, bool a_lower, cudaStream_t s);

// P_K = sum_i f_i X[i, off_K:] X[i, off_K:]^T packed at poff[K].
cudaError_t density_f64(const HView& h, const int64_t* poff, const double* X, int64_t Ns, int64_t ld,
                        const double* f, double* P, cudaStream_t s);

// Fermi level by bisection and occupations (one CTA).
cudaError_t occupations_f64(const double* ritz, int64_t Ns, double Ne, double kT, double* f, double* mu,
                            cudaStream_t s);

// G_e += alpha * sum_s w_s A[s, off_K + j] B[s, off_K' + j'] for every stored block e = (K, K')
// (values layout of H; w may be null).
cudaError_t block_outer_f64(const HView& h, const int32_t* blk_row, int64_t nnzb, const double* A, int64_t lda,
                            const double* B, int64_t ldb, const double* w, double alpha, int64_t Ns, double* G,
                            cudaStream_t s);
// C[i,r] = sum_l A[l,i] B[l,r]  (A: K x rows row-major, B: K x cols row-major).
cudaError_t gemm_tn_f64(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                        int64_t rows, int64_t cols, int64_t K, cudaStream_t s);
// out[i, r] = scale * g[i] * (HX[i, r] - lam[i] X[i, r]) for r < n.
cudaError_t scaled_residual_f64(const double* HX, const double* X, int64_t ld, const double* lam, const double* g,
                                double scale, int64_t Ns, int64_t n, double* out, int64_t ldo, cudaStream_t s);

// A[i,i] += coef * trace(A) for a row-major n x n matrix (one CTA, fixed
// summation order).
cudaError_t shift_diagonal_by_trace_f64(double* A, int64_t n, double coef, cudaStream_t s);
// Zero the strict upper triangle of a row-major n x n matrix.
cudaError_t zero_strict_upper_f64(double* A, int64_t n, int64_t lda, cudaStream_t s);
// flag[0] |= 1 if any of x[0..n) is not finite.
cudaError_t check_finite_f64(const double* x, int64_t n, int* flag, cudaStream_t s);

}  // namespace dg
