// Cholesky factor of the Gram matrix and its inverse from dense products
// (Alg. 1 step 3: S = U^T U, Y_hat = Y U^{-1}). The paper names the Cholesky
// factorisation, next to the eigensolve, as the part of the subspace problem
// to move onto dense matrix products (Conclusion); here it is a recursive
// blocked factorisation whose work is four products per level.
//
// Row-major lower view: S = L L^T with L = U^T lower, and what the step needs
// is L^{-1} = U^{-T} (Y_hat^T = L^{-1} Y^T). For the leading block split
// S = [S11, .; S21, S22] (n1 + n2 rows):
//   L11, L11^{-1}  from the block S11 (recursively),
//   L21 = S21 L11^{-T},
//   S22 <- S22 - L21 L21^T          (lower triangle only),
//   L22, L22^{-1}  from the updated S22 (recursively),
//   (L^{-1})21 = -L22^{-1} (L21 L11^{-1}),
// (Golub and Van Loan, Matrix Computations, 4th ed., Sec. 4.2 for the block
// Cholesky; the block form of the triangular inverse is the one of Sec. 3.1).
// Blocks of at most 64 rows are factored and inverted in shared memory by
// one CTA (the unblocked outer-product Cholesky and forward substitution of
// the unit vectors). Products with every side at least 512 run from exact
// BF16 slices on the tensor cores (sliced.cu), smaller ones on the FP64 cores.
// S is first equilibrated by powers of two (see k_equilibrate).
#include <algorithm>
#include <cmath>

#include "ctx.h"

namespace dg {

namespace {

constexpr int kLeaf = 64;        // rows of a block factored by one CTA
constexpr int64_t kSliced = 512;  // smallest product side run from slices

// One CTA factors the n x n block (n <= 64) whose lower triangle is at A
// (lda): L (lower) replaces it, the strict upper part is left as it was, and
// Li (ldl) receives L^{-1} with its strict upper part zeroed. A pivot that is
// not positive and finite stops the block: *info = col0 + j + 1 (1-based
// column of the whole matrix) if *info was 0.
__global__ void __launch_bounds__(256) k_chol_leaf(double* __restrict__ A, int64_t lda, double* __restrict__ Li,
                                                   int64_t ldl, int n, int64_t col0, int* __restrict__ info) {
  __shared__ double M[kLeaf][kLeaf + 1];
  __shared__ int bad;
  const int t = threadIdx.x;
  if (t == 0) bad = 0;
  for (int e = t; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    M[i][j] = j <= i ? A[(int64_t)i * lda + j] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (t == 0) {
      const double d = M[j][j];
      if (!(d > 0.0) || !isfinite(d)) {
        bad = 1;
        atomicCAS(info, 0, (int)(col0 + j + 1));
      } else {
        M[j][j] = sqrt(d);
      }
    }
    __syncthreads();
    if (bad) break;
    const double ljj = M[j][j];
    for (int i = j + 1 + t; i < n; i += blockDim.x) M[i][j] /= ljj;
    __syncthreads();
    // trailing update of the lower triangle: M[i][k] -= M[i][j] M[k][j], j < k <= i
    const int m = n - j - 1;
    for (int e = t; e < m * m; e += blockDim.x) {
      const int i = j + 1 + e / m, k = j + 1 + e % m;
      if (k <= i) M[i][k] -= M[i][j] * M[k][j];
    }
    __syncthreads();
  }
  if (bad) return;
  for (int e = t; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    if (j <= i) A[(int64_t)i * lda + j] = M[i][j];
  }
  // column c of L^{-1}: forward substitution of e_c (entries above c are zero)
  for (int c = t; c < n; c += blockDim.x) {
    double x[kLeaf];
    for (int i = 0; i < c; ++i) Li[(int64_t)i * ldl + c] = 0.0;
    for (int i = c; i < n; ++i) {
      double acc = i == c ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) acc -= M[i][k] * x[k];
      x[i] = acc / M[i][i];
      Li[(int64_t)i * ldl + c] = x[i];
    }
  }
}

// Y = alpha X + beta Y on rows x cols (row strides ldx, ldy); lower: only the
// entries c <= r.
__global__ void k_axpby_2d(double alpha, const double* __restrict__ X, int64_t ldx, double beta, double* Y,
                           int64_t ldy, int64_t rows, int64_t cols, int lower) {
  const int64_t tot = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    if (lower && c > r) continue;
    double* y = Y + r * ldy + c;
    *y = beta == 0.0 ? alpha * X[r * ldx + c] : alpha * X[r * ldx + c] + beta * *y;
  }
}

// Exact equilibration: d_i = 2^{-round(log2(S_ii) / 2)} (1 for a diagonal
// entry that is not positive and finite, which the factorisation then
// rejects), and the lower triangle of S scaled to d_i S_ij d_j, whose
// diagonal lies in [1/2, 2]. Powers of two change no bits, and the factor of
// the scaled matrix is D L, so L^{-1} = (D L)^{-1} D. The slices of a product
// share one exponent per row, so without this a matrix whose diagonal spans
// many orders keeps fewer significant bits in the rows' smaller entries.
__global__ void k_equilibrate(double* __restrict__ S, int64_t lda, int64_t n, double* __restrict__ d) {
  for (int64_t i = blockIdx.y; i < n; i += gridDim.y) {
    const double sii = S[i * lda + i];
    const double di = (sii > 0.0 && isfinite(sii)) ? ldexp(1.0, -(int)rint(0.5 * log2(sii))) : 1.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= i; j += (int64_t)gridDim.x * blockDim.x) {
      const double sjj = S[j * lda + j];
      const double dj = (sjj > 0.0 && isfinite(sjj)) ? ldexp(1.0, -(int)rint(0.5 * log2(sjj))) : 1.0;
      if (j != i) S[i * lda + j] *= di * dj;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) d[i] = di;
  }
}

// The diagonal after the rows' off-diagonal entries (those read the old diagonal).
__global__ void k_equilibrate_diag(double* __restrict__ S, int64_t lda, int64_t n, const double* __restrict__ d) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    S[i * lda + i] *= d[i] * d[i];
}

// S[i, j] = Li[i, j] d_j on the lower triangle (L^{-1} = (D L)^{-1} D).
__global__ void k_unscale_inverse(const double* __restrict__ Li, int64_t n, const double* __restrict__ d,
                                  double* __restrict__ S, int64_t lda) {
  const int64_t tot = n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    if (j <= i) S[i * lda + j] = Li[e] * d[j];
  }
}

unsigned grid_2d(int64_t tot) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((tot + 255) / 256, 152 * 16)); }

struct Chol {
  dgchefsi_ctx* ctx;
  double* A;     // the matrix (lower triangle), L on return
  int64_t lda;
  double* Li;    // L^{-1}, n x n, row stride n (strict upper zero)
  double* T;     // scratch, n x n, row stride n
  double* T2;    // scratch, n x n, row stride n
  int64_t n;
  int* info;     // device
  int* bad;      // device non-finite flag of the sliced products
  int slices;
  cudaStream_t st;

  // C (rows x cols, ldc) = X Z^T with X rows x K (ldx), Z cols x K (ldz);
  // tri: only the lower triangle (rows == cols).
  dgchefsi_status prod_nt(const double* X, int64_t ldx, const double* Z, int64_t ldz, double* C, int64_t ldc,
                          int64_t rows, int64_t cols, int64_t K, bool tri) {
    if (std::min(std::min(rows, cols), K) >= kSliced)
      return sliced_gemm(ctx, true, false, rows, cols, K, X, ldx, Z, ldz, C, ldc, slices, bad, tri ? rows : 0);
    DG_CUDA(gemm_nt_f64(X, ldx, Z, ldz, C, ldc, rows, cols, K, tri, false, st));
    return DGCHEFSI_OK;
  }
  // C = X Z with X rows x K (x_lower: lower triangular), Z K x cols.
  dgchefsi_status prod_nn(const double* X, int64_t ldx, const double* Z, int64_t ldz, double* C, int64_t ldc,
                          int64_t rows, int64_t cols, int64_t K, bool x_lower) {
    if (std::min(std::min(rows, cols), K) >= kSliced)
      return sliced_gemm(ctx, false, x_lower, rows, cols, K, X, ldx, Z, ldz, C, ldc, slices, bad);
    DG_CUDA(gemm_nn_f64(X, ldx, Z, ldz, C, ldc, rows, cols, K, x_lower, st));
    return DGCHEFSI_OK;
  }
  dgchefsi_status axpby(double alpha, const double* X, int64_t ldx, double beta, double* Y, int64_t ldy,
                        int64_t rows, int64_t cols, bool lower) {
    k_axpby_2d<<<grid_2d(rows * cols), 256, 0, st>>>(alpha, X, ldx, beta, Y, ldy, rows, cols, lower ? 1 : 0);
    count_launch();
    DG_CUDA(cudaGetLastError());
    return DGCHEFSI_OK;
  }

  // The diagonal block at (i0, i0) of m rows, its Schur complement applied.
  dgchefsi_status block(int64_t i0, int64_t m) {
    double* a = A + i0 * lda + i0;
    double* li = Li + i0 * n + i0;
    if (m <= kLeaf) {
      k_chol_leaf<<<1, 256, 0, st>>>(a, lda, li, n, (int)m, i0, info);
      count_launch();
      DG_CUDA(cudaGetLastError());
      return DGCHEFSI_OK;
    }
    // split on a multiple of the leaf (of 256 once blocks are large), near the middle
    const int64_t q = m >= 1024 ? 256 : kLeaf;
    const int64_t m1 = std::max<int64_t>(q, (m / 2 + q / 2) / q * q);
    const int64_t m2 = m - m1;
    DG_TRY(block(i0, m1));
    double* a21 = a + m1 * lda;
    double* a22 = a21 + m1;
    double* li11 = li;
    double* li21 = li + m1 * n;
    double* li22 = li21 + m1;
    // L21 = S21 L11^{-T}
    DG_TRY(prod_nt(a21, lda, li11, n, T, n, m2, m1, m1, false));
    DG_TRY(axpby(1.0, T, n, 0.0, a21, lda, m2, m1, false));
    // S22 <- S22 - L21 L21^T (lower)
    DG_TRY(prod_nt(a21, lda, a21, lda, T2, n, m2, m2, m1, true));
    DG_TRY(axpby(-1.0, T2, n, 1.0, a22, lda, m2, m2, true));
    DG_TRY(block(i0 + m1, m2));
    // (L^{-1})21 = -L22^{-1} (L21 L11^{-1})
    DG_TRY(prod_nn(a21, lda, li11, n, T, n, m2, m1, m1, false));
    DG_TRY(prod_nn(li22, n, T, n, T2, n, m2, m1, m2, true));
    DG_TRY(axpby(-1.0, T2, n, 0.0, li21, n, m2, m1, false));
    return DGCHEFSI_OK;
  }
};

}  // namespace

dgchefsi_status cholesky_inverse(dgchefsi_ctx* ctx, double* S, int64_t n, int64_t lda, int* info, int* bad) {
  if (n <= 0) return DGCHEFSI_OK;
  const size_t nn = (size_t)n * (size_t)n;
  DG_TRY(ensure(ctx, ctx->ws_chol, sizeof(double) * (3 * nn + (size_t)n), "Cholesky workspace"));
  double* Li = static_cast<double*>(ctx->ws_chol.p);
  double* d = Li + 3 * nn;
  Chol c{ctx, S, lda, Li, Li + nn, Li + 2 * nn, n, info, bad, std::max(ctx->products_slices, 10), ctx->stream};
  DG_CUDA(cudaMemsetAsync(Li, 0, sizeof(double) * nn, c.st));
  k_equilibrate<<<dim3((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)std::min<int64_t>(n, 65535)), 256,
                  0, c.st>>>(S, lda, n, d);
  k_equilibrate_diag<<<grid_2d(n), 256, 0, c.st>>>(S, lda, n, d);
  count_launch(2);
  DG_CUDA(cudaGetLastError());
  DG_TRY(c.block(0, n));
  // L^{-1} into the lower triangle of S (its strict upper part is left unspecified)
  k_unscale_inverse<<<grid_2d((int64_t)nn), 256, 0, c.st>>>(Li, n, d, S, lda);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return DGCHEFSI_OK;
}

}  // namespace dg
