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
// Blocks of at most 64 rows are factored and inverted by one CTA (the
// unblocked outer-product Cholesky, then Gauss-Jordan elimination of the
// identity, with the block's entries held in registers). Products with every
// side at least 512 run from exact BF16 slices on the tensor cores
// (sliced.cu), smaller ones on the FP64 cores as split-K tiles over the whole GPU.
// S is first equilibrated by powers of two (see k_equilibrate).
#include <algorithm>
#include <cmath>

#include "ctx.h"

namespace dg {

namespace {

// rows of a block factored by one CTA. A leaf runs on one SM, which does two
// FP64 multiply-adds per clock, and its ~2 kLeaf^3 / 3 of them are serial
// across the leaves: 64 keeps that near 3 ms at n = 4096 (128 took 4 ms per
// leaf; 32 gave the same Rayleigh-Ritz time as 64, the extra level of small
// products taking what the smaller leaves save), the levels above run over
// the whole GPU
constexpr int kLeaf = 64;
constexpr int64_t kSliced = 512;  // smallest product side run from slices
constexpr int kLeafThreads = 256;
constexpr int64_t kPartial = int64_t(1) << 20;  // doubles of partial tiles for the split-K products
constexpr int kOwn = (kLeaf * (kLeaf + 1) / 2 + kLeafThreads - 1) / kLeafThreads;  // entries per thread

// One CTA factors the n x n block (n <= 64) whose lower triangle is at A
// (lda): L (lower) replaces it, the strict upper part is left as it was, and
// Li (ldl) receives L^{-1} with its strict upper part zeroed.
// Factorisation: each thread owns up to kOwn entries of the lower triangle in
// registers, numbered by column from the last one (entry e of column k, row
// i, is e = (n-1-k)(n-k)/2 + i - k; thread e mod 256 owns it), so the
// entries a step updates (columns after j) are a prefix of the numbering and
// fill whole warps; one FP64 warp instruction occupies the SM's FP64 pipe for
// many clocks, so half-empty warps cost as much as full ones. Step j
// publishes column j, the pivot's owner also its root and reciprocals, and
// every owner of (i, k), j < k <= i, subtracts M_ij M_kj / M_jj; column j is
// then divided by sqrt(M_jj).
// Inverse: L goes to shared memory, and W = L^{-1} follows by Gauss-Jordan
// elimination of I with the entries of W owned by rows (e = i(i+1)/2 + k): step
// j publishes row j of W, row j is divided by L_jj, rows i > j lose L_ij times
// it. The shared rows and columns alternate between two buffers, so each step
// needs one barrier. A pivot that is not positive and finite stops the block:
// *info = col0 + j + 1 (1-based column of the whole matrix) if *info was 0.
__global__ void __launch_bounds__(kLeafThreads, 1) k_chol_leaf(double* __restrict__ A, int64_t lda,
                                                              double* __restrict__ Li, int64_t ldl, int n,
                                                              int64_t col0, int* __restrict__ info) {
  __shared__ double col[2][kLeaf], row[2][kLeaf], rd[kLeaf];
  __shared__ double Ls[kLeaf][kLeaf + 1];
  __shared__ double sc[2][4];  // the pivot, its square root and their reciprocals (one thread computes them)
  const int t = threadIdx.x;
  const int tot = n * (n + 1) / 2;
  double v[kOwn];
  int rc[kOwn];  // (row << 8) | column of the entry, -1 for none
#pragma unroll
  for (int q = 0; q < kOwn; ++q) {
    const int e = t + kLeafThreads * q;
    int m = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);  // columns after this one: m = n - 1 - k
    while ((m + 1) * (m + 2) / 2 <= e) ++m;
    while (m * (m + 1) / 2 > e) --m;
    const int k = n - 1 - m, i = k + (e - m * (m + 1) / 2);
    const bool ok = e < tot;
    rc[q] = ok ? (i << 8) | k : -1;
    v[q] = ok ? A[(int64_t)i * lda + k] : 0.0;
  }
  for (int j = 0; j < n; ++j) {
    const int b = j & 1;
#pragma unroll
    for (int q = 0; q < kOwn; ++q)
      if (rc[q] >= 0 && (rc[q] & 255) == j) {
        col[b][rc[q] >> 8] = v[q];
        if ((rc[q] >> 8) == j) {  // the pivot's owner
          const double pv = v[q], sq = sqrt(pv);
          sc[b][0] = pv;
          sc[b][1] = sq;
          sc[b][2] = 1.0 / sq;
          sc[b][3] = 1.0 / pv;
        }
      }
    __syncthreads();
    const double p = sc[b][0];
    if (!(p > 0.0) || !isfinite(p)) {  // the same value in every thread: all leave together
      if (t == 0) atomicCAS(info, 0, (int)(col0 + j + 1));
      return;
    }
    const double ljj = sc[b][1], rl = sc[b][2], rp = sc[b][3];
#pragma unroll
    for (int q = 0; q < kOwn; ++q) {
      if (rc[q] < 0) continue;
      const int i = rc[q] >> 8, k = rc[q] & 255;
      if (k == j)
        v[q] = i == j ? ljj : v[q] * rl;
      else if (k > j)
        v[q] -= col[b][i] * (col[b][k] * rp);
    }
  }
  // L to A and to shared memory; the reciprocals of its diagonal
#pragma unroll
  for (int q = 0; q < kOwn; ++q) {
    if (rc[q] < 0) continue;
    const int i = rc[q] >> 8, k = rc[q] & 255;
    A[(int64_t)i * lda + k] = v[q];
    Ls[i][k] = v[q];
  }
  __syncthreads();
  if (t < n) rd[t] = 1.0 / Ls[t][t];
  // W by rows: entry e = i(i+1)/2 + k
  double w[kOwn];
#pragma unroll
  for (int q = 0; q < kOwn; ++q) {
    const int e = t + kLeafThreads * q;
    int i = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
    while ((i + 1) * (i + 2) / 2 <= e) ++i;
    while (i * (i + 1) / 2 > e) --i;
    const int k = e - i * (i + 1) / 2;
    const bool ok = e < tot;
    rc[q] = ok ? (i << 8) | k : -1;
    w[q] = (ok && i == k) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const int b = j & 1;
#pragma unroll
    for (int q = 0; q < kOwn; ++q)
      if (rc[q] >= 0 && (rc[q] >> 8) == j) row[b][rc[q] & 255] = w[q];  // row j of W, before its division
    __syncthreads();
    const double rl = rd[j];
#pragma unroll
    for (int q = 0; q < kOwn; ++q) {
      if (rc[q] < 0) continue;
      const int i = rc[q] >> 8, k = rc[q] & 255;
      if (i == j)
        w[q] *= rl;
      else if (i > j && k <= j)
        w[q] -= Ls[i][j] * (row[b][k] * rl);
    }
  }
#pragma unroll
  for (int q = 0; q < kOwn; ++q) {
    if (rc[q] < 0) continue;
    Li[(int64_t)(rc[q] >> 8) * ldl + (rc[q] & 255)] = w[q];
  }
  for (int e = t; e < n * n; e += kLeafThreads) {
    const int i = e / n, k = e % n;
    if (k > i) Li[(int64_t)i * ldl + k] = 0.0;
  }
}

// Small FP64 products on the CUDA cores, spread over the whole GPU: 32 x 32
// output tiles, the K range split into `splits` parts (one CTA per tile and
// part) whose partial tiles go to P, then summed in a fixed order
// (deterministic). C = X op(Z): op(Z)[k, c] = Z[c, k] (zt, the X Z^T form)
// or Z[k, c]; x_lower: X[r, k] = 0 for k > r. One SM does two FP64 FMAs per
// clock, so a product of a few million multiply-adds needs many CTAs.
template <bool ZT, bool XLOWER>
__global__ void __launch_bounds__(256) k_small_gemm_part(const double* __restrict__ X, int64_t ldx,
                                                         const double* __restrict__ Z, int64_t ldz,
                                                         double* __restrict__ P, int64_t rows, int64_t cols,
                                                         int64_t K, int64_t kc) {
  __shared__ double Xs[32][33], Zs[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  const int64_t k0 = (int64_t)blockIdx.z * kc, k1 = K < k0 + kc ? K : k0 + kc;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t kk = k0; kk < k1; kk += 32) {
    for (int u = ty; u < 32; u += 8) {
      const int64_t r = r0 + u, k = kk + tx;
      Xs[u][tx] = (r < rows && k < k1 && (!XLOWER || k <= r)) ? X[r * ldx + k] : 0.0;
      const int64_t kz = kk + u, c = c0 + tx;
      Zs[u][tx] = (kz < k1 && c < cols) ? (ZT ? Z[c * ldz + kz] : Z[kz * ldz + c]) : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int i = 0; i < 32; ++i) {
      const double z = Zs[i][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] += Xs[ty + 8 * u][i] * z;
    }
    __syncthreads();
  }
  double* Pp = P + (int64_t)blockIdx.z * rows * cols;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t r = r0 + ty + 8 * u, c = c0 + tx;
    if (r < rows && c < cols) Pp[r * cols + c] = acc[u];
  }
}

// C[r, c] = sum_s P[s, r, c] in the order s = 0, 1, ...; tri: only c <= r.
__global__ void k_small_gemm_sum(const double* __restrict__ P, int splits, int64_t rows, int64_t cols,
                                 double* __restrict__ C, int64_t ldc, int tri) {
  const int64_t tot = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    if (tri && c > r) continue;
    double sum = 0.0;
    for (int sp = 0; sp < splits; ++sp) sum += P[(int64_t)sp * tot + e];
    C[r * ldc + c] = sum;
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
  double* P;     // partial tiles of the small products (kPartial doubles)
  int64_t n;
  int* info;     // device
  int* bad;      // device non-finite flag of the sliced products
  int slices;
  cudaStream_t st;

  // Split-K FP64 product on the CUDA cores for the small levels.
  template <bool ZT, bool XLOWER>
  dgchefsi_status small(const double* X, int64_t ldx, const double* Z, int64_t ldz, double* C, int64_t ldc,
                        int64_t rows, int64_t cols, int64_t K, bool tri) {
    const int64_t tiles = ((rows + 31) / 32) * ((cols + 31) / 32);
    int64_t splits = std::max<int64_t>(1, std::min<int64_t>((2 * 152 + tiles - 1) / tiles, (K + 31) / 32));
    splits = std::max<int64_t>(1, std::min<int64_t>(splits, kPartial / (rows * cols)));
    const int64_t kc = ((K + splits - 1) / splits + 31) / 32 * 32;
    splits = (K + kc - 1) / kc;
    k_small_gemm_part<ZT, XLOWER><<<dim3((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32), (unsigned)splits),
                                     256, 0, st>>>(X, ldx, Z, ldz, P, rows, cols, K, kc);
    k_small_gemm_sum<<<grid_2d(rows * cols), 256, 0, st>>>(P, (int)splits, rows, cols, C, ldc, tri ? 1 : 0);
    count_launch(2);
    DG_CUDA(cudaGetLastError());
    return DGCHEFSI_OK;
  }
  // C (rows x cols, ldc) = X Z^T with X rows x K (ldx), Z cols x K (ldz);
  // tri: only the lower triangle (rows == cols).
  dgchefsi_status prod_nt(const double* X, int64_t ldx, const double* Z, int64_t ldz, double* C, int64_t ldc,
                          int64_t rows, int64_t cols, int64_t K, bool tri) {
    if (std::min(std::min(rows, cols), K) >= kSliced)
      return sliced_gemm(ctx, true, false, rows, cols, K, X, ldx, Z, ldz, C, ldc, slices, bad, tri ? rows : 0);
    return small<true, false>(X, ldx, Z, ldz, C, ldc, rows, cols, K, tri);
  }
  // C = X Z with X rows x K (x_lower: lower triangular), Z K x cols.
  dgchefsi_status prod_nn(const double* X, int64_t ldx, const double* Z, int64_t ldz, double* C, int64_t ldc,
                          int64_t rows, int64_t cols, int64_t K, bool x_lower) {
    if (std::min(std::min(rows, cols), K) >= kSliced)
      return sliced_gemm(ctx, false, x_lower, rows, cols, K, X, ldx, Z, ldz, C, ldc, slices, bad);
    return x_lower ? small<false, true>(X, ldx, Z, ldz, C, ldc, rows, cols, K, false)
                   : small<false, false>(X, ldx, Z, ldz, C, ldc, rows, cols, K, false);
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
      k_chol_leaf<<<1, kLeafThreads, 0, st>>>(a, lda, li, n, (int)m, i0, info);
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
  DG_TRY(ensure(ctx, ctx->ws_chol, sizeof(double) * (3 * nn + (size_t)kPartial + (size_t)n), "Cholesky workspace"));
  double* Li = static_cast<double*>(ctx->ws_chol.p);
  double* d = Li + 3 * nn + kPartial;
  Chol c{ctx, S, lda, Li, Li + nn, Li + 2 * nn, Li + 3 * nn, n, info, bad, std::max(ctx->products_slices, 10),
         ctx->stream};
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
