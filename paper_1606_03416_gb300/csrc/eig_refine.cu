// Eigen-decomposition of the projected Hamiltonian H_hat (Alg. 1 step 4) from
// dense products. The paper's subspace problem is its largest cost at scale
// and its Conclusion proposes moving it onto matrix products; here the FP64
// eigenpairs come from a cheap approximate start improved by iterative
// refinement whose work is three dense products per step, run on the
// tensor cores from exact BF16 slices (sliced.cu).
//
// Refinement (Ogita and Aishima, "Iterative refinement for symmetric
// eigenvalue decomposition", Japan J. Indust. Appl. Math. 35, 2018; clustered
// eigenvalues after their part II, 2019). With X the approximate
// eigenvectors as columns (here V = X^T, one eigenvector per row):
//   G = X^T X,  S = X^T A X,  lambda_i = S_ii / G_ii,
//   e_ii = (1 - G_ii) / 2,
//   e_ij = (S_ij - lambda_j G_ij) / (lambda_j - lambda_i)        (i != j),
//   X <- X (I + E).
// These are the first-order conditions for X (I + E) to be orthonormal
// (E + E^T = I - G) and to diagonalise A; the error falls quadratically
// while every |e_ij| stays small. The coefficients are formed from the
// symmetrised G and S, so E + E^T = I - G holds over any gap; a coupling at
// the rounding level of the products (below kNoise u ||A||) over a gap too
// small to rotate safely gets only the orthonormalisation term.
// Pairs whose first-order correction would not be small
// (|lambda_j - lambda_i| <= kappa |S_ij - lambda_j G_ij|, or a gap at the
// rounding level) are joined into clusters: connected components, widened to
// the range of Rayleigh quotients they span. The columns of a cluster C are
// first rotated exactly: X_C <- X_C W with W = (I + R/2) Q, R = I - G_CC and
// Q the eigenvectors of M = S_CC + (R S_CC + S_CC R) / 2 (first order of
// G_CC^{-1/2} S_CC G_CC^{-1/2}), found by cyclic Jacobi (Golub and Van Loan,
// Matrix Computations, 4th ed., Sec. 8.5). Inside a cluster
// e_ij = (I - G)_ij / 2 then keeps X orthonormal.
//
// Start: a row of A whose first-order couplings |A_ij| / |A_jj - A_ii| all
// stay below the context's start threshold begins as its unit vector (a
// projected H of converging CheFSI cycles is nearly diagonal); the block of
// the other rows gets FP32 eigenvectors (this library's Jacobi kernel up to
// kJacobiMax rows, else cuSOLVER's single-precision solver), the whole matrix
// when more than half the rows are in it. With V = I the
// first step needs no products; with V = I outside a block of at most n/8
// rows, only small FP64 products on the block's rows and columns.
//
// Products per later step: T = V A, [G; S] = [V; T] V^T (one call, 2n x n,
// lower triangles) and the update V <- V + E^T V, all n x n x n on the
// slice-pair kernel; the update takes only the slices that the size of E
// needs (update_slices), fewer as the corrections shrink. Stop after the step whose largest correction is at most
// kStop, or whose correction, at the quadratic rate seen over the last two
// steps, predicts the next one below kPredict.

#include <algorithm>
#include <cfloat>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "ctx.h"

#define EIG_SOLVER(call)                                                                                   \
  do {                                                                                                     \
    cusolverStatus_t s_ = (call);                                                                          \
    if (s_ != CUSOLVER_STATUS_SUCCESS)                                                                     \
      return dg::set_error(DGCHEFSI_ERR_CUDA, "%s failed: cuSOLVER status %d", #call, (int)s_);             \
  } while (0)

namespace dg {

namespace {

constexpr int kMaxCluster = 32;    // largest cluster the Jacobi kernel takes
constexpr int kMaxSteps = 10;      // refinement steps before the FP64 fallback
constexpr double kKappa = 100.0;   // cluster when |e_ij| would exceed 1/kappa
constexpr double kStop = 1e-8;     // last step: the next correction is O(kStop^2)
constexpr double kPredict = 1e-15; // or when the next correction is predicted below this
constexpr double kNoise = 256.0;   // couplings below kNoise u ||A|| are rounding noise of the products

unsigned grid_for(int64_t n, int t = 256) { return (unsigned)std::min<int64_t>((n + t - 1) / t, 1 << 20); }

// B (FP32, n x n) = A (FP64, lda) with the lower triangle (row-major)
// mirrored into the upper one.
__global__ void k_lower_to_f32(const double* __restrict__ A, int64_t lda, int64_t n, float* __restrict__ B) {
  const int64_t tot = n * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / n, j = t % n;
    B[t] = (float)(j <= i ? A[i * lda + j] : A[j * lda + i]);
  }
}

// The upper triangle (row-major) of A is overwritten by the lower one.
__global__ void k_mirror_lower(double* A, int64_t lda, int64_t n) {
  const int64_t tot = n * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / n, j = t % n;
    if (j > i) A[i * lda + j] = A[j * lda + i];
  }
}

__global__ void k_f32_to_f64(const float* __restrict__ A, int64_t tot, double* __restrict__ B) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x)
    B[t] = (double)A[t];
}

// lam[i] = S[i, i] / G[i, i]  (G, S row-major n x n, ld n)
__global__ void k_rayleigh(const double* __restrict__ G, const double* __restrict__ S, int64_t n,
                           double* __restrict__ lam) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    lam[i] = S[i * n + i] / G[i * n + i];
}

// Symmetrised entries of the 32 x 32 tile (i0, j0) of G and S: the tile
// itself is read along j by the caller, the mirror tile (j0, i0) is staged
// here transposed, so Gt[r][c] = G[j0 + c, i0 + r] (likewise St).
__device__ __forceinline__ void stage_mirror(const double* __restrict__ G, const double* __restrict__ S, int64_t n,
                                             int64_t i0, int64_t j0, double (*Gt)[33], double (*St)[33]) {
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t j = j0 + r, i = i0 + threadIdx.x;
    if (j < n && i < n) {
      Gt[threadIdx.x][r] = G[j * n + i];
      St[threadIdx.x][r] = S[j * n + i];
    }
  }
}

// Pairs i < j whose first-order correction would not be small,
// |lambda_j - lambda_i| <= kappa |S_ij - lambda_j G_ij| (G, S symmetrised),
// or whose gap is at the rounding level: written to pairs[0..cap) (count
// keeps counting past cap). 32 x 32 tiles on and above the diagonal.
__global__ void __launch_bounds__(256) k_close_pairs(const double* __restrict__ G, const double* __restrict__ S,
                                                     int64_t n, const double* __restrict__ lam, double kappa,
                                                     double floor_gap, int2* __restrict__ pairs, int cap,
                                                     int* __restrict__ count) {
  __shared__ double Gt[32][33], St[32][33];
  if (blockIdx.y > blockIdx.x) return;
  const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
  stage_mirror(G, S, n, i0, j0, Gt, St);
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t i = i0 + r, j = j0 + threadIdx.x;
    if (i < n && j < n && j > i) {
      const double g = 0.5 * (G[i * n + j] + Gt[r][threadIdx.x]);
      const double sv = 0.5 * (S[i * n + j] + St[r][threadIdx.x]);
      const double li = lam[i], lj = lam[j];
      const double gap = fabs(lj - li);
      if (gap <= floor_gap || gap <= kappa * fabs(sv - lj * g)) {
        const int slot = atomicAdd(count, 1);
        if (slot < cap) pairs[slot] = make_int2((int)i, (int)j);
      }
    }
  }
}

// One warp per cluster q (members idx[cofs[q] .. cofs[q + 1]), c <= 32):
// W_q (c x c row-major at Wd + wofs[q]) = (I + R/2) Q with R = I - G_CC and
// Q the eigenvectors (columns) of M = S_CC + (R S_CC + S_CC R)/2, G_CC and
// S_CC symmetrised. M is exactly symmetric as computed (the two products
// take the same terms in the same order), and cyclic Jacobi sweeps run until
// the off-diagonal part is below 2^-56 of M in the Frobenius norm (at most
// 50 sweeps). Each rotation zeroes M_pr: tau = (M_rr - M_pp) / (2 M_pr),
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c.
__global__ void __launch_bounds__(32) k_cluster_rotations(const double* __restrict__ G, const double* __restrict__ S,
                                                         int64_t n, const int* __restrict__ idx,
                                                         const int* __restrict__ cofs, const int* __restrict__ wofs,
                                                         int ncl, double* __restrict__ Wd) {
  __shared__ double Ms[kMaxCluster][kMaxCluster + 1], Qs[kMaxCluster][kMaxCluster + 1];
  __shared__ double Rs[kMaxCluster][kMaxCluster + 1], Ss[kMaxCluster][kMaxCluster + 1];
  const int lane = threadIdx.x;
  for (int q = blockIdx.x; q < ncl; q += gridDim.x) {
    const int c0 = cofs[q], c = cofs[q + 1] - c0;
    __syncwarp();
    if (lane < c) {
      const int64_t ib = idx[c0 + lane];
      for (int a = 0; a < c; ++a) {
        const int64_t ia = idx[c0 + a];
        Ss[a][lane] = 0.5 * (S[ia * n + ib] + S[ib * n + ia]);
        Rs[a][lane] = (a == lane ? 1.0 : 0.0) - 0.5 * (G[ia * n + ib] + G[ib * n + ia]);
        Qs[a][lane] = a == lane ? 1.0 : 0.0;
      }
    }
    __syncwarp();
    if (lane < c) {
      for (int b = 0; b < c; ++b) {
        double rs = 0.0, sr = 0.0;
        for (int d = 0; d < c; ++d) {
          rs += Rs[lane][d] * Ss[d][b];
          sr += Ss[lane][d] * Rs[d][b];
        }
        Ms[lane][b] = Ss[lane][b] + 0.5 * (rs + sr);
      }
    }
    __syncwarp();
    for (int sweep = 0; sweep < 50; ++sweep) {
      double off = 0.0, tot = 0.0;
      if (lane < c)
        for (int b = 0; b < c; ++b) {
          const double m = Ms[lane][b];
          tot += m * m;
          if (b != lane) off += m * m;
        }
      for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(0xffffffffu, off, o);
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
      }
      if (!(off > 0x1p-112 * tot)) break;  // also ends on NaN
      for (int p = 0; p < c - 1; ++p) {
        for (int r = p + 1; r < c; ++r) {
          const double apr = Ms[p][r];
          if (apr == 0.0) continue;
          const double tau = (Ms[r][r] - Ms[p][p]) / (2.0 * apr);
          const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          const double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
          __syncwarp();
          if (lane < c) {  // M <- M J, Q <- Q J (columns p, r)
            const double mp = Ms[lane][p], mr = Ms[lane][r];
            Ms[lane][p] = cs * mp - sn * mr;
            Ms[lane][r] = sn * mp + cs * mr;
            const double qp = Qs[lane][p], qr = Qs[lane][r];
            Qs[lane][p] = cs * qp - sn * qr;
            Qs[lane][r] = sn * qp + cs * qr;
          }
          __syncwarp();
          if (lane < c) {  // M <- J^T M (rows p, r)
            const double mp = Ms[p][lane], mr = Ms[r][lane];
            Ms[p][lane] = cs * mp - sn * mr;
            Ms[r][lane] = sn * mp + cs * mr;
          }
          __syncwarp();
        }
      }
    }
    if (lane < c) {
      double* W = Wd + wofs[q];
      for (int b = 0; b < c; ++b) {
        double acc = 0.0;
        for (int d = 0; d < c; ++d) acc += Rs[lane][d] * Qs[d][b];
        W[lane * c + b] = Qs[lane][b] + 0.5 * acc;
      }
    }
  }
}

// Rows of every cluster in up to three matrices (blockIdx.z picks one; null
// skipped): X[C_b, j] <- sum_a W_ab X[C_a, j] for j < ncols.
__global__ void __launch_bounds__(256) k_rotate_rows(double* X0, double* X1, double* X2, int64_t ld, int64_t ncols,
                                                     const int* __restrict__ idx, const int* __restrict__ cofs,
                                                     const int* __restrict__ wofs, int ncl,
                                                     const double* __restrict__ Wd) {
  __shared__ double Ws[kMaxCluster * kMaxCluster];
  double* X = blockIdx.z == 0 ? X0 : (blockIdx.z == 1 ? X1 : X2);
  if (X == nullptr) return;
  for (int q = blockIdx.y; q < ncl; q += gridDim.y) {
    const int c0 = cofs[q], c = cofs[q + 1] - c0;
    __syncthreads();
    for (int t = threadIdx.x; t < c * c; t += blockDim.x) Ws[t] = Wd[wofs[q] + t];
    __syncthreads();
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < ncols; j += (int64_t)gridDim.x * blockDim.x) {
      double x[kMaxCluster];
      for (int a = 0; a < c; ++a) x[a] = X[(int64_t)idx[c0 + a] * ld + j];
      for (int b = 0; b < c; ++b) {
        double y = 0.0;
        for (int a = 0; a < c; ++a) y += Ws[a * c + b] * x[a];
        X[(int64_t)idx[c0 + b] * ld + j] = y;
      }
    }
  }
}

// Columns of every cluster in up to two matrices: X[i, C_b] <- sum_a X[i, C_a] W_ab.
__global__ void __launch_bounds__(256) k_rotate_cols(double* X0, double* X1, int64_t ld, int64_t nrows,
                                                     const int* __restrict__ idx, const int* __restrict__ cofs,
                                                     const int* __restrict__ wofs, int ncl,
                                                     const double* __restrict__ Wd) {
  __shared__ double Ws[kMaxCluster * kMaxCluster];
  double* X = blockIdx.z == 0 ? X0 : X1;
  if (X == nullptr) return;
  for (int q = blockIdx.y; q < ncl; q += gridDim.y) {
    const int c0 = cofs[q], c = cofs[q + 1] - c0;
    __syncthreads();
    for (int t = threadIdx.x; t < c * c; t += blockDim.x) Ws[t] = Wd[wofs[q] + t];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrows; i += (int64_t)gridDim.x * blockDim.x) {
      double x[kMaxCluster];
      for (int a = 0; a < c; ++a) x[a] = X[i * ld + idx[c0 + a]];
      for (int b = 0; b < c; ++b) {
        double y = 0.0;
        for (int a = 0; a < c; ++a) y += x[a] * Ws[a * c + b];
        X[i * ld + idx[c0 + b]] = y;
      }
    }
  }
}

// F = E^T (row-major n x n): F[j, i] = e_ij with, for G and S symmetrised,
// nu_ij = S_ij - lambda_j G_ij and D = lambda_j - lambda_i,
//   e_ii = (1 - G_ii)/2,
//   e_ij = nu_ij / D, except -G_ij/2 (orthonormalisation only) inside a
//          cluster (cl[i] == cl[j] >= 0), for |D| at the rounding level
//          (floor_gap), and for a coupling |S_ij - (lambda_i + lambda_j) G_ij / 2|
//          at the rounding level of the products (floor_num) whose rotation
//          would exceed stop (noise over a tiny gap, which a rotation would
//          only turn into a loss of orthonormality).
// Both branches are symmetric in (i, j), so E + E^T = I - G. emax (the bits
// of a non-negative double) = max |e_ij|, +inf on NaN. 32 x 32 tiles: read
// along j (the mirror tile staged transposed), written transposed.
__global__ void __launch_bounds__(256) k_update_coeffs(const double* __restrict__ G, const double* __restrict__ S,
                                                       int64_t n, const double* __restrict__ lam,
                                                       const int* __restrict__ cl, double floor_gap, double floor_num,
                                                       double stop, double* __restrict__ F,
                                                       unsigned long long* emax) {
  __shared__ double Gt[32][33], St[32][33], tile[32][33];
  __shared__ double red[8];
  const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
  stage_mirror(G, S, n, i0, j0, Gt, St);
  __syncthreads();
  double m = 0.0;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t i = i0 + r, j = j0 + threadIdx.x;
    double e = 0.0;
    if (i < n && j < n) {
      const double g = 0.5 * (G[i * n + j] + Gt[r][threadIdx.x]);
      if (i == j) {
        e = 0.5 * (1.0 - g);
      } else {
        const double sv = 0.5 * (S[i * n + j] + St[r][threadIdx.x]);
        const double li = lam[i], lj = lam[j], gap = lj - li;
        const int ci = cl[i];
        const double cpl = fabs(sv - 0.5 * (li + lj) * g);
        if ((ci >= 0 && ci == cl[j]) || fabs(gap) <= floor_gap || (cpl <= floor_num && cpl > stop * fabs(gap)))
          e = -0.5 * g;
        else
          e = (sv - lj * g) / gap;
      }
      const double ae = fabs(e);
      m = ae <= DBL_MAX ? fmax(m, ae) : INFINITY;
    }
    tile[r][threadIdx.x] = e;
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  const int warp = (threadIdx.y * 32 + threadIdx.x) >> 5;
  if ((threadIdx.x & 31) == 0) red[warp] = m;
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t j = j0 + r, i = i0 + threadIdx.x;
    if (i < n && j < n) F[j * n + i] = tile[threadIdx.x][r];
  }
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    double b = red[0];
    for (int w = 1; w < 8; ++w) b = fmax(b, red[w]);
    atomicMax(emax, (unsigned long long)__double_as_longlong(b));
  }
}

// FP32 eigenvectors of a small symmetric block by cyclic Jacobi (Golub and
// Van Loan, Matrix Computations, 4th ed., Sec. 8.5.5: the parallel ordering).
// B (m x m, m <= kJacobiMax, in: the block; the lower triangle is read); W
// (m x m, out) the eigenvectors as rows (W[k * m + l]: component l of vector
// k, the layout the scatter into V expects); w[k] the eigenvalues
// (unordered). Each round rotates M/2 disjoint index pairs at once, the
// round-robin tournament over M = m rounded up to even indices (index m, when
// m is odd, is idle): pairs (pos_k, pos_{M-1-k}) with pos_0 = 0, pos_i = 1 +
// (i - 1 + r) mod (M - 1). A rotation zeroes B_pq: tau = (B_qq - B_pp) /
// (2 B_pq), t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2),
// s = t c; B <- R^T B R and W <- R^T W with columns p, q of R equal to
// (c e_p - s e_q, s e_p + c e_q). Because the pairs of a round are disjoint,
// the 2 x 2 block of B on rows of pair k and columns of pair l receives
// exactly the column rotation of l and then the row rotation of k, so one
// pass over the blocks with l >= k applies the whole round. After each sweep
// (M - 1 rounds) the off-diagonal part is measured; the sweeps stop once its
// squared Frobenius norm is below 2^-32 of the whole (2^-16 in norm: near
// FP32 rounding, a start for the FP64 refinement) or after 40.
// B is held once per entry (jacobi_slot), so a block of 320 rows takes
// ~207 KB of shared memory. Every CTA of the grid runs the same iteration on
// its own copy of B (the arithmetic and its order are identical, so are the
// rotations) and keeps components [c0, c0 + cw) of the vectors, cw =
// ceil(m / gridDim.x), in shared memory.
constexpr int kJacobiMax = 320;
constexpr int kJacobiThreads = 1024;
constexpr int kJacobiCtas = 32;
constexpr int kJacobiChunks = (kJacobiMax / 2 + 31) / 32;  // 32-wide chunks of the pair index

// Slot of entry {i, j} (i, j < m) in the wrapped half storage of a symmetric
// matrix: with the odd modulus Mo = m | 1 and d = (j - i) mod Mo, exactly one
// of d and Mo - d is at most (Mo - 1) / 2; the entry is column d of row i in
// the first case, column Mo - d of row j in the second (column 0: the
// diagonal). Rows have ld >= (Mo + 1) / 2 columns, ld even: 32 consecutive
// j then fall on distinct banks in either case (strides 1 and ld - 1).
__device__ __forceinline__ int jacobi_slot(int i, int j, int Mo, int ld) {
  int d = j - i;
  d += d < 0 ? Mo : 0;
  return d <= (Mo >> 1) ? i * ld + d : j * ld + (Mo - d);
}

__host__ __device__ constexpr int jacobi_ld(int m) { return (((m | 1) + 1) / 2 + 1) & ~1; }

__global__ void __launch_bounds__(kJacobiThreads, 1) k_block_jacobi(const float* __restrict__ B, int m,
                                                                    float* __restrict__ W, float* __restrict__ w) {
  extern __shared__ float sm_j[];
  __shared__ float cs[kJacobiMax / 2], sn[kJacobiMax / 2];
  __shared__ int pp[kJacobiMax / 2], qq[kJacobiMax / 2];
  __shared__ float red[2][kJacobiThreads / 32];
  __shared__ int done;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
  const int cw = (m + (int)gridDim.x - 1) / (int)gridDim.x, c0 = (int)blockIdx.x * cw;
  const int Mo = m | 1, ld = jacobi_ld(m), ncol = (Mo + 1) / 2;
  float* As = sm_j;           // m x ld, wrapped half storage
  float* Ws = sm_j + m * ld;  // m x cw: components c0 .. c0 + cw - 1 of every vector
  const int M = m + (m & 1), half = M / 2;
  for (int i = warp; i < m; i += nw) {
    for (int d = lane; d < ld; d += 32) {
      int j = i + d;
      j -= j >= Mo ? Mo : 0;
      As[i * ld + d] = d < ncol && j < m ? B[(int64_t)max(i, j) * m + min(i, j)] : 0.0f;
    }
    for (int j = lane; j < cw; j += 32) Ws[i * cw + j] = c0 + j == i ? 1.0f : 0.0f;
  }
  if (t == 0) done = 0;
  __syncthreads();
  for (int sweep = 0; sweep < 40; ++sweep) {
    for (int r = 0; r < M - 1; ++r) {
      if (t < half) {  // pair t of this round and its rotation
        const int pa = t == 0 ? 0 : 1 + (t - 1 + r) % (M - 1);
        const int k2 = M - 1 - t;
        const int pb = k2 == 0 ? 0 : 1 + (k2 - 1 + r) % (M - 1);
        const int p = min(pa, pb), q = max(pa, pb);
        float c = 1.0f, sv = 0.0f;
        if (q < m) {
          const float apq = As[jacobi_slot(q, p, Mo, ld)];
          if (apq != 0.0f) {
            const float tau = (As[q * ld] - As[p * ld]) / (2.0f * apq);
            const float tt = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
            c = 1.0f / sqrtf(1.0f + tt * tt);
            sv = tt * c;
          }
        }
        pp[t] = p;
        qq[t] = q < m ? q : p;  // a pair with the idle index rotates nothing
        cs[t] = c;
        sn[t] = q < m ? sv : 0.0f;
      }
      __syncthreads();
      // block (k, l), l >= k: rows pp[k], qq[k] x columns pp[l], qq[l]; each
      // entry is in exactly one such block. Warp w takes k = w, w + nw, ...
      // and lane j the l = 32 c + j of chunk c, whose pair values it holds in
      // registers for the whole round.
      int pl[kJacobiChunks], ql[kJacobiChunks];
      float cl[kJacobiChunks], sl[kJacobiChunks];
#pragma unroll
      for (int c = 0; c < kJacobiChunks; ++c) {
        const int l = c * 32 + lane;
        const bool on = l < half;
        pl[c] = on ? pp[l] : 0;
        ql[c] = on ? qq[l] : 0;
        cl[c] = on ? cs[l] : 1.0f;
        sl[c] = on ? sn[l] : 0.0f;
      }
      for (int k = warp; k < half; k += nw) {
        const int pk = pp[k], qk = qq[k];
        const float ck = cs[k], sk = sn[k];
        const bool krot = qk != pk;
#pragma unroll
        for (int c = 0; c < kJacobiChunks; ++c) {
          const int l = c * 32 + lane;
          if (l < k || l >= half) continue;
          const bool lrot = ql[c] != pl[c];
          // on the pair's own block (l == k) slots sb and sd coincide
          const int sa = jacobi_slot(pk, pl[c], Mo, ld), sb = jacobi_slot(pk, ql[c], Mo, ld);
          const int sd = jacobi_slot(qk, pl[c], Mo, ld), se = jacobi_slot(qk, ql[c], Mo, ld);
          const float a = As[sa], b = As[sb], d = As[sd], e = As[se];
          const float a1 = cl[c] * a - sl[c] * b, b1 = sl[c] * a + cl[c] * b;
          const float d1 = cl[c] * d - sl[c] * e, e1 = sl[c] * d + cl[c] * e;
          As[sa] = ck * a1 - sk * d1;
          if (l == k) {
            if (krot) {
              As[sb] = ck * b1 - sk * e1;
              As[se] = sk * b1 + ck * e1;
            }
            continue;
          }
          if (lrot) As[sb] = ck * b1 - sk * e1;
          if (krot) {
            As[sd] = sk * a1 + ck * d1;
            if (lrot) As[se] = sk * b1 + ck * e1;
          }
        }
        if (krot)  // rows pk, qk of the W slab
          for (int j = lane; j < cw; j += 32) {
            const float vp = Ws[pk * cw + j], vq = Ws[qk * cw + j];
            Ws[pk * cw + j] = ck * vp - sk * vq;
            Ws[qk * cw + j] = sk * vp + ck * vq;
          }
      }
      __syncthreads();
    }
    float off = 0.0f, tot = 0.0f;
    for (int i = warp; i < m; i += nw)
      for (int d = lane; d < ncol; d += 32) {
        int j = i + d;
        j -= j >= Mo ? Mo : 0;
        if (j >= m) continue;
        const float a = As[i * ld + d];
        const float a2 = d == 0 ? a * a : 2.0f * a * a;  // an off-diagonal slot holds two entries
        tot += a2;
        if (d != 0) off += a2;
      }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if (lane == 0) {
      red[0][warp] = off;
      red[1][warp] = tot;
    }
    __syncthreads();
    if (t == 0) {
      float so = 0.0f, st = 0.0f;
      for (int k = 0; k < nw; ++k) {
        so += red[0][k];
        st += red[1][k];
      }
      done = !(so > 0x1p-32f * st);  // also ends on NaN
    }
    __syncthreads();
    if (done) break;
  }
  if (blockIdx.x == 0)
    for (int i = t; i < m; i += blockDim.x) w[i] = As[i * ld];
  for (int i = warp; i < m; i += nw)
    for (int j = lane; j < cw && c0 + j < m; j += 32) W[(int64_t)i * m + c0 + j] = Ws[i * cw + j];
}

// Start selection. Row i of A (symmetric, both triangles valid) is coupled
// when some j != i has a first-order correction |A_ij| / |A_jj - A_ii| of at
// least tau, i.e. |A_ij| >= tau |A_jj - A_ii|, with |A_ij| above the rounding
// floor: flag[i] = 1 then, else 0. diag[i] = A_ii. One CTA per row.
__global__ void __launch_bounds__(256) k_row_coupling(const double* __restrict__ A, int64_t lda, int64_t n,
                                                      double tau, double floor_num, int* __restrict__ flag,
                                                      double* __restrict__ diag) {
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const double aii = A[i * lda + i];
    int hit = 0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      const double aij = fabs(A[i * lda + j]);
      if (j != i && aij > floor_num && aij >= tau * fabs(A[j * lda + j] - aii)) hit = 1;
    }
    const int any = __syncthreads_or(hit);
    if (threadIdx.x == 0) {
      flag[i] = any;
      diag[i] = aii;
    }
  }
}

// B32 (m x m FP32) = A[rows[k], rows[l]].
__global__ void k_gather_block_f32(const double* __restrict__ A, int64_t lda, const int* __restrict__ rows, int64_t m,
                                   float* __restrict__ B32) {
  const int64_t tot = m * m;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x)
    B32[t] = (float)A[(int64_t)rows[t / m] * lda + rows[t % m]];
}

// V = I (n x n).
__global__ void k_identity(double* __restrict__ V, int64_t n) {
  const int64_t tot = n * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x)
    V[t] = (t / n == t % n) ? 1.0 : 0.0;
}

// Rows rows[k] of V (= I outside them) become the eigenvectors of the
// gathered block: V[rows[k], rows[l]] = W[k * m + l] (the FP32 solver's
// column-major eigenvectors read row-major).
__global__ void k_scatter_block(double* __restrict__ V, int64_t n, const int* __restrict__ rows, int64_t m,
                                const float* __restrict__ W) {
  const int64_t tot = m * m;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x)
    V[(int64_t)rows[t / m] * n + rows[t % m]] = (double)W[t];
}

// Block-structured V (the identity outside the rows and columns rows[0..m)):
// gathers and scatters of those rows and columns.
// R (m x ncols) = X[rows[k], :]
__global__ void k_gather_rows_of(const double* __restrict__ X, int64_t ldx, const int* __restrict__ rows, int64_t m,
                                 int64_t ncols, double* __restrict__ R) {
  const int64_t tot = m * ncols;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x)
    R[t] = X[(int64_t)rows[t / ncols] * ldx + t % ncols];
}
// X[rows[k], :] = R (m x ncols)
__global__ void k_scatter_rows_of(double* __restrict__ X, int64_t ldx, const int* __restrict__ rows, int64_t m,
                                  int64_t ncols, const double* __restrict__ R) {
  const int64_t tot = m * ncols;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x)
    X[(int64_t)rows[t / ncols] * ldx + t % ncols] = R[t];
}
// R (nrows x m) = X[:, cols[k]]
__global__ void k_gather_cols_of(const double* __restrict__ X, int64_t ldx, const int* __restrict__ cols, int64_t m,
                                 int64_t nrows, double* __restrict__ R) {
  const int64_t tot = m * nrows;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x)
    R[t] = X[(t / m) * ldx + cols[t % m]];
}
// X[i, cols[k]] = R[i, k] + (pos[i] >= 0 ? B[pos[i], k] : 0) for every row i
// (R nrows x m; B m x m, may be null)
__global__ void k_scatter_cols_of(double* __restrict__ X, int64_t ldx, const int* __restrict__ cols, int64_t m,
                                  int64_t nrows, const double* __restrict__ R, const int* __restrict__ pos,
                                  const double* __restrict__ B) {
  const int64_t tot = m * nrows;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / m, k = t % m;
    double v = R[t];
    if (B && pos[i] >= 0) v += B[(int64_t)pos[i] * m + k];
    X[i * ldx + cols[k]] = v;
  }
}
// X[rows[k], rows[l]] = B[k, l]  (B m x m)
__global__ void k_scatter_block_of(double* __restrict__ X, int64_t ldx, const int* __restrict__ rows, int64_t m,
                                   const double* __restrict__ B) {
  const int64_t tot = m * m;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x)
    X[(int64_t)rows[t / m] * ldx + rows[t % m]] = B[t];
}
// B (m x m) = X[rows[k], rows[l]]
__global__ void k_gather_block_of(const double* __restrict__ X, int64_t ldx, const int* __restrict__ rows, int64_t m,
                                  double* __restrict__ B) {
  const int64_t tot = m * m;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x)
    B[t] = X[(int64_t)rows[t / m] * ldx + rows[t % m]];
}

// For V = I: G = I and S = A (the products of a step, without computing them).
__global__ void k_identity_products(const double* __restrict__ A, int64_t lda, int64_t n, double* __restrict__ G,
                                    double* __restrict__ S) {
  const int64_t tot = n * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / n, j = t % n;
    G[t] = i == j ? 1.0 : 0.0;
    S[t] = A[i * lda + j];
  }
}

// A[r, :] = V[perm[r], :] (ld n -> lda) and w[r] = lam[perm[r]].
__global__ void k_gather_rows(const double* __restrict__ V, int64_t n, const int* __restrict__ perm,
                              const double* __restrict__ lam, double* __restrict__ A, int64_t lda,
                              double* __restrict__ w) {
  for (int64_t r = blockIdx.y; r < n; r += gridDim.y) {
    const int64_t src = perm[r];
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
      A[r * lda + j] = V[src * n + j];
    if (blockIdx.x == 0 && threadIdx.x == 0) w[r] = lam[src];
  }
}

}  // namespace

}  // namespace dg

namespace dg {

namespace {

// cuSOLVER's FP64 divide-and-conquer on the lower triangle (row-major) of A;
// its info goes to ctx->info_d[2].
dgchefsi_status eig_syevd(dgchefsi_ctx* ctx, double* A, int64_t n, int64_t lda, double* w) {
  if (n > INT32_MAX || lda > INT32_MAX)
    return set_error(DGCHEFSI_ERR_UNSUPPORTED, "eigensolve of order %lld", (long long)n);
  EIG_SOLVER(cusolverDnSetStream(ctx->solver, ctx->stream));
  int lw = 0;
  EIG_SOLVER(cusolverDnDsyevd_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, (int)n, A,
                                        (int)lda, w, &lw));
  DG_TRY(ensure(ctx, ctx->ws_solver, sizeof(double) * (size_t)lw, "cuSOLVER workspace"));
  EIG_SOLVER(cusolverDnDsyevd(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, (int)n, A, (int)lda, w,
                             static_cast<double*>(ctx->ws_solver.p), (int)(ctx->ws_solver.bytes / sizeof(double)),
                             ctx->info_d + 2));
  return DGCHEFSI_OK;
}

// Layout of the refinement's workspace for order n.
struct EigWs {
  float* A32;          // n x n: FP32 copy of A, then the FP32 start's vectors
  float* w32;          // n
  double* VT;          // 2n x n: V (rows = vectors), then T = V A
  double* GS;          // 2n x n: G = V V^T, S = T V^T; rows 0..n-1 reused for E^T V
  double* F;           // n x n: E^T
  double* lam;         // n
  double* Wd;          // cluster rotations (sum of c^2 <= 32 n)
  int2* pairs;         // cap
  int* cl;             // n: cluster of each row, -1 for none
  int* idx;            // n: cluster members
  int* cofs;           // n + 1
  int* wofs;           // n + 1
  int* perm;           // n: the block's rows in the first step, the final order at the end
  int* posb;           // n: position of a row in the block, -1 outside
  int* cnt;            // [0] close-pair count, [1] FP32 start info, [2] non-finite operand flag
  unsigned long long* emax;
  int cap;
  size_t bytes;
};

EigWs eig_layout(int64_t n, char* base) {
  EigWs w{};
  size_t o = 0;
  auto take = [&](size_t b) {
    const size_t at = o;
    o += (b + 255) / 256 * 256;
    return base ? base + at : nullptr;
  };
  const size_t nn = (size_t)n * (size_t)n;
  w.cap = (int)std::min<int64_t>(16 * n, 1 << 24);
  w.A32 = reinterpret_cast<float*>(take(sizeof(float) * nn));
  w.w32 = reinterpret_cast<float*>(take(sizeof(float) * (size_t)n));
  w.VT = reinterpret_cast<double*>(take(sizeof(double) * 2 * nn));
  w.GS = reinterpret_cast<double*>(take(sizeof(double) * 2 * nn));
  w.F = reinterpret_cast<double*>(take(sizeof(double) * nn));
  w.lam = reinterpret_cast<double*>(take(sizeof(double) * (size_t)n));
  w.Wd = reinterpret_cast<double*>(take(sizeof(double) * (size_t)n * kMaxCluster));
  w.pairs = reinterpret_cast<int2*>(take(sizeof(int2) * (size_t)w.cap));
  w.cl = reinterpret_cast<int*>(take(sizeof(int) * (size_t)n));
  w.idx = reinterpret_cast<int*>(take(sizeof(int) * (size_t)n));
  w.cofs = reinterpret_cast<int*>(take(sizeof(int) * (size_t)(n + 1)));
  w.wofs = reinterpret_cast<int*>(take(sizeof(int) * (size_t)(n + 1)));
  w.perm = reinterpret_cast<int*>(take(sizeof(int) * (size_t)n));
  w.posb = reinterpret_cast<int*>(take(sizeof(int) * (size_t)n));
  w.cnt = reinterpret_cast<int*>(take(sizeof(int) * 4));
  w.emax = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long)));
  w.bytes = o;
  return w;
}

// Outcome of the refinement other than an error: done, or hand over to the
// FP64 eigensolver (the reason is recorded in the context's statistics).
enum class Refine { kDone, kFallback };

int find_root(std::vector<int>& parent, int x) {
  while (parent[x] != x) {
    parent[x] = parent[parent[x]];
    x = parent[x];
  }
  return x;
}

}  // namespace

}  // namespace dg

namespace dg {

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t) { return std::chrono::duration<double, std::milli>(Clock::now() - t).count(); }

// The refinement. *reason = 0 when A and w hold the result, else the reason
// for handing over to the FP64 eigensolver (A's lower triangle is then
// untouched): 1 the FP32 start failed, 2 more close pairs than the table
// holds, 3 a cluster larger than kMaxCluster, 4 a correction that is not
// finite or not below 1, 5 no convergence in kMaxSteps steps.
// Fewest slices s' in [2, smax] of the refinement's update product E^T V
// whose splitting error, 2 L emax 2^{-6s'} (s' + 4) per K chunk, stays below
// u L = 2^-53 L; smax when none does.
static int update_slices(double emax, int smax) {
  for (int sp = 2; sp < smax; ++sp)
    if (2.0 * std::ldexp((double)(sp + 4), -6 * sp) * emax <= 0x1p-53) return sp;
  return smax;
}

dgchefsi_status eig_refined(dgchefsi_ctx* ctx, double* A, int64_t n, int64_t lda, double* w, int* reason) {
  *reason = 0;
  if (n > INT32_MAX / 2 || lda > INT32_MAX)
    return set_error(DGCHEFSI_ERR_UNSUPPORTED, "eigensolve of order %lld", (long long)n);
  cudaStream_t st = ctx->stream;
  const int s = std::max(ctx->products_slices, 10);
  EigWs ws = eig_layout(n, nullptr);
  DG_TRY(ensure(ctx, ctx->ws_eig, ws.bytes, "eigensolver workspace"));
  ws = eig_layout(n, static_cast<char*>(ctx->ws_eig.p));
  const int64_t nn = n * n;
  double* V = ws.VT;
  double* T = ws.VT + nn;
  double* Gm = ws.GS;
  double* Sm = ws.GS + nn;
  int* bad = ws.cnt + 2;
  const auto t0 = Clock::now();

  // Start. Rows whose first-order couplings are all below the context's
  // start threshold (0.001 by default) start from their unit vector; the
  // block of the other rows is solved in FP32 (k_block_jacobi up to
  // kJacobiMax rows, else cuSOLVER's single-precision solver) and its
  // eigenvectors placed on those rows. When more than half the rows are
  // coupled (a first projected H, a matrix without structure) the whole
  // matrix is solved in FP32 by cuSOLVER.
  k_mirror_lower<<<grid_for(nn), 256, 0, st>>>(A, lda, n);
  k_row_coupling<<<(unsigned)std::min<int64_t>(n, 1 << 16), 256, 0, st>>>(A, lda, n, ctx->eig_start_coupling, 0.0,
                                                                         ws.cl, ws.lam);
  count_launch(2);
  DG_CUDA(cudaGetLastError());
  std::vector<int> flag_h(n);
  std::vector<double> diag_h(n);
  DG_CUDA(cudaMemcpyAsync(flag_h.data(), ws.cl, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost, st));
  DG_CUDA(cudaMemcpyAsync(diag_h.data(), ws.lam, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, st));
  DG_CUDA(cudaStreamSynchronize(st));
  double norm = 0.0;
  for (double x : diag_h) norm = std::max(norm, std::fabs(x));
  std::vector<int> rows;
  for (int64_t i = 0; i < n; ++i)
    if (flag_h[i]) rows.push_back((int)i);
  const bool full = (int64_t)rows.size() * 2 > n;
  const int64_t m = full ? n : (int64_t)rows.size();
  float* W32 = ws.A32;  // the start block's FP32 eigenvectors, one per row
  ctx->eig_start_order = m;
  if (m > 0) {
    if (full) {
      k_lower_to_f32<<<grid_for(nn), 256, 0, st>>>(A, lda, n, ws.A32);
    } else {
      DG_CUDA(cudaMemcpyAsync(ws.idx, rows.data(), sizeof(int) * (size_t)m, cudaMemcpyHostToDevice, st));
      DG_CUDA(cudaMemcpyAsync(ws.perm, rows.data(), sizeof(int) * (size_t)m, cudaMemcpyHostToDevice, st));
      k_gather_block_f32<<<grid_for(m * m), 256, 0, st>>>(A, lda, ws.idx, m, ws.A32);
    }
    count_launch();
    DG_CUDA(cudaGetLastError());
    DG_CUDA(cudaMemsetAsync(ws.cnt, 0, 4 * sizeof(int), st));
    if (!full && m <= kJacobiMax) {
      // a small block: this library's Jacobi kernel, eigenvectors after the block
      W32 = ws.A32 + m * m;
      const int ctas = (int)std::min<int64_t>(kJacobiCtas, m);
      const int64_t cw = (m + ctas - 1) / ctas;
      const int smem = (int)(sizeof(float) * (m * jacobi_ld((int)m) + m * cw));
      DG_CUDA(cudaFuncSetAttribute(k_block_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      k_block_jacobi<<<ctas, kJacobiThreads, smem, st>>>(ws.A32, (int)m, W32, ws.w32);
      count_launch();
      DG_CUDA(cudaGetLastError());
      ctx->eig_start_solver = 1;
    } else {
      EIG_SOLVER(cusolverDnSetStream(ctx->solver, st));
      int lw = 0;
      EIG_SOLVER(cusolverDnSsyevd_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, (int)m,
                                             ws.A32, (int)m, ws.w32, &lw));
      DG_TRY(ensure(ctx, ctx->ws_solver, sizeof(float) * (size_t)lw, "cuSOLVER workspace"));
      EIG_SOLVER(cusolverDnSsyevd(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, (int)m, ws.A32,
                                  (int)m, ws.w32, static_cast<float*>(ctx->ws_solver.p),
                                  (int)(ctx->ws_solver.bytes / sizeof(float)), ws.cnt + 1));
      ctx->eig_start_solver = 2;
    }
    // column-major eigenvectors read row-major (the Jacobi kernel writes rows):
    // one eigenvector per row
    if (full) {
      k_f32_to_f64<<<grid_for(nn), 256, 0, st>>>(ws.A32, nn, V);
    } else {
      k_identity<<<grid_for(nn), 256, 0, st>>>(V, n);
      k_scatter_block<<<grid_for(m * m), 256, 0, st>>>(V, n, ws.idx, m, W32);
    }
    count_launch(full ? 1 : 2);
    DG_CUDA(cudaGetLastError());
    std::vector<float> w32(m);
    int sinfo = 0;
    DG_CUDA(cudaMemcpyAsync(&sinfo, ws.cnt + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    DG_CUDA(cudaMemcpyAsync(w32.data(), ws.w32, sizeof(float) * (size_t)m, cudaMemcpyDeviceToHost, st));
    DG_CUDA(cudaStreamSynchronize(st));
    for (float x : w32) norm = std::max(norm, (double)std::fabs(x));
    if (sinfo != 0) {
      *reason = 1;
      return DGCHEFSI_OK;
    }
  } else {
    k_identity<<<grid_for(nn), 256, 0, st>>>(V, n);
    count_launch();
    DG_CUDA(cudaGetLastError());
  }
  if (!std::isfinite(norm)) {
    *reason = 1;
    return DGCHEFSI_OK;
  }
  // gaps below this are rounding noise of the FP64 products
  const double floor_gap = 64.0 * 0x1p-53 * std::max(norm, DBL_MIN);
  const double floor_num = kNoise * 0x1p-53 * std::max(norm, DBL_MIN);
  ctx->eig_start_ms = ms_since(t0);

  std::vector<int2> pairs_h;
  std::vector<int> parent(n), order(n), pos(n), lo(n), hi(n), reach(n), cl_h(n), idx_h(n), cofs_h, wofs_h;
  std::vector<double> lam_h(n);
  std::vector<int> blk_h, pos_h(n);
  bool converged = false;
  bool unit = m == 0;  // V = I exactly: the step's products are known
  // V = I outside a small block (rows[] in ws.perm): the first step's products
  // and update come from products of the block's rows and columns alone
  bool block = m > 0 && !full && 8 * m <= n;
  double prev = -1.0;
  for (int step = 0; step < kMaxSteps && !converged; ++step) {
    if (unit) {
      k_identity_products<<<grid_for(nn), 256, 0, st>>>(A, lda, n, Gm, Sm);
      count_launch();
      DG_CUDA(cudaGetLastError());
    } else if (block) {
      // S = V A V^T: rows B become W A[B, :], then columns B become S[:, B] W^T;
      // G = V V^T: I outside B, W W^T on B x B (W: the block's eigenvectors, rows)
      double* Wb = T;             // m x m
      double* R1 = T + m * m;     // m x n, then n x m, then m x m
      double* R2 = R1 + m * n;    // m x n, then n x m
      k_f32_to_f64<<<grid_for(m * m), 256, 0, st>>>(W32, m * m, Wb);
      k_identity_products<<<grid_for(nn), 256, 0, st>>>(A, lda, n, Gm, Sm);
      k_gather_rows_of<<<grid_for(m * n), 256, 0, st>>>(A, lda, ws.perm, m, n, R1);
      count_launch(3);
      DG_CUDA(gemm_nn_f64(Wb, m, R1, n, R2, n, m, n, m, false, st));
      k_scatter_rows_of<<<grid_for(m * n), 256, 0, st>>>(Sm, n, ws.perm, m, n, R2);
      k_gather_cols_of<<<grid_for(m * n), 256, 0, st>>>(Sm, n, ws.perm, m, n, R1);
      count_launch(2);
      DG_CUDA(gemm_nt_f64(R1, m, Wb, m, R2, m, n, m, m, false, false, st));
      k_scatter_cols_of<<<grid_for(m * n), 256, 0, st>>>(Sm, n, ws.perm, m, n, R2, nullptr, nullptr);
      count_launch();
      DG_CUDA(gemm_nt_f64(Wb, m, Wb, m, R1, m, m, m, m, false, false, st));
      k_scatter_block_of<<<grid_for(m * m), 256, 0, st>>>(Gm, n, ws.perm, m, R1);
      count_launch();
      DG_CUDA(cudaGetLastError());
    } else {
      DG_TRY(sliced_gemm(ctx, true, false, n, n, n, V, n, A, lda, T, n, s, bad));  // T = V A
      // [G; S] = [V; T] V^T, both symmetric: lower triangles, then mirrored
      DG_TRY(sliced_gemm(ctx, true, false, 2 * n, n, n, ws.VT, n, V, n, ws.GS, n, s, bad, n));
      k_mirror_lower<<<grid_for(nn), 256, 0, st>>>(Gm, n, n);
      k_mirror_lower<<<grid_for(nn), 256, 0, st>>>(Sm, n, n);
      count_launch(2);
      DG_CUDA(cudaGetLastError());
    }
    k_rayleigh<<<grid_for(n), 256, 0, st>>>(Gm, Sm, n, ws.lam);
    DG_CUDA(cudaMemsetAsync(ws.cnt, 0, sizeof(int), st));
    const unsigned nt = (unsigned)((n + 31) / 32);
    k_close_pairs<<<dim3(nt, nt), dim3(32, 8), 0, st>>>(Gm, Sm, n, ws.lam, kKappa, floor_gap, ws.pairs, ws.cap,
                                                        ws.cnt);
    count_launch(2);
    DG_CUDA(cudaGetLastError());
    int npairs = 0;
    DG_CUDA(cudaMemcpyAsync(&npairs, ws.cnt, sizeof(int), cudaMemcpyDeviceToHost, st));
    DG_CUDA(cudaMemcpyAsync(lam_h.data(), ws.lam, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, st));
    DG_CUDA(cudaStreamSynchronize(st));
    if (npairs > ws.cap || npairs < 0) {
      *reason = 2;
      return DGCHEFSI_OK;
    }
    pairs_h.resize(npairs);
    if (npairs > 0) {
      DG_CUDA(cudaMemcpyAsync(pairs_h.data(), ws.pairs, sizeof(int2) * (size_t)npairs, cudaMemcpyDeviceToHost, st));
      DG_CUDA(cudaStreamSynchronize(st));
    }
    // Clusters: the connected components of the close pairs, each widened to
    // the range of Rayleigh quotients it spans (everything in between joins,
    // and overlapping ranges merge), so a cluster is a run of the sorted order.
    std::iota(parent.begin(), parent.end(), 0);
    for (const int2& p : pairs_h) {
      const int a = find_root(parent, p.x), b = find_root(parent, p.y);
      if (a != b) parent[std::max(a, b)] = std::min(a, b);
    }
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lam_h[a] < lam_h[b]; });
    for (int64_t k = 0; k < n; ++k) pos[order[k]] = (int)k;
    std::fill(lo.begin(), lo.end(), INT32_MAX);
    std::fill(hi.begin(), hi.end(), -1);
    for (int64_t i = 0; i < n; ++i) {
      const int r = find_root(parent, (int)i);
      lo[r] = std::min(lo[r], pos[i]);
      hi[r] = std::max(hi[r], pos[i]);
    }
    // reach[k]: the furthest sorted position a range starting at k covers
    std::fill(reach.begin(), reach.end(), -1);
    for (int64_t r = 0; r < n; ++r)
      if (hi[r] > lo[r]) reach[lo[r]] = std::max(reach[lo[r]], hi[r]);
    int ncl = 0, max_c = 1;
    cofs_h.assign(1, 0);
    for (int64_t k = 0; k < n;) {
      int end = reach[k];
      if (end <= k) {
        cl_h[order[k]] = -1;
        ++k;
        continue;
      }
      for (int64_t t = k; t <= end; ++t) end = std::max(end, reach[t]);
      for (int64_t t = k; t <= end; ++t) {
        cl_h[order[t]] = ncl;
        idx_h[cofs_h.back() + (t - k)] = order[t];
      }
      const int c = (int)(end - k + 1);
      cofs_h.push_back(cofs_h.back() + c);
      max_c = std::max(max_c, c);
      ++ncl;
      k = end + 1;
    }
    ctx->eig_max_cluster = std::max(ctx->eig_max_cluster, max_c);
    if (max_c > kMaxCluster) {
      *reason = 3;
      return DGCHEFSI_OK;
    }
    DG_CUDA(cudaMemcpyAsync(ws.cl, cl_h.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, st));
    if (ncl > 0) {
      wofs_h.assign(ncl + 1, 0);
      for (int q = 0; q < ncl; ++q) {
        const int c = cofs_h[q + 1] - cofs_h[q];
        wofs_h[q + 1] = wofs_h[q] + c * c;
      }
      DG_CUDA(cudaMemcpyAsync(ws.idx, idx_h.data(), sizeof(int) * (size_t)cofs_h[ncl], cudaMemcpyHostToDevice, st));
      DG_CUDA(cudaMemcpyAsync(ws.cofs, cofs_h.data(), sizeof(int) * (size_t)(ncl + 1), cudaMemcpyHostToDevice, st));
      DG_CUDA(cudaMemcpyAsync(ws.wofs, wofs_h.data(), sizeof(int) * (size_t)(ncl + 1), cudaMemcpyHostToDevice, st));
      const unsigned gy = (unsigned)std::min(ncl, 65535);
      k_cluster_rotations<<<(unsigned)std::min(ncl, 4096), 32, 0, st>>>(Gm, Sm, n, ws.idx, ws.cofs, ws.wofs, ncl,
                                                                        ws.Wd);
      k_rotate_rows<<<dim3(grid_for(n), gy, 3), 256, 0, st>>>(Gm, Sm, V, n, n, ws.idx, ws.cofs, ws.wofs, ncl, ws.Wd);
      k_rotate_cols<<<dim3(grid_for(n), gy, 2), 256, 0, st>>>(Gm, Sm, n, n, ws.idx, ws.cofs, ws.wofs, ncl, ws.Wd);
      k_rayleigh<<<grid_for(n), 256, 0, st>>>(Gm, Sm, n, ws.lam);
      count_launch(4);
      DG_CUDA(cudaGetLastError());
      // host tables must outlive the copies above
      DG_CUDA(cudaStreamSynchronize(st));
    }
    DG_CUDA(cudaMemsetAsync(ws.emax, 0, sizeof(unsigned long long), st));
    k_update_coeffs<<<dim3((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32)), dim3(32, 8), 0, st>>>(
        Gm, Sm, n, ws.lam, ws.cl, floor_gap, floor_num, kStop, ws.F, ws.emax);
    count_launch();
    DG_CUDA(cudaGetLastError());
    unsigned long long eb = 0;
    DG_CUDA(cudaMemcpyAsync(&eb, ws.emax, sizeof(eb), cudaMemcpyDeviceToHost, st));
    DG_CUDA(cudaStreamSynchronize(st));
    double emax = 0.0;
    std::memcpy(&emax, &eb, sizeof(emax));
    ctx->eig_steps = step + 1;
    ctx->eig_update = emax;
    if (step < 16) ctx->eig_history[step] = emax;
    if (!(emax < 1.0)) {
      *reason = 4;
      return DGCHEFSI_OK;
    }
    // the block of V that differs from I: the first step's block and this
    // step's cluster rows (the rotations mixed only those rows)
    int64_t mb = 0;
    if (block && !unit) {
      std::vector<char> in(n, 0);
      for (int r : rows) in[r] = 1;
      for (int q = 0; q < cofs_h[ncl]; ++q) in[idx_h[q]] = 1;
      blk_h.clear();
      for (int64_t i = 0; i < n; ++i)
        if (in[i]) blk_h.push_back((int)i);
      mb = (int64_t)blk_h.size();
      if (4 * mb > n) mb = 0;
    }
    if (unit && ncl == 0) {
      DG_CUDA(axpby_f64(1.0, ws.F, 1.0, V, V, nn, st));  // V <- I + E^T
    } else if (mb > 0) {
      // V <- V + E^T V: outside the block's columns E^T V = E^T; on them
      // E^T[:, B] V[B, B], and V[:, B] is zero outside the rows B
      std::fill(pos_h.begin(), pos_h.end(), -1);
      for (int64_t k = 0; k < mb; ++k) pos_h[blk_h[k]] = (int)k;
      DG_CUDA(cudaMemcpyAsync(ws.perm, blk_h.data(), sizeof(int) * (size_t)mb, cudaMemcpyHostToDevice, st));
      DG_CUDA(cudaMemcpyAsync(ws.posb, pos_h.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, st));
      double* VB = T;            // mb x mb
      double* FB = T + mb * mb;  // n x mb
      double* FV = FB + n * mb;  // n x mb
      k_gather_block_of<<<grid_for(mb * mb), 256, 0, st>>>(V, n, ws.perm, mb, VB);
      k_gather_cols_of<<<grid_for(mb * n), 256, 0, st>>>(ws.F, n, ws.perm, mb, n, FB);
      count_launch(2);
      DG_CUDA(gemm_nn_f64(FB, mb, VB, mb, FV, mb, n, mb, mb, false, st));
      DG_CUDA(axpby_f64(1.0, ws.F, 1.0, V, V, nn, st));
      k_scatter_cols_of<<<grid_for(mb * n), 256, 0, st>>>(V, n, ws.perm, mb, n, FV, ws.posb, VB);
      count_launch();
      DG_CUDA(cudaGetLastError());
      DG_CUDA(cudaStreamSynchronize(st));  // the host tables above are pageable copies' sources
    } else {
      // E^T V with the slices its size needs: the splitting error is at most
      // L max|F| max|V| 2^{-6s'} (s' + 4) per K chunk of length L (sliced.cu),
      // max|F| = emax and max|V| < 2, so 2^{-6s'} (s' + 4) 2 emax <= 2^-53
      // keeps it below u L, FP64's own bound for a product of V's size
      const int su = update_slices(emax, s);
      if (step < 16) ctx->eig_slices_history[step] = su;
      DG_TRY(sliced_gemm(ctx, false, false, n, n, n, ws.F, n, V, n, ws.GS, n, su, bad));  // E^T V
      DG_CUDA(axpby_f64(1.0, ws.GS, 1.0, V, V, nn, st));                                   // V <- V + E^T V
    }
    unit = false;
    block = false;
    // stop when this correction is small, or when the quadratic rate seen
    // over the last two steps puts the next one below kPredict
    const double rate = prev > 0.0 ? std::max(1.0, emax / (prev * prev)) : 0.0;
    converged = emax <= kStop || (prev > 0.0 && rate * emax * emax <= kPredict);
    prev = emax;
  }
  if (!converged) {
    *reason = 5;
    return DGCHEFSI_OK;
  }
  // ascending order: rows of V and their Rayleigh quotients gathered into A and w
  int nonfinite = 0;
  DG_CUDA(cudaMemcpyAsync(lam_h.data(), ws.lam, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, st));
  DG_CUDA(cudaMemcpyAsync(&nonfinite, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  DG_CUDA(cudaStreamSynchronize(st));
  if (nonfinite != 0) {
    *reason = 4;
    return DGCHEFSI_OK;
  }
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lam_h[a] < lam_h[b]; });
  DG_CUDA(cudaMemcpyAsync(ws.perm, order.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, st));
  k_gather_rows<<<dim3(grid_for(n), (unsigned)std::min<int64_t>(n, 65535)), 256, 0, st>>>(V, n, ws.perm, ws.lam, A,
                                                                                        lda, w);
  count_launch();
  DG_CUDA(cudaGetLastError());
  DG_CUDA(cudaStreamSynchronize(st));
  ctx->eig_refine_ms = ms_since(t0) - ctx->eig_start_ms;
  return DGCHEFSI_OK;
}

}  // namespace

dgchefsi_status subspace_eigh(dgchefsi_ctx* ctx, double* A, int64_t n, int64_t lda, double* w) {
  ctx->eig_steps = 0;
  ctx->eig_max_cluster = 0;
  ctx->eig_fallback = 0;
  ctx->eig_update = 0.0;
  ctx->eig_start_ms = ctx->eig_refine_ms = 0.0;
  ctx->eig_start_order = 0;
  ctx->eig_start_solver = 0;
  for (double& h : ctx->eig_history) h = 0.0;
  for (int& h : ctx->eig_slices_history) h = 0;
  ctx->eig_used = DGCHEFSI_EIG_SYEVD;
  if (n <= 0) return DGCHEFSI_OK;
  int mode = ctx->eig_mode;
  if (mode == DGCHEFSI_EIG_AUTO)
    mode = ctx->products_mode == DGCHEFSI_PRODUCTS_SLICED_BF16 && n >= 256 ? DGCHEFSI_EIG_REFINED : DGCHEFSI_EIG_SYEVD;
  if (mode == DGCHEFSI_EIG_REFINED && n >= 2) {
    int reason = 0;
    DG_TRY(eig_refined(ctx, A, n, lda, w, &reason));
    if (reason == 0) {
      ctx->eig_used = DGCHEFSI_EIG_REFINED;
      return DGCHEFSI_OK;
    }
    ctx->eig_fallback = reason;  // A's lower triangle is intact
  }
  return eig_syevd(ctx, A, n, lda, w);
}

}  // namespace dg
