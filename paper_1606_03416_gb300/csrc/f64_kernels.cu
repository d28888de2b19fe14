// FP64 kernels of the CheFSI cycle: block-sparse mat-vec with the Chebyshev
// recurrence fused into its epilogue (Alg. 1 step 2, Eq. matvec_3), the
// Lanczos vector operations (Alg. 1 step 1), the dense FP64 products of the
// subspace problem (Alg. 1 steps 3-5), the Fermi level and occupations, and the
// diagonal density blocks (Eq. densitymatrix).
//
// GB300 executes FP64 only on the CUDA-core DFMA pipe (tcgen05 has no FP64
// kind), at a small fraction of the tensor rate, so these kernels are
// ALU-bound by a wide margin: a 64x64 output tile per 256-thread CTA, 4x4
// register blocking, operands staged through shared memory in 16-deep slices.
#include <atomic>
#include <cmath>

#include "internal.h"

namespace dg {

static std::atomic<int64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

namespace {

constexpr int T = 64;       // output tile edge
constexpr int BK = 16;      // contraction slice
constexpr int TP = T + 1;   // padded shared-memory row
constexpr int NT = 256;     // threads per CTA (16 x 16, 4x4 outputs each)

__device__ __forceinline__ void fma_tile(const double (&As)[BK][TP], const double (&Bs)[BK][TP],
                                         double (&acc)[4][4], int tx, int ty) {
#pragma unroll
  for (int kk = 0; kk < BK; ++kk) {
    double a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  }
}

// One Chebyshev step on a (64 states) x (TJ rows of element K) tile:
// out = alpha * (sum_{K'} H_KK' in_K' - c in_K) - beta * prev_K.
// TJ = 64 when every element size is a multiple of 64, else 32, so uneven
// elements leave fewer idle columns in their last tile.
template <int TJ>
__global__ void __launch_bounds__(NT) k_filter_step_f64(HView h, const double* __restrict__ in, int64_t ld,
                                                        const double* prev, double* out, int64_t ldo,
                                                        int64_t Ns, double alpha, double c, double beta,
                                                        const double* __restrict__ coef, int step) {
  constexpr int JR = TJ / 16;  // output columns per thread
  if (coef) {  // coefficients in device memory ([c, alpha_0, beta_0, alpha_1, ...]; graph replays)
    c = coef[0];
    alpha = coef[1 + 2 * step];
    beta = coef[2 + 2 * step];
  }
  const int K = blockIdx.y;
  const int nK = h.nb[K];
  const int j0 = blockIdx.z * TJ;
  if (j0 >= nK) return;
  const int64_t s0 = (int64_t)blockIdx.x * T;
  __shared__ double As[BK][TP];
  __shared__ double Bs[BK][TJ + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][JR];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < JR; ++j) acc[i][j] = 0.0;
  const int64_t offK = h.off[K];
  const int64_t e_end = h.row_ptr[K + 1];
  for (int64_t e = h.row_ptr[K]; e < e_end; ++e) {
    const int Kp = h.col[e];
    const int nKp = h.nb[Kp];
    const int64_t offKp = h.off[Kp];
    const double* blk = h.vals + h.blk_off[e];
    for (int k0 = 0; k0 < nKp; k0 += BK) {
      const int kk = tid & 15;
      const bool kin = (k0 + kk) < nKp;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = (tid >> 4) + 16 * i;
        As[kk][r] = (kin && s0 + r < Ns) ? in[(s0 + r) * ld + offKp + k0 + kk] : 0.0;
      }
#pragma unroll
      for (int i = 0; i < JR; ++i) {
        const int r = (tid >> 4) + 16 * i;
        Bs[kk][r] = (kin && j0 + r < nK) ? blk[(int64_t)(j0 + r) * nKp + k0 + kk] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < BK; ++q) {
        double a[4], b[JR];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[q][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < JR; ++j) b[j] = Bs[q][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < JR; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t s = s0 + ty + 16 * i;
    if (s >= Ns) continue;
#pragma unroll
    for (int j = 0; j < JR; ++j) {
      const int jj = j0 + tx + 16 * j;
      if (jj >= nK) continue;
      const int64_t idx = s * ldo + offK + jj;
      double r = alpha * (acc[i][j] - c * in[s * ld + offK + jj]);
      if (beta != 0.0) r -= beta * prev[idx];
      out[idx] = r;
    }
  }
}

// y = H x: one warp per row of H, lanes stride over each neighbour block's row.
__global__ void k_spmv_f64(HView h, const double* __restrict__ x, double* __restrict__ y) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= h.N) return;
  int lo = 0, hi = h.M;  // find K with off[K] <= row < off[K+1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (h.off[mid] <= row) lo = mid; else hi = mid;
  }
  const int K = lo;
  const int j = (int)(row - h.off[K]);
  double sum = 0.0;
  for (int64_t e = h.row_ptr[K]; e < h.row_ptr[K + 1]; ++e) {
    const int Kp = h.col[e];
    const int nKp = h.nb[Kp];
    const double* brow = h.vals + h.blk_off[e] + (int64_t)j * nKp;
    const double* xs = x + h.off[Kp];
    for (int jp = lane; jp < nKp; jp += 32) sum = fma(brow[jp], xs[jp], sum);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) y[row] = sum;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  const int tid = threadIdx.x;
  red[tid] = v;
  __syncthreads();
  for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
    if (tid < s) red[tid] += red[tid + s];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

__global__ void k_dots_f64(const double* __restrict__ V, int64_t ldv, const double* __restrict__ w, int64_t n,
                           double* __restrict__ out) {
  __shared__ double red[256];
  const double* v = V + (int64_t)blockIdx.x * ldv;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(v[i], w[i], s);
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) out[blockIdx.x] = t;
}

__global__ void k_sub_combination_f64(double* __restrict__ w, const double* __restrict__ V, int64_t ldv,
                                      const double* __restrict__ coef, int nv, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int l = 0; l < nv; ++l) acc = fma(coef[l], V[(int64_t)l * ldv + i], acc);
    w[i] -= acc;
  }
}

__global__ void k_axpby_f64(double a, const double* __restrict__ x, double b, const double* y, double* yo, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    yo[i] = a * x[i] + b * y[i];
}

// C[i,j] = sum_r A[i,r] B[j,r]
__global__ void __launch_bounds__(NT) k_gemm_nt_f64(const double* __restrict__ A, int64_t lda,
                                                    const double* __restrict__ B, int64_t ldb, double* C,
                                                    int64_t ldc, int64_t rows, int64_t cols, int64_t K,
                                                    int lower_only) {
  if (lower_only && blockIdx.x > blockIdx.y) return;
  const int64_t i0 = (int64_t)blockIdx.y * T, j0 = (int64_t)blockIdx.x * T;
  __shared__ double As[BK][TP];
  __shared__ double Bs[BK][TP];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int64_t k0 = 0; k0 < K; k0 += BK) {
    const int kk = tid & 15;
    const bool kin = (k0 + kk) < K;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = (tid >> 4) + 16 * i;
      double v = 0.0, w = 0.0;
      if (kin && i0 + r < rows) v = A[(i0 + r) * lda + k0 + kk];
      if (kin && j0 + r < cols) w = B[(j0 + r) * ldb + k0 + kk];
      As[kk][r] = v;
      Bs[kk][r] = w;
    }
    __syncthreads();
    fma_tile(As, Bs, acc, tx, ty);
    __syncthreads();
  }
  const bool mirror = lower_only && blockIdx.x < blockIdx.y;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t ii = i0 + ty + 16 * i;
    if (ii >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t jj = j0 + tx + 16 * j;
      if (jj >= cols) continue;
      C[ii * ldc + jj] = acc[i][j];
      if (mirror) C[jj * ldc + ii] = acc[i][j];
    }
  }
}

__global__ void k_symmetrise_f64(double* C, int64_t n, int64_t ldc) {
  const int64_t i = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || j >= n || j <= i) return;
  const double v = 0.5 * (C[i * ldc + j] + C[j * ldc + i]);
  C[i * ldc + j] = v;
  C[j * ldc + i] = v;
}

// C[i,r] = sum_l A[i,l] B[l,r]
__global__ void __launch_bounds__(NT) k_gemm_nn_f64(const double* __restrict__ A, int64_t lda,
                                                    const double* __restrict__ B, int64_t ldb,
                                                    double* __restrict__ C, int64_t ldc, int64_t rows,
                                                    int64_t cols, int64_t K, int a_lower) {
  const int64_t i0 = (int64_t)blockIdx.y * T, r0 = (int64_t)blockIdx.x * T;
  __shared__ double As[BK][TP];
  __shared__ double Bs[BK][TP];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const int64_t kend = a_lower ? (K < i0 + T ? K : i0 + T) : K;
  for (int64_t k0 = 0; k0 < kend; k0 += BK) {
    {
      const int kk = tid & 15;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = (tid >> 4) + 16 * i;
        const int64_t l = k0 + kk, row = i0 + r;
        double v = 0.0;
        if (l < K && row < rows && (!a_lower || l <= row)) v = A[row * lda + l];
        As[kk][r] = v;
      }
    }
    {
      const int cc = tid & 63;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int kk = (tid >> 6) + 4 * i;
        const int64_t l = k0 + kk;
        double w = 0.0;
        if (l < K && r0 + cc < cols) w = B[l * ldb + r0 + cc];
        Bs[kk][cc] = w;
      }
    }
    __syncthreads();
    fma_tile(As, Bs, acc, tx, ty);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t ii = i0 + ty + 16 * i;
    if (ii >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t rr = r0 + tx + 16 * j;
      if (rr < cols) C[ii * ldc + rr] = acc[i][j];
    }
  }
}

// P_K[j, j'] = sum_i f_i X[i, off_K + j] X[i, off_K + j']
__global__ void __launch_bounds__(NT) k_density_f64(HView h, const int64_t* __restrict__ poff,
                                                    const double* __restrict__ X, int64_t Ns, int64_t ld,
                                                    const double* __restrict__ f, double* __restrict__ P) {
  const int K = blockIdx.x;
  const int nK = h.nb[K];
  const int j0 = blockIdx.y * T, jp0 = blockIdx.z * T;
  if (j0 >= nK || jp0 >= nK) return;
  const int64_t offK = h.off[K];
  __shared__ double As[BK][TP];
  __shared__ double Bs[BK][TP];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const int cc = tid & 63;
  for (int64_t i0 = 0; i0 < Ns; i0 += BK) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int kk = (tid >> 6) + 4 * i;
      const int64_t s = i0 + kk;
      double v = 0.0, w = 0.0;
      if (s < Ns) {
        const double* xr = X + s * ld + offK;
        if (j0 + cc < nK) v = f[s] * xr[j0 + cc];
        if (jp0 + cc < nK) w = xr[jp0 + cc];
      }
      As[kk][cc] = v;
      Bs[kk][cc] = w;
    }
    __syncthreads();
    fma_tile(As, Bs, acc, tx, ty);
    __syncthreads();
  }
  double* PK = P + poff[K];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int jj = j0 + ty + 16 * i;
    if (jj >= nK) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int jq = jp0 + tx + 16 * j;
      if (jq < nK) PK[(int64_t)jj * nK + jq] = acc[i][j];
    }
  }
}

__device__ __forceinline__ double fermi(double x) {
  if (x > 0.0) {
    const double e = exp(-x);
    return e / (1.0 + e);
  }
  return 1.0 / (1.0 + exp(x));
}

// Fermi level by bisection and occupations; one CTA of 256 threads.
__global__ void __launch_bounds__(256) k_occupations_f64(const double* __restrict__ lam, int64_t Ns, double Ne,
                                                        double kT, double* __restrict__ f, double* __restrict__ mu_out) {
  __shared__ double red[256];
  double vmin = INFINITY, vmax = -INFINITY;
  for (int64_t i = threadIdx.x; i < Ns; i += blockDim.x) {
    vmin = fmin(vmin, lam[i]);
    vmax = fmax(vmax, lam[i]);
  }
  red[threadIdx.x] = vmin;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  double lo = red[0] - 50.0 * kT;
  __syncthreads();
  red[threadIdx.x] = vmax;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  double hi = red[0] + 50.0 * kT;
  __syncthreads();
  const double tol = 1e-13 * Ne;
  double mu = 0.5 * (lo + hi);
  for (int it = 0; it < 200; ++it) {
    mu = 0.5 * (lo + hi);
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < Ns; i += blockDim.x) s += fermi((lam[i] - mu) / kT);
    const double count = 2.0 * block_sum(s, red);
    if (fabs(count - Ne) <= tol) break;
    if (count < Ne) lo = mu; else hi = mu;
  }
  for (int64_t i = threadIdx.x; i < Ns; i += blockDim.x) f[i] = fermi((lam[i] - mu) / kT);
  if (threadIdx.x == 0) *mu_out = mu;
}

__global__ void k_shift_diag_f64(double* A, int64_t n, double coef) {
  __shared__ double red[256];
  double t = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) t += A[i * n + i];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double sft = coef * red[0];
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) A[i * n + i] += sft;
}

__global__ void k_zero_strict_upper_f64(double* A, int64_t n, int64_t lda) {
  const int64_t i = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && j < n && j > i) A[i * lda + j] = 0.0;
}

__global__ void k_check_finite_f64(const double* __restrict__ x, int64_t n, int* flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) atomicOr(flag, 1);
}


// G_e += alpha * sum_s w_s A[s, off_K + j] B[s, off_K' + j'] for every stored
// block e = (K, K') (w may be null: unit weights).
__global__ void __launch_bounds__(NT) k_block_outer_f64(HView h, const int32_t* __restrict__ blk_row,
                                                        const double* __restrict__ A, int64_t lda,
                                                        const double* __restrict__ B, int64_t ldb,
                                                        const double* __restrict__ w, double alpha, int64_t Ns,
                                                        double* __restrict__ G) {
  const int64_t e = blockIdx.x;
  const int K = blk_row[e], Kp = h.col[e];
  const int nK = h.nb[K], nKp = h.nb[Kp];
  const int j0 = blockIdx.y * T, jp0 = blockIdx.z * T;
  if (j0 >= nK || jp0 >= nKp) return;
  const int64_t offK = h.off[K], offKp = h.off[Kp];
  __shared__ double As[BK][TP];
  __shared__ double Bs[BK][TP];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const int cc = tid & 63;
  for (int64_t i0 = 0; i0 < Ns; i0 += BK) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int kk = (tid >> 6) + 4 * i;
      const int64_t s = i0 + kk;
      double v = 0.0, u = 0.0;
      if (s < Ns) {
        if (j0 + cc < nK) v = (w ? w[s] : 1.0) * A[s * lda + offK + j0 + cc];
        if (jp0 + cc < nKp) u = B[s * ldb + offKp + jp0 + cc];
      }
      As[kk][cc] = v;
      Bs[kk][cc] = u;
    }
    __syncthreads();
    fma_tile(As, Bs, acc, tx, ty);
    __syncthreads();
  }
  double* Ge = G + h.blk_off[e];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int jj = j0 + ty + 16 * i;
    if (jj >= nK) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int jq = jp0 + tx + 16 * j;
      if (jq < nKp) Ge[(int64_t)jj * nKp + jq] += alpha * acc[i][j];
    }
  }
}

// C[i,r] = sum_l A[l,i] B[l,r]  (A: K x rows, B: K x cols, both row-major)
__global__ void __launch_bounds__(NT) k_gemm_tn_f64(const double* __restrict__ A, int64_t lda,
                                                    const double* __restrict__ B, int64_t ldb,
                                                    double* __restrict__ C, int64_t ldc, int64_t rows,
                                                    int64_t cols, int64_t K) {
  const int64_t i0 = (int64_t)blockIdx.y * T, r0 = (int64_t)blockIdx.x * T;
  __shared__ double As[BK][TP];
  __shared__ double Bs[BK][TP];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const int cc = tid & 63;
  for (int64_t k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int kk = (tid >> 6) + 4 * i;
      const int64_t l = k0 + kk;
      double v = 0.0, u = 0.0;
      if (l < K) {
        if (i0 + cc < rows) v = A[l * lda + i0 + cc];
        if (r0 + cc < cols) u = B[l * ldb + r0 + cc];
      }
      As[kk][cc] = v;
      Bs[kk][cc] = u;
    }
    __syncthreads();
    fma_tile(As, Bs, acc, tx, ty);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t ii = i0 + ty + 16 * i;
    if (ii >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t rr = r0 + tx + 16 * j;
      if (rr < cols) C[ii * ldc + rr] = acc[i][j];
    }
  }
}

// out[i, r] = scale * g[i] * (HX[i, r] - lam[i] * X[i, r]) for r < n
__global__ void k_scaled_residual_f64(const double* __restrict__ HX, const double* __restrict__ X, int64_t ld,
                                      const double* __restrict__ lam, const double* __restrict__ g, double scale,
                                      int64_t Ns, int64_t n, double* __restrict__ out, int64_t ldo) {
  const int64_t i = blockIdx.y;
  if (i >= Ns) return;
  const double gi = scale * g[i], li = lam[i];
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    out[i * ldo + r] = gi * (HX[i * ld + r] - li * X[i * ld + r]);
}

inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }
inline unsigned stream_grid(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t filter_step_f64(const HView& h, const double* in, int64_t ld_in, const double* prev, double* out,
                            int64_t ld_out, int64_t Ns, double alpha, double c, double beta, cudaStream_t s) {
  if (Ns == 0) return cudaSuccess;
  if (h.tj == 64)
    k_filter_step_f64<64><<<dim3(cdiv(Ns, T), (unsigned)h.M, cdiv(h.max_nb, 64)), NT, 0, s>>>(
        h, in, ld_in, prev, out, ld_out, Ns, alpha, c, beta, nullptr, 0);
  else
    k_filter_step_f64<32><<<dim3(cdiv(Ns, T), (unsigned)h.M, cdiv(h.max_nb, 32)), NT, 0, s>>>(
        h, in, ld_in, prev, out, ld_out, Ns, alpha, c, beta, nullptr, 0);
  count_launch();
  return cudaGetLastError();
}

cudaError_t filter_step_f64_dev(const HView& h, const double* in, int64_t ld_in, const double* prev, double* out,
                                int64_t ld_out, int64_t Ns, const double* coef, int step, cudaStream_t s) {
  if (Ns <= 0) return cudaSuccess;
  if (h.tj == 64)
    k_filter_step_f64<64><<<dim3(cdiv(Ns, T), (unsigned)h.M, cdiv(h.max_nb, 64)), NT, 0, s>>>(
        h, in, ld_in, prev, out, ld_out, Ns, 0.0, 0.0, 0.0, coef, step);
  else
    k_filter_step_f64<32><<<dim3(cdiv(Ns, T), (unsigned)h.M, cdiv(h.max_nb, 32)), NT, 0, s>>>(
        h, in, ld_in, prev, out, ld_out, Ns, 0.0, 0.0, 0.0, coef, step);
  count_launch();
  return cudaGetLastError();
}

// FP64 issue-rate probe: 8 independent DFMA chains per thread, nothing read
// from memory; the store happens only if the result hits a value it cannot
// take, which keeps the chains live without memory traffic.
__global__ void __launch_bounds__(256) k_dfma_rate(int64_t iters, double x, double* __restrict__ sink) {
  double a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = 1.0 + 1e-3 * (threadIdx.x + i);
  const double y = -0.5 * x;
  for (int64_t n = 0; n < iters; ++n) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fma(a[i], x, y);
  }
  double t = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) t += a[i];
  if (t == 1234.5678) sink[0] = t;
}

cudaError_t dfma_rate(int64_t iters, int blocks, double* sink, cudaStream_t s) {
  k_dfma_rate<<<blocks, 256, 0, s>>>(iters, 0.999999, sink);
  count_launch();
  return cudaGetLastError();
}

cudaError_t preload_lanczos_kernels() {
  // cudaFuncGetAttributes loads a kernel's module on a lazily loading runtime,
  // so a later launch of these kernels allocates no device memory for code.
  cudaFuncAttributes a;
  cudaError_t e;
  if ((e = cudaFuncGetAttributes(&a, k_spmv_f64)) != cudaSuccess) return e;
  if ((e = cudaFuncGetAttributes(&a, k_dots_f64)) != cudaSuccess) return e;
  if ((e = cudaFuncGetAttributes(&a, k_sub_combination_f64)) != cudaSuccess) return e;
  return cudaFuncGetAttributes(&a, k_axpby_f64);
}

cudaError_t spmv_f64(const HView& h, const double* x, double* y, cudaStream_t s) {
  const int64_t threads = h.N * 32;
  k_spmv_f64<<<cdiv(threads, 256), 256, 0, s>>>(h, x, y);
  count_launch();
  return cudaGetLastError();
}

cudaError_t dots_f64(const double* V, int64_t ldv, int nv, const double* w, int64_t n, double* out, cudaStream_t s) {
  if (nv <= 0) return cudaSuccess;
  k_dots_f64<<<nv, 256, 0, s>>>(V, ldv, w, n, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t sub_combination_f64(double* w, const double* V, int64_t ldv, const double* coef, int nv, int64_t n,
                                cudaStream_t s) {
  if (nv <= 0) return cudaSuccess;
  k_sub_combination_f64<<<stream_grid(n), 256, 0, s>>>(w, V, ldv, coef, nv, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t axpby_f64(double a, const double* x, double b, const double* y, double* y_out, int64_t n,
                      cudaStream_t s) {
  k_axpby_f64<<<stream_grid(n), 256, 0, s>>>(a, x, b, y, y_out, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t gemm_nt_f64(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                        int64_t rows, int64_t cols, int64_t K, bool lower_only, bool symmetrise, cudaStream_t s) {
  if (rows == 0 || cols == 0) return cudaSuccess;
  dim3 grid(cdiv(cols, T), cdiv(rows, T));
  k_gemm_nt_f64<<<grid, NT, 0, s>>>(A, lda, B, ldb, C, ldc, rows, cols, K, lower_only ? 1 : 0);
  count_launch();
  if (symmetrise && rows == cols) {
    dim3 b2(32, 8), g2(cdiv(rows, 32), cdiv(rows, 8));
    k_symmetrise_f64<<<g2, b2, 0, s>>>(C, rows, ldc);
    count_launch();
  }
  return cudaGetLastError();
}

cudaError_t gemm_nn_f64(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                        int64_t rows, int64_t cols, int64_t K, bool a_lower, cudaStream_t s) {
  if (rows == 0 || cols == 0) return cudaSuccess;
  dim3 grid(cdiv(cols, T), cdiv(rows, T));
  k_gemm_nn_f64<<<grid, NT, 0, s>>>(A, lda, B, ldb, C, ldc, rows, cols, K, a_lower ? 1 : 0);
  count_launch();
  return cudaGetLastError();
}

cudaError_t density_f64(const HView& h, const int64_t* poff, const double* X, int64_t Ns, int64_t ld,
                        const double* f, double* P, cudaStream_t s) {
  dim3 grid((unsigned)h.M, cdiv(h.max_nb, T), cdiv(h.max_nb, T));
  k_density_f64<<<grid, NT, 0, s>>>(h, poff, X, Ns, ld, f, P);
  count_launch();
  return cudaGetLastError();
}

cudaError_t occupations_f64(const double* ritz, int64_t Ns, double Ne, double kT, double* f, double* mu,
                            cudaStream_t s) {
  k_occupations_f64<<<1, 256, 0, s>>>(ritz, Ns, Ne, kT, f, mu);
  count_launch();
  return cudaGetLastError();
}

cudaError_t shift_diagonal_by_trace_f64(double* A, int64_t n, double coef, cudaStream_t s) {
  k_shift_diag_f64<<<1, 256, 0, s>>>(A, n, coef);
  count_launch();
  return cudaGetLastError();
}

cudaError_t zero_strict_upper_f64(double* A, int64_t n, int64_t lda, cudaStream_t s) {
  dim3 b(32, 8), g(cdiv(n, 32), cdiv(n, 8));
  k_zero_strict_upper_f64<<<g, b, 0, s>>>(A, n, lda);
  count_launch();
  return cudaGetLastError();
}


cudaError_t block_outer_f64(const HView& h, const int32_t* blk_row, int64_t nnzb, const double* A, int64_t lda,
                            const double* B, int64_t ldb, const double* w, double alpha, int64_t Ns, double* G,
                            cudaStream_t s) {
  if (nnzb == 0) return cudaSuccess;
  dim3 grid((unsigned)nnzb, cdiv(h.max_nb, T), cdiv(h.max_nb, T));
  k_block_outer_f64<<<grid, NT, 0, s>>>(h, blk_row, A, lda, B, ldb, w, alpha, Ns, G);
  count_launch();
  return cudaGetLastError();
}

cudaError_t gemm_tn_f64(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                        int64_t rows, int64_t cols, int64_t K, cudaStream_t s) {
  if (rows == 0 || cols == 0) return cudaSuccess;
  dim3 grid(cdiv(cols, T), cdiv(rows, T));
  k_gemm_tn_f64<<<grid, NT, 0, s>>>(A, lda, B, ldb, C, ldc, rows, cols, K);
  count_launch();
  return cudaGetLastError();
}

cudaError_t scaled_residual_f64(const double* HX, const double* X, int64_t ld, const double* lam, const double* g,
                                double scale, int64_t Ns, int64_t n, double* out, int64_t ldo, cudaStream_t s) {
  if (Ns == 0) return cudaSuccess;
  dim3 grid(cdiv(n, 256) > 64 ? 64 : cdiv(n, 256), (unsigned)Ns);
  k_scaled_residual_f64<<<grid, 256, 0, s>>>(HX, X, ld, lam, g, scale, Ns, n, out, ldo);
  count_launch();
  return cudaGetLastError();
}

cudaError_t check_finite_f64(const double* x, int64_t n, int* flag, cudaStream_t s) {
  k_check_finite_f64<<<stream_grid(n), 256, 0, s>>>(x, n, flag);
  count_launch();
  return cudaGetLastError();
}

}  // namespace dg
