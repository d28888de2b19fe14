// FP64 products of the Rayleigh-Ritz step (Alg. 1 steps 3-5: Gram matrix,
// Y U^{-1}, projected H, rotation) emulated on the BF16 tensor cores by exact
// splitting (the Ozaki scheme: Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59,
// 2012; BF16/FP16 tensor-core form after Mukunoki, Ozaki, Ogita, Imamura,
// ISC 2020).
//
// Over one K chunk of length L <= 4096, row r of A is written as
//   a[r,k] = 2^{e_r} sum_{i<s} q_i[r,k] 2^{-6(i+1)},  q_i integer, |q_0| <= 64, |q_i| <= 32,
// with 2^{e_r} > max_k |a[r,k]| (and likewise each column of the product's
// right operand with exponent f_c). Every q is exact in BF16, every product
// q_i q_j is at most 2^12, so a slice-pair product summed over L <= 4096 terms
// is an integer of magnitude <= 2^24: the tensor core's FP32 accumulation
// returns it exactly, whatever its summation order. The pairs with
// i + j <= s - 1 are kept; their FP32 results are summed per t = i + j in FP64
// (exact: integers below 2^53), combined by Horner in 2^{-6}, scaled by
// 2^{e_r + f_c - 12} and added over the chunks. The slice-pair products run
// on this library's tcgen05 kernel for pairs of SMs (pair_gemm.cu: 256 x 256
// tiles, every pair of a chunk in one persistent launch, FP32 slabs);
// splitting and the FP64 reduction are the kernels below.
//
// Error per chunk (row and column maxima m_r, n_c over the chunk): the
// remainders after s slices and the dropped pairs contribute at most
// L 2^{e_r + f_c} 2^{-6s} (s + 4)/4 <= L m_r n_c 2^{-6s} (s + 4); the FP64
// Horner sum and the sum over chunks add at most (5 + chunks) u L m_r n_c,
// u = 2^{-53}. For s = 10 the splitting term is below u L m_r n_c, the size of
// FP64's own worst-case bound. The bound is normwise per row and column:
// entries far below their row's maximum keep fewer significant bits than FP64.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <climits>

#include "ctx.h"

namespace dg {

static constexpr int kBeta = 6;      // bits per slice
static constexpr int64_t kL = 4096;  // K chunk: 4096 * 2^12 = 2^24

__device__ __forceinline__ void atomic_flag(int* flag) {
  if (flag) atomicOr(flag, 1);
}

// |x| = M 2^{E - 1075} with M normalised to [2^52, 2^53) (subnormals too).
// Returns 0 for zero, 1 for a finite nonzero x, 2 for NaN/Inf. The frexp
// exponent of x (|x| = f 2^e, f in [0.5, 1)) is E - 1022.
__device__ __forceinline__ int decompose(double x, int64_t& M, int& E) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int Eb = (int)((u >> 52) & 0x7ff);
  const long long m = (long long)(u & 0xfffffffffffffULL);
  if (Eb == 0x7ff) return 2;
  if (Eb == 0) {
    if (m == 0) return 0;
    const int sh = __clzll(m) - 11;  // bring the leading bit to position 52
    M = m << sh;
    E = 1 - sh;
    return 1;
  }
  M = m | (1LL << 52);
  E = Eb;
  return 1;
}

// Slices of v = x 2^{-e'} (|v| < 1), where x = (-1)^neg M 2^{E - 1075} and
// base = -1075 - e' + 6s, s <= 10: F = round(v 2^{6s}) as a 64-bit integer
// (|F| <= 2^60, |v 2^{6s} - F| <= 1/2), then its balanced base-64 digits
// q_{s-1}, ..., q_1 in [-32, 31] and the leading q_0 = the rest, |q_0| <= 64;
// v = sum_i q_i 2^{-6(i+1)} up to 2^{-6s}/2. Integer arithmetic only.
__device__ __forceinline__ void slice_fixed(int64_t M, int E, bool neg, int base, int s,
                                            __nv_bfloat16* __restrict__ q, int64_t stride) {
  const int sh = E + base;
  int64_t F = 0;
  if (M != 0) {
    if (sh >= 0)
      F = M << sh;
    else if (sh > -54)
      F = (M + (1LL << (-sh - 1))) >> (-sh);
  }
  if (neg) F = -F;
  for (int i = s - 1; i >= 1; --i) {
    const int64_t d = ((F + 32) & 63) - 32;
    q[i * stride] = __float2bfloat16_rn((float)(int)d);
    F = (F - d) >> 6;
  }
  q[0] = __float2bfloat16_rn((float)(int)F);
}

// The same digits for s > 10 (F would not fit 64 bits): v is scaled in FP64,
// each digit rounded to nearest and subtracted (every step exact).
__device__ __forceinline__ void slice_fp64(double v, int s, __nv_bfloat16* __restrict__ q, int64_t stride) {
  double r = v;
  for (int i = 0; i < s; ++i) {
    r *= 64.0;
    const double d = rint(r);
    r -= d;
    q[i * stride] = __float2bfloat16_rn((float)d);
  }
}

__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// One CTA per (row, chunk), 256 threads, 16 entries each. Q: s slices of
// rows x ldq BF16 (slice i at Q + i * sstride); E[row * nch + chunk] = e_r, the
// frexp exponent of the row's largest |entry| in the chunk (0 if all are zero).
// lower: entries k > row are zero (a lower-triangular operand). bal (may be
// null): entry k is split as X[row, k] 2^{bal[k]}. A row chunk holding NaN/Inf
// gets zero slices and raises flag.
__global__ void __launch_bounds__(256) k_split_rows(const double* __restrict__ X, int64_t ldx, int64_t K, int s,
                                                    int lower, const int32_t* __restrict__ bal,
                                                    __nv_bfloat16* __restrict__ Q, int64_t ldq, int64_t sstride,
                                                    int32_t* __restrict__ E, int nch, int* __restrict__ flag) {
  const int64_t row = blockIdx.x;
  const int chunk = blockIdx.y;
  const int64_t k0 = (int64_t)chunk * kL;
  double v[16];
  int emax = INT_MIN;
  bool bad = false;
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int64_t k = k0 + threadIdx.x + 256 * u;
    double x = 0.0;
    if (k < K && !(lower && k > row)) x = X[row * ldx + k];
    v[u] = x;
    int64_t M;
    int Ex;
    const int c = decompose(x, M, Ex);
    if (c == 2) bad = true;
    if (c == 1) emax = max(emax, Ex + (bal ? bal[k] : 0));
  }
  __shared__ int red[8];
  __shared__ int sbad;
  if (threadIdx.x == 0) sbad = 0;
  emax = warp_max(emax);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = emax;
  if (bad) sbad = 1;
  __syncthreads();
  emax = red[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) emax = max(emax, red[w]);
  const bool zero = sbad != 0;
  const int e = (emax == INT_MIN || zero) ? 0 : emax - 1022;
  if (threadIdx.x == 0) {
    E[row * nch + chunk] = e;
    if (zero) atomic_flag(flag);
  }
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int64_t k = k0 + threadIdx.x + 256 * u;
    if (k >= K) break;
    __nv_bfloat16* q = Q + row * ldq + k;
    const int b = bal ? bal[k] : 0;
    if (s <= 10) {
      int64_t M = 0;
      int Ex = 0;
      if (zero || decompose(v[u], M, Ex) != 1) M = 0;
      slice_fixed(M, Ex + b, v[u] < 0.0, -1075 - e + 6 * s, s, q, sstride);
    } else {
      slice_fp64(zero ? 0.0 : ldexp(v[u], b - e), s, q, sstride);
    }
  }
}

// bal[k] = frexp exponent of max_c |X[k, c]| (X row-major K x C), 0 for a row
// with no finite nonzero entry, and nbal[k] = -bal[k]. One CTA per row.
__global__ void __launch_bounds__(256) k_row_exponents(const double* __restrict__ X, int64_t ldx, int64_t C,
                                                       int32_t* __restrict__ bal, int32_t* __restrict__ nbal) {
  const int64_t k = blockIdx.x;
  int emax = INT_MIN;
  for (int64_t c = threadIdx.x; c < C; c += 256) {
    int64_t M;
    int Ex;
    if (decompose(X[k * ldx + c], M, Ex) == 1) emax = max(emax, Ex);
  }
  emax = warp_max(emax);
  __shared__ int red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = emax;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) emax = max(emax, red[w]);
    emax = max(emax, red[0]);
    bal[k] = emax == INT_MIN ? 0 : emax - 1022;
    nbal[k] = -bal[k];
  }
}

// C[r, n0 + c] (+)= 2^{e_r + f_{n0+c} - 12} sum_t 2^{-6t} g_t,  g_t = sum_{i+j=t} P_{ij}[r, c],
// for r < M, c < P. Pair (i, j) is slab i*S - i(i-1)/2 + j of Pw (M x P FP32).
// Each P_ij is an exact integer of magnitude <= 2^24, so g_t is summed in
// int32 (|g_t| <= 16 * 2^24), five consecutive t are combined exactly in int64
// (< 2^53, exact in FP64), and the blocks meet in FP64: one rounding per 30
// bits of weight. Every slab value is loaded once, all loads of an output
// before any use, so the kernel streams Pw at memory speed.
// cmap (may be null): column c of the slabs goes to column cmap[c] of C, and
// is skipped when cmap[c] < 0 (the padding columns of the element-padded layout).
// tri > 0: only the entries with n0 + c <= r mod tri are formed (the slice-pair
// kernel left the tiles above that line out); the others are not read or written.
template <int S>
__global__ void __launch_bounds__(256) k_sliced_reduce(const float* __restrict__ Pw, int64_t M, int64_t P,
                                                       const int32_t* __restrict__ Ea, const int32_t* __restrict__ Eb,
                                                       int nch, int chunk, int64_t n0, double* __restrict__ C,
                                                       int64_t ldc, int accumulate, const int32_t* __restrict__ cmap,
                                                       int64_t tri) {
  constexpr int NB = (S + 4) / 5;  // blocks of five t
  const int64_t total = M * P;
  const int64_t slab = M * P;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    if (tri > 0 && n0 + idx % P > (idx / P) % tri) continue;
    int g[S];
#pragma unroll
    for (int t = 0; t < S; ++t) g[t] = 0;
#pragma unroll
    for (int i = 0; i < S; ++i)
#pragma unroll
      for (int j = 0; j < S - i; ++j)
        g[i + j] += __float2int_rn(__ldcs(Pw + (int64_t)(i * S - i * (i - 1) / 2 + j) * slab + idx));
    // h = sum_b B_b 2^{-30 b}, B_b = sum_{t = 5b}^{5b+4} g_t 2^{6(5b + 4 - t)}; sum_t g_t 2^{-6t} = h 2^{-24}
    double h = 0.0;
#pragma unroll
    for (int b = NB - 1; b >= 0; --b) {
      int64_t B = 0;
#pragma unroll
      for (int t = 5 * b; t < 5 * b + 5; ++t) B = B * 64 + (t < S ? (int64_t)g[t] : 0);
      h = h * 0x1p-30 + (double)B;
    }
    const int64_t r = idx / P;
    const int64_t c = idx - r * P;
    const int64_t oc = cmap ? (int64_t)cmap[c] : n0 + c;
    if (oc < 0) continue;
    const double v = ldexp(h, Ea[r * nch + chunk] + Eb[(n0 + c) * nch + chunk] - 12 - 24);
    double* out = C + r * ldc + oc;
    *out = accumulate ? *out + v : v;
  }
}

// The same for P % 4 == 0, four consecutive outputs per thread: one 16-byte
// load per slab instead of four 4-byte ones (same sums, same roundings).
template <int S>
__global__ void __launch_bounds__(256) k_sliced_reduce4(const float* __restrict__ Pw, int64_t M, int64_t P,
                                                        const int32_t* __restrict__ Ea, const int32_t* __restrict__ Eb,
                                                        int nch, int chunk, int64_t n0, double* __restrict__ C,
                                                        int64_t ldc, int accumulate, const int32_t* __restrict__ cmap,
                                                        int64_t tri) {
  constexpr int NB = (S + 4) / 5;
  const int64_t slab = M * P;
  const int64_t total4 = slab / 4;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total4;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t idx = 4 * q;
    // the four entries share a row and a 256-column tile: when the first is
    // above the line all are, and otherwise the tile was computed
    const int64_t rdiag = tri > 0 ? (idx / P) % tri : 0;
    if (tri > 0 && n0 + idx % P > rdiag) continue;
    int g[4][S];
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
      for (int t = 0; t < S; ++t) g[e][t] = 0;
#pragma unroll
    for (int i = 0; i < S; ++i)
#pragma unroll
      for (int j = 0; j < S - i; ++j) {
        const float4 v =
            __ldcs(reinterpret_cast<const float4*>(Pw + (int64_t)(i * S - i * (i - 1) / 2 + j) * slab + idx));
        g[0][i + j] += __float2int_rn(v.x);
        g[1][i + j] += __float2int_rn(v.y);
        g[2][i + j] += __float2int_rn(v.z);
        g[3][i + j] += __float2int_rn(v.w);
      }
    const int64_t r = idx / P;
    const int64_t c0 = idx - r * P;
    const int er = Ea[r * nch + chunk];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      double h = 0.0;
#pragma unroll
      for (int b = NB - 1; b >= 0; --b) {
        int64_t B = 0;
#pragma unroll
        for (int t = 5 * b; t < 5 * b + 5; ++t) B = B * 64 + (t < S ? (int64_t)g[e][t] : 0);
        h = h * 0x1p-30 + (double)B;
      }
      const int64_t c = c0 + e;
      const int64_t oc = cmap ? (int64_t)cmap[c] : n0 + c;
      if (oc < 0 || (tri > 0 && n0 + c > rdiag)) continue;
      const double v = ldexp(h, er + Eb[(n0 + c) * nch + chunk] - 12 - 24);
      double* out = C + r * ldc + oc;
      *out = accumulate ? *out + v : v;
    }
  }
}

typedef void (*ReduceKernel)(const float*, int64_t, int64_t, const int32_t*, const int32_t*, int, int, int64_t,
                             double*, int64_t, int, const int32_t*, int64_t);

static ReduceKernel reduce_kernel(int s) {
  switch (s) {
#define DG_REDUCE_CASE(n) \
  case n: return k_sliced_reduce<n>;
    DG_REDUCE_CASE(2) DG_REDUCE_CASE(3) DG_REDUCE_CASE(4) DG_REDUCE_CASE(5) DG_REDUCE_CASE(6)
    DG_REDUCE_CASE(7) DG_REDUCE_CASE(8) DG_REDUCE_CASE(9) DG_REDUCE_CASE(10) DG_REDUCE_CASE(11)
    DG_REDUCE_CASE(12) DG_REDUCE_CASE(13) DG_REDUCE_CASE(14) DG_REDUCE_CASE(15) DG_REDUCE_CASE(16)
#undef DG_REDUCE_CASE
    default: return nullptr;
  }
}

static ReduceKernel reduce_kernel4(int s) {
  switch (s) {
#define DG_REDUCE_CASE(n) \
  case n: return k_sliced_reduce4<n>;
    DG_REDUCE_CASE(2) DG_REDUCE_CASE(3) DG_REDUCE_CASE(4) DG_REDUCE_CASE(5) DG_REDUCE_CASE(6)
    DG_REDUCE_CASE(7) DG_REDUCE_CASE(8) DG_REDUCE_CASE(9) DG_REDUCE_CASE(10) DG_REDUCE_CASE(11)
    DG_REDUCE_CASE(12) DG_REDUCE_CASE(13) DG_REDUCE_CASE(14) DG_REDUCE_CASE(15) DG_REDUCE_CASE(16)
#undef DG_REDUCE_CASE
    default: return nullptr;
  }
}

// The reduction over slabs of M x P: four outputs per thread when P % 4 == 0.
static cudaError_t launch_reduce(int s, const float* Pw, int64_t M, int64_t P, const int32_t* Ea, const int32_t* Eb,
                                 int nch, int chunk, int64_t n0, double* C, int64_t ldc, int accumulate,
                                 const int32_t* cmap, cudaStream_t st, int64_t tri = 0) {
  const bool v4 = P % 4 == 0;
  const int64_t work = v4 ? M * P / 4 : M * P;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 152 * 16));
  (v4 ? reduce_kernel4(s) : reduce_kernel(s))<<<grid, 256, 0, st>>>(Pw, M, P, Ea, Eb, nch, chunk, n0, C, ldc,
                                                                      accumulate, cmap, tri);
  count_launch();
  return cudaGetLastError();
}

static int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Workspace cap of the FP32 slice-pair products; wider outputs run in column panels.
static constexpr size_t kPairBytes = size_t(8) << 30;

// T (cols x rows, row-major, ldt) = X^T for X (rows x cols, row-major, ldx);
// 32 x 32 tiles through shared memory, 32 x 8 threads.
__global__ void __launch_bounds__(256) k_transpose_f64(const double* __restrict__ X, int64_t ldx, int64_t rows,
                                                       int64_t cols, double* __restrict__ T, int64_t ldt) {
  __shared__ double tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int64_t r = r0 + j, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[j][threadIdx.x] = X[r * ldx + c];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int64_t c = c0 + j, r = r0 + threadIdx.x;
    if (r < rows && c < cols) T[c * ldt + r] = tile[threadIdx.x][j];
  }
}

static dgchefsi_status transpose_f64(const double* X, int64_t ldx, int64_t rows, int64_t cols, double* T, int64_t ldt,
                                     cudaStream_t st) {
  if ((rows + 31) / 32 > 65535) return set_error(DGCHEFSI_ERR_UNSUPPORTED, "transpose of %lld rows", (long long)rows);
  k_transpose_f64<<<dim3((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32)), dim3(32, 8), 0, st>>>(
      X, ldx, rows, cols, T, ldt);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return DGCHEFSI_OK;
}

dgchefsi_status sliced_gemm(dgchefsi_ctx* ctx, bool b_rows, bool a_lower, int64_t M, int64_t Nc, int64_t K,
                            const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, int s,
                            int* flag, int64_t tri) {
  if (M <= 0 || Nc <= 0) return DGCHEFSI_OK;
  if (!reduce_kernel(s)) return set_error(DGCHEFSI_ERR_ARG, "slices = %d outside 2..16", s);
  cudaStream_t st = ctx->stream;
  if (K <= 0) {
    DG_CUDA(cudaMemset2DAsync(C, sizeof(double) * ldc, 0, sizeof(double) * Nc, M, st));
    return DGCHEFSI_OK;
  }
  const int nch = (int)((K + kL - 1) / kL);
  const int64_t pairs = (int64_t)s * (s + 1) / 2;
  // Slices of A: s x M x lqa, of the right operand as rows: s x Nc x lqb (K
  // contiguous in both; the A B form transposes B first).
  const int64_t lqa = round_up(K, 8);
  const int64_t lqb = round_up(K, 8);
  const int64_t sa = M * lqa;
  const int64_t sb = Nc * lqb;
  const bool same = b_rows && A == B && lda == ldb && M == Nc && !a_lower;
  const size_t qa_bytes = sizeof(__nv_bfloat16) * (size_t)(s * sa);
  const size_t qb_bytes = same ? 0 : sizeof(__nv_bfloat16) * (size_t)(s * sb);
  const size_t ea_bytes = sizeof(int32_t) * (size_t)(M * nch);
  const size_t eb_bytes = sizeof(int32_t) * (size_t)(Nc * nch);
  const size_t bal_bytes = b_rows ? 0 : 2 * sizeof(int32_t) * (size_t)K;
  const size_t a256 = 256;
  auto up = [&](size_t x) { return (x + a256 - 1) / a256 * a256; };
  // Column panel of the product (a multiple of the kernel's 128-column tiles)
  // so that the FP32 pair slabs stay under the cap; two slab buffers when the
  // product has more than one (panel, chunk) step, so that the reduction of
  // one step (on the context's reduction stream) overlaps the next step's
  // slice pairs.
  const bool multi = nch > 1 || (int64_t)(kPairBytes / (sizeof(float) * (size_t)pairs * (size_t)M)) < Nc;
  const int nbuf = multi ? 2 : 1;
  int64_t P = (int64_t)(kPairBytes / nbuf / (sizeof(float) * (size_t)pairs * (size_t)M));
  P = std::max<int64_t>(128, P / 128 * 128);
  if (P >= Nc) P = Nc;
  const size_t slab_set = sizeof(float) * (size_t)pairs * (size_t)M * (size_t)P;
  const size_t pw_bytes = (size_t)nbuf * up(slab_set);
  DG_TRY(ensure(ctx, ctx->ws_sliced,
                up(qa_bytes) + up(qb_bytes) + up(ea_bytes) + up(eb_bytes) + up(bal_bytes) + up(pw_bytes),
                "sliced-product workspace"));
  char* base = static_cast<char*>(ctx->ws_sliced.p);
  __nv_bfloat16* Qa = reinterpret_cast<__nv_bfloat16*>(base);
  __nv_bfloat16* Qb = same ? Qa : reinterpret_cast<__nv_bfloat16*>(base + up(qa_bytes));
  int32_t* Ea = reinterpret_cast<int32_t*>(base + up(qa_bytes) + up(qb_bytes));
  int32_t* Eb = same ? Ea : reinterpret_cast<int32_t*>(base + up(qa_bytes) + up(qb_bytes) + up(ea_bytes));
  int32_t* bal = b_rows ? nullptr
                        : reinterpret_cast<int32_t*>(base + up(qa_bytes) + up(qb_bytes) + up(ea_bytes) + up(eb_bytes));
  int32_t* nbal = b_rows ? nullptr : bal + K;
  float* Pw =
      reinterpret_cast<float*>(base + up(qa_bytes) + up(qb_bytes) + up(ea_bytes) + up(eb_bytes) + up(bal_bytes));

  // C = A B with B (K x Nc): every K index k is balanced first, row k of B by
  // 2^{-s_k} and column k of A by 2^{s_k} (exact), s_k the exponent of B's row
  // maximum, so that rows of B with very different norms (the filtered states
  // of Y_hat^T = U^{-T} Y^T) do not share one column scale. B is then
  // transposed (Nc x K) and split by rows like the A B^T form.
  const double* Br = B;
  int64_t ldbr = ldb;
  if (!b_rows) {
    k_row_exponents<<<(unsigned)K, 256, 0, st>>>(B, ldb, Nc, bal, nbal);
    count_launch();
    DG_CUDA(cudaGetLastError());
    DG_TRY(ensure(ctx, ctx->ws_sliced_b, sizeof(double) * (size_t)Nc * (size_t)K, "transposed right operand"));
    double* Bt = static_cast<double*>(ctx->ws_sliced_b.p);
    DG_TRY(transpose_f64(B, ldb, K, Nc, Bt, K, st));
    Br = Bt;
    ldbr = K;
  }
  k_split_rows<<<dim3((unsigned)M, (unsigned)nch), 256, 0, st>>>(A, lda, K, s, a_lower ? 1 : 0, bal, Qa, lqa, sa,
                                                                  Ea, nch, flag);
  count_launch();
  DG_CUDA(cudaGetLastError());
  if (!same) {
    k_split_rows<<<dim3((unsigned)Nc, (unsigned)nch), 256, 0, st>>>(Br, ldbr, K, s, 0, nbal, Qb, lqb, sb, Eb, nch,
                                                                     flag);
    count_launch();
    DG_CUDA(cudaGetLastError());
  }
  DG_TRY(pair_products_begin(ctx));
  cudaStream_t sr = st;
  if (multi) {
    if (!ctx->s_reduce) {
      DG_CUDA(cudaStreamCreateWithFlags(&ctx->s_reduce, cudaStreamNonBlocking));
      for (int i = 0; i < 2; ++i) {
        DG_CUDA(cudaEventCreateWithFlags(&ctx->ev_pairs[i], cudaEventDisableTiming));
        DG_CUDA(cudaEventCreateWithFlags(&ctx->ev_reduce[i], cudaEventDisableTiming));
      }
    }
    sr = ctx->s_reduce;
    // nothing of an earlier call may still read a slab buffer or write C
    DG_CUDA(cudaEventRecord(ctx->ev_pairs[0], st));
    DG_CUDA(cudaStreamWaitEvent(sr, ctx->ev_pairs[0], 0));
    for (int b = 0; b < 2; ++b) DG_CUDA(cudaEventRecord(ctx->ev_reduce[b], sr));
  }
  // timing events around every slice-pair launch (read after the status check)
  const int nsteps = (int)(((Nc + P - 1) / P) * nch);
  while ((int)ctx->ev_time.size() < 2 * nsteps) {
    cudaEvent_t e = nullptr;
    DG_CUDA(cudaEventCreate(&e));
    ctx->ev_time.push_back(e);
  }
  int step = 0;
  for (int64_t n0 = 0; n0 < Nc; n0 += P) {
    const int64_t pn = std::min<int64_t>(P, Nc - n0);
    for (int chunk = 0; chunk < nch; ++chunk, ++step) {
      const int64_t k0 = (int64_t)chunk * kL;
      const int64_t kc = std::min<int64_t>(kL, K - k0);
      const int b = step & 1;
      float* Pb = reinterpret_cast<float*>(reinterpret_cast<char*>(Pw) + (size_t)b * up(slab_set));
      // slab of pair (i, j): M x pn, Qa_i times the panel's rows of Qb_j over this chunk,
      // into buffer b once the reduction that last read it is done
      if (multi) DG_CUDA(cudaStreamWaitEvent(st, ctx->ev_reduce[b], 0));
      DG_CUDA(cudaEventRecord(ctx->ev_time[2 * step], st));
      DG_TRY(pair_products_2sm(ctx, Qa, lqa, sa, M, Qb, lqb, sb, Nc, K, k0, kc, n0, pn, s, Pb, a_lower, tri));
      DG_CUDA(cudaEventRecord(ctx->ev_time[2 * step + 1], st));
      if (multi) {
        DG_CUDA(cudaEventRecord(ctx->ev_pairs[b], st));
        DG_CUDA(cudaStreamWaitEvent(sr, ctx->ev_pairs[b], 0));
      }
      DG_CUDA(launch_reduce(s, Pb, M, pn, Ea, Eb, nch, chunk, n0, C, ldc, chunk > 0 ? 1 : 0, nullptr, sr, tri));
      if (multi) DG_CUDA(cudaEventRecord(ctx->ev_reduce[b], sr));
    }
  }
  if (multi) {  // the caller's stream sees C complete
    DG_CUDA(cudaEventRecord(ctx->ev_reduce[0], sr));
    DG_CUDA(cudaStreamWaitEvent(st, ctx->ev_reduce[0], 0));
  }
  DG_TRY(pair_products_status(ctx));  // synchronises the stream
  double ms = 0.0;
  for (int q = 0; q < step; ++q) {
    float t = 0.f;
    DG_CUDA(cudaEventElapsedTime(&t, ctx->ev_time[2 * q], ctx->ev_time[2 * q + 1]));
    ms += t;
  }
  ctx->pairs_ms = ms;
  ctx->pairs_launches = step;
  return DGCHEFSI_OK;
}

// ---------------------------------------------------------------------------
// H X from slices (the block-sparse product of Rayleigh-Ritz, W = H Y_hat).
// Row r of H (element K, row n) contracts over the columns of K's neighbour
// blocks only, at most 4096 of them, so one K chunk covers every row: its
// exponent e_r is over the whole row. Each state's exponent f_s is over all N
// of its components (a valid bound for every row's column range). H's digits
// are written in the block layout of the tensor-core filter's operand copy
// of H (64-column slices of each block, element-padded rows), the states'
// digits in its element-padded state-major layout, so the filter's step
// kernel multiplies one slice pair per launch (alpha = 1, beta = 0) into an
// FP32 slab, and k_sliced_reduce (with the padded-to-plain column map)
// combines the slabs.

// E[poff_K + n] = frexp exponent of max_j |H[(K, n), j]| over row n of element
// K's blocks (0 for an all-zero row, and for the padding rows n >= nb[K]).
// One CTA per element. A non-finite entry raises flag.
__global__ void __launch_bounds__(256) k_h_row_exponents(const int64_t* __restrict__ row_ptr,
                                                         const int32_t* __restrict__ col,
                                                         const int64_t* __restrict__ blk_off,
                                                         const double* __restrict__ vals,
                                                         const int32_t* __restrict__ nb,
                                                         const int32_t* __restrict__ pnb,
                                                         const int32_t* __restrict__ poff, int32_t* __restrict__ E,
                                                         int* __restrict__ flag) {
  __shared__ int emax[256];
  __shared__ int bad;
  const int K = blockIdx.x;
  const int nK = nb[K];
  for (int n = threadIdx.x; n < 256; n += blockDim.x) emax[n] = INT_MIN;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int64_t e = row_ptr[K]; e < row_ptr[K + 1]; ++e) {
    const int nKp = nb[col[e]];
    const double* blk = vals + blk_off[e];
    const int64_t total = (int64_t)nK * nKp;
    for (int64_t t = threadIdx.x; t < total; t += blockDim.x) {
      int64_t Mm;
      int Ex;
      const int c = decompose(blk[t], Mm, Ex);
      if (c == 2) bad = 1;
      if (c == 1) atomicMax(&emax[(int)(t / nKp)], Ex);
    }
  }
  __syncthreads();
  for (int n = threadIdx.x; n < pnb[K]; n += blockDim.x)
    E[poff[K] + n] = (n < nK && emax[n] != INT_MIN && !bad) ? emax[n] - 1022 : 0;
  if (threadIdx.x == 0 && bad) atomic_flag(flag);
}

// s digit copies of H in the filter's operand layout: block e, 64-column
// slice sl, padded row n at row brow[e] + sl * pnb[K] + n of each copy (copy i
// starts at Q + i * cstride); entries past the block (padding) are zero.
__global__ void __launch_bounds__(256) k_build_h_slices(const int32_t* __restrict__ blk_row,
                                                        const int32_t* __restrict__ col,
                                                        const int64_t* __restrict__ blk_off,
                                                        const double* __restrict__ vals,
                                                        const int32_t* __restrict__ nb,
                                                        const int32_t* __restrict__ pnb,
                                                        const int32_t* __restrict__ poff,
                                                        const int64_t* __restrict__ brow,
                                                        const int32_t* __restrict__ E, int s,
                                                        __nv_bfloat16* __restrict__ Q, int64_t cstride) {
  constexpr int W = 64;
  const int64_t e = blockIdx.x;
  const int K = blk_row[e], Kp = col[e];
  const int nK = nb[K], nKp = nb[Kp], pK = pnb[K];
  const int nsl = (pnb[Kp] + W - 1) / W;
  const double* blk = vals + blk_off[e];
  const int64_t total = (int64_t)nsl * pK * W;
  for (int64_t t = threadIdx.x; t < total; t += blockDim.x) {
    const int w = (int)(t % W);
    const int64_t rr = t / W;
    const int n = (int)(rr % pK);
    const int sl = (int)(rr / pK);
    const int jp = sl * W + w;
    const double v = (n < nK && jp < nKp) ? blk[(int64_t)n * nKp + jp] : 0.0;
    const int er = E[poff[K] + n];
    __nv_bfloat16* q = Q + (brow[e] + rr) * W + w;
    if (s <= 10) {
      int64_t Mm = 0;
      int Ex = 0;
      if (decompose(v, Mm, Ex) != 1) Mm = 0;
      slice_fixed(Mm, Ex, v < 0.0, -1075 - er + 6 * s, s, q, cstride);
    } else {
      slice_fp64(std::isfinite(v) ? ldexp(v, -er) : 0.0, s, q, cstride);
    }
  }
}

// s digit copies of the states X (Ns x ld, state-major) in the element-padded
// layout (Ns x ldp per copy, copy i at Q + i * cstride); cmap[c] is the
// column of padded column c (-1 for padding, written as zero). E[s] = frexp
// exponent of the state's largest |entry|. One CTA per state, two passes.
__global__ void __launch_bounds__(256) k_pack_state_slices(const double* __restrict__ X, int64_t ld, int64_t N,
                                                           const int32_t* __restrict__ cmap, int64_t ldp, int s,
                                                           __nv_bfloat16* __restrict__ Q, int64_t cstride,
                                                           int32_t* __restrict__ E, int* __restrict__ flag) {
  const int64_t st = blockIdx.x;
  const double* x = X + st * ld;
  int emax = INT_MIN;
  bool bad = false;
  for (int64_t c = threadIdx.x; c < N; c += blockDim.x) {
    int64_t Mm;
    int Ex;
    const int k = decompose(x[c], Mm, Ex);
    if (k == 2) bad = true;
    if (k == 1) emax = max(emax, Ex);
  }
  __shared__ int red[8];
  __shared__ int sbad;
  if (threadIdx.x == 0) sbad = 0;
  emax = warp_max(emax);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = emax;
  if (bad) sbad = 1;
  __syncthreads();
  emax = red[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) emax = max(emax, red[w]);
  const bool zero = sbad != 0;
  const int e = (emax == INT_MIN || zero) ? 0 : emax - 1022;
  if (threadIdx.x == 0) {
    E[st] = e;
    if (zero) atomic_flag(flag);
  }
  for (int64_t c = threadIdx.x; c < ldp; c += blockDim.x) {
    const int32_t oc = cmap[c];
    const double v = (oc >= 0 && !zero) ? x[oc] : 0.0;
    __nv_bfloat16* q = Q + st * ldp + c;
    if (s <= 10) {
      int64_t Mm = 0;
      int Ex = 0;
      if (decompose(v, Mm, Ex) != 1) Mm = 0;
      slice_fixed(Mm, Ex, v < 0.0, -1075 - e + 6 * s, s, q, cstride);
    } else {
      slice_fp64(ldexp(v, -e), s, q, cstride);
    }
  }
}

cudaError_t slices_of_h(const dgchefsi_ctx* ctx, const int32_t* blk_row, const int32_t* pnb, const int32_t* poff,
                        const int64_t* brow, int s, __nv_bfloat16* Q, int64_t cstride, int32_t* E, int* flag,
                        cudaStream_t st) {
  k_h_row_exponents<<<(unsigned)ctx->M, 256, 0, st>>>(ctx->row_ptr_d, ctx->col_d, ctx->blk_off_d, ctx->vals_d,
                                                      ctx->nb_d, pnb, poff, E, flag);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_build_h_slices<<<(unsigned)ctx->nnzb, 256, 0, st>>>(blk_row, ctx->col_d, ctx->blk_off_d, ctx->vals_d, ctx->nb_d,
                                                        pnb, poff, brow, E, s, Q, cstride);
  count_launch();
  return cudaGetLastError();
}

cudaError_t slices_of_states(const double* X, int64_t ld, int64_t Ns, int64_t N, const int32_t* cmap, int64_t ldp,
                             int s, __nv_bfloat16* Q, int64_t cstride, int32_t* E, int* flag, cudaStream_t st) {
  k_pack_state_slices<<<(unsigned)Ns, 256, 0, st>>>(X, ld, N, cmap, ldp, s, Q, cstride, E, flag);
  count_launch();
  return cudaGetLastError();
}

dgchefsi_status reduce_pair_slabs(const float* Pw, int64_t rows, int64_t cols, const int32_t* Erows,
                                  const int32_t* Ecols, const int32_t* cmap, double* C, int64_t ldc, int s,
                                  cudaStream_t st) {
  if (!reduce_kernel(s)) return set_error(DGCHEFSI_ERR_ARG, "slices = %d outside 2..16", s);
  DG_CUDA(launch_reduce(s, Pw, rows, cols, Erows, Ecols, 1, 0, 0, C, ldc, 0, cmap, st));
  return DGCHEFSI_OK;
}

dgchefsi_status sliced_gemm_tn(dgchefsi_ctx* ctx, int64_t M, int64_t Nc, int64_t K, const double* A, int64_t lda,
                               const double* B, int64_t ldb, double* C, int64_t ldc, int s, int* flag) {
  if (M <= 0 || Nc <= 0) return DGCHEFSI_OK;
  if (K > 0) {
    DG_TRY(ensure(ctx, ctx->ws_sliced_t, sizeof(double) * (size_t)M * (size_t)K, "transposed operand"));
    double* At = static_cast<double*>(ctx->ws_sliced_t.p);
    DG_TRY(transpose_f64(A, lda, K, M, At, K, ctx->stream));
    return sliced_gemm(ctx, false, false, M, Nc, K, At, K, B, ldb, C, ldc, s, flag);
  }
  return sliced_gemm(ctx, false, false, M, Nc, K, A, lda, B, ldb, C, ldc, s, flag);
}

void sliced_destroy(dgchefsi_ctx* ctx) { (void)ctx; }

}  // namespace dg
