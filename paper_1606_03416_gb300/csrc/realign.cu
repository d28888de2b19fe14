// Steps around the cycle: re-alignment of the coefficient block to the next
// SCF step's basis (Sec. III.B.3, Eq. basis_rotation_3) and density-matrix
// blocks on all of H's pattern (Eq. densitymatrix for neighbouring elements).
//
// Re-alignment, per element K with old size q = J_K^i, new size p = J_K^{i+1}
// and R_K sample points:
//   T_K = (V_K^{i+1})^T V_K^{i}                      (p x q, k_overlap_f64)
//   X_new[s, K, j'] = sum_j T_K[j', j] X_old[s, K, j] (k_realign_f64)
// i.e. the paper's two products, the small one first (R_K p q + N_s p q
// multiply-adds instead of R_K N_s (p + q)). Both in FP64 on the DFMA pipe.
#include <algorithm>
#include <vector>

#include "ctx.h"

namespace dg {
namespace {

// T_K = Vn_K^T Vo_K for every element; Vn_K (R x p), Vo_K (R x q) row-major.
__global__ void __launch_bounds__(256) k_overlap_f64(const int32_t* __restrict__ nb_new, const int32_t* __restrict__ nb_old,
                                                     const int32_t* __restrict__ nr, const int64_t* __restrict__ vn_off,
                                                     const int64_t* __restrict__ vo_off, const int64_t* __restrict__ t_off,
                                                     const double* __restrict__ Vn, const double* __restrict__ Vo,
                                                     double* __restrict__ T) {
  constexpr int TB = 32, RB = 32;
  const int K = blockIdx.x;
  const int p = nb_new[K], q = nb_old[K], R = nr[K];
  const int j0 = blockIdx.y * TB, i0 = blockIdx.z * TB;
  if (j0 >= p || i0 >= q) return;
  __shared__ double As[RB][TB + 1];
  __shared__ double Bs[RB][TB + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const double* vn = Vn + vn_off[K];
  const double* vo = Vo + vo_off[K];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int r0 = 0; r0 < R; r0 += RB) {
    for (int rr = ty; rr < RB; rr += 8) {
      const int r = r0 + rr;
      As[rr][tx] = (r < R && j0 + tx < p) ? vn[(int64_t)r * p + j0 + tx] : 0.0;
      Bs[rr][tx] = (r < R && i0 + tx < q) ? vo[(int64_t)r * q + i0 + tx] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < RB; ++rr) {
      const double b = Bs[rr][tx];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i] = fma(As[rr][ty + 8 * i], b, acc[i]);
    }
    __syncthreads();
  }
  double* t = T + t_off[K];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int jj = j0 + ty + 8 * i;
    if (jj < p && i0 + tx < q) t[(int64_t)jj * q + i0 + tx] = acc[i];
  }
}

// Y[s, on_K + j'] = sum_j X[s, oo_K + j] T_K[j', j]; 64 states x 64 new columns per CTA.
__global__ void __launch_bounds__(256) k_realign_f64(const int32_t* __restrict__ nb_new, const int32_t* __restrict__ nb_old,
                                                     const int64_t* __restrict__ off_new, const int64_t* __restrict__ off_old,
                                                     const int64_t* __restrict__ t_off, const double* __restrict__ T,
                                                     const double* __restrict__ X, int64_t ldx, double* __restrict__ Y,
                                                     int64_t ldy, int64_t Ns) {
  constexpr int TS = 64, TJ = 64, KB = 16;
  const int K = blockIdx.x;
  const int p = nb_new[K], q = nb_old[K];
  const int64_t s0 = (int64_t)blockIdx.y * TS;
  const int jp0 = blockIdx.z * TJ;
  if (s0 >= Ns || jp0 >= p) return;
  __shared__ double Xs[TS][KB + 1];
  __shared__ double Ts[KB][TJ + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const double* t = T + t_off[K];
  const int64_t oo = off_old[K], on = off_new[K];
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int j0 = 0; j0 < q; j0 += KB) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int e = tid + 256 * l;  // 1024 entries of each tile
      const int xr = e >> 4, xc = e & 15;
      const int64_t s = s0 + xr;
      Xs[xr][xc] = (s < Ns && j0 + xc < q) ? X[s * ldx + oo + j0 + xc] : 0.0;
      const int tr = e >> 6, tc = e & 63;  // Ts[j][j'] = T[j'][j]
      Ts[tr][tc] = (j0 + tr < q && jp0 + tc < p) ? t[(int64_t)(jp0 + tc) * q + j0 + tr] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KB; ++kk) {
      double xa[4], tb[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) xa[a] = Xs[ty + 16 * a][kk];
#pragma unroll
      for (int b = 0; b < 4; ++b) tb[b] = Ts[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(xa[a], tb[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t s = s0 + ty + 16 * a;
    if (s >= Ns) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int jp = jp0 + tx + 16 * b;
      if (jp < p) Y[s * ldy + on + jp] = acc[a][b];
    }
  }
}

}  // namespace
}  // namespace dg

using namespace dg;

extern "C" dgchefsi_status dgchefsi_realign(dgchefsi_ctx* ctx, const int32_t* nb_old, const int32_t* nr,
                                            const double* V_old, const double* V_new, const double* X_old, int64_t Ns,
                                            int64_t ld_old, double* X_new, int64_t ld) {
  clear_error();
  if (!ctx) return set_error(DGCHEFSI_ERR_ARG, "null context");
  if (!nb_old || !nr || !V_old || !V_new || !X_old || !X_new) return set_error(DGCHEFSI_ERR_ARG, "null pointer");
  if (Ns < 1) return set_error(DGCHEFSI_ERR_ARG, "Ns < 1");
  const int M = ctx->M;
  std::vector<int64_t> off_old(M + 1, 0), vo(M + 1, 0), vn(M + 1, 0), to(M + 1, 0);
  int max_old = 0;
  for (int K = 0; K < M; ++K) {
    const int q = nb_old[K], p = ctx->nb_h[K], R = nr[K];
    if (q < 1 || q > 256) return set_error(DGCHEFSI_ERR_ARG, "nb_old[%d] = %d outside 1..256", K, q);
    if (R < 1) return set_error(DGCHEFSI_ERR_ARG, "nr[%d] = %d < 1", K, R);
    off_old[K + 1] = off_old[K] + q;
    vo[K + 1] = vo[K] + (int64_t)R * q;
    vn[K + 1] = vn[K] + (int64_t)R * p;
    to[K + 1] = to[K] + (int64_t)p * q;
    max_old = std::max(max_old, q);
  }
  if (ld_old < off_old[M]) return set_error(DGCHEFSI_ERR_ARG, "ld_old < sum of old element sizes");
  if (ld < ctx->N) return set_error(DGCHEFSI_ERR_ARG, "ld < N");
  // the two blocks must not overlap
  const char* a0 = reinterpret_cast<const char*>(X_old);
  const char* a1 = a0 + sizeof(double) * ((size_t)(Ns - 1) * ld_old + off_old[M]);
  const char* b0 = reinterpret_cast<const char*>(X_new);
  const char* b1 = b0 + sizeof(double) * ((size_t)(Ns - 1) * ld + ctx->N);
  if (a0 < b1 && b0 < a1) return set_error(DGCHEFSI_ERR_ARG, "X_new overlaps X_old");
  cudaStream_t s = ctx->stream;
  // device copies of the per-element tables (4 x [M+1] int64, 2 x [M] int32) and T
  const size_t tab = sizeof(int64_t) * 4 * (size_t)(M + 1) + sizeof(int32_t) * 2 * (size_t)M;
  const size_t tab_al = (tab + 255) / 256 * 256;
  DG_TRY(ensure(ctx, ctx->ws_realign, tab_al + sizeof(double) * (size_t)std::max<int64_t>(to[M], 1), "re-alignment tables"));
  std::vector<char> host(tab);
  char* hp = host.data();
  auto put = [&](const void* src, size_t n) {
    std::copy(static_cast<const char*>(src), static_cast<const char*>(src) + n, hp);
    hp += n;
  };
  put(off_old.data(), sizeof(int64_t) * (M + 1));
  put(vo.data(), sizeof(int64_t) * (M + 1));
  put(vn.data(), sizeof(int64_t) * (M + 1));
  put(to.data(), sizeof(int64_t) * (M + 1));
  put(nb_old, sizeof(int32_t) * M);
  put(nr, sizeof(int32_t) * M);
  char* dbase = static_cast<char*>(ctx->ws_realign.p);
  DG_CUDA(cudaMemcpyAsync(dbase, host.data(), tab, cudaMemcpyHostToDevice, s));
  const int64_t* d_off_old = reinterpret_cast<const int64_t*>(dbase);
  const int64_t* d_vo = d_off_old + (M + 1);
  const int64_t* d_vn = d_vo + (M + 1);
  const int64_t* d_to = d_vn + (M + 1);
  const int32_t* d_nb_old = reinterpret_cast<const int32_t*>(d_to + (M + 1));
  const int32_t* d_nr = d_nb_old + M;
  double* T = reinterpret_cast<double*>(dbase + tab_al);
  const unsigned tp = (unsigned)((ctx->max_nb + 31) / 32), tq = (unsigned)((max_old + 31) / 32);
  k_overlap_f64<<<dim3((unsigned)M, tp, tq), 256, 0, s>>>(ctx->nb_d, d_nb_old, d_nr, d_vn, d_vo, d_to, V_new, V_old, T);
  count_launch();
  DG_CUDA(cudaGetLastError());
  const int64_t st = (Ns + 63) / 64;
  if (st > 65535) return set_error(DGCHEFSI_ERR_UNSUPPORTED, "Ns too large for one launch");
  k_realign_f64<<<dim3((unsigned)M, (unsigned)st, (unsigned)((ctx->max_nb + 63) / 64)), 256, 0, s>>>(
      ctx->nb_d, d_nb_old, ctx->off_d, d_off_old, d_to, T, X_old, ld_old, X_new, ld, Ns);
  count_launch();
  DG_CUDA(cudaGetLastError());
  // the host table must outlive the asynchronous copy from pageable memory
  DG_CUDA(cudaStreamSynchronize(s));
  return DGCHEFSI_OK;
}

extern "C" dgchefsi_status dgchefsi_density_pattern(dgchefsi_ctx* ctx, const double* X, int64_t Ns, int64_t ld,
                                                    const double* f, double* P) {
  clear_error();
  if (!ctx) return set_error(DGCHEFSI_ERR_ARG, "null context");
  if (!X || !f || !P) return set_error(DGCHEFSI_ERR_ARG, "null pointer");
  if (Ns < 1) return set_error(DGCHEFSI_ERR_ARG, "Ns < 1");
  if (ld < ctx->N) return set_error(DGCHEFSI_ERR_ARG, "ld < N");
  cudaStream_t s = ctx->stream;
  DG_CUDA(cudaMemsetAsync(P, 0, sizeof(double) * (size_t)ctx->n_values, s));
  DG_CUDA(block_outer_f64(ctx->view(), ctx->blk_row_d, ctx->nnzb, X, ld, X, ld, f, 1.0, Ns, P, s));
  return DGCHEFSI_OK;
}
