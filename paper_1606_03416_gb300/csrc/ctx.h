// Library context and host-side helpers shared by the API translation units.
#pragma once
#include <cuda_bf16.h>
#include <cusolverDn.h>

#include <cstdarg>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dgchefsi.h"
#include "internal.h"

namespace dg {

// Grow-only device buffer owned by a context.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct TcState;  // tensor-core filter state (tc_filter.cu)

}  // namespace dg

struct dgchefsi_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int32_t M = 0;
  int64_t N = 0;
  int32_t max_nb = 0;
  int64_t nnzb = 0;
  int64_t n_values = 0;
  std::vector<int32_t> nb_h;
  std::vector<int64_t> off_h, row_ptr_h, blk_off_h, poff_h;
  std::vector<int32_t> col_h;
  // device copy of H
  int32_t* nb_d = nullptr;
  int64_t* off_d = nullptr;
  int64_t* row_ptr_d = nullptr;
  int32_t* col_d = nullptr;
  int64_t* blk_off_d = nullptr;
  double* vals_d = nullptr;
  int64_t* poff_d = nullptr;  // packed density-block offsets
  int32_t* blk_row_d = nullptr;  // element row of each stored block
  // workspace
  dg::DevBuf ws_filter;   // filter ping-pong partner (Ns x ld FP64)
  dg::DevBuf ws_rr;       // Rayleigh-Ritz block (Ns x N FP64)
  dg::DevBuf ws_small;    // Ns x Ns FP64
  dg::DevBuf ws_solver;   // cuSOLVER device workspace
  dg::DevBuf ws_cycle;    // filtered block inside dgchefsi_cycle
  dg::DevBuf ws_lanczos;  // Lanczos basis and scalars
  dg::DevBuf ws_adjoint;  // checkpoints and blocks of the band-energy gradient
  dg::DevBuf ws_realign;  // per-element tables and overlaps of the re-alignment
  int orth_mode = 0;      // DGCHEFSI_ORTH_*: orthonormalisation of step 3
  // Rayleigh-Ritz products: DGCHEFSI_PRODUCTS_*, slice count of the sliced
  // BF16 form and its workspace
  int products_mode = 0;
  int products_slices = 10;
  dg::DevBuf ws_sliced;
  dg::DevBuf ws_sliced_t;  // transposed left operand of the A^T B form
  dg::DevBuf ws_sliced_b;  // transposed right operand of the A B form
  dg::DevBuf ws_pairs;     // tensor maps, pair and tile lists of the slice-pair kernel (regrown as needed)
  dg::DevBuf ws_pairs_err; // the slice-pair kernel's error word (its own buffer: never regrown mid-product)
  // the slab reduction of the sliced products runs on its own stream, one K
  // chunk behind the slice-pair kernel (double-buffered slabs)
  cudaStream_t s_reduce = nullptr;
  cudaEvent_t ev_pairs[2] = {nullptr, nullptr}, ev_reduce[2] = {nullptr, nullptr};
  // device time of the slice-pair kernel launches of the last sliced product
  // (dgchefsi_sliced_timing): timing events around each launch, read back
  // when the product's status is checked
  std::vector<cudaEvent_t> ev_time;
  double pairs_ms = 0.0;
  int64_t pairs_launches = 0;
  // eigensolver of the projected Hamiltonian (DGCHEFSI_EIG_*), its workspace
  // and what its last call did (dgchefsi_eigensolver_stats)
  int eig_mode = 0;
  int eig_used = 0, eig_steps = 0, eig_max_cluster = 0, eig_fallback = 0;
  double eig_update = 0.0, eig_start_ms = 0.0, eig_refine_ms = 0.0;
  int64_t eig_start_order = 0;
  int eig_start_solver = 0;  // 0 none (identity start), 1 this library's Jacobi kernel, 2 cuSOLVER FP32
  double eig_history[16] = {};     // largest correction of each refinement step
  int eig_slices_history[16] = {};  // slices of each step's update product (0: no full product)
  double eig_start_coupling = 0.001;  // first-order coupling that puts a row in the FP32 start block
  dg::DevBuf ws_eig;
  // Cholesky factorisation of step 3 (DGCHEFSI_CHOL_*) and the recursive
  // form's workspace (L^{-1} and two scratch blocks, 3 N_s^2 doubles)
  int chol_mode = 0;
  dg::DevBuf ws_chol;
  int32_t f64_tj = 64;    // column tile of the FP64 filter (set at create)
  // FP64 filter as a CUDA graph: coefficients copied from a pinned mirror at
  // every replay; the graph is captured again when X, Y, N_s, ld, m or the
  // workspace it refers to change
  cudaGraphExec_t f64_gexec = nullptr;
  cudaStream_t f64_cap = nullptr;
  double* f64_coef_d = nullptr;
  double* f64_coef_h = nullptr;
  int f64_coef_cap = 0, f64_m = 0;
  const void* f64_X = nullptr;
  void* f64_Y = nullptr;
  void* f64_T = nullptr;
  int64_t f64_Ns = 0, f64_ld = 0;
  // host-buffer filter: double-buffered device chunks, copy streams, events
  dg::DevBuf ws_hin[2], ws_hout[2];
  cudaStream_t h_in = nullptr, h_out = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_f[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
  std::vector<char> solver_host;
  int* info_d = nullptr;  // [4] cuSOLVER infos + finite flag
  cusolverDnHandle_t solver = nullptr;
  dg::TcState* tc = nullptr;

  dg::HView view() const {
    dg::HView h;
    h.M = M;
    h.N = N;
    h.nb = nb_d;
    h.off = off_d;
    h.row_ptr = row_ptr_d;
    h.col = col_d;
    h.blk_off = blk_off_d;
    h.vals = vals_d;
    h.max_nb = max_nb;
    h.tj = f64_tj;
    return h;
  }
};

namespace dg {

// Thread-local last error message; returns `st`.
dgchefsi_status set_error(dgchefsi_status st, const char* fmt, ...);
void clear_error();
// Make `b` hold at least `bytes` (synchronises the context's stream before a regrow).
dgchefsi_status ensure(dgchefsi_ctx* ctx, DevBuf& b, size_t bytes, const char* what);

// Tensor-core filter (tc_filter.cu). X, Y FP64 (Ns x ld) state-major.
// reuse_hop: the operand copy of H - cI built by the previous call of this
// precision with the same (a, b) is still valid (consecutive chunks of one
// host-buffer call), so it is not rebuilt.
dgchefsi_status filter_tc(dgchefsi_ctx* ctx, int prec, const double* X, double* Y, int64_t Ns, int64_t ld, int m,
                          double a, double b, double a0, bool reuse_hop = false);
// The same filter replayed from a CUDA graph captured for (prec, X, Y, Ns, ld, m).
dgchefsi_status filter_tc_graph(dgchefsi_ctx* ctx, int prec, const double* X, double* Y, int64_t Ns, int64_t ld,
                                int m, double a, double b, double a0);
dgchefsi_status tc_set_shape(dgchefsi_ctx* ctx, int prec, int G, int T, int layout);
dgchefsi_status tc_get_shape(dgchefsi_ctx* ctx, int prec, int* G, int* T, int* ACC, int* layout);
dgchefsi_status tc_wait_selftest(dgchefsi_ctx* ctx, int64_t limit_ns);
dgchefsi_status tc_set_unit_order(dgchefsi_ctx* ctx, int prec, int tgb);
dgchefsi_status tc_get_unit_order(dgchefsi_ctx* ctx, int prec, int* tgb);
// Band-energy gradient on the tensor-core filter. Forward: Y_m (FP64, Ns x N
// compact) from X, keeping FP32 iterate pairs every `stride` steps. Backward
// (same prec, m, stride, right after the forward): the reverse recurrence from
// W_m (FP64 compact), adding alpha_k W_{k+1} Y_k^T to H_bar (values layout,
// may be null) and writing W_0 to X_bar (ld_xbar, may be null).
dgchefsi_status tc_grad_forward(dgchefsi_ctx* ctx, int prec, const double* X, int64_t ld, int64_t Ns, int m,
                                double a, double b, double a0, int stride, double* Ym);
dgchefsi_status tc_grad_backward(dgchefsi_ctx* ctx, int prec, const double* Wm, int64_t Ns, int m, int stride,
                                 double* H_bar, double* X_bar, int64_t ld_xbar);
void tc_destroy(dgchefsi_ctx* ctx);

// C (M x Nc, row-major, ldc) = A B^T (b_rows: B is Nc x K) or A B (B is K x Nc),
// A (M x K, lda) row-major, all FP64, computed from s exact BF16 slices per
// operand on the tensor cores (sliced.cu). a_lower: entries k > r of A are
// zero and not read. flag (device int) gets 1 if an operand is not finite.
// tri > 0: only the entries C[r, c] with c <= r mod tri are computed (the lower
// triangle of a symmetric result, or of each of M / tri stacked ones); the
// others are left as they were.
dgchefsi_status sliced_gemm(dgchefsi_ctx* ctx, bool b_rows, bool a_lower, int64_t M, int64_t Nc, int64_t K,
                            const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, int s,
                            int* flag, int64_t tri = 0);
// C (M x Nc) = A^T B with A (K x M, lda) and B (K x Nc, ldb) row-major: A is
// transposed into a library buffer, then the A B form above.
dgchefsi_status sliced_gemm_tn(dgchefsi_ctx* ctx, int64_t M, int64_t Nc, int64_t K, const double* A, int64_t lda,
                               const double* B, int64_t ldb, double* C, int64_t ldc, int s, int* flag);
void sliced_destroy(dgchefsi_ctx* ctx);

// Slices for the block-sparse product H X (sliced.cu). slices_of_h: the row
// exponents E (element-padded rows) and s digit copies of H in the tensor-core
// operand layout (brow: first row of each block, cstride: elements per copy).
// slices_of_states: the state exponents E[Ns] and s digit copies of X in the
// element-padded layout (cmap: padded column -> column, -1 for padding).
// reduce_pair_slabs: C[r, cmap[c]] = the FP64 sum of the slice-pair slabs
// (rows x cols FP32 each, pair order of the dense form) scaled by Erows[r] + Ecols[c].
cudaError_t slices_of_h(const dgchefsi_ctx* ctx, const int32_t* blk_row, const int32_t* pnb, const int32_t* poff,
                        const int64_t* brow, int s, __nv_bfloat16* Q, int64_t cstride, int32_t* E, int* flag,
                        cudaStream_t st);
cudaError_t slices_of_states(const double* X, int64_t ld, int64_t Ns, int64_t N, const int32_t* cmap, int64_t ldp,
                             int s, __nv_bfloat16* Q, int64_t cstride, int32_t* E, int* flag, cudaStream_t st);
dgchefsi_status reduce_pair_slabs(const float* Pw, int64_t rows, int64_t cols, const int32_t* Erows,
                                  const int32_t* Ecols, const int32_t* cmap, double* C, int64_t ldc, int s,
                                  cudaStream_t st);
// The slice-pair products of the dense sliced GEMM (pair_gemm.cu: tcgen05 on
// pairs of SMs, cta_group::2, all pairs of the chunk in one persistent
// launch): for every pair i + j < s, Pw[pair i*s - i(i-1)/2 + j] (M x pn,
// row-major FP32) = Qa_i[:, k0:k0+kc] times Qb_j[n0:n0+pn, k0:k0+kc]^T, with
// Qa_i = Qa + i*sa (M x K, row stride lqa), Qb_j = Qb + j*sb (Nc x K, row
// stride lqb), entries k >= K read as zero; a_lower: A is lower triangular,
// so a row tile skips the K slices past its last row. Enqueued only.
// pair_products_begin clears the kernel's error word; pair_products_status
// synchronises and reports a pipeline timeout.
dgchefsi_status pair_products_2sm(dgchefsi_ctx* ctx, const __nv_bfloat16* Qa, int64_t lqa, int64_t sa, int64_t M,
                                  const __nv_bfloat16* Qb, int64_t lqb, int64_t sb, int64_t Nc, int64_t K, int64_t k0,
                                  int64_t kc, int64_t n0, int64_t pn, int s, float* Pw, bool a_lower,
                                  int64_t tri = 0);
dgchefsi_status pair_products_begin(dgchefsi_ctx* ctx);
dgchefsi_status pair_products_status(dgchefsi_ctx* ctx);
// Y = H X (X, Y: Ns x ld state-major FP64) from s BF16 slices of each operand on
// the tensor-core filter's step kernel (tc_filter.cu). *used = false when this
// H does not fit the form (a row longer than 4096 columns, or an element
// larger than 128): the caller then runs the FP64 product.
dgchefsi_status tc_sliced_matvec(dgchefsi_ctx* ctx, const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t Ns,
                                 int s, int* flag, bool* used);

// Eigen-decomposition of a symmetric A (eig_refine.cu) with the context's
// eigensolver: on entry the lower triangle (row-major) of A (n x n, lda)
// holds the matrix, the upper one may be overwritten; on exit row i of A is
// the eigenvector of w[i], w ascending. cuSOLVER's FP64 solver reports its
// info in ctx->info_d[2] (checked by the caller); the refined form
// synchronises and records its statistics in the context.
dgchefsi_status subspace_eigh(dgchefsi_ctx* ctx, double* A, int64_t n, int64_t lda, double* w);

// S = L L^T (lower triangle of S, row-major n x n, lda) factored by the
// recursive blocked form whose work is dense products (chol.cu); on return
// the lower triangle of S holds L^{-1} (= U^{-T} for S = U^T U) and the
// strict upper part is unspecified. A pivot that is not positive sets
// *info (device) to its 1-based column; a non-finite operand of a sliced
// product sets *bad. Enqueued on the context's stream (sliced products
// synchronise).
dgchefsi_status cholesky_inverse(dgchefsi_ctx* ctx, double* S, int64_t n, int64_t lda, int* info, int* bad);
// The recursive form for the context's setting: DGCHEFSI_CHOL_PRODUCTS, or
// DGCHEFSI_CHOL_AUTO with sliced subspace products.
inline bool use_own_cholesky(const dgchefsi_ctx* ctx) {
  return ctx->chol_mode == DGCHEFSI_CHOL_PRODUCTS ||
         (ctx->chol_mode == DGCHEFSI_CHOL_AUTO && ctx->products_mode == DGCHEFSI_PRODUCTS_SLICED_BF16);
}

// Set-up of dgchefsi_bounds_static for `device` (noalloc.cu), run by
// dgchefsi_create with that device current: looks up the device address of
// the fixed scratch array (which loads its module, so the array is resident
// from then on) and loads the Lanczos kernels' modules.
dgchefsi_status bounds_static_setup(int device);

}  // namespace dg

#define DG_CUDA(call)                                                                               \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      return dg::set_error(DGCHEFSI_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                           __FILE__, __LINE__);                                                     \
  } while (0)

#define DG_TRY(call)                          \
  do {                                        \
    dgchefsi_status st_ = (call);             \
    if (st_ != DGCHEFSI_OK) return st_;       \
  } while (0)
