// Band energy of one CheFSI cycle and its adjoint (differentiation of the
// cycle; the paper itself does not differentiate it).
//
// E(H, X) = sum_i f_i lambda_i after one cycle (Alg. 1 steps 2-5 and the
// occupations) with the filter bounds, N_e and kT held fixed. Backward:
//   * g_i = dE/dlambda_i = f_i + lambda_i f'_i - f'_i (sum_j lambda_j f'_j)/(sum_j f'_j),
//     f'_i = -f_i (1 - f_i)/kT (the Fermi level follows the eigenvalues);
//   * Rayleigh-Ritz: with Z = U^{-1} Q (X_new = Y~ Z) and R = H X_new - X_new Lambda,
//     dE/dH += sum_i g_i x_i x_i^T on H's block pattern and Y~bar = 2 R G Z^T;
//   * filter: the recurrence Y_{k+1} = alpha_k (H - cI) Y_k - beta_k Y_{k-1} run
//     backwards, W_m = Y~bar, dE/dH += alpha_k W_{k+1} Y_k^T,
//     W_k = alpha_k (H - cI) W_{k+1} - beta_{k+1} W_{k+2}, Xbar = W_0.
// The backward recurrence is the forward step kernel with other coefficients.
// With a tensor-core precision the filter, its checkpoints (FP32), the
// recomputed segments and the backward recurrence run on the tensor-core step
// kernel, and alpha_k W_{k+1} Y_k^T is accumulated from FP32 iterates into
// FP64; Cholesky-QR, Rayleigh-Ritz and their adjoint stay FP64.
// Iterates Y_k are not all stored: pairs (Y_{js}, Y_{js+1}) are kept every s
// steps (s = ceil(sqrt(m)) by default, a three-term restart needs two
// iterates) and each segment is recomputed in reverse order, so the memory is
// about 2 m/s + s blocks instead of m.
#include <cmath>
#include <vector>

#include "ctx.h"

namespace dg {
namespace {

#define ADJ_SOLVER(call)                                                                     \
  do {                                                                                       \
    cusolverStatus_t s_ = (call);                                                            \
    if (s_ != CUSOLVER_STATUS_SUCCESS)                                                       \
      return set_error(DGCHEFSI_ERR_CUDA, "%s failed (cusolver status %d)", #call, (int)s_); \
  } while (0)

struct Coeffs {
  double c = 0.0;
  std::vector<double> alpha, beta;  // alpha_k, beta_k for k = 0 .. m-1 (beta_0 = 0)
};

Coeffs coefficients(int m, double a, double b, double a0) {
  Coeffs r;
  const double e = 0.5 * (b - a);
  r.c = 0.5 * (b + a);
  const double s1 = e / (a0 - r.c);
  double sig = s1;
  r.alpha.push_back(s1 / e);
  r.beta.push_back(0.0);
  for (int k = 1; k < m; ++k) {
    const double sn = 1.0 / (2.0 / s1 - sig);
    r.alpha.push_back(2.0 * sn / e);
    r.beta.push_back(sig * sn);
    sig = sn;
  }
  return r;
}

}  // namespace
}  // namespace dg

using namespace dg;

extern "C" dgchefsi_status dgchefsi_set_values(dgchefsi_ctx* ctx, const double* values) {
  clear_error();
  if (!ctx) return set_error(DGCHEFSI_ERR_ARG, "null context");
  if (!values) return set_error(DGCHEFSI_ERR_ARG, "null values");
  DG_CUDA(cudaMemcpyAsync(ctx->vals_d, values, sizeof(double) * (size_t)ctx->n_values, cudaMemcpyDeviceToDevice,
                          ctx->stream));
  if (ctx->tc) tc_destroy(ctx);  // operand copies of H are rebuilt from the new values
  return DGCHEFSI_OK;
}

extern "C" dgchefsi_status dgchefsi_energy_grad(dgchefsi_ctx* ctx, int prec, const double* X, int64_t Ns, int64_t ld,
                                                int m, double a, double b, double a0, double Ne, double kT,
                                                int checkpoint_stride, double* energy, double* ritz, double* H_bar,
                                                double* X_bar) {
  clear_error();
  if (!ctx) return set_error(DGCHEFSI_ERR_ARG, "null context");
  if (prec != DGCHEFSI_F64 && prec != DGCHEFSI_TF32 && prec != DGCHEFSI_BF16 && prec != DGCHEFSI_BF16X3)
    return set_error(DGCHEFSI_ERR_ARG, "unknown precision %d", prec);
  const bool tc = prec != DGCHEFSI_F64;
  if (!X || !energy || Ns < 1) return set_error(DGCHEFSI_ERR_ARG, "need X, energy and Ns >= 1");
  if (ld < ctx->N) return set_error(DGCHEFSI_ERR_ARG, "ld < N");
  if (Ns > ctx->N) return set_error(DGCHEFSI_ERR_ARG, "Ns > N");
  if (m < 1 || !(a0 < a && a < b) || !std::isfinite(a) || !std::isfinite(b) || !std::isfinite(a0))
    return set_error(DGCHEFSI_ERR_ARG, "need m >= 1 and a0 < a < b");
  if (!(kT > 0.0) || !(Ne >= 0.0) || Ne > 2.0 * (double)Ns)
    return set_error(DGCHEFSI_ERR_ARG, "need kT > 0 and 0 <= Ne <= 2 Ns");
  if (checkpoint_stride < 0) return set_error(DGCHEFSI_ERR_ARG, "checkpoint stride < 0");
  const bool want_grad = H_bar || X_bar;
  const int64_t N = ctx->N;
  const int n = (int)Ns;
  cudaStream_t s = ctx->stream;
  const HView h = ctx->view();
  const Coeffs cf = coefficients(m, a, b, a0);
  int stride = checkpoint_stride > 0 ? checkpoint_stride : (int)std::ceil(std::sqrt((double)m));
  if (stride > m) stride = m;
  const int nseg = (m + stride - 1) / stride;

  // ---- workspace: every block is (Ns x N) FP64, compact (ld = N)
  const size_t blk = (size_t)Ns * (size_t)N;
  const int nbig = (want_grad && !tc) ? (2 * nseg + stride + 9) : (want_grad ? 9 : 8);
  const size_t small = (size_t)Ns * (size_t)Ns;
  DG_TRY(ensure(ctx, ctx->ws_adjoint, sizeof(double) * (blk * nbig + 3 * small + 4 * (size_t)Ns + 8),
                "band-energy workspace"));
  double* base = static_cast<double*>(ctx->ws_adjoint.p);
  int next_blk = 0;
  auto take = [&]() { return base + blk * (size_t)(next_blk++); };
  double* Yt = take();   // Y_m
  double* Yh = take();   // Y_hat
  double* HY = take();   // H Y_hat
  double* XN = take();   // X_new
  double* HXN = take();  // H X_new
  double* T0 = take();
  double* T1 = take();
  double* T2 = take();
  std::vector<double*> cp0(nseg), cp1(nseg), seg;
  if (want_grad && !tc) {
    for (int j = 0; j < nseg; ++j) {
      cp0[j] = take();
      cp1[j] = take();
    }
    for (int i = 0; i < stride; ++i) seg.push_back(take());
  }
  double* WA = want_grad ? take() : nullptr;
  double* S = base + blk * (size_t)nbig;
  double* L = S + small;
  double* Z = L + small;
  double* lam = Z + small;
  double* f = lam + Ns;
  double* g = f + Ns;
  double* mu = g + Ns;

  // ---- forward filter, copying the checkpoint pairs (Y_{js}, Y_{js+1})
  auto copy_blk = [&](double* dst, int64_t ldd, const double* src, int64_t lds) -> dgchefsi_status {
    DG_CUDA(cudaMemcpy2DAsync(dst, sizeof(double) * ldd, src, sizeof(double) * lds, sizeof(double) * N, Ns,
                              cudaMemcpyDeviceToDevice, s));
    return DGCHEFSI_OK;
  };
  if (tc && want_grad) {
    // tensor-core filter; FP32 checkpoints are kept inside the filter state
    DG_TRY(tc_grad_forward(ctx, prec, X, ld, Ns, m, a, b, a0, stride, Yt));
  } else if (tc) {
    // energy only: the ordinary tensor-core filter (same kernel, no checkpoints)
    // on a compact copy of X
    DG_TRY(copy_blk(T0, N, X, ld));
    DG_TRY(filter_tc(ctx, prec, T0, Yt, Ns, N, m, a, b, a0));
  } else {
    // Y_0 = X (caller layout ld); iterates in T0/T1/T2 rotation (ld = N)
    double* rot[3] = {T0, T1, T2};
    const double* prev = nullptr;
    const double* cur = X;
    int64_t ldc = ld;
    if (want_grad) DG_TRY(copy_blk(cp0[0], N, X, ld));
    for (int k = 0; k < m; ++k) {
      double* out = (k == m - 1) ? Yt : rot[k % 3];
      DG_CUDA(filter_step_f64(h, cur, ldc, k == 0 ? nullptr : prev, out, N, Ns, cf.alpha[k], cf.c,
                              k == 0 ? 0.0 : cf.beta[k], s));
      const int kk = k + 1;  // index of the iterate just produced
      if (want_grad && kk < m) {
        if (kk % stride == 0) DG_TRY(copy_blk(cp0[kk / stride], N, out, N));
        if (kk % stride == 1) DG_TRY(copy_blk(cp1[kk / stride], N, out, N));
      }
      prev = cur;
      cur = out;
      ldc = N;
    }
  }
  // ---- Cholesky-QR and Rayleigh-Ritz, keeping U^{-T} (L) and Q^T (row-major views).
  // The dense products run on the FP64 cores or from exact BF16 slices on the
  // tensor cores, as the context's product setting says (non-finite operands
  // of the sliced form raise info[3]).
  const bool sl = ctx->products_mode == DGCHEFSI_PRODUCTS_SLICED_BF16;
  const int nsl = ctx->products_slices;
  int* bad = ctx->info_d + 3;
  // C = A B^T, K = N, for a symmetric C of which only the lower triangle is
  // read (the Cholesky factorisation and the eigensolver)
  auto prod_nt = [&](const double* A_, const double* B_, double* C_) -> dgchefsi_status {
    if (sl) return sliced_gemm(ctx, true, false, Ns, Ns, N, A_, N, B_, N, C_, Ns, nsl, bad, Ns);
    DG_CUDA(gemm_nt_f64(A_, N, B_, N, C_, Ns, Ns, Ns, N, true, false, s));
    return DGCHEFSI_OK;
  };
  auto prod_nn = [&](const double* A_, const double* B_, int64_t ldb_, int64_t cols, double* C_, int64_t ldc_,
                     bool lower) -> dgchefsi_status {  // C = A B, A N_s x N_s, K = N_s
    if (sl) return sliced_gemm(ctx, false, lower, Ns, cols, Ns, A_, Ns, B_, ldb_, C_, ldc_, nsl, bad);
    DG_CUDA(gemm_nn_f64(A_, Ns, B_, ldb_, C_, ldc_, Ns, cols, Ns, lower, s));
    return DGCHEFSI_OK;
  };
  DG_CUDA(cudaMemsetAsync(ctx->info_d, 0, 4 * sizeof(int), s));
  DG_TRY(prod_nt(Yt, Yt, S));
  ADJ_SOLVER(cusolverDnSetStream(ctx->solver, s));
  int lw_potrf = 0, lw_syevd = 0;
  size_t lw_tr_d = 0, lw_tr_h = 0;
  ADJ_SOLVER(cusolverDnDpotrf_bufferSize(ctx->solver, CUBLAS_FILL_MODE_UPPER, n, S, n, &lw_potrf));
  ADJ_SOLVER(cusolverDnXtrtri_bufferSize(ctx->solver, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, Ns, CUDA_R_64F, S,
                                         Ns, &lw_tr_d, &lw_tr_h));
  ADJ_SOLVER(cusolverDnDsyevd_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, n, S, n, lam,
                                         &lw_syevd));
  size_t need = sizeof(double) * (size_t)std::max(lw_potrf, lw_syevd);
  if (lw_tr_d > need) need = lw_tr_d;
  DG_TRY(ensure(ctx, ctx->ws_solver, need, "cuSOLVER workspace"));
  if (ctx->solver_host.size() < lw_tr_h) ctx->solver_host.resize(lw_tr_h);
  double* work = static_cast<double*>(ctx->ws_solver.p);
  const int lwork = (int)(ctx->ws_solver.bytes / sizeof(double));
  const bool own_chol = use_own_cholesky(ctx);
  if (own_chol)
    DG_TRY(cholesky_inverse(ctx, S, Ns, Ns, ctx->info_d, bad));
  else
    ADJ_SOLVER(cusolverDnDpotrf(ctx->solver, CUBLAS_FILL_MODE_UPPER, n, S, n, work, lwork, ctx->info_d));
  int info[4] = {0, 0, 0, 0};
  DG_CUDA(cudaMemcpyAsync(info, ctx->info_d, sizeof(int), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  if (info[0] != 0) return set_error(DGCHEFSI_ERR_NOT_SPD, "Cholesky of S = Y^T Y failed at column %d", info[0]);
  if (!own_chol)
    ADJ_SOLVER(cusolverDnXtrtri(ctx->solver, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, Ns, CUDA_R_64F, S, Ns,
                                work, ctx->ws_solver.bytes,
                                ctx->solver_host.empty() ? nullptr : ctx->solver_host.data(), lw_tr_h,
                                ctx->info_d + 1));
  DG_CUDA(zero_strict_upper_f64(S, Ns, Ns, s));  // S now holds L = U^{-T} exactly (lower)
  DG_CUDA(cudaMemcpyAsync(L, S, sizeof(double) * small, cudaMemcpyDeviceToDevice, s));
  DG_TRY(prod_nn(L, Yt, N, N, Yh, N, true));
  bool hy_sliced = false;  // H Y_hat from BF16 slices too, when H fits that form
  if (sl) DG_TRY(tc_sliced_matvec(ctx, Yh, N, HY, N, Ns, nsl, bad, &hy_sliced));
  if (!hy_sliced) DG_CUDA(filter_step_f64(h, Yh, N, nullptr, HY, N, Ns, 1.0, 0.0, 0.0, s));
  DG_TRY(prod_nt(Yh, HY, S));
  DG_TRY(subspace_eigh(ctx, S, Ns, Ns, lam));
  DG_TRY(prod_nn(S, Yh, N, N, XN, N, false));   // X_new^T = Q^T Y_hat^T
  DG_TRY(prod_nn(S, HY, N, N, HXN, N, false));  // (H X_new)^T
  DG_CUDA(occupations_f64(lam, Ns, Ne, kT, f, mu, s));
  std::vector<double> lam_h(Ns), f_h(Ns);
  DG_CUDA(cudaMemcpyAsync(lam_h.data(), lam, sizeof(double) * Ns, cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaMemcpyAsync(f_h.data(), f, sizeof(double) * Ns, cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaMemcpyAsync(info, ctx->info_d, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  if (info[1] != 0) return set_error(DGCHEFSI_ERR_NOT_SPD, "triangular inverse failed (info %d)", info[1]);
  if (info[2] != 0) return set_error(DGCHEFSI_ERR_NO_CONVERGENCE, "dense eigensolver failed (info %d)", info[2]);
  if (sl && info[3] != 0) return set_error(DGCHEFSI_ERR_NONFINITE, "non-finite Rayleigh-Ritz operand");
  double E = 0.0;
  for (int64_t i = 0; i < Ns; ++i) E += f_h[i] * lam_h[i];
  if (!std::isfinite(E)) return set_error(DGCHEFSI_ERR_NONFINITE, "non-finite band energy");
  *energy = E;
  if (ritz) DG_CUDA(cudaMemcpyAsync(ritz, lam, sizeof(double) * Ns, cudaMemcpyDeviceToDevice, s));
  if (!want_grad) {
    DG_CUDA(cudaStreamSynchronize(s));
    return DGCHEFSI_OK;
  }

  // ---- backward: eigenvalue weights
  std::vector<double> g_h(Ns);
  double sfp = 0.0, slfp = 0.0;
  for (int64_t i = 0; i < Ns; ++i) {
    const double fp = -f_h[i] * (1.0 - f_h[i]) / kT;
    sfp += fp;
    slfp += lam_h[i] * fp;
  }
  const double shift = sfp != 0.0 ? slfp / sfp : 0.0;
  for (int64_t i = 0; i < Ns; ++i) {
    const double fp = -f_h[i] * (1.0 - f_h[i]) / kT;
    g_h[i] = f_h[i] + lam_h[i] * fp - fp * shift;
  }
  DG_CUDA(cudaMemcpyAsync(g, g_h.data(), sizeof(double) * Ns, cudaMemcpyHostToDevice, s));
  double* Hb = H_bar;
  if (Hb) {
    DG_CUDA(cudaMemsetAsync(Hb, 0, sizeof(double) * (size_t)ctx->n_values, s));
    DG_CUDA(block_outer_f64(h, ctx->blk_row_d, ctx->nnzb, XN, N, XN, N, g, 1.0, Ns, Hb, s));
  }
  // Y~bar = 2 R G Z^T, in state-major form Y~bar^T = Z (2 G R^T), Z^T = Q^T L
  DG_CUDA(scaled_residual_f64(HXN, XN, N, lam, g, 2.0, Ns, N, T0, N, s));
  DG_TRY(prod_nn(S, L, Ns, Ns, Z, Ns, false));  // Z^T = Q^T L
  if (sl)                                        // W_m = Z (2 G R^T)
    DG_TRY(sliced_gemm_tn(ctx, Ns, N, Ns, Z, Ns, T0, N, WA, N, nsl, bad));
  else
    DG_CUDA(gemm_tn_f64(Z, Ns, T0, N, WA, N, Ns, N, Ns, s));
  if (tc) {
    DG_TRY(tc_grad_backward(ctx, prec, WA, Ns, m, stride, Hb, X_bar, ld));
    DG_CUDA(cudaStreamSynchronize(s));
    return DGCHEFSI_OK;
  }
  // ---- filter backward, segment by segment from the last
  double* Wcur = WA;   // W_{k+1}
  double* Wprev = T1;  // W_{k+2} (unused while beta_{k+1} = 0)
  bool have_prev = false;
  for (int j = nseg - 1; j >= 0; --j) {
    const int k0 = j * stride, k1 = std::min(m, k0 + stride);
    // recompute Y_{k0} .. Y_{k1-1} into seg[0 .. k1-k0-1]
    DG_TRY(copy_blk(seg[0], N, cp0[j], N));
    if (k1 - k0 > 1) DG_TRY(copy_blk(seg[1], N, cp1[j], N));
    for (int kk = k0 + 2; kk < k1; ++kk) {
      const int q = kk - k0;
      DG_CUDA(filter_step_f64(h, seg[q - 1], N, seg[q - 2], seg[q], N, Ns, cf.alpha[kk - 1], cf.c, cf.beta[kk - 1], s));
    }
    for (int k = k1 - 1; k >= k0; --k) {
      if (Hb) DG_CUDA(block_outer_f64(h, ctx->blk_row_d, ctx->nnzb, Wcur, N, seg[k - k0], N, nullptr, cf.alpha[k], Ns,
                                      Hb, s));
      const double bnext = (k + 1 < m) ? cf.beta[k + 1] : 0.0;
      // W_k = alpha_k (H - cI) W_{k+1} - beta_{k+1} W_{k+2}, written over W_{k+2}
      double* out = Wprev;
      DG_CUDA(filter_step_f64(h, Wcur, N, have_prev ? Wprev : nullptr, out, N, Ns, cf.alpha[k], cf.c,
                              have_prev ? bnext : 0.0, s));
      Wprev = Wcur;
      Wcur = out;
      have_prev = true;
    }
  }
  if (X_bar) DG_TRY(copy_blk(X_bar, ld, Wcur, N));
  DG_CUDA(cudaStreamSynchronize(s));
  return DGCHEFSI_OK;
}
