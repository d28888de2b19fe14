// C ABI of the DG-CheFSI library: context set-up and validation, the FP64
// filter driver, Lanczos bounds, Cholesky-QR / Rayleigh-Ritz, occupations,
// density blocks and the full cycle (Alg. 1). Kernels live in f64_kernels.cu
// and tc_filter.cu; the dense factorisations (Cholesky, triangular inverse,
// symmetric eigensolve of the N_s x N_s projected matrix) are cuSOLVER calls.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>

#include "ctx.h"

namespace dg {

int64_t launch_count();

static thread_local std::string g_err;

dgchefsi_status set_error(dgchefsi_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

void clear_error() { g_err.clear(); }

dgchefsi_status ensure(dgchefsi_ctx* ctx, DevBuf& b, size_t bytes, const char* what) {
  if (b.bytes >= bytes && b.p) return DGCHEFSI_OK;
  if (b.p) {
    DG_CUDA(cudaStreamSynchronize(ctx->stream));
    DG_CUDA(cudaFree(b.p));
    b.p = nullptr;
    b.bytes = 0;
  }
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return set_error(DGCHEFSI_ERR_OOM, "cudaMalloc of %zu bytes for %s failed: %s", bytes, what,
                     cudaGetErrorString(e));
  }
  b.bytes = bytes;
  return DGCHEFSI_OK;
}

static void free_buf(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

static const char* solver_str(cusolverStatus_t s) {
  switch (s) {
    case CUSOLVER_STATUS_SUCCESS: return "success";
    case CUSOLVER_STATUS_NOT_INITIALIZED: return "not initialized";
    case CUSOLVER_STATUS_ALLOC_FAILED: return "alloc failed";
    case CUSOLVER_STATUS_INVALID_VALUE: return "invalid value";
    case CUSOLVER_STATUS_ARCH_MISMATCH: return "arch mismatch";
    case CUSOLVER_STATUS_EXECUTION_FAILED: return "execution failed";
    case CUSOLVER_STATUS_INTERNAL_ERROR: return "internal error";
    default: return "other cusolver error";
  }
}

#define DG_SOLVER(call)                                                                              \
  do {                                                                                               \
    cusolverStatus_t s_ = (call);                                                                    \
    if (s_ != CUSOLVER_STATUS_SUCCESS)                                                               \
      return dg::set_error(DGCHEFSI_ERR_CUDA, "%s failed: %s", #call, solver_str(s_));                \
  } while (0)

// Smallest / largest eigenvalue of the symmetric tridiagonal T (diag a, off b)
// by Sturm-sequence bisection.
static int sturm_count(const std::vector<double>& a, const std::vector<double>& b, double x) {
  int cnt = 0;
  double q = a[0] - x;
  const double tiny = 1e-300;
  if (q < 0) ++cnt;
  for (size_t i = 1; i < a.size(); ++i) {
    if (q == 0.0) q = tiny;
    q = (a[i] - x) - b[i - 1] * b[i - 1] / q;
    if (q < 0) ++cnt;
  }
  return cnt;
}

static double tridiag_eig(const std::vector<double>& a, const std::vector<double>& b, int which /*1-based*/) {
  double lo = a[0], hi = a[0];
  for (size_t i = 0; i < a.size(); ++i) {
    double r = 0;
    if (i > 0) r += std::fabs(b[i - 1]);
    if (i + 1 < a.size()) r += std::fabs(b[i]);
    lo = std::fmin(lo, a[i] - r);
    hi = std::fmax(hi, a[i] + r);
  }
  const double span = std::fmax(std::fabs(lo), std::fabs(hi));
  lo -= 1e-12 * span + 1e-300;
  hi += 1e-12 * span + 1e-300;
  for (int it = 0; it < 400; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(a, b, mid) >= which) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

static dgchefsi_status check_ctx(const dgchefsi_ctx* ctx) {
  if (!ctx) return set_error(DGCHEFSI_ERR_ARG, "null context");
  return DGCHEFSI_OK;
}

static dgchefsi_status check_block(const dgchefsi_ctx* ctx, const void* X, int64_t Ns, int64_t ld, const char* name) {
  if (Ns < 0) return set_error(DGCHEFSI_ERR_ARG, "Ns < 0");
  if (ld < ctx->N) return set_error(DGCHEFSI_ERR_ARG, "ld (%lld) < N (%lld)", (long long)ld, (long long)ctx->N);
  if (Ns > 0 && !X) return set_error(DGCHEFSI_ERR_ARG, "null %s", name);
  return DGCHEFSI_OK;
}

static bool overlaps(const void* a, const void* b, size_t bytes) {
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + bytes && pb < pa + bytes;
}

static dgchefsi_status filter_f64(dgchefsi_ctx* ctx, const double* X, double* Y, int64_t Ns, int64_t ld, int m,
                                  double a, double b, double a0) {
  const double e = 0.5 * (b - a), c = 0.5 * (b + a);
  const double s1 = e / (a0 - c);
  double* T = nullptr;
  if (m >= 2) {
    DG_TRY(ensure(ctx, ctx->ws_filter, sizeof(double) * (size_t)Ns * (size_t)ld, "filter iterate"));
    T = static_cast<double*>(ctx->ws_filter.p);
  }
  // Ping-pong: Y_odd -> A, Y_even -> B, so Y_m lands in Y. Y_{k+1} overwrites
  // Y_{k-1} in place (each output entry reads its own prev entry only).
  double* A = (m % 2 == 1) ? Y : T;
  double* B = (m % 2 == 1) ? T : Y;
  const HView h = ctx->view();
  DG_CUDA(filter_step_f64(h, X, ld, nullptr, A, ld, Ns, s1 / e, c, 0.0, ctx->stream));
  const double* prev = X;
  double* cur = A;
  double sig = s1;
  for (int k = 1; k < m; ++k) {
    const double sn = 1.0 / (2.0 / s1 - sig);
    double* out = (k % 2 == 1) ? B : A;
    DG_CUDA(filter_step_f64(h, cur, ld, prev, out, ld, Ns, 2.0 * sn / e, c, sig * sn, ctx->stream));
    prev = cur;
    cur = out;
    sig = sn;
  }
  return DGCHEFSI_OK;
}

// The FP64 filter captured once as a graph (coefficient copy + m steps, the
// same ping-pong as filter_f64) and replayed.
static dgchefsi_status filter_f64_graph(dgchefsi_ctx* ctx, const double* X, double* Y, int64_t Ns, int64_t ld, int m,
                                        double a, double b, double a0) {
  cudaStream_t s = ctx->stream;
  // the previous replay may still read the pinned mirror or the coefficients
  DG_CUDA(cudaStreamSynchronize(s));
  if (ctx->f64_coef_cap < 1 + 2 * m) {
    if (ctx->f64_gexec) {
      cudaGraphExecDestroy(ctx->f64_gexec);
      ctx->f64_gexec = nullptr;
    }
    cudaFree(ctx->f64_coef_d);
    cudaFreeHost(ctx->f64_coef_h);
    ctx->f64_coef_d = nullptr;
    ctx->f64_coef_h = nullptr;
    ctx->f64_coef_cap = 0;
    DG_CUDA(cudaMalloc(&ctx->f64_coef_d, sizeof(double) * (1 + 2 * m)));
    DG_CUDA(cudaMallocHost(&ctx->f64_coef_h, sizeof(double) * (1 + 2 * m)));
    ctx->f64_coef_cap = 1 + 2 * m;
  }
  const double e = 0.5 * (b - a), c = 0.5 * (b + a);
  const double s1 = e / (a0 - c);
  double* ch = ctx->f64_coef_h;
  ch[0] = c;
  ch[1] = s1 / e;
  ch[2] = 0.0;
  double sig = s1;
  for (int k = 1; k < m; ++k) {
    const double sn = 1.0 / (2.0 / s1 - sig);
    ch[1 + 2 * k] = 2.0 * sn / e;
    ch[2 + 2 * k] = sig * sn;
    sig = sn;
  }
  double* T = nullptr;
  if (m >= 2) {  // a regrow moves the workspace; the graph key below then differs
    DG_TRY(ensure(ctx, ctx->ws_filter, sizeof(double) * (size_t)Ns * (size_t)ld, "filter iterate"));
    T = static_cast<double*>(ctx->ws_filter.p);
  }
  const bool same = ctx->f64_gexec && ctx->f64_m == m && ctx->f64_X == X && ctx->f64_Y == Y && ctx->f64_Ns == Ns &&
                    ctx->f64_ld == ld && ctx->f64_T == (void*)T;
  if (!same) {
    if (ctx->f64_gexec) {
      cudaGraphExecDestroy(ctx->f64_gexec);
      ctx->f64_gexec = nullptr;
    }
    if (!ctx->f64_cap) DG_CUDA(cudaStreamCreateWithFlags(&ctx->f64_cap, cudaStreamNonBlocking));
    cudaStream_t cs = ctx->f64_cap;
    const HView h = ctx->view();
    double* A = (m % 2 == 1) ? Y : T;
    double* B = (m % 2 == 1) ? T : Y;
    cudaGraph_t graph = nullptr;
    DG_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = cudaMemcpyAsync(ctx->f64_coef_d, ctx->f64_coef_h, sizeof(double) * (1 + 2 * m),
                                      cudaMemcpyHostToDevice, cs);
    if (err == cudaSuccess) err = filter_step_f64_dev(h, X, ld, nullptr, A, ld, Ns, ctx->f64_coef_d, 0, cs);
    const double* prev = X;
    double* cur = A;
    for (int k = 1; k < m && err == cudaSuccess; ++k) {
      double* out = (k % 2 == 1) ? B : A;
      err = filter_step_f64_dev(h, cur, ld, prev, out, ld, Ns, ctx->f64_coef_d, k, cs);
      prev = cur;
      cur = out;
    }
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (err != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return set_error(DGCHEFSI_ERR_CUDA, "capture of the FP64 filter graph failed: %s",
                       cudaGetErrorString(err != cudaSuccess ? err : e2));
    }
    cudaError_t e3 = cudaGraphInstantiate(&ctx->f64_gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e3 != cudaSuccess) {
      ctx->f64_gexec = nullptr;
      return set_error(DGCHEFSI_ERR_CUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(e3));
    }
    ctx->f64_m = m;
    ctx->f64_T = T;
    ctx->f64_X = X;
    ctx->f64_Y = Y;
    ctx->f64_Ns = Ns;
    ctx->f64_ld = ld;
  }
  DG_CUDA(cudaGraphLaunch(ctx->f64_gexec, s));
  count_launch(m);
  return DGCHEFSI_OK;
}

static dgchefsi_status bounds_impl(dgchefsi_ctx* ctx, const double* v0, int k, double* b_upper, double* theta_min) {
  const int64_t N = ctx->N;
  if (k > N) k = (int)N;
  const size_t nvec = (size_t)k + 1;
  DG_TRY(ensure(ctx, ctx->ws_lanczos, sizeof(double) * (nvec * (size_t)N + (size_t)N + 72), "Lanczos basis"));
  double* V = static_cast<double*>(ctx->ws_lanczos.p);
  double* w = V + nvec * (size_t)N;
  double* sc = w + N;  // device scalars [72]
  cudaStream_t s = ctx->stream;
  double host[72];
  auto fetch = [&](int n) -> dgchefsi_status {
    DG_CUDA(cudaMemcpyAsync(host, sc, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaStreamSynchronize(s));
    return DGCHEFSI_OK;
  };
  DG_CUDA(dots_f64(v0, 0, 1, v0, N, sc, s));
  DG_TRY(fetch(1));
  const double nrm = std::sqrt(host[0]);
  if (!(nrm > 0.0) || !std::isfinite(nrm)) return set_error(DGCHEFSI_ERR_ARG, "Lanczos start vector is zero or not finite");
  DG_CUDA(axpby_f64(1.0 / nrm, v0, 0.0, v0, V, N, s));
  std::vector<double> al, be;
  double beta_prev = 0.0, beta_last = 0.0;
  const HView h = ctx->view();
  for (int j = 0; j < k; ++j) {
    double* vj = V + (size_t)j * N;
    DG_CUDA(spmv_f64(h, vj, w, s));
    if (j > 0) DG_CUDA(axpby_f64(-beta_prev, vj - N, 1.0, w, w, N, s));
    DG_CUDA(dots_f64(vj, 0, 1, w, N, sc, s));
    DG_TRY(fetch(1));
    const double alpha = host[0];
    DG_CUDA(axpby_f64(-alpha, vj, 1.0, w, w, N, s));
    DG_CUDA(dots_f64(V, N, j + 1, w, N, sc, s));
    DG_CUDA(sub_combination_f64(w, V, N, sc, j + 1, N, s));
    DG_CUDA(dots_f64(w, 0, 1, w, N, sc + 64, s));
    DG_CUDA(cudaMemcpyAsync(host, sc + 64, sizeof(double), cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaStreamSynchronize(s));
    const double beta = std::sqrt(host[0]);
    al.push_back(alpha);
    beta_last = beta;
    if (!std::isfinite(alpha) || !std::isfinite(beta))
      return set_error(DGCHEFSI_ERR_NONFINITE, "Lanczos produced a non-finite coefficient");
    if (j == k - 1 || beta == 0.0) break;
    be.push_back(beta);
    DG_CUDA(axpby_f64(1.0 / beta, w, 0.0, w, vj + N, N, s));
    beta_prev = beta;
  }
  const int n = (int)al.size();
  const double tmax = tridiag_eig(al, be, n);
  const double tmin = tridiag_eig(al, be, 1);
  *b_upper = tmax + std::fabs(beta_last);
  if (theta_min) *theta_min = tmin;
  return DGCHEFSI_OK;
}

static dgchefsi_status rr_impl(dgchefsi_ctx* ctx, double* Y, int64_t Ns, int64_t ld, double* ritz) {
  const int64_t N = ctx->N;
  cudaStream_t s = ctx->stream;
  DG_TRY(ensure(ctx, ctx->ws_rr, sizeof(double) * (size_t)Ns * (size_t)N, "Rayleigh-Ritz block"));
  DG_TRY(ensure(ctx, ctx->ws_small, sizeof(double) * (size_t)Ns * (size_t)Ns, "N_s x N_s matrix"));
  double* W = static_cast<double*>(ctx->ws_rr.p);
  double* S = static_cast<double*>(ctx->ws_small.p);
  const int n = (int)Ns;
  DG_SOLVER(cusolverDnSetStream(ctx->solver, s));
  // workspace sizes
  int lw_potrf = 0, lw_syevd = 0;
  size_t lw_trtri_d = 0, lw_trtri_h = 0;
  DG_SOLVER(cusolverDnDpotrf_bufferSize(ctx->solver, CUBLAS_FILL_MODE_UPPER, n, S, n, &lw_potrf));
  DG_SOLVER(cusolverDnXtrtri_bufferSize(ctx->solver, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, Ns, CUDA_R_64F, S,
                                        Ns, &lw_trtri_d, &lw_trtri_h));
  DG_SOLVER(cusolverDnDsyevd_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, n, S, n, ritz,
                                        &lw_syevd));
  size_t need = sizeof(double) * (size_t)std::max(lw_potrf, lw_syevd);
  if (lw_trtri_d > need) need = lw_trtri_d;
  DG_TRY(ensure(ctx, ctx->ws_solver, need, "cuSOLVER workspace"));
  if (ctx->solver_host.size() < lw_trtri_h) ctx->solver_host.resize(lw_trtri_h);
  double* work = static_cast<double*>(ctx->ws_solver.p);
  const int lwork = (int)(ctx->ws_solver.bytes / sizeof(double));
  DG_CUDA(cudaMemsetAsync(ctx->info_d, 0, 4 * sizeof(int), s));
  int info[4] = {0, 0, 0, 0};
  // Products on the FP64 cores, or from exact BF16 slices on the tensor cores
  // (non-finite operands there raise info[3], like a non-finite Ritz value).
  const bool sl = ctx->products_mode == DGCHEFSI_PRODUCTS_SLICED_BF16;
  const bool own_chol = use_own_cholesky(ctx);
  int* bad = ctx->info_d + 3;
  // Step 3: S = Y^T Y (lower tiles, mirrored), S = U^T U, Y_hat = Y U^{-1}.
  // CholeskyQR2 repeats the pass on Y_hat; shifted CholeskyQR3 factors
  // Y^T Y + s I first, s = 11 (N N_s + N_s (N_s + 1)) u ||Y||_F^2, then repeats
  // twice. Pass 1 reads Y and writes W; later passes read W, write Y and copy
  // back, so Y_hat always ends in W (state-major, ld N).
  const int passes = ctx->orth_mode == DGCHEFSI_ORTH_CHOLQR2 ? 2 : (ctx->orth_mode == DGCHEFSI_ORTH_SHIFTED_CHOLQR3 ? 3 : 1);
  for (int pass = 0; pass < passes; ++pass) {
    const double* in = pass == 0 ? Y : W;
    const int64_t ldi = pass == 0 ? ld : N;
    double* outp = pass == 0 ? W : Y;
    const int64_t ldo = pass == 0 ? N : ld;
    if (sl)
      DG_TRY(sliced_gemm(ctx, true, false, Ns, Ns, N, in, ldi, in, ldi, S, Ns, ctx->products_slices, bad, Ns));
    else
      DG_CUDA(gemm_nt_f64(in, ldi, in, ldi, S, Ns, Ns, Ns, N, true, false, s));
    if (pass == 0 && ctx->orth_mode == DGCHEFSI_ORTH_SHIFTED_CHOLQR3)
      DG_CUDA(shift_diagonal_by_trace_f64(S, Ns, 11.0 * ((double)N * (double)Ns + (double)Ns * (double)(Ns + 1)) *
                                                     0x1p-53, s));
    // S = U^T U and U^{-1}: column-major U^{-1} read row-major is U^{-T} (lower),
    // which the recursive form writes directly.
    if (own_chol) {
      DG_TRY(cholesky_inverse(ctx, S, Ns, Ns, ctx->info_d, bad));
    } else {
      DG_SOLVER(cusolverDnDpotrf(ctx->solver, CUBLAS_FILL_MODE_UPPER, n, S, n, work, lwork, ctx->info_d));
    }
    DG_CUDA(cudaMemcpyAsync(info, ctx->info_d, sizeof(int), cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaStreamSynchronize(s));
    if (info[0] != 0)
      return set_error(DGCHEFSI_ERR_NOT_SPD,
                       "Cholesky of S = Y^T Y failed at column %d (S not positive definite; orthonormalisation pass %d)",
                       info[0], pass + 1);
    if (!own_chol)
      DG_SOLVER(cusolverDnXtrtri(ctx->solver, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, Ns, CUDA_R_64F, S, Ns,
                                 work, ctx->ws_solver.bytes,
                                 ctx->solver_host.empty() ? nullptr : ctx->solver_host.data(), lw_trtri_h,
                                 ctx->info_d + 1));
    // Y_hat^T = U^{-T} Y^T
    if (sl)
      DG_TRY(sliced_gemm(ctx, false, true, Ns, N, Ns, S, Ns, in, ldi, outp, ldo, ctx->products_slices, bad));
    else
      DG_CUDA(gemm_nn_f64(S, Ns, in, ldi, outp, ldo, Ns, N, Ns, true, s));
    if (pass > 0)
      DG_CUDA(cudaMemcpy2DAsync(W, sizeof(double) * N, Y, sizeof(double) * ld, sizeof(double) * N, Ns,
                                cudaMemcpyDeviceToDevice, s));
  }
  // Step 4: H Y_hat into Y (Y is free now), H_hat = Y_hat^T (H Y_hat). H_hat is
  // symmetric up to rounding and the eigensolver reads one triangle (row-major
  // lower = column-major upper), so only the tiles on and below the diagonal
  // are computed.
  // With sliced products H Y_hat also runs from BF16 slices, on the
  // tensor-core filter's block-sparse step kernel, when H fits that form.
  bool hx_sliced = false;
  if (sl) DG_TRY(tc_sliced_matvec(ctx, W, N, Y, ld, Ns, ctx->products_slices, bad, &hx_sliced));
  if (!hx_sliced) DG_CUDA(filter_step_f64(ctx->view(), W, N, nullptr, Y, ld, Ns, 1.0, 0.0, 0.0, s));
  if (sl)
    DG_TRY(sliced_gemm(ctx, true, false, Ns, Ns, N, W, N, Y, ld, S, Ns, ctx->products_slices, bad, Ns));
  else
    DG_CUDA(gemm_nt_f64(W, N, Y, ld, S, Ns, Ns, Ns, N, true, false, s));
  // The eigensolver reads the lower triangle (row-major), the one computed.
  DG_TRY(subspace_eigh(ctx, S, Ns, Ns, ritz));
  // Step 5: X_new^T = Q^T Y_hat^T (column-major Q read row-major is Q^T).
  if (sl)
    DG_TRY(sliced_gemm(ctx, false, false, Ns, N, Ns, S, Ns, W, N, Y, ld, ctx->products_slices, bad));
  else
    DG_CUDA(gemm_nn_f64(S, Ns, W, N, Y, ld, Ns, N, Ns, false, s));
  DG_CUDA(check_finite_f64(ritz, Ns, ctx->info_d + 3, s));
  DG_CUDA(cudaMemcpyAsync(info, ctx->info_d, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  if (info[1] != 0) return set_error(DGCHEFSI_ERR_NOT_SPD, "triangular inverse failed (info %d)", info[1]);
  if (info[2] != 0) return set_error(DGCHEFSI_ERR_NO_CONVERGENCE, "dense eigensolver failed (info %d)", info[2]);
  if (info[3] != 0)
    return set_error(DGCHEFSI_ERR_NONFINITE, sl ? "non-finite Ritz value or Rayleigh-Ritz operand" : "non-finite Ritz value");
  return DGCHEFSI_OK;
}

}  // namespace dg

using namespace dg;

extern "C" {

const char* dgchefsi_last_error(void) { return g_err.c_str(); }

int64_t dgchefsi_launch_count(void) { return dg::launch_count(); }

dgchefsi_status dgchefsi_create(int32_t M, const int32_t* nb, const int64_t* row_ptr, const int32_t* col,
                                const int64_t* blk_off, const double* values, int64_t n_values, void* stream,
                                dgchefsi_ctx** out) {
  clear_error();
  if (!out) return set_error(DGCHEFSI_ERR_ARG, "null output pointer");
  *out = nullptr;
  if (M < 1 || !nb || !row_ptr || !col || !blk_off || !values || n_values < 1)
    return set_error(DGCHEFSI_ERR_ARG, "need M >= 1 and non-null host arrays");
  dgchefsi_ctx* ctx = nullptr;
  try {
    ctx = new dgchefsi_ctx();
  } catch (const std::bad_alloc&) {
    return set_error(DGCHEFSI_ERR_OOM, "host allocation failed");
  }
  auto bail = [&](dgchefsi_status st) {
    dgchefsi_destroy(ctx);
    return st;
  };
  try {
    ctx->M = M;
    ctx->nb_h.assign(nb, nb + M);
    ctx->off_h.assign(M + 1, 0);
    for (int K = 0; K < M; ++K) {
      if (nb[K] < 1 || nb[K] > 256) return bail(set_error(DGCHEFSI_ERR_ARG, "nb[%d] = %d outside 1..256", K, nb[K]));
      ctx->off_h[K + 1] = ctx->off_h[K] + nb[K];
      ctx->max_nb = std::max(ctx->max_nb, nb[K]);
    }
    ctx->N = ctx->off_h[M];
    ctx->f64_tj = 64;
    for (int K = 0; K < M; ++K)
      if (nb[K] % 64 != 0) ctx->f64_tj = 32;
    if (row_ptr[0] != 0) return bail(set_error(DGCHEFSI_ERR_ARG, "row_ptr[0] != 0"));
    for (int K = 0; K < M; ++K)
      if (row_ptr[K + 1] < row_ptr[K]) return bail(set_error(DGCHEFSI_ERR_ARG, "row_ptr decreases at %d", K));
    const int64_t nnzb = row_ptr[M];
    ctx->nnzb = nnzb;
    ctx->n_values = n_values;
    ctx->row_ptr_h.assign(row_ptr, row_ptr + M + 1);
    ctx->col_h.assign(col, col + nnzb);
    ctx->blk_off_h.assign(blk_off, blk_off + nnzb);
    for (int K = 0; K < M; ++K) {
      bool diag = false;
      for (int64_t e = row_ptr[K]; e < row_ptr[K + 1]; ++e) {
        const int Kp = col[e];
        if (Kp < 0 || Kp >= M) return bail(set_error(DGCHEFSI_ERR_ARG, "col[%lld] = %d out of range", (long long)e, Kp));
        if (e > row_ptr[K] && col[e - 1] >= Kp)
          return bail(set_error(DGCHEFSI_ERR_ARG, "columns of row %d not strictly ascending", K));
        if (Kp == K) diag = true;
        const int64_t sz = (int64_t)nb[K] * nb[Kp];
        if (blk_off[e] < 0 || blk_off[e] + sz > n_values)
          return bail(set_error(DGCHEFSI_ERR_ARG, "block %lld lies outside values", (long long)e));
      }
      if (!diag) return bail(set_error(DGCHEFSI_ERR_ARG, "row %d has no diagonal block", K));
    }
    for (int64_t i = 0; i < n_values; ++i)
      if (!std::isfinite(values[i])) return bail(set_error(DGCHEFSI_ERR_ARG, "values[%lld] not finite", (long long)i));
    // symmetry: pattern and H_{K';K} == H_{K;K'}^T exactly
    for (int K = 0; K < M; ++K) {
      for (int64_t e = row_ptr[K]; e < row_ptr[K + 1]; ++e) {
        const int Kp = col[e];
        int64_t lo = row_ptr[Kp], hi = row_ptr[Kp + 1] - 1, f = -1;
        while (lo <= hi) {
          const int64_t mid = (lo + hi) / 2;
          if (col[mid] == K) { f = mid; break; }
          if (col[mid] < K) lo = mid + 1; else hi = mid - 1;
        }
        if (f < 0) return bail(set_error(DGCHEFSI_ERR_ARG, "pattern not symmetric: (%d,%d) without (%d,%d)", K, Kp, Kp, K));
        const double* A = values + blk_off[e];
        const double* B = values + blk_off[f];
        const int nK = nb[K], nKp = nb[Kp];
        for (int i = 0; i < nK; ++i)
          for (int j = 0; j < nKp; ++j)
            if (A[(int64_t)i * nKp + j] != B[(int64_t)j * nK + i])
              return bail(set_error(DGCHEFSI_ERR_ARG, "H not symmetric in block (%d,%d) at (%d,%d)", K, Kp, i, j));
      }
    }
    ctx->poff_h.assign(M + 1, 0);
    for (int K = 0; K < M; ++K) ctx->poff_h[K + 1] = ctx->poff_h[K] + (int64_t)nb[K] * nb[K];
  } catch (const std::bad_alloc&) {
    return bail(set_error(DGCHEFSI_ERR_OOM, "host allocation failed"));
  }
  if (cudaGetDevice(&ctx->device) != cudaSuccess) return bail(set_error(DGCHEFSI_ERR_CUDA, "no CUDA device"));
  ctx->stream = static_cast<cudaStream_t>(stream);
  auto dmalloc = [&](void** p, size_t bytes) -> dgchefsi_status {
    if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
      cudaGetLastError();
      return set_error(DGCHEFSI_ERR_OOM, "cudaMalloc of %zu bytes for H failed", bytes);
    }
    return DGCHEFSI_OK;
  };
  dgchefsi_status st;
  if ((st = dmalloc((void**)&ctx->nb_d, sizeof(int32_t) * M)) ||
      (st = dmalloc((void**)&ctx->off_d, sizeof(int64_t) * (M + 1))) ||
      (st = dmalloc((void**)&ctx->row_ptr_d, sizeof(int64_t) * (M + 1))) ||
      (st = dmalloc((void**)&ctx->col_d, sizeof(int32_t) * ctx->nnzb)) ||
      (st = dmalloc((void**)&ctx->blk_off_d, sizeof(int64_t) * ctx->nnzb)) ||
      (st = dmalloc((void**)&ctx->vals_d, sizeof(double) * n_values)) ||
      (st = dmalloc((void**)&ctx->poff_d, sizeof(int64_t) * (M + 1))) ||
      (st = dmalloc((void**)&ctx->blk_row_d, sizeof(int32_t) * std::max<int64_t>(ctx->nnzb, 1))) ||
      (st = dmalloc((void**)&ctx->info_d, sizeof(int) * 4)))
    return bail(st);
  auto h2d = [&](void* d, const void* h, size_t bytes) { return cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice); };
  std::vector<int32_t> blk_row(ctx->nnzb);
  for (int K = 0; K < M; ++K)
    for (int64_t e = row_ptr[K]; e < row_ptr[K + 1]; ++e) blk_row[e] = K;
  if (ctx->nnzb > 0 && h2d(ctx->blk_row_d, blk_row.data(), sizeof(int32_t) * ctx->nnzb))
    return bail(set_error(DGCHEFSI_ERR_CUDA, "copy of the block rows to the device failed"));
  if (h2d(ctx->nb_d, nb, sizeof(int32_t) * M) || h2d(ctx->off_d, ctx->off_h.data(), sizeof(int64_t) * (M + 1)) ||
      h2d(ctx->row_ptr_d, row_ptr, sizeof(int64_t) * (M + 1)) || h2d(ctx->col_d, col, sizeof(int32_t) * ctx->nnzb) ||
      h2d(ctx->blk_off_d, blk_off, sizeof(int64_t) * ctx->nnzb) ||
      h2d(ctx->vals_d, values, sizeof(double) * n_values) ||
      h2d(ctx->poff_d, ctx->poff_h.data(), sizeof(int64_t) * (M + 1)))
    return bail(set_error(DGCHEFSI_ERR_CUDA, "copy of H to the device failed"));
  if (cusolverDnCreate(&ctx->solver) != CUSOLVER_STATUS_SUCCESS)
    return bail(set_error(DGCHEFSI_ERR_CUDA, "cusolverDnCreate failed"));
  // the fixed array of dgchefsi_bounds_static becomes resident here, while the
  // caller can still allocate, not at that entry point's first call
  if ((st = bounds_static_setup(ctx->device))) return bail(st);
  *out = ctx;
  return DGCHEFSI_OK;
}

void dgchefsi_destroy(dgchefsi_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream || ctx->vals_d) cudaStreamSynchronize(ctx->stream);
  tc_destroy(ctx);
  sliced_destroy(ctx);
  if (ctx->solver) cusolverDnDestroy(ctx->solver);
  cudaFree(ctx->nb_d);
  cudaFree(ctx->off_d);
  cudaFree(ctx->row_ptr_d);
  cudaFree(ctx->col_d);
  cudaFree(ctx->blk_off_d);
  cudaFree(ctx->vals_d);
  cudaFree(ctx->poff_d);
  cudaFree(ctx->blk_row_d);
  cudaFree(ctx->info_d);
  free_buf(ctx->ws_filter);
  free_buf(ctx->ws_rr);
  free_buf(ctx->ws_small);
  free_buf(ctx->ws_solver);
  free_buf(ctx->ws_cycle);
  free_buf(ctx->ws_lanczos);
  free_buf(ctx->ws_adjoint);
  free_buf(ctx->ws_realign);
  free_buf(ctx->ws_sliced);
  free_buf(ctx->ws_sliced_t);
  free_buf(ctx->ws_sliced_b);
  free_buf(ctx->ws_pairs);
  free_buf(ctx->ws_pairs_err);
  free_buf(ctx->ws_eig);
  free_buf(ctx->ws_chol);
  if (ctx->s_reduce) cudaStreamSynchronize(ctx->s_reduce);
  for (int i = 0; i < 2; ++i) {
    if (ctx->ev_pairs[i]) cudaEventDestroy(ctx->ev_pairs[i]);
    if (ctx->ev_reduce[i]) cudaEventDestroy(ctx->ev_reduce[i]);
  }
  if (ctx->s_reduce) cudaStreamDestroy(ctx->s_reduce);
  for (cudaEvent_t e : ctx->ev_time) cudaEventDestroy(e);
  for (int i = 0; i < 2; ++i) {
    free_buf(ctx->ws_hin[i]);
    free_buf(ctx->ws_hout[i]);
    if (ctx->ev_in[i]) cudaEventDestroy(ctx->ev_in[i]);
    if (ctx->ev_f[i]) cudaEventDestroy(ctx->ev_f[i]);
    if (ctx->ev_out[i]) cudaEventDestroy(ctx->ev_out[i]);
  }
  if (ctx->h_in) cudaStreamDestroy(ctx->h_in);
  if (ctx->h_out) cudaStreamDestroy(ctx->h_out);
  if (ctx->f64_gexec) cudaGraphExecDestroy(ctx->f64_gexec);
  if (ctx->f64_cap) cudaStreamDestroy(ctx->f64_cap);
  cudaFree(ctx->f64_coef_d);
  cudaFreeHost(ctx->f64_coef_h);
  delete ctx;
}

dgchefsi_status dgchefsi_set_stream(dgchefsi_ctx* ctx, void* stream) {
  clear_error();
  DG_TRY(check_ctx(ctx));
  ctx->stream = static_cast<cudaStream_t>(stream);
  return DGCHEFSI_OK;
}

dgchefsi_status dgchefsi_dims(const dgchefsi_ctx* ctx, int64_t* N, int32_t* M) {
  clear_error();
  DG_TRY(check_ctx(ctx));
  if (N) *N = ctx->N;
  if (M) *M = ctx->M;
  return DGCHEFSI_OK;
}

dgchefsi_status dgchefsi_matvec(dgchefsi_ctx* ctx, const double* X, double* Y, int64_t Ns, int64_t ld) {
  clear_error();
  DG_TRY(check_ctx(ctx));
  DG_TRY(check_block(ctx, X, Ns, ld, "X"));
  DG_TRY(check_block(ctx, Y, Ns, ld, "Y"));
  if (Ns == 0) return DGCHEFSI_OK;
  if (overlaps(X, Y, sizeof(double) * (size_t)Ns * ld)) return set_error(DGCHEFSI_ERR_ARG, "X and Y overlap");
  DG_CUDA(filter_step_f64(ctx->view(), X, ld, nullptr, Y, ld, Ns, 1.0, 0.0, 0.0, ctx->stream));
  return DGCHEFSI_OK;
}

dgchefsi_status dgchefsi_bounds(dgchefsi_ctx* ctx, const double* v0, int k, double* b_upper, double* theta_min) {
  clear_error();
  DG_TRY(check_ctx(ctx));
  if (!v0 || !b_upper) return set_error(DGCHEFSI_ERR_ARG, "null v0 or b_upper");
  if (k < 1 || k > 64) return set_error(DGCHEFSI_ERR_ARG, "k = %d outside 1..64", k);
  return bounds_impl(ctx, v0, k, b_upper, theta_min);
}

static dgchefsi_status check_filter_args(dgchefsi_ctx* ctx, int prec, const double* X, double* Y, int64_t Ns,
                                         int64_t ld, int m, double a, double b, double a0) {
  DG_TRY(check_ctx(ctx));
  DG_TRY(check_block(ctx, X, Ns, ld, "X"));
  DG_TRY(check_block(ctx, Y, Ns, ld, "Y"));
  if (prec < DGCHEFSI_F64 || prec > DGCHEFSI_BF16X3) return set_error(DGCHEFSI_ERR_ARG, "unknown precision %d", prec);
  if (m < 1) return set_error(DGCHEFSI_ERR_ARG, "filter degree m = %d < 1", m);
  if (!(std::isfinite(a) && std::isfinite(b) && std::isfinite(a0)) || !(a0 < a && a < b))
    return set_error(DGCHEFSI_ERR_ARG, "need a0 < a < b (got a0=%g a=%g b=%g)", a0, a, b);
  if (Ns > 0 && overlaps(X, Y, sizeof(double) * (size_t)Ns * ld)) return set_error(DGCHEFSI_ERR_ARG, "X and Y overlap");
  return DGCHEFSI_OK;
}

dgchefsi_status dgchefsi_filter(dgchefsi_ctx* ctx, int prec, const double* X, double* Y, int64_t Ns, int64_t ld,
                                int m, double a, double b, double a0) {
  clear_error();
  DG_TRY(check_filter_args(ctx, prec, X, Y, Ns, ld, m, a, b, a0));
  if (Ns == 0) return DGCHEFSI_OK;
  if (prec == DGCHEFSI_F64) return filter_f64(ctx, X, Y, Ns, ld, m, a, b, a0);
  return filter_tc(ctx, prec, X, Y, Ns, ld, m, a, b, a0);
}

dgchefsi_status dgchefsi_filter_graph(dgchefsi_ctx* ctx, int prec, const double* X, double* Y, int64_t Ns,
                                      int64_t ld, int m, double a, double b, double a0) {
  clear_error();
  DG_TRY(check_filter_args(ctx, prec, X, Y, Ns, ld, m, a, b, a0));
  if (Ns == 0) return DGCHEFSI_OK;
  if (prec == DGCHEFSI_F64) return filter_f64_graph(ctx, X, Y, Ns, ld, m, a, b, a0);
  return filter_tc_graph(ctx, prec, X, Y, Ns, ld, m, a, b, a0);
}

// Host-buffer filter: chunks of states pipelined over three streams (upload
// of chunk k+1 and download of chunk k-1 overlap the filter of chunk k).
static dgchefsi_status filter_host_impl(dgchefsi_ctx* ctx, int prec, const double* X, double* Y, int64_t Ns,
                                        int64_t ld, int m, double a, double b, double a0,
                                        const std::vector<int64_t>& start) {
  // chunk k holds states start[k] .. start[k+1]-1
  int64_t chunk = 0;
  for (size_t k = 0; k + 1 < start.size(); ++k) chunk = std::max(chunk, start[k + 1] - start[k]);
  const int64_t N = ctx->N;
  cudaStream_t s = ctx->stream;
  if (!ctx->h_in) DG_CUDA(cudaStreamCreateWithFlags(&ctx->h_in, cudaStreamNonBlocking));
  if (!ctx->h_out) DG_CUDA(cudaStreamCreateWithFlags(&ctx->h_out, cudaStreamNonBlocking));
  for (int i = 0; i < 2; ++i) {
    if (!ctx->ev_in[i]) DG_CUDA(cudaEventCreateWithFlags(&ctx->ev_in[i], cudaEventDisableTiming));
    if (!ctx->ev_f[i]) DG_CUDA(cudaEventCreateWithFlags(&ctx->ev_f[i], cudaEventDisableTiming));
    if (!ctx->ev_out[i]) DG_CUDA(cudaEventCreateWithFlags(&ctx->ev_out[i], cudaEventDisableTiming));
  }
  // nothing of an earlier call may still use the chunk buffers or events
  DG_CUDA(cudaStreamSynchronize(ctx->h_in));
  DG_CUDA(cudaStreamSynchronize(ctx->h_out));
  const size_t cb = sizeof(double) * (size_t)chunk * (size_t)N;
  for (int i = 0; i < 2; ++i) {
    DG_TRY(ensure(ctx, ctx->ws_hin[i], cb, "host-filter input chunk"));
    DG_TRY(ensure(ctx, ctx->ws_hout[i], cb, "host-filter output chunk"));
  }
  const int64_t nch = (int64_t)start.size() - 1;
  auto rows = [&](int64_t k) { return start[k + 1] - start[k]; };
  auto upload = [&](int64_t k) -> dgchefsi_status {
    const int i = (int)(k & 1);
    if (k >= 2) DG_CUDA(cudaStreamWaitEvent(ctx->h_in, ctx->ev_f[i], 0));  // filter k-2 done with it
    DG_CUDA(cudaMemcpy2DAsync(ctx->ws_hin[i].p, sizeof(double) * N, X + start[k] * ld, sizeof(double) * ld,
                              sizeof(double) * N, rows(k), cudaMemcpyHostToDevice, ctx->h_in));
    DG_CUDA(cudaEventRecord(ctx->ev_in[i], ctx->h_in));
    return DGCHEFSI_OK;
  };
  dgchefsi_status st = upload(0);
  for (int64_t k = 0; k < nch && st == DGCHEFSI_OK; ++k) {
    const int i = (int)(k & 1);
    if (k + 1 < nch) st = upload(k + 1);
    if (st != DGCHEFSI_OK) break;
    cudaError_t e = cudaStreamWaitEvent(s, ctx->ev_in[i], 0);
    if (e == cudaSuccess && k >= 2) e = cudaStreamWaitEvent(s, ctx->ev_out[i], 0);  // download k-2 done
    if (e != cudaSuccess) {
      st = set_error(DGCHEFSI_ERR_CUDA, "stream wait failed: %s", cudaGetErrorString(e));
      break;
    }
    const double* xi = static_cast<const double*>(ctx->ws_hin[i].p);
    double* yo = static_cast<double*>(ctx->ws_hout[i].p);
    st = prec == DGCHEFSI_F64 ? filter_f64(ctx, xi, yo, rows(k), N, m, a, b, a0)
                              : filter_tc(ctx, prec, xi, yo, rows(k), N, m, a, b, a0, /*reuse_hop=*/k > 0);
    if (st != DGCHEFSI_OK) break;
    e = cudaEventRecord(ctx->ev_f[i], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->h_out, ctx->ev_f[i], 0);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(Y + start[k] * ld, sizeof(double) * ld, yo, sizeof(double) * N, sizeof(double) * N,
                            rows(k), cudaMemcpyDeviceToHost, ctx->h_out);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_out[i], ctx->h_out);
    if (e != cudaSuccess) st = set_error(DGCHEFSI_ERR_CUDA, "chunk download failed: %s", cudaGetErrorString(e));
  }
  // drain all three streams whatever happened, so no copy is left in flight
  cudaError_t e1 = cudaStreamSynchronize(ctx->h_in);
  cudaError_t e2 = cudaStreamSynchronize(s);
  cudaError_t e3 = cudaStreamSynchronize(ctx->h_out);
  if (st != DGCHEFSI_OK) return st;
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)
    return set_error(DGCHEFSI_ERR_CUDA, "host-filter pipeline failed: %s",
                     cudaGetErrorString(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3)));
  return DGCHEFSI_OK;
}

dgchefsi_status dgchefsi_filter_host(dgchefsi_ctx* ctx, int prec, const double* X, double* Y, int64_t Ns,
                                     int64_t ld, int m, double a, double b, double a0, int64_t chunk) {
  clear_error();
  DG_TRY(check_filter_args(ctx, prec, X, Y, Ns, ld, m, a, b, a0));
  if (chunk < 0) return set_error(DGCHEFSI_ERR_ARG, "chunk < 0");
  if (Ns == 0) return DGCHEFSI_OK;
  std::vector<int64_t> start{0};
  if (chunk > 0) {
    for (int64_t s0 = chunk; s0 < Ns; s0 += chunk) start.push_back(s0);
  } else if (Ns >= 2048) {
    // small first and last chunks (their copies are the only ones not
    // overlapped), three equal chunks of 256-state multiples between
    const int64_t edge = std::max<int64_t>(256, Ns / 16 / 256 * 256);
    const int64_t span = Ns - 2 * edge;
    start.push_back(edge);
    for (int q = 1; q < 3; ++q) {
      const int64_t b = edge + (q * span / 3 + 255) / 256 * 256;
      if (b > start.back() && b < Ns - edge) start.push_back(b);
    }
    start.push_back(Ns - edge);
  } else {
    const int64_t c = std::max<int64_t>(256, (Ns / 4 + 255) / 256 * 256);
    for (int64_t s0 = c; s0 < Ns; s0 += c) start.push_back(s0);
  }
  start.push_back(Ns);
  return filter_host_impl(ctx, prec, X, Y, Ns, ld, m, a, b, a0, start);
}

dgchefsi_status dgchefsi_set_orthonormalisation(dgchefsi_ctx* ctx, int mode) {
  clear_error();
  if (!ctx) return set_error(DGCHEFSI_ERR_ARG, "null context");
  if (mode != DGCHEFSI_ORTH_CHOLQR && mode != DGCHEFSI_ORTH_CHOLQR2 && mode != DGCHEFSI_ORTH_SHIFTED_CHOLQR3)
    return set_error(DGCHEFSI_ERR_ARG, "unknown orthonormalisation %d", mode);
  ctx->orth_mode = mode;
  return DGCHEFSI_OK;
}

dgchefsi_status dgchefsi_set_subspace_products(dgchefsi_ctx* ctx, int mode, int slices) {
  clear_error();
  if (!ctx) return set_error(DGCHEFSI_ERR_ARG, "null context");
  if (mode != DGCHEFSI_PRODUCTS_F64 && mode != DGCHEFSI_PRODUCTS_SLICED_BF16)
    return set_error(DGCHEFSI_ERR_ARG, "unknown product arithmetic %d", mode);
  if (mode == DGCHEFSI_PRODUCTS_SLICED_BF16 && (slices < 2 || slices > 16))
    return set_error(DGCHEFSI_ERR_ARG, "slices = %d outside 2..16", slices);
  ctx->products_mode = mode;
  if (mode == DGCHEFSI_PRODUCTS_SLICED_BF16) ctx->products_slices = slices;
  return DGCHEFSI_OK;
}

dgchefsi_status dgchefsi_sliced_gemm(dgchefsi_ctx* ctx, int b_rows, int a_lower, int64_t M, int64_t Nc, int64_t K,
                                     const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                                     int64_t ldc, int slices, int64_t tri) {
  clear_error();
  DG_TRY(check_ctx(ctx));
  if (M < 0 || Nc < 0 || K < 0 || tri < 0) return set_error(DGCHEFSI_ERR_ARG, "negative size");
  if (slices < 2 || slices > 16) return set_error(DGCHEFSI_ERR_ARG, "slices = %d outside 2..16", slices);
  if (M == 0 || Nc == 0) return DGCHEFSI_OK;
  if (!C || (K > 0 && (!A || !B))) return set_error(DGCHEFSI_ERR_ARG, "null matrix pointer");
  if (ldc < Nc || (K > 0 && (lda < K || ldb < (b_rows ? K : Nc))))
    return set_error(DGCHEFSI_ERR_ARG, "leading dimension smaller than the row length");
  if ((K + 4095) / 4096 > 65535 || M > 0x7fffffff || Nc > 0x7fffffff)
    return set_error(DGCHEFSI_ERR_UNSUPPORTED, "sizes beyond this build's grid limits");
  DG_CUDA(cudaMemsetAsync(ctx->info_d + 3, 0, sizeof(int), ctx->stream));
  DG_TRY(sliced_gemm(ctx, b_rows != 0, a_lower != 0, M, Nc, K, A, lda, B, ldb, C, ldc, slices, ctx->info_d + 3,
                     tri));
  int bad = 0;
  DG_CUDA(cudaMemcpyAsync(&bad, ctx->info_d + 3, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  DG_CUDA(cudaStreamSynchronize(ctx->stream));
  if (bad) return set_error(DGCHEFSI_ERR_NONFINITE, "non-finite entry in A or B");
  return DGCHEFSI_OK;
}

dgchefsi_status dgchefsi_sliced_matvec(dgchefsi_ctx* ctx, const double* X, double* Y, int64_t Ns, int64_t ld,
                                       int slices) {
  clear_error();
  DG_TRY(check_ctx(ctx));
  DG_TRY(check_block(ctx, X, Ns, ld, "X"));
  DG_TRY(check_block(ctx, Y, Ns, ld, "Y"));
  if (slices < 2 || slices > 16) return set_error(DGCHEFSI_ERR_ARG, "slices = %d outside 2..16", slices);
  if (Ns == 0) return DGCHEFSI_OK;
  if (overlaps(X, Y, sizeof(double) * (size_t)((Ns - 1) * ld + ctx->N)))
    return set_error(DGCHEFSI_ERR_ARG, "Y overlaps X");
  DG_CUDA(cudaMemsetAsync(ctx->info_d + 3, 0, sizeof(int), ctx->stream));
  bool used = false;
  DG_TRY(tc_sliced_matvec(ctx, X, ld, Y, ld, Ns, slices, ctx->info_d + 3, &used));
  if (!used)
    return set_error(DGCHEFSI_ERR_UNSUPPORTED,
                     "H does not fit the sliced product (a block row longer than 4096 columns or an element "
                     "larger than 128)");
  int bad = 0;
  DG_CUDA(cudaMemcpyAsync(&bad, ctx->info_d + 3, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  DG_CUDA(cudaStreamSynchronize(ctx->stream));
  if (bad) return set_error(DGCHEFSI_ERR_NONFINITE, "non-finite entry in H or X");
  return DGCHEFSI_OK;
}

dgchefsi_status dgchefsi_sliced_timing(dgchefsi_ctx* ctx, double* pairs_ms, int64_t* launches) {
  clear_error();
  DG_TRY(check_ctx(ctx));
  if (pairs_ms) *pairs_ms = ctx->pairs_ms;
  if (launches) *launches = ctx->pairs_launches;
  return DGCHEFSI_OK;
}

dgchefsi_status dgchefsi_set_refinement_start(dgchefsi_ctx* ctx, double coupling) {
  clear_error();
  if (!ctx) return set_error(DGCHEFSI_ERR_ARG, "null context");
  if (!(coupling > 0.0 && coupling <= 1.0)) return set_error(DGCHEFSI_ERR_ARG, "coupling threshold outside (0, 1]");
  ctx->eig_start_coupling = coupling;
  return DGCHEFSI_OK;
}

dgchefsi_status dgchefsi_eigensolver_history(const dgchefsi_ctx* ctx, double* corrections, int* slices, int cap,
                                             int* count) {
  clear_error();
  DG_TRY(check_ctx(ctx));
  const int k = std::min(ctx->eig_steps, 16);
  if (count) *count = k;
  for (int i = 0; corrections && i < std::min(k, cap); ++i) corrections[i] = ctx->eig_history[i];
  for (int i = 0; slices && i < std::min(k, cap); ++i) slices[i] = ctx->eig_slices_history[i];
  return DGCHEFSI_OK;
}

dgchefsi_status dgchefsi_set_cholesky(dgchefsi_ctx* ctx, int mode) {
  clear_error();
  if (!ctx) return set_error(DGCHEFSI_ERR_ARG, "null context");
  if (mode != DGCHEFSI_CHOL_AUTO && mode != DGCHEFSI_CHOL_CUSOLVER && mode != DGCHEFSI_CHOL_PRODUCTS)
    return set_error(DGCHEFSI_ERR_ARG, "unknown Cholesky form %d", mode);
  ctx->chol_mode = mode;
  return DGCHEFSI_OK;
}

dgchefsi_status dgchefsi_cholesky_inverse(dgchefsi_ctx* ctx, double* S, int64_t n, int64_t lda) {
  clear_error();
  DG_TRY(check_ctx(ctx));
  if (n < 0 || lda < n || (n > 0 && !S)) return set_error(DGCHEFSI_ERR_ARG, "bad Cholesky arguments");
  if (n == 0) return DGCHEFSI_OK;
  cudaStream_t s = ctx->stream;
  DG_CUDA(cudaMemsetAsync(ctx->info_d, 0, 4 * sizeof(int), s));
  if (use_own_cholesky(ctx)) {
    DG_TRY(cholesky_inverse(ctx, S, n, lda, ctx->info_d, ctx->info_d + 3));
  } else {
    if (n > INT32_MAX || lda > INT32_MAX) return set_error(DGCHEFSI_ERR_UNSUPPORTED, "order beyond cuSOLVER's int");
    DG_SOLVER(cusolverDnSetStream(ctx->solver, s));
    int lw = 0;
    size_t lw_d = 0, lw_h = 0;
    DG_SOLVER(cusolverDnDpotrf_bufferSize(ctx->solver, CUBLAS_FILL_MODE_UPPER, (int)n, S, (int)lda, &lw));
    DG_SOLVER(cusolverDnXtrtri_bufferSize(ctx->solver, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, n, CUDA_R_64F, S,
                                          lda, &lw_d, &lw_h));
    DG_TRY(ensure(ctx, ctx->ws_solver, std::max(sizeof(double) * (size_t)lw, lw_d), "cuSOLVER workspace"));
    if (ctx->solver_host.size() < lw_h) ctx->solver_host.resize(lw_h);
    DG_SOLVER(cusolverDnDpotrf(ctx->solver, CUBLAS_FILL_MODE_UPPER, (int)n, S, (int)lda,
                               static_cast<double*>(ctx->ws_solver.p), (int)(ctx->ws_solver.bytes / sizeof(double)),
                               ctx->info_d));
    int f = 0;
    DG_CUDA(cudaMemcpyAsync(&f, ctx->info_d, sizeof(int), cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaStreamSynchronize(s));
    if (f != 0) return set_error(DGCHEFSI_ERR_NOT_SPD, "Cholesky failed at column %d", f);
    DG_SOLVER(cusolverDnXtrtri(ctx->solver, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, n, CUDA_R_64F, S, lda,
                               ctx->ws_solver.p, ctx->ws_solver.bytes,
                               ctx->solver_host.empty() ? nullptr : ctx->solver_host.data(), lw_h, ctx->info_d + 1));
  }
  int info[4] = {0, 0, 0, 0};
  DG_CUDA(cudaMemcpyAsync(info, ctx->info_d, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  if (info[0] != 0) return set_error(DGCHEFSI_ERR_NOT_SPD, "Cholesky failed at column %d", info[0]);
  if (info[1] != 0) return set_error(DGCHEFSI_ERR_NOT_SPD, "triangular inverse failed (info %d)", info[1]);
  if (info[3] != 0) return set_error(DGCHEFSI_ERR_NONFINITE, "non-finite entry in S");
  return DGCHEFSI_OK;
}

dgchefsi_status dgchefsi_set_eigensolver(dgchefsi_ctx* ctx, int mode) {
  clear_error();
  if (!ctx) return set_error(DGCHEFSI_ERR_ARG, "null context");
  if (mode != DGCHEFSI_EIG_AUTO && mode != DGCHEFSI_EIG_SYEVD && mode != DGCHEFSI_EIG_REFINED)
    return set_error(DGCHEFSI_ERR_ARG, "unknown eigensolver %d", mode);
  ctx->eig_mode = mode;
  return DGCHEFSI_OK;
}

dgchefsi_status dgchefsi_subspace_eigh(dgchefsi_ctx* ctx, double* A, int64_t n, int64_t lda, double* w) {
  clear_error();
  DG_TRY(check_ctx(ctx));
  if (n < 0 || lda < n || (n > 0 && (!A || !w))) return set_error(DGCHEFSI_ERR_ARG, "bad eigensolve arguments");
  if (n > 0) {
    const char* a0 = reinterpret_cast<const char*>(A);
    const char* a1 = a0 + sizeof(double) * (size_t)((n - 1) * lda + n);
    const char* w0 = reinterpret_cast<const char*>(w);
    if (w0 < a1 && a0 < w0 + sizeof(double) * (size_t)n) return set_error(DGCHEFSI_ERR_ARG, "w overlaps A");
  }
  cudaStream_t s = ctx->stream;
  DG_CUDA(cudaMemsetAsync(ctx->info_d, 0, 4 * sizeof(int), s));
  DG_TRY(subspace_eigh(ctx, A, n, lda, w));
  if (n > 0) DG_CUDA(check_finite_f64(w, n, ctx->info_d + 3, s));
  int info[4] = {0, 0, 0, 0};
  DG_CUDA(cudaMemcpyAsync(info, ctx->info_d, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  if (info[2] != 0) return set_error(DGCHEFSI_ERR_NO_CONVERGENCE, "dense eigensolver failed (info %d)", info[2]);
  if (info[3] != 0) return set_error(DGCHEFSI_ERR_NONFINITE, "non-finite eigenvalue");
  return DGCHEFSI_OK;
}

dgchefsi_status dgchefsi_eigensolver_stats(const dgchefsi_ctx* ctx, int* used, int* steps, int* max_cluster,
                                           int* fallback, double* update, double* start_ms, double* refine_ms,
                                           int64_t* start_order, int* start_solver) {
  clear_error();
  DG_TRY(check_ctx(ctx));
  if (used) *used = ctx->eig_used;
  if (steps) *steps = ctx->eig_steps;
  if (max_cluster) *max_cluster = ctx->eig_max_cluster;
  if (fallback) *fallback = ctx->eig_fallback;
  if (update) *update = ctx->eig_update;
  if (start_ms) *start_ms = ctx->eig_start_ms;
  if (refine_ms) *refine_ms = ctx->eig_refine_ms;
  if (start_order) *start_order = ctx->eig_start_order;
  if (start_solver) *start_solver = ctx->eig_start_solver;
  return DGCHEFSI_OK;
}

dgchefsi_status dgchefsi_set_tile_shape(dgchefsi_ctx* ctx, int prec, int G, int T, int layout) {
  clear_error();
  DG_TRY(check_ctx(ctx));
  if (prec < DGCHEFSI_TF32 || prec > DGCHEFSI_BF16X3) return set_error(DGCHEFSI_ERR_ARG, "not a tensor-core precision");
  if (G < 0 || T < 0 || (G == 0) != (T == 0)) return set_error(DGCHEFSI_ERR_ARG, "need G, T both > 0 or both 0");
  if (layout < 0 || layout > 2) return set_error(DGCHEFSI_ERR_ARG, "layout must be 0, 1 or 2");
  return tc_set_shape(ctx, prec, G, T, layout);
}

dgchefsi_status dgchefsi_get_tile_shape(dgchefsi_ctx* ctx, int prec, int* G, int* T, int* ACC, int* layout) {
  clear_error();
  DG_TRY(check_ctx(ctx));
  if (!G || !T || !ACC || !layout) return set_error(DGCHEFSI_ERR_ARG, "null output");
  if (prec < DGCHEFSI_TF32 || prec > DGCHEFSI_BF16X3) return set_error(DGCHEFSI_ERR_ARG, "not a tensor-core precision");
  return tc_get_shape(ctx, prec, G, T, ACC, layout);
}

dgchefsi_status dgchefsi_set_unit_order(dgchefsi_ctx* ctx, int prec, int tgb) {
  clear_error();
  DG_TRY(check_ctx(ctx));
  if (prec < DGCHEFSI_TF32 || prec > DGCHEFSI_BF16X3) return set_error(DGCHEFSI_ERR_ARG, "not a tensor-core precision");
  if (tgb < -1 || tgb > 65535) return set_error(DGCHEFSI_ERR_ARG, "unit order %d outside -1..65535", tgb);
  return tc_set_unit_order(ctx, prec, tgb);
}

dgchefsi_status dgchefsi_get_unit_order(dgchefsi_ctx* ctx, int prec, int* tgb) {
  clear_error();
  DG_TRY(check_ctx(ctx));
  if (prec < DGCHEFSI_TF32 || prec > DGCHEFSI_BF16X3) return set_error(DGCHEFSI_ERR_ARG, "not a tensor-core precision");
  if (!tgb) return set_error(DGCHEFSI_ERR_ARG, "null output");
  return tc_get_unit_order(ctx, prec, tgb);
}

dgchefsi_status dgchefsi_selftest_wait(dgchefsi_ctx* ctx, int64_t limit_ns) {
  clear_error();
  DG_TRY(check_ctx(ctx));
  if (limit_ns < 1 || limit_ns > 10000000000LL) return set_error(DGCHEFSI_ERR_ARG, "limit_ns outside 1 ns .. 10 s");
  return tc_wait_selftest(ctx, limit_ns);
}

dgchefsi_status dgchefsi_selftest_fp64_rate(dgchefsi_ctx* ctx, int reps, double* flops_per_s) {
  clear_error();
  DG_TRY(check_ctx(ctx));
  if (reps < 1 || reps > 100 || !flops_per_s) return set_error(DGCHEFSI_ERR_ARG, "need 1 <= reps <= 100 and an output");
  int nsm = 0;
  DG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
  const int blocks = 8 * nsm;
  const int64_t iters = 1 << 15;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  DG_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return set_error(DGCHEFSI_ERR_CUDA, "cudaEventCreate failed");
  }
  double* sink = reinterpret_cast<double*>(ctx->info_d);
  float best = 0.f;
  cudaError_t err = dfma_rate(iters / 8, blocks, sink, ctx->stream);  // warm-up
  for (int r = 0; r < reps && err == cudaSuccess; ++r) {
    cudaEventRecord(e0, ctx->stream);
    err = dfma_rate(iters, blocks, sink, ctx->stream);
    cudaEventRecord(e1, ctx->stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && (best == 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return set_error(DGCHEFSI_ERR_CUDA, "FP64 rate probe failed: %s", cudaGetErrorString(err));
  *flops_per_s = 16.0 * (double)iters * (double)blocks * 256.0 / (1e-3 * (double)best);
  return DGCHEFSI_OK;
}

dgchefsi_status dgchefsi_gram(dgchefsi_ctx* ctx, const double* Y, int64_t Ns, int64_t ld, double* S) {
  clear_error();
  DG_TRY(check_ctx(ctx));
  DG_TRY(check_block(ctx, Y, Ns, ld, "Y"));
  if (Ns > 0 && !S) return set_error(DGCHEFSI_ERR_ARG, "null S");
  DG_CUDA(gemm_nt_f64(Y, ld, Y, ld, S, Ns, Ns, Ns, ctx->N, true, false, ctx->stream));
  return DGCHEFSI_OK;
}

dgchefsi_status dgchefsi_rayleigh_ritz(dgchefsi_ctx* ctx, double* Y, int64_t Ns, int64_t ld, double* ritz) {
  clear_error();
  DG_TRY(check_ctx(ctx));
  DG_TRY(check_block(ctx, Y, Ns, ld, "Y"));
  if (Ns > 0 && !ritz) return set_error(DGCHEFSI_ERR_ARG, "null ritz");
  if (Ns > ctx->N) return set_error(DGCHEFSI_ERR_ARG, "Ns (%lld) > N (%lld)", (long long)Ns, (long long)ctx->N);
  if (Ns > 2147483647LL) return set_error(DGCHEFSI_ERR_UNSUPPORTED, "Ns too large for the dense eigensolver");
  if (Ns == 0) return DGCHEFSI_OK;
  return rr_impl(ctx, Y, Ns, ld, ritz);
}

dgchefsi_status dgchefsi_occupations(dgchefsi_ctx* ctx, const double* ritz, int64_t Ns, double Ne, double kT,
                                     double* f, double* mu) {
  clear_error();
  DG_TRY(check_ctx(ctx));
  if (Ns < 1 || !ritz || !f || !mu) return set_error(DGCHEFSI_ERR_ARG, "need Ns >= 1 and non-null ritz, f, mu");
  if (!(kT > 0.0) || !std::isfinite(kT)) return set_error(DGCHEFSI_ERR_ARG, "kT must be > 0");
  if (!(Ne >= 0.0) || Ne > 2.0 * (double)Ns)
    return set_error(DGCHEFSI_ERR_ARG, "need 0 <= Ne <= 2 Ns (Ne = %g, Ns = %lld)", Ne, (long long)Ns);
  DG_CUDA(occupations_f64(ritz, Ns, Ne, kT, f, mu, ctx->stream));
  return DGCHEFSI_OK;
}

dgchefsi_status dgchefsi_density_blocks(dgchefsi_ctx* ctx, const double* X, int64_t Ns, int64_t ld, const double* f,
                                        double* P) {
  clear_error();
  DG_TRY(check_ctx(ctx));
  DG_TRY(check_block(ctx, X, Ns, ld, "X"));
  if (!P || (Ns > 0 && !f)) return set_error(DGCHEFSI_ERR_ARG, "null f or P");
  DG_CUDA(density_f64(ctx->view(), ctx->poff_d, X, Ns, ld, f, P, ctx->stream));
  return DGCHEFSI_OK;
}

dgchefsi_status dgchefsi_cycle(dgchefsi_ctx* ctx, int prec, double* X, int64_t Ns, int64_t ld, int m, double Ne,
                               double kT, const double* v0, int k_lanczos, const double* prev_ritz, double* bounds,
                               int use_bounds, double* ritz, double* f, double* mu, double* P) {
  clear_error();
  DG_TRY(check_ctx(ctx));
  DG_TRY(check_block(ctx, X, Ns, ld, "X"));
  if (Ns < 1 || !ritz || !f || !mu || !P) return set_error(DGCHEFSI_ERR_ARG, "need Ns >= 1 and non-null outputs");
  if (Ns > ctx->N) return set_error(DGCHEFSI_ERR_ARG, "Ns > N");
  if (!(kT > 0.0) || !(Ne >= 0.0) || Ne > 2.0 * (double)Ns)
    return set_error(DGCHEFSI_ERR_ARG, "need kT > 0 and 0 <= Ne <= 2 Ns");
  double a, b, a0;
  if (use_bounds) {
    if (!bounds) return set_error(DGCHEFSI_ERR_ARG, "use_bounds without bounds");
    a = bounds[0];
    b = bounds[1];
    a0 = bounds[2];
  } else {
    if (!v0) return set_error(DGCHEFSI_ERR_ARG, "null Lanczos start vector");
    if (k_lanczos < 1 || k_lanczos > 64) return set_error(DGCHEFSI_ERR_ARG, "k_lanczos outside 1..64");
    double tmin = 0.0;
    DG_TRY(bounds_impl(ctx, v0, k_lanczos, &b, &tmin));
    if (prev_ritz) {
      a = -std::numeric_limits<double>::infinity();
      a0 = std::numeric_limits<double>::infinity();
      for (int64_t i = 0; i < Ns; ++i) {
        a = std::fmax(a, prev_ritz[i]);
        a0 = std::fmin(a0, prev_ritz[i]);
      }
    } else {
      a0 = tmin;
      a = a0 + (b - a0) * (double)Ns / (double)ctx->N;
    }
  }
  DG_TRY(check_filter_args(ctx, prec, X, X + 0, 0, ld, m, a, b, a0));
  DG_TRY(ensure(ctx, ctx->ws_cycle, sizeof(double) * (size_t)Ns * (size_t)ld, "filtered block"));
  double* Yw = static_cast<double*>(ctx->ws_cycle.p);
  if (prec == DGCHEFSI_F64)
    DG_TRY(filter_f64(ctx, X, Yw, Ns, ld, m, a, b, a0));
  else
    DG_TRY(filter_tc(ctx, prec, X, Yw, Ns, ld, m, a, b, a0));
  DG_TRY(rr_impl(ctx, Yw, Ns, ld, ritz));
  DG_CUDA(cudaMemcpy2DAsync(X, sizeof(double) * ld, Yw, sizeof(double) * ld, sizeof(double) * ctx->N, Ns,
                            cudaMemcpyDeviceToDevice, ctx->stream));
  DG_CUDA(occupations_f64(ritz, Ns, Ne, kT, f, mu, ctx->stream));
  DG_CUDA(density_f64(ctx->view(), ctx->poff_d, X, Ns, ld, f, P, ctx->stream));
  if (bounds) {
    bounds[0] = a;
    bounds[1] = b;
    bounds[2] = a0;
  }
  DG_CUDA(cudaStreamSynchronize(ctx->stream));
  return DGCHEFSI_OK;
}

}  // extern "C"
