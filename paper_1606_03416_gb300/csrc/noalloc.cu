// Allocation-free Lanczos bound (dgchefsi_bounds_static).
//
// Some callers cannot allocate device memory while they run: their GPU memory
// is already reserved by another framework's caching allocator, or they sit in
// a loop that cannot absorb the device-wide synchronisation of cudaMalloc /
// cudaFree. For them the Krylov basis of the bound lives in one fixed
// file-scope device array instead of the context's grow-only workspace. The
// arithmetic and launch sequence are those of dgchefsi_bounds.
#include <cmath>
#include <mutex>

#include "ctx.h"
#include "internal.h"

namespace dg {
namespace {

constexpr int64_t kStaticDoubles = DGCHEFSI_BOUNDS_STATIC_DOUBLES;
constexpr int kMaxDevices = 64;
constexpr int kMaxSteps = 64;

// The scratch itself. In host code this name is only a handle for
// cudaGetSymbolAddress: its device address is looked up once per device.
static __device__ __align__(256) double g_bounds_scratch[kStaticDoubles];

std::mutex g_addr_mu;
double* g_addr[kMaxDevices] = {};

// Looks up the device address of g_bounds_scratch on `dev` (made current for
// the lookup) and caches it. The lookup loads this file's module if it is not
// loaded yet, which is when the array itself is allocated on the device.
dgchefsi_status lookup_scratch(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return set_error(DGCHEFSI_ERR_UNSUPPORTED, "device index %d too large", dev);
  int cur = 0;
  DG_CUDA(cudaGetDevice(&cur));
  if (cur != dev) DG_CUDA(cudaSetDevice(dev));
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_bounds_scratch);
  if (cur != dev) cudaSetDevice(cur);
  if (e != cudaSuccess)
    return set_error(DGCHEFSI_ERR_CUDA, "cudaGetSymbolAddress of the bound scratch failed: %s", cudaGetErrorString(e));
  g_addr[dev] = static_cast<double*>(p);
  return DGCHEFSI_OK;
}

// Cached device address of g_bounds_scratch on `dev`.
dgchefsi_status scratch_address(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return set_error(DGCHEFSI_ERR_UNSUPPORTED, "device index %d too large", dev);
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[dev]) DG_TRY(lookup_scratch(dev));
  *out = g_addr[dev];
  return DGCHEFSI_OK;
}

int sturm_count_n(const double* a, const double* b, int n, double x) {
  int cnt = 0;
  double q = a[0] - x;
  if (q < 0) ++cnt;
  for (int i = 1; i < n; ++i) {
    if (q == 0.0) q = 1e-300;
    q = (a[i] - x) - b[i - 1] * b[i - 1] / q;
    if (q < 0) ++cnt;
  }
  return cnt;
}

// `which`-th smallest eigenvalue (1-based) of the n x n symmetric tridiagonal
// matrix with diagonal a and off-diagonal b, by Sturm bisection.
double tridiag_eig_n(const double* a, const double* b, int n, int which) {
  double lo = a[0], hi = a[0];
  for (int i = 0; i < n; ++i) {
    double r = 0.0;
    if (i > 0) r += std::fabs(b[i - 1]);
    if (i + 1 < n) r += std::fabs(b[i]);
    lo = std::fmin(lo, a[i] - r);
    hi = std::fmax(hi, a[i] + r);
  }
  const double span = std::fmax(std::fabs(lo), std::fabs(hi));
  lo -= 1e-12 * span + 1e-300;
  hi += 1e-12 * span + 1e-300;
  for (int it = 0; it < 400; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count_n(a, b, n, mid) >= which) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

}  // namespace

// Run by dgchefsi_create with `device` current. Every new context refreshes
// the cached address, so a context created after a cudaDeviceReset (which
// unloads modules and frees the array) gets the reloaded array's address.
dgchefsi_status bounds_static_setup(int device) {
  {
    std::lock_guard<std::mutex> lock(g_addr_mu);
    DG_TRY(lookup_scratch(device));
  }
  DG_CUDA(preload_lanczos_kernels());
  return DGCHEFSI_OK;
}

}  // namespace dg

using namespace dg;

extern "C" dgchefsi_status dgchefsi_bounds_static(dgchefsi_ctx* ctx, const double* v0, int k, double* b_upper,
                                                  double* theta_min) {
  clear_error();
  if (!ctx) return set_error(DGCHEFSI_ERR_ARG, "null context");
  if (!v0 || !b_upper) return set_error(DGCHEFSI_ERR_ARG, "null v0 or b_upper");
  if (k < 1 || k > kMaxSteps) return set_error(DGCHEFSI_ERR_ARG, "k = %d outside 1..%d", k, kMaxSteps);
  const int64_t N = ctx->N;
  if (k > N) k = (int)N;
  const int64_t need = ((int64_t)k + 2) * N + 72;
  if (need > kStaticDoubles)
    return set_error(DGCHEFSI_ERR_ARG,
                     "dgchefsi_bounds_static needs (k+2)*N+72 = %lld doubles of fixed scratch but the library holds "
                     "%lld; use dgchefsi_bounds or fewer steps",
                     (long long)need, (long long)kStaticDoubles);
  double* V = nullptr;
  DG_TRY(scratch_address(ctx->device, &V));
  double* w = V + ((size_t)k + 1) * (size_t)N;
  double* sc = w + N;  // 72 device scalars
  cudaStream_t s = ctx->stream;
  double host[2];
  DG_CUDA(dots_f64(v0, 0, 1, v0, N, sc, s));
  DG_CUDA(cudaMemcpyAsync(host, sc, sizeof(double), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  const double nrm = std::sqrt(host[0]);
  if (!(nrm > 0.0) || !std::isfinite(nrm)) return set_error(DGCHEFSI_ERR_ARG, "Lanczos start vector is zero or not finite");
  DG_CUDA(axpby_f64(1.0 / nrm, v0, 0.0, v0, V, N, s));
  double al[kMaxSteps], be[kMaxSteps];
  int n = 0;
  double beta_prev = 0.0, beta_last = 0.0;
  const HView h = ctx->view();
  for (int j = 0; j < k; ++j) {
    double* vj = V + (size_t)j * N;
    DG_CUDA(spmv_f64(h, vj, w, s));
    if (j > 0) DG_CUDA(axpby_f64(-beta_prev, vj - N, 1.0, w, w, N, s));
    DG_CUDA(dots_f64(vj, 0, 1, w, N, sc, s));
    DG_CUDA(cudaMemcpyAsync(host, sc, sizeof(double), cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaStreamSynchronize(s));
    const double alpha = host[0];
    DG_CUDA(axpby_f64(-alpha, vj, 1.0, w, w, N, s));
    DG_CUDA(dots_f64(V, N, j + 1, w, N, sc, s));
    DG_CUDA(sub_combination_f64(w, V, N, sc, j + 1, N, s));
    DG_CUDA(dots_f64(w, 0, 1, w, N, sc + 64, s));
    DG_CUDA(cudaMemcpyAsync(host, sc + 64, sizeof(double), cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaStreamSynchronize(s));
    const double beta = std::sqrt(host[0]);
    al[n++] = alpha;
    beta_last = beta;
    if (!std::isfinite(alpha) || !std::isfinite(beta))
      return set_error(DGCHEFSI_ERR_NONFINITE, "Lanczos produced a non-finite coefficient");
    if (j == k - 1 || beta == 0.0) break;
    be[n - 1] = beta;
    DG_CUDA(axpby_f64(1.0 / beta, w, 0.0, w, vj + N, N, s));
    beta_prev = beta;
  }
  *b_upper = tridiag_eig_n(al, be, n, n) + std::fabs(beta_last);
  if (theta_min) *theta_min = tridiag_eig_n(al, be, n, 1);
  return DGCHEFSI_OK;
}
