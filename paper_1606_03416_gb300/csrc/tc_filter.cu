// Host side of the tensor-core Chebyshev filter: operand layouts, element
// groups and slice schedules per unit shape, an autotuner over unit shapes,
// and a CUDA-graph form of the whole filter. The step kernel itself is in
// tc_kernel.cuh (instantiated in tc_tf32.cu, tc_bf16.cu, tc_bf16x3.cu).
#include <algorithm>
#include <cmath>
#include <map>

#include "tc_kernel.cuh"

namespace dg {
namespace {

// X (FP64, natural layout, ld) -> FP32 master + BF16 hi / lo copies in the
// padded layout. Block (x, K) strides over the flattened (state, column)
// pairs of element K, so every thread has work whatever n_K is.
__global__ void k_pack(const double* __restrict__ X, int64_t ld, int64_t Ns, const int64_t* __restrict__ off,
                       const int32_t* __restrict__ nb, const int32_t* __restrict__ poff, int64_t ldp,
                       float* __restrict__ F, __nv_bfloat16* __restrict__ Hh, __nv_bfloat16* __restrict__ Hl) {
  const int K = blockIdx.y;
  const int n = nb[K];
  const int64_t o = off[K];
  const int po = poff[K];
  const int64_t total = Ns * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = t / n;
    const int j = (int)(t - s * n);
    const float v = (float)X[s * ld + o + j];
    const int64_t q = s * ldp + po + j;
    F[q] = v;
    if (Hh) {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      Hh[q] = h;
      if (Hl) Hl[q] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
  }
}

// FP32 padded layout -> FP64 natural layout (same flattened mapping).
__global__ void k_unpack(const float* __restrict__ F, int64_t ldp, int64_t Ns, const int64_t* __restrict__ off,
                         const int32_t* __restrict__ nb, const int32_t* __restrict__ poff, double* __restrict__ Y,
                         int64_t ld) {
  const int K = blockIdx.y;
  const int n = nb[K];
  const int64_t o = off[K];
  const int po = poff[K];
  const int64_t total = Ns * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = t / n;
    const int j = (int)(t - s * n);
    Y[s * ld + o + j] = (double)F[s * ldp + po + j];
  }
}

// Grid of k_pack / k_unpack: blocks of 256 threads per element, about four
// (state, column) pairs per thread.
static dim3 pack_grid(int64_t Ns, int max_nb, int M) {
  const int64_t per = (Ns * (int64_t)max_nb + 1023) / 1024;
  return dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(per, 65535)), (unsigned)M);
}

// Operand copy of (H - cI): for block e = (K, K') and slice sl of K', rows
// brow[e] + sl * pnb[K] + n (n < pnb[K]), W columns each; zero outside the block.
__global__ void k_build_hop(const int32_t* __restrict__ blk_row, const int32_t* __restrict__ col,
                            const int64_t* __restrict__ blk_off, const double* __restrict__ vals,
                            const int32_t* __restrict__ nb, const int32_t* __restrict__ pnb,
                            const int64_t* __restrict__ brow, int W, const double* __restrict__ coef, int mode,
                            int64_t lo_rows,
                            float* __restrict__ H32, __nv_bfloat16* __restrict__ H16) {
  const int64_t e = blockIdx.x;
  const double c = coef[0];
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
    double v = 0.0;
    if (n < nK && jp < nKp) {
      v = blk[(int64_t)n * nKp + jp];
      if (K == Kp && n == jp) v -= c;
    }
    const int64_t q = (brow[e] + rr) * W + w;
    if (mode == MODE_TF32) {
      H32[q] = (float)v;
    } else {
      const float f = (float)v;
      const __nv_bfloat16 h = __float2bfloat16_rn(f);
      H16[q] = h;
      if (mode == MODE_BF16X3) H16[q + lo_rows * W] = __float2bfloat16_rn(f - __bfloat162float(h));
    }
  }
}

// BF16 operand copies (hi, and lo = bf16(v - hi)) of an FP32 iterate in the padded layout.
__global__ void k_shadow(const float* __restrict__ F, int64_t n, __nv_bfloat16* __restrict__ Hh,
                         __nv_bfloat16* __restrict__ Hl) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = F[i];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    Hh[i] = h;
    if (Hl) Hl[i] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// G_e += alpha * sum_s W[s, poff_K + j] Y[s, poff_K' + j'] for every stored block
// e = (K, K'); W, Y FP32 in the padded layout (ld ldp), FP32 accumulation per
// 64 x 64 tile, FP64 update of G (values layout of H).
__global__ void __launch_bounds__(256) k_block_outer_f32(const int32_t* __restrict__ blk_row,
                                                         const int32_t* __restrict__ col, const int64_t* __restrict__ blk_off,
                                                         const int32_t* __restrict__ nb, const int32_t* __restrict__ poff,
                                                         const float* __restrict__ W, const float* __restrict__ Y,
                                                         int64_t ldp, int64_t Ns, double alpha, double* __restrict__ G) {
  constexpr int TT = 64, KB = 16, TPAD = TT + 4;
  const int64_t e = blockIdx.x;
  const int K = blk_row[e], Kp = col[e];
  const int nK = nb[K], nKp = nb[Kp];
  const int j0 = blockIdx.y * TT, jp0 = blockIdx.z * TT;
  if (j0 >= nK || jp0 >= nKp) return;
  const int64_t oK = poff[K], oKp = poff[Kp];
  __shared__ float As[KB][TPAD];
  __shared__ float Bs[KB][TPAD];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  const int cc = tid & 63;
  for (int64_t i0 = 0; i0 < Ns; i0 += KB) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int kk = (tid >> 6) + 4 * i;
      const int64_t st = i0 + kk;
      float v = 0.f, u = 0.f;
      if (st < Ns) {
        if (j0 + cc < nK) v = W[st * ldp + oK + j0 + cc];
        if (jp0 + cc < nKp) u = Y[st * ldp + oKp + jp0 + cc];
      }
      As[kk][cc] = v;
      Bs[kk][cc] = u;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KB; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  double* Ge = G + blk_off[e];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int jj = j0 + ty + 16 * i;
    if (jj >= nK) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int jq = jp0 + tx + 16 * j;
      if (jq < nKp) Ge[(int64_t)jj * nKp + jq] += alpha * (double)acc[i][j];
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }
  return fn;
}

// Self-test of the bounded wait: one thread waits on an mbarrier whose phase
// nothing completes; the wait must give up after limit_ns and report it.
__global__ void k_wait_selftest(uint64_t limit_ns, int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const bool completed = mbar_wait_for(smem_u32(&bar), 0u, limit_ns);
    *status = completed ? 0 : 1;
  }
}

}  // namespace

dgchefsi_status tc_wait_selftest(dgchefsi_ctx* ctx, int64_t limit_ns) {
  int* d = nullptr;
  if (ctx->ws_small.bytes < sizeof(int)) DG_TRY(ensure(ctx, ctx->ws_small, sizeof(int) * 4, "self-test status"));
  d = static_cast<int*>(ctx->ws_small.p);
  DG_CUDA(cudaMemsetAsync(d, 0xff, sizeof(int), ctx->stream));
  k_wait_selftest<<<1, 32, 0, ctx->stream>>>((uint64_t)limit_ns, d);
  count_launch();
  DG_CUDA(cudaGetLastError());
  int st = -1;
  DG_CUDA(cudaMemcpyAsync(&st, d, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  DG_CUDA(cudaStreamSynchronize(ctx->stream));
  if (st == 1) return set_error(DGCHEFSI_ERR_TIMEOUT, "bounded device wait gave up after %lld ns (self-test)",
                                (long long)limit_ns);
  return DGCHEFSI_OK;
}

// Element groups of G consecutive elements and, per group, the slices of the
// union of its members' neighbour lists: [A x coordinate, B row per member].
struct Plan {
  int G = 0, W = 0, ngroups = 0, maxent = 0;
  int32_t* grp_elem_d = nullptr;
  int32_t* sched_d = nullptr;
  int32_t* sched_ptr_d = nullptr;
  uint8_t* nsub_d = nullptr;    // 64-byte ring slots per slice entry (1 or 2)
  int32_t* gslots_d = nullptr;  // 64-byte ring slots per element group
};

struct TcState {
  int64_t Ns = -1, ldp = 0;
  int mode = -1;  // precision the operand copy of H is laid out for
  int boxn = 16, ACC = 64, num_sms = 0;
  std::vector<int32_t> pnb_h, poff_h, blk_row_h;
  std::vector<int64_t> brow_h;
  int64_t b_rows = 0, zero_row = 0;
  int32_t *pnb_d = nullptr, *poff_d = nullptr, *blk_row_d = nullptr;
  int64_t* brow_d = nullptr;
  DevBuf F[2], Sh[2], Sl[2], Hop;
  int* err_d = nullptr;
  double* coef_d = nullptr;  // [1 + 2m] c, alpha_k, beta_k
  double* coef_h = nullptr;  // pinned mirror
  int coef_cap = 0;
  std::map<int, Plan> plans;  // keyed by G
  int shapeG[3] = {0, 0, 0}, shapeT[3] = {0, 0, 0}, shapeL[3] = {0, 0, 0};  // chosen per precision
  int forceG[3] = {0, 0, 0}, forceT[3] = {0, 0, 0}, forceL[3] = {0, 0, 0};  // dgchefsi_set_tile_shape
  int tgb[3] = {-1, -1, -1};  // unit order (Params::tgb) chosen per precision; -1 = not tuned yet
  int force_tgb[3] = {-1, -1, -1};  // dgchefsi_set_unit_order (-1 = tune)
  float tuned_ms[3][NSHAPES] = {};
  // graph form
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int g_mode = -1, g_m = 0, g_G = 0, g_T = 0, g_L = 0;
  // bumped whenever a buffer or plan a captured graph may refer to is
  // (re)allocated or freed; a graph is replayed only under the same generation
  uint64_t gen = 1, g_gen = 0;
  const void* g_X = nullptr;
  void* g_Y = nullptr;
  int64_t g_Ns = 0, g_ld = 0;
  // band-energy gradient: FP32 checkpoints, segment and backward iterates
  DevBuf gbuf;
  double* coefb_d = nullptr;  // [1 + 2m] c, then alpha_k, beta_{k+1} of each backward step
  int coefb_cap = 0;
  int g_stride = 0, g_nseg = 0, g_mG = 0, g_mT = 0, g_mL = 0, g_mm = 0;
  std::vector<float*> cp0, cp1, segb;
  // H X from BF16 slices (tc_sliced_matvec): H's digits in the W = 64 operand
  // layout (s copies), the states' digits (s copies, element-padded), the
  // FP32 slice-pair slabs of one state panel, the exponents and the padded
  // column map
  struct {
    bool layout = false, h_built = false;
    int h_slices = 0;
    std::vector<int64_t> brow_h;
    int64_t b_rows = 0, zero_row = 0, max_row_len = 0;
    int64_t* brow_d = nullptr;
    int32_t* cmap_d = nullptr;
    int32_t* eh_d = nullptr;   // [ldp] H row exponents
    double* coef_d = nullptr;  // {c = 0, alpha = 1, beta = 0}
    Plan plan;
    DevBuf Hs, Xs, Pw, ex;
  } sx;
  float* R[3] = {nullptr, nullptr, nullptr};
  float* WF[2] = {nullptr, nullptr};
  __nv_bfloat16* WSh[2] = {nullptr, nullptr};
  __nv_bfloat16* WSl[2] = {nullptr, nullptr};
};

static FilterKernel pick_kernel(int mode, int G, int T, int ACC, int layout) {
  if (mode == MODE_TF32) return pick_kernel_tf32(G, T, ACC, layout);
  if (mode == MODE_BF16) return pick_kernel_bf16(G, T, ACC, layout);
  return pick_kernel_bf16x3(G, T, ACC, layout);
}

static void free_plan(Plan& pl) {
  cudaFree(pl.grp_elem_d);
  cudaFree(pl.sched_d);
  cudaFree(pl.sched_ptr_d);
  cudaFree(pl.nsub_d);
  cudaFree(pl.gslots_d);
  pl = Plan();
}

static dgchefsi_status ensure_layout(dgchefsi_ctx* ctx, TcState& t) {
  if (!t.pnb_h.empty()) return DGCHEFSI_OK;
  const int M = ctx->M;
  t.pnb_h.resize(M);
  t.poff_h.resize(M + 1);
  t.poff_h[0] = 0;
  int boxn = 16;
  for (int K = 0; K < M; ++K) {
    t.pnb_h[K] = (ctx->nb_h[K] + 15) / 16 * 16;
    t.poff_h[K + 1] = t.poff_h[K] + t.pnb_h[K];
    boxn = std::max(boxn, t.pnb_h[K]);
  }
  t.ldp = t.poff_h[M];
  t.ACC = boxn <= 32 ? 32 : (boxn <= 64 ? 64 : 128);
  t.boxn = t.ACC;  // B boxes are ACC rows high so the tiles of G elements stack along N
  t.blk_row_h.resize(ctx->nnzb);
  for (int K = 0; K < M; ++K)
    for (int64_t e = ctx->row_ptr_h[K]; e < ctx->row_ptr_h[K + 1]; ++e) t.blk_row_h[e] = K;
  int dev = 0;
  DG_CUDA(cudaGetDevice(&dev));
  DG_CUDA(cudaDeviceGetAttribute(&t.num_sms, cudaDevAttrMultiProcessorCount, dev));
  DG_CUDA(cudaMalloc(&t.pnb_d, sizeof(int32_t) * M));
  DG_CUDA(cudaMalloc(&t.poff_d, sizeof(int32_t) * (M + 1)));
  DG_CUDA(cudaMalloc(&t.blk_row_d, sizeof(int32_t) * std::max<int64_t>(ctx->nnzb, 1)));
  DG_CUDA(cudaMalloc(&t.brow_d, sizeof(int64_t) * std::max<int64_t>(ctx->nnzb, 1)));
  DG_CUDA(cudaMalloc(&t.err_d, sizeof(int)));
  DG_CUDA(cudaMemcpy(t.pnb_d, t.pnb_h.data(), sizeof(int32_t) * M, cudaMemcpyHostToDevice));
  DG_CUDA(cudaMemcpy(t.poff_d, t.poff_h.data(), sizeof(int32_t) * (M + 1), cudaMemcpyHostToDevice));
  DG_CUDA(cudaMemcpy(t.blk_row_d, t.blk_row_h.data(), sizeof(int32_t) * ctx->nnzb, cudaMemcpyHostToDevice));
  return DGCHEFSI_OK;
}

// Row layout of the operand copy of H for one slice width; plans depend on it.
static dgchefsi_status ensure_mode(dgchefsi_ctx* ctx, TcState& t, int mode) {
  if (t.mode == mode) return DGCHEFSI_OK;
  const int W = mode == MODE_TF32 ? 32 : 64;
  ++t.gen;
  for (auto& kv : t.plans) free_plan(kv.second);
  t.plans.clear();
  t.brow_h.resize(ctx->nnzb);
  int64_t r = 0;
  for (int64_t e = 0; e < ctx->nnzb; ++e) {
    t.brow_h[e] = r;
    const int Kp = ctx->col_h[e];
    r += (int64_t)((t.pnb_h[Kp] + W - 1) / W) * t.pnb_h[t.blk_row_h[e]];
  }
  t.zero_row = r;                                       // ZERO_TILES zero tiles of ACC rows
  t.b_rows = r + (int64_t)ZERO_TILES * t.boxn + t.boxn;  // plus slack for a full-height box
  if (t.b_rows * (mode == MODE_BF16X3 ? 2 : 1) > 2147483647LL)
    return set_error(DGCHEFSI_ERR_UNSUPPORTED, "operand copy of H too large for 32-bit TMA rows");
  DG_CUDA(cudaMemcpy(t.brow_d, t.brow_h.data(), sizeof(int64_t) * ctx->nnzb, cudaMemcpyHostToDevice));
  const size_t esz = mode == MODE_TF32 ? 4 : 2;
  const size_t copies = mode == MODE_BF16X3 ? 2 : 1;
  DG_TRY(ensure(ctx, t.Hop, (size_t)t.b_rows * copies * W * esz, "operand copy of H"));
  DG_CUDA(cudaMemsetAsync(t.Hop.p, 0, t.Hop.bytes, ctx->stream));
  t.mode = mode;
  return DGCHEFSI_OK;
}

static dgchefsi_status make_plan(dgchefsi_ctx* ctx, const TcState& t, int G, int W,
                                 const std::vector<int64_t>& brow_h, int64_t zero_row, Plan& out);

static dgchefsi_status get_plan(dgchefsi_ctx* ctx, TcState& t, int G, Plan** out) {
  auto it = t.plans.find(G);
  if (it != t.plans.end()) {
    *out = &it->second;
    return DGCHEFSI_OK;
  }
  Plan pl;
  DG_TRY(make_plan(ctx, t, G, t.mode == MODE_TF32 ? 32 : 64, t.brow_h, t.zero_row, pl));
  t.plans[G] = pl;
  *out = &t.plans[G];
  return DGCHEFSI_OK;
}

// Element groups and their slice schedules for an operand copy of H laid out
// with W-column slices, blocks starting at rows brow_h and zero tiles at zero_row.
static dgchefsi_status make_plan(dgchefsi_ctx* ctx, const TcState& t, int G, int W,
                                 const std::vector<int64_t>& brow_h, int64_t zero_row, Plan& out) {
  const int M = ctx->M;
  Plan pl;
  pl.G = G;
  pl.W = W;
  pl.ngroups = (M + G - 1) / G;
  std::vector<int32_t> grp((size_t)pl.ngroups * G, -1);
  for (int K = 0; K < M; ++K) grp[K] = K;  // group eg holds elements eg*G .. eg*G+G-1
  std::vector<int32_t> sched, sptr(pl.ngroups + 1, 0), gslots(pl.ngroups, 0);
  std::vector<uint8_t> nsub;
  for (int eg = 0; eg < pl.ngroups; ++eg) {
    std::vector<int> nbrs;
    for (int g = 0; g < G; ++g) {
      const int K = grp[(size_t)eg * G + g];
      if (K < 0) continue;
      for (int64_t e = ctx->row_ptr_h[K]; e < ctx->row_ptr_h[K + 1]; ++e) nbrs.push_back(ctx->col_h[e]);
    }
    std::sort(nbrs.begin(), nbrs.end());
    nbrs.erase(std::unique(nbrs.begin(), nbrs.end()), nbrs.end());
    for (int Kp : nbrs) {
      const int nsl = (t.pnb_h[Kp] + W - 1) / W;
      for (int sl = 0; sl < nsl; ++sl) {
        sched.push_back(t.poff_h[Kp] + sl * W);
        // with 64-byte slots a slice is two halves of W/2 columns; the second
        // is skipped when it lies past K''s padded size (H is zero there)
        const uint8_t ns = (t.pnb_h[Kp] - sl * W) <= W / 2 ? 1 : 2;
        nsub.push_back(ns);
        gslots[eg] += ns;
        for (int g = 0; g < G; ++g) {
          const int K = grp[(size_t)eg * G + g];
          // a zero tile (one of ZERO_TILES, spread over L2) when K does not couple to K'
          int32_t row = (int32_t)(zero_row + (int64_t)(eg % ZERO_TILES) * t.boxn);
          if (K >= 0) {
            int64_t lo = ctx->row_ptr_h[K], hi = ctx->row_ptr_h[K + 1] - 1;
            while (lo <= hi) {
              const int64_t mid = (lo + hi) / 2;
              const int cm = ctx->col_h[mid];
              if (cm == Kp) {
                row = (int32_t)(brow_h[mid] + (int64_t)sl * t.pnb_h[K]);
                break;
              }
              if (cm < Kp) lo = mid + 1; else hi = mid - 1;
            }
          }
          sched.push_back(row);
        }
      }
    }
    sptr[eg + 1] = (int32_t)(sched.size() / (1 + G));
    pl.maxent = std::max(pl.maxent, sptr[eg + 1] - sptr[eg]);
  }
  DG_CUDA(cudaMalloc(&pl.grp_elem_d, sizeof(int32_t) * grp.size()));
  DG_CUDA(cudaMalloc(&pl.sched_d, sizeof(int32_t) * std::max<size_t>(sched.size(), 1)));
  DG_CUDA(cudaMalloc(&pl.sched_ptr_d, sizeof(int32_t) * sptr.size()));
  DG_CUDA(cudaMemcpy(pl.grp_elem_d, grp.data(), sizeof(int32_t) * grp.size(), cudaMemcpyHostToDevice));
  DG_CUDA(cudaMemcpy(pl.sched_d, sched.data(), sizeof(int32_t) * sched.size(), cudaMemcpyHostToDevice));
  DG_CUDA(cudaMemcpy(pl.sched_ptr_d, sptr.data(), sizeof(int32_t) * sptr.size(), cudaMemcpyHostToDevice));
  DG_CUDA(cudaMalloc(&pl.nsub_d, std::max<size_t>(nsub.size(), 1)));
  DG_CUDA(cudaMalloc(&pl.gslots_d, sizeof(int32_t) * std::max<size_t>(gslots.size(), 1)));
  if (!nsub.empty()) DG_CUDA(cudaMemcpy(pl.nsub_d, nsub.data(), nsub.size(), cudaMemcpyHostToDevice));
  DG_CUDA(cudaMemcpy(pl.gslots_d, gslots.data(), sizeof(int32_t) * gslots.size(), cudaMemcpyHostToDevice));
  out = pl;
  return DGCHEFSI_OK;
}

static dgchefsi_status grow_iterates(dgchefsi_ctx* ctx, TcState& t, int mode, int64_t Ns);

static dgchefsi_status ensure_iterates(dgchefsi_ctx* ctx, TcState& t, int mode, int64_t Ns) {
  const void* before[6] = {t.F[0].p, t.F[1].p, t.Sh[0].p, t.Sh[1].p, t.Sl[0].p, t.Sl[1].p};
  DG_TRY(grow_iterates(ctx, t, mode, Ns));
  const void* after[6] = {t.F[0].p, t.F[1].p, t.Sh[0].p, t.Sh[1].p, t.Sl[0].p, t.Sl[1].p};
  for (int i = 0; i < 6; ++i)
    if (before[i] != after[i]) ++t.gen;
  return DGCHEFSI_OK;
}

static dgchefsi_status grow_iterates(dgchefsi_ctx* ctx, TcState& t, int mode, int64_t Ns) {
  if (t.Ns < Ns || t.F[0].p == nullptr) {
    const size_t n = (size_t)Ns * (size_t)t.ldp;
    for (int i = 0; i < 2; ++i) {
      DG_TRY(ensure(ctx, t.F[i], n * sizeof(float), "FP32 iterate"));
      DG_CUDA(cudaMemsetAsync(t.F[i].p, 0, t.F[i].bytes, ctx->stream));
    }
    t.Ns = Ns;
  }
  if (mode != MODE_TF32) {
    const size_t n = (size_t)Ns * (size_t)t.ldp * sizeof(__nv_bfloat16);
    for (int i = 0; i < 2; ++i) {
      if (t.Sh[i].bytes < n) {
        DG_TRY(ensure(ctx, t.Sh[i], n, "BF16 iterate"));
        DG_CUDA(cudaMemsetAsync(t.Sh[i].p, 0, t.Sh[i].bytes, ctx->stream));
      }
      if (mode == MODE_BF16X3 && t.Sl[i].bytes < n) {
        DG_TRY(ensure(ctx, t.Sl[i], n, "BF16 low iterate"));
        DG_CUDA(cudaMemsetAsync(t.Sl[i].p, 0, t.Sl[i].bytes, ctx->stream));
      }
    }
  }
  return DGCHEFSI_OK;
}

// row_stride: elements between rows (0 = inner, a packed matrix).
static dgchefsi_status make_map(CUtensorMap* map, void* base, bool f32, uint64_t inner, uint64_t rows,
                                uint32_t box_inner, uint32_t box_rows, bool swizzle64 = false,
                                uint64_t row_stride = 0) {
  auto enc = encode_fn();
  if (!enc) return set_error(DGCHEFSI_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  const size_t esz = f32 ? 4 : 2;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {(row_stride ? row_stride : inner) * esz};
  cuuint32_t box[2] = {box_inner, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   swizzle64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(DGCHEFSI_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return DGCHEFSI_OK;
}

static int mode_of(int prec) {
  return prec == DGCHEFSI_TF32 ? MODE_TF32 : (prec == DGCHEFSI_BF16 ? MODE_BF16 : MODE_BF16X3);
}

// Everything one filter call enqueues, for a given unit shape.
struct Launch {
  FilterKernel kern = nullptr;
  Params p{};
  CUtensorMap A0[2], A1[2], B;
  dim3 grid;
  int smem = 0;
  int layout = 0;
};

// A-operand tensor maps of one iterate: the FP32 master itself for TF32, the
// BF16 hi (A0) and lo (A1) copies otherwise.
static dgchefsi_status bind_iterate(TcState& t, int mode, int layout, int64_t Ns, const float* F,
                                    const __nv_bfloat16* Sh, const __nv_bfloat16* Sl, CUtensorMap* A0,
                                    CUtensorMap* A1) {
  const uint32_t xrows = layout >= 1 ? 256u : (uint32_t)BM;  // states per box of Y_k
  const bool sw64 = layout == 2;                              // 64-byte slots
  if (mode == MODE_TF32) {
    DG_TRY(make_map(A0, const_cast<float*>(F), true, (uint64_t)t.ldp, (uint64_t)Ns, sw64 ? 16 : 32, xrows, sw64));
    *A1 = *A0;
    return DGCHEFSI_OK;
  }
  DG_TRY(make_map(A0, const_cast<__nv_bfloat16*>(Sh), false, (uint64_t)t.ldp, (uint64_t)Ns, sw64 ? 32 : 64, xrows,
                  sw64));
  if (mode == MODE_BF16X3)
    DG_TRY(make_map(A1, const_cast<__nv_bfloat16*>(Sl), false, (uint64_t)t.ldp, (uint64_t)Ns, sw64 ? 32 : 64, xrows,
                    sw64));
  else *A1 = *A0;
  return DGCHEFSI_OK;
}

static dgchefsi_status prepare_launch(dgchefsi_ctx* ctx, TcState& t, int mode, int G, int T, int layout,
                                      int64_t Ns, Launch& L) {
  const bool f32 = mode == MODE_TF32;
  const int W = f32 ? 32 : 64;
  Plan* pl = nullptr;
  DG_TRY(get_plan(ctx, t, G, &pl));
  L.kern = pick_kernel(mode, G, T, t.ACC, layout);
  if (!L.kern)
    return set_error(DGCHEFSI_ERR_UNSUPPORTED, "no filter kernel for G=%d T=%d ACC=%d layout %d", G, T, t.ACC, layout);
  L.layout = layout;
  for (int i = 0; i < 2; ++i)
    DG_TRY(bind_iterate(t, mode, layout, Ns, static_cast<float*>(t.F[i].p), static_cast<__nv_bfloat16*>(t.Sh[i].p),
                        static_cast<__nv_bfloat16*>(t.Sl[i].p), &L.A0[i], &L.A1[i]));
  const uint64_t brows_total = (uint64_t)t.b_rows * (mode == MODE_BF16X3 ? 2 : 1);
  const int sb = layout == 2 ? 64 : SLICE_BYTES;  // ring-slot K extent in bytes
  DG_TRY(make_map(&L.B, t.Hop.p, f32, (uint64_t)W, brows_total, (uint32_t)(W * sb / SLICE_BYTES), (uint32_t)t.boxn,
                  layout == 2));
  const int na = mode == MODE_BF16X3 ? 2 : 1;
  const int stage_bytes = layout >= 1 ? na * (128 * sb + 256 * sb) : na * (T * A_BYTES + G * t.ACC * SLICE_BYTES);
  const int stages = layout >= 1 ? TN_RING_BYTES / stage_bytes : (mode == MODE_BF16X3 ? STAGES / 2 : STAGES);
  L.smem = stages * stage_bytes + (2 * stages + 4) * 8 + 2 * pl->maxent * (1 + G) * 4 + 1024;
  if (L.smem > 227 * 1024) return set_error(DGCHEFSI_ERR_UNSUPPORTED, "filter schedule too large for shared memory");
  DG_CUDA(cudaFuncSetAttribute(L.kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.smem));
  Params& p = L.p;
  p = Params{};
  p.sched = pl->sched_d;
  p.sched_ptr = pl->sched_ptr_d;
  p.nsub = pl->nsub_d;
  p.gslots = pl->gslots_d;
  p.grp_elem = pl->grp_elem_d;
  p.nb = ctx->nb_d;
  p.pnb = t.pnb_d;
  p.poff = t.poff_d;
  p.lo_rows = t.b_rows;
  p.Ns = Ns;
  p.ldp = t.ldp;
  p.coef = t.coef_d;
  p.W = W;
  p.mode = mode;
  p.boxn = t.boxn;
  p.G = G;
  p.T = T;
  p.ACC = t.ACC;
  p.NBUF = 2;
  p.stages = stages;
  p.ngroups = pl->ngroups;
  p.ntg = (int)((Ns + (int64_t)BM * T - 1) / ((int64_t)BM * T));
  p.maxent = pl->maxent;
  p.err = t.err_d;
  p.tgb = t.tgb[mode] > 0 ? t.tgb[mode] : 0;
  const int64_t nunits = (int64_t)p.ngroups * p.ntg;
  L.grid = dim3((unsigned)std::min<int64_t>(nunits, t.num_sms));
  return DGCHEFSI_OK;
}

// Step k: Y_{k+1} from Y_k (buffer k%2) and Y_{k-1} (buffer (k+1)%2).
static dgchefsi_status launch_step(dgchefsi_ctx* ctx, TcState& t, int mode, Launch& L, int k, cudaStream_t s) {
  const int cur = k & 1, nxt = cur ^ 1;
  Params p = L.p;
  p.step = k;
  p.Fprev = static_cast<float*>(t.F[nxt].p);
  p.Fout = static_cast<float*>(t.F[nxt].p);
  p.Hout = mode == MODE_TF32 ? nullptr : static_cast<__nv_bfloat16*>(t.Sh[nxt].p);
  p.Lout = mode == MODE_BF16X3 ? static_cast<__nv_bfloat16*>(t.Sl[nxt].p) : nullptr;
  L.kern<<<L.grid, NTHREADS, L.smem, s>>>(L.A0[cur], L.A1[cur], L.B, p);
  count_launch();
  DG_CUDA(cudaGetLastError());
  (void)ctx;
  return DGCHEFSI_OK;
}

// Iterate addresses of one step given explicitly (the gradient keeps its
// iterates in checkpoint and segment buffers rather than the ping-pong pair).
struct StepIO {
  const float* Fin = nullptr;          // Y_k, FP32 (the A operand for TF32)
  const __nv_bfloat16* Shin = nullptr;  // Y_k hi / lo operand copies (BF16 forms)
  const __nv_bfloat16* Slin = nullptr;
  const float* Fprev = nullptr;  // Y_{k-1} (not read while beta_k = 0)
  float* Fout = nullptr;         // Y_{k+1}; may alias Fprev
  __nv_bfloat16* Hout = nullptr;
  __nv_bfloat16* Lout = nullptr;
};

static dgchefsi_status launch_io(TcState& t, int mode, Launch& L, int k, const double* coef, const StepIO& io,
                                 cudaStream_t s) {
  CUtensorMap A0, A1;
  DG_TRY(bind_iterate(t, mode, L.layout, L.p.Ns, io.Fin, io.Shin, io.Slin, &A0, &A1));
  Params p = L.p;
  p.step = k;
  p.coef = coef;
  p.Fprev = io.Fprev ? io.Fprev : io.Fout;
  p.Fout = io.Fout;
  p.Hout = mode == MODE_TF32 ? nullptr : io.Hout;
  p.Lout = mode == MODE_BF16X3 ? io.Lout : nullptr;
  L.kern<<<L.grid, NTHREADS, L.smem, s>>>(A0, A1, L.B, p);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return DGCHEFSI_OK;
}

static dgchefsi_status upload_coefficients(dgchefsi_ctx* ctx, TcState& t, int m, double a, double b, double a0) {
  if (t.coef_cap < 1 + 2 * m) {
    if (t.gexec) {  // a captured graph refers to the old buffers
      DG_CUDA(cudaStreamSynchronize(ctx->stream));
      cudaGraphExecDestroy(t.gexec);
      t.gexec = nullptr;
    }
    cudaFree(t.coef_d);
    cudaFreeHost(t.coef_h);
    t.coef_d = nullptr;
    t.coef_h = nullptr;
    t.coef_cap = 0;
    DG_CUDA(cudaMalloc(&t.coef_d, sizeof(double) * (1 + 2 * m)));
    DG_CUDA(cudaMallocHost(&t.coef_h, sizeof(double) * (1 + 2 * m)));
    t.coef_cap = 1 + 2 * m;
  }
  const double e = 0.5 * (b - a), c = 0.5 * (b + a);
  const double s1 = e / (a0 - c);
  t.coef_h[0] = c;
  double sig = s1;
  for (int k = 0; k < m; ++k) {
    double alpha, beta;
    if (k == 0) {
      alpha = s1 / e;
      beta = 0.0;
    } else {
      const double sn = 1.0 / (2.0 / s1 - sig);
      alpha = 2.0 * sn / e;
      beta = sig * sn;
      sig = sn;
    }
    t.coef_h[1 + 2 * k] = alpha;
    t.coef_h[2 + 2 * k] = beta;
  }
  return DGCHEFSI_OK;
}

// build_hop -> pack -> steps -> unpack, all on stream s (the coefficients must be on the device).
static dgchefsi_status enqueue_filter(dgchefsi_ctx* ctx, TcState& t, int mode, Launch& L, const double* X,
                                      double* Y, int64_t Ns, int64_t ld, int m, cudaStream_t s,
                                      bool reuse_hop = false) {
  const bool f32 = mode == MODE_TF32;
  const int W = f32 ? 32 : 64;
  if (!reuse_hop) {
    k_build_hop<<<(unsigned)ctx->nnzb, 256, 0, s>>>(
        t.blk_row_d, ctx->col_d, ctx->blk_off_d, ctx->vals_d, ctx->nb_d, t.pnb_d, t.brow_d, W, t.coef_d, mode,
        t.b_rows, f32 ? static_cast<float*>(t.Hop.p) : nullptr, f32 ? nullptr : static_cast<__nv_bfloat16*>(t.Hop.p));
    count_launch();
    DG_CUDA(cudaGetLastError());
  }
  const dim3 g = pack_grid(Ns, ctx->max_nb, ctx->M);
  k_pack<<<g, 256, 0, s>>>(X, ld, Ns, ctx->off_d, ctx->nb_d, t.poff_d, t.ldp, static_cast<float*>(t.F[0].p),
                           f32 ? nullptr : static_cast<__nv_bfloat16*>(t.Sh[0].p),
                           mode == MODE_BF16X3 ? static_cast<__nv_bfloat16*>(t.Sl[0].p) : nullptr);
  count_launch();
  DG_CUDA(cudaGetLastError());
  for (int k = 0; k < m; ++k) DG_TRY(launch_step(ctx, t, mode, L, k, s));
  k_unpack<<<g, 256, 0, s>>>(static_cast<float*>(t.F[m & 1].p), t.ldp, Ns, ctx->off_d, ctx->nb_d, t.poff_d, Y, ld);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return DGCHEFSI_OK;
}

// Pick the unit shape for this precision: a forced one, the tuned one, or time
// step 0 with every candidate whose accumulator width fits and keep the fastest.
static dgchefsi_status tune_unit_order(dgchefsi_ctx* ctx, TcState& t, int mode, int64_t Ns, int G, int T,
                                       int layout);

static dgchefsi_status choose_shape(dgchefsi_ctx* ctx, TcState& t, int mode, int64_t Ns, int* G, int* T,
                                    int* layout) {
  if (t.forceG[mode]) {
    *G = t.forceG[mode];
    *T = t.forceT[mode];
    *layout = t.forceL[mode];
    return tune_unit_order(ctx, t, mode, Ns, *G, *T, *layout);
  }
  if (t.shapeG[mode]) {
    *G = t.shapeG[mode];
    *T = t.shapeT[mode];
    *layout = t.shapeL[mode];
    return tune_unit_order(ctx, t, mode, Ns, *G, *T, *layout);
  }
  cudaStream_t s = ctx->stream;
  cudaEvent_t e0, e1;
  DG_CUDA(cudaEventCreate(&e0));
  DG_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int bG = 0, bT = 0, bL = 0;
  for (int i = 0; i < NSHAPES; ++i) {
    if (SHAPES[i][2] != t.ACC) continue;
    Launch L;
    dgchefsi_status st = prepare_launch(ctx, t, mode, SHAPES[i][0], SHAPES[i][1], SHAPES[i][3], Ns, L);
    if (st != DGCHEFSI_OK) continue;
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {  // the first launch warms caches and the L2
      DG_CUDA(cudaEventRecord(e0, s));
      DG_TRY(launch_step(ctx, t, mode, L, 0, s));
      DG_CUDA(cudaEventRecord(e1, s));
      DG_CUDA(cudaEventSynchronize(e1));
      DG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    }
    t.tuned_ms[mode][i] = ms;
    if (ms < best) {
      best = ms;
      bG = SHAPES[i][0];
      bT = SHAPES[i][1];
      bL = SHAPES[i][3];
    }
  }
  if (!bG) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return set_error(DGCHEFSI_ERR_UNSUPPORTED, "no tensor-core unit shape for accumulator width %d", t.ACC);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  t.shapeG[mode] = *G = bG;
  t.shapeT[mode] = *T = bT;
  t.shapeL[mode] = *layout = bL;
  clear_error();  // a candidate without a kernel is skipped, not an error
  return tune_unit_order(ctx, t, mode, Ns, bG, bT, bL);
}

// Unit order of a shape: state tiles in blocks of 2, 4 or 8 per pass over the
// element groups (the Y_k slices one pass touches stay in L2; H is read once
// per pass), or all state tiles of a group back to back (0). A forced order
// is taken as is; otherwise step 0 is timed with each and the fastest kept.
static dgchefsi_status tune_unit_order(dgchefsi_ctx* ctx, TcState& t, int mode, int64_t Ns, int G, int T,
                                       int layout) {
  if (t.force_tgb[mode] >= 0) {
    t.tgb[mode] = t.force_tgb[mode];
    return DGCHEFSI_OK;
  }
  if (t.tgb[mode] >= 0) return DGCHEFSI_OK;
  cudaStream_t s = ctx->stream;
  cudaEvent_t e0, e1;
  DG_CUDA(cudaEventCreate(&e0));
  DG_CUDA(cudaEventCreate(&e1));
  Launch L;
  dgchefsi_status st = prepare_launch(ctx, t, mode, G, T, layout, Ns, L);
  float best = 1e30f;
  int bo = 0;
  for (int o : {0, 2, 4, 8}) {
    if (st != DGCHEFSI_OK || (o > 0 && o >= L.p.ntg)) continue;
    L.p.tgb = o;
    float ms = 0.f;
    for (int rep = 0; rep < 2 && st == DGCHEFSI_OK; ++rep) {  // the first launch warms caches
      cudaEventRecord(e0, s);
      st = launch_step(ctx, t, mode, L, 0, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        st = set_error(DGCHEFSI_ERR_CUDA, "timing the unit order failed");
    }
    if (st == DGCHEFSI_OK && ms < best) {
      best = ms;
      bo = o;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != DGCHEFSI_OK) return st;
  t.tgb[mode] = bo;
  return DGCHEFSI_OK;
}

static dgchefsi_status check_err(TcState& t, cudaStream_t s) {
  int err = 0;
  DG_CUDA(cudaMemcpyAsync(&err, t.err_d, sizeof(int), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  if (err) return set_error(DGCHEFSI_ERR_TIMEOUT, "a tensor-core filter CTA gave up waiting on a pipeline barrier");
  return DGCHEFSI_OK;
}

// The unit shape for X: when nothing is forced or tuned yet, H's operand copy
// is built and X packed into the ping-pong pair first, so that the autotuner
// times step 0 on the caller's data.
static dgchefsi_status select_shape(dgchefsi_ctx* ctx, TcState& t, int mode, const double* X, int64_t ld, int64_t Ns,
                                    int* G, int* T, int* layout) {
  if (!t.forceG[mode] && !t.shapeG[mode]) {
    cudaStream_t s = ctx->stream;
    const bool f32 = mode == MODE_TF32;
    k_build_hop<<<(unsigned)ctx->nnzb, 256, 0, s>>>(
        t.blk_row_d, ctx->col_d, ctx->blk_off_d, ctx->vals_d, ctx->nb_d, t.pnb_d, t.brow_d, f32 ? 32 : 64, t.coef_d,
        mode, t.b_rows, f32 ? static_cast<float*>(t.Hop.p) : nullptr,
        f32 ? nullptr : static_cast<__nv_bfloat16*>(t.Hop.p));
    count_launch();
    const dim3 g = pack_grid(Ns, ctx->max_nb, ctx->M);
    k_pack<<<g, 256, 0, s>>>(X, ld, Ns, ctx->off_d, ctx->nb_d, t.poff_d, t.ldp, static_cast<float*>(t.F[0].p),
                             f32 ? nullptr : static_cast<__nv_bfloat16*>(t.Sh[0].p),
                             mode == MODE_BF16X3 ? static_cast<__nv_bfloat16*>(t.Sl[0].p) : nullptr);
    count_launch();
    DG_CUDA(cudaGetLastError());
  }
  return choose_shape(ctx, t, mode, Ns, G, T, layout);
}

static dgchefsi_status tc_prepare(dgchefsi_ctx* ctx, int prec, int64_t Ns, int m, double a, double b, double a0,
                                  int* mode_out) {
  if (ctx->max_nb > 128)
    return set_error(DGCHEFSI_ERR_UNSUPPORTED, "tensor-core filter supports element sizes up to 128 (got %d)",
                     ctx->max_nb);
  if (Ns > 2147483647LL / 2 - 4 * BM) return set_error(DGCHEFSI_ERR_UNSUPPORTED, "Ns too large");
  if (!ctx->tc) ctx->tc = new TcState();
  TcState& t = *ctx->tc;
  const int mode = mode_of(prec);
  DG_TRY(ensure_layout(ctx, t));
  DG_TRY(ensure_mode(ctx, t, mode));
  DG_TRY(ensure_iterates(ctx, t, mode, Ns));
  DG_TRY(upload_coefficients(ctx, t, m, a, b, a0));
  *mode_out = mode;
  return DGCHEFSI_OK;
}

dgchefsi_status filter_tc(dgchefsi_ctx* ctx, int prec, const double* X, double* Y, int64_t Ns, int64_t ld, int m,
                          double a, double b, double a0, bool reuse_hop) {
  int mode = 0;
  DG_TRY(tc_prepare(ctx, prec, Ns, m, a, b, a0, &mode));
  TcState& t = *ctx->tc;
  cudaStream_t s = ctx->stream;
  DG_CUDA(cudaMemcpyAsync(t.coef_d, t.coef_h, sizeof(double) * (1 + 2 * m), cudaMemcpyHostToDevice, s));
  DG_CUDA(cudaMemsetAsync(t.err_d, 0, sizeof(int), s));
  int G = 0, T = 0, layout = 0;
  DG_TRY(select_shape(ctx, t, mode, X, ld, Ns, &G, &T, &layout));
  Launch L;
  DG_TRY(prepare_launch(ctx, t, mode, G, T, layout, Ns, L));
  DG_TRY(enqueue_filter(ctx, t, mode, L, X, Y, Ns, ld, m, s, reuse_hop && t.shapeG[mode] + t.forceG[mode] > 0));
  return check_err(t, s);
}

dgchefsi_status filter_tc_graph(dgchefsi_ctx* ctx, int prec, const double* X, double* Y, int64_t Ns, int64_t ld,
                                int m, double a, double b, double a0) {
  int mode = 0;
  DG_TRY(tc_prepare(ctx, prec, Ns, m, a, b, a0, &mode));
  TcState& t = *ctx->tc;
  cudaStream_t s = ctx->stream;
  if (!t.forceG[mode] && !t.shapeG[mode]) {
    // tune with one ordinary call (host synchronisation is not allowed under capture)
    DG_TRY(filter_tc(ctx, prec, X, Y, Ns, ld, m, a, b, a0));
    DG_TRY(upload_coefficients(ctx, t, m, a, b, a0));
  }
  int G = 0, T = 0, layout = 0;
  DG_TRY(choose_shape(ctx, t, mode, Ns, &G, &T, &layout));
  const bool same = t.gexec && t.g_mode == mode && t.g_m == m && t.g_G == G && t.g_T == T && t.g_L == layout &&
                    t.g_X == X && t.g_Y == Y && t.g_Ns == Ns && t.g_ld == ld && t.g_gen == t.gen;
  if (!same) {
    if (t.gexec) {
      DG_CUDA(cudaStreamSynchronize(s));
      cudaGraphExecDestroy(t.gexec);
      t.gexec = nullptr;
    }
    if (!t.cap_stream) DG_CUDA(cudaStreamCreateWithFlags(&t.cap_stream, cudaStreamNonBlocking));
    Launch L;
    DG_TRY(prepare_launch(ctx, t, mode, G, T, layout, Ns, L));
    cudaGraph_t graph = nullptr;
    DG_CUDA(cudaStreamBeginCapture(t.cap_stream, cudaStreamCaptureModeThreadLocal));
    // the coefficients are copied from the pinned host mirror at every replay
    cudaError_t e1 = cudaMemcpyAsync(t.coef_d, t.coef_h, sizeof(double) * (1 + 2 * m), cudaMemcpyHostToDevice,
                                     t.cap_stream);
    cudaError_t e2 = cudaMemsetAsync(t.err_d, 0, sizeof(int), t.cap_stream);
    dgchefsi_status st = DGCHEFSI_OK;
    if (e1 == cudaSuccess && e2 == cudaSuccess) st = enqueue_filter(ctx, t, mode, L, X, Y, Ns, ld, m, t.cap_stream);
    cudaError_t e3 = cudaStreamEndCapture(t.cap_stream, &graph);
    if (e1 != cudaSuccess || e2 != cudaSuccess || st != DGCHEFSI_OK || e3 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      if (st != DGCHEFSI_OK) return st;
      return set_error(DGCHEFSI_ERR_CUDA, "capture of the filter graph failed");
    }
    cudaError_t e4 = cudaGraphInstantiate(&t.gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e4 != cudaSuccess) {
      t.gexec = nullptr;
      return set_error(DGCHEFSI_ERR_CUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(e4));
    }
    t.g_mode = mode;
    t.g_gen = t.gen;
    t.g_m = m;
    t.g_G = G;
    t.g_T = T;
    t.g_L = layout;
    t.g_X = X;
    t.g_Y = Y;
    t.g_Ns = Ns;
    t.g_ld = ld;
  }
  DG_CUDA(cudaGraphLaunch(t.gexec, s));
  count_launch(m + 3);
  return check_err(t, s);
}

// ---- band-energy gradient on the tensor-core filter

// Workspace of the gradient: 2 nseg checkpoint blocks, stride - 2 segment
// blocks, 3 rotation blocks and the backward pair, all FP32 in the padded
// layout, plus BF16 operand copies of the backward pair. Zeroed when
// (re)allocated so element pads read as zero.
static dgchefsi_status ensure_grad(dgchefsi_ctx* ctx, TcState& t, int mode, int64_t Ns, int m, int stride) {
  const int nseg = (m + stride - 1) / stride;
  const size_t fblk = ((size_t)Ns * (size_t)t.ldp * sizeof(float) + 255) / 256 * 256;
  const size_t hblk = ((size_t)Ns * (size_t)t.ldp * sizeof(__nv_bfloat16) + 255) / 256 * 256;
  const int nf = 2 * nseg + std::max(stride - 2, 0) + 3 + 2;
  const int nh = mode == MODE_TF32 ? 0 : (mode == MODE_BF16X3 ? 4 : 2);
  const size_t need = fblk * nf + hblk * nh;
  DG_TRY(ensure(ctx, t.gbuf, need, "gradient checkpoints"));
  DG_CUDA(cudaMemsetAsync(t.gbuf.p, 0, need, ctx->stream));  // block offsets move with Ns
  char* base = static_cast<char*>(t.gbuf.p);
  size_t o = 0;
  auto takef = [&]() { float* q = reinterpret_cast<float*>(base + o); o += fblk; return q; };
  auto takeh = [&]() { __nv_bfloat16* q = reinterpret_cast<__nv_bfloat16*>(base + o); o += hblk; return q; };
  t.cp0.assign(nseg, nullptr);
  t.cp1.assign(nseg, nullptr);
  for (int j = 0; j < nseg; ++j) {
    t.cp0[j] = takef();
    t.cp1[j] = takef();
  }
  t.segb.assign(std::max(stride - 2, 0), nullptr);
  for (auto& q : t.segb) q = takef();
  for (auto& q : t.R) q = takef();
  for (auto& q : t.WF) q = takef();
  for (int i = 0; i < 2; ++i) {
    t.WSh[i] = mode == MODE_TF32 ? nullptr : takeh();
    t.WSl[i] = mode == MODE_BF16X3 ? takeh() : nullptr;
  }
  t.g_stride = stride;
  t.g_nseg = nseg;
  t.g_mm = m;
  return DGCHEFSI_OK;
}

static __nv_bfloat16* bf_ptr(DevBuf& b) { return static_cast<__nv_bfloat16*>(b.p); }

dgchefsi_status tc_grad_forward(dgchefsi_ctx* ctx, int prec, const double* X, int64_t ld, int64_t Ns, int m,
                                double a, double b, double a0, int stride, double* Ym) {
  int mode = 0;
  DG_TRY(tc_prepare(ctx, prec, Ns, m, a, b, a0, &mode));
  TcState& t = *ctx->tc;
  cudaStream_t s = ctx->stream;
  DG_CUDA(cudaMemcpyAsync(t.coef_d, t.coef_h, sizeof(double) * (1 + 2 * m), cudaMemcpyHostToDevice, s));
  DG_CUDA(cudaMemsetAsync(t.err_d, 0, sizeof(int), s));
  int G = 0, T = 0, layout = 0;
  DG_TRY(select_shape(ctx, t, mode, X, ld, Ns, &G, &T, &layout));
  DG_TRY(ensure_grad(ctx, t, mode, Ns, m, stride));
  Launch L;
  DG_TRY(prepare_launch(ctx, t, mode, G, T, layout, Ns, L));
  t.g_mG = G;
  t.g_mT = T;
  t.g_mL = layout;
  const bool f32 = mode == MODE_TF32;
  const int W = f32 ? 32 : 64;
  k_build_hop<<<(unsigned)ctx->nnzb, 256, 0, s>>>(
      t.blk_row_d, ctx->col_d, ctx->blk_off_d, ctx->vals_d, ctx->nb_d, t.pnb_d, t.brow_d, W, t.coef_d, mode, t.b_rows,
      f32 ? static_cast<float*>(t.Hop.p) : nullptr, f32 ? nullptr : bf_ptr(t.Hop));
  count_launch();
  const dim3 g = pack_grid(Ns, ctx->max_nb, ctx->M);
  k_pack<<<g, 256, 0, s>>>(X, ld, Ns, ctx->off_d, ctx->nb_d, t.poff_d, t.ldp, t.cp0[0], f32 ? nullptr : bf_ptr(t.Sh[0]),
                           mode == MODE_BF16X3 ? bf_ptr(t.Sl[0]) : nullptr);
  count_launch();
  DG_CUDA(cudaGetLastError());
  // Y_{k+1} goes straight to its checkpoint slot, else to the rotation block
  // that holds neither Y_k nor Y_{k-1}.
  std::vector<float*> pos(m + 1, nullptr);
  pos[0] = t.cp0[0];
  for (int k = 0; k < m; ++k) {
    const int kk = k + 1;
    float* out = t.R[kk % 3];
    if (kk < m && kk % stride == 0) out = t.cp0[kk / stride];
    else if (kk < m && stride > 1 && kk % stride == 1) out = t.cp1[kk / stride];
    StepIO io;
    io.Fin = pos[k];
    io.Shin = f32 ? nullptr : bf_ptr(t.Sh[k & 1]);
    io.Slin = mode == MODE_BF16X3 ? bf_ptr(t.Sl[k & 1]) : nullptr;
    io.Fprev = k > 0 ? pos[k - 1] : out;
    io.Fout = out;
    io.Hout = f32 ? nullptr : bf_ptr(t.Sh[kk & 1]);
    io.Lout = mode == MODE_BF16X3 ? bf_ptr(t.Sl[kk & 1]) : nullptr;
    DG_TRY(launch_io(t, mode, L, k, t.coef_d, io, s));
    pos[kk] = out;
  }
  k_unpack<<<g, 256, 0, s>>>(pos[m], t.ldp, Ns, ctx->off_d, ctx->nb_d, t.poff_d, Ym, ctx->N);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return check_err(t, s);
}

dgchefsi_status tc_grad_backward(dgchefsi_ctx* ctx, int prec, const double* Wm, int64_t Ns, int m, int stride,
                                 double* H_bar, double* X_bar, int64_t ld_xbar) {
  if (!ctx->tc || ctx->tc->g_stride != stride || ctx->tc->g_mm != m || ctx->tc->Ns < Ns)
    return set_error(DGCHEFSI_ERR_ARG, "tensor-core gradient backward without its forward");
  TcState& t = *ctx->tc;
  const int mode = mode_of(prec);
  if (t.mode != mode) return set_error(DGCHEFSI_ERR_ARG, "backward precision differs from the forward's");
  cudaStream_t s = ctx->stream;
  const bool f32 = mode == MODE_TF32;
  const int nseg = t.g_nseg;
  // backward coefficients from the forward ones on the pinned mirror:
  // step j computes W_k, k = m-1-j, with alpha_k and beta_{k+1} (0 for j = 0)
  if (t.coefb_cap < 1 + 2 * m) {
    cudaFree(t.coefb_d);
    t.coefb_d = nullptr;
    t.coefb_cap = 0;
    DG_CUDA(cudaMalloc(&t.coefb_d, sizeof(double) * (1 + 2 * m)));
    t.coefb_cap = 1 + 2 * m;
  }
  std::vector<double> cb(1 + 2 * m);
  cb[0] = t.coef_h[0];
  for (int j = 0; j < m; ++j) {
    const int k = m - 1 - j;
    cb[1 + 2 * j] = t.coef_h[1 + 2 * k];
    cb[2 + 2 * j] = j == 0 ? 0.0 : t.coef_h[2 + 2 * (k + 1)];
  }
  DG_CUDA(cudaMemcpyAsync(t.coefb_d, cb.data(), sizeof(double) * cb.size(), cudaMemcpyHostToDevice, s));
  DG_CUDA(cudaMemsetAsync(t.err_d, 0, sizeof(int), s));
  Launch L;
  DG_TRY(prepare_launch(ctx, t, mode, t.g_mG, t.g_mT, t.g_mL, Ns, L));
  const dim3 g = pack_grid(Ns, ctx->max_nb, ctx->M);
  k_pack<<<g, 256, 0, s>>>(Wm, ctx->N, Ns, ctx->off_d, ctx->nb_d, t.poff_d, t.ldp, t.WF[0], t.WSh[0], t.WSl[0]);
  count_launch();
  DG_CUDA(cudaGetLastError());
  const int tiles = (ctx->max_nb + 63) / 64;
  const dim3 go((unsigned)ctx->nnzb, (unsigned)tiles, (unsigned)tiles);
  const int64_t nsh = Ns * t.ldp;
  const unsigned gsh = (unsigned)std::min<int64_t>((nsh + 255) / 256, 8 * (int64_t)t.num_sms);
  int jb = 0;
  std::vector<const float*> ypos(stride + 1, nullptr);
  for (int j = nseg - 1; j >= 0; --j) {
    const int k0 = j * stride, k1 = std::min(m, k0 + stride);
    ypos[0] = t.cp0[j];
    if (k1 - k0 > 1) ypos[1] = t.cp1[j];
    if (k1 - k0 > 2) {
      if (!f32) {
        k_shadow<<<gsh, 256, 0, s>>>(t.cp1[j], nsh, bf_ptr(t.Sh[(k0 + 1) & 1]),
                                     mode == MODE_BF16X3 ? bf_ptr(t.Sl[(k0 + 1) & 1]) : nullptr);
        count_launch();
        DG_CUDA(cudaGetLastError());
      }
      for (int kk = k0 + 2; kk < k1; ++kk) {
        const int q = kk - k0;
        StepIO io;
        io.Fin = ypos[q - 1];
        io.Shin = f32 ? nullptr : bf_ptr(t.Sh[(kk - 1) & 1]);
        io.Slin = mode == MODE_BF16X3 ? bf_ptr(t.Sl[(kk - 1) & 1]) : nullptr;
        io.Fprev = ypos[q - 2];
        io.Fout = t.segb[q - 2];
        io.Hout = f32 ? nullptr : bf_ptr(t.Sh[kk & 1]);
        io.Lout = mode == MODE_BF16X3 ? bf_ptr(t.Sl[kk & 1]) : nullptr;
        DG_TRY(launch_io(t, mode, L, kk - 1, t.coef_d, io, s));
        ypos[q] = t.segb[q - 2];
      }
    }
    for (int k = k1 - 1; k >= k0; --k, ++jb) {
      const int cur = jb & 1, nxt = cur ^ 1;
      if (H_bar) {
        k_block_outer_f32<<<go, 256, 0, s>>>(t.blk_row_d, ctx->col_d, ctx->blk_off_d, ctx->nb_d, t.poff_d, t.WF[cur],
                                             ypos[k - k0], t.ldp, Ns, t.coef_h[1 + 2 * k], H_bar);
        count_launch();
        DG_CUDA(cudaGetLastError());
      }
      // W_k = alpha_k (H - cI) W_{k+1} - beta_{k+1} W_{k+2}, over W_{k+2}
      StepIO io;
      io.Fin = t.WF[cur];
      io.Shin = t.WSh[cur];
      io.Slin = t.WSl[cur];
      io.Fprev = t.WF[nxt];
      io.Fout = t.WF[nxt];
      io.Hout = t.WSh[nxt];
      io.Lout = t.WSl[nxt];
      DG_TRY(launch_io(t, mode, L, jb, t.coefb_d, io, s));
    }
  }
  if (X_bar) {
    k_unpack<<<g, 256, 0, s>>>(t.WF[m & 1], t.ldp, Ns, ctx->off_d, ctx->nb_d, t.poff_d, X_bar, ld_xbar);
    count_launch();
    DG_CUDA(cudaGetLastError());
  }
  return check_err(t, s);
}

// Workspace cap of the FP32 slice-pair slabs of the sliced H X; the states run
// in panels of 256-state multiples below it.
static constexpr size_t kSlabBytes = size_t(8) << 30;

dgchefsi_status tc_sliced_matvec(dgchefsi_ctx* ctx, const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t Ns,
                                 int s, int* flag, bool* used) {
  *used = false;
  if (Ns <= 0) {
    *used = true;
    return DGCHEFSI_OK;
  }
  if (ctx->max_nb > 128 || s < 2 || s > 16) return DGCHEFSI_OK;
  if (!ctx->tc) ctx->tc = new TcState();
  TcState& t = *ctx->tc;
  DG_TRY(ensure_layout(ctx, t));
  auto& sx = t.sx;
  constexpr int W = 64;
  cudaStream_t st = ctx->stream;
  if (!sx.layout) {
    // W = 64 block layout of the slice copies (the BF16 filter's), the longest
    // row (padded columns of its neighbour blocks) and the padded column map
    sx.brow_h.resize(ctx->nnzb);
    int64_t r = 0;
    for (int64_t e = 0; e < ctx->nnzb; ++e) {
      sx.brow_h[e] = r;
      r += (int64_t)((t.pnb_h[ctx->col_h[e]] + W - 1) / W) * t.pnb_h[t.blk_row_h[e]];
    }
    sx.zero_row = r;
    sx.b_rows = r + (int64_t)ZERO_TILES * t.boxn + t.boxn;
    for (int K = 0; K < ctx->M; ++K) {
      int64_t len = 0;
      for (int64_t e = ctx->row_ptr_h[K]; e < ctx->row_ptr_h[K + 1]; ++e) len += ctx->nb_h[ctx->col_h[e]];
      sx.max_row_len = std::max(sx.max_row_len, len);
    }
    std::vector<int32_t> cmap((size_t)t.ldp, -1);
    for (int K = 0; K < ctx->M; ++K)
      for (int j = 0; j < ctx->nb_h[K]; ++j) cmap[(size_t)t.poff_h[K] + j] = (int32_t)(ctx->off_h[K] + j);
    DG_CUDA(cudaMalloc(&sx.brow_d, sizeof(int64_t) * std::max<int64_t>(ctx->nnzb, 1)));
    DG_CUDA(cudaMalloc(&sx.cmap_d, sizeof(int32_t) * (size_t)t.ldp));
    DG_CUDA(cudaMalloc(&sx.eh_d, sizeof(int32_t) * (size_t)t.ldp));
    DG_CUDA(cudaMalloc(&sx.coef_d, sizeof(double) * 3));
    const double coef[3] = {0.0, 1.0, 0.0};
    DG_CUDA(cudaMemcpy(sx.brow_d, sx.brow_h.data(), sizeof(int64_t) * ctx->nnzb, cudaMemcpyHostToDevice));
    DG_CUDA(cudaMemcpy(sx.cmap_d, cmap.data(), sizeof(int32_t) * (size_t)t.ldp, cudaMemcpyHostToDevice));
    DG_CUDA(cudaMemcpy(sx.coef_d, coef, sizeof(coef), cudaMemcpyHostToDevice));
    DG_TRY(make_plan(ctx, t, 128 / t.ACC, W, sx.brow_h, sx.zero_row, sx.plan));
    sx.layout = true;
  }
  // every pair sum must stay an exact FP32 integer: at most 4096 terms per row
  if (sx.max_row_len > 4096) return DGCHEFSI_OK;
  if (sx.b_rows * (int64_t)W > ((int64_t)1 << 31) || Ns * t.ldp > ((int64_t)1 << 40)) return DGCHEFSI_OK;
  const int G = 128 / t.ACC, T = 2;
  FilterKernel kern = pick_kernel(MODE_BF16, G, T, t.ACC, 1);
  if (!kern) return DGCHEFSI_OK;
  // H's digits (once per H and slice count)
  const int64_t hcopy = sx.b_rows * W;
  if (!sx.h_built || sx.h_slices != s) {
    if (sx.Hs.bytes < sizeof(__nv_bfloat16) * (size_t)(s * hcopy)) {
      DG_TRY(ensure(ctx, sx.Hs, sizeof(__nv_bfloat16) * (size_t)(s * hcopy), "slices of H"));
      DG_CUDA(cudaMemsetAsync(sx.Hs.p, 0, sx.Hs.bytes, st));  // zero tiles and slack rows
    }
    DG_CUDA(slices_of_h(ctx, t.blk_row_d, t.pnb_d, t.poff_d, sx.brow_d, s, static_cast<__nv_bfloat16*>(sx.Hs.p), hcopy,
                        sx.eh_d, flag, st));
    sx.h_built = true;
    sx.h_slices = s;
  }
  // the states' digits and exponents
  const int64_t xcopy = Ns * t.ldp;
  DG_TRY(ensure(ctx, sx.Xs, sizeof(__nv_bfloat16) * (size_t)(s * xcopy), "slices of the states"));
  DG_TRY(ensure(ctx, sx.ex, sizeof(int32_t) * (size_t)Ns, "state exponents"));
  __nv_bfloat16* Xq = static_cast<__nv_bfloat16*>(sx.Xs.p);
  int32_t* ex = static_cast<int32_t*>(sx.ex.p);
  DG_CUDA(slices_of_states(X, ldx, Ns, ctx->N, sx.cmap_d, t.ldp, s, Xq, xcopy, ex, flag, st));
  // state panels whose slabs fit the cap
  const int pairs = s * (s + 1) / 2;
  const int64_t per_state = (int64_t)pairs * t.ldp * (int64_t)sizeof(float);
  int64_t P = (int64_t)(kSlabBytes / (size_t)per_state) / 256 * 256;
  if (P < 256) P = 256;
  if (P > Ns) P = Ns;
  DG_TRY(ensure(ctx, sx.Pw, (size_t)per_state * (size_t)P, "slice-pair slabs"));
  float* Pw = static_cast<float*>(sx.Pw.p);
  // launch configuration of the transposed step kernel (layout 1, 128-byte slots)
  const int stage_bytes = 128 * SLICE_BYTES + 256 * SLICE_BYTES;
  const int stages = TN_RING_BYTES / stage_bytes;
  const int smem = stages * stage_bytes + (2 * stages + 4) * 8 + 2 * sx.plan.maxent * (1 + G) * 4 + 1024;
  if (smem > 227 * 1024) return DGCHEFSI_OK;
  DG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  Params p{};
  p.sched = sx.plan.sched_d;
  p.sched_ptr = sx.plan.sched_ptr_d;
  p.nsub = sx.plan.nsub_d;
  p.gslots = sx.plan.gslots_d;
  p.grp_elem = sx.plan.grp_elem_d;
  p.nb = ctx->nb_d;
  p.pnb = t.pnb_d;
  p.poff = t.poff_d;
  p.lo_rows = 0;
  p.ldp = t.ldp;
  p.coef = sx.coef_d;
  p.step = 0;
  p.W = W;
  p.mode = MODE_BF16;
  p.boxn = t.boxn;
  p.G = G;
  p.T = T;
  p.ACC = t.ACC;
  p.NBUF = 2;
  p.stages = stages;
  p.ngroups = sx.plan.ngroups;
  p.maxent = sx.plan.maxent;
  p.err = t.err_d;
  p.Hout = nullptr;
  p.Lout = nullptr;
  DG_CUDA(cudaMemsetAsync(t.err_d, 0, sizeof(int), st));
  std::vector<CUtensorMap> hmap(s);
  for (int i = 0; i < s; ++i)
    DG_TRY(make_map(&hmap[i], static_cast<__nv_bfloat16*>(sx.Hs.p) + (size_t)i * hcopy, false, (uint64_t)W,
                    (uint64_t)sx.b_rows, (uint32_t)W, (uint32_t)t.boxn));
  for (int64_t s0 = 0; s0 < Ns; s0 += P) {
    const int64_t pn = std::min<int64_t>(P, Ns - s0);
    p.Ns = pn;
    p.ntg = (int)((pn + 255) / 256);
    const unsigned grid = (unsigned)std::min<int64_t>((int64_t)p.ngroups * p.ntg, t.num_sms);
    for (int j = 0; j < s; ++j) {
      CUtensorMap xmap;
      DG_TRY(make_map(&xmap, Xq + (size_t)j * xcopy + (size_t)s0 * t.ldp, false, (uint64_t)t.ldp, (uint64_t)pn,
                      (uint32_t)W, 256u));
      for (int i = 0; i + j < s; ++i) {
        p.Fout = Pw + (size_t)(i * s - i * (i - 1) / 2 + j) * (size_t)(pn * t.ldp);
        p.Fprev = p.Fout;
        kern<<<grid, NTHREADS, smem, st>>>(xmap, xmap, hmap[i], p);
        count_launch();
        DG_CUDA(cudaGetLastError());
      }
    }
    DG_TRY(reduce_pair_slabs(Pw, pn, t.ldp, ex + s0, sx.eh_d, sx.cmap_d, Y + s0 * ldy, ldy, s, st));
  }
  DG_TRY(check_err(t, st));
  *used = true;
  return DGCHEFSI_OK;
}

dgchefsi_status tc_set_shape(dgchefsi_ctx* ctx, int prec, int G, int T, int layout) {
  if (!ctx->tc) ctx->tc = new TcState();
  TcState& t = *ctx->tc;
  DG_TRY(ensure_layout(ctx, t));
  const int mode = mode_of(prec);
  if (G == 0 && T == 0) {
    t.forceG[mode] = t.forceT[mode] = t.forceL[mode] = 0;
    if (t.force_tgb[mode] < 0) t.tgb[mode] = -1;
    return DGCHEFSI_OK;
  }
  if (!pick_kernel(mode, G, T, t.ACC, layout))
    return set_error(DGCHEFSI_ERR_UNSUPPORTED, "no kernel for G=%d T=%d layout %d with accumulator width %d", G, T,
                     layout, t.ACC);
  t.forceG[mode] = G;
  t.forceT[mode] = T;
  t.forceL[mode] = layout;
  t.tgb[mode] = -1;  // a new shape gets its unit order tuned again
  return DGCHEFSI_OK;
}

dgchefsi_status tc_set_unit_order(dgchefsi_ctx* ctx, int prec, int tgb) {
  if (!ctx->tc) ctx->tc = new TcState();
  TcState& t = *ctx->tc;
  const int mode = mode_of(prec);
  t.force_tgb[mode] = tgb;
  t.tgb[mode] = tgb;
  return DGCHEFSI_OK;
}

dgchefsi_status tc_get_unit_order(dgchefsi_ctx* ctx, int prec, int* tgb) {
  *tgb = (ctx->tc && ctx->tc->tgb[mode_of(prec)] >= 0) ? ctx->tc->tgb[mode_of(prec)] : -1;
  return DGCHEFSI_OK;
}

dgchefsi_status tc_get_shape(dgchefsi_ctx* ctx, int prec, int* G, int* T, int* ACC, int* layout) {
  if (!ctx->tc) {
    *G = *T = *ACC = *layout = 0;
    return DGCHEFSI_OK;
  }
  TcState& t = *ctx->tc;
  const int mode = mode_of(prec);
  *G = t.forceG[mode] ? t.forceG[mode] : t.shapeG[mode];
  *T = t.forceG[mode] ? t.forceT[mode] : t.shapeT[mode];
  *layout = t.forceG[mode] ? t.forceL[mode] : t.shapeL[mode];
  *ACC = t.ACC;
  return DGCHEFSI_OK;
}

void tc_destroy(dgchefsi_ctx* ctx) {
  if (!ctx->tc) return;
  TcState& t = *ctx->tc;
  if (t.gexec) cudaGraphExecDestroy(t.gexec);
  if (t.cap_stream) cudaStreamDestroy(t.cap_stream);
  for (auto& kv : t.plans) free_plan(kv.second);
  cudaFree(t.pnb_d);
  cudaFree(t.poff_d);
  cudaFree(t.blk_row_d);
  cudaFree(t.brow_d);
  cudaFree(t.err_d);
  cudaFree(t.coef_d);
  cudaFreeHost(t.coef_h);
  for (int i = 0; i < 2; ++i) {
    cudaFree(t.F[i].p);
    cudaFree(t.Sh[i].p);
    cudaFree(t.Sl[i].p);
  }
  cudaFree(t.Hop.p);
  free_plan(t.sx.plan);
  cudaFree(t.sx.brow_d);
  cudaFree(t.sx.cmap_d);
  cudaFree(t.sx.eh_d);
  cudaFree(t.sx.coef_d);
  cudaFree(t.sx.Hs.p);
  cudaFree(t.sx.Xs.p);
  cudaFree(t.sx.Pw.p);
  cudaFree(t.sx.ex.p);
  cudaFree(t.gbuf.p);
  cudaFree(t.coefb_d);
  delete ctx->tc;
  ctx->tc = nullptr;
}

}  // namespace dg
