// Chebyshev filter on the tcgen05 tensor cores (Alg. 1 step 2; Eq. matvec_3).
//
// One step of the scaled recurrence is, per element K and per tile of 128 states,
//     Y_{k+1}[s, K] = alpha_k * sum_{K' in N(K)} (H - cI)_{KK'} Y_k[s, K'] - beta_k * Y_{k-1}[s, K]
// i.e. a dense GEMM with M = 128 states, N = n_K (padded to 16) and a K dimension
// that runs over the neighbour blocks, followed by the recurrence update. One CTA
// owns one (state tile, element) output tile:
//   * warp 0 / lane 0 streams 128-byte-wide K slices of Y_k (A operand, 128 rows)
//     and of (H - cI) (B operand, n_K rows) with TMA into a 4-stage shared-memory
//     ring (SWIZZLE_128B, K-major), signalling mbarriers;
//   * warp 1 / lane 0 issues tcgen05.mma (kind::f16 for BF16, kind::tf32 for
//     TF32) into a 128 x n_K FP32 accumulator in tensor memory and frees each
//     ring slot with tcgen05.commit;
//   * all four warps then read the accumulator (tcgen05.ld, one state row per
//     thread) and apply alpha_k, -beta_k Y_{k-1} (FP32 master copy), writing the
//     FP32 master of Y_{k+1} and, for the BF16 forms, its BF16 operand copies.
// The shift -cI is folded into the diagonal block of the operand copy of H,
// rebuilt once per filter call. Iterates live in an element-padded layout
// (every element starts on a 16-column boundary, pads held at zero) so TMA
// coordinates are always 16-byte aligned; pads of H are zero so neighbouring
// columns read by a wide K slice contribute nothing.
//
// BF16X3 splits every operand v into hi = bf16(v) and lo = bf16(v - hi) and
// accumulates hi*hi + hi*lo + lo*hi (three K passes over the same neighbours),
// which recovers close to FP32 accuracy on the BF16 tensor pipe.
//
// Every wait on an mbarrier is bounded by wall-clock time; on expiry the CTA
// records DGCHEFSI_ERR_TIMEOUT in a device word, drains its own copies in
// flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "ctx.h"

namespace dg {

namespace {

constexpr int BM = 128;           // states per tile (MMA M)
constexpr int SLICE_BYTES = 128;  // K extent of one ring slot in bytes (one swizzle row)
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * SLICE_BYTES;
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // 2 s per wait

enum Mode { MODE_TF32 = 0, MODE_BF16 = 1, MODE_BF16X3 = 2 };

struct Params {
  const int64_t* row_ptr;
  const int32_t* col;
  const int32_t* nb;
  const int32_t* pnb;   // padded element sizes (multiple of 16)
  const int32_t* poff;  // padded element offsets
  const int64_t* brow;  // first row of block e in the B operand tensor
  int64_t lo_rows;      // BF16X3: row offset of the lo copy of H
  int64_t Ns, ldp;
  const float* Fprev;
  float* Fout;
  __nv_bfloat16* Hout;
  __nv_bfloat16* Lout;
  float alpha, beta;
  int W;      // elements per slice: 64 (BF16) or 32 (TF32)
  int mode;
  int boxn;   // rows of a B box (max padded element size)
  int* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: true once the phase with the given parity has completed.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtime();
  while (true) {
    for (int i = 0; i < 32; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (gtime() - t0 > WAIT_LIMIT_NS) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor: FP32 accumulate, A/B format code `fmt` (1 = BF16 for
// kind::f16, 2 = TF32 for kind::tf32), both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc(uint32_t fmt, uint32_t n) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(128, 1)
    k_filter_step_tc(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
                     const __grid_constant__ CUtensorMap tmB, const Params p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int b_bytes = p.boxn * SLICE_BYTES;
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + STAGES * b_bytes);  // full[S], empty[S], acc
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int K = blockIdx.y;
  const int64_t s0 = (int64_t)blockIdx.x * BM;
  const int nK = p.nb[K];
  const int pK = p.pnb[K];
  const uint32_t ncols = pK <= 32 ? 32u : (pK <= 64 ? 64u : 128u);
  const int npass = p.mode == MODE_BF16X3 ? 3 : 1;
  const int64_t e0 = p.row_ptr[K], e1 = p.row_ptr[K + 1];

  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), accb = smem_u32(bars + 2 * STAGES);
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(accb, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0 && lane == 0) {
    // ---------------- producer: TMA into the ring
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA0)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
    int c = 0;
    bool ok = true;
    for (int64_t e = e0; e < e1 && ok; ++e) {
      const int Kp = p.col[e];
      const int nsl = (p.pnb[Kp] + p.W - 1) / p.W;
      const int x0 = p.poff[Kp];
      const int64_t r0 = p.brow[e];
      for (int sl = 0; sl < nsl && ok; ++sl) {
        for (int pass = 0; pass < npass; ++pass) {
          const int st = c % STAGES;
          const uint32_t ph = (uint32_t)(c / STAGES) & 1u;
          if (!mbar_wait(empty0 + 8 * st, ph ^ 1u)) {
            ok = false;
            break;
          }
          mbar_expect_tx(full0 + 8 * st, (uint32_t)(A_BYTES + b_bytes));
          tma_load_2d(smem_u32(sA + st * A_BYTES), pass == 2 ? &tmA1 : &tmA0, x0 + sl * p.W, (int)s0,
                      full0 + 8 * st);
          const int64_t brow = r0 + (int64_t)sl * pK + (pass == 1 ? p.lo_rows : 0);
          tma_load_2d(smem_u32(sB + st * b_bytes), &tmB, 0, (int)brow, full0 + 8 * st);
          ++c;
        }
      }
    }
    if (!ok) {
      atomicOr(p.err, 1);
      atomicExch(&abort_sh, 1);
    }
    // drain: every issued copy must land before the CTA may exit
    for (int i = std::max(0, c - STAGES); i < c; ++i)
      if (!mbar_wait(full0 + 8 * (i % STAGES), (uint32_t)(i / STAGES) & 1u)) atomicOr(p.err, 1);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    int total = 0;
    for (int64_t e = e0; e < e1; ++e) total += (p.pnb[p.col[e]] + p.W - 1) / p.W;
    total *= npass;
    const uint32_t id = idesc(p.mode == MODE_TF32 ? 2u : 1u, (uint32_t)pK);
    for (int c = 0; c < total; ++c) {
      const int st = c % STAGES;
      const uint32_t ph = (uint32_t)(c / STAGES) & 1u;
      if (!mbar_wait(full0 + 8 * st, ph)) {
        atomicOr(p.err, 1);
        atomicExch(&abort_sh, 1);
        break;
      }
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA + st * A_BYTES), b0 = smem_u32(sB + st * b_bytes);
#pragma unroll
      for (int kk = 0; kk < SLICE_BYTES / 32; ++kk) {
        const uint64_t ad = sdesc(a0 + 32 * kk), bd = sdesc(b0 + 32 * kk);
        const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
        if (p.mode == MODE_TF32) mma_tf32(tmem, ad, bd, id, acc);
        else mma_bf16(tmem, ad, bd, id, acc);
      }
      mma_commit(empty0 + 8 * st);
    }
    mma_commit(accb);
  }

  // ---------------- epilogue: every thread owns one state row
  __syncwarp();
  bool ready = mbar_wait(accb, 0);
  ready = __all_sync(0xffffffffu, ready);
  tc_fence_after();
  if (!ready && lane == 0) atomicOr(p.err, 1);
  const bool store = ready && (*(volatile int*)&abort_sh == 0);
  const int row = warp * 32 + lane;
  const int64_t s = s0 + row;
  const bool live = store && s < p.Ns;
  const int64_t base = s * p.ldp + p.poff[K];
  for (int j0 = 0; j0 < pK; j0 += 16) {
    float v[16];
    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)j0, v);
    if (!live) continue;
    const int jn = min(16, nK - j0);
    if (jn <= 0) continue;
    float y[16];
    if (jn == 16) {
      const float4* pv = reinterpret_cast<const float4*>(p.Fprev + base + j0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float4 pr = make_float4(0.f, 0.f, 0.f, 0.f);
        if (p.beta != 0.f) pr = pv[q];
        y[4 * q + 0] = p.alpha * v[4 * q + 0] - p.beta * pr.x;
        y[4 * q + 1] = p.alpha * v[4 * q + 1] - p.beta * pr.y;
        y[4 * q + 2] = p.alpha * v[4 * q + 2] - p.beta * pr.z;
        y[4 * q + 3] = p.alpha * v[4 * q + 3] - p.beta * pr.w;
      }
      float4* po = reinterpret_cast<float4*>(p.Fout + base + j0);
#pragma unroll
      for (int q = 0; q < 4; ++q) po[q] = make_float4(y[4 * q], y[4 * q + 1], y[4 * q + 2], y[4 * q + 3]);
      if (p.mode != MODE_TF32) {
        uint32_t hw[8], lw[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(y[2 * q], y[2 * q + 1]);
          const float2 hf = __bfloat1622float2(h2);
          const __nv_bfloat162 l2 = __floats2bfloat162_rn(y[2 * q] - hf.x, y[2 * q + 1] - hf.y);
          hw[q] = *reinterpret_cast<const uint32_t*>(&h2);
          lw[q] = *reinterpret_cast<const uint32_t*>(&l2);
        }
        uint4* ph = reinterpret_cast<uint4*>(p.Hout + base + j0);
        ph[0] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        ph[1] = make_uint4(hw[4], hw[5], hw[6], hw[7]);
        if (p.mode == MODE_BF16X3) {
          uint4* pl = reinterpret_cast<uint4*>(p.Lout + base + j0);
          pl[0] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
          pl[1] = make_uint4(lw[4], lw[5], lw[6], lw[7]);
        }
      }
    } else {
      for (int q = 0; q < jn; ++q) {
        const int64_t idx = base + j0 + q;
        const float pr = p.beta != 0.f ? p.Fprev[idx] : 0.f;
        const float yv = p.alpha * v[q] - p.beta * pr;
        p.Fout[idx] = yv;
        if (p.mode != MODE_TF32) {
          const __nv_bfloat16 h = __float2bfloat16_rn(yv);
          p.Hout[idx] = h;
          if (p.mode == MODE_BF16X3) p.Lout[idx] = __float2bfloat16_rn(yv - __bfloat162float(h));
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

// X (FP64, natural layout, ld) -> FP32 master + BF16 hi / lo copies in the padded layout.
__global__ void k_pack(const double* __restrict__ X, int64_t ld, int64_t Ns, const int64_t* __restrict__ off,
                       const int32_t* __restrict__ nb, const int32_t* __restrict__ poff, int64_t ldp,
                       float* __restrict__ F, __nv_bfloat16* __restrict__ Hh, __nv_bfloat16* __restrict__ Hl) {
  const int K = blockIdx.y;
  const int n = nb[K];
  const int64_t o = off[K];
  const int po = poff[K];
  for (int64_t s = blockIdx.x; s < Ns; s += gridDim.x) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
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
}

// FP32 padded layout -> FP64 natural layout.
__global__ void k_unpack(const float* __restrict__ F, int64_t ldp, int64_t Ns, const int64_t* __restrict__ off,
                         const int32_t* __restrict__ nb, const int32_t* __restrict__ poff, double* __restrict__ Y,
                         int64_t ld) {
  const int K = blockIdx.y;
  const int n = nb[K];
  const int64_t o = off[K];
  const int po = poff[K];
  for (int64_t s = blockIdx.x; s < Ns; s += gridDim.x)
    for (int j = threadIdx.x; j < n; j += blockDim.x) Y[s * ld + o + j] = (double)F[s * ldp + po + j];
}

// Operand copy of (H - cI): for block e = (K, K') and slice sl of K', rows
// brow[e] + sl * pnb[K] + n (n < pnb[K]), W columns each; zero outside the block.
__global__ void k_build_hop(const int32_t* __restrict__ blk_row, const int32_t* __restrict__ col,
                            const int64_t* __restrict__ blk_off, const double* __restrict__ vals,
                            const int32_t* __restrict__ nb, const int32_t* __restrict__ pnb,
                            const int64_t* __restrict__ brow, int W, double c, int mode, int64_t lo_rows,
                            float* __restrict__ H32, __nv_bfloat16* __restrict__ H16) {
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

}  // namespace

struct TcState {
  int64_t Ns = -1, ldp = 0;
  int mode = -1;
  std::vector<int32_t> pnb_h, poff_h, blk_row_h;
  std::vector<int64_t> brow_h;
  int64_t b_rows = 0;  // rows of one copy of H in the operand tensor
  int boxn = 0;
  int32_t *pnb_d = nullptr, *poff_d = nullptr, *blk_row_d = nullptr;
  int64_t* brow_d = nullptr;
  DevBuf F[2], Sh[2], Sl[2], Hop;
  int* err_d = nullptr;
};

static dgchefsi_status tc_setup(dgchefsi_ctx* ctx, int mode, int64_t Ns) {
  if (!ctx->tc) ctx->tc = new TcState();
  TcState& t = *ctx->tc;
  const int M = ctx->M;
  const int W = mode == MODE_TF32 ? 32 : 64;
  if (t.pnb_h.empty()) {
    t.pnb_h.resize(M);
    t.poff_h.resize(M + 1);
    t.poff_h[0] = 0;
    int boxn = 16;
    for (int K = 0; K < M; ++K) {
      t.pnb_h[K] = (ctx->nb_h[K] + 15) / 16 * 16;
      t.poff_h[K + 1] = t.poff_h[K] + t.pnb_h[K];
      boxn = std::max(boxn, t.pnb_h[K]);
    }
    t.boxn = boxn;
    t.ldp = t.poff_h[M];
    t.blk_row_h.resize(ctx->nnzb);
    for (int K = 0; K < M; ++K)
      for (int64_t e = ctx->row_ptr_h[K]; e < ctx->row_ptr_h[K + 1]; ++e) t.blk_row_h[e] = K;
    DG_CUDA(cudaMalloc(&t.pnb_d, sizeof(int32_t) * M));
    DG_CUDA(cudaMalloc(&t.poff_d, sizeof(int32_t) * (M + 1)));
    DG_CUDA(cudaMalloc(&t.blk_row_d, sizeof(int32_t) * std::max<int64_t>(ctx->nnzb, 1)));
    DG_CUDA(cudaMalloc(&t.brow_d, sizeof(int64_t) * std::max<int64_t>(ctx->nnzb, 1)));
    DG_CUDA(cudaMalloc(&t.err_d, sizeof(int)));
    DG_CUDA(cudaMemcpy(t.pnb_d, t.pnb_h.data(), sizeof(int32_t) * M, cudaMemcpyHostToDevice));
    DG_CUDA(cudaMemcpy(t.poff_d, t.poff_h.data(), sizeof(int32_t) * (M + 1), cudaMemcpyHostToDevice));
    DG_CUDA(cudaMemcpy(t.blk_row_d, t.blk_row_h.data(), sizeof(int32_t) * ctx->nnzb, cudaMemcpyHostToDevice));
  }
  if (t.mode != mode) {  // B row layout depends on the slice width
    t.brow_h.resize(ctx->nnzb);
    int64_t r = 0;
    for (int64_t e = 0; e < ctx->nnzb; ++e) {
      t.brow_h[e] = r;
      const int Kp = ctx->col_h[e];
      r += (int64_t)((t.pnb_h[Kp] + W - 1) / W) * t.pnb_h[t.blk_row_h[e]];
    }
    t.b_rows = r + t.boxn;  // slack so a full-height box never leaves the tensor
    DG_CUDA(cudaMemcpy(t.brow_d, t.brow_h.data(), sizeof(int64_t) * ctx->nnzb, cudaMemcpyHostToDevice));
    const size_t esz = mode == MODE_TF32 ? 4 : 2;
    const size_t copies = mode == MODE_BF16X3 ? 2 : 1;
    DG_TRY(ensure(ctx, t.Hop, (size_t)t.b_rows * copies * W * esz, "operand copy of H"));
    DG_CUDA(cudaMemsetAsync(t.Hop.p, 0, t.Hop.bytes, ctx->stream));
    t.mode = mode;
  }
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

static dgchefsi_status make_map(CUtensorMap* map, void* base, bool f32, uint64_t inner, uint64_t rows,
                                uint32_t box_inner, uint32_t box_rows) {
  auto enc = encode_fn();
  if (!enc) return set_error(DGCHEFSI_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  const size_t esz = f32 ? 4 : 2;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * esz};
  cuuint32_t box[2] = {box_inner, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(DGCHEFSI_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return DGCHEFSI_OK;
}

dgchefsi_status filter_tc(dgchefsi_ctx* ctx, int prec, const double* X, double* Y, int64_t Ns, int64_t ld, int m,
                          double a, double b, double a0) {
  if (ctx->max_nb > 128)
    return set_error(DGCHEFSI_ERR_UNSUPPORTED, "tensor-core filter supports element sizes up to 128 (got %d)",
                     ctx->max_nb);
  if (Ns > 2147483647LL - BM) return set_error(DGCHEFSI_ERR_UNSUPPORTED, "Ns too large");
  const int mode = prec == DGCHEFSI_TF32 ? MODE_TF32 : (prec == DGCHEFSI_BF16 ? MODE_BF16 : MODE_BF16X3);
  const int W = mode == MODE_TF32 ? 32 : 64;
  DG_TRY(tc_setup(ctx, mode, Ns));
  TcState& t = *ctx->tc;
  cudaStream_t s = ctx->stream;
  const double e = 0.5 * (b - a), c = 0.5 * (b + a);
  const double s1 = e / (a0 - c);
  const bool f32 = mode == MODE_TF32;
  __nv_bfloat16* Hop16 = f32 ? nullptr : static_cast<__nv_bfloat16*>(t.Hop.p);
  float* Hop32 = f32 ? static_cast<float*>(t.Hop.p) : nullptr;
  k_build_hop<<<(unsigned)ctx->nnzb, 256, 0, s>>>(t.blk_row_d, ctx->col_d, ctx->blk_off_d, ctx->vals_d, ctx->nb_d,
                                                  t.pnb_d, t.brow_d, W, c, mode, t.b_rows, Hop32, Hop16);
  count_launch();
  DG_CUDA(cudaGetLastError());
  // Y_0 = X in buffer 0
  auto sh = [&](int i) { return static_cast<__nv_bfloat16*>(t.Sh[i].p); };
  auto sl = [&](int i) { return static_cast<__nv_bfloat16*>(t.Sl[i].p); };
  auto fb = [&](int i) { return static_cast<float*>(t.F[i].p); };
  {
    dim3 g((unsigned)std::min<int64_t>(Ns, 1024), (unsigned)ctx->M);
    k_pack<<<g, 128, 0, s>>>(X, ld, Ns, ctx->off_d, ctx->nb_d, t.poff_d, t.ldp, fb(0), f32 ? nullptr : sh(0),
                             mode == MODE_BF16X3 ? sl(0) : nullptr);
    count_launch();
    DG_CUDA(cudaGetLastError());
  }
  CUtensorMap mapF[2], mapH[2], mapL[2], mapB;
  for (int i = 0; i < 2; ++i) {
    if (f32) {
      DG_TRY(make_map(&mapF[i], t.F[i].p, true, (uint64_t)t.ldp, (uint64_t)Ns, 32, BM));
    } else {
      DG_TRY(make_map(&mapH[i], t.Sh[i].p, false, (uint64_t)t.ldp, (uint64_t)Ns, 64, BM));
      if (mode == MODE_BF16X3) DG_TRY(make_map(&mapL[i], t.Sl[i].p, false, (uint64_t)t.ldp, (uint64_t)Ns, 64, BM));
      else mapL[i] = mapH[i];
    }
  }
  const uint64_t brows_total = (uint64_t)t.b_rows * (mode == MODE_BF16X3 ? 2 : 1);
  DG_TRY(make_map(&mapB, t.Hop.p, f32, (uint64_t)W, brows_total, (uint32_t)W, (uint32_t)t.boxn));

  const int smem = STAGES * (A_BYTES + t.boxn * SLICE_BYTES) + (2 * STAGES + 1) * 8 + 1024;
  DG_CUDA(cudaFuncSetAttribute(k_filter_step_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  DG_CUDA(cudaMemsetAsync(t.err_d, 0, sizeof(int), s));
  Params p{};
  p.row_ptr = ctx->row_ptr_d;
  p.col = ctx->col_d;
  p.nb = ctx->nb_d;
  p.pnb = t.pnb_d;
  p.poff = t.poff_d;
  p.brow = t.brow_d;
  p.lo_rows = t.b_rows;
  p.Ns = Ns;
  p.ldp = t.ldp;
  p.W = W;
  p.mode = mode;
  p.boxn = t.boxn;
  p.err = t.err_d;
  dim3 grid((unsigned)((Ns + BM - 1) / BM), (unsigned)ctx->M);
  double sig = s1;
  for (int k = 0; k < m; ++k) {
    // step k: Y_{k+1} from Y_k (buffer k%2) and Y_{k-1} (buffer (k+1)%2)
    const int cur = k & 1, nxt = cur ^ 1;
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
    p.alpha = (float)alpha;
    p.beta = (float)beta;
    p.Fprev = fb(nxt);
    p.Fout = fb(nxt);
    p.Hout = f32 ? nullptr : sh(nxt);
    p.Lout = mode == MODE_BF16X3 ? sl(nxt) : nullptr;
    const CUtensorMap& A0 = f32 ? mapF[cur] : mapH[cur];
    const CUtensorMap& A1 = f32 ? mapF[cur] : mapL[cur];
    k_filter_step_tc<<<grid, 128, smem, s>>>(A0, A1, mapB, p);
    count_launch();
    DG_CUDA(cudaGetLastError());
  }
  {
    dim3 g((unsigned)std::min<int64_t>(Ns, 1024), (unsigned)ctx->M);
    k_unpack<<<g, 128, 0, s>>>(fb(m & 1), t.ldp, Ns, ctx->off_d, ctx->nb_d, t.poff_d, Y, ld);
    count_launch();
    DG_CUDA(cudaGetLastError());
  }
  int err = 0;
  DG_CUDA(cudaMemcpyAsync(&err, t.err_d, sizeof(int), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  if (err) return set_error(DGCHEFSI_ERR_TIMEOUT, "a tensor-core filter CTA gave up waiting on a pipeline barrier");
  return DGCHEFSI_OK;
}

void tc_destroy(dgchefsi_ctx* ctx) {
  if (!ctx->tc) return;
  TcState& t = *ctx->tc;
  cudaFree(t.pnb_d);
  cudaFree(t.poff_d);
  cudaFree(t.blk_row_d);
  cudaFree(t.brow_d);
  cudaFree(t.err_d);
  for (int i = 0; i < 2; ++i) {
    cudaFree(t.F[i].p);
    cudaFree(t.Sh[i].p);
    cudaFree(t.Sl[i].p);
  }
  cudaFree(t.Hop.p);
  delete ctx->tc;
  ctx->tc = nullptr;
}

}  // namespace dg
