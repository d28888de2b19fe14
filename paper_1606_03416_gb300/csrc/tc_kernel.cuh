// Chebyshev filter on the tcgen05 tensor cores (Alg. 1 step 2; Eq. matvec_3).
//
// One step of the scaled recurrence is, per element K and state tile,
//     Y_{k+1}[s, K] = alpha_k * sum_{K' in N(K)} (H - cI)_{KK'} Y_k[s, K'] - beta_k * Y_{k-1}[s, K]
// i.e. a dense GEMM with M = 128 states, N = n_K (padded to 16) and a K dimension
// running over the neighbour blocks, followed by the recurrence update.
//
// Persistent, warp-specialised kernel, one CTA per SM (320 threads):
//   * warp 0 (one lane) streams 128-byte-wide K slices with TMA into a
//     shared-memory ring (SWIZZLE_128B, K-major): per slot, T state tiles of
//     Y_k (A operands, 128 rows each) and the blocks of (H - cI) that couple the
//     slice's element K' to each of the G output elements of the work unit
//     (B operands);
//   * warp 1 (one lane) issues tcgen05.mma (kind::f16 for BF16, kind::tf32 for
//     TF32) into G x T FP32 accumulators in tensor memory, double-buffered
//     across work units, and frees ring slots with tcgen05.commit;
//   * warps 2-9 drain a finished unit's accumulators (tcgen05.ld, one state row
//     per thread) while the next unit is multiplied, apply alpha_k and
//     -beta_k Y_{k-1} (FP32 master), and write the FP32 master of Y_{k+1} and,
//     for the BF16 forms, its BF16 operand copies.
// A work unit is G consecutive elements x T consecutive state tiles; it walks
// the union of the G elements' neighbour lists, so each A slice loaded is used
// for every element of the unit that couples to it, and each B block for all
// T state tiles. The shift -cI is folded into the diagonal blocks of the
// operand copy of H, rebuilt once per filter call. Iterates live in an
// element-padded layout (every element starts on a 16-column boundary, pads
// held at zero) so TMA coordinates stay 16-byte aligned; pads of H are zero,
// so columns of a neighbouring element read by a wide slice contribute nothing.
//
// BF16X3 splits every operand v into hi = bf16(v) and lo = bf16(v - hi) and
// accumulates hi*hi + hi*lo + lo*hi (three passes per slice), which recovers
// close to FP32 accuracy on the BF16 tensor pipe.
//
// Every wait on an mbarrier is bounded by wall-clock time; on expiry the CTA
// records DGCHEFSI_ERR_TIMEOUT in a device word, drains its own copies in
// flight, frees its tensor memory and returns.
#pragma once
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
constexpr int NTHREADS = 320;  // producer warp, MMA warp, 8 epilogue warps
constexpr int EPI_WARPS = 8;
constexpr int STAGES = 4;       // ring slots (each T A-tiles + G B-tiles)
constexpr int ZERO_TILES = 64;  // zero B tiles for non-coupling elements, spread over L2
constexpr int A_BYTES = BM * SLICE_BYTES;
constexpr int TN_RING_BYTES = 192 * 1024;  // ring of the transposed kernel (any slot size)
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // 2 s per wait

constexpr int MAXG = 4;

enum Mode { MODE_TF32 = 0, MODE_BF16 = 1, MODE_BF16X3 = 2 };

struct Params {
  const int32_t* sched;      // slice entries: [A x coordinate, B row for each of the G elements or -1]
  const int32_t* sched_ptr;  // [ngroups + 1] first entry of each element group
  const int32_t* grp_elem;   // [ngroups * G] elements of each group (-1 past the end)
  const int32_t* nb;
  const int32_t* pnb;   // padded element sizes (multiple of 16)
  const int32_t* poff;  // padded element offsets
  int64_t lo_rows;      // BF16X3: row offset of the lo copy of H
  int64_t Ns, ldp;
  const float* Fprev;
  float* Fout;
  __nv_bfloat16* Hout;
  __nv_bfloat16* Lout;
  const double* coef;  // [1 + 2m]: c, then alpha_k, beta_k of each step (device)
  int step;            // k: this launch computes Y_{k+1}
  int W;      // elements per slice: 64 (BF16) or 32 (TF32)
  int mode;
  int boxn;   // rows of a B box (max padded element size)
  int G, T, ACC, NBUF, stages;
  int ngroups, ntg;
  int maxent;  // most slice entries of any element group (shared-memory copy size)
  int* err;
  // 64-byte ring slots only: ring slots of each slice entry (1 when the slice's
  // second half lies past its element's padded size, so its H columns are all
  // zero) and of each element group
  const uint8_t* nsub;
  const int32_t* gslots;
  // unit order: blocks of tgb state tiles, each walking every element group
  // (tgb consecutive units per group) before the next block; 0 = all state
  // tiles of a group back to back (one block)
  int tgb;
};

// Element group and state tile of work unit u.
__device__ __forceinline__ void unit_coords(const Params& p, int u, int& eg, int& tg) {
  const int b = p.tgb > 0 && p.tgb < p.ntg ? p.tgb : p.ntg;
  const int tb = u / (p.ngroups * b);
  const int rem = u - tb * p.ngroups * b;
  const int cnt = min(b, p.ntg - tb * b);
  eg = rem / cnt;
  tg = tb * b + (rem - eg * cnt);
}

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

// Bounded wait: true once the phase with the given parity has completed,
// false after limit_ns of wall-clock time.
__device__ __noinline__ bool mbar_wait_for(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtime();
  while (true) {
    for (int i = 0; i < 32; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (gtime() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  return mbar_wait_for(bar, parity, WAIT_LIMIT_NS);
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

// The same for rows of SB bytes (128: 128-byte swizzle, layout code 2; 64:
// 64-byte swizzle, layout code 4), 8-row groups 8 * SB bytes apart.
template <int SB>
__device__ __forceinline__ uint64_t sdesc_sb(uint32_t addr) {
  static_assert(SB == 128 || SB == 64, "slice width");
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)((8 * SB) >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)(SB == 128 ? 2 : 4) << 61);
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


__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// Epilogue of one 16-column chunk of one state row.
__device__ __forceinline__ void store_chunk(const Params& p, float alpha, float beta, int64_t idx, int jn,
                                            const float (&v)[16], const float4 (&pr)[4]) {
  float y[16];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    y[4 * q + 0] = alpha * v[4 * q + 0] - beta * pr[q].x;
    y[4 * q + 1] = alpha * v[4 * q + 1] - beta * pr[q].y;
    y[4 * q + 2] = alpha * v[4 * q + 2] - beta * pr[q].z;
    y[4 * q + 3] = alpha * v[4 * q + 3] - beta * pr[q].w;
  }
  if (jn == 16) {
    float4* po = reinterpret_cast<float4*>(p.Fout + idx);
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
      uint4* ph = reinterpret_cast<uint4*>(p.Hout + idx);
      ph[0] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      ph[1] = make_uint4(hw[4], hw[5], hw[6], hw[7]);
      if (p.mode == MODE_BF16X3) {
        uint4* pl = reinterpret_cast<uint4*>(p.Lout + idx);
        pl[0] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        pl[1] = make_uint4(lw[4], lw[5], lw[6], lw[7]);
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      if (q < jn) {
        p.Fout[idx + q] = y[q];
        if (p.mode != MODE_TF32) {
          const __nv_bfloat16 h = __float2bfloat16_rn(y[q]);
          p.Hout[idx + q] = h;
          if (p.mode == MODE_BF16X3) p.Lout[idx + q] = __float2bfloat16_rn(y[q] - __bfloat162float(h));
        }
      }
    }
  }
}

// Fprev for one chunk (zeros when beta == 0 or the row is not live).
__device__ __forceinline__ void load_prev(const Params& p, float beta, int64_t idx, int jn, bool live,
                                          float4 (&pr)[4]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) pr[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (!live || beta == 0.f || jn <= 0) return;
  if (jn == 16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) pr[q] = ld4(p.Fprev + idx + 4 * q);
  } else {
    float t[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) t[q] = q < jn ? p.Fprev[idx + q] : 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) pr[q] = make_float4(t[4 * q], t[4 * q + 1], t[4 * q + 2], t[4 * q + 3]);
  }
}

// MODE_, G, T and ACC (accumulator columns per element) are compile-time so
// the single MMA-issuing thread runs a fully unrolled loop of descriptor adds:
// with N = 64 each MMA is only ~32 tensor-core cycles, so issue overhead
// would otherwise dominate.
template <int MODE_, int G, int T, int ACC>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_filter_step_tc(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
                     const __grid_constant__ CUtensorMap tmB, const Params p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  // BF16X3 keeps the hi and lo copies of both operands in one ring slot (its
  // three products reuse them), so its slots are twice as large and half as many.
  constexpr int NA = MODE_ == MODE_BF16X3 ? 2 : 1;
  constexpr int S = MODE_ == MODE_BF16X3 ? STAGES / 2 : STAGES;
  constexpr int b_bytes = ACC * SLICE_BYTES;  // one element's B tile: ACC rows of 128 bytes
  constexpr int a_part = NA * T * A_BYTES;    // [A hi x T][A lo x T]
  constexpr int stage_bytes = a_part + NA * G * b_bytes;  // then [B hi x G][B lo x G]
  constexpr uint32_t NMMA = (uint32_t)(G * ACC);  // the G elements' B tiles are stacked along N
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * stage_bytes);
  // per-role copies of the current group's slice entries (producer, MMA issuer)
  int32_t* sched_sh0 = reinterpret_cast<int32_t*>(bars + 2 * S + 4);
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nunits = p.ngroups * p.ntg;
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * S;
  const uint32_t accf0 = empty0 + 8 * S, acce0 = accf0 + 16;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, EPI_WARPS);
    }
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0) {
    // ---------------- producer: TMA into the ring (lane 0 issues; the warp copies schedules)
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA0)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
    }
    int c = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
      int eg, tg;
      unit_coords(p, u, eg, tg);
      const int s0 = tg * BM * T;
      const int e0 = p.sched_ptr[eg], ne = p.sched_ptr[eg + 1] - e0;
      __syncwarp();
      for (int z = lane; z < ne * (1 + G); z += 32) sched_sh0[z] = p.sched[(int64_t)e0 * (1 + G) + z];
      __syncwarp();
      if (lane == 0 && ok) {
        for (int e = 0; e < ne && ok; ++e) {
          const int32_t* ent = sched_sh0 + e * (1 + G);
          const int ax = ent[0];
          {
            const int st = c & (S - 1);
            const uint32_t ph = (uint32_t)(c / S) & 1u;
            if (!mbar_wait(empty0 + 8 * st, ph ^ 1u)) {
              ok = false;
              break;
            }
            const uint32_t fb = full0 + 8 * st;
            mbar_expect_tx(fb, (uint32_t)stage_bytes);
            uint8_t* sst = smem + st * stage_bytes;
#pragma unroll
            for (int v = 0; v < NA; ++v)
#pragma unroll
              for (int t = 0; t < T; ++t)
                tma_load_2d(smem_u32(sst + (v * T + t) * A_BYTES), v == 1 ? &tmA1 : &tmA0, ax, s0 + BM * t, fb);
#pragma unroll
            for (int v = 0; v < NA; ++v)
#pragma unroll
              for (int g = 0; g < G; ++g) {
                const int r = ent[1 + g];  // a zero block when element g does not couple to this slice
                tma_load_2d(smem_u32(sst + a_part + (v * G + g) * b_bytes), &tmB, 0,
                            (int)(r + (v == 1 ? p.lo_rows : 0)), fb);
              }
            ++c;
          }
        }
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
    }
    if (lane == 0) {
      if (!ok) {
        atomicOr(p.err, 1);
        atomicExch(&abort_sh, 1);
      }
      // drain: every issued copy must land before the CTA may exit
      for (int i = c - S < 0 ? 0 : c - S; i < c; ++i)
        if (!mbar_wait(full0 + 8 * (i & (S - 1)), (uint32_t)(i / S) & 1u)) atomicOr(p.err, 1);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (lane 0 issues; the warp copies schedules)
    constexpr uint32_t fmt = MODE_ == MODE_TF32 ? 2u : 1u;
    // descriptor of the ring's first byte; every operand is an offset from it
    const uint64_t desc0 = sdesc(smem_u32(smem));
    int c = 0, i = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < nunits; u += gridDim.x, ++i) {
      int eg, tg_;
      unit_coords(p, u, eg, tg_);
      const int ne = p.sched_ptr[eg + 1] - p.sched_ptr[eg];
      if (lane == 0 && ok) {
        const int buf = p.NBUF == 2 ? (i & 1) : 0;
        const int use = p.NBUF == 2 ? (i >> 1) : i;
        if (!mbar_wait(acce0 + 8 * buf, ((uint32_t)use & 1u) ^ 1u)) ok = false;
        tc_fence_after();
        constexpr uint32_t ID = idesc(fmt, NMMA);
        const uint32_t dbuf = tmem + (uint32_t)(buf * T * G * ACC);
        uint32_t first = 0;  // the unit's first slice overwrites the accumulators
        for (int e = 0; e < ne && ok; ++e) {
          const int st = c & (S - 1);
          const uint32_t ph = (uint32_t)(c / S) & 1u;
          if (!mbar_wait(full0 + 8 * st, ph)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t da = desc0 + (uint64_t)((st * stage_bytes) >> 4);  // A hi
          const uint64_t db = da + (uint64_t)(a_part >> 4);                   // B hi
#pragma unroll
          for (int t = 0; t < T; ++t) {
            const uint32_t d = dbuf + (uint32_t)(t * G * ACC);
#pragma unroll
            for (int kk = 0; kk < SLICE_BYTES / 32; ++kk) {
              const uint64_t ad = da + (uint64_t)((t * A_BYTES + 32 * kk) >> 4);
              const uint64_t bd = db + (uint64_t)((32 * kk) >> 4);
              const uint32_t acc = kk > 0 ? 1u : first;
              if constexpr (MODE_ == MODE_TF32) {
                mma_tf32(d, ad, bd, ID, acc);
              } else {
                mma_bf16(d, ad, bd, ID, acc);
                if constexpr (MODE_ == MODE_BF16X3) {
                  // hi * lo(H) and lo * hi(H)
                  mma_bf16(d, ad, bd + (uint64_t)((G * b_bytes) >> 4), ID, 1u);
                  mma_bf16(d, ad + (uint64_t)((T * A_BYTES) >> 4), bd, ID, 1u);
                }
              }
            }
          }
          first = 1u;
          mma_commit(empty0 + 8 * st);
          ++c;
        }
        mma_commit(accf0 + 8 * buf);
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
    }
    if (lane == 0 && !ok) {
      atomicOr(p.err, 1);
      atomicExch(&abort_sh, 1);
    }
  } else {
    // ---------------- epilogue: warps 2..9; two warps per TMEM lane quarter split
    // the 16-column chunks of each accumulator; one state row per thread.
    const float alpha = (float)p.coef[1 + 2 * p.step], beta = (float)p.coef[2 + 2 * p.step];
    const int q = warp & 3;          // TMEM lane quarter this warp may access
    const int h = (warp - 2) >> 2;   // which half of the chunks
    int i = 0;
    for (int u = blockIdx.x; u < nunits; u += gridDim.x, ++i) {
      const int buf = p.NBUF == 2 ? (i & 1) : 0;
      const int use = p.NBUF == 2 ? (i >> 1) : i;
      int eg, tg;
      unit_coords(p, u, eg, tg);
      const int64_t s0 = (int64_t)tg * BM * T;
      bool ready = mbar_wait(accf0 + 8 * buf, (uint32_t)use & 1u);
      ready = __all_sync(0xffffffffu, ready);
      if (!ready) {
        if (lane == 0) atomicOr(p.err, 1);
        break;
      }
      tc_fence_after();
      const bool go = *(volatile int*)&abort_sh == 0;
      for (int g = 0; g < G; ++g) {
        const int K = p.grp_elem[eg * G + g];
        if (K < 0) continue;
        const int nK = p.nb[K], pK = p.pnb[K];
        const int nch = pK >> 4;
        const int64_t col = p.poff[K];
        for (int t = 0; t < T; ++t) {
          const int64_t s = s0 + BM * t + 32 * q + lane;
          const bool live = go && s < p.Ns;
          const int64_t rbase = s * p.ldp + col;
          const uint32_t ta = tmem + (uint32_t)(((buf * T + t) * G + g) * ACC) + ((uint32_t)(32 * q) << 16);
          // all loads of Y_{k-1} for this warp's chunks first (memory-level parallelism)
          float4 pr[4][4];
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            const int c = h + 2 * cc;
            const int jn = nK - 16 * c;
            load_prev(p, beta, rbase + 16 * c, jn > 16 ? 16 : jn, live && c < nch, pr[cc]);
          }
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            const int c = h + 2 * cc;
            if (c < nch) {
              float v[16];
              tmem_ld16(ta + (uint32_t)(16 * c), v);
              const int jn = nK - 16 * c;
              if (live && jn > 0) store_chunk(p, alpha, beta, rbase + 16 * c, jn > 16 ? 16 : jn, v, pr[cc]);
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce0 + 8 * buf);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}



// Transposed orientation: the MMA's M = 128 rows are the H rows of the unit's
// G = 128/ACC elements stacked (A operand: the blocks (H - cI)_{K_g K'} of one
// slice), and N = 256 states (B operand: the slice of Y_k for 256 states).
// Per ring slot 16 KB of A and 32 KB of B feed four 128x256x16 MMAs, so the
// tensor core reads 48 KB of shared memory per slot instead of 64 KB, issues
// half as many instructions, and the epilogue (tensor-memory lane = element
// row, column = state) writes along element rows, coalesced across the warp.
// SB is the K extent of a ring slot in bytes: 128 (one 128-byte swizzle row per
// slice of the schedule) or 64 (each slice split into two slots with 64-byte
// swizzle), which halves the slot and doubles the ring depth in the same
// shared memory, so a refill has three slots of MMA time to land instead of one.
template <int MODE_, int ACC, int SB = SLICE_BYTES>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_filter_step_tn(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
                     const __grid_constant__ CUtensorMap tmB, const Params p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  constexpr int G = 128 / ACC;   // elements stacked along M
  constexpr int NS = 256;        // states per unit (MMA N)
  constexpr int NA = MODE_ == MODE_BF16X3 ? 2 : 1;
  constexpr int h_bytes = ACC * SB;             // one element's H tile
  constexpr int a_bytes = G * h_bytes;          // 128 SB: the stacked H tiles (MMA A)
  constexpr int x_bytes = NS * SB;              // 256 SB: the Y_k slice (MMA B)
  constexpr int stage_bytes = NA * (a_bytes + x_bytes);  // [H hi][H lo][X hi][X lo]
  constexpr int S = TN_RING_BYTES / stage_bytes;          // 2, 4 or 8 slots
  constexpr int NSUB = SLICE_BYTES / SB;                  // ring slots per schedule slice
  constexpr int ESZ = MODE_ == MODE_TF32 ? 4 : 2;
  static_assert((S & (S - 1)) == 0, "ring depth must be a power of two");
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * stage_bytes);
  int32_t* sched_sh0 = reinterpret_cast<int32_t*>(bars + 2 * S + 4);
  int32_t* sched_sh1 = sched_sh0 + p.maxent * (1 + G);
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nunits = p.ngroups * p.ntg;
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * S;
  const uint32_t accf0 = empty0 + 8 * S, acce0 = accf0 + 16;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, EPI_WARPS);
    }
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0) {
    // ---------------- producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA0)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
    }
    int c = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
      int eg, tg;
      unit_coords(p, u, eg, tg);
      const int s0 = tg * NS;
      const int e0 = p.sched_ptr[eg], ne = p.sched_ptr[eg + 1] - e0;
      __syncwarp();
      for (int z = lane; z < ne * (1 + G); z += 32) sched_sh0[z] = p.sched[(int64_t)e0 * (1 + G) + z];
      if constexpr (NSUB > 1)  // ring slots per entry, staged beside the schedule
        for (int z = lane; z < ne; z += 32) sched_sh1[z] = p.nsub[e0 + z];
      __syncwarp();
      if (lane == 0 && ok) {
        for (int e = 0; e < ne && ok; ++e) {
          const int32_t* ent = sched_sh0 + e * (1 + G);
          const int nsub = NSUB == 1 ? 1 : sched_sh1[e];
          for (int sub = 0; sub < nsub; ++sub) {
            const int st = c & (S - 1);
            const uint32_t ph = (uint32_t)(c / S) & 1u;
            if (!mbar_wait(empty0 + 8 * st, ph ^ 1u)) {
              ok = false;
              break;
            }
            const uint32_t fb = full0 + 8 * st;
            mbar_expect_tx(fb, (uint32_t)stage_bytes);
            uint8_t* sst = smem + st * stage_bytes;
            const int xo = sub * (SB / ESZ);  // element offset of this K part (16-byte multiple)
#pragma unroll
            for (int v = 0; v < NA; ++v) {
#pragma unroll
              for (int g = 0; g < G; ++g)  // H tiles (zero tiles for non-coupling elements)
                tma_load_2d(smem_u32(sst + v * a_bytes + g * h_bytes), &tmB, xo,
                            (int)(ent[1 + g] + (v == 1 ? p.lo_rows : 0)), fb);
              tma_load_2d(smem_u32(sst + NA * a_bytes + v * x_bytes), v == 1 ? &tmA1 : &tmA0, ent[0] + xo, s0, fb);
            }
            ++c;
          }
        }
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
    }
    if (lane == 0) {
      if (!ok) {
        atomicOr(p.err, 1);
        atomicExch(&abort_sh, 1);
      }
      for (int i = c - S < 0 ? 0 : c - S; i < c; ++i)
        if (!mbar_wait(full0 + 8 * (i & (S - 1)), (uint32_t)(i / S) & 1u)) atomicOr(p.err, 1);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    constexpr uint32_t fmt = MODE_ == MODE_TF32 ? 2u : 1u;
    constexpr uint32_t ID = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(NS >> 3) << 17) |
                            ((uint32_t)(128 >> 4) << 24);
    const uint64_t desc0 = sdesc_sb<SB>(smem_u32(smem));
    int c = 0, i = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x, ++i) {
      int eg, tg_;
      unit_coords(p, u, eg, tg_);
      const int ne = p.sched_ptr[eg + 1] - p.sched_ptr[eg];
      if (lane == 0) {
        const int buf = i & 1;
        const int use = i >> 1;
        if (!mbar_wait(acce0 + 8 * buf, ((uint32_t)use & 1u) ^ 1u)) ok = false;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * NS);
        uint32_t first = 0;
        const int nslots = NSUB == 1 ? ne : p.gslots[eg];
        for (int e = 0; e < nslots && ok; ++e) {  // one iteration per ring slot
          const int st = c & (S - 1);
          const uint32_t ph = (uint32_t)(c / S) & 1u;
          if (!mbar_wait(full0 + 8 * st, ph)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t dh = desc0 + (uint64_t)((st * stage_bytes) >> 4);  // H hi (A)
          const uint64_t dx = dh + (uint64_t)((NA * a_bytes) >> 4);         // X hi (B)
#pragma unroll
          for (int kk = 0; kk < SB / 32; ++kk) {
            const uint64_t ad = dh + (uint64_t)((32 * kk) >> 4);
            const uint64_t bd = dx + (uint64_t)((32 * kk) >> 4);
            const uint32_t acc = kk > 0 ? 1u : first;
            if constexpr (MODE_ == MODE_TF32) {
              mma_tf32(d, ad, bd, ID, acc);
            } else {
              mma_bf16(d, ad, bd, ID, acc);
              if constexpr (MODE_ == MODE_BF16X3) {
                mma_bf16(d, ad + (uint64_t)(a_bytes >> 4), bd, ID, 1u);  // lo(H) * hi(X)
                mma_bf16(d, ad, bd + (uint64_t)(x_bytes >> 4), ID, 1u);  // hi(H) * lo(X)
              }
            }
          }
          first = 1u;
          mma_commit(empty0 + 8 * st);
          ++c;
        }
        mma_commit(accf0 + 8 * buf);
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
    }
    if (lane == 0 && !ok) {
      atomicOr(p.err, 1);
      atomicExch(&abort_sh, 1);
    }
  } else {
    // ---------------- epilogue: warps 2..9; lane quarter q = element rows 32q..32q+31,
    // the two warps of a quarter take alternate 16-state chunks
    const float alpha = (float)p.coef[1 + 2 * p.step], beta = (float)p.coef[2 + 2 * p.step];
    const int q = warp & 3;
    const int h = (warp - 2) >> 2;
    const int r = 32 * q + lane;        // row of the stacked M = 128
    const int g = r / ACC, j = r % ACC;
    int i = 0;
    for (int u = blockIdx.x; u < nunits; u += gridDim.x, ++i) {
      const int buf = i & 1;
      const int use = i >> 1;
      int eg, tg;
      unit_coords(p, u, eg, tg);
      const int64_t s0 = (int64_t)tg * NS;
      bool ready = mbar_wait(accf0 + 8 * buf, (uint32_t)use & 1u);
      ready = __all_sync(0xffffffffu, ready);
      if (!ready) {
        if (lane == 0) atomicOr(p.err, 1);
        break;
      }
      tc_fence_after();
      const bool go = *(volatile int*)&abort_sh == 0;
      const int K = p.grp_elem[eg * G + g];
      const bool row_ok = go && K >= 0 && j < (K >= 0 ? p.nb[K] : 0);
      const int64_t col = (K >= 0 ? (int64_t)p.poff[K] : 0) + j;
      const uint32_t ta = tmem + (uint32_t)(buf * NS) + ((uint32_t)(32 * q) << 16);
      const int64_t ldp = p.ldp;
      const bool need_prev = row_ok && beta != 0.f;
      const bool write_ops = p.Hout != nullptr;
#pragma unroll 1
      for (int cc = 0; cc < NS / 32; ++cc) {
        const int c0 = 16 * (h + 2 * cc);
        const int64_t sb = s0 + c0;
        const int nz = (int)(p.Ns - sb < 16 ? p.Ns - sb : 16);  // states of this chunk inside N_s
        const int64_t base = sb * ldp + col;                      // dereferenced only for z < nz
        float pr[16];
        if (need_prev && nz == 16) {
#pragma unroll
          for (int z = 0; z < 16; ++z) pr[z] = p.Fprev[base + z * ldp];
        } else {
#pragma unroll
          for (int z = 0; z < 16; ++z) pr[z] = (need_prev && z < nz) ? p.Fprev[base + z * ldp] : 0.f;
        }
        float v[16];
        tmem_ld16(ta + (uint32_t)c0, v);
        if (row_ok) {
#pragma unroll
          for (int z = 0; z < 16; ++z) {
            if (z < nz) {
              const int64_t idx = base + z * ldp;
              const float y = alpha * v[z] - beta * pr[z];
              p.Fout[idx] = y;
              if constexpr (MODE_ != MODE_TF32) {
                if (write_ops) {  // no operand copies for a plain product (slice pairs)
                  const __nv_bfloat16 hb = __float2bfloat16_rn(y);
                  p.Hout[idx] = hb;
                  if constexpr (MODE_ == MODE_BF16X3) p.Lout[idx] = __float2bfloat16_rn(y - __bfloat162float(hb));
                }
              }
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce0 + 8 * buf);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

using FilterKernel = void (*)(const CUtensorMap, const CUtensorMap, const CUtensorMap, const Params);

// Unit shapes {G elements, T tiles of 128 states, ACC accumulator columns per
// element, layout} that have kernels; layout 0 = states along the MMA's M
// (k_filter_step_tc), 1 = element rows along M, 256 states along N
// (k_filter_step_tn, G = 128/ACC, T = 2), 2 = layout 1 with 64-byte ring
// slots. The autotuner picks among those matching ACC.
constexpr int NSHAPES = 13;
constexpr int SHAPES[NSHAPES][4] = {{2, 2, 64, 0}, {1, 2, 64, 0}, {2, 1, 64, 0}, {4, 2, 32, 0}, {2, 2, 32, 0},
                                    {2, 1, 128, 0}, {1, 2, 128, 0}, {2, 2, 64, 1}, {4, 2, 32, 1},
                                    {1, 2, 128, 1}, {2, 2, 64, 2}, {4, 2, 32, 2}, {1, 2, 128, 2}};

template <int MODE_>
FilterKernel pick_shape(int G, int T, int ACC, int layout) {
  if (layout == 1) {
    if (ACC == 64 && G == 2 && T == 2) return k_filter_step_tn<MODE_, 64>;
    if (ACC == 32 && G == 4 && T == 2) return k_filter_step_tn<MODE_, 32>;
    if (ACC == 128 && G == 1 && T == 2) return k_filter_step_tn<MODE_, 128>;
    return nullptr;
  }
  if (layout == 2) {
    if (ACC == 64 && G == 2 && T == 2) return k_filter_step_tn<MODE_, 64, 64>;
    if (ACC == 32 && G == 4 && T == 2) return k_filter_step_tn<MODE_, 32, 64>;
    if (ACC == 128 && G == 1 && T == 2) return k_filter_step_tn<MODE_, 128, 64>;
    return nullptr;
  }
  if (layout != 0) return nullptr;
  if (G == 2 && T == 2 && ACC == 64) return k_filter_step_tc<MODE_, 2, 2, 64>;
  if (G == 1 && T == 2 && ACC == 64) return k_filter_step_tc<MODE_, 1, 2, 64>;
  if (G == 2 && T == 1 && ACC == 64) return k_filter_step_tc<MODE_, 2, 1, 64>;
  if (G == 4 && T == 2 && ACC == 32) return k_filter_step_tc<MODE_, 4, 2, 32>;
  if (G == 2 && T == 2 && ACC == 32) return k_filter_step_tc<MODE_, 2, 2, 32>;
  if (G == 2 && T == 1 && ACC == 128) return k_filter_step_tc<MODE_, 2, 1, 128>;
  if (G == 1 && T == 2 && ACC == 128) return k_filter_step_tc<MODE_, 1, 2, 128>;
  return nullptr;
}

}  // namespace

// One translation unit per precision instantiates the kernels (compiled in parallel).
FilterKernel pick_kernel_tf32(int G, int T, int ACC, int layout);
FilterKernel pick_kernel_bf16(int G, int T, int ACC, int layout);
FilterKernel pick_kernel_bf16x3(int G, int T, int ACC, int layout);

}  // namespace dg
