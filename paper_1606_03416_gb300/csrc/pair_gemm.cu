// Slice-pair products of the FP64-from-BF16-slices GEMM (the Ozaki scheme of
// sliced.cu; Alg. 1 steps 3-5) on pairs of SMs: tcgen05 with cta_group::2.
//
// Every slice pair (i, j) of a K chunk is a plain BF16 GEMM with FP32
// accumulation, P_ij = A_i B_j^T, written as an FP32 slab. One CTA pair (a
// cluster of two) computes a 256 x 256 tile of one pair at a time: each CTA
// stages its own 128 rows of A_i and its own 128 rows of B_j (32 KB per
// 64-wide K slice), the first CTA of the pair issues 256 x 256 x 16 MMAs that
// read both CTAs' halves, and each CTA's tensor memory holds its 128 rows of
// the tile. Per SM that is 8 KB of operands per 128-clock MMA, half of what a
// single-SM 128 x 256 tile reads, which leaves shared-memory bandwidth for the
// TMA refills. The kernel is persistent over (pair, tile) units, the tiles of
// one pair back to back so that the units in flight read the same two slices
// from L2, and the tensor maps of all slices sit in device memory, so one
// launch covers every pair of a chunk.
//
// Roles per CTA (320 threads): warp 0 lane 0 loads its halves with TMA into a
// 6-slot ring and signals the first CTA's "full" barrier (its expect-tx counts
// both CTAs' bytes); warp 1 lane 0 of the first CTA issues the MMAs, frees
// ring slots in both CTAs and announces finished accumulators to both
// (multicast commits); warps 2-9 drain their CTA's accumulator
// (double-buffered, 2 x 256 columns) and report to the first CTA's "empty"
// accumulator barrier. Every wait is bounded; on expiry the CTA records an
// error word and both CTAs still meet at the final cluster barrier.
#include <algorithm>
#include <cstring>
#include <vector>

#include "tc_kernel.cuh"

namespace dg {
namespace {

constexpr int PG_THREADS = 320;
constexpr int PG_HALF = 128 * SLICE_BYTES;  // 128 rows x 64 BF16 of one operand
constexpr int PG_STAGE = 2 * PG_HALF;       // A half + B half per CTA
constexpr int PG_STAGES = 6;

struct PairJob {
  const CUtensorMap* maps;  // device, 64-byte aligned: [s] maps of A_i, then [s] maps of B_j
  const int32_t* pair_i;    // [npairs]
  const int32_t* pair_j;
  int npairs, s;
  int64_t M;        // rows of A (the slab's rows)
  int64_t pn;       // columns of the slab (rows n0 .. n0 + pn - 1 of B)
  int n0, k0, nk;   // first B row, first K column, 64-wide K slices of the chunk
  int nmt, nnt;     // 256-row tiles along M and along the panel
  int lower;        // A is lower triangular: a row tile stops at the chunk's last K slice it reaches
  const int2* tiles;  // null: every (row tile, column tile); else the ntl tiles to compute
  int ntl;
  float* Pw;        // slab of pair p at Pw + p * M * pn, row-major M x pn
  int* err;
};

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t map_to_rank(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

// TMA load into this CTA's shared memory, completing on a barrier that may sit
// in the peer CTA of the pair.
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void mma_bf16_pair(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}

// Arrive on the barrier at this offset in both CTAs of the pair once the MMAs
// issued so far have completed.
__device__ __forceinline__ void commit_pair(uint32_t bar) {
  const uint16_t mask = 3;
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
      "h"(mask)
      : "memory");
}

// Pair and tile of work unit u: pairs outermost (in the table's order, one
// slice of A with the slices of B in turn), the tiles of one pair back to back
// (row tiles fastest), so the units in flight share one A slice and one or two
// B slices, which stay in L2.
__device__ __forceinline__ void unit_of(const PairJob& J, int64_t u, int& p, int& mt, int& nt) {
  if (J.tiles) {
    p = (int)(u / J.ntl);
    const int2 t = J.tiles[u - (int64_t)p * J.ntl];
    mt = t.x;
    nt = t.y;
    return;
  }
  const int64_t ntiles = (int64_t)J.nmt * J.nnt;
  p = (int)(u / ntiles);
  const int64_t tile = u - (int64_t)p * ntiles;
  mt = (int)(tile % J.nmt);
  nt = (int)(tile / J.nmt);
}

// K slices of the chunk that row tile mt needs: all of them, or for a lower
// triangular A those up to its last row (at least one, so that the tile's
// accumulator is written).
__device__ __forceinline__ int slices_of_tile(const PairJob& J, int mt) {
  if (!J.lower) return J.nk;
  const int need = (mt * 256 + 256 - J.k0 + 63) / 64;
  return max(1, min(J.nk, need));
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(PG_THREADS, 1) k_slice_pairs_2sm(const PairJob J) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + PG_STAGES * PG_STAGE);
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;

  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;
  const int64_t nunits = (J.tiles ? (int64_t)J.ntl : (int64_t)J.nmt * J.nnt) * J.npairs;
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * PG_STAGES;
  const uint32_t accf0 = empty0 + 8 * PG_STAGES, acce0 = accf0 + 16;

  if (threadIdx.x == 0) {
    for (int s = 0; s < PG_STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, 2 * EPI_WARPS);  // the epilogue warps of both CTAs
    }
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {  // both CTAs allocate the same columns together
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // barriers of both CTAs initialised before any remote use
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0) {
    // ---------------- producer: this CTA's halves, completing on the first CTA's barrier
    if (lane == 0) {
      const uint32_t full_l = map_to_rank(full0, 0);
      int c = 0;
      bool ok = true;
      for (int64_t u = cid; u < nunits && ok; u += ncl) {
        int p, mt, nt;
        unit_of(J, u, p, mt, nt);
        const CUtensorMap* am = J.maps + J.pair_i[p];
        const CUtensorMap* bm = J.maps + J.s + J.pair_j[p];
        const int ya = mt * 256 + (int)rank * 128;
        const int yb = J.n0 + nt * 256 + (int)rank * 128;
        const int nk = slices_of_tile(J, mt);
        for (int ks = 0; ks < nk; ++ks) {
          const int st = c % PG_STAGES;
          const uint32_t ph = (uint32_t)(c / PG_STAGES) & 1u;
          if (!mbar_wait(empty0 + 8 * st, ph ^ 1u)) {
            ok = false;
            break;
          }
          if (leader) mbar_expect_tx(full0 + 8 * st, (uint32_t)(2 * PG_STAGE));
          const uint32_t dst = smem_u32(smem + st * PG_STAGE);
          const int x = J.k0 + ks * (SLICE_BYTES / 2);
          tma_load_2d_pair(dst, am, x, ya, full_l + 8 * st);
          tma_load_2d_pair(dst + PG_HALF, bm, x, yb, full_l + 8 * st);
          ++c;
        }
      }
      if (!ok) {
        atomicOr(J.err, 1);
        atomicExch(&abort_sh, 1);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: the first CTA of the pair only
    if (leader && lane == 0) {
      constexpr uint32_t ID = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(256 >> 3) << 17) |
                              ((uint32_t)(256 >> 4) << 24);
      const uint64_t desc0 = sdesc(smem_u32(smem));
      int c = 0, i = 0;
      bool ok = true;
      for (int64_t u = cid; u < nunits && ok; u += ncl, ++i) {
        const int buf = i & 1;
        const uint32_t use = (uint32_t)(i >> 1);
        if (!mbar_wait(acce0 + 8 * buf, (use & 1u) ^ 1u)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * 256);
        int p_, mt, nt_;
        unit_of(J, u, p_, mt, nt_);
        const int nk = slices_of_tile(J, mt);
        for (int ks = 0; ks < nk && ok; ++ks) {
          const int st = c % PG_STAGES;
          const uint32_t ph = (uint32_t)(c / PG_STAGES) & 1u;
          if (!mbar_wait(full0 + 8 * st, ph)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t da = desc0 + (uint64_t)((st * PG_STAGE) >> 4);
          const uint64_t db = da + (uint64_t)(PG_HALF >> 4);
#pragma unroll
          for (int kk = 0; kk < SLICE_BYTES / 32; ++kk)
            mma_bf16_pair(d, da + (uint64_t)((32 * kk) >> 4), db + (uint64_t)((32 * kk) >> 4), ID,
                          (ks > 0 || kk > 0) ? 1u : 0u);
          commit_pair(empty0 + 8 * st);
          ++c;
        }
        if (ok) commit_pair(accf0 + 8 * buf);
      }
      if (!ok) {
        atomicOr(J.err, 1);
        atomicExch(&abort_sh, 1);
      }
    }
  } else {
    // ---------------- epilogue: warps 2..9, lane quarter q = tile rows 32q..32q+31 of this
    // CTA's half; the two warps of a quarter take alternate 16-column chunks
    const int q = warp & 3;
    const int h = (warp - 2) >> 2;
    const uint32_t acce_l = map_to_rank(acce0, 0);
    int i = 0;
    for (int64_t u = cid; u < nunits; u += ncl, ++i) {
      const int buf = i & 1;
      const uint32_t use = (uint32_t)(i >> 1);
      bool ready = mbar_wait(accf0 + 8 * buf, use & 1u);
      ready = __all_sync(0xffffffffu, ready);
      if (!ready) {
        if (lane == 0) atomicOr(J.err, 1);
        break;
      }
      tc_fence_after();
      int p, mt, nt;
      unit_of(J, u, p, mt, nt);
      const int64_t r = (int64_t)mt * 256 + rank * 128 + 32 * q + lane;
      const bool row_ok = r < J.M && *(volatile int*)&abort_sh == 0;
      float* out = J.Pw + (size_t)p * (size_t)(J.M * J.pn) + (size_t)(r < J.M ? r : 0) * (size_t)J.pn;
      const uint32_t ta = tmem + (uint32_t)(buf * 256) + ((uint32_t)(32 * q) << 16);
#pragma unroll 1
      for (int cc = 0; cc < 8; ++cc) {
        const int c0 = 16 * (h + 2 * cc);
        float v[16];
        tmem_ld16(ta + (uint32_t)c0, v);
        const int64_t col = (int64_t)nt * 256 + c0;
        if (row_ok) {
          if (col + 16 <= J.pn && (J.pn & 3) == 0) {  // rows start on 16 bytes only when pn % 4 == 0
            float4* o = reinterpret_cast<float4*>(out + col);
#pragma unroll
            for (int z = 0; z < 4; ++z) o[z] = make_float4(v[4 * z], v[4 * z + 1], v[4 * z + 2], v[4 * z + 3]);
          } else {
#pragma unroll
            for (int z = 0; z < 16; ++z)
              if (col + z < J.pn) out[col + z] = v[z];
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) arrive_remote(acce_l + 8 * buf);
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // neither CTA leaves while the pair's MMAs or arrivals may still touch it
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &qr) ==
            cudaSuccess &&
        qr == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }
  return fn;
}

// BF16 matrix rows x inner (row stride `stride` elements), boxes of 64 x 128, 128-byte swizzle.
dgchefsi_status slice_map(CUtensorMap* map, const __nv_bfloat16* base, uint64_t inner, uint64_t rows,
                          uint64_t stride) {
  auto enc = tensor_map_encoder();
  if (!enc) return set_error(DGCHEFSI_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {stride * 2};
  cuuint32_t box[2] = {64, 128};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims, strides, box,
                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(DGCHEFSI_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return DGCHEFSI_OK;
}

}  // namespace

dgchefsi_status pair_products_2sm(dgchefsi_ctx* ctx, const __nv_bfloat16* Qa, int64_t lqa, int64_t sa, int64_t M,
                                  const __nv_bfloat16* Qb, int64_t lqb, int64_t sb, int64_t Nc, int64_t K, int64_t k0,
                                  int64_t kc, int64_t n0, int64_t pn, int s, float* Pw, bool a_lower, int64_t tri) {
  if (M > 2147483647LL - 256 || Nc > 2147483647LL - 256 || K > 2147483647LL)
    return set_error(DGCHEFSI_ERR_UNSUPPORTED, "slice-pair product too large for 32-bit TMA coordinates");
  cudaStream_t st = ctx->stream;
  const int npairs = s * (s + 1) / 2;
  const int nmt = (int)((M + 255) / 256), nnt = (int)((pn + 255) / 256);
  // tri > 0: only entries (r, n0 + c) with n0 + c <= r mod tri are wanted (the
  // lower triangle of a symmetric product, or of each of several stacked
  // ones); tiles entirely above it are left out.
  std::vector<int2> tl;
  if (tri > 0) {
    for (int nt = 0; nt < nnt; ++nt)
      for (int mt = 0; mt < nmt; ++mt) {
        const int64_t r0 = (int64_t)mt * 256, r1 = std::min<int64_t>(r0 + 256, M) - 1;
        const int64_t c0 = n0 + (int64_t)nt * 256;
        const bool wrap = r0 / tri != r1 / tri;
        if (wrap || c0 <= r1 % tri) tl.push_back(make_int2(mt, nt));
      }
    if (tl.empty()) return DGCHEFSI_OK;
  }
  // tables: 2s tensor maps (64-byte aligned), then the pair lists, then the tile list
  const size_t maps_bytes = sizeof(CUtensorMap) * (size_t)(2 * s);
  const size_t pairs_bytes = sizeof(int32_t) * (size_t)(2 * npairs);
  const size_t tiles_at = (maps_bytes + pairs_bytes + 15) / 16 * 16;
  std::vector<uint8_t> host(tiles_at + sizeof(int2) * tl.size());
  CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(host.data());
  for (int i = 0; i < s; ++i) {
    DG_TRY(slice_map(&maps[i], Qa + (size_t)i * sa, (uint64_t)K, (uint64_t)M, (uint64_t)lqa));
    DG_TRY(slice_map(&maps[s + i], Qb + (size_t)i * sb, (uint64_t)K, (uint64_t)Nc, (uint64_t)lqb));
  }
  int32_t* pi = reinterpret_cast<int32_t*>(host.data() + maps_bytes);
  int32_t* pj = pi + npairs;
  int n = 0;
  for (int i = 0; i < s; ++i)
    for (int j = 0; i + j < s; ++j, ++n) {
      pi[n] = i;
      pj[n] = j;
    }
  if (!tl.empty()) std::memcpy(host.data() + tiles_at, tl.data(), sizeof(int2) * tl.size());
  // the context's table buffer (may be regrown here: it holds no state across launches)
  DevBuf& tables = ctx->ws_pairs;
  DG_TRY(ensure(ctx, tables, host.size(), "slice-pair tensor maps"));
  uint8_t* tab = static_cast<uint8_t*>(tables.p);
  DG_CUDA(cudaMemcpyAsync(tab, host.data(), host.size(), cudaMemcpyHostToDevice, st));
  // the pageable copy above has been staged before it returns, so `host` may go
  PairJob J{};
  J.maps = reinterpret_cast<const CUtensorMap*>(tab);
  J.pair_i = reinterpret_cast<const int32_t*>(tab + maps_bytes);
  J.pair_j = J.pair_i + npairs;
  J.npairs = npairs;
  J.s = s;
  J.M = M;
  J.pn = pn;
  J.n0 = (int)n0;
  J.k0 = (int)k0;
  J.nk = (int)((kc + 63) / 64);
  J.nmt = nmt;
  J.nnt = nnt;
  J.lower = a_lower ? 1 : 0;
  J.tiles = tl.empty() ? nullptr : reinterpret_cast<const int2*>(tab + tiles_at);
  J.ntl = (int)tl.size();
  J.Pw = Pw;
  if (!ctx->ws_pairs_err.p) return set_error(DGCHEFSI_ERR_CUDA, "slice-pair products not begun");
  J.err = static_cast<int*>(ctx->ws_pairs_err.p);
  int nsm = 0;
  DG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
  const int64_t units = (J.tiles ? (int64_t)J.ntl : (int64_t)J.nmt * J.nnt) * npairs;
  const int clusters = (int)std::min<int64_t>(units, std::max(nsm / 2, 1));
  const int smem = PG_STAGES * PG_STAGE + (2 * PG_STAGES + 4) * 8 + 1024;
  DG_CUDA(cudaFuncSetAttribute(k_slice_pairs_2sm, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  k_slice_pairs_2sm<<<2 * clusters, PG_THREADS, smem, st>>>(J);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return DGCHEFSI_OK;
}

dgchefsi_status pair_products_begin(dgchefsi_ctx* ctx) {
  DG_TRY(ensure(ctx, ctx->ws_pairs_err, 256, "slice-pair error word"));
  DG_CUDA(cudaMemsetAsync(ctx->ws_pairs_err.p, 0, sizeof(int), ctx->stream));
  return DGCHEFSI_OK;
}

dgchefsi_status pair_products_status(dgchefsi_ctx* ctx) {
  if (!ctx->ws_pairs_err.p) return DGCHEFSI_OK;
  int err = 0;
  DG_CUDA(cudaMemcpyAsync(&err, ctx->ws_pairs_err.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  DG_CUDA(cudaStreamSynchronize(ctx->stream));
  if (err) return set_error(DGCHEFSI_ERR_TIMEOUT, "a slice-pair CTA gave up waiting on a pipeline barrier");
  return DGCHEFSI_OK;
}

}  // namespace dg
