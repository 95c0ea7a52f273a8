// Latency mode of the tensor-core decoder for launches with few tiles (the
// shrinking tail of a march): each tile is spread over a cluster of WC CTAs,
// CTA r computing output columns [r N/WC, (r+1) N/WC) of every layer for all
// of the tile's rows.  The per-layer tensor-core work of one SM drops by WC;
// the CTAs exchange the next layer's operand through an L2-resident staging
// image (each stores its column slice there with one bulk copy, then bulk-
// loads the others').  Every output
// column is accumulated over K in the same order and through the same
// epilogue arithmetic as in mlp_tc_kernel, and the head adds the same 32-column
// chunk sums in the same order, so a row's f is the same in either kernel.
//
// Roles per CTA (10 warps): warp 0 streams this CTA's weight rows through a
// TMA ring, warp 1 issues the MMAs (N = 128, or 64 for the 256-wide layer),
// warps 2..9 are the epilogue (TMEM lane quadrant warp & 3, one half of the
// CTA's columns each); lane 0 of warp 2 also loads the peers' operand
// slices.  Waits are bounded like the main kernel's.
#include <cmath>
#include <cstring>

#include "step.cuh"
#include "tc_common.cuh"

namespace dist {

namespace {

constexpr int WC = 4;                          // CTAs per tile
constexpr int WT_MAX = 37;                     // clusters per launch: 148 SMs / WC
constexpr int W_BN = 128;                      // weight rows per stage (= 512 / WC)
constexpr int W_STAGE = 2 * W_BN * BK * 2;     // 32 KB: two 64-column chunks, one TMA copy
constexpr int W_NST = 3;
constexpr int W_EPI = 8;                       // epilogue warps: two per TMEM lane quadrant
constexpr int W_THREADS = (2 + W_EPI) * 32;
constexpr int W_BAR_BYTES = 256;
constexpr int W_SMEM = 1024 + ACT_BYTES + W_NST * W_STAGE + W_BAR_BYTES;
static_assert(W_SMEM <= 232448, "wide kernel shared memory");
constexpr int QPT_XW = 64;                     // FP32-class queries per tile

struct WideArgs {
  const TCConst* K;
  const float* bfold0;
  const float* bfold4;
  RowSrc src[3];       // lists as in mlp_tc_kernel: 16-bit, FP32-class, FP16 stage
  float* fout[3];
  int* err;
  float inv_scale[NUM_GEMM];
  int fuse_step;
  StepFuse step;
  uint8_t* stage_g;    // [clusters][2][ACT_BYTES] operand images
  float* head_g;       // [clusters][BM][16] head chunk sums
  int nsm;             // CTAs of the mlp_tc_kernel launch of the same step
};

__device__ __forceinline__ uint32_t wide_idesc(bool f16, int n) {
  return (1u << 4) | ((f16 ? 0u : 1u) << 7) | ((f16 ? 0u : 1u) << 10) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

// Two [128 x 64] chunks (z, z + 1) of a 3D weight view, rows from y.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int y,
                                            int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(0), "r"(y), "r"(z)
      : "memory");
}

__device__ __forceinline__ void prefetch_l1(const float* q) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(q));
}

// Shared -> global bulk copy (16-byte aligned, size a multiple of 16),
// waited for to completion.
__device__ __forceinline__ void bulk_store(uint8_t* dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(
                   reinterpret_cast<uint64_t>(dst)),
               "r"(src), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

template <bool F16>
__global__ void __launch_bounds__(W_THREADS, 1)
mlp_tc_wide_kernel(const __grid_constant__ TCMaps wmaps, const __grid_constant__ TCMaps wxmaps,
                   const __grid_constant__ TCMaps wmaps16, const WideArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint8_t* act = smem;
  uint8_t* wst = smem + ACT_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(wst + W_NST * W_STAGE);
  uint64_t* full = bars;                        // [W_NST]
  uint64_t* empty = bars + W_NST;               // [W_NST]
  uint64_t* acc_full = bars + 2 * W_NST;        // MMA -> epilogue
  uint64_t* act_full = bars + 2 * W_NST + 1;    // operand complete -> MMA
  // [2] every CTA's slice of exchange x is in the staging image: barrier
  // x & 1, so that a CTA already one exchange ahead cannot complete a phase
  // a slower peer's arrival still belongs to
  uint64_t* slice_ready = bars + 2 * W_NST + 2;
  uint64_t* a_loaded = bars + 2 * W_NST + 4;    // peers' slices copied in
  uint64_t* head_ready = bars + 2 * W_NST + 5;  // (rank 0) every CTA's head chunk sums
  uint64_t* drain = bars + 2 * W_NST + 6;       // every issued MMA complete
  // the other epilogue warps' parts of an operand slice are written -> warp 2
  // (an mbarrier, so that warp 2's wait is bounded like every other)
  uint64_t* epi_done = bars + 2 * W_NST + 7;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * W_NST + 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  static_assert((2 * W_NST + 8) * 8 + 8 <= W_BAR_BYTES, "barrier block");

  // Launched behind this step's mlp_tc_kernel (programmatic dependent
  // launch), possibly to decode some of the step's tiles beside it.  This
  // step's inputs are acquired through the sequence number that grid
  // releases before it lets this one launch (so the bounded wait below finds
  // it at once; it never waits for the other grid to make progress).  Each
  // CTA that decodes, and CTA 0, waits for that grid before it exits, so the
  // next step, launched behind this grid, starts only once both are done.
  grid_dep_launch();

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int rank = (int)cluster_rank();
  const int cid = (int)(blockIdx.x / WC);
  const int ncl = (int)(gridDim.x / WC);
  int fresh = 1;
  if (threadIdx.x == 0) {
    const unsigned long long t0 = globaltimer();
    while (seq_acquire(a.step.seq_flag) != a.step.seq) {
      if (globaltimer() - t0 > kTimeoutNs) {
        fresh = 0;
        atomicOr(a.err, 4);
        break;
      }
    }
  }
  fresh = __syncthreads_or(fresh && threadIdx.x == 0);
  const int n0 = fresh ? rowsrc_count(a.src[0]) : 0;
  const int n1 = fresh ? rowsrc_count(a.src[1]) : 0;
  const int n2 = fresh ? rowsrc_count(a.src[2]) : 0;
  const int t1 = (n1 + QPT_XW - 1) / QPT_XW;         // FP32-class tiles: [0, t1)
  const int t2 = t1 + (n2 + BM - 1) / BM;            // FP16-stage tiles: [t1, t2)
  const int n_tiles = t2 + (n0 + BM - 1) / BM;
  // this kernel's tiles [0, nw): the same decision as mlp_tc_kernel's from
  // the same counts (wide_share); uniform over a cluster
  const int nw = wide_share(n_tiles, t1, ncl, a.nsm);
  if (cid >= nw) {
    if (blockIdx.x == 0) grid_dep_wait();
    return;
  }
  if (nw == n_tiles && a.fuse_step && a.step.queries && cid == 0 && rank == 0 &&
      threadIdx.x == 0) {
    atomicAdd(a.step.queries + 0, (unsigned long long)(n0 + n2));
    atomicAdd(a.step.queries + 1, (unsigned long long)n1);
  }
  // row list of tile t and its first row in the list
  auto tile_list = [&](int t) { return t < t1 ? 1 : (t < t2 ? 2 : 0); };
  auto tile_row0 = [&](int t) { return t < t1 ? t * QPT_XW : (t - (t < t2 ? t1 : t2)) * BM; };
  if (threadIdx.x == 0) {
    for (int s = 0; s < W_NST; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(act_full, 1);
    mbar_init(slice_ready + 0, WC);   // one arrival per CTA (its loader)
    mbar_init(slice_ready + 1, WC);
    mbar_init(a_loaded, 1);
    mbar_init(head_ready, W_EPI * WC);
    mbar_init(drain, 1);
    mbar_init(epi_done, W_EPI - 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, 128);
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();   // every CTA's barriers exist before remote arrivals
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------ weight rows of this CTA
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_parity[W_NST];
      bool issued[W_NST];
      for (int s = 0; s < W_NST; ++s) issued[s] = false;
      bool ok = true;
      for (int tile = cid; ok && tile < nw; tile += ncl) {
        const bool xt = tile < t1;
        const bool mid = tile_list(tile) == 2;
        for (int g = 0; ok && g < NUM_GEMM; ++g) {
          const CUtensorMap* map = xt ? &wxmaps.m[g] : (mid ? &wmaps16.m[g] : &wmaps.m[g]);
          const int nkc = gemm_k(g) / BK;
          const int row0 = (gemm_n(g) / WC) * rank;
          // stages of two K chunks (nkc is even, so a pair never straddles
          // the FP32-class tiles' W_lo / W_hi passes)
          for (int kc = 0; kc < (xt ? 2 : 1) * nkc; kc += 2) {
            if (!mbar_wait(empty + stage, phase ^ 1u, abort_flag)) { ok = false; break; }
            mbar_expect_tx(full + stage, W_STAGE);
            const int xk = !xt ? kc : (kc < nkc ? nkc + kc : kc - nkc);
            tma_load_3d(wst + stage * W_STAGE, map, full + stage, row0, xk);
            issued[stage] = true;
            issued_parity[stage] = phase;
            if (++stage == W_NST) { stage = 0; phase ^= 1u; }
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(a.err, 1);
      }
      for (int s = 0; s < W_NST; ++s) {
        if (!issued[s]) continue;
        const unsigned long long t0 = globaltimer();
        while (!mbar_try_wait(full + s, issued_parity[s]) && globaltimer() - t0 < kTimeoutNs) {
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------- MMAs
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, act_phase = 0;
      bool ok = true;
      for (int tile = cid; ok && tile < nw; tile += ncl) {
        const bool xt = tile < t1;
        const bool f16 = xt || F16 || tile_list(tile) == 2;
        for (int g = 0; ok && g < NUM_GEMM; ++g) {
          const int nkc = gemm_k(g) / BK;
          const uint32_t idesc = wide_idesc(f16, gemm_n(g) / WC);
          if (!mbar_wait(act_full, act_phase, abort_flag)) { ok = false; break; }
          act_phase ^= 1u;
          tc_fence_after();
          for (int kc = 0; kc < (xt ? 2 : 1) * nkc; kc += 2) {
            if (!mbar_wait(full + stage, phase, abort_flag)) { ok = false; break; }
            tc_fence_after();
            const uint32_t a_base = smem_u32(act + (kc < nkc ? kc : kc - nkc) * CHUNK_BYTES);
            const uint32_t b_base = smem_u32(wst + stage * W_STAGE);
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
              for (int k = 0; k < BK / 16; ++k)
                mma_bf16(tmem, sw128_desc(a_base + c * CHUNK_BYTES + 32 * k),
                         sw128_desc(b_base + c * (W_BN * BK * 2) + 32 * k), idesc,
                         (kc | c | k) != 0);
            mma_commit(empty + stage);
            if (++stage == W_NST) { stage = 0; phase ^= 1u; }
          }
          if (ok) mma_commit(acc_full);
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(a.err, 2);
      }
      mma_commit(drain);      // every issued MMA completes before TMEM is released
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(drain, 0) && globaltimer() - t0 < kTimeoutNs) {
      }
    }
  } else {
    // ------------------------------------------------------------- epilogue
    const int quad = warp & 3;
    const int half = (warp - 2) >> 2;            // 0: first half of each column range
    const int row = quad * 32 + lane;            // 16-bit tiles
    const int part = lane >> 4;                  // FP32-class tiles
    const int jr = quad * 16 + (lane & 15);
    const int rhi = quad * 32 + (lane & 15);
    const int rlo = rhi + 16;
    const uint32_t t_row = tmem + ((uint32_t)(quad * 32) << 16);
    const TCConst* K = a.K;
    uint32_t acc_phase = 0, load_phase = 0, head_phase = 0, epi_phase = 0;
    int xs = 0;                                   // exchanges so far
    bool ok = true;
    float vmax = 0.f;
    bool xt = false, valid = false, f16 = F16;
    int list = 0, j = 0, shape = 0;
    float3 p = make_float3(0.f, 0.f, 0.f);
    uint8_t* stage_base = nullptr;

    // operand words at column c (8-aligned) of this thread's row(s)
    auto put4 = [&](uint32_t off, uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3) {
      st_shared_v4(smem_u32(act) + off, w0, w1, w2, w3);
    };
    auto put = [&](int c, const uint32_t (&h)[16]) {
      if (!xt) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int col = c + 8 * q;
          const uint32_t off = (uint32_t)((col >> 6) * CHUNK_BYTES) + swz(row, (col & 63) >> 3);
          put4(off, h[4 * q], h[4 * q + 1], h[4 * q + 2], h[4 * q + 3]);
        }
      } else {
        const int cc = c + 16 * part;
        const uint32_t ch = (uint32_t)((cc >> 6) * CHUNK_BYTES);
        const uint32_t u = (uint32_t)((cc & 63) >> 3);
        put4(ch + swz(rhi, u), h[0], h[1], h[2], h[3]);
        put4(ch + swz(rhi, u + 1), h[4], h[5], h[6], h[7]);
        put4(ch + swz(rlo, u), h[8], h[9], h[10], h[11]);
        put4(ch + swz(rlo, u + 1), h[12], h[13], h[14], h[15]);
      }
    };
    auto split_pack = [&](float (&v)[16], uint32_t (&h)[16]) {
      uint32_t hi[8], lo[8];
      relu_split16(v, hi, lo, vmax);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        h[i] = hi[i];
        h[8 + i] = lo[i];
      }
    };
    // layer 0 (CUDA cores), 32 columns from c
    auto layer0 = [&](int c, uint32_t (&h)[16]) {
      const float* bf0 = a.bfold0 + (size_t)shape * 512;
      if (!xt) {
        float v[32];
        layer0_32(K, bf0, c, p, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) h[i] = pack16r(f16, v[2 * i], v[2 * i + 1]);
      } else {
        float v[16];
        layer0_16(K, bf0, c + 16 * part, p, v);
        split_pack(v, h);
      }
    };
    // GEMM layer g, 32 accumulator columns at TMEM column tc (output column c)
    auto hold = [&](int g, const float* bf4, int tc, int c, uint32_t (&h)[16]) {
      uint32_t r[32];
      tmem_ld32(t_row + (uint32_t)tc, r);
      const bool point = g == 2 && c == 224;
      if (!xt) {
        const float* bias = g == 3 ? bf4 : K->bias[g];
#pragma unroll
        for (int i = 0; i < 32; i += 4) {
          const float4 b = ldg4(bias + c + i);
          h[i / 2] = pack16r(f16, fmaxf(__uint_as_float(r[i]) + b.x, 0.f),
                                 fmaxf(__uint_as_float(r[i + 1]) + b.y, 0.f));
          h[i / 2 + 1] = pack16r(f16, fmaxf(__uint_as_float(r[i + 2]) + b.z, 0.f),
                                     fmaxf(__uint_as_float(r[i + 3]) + b.w, 0.f));
        }
        if (point) {
          const float b28 = __ldg(K->bias[g] + 252);
          h[14] = pack16r(f16, fmaxf(__uint_as_float(r[28]) + b28, 0.f), p.x);
          h[15] = pack16r(f16, p.y, p.z);
        }
      } else {
        float m[16], v[16];
        pair_sum16(r, part, m);
        affine16(K, g, bf4, c + 16 * part, p, a.inv_scale[g], m, v, false);
        const float v12 = fmaxf(v[12], 0.f);
        split_pack(v, h);
        if (point && part == 1) {
          split_pair(v12, p.x, h[6], h[14]);
          split_pair(p.y, p.z, h[7], h[15]);
        }
      }
    };
    // this CTA's slice of the next operand is in place: make it visible to
    // the tensor core; then (loader: lane 0 of warp 2) store it to the
    // staging image with one bulk copy, tell the peers, and bring in theirs
    auto exchange = [&](int width) -> bool {
      uint64_t* ready = slice_ready + (xs & 1);
      const uint32_t slice = (uint32_t)(width / WC) * 2u * BM;   // bytes per CTA slice
      fence_async_shared();
      bool good = true;
      __syncwarp();
      if (warp != 2) {
        if (lane == 0) mbar_arrive(epi_done);
      } else {
        // every epilogue warp's part of the slice is in act
        good = mbar_wait(epi_done, epi_phase, abort_flag);
        epi_phase ^= 1u;
        if (good && lane == 0) {
          bulk_store(stage_base + (size_t)slice * rank, smem_u32(act) + slice * rank, slice);
          // the store is complete before the peers hear of it
          asm volatile("fence.proxy.async.global;" ::: "memory");
          for (int d = 0; d < WC; ++d) mbar_arrive_remote(map_rank(smem_u32(ready), (uint32_t)d));
          good = mbar_wait_cl(ready, (uint32_t)(xs >> 1) & 1u, abort_flag);
          if (good) {
            asm volatile("fence.proxy.async.global;" ::: "memory");
            mbar_expect_tx(a_loaded, slice * (WC - 1));
            for (int d = 0; d < WC; ++d) {
              if (d == rank) continue;
              asm volatile(
                  "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], "
                  "%2, [%3];" ::"r"(smem_u32(act) + slice * d),
                  "l"(reinterpret_cast<uint64_t>(stage_base + (size_t)slice * d)), "r"(slice),
                  "r"(smem_u32(a_loaded))
                  : "memory");
            }
            good = mbar_wait(a_loaded, load_phase, abort_flag);
            load_phase ^= 1u;
            if (good) mbar_arrive(act_full);
          }
        }
        good = __shfl_sync(0xffffffffu, good ? 1 : 0, 0) != 0;
      }
      ++xs;
      stage_base = a.stage_g + ((size_t)cid * 2 + (xs & 1)) * ACT_BYTES;
      return good;
    };
    auto wait_acc = [&]() -> bool {
      if (!mbar_wait(acc_full, acc_phase, abort_flag)) return false;
      acc_phase ^= 1u;
      tc_fence_after();
      return true;
    };

    stage_base = a.stage_g + ((size_t)cid * 2 + (xs & 1)) * ACT_BYTES;
    for (int tile = cid; ok && tile < nw; tile += ncl) {
      list = tile_list(tile);
      xt = list == 1;
      f16 = F16 || list == 2;
      j = tile_row0(tile) + (xt ? jr : row);
      valid = j < (list == 1 ? n1 : (list == 2 ? n2 : n0));
      p = make_float3(0.f, 0.f, 0.f);
      shape = 0;
      if (valid) rowsrc_load(a.src[list], j, p, shape);
      const float* bf4 = a.bfold4 + (size_t)shape * 512;
      // layer 0: this CTA's 128 columns
#pragma unroll 1
      for (int k = 2 * half; k < 2 * half + 2; ++k) {
        uint32_t h[16];
        layer0(W_BN * rank + 32 * k, h);
        put(W_BN * rank + 32 * k, h);
      }
      if (!exchange(512)) { ok = false; break; }
      float hc[4] = {0.f, 0.f, 0.f, 0.f};
      for (int g = 0; g < NUM_GEMM; ++g) {
        const int nr = gemm_n(g) / WC;
        const int c0 = nr * rank;
        // this layer's epilogue constants into L1 while its MMAs run
        for (int k = half * nr / 64; k < (half + 1) * nr / 64; ++k) {
          prefetch_l1((g == 3 ? bf4 : K->bias[g]) + c0 + 32 * k);
          if (g == NUM_GEMM - 1) prefetch_l1(K->w_head + c0 + 32 * k);
        }
        if (!wait_acc()) { ok = false; break; }
        if (g < NUM_GEMM - 1) {
#pragma unroll 1
          for (int k = half * nr / 64; k < (half + 1) * nr / 64; ++k) {
            uint32_t h[16];
            hold(g, bf4, 32 * k, c0 + 32 * k, h);
            put(c0 + 32 * k, h);
          }
          tc_fence_before();
          if (!exchange(gemm_n(g))) { ok = false; break; }
        } else {
          // head chunk sums of this CTA's quarter (q = rank, groups k)
#pragma unroll 1
          for (int k = 2 * half; k < 2 * half + 2; ++k) {
            uint32_t r[32];
            tmem_ld32(t_row + (uint32_t)(32 * k), r);
            hc[k] = head_chunk_sum<F16>(K, xt, bf4, p, c0 + 32 * k, part,
                                        a.inv_scale[NUM_GEMM - 1], r);
          }
          tc_fence_before();
        }
      }
      if (!ok) break;
      // head: rank 0 adds the 16 chunk sums of each row in the single-CTA
      // kernel's order: per group k, quarters 0..3; then groups 0..3
      const int hr = xt ? jr : row;
      float* hg = a.head_g + ((size_t)cid * BM + hr) * 16;
      if (!xt || part == 0)
        for (int k = 2 * half; k < 2 * half + 2; ++k) hg[rank * 4 + k] = hc[k];
      __threadfence();
      __syncwarp();
      if (lane == 0) mbar_arrive_remote(map_rank(smem_u32(head_ready), 0u));
      if (rank == 0 && half == 0) {
        if (!mbar_wait_cl(head_ready, head_phase, abort_flag)) { ok = false; break; }
        head_phase ^= 1u;
        float total = 0.f;
        for (int k = 0; k < 4; ++k) {
          float hk = 0.f;
          for (int q = 0; q < 4; ++q) hk += __ldcg(hg + q * 4 + k);
          total = k == 0 ? hk : total + hk;
        }
        const float f = tanhf(total + __ldg(&K->b_head));
        const bool mine = valid && (!xt || part == 0);
        if (a.fuse_step) {
          int keep = -1, ray = 0;
          if (mine) {
            ray = a.src[list].idx[j];
            keep = step_ray(a.step.t, list, ray, f);
          }
          const int s0 = warp_append(keep == 0, a.step.cnt_out[0]);
          const int s1 = warp_append(keep == 1, a.step.cnt_out[1]);
          const int s2 = warp_append(keep == 2, a.step.cnt_out[2]);
          if (s0 >= 0) a.step.out[0][s0] = ray;
          if (s1 >= 0) a.step.out[1][s1] = ray;
          if (s2 >= 0) a.step.out[2][s2] = ray;
        } else if (mine) {
          a.fout[list][j] = f;
        }
      }
    }
    if (!ok) {
      *abort_flag = 1;
      atomicOr(a.err, 4);
    }
    if (!(vmax <= 65504.f)) atomicOr(a.err, 64);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 128);
  }
  cluster_sync_all();   // no CTA leaves while a peer may still arrive on its barriers
  grid_dep_wait();      // this step's mlp_tc_kernel is complete
}

}  // namespace

// Clusters of WC CTAs that can be resident at once (at most WT_MAX): the
// largest tile count the latency mode takes.
int tc_wide_max_tiles() {
  // computed once per process (thread-safe static initialisation)
  static const int n = [] {
    if (cudaFuncSetAttribute(mlp_tc_wide_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             W_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(mlp_tc_wide_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             W_SMEM) != cudaSuccess) {
      (void)cudaGetLastError();
      return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(WC * WT_MAX);
    cfg.blockDim = dim3(W_THREADS);
    cfg.dynamicSmemBytes = W_SMEM;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = WC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int c = 0;
    if (cudaOccupancyMaxActiveClusters(&c, mlp_tc_wide_kernel<true>, &cfg) != cudaSuccess) {
      (void)cudaGetLastError();
      c = 0;
    }
    return c < WT_MAX ? c : WT_MAX;
  }();
  return n;
}

cudaError_t mlp_tc_wide(const dist_decoder* dec, const RowSrc& src16, float* f16out,
                        const RowSrc& srcx, float* fxout, const float* bfold0,
                        const float* bfolds, cudaStream_t st, bool f16, const StepFuse* step,
                        void* scratch, const RowSrc* srcm, float* fmout) {
  WideArgs a;
  memset(&a, 0, sizeof(a));
  a.K = dec->tc.cst;
  a.bfold0 = bfold0;
  a.bfold4 = bfolds;
  a.src[0] = src16;
  a.src[1] = srcx;
  if (srcm) a.src[2] = *srcm;       // else count 0 (zeroed above)
  a.fout[0] = f16out;
  a.fout[1] = fxout;
  a.fout[2] = fmout;
  a.err = dec->tc.err;
  for (int g = 0; g < NUM_GEMM; ++g) a.inv_scale[g] = dec->tc.x_inv_scale[g];
  a.fuse_step = step ? 1 : 0;
  if (step) a.step = *step;
  a.stage_g = static_cast<uint8_t*>(scratch);
  a.head_g = reinterpret_cast<float*>(a.stage_g + (size_t)WT_MAX * 2 * ACT_BYTES);
  a.nsm = num_sms();
  const int wt = tc_wide_max_tiles();
  if (wt <= 0) return cudaErrorNotSupported;
  auto kern = f16 ? mlp_tc_wide_kernel<true> : mlp_tc_wide_kernel<false>;
  const TCMaps& maps = f16 ? dec->tc.wmaps16 : dec->tc.wmaps;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(WC * wt);
  cfg.blockDim = dim3(W_THREADS);
  cfg.dynamicSmemBytes = W_SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = WC;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, maps, dec->tc.wxmaps, dec->tc.wmaps16, a);
  count_launch(1);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

size_t tc_wide_scratch_bytes() {
  return (size_t)WT_MAX * 2 * ACT_BYTES + (size_t)WT_MAX * BM * 16 * sizeof(float) + 256;
}

unsigned long long* tc_wide_seq_flag(void* scratch) {
  return reinterpret_cast<unsigned long long*>(static_cast<uint8_t*>(scratch) +
                                               tc_wide_scratch_bytes() - 256);
}

}  // namespace dist
