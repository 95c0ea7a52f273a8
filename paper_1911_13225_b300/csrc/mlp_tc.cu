// tcgen05 decoder forward for the DeepSDF shape: 8 hidden layers of 512,
// latent 256 folded into per-shape biases of layer 0 and the skip layer 4,
// ReLU, tanh head (Sec. B.1).  GEMM layers 1..7 run on the 5th generation
// tensor cores with FP32 accumulation in tensor memory; layer 0 (3 inputs),
// the xyz columns of layer 4 and the 512 -> 1 head run on CUDA cores in FP32
// inside the epilogue.  One launch decodes two row lists: 16-bit operands
// (BF16 or FP16) and FP32-class operands (each a sum of two FP16 numbers).
//
// One persistent CTA per SM, 128-row tiles (one row per TMEM lane):
//   warp 0      TMA producer: weight slices [256 N x 64 K] (128B swizzle)
//               into a 3-stage ring;
//   warp 1      TMEM owner and single-thread MMA issuer
//               (M = 128, N = 256, K = 16 per instruction);
//   warps 2-17  epilogue: four warps per TMEM lane quadrant split the
//               columns; tcgen05.ld the accumulator, add bias (+ xyz term),
//               ReLU, round to the operand format and write the next layer's
//               A operand into the shared activation tile in the same
//               128B-swizzled K-major layout the MMA descriptors describe.
// Activations never leave the SM.  Every wait is bounded (1 s): on timeout
// the CTA raises an error word, drains its MMAs and frees its TMEM.
//
// FP32-class tiles: 64 queries per tile.  In TMEM lane quadrant q, rows
// 32q + i (i < 16) hold the hi parts of the activations of query 16q + i and
// rows 32q + 16 + i their lo parts.  Each layer runs its K loop twice, first
// against W_lo, then against W_hi (weights of layer l scaled by 2^s_l so
// that W_lo stays a normal FP16 number), into one FP32 accumulator, so rows
// 32q + i and 32q + 16 + i hold a_hi (W_hi + W_lo) and a_lo (W_hi + W_lo);
// their sum, one warp shuffle apart, is (a_hi + a_lo)(W_hi + W_lo): all four
// partial products, nothing dropped beyond the two split residuals.  The
// work per query is four times a 16-bit query.
// Accuracy: emulated with exact accumulation this arithmetic is as close to
// the FP64 decoder as FP32 CUDA-core arithmetic (~1e-7 in f), but the tensor
// core's FP32 accumulator does not round to nearest: measured on B300 each
// K step loses a fraction of an ulp of the running sum, always towards zero,
// which leaves a systematic error of ~2e-6 in f.  The small W_lo pass runs
// first so that only the W_hi pass adds into a large accumulator.
#include <cmath>
#include <cstring>
#include <vector>

#include "step.cuh"
#include "tc_common.cuh"

namespace dist {

namespace {

// Forward arguments: three row lists decoded in one launch.  List 0 runs
// with 16-bit operands (BF16, or FP16 with the F16 variant), 128 rows per
// tile; list 1 is FP32-class: every operand a sum of two FP16 numbers (hi +
// lo, weights scaled by 2^s_l), 64 queries per tile, see tc_common.cuh; list
// 2 runs with FP16 operands, 128 rows per tile (the FP16 stage between a
// BF16 march and its FP32-class queries; empty otherwise).
struct TCArgs {
  const TCConst* K;              // epilogue constants (device)
  const float* bfold0;           // [shape][512] folded bias of layer 0
  const float* bfold4;           // [shape][512] folded bias of the skip layer 4
  RowSrc src[3];
  float* fout[3];
  int* err;
  float inv_scale[NUM_GEMM];     // list 1: 2^-s_l of GEMM layer g
  float* cpart;                  // colour decoder: [row][4 column groups][3] head partials
  int fuse_step;                 // apply `step` to each row instead of writing f
  StepFuse step;
  int wide_tiles;                // > 0: launches of at most this many latency-mode tiles
                                 // are left to mlp_tc_wide_kernel
  unsigned long long wait_ns;    // limit of every wait of the decoding loop
  int withhold;                  // tests: the TMA producer issues no weight copies, so
                                 // the MMA warp's first wait runs out
};

constexpr int QPT_X = 64;        // FP32-class queries per tile

// Tile of round r for CTA pid in a launch of npid: serpentine order.
// The FP32-class tiles (twice a 16-bit tile's work) come first in the tile
// list, so odd rounds run backwards and hand their tiles to the CTAs that took
// the cheaper tiles of the round before.  Increasing in r for a fixed pid.
__device__ __forceinline__ int tile_of(int r, int pid, int npid) {
  return r * npid + ((r & 1) ? npid - 1 - pid : pid);
}


// Forward pipeline.  A tile is one of the two kinds; the FP32-class tiles
// come first in tile order (they take twice as long).  A tile's K loop runs
// once (16-bit) or twice (FP32-class: against W_lo, then W_hi).  The
// accumulator of a 512-wide layer completes in two 256-column halves
// (acc_full[0], acc_full[1]); the next layer's operand is handed back in four
// 128-column K quarters (act_full[0..3]).
//   epilogue (16 warps, four per TMEM lane quadrant, one 32-column chunk of
//     each quarter per warp): after acc_full[0] it reads quarters 0 and 1
//     into registers while the tensor core computes half 1; once
//     acc_full[1] says the layer's MMAs (which read the operand tile) are
//     done it writes them and releases act_full[0] and [1], then reads,
//     converts and writes quarter 2, releases it, and quarter 3.
//   MMA: the next layer's first output half starts on K quarter 0 as soon as
//     act_full[0] arrives, so it overlaps the epilogue's second half;
//     act_full[3] also certifies that TMEM columns 256..511 have been read.
// On the last layer the released operand tile takes the next tile's layer 0
// (in the next tile's format), so the next tile's GEMMs overlap this tile's
// head.
//
// (A CTA-pair variant -- cta_group::2, M = 256, each SM streaming half of
// every weight stage -- measured slower on B300, 973 against 1,183 TFLOP/s
// on large launches and 92 against 78 us for one tile: the cross-CTA
// hand-offs cost more than the halved weight stream saves.  Not kept.)
template <bool F16, bool COLOR>
__global__ void __launch_bounds__(FWD_THREADS, 1)
mlp_tc_kernel(const __grid_constant__ TCMaps maps, const __grid_constant__ TCMaps xmaps,
              const __grid_constant__ TCMaps maps16, const TCArgs a) {
  constexpr int NST = STAGES;          // weight ring stages
  constexpr int SB = STAGE_BYTES;      // bytes per stage
  static_assert((2 * NST + 10) * 8 + 8 <= BAR_BYTES, "barrier block");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint8_t* act = smem;
  uint8_t* wst = smem + ACT_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(wst + NST * SB);
  uint64_t* full = bars;                     // [NST]
  uint64_t* empty = bars + NST;              // [NST]
  uint64_t* acc_full = bars + 2 * NST;       // [2] MMA -> epilogue, per N half
  uint64_t* act_full = bars + 2 * NST + 2;   // [4] epilogue -> MMA, per K quarter
  uint64_t* drain = bars + 2 * NST + 6;      // final MMA completion
  uint64_t* head_bar = bars + 2 * NST + 7;   // head partial sums -> column group 0
  uint64_t* step_full = bars + 2 * NST + 8;  // f of a tile's rows -> step warps
  uint64_t* step_empty = bars + 2 * NST + 9; // step warps have read them
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NST + 10);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* head_part = reinterpret_cast<float*>(smem + ACT_BYTES + NST * SB + BAR_BYTES);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const unsigned long long wlim = a.wait_ns;
  const int pid = (int)blockIdx.x;
  const int npid = (int)gridDim.x;
  // shared-memory barriers and TMEM read nothing the previous grid writes:
  // set them up before waiting for it (the other TMEM users of this library
  // need as much shared memory as this kernel, so none of their CTAs shares
  // an SM with this one and holds TMEM it would wait for)
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int h = 0; h < 2; ++h) mbar_init(acc_full + h, 1);
    for (int q = 0; q < 4; ++q) mbar_init(act_full + q, FWD_EPI);
    mbar_init(drain, 1);
    mbar_init(head_bar, (FWD_EPI - 4) * 32);
    mbar_init(step_full, 4);
    mbar_init(step_empty, FWD_STEP_WARPS);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // launched early behind the previous grid (programmatic dependent
  // launch): nothing it writes is read before this wait
  grid_dep_wait();
  if (a.wide_tiles > 0) {
    // mlp_tc_wide_kernel, launched behind this grid, may run beside it: it
    // acquires this step's inputs (complete and visible here) through the
    // release of the step's sequence number, written before any CTA of this
    // grid lets it launch
    if (pid == 0 && threadIdx.x == 0) seq_release(a.step.seq_flag, a.step.seq);
    __syncthreads();
  }
  grid_dep_launch();
  const int n0 = rowsrc_count(a.src[0]);
  const int n1 = rowsrc_count(a.src[1]);
  const int n2 = rowsrc_count(a.src[2]);
  const int t1 = (n1 + QPT_X - 1) / QPT_X;   // FP32-class tiles: [0, t1)
  const int t2 = t1 + (n2 + BM - 1) / BM;     // FP16-stage tiles: [t1, t2)
  const int n_tiles = t2 + (n0 + BM - 1) / BM;
  // tiles [0, tb) go to the latency-mode kernel (all of a small launch, or
  // the FP32-class tiles of a launch that leaves room for both, see
  // wide_share); this grid takes [tb, n_tiles)
  const int tb = wide_share(n_tiles, t1, a.wide_tiles, npid);
  if (tb + pid >= n_tiles) {
    if (warp == 1) tmem_dealloc(tmem, 512);
    return;
  }
  // tile of round r for this CTA
  auto tile_at = [&](int r) { return tb + tile_of(r, pid, npid); };
  if (a.fuse_step && a.step.queries && pid == 0 && threadIdx.x == 0) {
    atomicAdd(a.step.queries + 0, (unsigned long long)(n0 + n2));
    atomicAdd(a.step.queries + 1, (unsigned long long)n1);
  }
  // row list of tile t, and the first row of its list in this CTA
  auto tile_list = [&](int t) { return t < t1 ? 1 : (t < t2 ? 2 : 0); };
  auto tile_row0 = [&](int t) {
    return t < t1 ? t * QPT_X : (t - (t < t2 ? t1 : t2)) * BM;
  };


  if (warp == 0) {
    // ------------------------------------------------------ TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_parity[NST];
      bool issued[NST];
      for (int s = 0; s < NST; ++s) issued[s] = false;
      bool ok = true;
      // (a.withhold, tests only: no copy is issued, so the MMA warp's first
      // wait for a weight stage runs out and the CTA takes its abort path)
      for (int r = 0, tile = tile_at(0); ok && !a.withhold && tile < n_tiles; tile = tile_at(++r)) {
        const bool xt = tile < t1;
        const bool mid = tile_list(tile) == 2;
        for (int g = 0; ok && g < NUM_GEMM; ++g) {
          const CUtensorMap* map = xt ? &xmaps.m[g] : (mid ? &maps16.m[g] : &maps.m[g]);
          const int nkc = gemm_k(g) / BK;
          for (int nh = 0; ok && nh < gemm_n(g) / BN; ++nh) {
            for (int kc = 0; kc < (xt ? 2 : 1) * nkc; ++kc) {
              if (!mbar_wait(empty + stage, phase ^ 1u, abort_flag, wlim)) { ok = false; break; }
              mbar_expect_tx(full + stage, SB);
              // FP32-class: the W_lo pass (columns K..2K-1) first, then W_hi
              const int xk = !xt ? kc : (kc < nkc ? nkc + kc : kc - nkc);
              tma_load_2d(wst + stage * SB, map, full + stage, xk * BK, nh * BN);
              issued[stage] = true;
              issued_parity[stage] = phase;
              if (++stage == NST) { stage = 0; phase ^= 1u; }
            }
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(a.err, 1);
      }
      // every issued copy must land before the CTA exits
      for (int s = 0; s < NST; ++s) {
        if (!issued[s]) continue;
        const unsigned long long t0 = globaltimer();
        while (!mbar_try_wait(full + s, issued_parity[s]) && globaltimer() - t0 < kTimeoutNs) {
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t act_phase[4] = {0u, 0u, 0u, 0u};
      bool ok = true;
      auto commit = [&](uint64_t* bar) { mma_commit(bar); };
      for (int r = 0, tile = tile_at(0); ok && tile < n_tiles; tile = tile_at(++r)) {
        const bool xt = tile < t1;
        const uint32_t idesc = instr_desc_m(xt || F16 || tile_list(tile) == 2, BM);
        for (int g = 0; ok && g < NUM_GEMM; ++g) {
          const int nkc = gemm_k(g) / BK;
          for (int nh = 0; ok && nh < gemm_n(g) / BN; ++nh) {
            for (int kc = 0; kc < (xt ? 2 : 1) * nkc; ++kc) {
              if (nh == 0 && kc < nkc && (kc & 1) == 0) {
                const int q = kc >> 1;
                if (!mbar_wait(act_full + q, act_phase[q], abort_flag, wlim)) { ok = false; break; }
                act_phase[q] ^= 1u;
                tc_fence_after();
              }
              if (!mbar_wait(full + stage, phase, abort_flag, wlim)) { ok = false; break; }
              tc_fence_after();
              const uint32_t a_base = smem_u32(act + (kc < nkc ? kc : kc - nkc) * CHUNK_BYTES);
              const uint32_t b_base = smem_u32(wst + stage * SB);
#pragma unroll
              for (int k = 0; k < BK / 16; ++k)
                mma_bf16(tmem + (uint32_t)(nh * BN), sw128_desc(a_base + 32 * k),
                         sw128_desc(b_base + 32 * k), idesc, (kc | k) != 0);
              commit(empty + stage);
              if (++stage == NST) { stage = 0; phase ^= 1u; }
            }
            if (ok) commit(acc_full + nh);
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(a.err, 2);
      }
      // all issued MMAs complete before TMEM is released
      commit(drain);
    }
    if (lane == 0) {
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(drain, 0) && globaltimer() - t0 < kTimeoutNs) {
      }
    }
  } else if (warp >= 2 + FWD_EPI) {
    // ----------------------------------------------------- march step
    // With a fused step, thread s applies the step update to rows s, s + 64
    // of each of this CTA's tiles once column group 0 has put their f in
    // head_part (the step update is off the decoder's critical path).
    if (a.fuse_step) {
      constexpr int SW = FWD_STEP_WARPS * 32;
      constexpr int RPT = BM / SW;   // rows per step thread
      const int s = threadIdx.x - (2 + FWD_EPI) * 32;
      uint32_t sphase = 0;
      for (int r = 0, t = tile_at(0); t < n_tiles; t = tile_at(++r)) {
        const bool xt = t < t1;
        const int list = tile_list(t);
        const int j0 = tile_row0(t);
        const int rows = xt ? QPT_X : BM;
        const int n = list == 1 ? n1 : (list == 2 ? n2 : n0);
        // the rows' ray state is read while the tile is being decoded
        int ray[RPT];
        bool valid[RPT];
        RayState rs[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
          const int r = s + k * SW;
          valid[k] = r < rows && j0 + r < n;
          ray[k] = valid[k] ? a.src[list].idx[j0 + r] : 0;
          if (valid[k]) load_ray(a.step.t, list, ray[k], rs[k]);
        }
        if (!mbar_wait(step_full, sphase, abort_flag, wlim)) {
          *abort_flag = 1;
          atomicOr(a.err, 4);
          break;
        }
        sphase ^= 1u;
        float f[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) f[k] = head_part[s + k * SW];
        __syncwarp();
        if (lane == 0) mbar_arrive(step_empty);
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
          const int keep = valid[k] ? apply_step(a.step.t, list, ray[k], f[k], rs[k]) : -1;
          const int s0 = warp_append(keep == 0, a.step.cnt_out[0]);
          const int s1 = warp_append(keep == 1, a.step.cnt_out[1]);
          const int s2 = warp_append(keep == 2, a.step.cnt_out[2]);
          if (s0 >= 0) a.step.out[0][s0] = ray[k];
          if (s1 >= 0) a.step.out[1][s1] = ray[k];
          if (s2 >= 0) a.step.out[2][s2] = ray[k];
        }
      }
    }
  } else {
    // --------------------------------------------------------- epilogue
    // 16-bit tile: this thread owns tile row 32 quad + lane.  FP32-class
    // tile: lanes i and i + 16 of a warp own query 16 quad + i, lane i its
    // hi operand row 32 quad + i and lane i + 16 its lo row 32 quad + 16 + i;
    // each keeps 16 of the warp's 32 columns after their pair sum.
    const int ew = warp - 2;                  // 0..FWD_EPI-1
    const int quad = warp & 3;                // TMEM lane quadrant of this warp
    const int grp = ew >> 2;                  // 32-column chunk inside each quarter
    const int cg = grp * 32;
    const int row = quad * 32 + lane;         // 16-bit tiles
    const int part = lane >> 4;               // FP32-class tiles
    const int jr = quad * 16 + (lane & 15);
    const int rhi = quad * 32 + (lane & 15);
    const int rlo = rhi + 16;
    const uint32_t t_row = tmem + ((uint32_t)(quad * 32) << 16);
    const TCConst* K = a.K;
    uint32_t acc_phase[2] = {0u, 0u};
    uint32_t head_phase = 0;
    bool ok = true;
    float vmax = 0.f;

    // rows of tile t for this thread (list, operand format: f16 for the
    // FP16 stage, or for every 16-bit tile of the F16 variant)
    bool xt = false, valid = false, f16 = F16;
    int list = 0, j = 0, shape = 0;
    float3 p = make_float3(0.f, 0.f, 0.f);
    auto load_rows = [&](int t) {
      list = tile_list(t);
      xt = list == 1;
      f16 = F16 || list == 2;
      j = tile_row0(t) + (xt ? jr : row);
      valid = j < (list == 1 ? n1 : (list == 2 ? n2 : n0));
      p = make_float3(0.f, 0.f, 0.f);
      shape = 0;
      if (valid) rowsrc_load(a.src[list], j, p, shape);
    };
    auto wait_acc = [&](int h) -> bool {
      if (!mbar_wait(acc_full + h, acc_phase[h], abort_flag, wlim)) return false;
      acc_phase[h] ^= 1u;
      tc_fence_after();
      return true;
    };
    // one arrival per warp on act_full[q]
    auto release = [&](int q) {
      fence_async_shared();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(act_full + q);
    };
    // operand words of quarter q: 16 packed pairs (16-bit tile) or 8 hi + 8
    // lo pairs (FP32-class tile), written to the operand tile by put()
    auto put = [&](int q, const uint32_t (&h)[16]) {
      if (!xt) {
        store_packed<16>(act, row, 128 * q + cg, h);
      } else {
        const int c = 128 * q + cg + 16 * part;
        const uint32_t ch = (uint32_t)((c >> 6) * CHUNK_BYTES);
        const uint32_t u = (uint32_t)((c & 63) >> 3);
        const uint32_t base = smem_u32(act) + ch;
        st_shared_v4(base + swz(rhi, u), h[0], h[1], h[2], h[3]);
        st_shared_v4(base + swz(rhi, u + 1), h[4], h[5], h[6], h[7]);
        st_shared_v4(base + swz(rlo, u), h[8], h[9], h[10], h[11]);
        st_shared_v4(base + swz(rlo, u + 1), h[12], h[13], h[14], h[15]);
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
    // layer 0 of the current rows, quarter q
    auto layer0 = [&](int q, uint32_t (&h)[16]) {
      const float* bf0 = a.bfold0 + (size_t)shape * 512;
      if (!xt) {
        float v[32];
        layer0_32(K, bf0, 128 * q + cg, p, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) h[i] = pack16r(f16, v[2 * i], v[2 * i + 1]);
      } else {
        float v[16];
        layer0_16(K, bf0, 128 * q + cg + 16 * part, p, v);
        split_pack(v, h);
      }
    };
    // quarter q of GEMM layer g (rows at p): operand words of relu(acc + bias).
    // Layer 3's padding columns 253..255 carry the ray point instead (the
    // skip layer's GEMM multiplies them by its xyz weights).
    auto hold = [&](int g, const float* bf4, const float3& pp, int q, uint32_t (&h)[16]) {
      uint32_t r[32];
      tmem_ld32(t_row + (uint32_t)(128 * q + cg), r);
      const bool point = g == 2 && 128 * q + cg == 224;
      if (!xt) {
        // bias, ReLU and packing in place, 4 columns at a time (keeps the
        // live registers to the accumulator words and the packed result)
        const float* bias = g == 3 ? bf4 : K->bias[g];
#pragma unroll
        for (int i = 0; i < 32; i += 4) {
          const float4 b = ldg4(bias + 128 * q + cg + i);
          h[i / 2] = pack16r(f16, fmaxf(__uint_as_float(r[i]) + b.x, 0.f),
                                 fmaxf(__uint_as_float(r[i + 1]) + b.y, 0.f));
          h[i / 2 + 1] = pack16r(f16, fmaxf(__uint_as_float(r[i + 2]) + b.z, 0.f),
                                     fmaxf(__uint_as_float(r[i + 3]) + b.w, 0.f));
        }
        if (point) {
          const float b28 = __ldg(K->bias[g] + 252);
          h[14] = pack16r(f16, fmaxf(__uint_as_float(r[28]) + b28, 0.f), pp.x);
          h[15] = pack16r(f16, pp.y, pp.z);
        }
      } else {
        float m[16], v[16];
        pair_sum16(r, part, m);
        affine16(K, g, bf4, 128 * q + cg + 16 * part, pp, a.inv_scale[g], m, v, false);
        const float v12 = fmaxf(v[12], 0.f);
        split_pack(v, h);
        if (point && part == 1) {      // this lane's columns 240..255
          split_pair(v12, pp.x, h[6], h[14]);
          split_pair(pp.y, pp.z, h[7], h[15]);
        }
      }
    };
    // head term of the 32-column chunk of quarter q of the last layer (tile
    // kind `kx`): its own sum, so that the per-row total is the same fixed-
    // order sum of 16 chunk sums as in the latency mode (mlp_tc_wide_kernel)
    auto head_q = [&](bool kx, const float* bf4, const float3& pp, int q) -> float {
      uint32_t r[32];
      tmem_ld32(t_row + (uint32_t)(128 * q + cg), r);
      return head_chunk_sum<F16>(K, kx, bf4, pp, 128 * q + cg, part, a.inv_scale[NUM_GEMM - 1], r);
    };

    uint32_t step_phase = 0;   // column group 1: step_empty parity
    int tile = tile_at(0);
    int rnd = 0;
    load_rows(tile);
    for (int q = 0; q < 4; ++q) {
      uint32_t h[16];
      layer0(q, h);
      put(q, h);
      release(q);
    }
    for (; tile < n_tiles; tile = tile_at(++rnd)) {
      const float* bf4 = a.bfold4 + (size_t)shape * 512;
      const int next = tile_at(rnd + 1);
      const bool has_next = next < n_tiles;
      for (int g = 0; g < NUM_GEMM - 1; ++g) {
        if (!wait_acc(0)) { ok = false; break; }
        if (gemm_n(g) == 256) {
          // one output half: the layer's MMAs are done, write directly
          for (int q = 0; q < 2; ++q) {
            uint32_t h[16];
            hold(g, bf4, p, q, h);
            put(q, h);
            release(q);
          }
          continue;
        }
        uint32_t h0[16], h1[16];
        hold(g, bf4, p, 0, h0);
        hold(g, bf4, p, 1, h1);
        if (!wait_acc(1)) { ok = false; break; }
        put(0, h0);
        release(0);
        put(1, h1);
        release(1);
        for (int q = 2; q < 4; ++q) {
          uint32_t h[16];
          hold(g, bf4, p, q, h);
          put(q, h);
          release(q);
        }
      }
      if (!ok) break;
      // ---- last layer: head partial sums; the operand tile takes the next
      // tile's layer 0 once this layer's MMAs are done
      const bool cur_xt = xt;
      const int cur_list = list;
      const int cur_j = j;
      const bool cur_valid = valid;
      const float3 cur_p = p;
      float head = 0.f;
      // colour decoder (16-bit rows): the three head rows' partial dot
      // products over this thread's 32 columns of each quarter, in order
      float cacc[3] = {0.f, 0.f, 0.f};
      auto color_q = [&](int q) {
        if constexpr (COLOR) {
          uint32_t r[32];
          tmem_ld32(t_row + (uint32_t)(128 * q + cg), r);
          float v[32];
          bias32(K, NUM_GEMM - 1, bf4, 128 * q + cg, cur_p, r, v);
#pragma unroll
          for (int o = 0; o < 3; ++o)
#pragma unroll
            for (int i = 0; i < 32; i += 4) {
              const float4 w = ldg4(K->w_c[o] + 128 * q + cg + i);
              cacc[o] = fmaf(fmaxf(v[i], 0.f), w.x,
                             fmaf(fmaxf(v[i + 1], 0.f), w.y,
                                  fmaf(fmaxf(v[i + 2], 0.f), w.z,
                                       fmaf(fmaxf(v[i + 3], 0.f), w.w, cacc[o]))));
            }
        }
      };
      if (!wait_acc(0)) { ok = false; break; }
      head += head_q(cur_xt, bf4, cur_p, 0);
      color_q(0);
      head += head_q(cur_xt, bf4, cur_p, 1);
      color_q(1);
      // from here on xt/j/p/shape describe the next tile's rows (layer 0 in
      // its format): quarters 0 and 1 of it are computed while the tensor
      // core finishes this layer; quarter q is released once this tile's
      // quarter q has been read from TMEM
      uint32_t n0h[16], n1h[16];
      if (has_next) {
        load_rows(next);
        layer0(0, n0h);
        layer0(1, n1h);
      }
      if (!wait_acc(1)) { ok = false; break; }
      if (has_next) {
        put(0, n0h);
        release(0);
        put(1, n1h);
        release(1);
      }
      for (int q = 2; q < 4; ++q) {
        head += head_q(cur_xt, bf4, cur_p, q);
        color_q(q);
        if (has_next) {
          uint32_t h[16];
          layer0(q, h);
          put(q, h);
          release(q);
        }
      }
      if (!has_next) tc_fence_before();
      if constexpr (COLOR) {
        if (cur_valid && !cur_xt)
#pragma unroll
          for (int o = 0; o < 3; ++o) a.cpart[((size_t)cur_j * 4 + grp) * 3 + o] = cacc[o];
      }
      // head: f = tanh(w . h7 + b); column groups 1..3 hand their partial
      // sums to group 0 (head_part is rewritten only after the next tile's
      // layers, which group 0 takes part in, so one phase per tile suffices)
      const int hr = cur_xt ? jr : row;
      if (grp > 0) {
        // with a fused step, head_part[0..BM) carries the previous tile's f
        // to the step warps: group 1 overwrites it once they have read it
        if (a.fuse_step && grp == 1 && rnd > 0) {
          if (!mbar_wait(step_empty, step_phase, abort_flag, wlim)) { ok = false; break; }
          step_phase ^= 1u;
        }
        head_part[(grp - 1) * BM + hr] = head;
        mbar_arrive(head_bar);
      } else {
        if (!mbar_wait(head_bar, head_phase, abort_flag, wlim)) { ok = false; break; }
#pragma unroll
        for (int q = 0; q < FWD_GRPS - 1; ++q) head += head_part[q * BM + hr];
        const bool mine = cur_valid && (!cur_xt || part == 0);
        if (a.fuse_step) {
          // f to the step warps (rows past the list end included); in an
          // FP32-class tile both lanes of a query read slot hr above
          __syncwarp();
          if (!cur_xt || part == 0) head_part[hr] = tanhf(head + __ldg(&K->b_head));
          __syncwarp();
          if (lane == 0) mbar_arrive(step_full);
        } else if (mine) {
          a.fout[cur_list][cur_j] = tanhf(head + __ldg(&K->b_head));
        }
      }
      head_phase ^= 1u;
    }
    if (!ok) {
      *abort_flag = 1;
      atomicOr(a.err, 4);
    }
    if (!(vmax <= 65504.f)) atomicOr(a.err, 64);   // an FP32-class activation overflowed FP16
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------- adjoint
//
// The same pipeline runs 14 GEMMs per 128-probe tile: the 7 forward layers
// again (recording ReLU masks), then, from g_7 = (1 - f^2) w_head * 1[a_7 > 0],
// the 7 backward GEMMs g_{l-1} = (W_l^T g_l) * 1[a_{l-1} > 0] with W_l^T tiles
// (TMA maps over the transposed weights).  The skip layer's gradient g_4 and
// layer 0's g_0 give grad_p f = Wx0^T g_0 + Wx4^T g_4 and the latent
// gradient W_z0^T g_0 + W_z4^T g_4; per probe coefficients c (the paper's
// first-term weight, or -w / (grad f . v) for the exact depth gradient) scale
// g_0 and g_4, which are summed over rays into FP64 per-shape accumulators
// (a warp transpose-reduction over 32 rays in FP32, then FP64 atomics).
//
// Each GEMM's accumulator completes in two 256-column halves (acc_half[0],
// acc_half[1]); the epilogue warps of a lane quadrant split every layer's
// columns between two sides, each side taking 128 columns of each half, and
// hold their half-0 results in registers until the half-1 MMAs (which still
// read the operand tile) are done, so half 0's epilogue overlaps half 1's
// MMAs.  The two sides of a row meet through a small exchange buffer and
// two mbarriers (side 1 -> side 0: head and gradient partial sums; side 0 ->
// side 1: 1 - f^2 and the coefficient).
//
// FP32-class variant (X): 64 probes per tile in the forward kernel's hi / lo
// row layout, every GEMM's K loop twice (W_lo, then W_hi; the backward
// GEMMs over the transposed split), the lane pair of a probe adding its two
// rows.  The backward operand g is scaled by 2^kGradExp before its split, so
// that its lo parts stay normal FP16 numbers (the backward is linear in g;
// the scale is exact and removed before any result leaves the kernel).

constexpr int XFER_BYTES = 3 * BM * 4;
constexpr int ADJ_SMEM_BYTES = 1024 + ACT_BYTES + STAGES * STAGE_BYTES + BAR_BYTES + XFER_BYTES;
constexpr int NUM_ADJ_GEMM = 14;
constexpr size_t kMaskWordsPerCta = (size_t)8 * 128 * 2 * 8;

// GEMM e of a tile: forward layers 1..7 (e < 7), then backward layers 7..1.
__device__ __forceinline__ int adj_n(int e) { return e < 7 ? gemm_n(e) : gemm_k(13 - e); }
__device__ __forceinline__ int adj_k(int e) { return e < 7 ? gemm_k(e) : gemm_n(13 - e); }

constexpr int kGradExp = 8;   // FP32-class adjoint: g scaled by 2^8 before its split

struct TCAdjArgs {
  const TCConst* K;
  const float* bfold0;
  const float* bfold4;
  const float4* pp;
  const float4* pq;
  const int* count;
  float* out4;
  double* gacc0;
  double* gacc4;
  int accumulate;
  uint8_t* scratch;   // gridDim.x * kTcAdjScratchPerCta bytes
  int* err;
  float inv_scale[NUM_GEMM];   // X: 2^-s_l of GEMM layer g
  // X, optional: probes with a ReLU input within redo_tau of 0 are appended
  // to (redo_p, redo_q) instead of being accumulated (at most redo_cap; the
  // rest are accumulated here), for an FP32 adjoint to redo
  float4* redo_p;
  float4* redo_q;
  int* redo_count;
  int redo_cap;
  float redo_tau;
};

// Sum of v[0..31] over the 32 lanes of the warp, column by column: lane L
// returns the column-L total (recursive halving, 31 shuffles).
__device__ __forceinline__ float warp_column_sum(float (&v)[32], int lane) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const float send = upper ? v[i] : v[i + o];
      const float recv = __shfl_xor_sync(0xffffffffu, send, o);
      v[i] = (upper ? v[i + o] : v[i]) + recv;
    }
  }
  return v[0];
}

template <bool F16, bool X>
__global__ void __launch_bounds__(THREADS, 1)
mlp_tc_adj_kernel(const __grid_constant__ TCMaps fmaps, const __grid_constant__ TCMaps bmaps,
                  const TCAdjArgs a) {
  static_assert(!X || F16, "FP32-class operands are FP16 pairs");
  constexpr uint32_t kIdesc = instr_desc<F16>();
  constexpr int QPT = X ? 64 : BM;     // probes per tile
  constexpr int NPASS = X ? 2 : 1;     // K passes per GEMM (X: W_lo, then W_hi)
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint8_t* act = smem;
  uint8_t* wst = smem + ACT_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(wst + STAGES * STAGE_BYTES);
  uint64_t* full = bars;
  uint64_t* empty = bars + STAGES;
  uint64_t* acc_half = bars + 2 * STAGES;     // [2]: accumulator columns 0..255, 256..511
  uint64_t* act_lo = bars + 2 * STAGES + 2;   // operand columns 0..255 written
  uint64_t* act_hi = bars + 2 * STAGES + 3;   // operand columns 256..511 written
  uint64_t* drain = bars + 2 * STAGES + 4;
  uint64_t* h2l = bars + 2 * STAGES + 5;      // side 1 -> side 0
  uint64_t* l2h = bars + 2 * STAGES + 6;      // side 0 -> side 1
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 7);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* xfer = reinterpret_cast<float*>(smem + ACT_BYTES + STAGES * STAGE_BYTES + BAR_BYTES);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int n = *a.count;
  const int n_tiles = (n + QPT - 1) / QPT;
  if ((int)blockIdx.x >= n_tiles) return;
  uint32_t* masks = reinterpret_cast<uint32_t*>(a.scratch + (size_t)blockIdx.x * kTcAdjScratchPerCta);
  float* g4s = reinterpret_cast<float*>(masks + kMaskWordsPerCta);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(acc_half, 1);
    mbar_init(acc_half + 1, 1);
    mbar_init(act_lo, NUM_EPI * 32);
    mbar_init(act_hi, NUM_EPI * 32);
    mbar_init(drain, 1);
    mbar_init(h2l, NUM_EPI * 16);
    mbar_init(l2h, NUM_EPI * 16);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------ TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_parity[STAGES];
      bool issued[STAGES];
      for (int s = 0; s < STAGES; ++s) issued[s] = false;
      bool ok = true;
      for (int tile = blockIdx.x; ok && tile < n_tiles; tile += gridDim.x) {
        for (int e = 0; ok && e < NUM_ADJ_GEMM; ++e) {
          const CUtensorMap* map = e < 7 ? &fmaps.m[e] : &bmaps.m[13 - e];
          const int nkc = adj_k(e) / BK;
          for (int nh = 0; ok && nh < adj_n(e) / BN; ++nh) {
            for (int kc = 0; kc < NPASS * nkc; ++kc) {
              if (!mbar_wait(empty + stage, phase ^ 1u, abort_flag)) { ok = false; break; }
              mbar_expect_tx(full + stage, STAGE_BYTES);
              // X: the split rows hold [hi | lo]; the lo half comes first
              const int xk = !X ? kc : (kc < nkc ? nkc + kc : kc - nkc);
              tma_load_2d(wst + stage * STAGE_BYTES, map, full + stage, xk * BK, nh * BN);
              issued[stage] = true;
              issued_parity[stage] = phase;
              if (++stage == STAGES) { stage = 0; phase ^= 1u; }
            }
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(a.err, 8);
      }
      for (int s = 0; s < STAGES; ++s) {
        if (!issued[s]) continue;
        const unsigned long long t0 = globaltimer();
        while (!mbar_try_wait(full + s, issued_parity[s]) && globaltimer() - t0 < kTimeoutNs) {
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, lo_phase = 0, hi_phase = 0;
      bool ok = true;
      for (int tile = blockIdx.x; ok && tile < n_tiles; tile += gridDim.x) {
        for (int e = 0; ok && e < NUM_ADJ_GEMM; ++e) {
          const int nkc = adj_k(e) / BK;
          for (int nh = 0; ok && nh < adj_n(e) / BN; ++nh) {
            for (int kc = 0; kc < NPASS * nkc; ++kc) {
              // the operand arrives in two 256-column halves: the first K
              // chunks start as soon as their half is written
              if (nh == 0 && (kc == 0 || (kc == 4 && nkc == 8))) {
                uint64_t* bar = kc == 0 ? act_lo : act_hi;
                uint32_t& ph = kc == 0 ? lo_phase : hi_phase;
                if (!mbar_wait(bar, ph, abort_flag)) { ok = false; break; }
                ph ^= 1u;
                tc_fence_after();
              }
              if (!mbar_wait(full + stage, phase, abort_flag)) { ok = false; break; }
              tc_fence_after();
              const uint32_t a_base = smem_u32(act + (kc % nkc) * CHUNK_BYTES);
              const uint32_t b_base = smem_u32(wst + stage * STAGE_BYTES);
#pragma unroll
              for (int k = 0; k < BK / 16; ++k)
                mma_bf16(tmem + (uint32_t)(nh * BN), sw128_desc(a_base + 32 * k),
                         sw128_desc(b_base + 32 * k), kIdesc, (kc | k) != 0);
              mma_commit(empty + stage);
              if (++stage == STAGES) { stage = 0; phase ^= 1u; }
            }
            if (ok) mma_commit(acc_half + nh);   // this 256-column half is done
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(a.err, 16);
      }
      mma_commit(drain);
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(drain, 0) && globaltimer() - t0 < kTimeoutNs) {
      }
    }
  } else if constexpr (!X) {
    // --------------------------------------------------------- epilogue
    // Warp (lane quadrant q, side s) owns TMEM lanes 32q..32q+31, one probe
    // row each, and of a layer's output columns the chunks col(w): of a
    // 512-wide layer columns s*128 + [0, 128) of each 256-column accumulator
    // half (chunks 0..3 in half 0, 4..7 in half 1), of a 256-wide layer
    // chunks 0..3.  Half 0's results wait in registers while half 1's MMAs,
    // which still read the operand tile, run; then both are written.
    const int ew = warp - 2;
    const int quad = warp & 3;
    const int side = ew >> 2;
    const int row = quad * 32 + lane;
    const uint32_t t_row = tmem + ((uint32_t)(quad * 32) << 16);
    uint32_t acc_phase[2] = {0u, 0u};
    uint32_t h2l_phase = 0, l2h_phase = 0;
    bool ok = true;
    auto col = [&](int w) { return side * 128 + 32 * (w & 3) + 256 * (w >> 2); };
    // mask words of (layer, row, side): word w covers chunk col(w)
    auto mask_ptr = [&](int layer) { return masks + ((size_t)(layer * BM + row) * 2 + side) * 8; };
    auto wait_acc = [&](int h) -> bool {
      if (!mbar_wait(acc_half + h, acc_phase[h], abort_flag)) return false;
      acc_phase[h] ^= 1u;
      tc_fence_after();
      return true;
    };
    auto store_masks = [&](int layer, const uint32_t (&mw)[8]) {
      uint4* mp = reinterpret_cast<uint4*>(mask_ptr(layer));
      mp[0] = make_uint4(mw[0], mw[1], mw[2], mw[3]);
      mp[1] = make_uint4(mw[4], mw[5], mw[6], mw[7]);
    };
    auto store_held = [&](const uint32_t (&held)[4][16]) {
#pragma unroll
      for (int w = 0; w < 4; ++w) store_packed<16>(act, row, col(w), held[w]);
    };
    // operand columns 0..255 (lo) or 256..511 (hi) of this thread written
    auto release = [&](uint64_t* bar) {
      tc_fence_before();
      fence_async_shared();
      mbar_arrive(bar);
    };
    for (int tile = blockIdx.x; ok && tile < n_tiles; tile += gridDim.x) {
      const int j = tile * BM + row;
      const bool valid = j < n;
      float4 pv = valid ? a.pp[j] : make_float4(0.f, 0.f, 0.f, __int_as_float(0));
      const float3 p = make_float3(pv.x, pv.y, pv.z);
      const int shape = __float_as_int(pv.w);
      const float* bf4 = a.bfold4 + (size_t)shape * 512;
      // ---- forward recompute with ReLU masks (the operand tile is free:
      // the previous tile's last GEMM is complete)
      {
        const float* bf = a.bfold0 + (size_t)shape * 512;
        uint32_t mw[8];
        for (int w = 0; w < 8; ++w) {
          const int c = col(w);
          float v[32];
          layer0_32(a.K, bf, c, p, v);
          uint32_t bits = 0;
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            bits |= (v[i] > 0.f ? 1u : 0u) << i;
            v[i] = fmaxf(v[i], 0.f);
          }
          mw[w] = bits;
          store_act32<F16>(act, row, c, v);
          if (w == 3) release(act_lo);
        }
        store_masks(0, mw);
        release(act_hi);
      }
      float head = 0.f;
      for (int g = 0; g < NUM_GEMM; ++g) {
        const bool last = g == NUM_GEMM - 1;
        uint32_t mw[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        // chunk w: bias, ReLU mask, then the head term or the operand values
        auto chunk = [&](int w, float (&v)[32]) {
          const int c = col(w);
          uint32_t r[32];
          tmem_ld32(t_row + (uint32_t)c, r);
          bias32(a.K, g, bf4, c, p, r, v);
          uint32_t bits = 0;
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            bits |= (v[i] > 0.f ? 1u : 0u) << i;
            v[i] = fmaxf(v[i], 0.f);
          }
          mw[w] = bits;
          if (last) head = head32(a.K, c, v, head);
        };
        uint32_t held[4][16];
        if (!wait_acc(0)) { ok = false; break; }
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          float v[32];
          chunk(w, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) held[w][i] = pack16<F16>(v[2 * i], v[2 * i + 1]);
        }
        if (gemm_n(g) == 512) {
          if (!wait_acc(1)) { ok = false; break; }
          if (!last) {
            store_held(held);
            release(act_lo);
          }
          for (int w = 4; w < 8; ++w) {
            float v[32];
            chunk(w, v);
            if (!last) store_act32<F16>(act, row, col(w), v);
          }
          if (!last) release(act_hi);
        } else if (!last) {
          store_held(held);
          release(act_lo);
        }
        store_masks(g + 1, mw);
        tc_fence_before();
      }
      if (!ok) break;
      // ---- head: f, then 1 - f^2 to both sides
      float fval = 0.f, dfs = 0.f;
      if (side == 1) {
        xfer[row] = head;
        mbar_arrive(h2l);
        if (!mbar_wait(l2h, l2h_phase, abort_flag)) { ok = false; break; }
        dfs = xfer[row];
      } else {
        if (!mbar_wait(h2l, h2l_phase, abort_flag)) { ok = false; break; }
        fval = tanhf(head + xfer[row] + __ldg(&a.K->b_head));
        dfs = 1.f - fval * fval;
        xfer[row] = dfs;
        mbar_arrive(l2h);
      }
      h2l_phase ^= 1u;
      l2h_phase ^= 1u;
      // ---- g_7 = (1 - f^2) w_head * mask_7 into the A tile
      {
        const uint32_t* mw = mask_ptr(7);
        for (int w = 0; w < 8; ++w) {
          const int c = col(w);
          const uint32_t bits = mw[w];
          float v[32];
#pragma unroll
          for (int i = 0; i < 32; i += 4) {
            const float4 wh = ldg4(a.K->w_head + c + i);
            v[i + 0] = ((bits >> (i + 0)) & 1u) ? dfs * wh.x : 0.f;
            v[i + 1] = ((bits >> (i + 1)) & 1u) ? dfs * wh.y : 0.f;
            v[i + 2] = ((bits >> (i + 2)) & 1u) ? dfs * wh.z : 0.f;
            v[i + 3] = ((bits >> (i + 3)) & 1u) ? dfs * wh.w : 0.f;
          }
          store_act32<F16>(act, row, c, v);
          if (w == 3) release(act_lo);
        }
        release(act_hi);
      }
      // ---- backward GEMMs for layers 7..1: g_{l-1} = acc * mask_{l-1}
      float gx = 0.f, gy = 0.f, gz = 0.f;
      for (int l = 7; l >= 1; --l) {
        const uint32_t* mw = mask_ptr(l - 1);
        const bool more = l > 1;              // g_{l-1} is the next GEMM's operand
        auto chunk = [&](int w, float (&v)[32]) {
          const int c = col(w);
          uint32_t r[32];
          tmem_ld32(t_row + (uint32_t)c, r);
          const uint32_t bits = mw[w];
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = ((bits >> i) & 1u) ? __uint_as_float(r[i]) : 0.f;
          if (l == 5 || l == 1) {
            // g_4 or g_0: the xyz columns of that layer give grad_p f
            const float(*Wx)[512] = l == 5 ? a.K->wx4 : a.K->wx0;
#pragma unroll
            for (int i = 0; i < 32; i += 4) {
              const float4 x = ldg4(Wx[0] + c + i), y = ldg4(Wx[1] + c + i), z = ldg4(Wx[2] + c + i);
              gx = fmaf(v[i], x.x, fmaf(v[i + 1], x.y, fmaf(v[i + 2], x.z, fmaf(v[i + 3], x.w, gx))));
              gy = fmaf(v[i], y.x, fmaf(v[i + 1], y.y, fmaf(v[i + 2], y.z, fmaf(v[i + 3], y.w, gy))));
              gz = fmaf(v[i], z.x, fmaf(v[i + 1], z.y, fmaf(v[i + 2], z.z, fmaf(v[i + 3], z.w, gz))));
            }
            if (l == 5) {
              float4* dst = reinterpret_cast<float4*>(g4s + (size_t)row * 512 + c);
#pragma unroll
              for (int i = 0; i < 32; i += 4) dst[i / 4] = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
            }
          }
        };
        uint32_t held[4][16];
        if (!wait_acc(0)) { ok = false; break; }
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          float v[32];
          chunk(w, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) held[w][i] = pack16<F16>(v[2 * i], v[2 * i + 1]);
        }
        if (gemm_k(l - 1) == 512) {
          if (!wait_acc(1)) { ok = false; break; }
          if (more) {
            store_held(held);
            release(act_lo);
          }
          for (int w = 4; w < 8; ++w) {
            float v[32];
            chunk(w, v);
            if (more) store_act32<F16>(act, row, col(w), v);
          }
          if (more) release(act_hi);
        } else if (more) {
          store_held(held);
          release(act_lo);
        }
        tc_fence_before();
      }
      if (!ok) break;
      // ---- grad_p f and the probe coefficient
      float coef = 0.f;
      if (side == 1) {
        xfer[row] = gx;
        xfer[BM + row] = gy;
        xfer[2 * BM + row] = gz;
        mbar_arrive(h2l);
        if (!mbar_wait(l2h, l2h_phase, abort_flag)) { ok = false; break; }
        coef = xfer[row];
      } else {
        if (!mbar_wait(h2l, h2l_phase, abort_flag)) { ok = false; break; }
        gx += xfer[row];
        gy += xfer[BM + row];
        gz += xfer[2 * BM + row];
        if (valid) {
          if (a.out4) reinterpret_cast<float4*>(a.out4)[j] = make_float4(fval, gx, gy, gz);
          const float4 q4 = a.pq ? a.pq[j] : make_float4(0.f, 0.f, 0.f, 0.f);
          coef = q4.w;
          if (q4.x != 0.f || q4.y != 0.f || q4.z != 0.f) {
            const float gv = gx * q4.x + gy * q4.y + gz * q4.z;
            const float gn = sqrtf(gx * gx + gy * gy + gz * gz);
            coef = (fabsf(gv) >= 1e-3f * gn && gv != 0.f) ? -q4.w / gv : 0.f;
          }
        }
        xfer[row] = coef;
        mbar_arrive(l2h);
      }
      h2l_phase ^= 1u;
      l2h_phase ^= 1u;
      // ---- sum coef * g_0 and coef * g_4 over the tile's rays per shape
      if (a.accumulate) {
        const uint32_t* m0 = mask_ptr(0);
        unsigned todo = __ballot_sync(0xffffffffu, valid && coef != 0.f);
        while (todo) {
          const int leader = __ffs(todo) - 1;
          const int s = __shfl_sync(0xffffffffu, shape, leader);
          const bool mine = valid && coef != 0.f && shape == s;
          const float cc = mine ? coef : 0.f;
          for (int which = 0; which < 2; ++which) {
            double* dst = (which == 0 ? a.gacc0 : a.gacc4) + (size_t)s * 512;
            for (int w = 0; w < 8; ++w) {
              const int c = col(w);
              float v[32];
              if (which == 0) {
                uint32_t r[32];
                tmem_ld32(t_row + (uint32_t)c, r);
                const uint32_t bits = m0[w];
#pragma unroll
                for (int i = 0; i < 32; ++i)
                  v[i] = ((bits >> i) & 1u) ? cc * __uint_as_float(r[i]) : 0.f;
              } else {
                const float4* src = reinterpret_cast<const float4*>(g4s + (size_t)row * 512 + c);
#pragma unroll
                for (int i = 0; i < 32; i += 4) {
                  const float4 t = src[i / 4];
                  v[i] = cc * t.x; v[i + 1] = cc * t.y; v[i + 2] = cc * t.z; v[i + 3] = cc * t.w;
                }
              }
              const float colsum = warp_column_sum(v, lane);
              if (colsum != 0.f) atomicAdd(dst + c + lane, (double)colsum);
            }
          }
          todo &= ~__ballot_sync(0xffffffffu, mine);
        }
      }
      tc_fence_before();
    }
    if (!ok) {
      *abort_flag = 1;
      atomicOr(a.err, 32);
    }
  } else {
    // ------------------------------------------- epilogue, FP32-class tiles
    // Lane pair (i, i + 16) of quadrant q holds probe 16q + i: lane i the hi
    // row, lane i + 16 the lo row.  After the pair sum each lane owns 16 of a
    // 32-column chunk (`part`) and writes both rows of those columns.  The
    // chunks of a side are the 16-bit epilogue's; the operand is written once
    // a layer's MMAs are all done (no hold-back of half 0, see below).
    const int ew = warp - 2;
    const int quad = warp & 3;
    const int side = ew >> 2;
    const int part = lane >> 4;
    const int jq = quad * 16 + (lane & 15);
    const int rhi = quad * 32 + (lane & 15), rlo = rhi + 16;
    const uint32_t t_row = tmem + ((uint32_t)(quad * 32) << 16);
    constexpr float kGS = (float)(1 << kGradExp), kInvGS = 1.f / (float)(1 << kGradExp);
    uint32_t acc_phase[2] = {0u, 0u};
    uint32_t h2l_phase = 0, l2h_phase = 0;
    bool ok = true;
    float vmax = 0.f;
    auto col = [&](int w) { return side * 128 + 32 * (w & 3) + 256 * (w >> 2); };
    auto mask_ptr = [&](int layer) { return masks + ((size_t)(layer * BM + jq) * 2 + side) * 8; };
    // warp-uniform waits: the lane pairs exchange values after every wait, so
    // a warp never splits on a wait that runs out
    auto wait_all = [&](uint64_t* bar, uint32_t parity) {
      return __all_sync(0xffffffffu, mbar_wait(bar, parity, abort_flag));
    };
    auto wait_acc = [&](int h) -> bool {
      if (!wait_all(acc_half + h, acc_phase[h])) return false;
      acc_phase[h] ^= 1u;
      tc_fence_after();
      return true;
    };
    // hi / lo words of this lane's 16 columns from column cc into both rows
    auto putx = [&](int cc, const uint32_t (&hi)[8], const uint32_t (&lo)[8]) {
      const uint32_t base = smem_u32(act) + (uint32_t)((cc >> 6) * CHUNK_BYTES);
      const int u = (cc & 63) >> 3;
      st_shared_v4(base + swz(rhi, u), hi[0], hi[1], hi[2], hi[3]);
      st_shared_v4(base + swz(rhi, u + 1), hi[4], hi[5], hi[6], hi[7]);
      st_shared_v4(base + swz(rlo, u), lo[0], lo[1], lo[2], lo[3]);
      st_shared_v4(base + swz(rlo, u + 1), lo[4], lo[5], lo[6], lo[7]);
    };
    // the two-term split of 16 signed values (backward operands)
    auto splitx = [&](const float (&v)[16], uint32_t (&hi)[8], uint32_t (&lo)[8]) {
#pragma unroll
      for (int i = 0; i < 16; i += 2) {
        vmax = fmaxf(vmax, fmaxf(fabsf(v[i]), fabsf(v[i + 1])));
        split_pair(v[i], v[i + 1], hi[i / 2], lo[i / 2]);
      }
    };
    // 32-bit mask word of a chunk from the pair's two 16-bit halves
    auto join = [&](uint32_t b16) {
      const uint32_t o = __shfl_xor_sync(0xffffffffu, b16, 16);
      return part ? (o | (b16 << 16)) : (b16 | (o << 16));
    };
    auto store_masks = [&](int layer, const uint32_t (&mw)[8]) {
      if (part == 0) {
        uint4* mp = reinterpret_cast<uint4*>(mask_ptr(layer));
        mp[0] = make_uint4(mw[0], mw[1], mw[2], mw[3]);
        mp[1] = make_uint4(mw[4], mw[5], mw[6], mw[7]);
      }
    };
    // this lane's accumulator columns col(w) + 16 part .. + 15, times s
    auto pair_acc = [&](int w, float s, float (&m)[16]) {
      uint32_t r[32];
      tmem_ld32(t_row + (uint32_t)col(w), r);
      pair_sum16(r, part, m);
#pragma unroll
      for (int i = 0; i < 16; ++i) m[i] *= s;
    };
    auto release = [&](uint64_t* bar) {
      tc_fence_before();
      fence_async_shared();
      mbar_arrive(bar);
    };
    for (int tile = blockIdx.x; ok && tile < n_tiles; tile += gridDim.x) {
      const int j = tile * QPT + jq;
      const bool valid = j < n;
      float4 pv = valid ? a.pp[j] : make_float4(0.f, 0.f, 0.f, __int_as_float(0));
      const float3 p = make_float3(pv.x, pv.y, pv.z);
      const int shape = __float_as_int(pv.w);
      const float* bf4 = a.bfold4 + (size_t)shape * 512;
      float pmin = __builtin_huge_valf();   // smallest |ReLU input| of the probe
      // ---- forward recompute with ReLU masks
      {
        const float* bf = a.bfold0 + (size_t)shape * 512;
        uint32_t mw[8];
        for (int w = 0; w < 8; ++w) {
          const int cc = col(w) + 16 * part;
          float v[16];
          layer0_16(a.K, bf, cc, p, v);
          uint32_t bits = 0;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            bits |= (v[i] > 0.f ? 1u : 0u) << i;
            pmin = fminf(pmin, fabsf(v[i]));
          }
          mw[w] = join(bits);
          uint32_t hi[8], lo[8];
          relu_split16(v, hi, lo, vmax);
          putx(cc, hi, lo);
          if (w == 3) release(act_lo);
        }
        store_masks(0, mw);
        release(act_hi);
      }
      float head = 0.f;
      for (int g = 0; g < NUM_GEMM; ++g) {
        const bool last = g == NUM_GEMM - 1;
        uint32_t mw[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        auto chunk = [&](int w, uint32_t (&hi)[8], uint32_t (&lo)[8]) {
          float m[16], v[16];
          pair_acc(w, 1.f, m);
          const int cc = col(w) + 16 * part;
          affine16(a.K, g, bf4, cc, p, a.inv_scale[g], m, v);
          uint32_t bits = 0;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            bits |= (v[i] > 0.f ? 1u : 0u) << i;
            // (layer 3's padding columns 253..255 are no neurons)
            if (g != 2 || cc + i < 253) pmin = fminf(pmin, fabsf(v[i]));
          }
          mw[w] = join(bits);
          if (last) {
#pragma unroll
            for (int i = 0; i < 16; i += 4) {
              const float4 wh = ldg4(a.K->w_head + cc + i);
              head = fmaf(fmaxf(v[i], 0.f), wh.x,
                          fmaf(fmaxf(v[i + 1], 0.f), wh.y,
                               fmaf(fmaxf(v[i + 2], 0.f), wh.z, fmaf(fmaxf(v[i + 3], 0.f), wh.w, head))));
            }
          } else {
            relu_split16(v, hi, lo, vmax);
          }
        };
        // (FP32-class tiles write straight after the layer's last MMAs: holding
        // half 0 in registers spilled at the 168-register cap and measured no
        // faster)
        if (!wait_acc(0)) { ok = false; break; }
        const bool wide_out = gemm_n(g) == 512;
        if (wide_out && !wait_acc(1)) { ok = false; break; }
        for (int w = 0; w < (wide_out ? 8 : 4); ++w) {
          uint32_t hi[8], lo[8];
          chunk(w, hi, lo);
          if (!last) putx(col(w) + 16 * part, hi, lo);
          if (!last && w == 3) release(act_lo);
        }
        if (!last && wide_out) release(act_hi);
        store_masks(g + 1, mw);
        tc_fence_before();
      }
      if (!ok) break;
      head += __shfl_xor_sync(0xffffffffu, head, 16);
      pmin = fminf(pmin, __shfl_xor_sync(0xffffffffu, pmin, 16));
      // ---- head: f, then 1 - f^2 to both sides (and side 1's pmin to side 0)
      float fval = 0.f, dfs = 0.f;
      if (side == 1) {
        if (part == 0) {
          xfer[jq] = head;
          xfer[BM + jq] = pmin;
        }
        mbar_arrive(h2l);
        if (!wait_all(l2h, l2h_phase)) { ok = false; break; }
        dfs = xfer[jq];
      } else {
        if (!wait_all(h2l, h2l_phase)) { ok = false; break; }
        pmin = fminf(pmin, xfer[BM + jq]);
        fval = tanhf(head + xfer[jq] + __ldg(&a.K->b_head));
        dfs = 1.f - fval * fval;
        __syncwarp();
        if (part == 0) xfer[jq] = dfs;
        mbar_arrive(l2h);
      }
      h2l_phase ^= 1u;
      l2h_phase ^= 1u;
      // ---- g_7 = 2^kGradExp (1 - f^2) w_head * mask_7 into the A tile
      {
        const uint32_t* mw = mask_ptr(7);
        const float ds = dfs * kGS;
        for (int w = 0; w < 8; ++w) {
          const uint32_t bits = mw[w] >> (16 * part);
          const int cc = col(w) + 16 * part;
          float v[16];
#pragma unroll
          for (int i = 0; i < 16; i += 4) {
            const float4 wh = ldg4(a.K->w_head + cc + i);
            v[i + 0] = ((bits >> (i + 0)) & 1u) ? ds * wh.x : 0.f;
            v[i + 1] = ((bits >> (i + 1)) & 1u) ? ds * wh.y : 0.f;
            v[i + 2] = ((bits >> (i + 2)) & 1u) ? ds * wh.z : 0.f;
            v[i + 3] = ((bits >> (i + 3)) & 1u) ? ds * wh.w : 0.f;
          }
          uint32_t hi[8], lo[8];
          splitx(v, hi, lo);
          putx(cc, hi, lo);
          if (w == 3) release(act_lo);
        }
        release(act_hi);
      }
      // ---- backward GEMMs for layers 7..1: g_{l-1} = acc * mask_{l-1}
      float gx = 0.f, gy = 0.f, gz = 0.f;
      for (int l = 7; l >= 1; --l) {
        const uint32_t* mw = mask_ptr(l - 1);
        const bool more = l > 1;
        auto chunk = [&](int w, uint32_t (&hi)[8], uint32_t (&lo)[8]) {
          float m[16];
          pair_acc(w, a.inv_scale[l - 1], m);
          const uint32_t bits = mw[w] >> (16 * part);
          const int cc = col(w) + 16 * part;
          float v[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = ((bits >> i) & 1u) ? m[i] : 0.f;
          if (l == 5 || l == 1) {
            const float(*Wx)[512] = l == 5 ? a.K->wx4 : a.K->wx0;
#pragma unroll
            for (int i = 0; i < 16; i += 4) {
              const float4 x = ldg4(Wx[0] + cc + i), y = ldg4(Wx[1] + cc + i), z = ldg4(Wx[2] + cc + i);
              gx = fmaf(v[i], x.x, fmaf(v[i + 1], x.y, fmaf(v[i + 2], x.z, fmaf(v[i + 3], x.w, gx))));
              gy = fmaf(v[i], y.x, fmaf(v[i + 1], y.y, fmaf(v[i + 2], y.z, fmaf(v[i + 3], y.w, gy))));
              gz = fmaf(v[i], z.x, fmaf(v[i + 1], z.y, fmaf(v[i + 2], z.z, fmaf(v[i + 3], z.w, gz))));
            }
            if (l == 5) {
              float4* dst = reinterpret_cast<float4*>(g4s + (size_t)jq * 512 + cc);
#pragma unroll
              for (int i = 0; i < 16; i += 4) dst[i / 4] = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
            }
          }
          if (more) splitx(v, hi, lo);
        };
        if (!wait_acc(0)) { ok = false; break; }
        const bool wide_out = gemm_k(l - 1) == 512;
        if (wide_out && !wait_acc(1)) { ok = false; break; }
        for (int w = 0; w < (wide_out ? 8 : 4); ++w) {
          uint32_t hi[8], lo[8];
          chunk(w, hi, lo);
          if (more) putx(col(w) + 16 * part, hi, lo);
          if (more && w == 3) release(act_lo);
        }
        if (more && wide_out) release(act_hi);
        tc_fence_before();
      }
      if (!ok) break;
      gx += __shfl_xor_sync(0xffffffffu, gx, 16);
      gy += __shfl_xor_sync(0xffffffffu, gy, 16);
      gz += __shfl_xor_sync(0xffffffffu, gz, 16);
      // ---- grad_p f and the probe coefficient
      float coef = 0.f;
      if (side == 1) {
        if (part == 0) {
          xfer[jq] = gx;
          xfer[BM + jq] = gy;
          xfer[2 * BM + jq] = gz;
        }
        mbar_arrive(h2l);
        if (!wait_all(l2h, l2h_phase)) { ok = false; break; }
        coef = xfer[jq];
      } else {
        if (!wait_all(h2l, h2l_phase)) { ok = false; break; }
        gx = (gx + xfer[jq]) * kInvGS;
        gy = (gy + xfer[BM + jq]) * kInvGS;
        gz = (gz + xfer[2 * BM + jq]) * kInvGS;
        if (valid) {
          if (a.out4 && part == 0) reinterpret_cast<float4*>(a.out4)[j] = make_float4(fval, gx, gy, gz);
          const float4 q4 = a.pq ? a.pq[j] : make_float4(0.f, 0.f, 0.f, 0.f);
          coef = q4.w;
          if (q4.x != 0.f || q4.y != 0.f || q4.z != 0.f) {
            const float gv = gx * q4.x + gy * q4.y + gz * q4.z;
            const float gn = sqrtf(gx * gx + gy * gy + gz * gz);
            coef = (fabsf(gv) >= 1e-3f * gn && gv != 0.f) ? -q4.w / gv : 0.f;
          }
        }
        // a probe whose ReLU masks the FP32-class recompute may have got
        // wrong goes to the FP32 redo list instead (its lane pair agrees)
        int slot = -1;
        if (a.redo_p && part == 0 && valid && pmin < a.redo_tau) {
          slot = atomicAdd(a.redo_count, 1);
          if (slot < a.redo_cap) {
            a.redo_p[slot] = pv;
            a.redo_q[slot] = a.pq ? a.pq[j] : make_float4(0.f, 0.f, 0.f, 0.f);
          } else {
            atomicSub(a.redo_count, 1);   // the count settles at redo_cap
            slot = -1;
          }
        }
        slot = __shfl_sync(0xffffffffu, slot, lane & 15);
        if (slot >= 0) coef = 0.f;
        __syncwarp();
        if (part == 0) xfer[jq] = coef;
        mbar_arrive(l2h);
      }
      h2l_phase ^= 1u;
      l2h_phase ^= 1u;
      // ---- sum coef * g_0 and coef * g_4 over the tile's probes per shape
      // (g carries 2^kGradExp: the coefficient takes it back)
      if (a.accumulate) {
        const uint32_t* m0 = mask_ptr(0);
        const bool live = valid && coef != 0.f;
        unsigned todo = __ballot_sync(0xffffffffu, live);
        while (todo) {
          const int leader = __ffs(todo) - 1;
          const int s = __shfl_sync(0xffffffffu, shape, leader);
          const bool mine = live && shape == s;
          const float cc = mine ? coef * kInvGS : 0.f;
          for (int which = 0; which < 2; ++which) {
            double* dst = (which == 0 ? a.gacc0 : a.gacc4) + (size_t)s * 512;
            for (int w = 0; w < 8; ++w) {
              const int c = col(w);
              float u[16];
              if (which == 0) {
                float m[16];
                pair_acc(w, a.inv_scale[0], m);
                const uint32_t bits = m0[w] >> (16 * part);
#pragma unroll
                for (int i = 0; i < 16; ++i) u[i] = ((bits >> i) & 1u) ? cc * m[i] : 0.f;
              } else {
                const float4* src = reinterpret_cast<const float4*>(g4s + (size_t)jq * 512 + c + 16 * part);
#pragma unroll
                for (int i = 0; i < 16; i += 4) {
                  const float4 t = src[i / 4];
                  u[i] = cc * t.x; u[i + 1] = cc * t.y; u[i + 2] = cc * t.z; u[i + 3] = cc * t.w;
                }
              }
              // the lane's 16 columns in its half of a 32-column row, zeros
              // in the other half: column sums over the warp's 16 probes
              float v[32];
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                v[i] = part ? 0.f : u[i];
                v[16 + i] = part ? u[i] : 0.f;
              }
              const float colsum = warp_column_sum(v, lane);
              if (colsum != 0.f) atomicAdd(dst + c + lane, (double)colsum);
            }
          }
          todo &= ~__ballot_sync(0xffffffffu, mine);
        }
      }
      tc_fence_before();
    }
    if (!ok) {
      *abort_flag = 1;
      atomicOr(a.err, 32);
    }
    if (!(vmax <= 65504.f)) atomicOr(a.err, 64);   // an FP32-class operand overflowed FP16
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

}  // namespace

// Source column in W_l of GEMM column k: the skip layer's GEMM runs over its
// 253 h columns and, in the three padding columns 253..255, its xyz columns,
// so that with the ray point written into those operand columns the tensor
// cores add W_xyz p.  (The adjoint writes zeros there and adds W_xyz p in its
// epilogue; the transposed copy's extra rows meet a zero ReLU mask.)
static int skip_col(int l, int k) { return (l == 4 && k >= 253) ? 253 + 256 + (k - 253) : k; }

// Weights of GEMM layers 1..7 as [N rows][2K cols] fp16: columns 0..K-1 hold
// W_hi, K..2K-1 hold W_lo, both of W * 2^s_l.
dist_status pack_tcx(dist_decoder* d, const float* const* W) {
  auto enc = tensor_map_encoder();
  DIST_CHECK(enc != nullptr, DIST_E_CUDA, "cuTensorMapEncodeTiled entry point not available");
  const int L = 256, Hh = 253;
  for (int g = 0; g < NUM_GEMM; ++g) {
    const int l = g + 1;
    const int N = gemm_n(g), K = gemm_k(g);
    const int n_real = (l == 3) ? Hh : 512;
    const int k_real = (l == 4) ? Hh + 3 : 512;
    const int in_dim = (l == 4) ? Hh + L + 3 : 512;
    float amax = 0.f;
    for (int nn = 0; nn < n_real; ++nn)
      for (int k = 0; k < k_real; ++k)
        amax = std::fmax(amax, std::fabs(W[l][(size_t)nn * in_dim + skip_col(l, k)]));
    // largest power of two with amax * 2^s <= 2^14
    int s = 0;
    if (amax > 0.f) s = (int)std::floor(std::log2(16384.0 / (double)amax));
    s = s < -24 ? -24 : (s > 24 ? 24 : s);
    const float scale = std::ldexp(1.f, s);
    d->tc.x_inv_scale[g] = std::ldexp(1.f, -s);
    std::vector<uint16_t> h((size_t)N * 2 * K, 0);
    for (int nn = 0; nn < n_real; ++nn)
      for (int k = 0; k < k_real; ++k) {
        const float w = W[l][(size_t)nn * in_dim + skip_col(l, k)] * scale;
        const __half hi = __float2half_rn(w);
        const __half lo = __float2half_rn(w - __half2float(hi));
        h[(size_t)nn * 2 * K + k] = *reinterpret_cast<const uint16_t*>(&hi);
        h[(size_t)nn * 2 * K + K + k] = *reinterpret_cast<const uint16_t*>(&lo);
      }
    void* q = nullptr;
    DIST_CUDA_TRY(cudaMalloc(&q, h.size() * sizeof(uint16_t)));
    d->allocations.push_back(q);
    DIST_CUDA_TRY(cudaMemcpy(q, h.data(), h.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    cuuint64_t dims[2] = {(cuuint64_t)(2 * K), (cuuint64_t)N};
    cuuint64_t strides[1] = {(cuuint64_t)(2 * K) * sizeof(uint16_t)};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BN};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&d->tc.xmaps.m[g], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, q, dims, strides, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    DIST_CHECK(r == CUDA_SUCCESS, DIST_E_CUDA, "cuTensorMapEncodeTiled failed (split weights)");
    // 3D view for the latency mode: one copy brings two 64-column chunks of
    // 128 rows (a TMA copy costs ~160 ns whether it moves 16 or 32 KB)
    {
      cuuint64_t d3[3] = {(cuuint64_t)BK, (cuuint64_t)N, (cuuint64_t)(2 * K / BK)};
      cuuint64_t s3[2] = {(cuuint64_t)(2 * K) * sizeof(uint16_t), (cuuint64_t)BK * sizeof(uint16_t)};
      cuuint32_t b3[3] = {(cuuint32_t)BK, (cuuint32_t)(BN / 2), 2};
      cuuint32_t e3[3] = {1, 1, 1};
      r = enc(&d->tc.wxmaps.m[g], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, q, d3, s3, b3, e3,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      DIST_CHECK(r == CUDA_SUCCESS, DIST_E_CUDA, "cuTensorMapEncodeTiled failed (split, 3D)");
    }
    // the transposed split [K rows][2N cols] (W^T_hi | W^T_lo) for the
    // FP32-class adjoint's backward GEMMs
    std::vector<uint16_t> t((size_t)K * 2 * N, 0);
    for (int nn = 0; nn < N; ++nn)
      for (int k = 0; k < K; ++k) {
        t[(size_t)k * 2 * N + nn] = h[(size_t)nn * 2 * K + k];
        t[(size_t)k * 2 * N + N + nn] = h[(size_t)nn * 2 * K + K + k];
      }
    void* qt = nullptr;
    DIST_CUDA_TRY(cudaMalloc(&qt, t.size() * sizeof(uint16_t)));
    d->allocations.push_back(qt);
    DIST_CUDA_TRY(cudaMemcpy(qt, t.data(), t.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    cuuint64_t tdims[2] = {(cuuint64_t)(2 * N), (cuuint64_t)K};
    cuuint64_t tstrides[1] = {(cuuint64_t)(2 * N) * sizeof(uint16_t)};
    r = enc(&d->tc.bxmaps.m[g], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, qt, tdims, tstrides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    DIST_CHECK(r == CUDA_SUCCESS, DIST_E_CUDA, "cuTensorMapEncodeTiled failed (split transpose)");
  }
  return DIST_OK;
}

dist_status pack_tc(dist_decoder* d, const float* const* W, const float* const* b) {
  d->tc.ok = false;
  auto enc = tensor_map_encoder();
  DIST_CHECK(enc != nullptr, DIST_E_CUDA, "cuTensorMapEncodeTiled entry point not available");
  const int L = 256, Hh = 253;   // latent, h-part of the skip input
  const int L0 = d->f32.latent0; // layer-0 code length (L, or longer for a colour decoder)
  {
    // epilogue constants; layer 3 has Hh real outputs, the rest stay 0
    TCConst* c = new TCConst();
    for (int g = 0; g < NUM_GEMM; ++g) {
      const int n_real = (g + 1 == 3) ? Hh : 512;
      for (int j = 0; j < n_real; ++j) c->bias[g][j] = b[g + 1][j];
    }
    for (int j = 0; j < 512; ++j)
      for (int ax = 0; ax < 3; ++ax) {
        c->wx0[ax][j] = W[0][(size_t)j * (L0 + 3) + L0 + ax];
        c->wx4[ax][j] = W[4][(size_t)j * 512 + Hh + L + ax];
      }
    for (int j = 0; j < 512; ++j) c->w_head[j] = W[8][j];
    c->b_head = b[8][0];
    if (d->f32.out_dim == 3) {
      for (int o = 0; o < 3; ++o) {
        for (int j = 0; j < 512; ++j) c->w_c[o][j] = W[8][(size_t)o * 512 + j];
        c->b_c[o] = b[8][o];
      }
    }
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(TCConst));
    if (e == cudaSuccess) {
      d->allocations.push_back(q);
      e = cudaMemcpy(q, c, sizeof(TCConst), cudaMemcpyHostToDevice);
    }
    delete c;
    if (e != cudaSuccess) {
      set_error(std::string("TCConst upload: ") + cudaGetErrorString(e));
      return DIST_E_CUDA;
    }
    d->tc.cst = static_cast<const TCConst*>(q);
  }
  for (int f16 = 0; f16 < 2; ++f16) {
    for (int g = 0; g < NUM_GEMM; ++g) {
      const int l = g + 1;
      const int N = gemm_n(g), K = gemm_k(g);
      std::vector<uint16_t> h((size_t)N * K, 0);   // +0 in both formats
      const int n_real = (l == 3) ? Hh : 512;
      const int k_real = (l == 4) ? Hh + 3 : 512;
      const int in_dim = (l == 4) ? Hh + L + 3 : 512;
      for (int n = 0; n < n_real; ++n)
        for (int k = 0; k < k_real; ++k) {
          const float w = W[l][(size_t)n * in_dim + skip_col(l, k)];
          if (f16) {
            __half v = __float2half_rn(w);
            h[(size_t)n * K + k] = *reinterpret_cast<uint16_t*>(&v);
          } else {
            __nv_bfloat16 v = __float2bfloat16_rn(w);
            h[(size_t)n * K + k] = *reinterpret_cast<uint16_t*>(&v);
          }
        }
      void* p = nullptr;
      DIST_CUDA_TRY(cudaMalloc(&p, h.size() * sizeof(uint16_t)));
      d->allocations.push_back(p);
      DIST_CUDA_TRY(cudaMemcpy(p, h.data(), h.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
      cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)N};
      cuuint64_t strides[1] = {(cuuint64_t)K * sizeof(uint16_t)};
      cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BN};
      cuuint32_t estr[2] = {1, 1};
      CUtensorMap* m = f16 ? &d->tc.maps16.m[g] : &d->tc.maps.m[g];
      CUresult r = enc(m, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                       2, p, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      DIST_CHECK(r == CUDA_SUCCESS, DIST_E_CUDA, "cuTensorMapEncodeTiled failed");
      {
        cuuint64_t d3[3] = {(cuuint64_t)BK, (cuuint64_t)N, (cuuint64_t)(K / BK)};
        cuuint64_t s3[2] = {(cuuint64_t)K * sizeof(uint16_t), (cuuint64_t)BK * sizeof(uint16_t)};
        cuuint32_t b3[3] = {(cuuint32_t)BK, (cuuint32_t)(BN / 2), 2};
        cuuint32_t e3[3] = {1, 1, 1};
        CUtensorMap* mw = f16 ? &d->tc.wmaps16.m[g] : &d->tc.wmaps.m[g];
        r = enc(mw, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, p,
                d3, s3, b3, e3, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        DIST_CHECK(r == CUDA_SUCCESS, DIST_E_CUDA, "cuTensorMapEncodeTiled failed (3D)");
      }
      // the transpose [K rows][N cols] for the adjoint's backward GEMM
      std::vector<uint16_t> t((size_t)K * N, 0);
      for (int nn = 0; nn < N; ++nn)
        for (int k = 0; k < K; ++k) t[(size_t)k * N + nn] = h[(size_t)nn * K + k];
      void* q = nullptr;
      DIST_CUDA_TRY(cudaMalloc(&q, t.size() * sizeof(uint16_t)));
      d->allocations.push_back(q);
      DIST_CUDA_TRY(cudaMemcpy(q, t.data(), t.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
      cuuint64_t tdims[2] = {(cuuint64_t)N, (cuuint64_t)K};
      cuuint64_t tstrides[1] = {(cuuint64_t)N * sizeof(uint16_t)};
      CUtensorMap* mt = f16 ? &d->tc.bmaps16.m[g] : &d->tc.bmaps.m[g];
      r = enc(mt, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, q,
              tdims, tstrides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      DIST_CHECK(r == CUDA_SUCCESS, DIST_E_CUDA, "cuTensorMapEncodeTiled failed (transpose)");
    }
  }
  {
    dist_status xs = pack_tcx(d, W);
    if (xs != DIST_OK) return xs;
  }
  void* e = nullptr;
  DIST_CUDA_TRY(cudaMalloc(&e, sizeof(int)));
  d->allocations.push_back(e);
  DIST_CUDA_TRY(cudaMemset(e, 0, sizeof(int)));
  d->tc.err = static_cast<int*>(e);
  d->tc.wait_ns = kTimeoutNs;
  d->tc.withhold = 0;
  d->tc.ok = true;
  return DIST_OK;
}

template <bool F16, bool COLOR = false>
cudaError_t launch_fused(const dist_decoder* dec, const TCArgs& a, cudaStream_t st) {
  // set once per process (thread-safe static initialisation)
  static const cudaError_t configured = cudaFuncSetAttribute(
      mlp_tc_kernel<F16, COLOR>, cudaFuncAttributeMaxDynamicSharedMemorySize, FWD_SMEM_BYTES);
  if (configured != cudaSuccess) return configured;
  const TCMaps& maps = F16 ? dec->tc.maps16 : dec->tc.maps;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(num_sms());
  cfg.blockDim = dim3(FWD_THREADS);
  cfg.dynamicSmemBytes = FWD_SMEM_BYTES;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // (dec->tc.maps16 also serves the FP16-stage tiles of a BF16 march)
  cudaError_t e = cudaLaunchKernelEx(&cfg, mlp_tc_kernel<F16, COLOR>, maps, dec->tc.xmaps,
                                     dec->tc.maps16, a);
  count_launch(1);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t mlp_tc_fused(const dist_decoder* dec, const RowSrc& src16, float* f16out,
                         const RowSrc& srcx, float* fxout, const float* bfold0,
                         const float* bfolds, cudaStream_t st, bool f16,
                         const StepFuse* step, const RowSrc* srcm, float* fmout) {
  if (!dec->tc.ok) return cudaErrorNotSupported;
  TCArgs a;
  a.K = dec->tc.cst;
  a.bfold0 = bfold0;
  a.bfold4 = bfolds;
  a.src[0] = src16;
  a.src[1] = srcx;
  a.src[2] = srcm ? *srcm : RowSrc{};     // no FP16-stage list: count 0
  a.fout[0] = f16out;
  a.fout[1] = fxout;
  a.fout[2] = fmout;
  a.err = dec->tc.err;
  for (int g = 0; g < NUM_GEMM; ++g) a.inv_scale[g] = dec->tc.x_inv_scale[g];
  a.cpart = nullptr;
  a.fuse_step = step ? 1 : 0;
  if (step) a.step = *step;
  else memset(&a.step, 0, sizeof(a.step));
  // with a fused step and latency-mode scratch, both kernels are launched;
  // each decides from the list lengths on the device which one decodes
  a.wide_tiles = (step && step->wide) ? tc_wide_max_tiles() : 0;
  a.wait_ns = dec->tc.wait_ns;
  a.withhold = dec->tc.withhold;
  cudaError_t e = f16 ? launch_fused<true>(dec, a, st) : launch_fused<false>(dec, a, st);
  if (e != cudaSuccess || a.wide_tiles <= 0) return e;
  return mlp_tc_wide(dec, src16, f16out, srcx, fxout, bfold0, bfolds, st, f16, step, step->wide,
                     srcm, fmout);
}

cudaError_t mlp_tc_color(const dist_decoder* dec, const RowSrc& src, const float* bfold0,
                         const float* bfolds, float* scratch, float* cpart, cudaStream_t st,
                         bool f16) {
  if (!dec->tc.ok) return cudaErrorNotSupported;
  TCArgs a;
  memset(&a, 0, sizeof(a));
  a.K = dec->tc.cst;
  a.bfold0 = bfold0;
  a.bfold4 = bfolds;
  a.src[0] = src;
  a.fout[0] = scratch;
  a.err = dec->tc.err;
  for (int g = 0; g < NUM_GEMM; ++g) a.inv_scale[g] = dec->tc.x_inv_scale[g];
  a.cpart = cpart;
  a.wait_ns = dec->tc.wait_ns;
  a.withhold = dec->tc.withhold;
  return f16 ? launch_fused<true, true>(dec, a, st) : launch_fused<false, true>(dec, a, st);
}

cudaError_t mlp_tc_forward(const dist_decoder* dec, const RowSrc& src, const float* bfold0,
                           const float* bfolds, float* fout, cudaStream_t st, bool f16) {
  RowSrc none{};
  return mlp_tc_fused(dec, src, fout, none, nullptr, bfold0, bfolds, st, f16);
}

cudaError_t mlp_tcx_forward(const dist_decoder* dec, const RowSrc& src, const float* bfold0,
                            const float* bfolds, float* fout, cudaStream_t st) {
  RowSrc none{};
  return mlp_tc_fused(dec, none, nullptr, src, fout, bfold0, bfolds, st, false);
}

namespace {

template <bool F16, bool X>
cudaError_t launch_adjoint(const TCMaps& fmaps, const TCMaps& bmaps, const TCAdjArgs& a,
                           cudaStream_t st) {
  // set once per process and variant (thread-safe static initialisation)
  static const cudaError_t configured = cudaFuncSetAttribute(
      mlp_tc_adj_kernel<F16, X>, cudaFuncAttributeMaxDynamicSharedMemorySize, ADJ_SMEM_BYTES);
  if (configured != cudaSuccess) return configured;
  prof_mlp_begin(st, 2);
  mlp_tc_adj_kernel<F16, X><<<num_sms(), THREADS, ADJ_SMEM_BYTES, st>>>(fmaps, bmaps, a);
  prof_mlp_end(st);
  count_launch(1);
  return cudaGetLastError();
}

TCAdjArgs adj_args(const dist_decoder* dec, const float4* pp, const float4* pq, const int* count,
                   const float* bfold0, const float* bfolds, float* out4, double* gacc0,
                   double* gaccs, int accumulate, void* scratch) {
  TCAdjArgs a;
  a.K = dec->tc.cst;
  a.bfold0 = bfold0;
  a.bfold4 = bfolds;
  a.pp = pp;
  a.pq = pq;
  a.count = count;
  a.out4 = out4;
  a.gacc0 = gacc0;
  a.gacc4 = gaccs;
  a.accumulate = accumulate;
  a.scratch = static_cast<uint8_t*>(scratch);
  a.err = dec->tc.err;
  for (int g = 0; g < NUM_GEMM; ++g) a.inv_scale[g] = dec->tc.x_inv_scale[g];
  a.redo_p = nullptr;
  a.redo_q = nullptr;
  a.redo_count = nullptr;
  a.redo_cap = 0;
  a.redo_tau = 0.f;
  return a;
}

}  // namespace

cudaError_t mlp_tc_adjoint(const dist_decoder* dec, const float4* pp, const float4* pq,
                           const int* count, const float* bfold0, const float* bfolds,
                           float* out4, double* gacc0, double* gaccs, int accumulate,
                           void* scratch, cudaStream_t st, bool f16) {
  if (!dec->tc.ok) return cudaErrorNotSupported;
  const TCAdjArgs a = adj_args(dec, pp, pq, count, bfold0, bfolds, out4, gacc0, gaccs,
                               accumulate, scratch);
  return f16 ? launch_adjoint<true, false>(dec->tc.maps16, dec->tc.bmaps16, a, st)
             : launch_adjoint<false, false>(dec->tc.maps, dec->tc.bmaps, a, st);
}

cudaError_t mlp_tcx_adjoint(const dist_decoder* dec, const float4* pp, const float4* pq,
                            const int* count, const float* bfold0, const float* bfolds,
                            float* out4, double* gacc0, double* gaccs, int accumulate,
                            void* scratch, cudaStream_t st, const RedoList* redo) {
  if (!dec->tc.ok) return cudaErrorNotSupported;
  TCAdjArgs a = adj_args(dec, pp, pq, count, bfold0, bfolds, out4, gacc0, gaccs, accumulate,
                         scratch);
  if (redo) {
    a.redo_p = redo->p;
    a.redo_q = redo->q;
    a.redo_count = redo->count;
    a.redo_cap = redo->cap;
    a.redo_tau = redo->tau;
  }
  return launch_adjoint<true, true>(dec->tc.xmaps, dec->tc.bxmaps, a, st);
}

}  // namespace dist
