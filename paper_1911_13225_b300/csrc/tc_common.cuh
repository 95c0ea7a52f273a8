// Internal: tcgen05 / TMA / mbarrier helpers and epilogue pieces shared by the
// tensor-core decoder kernels (mlp_tc.cu, mlp_tc_wide.cu).
#pragma once

#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace dist {
namespace {

constexpr int BM = 128;                       // rows per tile == TMEM lanes
constexpr int BN = 256;                       // N per stage and per MMA
constexpr int BK = 64;                        // K per stage: one 128-byte bf16 row
constexpr int STAGES = 3;
constexpr int NUM_EPI = 8;                    // epilogue warps
constexpr int THREADS = 64 + NUM_EPI * 32;
constexpr int ACT_BYTES = BM * 512 * 2;       // 8 K-chunks of [128 x 64] bf16
constexpr int CHUNK_BYTES = BM * BK * 2;      // 16 KB
constexpr int STAGE_BYTES = BN * BK * 2;      // 32 KB
constexpr int NUM_GEMM = 7;                   // layers 1..7
constexpr int BAR_BYTES = 256;
constexpr int SMEM_BYTES =
    1024 + ACT_BYTES + STAGES * STAGE_BYTES + BAR_BYTES + (NUM_EPI / 4 - 1) * BM * 4;
constexpr unsigned long long kTimeoutNs = 1000000000ull;
// Forward kernels: 16 epilogue warps, four per TMEM lane quadrant.
constexpr int FWD_EPI = 16;
constexpr int FWD_STEP_WARPS = 2;   // march step update of a tile's rows
constexpr int FWD_THREADS = 64 + FWD_EPI * 32 + FWD_STEP_WARPS * 32;
constexpr int FWD_GRPS = FWD_EPI / 4;
constexpr int FWD_SMEM_BYTES =
    1024 + ACT_BYTES + STAGES * STAGE_BYTES + BAR_BYTES + (FWD_GRPS - 1) * BM * 4;
static_assert(FWD_SMEM_BYTES <= 232448, "forward kernel shared memory");

// Programmatic dependent launch: wait for the previous grid in the stream
// (complete, its writes visible); let the next grid start launching.
__device__ __forceinline__ void grid_dep_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void grid_dep_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Instruction descriptor, kind::f16: D fp32 (bits 4-5 = 1), A bf16 (7-9 = 1),
// B bf16 (10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
// With F16 the operand formats (bits 7-9, 10-12) are 0 = fp16 instead of bf16.
template <bool F16>
__host__ __device__ constexpr uint32_t instr_desc() {
  return (1u << 4) | ((F16 ? 0u : 1u) << 7) | ((F16 ? 0u : 1u) << 10) |
         ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

// The same for a runtime operand format and M.
__host__ __device__ constexpr uint32_t instr_desc_m(bool f16, int m) {
  return (1u << 4) | ((f16 ? 0u : 1u) << 7) | ((f16 ? 0u : 1u) << 10) |
         ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__host__ __device__ constexpr int gemm_k(int g) { return g == 3 ? 256 : 512; }
__host__ __device__ constexpr int gemm_n(int g) { return g == 2 ? 256 : 512; }

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with `parity` to complete; false after
// `limit_ns` or when another role has aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          unsigned long long limit_ns = kTimeoutNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63) == 0) {
      if (*abort_flag) return false;
      if (globaltimer() - t0 > limit_ns) return false;
    }
  }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// This warp's 32 TMEM lanes x 32 consecutive fp32 columns.  The wait is tied
// to the destination registers so that no use of them is scheduled before it.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]),
                 "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                 "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]),
                 "+r"(r[30]), "+r"(r[31]));
}

// This warp's 32 TMEM lanes x 16 consecutive fp32 columns.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]));
}

// ---- clusters

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_index() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
// shared::cluster address of the same shared variable in CTA `rank`
__device__ __forceinline__ uint32_t map_rank(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_acq_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait with cluster-scope acquire (barriers other CTAs arrive on).
__device__ __forceinline__ bool mbar_wait_cl(uint64_t* bar, uint32_t parity,
                                             volatile int* abort_flag,
                                             unsigned long long limit_ns = kTimeoutNs) {
  if (mbar_try_wait_acq_cluster(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait_acq_cluster(bar, parity)) return true;
    if ((it & 63) == 0) {
      if (*abort_flag) return false;
      if (globaltimer() - t0 > limit_ns) return false;
    }
  }
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), version 1 (bit 46), swizzle mode 2 (bits 61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Byte offset of bf16 column group u (8 columns = 16 bytes) of row r inside a
// 128B-swizzled [128 x 64] chunk.
__device__ __forceinline__ uint32_t swz(int r, int u) {
  return (uint32_t)(r * 128 + ((u ^ (r & 7)) << 4));
}

// Two floats rounded to the operand type (nearest even), packed.
template <bool F16>
__device__ __forceinline__ uint32_t pack16(float a, float b) {
  if constexpr (F16) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  } else {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
}

// pack16 with the operand type chosen at run time (uniform over a warp).
__device__ __forceinline__ uint32_t pack16r(bool f16, float a, float b) {
  return f16 ? pack16<true>(a, b) : pack16<false>(a, b);
}

// Store 32 consecutive activations (columns c..c+31, c % 32 == 0) of row r.
template <bool F16>
__device__ __forceinline__ void store_act32(uint8_t* act, int r, int c, const float (&v)[32]) {
  uint8_t* chunk = act + (c >> 6) * CHUNK_BYTES;
  const int u0 = (c & 63) >> 3;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t off = swz(r, u0 + q);
    const uint32_t a = pack16<F16>(v[8 * q + 0], v[8 * q + 1]);
    const uint32_t b = pack16<F16>(v[8 * q + 2], v[8 * q + 3]);
    const uint32_t cc = pack16<F16>(v[8 * q + 4], v[8 * q + 5]);
    const uint32_t d = pack16<F16>(v[8 * q + 6], v[8 * q + 7]);
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(smem_u32(chunk + off)), "r"(a),
                 "r"(b), "r"(cc), "r"(d)
                 : "memory");
  }
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
               "r"(d)
               : "memory");
}

// Store NP packed pairs (columns c..c+2*NP-1, c % 8 == 0) of row r.
template <int NP>
__device__ __forceinline__ void store_packed(uint8_t* act, int r, int c, const uint32_t (&h)[NP]) {
#pragma unroll
  for (int q = 0; q < NP / 4; ++q) {
    const int col = c + 8 * q;
    const uint32_t off = (uint32_t)((col >> 6) * CHUNK_BYTES) + swz(r, (col & 63) >> 3);
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(smem_u32(act + off)),
                 "r"(h[4 * q]), "r"(h[4 * q + 1]), "r"(h[4 * q + 2]), "r"(h[4 * q + 3])
                 : "memory");
  }
}

__device__ __forceinline__ float4 ldg4(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}

// v = relu(Wx0 p + b0'), columns c..c+31 of layer 0
__device__ __forceinline__ void layer0_32(const TCConst* K, const float* bf, int c, const float3& p,
                                          float (&v)[32]) {
#pragma unroll
  for (int i = 0; i < 32; i += 4) {
    const float4 b = ldg4(bf + c + i);
    const float4 x = ldg4(K->wx0[0] + c + i);
    const float4 y = ldg4(K->wx0[1] + c + i);
    const float4 z = ldg4(K->wx0[2] + c + i);
    v[i + 0] = fmaxf(fmaf(x.x, p.x, fmaf(y.x, p.y, fmaf(z.x, p.z, b.x))), 0.f);
    v[i + 1] = fmaxf(fmaf(x.y, p.x, fmaf(y.y, p.y, fmaf(z.y, p.z, b.y))), 0.f);
    v[i + 2] = fmaxf(fmaf(x.z, p.x, fmaf(y.z, p.y, fmaf(z.z, p.z, b.z))), 0.f);
    v[i + 3] = fmaxf(fmaf(x.w, p.x, fmaf(y.w, p.y, fmaf(z.w, p.z, b.w))), 0.f);
  }
}

// v = accumulator + bias of GEMM layer g (the skip layer: folded bias, plus
// Wx4 p when `xyz`; the forward kernel has the tensor cores add Wx4 p),
// columns c..c+W-1.
template <int W>
__device__ __forceinline__ void bias_cols(const TCConst* K, int g, const float* bf4, int c,
                                          const float3& p, const uint32_t (&r)[W], float (&v)[W],
                                          bool xyz = true) {
  if (g == 3 && !xyz) {
#pragma unroll
    for (int i = 0; i < W; i += 4) {
      const float4 b = ldg4(bf4 + c + i);
      v[i + 0] = __uint_as_float(r[i + 0]) + b.x;
      v[i + 1] = __uint_as_float(r[i + 1]) + b.y;
      v[i + 2] = __uint_as_float(r[i + 2]) + b.z;
      v[i + 3] = __uint_as_float(r[i + 3]) + b.w;
    }
  } else if (g == 3) {
#pragma unroll
    for (int i = 0; i < W; i += 4) {
      const float4 b = ldg4(bf4 + c + i);
      const float4 x = ldg4(K->wx4[0] + c + i);
      const float4 y = ldg4(K->wx4[1] + c + i);
      const float4 z = ldg4(K->wx4[2] + c + i);
      v[i + 0] = fmaf(x.x, p.x, fmaf(y.x, p.y, fmaf(z.x, p.z, __uint_as_float(r[i + 0]) + b.x)));
      v[i + 1] = fmaf(x.y, p.x, fmaf(y.y, p.y, fmaf(z.y, p.z, __uint_as_float(r[i + 1]) + b.y)));
      v[i + 2] = fmaf(x.z, p.x, fmaf(y.z, p.y, fmaf(z.z, p.z, __uint_as_float(r[i + 2]) + b.z)));
      v[i + 3] = fmaf(x.w, p.x, fmaf(y.w, p.y, fmaf(z.w, p.z, __uint_as_float(r[i + 3]) + b.w)));
    }
  } else {
    const float* bias = K->bias[g];
#pragma unroll
    for (int i = 0; i < W; i += 4) {
      const float4 b = ldg4(bias + c + i);
      v[i + 0] = __uint_as_float(r[i + 0]) + b.x;
      v[i + 1] = __uint_as_float(r[i + 1]) + b.y;
      v[i + 2] = __uint_as_float(r[i + 2]) + b.z;
      v[i + 3] = __uint_as_float(r[i + 3]) + b.w;
    }
  }
}
__device__ __forceinline__ void bias32(const TCConst* K, int g, const float* bf4, int c,
                                       const float3& p, const uint32_t (&r)[32], float (&v)[32],
                                       bool xyz = true) {
  bias_cols<32>(K, g, bf4, c, p, r, v, xyz);
}
__device__ __forceinline__ void bias16(const TCConst* K, int g, const float* bf4, int c,
                                       const float3& p, const uint32_t (&r)[16], float (&v)[16]) {
  bias_cols<16>(K, g, bf4, c, p, r, v);
}

__device__ __forceinline__ float head32(const TCConst* K, int c, const float (&v)[32], float acc) {
#pragma unroll
  for (int i = 0; i < 32; i += 4) {
    const float4 w = ldg4(K->w_head + c + i);
    acc = fmaf(v[i], w.x, fmaf(v[i + 1], w.y, fmaf(v[i + 2], w.z, fmaf(v[i + 3], w.w, acc))));
  }
  return acc;
}

// ---- FP32-class (two-term FP16 split) epilogue pieces

// v = m * scale + bias of GEMM layer g (the skip layer: folded bias, plus
// Wx4 p when `xyz`), 16 columns from c.
__device__ __forceinline__ void affine16(const TCConst* K, int g, const float* bf4, int c,
                                         const float3& p, float scale, const float (&m)[16],
                                         float (&v)[16], bool xyz = true) {
  if (g == 3 && !xyz) {
#pragma unroll
    for (int i = 0; i < 16; i += 4) {
      const float4 b = ldg4(bf4 + c + i);
      v[i + 0] = fmaf(m[i + 0], scale, b.x);
      v[i + 1] = fmaf(m[i + 1], scale, b.y);
      v[i + 2] = fmaf(m[i + 2], scale, b.z);
      v[i + 3] = fmaf(m[i + 3], scale, b.w);
    }
  } else if (g == 3) {
#pragma unroll
    for (int i = 0; i < 16; i += 4) {
      const float4 b = ldg4(bf4 + c + i);
      const float4 x = ldg4(K->wx4[0] + c + i);
      const float4 y = ldg4(K->wx4[1] + c + i);
      const float4 z = ldg4(K->wx4[2] + c + i);
      v[i + 0] = fmaf(x.x, p.x, fmaf(y.x, p.y, fmaf(z.x, p.z, fmaf(m[i + 0], scale, b.x))));
      v[i + 1] = fmaf(x.y, p.x, fmaf(y.y, p.y, fmaf(z.y, p.z, fmaf(m[i + 1], scale, b.y))));
      v[i + 2] = fmaf(x.z, p.x, fmaf(y.z, p.y, fmaf(z.z, p.z, fmaf(m[i + 2], scale, b.z))));
      v[i + 3] = fmaf(x.w, p.x, fmaf(y.w, p.y, fmaf(z.w, p.z, fmaf(m[i + 3], scale, b.w))));
    }
  } else {
    const float* bias = K->bias[g];
#pragma unroll
    for (int i = 0; i < 16; i += 4) {
      const float4 b = ldg4(bias + c + i);
      v[i + 0] = fmaf(m[i + 0], scale, b.x);
      v[i + 1] = fmaf(m[i + 1], scale, b.y);
      v[i + 2] = fmaf(m[i + 2], scale, b.z);
      v[i + 3] = fmaf(m[i + 3], scale, b.w);
    }
  }
}

// Layer 0 pre-activation, 16 columns from c: Wx0 p + b0'.
__device__ __forceinline__ void layer0_16(const TCConst* K, const float* bf, int c, const float3& p,
                                          float (&v)[16]) {
#pragma unroll
  for (int i = 0; i < 16; i += 4) {
    const float4 b = ldg4(bf + c + i);
    const float4 x = ldg4(K->wx0[0] + c + i);
    const float4 y = ldg4(K->wx0[1] + c + i);
    const float4 z = ldg4(K->wx0[2] + c + i);
    v[i + 0] = fmaf(x.x, p.x, fmaf(y.x, p.y, fmaf(z.x, p.z, b.x)));
    v[i + 1] = fmaf(x.y, p.x, fmaf(y.y, p.y, fmaf(z.y, p.z, b.y)));
    v[i + 2] = fmaf(x.z, p.x, fmaf(y.z, p.y, fmaf(z.z, p.z, b.z)));
    v[i + 3] = fmaf(x.w, p.x, fmaf(y.w, p.y, fmaf(z.w, p.z, b.w)));
  }
}

// ReLU, then the two-term FP16 split of 16 values, packed in pairs.
// `vmax` tracks the largest activation (an FP16 overflow check).
__device__ __forceinline__ void relu_split16(float (&v)[16], uint32_t (&hi)[8], uint32_t (&lo)[8],
                                             float& vmax) {
#pragma unroll
  for (int i = 0; i < 16; i += 2) {
    const float a = fmaxf(v[i], 0.f), b = fmaxf(v[i + 1], 0.f);
    vmax = fmaxf(vmax, fmaxf(a, b));
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    hi[i / 2] = *reinterpret_cast<const uint32_t*>(&h);
    lo[i / 2] = *reinterpret_cast<const uint32_t*>(&l);
  }
}

// The two-term FP16 split of a pair without ReLU (operand columns that carry
// the ray point).
__device__ __forceinline__ void split_pair(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(a, b);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Sum of the hi-row and lo-row accumulators of one query for the 16 columns
// this lane owns in a 32-column chunk: lanes i and i + 16 exchange the half
// of the chunk the other one keeps (16 shuffles).
__device__ __forceinline__ void pair_sum16(const uint32_t (&r)[32], int part, float (&m)[16]) {
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const float keep = __uint_as_float(part ? r[16 + i] : r[i]);
    const float send = __uint_as_float(part ? r[i] : r[16 + i]);
    m[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
}

// Head term w_head . relu(acc + bias) of one 32-column chunk at column c of
// the last GEMM layer, summed from zero in a fixed order, for the row of this
// thread (16-bit tile) or of this lane pair (FP32-class tile: each lane sums
// its 16 columns, then the pair adds the two halves).  The forward kernels
// add these chunk sums in one fixed order, so a row's f does not depend on
// which kernel or batch decoded it.
template <bool F16>
__device__ __forceinline__ float head_chunk_sum(const TCConst* K, bool kx, const float* bf4,
                                                const float3& pp, int c, int part, float scale,
                                                const uint32_t (&r)[32]) {
  if (!kx) {
    float v[32];
    bias32(K, NUM_GEMM - 1, bf4, c, pp, r, v);
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = fmaxf(v[i], 0.f);
    return head32(K, c, v, 0.f);
  }
  float m[16], v[16];
  pair_sum16(r, part, m);
  const int cc = c + 16 * part;
  affine16(K, NUM_GEMM - 1, bf4, cc, pp, scale, m, v);
  float acc = 0.f;
#pragma unroll
  for (int i = 0; i < 16; i += 4) {
    const float4 w = ldg4(K->w_head + cc + i);
    acc = fmaf(fmaxf(v[i], 0.f), w.x,
               fmaf(fmaxf(v[i + 1], 0.f), w.y,
                    fmaf(fmaxf(v[i + 2], 0.f), w.z, fmaf(fmaxf(v[i + 3], 0.f), w.w, acc))));
  }
  // part 0 holds the chunk's first 16 columns: first + second, in both lanes
  const float other = __shfl_xor_sync(0xffffffffu, acc, 16);
  return part ? other + acc : acc + other;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point query.
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace
}  // namespace dist
