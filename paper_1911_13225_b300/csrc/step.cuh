// Internal: the per-ray step/converge update of the march (Alg. 1, Sec. 3.2,
// Eq. 1), shared by the step kernel and the decoder kernel's epilogue.
#pragma once

#include "common.cuh"

namespace dist {

constexpr float kInf = __builtin_huge_valf();

struct TraceArgs {
  const CamDev* cams;
  int n_cams;
  long long n_pix;
  long long pix0;       // first pixel index handled (0 for a whole batch)
  int cam_fixed;        // >= 0: every pixel belongs to this camera
  float radius;
  int K;
  float eps, alpha, eps_bf16;
  float eps_mid;        // BF16 march: > 0 = rays hand over to FP16 queries (list 2)
                        // at |f| < eps_bf16, and from there to FP32-class queries
                        // at |f| < eps_mid; 0 = straight to FP32-class
  int max_steps;
  float alpha_fp32;     // step factor of FP32-list rays
  int refine;           // refine_steps for a tensor-core march, else 0
  int secant;           // secant rule for FP32-list rays of a tensor-core march
  dist_trace_out o;
  float4* st;
  float4* dir;
  int* fq;              // FP32 queries per ray after the low-precision phase
  float* fprev;         // previous low-precision sample (then FP32-class, secant)
  float* dprev;         // distance of the previous FP32-class sample (secant)
  int c2f;              // coarse-to-fine trace: o.status holds -1 / -2 for a
                        // ray marching in list 0 / list 1 until it ends
  int c2f_start;        // the code of a ray that starts marching
  int last;             // coarse-to-fine: this is the last march iteration, so
                        // a ray that started late also ends here (MAX_STEPS)
};

// The step update applied by the decoder kernel itself: the thread that
// computes a ray's f updates the ray and appends it to the next step's list.
struct StepFuse {
  TraceArgs t;
  int* out[3];                   // next step's lists (0: 16-bit, 1: FP32-class,
                                 // 2: FP16 stage of a BF16 march)
  int* cnt_out[3];               // their append counters
  unsigned long long* queries;   // per-list query counters, or null
  uint8_t* wide;                 // latency-mode scratch (tc_wide_scratch_bytes()), or
                                 // null: every launch on the one-tile-per-SM kernel
  unsigned long long* seq_flag;  // with `wide`: device word through which mlp_tc_kernel
  unsigned long long seq;        // hands this step's inputs to mlp_tc_wide_kernel
                                 // (seq: distinct per fused step on this word)
};

// Tiles of a fused step that mlp_tc_wide_kernel decodes: the first ones in
// tile order (FP32-class tiles first), mlp_tc_kernel the rest.  All of them
// when they fit on the resident clusters (wt); the FP32-class tiles alone
// (a four-SM cluster each) when those fit too and the other tiles take one
// round on the SMs left over (4 t1 + (n_tiles - t1) <= nsm): the two kernels
// then run side by side; else none.  Both kernels make this decision from
// the same counts.
__host__ __device__ __forceinline__ int wide_share(int n_tiles, int t1, int wt, int nsm) {
  if (wt <= 0) return 0;
  if (n_tiles <= wt) return n_tiles;
  if (t1 > 0 && t1 <= wt && 3 * t1 + n_tiles <= nsm) return t1;
  return 0;
}

// Release / acquire of the step sequence word (gpu scope).
__device__ __forceinline__ void seq_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long seq_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Warp-aggregated append over the lanes in `active`: one atomic per warp.
__device__ __forceinline__ int warp_append(bool pred, int* counter,
                                           unsigned active = 0xffffffffu) {
  const unsigned m = __ballot_sync(active, pred);
  if (m == 0) return -1;
  const int leader = __ffs(m) - 1;
  int base = 0;
  if (lane_id() == leader) base = atomicAdd(counter, __popc(m));
  base = __shfl_sync(active, base, leader);
  return pred ? base + __popc(m & ((1u << lane_id()) - 1u)) : -1;
}

// The per-ray state a step reads: loaded ahead of the query result where
// the caller can (the fused step), right before it otherwise.
struct RayState {
  float4 s;                // (d, t_in, t_out, camera bits)
  int steps;
  float fm[kMaxK], dm[kMaxK];
  int fq;
  float fprev, dprev, dirw;
};

__device__ __forceinline__ void load_ray(const TraceArgs& a, int list, int i, RayState& r) {
  r.s = a.st[i];
  r.steps = a.o.steps[i];
  const float* fm = a.o.f_min + (size_t)i * a.K;
  const float* dm = a.o.d_min + (size_t)i * a.K;
#pragma unroll
  for (int k = 0; k < kMaxK; ++k) {
    r.fm[k] = k < a.K ? fm[k] : kInf;
    r.dm[k] = k < a.K ? dm[k] : 0.f;
  }
  const bool ref = list == 1 && (a.refine > 0 || a.secant);
  r.fq = ref ? a.fq[i] : 0;
  r.fprev = (list != 1 || a.secant) ? a.fprev[i] : 0.f;
  r.dprev = (list == 1 && a.secant) ? a.dprev[i] : 0.f;
  r.dirw = a.dir[i].w;
}

// One query's update of ray i (list 0: low-precision, 1: FP32 / FP32-class,
// 2: the FP16 stage of a BF16 march) with decoder value f and its state r:
// step count, the k smallest |f| (silhouette and the paper's gradient),
// hand-over, convergence (|f| < eps: hit at the unit final step d + f), the
// aggressive step d += alpha f, leaving the bounding sphere and the step
// budget.  Returns the list the ray continues in, or -1.
__device__ __forceinline__ int apply_step(const TraceArgs& a, int list, int i, float f,
                                          const RayState& r) {
  int keep = -1;
  float4 s = r.s;
  const float d = s.x;
  const int steps = r.steps + 1;
  a.o.steps[i] = steps;
  const float af = fabsf(f);
  const bool low = list != 1;             // a 16-bit sample (BF16, or FP16)
  const float track = low ? fmaxf(af, a.eps) : af;
  // k smallest |f|, ascending; changed entries are written back
  float fm0 = r.fm[0];
  {
    float* fm = a.o.f_min + (size_t)i * a.K;
    float* dm = a.o.d_min + (size_t)i * a.K;
    float cf = copysignf(track, f), cd = d;
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) {
      if (k < a.K && fabsf(cf) < fabsf(r.fm[k])) {
        const float of = r.fm[k], od = r.dm[k];
        if (k == 0) fm0 = cf;
        fm[k] = cf; dm[k] = cd;
        cf = of; cd = od;
      }
    }
  }
  int outcome = -1;   // -1 keep marching
  float dn = d;
  bool accepted = false;
  int q = 0;
  if (list == 1 && (a.refine > 0 || a.secant)) {
    // FP32 refinement after a tensor-core march: after `refine` FP32
    // queries a ray within 4 eps_bf16 of the surface is accepted
    q = r.fq + 1;
    a.fq[i] = q;
    accepted = a.refine > 0 && q >= a.refine && af >= a.eps && af < 4.f * a.eps_bf16;
  }
  bool crossed = false;
  const float eps_lo = list == 2 ? a.eps_mid : a.eps_bf16;
  if (low) {
    // a low-precision march that steps across the surface close to it
    // hands over to FP32 even if its noisy |f| never drops below its
    // threshold
    const float fp = r.fprev;
    a.fprev[i] = f;
    crossed = fp != 0.f && ((fp > 0.f) != (f > 0.f)) && af < 16.f * eps_lo;
  }
  if (list == 1 && (af < a.eps || accepted)) {
    outcome = DIST_RAY_HIT;
  } else if (low && (af < eps_lo || crossed)) {
    // switch to FP32-class queries at the same point (from a BF16 march with
    // an FP16 stage: BF16 rays close to the surface or across it go to FP16
    // first)
    keep = (list == 0 && a.eps_mid > 0.f) ? 2 : 1;
    if (a.c2f) a.o.status[i] = -2;
  } else {
    dn = fmaf(list == 1 ? a.alpha_fp32 : a.alpha, f, d);
    if (list == 1 && a.secant) {
      // unit step first, then secant steps through the last two samples
      if (q == 1) {
        dn = d + f;
      } else {
        const float dd = d - r.dprev;
        const float sl = dd != 0.f ? (f - r.fprev) / dd : 0.f;
        const float stp = sl < -1e-3f ? -f / sl : 0.f;
        if (sl < -1e-3f && fabsf(stp) <= 8.f * af) dn = d + stp;
      }
      a.dprev[i] = d;
      a.fprev[i] = f;
    }
    if (dn > s.z || dn < s.y) outcome = DIST_RAY_LEFT;
    else keep = list;
  }
  if (outcome < 0 && (steps >= a.max_steps || a.last)) {
    outcome = DIST_RAY_MAX_STEPS;
    keep = -1;
  }
  if (outcome == DIST_RAY_HIT) {
    const float dh = d + f;
    a.o.d_hit[i] = dh;
    a.o.depth[i] = dh * r.dirw;
    a.o.mask[i] = 1;
    a.o.sil[i] = accepted ? af - 4.f * a.eps_bf16 : fabsf(fm0) - a.eps;
  } else if (outcome >= 0) {
    a.o.d_hit[i] = kInf;
    a.o.depth[i] = kInf;
    a.o.mask[i] = 0;
    a.o.sil[i] = fabsf(fm0) - a.eps;
  } else if (keep == list) {
    s.x = dn;
    a.st[i] = s;
  }
  if (outcome >= 0 && a.o.status) a.o.status[i] = outcome;
  return keep;
}

__device__ __forceinline__ int step_ray(const TraceArgs& a, int list, int i, float f) {
  RayState r;
  load_ray(a, list, i, r);
  return apply_step(a, list, i, f, r);
}

}  // namespace dist
