// Sphere tracing on the device: ray generation with unit-sphere
// initialisation, the per-step converge/step/compact update, normals, the
// backward probes and the image-plane losses, plus their C-ABI entry points.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

#include "step.cuh"

namespace dist {

namespace {

// Warp-aggregated append of `k` consecutive slots per lane (k may be 0).
__device__ __forceinline__ int warp_append_n(int k, int* counter) {
  int incl = k;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane_id() >= o) incl += y;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  int base = 0;
  if (total > 0 && lane_id() == 31) base = atomicAdd(counter, total);
  base = __shfl_sync(0xffffffffu, base, 31);
  return base + incl - k;
}

// Block-aggregated append to two lists: one atomic per list per block call
// (warp-level appends put one atomic per warp on the same two counters).
// Every thread of the block must call it; it synchronises the block.
template <int WARPS>
__device__ __forceinline__ void block_append2(bool p0, bool p1, int* c0, int* c1, int& s0,
                                              int& s1) {
  __shared__ int wcnt[2][WARPS];
  __shared__ int wbase[2][WARPS];
  const int lane = lane_id(), w = threadIdx.x >> 5;
  const unsigned m0 = __ballot_sync(0xffffffffu, p0), m1 = __ballot_sync(0xffffffffu, p1);
  if (lane == 0) {
    wcnt[0][w] = __popc(m0);
    wcnt[1][w] = __popc(m1);
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    const int l = threadIdx.x;
    int tot = 0;
    for (int q = 0; q < WARPS; ++q) {
      wbase[l][q] = tot;
      tot += wcnt[l][q];
    }
    const int b = tot ? atomicAdd(l ? c1 : c0, tot) : 0;
    for (int q = 0; q < WARPS; ++q) wbase[l][q] += b;
  }
  __syncthreads();
  const unsigned below = (1u << lane) - 1u;
  s0 = p0 ? wbase[0][w] + __popc(m0 & below) : -1;
  s1 = p1 ? wbase[1][w] + __popc(m1 & below) : -1;
}

__device__ __forceinline__ int find_cam(const CamDev* cams, int n_cams, long long i) {
  int lo = 0, hi = n_cams - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cams[mid].offset <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------- cameras

constexpr int kCamChunk = 40;
struct CamChunk {
  CamDev c[kCamChunk];
  int n, first;
};

// Cameras travel as kernel parameters, so no host staging buffer has to
// outlive the call.
__global__ void write_cams_kernel(CamChunk ch, CamDev* dst) {
  const int t = threadIdx.x;
  if (t < ch.n) dst[ch.first + t] = ch.c[t];
}

// --------------------------------------------------------- latent folding

// b'[s][j] = b[j] + sum_k W_z[j][k] z[s][k] for layer 0 (y = 0) and the skip
// layer (y = 1): the latent part of the concatenated input [z, p] is the same
// for every query of a shape, so it is applied once per shape.
__global__ void fold_bias_kernel(DecoderF32 d, const float* __restrict__ z, int n_shapes,
                                 float* bfold0, float* bfolds) {
  const int s = blockIdx.x;
  const int which = blockIdx.y;
  if (which == 1 && d.skip < 0) return;
  const float* Wz = which == 0 ? d.Wz0 : d.Wzs;
  const float* b = which == 0 ? d.b[0] : d.b[d.skip];
  float* out = (which == 0 ? bfold0 : bfolds) + (size_t)s * d.width;
  // layer 0 reads the whole code, the skip layer its last `latent` entries
  const int Lz = which == 0 ? d.latent0 : d.latent;
  const float* zs = z + (size_t)s * d.latent0 + (which == 0 ? 0 : d.latent0 - d.latent);
  const int warp = threadIdx.x >> 5, lane = lane_id();
  for (int j = blockIdx.z * 8 + warp; j < d.width; j += gridDim.z * 8) {
    double acc = 0.0;
    for (int k = lane; k < Lz; k += 32)
      acc += (double)Wz[(size_t)j * Lz + k] * (double)zs[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[j] = (float)(acc + (double)b[j]);
  }
}

// -------------------------------------------------------------- ray setup


// The ray through image point (u, v) of camera c (Sec. 3.2 "Initialization"):
// its world direction, 1/sqrt(x~^2 + y~^2 + 1) for the depth (Sec. 3.3), its
// entry/exit distances into the bounding sphere and, for a ray that misses
// it, the distance from the origin to the ray (Sec. A.3).
struct RayGeom {
  float vx, vy, vz, inv, t_in, t_out, dist;
  bool enters;
};

__device__ __forceinline__ RayGeom ray_geom(const CamDev& c, float radius, float u, float v) {
  RayGeom g;
  const float xt = (u - c.cx) / c.fx;
  const float yt = (v - c.cy) / c.fy;
  const float inv = 1.0f / sqrtf(xt * xt + yt * yt + 1.0f);
  const float vx0 = xt * inv, vy0 = yt * inv, vz0 = inv;
  float vx = c.R[0] * vx0 + c.R[1] * vy0 + c.R[2] * vz0;
  float vy = c.R[3] * vx0 + c.R[4] * vy0 + c.R[5] * vz0;
  float vz = c.R[6] * vx0 + c.R[7] * vy0 + c.R[8] * vz0;
  const float vn = 1.0f / sqrtf(vx * vx + vy * vy + vz * vz);
  vx *= vn; vy *= vn; vz *= vn;
  const float b = vx * c.c[0] + vy * c.c[1] + vz * c.c[2];
  // squared distance from the origin to the line, without cancellation
  const float qx = c.c[0] - b * vx, qy = c.c[1] - b * vy, qz = c.c[2] - b * vz;
  const float qq = qx * qx + qy * qy + qz * qz;
  const float disc = radius * radius - qq;
  const float sq = sqrtf(fmaxf(disc, 0.f));
  g.vx = vx; g.vy = vy; g.vz = vz; g.inv = inv;
  g.t_in = -b - sq;
  g.t_out = -b + sq;
  g.enters = disc > 0.f && g.t_out > 0.f;
  const float cc = c.c[0] * c.c[0] + c.c[1] * c.c[1] + c.c[2] * c.c[2];
  g.dist = b < 0.f ? sqrtf(qq) : sqrtf(cc);
  return g;
}

// Image coordinate of the centre of block X of a 2^level-coarser image:
// (X + 1/2) 2^level, exact in float (x + 0.5 at level 0).
__device__ __forceinline__ float block_centre(int X, int level) {
  return (float)(2 * X + 1) * (float)(1 << level) * 0.5f;
}

// Ray q of a 2^level-coarser image (coarse-to-fine tracing, Sec. 3.2): its
// camera, the full-resolution pixel that holds its state (the top-left pixel
// of its block) and its block coordinates.  Every camera's H and W are
// multiples of 2^level, so camera offsets are multiples of 4^level.
__device__ __forceinline__ long long coarse_ray(const TraceArgs& a, long long q, int level,
                                                int& ci, int& X, int& Y) {
  ci = find_cam(a.cams, a.n_cams, q << (2 * level));
  const CamDev& c = a.cams[ci];
  const long long lq = q - (c.offset >> (2 * level));
  const int Wl = c.W >> level;
  X = (int)(lq % Wl);
  Y = (int)(lq / Wl);
  return c.offset + ((long long)Y << level) * c.W + ((long long)X << level);
}

__device__ __forceinline__ void write_miss(const TraceArgs& a, long long i, float sil, int status) {
  a.o.depth[i] = kInf;
  a.o.d_hit[i] = kInf;
  a.o.mask[i] = 0;
  a.o.sil[i] = sil;
  if (a.o.status) a.o.status[i] = status;
}

// A ray that starts marching at its own entry point: no queries, no samples.
__device__ __forceinline__ void start_ray(const TraceArgs& a, long long i, const RayGeom& g,
                                          int ci) {
  a.o.steps[i] = 0;
  for (int k = 0; k < a.K; ++k) {
    a.o.d_min[i * a.K + k] = __int_as_float(0x7fc00000);
    a.o.f_min[i * a.K + k] = kInf;
  }
  if (g.enters) {
    a.st[i] = make_float4(g.t_in, g.t_in, g.t_out, __int_as_float(ci));
    a.fq[i] = 0;
    a.fprev[i] = 0.f;
    if (a.c2f) a.o.status[i] = a.c2f_start;
  } else {
    write_miss(a, i, g.dist - a.radius, DIST_RAY_INIT_MISS);
  }
}

// One thread per ray (Sec. 3.2 "Initialization"): the ray through the pixel
// centre (level 0) or through the centre of its block of a 2^level-coarser
// image (coarse-to-fine tracing), its entry/exit distances into the bounding
// sphere, and the background outputs of rays that miss it (depth +inf,
// silhouette = distance from the origin to the ray minus the radius,
// Sec. A.3).  Rays that enter are appended to `list0`.
__global__ void raygen_kernel(TraceArgs a, int level, int* list0, int* count0) {
  const long long n = a.n_pix >> (2 * level);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll;
       base < n; base += stride) {
    long long i = 0;
    bool enters = false;
    if (base + lane_id() < n) {
      int ci, X, Y;
      if (level == 0) {
        i = a.pix0 + base + lane_id();
        ci = a.cam_fixed >= 0 ? a.cam_fixed : find_cam(a.cams, a.n_cams, i);
        const long long li = i - a.cams[ci].offset;
        X = (int)(li % a.cams[ci].W);
        Y = (int)(li / a.cams[ci].W);
      } else {
        i = coarse_ray(a, base + lane_id(), level, ci, X, Y);
      }
      const RayGeom g = ray_geom(a.cams[ci], a.radius, block_centre(X, level),
                                 block_centre(Y, level));
      a.dir[i] = make_float4(g.vx, g.vy, g.vz, g.inv);
      start_ray(a, i, g, ci);
      enters = g.enters;
    }
    const int slot = warp_append(enters, count0);
    if (slot >= 0) list0[slot] = (int)i;
  }
}

// Coarse-to-fine split (Sec. 3.2): every ray of level `level` becomes its
// four children of level - 1.  One thread per parent reads the parent's state
// (held at its block's top-left pixel, which is also its first child's) and
// writes the children's.  What a child inherits is not stated in the paper;
// the reading: a child has its own direction and bounding-sphere interval (a
// child that misses the sphere is background); a child of a parent that
// missed the sphere starts at its own entry; otherwise it inherits the step
// count and the k smallest-|f| samples with |f| raised to eps, and
//  * a marching or converged parent's ray distance d, raised to the child's
//    t_in (past its t_out the child has left the sphere): the child marches
//    on from there, in the parent's list (a converged parent's children in
//    the FP32 list), or ends as MAX_STEPS when no query is left (`final`);
//  * a parent that left the sphere or ran out of queries: the same outcome.
__global__ void split_kernel(TraceArgs a, int level, int final, int* list0, int* list1,
                             int* count0, int* count1) {
  const long long n = a.n_pix >> (2 * level);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll;
       base < n; base += stride) {
    // per lane: up to 4 children appended to list 0 / list 1
    int add0[4] = {-1, -1, -1, -1}, add1[4] = {-1, -1, -1, -1};
    if (base + lane_id() < n) {
      int ci, X, Y;
      const long long ip = coarse_ray(a, base + lane_id(), level, ci, X, Y);
      const CamDev& c = a.cams[ci];
      const int status = a.o.status[ip];
      const float4 sp = a.st[ip];
      const int steps = a.o.steps[ip];
      float fm[kMaxK], dm[kMaxK];
      for (int k = 0; k < kMaxK; ++k) {
        fm[k] = k < a.K ? a.o.f_min[ip * a.K + k] : kInf;
        dm[k] = k < a.K ? a.o.d_min[ip * a.K + k] : 0.f;
      }
      const int fq = a.fq[ip];
      const float fprev = a.fprev[ip], dprev = a.dprev[ip];
      const bool marching = status < 0 || status == DIST_RAY_HIT;
      const int list = status == DIST_RAY_HIT ? 1 : (status == -1 ? 0 : 1);
#pragma unroll
      for (int ch = 0; ch < 4; ++ch) {
        const int cx = 2 * X + (ch & 1), cy = 2 * Y + (ch >> 1);
        const long long i = c.offset + ((long long)cy << (level - 1)) * c.W +
                            ((long long)cx << (level - 1));
        const RayGeom g = ray_geom(c, a.radius, block_centre(cx, level - 1),
                                   block_centre(cy, level - 1));
        a.dir[i] = make_float4(g.vx, g.vy, g.vz, g.inv);
        if (!g.enters || status == DIST_RAY_INIT_MISS) {
          start_ray(a, i, g, ci);
          if (g.enters) {
            if (final) {
              write_miss(a, i, kInf, DIST_RAY_MAX_STEPS);
            } else if (a.c2f_start == -1) {
              add0[ch] = (int)i;
            } else {
              add1[ch] = (int)i;
            }
          }
          continue;
        }
        a.o.steps[i] = steps;
        float fm0 = kInf;
        for (int k = 0; k < a.K; ++k) {
          const float f = copysignf(fmaxf(fabsf(fm[k]), a.eps), fm[k]);
          a.o.f_min[i * a.K + k] = f;
          a.o.d_min[i * a.K + k] = dm[k];
          if (k == 0) fm0 = fabsf(f);
        }
        if (!marching) {
          write_miss(a, i, fm0 - a.eps, status);
          continue;
        }
        const float d = fmaxf(sp.x, g.t_in);
        if (d > g.t_out) {
          write_miss(a, i, fm0 - a.eps, DIST_RAY_LEFT);
        } else if (final) {
          write_miss(a, i, fm0 - a.eps, DIST_RAY_MAX_STEPS);
        } else {
          a.st[i] = make_float4(d, g.t_in, g.t_out, __int_as_float(ci));
          a.fq[i] = fq;
          a.fprev[i] = fprev;
          a.dprev[i] = dprev;
          a.o.status[i] = list == 0 ? -1 : -2;
          if (list == 0) add0[ch] = (int)i;
          else add1[ch] = (int)i;
        }
      }
    }
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
      const int s0 = warp_append(add0[ch] >= 0, count0);
      if (s0 >= 0) list0[s0] = add0[ch];
      const int s1 = warp_append(add1[ch] >= 0, count1);
      if (s1 >= 0) list1[s1] = add1[ch];
    }
  }
}

// ------------------------------------------------------------- march step

struct StepLists {
  const int* cnt_in[2];   // list lengths: [0] low-precision list, [1] FP32 list
  int* cnt_out[2];        // append counters of the output lists
  const int* in[2];
  const float* f[2];
  int* out[2];
};

// One march step for every ray that was queried this step (Alg. 1 with the
// aggressive update of Sec. 3.2 and the stopping rules of Sec. 3.2 / B.2):
//  * track the k smallest |f| (Sec. 3.4, B.2) -- ties keep the earlier sample;
//  * |f| < eps: hit; the last query is a unit step, d_hit = d + f (Eq. 1);
//  * else d += alpha f; leaving [t_in, t_out] or using the last query makes
//    the ray background (Sec. B.2, A.2);
//  * survivors are appended to the next step's list (dynamic synchronized
//    inference, Sec. 3.2) with a warp-aggregated atomic.
// BF16-phase rays (list 0) use eps_bf16 to switch to FP32 queries at the
// same point; their samples enter the |f| tracking as max(|f|, eps) so that
// only FP32 samples can make the silhouette negative.
constexpr int kStepThreads = 256;
__global__ void __launch_bounds__(kStepThreads) step_kernel(TraceArgs a, StepLists L,
                                                            unsigned long long* queries) {
  const int n0 = *L.cnt_in[0], n1 = *L.cnt_in[1];
  const int n = n0 + n1;
  if (queries && blockIdx.x == 0 && threadIdx.x == 0) {
    atomicAdd(queries + 0, (unsigned long long)n0);
    atomicAdd(queries + 1, (unsigned long long)n1);
  }
  const int stride = gridDim.x * blockDim.x;
  // block-uniform rounds (block_append2 synchronises the block)
  for (int r0 = blockIdx.x * blockDim.x; r0 < n; r0 += stride) {
    const int j = r0 + threadIdx.x;
    int keep = -1, ray = -1;
    if (j < n) {
      const int list = j < n0 ? 0 : 1;
      const int jj = list == 0 ? j : j - n0;
      const int i = L.in[list][jj];
      const float f = L.f[list][jj];
      ray = i;
      keep = step_ray(a, list, i, f);
    }
    int s0, s1;
    block_append2<kStepThreads / 32>(keep == 0, keep == 1, L.cnt_out[0], L.cnt_out[1], s0, s1);
    if (s0 >= 0) L.out[0][s0] = ray;
    if (s1 >= 0) L.out[1][s1] = ray;
  }
}

// ---------------------------------------------------------------- probes

struct ProbeArgs {
  const CamDev* cams;
  const float4* st;       // unused after the trace except for the camera id
  const float4* dir;
  long long n_pix;
  long long pix0;         // first pixel handled (probes_bwd_kernel)
  int cam_fixed;          // >= 0: all pixels belong to this camera (probes_bwd_kernel)
  int n_cams;
  int K;
  dist_trace_out o;
  float4* pp;
  float4* pq;
  int* pix;
  int* count;
  // Ordered append (pixel order, so the backward pass sums its probes in the
  // same grouping on every run): null = atomic append in arrival order; else
  // phase 0 writes each 32-pixel chunk's probe count to chunk[base / 32],
  // chunk_scan_kernel turns the counts into offsets, and phase 1 writes the
  // probes at them.
  int* chunk;
  int phase;
};

// Slot of the first of this lane's k probes for the 32-pixel chunk at
// `base` (all lanes of the warp call it), or -1 when nothing is written
// (the counting phase of an ordered append).
__device__ __forceinline__ int probe_slot(const ProbeArgs& a, long long base, int k) {
  if (!a.chunk) return warp_append_n(k, a.count);
  int incl = k;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane_id() >= o) incl += y;
  }
  if (a.phase == 0) {
    if (lane_id() == 31) a.chunk[base >> 5] = incl;
    return -1;
  }
  return a.chunk[base >> 5] + incl - k;
}

// In-place exclusive scan of the per-chunk probe counts of an ordered append
// (one block); *total = their sum, the probe count the adjoint reads.
__global__ void __launch_bounds__(1024) chunk_scan_kernel(int* c, long long n, int* total) {
  __shared__ int part[1024];
  const long long per = (n + blockDim.x - 1) / blockDim.x;
  const long long lo = min(n, per * threadIdx.x), hi = min(n, lo + per);
  int s = 0;
  for (long long i = lo; i < hi; ++i) s += c[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {
    const int v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - s;      // exclusive prefix of this thread's range
  for (long long i = lo; i < hi; ++i) {
    const int v = c[i];
    c[i] = run;
    run += v;
  }
  if (threadIdx.x == blockDim.x - 1) *total = part[threadIdx.x];
}

__device__ __forceinline__ float4 ray_point(const CamDev& c, const float4& v, float d, int shape) {
  return make_float4(fmaf(d, v.x, c.c[0]), fmaf(d, v.y, c.c[1]), fmaf(d, v.z, c.c[2]),
                     __int_as_float(shape));
}

// Hit points of the trace (normals): one probe per hit pixel.
__global__ void probes_hits_kernel(ProbeArgs a) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll;
       base < a.n_pix; base += stride) {
    const long long i = base + lane_id();
    const bool hit = i < a.n_pix && a.o.mask[i];
    const int slot = warp_append(hit, a.count);
    if (slot >= 0) {
      const CamDev& c = a.cams[find_cam(a.cams, a.n_cams, i)];
      a.pp[slot] = ray_point(c, a.dir[i], a.o.d_hit[i], c.shape);
      a.pq[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
      a.pix[slot] = (int)i;
    }
  }
}

// Six probes per hit pixel at p_hit +- delta e_a (Sec. 3.3 central
// differences), in the order +x, -x, +y, -y, +z, -z.  With `g_normal`
// non-null only pixels with a non-zero normal gradient get probes.
__global__ void probes_fd_kernel(ProbeArgs a, float delta, const float* g_normal) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll;
       base < a.n_pix; base += stride) {
    const long long i = base + lane_id();
    bool take = i < a.n_pix && a.o.mask[i];
    if (take && g_normal)
      take = g_normal[3 * i] != 0.f || g_normal[3 * i + 1] != 0.f || g_normal[3 * i + 2] != 0.f;
    const int slot = probe_slot(a, base, take ? 6 : 0);
    if (take && slot >= 0) {
      const CamDev& c = a.cams[find_cam(a.cams, a.n_cams, i)];
      const float4 p = ray_point(c, a.dir[i], a.o.d_hit[i], c.shape);
      for (int e = 0; e < 6; ++e) {
        float4 q = p;
        const float dlt = (e & 1) ? -delta : delta;
        if (e < 2) q.x += dlt; else if (e < 4) q.y += dlt; else q.z += dlt;
        a.pp[slot + e] = q;
        a.pq[slot + e] = make_float4(0.f, 0.f, 0.f, 0.f);
        a.pix[slot + e] = (int)i;
      }
    }
  }
}

__global__ void normals_from_grad_kernel(const float* out4, const int* pix, const int* count,
                                         float* normal) {
  const int n = *count;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const float4 g = out4 ? reinterpret_cast<const float4*>(out4)[j] : make_float4(0, 0, 0, 0);
    const float nn = sqrtf(g.y * g.y + g.z * g.z + g.w * g.w);
    const float s = nn > 0.f ? 1.f / nn : 0.f;
    const int i = pix[j];
    normal[3 * i] = g.y * s; normal[3 * i + 1] = g.z * s; normal[3 * i + 2] = g.w * s;
  }
}

__global__ void normals_from_fd_kernel(const float* f6, const int* pix, const int* count,
                                       float delta, float* normal, float* grad_len) {
  const int n = *count / 6;
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) {
    const float* f = f6 + 6 * h;
    const float inv = 1.f / (2.f * delta);
    const float gx = (f[0] - f[1]) * inv, gy = (f[2] - f[3]) * inv, gz = (f[4] - f[5]) * inv;
    const float nn = sqrtf(gx * gx + gy * gy + gz * gz);
    const float s = nn > 0.f ? 1.f / nn : 0.f;
    const int i = pix[6 * h];
    normal[3 * i] = gx * s; normal[3 * i + 1] = gy * s; normal[3 * i + 2] = gz * s;
    if (grad_len) grad_len[i] = nn;
  }
}

// Backward probes for the depth and silhouette terms.
//  exact depth: the hit point, q = (v, g_depth * inv_norm); the adjoint
//    turns it into -q.w / (grad f . v) (implicit differentiation);
//  paper depth: the k smallest-|f| samples, coefficient alpha g_depth inv_norm
//    (first term of Eq. 2);
//  silhouette: the smallest-|f| sample, coefficient g_sil sign(f_min).
__global__ void probes_bwd_kernel(ProbeArgs a, const float* g_depth, const float* g_sil,
                                  int paper, float alpha) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll;
       base < a.n_pix; base += stride) {
    const long long i = a.pix0 + base + lane_id();
    int nd = 0, ns = 0;
    float gd = 0.f, gs = 0.f;
    if (base + lane_id() < a.n_pix) {
      gd = g_depth ? g_depth[i] : 0.f;
      gs = g_sil ? g_sil[i] : 0.f;
      if (a.o.mask[i] && gd != 0.f) {
        if (!paper) nd = 1;
        else
          for (int k = 0; k < a.K; ++k) nd += isnan(a.o.d_min[i * a.K + k]) ? 0 : 1;
      }
      const float fm0 = a.o.f_min[i * a.K];
      if (gs != 0.f && !isnan(a.o.d_min[i * a.K]) && fm0 != 0.f) ns = 1;
    }
    int slot = probe_slot(a, base, nd + ns);
    if (nd + ns > 0 && slot >= 0) {
      const CamDev& c = a.cams[a.cam_fixed >= 0 ? a.cam_fixed : find_cam(a.cams, a.n_cams, i)];
      const float4 v = a.dir[i];
      if (nd > 0 && !paper) {
        a.pp[slot] = ray_point(c, v, a.o.d_hit[i], c.shape);
        a.pq[slot] = make_float4(v.x, v.y, v.z, gd * v.w);
        a.pix[slot] = (int)i;
        ++slot;
      } else if (nd > 0) {
        for (int k = 0; k < a.K; ++k) {
          const float dk = a.o.d_min[i * a.K + k];
          if (isnan(dk)) continue;
          a.pp[slot] = ray_point(c, v, dk, c.shape);
          a.pq[slot] = make_float4(0.f, 0.f, 0.f, alpha * gd * v.w);
          a.pix[slot] = (int)i;
          ++slot;
        }
      }
      if (ns) {
        const float fm0 = a.o.f_min[i * a.K];
        a.pp[slot] = ray_point(c, v, a.o.d_min[i * a.K], c.shape);
        a.pq[slot] = make_float4(0.f, 0.f, 0.f, fm0 > 0.f ? gs : -gs);
        a.pix[slot] = (int)i;
      }
    }
  }
}

// ------------------------------------------------------ camera gradients

constexpr int kCamSil = 1 << 30;   // probe_pix flag: silhouette probe (else depth)

// Probes for the camera gradient: at the hit of every pixel with a depth
// gradient, and at the smallest-|f| sample of every pixel with a silhouette
// gradient whose ray entered the sphere and was queried.
__global__ void probes_cam_kernel(ProbeArgs a, const float* g_depth, const float* g_sil) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll;
       base < a.n_pix; base += stride) {
    const long long i = base + lane_id();
    int nd = 0, ns = 0;
    if (i < a.n_pix) {
      nd = g_depth && a.o.mask[i] && g_depth[i] != 0.f ? 1 : 0;
      ns = g_sil && g_sil[i] != 0.f && !isnan(a.o.d_min[i * a.K]) ? 1 : 0;
    }
    int slot = probe_slot(a, base, nd + ns);
    if (nd + ns > 0 && slot >= 0) {
      const CamDev& c = a.cams[find_cam(a.cams, a.n_cams, i)];
      const float4 v = a.dir[i];
      if (nd) {
        a.pp[slot] = ray_point(c, v, a.o.d_hit[i], c.shape);
        a.pix[slot] = (int)i;
        ++slot;
      }
      if (ns) {
        a.pp[slot] = ray_point(c, v, a.o.d_min[i * a.K], c.shape);
        a.pix[slot] = (int)i | kCamSil;
      }
    }
  }
}

// Adds the 12 values of one ray's dL/d(c, R) to its camera's FP64 sums: one
// set of atomics per warp when the warp's lanes share a camera.
__device__ __forceinline__ void cam_accumulate(double* G, int ci, bool have, const double (&v)[12]) {
  const unsigned act = __activemask();
  const unsigned peers = __match_any_sync(act, have ? ci : -1);
  const bool uniform = __all_sync(act, have) && peers == act;
  if (uniform) {
    double r[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      double x = v[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(act, x, o);
      r[k] = x;
    }
    if (lane_id() == __ffs(act) - 1) {
#pragma unroll
      for (int k = 0; k < 12; ++k)
        if (r[k] != 0.0) atomicAdd(G + (size_t)ci * 12 + k, r[k]);
    }
  } else if (have) {
#pragma unroll
    for (int k = 0; k < 12; ++k)
      if (v[k] != 0.0) atomicAdd(G + (size_t)ci * 12 + k, v[k]);
  }
}

// The camera frame direction of pixel i: v_cam = (x~, y~, 1)/|.|, and
// u = R v_cam (the world direction before normalisation).
__device__ __forceinline__ void pixel_frame(const CamDev& c, long long i, double (&vc)[3],
                                            double (&u)[3]) {
  const long long li = i - c.offset;
  const int x = (int)(li % c.W), y = (int)(li / c.W);
  const double xt = ((double)x + 0.5 - c.cx) / c.fx;
  const double yt = ((double)y + 0.5 - c.cy) / c.fy;
  const double inv = 1.0 / sqrt(xt * xt + yt * yt + 1.0);
  vc[0] = xt * inv; vc[1] = yt * inv; vc[2] = inv;
  for (int a = 0; a < 3; ++a)
    u[a] = c.R[3 * a] * vc[0] + c.R[3 * a + 1] * vc[1] + c.R[3 * a + 2] * vc[2];
}

// dL/dR from dL/dv: v = u/|u|, u = R v_cam.
__device__ __forceinline__ void cam_pack(const double (&dc)[3], const double (&dv)[3],
                                         const double (&vc)[3], const double (&u)[3],
                                         double (&out)[12]) {
  const double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  const double v[3] = {u[0] / un, u[1] / un, u[2] / un};
  const double vd = v[0] * dv[0] + v[1] * dv[1] + v[2] * dv[2];
  for (int a = 0; a < 3; ++a) {
    out[a] = dc[a];
    const double du = (dv[a] - v[a] * vd) / un;
    for (int b = 0; b < 3; ++b) out[3 + 3 * a + b] = du * vc[b];
  }
}

// Per probe: the depth (implicit) or entering-silhouette (first-term)
// contribution to the camera gradient, from grad_p f of the adjoint.
__global__ void cam_probe_grad_kernel(ProbeArgs a, const float* out4, const float* g_depth,
                                      const float* g_sil, double* G) {
  const int n = *a.count;
  for (int base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; base < n;
       base += gridDim.x * blockDim.x) {
    const int j = base + lane_id();
    double val[12];
    for (int k = 0; k < 12; ++k) val[k] = 0.0;
    bool have = false;
    int ci = 0;
    if (j < n) {
      const int pj = a.pix[j];
      const bool sil = (pj & kCamSil) != 0;
      const long long i = pj & (kCamSil - 1);
      ci = find_cam(a.cams, a.n_cams, i);
      const CamDev& c = a.cams[ci];
      double vc[3], u[3];
      pixel_frame(c, i, vc, u);
      const float4 g4 = reinterpret_cast<const float4*>(out4)[j];
      const double gp[3] = {g4.y, g4.z, g4.w};
      const float4 v4 = a.dir[i];
      const double v[3] = {v4.x, v4.y, v4.z};
      double dc[3] = {0.0, 0.0, 0.0}, dv[3] = {0.0, 0.0, 0.0};
      if (!sil) {
        const double gv = gp[0] * v[0] + gp[1] * v[1] + gp[2] * v[2];
        const double gn = sqrt(gp[0] * gp[0] + gp[1] * gp[1] + gp[2] * gp[2]);
        if (fabs(gv) >= 1e-3 * gn && gv != 0.0) {
          const double w = (double)g_depth[i] * (double)v4.w / gv;
          const double d = a.o.d_hit[i];
          for (int k = 0; k < 3; ++k) { dc[k] = -w * gp[k]; dv[k] = -w * d * gp[k]; }
          have = true;
        }
      } else {
        const float fm = a.o.f_min[i * a.K];
        const double s = (fm > 0.f ? 1.0 : (fm < 0.f ? -1.0 : 0.0)) * (double)g_sil[i];
        const double d = a.o.d_min[i * a.K];
        for (int k = 0; k < 3; ++k) { dc[k] = s * gp[k]; dv[k] = s * d * gp[k]; }
        have = true;
      }
      if (have) cam_pack(dc, dv, vc, u, val);
    }
    cam_accumulate(G, ci, have, val);
  }
}

// Rays that missed the bounding sphere: S = dist(origin, ray) - radius
// (Sec. A.3), differentiated exactly; such a ray made no query (steps 0)
// and has a finite silhouette.
__global__ void cam_miss_grad_kernel(ProbeArgs a, const float* g_sil, double* G) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll;
       base < a.n_pix; base += stride) {
    const long long i = base + lane_id();
    double val[12];
    for (int k = 0; k < 12; ++k) val[k] = 0.0;
    bool have = false;
    int ci = 0;
    if (i < a.n_pix && g_sil[i] != 0.f && a.o.steps[i] == 0 && isfinite(a.o.sil[i])) {
      ci = find_cam(a.cams, a.n_cams, i);
      const CamDev& c = a.cams[ci];
      double vc[3], u[3];
      pixel_frame(c, i, vc, u);
      const float4 v4 = a.dir[i];
      const double v[3] = {v4.x, v4.y, v4.z};
      const double cc[3] = {c.c[0], c.c[1], c.c[2]};
      const double b = v[0] * cc[0] + v[1] * cc[1] + v[2] * cc[2];
      const double c2 = cc[0] * cc[0] + cc[1] * cc[1] + cc[2] * cc[2];
      const double g = g_sil[i];
      double dc[3], dv[3];
      if (b < 0.0) {
        const double dist = sqrt(fmax(c2 - b * b, 0.0));
        for (int k = 0; k < 3; ++k) {
          dc[k] = g * (cc[k] - b * v[k]) / dist;
          dv[k] = -g * b * cc[k] / dist;
        }
      } else {
        const double dist = sqrt(c2);
        for (int k = 0; k < 3; ++k) { dc[k] = g * cc[k] / dist; dv[k] = 0.0; }
      }
      cam_pack(dc, dv, vc, u, val);
      have = true;
    }
    cam_accumulate(G, ci, have, val);
  }
}

__global__ void cam_finalize_kernel(const double* G, int n, float* out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    out[k] = (float)G[k];
}

// ------------------------------------------------- photometric warp loss

struct PhotoArgs {
  const CamDev* cams;
  int vi, vj;            // warp view vj onto view vi
  const float* depth;    // [n_pix] rendered depth of all views (inf = background)
  const float* img;      // [n_pix][C] colour images of all views
  int C;
  double vis_thresh;
  double* sums;          // [0] sum of |I_i - I_{j->i}|, [1] visible pixels
  float* g_depth;        // += d(sum)/d depth_i (normalised afterwards)
};

// One thread per pixel of view vi (Sec. 4.2 multi-view loss, Sec. B.3
// visibility): lift the hit to P = c_i + d v, project into view vj, sample
// its image and depth bilinearly between pixel centres, test visibility
// ((z_j(P) - D_j)^2 below the threshold, all four neighbours hit and inside)
// and add the L1 colour difference and its derivative with respect to the
// rendered depth of view vi.  Double precision (a small kernel; it keeps the
// cell and visibility decisions those of the reference arithmetic).
__global__ void photo_pair_kernel(PhotoArgs a) {
  const CamDev& ci = a.cams[a.vi];
  const CamDev& cj = a.cams[a.vj];
  const long long n = (long long)ci.H * ci.W;
  double lsum = 0.0, lcnt = 0.0;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (long long)gridDim.x * blockDim.x) {
    const long long gi = ci.offset + x;
    const float Di = a.depth[gi];
    if (!isfinite(Di)) continue;
    const int px = (int)(x % ci.W), py = (int)(x / ci.W);
    const double xt = ((double)px + 0.5 - ci.cx) / ci.fx;
    const double yt = ((double)py + 0.5 - ci.cy) / ci.fy;
    const double nrm = sqrt(xt * xt + yt * yt + 1.0);
    const double vc[3] = {xt / nrm, yt / nrm, 1.0 / nrm};
    double v[3];
    for (int r = 0; r < 3; ++r)
      v[r] = ci.R[3 * r] * vc[0] + ci.R[3 * r + 1] * vc[1] + ci.R[3 * r + 2] * vc[2];
    const double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int r = 0; r < 3; ++r) v[r] /= vn;
    const double inv = 1.0 / nrm;
    const double d = (double)Di / inv;
    double w3[3], pc[3] = {0.0, 0.0, 0.0}, q[3] = {0.0, 0.0, 0.0};
    for (int r = 0; r < 3; ++r) w3[r] = ci.c[r] + d * v[r] - cj.c[r];
    // R_j^T (P - c_j) and R_j^T v
    for (int k = 0; k < 3; ++k)
      for (int r = 0; r < 3; ++r) {
        pc[k] += cj.R[3 * r + k] * w3[r];
        q[k] += cj.R[3 * r + k] * v[r];
      }
    if (!(pc[2] > 1e-9)) continue;
    const double pz = pc[2];
    const double u = cj.fx * pc[0] / pz + cj.cx;
    const double vv = cj.fy * pc[1] / pz + cj.cy;
    const double sx = u - 0.5, sy = vv - 0.5;
    const double fx0 = floor(sx), fy0 = floor(sy);
    if (!(fx0 >= 0.0 && fy0 >= 0.0 && fx0 <= (double)(cj.W - 2) && fy0 <= (double)(cj.H - 2)))
      continue;
    const int x0 = (int)fx0, y0 = (int)fy0;
    const double fx = sx - fx0, fy = sy - fy0;
    const long long b00 = cj.offset + (long long)y0 * cj.W + x0;
    const long long b01 = b00 + 1, b10 = b00 + cj.W, b11 = b10 + 1;
    const float d00 = a.depth[b00], d01 = a.depth[b01], d10 = a.depth[b10], d11 = a.depth[b11];
    if (!(isfinite(d00) && isfinite(d01) && isfinite(d10) && isfinite(d11))) continue;
    const double Dj = (1 - fy) * ((1 - fx) * d00 + fx * d01) + fy * ((1 - fx) * d10 + fx * d11);
    if (!((pz - Dj) * (pz - Dj) < a.vis_thresh)) continue;
    const double dudd = cj.fx * (q[0] * pz - pc[0] * q[2]) / (pz * pz);
    const double dvdd = cj.fy * (q[1] * pz - pc[1] * q[2]) / (pz * pz);
    double term = 0.0, dterm = 0.0;
    for (int c = 0; c < a.C; ++c) {
      const double i00 = a.img[b00 * a.C + c], i01 = a.img[b01 * a.C + c];
      const double i10 = a.img[b10 * a.C + c], i11 = a.img[b11 * a.C + c];
      const double val = (1 - fy) * ((1 - fx) * i00 + fx * i01) + fy * ((1 - fx) * i10 + fx * i11);
      const double du = (1 - fy) * (i01 - i00) + fy * (i11 - i10);
      const double dv = (1 - fx) * (i10 - i00) + fx * (i11 - i01);
      const double r = (double)a.img[gi * a.C + c] - val;
      term += fabs(r);
      const double sg = r > 0.0 ? 1.0 : (r < 0.0 ? -1.0 : 0.0);
      dterm -= sg * (du * dudd + dv * dvdd);
    }
    lsum += term;
    lcnt += 1.0;
    a.g_depth[gi] += (float)(dterm / inv);
  }
  // block sums, one atomic pair per block
  __shared__ double s_sum[8], s_cnt[8];
  for (int o = 16; o > 0; o >>= 1) {
    lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    lcnt += __shfl_xor_sync(0xffffffffu, lcnt, o);
  }
  const int w = threadIdx.x >> 5;
  if (lane_id() == 0) { s_sum[w] = lsum; s_cnt[w] = lcnt; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ts = 0.0, tc = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { ts += s_sum[k]; tc += s_cnt[k]; }
    if (tc > 0.0) {
      atomicAdd(a.sums, ts);
      atomicAdd(a.sums + 1, tc);
    }
  }
}

// loss = w sum / count and g_depth *= w / count (0 without visible pixels).
__global__ void photo_finalize_kernel(const double* sums, double w, long long n, float* g_depth,
                                      double* loss) {
  const double cnt = sums[1];
  const double s = cnt > 0.0 ? w / cnt : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) *loss = sums[0] * s;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    g_depth[k] = (float)((double)g_depth[k] * s);
}

// ------------------------------------------------------- texture colour

// rgb of hit pixels from the FP32 colour rows (tanh applied).
__global__ void color_scatter_kernel(const float* rows, const int* pix, const int* count,
                                     float* rgb) {
  const int n = *count;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const int i = pix[j];
    for (int o = 0; o < 3; ++o) rgb[3 * (size_t)i + o] = rows[3 * (size_t)j + o];
  }
}

// rgb = tanh(sum of the four column-group partials, in order, + b) from the
// tensor-core colour decoder.
__global__ void color_finalize_kernel(const float* cpart, const int* pix, const int* count,
                                      float b0, float b1, float b2, float* rgb) {
  const int n = *count;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const int i = pix[j];
    const float b[3] = {b0, b1, b2};
    for (int o = 0; o < 3; ++o) {
      float s = 0.f;
      for (int g = 0; g < 4; ++g) s += cpart[((size_t)j * 4 + g) * 3 + o];
      rgb[3 * (size_t)i + o] = tanhf(s + b[o]);
    }
  }
}

// Normal-loss coefficients: with g = FD gradient from the six probe values
// and n = g / |g|, dL/dg = (g_n - n (n . g_n)) / |g|; probe +a gets
// dL/dg_a / (2 delta), probe -a its negative (hit point held fixed).
// Probe coefficients of the central-difference normal n = g / |g|: the VJP
// of dL/dn through the normalisation, (dL/dn - n (n . dL/dn)) / |g|, times
// +-1 / (2 delta) for the probes at p +- delta e_a.
__device__ __forceinline__ void fd_coef_store(const double (&nv)[3], double gn, double inv,
                                              const float* g_normal, int i, float4* pq6) {
  const double up[3] = {g_normal[3 * i], g_normal[3 * i + 1], g_normal[3 * i + 2]};
  double c[3] = {0, 0, 0};
  if (gn > 0) {
    const double nu = nv[0] * up[0] + nv[1] * up[1] + nv[2] * up[2];
    for (int e = 0; e < 3; ++e) c[e] = (up[e] - nv[e] * nu) / gn * inv;
  }
  for (int e = 0; e < 3; ++e) {
    pq6[2 * e] = make_float4(0.f, 0.f, 0.f, (float)c[e]);
    pq6[2 * e + 1] = make_float4(0.f, 0.f, 0.f, (float)-c[e]);
  }
}

// ... from the six probe values.
__global__ void fd_coef_kernel(const float* f6, const int* pix, const int* count, float delta,
                               const float* g_normal, float4* pq) {
  const int n = *count / 6;
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) {
    const float* f = f6 + 6 * h;
    const double inv = 1.0 / (2.0 * (double)delta);
    const double g[3] = {(f[0] - f[1]) * inv, (f[2] - f[3]) * inv, (f[4] - f[5]) * inv};
    const double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    double nv[3] = {0, 0, 0};
    if (gn > 0)
      for (int e = 0; e < 3; ++e) nv[e] = g[e] / gn;
    fd_coef_store(nv, gn, inv, g_normal, pix[6 * h], pq + 6 * h);
  }
}

// ... from the forward's normal and |g| (dist_trace_out.grad_len).
__global__ void fd_coef_from_normal_kernel(const float* normal, const float* grad_len,
                                           const int* pix, const int* count, float delta,
                                           const float* g_normal, float4* pq) {
  const int n = *count / 6;
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) {
    const int i = pix[6 * h];
    const double inv = 1.0 / (2.0 * (double)delta);
    const double nv[3] = {normal[3 * i], normal[3 * i + 1], normal[3 * i + 2]};
    fd_coef_store(nv, (double)grad_len[i], inv, g_normal, i, pq + 6 * h);
  }
}

// dz[s][k] += sum_j Wz0[j][k] G0[s][j] + sum_j Wzs[j][k] Gs[s][j]  (FP64).
// dz[s] += W_z0^T G0[s] + W_zs^T Gs[s] (Eq. 2's latent factor), in FP64.
// Block (k-chunk of 32, shape s): lane = latent index, the 16 warps split the
// width and a fixed-order shared-memory sum combines them (deterministic).
constexpr int kFinalizeWarps = 16;
__global__ void __launch_bounds__(kFinalizeWarps * 32)
latent_finalize_kernel(DecoderF32 d, const double* G0, const double* Gs, int n_shapes, float* dz) {
  __shared__ double part[kFinalizeWarps][32];
  const int s = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int k = blockIdx.x * 32 + lane;
  const int per = (d.width + kFinalizeWarps - 1) / kFinalizeWarps;
  const int j0 = w * per, j1 = min(d.width, j0 + per);
  double acc = 0.0;
  if (k < d.latent) {
    const double* g0 = G0 + (size_t)s * d.width;
    const double* gs = Gs + (size_t)s * d.width;
    for (int j = j0; j < j1; ++j) {
      acc = fma((double)d.Wz0[(size_t)j * d.latent + k], g0[j], acc);
      if (d.skip > 0) acc = fma((double)d.Wzs[(size_t)j * d.latent + k], gs[j], acc);
    }
  }
  part[w][lane] = acc;
  __syncthreads();
  if (w == 0 && k < d.latent) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < kFinalizeWarps; ++q) t += part[q][lane];
    dz[(size_t)s * d.latent + k] += (float)t;
  }
}

// ------------------------------------------------------------------ losses

__device__ __forceinline__ double block_sum_d(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5;
  if (lane_id() == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
  __syncthreads();
  return t;
}

__global__ void loss_count_kernel(long long n, const uint8_t* mask, const float* tgt, int* cnt) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll; base < n;
       base += stride) {
    const long long i = base + lane_id();
    const bool m = i < n && mask[i] && isfinite(tgt[i]);
    const unsigned b = __ballot_sync(0xffffffffu, m);
    if (lane_id() == 0 && b) atomicAdd(cnt, __popc(b));
  }
}

struct LossArgs {
  double* part;            // [gridDim.x] block sums and
  unsigned int* ticket;    // a zeroed counter: fixed-order sum; or null: FP64 atomics
  long long n;
  const float *depth, *sil, *normal, *tgt_depth, *tgt_normal, *tgt_sil;
  const uint8_t* mask;
  dist_loss_weights w;
  const int* cnt;
  double* loss;
  float *g_depth, *g_normal, *g_sil;
};

// Per-pixel loss terms and upstream gradients (Sec. B.3; silhouette Eq. 4 of
// Sec. A.3); FP64 block sums.  The means' weights w / |M| and w / n are
// formed once per thread (FP64 division is slow on B300) and each term's
// pixel sum is scaled by them at the end.
__global__ void loss_terms_kernel(LossArgs a) {
  __shared__ double sh[32];
  const double sd = (double)a.w.w_depth / (double)max(*a.cnt, 1);
  const double sn = (double)a.w.w_normal / (double)max(*a.cnt, 1);
  const double ss = (double)a.w.w_sil / (double)a.n;
  const float gd = (float)sd;
  double acc_d = 0.0, acc_n = 0.0, acc_s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n;
       i += (long long)gridDim.x * blockDim.x) {
    const bool M = a.mask[i] && isfinite(a.tgt_depth[i]);
    if (a.w.w_depth != 0.f) {
      const double r = M ? (double)a.depth[i] - (double)a.tgt_depth[i] : 0.0;
      acc_d += fabs(r);
      a.g_depth[i] = r > 0 ? gd : (r < 0 ? -gd : 0.f);
    } else if (a.g_depth) {
      a.g_depth[i] = 0.f;
    }
    if (a.w.w_normal != 0.f) {
      double dot = 0.0;
      for (int e = 0; e < 3; ++e) dot += (double)a.normal[3 * i + e] * (double)a.tgt_normal[3 * i + e];
      if (M) acc_n -= dot;
      for (int e = 0; e < 3; ++e)
        a.g_normal[3 * i + e] = M ? (float)(-sn * a.tgt_normal[3 * i + e]) : 0.f;
    } else if (a.g_normal) {
      for (int e = 0; e < 3; ++e) a.g_normal[3 * i + e] = 0.f;
    }
    if (a.w.w_sil != 0.f) {
      const double S = a.sil[i], Sg = a.tgt_sil[i];
      acc_s += Sg * fmax(0.0, S) + (1.0 - Sg) * fmax(0.0, -S);
      a.g_sil[i] = (float)(ss * (Sg * (S > 0 ? 1.0 : 0.0) - (1.0 - Sg) * (S < 0 ? 1.0 : 0.0)));
    } else if (a.g_sil) {
      a.g_sil[i] = 0.f;
    }
  }
  const double t = block_sum_d(sd * acc_d + sn * acc_n + ss * acc_s, sh);
  if (!a.part) {
    if (threadIdx.x == 0 && t != 0.0) atomicAdd(a.loss, t);
    return;
  }
  // block sums to part[], the last block to finish adds them in block order
  // (one FP64 atomic per block on one word serialised at the L2; this sum
  // is also the same on every run)
  __shared__ bool last;
  if (threadIdx.x == 0) {
    a.part[blockIdx.x] = t;
    __threadfence();
    last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double v = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
    v += reinterpret_cast<volatile const double*>(a.part)[b];
  const double tot = block_sum_d(v, sh);
  if (threadIdx.x == 0) {
    *a.loss += tot;
    *a.ticket = 0u;
  }
}

// ||z||^2 regulariser (Sec. B.4): loss += w sum z^2, dz = 2 w z.
__global__ void loss_reg_kernel(const float* z, long long nz, float w, double* loss, float* dz) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nz;
       i += (long long)gridDim.x * blockDim.x) {
    const double zi = z[i];
    acc += (double)w * zi * zi;
    if (dz) dz[i] = (float)(2.0 * w * zi);
  }
  const double t = block_sum_d(acc, sh);
  if (threadIdx.x == 0 && t != 0.0) atomicAdd(loss, t);
}

// Shape indices are clamped into [0, n_shapes) so no kernel reads outside the
// folded-bias table.
__global__ void pack_points_kernel(const float* __restrict__ pts, const int* __restrict__ shape,
                                   long long n, int n_shapes, float4* out, int* count) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *count = (int)n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int s = min(max(shape[i], 0), n_shapes - 1);
    out[i] = make_float4(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], __int_as_float(s));
  }
}

__global__ void unpack_grad_kernel(const float* out4, long long n, float* f, float* grad) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float4 v = reinterpret_cast<const float4*>(out4)[i];
    f[i] = v.x;
    grad[3 * i] = v.y; grad[3 * i + 1] = v.z; grad[3 * i + 2] = v.w;
  }
}

// -------------------------------------------------------------- host side

int grid_for(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  const long long cap = (long long)num_sms() * 8;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

struct Prepared {
  long long n_pix;
  cudaStream_t st;
};

// Validates the cameras and writes the workspace's camera table; *n_pix is
// the total pixel count (cameras' pixels concatenated in order).
dist_status upload_cameras(const dist_camera* cams, int n_cams, float radius, dist_workspace* ws,
                           cudaStream_t st, long long* n_pix_out) {
  DIST_CHECK(cams && ws, DIST_E_INVALID, "NULL argument");
  DIST_CHECK(n_cams >= 1 && n_cams <= ws->max_cams, DIST_E_INVALID, "n_cams out of range");
  long long n_pix = 0;
  CamChunk ch;
  std::memset(&ch, 0, sizeof(ch));
  for (int c = 0; c < n_cams; ++c) {
    const dist_camera& k = cams[c];
    DIST_CHECK(k.H > 0 && k.W > 0 && (long long)k.H * k.W <= (1ll << 31), DIST_E_INVALID,
               "camera image size out of range");
    DIST_CHECK(k.fx != 0.f && k.fy != 0.f, DIST_E_INVALID, "zero focal length");
    const double cc = (double)k.c[0] * k.c[0] + (double)k.c[1] * k.c[1] + (double)k.c[2] * k.c[2];
    DIST_CHECK(cc > (double)radius * radius, DIST_E_INVALID, "camera inside the bounding sphere");
    CamDev& d = ch.c[c % kCamChunk];
    std::memcpy(d.c, k.c, sizeof(d.c));
    std::memcpy(d.R, k.R, sizeof(d.R));
    d.fx = k.fx; d.fy = k.fy; d.cx = k.cx; d.cy = k.cy;
    d.H = k.H; d.W = k.W; d.shape = k.shape; d.pad = 0;
    d.offset = n_pix;
    n_pix += (long long)k.H * k.W;
    if (c % kCamChunk == kCamChunk - 1 || c == n_cams - 1) {
      ch.n = c % kCamChunk + 1;
      ch.first = c - (c % kCamChunk);
      write_cams_kernel<<<1, 64, 0, st>>>(ch, ws->cams);
      DIST_LAUNCH_CHECK();
    }
  }
  DIST_CHECK(n_pix <= ws->max_rays, DIST_E_INVALID, "more pixels than the workspace holds");
  *n_pix_out = n_pix;
  return DIST_OK;
}

dist_status validate_and_upload(const dist_decoder* dec, const float* z, int n_shapes,
                                const dist_camera* cams, int n_cams,
                                const dist_trace_params* p, const dist_trace_out* o,
                                dist_workspace* ws, void* stream, Prepared* out) {
  DIST_CHECK(dec && z && cams && p && o && ws, DIST_E_INVALID, "NULL argument");
  DIST_CHECK(is_sdf_decoder(dec->desc), DIST_E_INVALID,
             "tracing needs an SDF decoder (out_dim 1, latent_dim0 = latent_dim)");
  DIST_CHECK(n_cams >= 1 && n_cams <= ws->max_cams, DIST_E_INVALID, "n_cams out of range");
  DIST_CHECK(n_shapes >= 1 && n_shapes <= kMaxShapes, DIST_E_INVALID, "n_shapes out of range");
  DIST_CHECK(p->max_steps >= 1 && p->max_steps <= ws->max_steps, DIST_E_INVALID,
             "max_steps must be 1..workspace max_steps");
  DIST_CHECK(p->k_min >= 1 && p->k_min <= kMaxK, DIST_E_INVALID, "k_min must be 1..3");
  DIST_CHECK(p->eps > 0.f && p->alpha > 0.f && p->radius > 0.f && p->normal_delta >= 0.f,
             DIST_E_INVALID, "eps, alpha, radius must be > 0 and normal_delta >= 0");
  DIST_CHECK(valid_precision(p->precision), DIST_E_INVALID, "bad precision");
  DIST_CHECK(p->refine_steps >= 0, DIST_E_INVALID, "refine_steps must be >= 0");
  DIST_CHECK(p->refine_engine == DIST_REFINE_TC || p->refine_engine == DIST_REFINE_SIMT,
             DIST_E_INVALID, "bad refine_engine");
  DIST_CHECK(p->refine_rule == DIST_REFINE_MARCH || p->refine_rule == DIST_REFINE_SECANT,
             DIST_E_INVALID, "bad refine_rule");
  DIST_CHECK(p->grad_mode == DIST_GRAD_EXACT || p->grad_mode == DIST_GRAD_PAPER, DIST_E_INVALID,
             "bad grad_mode");
  DIST_CHECK(p->coarse_levels >= 0 && p->coarse_levels <= kMaxCoarseLevels &&
                 p->coarse_every >= 1,
             DIST_E_INVALID, "coarse_levels must be 0..4 and coarse_every >= 1");
  DIST_CHECK(p->latency_mode == 0 || p->latency_mode == 1, DIST_E_INVALID,
             "latency_mode must be 0 or 1");
  DIST_CHECK(p->coarse_levels == 0 || !is_tc(p->precision) ||
                 (fp32_on_tc(*p) && p->refine_steps == 0),
             DIST_E_INVALID,
             "coarse-to-fine tracing with a BF16/FP16 march needs refine_steps 0 and the TC "
             "refine engine");
  DIST_CHECK(p->precision != DIST_PREC_BF16 || p->eps_mid == 0.f ||
                 (p->eps_mid > 0.f && p->eps_mid < p->eps_bf16 && fp32_on_tc(*p) &&
                  p->refine_steps == 0 && p->refine_rule == DIST_REFINE_MARCH &&
                  p->coarse_levels == 0),
             DIST_E_INVALID,
             "eps_mid (the FP16 stage of a BF16 march) must be 0, or in (0, eps_bf16) with the "
             "TC refine engine, refine_steps 0, the MARCH rule and no coarse-to-fine levels");
  DIST_CHECK(!(is_tc(p->precision) || fp32_on_tc(*p)) || dec->tc.ok, DIST_E_UNSUPPORTED,
             "the tensor-core decoder covers only the DeepSDF shape (512 x 8, skip 4, latent 256)");
  DIST_CHECK(o->depth && o->sil && o->mask && o->steps && o->d_hit && o->d_min && o->f_min,
             DIST_E_INVALID, "dist_trace_out: NULL required buffer");
  cudaStream_t st = (cudaStream_t)stream;
  for (int c = 0; c < n_cams; ++c) {
    DIST_CHECK(cams[c].shape >= 0 && cams[c].shape < n_shapes, DIST_E_INVALID,
               "camera shape index out of range");
    DIST_CHECK(cams[c].H % (1 << p->coarse_levels) == 0 && cams[c].W % (1 << p->coarse_levels) == 0,
               DIST_E_INVALID, "coarse-to-fine tracing: H and W must be multiples of "
               "2^coarse_levels");
  }
  long long n_pix = 0;
  {
    dist_status cs = upload_cameras(cams, n_cams, p->radius, ws, st, &n_pix);
    if (cs != DIST_OK) return cs;
  }
  DIST_CHECK(n_pix <= ws->max_rays, DIST_E_INVALID, "more pixels than the workspace holds");
  const DecoderF32& d = dec->f32;
  dim3 g(n_shapes, 2, (d.width + 7) / 8);   // one output per warp
  fold_bias_kernel<<<g, 256, 0, st>>>(d, z, n_shapes, ws->bfold, ws->bfold + kMaxShapes * 512);
  DIST_LAUNCH_CHECK();
  out->n_pix = n_pix;
  out->st = st;
  return DIST_OK;
}

TraceArgs make_args(const dist_trace_params* p, const dist_trace_out* o, dist_workspace* ws,
                    int n_cams, long long n_pix) {
  TraceArgs a;
  a.cams = ws->cams; a.n_cams = n_cams; a.n_pix = n_pix; a.radius = p->radius; a.K = p->k_min;
  a.pix0 = 0; a.cam_fixed = -1;
  a.eps = p->eps; a.alpha = p->alpha; a.eps_bf16 = p->eps_bf16; a.max_steps = p->max_steps;
  a.eps_mid = p->precision == DIST_PREC_BF16 ? p->eps_mid : 0.f;
  a.refine = is_tc(p->precision) ? p->refine_steps : 0;
  a.secant = is_tc(p->precision) && p->refine_rule == DIST_REFINE_SECANT ? 1 : 0;
  a.alpha_fp32 = (is_tc(p->precision) && p->alpha_refine > 0.f) ? p->alpha_refine : p->alpha;
  a.o = *o; a.st = ws->st; a.dir = ws->dir; a.fq = ws->fq; a.fprev = ws->fprev;
  a.dprev = ws->dprev;
  a.c2f = p->coarse_levels > 0 ? 1 : 0;
  a.c2f_start = is_tc(p->precision) ? -1 : -2;
  a.last = 0;
  if (a.c2f && !a.o.status) a.o.status = ws->rstat;
  return a;
}

ProbeArgs make_probe_args(const dist_trace_params* p, const dist_trace_out* o, dist_workspace* ws,
                          int n_cams, long long n_pix, long long offset, int count_slot) {
  ProbeArgs a;
  a.cams = ws->cams; a.st = ws->st; a.dir = ws->dir; a.n_pix = n_pix; a.n_cams = n_cams;
  a.pix0 = 0; a.cam_fixed = -1;
  a.K = p->k_min; a.o = *o;
  a.pp = ws->probe_p + offset; a.pq = ws->probe_q + offset; a.pix = ws->probe_pix + offset;
  a.count = ws->probe_count + count_slot;
  a.chunk = nullptr;
  a.phase = 0;
  return a;
}

// An ordered append of probes: the kernel's counting phase, the scan of the
// chunk counts (in ws->chunk) and the writing phase.
template <class Launch>
cudaError_t ordered_probes(ProbeArgs a, dist_workspace* ws, long long n_pix, cudaStream_t st,
                           Launch launch) {
  a.chunk = ws->chunk;
  a.phase = 0;
  launch(a);
  count_launch(1);
  const long long n_chunks = (n_pix + 31) / 32;
  chunk_scan_kernel<<<1, 1024, 0, st>>>(a.chunk, n_chunks, a.count);
  count_launch(1);
  a.phase = 1;
  launch(a);
  count_launch(1);
  return cudaGetLastError();
}

// The decoder adjoint in the trace's precision: tcgen05 with BF16 / FP16
// operands after a tensor-core march, with FP32-class operands after an
// FP32_TC trace, FP32 SIMT otherwise.
cudaError_t adjoint(const dist_decoder* dec, const dist_trace_params* p, dist_workspace* ws,
                    const float4* pp, const float4* pq, const int* count, const float* b0,
                    const float* bs, float* out4, double* G0, double* Gs, int acc,
                    cudaStream_t st) {
  if (is_tc(p->precision) && dec->tc.ok)
    return mlp_tc_adjoint(dec, pp, pq, count, b0, bs, out4, G0, Gs, acc, ws->tc_scratch, st,
                          p->precision == DIST_PREC_FP16);
  if (p->precision == DIST_PREC_FP32_TC && dec->tc.ok)
    return mlp_tcx_adjoint(dec, pp, pq, count, b0, bs, out4, G0, Gs, acc, ws->tc_scratch, st);
  return mlp_fp32_adjoint(dec->f32, pp, pq, count, b0, bs, out4, G0, Gs, acc, st);
}

// The decoder adjoint at FP32-class accuracy whatever the march's precision
// (silhouette probes, too few for 16-bit rounding errors to average out, and
// the central-difference probes, whose gradients are differenced): the
// FP32-class tensor-core adjoint where the trace runs its FP32-class queries
// on the tensor cores, else the FP32 CUDA-core adjoint.
// With `redo` (central-difference probes), the probes the FP32-class kernel
// hands back (a ReLU input within kMaskMargin of 0) go through the FP32
// adjoint after it.
constexpr float kMaskMargin = 5e-7f;

cudaError_t fine_adjoint(const dist_decoder* dec, const dist_trace_params* p, dist_workspace* ws,
                         const float4* pp, const float4* pq, const int* count, const float* b0,
                         const float* bs, double* G0, double* Gs, cudaStream_t st,
                         const RedoList* redo = nullptr) {
  if (fp32_on_tc(*p) && dec->tc.ok) {
    cudaError_t e = mlp_tcx_adjoint(dec, pp, pq, count, b0, bs, nullptr, G0, Gs, 1,
                                    ws->tc_scratch, st, redo);
    if (e != cudaSuccess || !redo) return e;
    return mlp_fp32_adjoint(dec->f32, redo->p, redo->q, redo->count, b0, bs, nullptr, G0, Gs, 1,
                            st);
  }
  return mlp_fp32_adjoint(dec->f32, pp, pq, count, b0, bs, nullptr, G0, Gs, 1, st);
}

// Queries of the central-difference probes (normals and their gradient):
// differences of nearby values, so FP32-class precision whatever the march's:
// the FP32_TC tensor-core kernel (two-term FP16 split; its ~2e-6 error in f
// is mostly a common offset that cancels in the differences) when the trace
// runs its FP32-class queries there, else the FP32 CUDA-core kernel.
cudaError_t fd_forward(const dist_decoder* dec, const dist_trace_params* p, const RowSrc& src,
                       const float* b0, const float* bs, float* out, cudaStream_t st) {
  if (fp32_on_tc(*p) && dec->tc.ok) return mlp_tcx_forward(dec, src, b0, bs, out, st);
  return mlp_fp32_forward(dec->f32, src, b0, bs, out, st);
}

dist_status normals_impl(const dist_decoder* dec, const dist_trace_params* p,
                         const dist_trace_out* o, float* normal, dist_workspace* ws,
                         int n_cams, long long n_pix, cudaStream_t st) {
  const float* b0 = ws->bfold;
  const float* bs = ws->bfold + kMaxShapes * 512;
  DIST_CUDA_TRY(cudaMemsetAsync(normal, 0, (size_t)n_pix * 3 * sizeof(float), st));
  DIST_CUDA_TRY(cudaMemsetAsync(ws->probe_count, 0, 8 * sizeof(int), st));
  // |g| beside the normal it belongs to (the forward's own normal buffer)
  float* glen = o->grad_len && normal == o->normal ? o->grad_len : nullptr;
  if (glen) DIST_CUDA_TRY(cudaMemsetAsync(glen, 0, (size_t)n_pix * sizeof(float), st));
  const int g = grid_for(n_pix, 256);
  if (p->normal_delta == 0.f) {
    ProbeArgs a = make_probe_args(p, o, ws, n_cams, n_pix, 0, 0);
    probes_hits_kernel<<<g, 256, 0, st>>>(a);
    DIST_LAUNCH_CHECK();
    DIST_CUDA_TRY(adjoint(dec, p, ws, ws->probe_p, nullptr, ws->probe_count, b0, bs,
                          ws->probe_out, nullptr, nullptr, 0, st));
    normals_from_grad_kernel<<<g, 256, 0, st>>>(ws->probe_out, ws->probe_pix, ws->probe_count,
                                                 normal);
    DIST_LAUNCH_CHECK();
  } else {
    ProbeArgs a = make_probe_args(p, o, ws, n_cams, n_pix, 0, 0);
    probes_fd_kernel<<<g, 256, 0, st>>>(a, p->normal_delta, nullptr);
    DIST_LAUNCH_CHECK();
    RowSrc src{};
    src.count = ws->probe_count;
    src.pts = ws->probe_p;
    DIST_CUDA_TRY(fd_forward(dec, p, src, b0, bs, ws->probe_out, st));
    normals_from_fd_kernel<<<g, 256, 0, st>>>(ws->probe_out, ws->probe_pix, ws->probe_count,
                                               p->normal_delta, normal, glen);
    DIST_LAUNCH_CHECK();
  }
  return DIST_OK;
}

}  // namespace

// Launchers of the point-evaluation kernels for callers that bring their own
// scratch memory instead of a workspace.
cudaError_t launch_fold_bias(const DecoderF32& d, const float* z, int n_shapes, float* bfold0,
                             float* bfolds, cudaStream_t st) {
  dim3 g(n_shapes, 2, (d.width + 7) / 8);   // one output per warp
  fold_bias_kernel<<<g, 256, 0, st>>>(d, z, n_shapes, bfold0, bfolds);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_pack_points(const float* pts, const int* shape, long long n, int n_shapes,
                               float4* out, int* count, cudaStream_t st) {
  pack_points_kernel<<<grid_for(n, 256), 256, 0, st>>>(pts, shape, n, n_shapes, out, count);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_unpack_grad(const float* out4, long long n, float* f, float* grad,
                               cudaStream_t st) {
  unpack_grad_kernel<<<grid_for(n, 256), 256, 0, st>>>(out4, n, f, grad);
  count_launch(1);
  return cudaGetLastError();
}

// ---- serving: the server drives the same kernels one step at a time over a
// pool of rays that belong to many requests (one camera slot per request).

static TraceArgs pool_args(const RayPool& P) {
  TraceArgs a;
  a.cams = P.cams; a.n_cams = 0; a.n_pix = 0; a.pix0 = 0; a.cam_fixed = -1;
  a.radius = P.radius; a.K = P.K; a.eps = P.eps; a.alpha = P.alpha; a.eps_bf16 = P.eps_bf16;
  a.max_steps = P.max_steps; a.o = P.o; a.st = P.st; a.dir = P.dir;
  a.fq = P.fq; a.fprev = P.fprev; a.dprev = P.dprev; a.refine = P.refine;
  a.secant = P.secant; a.alpha_fp32 = P.alpha_fp32;
  a.eps_mid = P.eps_mid;
  a.c2f = 0; a.c2f_start = 0; a.last = 0;
  return a;
}

cudaError_t pool_write_cam(const CamDev& c, int slot, CamDev* dst, cudaStream_t st) {
  CamChunk ch;
  std::memset(&ch, 0, sizeof(ch));
  ch.c[0] = c;
  ch.n = 1;
  ch.first = slot;
  write_cams_kernel<<<1, 64, 0, st>>>(ch, dst);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t pool_raygen(const RayPool& P, int cam, long long pix0, long long n, int* list0,
                        int* count0, cudaStream_t st) {
  TraceArgs a = pool_args(P);
  a.n_pix = n; a.pix0 = pix0; a.cam_fixed = cam;
  raygen_kernel<<<grid_for(n, 256), 256, 0, st>>>(a, 0, list0, count0);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t pool_step(const RayPool& P, const int* cnt_in, int* cnt_out, int* const in[2],
                      const float* const f[2], int* const out[2], cudaStream_t st) {
  StepLists L;
  L.cnt_in[0] = cnt_in; L.cnt_in[1] = cnt_in + 1;
  L.cnt_out[0] = cnt_out; L.cnt_out[1] = cnt_out + 1;
  for (int k = 0; k < 2; ++k) { L.in[k] = in[k]; L.f[k] = f[k]; L.out[k] = out[k]; }
  step_kernel<<<num_sms() * 4, kStepThreads, 0, st>>>(pool_args(P), L, P.o.queries);
  count_launch(1);
  return cudaGetLastError();
}

void pool_step_fuse(const RayPool& P, int* cnt_out, int* const out[2], StepFuse* sf) {
  sf->t = pool_args(P);
  for (int k = 0; k < 2; ++k) { sf->out[k] = out[k]; sf->cnt_out[k] = cnt_out + k; }
  sf->out[2] = nullptr;   // set by the caller when the march has an FP16 stage
  sf->cnt_out[2] = nullptr;
  sf->queries = P.o.queries;
  sf->wide = nullptr;
  sf->seq_flag = nullptr;   // set with `wide` by the caller
  sf->seq = 0;
}

cudaError_t pool_probes_depth(const RayPool& P, int cam, long long pix0, long long n,
                              const float* g_depth, float4* pp, float4* pq, int* pix, int* count,
                              cudaStream_t st) {
  ProbeArgs a;
  a.cams = P.cams; a.st = P.st; a.dir = P.dir; a.n_pix = n; a.pix0 = pix0; a.cam_fixed = cam;
  a.n_cams = 0; a.K = P.K; a.o = P.o; a.pp = pp; a.pq = pq; a.pix = pix; a.count = count;
  a.chunk = nullptr; a.phase = 0;
  probes_bwd_kernel<<<grid_for(n, 256), 256, 0, st>>>(a, g_depth, nullptr, 0, P.alpha);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t pool_loss_depth(long long n, const float* depth, const uint8_t* mask, const float* tgt,
                            double* loss, float* g_depth, int* cnt, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  loss_count_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, mask, tgt, cnt);
  LossArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = n; a.depth = depth; a.tgt_depth = tgt; a.mask = mask; a.cnt = cnt; a.loss = loss;
  a.g_depth = g_depth;
  a.w.w_depth = 1.f;
  loss_terms_kernel<<<grid_for(n, 256), 256, 0, st>>>(a);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t pool_latent_finalize(const DecoderF32& d, const double* G0, const double* Gs,
                                 float* dz, cudaStream_t st) {
  dim3 fg((d.latent + 31) / 32, 1);
  latent_finalize_kernel<<<fg, kFinalizeWarps * 32, 0, st>>>(d, G0, Gs, 1, dz);
  count_launch(1);
  return cudaGetLastError();
}

}  // namespace dist

using namespace dist;

extern "C" {

dist_status dist_trace_fwd(const dist_decoder* dec, const float* z, int n_shapes,
                           const dist_camera* cams, int n_cams, const dist_trace_params* p,
                           const dist_trace_out* o, dist_workspace* ws, void* stream) {
  DIST_NVTX("dist_trace_fwd");
  Prepared pr;
  dist_status s = validate_and_upload(dec, z, n_shapes, cams, n_cams, p, o, ws, stream, &pr);
  if (s != DIST_OK) return s;
  cudaStream_t st = pr.st;
  const long long n_pix = pr.n_pix;
  TraceArgs a = make_args(p, o, ws, n_cams, n_pix);
  // list lengths: cA[s] low-precision list at step s, cB[t] FP32 list at
  // FP32 step t, a constant zero for a list that is not used, and the two
  // lists made by each coarse-to-fine split
  const int M = p->max_steps;
  int* cA = ws->counts;
  int* cB = ws->counts + (M + 1);
  int* zero = ws->counts + 2 * (M + 1);
  int* cSplit = zero + 1;
  int* cC = cSplit + 2 * kMaxCoarseLevels;   // FP16-stage list of a BF16 march
  DIST_CUDA_TRY(cudaMemsetAsync(
      ws->counts, 0, (size_t)(3 * (M + 1) + 1 + 2 * kMaxCoarseLevels) * sizeof(int), st));
  const bool tc = is_tc(p->precision);
  const int L = p->coarse_levels;
  // coarse-to-fine: rays start 2^L coarser per side; before march iteration
  // `every * k` (k = 1..L) every ray splits into its four children
  int level = L;
  auto split_due = [&](int it) { return level > 0 && it == p->coarse_every * (L - level + 1); };
  int par = 0;
  auto split = [&](int final, const int*& in0, const int*& in1) -> cudaError_t {
    int* c0 = cSplit + 2 * (L - level);
    split_kernel<<<grid_for(n_pix >> (2 * level), 256), 256, 0, st>>>(
        a, level, final, ws->act[par ^ 1][0], ws->act[par ^ 1][1], c0, c0 + 1);
    count_launch(1);
    --level;
    par ^= 1;
    in0 = c0;
    in1 = c0 + 1;
    return cudaGetLastError();
  };
  const long long n0 = n_pix >> (2 * L);
  if (tc)
    raygen_kernel<<<grid_for(n0, 256), 256, 0, st>>>(a, L, ws->act[0][0], cA);
  else
    raygen_kernel<<<grid_for(n0, 256), 256, 0, st>>>(a, L, ws->act[0][1], cB);
  DIST_LAUNCH_CHECK();
  const float* b0 = ws->bfold;
  const float* bs = ws->bfold + kMaxShapes * 512;
  const int step_grid = num_sms() * 4;
  RowSrc src{};
  src.st = ws->st; src.dir = ws->dir; src.cams = ws->cams;
  if (fp32_on_tc(*p)) {
    // Tensor-core march with FP32-class tensor-core queries (to convergence,
    // or refine_steps of them; FP32_TC: every query, the 16-bit list stays
    // empty): one launch per step decodes both lists
    // (16-bit rows and handed-over rays), so the two share the latency of
    // the shrinking tail of steps, which the latency mode shortens.  (With
    // refine_steps > 0 this measured faster than one deferred batch of the
    // FP32-class queries after the 16-bit march.)
    const int* in0 = cA;
    const int* in1 = cB;
    const int* in2 = cC;
    const bool mid = a.eps_mid > 0.f;
    for (int s = 0; s < M; ++s) {
      DIST_NVTX("march step");
      if (split_due(s)) DIST_CUDA_TRY(split(0, in0, in1));
      RowSrc sx = src;
      RowSrc sm = src;
      src.count = in0;
      src.idx = ws->act[par][0];
      sx.count = in1;
      sx.idx = ws->act[par][1];
      sm.count = in2;
      sm.idx = ws->act[par][2];
      // the decoder kernel applies the step update itself
      StepFuse sf;
      sf.t = a;
      sf.t.last = a.c2f && s == M - 1;
      for (int k = 0; k < 3; ++k) sf.out[k] = ws->act[par ^ 1][k];
      sf.cnt_out[0] = cA + s + 1; sf.cnt_out[1] = cB + s + 1; sf.cnt_out[2] = cC + s + 1;
      sf.queries = o->queries;
      sf.wide = p->latency_mode ? static_cast<uint8_t*>(ws->wide_scratch) : nullptr;
      sf.seq_flag = tc_wide_seq_flag(ws->wide_scratch);
      sf.seq = ++ws->step_seq;
      prof_mlp_begin(st, 0);
      DIST_CUDA_TRY(mlp_tc_fused(dec, src, ws->fbuf[0], sx, ws->fbuf[1], b0, bs, st,
                                 p->precision == DIST_PREC_FP16, &sf, mid ? &sm : nullptr,
                                 ws->fbuf[2]));
      prof_mlp_end(st);
      in0 = cA + s + 1;
      in1 = cB + s + 1;
      in2 = cC + s + 1;
      par ^= 1;
    }
    while (level > 0) DIST_CUDA_TRY(split(1, in0, in1));
    if (o->normal) return normals_impl(dec, p, o, o->normal, ws, n_cams, n_pix, st);
    return DIST_OK;
  }
  if (tc) {
    // Tensor-core march with FP32 CUDA-core queries.  Rays whose
    // low-precision |f| is small enough move to one FP32 list that grows
    // over all steps: their FP32 queries run together afterwards instead of
    // as a small launch every step.  A ray's result does not depend on when
    // its queries run.  (No coarse-to-fine here: validated.)
    for (int s = 0; s < M; ++s) {
      const int par = s & 1;
      src.count = cA + s;
      src.idx = ws->act[par][0];
      prof_mlp_begin(st, 0);
      DIST_CUDA_TRY(mlp_tc_forward(dec, src, b0, bs, ws->fbuf[0], st,
                                   p->precision == DIST_PREC_FP16));
      prof_mlp_end(st);
      StepLists L;
      L.cnt_in[0] = cA + s; L.cnt_in[1] = zero;
      L.cnt_out[0] = cA + s + 1; L.cnt_out[1] = cB;
      L.in[0] = ws->act[par][0]; L.in[1] = ws->act[0][1];
      L.f[0] = ws->fbuf[0]; L.f[1] = ws->fbuf[1];
      L.out[0] = ws->act[par ^ 1][0]; L.out[1] = ws->act[0][1];
      step_kernel<<<step_grid, kStepThreads, 0, st>>>(a, L, o->queries);
      DIST_LAUNCH_CHECK();
    }
  }
  // FP32 march (all rays for FP32 precision; the handed-over rays otherwise).
  // After the tensor-core march the first FP32 launch holds every handed-over
  // ray (64-row tiles for throughput); the shrinking tail after it runs in
  // 16-row tiles, whose launch latency is a quarter of a 64-row tile's.
  const int* in0 = zero;
  const int* in1 = cB;
  for (int t = 0; t < M; ++t) {
    DIST_NVTX("march step (FP32 list)");
    if (split_due(t)) DIST_CUDA_TRY(split(0, in0, in1));
    src.count = in1;
    src.idx = ws->act[par][1];
    prof_mlp_begin(st, 1);
    // (FP32-class queries on the tensor cores take the fused march above)
    DIST_CUDA_TRY(mlp_fp32_forward(dec->f32, src, b0, bs, ws->fbuf[1], st, tc && t > 0));
    prof_mlp_end(st);
    StepLists L;
    L.cnt_in[0] = zero; L.cnt_in[1] = in1;
    L.cnt_out[0] = zero; L.cnt_out[1] = cB + t + 1;
    L.in[0] = ws->act[0][0]; L.in[1] = ws->act[par][1];
    L.f[0] = ws->fbuf[0]; L.f[1] = ws->fbuf[1];
    L.out[0] = ws->act[0][0]; L.out[1] = ws->act[par ^ 1][1];
    TraceArgs at = a;
    at.last = a.c2f && t == M - 1;
    step_kernel<<<step_grid, kStepThreads, 0, st>>>(at, L, o->queries);
    DIST_LAUNCH_CHECK();
    in1 = cB + t + 1;
    par ^= 1;
  }
  while (level > 0) DIST_CUDA_TRY(split(1, in0, in1));
  if (o->normal) return normals_impl(dec, p, o, o->normal, ws, n_cams, n_pix, st);
  return DIST_OK;
}

dist_status dist_render_normals(const dist_decoder* dec, const float* z, int n_shapes,
                                const dist_camera* cams, int n_cams, const dist_trace_params* p,
                                const dist_trace_out* fwd, float* normal, dist_workspace* ws,
                                void* stream) {
  DIST_NVTX("dist_render_normals");
  DIST_CHECK(normal, DIST_E_INVALID, "dist_render_normals: NULL normal");
  Prepared pr;
  dist_status s = validate_and_upload(dec, z, n_shapes, cams, n_cams, p, fwd, ws, stream, &pr);
  if (s != DIST_OK) return s;
  return normals_impl(dec, p, fwd, normal, ws, n_cams, pr.n_pix, pr.st);
}

dist_status dist_trace_bwd(const dist_decoder* dec, const float* z, int n_shapes,
                           const dist_camera* cams, int n_cams, const dist_trace_params* p,
                           const dist_trace_out* fwd, const float* g_depth,
                           const float* g_normal, const float* g_sil, float* dz,
                           dist_workspace* ws, void* stream) {
  DIST_NVTX("dist_trace_bwd");
  DIST_CHECK(dz, DIST_E_INVALID, "dist_trace_bwd: NULL dz");
  DIST_CHECK(!g_normal || p == nullptr || p->normal_delta > 0.f, DIST_E_INVALID,
             "dist_trace_bwd: a normal gradient needs normal_delta > 0 (the analytic normal of a "
             "ReLU decoder has zero latent gradient almost everywhere)");
  Prepared pr;
  dist_status s = validate_and_upload(dec, z, n_shapes, cams, n_cams, p, fwd, ws, stream, &pr);
  if (s != DIST_OK) return s;
  cudaStream_t st = pr.st;
  const long long n_pix = pr.n_pix;
  const DecoderF32& d = dec->f32;
  const float* b0 = ws->bfold;
  const float* bs = ws->bfold + kMaxShapes * 512;
  double* G0 = ws->gacc;
  double* Gs = ws->gacc + kMaxShapes * 512;
  DIST_CUDA_TRY(cudaMemsetAsync(G0, 0, (size_t)n_shapes * d.width * sizeof(double), st));
  DIST_CUDA_TRY(cudaMemsetAsync(Gs, 0, (size_t)n_shapes * d.width * sizeof(double), st));
  DIST_CUDA_TRY(cudaMemsetAsync(ws->probe_count, 0, 8 * sizeof(int), st));
  const int g = grid_for(n_pix, 256);
  if (g_depth) {
    // depth probes (<= k_min per pixel) in [0, 3 max_rays), in the trace's precision
    ProbeArgs a = make_probe_args(p, fwd, ws, n_cams, n_pix, 0, 0);
    const int paper = p->grad_mode == DIST_GRAD_PAPER;
    const float alpha = p->alpha;
    DIST_CUDA_TRY(ordered_probes(a, ws, n_pix, st, [&](const ProbeArgs& b) {
      probes_bwd_kernel<<<g, 256, 0, st>>>(b, g_depth, nullptr, paper, alpha);
    }));
    DIST_CUDA_TRY(adjoint(dec, p, ws, ws->probe_p, ws->probe_q, ws->probe_count, b0, bs, nullptr,
                          G0, Gs, 1, st));
  }
  if (g_sil) {
    // silhouette probes (<= 1 per pixel) in [3, 4) max_rays: only rays whose
    // soft silhouette disagrees with the target contribute, too few for
    // 16-bit rounding errors to average out, so an FP32-class adjoint
    const long long off = 3 * (long long)ws->max_rays;
    ProbeArgs a = make_probe_args(p, fwd, ws, n_cams, n_pix, off, 2);
    const float alpha = p->alpha;
    DIST_CUDA_TRY(ordered_probes(a, ws, n_pix, st, [&](const ProbeArgs& b) {
      probes_bwd_kernel<<<g, 256, 0, st>>>(b, nullptr, g_sil, 0, alpha);
    }));
    DIST_CUDA_TRY(fine_adjoint(dec, p, ws, ws->probe_p + off, ws->probe_q + off,
                               ws->probe_count + 2, b0, bs, G0, Gs, st));
  }
  if (g_normal) {
    // central-difference normals difference nearby values: FP32-class
    // queries (fd_forward) and an FP32-class adjoint whatever the march precision
    const long long off = 4 * (long long)ws->max_rays;
    ProbeArgs a = make_probe_args(p, fwd, ws, n_cams, n_pix, off, 1);
    const float delta = p->normal_delta;
    DIST_CUDA_TRY(ordered_probes(a, ws, n_pix, st, [&](const ProbeArgs& b) {
      probes_fd_kernel<<<g, 256, 0, st>>>(b, delta, g_normal);
    }));
    if (fwd->normal && fwd->grad_len) {
      // the forward's central difference: its normal and |g| give the
      // coefficients without evaluating the probes again
      fd_coef_from_normal_kernel<<<g, 256, 0, st>>>(fwd->normal, fwd->grad_len,
                                                    ws->probe_pix + off, ws->probe_count + 1,
                                                    p->normal_delta, g_normal,
                                                    ws->probe_q + off);
    } else {
      RowSrc src{};
      src.count = ws->probe_count + 1;
      src.pts = ws->probe_p + off;
      float* f6 = ws->probe_out + off * 4;
      DIST_CUDA_TRY(fd_forward(dec, p, src, b0, bs, f6, st));
      fd_coef_kernel<<<g, 256, 0, st>>>(f6, ws->probe_pix + off, ws->probe_count + 1,
                                        p->normal_delta, g_normal, ws->probe_q + off);
    }
    DIST_LAUNCH_CHECK();
    // the redo list lives in the probe outputs of these probes (their f,
    // read by fd_coef_kernel, is no longer needed): two float4 arrays
    const long long cap = ((long long)kProbesPerRay * ws->max_rays - off) / 2;
    float4* redo_p = reinterpret_cast<float4*>(ws->probe_out + off * 4);
    RedoList redo{redo_p, redo_p + cap, ws->probe_count + 4, (int)std::min<long long>(cap, INT_MAX),
                  kMaskMargin};
    DIST_CUDA_TRY(fine_adjoint(dec, p, ws, ws->probe_p + off, ws->probe_q + off,
                               ws->probe_count + 1, b0, bs, G0, Gs, st, &redo));
  }
  dim3 fg((d.latent + 31) / 32, n_shapes);
  latent_finalize_kernel<<<fg, kFinalizeWarps * 32, 0, st>>>(d, G0, Gs, n_shapes, dz);
  DIST_LAUNCH_CHECK();
  return DIST_OK;
}

dist_status dist_trace_bwd_camera(const dist_decoder* dec, const float* z, int n_shapes,
                                  const dist_camera* cams, int n_cams, const dist_trace_params* p,
                                  const dist_trace_out* fwd, const float* g_depth,
                                  const float* g_sil, float* dcam, dist_workspace* ws,
                                  void* stream) {
  DIST_NVTX("dist_trace_bwd_camera");
  DIST_CHECK(dcam, DIST_E_INVALID, "dist_trace_bwd_camera: NULL dcam");
  Prepared pr;
  dist_status s = validate_and_upload(dec, z, n_shapes, cams, n_cams, p, fwd, ws, stream, &pr);
  if (s != DIST_OK) return s;
  cudaStream_t st = pr.st;
  const long long n_pix = pr.n_pix;
  const float* b0 = ws->bfold;
  const float* bs = ws->bfold + kMaxShapes * 512;
  double* G = ws->gacc;   // [n_cams][12] (the latent accumulators are free here)
  DIST_CUDA_TRY(cudaMemsetAsync(G, 0, (size_t)n_cams * 12 * sizeof(double), st));
  DIST_CUDA_TRY(cudaMemsetAsync(ws->probe_count, 0, 8 * sizeof(int), st));
  const int g = grid_for(n_pix, 256);
  ProbeArgs a = make_probe_args(p, fwd, ws, n_cams, n_pix, 0, 0);
  if (g_depth || g_sil) {
    probes_cam_kernel<<<g, 256, 0, st>>>(a, g_depth, g_sil);
    DIST_LAUNCH_CHECK();
    DIST_CUDA_TRY(adjoint(dec, p, ws, ws->probe_p, nullptr, ws->probe_count, b0, bs,
                          ws->probe_out, nullptr, nullptr, 0, st));
    cam_probe_grad_kernel<<<grid_for(2 * n_pix, 256), 256, 0, st>>>(a, ws->probe_out, g_depth,
                                                                     g_sil, G);
    DIST_LAUNCH_CHECK();
  }
  if (g_sil) {
    cam_miss_grad_kernel<<<g, 256, 0, st>>>(a, g_sil, G);
    DIST_LAUNCH_CHECK();
  }
  cam_finalize_kernel<<<grid_for(n_cams * 12, 256), 256, 0, st>>>(G, n_cams * 12, dcam);
  DIST_LAUNCH_CHECK();
  return DIST_OK;
}

dist_status dist_photo_loss(const dist_camera* cams, int n_cams, const float* depth,
                           const float* images, int channels, const int32_t* pairs, int n_pairs,
                           float w, double* loss, float* g_depth, dist_workspace* ws,
                           void* stream) {
  DIST_NVTX("dist_photo_loss");
  DIST_CHECK(cams && depth && images && pairs && loss && g_depth && ws, DIST_E_INVALID,
             "dist_photo_loss: NULL argument");
  DIST_CHECK(channels >= 1 && channels <= 4, DIST_E_INVALID, "dist_photo_loss: channels 1..4");
  DIST_CHECK(n_pairs >= 1, DIST_E_INVALID, "dist_photo_loss: no pair");
  for (int k = 0; k < n_pairs; ++k)
    DIST_CHECK(pairs[2 * k] >= 0 && pairs[2 * k] < n_cams && pairs[2 * k + 1] >= 0 &&
                   pairs[2 * k + 1] < n_cams,
               DIST_E_INVALID, "dist_photo_loss: view index out of range");
  cudaStream_t st = (cudaStream_t)stream;
  long long n_pix = 0;
  {
    dist_status cs = upload_cameras(cams, n_cams, 0.f, ws, st, &n_pix);
    if (cs != DIST_OK) return cs;
  }
  DIST_CUDA_TRY(cudaMemsetAsync(g_depth, 0, (size_t)n_pix * sizeof(float), st));
  DIST_CUDA_TRY(cudaMemsetAsync(ws->red, 0, 2 * sizeof(double), st));
  for (int k = 0; k < n_pairs; ++k) {
    PhotoArgs a;
    a.cams = ws->cams;
    a.vi = pairs[2 * k];
    a.vj = pairs[2 * k + 1];
    a.depth = depth;
    a.img = images;
    a.C = channels;
    a.vis_thresh = 1e-3;
    a.sums = ws->red;
    a.g_depth = g_depth;
    photo_pair_kernel<<<grid_for((long long)cams[a.vi].H * cams[a.vi].W, 256), 256, 0, st>>>(a);
    DIST_LAUNCH_CHECK();
  }
  photo_finalize_kernel<<<grid_for(n_pix, 256), 256, 0, st>>>(ws->red, (double)w, n_pix, g_depth,
                                                              loss);
  DIST_LAUNCH_CHECK();
  return DIST_OK;
}

dist_status dist_render_color(const dist_decoder* tex, const float* codes, int n_shapes,
                              const dist_camera* cams, int n_cams, const dist_trace_out* fwd,
                              int precision, float* rgb, dist_workspace* ws, void* stream) {
  DIST_NVTX("dist_render_color");
  DIST_CHECK(tex && codes && cams && fwd && rgb && ws, DIST_E_INVALID,
             "dist_render_color: NULL argument");
  DIST_CHECK(tex->f32.out_dim == 3, DIST_E_INVALID, "dist_render_color: decoder out_dim must be 3");
  DIST_CHECK(fwd->mask && fwd->d_hit, DIST_E_INVALID, "dist_render_color: NULL trace output");
  DIST_CHECK(n_shapes >= 1 && n_shapes <= kMaxShapes, DIST_E_INVALID, "n_shapes out of range");
  DIST_CHECK(precision == DIST_PREC_FP32 || is_tc(precision), DIST_E_INVALID,
             "dist_render_color: precision must be FP32, BF16 or FP16");
  DIST_CHECK(precision == DIST_PREC_FP32 || tex->tc.ok, DIST_E_UNSUPPORTED,
             "the tensor-core decoder covers only the DeepSDF layer shape");
  for (int c = 0; c < n_cams; ++c)
    DIST_CHECK(cams[c].shape >= 0 && cams[c].shape < n_shapes, DIST_E_INVALID,
               "camera shape index out of range");
  cudaStream_t st = (cudaStream_t)stream;
  long long n_pix = 0;
  {
    dist_status cs = upload_cameras(cams, n_cams, 0.f, ws, st, &n_pix);
    if (cs != DIST_OK) return cs;
  }
  float* b0 = ws->bfold;
  float* bs = ws->bfold + kMaxShapes * 512;
  DIST_CUDA_TRY(launch_fold_bias(tex->f32, codes, n_shapes, b0, bs, st));
  DIST_CUDA_TRY(cudaMemsetAsync(rgb, 0, (size_t)n_pix * 3 * sizeof(float), st));
  DIST_CUDA_TRY(cudaMemsetAsync(ws->probe_count, 0, 8 * sizeof(int), st));
  ProbeArgs a;
  std::memset(&a, 0, sizeof(a));
  a.cams = ws->cams; a.st = ws->st; a.dir = ws->dir; a.n_pix = n_pix; a.n_cams = n_cams;
  a.cam_fixed = -1; a.K = 1; a.o = *fwd;
  a.pp = ws->probe_p; a.pq = ws->probe_q; a.pix = ws->probe_pix; a.count = ws->probe_count;
  const int g = grid_for(n_pix, 256);
  probes_hits_kernel<<<g, 256, 0, st>>>(a);
  DIST_LAUNCH_CHECK();
  RowSrc src{};
  src.count = ws->probe_count;
  src.pts = ws->probe_p;
  if (precision == DIST_PREC_FP32) {
    DIST_CUDA_TRY(mlp_fp32_forward(tex->f32, src, b0, bs, ws->probe_out, st));
    color_scatter_kernel<<<g, 256, 0, st>>>(ws->probe_out, ws->probe_pix, ws->probe_count, rgb);
  } else {
    DIST_CUDA_TRY(mlp_tc_color(tex, src, b0, bs, ws->fbuf[0], ws->probe_out, st,
                               precision == DIST_PREC_FP16));
    color_finalize_kernel<<<g, 256, 0, st>>>(ws->probe_out, ws->probe_pix, ws->probe_count,
                                             tex->f32.b_out[0], tex->f32.b_out[1],
                                             tex->f32.b_out[2], rgb);
  }
  DIST_LAUNCH_CHECK();
  return DIST_OK;
}

dist_status dist_sdf_eval(const dist_decoder* dec, const float* z, int n_shapes,
                          const float* pts, const int32_t* shape, int64_t n, int precision,
                          float* f, float* grad, dist_workspace* ws, void* stream) {
  DIST_NVTX("dist_sdf_eval");
  DIST_CHECK(dec && z && pts && shape && f && ws, DIST_E_INVALID, "dist_sdf_eval: NULL argument");
  DIST_CHECK(is_sdf_decoder(dec->desc), DIST_E_INVALID,
             "dist_sdf_eval needs an SDF decoder (out_dim 1, latent_dim0 = latent_dim)");
  DIST_CHECK(n >= 1 && n <= ws->max_rays * kProbesPerRay, DIST_E_INVALID,
             "dist_sdf_eval: n must be 1..10 * workspace max_rays");
  DIST_CHECK(n_shapes >= 1 && n_shapes <= kMaxShapes, DIST_E_INVALID, "n_shapes out of range");
  DIST_CHECK(precision == DIST_PREC_FP32 || precision == DIST_PREC_FP32_TC ||
                 (valid_precision(precision) && !grad),
             DIST_E_INVALID,
             "dist_sdf_eval: bad precision (gradients need FP32 or FP32_TC)");
  DIST_CHECK(precision == DIST_PREC_FP32 || dec->tc.ok, DIST_E_UNSUPPORTED,
             "BF16 tensor-core MLP covers only the DeepSDF decoder shape");
  cudaStream_t st = (cudaStream_t)stream;
  const DecoderF32& d = dec->f32;
  dim3 fg(n_shapes, 2, (d.width + 7) / 8);
  fold_bias_kernel<<<fg, 256, 0, st>>>(d, z, n_shapes, ws->bfold, ws->bfold + kMaxShapes * 512);
  DIST_LAUNCH_CHECK();
  const float* b0 = ws->bfold;
  const float* bs = ws->bfold + kMaxShapes * 512;
  const int g = grid_for(n, 256);
  pack_points_kernel<<<g, 256, 0, st>>>(pts, shape, n, n_shapes, ws->probe_p, ws->probe_count);
  DIST_LAUNCH_CHECK();
  RowSrc src{};
  src.count = ws->probe_count;
  src.pts = ws->probe_p;
  if (is_tc(precision)) {
    DIST_CUDA_TRY(mlp_tc_forward(dec, src, b0, bs, f, st, precision == DIST_PREC_FP16));
  } else if (precision == DIST_PREC_FP32_TC && !grad) {
    DIST_CUDA_TRY(mlp_tcx_forward(dec, src, b0, bs, f, st));
  } else if (precision == DIST_PREC_FP32_TC) {
    // f and grad_p f from the FP32-class adjoint (its own forward recompute)
    DIST_CUDA_TRY(mlp_tcx_adjoint(dec, ws->probe_p, nullptr, ws->probe_count, b0, bs,
                                  ws->probe_out, nullptr, nullptr, 0, ws->tc_scratch, st));
    unpack_grad_kernel<<<g, 256, 0, st>>>(ws->probe_out, n, f, grad);
    DIST_LAUNCH_CHECK();
  } else if (!grad) {
    DIST_CUDA_TRY(mlp_fp32_forward(d, src, b0, bs, f, st));
  } else {
    DIST_CUDA_TRY(mlp_fp32_adjoint(d, ws->probe_p, nullptr, ws->probe_count, b0, bs,
                                   ws->probe_out, nullptr, nullptr, 0, st));
    unpack_grad_kernel<<<g, 256, 0, st>>>(ws->probe_out, n, f, grad);
    DIST_LAUNCH_CHECK();
  }
  return DIST_OK;
}

dist_status dist_loss(int64_t n, const float* depth, const uint8_t* mask, const float* sil,
                      const float* normal, const float* tgt_depth, const float* tgt_normal,
                      const float* tgt_sil, const float* z, int n_shapes, int latent_dim,
                      const dist_loss_weights* w, double* loss, float* g_depth, float* g_normal,
                      float* g_sil, float* dz, dist_workspace* ws, void* stream) {
  DIST_NVTX("dist_loss");
  DIST_CHECK(n >= 1 && depth && mask && tgt_depth && w && loss && ws, DIST_E_INVALID,
             "dist_loss: NULL argument or empty batch");
  DIST_CHECK(w->w_depth == 0.f || g_depth, DIST_E_INVALID, "dist_loss: g_depth required");
  DIST_CHECK(w->w_normal == 0.f || (normal && tgt_normal && g_normal), DIST_E_INVALID,
             "dist_loss: normal terms need normal, tgt_normal and g_normal");
  DIST_CHECK(w->w_sil == 0.f || (sil && tgt_sil && g_sil), DIST_E_INVALID,
             "dist_loss: silhouette terms need sil, tgt_sil and g_sil");
  DIST_CHECK(w->w_reg == 0.f || (z && n_shapes > 0 && latent_dim > 0), DIST_E_INVALID,
             "dist_loss: regulariser needs z");
  cudaStream_t st = (cudaStream_t)stream;
  DIST_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(double), st));
  DIST_CUDA_TRY(cudaMemsetAsync(ws->ired, 0, 2 * sizeof(int), st));
  const int g = grid_for(n, 256);
  loss_count_kernel<<<g, 256, 0, st>>>(n, mask, tgt_depth, ws->ired);
  DIST_LAUNCH_CHECK();
  LossArgs a;
  // block sums in the FP64 accumulators of the backward pass, which zeroes
  // them before its own use
  a.part = ws->gacc;
  a.ticket = reinterpret_cast<unsigned int*>(ws->ired + 1);
  a.n = n; a.depth = depth; a.sil = sil; a.normal = normal; a.tgt_depth = tgt_depth;
  a.tgt_normal = tgt_normal; a.tgt_sil = tgt_sil; a.mask = mask; a.w = *w; a.cnt = ws->ired;
  a.loss = loss; a.g_depth = g_depth; a.g_normal = g_normal; a.g_sil = g_sil;
  loss_terms_kernel<<<std::min(g, 2 * num_sms()), 256, 0, st>>>(a);
  DIST_LAUNCH_CHECK();
  if (dz && z && n_shapes > 0 && latent_dim > 0) {
    const long long nz = (long long)n_shapes * latent_dim;
    loss_reg_kernel<<<grid_for(nz, 256), 256, 0, st>>>(z, nz, w->w_reg, loss, dz);
    DIST_LAUNCH_CHECK();
  }
  return DIST_OK;
}

}  // extern "C"
