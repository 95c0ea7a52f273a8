// FP32 SIMT decoder kernels: the FP32-parity path and the plain FP32 GPU
// baseline.  f(p, z) is the DeepSDF decoder (Sec. B.1) with the latent
// columns of layer 0 and of the skip layer folded into per-shape biases
// (b' = W_z z + b), which is algebraically the concatenated input [z, p].
//
// Tiling: a CTA owns TM rows (queries).  Warp w owns rows 4w..4w+3; lane l
// owns the float4 column groups 4l + 128q (q < WIDTH/128), so each thread
// keeps a 4 x 4*(WIDTH/128) accumulator block.  Activations of the current
// layer live in shared memory (TM x WIDTH fp32); weights stream from L2 as
// coalesced float4 rows of a pre-transposed copy.
#include "common.cuh"

namespace dist {

namespace {

constexpr int kFwdRows = 64;   // rows per CTA, forward
constexpr int kAdjRows = 32;   // rows per CTA, adjoint

template <int WIDTH>
struct Tile {
  static constexpr int Q = WIDTH / 128;   // float4 column groups per lane
};

// acc[r][q] += A[r][0:K] . Wt[0:K][col(q)]  for the RPT rows of this warp.
// With 8 rows per thread every weight float4 feeds 32 FMAs, halving the L1
// weight traffic per FMA of the 4-row tile.
template <int WIDTH, int RPT = 4>
__device__ __forceinline__ void gemm_rows(float4 (&acc)[RPT][WIDTH / 128], const float* A,
                                          int row0, const float* __restrict__ Wt, int K,
                                          int lane) {
  constexpr int Q = WIDTH / 128;
  const float4* W4 = reinterpret_cast<const float4*>(Wt);
  if constexpr (RPT > 4) {
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
      float4 w[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) w[q] = __ldg(W4 + k * (WIDTH / 4) + lane + 32 * q);
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        const float av = A[(row0 + r) * WIDTH + k];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          acc[r][q].x = fmaf(av, w[q].x, acc[r][q].x);
          acc[r][q].y = fmaf(av, w[q].y, acc[r][q].y);
          acc[r][q].z = fmaf(av, w[q].z, acc[r][q].z);
          acc[r][q].w = fmaf(av, w[q].w, acc[r][q].w);
        }
      }
    }
    return;
  }
  for (int k = 0; k < K; k += 4) {
    float4 a[4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
      a[r] = *reinterpret_cast<const float4*>(A + (row0 + r) * WIDTH + k);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      float4 w[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) w[q] = __ldg(W4 + (k + kk) * (WIDTH / 4) + lane + 32 * q);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float av = kk == 0 ? a[r].x : kk == 1 ? a[r].y : kk == 2 ? a[r].z : a[r].w;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          acc[r][q].x = fmaf(av, w[q].x, acc[r][q].x);
          acc[r][q].y = fmaf(av, w[q].y, acc[r][q].y);
          acc[r][q].z = fmaf(av, w[q].z, acc[r][q].z);
          acc[r][q].w = fmaf(av, w[q].w, acc[r][q].w);
        }
      }
    }
  }
}

__device__ __forceinline__ float comp(const float4& v, int e) {
  return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
}
__device__ __forceinline__ void set_comp(float4& v, int e, float x) {
  if (e == 0) v.x = x; else if (e == 1) v.y = x; else if (e == 2) v.z = x; else v.w = x;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Pre-activation of hidden layer l for this thread's RPT rows: GEMM over the
// h-part plus, for layer 0 and the skip layer, the xyz columns and the
// folded per-shape bias; otherwise the plain bias.
template <int WIDTH, int RPT = 4>
__device__ __forceinline__ void layer_preact(const DecoderF32& d, int l,
                                             float4 (&acc)[RPT][WIDTH / 128],
                                             const float* A, int row0, const float4* pos,
                                             const float* bfold0, const float* bfolds, int lane) {
  constexpr int Q = WIDTH / 128;
#pragma unroll
  for (int r = 0; r < RPT; ++r)
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[r][q] = make_float4(0.f, 0.f, 0.f, 0.f);
  const int K = (d.kh[l] + 3) & ~3;
  if (K > 0) gemm_rows<WIDTH, RPT>(acc, A, row0, d.Wt[l], K, lane);
  const bool folded = (l == 0) || (l == d.skip);
  const float* Wx = (l == 0) ? d.Wx0 : d.Wxs;
  const float* bf = (l == 0) ? bfold0 : bfolds;
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const float4 p = pos[row0 + r];
    const int shape = __float_as_int(p.w);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int col = 4 * lane + 128 * q + e;
        float v = comp(acc[r][q], e);
        if (folded) {
          const float4 wx = __ldg(reinterpret_cast<const float4*>(Wx) + col);
          v = fmaf(wx.x, p.x, fmaf(wx.y, p.y, fmaf(wx.z, p.z, v)));
          v += __ldg(bf + (size_t)shape * WIDTH + col);
        } else {
          v += __ldg(d.b[l] + col);
        }
        set_comp(acc[r][q], e, v);
      }
    }
  }
}

template <int WIDTH, int RPT = 4>
__device__ __forceinline__ void store_rows(float* A, int row0, const float4 (&acc)[RPT][WIDTH / 128],
                                           int lane) {
  constexpr int Q = WIDTH / 128;
#pragma unroll
  for (int r = 0; r < RPT; ++r)
#pragma unroll
    for (int q = 0; q < Q; ++q)
      *reinterpret_cast<float4*>(A + (row0 + r) * WIDTH + 4 * lane + 128 * q) = acc[r][q];
}

template <int WIDTH, int RPT = 4>
__device__ __forceinline__ void relu_rows(float4 (&acc)[RPT][WIDTH / 128]) {
  constexpr int Q = WIDTH / 128;
#pragma unroll
  for (int r = 0; r < RPT; ++r)
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      acc[r][q].x = fmaxf(acc[r][q].x, 0.f);
      acc[r][q].y = fmaxf(acc[r][q].y, 0.f);
      acc[r][q].z = fmaxf(acc[r][q].z, 0.f);
      acc[r][q].w = fmaxf(acc[r][q].w, 0.f);
    }
}

// ---------------------------------------------------------------- forward

// RPT rows per thread (warp); TM / RPT warps per CTA.
// (8 rows per thread halves L1 weight traffic but, with 8 warps per SM and
// 255 registers, measured slower on B300: 24.1 vs 25.7 TFLOP/s; 4 is used.)
template <int TM>
__host__ __device__ constexpr int fwd_rpt() { return 4; }
template <int TM>
__host__ __device__ constexpr int fwd_threads() { return TM / fwd_rpt<TM>() * 32; }

template <int WIDTH, int TM>
__global__ void __launch_bounds__(fwd_threads<TM>(), TM >= 64 ? 1 : 4)
mlp_fp32_fwd_kernel(DecoderF32 d, RowSrc src, const float* bfold0, const float* bfolds,
                    float* __restrict__ fout) {
  constexpr int RPT = fwd_rpt<TM>();
  extern __shared__ __align__(16) float smem[];
  float* A = smem;                                         // [TM][WIDTH]
  float4* pos = reinterpret_cast<float4*>(A + TM * WIDTH);   // [TM]
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int row0 = warp * RPT;
  const int n = rowsrc_count(src);
  for (int tile = blockIdx.x; tile * TM < n; tile += gridDim.x) {
    const int base = tile * TM;
    if (threadIdx.x < TM) {
      const int j = base + threadIdx.x;
      float3 p = make_float3(0.f, 0.f, 0.f);
      int shape = 0;
      if (j < n) rowsrc_load(src, j, p, shape);
      pos[threadIdx.x] = make_float4(p.x, p.y, p.z, __int_as_float(shape));
    }
    __syncthreads();
    float4 acc[RPT][WIDTH / 128];
    for (int l = 0; l < d.n_hidden; ++l) {
      layer_preact<WIDTH, RPT>(d, l, acc, A, row0, pos, bfold0, bfolds, lane);
      relu_rows<WIDTH, RPT>(acc);
      __syncthreads();                 // all reads of the previous layer done
      store_rows<WIDTH, RPT>(A, row0, acc, lane);
      __syncthreads();
    }
    // head: s = w . h + b, f = tanh(s) (out_dim outputs per row: fout[j][o])
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      for (int o = 0; o < d.out_dim; ++o) {
        const float* wo = d.w_head + (size_t)o * WIDTH;
        float s = 0.f;
#pragma unroll
        for (int q = 0; q < WIDTH / 128; ++q) {
          const float4 h = *reinterpret_cast<const float4*>(A + (row0 + r) * WIDTH + 4 * lane + 128 * q);
          const float4 w = __ldg(reinterpret_cast<const float4*>(wo) + lane + 32 * q);
          s = fmaf(h.x, w.x, fmaf(h.y, w.y, fmaf(h.z, w.z, fmaf(h.w, w.w, s))));
        }
        s = warp_sum(s);
        const int j = base + row0 + r;
        if (lane == 0 && j < n) fout[(size_t)j * d.out_dim + o] = tanhf(s + d.b_out[o]);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- adjoint

// Per probe: forward with ReLU masks, then reverse through the layers:
//   g_head = 1 - tanh(s)^2;  g_l = (W_{l+1}^T g_{l+1}) * 1[a_l > 0];
// the skip layer's pre-activation gradient g_s and layer 0's g_0 give
//   grad_p f = Wx0^T g_0 + Wxs^T g_s,   df/dz = Wz0^T g_0 + Wzs^T g_s.
// The CTA then adds sum_rows coef * g_0 and coef * g_s into FP64 per-shape
// accumulators; the Wz^T products are applied once per shape afterwards.
template <int WIDTH>
__global__ void __launch_bounds__(kAdjRows * 8, 1)
mlp_fp32_adj_kernel(DecoderF32 d, const float4* __restrict__ pp, const float4* __restrict__ pq,
                    const int* count, const float* bfold0, const float* bfolds,
                    float* __restrict__ out4, double* gacc0, double* gaccs, int accumulate) {
  constexpr int TM = kAdjRows;
  constexpr int Q = WIDTH / 128;
  constexpr int WORDS = WIDTH / 32;                 // mask words per row per layer
  extern __shared__ __align__(16) float smem[];
  float* A = smem;                                   // [TM][WIDTH] activations / gradients
  float* Gs = A + TM * WIDTH;                        // [TM][WIDTH] skip-layer gradient
  uint32_t* masks = reinterpret_cast<uint32_t*>(Gs + TM * WIDTH);  // [TM][16][WORDS]
  float4* pos = reinterpret_cast<float4*>(masks + TM * 16 * WORDS);  // [TM]
  float* coef = reinterpret_cast<float*>(pos + TM);                 // [TM]
  double* red = reinterpret_cast<double*>(coef + TM);               // [8][WIDTH]
  __shared__ int s_next;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int row0 = warp * 4;
  const int n = *count;
  for (int tile = blockIdx.x; tile * TM < n; tile += gridDim.x) {
    const int base = tile * TM;
    if (threadIdx.x < TM) {
      const int j = base + threadIdx.x;
      pos[threadIdx.x] = j < n ? pp[j] : make_float4(0.f, 0.f, 0.f, __int_as_float(0));
    }
    __syncthreads();
    float4 acc[4][Q];
    // forward, recording ReLU masks (bit = lane, word = 4q + e)
    for (int l = 0; l < d.n_hidden; ++l) {
      layer_preact<WIDTH>(d, l, acc, A, row0, pos, bfold0, bfolds, lane);
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const uint32_t m = __ballot_sync(0xffffffffu, comp(acc[r][q], e) > 0.f);
            if (lane == 0) masks[((row0 + r) * 16 + l) * WORDS + 4 * q + e] = m;
          }
      relu_rows<WIDTH>(acc);
      __syncthreads();
      store_rows<WIDTH>(A, row0, acc, lane);
      __syncthreads();
    }
    // head value and its derivative; g for the last hidden layer
    float fval[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      float s = 0.f;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const float4 h = *reinterpret_cast<const float4*>(A + (row0 + r) * WIDTH + 4 * lane + 128 * q);
        const float4 w = __ldg(reinterpret_cast<const float4*>(d.w_head) + lane + 32 * q);
        s = fmaf(h.x, w.x, fmaf(h.y, w.y, fmaf(h.z, w.z, fmaf(h.w, w.w, s))));
      }
      s = warp_sum(s);
      fval[r] = tanhf(s + d.b_head);
    }
    {
      const int L = d.n_hidden - 1;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float dfs = 1.f - fval[r] * fval[r];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const float4 w = __ldg(reinterpret_cast<const float4*>(d.w_head) + lane + 32 * q);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const uint32_t m = masks[((row0 + r) * 16 + L) * WORDS + 4 * q + e];
            set_comp(acc[r][q], e, ((m >> lane) & 1u) ? dfs * comp(w, e) : 0.f);
          }
        }
      }
      __syncthreads();
      store_rows<WIDTH>(A, row0, acc, lane);
      if (L == d.skip) store_rows<WIDTH>(Gs, row0, acc, lane);
      __syncthreads();
    }
    // reverse through layers L..1: g_{l-1} = (W_l^T g_l) * mask_{l-1}
    for (int l = d.n_hidden - 1; l >= 1; --l) {
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < Q; ++q) acc[r][q] = make_float4(0.f, 0.f, 0.f, 0.f);
      gemm_rows<WIDTH>(acc, A, row0, d.Wb[l], WIDTH, lane);
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const uint32_t m = masks[((row0 + r) * 16 + (l - 1)) * WORDS + 4 * q + e];
            if (!((m >> lane) & 1u)) set_comp(acc[r][q], e, 0.f);
          }
      __syncthreads();
      store_rows<WIDTH>(A, row0, acc, lane);
      if (l - 1 == d.skip) store_rows<WIDTH>(Gs, row0, acc, lane);
      __syncthreads();
    }
    // A now holds g_0.  grad_p f = Wx0^T g_0 + Wxs^T g_s
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
      for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int col = 4 * lane + 128 * q + e;
          const float g0 = A[(row0 + r) * WIDTH + col];
          const float4 w0 = __ldg(reinterpret_cast<const float4*>(d.Wx0) + col);
          gx = fmaf(g0, w0.x, gx); gy = fmaf(g0, w0.y, gy); gz = fmaf(g0, w0.z, gz);
          if (d.skip > 0) {
            const float gs = Gs[(row0 + r) * WIDTH + col];
            const float4 ws = __ldg(reinterpret_cast<const float4*>(d.Wxs) + col);
            gx = fmaf(gs, ws.x, gx); gy = fmaf(gs, ws.y, gy); gz = fmaf(gs, ws.z, gz);
          }
        }
      gx = warp_sum(gx); gy = warp_sum(gy); gz = warp_sum(gz);
      const int j = base + row0 + r;
      if (lane == 0) {
        float c = 0.f;
        if (j < n) {
          if (out4) reinterpret_cast<float4*>(out4)[j] = make_float4(fval[r], gx, gy, gz);
          const float4 q4 = pq ? pq[j] : make_float4(0.f, 0.f, 0.f, 0.f);
          c = q4.w;
          if (q4.x != 0.f || q4.y != 0.f || q4.z != 0.f) {
            // exact depth gradient: dd/dz = -(df/dz) / (grad f . v), grazing -> 0
            const float gv = gx * q4.x + gy * q4.y + gz * q4.z;
            const float gn = sqrtf(gx * gx + gy * gy + gz * gz);
            c = (fabsf(gv) >= 1e-3f * gn && gv != 0.f) ? -q4.w / gv : 0.f;
          }
        }
        coef[row0 + r] = c;
      }
    }
    __syncthreads();
    if (accumulate) {
      // one pass per distinct shape in the tile (almost always one)
      uint32_t done = 0;   // bit r: row already reduced (identical in all threads)
      for (int guard = 0; guard < TM; ++guard) {
        if (threadIdx.x == 0) {
          int s = -1;
          for (int r = 0; r < TM; ++r)
            if (!((done >> r) & 1u) && base + r < n) { s = __float_as_int(pos[r].w); break; }
          s_next = s;
        }
        __syncthreads();
        const int shape = s_next;
        __syncthreads();
        if (shape < 0) break;
        for (int pass = 0; pass < (d.skip > 0 ? 2 : 1); ++pass) {
          const float* G = pass == 0 ? A : Gs;
#pragma unroll
          for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int col = 4 * lane + 128 * q + e;
              double t = 0.0;
#pragma unroll
              for (int r = 0; r < 4; ++r) {
                const int rr = row0 + r;
                if (base + rr < n && __float_as_int(pos[rr].w) == shape)
                  t += (double)coef[rr] * (double)G[rr * WIDTH + col];
              }
              red[warp * WIDTH + col] = t;
            }
          __syncthreads();
          double* dst = (pass == 0 ? gacc0 : gaccs) + (size_t)shape * WIDTH;
          for (int col = threadIdx.x; col < WIDTH; col += blockDim.x) {
            double t = 0.0;
            for (int w = 0; w < TM / 4; ++w) t += red[w * WIDTH + col];
            if (t != 0.0) atomicAdd(dst + col, t);
          }
          __syncthreads();
        }
        for (int r = 0; r < TM; ++r)
          if (base + r < n && __float_as_int(pos[r].w) == shape) done |= 1u << r;
      }
    }
    __syncthreads();
  }
}

template <int WIDTH, int TM>
size_t fwd_smem() { return (size_t)TM * WIDTH * 4 + TM * 16; }

template <int WIDTH>
size_t adj_smem() {
  return (size_t)kAdjRows * WIDTH * 4 * 2 + (size_t)kAdjRows * 16 * (WIDTH / 32) * 4 +
         kAdjRows * 16 + kAdjRows * 4 + (size_t)(kAdjRows / 4) * WIDTH * 8;
}

// TM = 64 rows per CTA (one CTA per SM) for large batches; TM = 16 (four
// CTAs per SM) for the sparse lists of the march, where the latency of one
// tile, not throughput, sets the launch time.
template <int WIDTH, int TM>
cudaError_t launch_fwd(const DecoderF32& d, const RowSrc& src, const float* b0, const float* bs,
                       float* fout, cudaStream_t st) {
  const size_t sm = fwd_smem<WIDTH, TM>();
  // set once per process (thread-safe static initialisation)
  static const cudaError_t configured = cudaFuncSetAttribute(
      mlp_fp32_fwd_kernel<WIDTH, TM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (configured != cudaSuccess) return configured;
  const int grid = num_sms() * (TM >= 64 ? 1 : 4);
  mlp_fp32_fwd_kernel<WIDTH, TM><<<grid, fwd_threads<TM>(), sm, st>>>(d, src, b0, bs, fout);
  count_launch(1);
  return cudaGetLastError();
}

template <int WIDTH>
cudaError_t launch_adj(const DecoderF32& d, const float4* pp, const float4* pq, const int* count,
                       const float* b0, const float* bs, float* out4, double* g0, double* gs,
                       int acc, cudaStream_t st) {
  const size_t sm = adj_smem<WIDTH>();
  static const cudaError_t configured = cudaFuncSetAttribute(
      mlp_fp32_adj_kernel<WIDTH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (configured != cudaSuccess) return configured;
  prof_mlp_begin(st, 2);
  mlp_fp32_adj_kernel<WIDTH><<<num_sms(), kAdjRows * 8, sm, st>>>(d, pp, pq, count, b0, bs, out4,
                                                                    g0, gs, acc);
  prof_mlp_end(st);
  count_launch(1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t mlp_fp32_forward(const DecoderF32& d, const RowSrc& src, const float* bfold0,
                             const float* bfolds, float* fout, cudaStream_t st, bool small_tiles) {
  if (small_tiles) {
    switch (d.width) {
      case 128: return launch_fwd<128, 16>(d, src, bfold0, bfolds, fout, st);
      case 256: return launch_fwd<256, 16>(d, src, bfold0, bfolds, fout, st);
      case 384: return launch_fwd<384, 16>(d, src, bfold0, bfolds, fout, st);
      case 512: return launch_fwd<512, 16>(d, src, bfold0, bfolds, fout, st);
    }
  } else {
    switch (d.width) {
      case 128: return launch_fwd<128, kFwdRows>(d, src, bfold0, bfolds, fout, st);
      case 256: return launch_fwd<256, kFwdRows>(d, src, bfold0, bfolds, fout, st);
      case 384: return launch_fwd<384, kFwdRows>(d, src, bfold0, bfolds, fout, st);
      case 512: return launch_fwd<512, kFwdRows>(d, src, bfold0, bfolds, fout, st);
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t mlp_fp32_adjoint(const DecoderF32& d, const float4* pp, const float4* pq,
                             const int* count, const float* bfold0, const float* bfolds,
                             float* out4, double* gacc0, double* gaccs, int accumulate,
                             cudaStream_t st) {
  switch (d.width) {
    case 128: return launch_adj<128>(d, pp, pq, count, bfold0, bfolds, out4, gacc0, gaccs, accumulate, st);
    case 256: return launch_adj<256>(d, pp, pq, count, bfold0, bfolds, out4, gacc0, gaccs, accumulate, st);
    case 384: return launch_adj<384>(d, pp, pq, count, bfold0, bfolds, out4, gacc0, gaccs, accumulate, st);
    case 512: return launch_adj<512>(d, pp, pq, count, bfold0, bfolds, out4, gacc0, gaccs, accumulate, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace dist
