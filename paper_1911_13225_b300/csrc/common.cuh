// Internal definitions shared by the libdist translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/dist.h"

namespace dist {

// ------------------------------------------------------------------ errors

void set_error(const std::string& msg);

#define DIST_CUDA_TRY(call)                                                   \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      ::dist::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));  \
      return DIST_E_CUDA;                                                     \
    }                                                                         \
  } while (0)

void count_launch(int n = 1);
void prof_mlp_begin(cudaStream_t st, int kind);   // kind 0: BF16 tensor core, 1: FP32 SIMT
void prof_mlp_end(cudaStream_t st);

// After a kernel launch: count it (measurement) and check the launch error.
#define DIST_LAUNCH_CHECK()                                                   \
  do {                                                                        \
    ::dist::count_launch(1);                                                  \
    DIST_CUDA_TRY(cudaGetLastError());                                        \
  } while (0)

// NVTX range over a scope: each entry point and march step shows up by name
// in Nsight Systems and under `ncu --nvtx`; without a tool attached the
// push/pop are no-ops (NVTX v3 is header-only, nothing to link).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define DIST_NVTX(name) ::dist::NvtxRange dist_nvtx_range_(name)

#define DIST_CHECK(cond, code, msg)                                           \
  do {                                                                        \
    if (!(cond)) {                                                            \
      ::dist::set_error(msg);                                                 \
      return code;                                                            \
    }                                                                         \
  } while (0)

// A decoder of the SDF (one output, one code): what tracing needs.
inline bool is_sdf_decoder(const dist_decoder_desc& d) {
  return (d.out_dim == 0 || d.out_dim == 1) && (d.latent_dim0 == 0 || d.latent_dim0 == d.latent_dim);
}

// Precisions whose march runs on the tensor cores.
inline bool is_tc(int precision) {
  return precision == DIST_PREC_BF16 || precision == DIST_PREC_FP16;
}

// Precisions accepted by the trace and evaluation entry points.
inline bool valid_precision(int precision) {
  return precision == DIST_PREC_FP32 || is_tc(precision) || precision == DIST_PREC_FP32_TC;
}

// The FP32-class queries of a trace (its FP32 list) run on the tensor cores.
inline bool fp32_on_tc(const dist_trace_params& p) {
  return p.precision == DIST_PREC_FP32_TC ||
         (is_tc(p.precision) && p.refine_engine == DIST_REFINE_TC);
}

constexpr int kMaxShapes = 1024;    // folded-bias capacity of a workspace
constexpr int kMaxK = 3;            // k_min upper bound (Sec. B.4 uses 1 or 3)
constexpr int kMaxCoarseLevels = 4; // coarse-to-fine: at most 16x coarser per side
constexpr int kProbesPerRay = 10;   // probe capacity per pixel in a workspace:
                                    // <= 4 depth/silhouette + 6 normal probes

// ------------------------------------------------------------- camera table

// One camera as the kernels see it.
struct CamDev {
  float c[3];
  float R[9];
  float fx, fy, cx, cy;
  int H, W;
  int shape;
  int pad;
  long long offset;   // first pixel index of this camera
};

// ------------------------------------------------------------------ decoder

// Weights repacked for the FP32 SIMT kernels.  Every hidden layer is padded
// to a square WIDTH x WIDTH block with zeros so that all layers share one
// tiling; padded outputs have zero weight and bias and so stay 0 after ReLU.
struct DecoderF32 {
  int width, n_hidden, skip, latent;
  int kh[16];          // h-part input count of each hidden layer (0 for layer 0)
  int nout[16];        // real output count of each hidden layer
  const float* Wt[16];   // [WIDTH k][WIDTH j] = W_l[j][h-col k]   (forward)
  const float* Wb[16];   // [WIDTH j][WIDTH k] = W_l[j][h-col k]   (backward)
  const float* b[16];    // [WIDTH]
  const float* Wx0;      // [WIDTH][4]  xyz columns of layer 0
  const float* Wxs;      // [WIDTH][4]  xyz columns of the skip layer (or null)
  const float* Wz0;      // [WIDTH][latent] latent columns of layer 0
  const float* Wzs;      // [WIDTH][latent] latent columns of the skip layer
  const float* w_head;   // [out_dim][WIDTH] (row 0: the SDF head)
  float b_head;          // b of output 0
  int latent0;           // layer-0 code length (the skip layer reads its last `latent`)
  int out_dim;           // 1 (SDF) or 3 (colour)
  float b_out[4];        // head biases
};

// BF16 tensor-core packing of the DeepSDF shape (width 512, 8 hidden, skip 4):
// GEMM layers 1..7 as bf16 [N rows][K cols] (K contiguous) with one TMA
// tensor map each (box 64 K x 256 N, 128-byte swizzle).
struct TCMaps {
  CUtensorMap m[7];
};
// Per-column constants of the tensor-core epilogues (device copy); the
// epilogue reads them warp-uniformly as float4 rows.
struct TCConst {
  float bias[7][512];            // layers 1..7 (entry 3, the skip layer, unused: folded)
  float wx0[3][512];             // xyz columns of layer 0, by axis
  float wx4[3][512];             // xyz columns of the skip layer 4, by axis
  float w_head[512];
  float w_c[3][512];             // colour decoder: the three head rows (read as float4)
  float b_head;
  float b_c[3];
};
static_assert(offsetof(TCConst, w_c) % 16 == 0 && offsetof(TCConst, w_head) % 16 == 0 &&
                  offsetof(TCConst, wx0) % 16 == 0 && offsetof(TCConst, wx4) % 16 == 0,
              "TCConst rows are read as float4");
struct DecoderTC {
  bool ok;
  TCMaps maps;                   // bf16 operands
  TCMaps maps16;                 // fp16 operands (same layout)
  TCMaps bmaps;                  // W_l^T for the adjoint's backward GEMMs (bf16)
  TCMaps bmaps16;                // same, fp16
  TCMaps xmaps;                  // [N][2K] fp16 hi | lo split of 2^s_l W_l (FP32-class kernel)
  TCMaps bxmaps;                 // [K][2N] its transpose (FP32-class adjoint)
  TCMaps wmaps, wmaps16, wxmaps; // the same three as 3D views [K/64][N][64] with boxes of
                                 // two 128-row x 64-column chunks (latency-mode kernel)
  float x_inv_scale[7];          // 2^-s_l
  const TCConst* cst;            // epilogue constants (device)
  int* err;                      // device error word of the bounded waits
  unsigned long long wait_ns;    // limit of the forward kernel's waits (default 1 s)
  int withhold;                  // tests: the forward kernel's loader issues no copies
};

// Per-CTA global scratch of the tensor-core adjoint: ReLU masks and the
// skip layer's pre-activation gradient of one 128-row tile.
constexpr size_t kTcAdjScratchPerCta = (size_t)8 * 128 * 2 * 8 * 4 + (size_t)128 * 512 * 4;

}  // namespace dist

struct dist_decoder {
  dist_decoder_desc desc;
  dist::DecoderF32 f32;
  dist::DecoderTC tc;
  std::vector<void*> allocations;
};

struct dist_workspace {
  int64_t max_rays;
  int max_steps;
  // ray state
  float4* dir;        // (vx, vy, vz, 1/sqrt(x~^2+y~^2+1))
  float4* st;         // (d, t_in, t_out, camera index as int bits)
  int* fq;            // FP32 queries a ray made after its low-precision phase
  float* fprev;       // previous low-precision sample of each ray (its FP32-class
                      // sample after the hand-over, secant rule)
  float* dprev;       // distance of the previous FP32-class sample (secant rule)
  int* act[2][3];     // [parity][0 = BF16 list, 1 = FP32 list, 2 = FP16 stage] ray ids
  float* fbuf[3];     // MLP outputs for the three lists
  int* counts;        // [(max_steps + 2) * 3 + 2 kMaxCoarseLevels] list lengths
                      // per step, then per coarse-to-fine split
  int* rstat;         // per-ray status when the caller asks for none
  int* chunk;         // (max_rays + 31) / 32 probe counts / offsets (ordered append)
  dist::CamDev* cams; // camera table (device)
  int max_cams;
  float* bfold;       // [2][kMaxShapes][512] folded latent biases
  double* gacc;       // [2][kMaxShapes][512] FP64 latent-gradient accumulators
  float4* probe_p;    // [max_rays * kProbesPerRay] (x, y, z, shape bits)
  float4* probe_q;    // (vx, vy, vz, coefficient)
  int* probe_pix;     // pixel of each probe
  float* probe_out;   // [max_rays * kProbesPerRay][4] f and grad_p per probe
  int* probe_count;   // [4]
  double* red;        // [8] small FP64 reduction scratch
  int* ired;          // [8] small integer scratch
  void* tc_scratch;   // num_sms() * kTcAdjScratchPerCta bytes (tensor-core adjoint)
  void* wide_scratch; // tc_wide_scratch_bytes(): latency-mode operand images
  unsigned long long step_seq;  // host: sequence number of the last fused step
  std::vector<void*> allocations;
};

namespace dist {

// ------------------------------------------------------- device helpers

__device__ __forceinline__ float3 cam_origin(const CamDev& c) {
  return make_float3(c.c[0], c.c[1], c.c[2]);
}

// Row sources for the MLP kernels: rays of an active list, or explicit points.
struct RowSrc {
  const int* count;        // device: number of rows (null -> n_rows)
  int n_rows;
  const int* idx;          // active list of ray ids (rays mode)
  const float4* st;
  const float4* dir;
  const CamDev* cams;
  const float4* pts;       // points mode: (x, y, z, shape as int bits)
};

__device__ __forceinline__ int rowsrc_count(const RowSrc& s) {
  return s.count ? *s.count : s.n_rows;
}

__device__ __forceinline__ void rowsrc_load(const RowSrc& s, int j, float3& p, int& shape) {
  if (s.pts) {
    float4 q = s.pts[j];
    p = make_float3(q.x, q.y, q.z);
    shape = __float_as_int(q.w);
  } else {
    int i = s.idx[j];
    float4 st = s.st[i];
    float4 dv = s.dir[i];
    const CamDev& c = s.cams[__float_as_int(st.w)];
    p = make_float3(fmaf(st.x, dv.x, c.c[0]), fmaf(st.x, dv.y, c.c[1]), fmaf(st.x, dv.z, c.c[2]));
    shape = c.shape;
  }
}

// ------------------------------------------------------------ launchers

int num_sms();

// FP32 SIMT decoder forward over `src` rows: fout[j] = f(p_j, z_shape_j).
// small_tiles: 16-row tiles (for short, latency-bound row lists).
cudaError_t mlp_fp32_forward(const DecoderF32& d, const RowSrc& src, const float* bfold0,
                             const float* bfolds, float* fout, cudaStream_t st,
                             bool small_tiles = false);

// FP32 SIMT adjoint over probes: f and grad_p f per probe (out4, optional) and
// FP64 accumulation of coef * (pre-activation gradients at layer 0 and the
// skip layer) into gacc0 / gaccs [shape][WIDTH] (when accumulate != 0).
cudaError_t mlp_fp32_adjoint(const DecoderF32& d, const float4* pp, const float4* pq,
                             const int* count, const float* bfold0, const float* bfolds,
                             float* out4, double* gacc0, double* gaccs, int accumulate,
                             cudaStream_t st);

// Point-evaluation helpers (trace.cu) for callers with their own scratch.
cudaError_t launch_fold_bias(const DecoderF32& d, const float* z, int n_shapes, float* bfold0,
                             float* bfolds, cudaStream_t st);
cudaError_t launch_pack_points(const float* pts, const int* shape, long long n, int n_shapes,
                               float4* out, int* count, cudaStream_t st);
cudaError_t launch_unpack_grad(const float* out4, long long n, float* f, float* grad,
                               cudaStream_t st);

// A pool of rays driven one march step at a time (serving).  Pixel indices
// are pool indices; camera index == request slot == latent index.
struct RayPool {
  const CamDev* cams;
  float4* st;
  float4* dir;
  int* fq;
  float* fprev;
  float* dprev;
  int refine;
  int secant;
  float alpha_fp32;
  dist_trace_out o;
  int K;
  float eps, alpha, eps_bf16, radius;
  float eps_mid;      // FP16 stage of a BF16 march (0: none)
  int max_steps;
};
cudaError_t pool_write_cam(const CamDev& c, int slot, CamDev* dst, cudaStream_t st);
cudaError_t pool_raygen(const RayPool& P, int cam, long long pix0, long long n, int* list0,
                        int* count0, cudaStream_t st);
cudaError_t pool_step(const RayPool& P, const int* cnt_in, int* cnt_out, int* const in[2],
                      const float* const f[2], int* const out[2], cudaStream_t st);
struct StepFuse;

// The same step update, applied by the fused decoder kernel (StepFuse).
void pool_step_fuse(const RayPool& P, int* cnt_out, int* const out[2], StepFuse* sf);
cudaError_t pool_probes_depth(const RayPool& P, int cam, long long pix0, long long n,
                              const float* g_depth, float4* pp, float4* pq, int* pix, int* count,
                              cudaStream_t st);
cudaError_t pool_loss_depth(long long n, const float* depth, const uint8_t* mask, const float* tgt,
                            double* loss, float* g_depth, int* cnt, cudaStream_t st);
cudaError_t pool_latent_finalize(const DecoderF32& d, const double* G0, const double* Gs,
                                 float* dz, cudaStream_t st);

// tcgen05 decoder forward with BF16 (f16 = false) or FP16 operands
// (DeepSDF shape only).
cudaError_t mlp_tc_forward(const dist_decoder* dec, const RowSrc& src, const float* bfold0,
                           const float* bfolds, float* fout, cudaStream_t st, bool f16);

// FP32-class tcgen05 decoder forward (two-term FP16 split of weights and
// activations; DeepSDF shape only).
cudaError_t mlp_tcx_forward(const dist_decoder* dec, const RowSrc& src, const float* bfold0,
                            const float* bfolds, float* fout, cudaStream_t st);

// Both in one launch: src16 with 16-bit operands into f16out, srcx
// FP32-class into fxout (either list may be empty: count null, n_rows 0).
// With `step` (rays mode only) the kernel applies the march step update to
// each queried ray instead of writing f: see StepFuse.
cudaError_t mlp_tc_fused(const dist_decoder* dec, const RowSrc& src16, float* f16out,
                         const RowSrc& srcx, float* fxout, const float* bfold0,
                         const float* bfolds, cudaStream_t st, bool f16,
                         const StepFuse* step = nullptr, const RowSrc* srcm = nullptr,
                         float* fmout = nullptr);

// Latency mode of the fused decoder (a launch of at most tc_wide_max_tiles()
// tiles of 128 16-bit rows or 64 FP32-class queries): each tile on a cluster
// of four CTAs, one quarter of every layer's output columns each.  Same
// arguments as mlp_tc_fused plus `scratch` (tc_wide_scratch_bytes() of
// device memory); the kernel does nothing when the lists are longer.
cudaError_t mlp_tc_wide(const dist_decoder* dec, const RowSrc& src16, float* f16out,
                        const RowSrc& srcx, float* fxout, const float* bfold0,
                        const float* bfolds, cudaStream_t st, bool f16, const StepFuse* step,
                        void* scratch, const RowSrc* srcm = nullptr, float* fmout = nullptr);
int tc_wide_max_tiles();
size_t tc_wide_scratch_bytes();
// The step sequence word inside that scratch (zeroed with it by its owner).
unsigned long long* tc_wide_seq_flag(void* scratch);

// Colour decoder on the tensor cores (16-bit rows only): per row the three
// head dot products of its last hidden layer in four partial sums (one per
// 32-column group, each over the four quarters in order),
// cpart[row][4][3]; bias and tanh are applied afterwards.
cudaError_t mlp_tc_color(const dist_decoder* dec, const RowSrc& src, const float* bfold0,
                         const float* bfolds, float* scratch, float* cpart, cudaStream_t st,
                         bool f16);

// tcgen05 decoder adjoint over probes (same contract as mlp_fp32_adjoint;
// `scratch` holds num_sms() * kTcAdjScratchPerCta bytes).
cudaError_t mlp_tc_adjoint(const dist_decoder* dec, const float4* pp, const float4* pq,
                           const int* count, const float* bfold0, const float* bfolds,
                           float* out4, double* gacc0, double* gaccs, int accumulate,
                           void* scratch, cudaStream_t st, bool f16);

// Probes handed from the FP32-class adjoint to the FP32 one: device arrays
// of `cap` entries, the device count (zeroed by the caller; it ends at most
// at cap) and the |ReLU input| below which a probe is handed over.
struct RedoList {
  float4* p;
  float4* q;
  int* count;
  int cap;
  float tau;
};

// The same adjoint with FP32-class operands (two-term FP16 splits, 64 probes
// per tile, four times a 16-bit probe's tensor work).  Its pre-activations
// carry ~1e-6 of truncation error, so a ReLU input that close to 0 may take
// the other side: with `redo`, such probes are left to the caller's FP32
// adjoint (the gradient of a central-difference normal differences two
// Jacobians 2 delta apart, and one flipped mask in either is amplified by
// 1 / (2 delta)).
cudaError_t mlp_tcx_adjoint(const dist_decoder* dec, const float4* pp, const float4* pq,
                            const int* count, const float* bfold0, const float* bfolds,
                            float* out4, double* gacc0, double* gaccs, int accumulate,
                            void* scratch, cudaStream_t st, const RedoList* redo = nullptr);

}  // namespace dist
