// Allocation-free point evaluation of the decoder.
//
// The scratch that dist_sdf_eval takes from a workspace (folded latent
// biases, packed points, gradient staging, a row count) lives here in one
// file-scope device array instead, so a call needs no cudaMalloc.  Host code
// cannot use the array's name as a device address: the address is looked up
// with cudaGetSymbolAddress once per device, on the first call made while
// that device is current, and handed to the kernels.
#include <mutex>

#include "common.cuh"

namespace dist {
namespace {

constexpr long long kStaticMaxPoints = 65536;
constexpr int kStaticMaxShapes = 64;
constexpr size_t kOffBias0 = 0;
constexpr size_t kOffBiasS = kOffBias0 + (size_t)kStaticMaxShapes * 512 * sizeof(float);
constexpr size_t kOffPoints = kOffBiasS + (size_t)kStaticMaxShapes * 512 * sizeof(float);
constexpr size_t kOffOut = kOffPoints + (size_t)kStaticMaxPoints * sizeof(float4);
constexpr size_t kOffCount = kOffOut + (size_t)kStaticMaxPoints * sizeof(float4);
constexpr size_t kStaticBytes = kOffCount + 256;   // 2,359,552 bytes

static __device__ __align__(256) unsigned char g_eval_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_eval_scratch on the current device (looked up once).
dist_status scratch_on_current_device(unsigned char** out) {
  int dev = 0;
  DIST_CUDA_TRY(cudaGetDevice(&dev));
  DIST_CHECK(dev >= 0 && dev < kMaxDevices, DIST_E_INVALID,
             "dist_sdf_eval_static: device index out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    DIST_CUDA_TRY(cudaGetSymbolAddress(&p, g_eval_scratch));
    DIST_CHECK(p != nullptr, DIST_E_CUDA, "cudaGetSymbolAddress returned NULL");
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return DIST_OK;
}

}  // namespace
}  // namespace dist

using namespace dist;

extern "C" dist_status dist_sdf_eval_static(const dist_decoder* dec, const float* z, int n_shapes,
                                            const float* pts, const int32_t* shape, int64_t n,
                                            int precision, float* f, float* grad, void* stream) {
  DIST_CHECK(dec && z && pts && shape && f, DIST_E_INVALID,
             "dist_sdf_eval_static: NULL argument");
  DIST_CHECK(is_sdf_decoder(dec->desc), DIST_E_INVALID,
             "dist_sdf_eval_static needs an SDF decoder (out_dim 1, latent_dim0 = latent_dim)");
  DIST_CHECK(n >= 1 && n <= kStaticMaxPoints, DIST_E_INVALID,
             "dist_sdf_eval_static: n must be 1..65536 (size of the built-in scratch)");
  DIST_CHECK(n_shapes >= 1 && n_shapes <= kStaticMaxShapes, DIST_E_INVALID,
             "dist_sdf_eval_static: n_shapes must be 1..64 (size of the built-in scratch)");
  DIST_CHECK(precision == DIST_PREC_FP32 || (valid_precision(precision) && !grad),
             DIST_E_INVALID,
             "dist_sdf_eval_static: bad precision (the tensor-core kernels have no gradient)");
  DIST_CHECK(precision == DIST_PREC_FP32 || dec->tc.ok, DIST_E_UNSUPPORTED,
             "BF16 tensor-core MLP covers only the DeepSDF decoder shape");
  unsigned char* base = nullptr;
  dist_status s = scratch_on_current_device(&base);
  if (s != DIST_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const DecoderF32& d = dec->f32;
  // the bias table is laid out [shape][width]; every entry the kernels read
  // (shapes < n_shapes) is rewritten below, and the row count is rewritten
  // by the pack kernel, so nothing depends on what a previous call left
  float* b0 = reinterpret_cast<float*>(base + kOffBias0);
  float* bs = reinterpret_cast<float*>(base + kOffBiasS);
  float4* pts4 = reinterpret_cast<float4*>(base + kOffPoints);
  float* out4 = reinterpret_cast<float*>(base + kOffOut);
  int* count = reinterpret_cast<int*>(base + kOffCount);
  DIST_CUDA_TRY(launch_fold_bias(d, z, n_shapes, b0, bs, st));
  DIST_CUDA_TRY(launch_pack_points(pts, shape, n, n_shapes, pts4, count, st));
  RowSrc src{};
  src.count = count;
  src.pts = pts4;
  if (is_tc(precision)) {
    DIST_CUDA_TRY(mlp_tc_forward(dec, src, b0, bs, f, st, precision == DIST_PREC_FP16));
  } else if (precision == DIST_PREC_FP32_TC) {
    DIST_CUDA_TRY(mlp_tcx_forward(dec, src, b0, bs, f, st));
  } else if (!grad) {
    DIST_CUDA_TRY(mlp_fp32_forward(d, src, b0, bs, f, st));
  } else {
    DIST_CUDA_TRY(mlp_fp32_adjoint(d, pts4, nullptr, count, b0, bs, out4, nullptr, nullptr, 0, st));
    DIST_CUDA_TRY(launch_unpack_grad(out4, n, f, grad, st));
  }
  return DIST_OK;
}
