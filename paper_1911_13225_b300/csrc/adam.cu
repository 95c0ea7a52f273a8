// Adam update of the latent codes: the optimiser of the inverse problem
// (Sec. 4.2, shape from depth by optimising z; Sec. B.4: Adam, lr 1e-2).
//
// Adam as published (Kingma & Ba, ICLR 2015, Algorithm 1) with the bias
// corrections folded into the step size:
//   m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2,
//   z <- z - lr / (1 - b1^t) * m / (sqrt(v / (1 - b2^t)) + eps).
// One thread per latent entry; the update is element-wise and memory bound
// (n_shapes x latent_dim floats: 32 KB for 32 shapes of 256), so its cost is
// the launch.  The arithmetic is FP32 with the bias corrections formed in
// FP64 on the host, so a run is reproducible bit for bit from (z, m, v, t).
#include <cmath>

#include "common.cuh"

namespace dist {
namespace {

__global__ void adam_kernel(float* __restrict__ z, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, long long n, float b1,
                            float b2, float step, float inv_sqrt_bc2, float eps) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
  const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
  m[i] = mi;
  v[i] = vi;
  z[i] -= step * mi / (sqrtf(vi) * inv_sqrt_bc2 + eps);
}

}  // namespace
}  // namespace dist

using namespace dist;

extern "C" dist_status dist_adam_step(float* z, const float* dz, float* m, float* v, int64_t n,
                                      int t, float lr, float beta1, float beta2, float eps,
                                      void* stream) {
  DIST_CHECK(z && dz && m && v, DIST_E_INVALID, "dist_adam_step: NULL argument");
  DIST_CHECK(n >= 1 && n <= ((int64_t)1 << 31), DIST_E_INVALID, "dist_adam_step: bad n");
  DIST_CHECK(t >= 1, DIST_E_INVALID, "dist_adam_step: t counts steps from 1");
  DIST_CHECK(lr > 0.f && beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f &&
                 eps > 0.f,
             DIST_E_INVALID, "dist_adam_step: bad hyper-parameters");
  const double bc1 = 1.0 - std::pow((double)beta1, (double)t);
  const double bc2 = 1.0 - std::pow((double)beta2, (double)t);
  const float step = (float)((double)lr / bc1);
  const float inv_sqrt_bc2 = (float)(1.0 / std::sqrt(bc2));
  const int threads = 256;
  const long long blocks = (n + threads - 1) / threads;
  adam_kernel<<<(unsigned)blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(
      z, dz, m, v, n, beta1, beta2, step, inv_sqrt_bc2, eps);
  DIST_LAUNCH_CHECK();
  return DIST_OK;
}
