// BF16 tcgen05 decoder forward (DeepSDF shape).  Placeholder until the
// tensor-core kernel lands: the decoder reports no BF16 support.
#include "common.cuh"

namespace dist {

dist_status pack_tc(dist_decoder* d, const float* const* W) {
  (void)W;
  d->tc.ok = false;
  return DIST_OK;
}

cudaError_t mlp_tc_forward(const dist_decoder*, const RowSrc&, const float*, const float*, float*,
                           cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace dist
