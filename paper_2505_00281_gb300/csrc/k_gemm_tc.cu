// tcgen05 BF16 block product (placeholder until the tensor-core kernel lands):
// reports every shape as unsupported so rr_gemm_lowp uses the SIMT kernel.
#include "rr_common.cuh"

namespace rr {
int& gemm_force_simt() {
  static int v = 0;
  return v;
}
bool gemm_bf16_tc_supported(int64_t, int64_t, int64_t, int64_t, int64_t, const void*, const void*) {
  return false;
}
rr_status gemm_bf16_tc(int64_t, int64_t, int64_t, const __nv_bfloat16*, int64_t, const __nv_bfloat16*,
                       int64_t, float*, int64_t, const double*, int64_t, const double*, cudaStream_t) {
  return RR_ERR_ARG;
}
}  // namespace rr
