// bwd_nc8.cu -- adjoint kernel for plans whose largest n_f is in the n class 8 (one
// translation unit per class so they compile in parallel).
#include "bwd_impl.cuh"

namespace mhc {

cudaError_t launch_bwd_nc8(const BwdArgs& b, int T, int64_t ctas, size_t smem, cudaStream_t s) {
  return launch_bwd_nc<8>(b, T, ctas, smem, s);
}

cudaError_t launch_kinv_nc8(const BwdArgs& b, int64_t n_fam, cudaStream_t s) {
  return launch_kinv_nc<8>(b, n_fam, s);
}

}  // namespace mhc
