// bwd_nc32.cu -- adjoint kernel for plans whose largest n_f is in the n class 32 (one
// translation unit per class so they compile in parallel).
#include "bwd_impl.cuh"

namespace mhc {

cudaError_t launch_bwd_nc32(const BwdArgs& b, int T, int64_t ctas, size_t smem, cudaStream_t s) {
  return launch_bwd_nc<32>(b, T, ctas, smem, s);
}

}  // namespace mhc
