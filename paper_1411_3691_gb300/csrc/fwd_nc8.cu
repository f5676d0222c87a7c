// fwd_nc8.cu -- forward and per-pair kernels for plans whose largest n_f is in the
// n class 8 (one translation unit per class so they compile in parallel).
#include "fwd_impl.cuh"

namespace mhc {

cudaError_t launch_fwd_nc8(const FwdArgs& a, int tile, int64_t items, size_t smem, cudaStream_t s) {
  return launch_fwd_nc<8>(a, tile, items, smem, s);
}

cudaError_t launch_pairs_nc8(const FwdArgs& a, int64_t n_pairs, int64_t n_src, const int64_t* ii,
                              const int64_t* jj, const int32_t* src_member, const int32_t* mem_family,
                              double* dets, int32_t* path, cudaStream_t s) {
  return launch_pairs_nc<8>(a, n_pairs, n_src, ii, jj, src_member, mem_family, dets, path, s);
}

}  // namespace mhc
