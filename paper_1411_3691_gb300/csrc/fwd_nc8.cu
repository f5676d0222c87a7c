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

cudaError_t launch_batch_nc8(int grid, int T, size_t smem, cudaStream_t s, const FwdArgs* desc,
                               const BatchItem* items, int64_t n_items, unsigned long long* head,
                               const int64_t* part_off, double2* partials) {
  return launch_batch_nc<8>(grid, T, smem, s, desc, items, n_items, head, part_off, partials);
}

int batch_occupancy_nc8(int T, size_t smem) { return batch_occupancy_nc<8>(T, smem); }

cudaError_t launch_kfac_batch_nc8(const FwdArgs* desc, const int64_t* kpref, const int64_t* nfam,
                                  int count, int64_t total, int big, cudaStream_t s) {
  return launch_kfac_batch_nc<8>(desc, kpref, nfam, count, total, big, s);
}

cudaError_t launch_kfac_nc8(const FwdArgs& a, int64_t n_fam, cudaStream_t s) {
  return launch_kfac_nc<8>(a, n_fam, s);
}

}  // namespace mhc
