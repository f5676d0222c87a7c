// forward.cu -- host launchers of the forward correlator and the deterministic reduction
// of the per-work-item partial sums.
#include "kernels.cuh"
#include "trace.h"

namespace mhc {

namespace {

// Sum of the per-item partials in a fixed order (one block of 1024 threads).
__global__ void __launch_bounds__(1024) reduce_kernel(const double2* __restrict__ partials,
                                                      int64_t n, double* out) {
  __shared__ double2 red[32];
  double2 s = make_double2(0.0, 0.0);
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    s.x += partials[i].x;
    s.y += partials[i].y;
  }
  s = dev::warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 t = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
      t.x += red[w].x;
      t.y += red[w].y;
    }
    out[0] = t.x;
    out[1] = t.y;
  }
}

}  // namespace

// Complex weights by bilinearity: with w_i = a_i + i b_i and w_j = c_j + i d_j,
// C = C(a, c) - C(b, d) + i (C(a, d) + C(b, c)), each C(x, y) a real-weight correlator.
// t holds C(a, c), C(a, d), C(b, c), C(b, d) as (Re, Im) pairs.
__global__ void combine_cw(const double* __restrict__ t, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    out[0] = t[0] - t[6] - (t[3] + t[5]);
    out[1] = t[1] - t[7] + (t[2] + t[4]);
  }
}

size_t forward_smem_bytes(int slots, int tile) {
  const size_t cache = (size_t)slots * tile * sizeof(double2);
  const size_t queue = (size_t)(tile / 32) * kQueueCap * kQueueEntryBytes;
  const size_t z1 = (size_t)(tile / 32) * kZ1Bytes;
  const size_t walk = (size_t)(tile / 32) * kWalkBytes;
  return cache + queue + z1 + walk;
}

// fwd_kernel over items [0, items): one launch per layout range, each with its own y
// cache, or one launch with the plan's layout (smem: its size).
static cudaError_t launch_fwd_items(const FwdArgs& a, int ncmax, int tile, int64_t items, size_t smem,
                                    cudaStream_t s) {
  auto one = [&](const FwdArgs& x, int64_t count, size_t bytes) {
    return ncmax <= 8 ? launch_fwd_nc8(x, tile, count, bytes, s)
                      : (ncmax <= 18 ? launch_fwd_nc18(x, tile, count, bytes, s)
                                     : launch_fwd_nc32(x, tile, count, bytes, s));
  };
  if (!a.fam_order || a.n_ranges <= 0) return one(a, items, smem);
  for (int r = 0; r < a.n_ranges; r++) {
    const FwdRange& g = a.ranges[r];
    if (g.count <= 0) continue;
    FwdArgs ar = a;
    ar.slots = g.slots;
    for (int f = 0; f < MHC_FMAX; f++) ar.yoff[f] = g.yoff[f];
    ar.item0 = g.first * a.n_tiles;
    const cudaError_t e = one(ar, g.count * a.n_tiles, forward_smem_bytes(g.slots, tile));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_forward(const FwdArgs& a, int ncmax, int tile, int64_t n_fam, int64_t items,
                           size_t smem, double* out, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (a.snk_orig) {  // two-sided update: the LU factors of every (family, sink family) block first
    TraceRange trace("block factors");
    if (ncmax <= 8)
      e = launch_kfac_nc8(a, n_fam, s);
    else if (ncmax <= 18)
      e = launch_kfac_nc18(a, n_fam, s);
    else
      e = launch_kfac_nc32(a, n_fam, s);
    if (e != cudaSuccess) return e;
  }
  {
    TraceRange trace("forward kernel");
    if ((e = launch_fwd_items(a, ncmax, tile, items, smem, s)) != cudaSuccess) return e;
  }
  TraceRange trace("reduce");
  return launch_reduce(a.partials, items, out, s);
}

cudaError_t launch_forward_cw(const FwdArgs& a0, const double* const* ws, const double* const* wk,
                              int ncmax, int tile, int64_t n_fam, int64_t items, size_t smem, double* tmp,
                              double* out, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (a0.snk_orig) {  // the block factors do not depend on the weights: once for the four passes
    e = ncmax <= 8 ? launch_kfac_nc8(a0, n_fam, s)
                   : (ncmax <= 18 ? launch_kfac_nc18(a0, n_fam, s) : launch_kfac_nc32(a0, n_fam, s));
    if (e != cudaSuccess) return e;
  }
  for (int k = 0; k < 4; k++) {
    FwdArgs a = a0;
    a.w_src = ws[k >> 1];
    a.w_snk = wk[k & 1];
    if ((e = launch_fwd_items(a, ncmax, tile, items, smem, s)) != cudaSuccess) return e;
    if ((e = launch_reduce(a.partials, items, tmp + 2 * k, s)) != cudaSuccess) return e;
  }
  combine_cw<<<1, 32, 0, s>>>(tmp, out);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const double2* partials, int64_t items, double* out, cudaStream_t s) {
  reduce_kernel<<<1, 1024, 0, s>>>(partials, items, out);
  return cudaGetLastError();
}

cudaError_t launch_pairs(const FwdArgs& a, int ncmax, int64_t n_pairs, int64_t n_src,
                         const int64_t* ii, const int64_t* jj, const int32_t* src_member,
                         const int32_t* mem_family, double* dets, int32_t* path, cudaStream_t s) {
  if (ncmax <= 8) return launch_pairs_nc8(a, n_pairs, n_src, ii, jj, src_member, mem_family, dets, path, s);
  if (ncmax <= 18) return launch_pairs_nc18(a, n_pairs, n_src, ii, jj, src_member, mem_family, dets, path, s);
  return launch_pairs_nc32(a, n_pairs, n_src, ii, jj, src_member, mem_family, dets, path, s);
}

}  // namespace mhc
