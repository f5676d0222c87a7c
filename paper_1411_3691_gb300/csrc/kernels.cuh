// kernels.cuh -- argument blocks and dispatch shared by the forward, pair-probe, batched
// and adjoint kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/mhc.h"
#include "device.cuh"
#include "layout.h"

namespace mhc {

// status bits of the device status word (counters[0])
enum : unsigned long long {
  kStatusNonFinite = 1ull,
  kStatusBadIndex = 2ull,
  kStatusTimeout = 4ull,
  kStatusUnsupported = 8ull,  // reserved: a request the kernels could not complete
};

// Everything one forward evaluation of one plan needs on the device.
struct FwdArgs {
  int F, Tn, n_tiles, slots, kp, kc;
  int rowdiff;               // 1: the row-difference update before a lemma-guard refactor
  int64_t n_snk;
  int n_f[MHC_FMAX], L_f[MHC_FMAX], off_f[MHC_FMAX], yoff[MHC_FMAX];
  const double2* S[MHC_FMAX];
  const int32_t* fam_info;   // [W][4]: member offset, member count
  const int32_t* fam_rank;   // [W][F]
  const int32_t* fam_arow;   // [W][Tn]
  const int32_t* mem_term;   // [members]
  const int32_t* mem_par;    // [members] bit f = sign parity of flavour f
  const int32_t* mem_lab;    // [members][F][MHC_MAX_RANK]
  const int32_t* snk_lab;    // [n_snk][Tn]
  const double* w_src;
  const double* w_snk;
  double2* partials;         // [items]
  unsigned long long* counters;
  // two-sided update; snk_orig == nullptr selects the one-sided update with the sinks
  // in their own order and labels from snk_lab
  const int32_t* snk_pos;    // [n_snk][Tn] aligned column labels of the sink at position j
  const int32_t* snk_orig;   // [n_snk] original sink index at position j
  const int32_t* snk_par;    // [n_snk] bit f: column-permutation parity
  const int32_t* snk_q;      // [n_snk] sink family of position j
  const int32_t* q_two;      // [Q] 1: the family uses the two-sided update
  const int32_t* q_rank;     // [Q][F] changed columns (1 or 2) of the sink family
  const int32_t* q_off;      // [Q + 1] first position of each sink family
  const double2* kbuf;       // [W][Q][kstride]: per flavour the LU factors of B (see kapply)
  int32_t* kguard;           // [W][Q][F] 1: the block's pivot guard fired
  int64_t n_q;
  int kstride;
  int koff[MHC_FMAX];
  // work order of fwd_kernel by y-cache layout: the families are grouped by the rank of
  // each flavour (n slots for rank 1, r n + 1 for rank r >= 2), the all-rank-1 group first,
  // and each group runs in a launch of its own with a cache sized for it, so that more
  // blocks fit on an SM.  Range r covers work positions [first, first + count) with layout
  // (yoff, slots); fam_order == nullptr: natural order, one launch with the plan's layout.
  const int32_t* fam_order;  // [n_fam] family at each work position
  int64_t item0;             // first work item of the launch
  int n_ranges;
  FwdRange ranges[kMaxFwdRanges];
};

namespace dev {

// Per-(n, rank) dispatch to the register-resident specialisations (n <= 6) or the generic
// runtime-n routine with arrays sized for the n class NCMAX.
template <int NCMAX>
__device__ __forceinline__ bool dispatch_shared(int n, int rho, const cd* S, int L,
                                                const int32_t* arow, const int32_t* col, cd* Y,
                                                int ys, int* ey, int kp) {
#define MHC_SR(N)                                                                   \
  case N:                                                                           \
    return rho == 1 ? shared_rows<N, N, 1>(S, L, N, arow, col, Y, ys, ey, kp)       \
                    : shared_rows<N, N, (N >= 2 ? 2 : 1)>(S, L, N, arow, col, Y, ys, ey, kp);
  switch (n) {
    MHC_SR(1)
    MHC_SR(2)
    MHC_SR(3)
    MHC_SR(4)
    MHC_SR(5)
    MHC_SR(6)
    default:
      break;
  }
#undef MHC_SR
  if constexpr (NCMAX >= 14) {  // three changed rows (n_f >= 14 only)
    if (rho == 3) return shared_rows<NCMAX, 0, 3>(S, L, n, arow, col, Y, ys, ey, kp);
  }
  if constexpr (NCMAX >= 18) {  // rank k for n_f >= 4k + 2: 4 from n_f = 18
    if (rho == 4) return shared_rows<NCMAX, 0, 4>(S, L, n, arow, col, Y, ys, ey, kp);
  }
  if constexpr (NCMAX >= 32) {  // 5 from n_f = 22, 6 from n_f = 26
    if (rho == 5) return shared_rows<NCMAX, 0, 5>(S, L, n, arow, col, Y, ys, ey, kp);
    if (rho == 6) return shared_rows<NCMAX, 0, 6>(S, L, n, arow, col, Y, ys, ey, kp);
  }
  return rho == 1 ? shared_rows<NCMAX, 0, 1>(S, L, n, arow, col, Y, ys, ey, kp)
                  : shared_rows<NCMAX, 0, 2>(S, L, n, arow, col, Y, ys, ey, kp);
}

template <int NCMAX>
__device__ __forceinline__ cd dispatch_member(int n, int rho, const cd* S, int L,
                                              const int32_t* lab, const int32_t* col,
                                              const cd* Y, int ys, int ey, int kc, bool* fail) {
#define MHC_MD(N)                                                                      \
  case N:                                                                              \
    return rho == 1 ? member_det<N, N, 1>(S, L, N, lab, col, Y, ys, ey, kc, fail)      \
                    : member_det<N, N, (N >= 2 ? 2 : 1)>(S, L, N, lab, col, Y, ys, ey, kc, fail);
  switch (n) {
    MHC_MD(1)
    MHC_MD(2)
    MHC_MD(3)
    MHC_MD(4)
    MHC_MD(5)
    MHC_MD(6)
    default:
      break;
  }
#undef MHC_MD
  if constexpr (NCMAX >= 14) {  // three changed rows (n_f >= 14 only)
    if (rho == 3) return member_det<NCMAX, 0, 3>(S, L, n, lab, col, Y, ys, ey, kc, fail);
  }
  if constexpr (NCMAX >= 18) {
    if (rho == 4) return member_det<NCMAX, 0, 4>(S, L, n, lab, col, Y, ys, ey, kc, fail);
  }
  if constexpr (NCMAX >= 32) {
    if (rho == 5) return member_det<NCMAX, 0, 5>(S, L, n, lab, col, Y, ys, ey, kc, fail);
    if (rho == 6) return member_det<NCMAX, 0, 6>(S, L, n, lab, col, Y, ys, ey, kc, fail);
  }
  if constexpr (NCMAX >= 18) {  // the n of the large-nucleus and batched workloads
    if (n == 9)
      return rho == 1 ? member_det<9, 9, 1>(S, L, 9, lab, col, Y, ys, ey, kc, fail)
                      : member_det<9, 9, 2>(S, L, 9, lab, col, Y, ys, ey, kc, fail);
    if (n == 12)
      return rho == 1 ? member_det<12, 12, 1>(S, L, 12, lab, col, Y, ys, ey, kc, fail)
                      : member_det<12, 12, 2>(S, L, 12, lab, col, Y, ys, ey, kc, fail);
    if (n == 18)
      return rho == 1 ? member_det<18, 18, 1>(S, L, 18, lab, col, Y, ys, ey, kc, fail)
                      : member_det<18, 18, 2>(S, L, 18, lab, col, Y, ys, ey, kc, fail);
  }
  return rho == 1 ? member_det<NCMAX, 0, 1>(S, L, n, lab, col, Y, ys, ey, kc, fail)
                  : member_det<NCMAX, 0, 2>(S, L, n, lab, col, Y, ys, ey, kc, fail);
}

template <int NCMAX>
__device__ __forceinline__ void dispatch_dots_z1(int n, const cd* S, int L, const int32_t* lab,
                                                 const int32_t* col, const cd* Y, int ys, cd* d11,
                                                 cd* d21) {
  if constexpr (NCMAX >= 18) {
    if (n == 12) { member_dots_z1<12, 12>(S, L, 12, lab, col, Y, ys, d11, d21); return; }
    if (n == 18) { member_dots_z1<18, 18>(S, L, 18, lab, col, Y, ys, d11, d21); return; }
  }
  member_dots_z1<NCMAX, 0>(S, L, n, lab, col, Y, ys, d11, d21);
}

template <int NCMAX>
__device__ __forceinline__ cd dispatch_member_z1(int n, const cd* S, int L, const int32_t* lab,
                                                 const int32_t* col, const cd* Y, int ys, int ey, int kc,
                                                 bool* fail, cd d11, cd d21) {
  if constexpr (NCMAX >= 18) {
    if (n == 12) return member_det_z1<12, 12>(S, L, 12, lab, col, Y, ys, ey, kc, fail, d11, d21);
    if (n == 18) return member_det_z1<18, 18>(S, L, 18, lab, col, Y, ys, ey, kc, fail, d11, d21);
  }
  return member_det_z1<NCMAX, 0>(S, L, n, lab, col, Y, ys, ey, kc, fail, d11, d21);
}

template <int NCMAX>
__device__ __forceinline__ void dispatch_kapply(int n, const cd* S, int L, const int32_t* arow,
                                                const int32_t* col, const cd* K, cd* Y, int ys,
                                                int* ey) {
  switch (n) {
    case 1: kapply<1, 1>(S, L, 1, arow, col, K, Y, ys, ey); return;
    case 2: kapply<2, 2>(S, L, 2, arow, col, K, Y, ys, ey); return;
    case 3: kapply<3, 3>(S, L, 3, arow, col, K, Y, ys, ey); return;
    case 4: kapply<4, 4>(S, L, 4, arow, col, K, Y, ys, ey); return;
    case 5: kapply<5, 5>(S, L, 5, arow, col, K, Y, ys, ey); return;
    case 6: kapply<6, 6>(S, L, 6, arow, col, K, Y, ys, ey); return;
    default: break;
  }
  if constexpr (NCMAX >= 18) {
    if (n == 9) { kapply<9, 9>(S, L, 9, arow, col, K, Y, ys, ey); return; }
    if (n == 12) { kapply<12, 12>(S, L, 12, arow, col, K, Y, ys, ey); return; }
    if (n == 18) { kapply<18, 18>(S, L, 18, arow, col, K, Y, ys, ey); return; }
  }
  kapply<NCMAX, 0>(S, L, n, arow, col, K, Y, ys, ey);
}

template <int NCMAX>
__device__ __forceinline__ void dispatch_kapply2(int n, const cd* S, int L, const int32_t* arow,
                                                 const int32_t* col, const cd* K, cd* Y, int ys,
                                                 int* ey) {
  switch (n) {
    case 2: kapply2<2, 2>(S, L, 2, arow, col, K, Y, ys, ey); return;
    case 3: kapply2<3, 3>(S, L, 3, arow, col, K, Y, ys, ey); return;
    case 4: kapply2<4, 4>(S, L, 4, arow, col, K, Y, ys, ey); return;
    case 5: kapply2<5, 5>(S, L, 5, arow, col, K, Y, ys, ey); return;
    case 6: kapply2<6, 6>(S, L, 6, arow, col, K, Y, ys, ey); return;
    default: break;
  }
  if constexpr (NCMAX >= 18) {
    if (n == 12) { kapply2<12, 12>(S, L, 12, arow, col, K, Y, ys, ey); return; }
    if (n == 18) { kapply2<18, 18>(S, L, 18, arow, col, K, Y, ys, ey); return; }
  }
  kapply2<NCMAX, 0>(S, L, n, arow, col, K, Y, ys, ey);
}

template <int NCMAX>
__device__ __forceinline__ void dispatch_kapply22(int n, const cd* S, int L, const int32_t* arow,
                                                  const int32_t* col, const cd* K, cd* Y, int ys,
                                                  int* ey) {
  if constexpr (NCMAX >= 18) {
    if (n == 12) { kapply22<12, 12>(S, L, 12, arow, col, K, Y, ys, ey); return; }
    if (n == 18) { kapply22<18, 18>(S, L, 18, arow, col, K, Y, ys, ey); return; }
  }
  kapply22<NCMAX, 0>(S, L, n, arow, col, K, Y, ys, ey);
}

template <int NCMAX>
__device__ __forceinline__ void dispatch_kapply12(int n, const cd* S, int L, const int32_t* arow,
                                                  const int32_t* col, const cd* K, cd* Y, int ys,
                                                  int* ey) {
  switch (n) {
    case 2: kapply12<2, 2>(S, L, 2, arow, col, K, Y, ys, ey); return;
    case 3: kapply12<3, 3>(S, L, 3, arow, col, K, Y, ys, ey); return;
    case 4: kapply12<4, 4>(S, L, 4, arow, col, K, Y, ys, ey); return;
    case 5: kapply12<5, 5>(S, L, 5, arow, col, K, Y, ys, ey); return;
    case 6: kapply12<6, 6>(S, L, 6, arow, col, K, Y, ys, ey); return;
    default: break;
  }
  if constexpr (NCMAX >= 18) {
    if (n == 12) { kapply12<12, 12>(S, L, 12, arow, col, K, Y, ys, ey); return; }
    if (n == 18) { kapply12<18, 18>(S, L, 18, arow, col, K, Y, ys, ey); return; }
  }
  kapply12<NCMAX, 0>(S, L, n, arow, col, K, Y, ys, ey);
}

template <int NCMAX>
__device__ __forceinline__ cd dispatch_fresh(int n, const cd* S, int L, const int32_t* rows,
                                             const int32_t* col) {
#define MHC_FD(N) \
  case N:         \
    return fresh_det<N, N>(S, L, N, rows, col);
  switch (n) {
    MHC_FD(1)
    MHC_FD(2)
    MHC_FD(3)
    MHC_FD(4)
    MHC_FD(5)
    MHC_FD(6)
    default:
      break;
  }
#undef MHC_FD
  return fresh_det<NCMAX, 0>(S, L, n, rows, col);
}

// column labels of the sink at position j (aligned order in the two-sided update)
__device__ __forceinline__ const int32_t* sink_cols(const FwdArgs& a, int64_t j) {
  return (a.snk_orig ? a.snk_pos : a.snk_lab) + j * a.Tn;
}

// Rows of member m in flavour f for a fresh factorisation: the shared rows, then the
// member's labels at the changed rows (the same order as the cached path).
__device__ __forceinline__ void member_rows(const FwdArgs& a, int W, int m, int f, int rho,
                                           int32_t* rows) {
  const int n = a.n_f[f];
  const int32_t* ar = a.fam_arow + (int64_t)W * a.Tn + a.off_f[f];
  for (int i = 0; i < n - rho; i++) rows[i] = ar[i];
  for (int t = 0; t < rho; t++) rows[n - rho + t] = a.mem_lab[((int64_t)m * a.F + f) * MHC_MAX_RANK + t];
}

// Per-flavour exponent scales of the member guard, packed 16 bits per flavour into two 64-bit
// registers: an array indexed by the runtime flavour would live in local memory, and the
// member loop reads it for every member and flavour.  (The n <= 8 class keeps the array:
// its loads hit L1, and packing measured no faster there.)
struct FlavourScalesArray {
  int e[MHC_FMAX];
  __device__ __forceinline__ void set(int f, int v) { e[f] = v; }
  __device__ __forceinline__ int get(int f) const { return e[f]; }
};
struct FlavourScales {
  unsigned long long w[2] = {0ull, 0ull};
  __device__ __forceinline__ void set(int f, int v) {
    const int s = 16 * (f & 3);
    const unsigned long long m = 0xffffull << s;
    const unsigned long long x = (unsigned long long)(unsigned short)(short)v << s;
    if (f < 4) w[0] = (w[0] & ~m) | x; else w[1] = (w[1] & ~m) | x;
  }
  __device__ __forceinline__ int get(int f) const {
    return (int)(short)(unsigned short)(((f < 4) ? w[0] : w[1]) >> (16 * (f & 3)));
  }
};
template <int NCMAX>
using ScalesFor = typename std::conditional<(NCMAX > 8), FlavourScales, FlavourScalesArray>::type;

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

__device__ __forceinline__ bool finite2(double2 v) {
  // exponent field all ones means Inf or NaN
  return ((__double2hiint(v.x) & 0x7ff00000) != 0x7ff00000) &&
         ((__double2hiint(v.y) & 0x7ff00000) != 0x7ff00000);
}

}  // namespace dev

// one work item of the persistent batched launch
struct BatchItem {
  int32_t corr, W, tile, pad;
};

// per-warp refactor queue of the forward kernel
constexpr int kQueueCap = 64;         // entries per warp
constexpr int kQueueEntryBytes = 48;  // sizeof(fwd::QEntry)
// per-warp store of the members' dots with a block's first null vector (rank-2 families
// against one-column sink families): two flavours, 32 members, two complex values
constexpr int kZ1Flavours = 2;
constexpr int kZ1Bytes = kZ1Flavours * 32 * 2 * 16;
// per-warp scratch of the grouped refactors: the multipliers of the shared elimination by
// step, packed (n - 1 + n - 2 + ... + 1 complex values for n <= 18)
constexpr int kWalkMaxN = 18;
constexpr int kWalkBytes = kWalkMaxN * (kWalkMaxN - 1) / 2 * 16;

// host-side launchers (forward.cu and fwd_nc*.cu)
cudaError_t launch_forward(const FwdArgs& a, int ncmax, int tile, int64_t n_fam, int64_t items,
                           size_t smem, double* out, cudaStream_t s);
cudaError_t launch_reduce(const double2* partials, int64_t items, double* out, cudaStream_t s);
cudaError_t launch_forward_cw(const FwdArgs& a0, const double* const* ws, const double* const* wk,
                              int ncmax, int tile, int64_t n_fam, int64_t items, size_t smem, double* tmp,
                              double* out, cudaStream_t s);
cudaError_t launch_pairs(const FwdArgs& a, int ncmax, int64_t n_pairs, int64_t n_src,
                         const int64_t* ii, const int64_t* jj, const int32_t* src_member,
                         const int32_t* mem_family, double* dets, int32_t* path, cudaStream_t s);
size_t forward_smem_bytes(int slots, int tile);
#define MHC_DECL_NC(NC)                                                                       \
  cudaError_t launch_fwd_nc##NC(const FwdArgs& a, int tile, int64_t items, size_t smem,       \
                                cudaStream_t s);                                              \
  cudaError_t launch_pairs_nc##NC(const FwdArgs& a, int64_t n_pairs, int64_t n_src,           \
                                  const int64_t* ii, const int64_t* jj,                       \
                                  const int32_t* src_member, const int32_t* mem_family,       \
                                  double* dets, int32_t* path, cudaStream_t s);      \
  cudaError_t launch_batch_nc##NC(int grid, int T, size_t smem, cudaStream_t s,               \
                                  const FwdArgs* desc, const BatchItem* items,                \
                                  int64_t n_items, unsigned long long* head,                  \
                                  const int64_t* part_off, double2* partials);                \
  int batch_occupancy_nc##NC(int T, size_t smem);                                            \
  cudaError_t launch_kfac_nc##NC(const FwdArgs& a, int64_t n_fam, cudaStream_t s);           \
  cudaError_t launch_kfac_batch_nc##NC(const FwdArgs* desc, const int64_t* kpref,            \
                                       const int64_t* nfam, int count, int64_t total,         \
                                       int big, cudaStream_t s);
MHC_DECL_NC(8)
MHC_DECL_NC(18)
MHC_DECL_NC(32)
#undef MHC_DECL_NC

}  // namespace mhc
