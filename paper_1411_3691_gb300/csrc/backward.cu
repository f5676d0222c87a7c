// backward.cu -- host side of the adjoint: workspace, launch, and the fixed-order final
// reductions of the per-warp accumulators into dS_f, dw_src and dw_snk.
#include <algorithm>
#include <string>
#include <vector>

#include "bwd_impl.cuh"
#include "plan.h"
#include "trace.h"

namespace mhc {

cudaError_t launch_bwd_nc8(const BwdArgs& b, int T, int64_t ctas, size_t smem, cudaStream_t s);
cudaError_t launch_bwd_nc18(const BwdArgs& b, int T, int64_t ctas, size_t smem, cudaStream_t s);
cudaError_t launch_bwd_nc32(const BwdArgs& b, int T, int64_t ctas, size_t smem, cudaStream_t s);
cudaError_t launch_kinv_nc8(const BwdArgs& b, int64_t n_fam, cudaStream_t s);
cudaError_t launch_kinv_nc18(const BwdArgs& b, int64_t n_fam, cudaStream_t s);
cudaError_t launch_kinv_nc32(const BwdArgs& b, int64_t n_fam, cudaStream_t s);
int plan_ncmax(const Plan& p);
mhc_status ensure_device(Plan& p);
mhc_status fill_fwd_args(Plan& p, const double* const* S_f, const double* w_src,
                         const double* w_snk, FwdArgs& a);

namespace {

// dS_f[a][b] = g conj(sum over (W, slot) rows labelled a, chunks, warps of the partials).
// One block per (row a, group of 32 columns): lane = column, the 32 warps take the terms
// (row entry, chunk, warp) round-robin in a fixed order, then a fixed-order sum over the
// warps -- the same result on every call.
constexpr int kFinWarps = 32;
__global__ void __launch_bounds__(32 * kFinWarps)
    fin_dS_kernel(int f, int L, const int32_t* __restrict__ list_off, const int2* __restrict__ list,
                  const double2* __restrict__ part, int n_chunks, int warps, int F, int slots_max,
                  int Lmax, const double* __restrict__ g, double2* __restrict__ dS) {
  __shared__ double2 red[kFinWarps][32];
  const int a = blockIdx.y;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int b = blockIdx.x * 32 + lane;
  const int bc = b < L ? b : L - 1;
  const int k0 = list_off[a];
  const int64_t per = (int64_t)n_chunks * warps;
  const int nk = list_off[a + 1] - k0;
  double2 s = make_double2(0.0, 0.0);
  // term t = k * per + cw (cw = chunk * warps + warp); this warp takes t = wp, wp + kFinWarps, ...
  int k = 0;
  int64_t cw = wp;
  while (cw >= per) {
    cw -= per;
    k++;
  }
  while (k < nk) {
    const int2 ws = list[k0 + k];
    const int64_t row = (((int64_t)ws.x * per + cw) * F + f) * slots_max + ws.y;
    const double2 v = part[row * Lmax + bc];
    s.x += v.x;
    s.y += v.y;
    cw += kFinWarps;
    while (cw >= per) {
      cw -= per;
      k++;
    }
  }
  red[wp][lane] = s;
  __syncthreads();
  if (wp == 0 && b < L) {
    double2 t = red[0][lane];
    for (int w = 1; w < kFinWarps; w++) {
      t.x += red[w][lane].x;
      t.y += red[w][lane].y;
    }
    const double gr = g[0], gi = g[1];
    dS[(int64_t)a * L + b] = make_double2(gr * t.x + gi * t.y, gi * t.x - gr * t.y);
  }
}

// dw_src[i] = Re(conj(g) sum_chunks part[member(i)][chunk])
__global__ void fin_dwsrc_kernel(int64_t n_src, const int32_t* __restrict__ src_member,
                                 const double2* __restrict__ part, int n_chunks,
                                 const double* __restrict__ g, double* __restrict__ dw) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_src) return;
  const int64_t m = src_member[i];
  double2 s = make_double2(0.0, 0.0);
  for (int c = 0; c < n_chunks; c++) {
    s.x += part[m * n_chunks + c].x;
    s.y += part[m * n_chunks + c].y;
  }
  dw[i] = g[0] * s.x + g[1] * s.y;
}

// dw_snk[j] = Re(conj(g) sum_W part[W][j])
__global__ void fin_dwsnk_kernel(int64_t n_snk, int64_t n_fam, const double2* __restrict__ part,
                                 const double* __restrict__ g, double* __restrict__ dw) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_snk) return;
  double2 s = make_double2(0.0, 0.0);
  for (int64_t W = 0; W < n_fam; W++) {
    s.x += part[W * n_snk + j].x;
    s.y += part[W * n_snk + j].y;
  }
  dw[j] = g[0] * s.x + g[1] * s.y;
}

template <typename T>
mhc_status dev_alloc(T** p, size_t count, size_t* have) {
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  if (*p && *have >= bytes) return MHC_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    set_error(std::string("mhc_correlator_backward: cudaMalloc: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MHC_ENOMEM : MHC_ECUDA;
  }
  *have = bytes;
  return MHC_OK;
}

}  // namespace
}  // namespace mhc

using namespace mhc;

extern "C" mhc_status mhc_correlator_backward(mhc_plan_t plan, const double* const* S_f,
                                              const double* w_src_dev, const double* w_snk_dev,
                                              const double* g_out_dev, double* const* dS_f,
                                              double* dw_src_dev, double* dw_snk_dev,
                                              mhc_stream_t stream) {
  if (!plan || !g_out_dev) {
    set_error("mhc_correlator_backward: NULL plan or g_out");
    return MHC_EINVAL;
  }
  Plan& p = *reinterpret_cast<Plan*>(plan);
  TraceRange trace("mhc_correlator_backward");
  int max_rank = 1;  // families of rank k >= 2: k member rows per member, k^2 coefficients
  for (int64_t W = 0; W < p.n_fam; W++)
    for (int f = 0; f < p.F; f++) max_rank = std::max(max_rank, (int)p.fam_rank[W * p.F + f]);
  const bool any_r2 = max_rank >= 2;
  mhc_status st = ensure_device(p);
  if (st != MHC_OK) return st;
  BwdArgs b;
  if ((st = fill_fwd_args(p, S_f, w_src_dev, w_snk_dev, b.a)) != MHC_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int F = p.F;
  int ysl = b.a.slots, mn_max = 1, Mmax = 0, Lmax = 1;  // ysl: the cached solves' slots
  for (int f = 0; f < F; f++) {
    mn_max = std::max(mn_max, std::max(p.n_f[f] - 1, 0) * p.n_f[f]);
    Mmax = std::max(Mmax, p.n_f[f] - 1);
    Lmax = std::max(Lmax, (int)p.L_f[f]);
  }
  ysl = std::max(ysl, 1);
  const int kmax = std::max(p.max_members, 1);
  // one warp per block: the per-sink state (cached solves, member determinants, weight
  // accumulators) is all that lives in shared memory, so several warps fit per SM
  const int T = 32;
  // cached solves [ysl][t] (the member dets are global scratch of the block)
  auto smem_of = [&](int t) { return (size_t)ysl * t * sizeof(double2); };
  if (smem_of(T) > 220 * 1024) {
    set_error("mhc_correlator_backward: a family is too large for the adjoint's shared memory; "
              "plan with a smaller opts.max_family");
    return MHC_EUNSUPPORTED;
  }
  const size_t smem = smem_of(T);
  const int warps = T / 32;
  const int n_tiles = (int)((p.n_snk + T - 1) / T);
  const int slots_max = Mmax + max_rank * kmax;
  const size_t per_cta = (size_t)warps * F * slots_max * Lmax * sizeof(double2);
  int n_chunks = (int)std::min<int64_t>(n_tiles, std::max<int64_t>(1, (48 * 152 + p.n_fam - 1) / p.n_fam));
  while (n_chunks > 1 && (double)per_cta * p.n_fam * n_chunks > 1.0e9) n_chunks = (n_chunks + 1) / 2;
  const int tiles_per_cta = (n_tiles + n_chunks - 1) / n_chunks;
  n_chunks = (n_tiles + tiles_per_cta - 1) / tiles_per_cta;
  const int64_t ctas = p.n_fam * n_chunks;

  DevicePlan& d = p.dev;
  if ((st = dev_alloc(reinterpret_cast<double2**>(&d.bwd_rows), (size_t)ctas * per_cta / sizeof(double2),
                      &d.bwd_rows_bytes)) != MHC_OK)
    return st;
  if ((st = dev_alloc(reinterpret_cast<double2**>(&d.bwd_wsrc), (size_t)p.n_src * n_chunks,
                      &d.bwd_wsrc_bytes)) != MHC_OK)
    return st;
  if ((st = dev_alloc(reinterpret_cast<double2**>(&d.bwd_wsnk), (size_t)p.n_fam * p.n_snk,
                      &d.bwd_wsnk_bytes)) != MHC_OK)
    return st;
  if ((st = dev_alloc(reinterpret_cast<double2**>(&d.bwd_stage), (size_t)ctas * T * mn_max,
                      &d.bwd_stage_bytes)) != MHC_OK)
    return st;
  if ((st = dev_alloc(reinterpret_cast<double2**>(&d.bwd_accs), (size_t)ctas * kmax * T,
                      &d.bwd_accs_bytes)) != MHC_OK)
    return st;
  if ((st = dev_alloc(reinterpret_cast<double2**>(&d.bwd_dets), (size_t)ctas * F * kmax * (T + 1),
                      &d.bwd_dets_bytes)) != MHC_OK)
    return st;
  if (any_r2 && (st = dev_alloc(reinterpret_cast<double2**>(&d.bwd_r2),
                                (size_t)ctas * kmax * max_rank * max_rank * T, &d.bwd_r2_bytes)) != MHC_OK)
    return st;
  // row-label index of the accumulators, per flavour: label -> (family, slot) pairs
  if (d.bwd_index.empty()) {
    d.bwd_index.resize(F);
    for (int f = 0; f < F; f++) {
      const int L = p.L_f[f], n = p.n_f[f];
      std::vector<std::vector<std::pair<int, int>>> lists(L);
      if (n > 0) {
        for (int64_t W = 0; W < p.n_fam; W++) {
          // slots: shared rows m < n - rho, then the member rows (two per member, rank 2)
          const int rho = p.fam_rank[W * F + f];
          for (int m = 0; m < n - rho; m++) lists[p.fam_arow[W * p.Tn + p.off_f[f] + m]].push_back({(int)W, m});
          for (int64_t c = 0; c < p.fam_off[W + 1] - p.fam_off[W]; c++) {
            const int64_t mm = p.fam_off[W] + c;
            for (int t = 0; t < rho; t++)
              lists[p.mem_lab[(mm * F + f) * MHC_MAX_RANK + t]].push_back({(int)W, (int)(n - rho + rho * c + t)});
          }
        }
      }
      std::vector<int32_t> off(L + 1, 0);
      std::vector<int2> ent;
      for (int a = 0; a < L; a++) {
        for (auto& x : lists[a]) ent.push_back(make_int2(x.first, x.second));
        off[a + 1] = (int32_t)ent.size();
      }
      DevicePlan::BwdIndex& bi = d.bwd_index[f];
      if (cudaMalloc(&bi.off, off.size() * sizeof(int32_t)) != cudaSuccess ||
          cudaMalloc(&bi.ent, std::max<size_t>(ent.size(), 1) * sizeof(int2)) != cudaSuccess) {
        set_error("mhc_correlator_backward: cudaMalloc failed for the row index");
        return MHC_ENOMEM;
      }
      cudaMemcpy(bi.off, off.data(), off.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
      if (!ent.empty()) cudaMemcpy(bi.ent, ent.data(), ent.size() * sizeof(int2), cudaMemcpyHostToDevice);
    }
  }

  b.tiles_per_cta = tiles_per_cta;
  b.n_chunks = n_chunks;
  b.warps = warps;
  b.kmax = kmax;
  b.slots_max = slots_max;
  b.Lmax = Lmax;
  b.mn_max = mn_max;
  b.ysl = ysl;
  b.a.n_tiles = n_tiles;  // the cached-solve layout (a.yoff, a.slots) stays the forward's
  b.dS_part = reinterpret_cast<double2*>(d.bwd_rows);
  b.dwsrc_part = reinterpret_cast<double2*>(d.bwd_wsrc);
  b.dwsnk_part = reinterpret_cast<double2*>(d.bwd_wsnk);
  b.stage = reinterpret_cast<double2*>(d.bwd_stage);
  b.accs = reinterpret_cast<double2*>(d.bwd_accs);
  b.r2 = reinterpret_cast<double2*>(d.bwd_r2);
  b.dets = reinterpret_cast<double2*>(d.bwd_dets);
  b.rk2 = max_rank * max_rank;
  const int nc = plan_ncmax(p);
  b.kinv = nullptr;
  if (b.a.snk_orig) {  // two-sided blocks: the factors of B, then B^{-1} for the cofactors
    size_t kis = 0;
    for (int f = 0; f < F; f++) {
      b.kioff[f] = (int)kis;
      kis += p.n_f[f] > 1 ? (size_t)(p.n_f[f] - 1) * (p.n_f[f] - 1) : 0;
    }
    b.kistride = (int)std::max<size_t>(kis, 1);
    const size_t kcount = (size_t)p.n_fam * p.n_qfam * b.kistride;
    if ((double)kcount * 16.0 <= 16e9) {
      if ((st = dev_alloc(reinterpret_cast<double2**>(&d.kinv), kcount, &d.kinv_bytes)) != MHC_OK) return st;
      b.kinv = reinterpret_cast<const double2*>(d.kinv);
    }
    cudaError_t ek = nc <= 8 ? launch_kfac_nc8(b.a, p.n_fam, s)
                             : (nc <= 18 ? launch_kfac_nc18(b.a, p.n_fam, s) : launch_kfac_nc32(b.a, p.n_fam, s));
    if (ek == cudaSuccess && b.kinv)
      ek = nc <= 8 ? launch_kinv_nc8(b, p.n_fam, s)
                   : (nc <= 18 ? launch_kinv_nc18(b, p.n_fam, s) : launch_kinv_nc32(b, p.n_fam, s));
    if (ek != cudaSuccess) {
      set_error(std::string("mhc_correlator_backward: launch: ") + cudaGetErrorString(ek));
      return MHC_ECUDA;
    }
  }
  cudaError_t e = nc <= 8 ? launch_bwd_nc8(b, T, ctas, smem, s)
                          : (nc <= 18 ? launch_bwd_nc18(b, T, ctas, smem, s) : launch_bwd_nc32(b, T, ctas, smem, s));
  if (e != cudaSuccess) {
    set_error(std::string("mhc_correlator_backward: launch: ") + cudaGetErrorString(e));
    return MHC_ECUDA;
  }
  for (int f = 0; f < F; f++) {
    if (!dS_f || !dS_f[f]) continue;
    const int L = p.L_f[f];  // 1 <= L <= 4096 (validated by the planner)
    fin_dS_kernel<<<dim3((unsigned)((L + 31) / 32), (unsigned)L), 32 * kFinWarps, 0, s>>>(
        f, L, d.bwd_index[f].off, d.bwd_index[f].ent, b.dS_part, n_chunks, warps, F, slots_max,
        Lmax, g_out_dev, reinterpret_cast<double2*>(dS_f[f]));
  }
  if (dw_src_dev)
    fin_dwsrc_kernel<<<(unsigned)((p.n_src + 255) / 256), 256, 0, s>>>(p.n_src, d.src_member, b.dwsrc_part,
                                                                        n_chunks, g_out_dev, dw_src_dev);
  if (dw_snk_dev)
    fin_dwsnk_kernel<<<(unsigned)((p.n_snk + 255) / 256), 256, 0, s>>>(p.n_snk, p.n_fam, b.dwsnk_part,
                                                                        g_out_dev, dw_snk_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("mhc_correlator_backward: ") + cudaGetErrorString(e));
    return MHC_ECUDA;
  }
  return MHC_OK;
}
