// runtime.cu -- plan upload, workspaces, launches and status of the C ABI.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "plan.h"
#include "trace.h"

namespace mhc {

namespace {

#define MHC_CUDA(call)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                       \
      return MHC_ECUDA;                                                                    \
    }                                                                                      \
  } while (0)

template <typename T>
mhc_status upload(T** dst, const T* src, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(dst, count * sizeof(T));
  if (e != cudaSuccess) {
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MHC_ENOMEM : MHC_ECUDA;
  }
  if (src) {
    e = cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      set_error(std::string("cudaMemcpy: ") + cudaGetErrorString(e));
      return MHC_ECUDA;
    }
  }
  return MHC_OK;
}

void free_device(DevicePlan& d) {
  void* ptrs[] = {d.fam_info, d.fam_rank, d.fam_arow, d.fam_order, d.mem_term, d.mem_par, d.mem_lab,
                  d.snk_lab, d.src_member, d.mem_family, d.w_src, d.w_snk, d.partials,
                  d.counters, d.bwd_rows, d.bwd_wsrc, d.bwd_wsnk, d.snk_order, d.snk_lab2,
                  d.snk_par2, d.snk_q, d.q_off, d.q_two, d.q_rank, d.kbuf, d.kguard, d.kinv, d.bwd_stage,
                  d.bwd_accs, d.bwd_r2, d.bwd_dets, d.cw_tmp};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (auto& bi : d.bwd_index) {
    if (bi.off) cudaFree(bi.off);
    if (bi.ent) cudaFree(bi.ent);
  }
  d = DevicePlan();
}

int log2_inv(double tau) {
  if (!(tau > 0.0)) return 4096;
  return (int)std::floor(-std::log2(tau) + 0.5);
}

}  // namespace

// complex entries of one two-sided block of a flavour with n labels (see kapply/kapply2)
size_t kblock_size(int n) {
  if (n <= 0) return 0;
  const size_t m1 = (size_t)(n - 1), m2 = n >= 2 ? (size_t)(n - 2) : 0;
  return std::max(m1 * m1 + m1 + 2, m2 * m2 + 2 * m2 + 1);
}

int plan_ncmax(const Plan& p) { return p.max_n <= 8 ? 8 : (p.max_n <= 18 ? 18 : 32); }

int plan_tile(const Plan& p) {
  if (p.opts.sink_tile) return p.opts.sink_tile;
  return p.max_n <= 8 ? 128 : (p.max_n <= 12 ? 64 : 32);
}

// y-cache slots per flavour: n for rank-1 families, r n + 1 when some family has rank r >= 2
void plan_slots(const Plan& p, int* yoff, int* total) {
  int s = 0;
  for (int f = 0; f < p.F; f++) {
    int r = 0;
    for (int64_t W = 0; W < p.n_fam; W++) r = std::max(r, (int)p.fam_rank[W * p.F + f]);
    yoff[f] = s;
    const int n = p.n_f[f];
    s += (r >= 2) ? r * n + 1 : n;  // rank r >= 2: r null vectors and sd
  }
  *total = std::max(s, 1);
}

mhc_status ensure_device(Plan& p) {
  int cur = 0;
  MHC_CUDA(cudaGetDevice(&cur));
  DevicePlan& d = p.dev;
  if (d.device == cur) return MHC_OK;
  if (d.device >= 0) {
    int prev = cur;
    cudaSetDevice(d.device);
    cudaDeviceSynchronize();
    free_device(d);
    cudaSetDevice(prev);
  }
  const int F = p.F;
  std::vector<int32_t> info(4 * p.n_fam, 0);
  for (int64_t W = 0; W < p.n_fam; W++) {
    info[4 * W] = (int32_t)p.fam_off[W];
    info[4 * W + 1] = (int32_t)(p.fam_off[W + 1] - p.fam_off[W]);
  }
  std::vector<int32_t> term(p.mem_term.begin(), p.mem_term.end());
  mhc_status st;
  if ((st = upload(&d.fam_info, info.data(), info.size())) != MHC_OK) return st;
  if ((st = upload(&d.fam_rank, p.fam_rank.data(), p.fam_rank.size())) != MHC_OK) return st;
  if ((st = upload(&d.fam_arow, p.fam_arow.data(), p.fam_arow.size())) != MHC_OK) return st;
  // work order by y-cache layout (see FwdArgs::fam_order): families grouped by the rank of
  // each flavour, each group in plan order, the groups by cache size (the all-rank-1 group
  // first); beyond kMaxFwdRanges groups the largest layouts share the plan's layout, which
  // holds any family.  One group: natural order, one launch.
  {
    std::map<std::vector<int>, std::vector<int32_t>> groups;
    for (int64_t W = 0; W < p.n_fam; W++) {
      std::vector<int> key(F);
      for (int f = 0; f < F; f++) key[f] = p.n_f[f] > 0 ? std::max(1, (int)p.fam_rank[W * F + f]) : 0;
      groups[key].push_back((int32_t)W);
    }
    struct G {
      int slots;
      std::vector<int> yoff;
      const std::vector<int32_t>* fams;
    };
    std::vector<G> gs;
    for (auto& kv : groups) {
      G g{0, std::vector<int>(F, 0), &kv.second};
      for (int f = 0; f < F; f++) {
        g.yoff[f] = g.slots;
        const int r = kv.first[f], n = p.n_f[f];
        g.slots += r >= 2 ? r * n + 1 : n;
      }
      g.slots = std::max(g.slots, 1);
      gs.push_back(std::move(g));
    }
    std::stable_sort(gs.begin(), gs.end(), [](const G& x, const G& y) { return x.slots < y.slots; });
    d.n_ranges = 0;
    if (gs.size() >= 2) {
      int yw[MHC_FMAX], sw = 0;
      plan_slots(p, yw, &sw);
      std::vector<int32_t> order;
      order.reserve(p.n_fam);
      for (size_t k = 0; k < gs.size(); k++) {
        const bool merged = k + 1 >= (size_t)kMaxFwdRanges;  // the last range takes the rest
        FwdRange& r = d.ranges[d.n_ranges];
        if (!merged || k + 1 == (size_t)kMaxFwdRanges) {
          r.first = (int64_t)order.size();
          r.count = 0;
          r.slots = merged ? sw : gs[k].slots;
          for (int f = 0; f < MHC_FMAX; f++) r.yoff[f] = f < F ? (merged ? yw[f] : gs[k].yoff[f]) : 0;
          d.n_ranges++;
        }
        order.insert(order.end(), gs[k].fams->begin(), gs[k].fams->end());
        d.ranges[d.n_ranges - 1].count += (int64_t)gs[k].fams->size();
      }
      if ((st = upload(&d.fam_order, order.data(), order.size())) != MHC_OK) return st;
    }
  }
  if ((st = upload(&d.mem_term, term.data(), term.size())) != MHC_OK) return st;
  if ((st = upload(&d.mem_par, p.mem_par.data(), p.mem_par.size())) != MHC_OK) return st;
  if ((st = upload(&d.mem_lab, p.mem_lab.data(), p.mem_lab.size())) != MHC_OK) return st;
  if ((st = upload(&d.snk_lab, p.labels_snk.data(), p.labels_snk.size())) != MHC_OK) return st;
  if ((st = upload(&d.src_member, p.src_member.data(), p.src_member.size())) != MHC_OK) return st;
  if ((st = upload(&d.mem_family, p.mem_family.data(), p.mem_family.size())) != MHC_OK) return st;
  if ((st = upload(&d.w_src, p.w_src.data(), p.w_src.size())) != MHC_OK) return st;
  if ((st = upload(&d.w_snk, p.w_snk.data(), p.w_snk.size())) != MHC_OK) return st;
  // two-sided update: sink tables and the block-factor store (skipped above 16 GB)
  size_t kstride = 0;
  for (int f = 0; f < p.F; f++) kstride += kblock_size(p.n_f[f]);
  const double kbytes = (double)p.n_fam * (double)p.n_qfam * (double)kstride * 16.0;
  d.two_sided = !p.opts.one_sided && p.two_sided_pairs > 0 && kbytes <= 16e9;
  if (d.two_sided) {
    if ((st = upload(&d.snk_order, p.snk_order.data(), p.snk_order.size())) != MHC_OK) return st;
    if ((st = upload(&d.snk_lab2, p.snk_lab2.data(), p.snk_lab2.size())) != MHC_OK) return st;
    if ((st = upload(&d.snk_par2, p.snk_par2.data(), p.snk_par2.size())) != MHC_OK) return st;
    if ((st = upload(&d.snk_q, p.snk_q.data(), p.snk_q.size())) != MHC_OK) return st;
    if ((st = upload(&d.q_off, p.q_off.data(), p.q_off.size())) != MHC_OK) return st;
    if ((st = upload(&d.q_two, p.q_two.data(), p.q_two.size())) != MHC_OK) return st;
    if ((st = upload(&d.q_rank, p.q_rank.data(), p.q_rank.size())) != MHC_OK) return st;
    if ((st = upload<double>(&d.kbuf, nullptr, 2 * (size_t)p.n_fam * p.n_qfam * kstride)) != MHC_OK) return st;
    if ((st = upload<int32_t>(&d.kguard, nullptr, (size_t)p.n_fam * p.n_qfam * p.F)) != MHC_OK) return st;
    d.kstride = (int)kstride;
  }
  d.tile = plan_tile(p);
  d.n_tiles = (int32_t)((p.n_snk + d.tile - 1) / d.tile);
  d.n_items = p.n_fam * d.n_tiles;
  if ((st = upload<double>(&d.partials, nullptr, 2 * (size_t)d.n_items)) != MHC_OK) return st;
  if ((st = upload<unsigned long long>(&d.counters, nullptr, kNumCounters)) != MHC_OK) return st;
  MHC_CUDA(cudaMemset(d.counters, 0, kNumCounters * sizeof(unsigned long long)));
  (void)F;
  d.device = cur;
  return MHC_OK;
}

mhc_status fill_fwd_args(Plan& p, const double* const* S_f, const double* w_src,
                         const double* w_snk, FwdArgs& a) {
  std::memset(&a, 0, sizeof(a));
  a.F = p.F;
  a.Tn = p.Tn;
  a.n_snk = p.n_snk;
  a.n_tiles = p.dev.n_tiles;
  plan_slots(p, a.yoff, &a.slots);
  a.kp = log2_inv(p.opts.tau_parent);
  a.kc = log2_inv(p.opts.tau_child);
  a.rowdiff = p.opts.row_difference ? 1 : 0;
  for (int f = 0; f < p.F; f++) {
    a.n_f[f] = p.n_f[f];
    a.L_f[f] = p.L_f[f];
    a.off_f[f] = p.off_f[f];
    if (p.n_f[f] > 0 && (!S_f || !S_f[f])) {
      set_error("S_f[" + std::to_string(f) + "] is NULL");
      return MHC_EINVAL;
    }
    a.S[f] = p.n_f[f] > 0 ? reinterpret_cast<const double2*>(S_f[f]) : nullptr;
  }
  a.fam_info = p.dev.fam_info;
  a.fam_rank = p.dev.fam_rank;
  a.fam_arow = p.dev.fam_arow;
  a.mem_term = p.dev.mem_term;
  a.mem_par = p.dev.mem_par;
  a.mem_lab = p.dev.mem_lab;
  a.snk_lab = p.dev.snk_lab;
  a.w_src = w_src ? w_src : p.dev.w_src;
  a.w_snk = w_snk ? w_snk : p.dev.w_snk;
  a.partials = reinterpret_cast<double2*>(p.dev.partials);
  a.counters = p.dev.counters;
  a.fam_order = p.dev.fam_order;
  a.n_ranges = p.dev.fam_order ? p.dev.n_ranges : 0;
  for (int r = 0; r < a.n_ranges; r++) a.ranges[r] = p.dev.ranges[r];
  if (p.dev.two_sided) {
    a.snk_pos = p.dev.snk_lab2;
    a.snk_orig = p.dev.snk_order;
    a.snk_par = p.dev.snk_par2;
    a.snk_q = p.dev.snk_q;
    a.q_two = p.dev.q_two;
    a.q_rank = p.dev.q_rank;
    a.q_off = p.dev.q_off;
    a.kbuf = reinterpret_cast<const double2*>(p.dev.kbuf);
    a.kguard = p.dev.kguard;
    a.n_q = p.n_qfam;
    a.kstride = p.dev.kstride;
    for (int f = 0, o = 0; f < p.F; f++) {
      a.koff[f] = o;
      o += (int)kblock_size(p.n_f[f]);
    }
  }
  return MHC_OK;
}

cudaError_t launch_pairs(const FwdArgs& a, int ncmax, int64_t n_pairs, int64_t n_src,
                         const int64_t* ii, const int64_t* jj, const int32_t* src_member,
                         const int32_t* mem_family, double* dets, int32_t* path, cudaStream_t s);

}  // namespace mhc

using namespace mhc;

extern "C" {

void mhc_plan_destroy(mhc_plan_t plan) {
  if (!plan) return;
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (p->dev.device >= 0) {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(p->dev.device);
    cudaDeviceSynchronize();
    free_device(p->dev);
    cudaSetDevice(prev);
  }
  delete p;
}

mhc_status mhc_correlator(mhc_plan_t plan, const double* const* S_f, const double* w_src_dev,
                          const double* w_snk_dev, double* out_dev, mhc_stream_t stream) {
  if (!plan || !out_dev) {
    set_error("mhc_correlator: NULL plan or output");
    return MHC_EINVAL;
  }
  Plan& p = *reinterpret_cast<Plan*>(plan);
  TraceRange trace("mhc_correlator");
  mhc_status st = ensure_device(p);
  if (st != MHC_OK) return st;
  FwdArgs a;
  if ((st = fill_fwd_args(p, S_f, w_src_dev, w_snk_dev, a)) != MHC_OK) return st;
  const int tile = p.dev.tile;
  const size_t smem = forward_smem_bytes(a.slots, tile);
  MHC_CUDA(launch_forward(a, plan_ncmax(p), tile, p.n_fam, p.dev.n_items, smem, out_dev,
                          reinterpret_cast<cudaStream_t>(stream)));
  return MHC_OK;
}

mhc_status mhc_correlator_cw(mhc_plan_t plan, const double* const* S_f, const double* w_src_re,
                             const double* w_src_im, const double* w_snk_re, const double* w_snk_im,
                             double* out_dev, mhc_stream_t stream) {
  if (!plan || !out_dev || !w_src_re || !w_src_im || !w_snk_re || !w_snk_im) {
    set_error("mhc_correlator_cw: NULL plan, weight or output");
    return MHC_EINVAL;
  }
  Plan& p = *reinterpret_cast<Plan*>(plan);
  mhc_status st = ensure_device(p);
  if (st != MHC_OK) return st;
  if (!p.dev.cw_tmp && cudaMalloc(&p.dev.cw_tmp, 8 * sizeof(double)) != cudaSuccess) {
    set_error("mhc_correlator_cw: cudaMalloc failed");
    return MHC_ENOMEM;
  }
  FwdArgs a;
  if ((st = fill_fwd_args(p, S_f, w_src_re, w_snk_re, a)) != MHC_OK) return st;
  const double* ws[2] = {w_src_re, w_src_im};
  const double* wk[2] = {w_snk_re, w_snk_im};
  const int tile = p.dev.tile;
  const size_t smem = forward_smem_bytes(a.slots, tile);
  MHC_CUDA(launch_forward_cw(a, ws, wk, plan_ncmax(p), tile, p.n_fam, p.dev.n_items, smem, p.dev.cw_tmp,
                             out_dev, reinterpret_cast<cudaStream_t>(stream)));
  return MHC_OK;
}

mhc_status mhc_pair_dets(mhc_plan_t plan, const double* const* S_f, int64_t n_pairs,
                         const int64_t* i_dev, const int64_t* j_dev, double* dets_dev,
                         int32_t* path_dev, mhc_stream_t stream) {
  if (!plan || n_pairs < 0 || (n_pairs > 0 && (!i_dev || !j_dev || !dets_dev))) {
    set_error("mhc_pair_dets: bad argument");
    return MHC_EINVAL;
  }
  Plan& p = *reinterpret_cast<Plan*>(plan);
  mhc_status st = ensure_device(p);
  if (st != MHC_OK) return st;
  FwdArgs a;
  if ((st = fill_fwd_args(p, S_f, nullptr, nullptr, a)) != MHC_OK) return st;
  MHC_CUDA(launch_pairs(a, plan_ncmax(p), n_pairs, p.n_src, i_dev, j_dev, p.dev.src_member,
                        p.dev.mem_family, dets_dev, path_dev,
                        reinterpret_cast<cudaStream_t>(stream)));
  return MHC_OK;
}

mhc_status mhc_get_status(mhc_plan_t plan, mhc_stream_t stream) {
  if (!plan) {
    set_error("mhc_get_status: NULL plan");
    return MHC_EINVAL;
  }
  Plan& p = *reinterpret_cast<Plan*>(plan);
  if (p.dev.device < 0) return MHC_OK;
  unsigned long long c[kNumCounters] = {0, 0, 0, 0, 0};
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  MHC_CUDA(cudaStreamSynchronize(s));
  MHC_CUDA(cudaMemcpy(c, p.dev.counters, sizeof(c), cudaMemcpyDeviceToHost));
  MHC_CUDA(cudaMemset(p.dev.counters, 0, sizeof(c)));
  p.stats.refactor_parent = (int64_t)c[1];
  p.stats.refactor_child = (int64_t)c[2];
  p.stats.refactor_flops = (double)c[3];
  p.stats.row_difference = (int64_t)c[4];
  if (c[0] & kStatusTimeout) {
    set_error("a bounded device wait ran out");
    return MHC_ETIMEOUT;
  }
  if (c[0] & kStatusBadIndex) {
    set_error("a pair index was out of range");
    return MHC_EINVAL;
  }
  if (c[0] & kStatusUnsupported) {
    set_error("a kernel could not complete a request it does not support");
    return MHC_EUNSUPPORTED;
  }
  if (c[0] & kStatusNonFinite) {
    set_error("a non-finite value reached a result");
    return MHC_ENONFINITE;
  }
  return MHC_OK;
}

}  // extern "C"
