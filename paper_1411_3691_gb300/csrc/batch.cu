// batch.cu -- many independent correlators in one persistent launch, captured once into
// a CUDA graph, with the sink tile (threads per block: one thread per sink, so the tile is
// also the number of warps per block times 32) chosen by measurement for each n class and
// remembered in a small cache file.
//
// The work items of all correlators, (correlator, family, sink tile), are listed on the
// host in decreasing order of their FLOP count (largest first), and a grid of one wave of
// thread blocks pulls them from that list through one atomic counter.  Each item writes
// its partial sum to a slot indexed by the item, not by the block that ran it, and each
// correlator's slots are summed in a fixed order afterwards: results do not depend on the
// dynamic assignment.  There is no waiting between blocks, so no bounded wait is needed.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <set>
#include <sstream>
#include <string>
#include <vector>

#include <fcntl.h>
#include <sys/stat.h>
#include <unistd.h>

#include "kernels.cuh"
#include "plan.h"
#include "trace.h"

struct mhc_batch_s;

namespace mhc {

int plan_ncmax(const Plan& p);
mhc_status ensure_device(Plan& p);
mhc_status fill_fwd_args(Plan& p, const double* const* S_f, const double* w_src,
                         const double* w_snk, FwdArgs& a);
void plan_slots(const Plan& p, int* yoff, int* total);

namespace {

// fixed-order sum of each correlator's item partials (one block per correlator)
__global__ void __launch_bounds__(256) batch_reduce(const double2* __restrict__ partials,
                                                    const int64_t* __restrict__ part_off,
                                                    double* const* __restrict__ outs) {
  __shared__ double2 red[8];
  const int b = blockIdx.x;
  const int64_t i0 = part_off[b], i1 = part_off[b + 1];
  double2 s = make_double2(0.0, 0.0);
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
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
    outs[b][0] = t.x;
    outs[b][1] = t.y;
  }
}

// deterministic finite scratch propagators for the autotuner: entries in [-1, 1] + 2 I
__global__ void scratch_S(double2* S, int L, uint32_t seed) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)L * L) return;
  uint32_t x = (uint32_t)e * 2654435761u ^ seed;
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  uint32_t y = x * 0x846ca68bu;
  y ^= y >> 16;
  const double re = (double)(x & 0xffffff) / 8388608.0 - 1.0;
  const double im = (double)(y & 0xffffff) / 8388608.0 - 1.0;
  S[e] = make_double2(re + ((e / L) == (e % L) ? 2.0 : 0.0), im);
}

}  // namespace

// The correlators of a batch by n class (largest n_f of the plan <= 8, 18, 32): each class
// has its own item queue and its own persistent kernel, compiled for that class, so the
// small-n correlators keep the register budget (and occupancy) of their class.
constexpr int kClasses = 3;
constexpr int kClassNc[kClasses] = {8, 18, 32};

// One launch configuration of a batch: a sink tile T[c] per n class.
struct BatchShape {
  int T[kClasses] = {0, 0, 0};
  int ncmax = 8;
  int64_t n_items = 0;
  std::vector<BatchItem> items;   // class by class, each in decreasing cost
  std::vector<int64_t> part_off;  // [count + 1]
  std::vector<int> n_tiles;       // per correlator
  int64_t cls_off[kClasses + 1] = {0, 0, 0, 0};  // items of class c: [cls_off[c], cls_off[c + 1])
  int cls_grid[kClasses] = {0, 0, 0};
  size_t cls_smem[kClasses] = {0, 0, 0};
};

}  // namespace mhc

using namespace mhc;

struct mhc_batch_s {
  int count = 0;
  int device = -1;
  std::vector<Plan*> plans;
  BatchShape shape;
  FwdArgs* d_desc = nullptr;
  BatchItem* d_items = nullptr;
  int64_t* d_part_off = nullptr;
  double2* d_partials = nullptr;
  unsigned long long* d_head = nullptr;
  double** d_outs = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<FwdArgs> h_desc;    // host copies of the descriptors
  int64_t* d_kpref = nullptr;     // [count + 1] first two-sided block thread of each plan
  int64_t* d_nfam = nullptr;      // [count] families per plan
  int64_t k_total = 0;
  int k_big = 0;                  // a two-sided plan has a flavour with n > 6
  // a plan given more than once (one plan, several propagator sets: gauge configurations,
  // time slices) gets batch-owned block factors and guard flags for its later entries
  std::vector<void*> own_kbuf, own_kguard;  // [count], null where the plan's own are used
  cudaStream_t side = nullptr;    // second branch: the class kernels run concurrently
  cudaEvent_t fork = nullptr, join = nullptr;
  std::vector<const void*> key;  // S and out pointers the graph was captured with
  double tune_ms[kClasses][3] = {};  // measured class time per candidate tile (32, 64, 128); 0: not run
  int from_cache[kClasses] = {0, 0, 0};  // 1: the class's tile came from the tuning cache
};

namespace {

int class_of(const Plan& p) {
  const int nc = plan_ncmax(p);
  return nc <= 8 ? 0 : (nc <= 18 ? 1 : 2);
}

BatchShape make_shape(const mhc_batch_s& b, const int (&Tc)[kClasses]) {
  BatchShape sh;
  for (int c = 0; c < kClasses; c++) sh.T[c] = Tc[c];
  struct Cost {
    double c;
    BatchItem it;
  };
  std::vector<Cost> all[kClasses];
  sh.part_off.push_back(0);
  int max_slots[kClasses] = {1, 1, 1};
  for (int k = 0; k < b.count; k++) {
    const Plan& p = *b.plans[k];
    const int cl = class_of(p);
    const int T = Tc[cl];
    const int nt = (int)((p.n_snk + T - 1) / T);
    sh.n_tiles.push_back(nt);
    sh.ncmax = std::max(sh.ncmax, plan_ncmax(p));
    int yoff[MHC_FMAX], slots = 0;
    plan_slots(p, yoff, &slots);
    max_slots[cl] = std::max(max_slots[cl], slots);
    for (int64_t W = 0; W < p.n_fam; W++) {
      double c = 0.0;
      const double kW = (double)(p.fam_off[W + 1] - p.fam_off[W]);
      for (int f = 0; f < p.F; f++) {
        const int n = p.n_f[f], rho = p.fam_rank[W * p.F + f];
        if (n > 0) c += flops_shared_rows(n, rho) + kW * flops_member(n, rho);
      }
      for (int t = 0; t < nt; t++) {
        const double width = (double)std::min<int64_t>(T, p.n_snk - (int64_t)t * T);
        all[cl].push_back({c * width, BatchItem{k, (int32_t)W, t, 0}});
      }
    }
    sh.part_off.push_back(sh.part_off.back() + p.n_fam * nt);
  }
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b.device);
  for (int c = 0; c < kClasses; c++) {
    std::stable_sort(all[c].begin(), all[c].end(), [](const Cost& x, const Cost& y) { return x.c > y.c; });
    sh.cls_off[c] = (int64_t)sh.items.size();
    for (auto& x : all[c]) sh.items.push_back(x.it);
    const int64_t n = (int64_t)all[c].size();
    if (n == 0) continue;
    sh.cls_smem[c] = forward_smem_bytes(max_slots[c], Tc[c]);
    const int occ = c == 0 ? batch_occupancy_nc8(Tc[c], sh.cls_smem[c])
                           : (c == 1 ? batch_occupancy_nc18(Tc[c], sh.cls_smem[c])
                                     : batch_occupancy_nc32(Tc[c], sh.cls_smem[c]));
    sh.cls_grid[c] = (int)std::min<int64_t>((int64_t)sms * occ, n);
  }
  sh.cls_off[kClasses] = (int64_t)sh.items.size();
  sh.n_items = (int64_t)sh.items.size();
  return sh;
}

// the tiles the tuner tries, and the shared memory limit a class's launch must fit in
constexpr int kTiles[3] = {32, 64, 128};
constexpr size_t kSmemLimit = 200 * 1024;

// ---- tuning cache ---------------------------------------------------------------------
// One JSON object per line: {"key": "...", "tile": T, "ms": [t32, t64, t128]}; the last
// line with a key wins.  The file is MHC_TUNE_CACHE if that variable is set (empty: no
// cache), else $HOME/.cache/mhc/tune.jsonl.  Lines are appended with one write() each.
std::mutex g_cache_mutex;

std::string cache_path() {
  const char* e = std::getenv("MHC_TUNE_CACHE");
  if (e) return std::string(e);
  const char* h = std::getenv("HOME");
  if (!h || !*h) return std::string();
  const std::string dir = std::string(h) + "/.cache/mhc";
  mkdir((std::string(h) + "/.cache").c_str(), 0755);
  mkdir(dir.c_str(), 0755);
  return dir + "/tune.jsonl";
}

bool cache_get(const std::string& key, int* tile) {
  const std::string path = cache_path();
  if (path.empty()) return false;
  std::lock_guard<std::mutex> lock(g_cache_mutex);
  std::ifstream in(path);
  if (!in) return false;
  const std::string want = "\"key\": \"" + key + "\"";
  std::string line;
  int found = 0;
  while (std::getline(in, line)) {
    if (line.find(want) == std::string::npos) continue;
    const size_t t = line.find("\"tile\": ");
    if (t == std::string::npos) continue;
    const int v = std::atoi(line.c_str() + t + 8);
    if (v == 32 || v == 64 || v == 128) found = v;
  }
  if (found) *tile = found;
  return found != 0;
}

bool cache_put(const std::string& key, int tile, const double* ms) {
  const std::string path = cache_path();
  if (path.empty()) return false;
  std::ostringstream o;
  o << "{\"key\": \"" << key << "\", \"tile\": " << tile << ", \"ms\": [";
  for (int i = 0; i < 3; i++) o << (i ? ", " : "") << (ms ? ms[i] : 0.0);
  o << "]}\n";
  const std::string line = o.str();
  std::lock_guard<std::mutex> lock(g_cache_mutex);
  const int fd = open(path.c_str(), O_WRONLY | O_CREAT | O_APPEND, 0644);
  if (fd < 0) return false;
  const bool ok = write(fd, line.data(), line.size()) == (ssize_t)line.size();
  close(fd);
  return ok;
}

// The cache key of class c of a batch: the GPU, this build of the library, the class and
// the (n_f, L_f) signatures of its correlators.
std::string class_key(const mhc_batch_s& b, int c) {
  std::set<std::string> sig;
  for (const Plan* p : b.plans) {
    if (class_of(*p) != c) continue;
    std::ostringstream o;
    for (int f = 0; f < p->F; f++) o << (f ? "," : "") << p->n_f[f] << "/" << p->L_f[f];
    sig.insert(o.str());
  }
  if (sig.empty()) return std::string();
  cudaDeviceProp prop;
  std::string gpu = "unknown";
  if (cudaGetDeviceProperties(&prop, b.device) == cudaSuccess) {
    gpu = prop.name;
    gpu += " sm" + std::to_string(prop.multiProcessorCount);
  }
  std::ostringstream o;
  o << "gpu=" << gpu << ";build=" << __DATE__ << " " << __TIME__ << ";nc=" << kClassNc[c] << ";shapes=";
  bool first = true;
  for (const auto& x : sig) {
    o << (first ? "" : " ") << x;
    first = false;
  }
  std::string k = o.str();
  for (char& ch : k)
    if (ch == '"' || ch == '\\' || ch == '\n') ch = '_';
  return k;
}

mhc_status fill_descs(mhc_batch_s& b, const BatchShape& sh, const double* const* const* S,
                      std::vector<FwdArgs>& desc) {
  desc.resize(b.count);
  b.own_kbuf.resize(b.count, nullptr);
  b.own_kguard.resize(b.count, nullptr);
  for (int k = 0; k < b.count; k++) {
    const Plan& p = *b.plans[k];
    mhc_status st = fill_fwd_args(*b.plans[k], S[k], nullptr, nullptr, desc[k]);
    if (st != MHC_OK) return st;
    desc[k].n_tiles = sh.n_tiles[k];
    bool repeat = false;
    for (int k2 = 0; k2 < k; k2++) repeat |= b.plans[k2] == b.plans[k];
    if (repeat && desc[k].snk_orig) {
      if (!b.own_kbuf[k]) {
        const size_t nk = (size_t)p.n_fam * p.n_qfam * desc[k].kstride * sizeof(double2);
        const size_t ng = (size_t)p.n_fam * p.n_qfam * p.F * sizeof(int32_t);
        if (cudaMalloc(&b.own_kbuf[k], std::max<size_t>(nk, 16)) != cudaSuccess ||
            cudaMalloc(&b.own_kguard[k], std::max<size_t>(ng, 16)) != cudaSuccess) {
          set_error("mhc_batch: cudaMalloc failed for a repeated plan's block factors");
          return MHC_ENOMEM;
        }
      }
      desc[k].kbuf = reinterpret_cast<const double2*>(b.own_kbuf[k]);
      desc[k].kguard = reinterpret_cast<int32_t*>(b.own_kguard[k]);
    }
  }
  return MHC_OK;
}

mhc_status upload_shape(mhc_batch_s& b, const BatchShape& sh) {
  if (b.d_items) cudaFree(b.d_items);
  if (b.d_part_off) cudaFree(b.d_part_off);
  if (b.d_partials) cudaFree(b.d_partials);
  b.d_items = nullptr;
  b.d_part_off = nullptr;
  b.d_partials = nullptr;
  if (cudaMalloc(&b.d_items, std::max<size_t>(sh.items.size(), 1) * sizeof(BatchItem)) != cudaSuccess ||
      cudaMalloc(&b.d_part_off, sh.part_off.size() * sizeof(int64_t)) != cudaSuccess ||
      cudaMalloc(&b.d_partials, std::max<int64_t>(sh.part_off.back(), 1) * sizeof(double2)) != cudaSuccess) {
    set_error("mhc_batch: cudaMalloc failed");
    return MHC_ENOMEM;
  }
  if (!sh.items.empty())
    cudaMemcpy(b.d_items, sh.items.data(), sh.items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
  cudaMemcpy(b.d_part_off, sh.part_off.data(), sh.part_off.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  return MHC_OK;
}

cudaError_t launch_class(const mhc_batch_s& b, const BatchShape& sh, int c, cudaStream_t s) {
  const BatchItem* items = b.d_items + sh.cls_off[c];
  const int64_t n = sh.cls_off[c + 1] - sh.cls_off[c];
  unsigned long long* head = b.d_head + c;
  const int T = sh.T[c];
  if (c == 0)
    return launch_batch_nc8(sh.cls_grid[c], T, sh.cls_smem[c], s, b.d_desc, items, n, head, b.d_part_off,
                            b.d_partials);
  if (c == 1)
    return launch_batch_nc18(sh.cls_grid[c], T, sh.cls_smem[c], s, b.d_desc, items, n, head, b.d_part_off,
                             b.d_partials);
  return launch_batch_nc32(sh.cls_grid[c], T, sh.cls_smem[c], s, b.d_desc, items, n, head, b.d_part_off,
                           b.d_partials);
}

cudaError_t launch_kfac(const mhc_batch_s& b, const BatchShape& sh, cudaStream_t s) {
  if (sh.ncmax <= 8) return launch_kfac_batch_nc8(b.d_desc, b.d_kpref, b.d_nfam, b.count, b.k_total, b.k_big, s);
  if (sh.ncmax <= 18) return launch_kfac_batch_nc18(b.d_desc, b.d_kpref, b.d_nfam, b.count, b.k_total, b.k_big, s);
  return launch_kfac_batch_nc32(b.d_desc, b.d_kpref, b.d_nfam, b.count, b.k_total, b.k_big, s);
}

cudaError_t enqueue(mhc_batch_s& b, const BatchShape& sh, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b.d_head, 0, sizeof(unsigned long long) * kClasses, s);
  if (e != cudaSuccess) return e;
  // two-sided update: the factors of every (family, sink family) block of every
  // correlator, in one launch (two when some flavour has n > 6)
  if ((e = launch_kfac(b, sh, s)) != cudaSuccess) return e;
  // the class with the most work on s, the others on the side branch: a class's blocks
  // take the SMs that the other class's queue releases as it drains
  int main_cls = -1;
  double most = -1.0;
  for (int c = 0; c < kClasses; c++) {
    const double n = (double)(sh.cls_off[c + 1] - sh.cls_off[c]) * (double)kClassNc[c] * kClassNc[c];
    if (sh.cls_off[c + 1] > sh.cls_off[c] && n > most) {
      most = n;
      main_cls = c;
    }
  }
  bool forked = false;
  for (int c = 0; c < kClasses; c++) {
    if (c == main_cls || sh.cls_off[c + 1] == sh.cls_off[c]) continue;
    if (!forked) {
      if ((e = cudaEventRecord(b.fork, s)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(b.side, b.fork, 0)) != cudaSuccess) return e;
      forked = true;
    }
    if ((e = launch_class(b, sh, c, b.side)) != cudaSuccess) return e;
  }
  if (main_cls >= 0 && (e = launch_class(b, sh, main_cls, s)) != cudaSuccess) return e;
  if (forked) {
    if ((e = cudaEventRecord(b.join, b.side)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s, b.join, 0)) != cudaSuccess) return e;
  }
  batch_reduce<<<b.count, 256, 0, s>>>(b.d_partials, b.d_part_off, b.d_outs);
  return cudaGetLastError();
}

void destroy(mhc_batch_s* b) {
  if (!b) return;
  if (b->device >= 0) {
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
  }
  if (b->exec) cudaGraphExecDestroy(b->exec);
  void* ptrs[] = {b->d_desc, b->d_items, b->d_part_off, b->d_partials, b->d_head, b->d_outs,
                  b->d_kpref, b->d_nfam};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (void* p : b->own_kbuf)
    if (p) cudaFree(p);
  for (void* p : b->own_kguard)
    if (p) cudaFree(p);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  delete b;
}

}  // namespace

extern "C" {

mhc_status mhc_batch_create(mhc_batch_t* out, int32_t count, const mhc_plan_t* plans) {
  TraceRange trace("mhc_batch_create");
  if (!out || count <= 0 || !plans) {
    set_error("mhc_batch_create: bad argument");
    return MHC_EINVAL;
  }
  *out = nullptr;
  mhc_batch_s* b = new mhc_batch_s();
  b->count = count;
  cudaGetDevice(&b->device);
  for (int k = 0; k < count; k++) {
    if (!plans[k]) {
      delete b;
      set_error("mhc_batch_create: NULL plan");
      return MHC_EINVAL;
    }
    Plan* p = reinterpret_cast<Plan*>(plans[k]);
    mhc_status st = ensure_device(*p);
    if (st != MHC_OK) {
      delete b;
      return st;
    }
    b->plans.push_back(p);
  }
  std::vector<int64_t> kpref(1, 0), nfam;
  for (int k = 0; k < count; k++) {
    const Plan& p = *b->plans[k];
    nfam.push_back(p.n_fam);
    kpref.push_back(kpref.back() + (p.dev.two_sided ? p.n_fam * p.n_qfam * p.F : 0));
    for (int f = 0; f < p.F; f++) b->k_big |= (p.dev.two_sided && p.n_f[f] > 6) ? 1 : 0;
  }
  b->k_total = kpref.back();
  if (cudaMalloc(&b->d_kpref, sizeof(int64_t) * (count + 1)) != cudaSuccess ||
      cudaMalloc(&b->d_nfam, sizeof(int64_t) * count) != cudaSuccess) {
    destroy(b);
    set_error("mhc_batch_create: CUDA allocation failed");
    return MHC_ENOMEM;
  }
  cudaMemcpy(b->d_kpref, kpref.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_nfam, nfam.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice);
  if (cudaMalloc(&b->d_desc, sizeof(FwdArgs) * count) != cudaSuccess ||
      cudaMalloc(&b->d_head, sizeof(unsigned long long) * kClasses) != cudaSuccess ||
      cudaMalloc(&b->d_outs, sizeof(double*) * count) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming) != cudaSuccess) {
    destroy(b);
    set_error("mhc_batch_create: CUDA allocation failed");
    return MHC_ENOMEM;
  }
  // ---- the sink tile of each n class: from the tuning cache, else timed on scratch
  // propagators (each class's persistent kernel alone, after the block factors) --------
  int Tc[kClasses] = {32, 32, 32};
  bool present[kClasses] = {false, false, false}, tune[kClasses] = {false, false, false};
  std::string keys[kClasses];
  for (const Plan* p : b->plans) present[class_of(*p)] = true;
  bool any_tune = false;
  for (int c = 0; c < kClasses; c++) {
    if (!present[c]) continue;
    keys[c] = class_key(*b, c);
    if (cache_get(keys[c], &Tc[c])) {
      b->from_cache[c] = 1;
    } else {
      tune[c] = true;
      any_tune = true;
    }
  }
  mhc_status st = MHC_OK;
  if (any_tune) {
    std::vector<std::vector<double2*>> scratch(count);
    std::vector<std::vector<const double*>> sp(count);
    std::vector<const double* const*> S(count);
    double* scratch_out = nullptr;
    std::vector<double*> outs(count);
    if (cudaMalloc(&scratch_out, sizeof(double) * 2 * count) != cudaSuccess) st = MHC_ENOMEM;
    for (int k = 0; k < count && st == MHC_OK; k++) {
      const Plan& p = *b->plans[k];
      for (int f = 0; f < p.F; f++) {
        double2* sc = nullptr;
        const int L = p.L_f[f];
        if (cudaMalloc(&sc, sizeof(double2) * L * L) != cudaSuccess) {
          st = MHC_ENOMEM;
          break;
        }
        scratch_S<<<(L * L + 255) / 256, 256, 0, b->cap>>>(sc, L, 977u * k + f);
        scratch[k].push_back(sc);
        sp[k].push_back(reinterpret_cast<const double*>(sc));
      }
      S[k] = sp[k].data();
      outs[k] = scratch_out + 2 * k;
    }
    if (st == MHC_ENOMEM) set_error("mhc_batch_create: scratch allocation failed");
    if (st == MHC_OK)
      cudaMemcpy(b->d_outs, outs.data(), sizeof(double*) * count, cudaMemcpyHostToDevice);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int ti = 0; ti < 3 && st == MHC_OK; ti++) {
      int Tt[kClasses];
      for (int c = 0; c < kClasses; c++) Tt[c] = tune[c] ? kTiles[ti] : Tc[c];
      BatchShape sh = make_shape(*b, Tt);
      std::vector<FwdArgs> desc;
      if ((st = fill_descs(*b, sh, S.data(), desc)) != MHC_OK) break;
      cudaMemcpy(b->d_desc, desc.data(), sizeof(FwdArgs) * count, cudaMemcpyHostToDevice);
      b->h_desc = desc;
      if ((st = upload_shape(*b, sh)) != MHC_OK) break;
      cudaError_t e = launch_kfac(*b, sh, b->cap);
      for (int c = 0; c < kClasses && e == cudaSuccess; c++) {
        if (!tune[c]) continue;
        if (sh.cls_smem[c] > kSmemLimit) {
          b->tune_ms[c][ti] = -1.0;
          continue;
        }
        float ms = 0.f;
        for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {
          e = cudaMemsetAsync(b->d_head + c, 0, sizeof(unsigned long long), b->cap);
          if (e == cudaSuccess) e = cudaEventRecord(e0, b->cap);
          if (e == cudaSuccess) e = launch_class(*b, sh, c, b->cap);
          if (e == cudaSuccess) e = cudaEventRecord(e1, b->cap);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        }
        b->tune_ms[c][ti] = ms;
      }
      if (e != cudaSuccess) {
        set_error(std::string("mhc_batch_create: tuning launch failed: ") + cudaGetErrorString(e));
        st = MHC_ECUDA;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (auto& v : scratch)
      for (auto* x : v) cudaFree(x);
    if (scratch_out) cudaFree(scratch_out);
    for (int c = 0; c < kClasses && st == MHC_OK; c++) {
      if (!tune[c]) continue;
      int best = -1;
      for (int ti = 0; ti < 3; ti++)
        if (b->tune_ms[c][ti] > 0.0 && (best < 0 || b->tune_ms[c][ti] < b->tune_ms[c][best])) best = ti;
      if (best < 0) {
        set_error("mhc_batch_create: no launch shape fits in shared memory");
        st = MHC_EUNSUPPORTED;
        break;
      }
      Tc[c] = kTiles[best];
      cache_put(keys[c], Tc[c], b->tune_ms[c]);
    }
  }
  if (st == MHC_OK) {
    b->shape = make_shape(*b, Tc);
    st = upload_shape(*b, b->shape);
  }
  if (st != MHC_OK) {
    destroy(b);
    return st;
  }
  *out = reinterpret_cast<mhc_batch_t>(b);
  return MHC_OK;
}

void mhc_batch_destroy(mhc_batch_t batch) { destroy(reinterpret_cast<mhc_batch_s*>(batch)); }

mhc_status mhc_batch_correlator(mhc_batch_t batch, const double* const* const* S, double* const* outs,
                                mhc_stream_t stream) {
  TraceRange trace("mhc_batch_correlator");
  if (!batch || !S || !outs) {
    set_error("mhc_batch_correlator: NULL argument");
    return MHC_EINVAL;
  }
  mhc_batch_s& b = *reinterpret_cast<mhc_batch_s*>(batch);
  std::vector<const void*> key;
  for (int k = 0; k < b.count; k++) {
    if (!S[k] || !outs[k]) {
      set_error("mhc_batch_correlator: NULL propagator list or output");
      return MHC_EINVAL;
    }
    for (int f = 0; f < b.plans[k]->F; f++) key.push_back(S[k][f]);
    key.push_back(outs[k]);
  }
  if (!b.exec || key != b.key) {
    // new pointers: refresh the descriptors and capture the launch sequence once
    std::vector<FwdArgs> desc;
    mhc_status st = fill_descs(b, b.shape, S, desc);
    if (st != MHC_OK) return st;
    b.h_desc = desc;
    if (cudaStreamSynchronize(b.cap) != cudaSuccess ||
        cudaMemcpy(b.d_desc, desc.data(), sizeof(FwdArgs) * b.count, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b.d_outs, outs, sizeof(double*) * b.count, cudaMemcpyHostToDevice) != cudaSuccess) {
      set_error("mhc_batch_correlator: descriptor upload failed");
      return MHC_ECUDA;
    }
    if (b.exec) {
      cudaGraphExecDestroy(b.exec);
      b.exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b.cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e2 = enqueue(b, b.shape, b.cap);
      e = cudaStreamEndCapture(b.cap, &g);
      if (e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b.exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      set_error(std::string("mhc_batch_correlator: graph capture: ") + cudaGetErrorString(e));
      return MHC_ECUDA;
    }
    b.key = key;
  }
  cudaError_t e = cudaGraphLaunch(b.exec, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    set_error(std::string("mhc_batch_correlator: graph launch: ") + cudaGetErrorString(e));
    return MHC_ECUDA;
  }
  return MHC_OK;
}

mhc_status mhc_batch_info(mhc_batch_t batch, int32_t* threads_per_block, int32_t* tiles_total) {
  if (!batch) {
    set_error("mhc_batch_info: NULL batch");
    return MHC_EINVAL;
  }
  const mhc_batch_s& b = *reinterpret_cast<const mhc_batch_s*>(batch);
  int main_cls = 0;  // the class with the most work items
  for (int c = 1; c < kClasses; c++)
    if (b.shape.cls_off[c + 1] - b.shape.cls_off[c] > b.shape.cls_off[main_cls + 1] - b.shape.cls_off[main_cls])
      main_cls = c;
  if (threads_per_block) *threads_per_block = b.shape.T[main_cls];
  if (tiles_total) *tiles_total = (int32_t)b.shape.n_items;
  return MHC_OK;
}

mhc_status mhc_batch_shape(mhc_batch_t batch, int32_t* tiles, int32_t* from_cache, double* tune_ms) {
  if (!batch || !tiles) {
    set_error("mhc_batch_shape: NULL batch or tiles");
    return MHC_EINVAL;
  }
  const mhc_batch_s& b = *reinterpret_cast<const mhc_batch_s*>(batch);
  for (int c = 0; c < kClasses; c++) {
    const bool used = b.shape.cls_off[c + 1] > b.shape.cls_off[c];
    tiles[c] = used ? b.shape.T[c] : 0;
    if (from_cache) from_cache[c] = used ? b.from_cache[c] : 0;
    if (tune_ms)
      for (int t = 0; t < 3; t++) tune_ms[3 * c + t] = b.tune_ms[c][t];
  }
  return MHC_OK;
}

mhc_status mhc_tune_cache_get(const char* key, int32_t* tile) {
  if (!key || !tile) {
    set_error("mhc_tune_cache_get: NULL argument");
    return MHC_EINVAL;
  }
  int t = 0;
  *tile = cache_get(key, &t) ? t : 0;
  return MHC_OK;
}

mhc_status mhc_tune_cache_put(const char* key, int32_t tile) {
  if (!key || !*key || !(tile == 32 || tile == 64 || tile == 128) || std::strchr(key, '"') ||
      std::strchr(key, '\\') || std::strchr(key, '\n')) {
    set_error("mhc_tune_cache_put: key must be non-empty without quotes, backslashes or newlines; "
              "tile 32, 64 or 128");
    return MHC_EINVAL;
  }
  if (!cache_put(key, tile, nullptr)) {
    set_error("mhc_tune_cache_put: the cache file is disabled (MHC_TUNE_CACHE empty) or not writable");
    return MHC_EINVAL;
  }
  return MHC_OK;
}

}  // extern "C"
