// noalloc.cu -- mhc_correlator_noalloc: the forward correlator without any device
// allocation by the call.
//
// The forward kernel needs one scratch slot per work item for its partial sums.  The
// ordinary entry point keeps that scratch in a buffer the plan allocates with cudaMalloc.
// Some callers cannot have the library allocate: for example a serving process whose
// device memory is entirely reserved up front by its own pool allocator (a cudaMalloc can
// then fail, or fragment what the pool expects to own), or a latency-critical loop that
// must not pay for an allocation (cudaMalloc and cudaFree may synchronise the device).
// For them this entry point keeps the scratch in a fixed-size array that lives in the
// library's own device memory for as long as the library is loaded.
#include <mutex>
#include <string>

#include "kernels.cuh"
#include "plan.h"

namespace mhc {

// The partial sums of at most this many work items fit in the array (1 MiB).
constexpr int64_t kNoAllocMaxItems = MHC_NOALLOC_MAX_ITEMS;

namespace {

// Scratch of the allocation-free forward call.  Every GPU that loads the library holds
// one copy until the process exits.  Every call on a device shares it.
static __device__ __align__(256) double2 g_noalloc_partials[kNoAllocMaxItems];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double2* g_scratch_ptr[kMaxDevices] = {nullptr};  // device address of the array, per device

// Host code cannot use g_noalloc_partials directly: on the host that name denotes a
// host-side stand-in, not device memory.  Look up its device address once per device,
// with that device current.
mhc_status scratch_for_current_device(double2** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error(std::string("mhc_correlator_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    return MHC_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("mhc_correlator_noalloc: device ordinal beyond the supported 64");
    return MHC_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
    if (e != cudaSuccess || !ptr) {
      set_error(std::string("mhc_correlator_noalloc: cudaGetSymbolAddress: ") +
                cudaGetErrorString(e));
      return MHC_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double2*>(ptr);
  }
  *out = g_scratch_ptr[dev];
  return MHC_OK;
}

}  // namespace

int plan_ncmax(const Plan& p);
mhc_status fill_fwd_args(Plan& p, const double* const* S_f, const double* w_src,
                         const double* w_snk, FwdArgs& a);

}  // namespace mhc

using namespace mhc;

extern "C" mhc_status mhc_correlator_noalloc(mhc_plan_t plan, const double* const* S_f,
                                             const double* w_src_dev, const double* w_snk_dev,
                                             double* out_dev, mhc_stream_t stream) {
  if (!plan || !out_dev) {
    set_error("mhc_correlator_noalloc: NULL plan or output");
    return MHC_EINVAL;
  }
  Plan& p = *reinterpret_cast<Plan*>(plan);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || p.dev.device != dev) {
    set_error("mhc_correlator_noalloc: the plan's tables are not on the current device yet; "
              "call mhc_correlator once with this plan on this device first (that call "
              "allocates and uploads them)");
    return MHC_EINVAL;
  }
  // the launch shape the upload fixed (the same one mhc_correlator launches with)
  const int tile = p.dev.tile;
  const int64_t items = p.dev.n_items;
  if (items > kNoAllocMaxItems) {
    set_error("mhc_correlator_noalloc: the plan has " + std::to_string(items) +
              " work items (families x sink tiles); the fixed scratch holds at most " +
              std::to_string(kNoAllocMaxItems) + ". Use mhc_correlator for this plan.");
    return MHC_EINVAL;
  }
  double2* scratch = nullptr;
  mhc_status st = scratch_for_current_device(&scratch);
  if (st != MHC_OK) return st;
  FwdArgs a;
  if ((st = fill_fwd_args(p, S_f, w_src_dev, w_snk_dev, a)) != MHC_OK) return st;
  // Every work item writes its own slot before the reduction reads it, so the array
  // needs no clearing between calls.
  a.partials = scratch;
  const size_t smem = forward_smem_bytes(a.slots, tile);
  cudaError_t e = launch_forward(a, plan_ncmax(p), tile, p.n_fam, items, smem, out_dev,
                                 reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    set_error(std::string("mhc_correlator_noalloc: launch: ") + cudaGetErrorString(e));
    return MHC_ECUDA;
  }
  return MHC_OK;
}
