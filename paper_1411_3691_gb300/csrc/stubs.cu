// stubs.cu -- entry points not built yet.
#include "plan.h"

using namespace mhc;

extern "C" {
mhc_status mhc_batch_create(mhc_batch_t* out, int32_t, const mhc_plan_t*) {
  if (out) *out = nullptr;
  set_error("mhc_batch_create: not built yet");
  return MHC_EUNSUPPORTED;
}
void mhc_batch_destroy(mhc_batch_t) {}
mhc_status mhc_batch_correlator(mhc_batch_t, const double* const* const*, double* const*, mhc_stream_t) {
  set_error("mhc_batch_correlator: not built yet");
  return MHC_EUNSUPPORTED;
}
mhc_status mhc_batch_info(mhc_batch_t, int32_t*, int32_t*) {
  set_error("mhc_batch_info: not built yet");
  return MHC_EUNSUPPORTED;
}
}
