// probe.cu -- FP64 peak probe: independent DFMA chains on every SM, timed with CUDA events.
// It states the roofline denominator on the same GPU, at the same clocks, as the kernels
// it is compared with.
#include <string>

#include "kernels.cuh"
#include "plan.h"

namespace mhc {
namespace {

__global__ void __launch_bounds__(256) dfma_chains(double* out, int iters, double b, double c) {
  double a[8];
#pragma unroll
  for (int i = 0; i < 8; i++) a[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < 8; i++) a[i] = fma(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; i++) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The complex reciprocal every pivot of the factorisations uses (dev::crcp), elementwise.
__global__ void crcp_kernel(int64_t n, const double2* __restrict__ z, double2* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = dev::crcp(z[i]);
}

}  // namespace
}  // namespace mhc

using namespace mhc;

extern "C" mhc_status mhc_complex_reciprocal(int64_t n, const double* z_dev, double* out_dev,
                                             mhc_stream_t stream) {
  if (n < 0 || (n > 0 && (!z_dev || !out_dev))) {
    set_error("mhc_complex_reciprocal: bad argument");
    return MHC_EINVAL;
  }
  if (n == 0) return MHC_OK;
  crcp_kernel<<<(unsigned)((n + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      n, reinterpret_cast<const double2*>(z_dev), reinterpret_cast<double2*>(out_dev));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("mhc_complex_reciprocal: ") + cudaGetErrorString(e));
    return MHC_ECUDA;
  }
  return MHC_OK;
}

extern "C" mhc_status mhc_fp64_peak(int32_t iters, double* flops, mhc_stream_t stream) {
  if (iters <= 0 || !flops) {
    set_error("mhc_fp64_peak: bad argument");
    return MHC_EINVAL;
  }
  int dev = 0, sms = 0;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    set_error("mhc_fp64_peak: no CUDA device");
    return MHC_ECUDA;
  }
  const int blocks = sms * 2, threads = 256;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) {
    set_error("mhc_fp64_peak: cudaMalloc failed");
    return MHC_ENOMEM;
  }
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  dfma_chains<<<blocks, threads, 0, s>>>(out, 16, 0.999, 1e-3);
  cudaEventRecord(e0, s);
  dfma_chains<<<blocks, threads, 0, s>>>(out, iters, 0.999, 1e-3);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) {
    set_error(std::string("mhc_fp64_peak: ") + cudaGetErrorString(e));
    return MHC_ECUDA;
  }
  *flops = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3);
  return MHC_OK;
}
