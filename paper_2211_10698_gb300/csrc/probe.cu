// The FP64 fused multiply-add rate of the GPU, measured: the denominator of the roofline of the
// FP64-bound kernels (the Poisson PCG iterations are bound by the FP64 pipe, not by memory).
// Eight independent FMA chains per thread keep the pipe fed; the result is only stored when a
// value no chain reaches appears, so the compiler keeps every FMA.
#include "ccm_host.h"

namespace {

__global__ void __launch_bounds__(256) k_fp64_fma(double* out, int iters, double b, double c) {
  double a[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) a[q] = 1e-3 * (threadIdx.x + q);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = fma(a[q], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += a[q];
  if (s == -1.0) out[0] = s;
}

}  // namespace

extern "C" ccm_status ccm_measure_fp64_rate(double* tflops) {
  ccm::set_last_error("");
  if (!tflops) {
    ccm::set_last_error("null argument");
    return CCM_E_INVALID;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = 4 * sms, threads = 256, iters = 4096;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.0f;
  for (int run = 0; run < 4 && e == cudaSuccess; ++run) {
    cudaEventRecord(e0);
    k_fp64_fma<<<blocks, threads>>>(out, iters, 0.999999999, 1e-12);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (run > 0 && (best == 0.0f || ms < best)) best = ms;  // the first run warms up
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (e != cudaSuccess || best <= 0.0f) {
    ccm::set_last_error(std::string("fp64 rate probe: ") + cudaGetErrorString(e));
    return CCM_E_CUDA;
  }
  *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
  return CCM_OK;
}
