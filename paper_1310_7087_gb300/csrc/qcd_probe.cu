// qcd_probe.cu -- measured FP64 arithmetic rate of the current GPU.
//
// The FP64-plain sweep is bound by the FP64 pipe, not by memory, so its
// roofline needs the device's FP64 fused multiply-add rate.  This kernel
// measures it: every thread runs eight independent FMA chains (enough to
// cover the pipe's latency), the grid fills every SM several times over, and
// CUDA events time the launch.  It changes no clock or device setting.
#include "qcd.h"
#include "qcd_internal.h"

#include <algorithm>
#include <cstdio>

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;
constexpr int kThreads = 256;

// Receives the chains' sums when a (never met) condition holds, so the
// compiler must keep the chains.
__device__ double g_probe_sink;

// x <- x * m + c with |m| < 1 keeps every chain bounded (it tends to
// c / (1 - m) = 1); the sum is compared with a value it cannot reach.
__global__ void __launch_bounds__(kThreads) fp64_fma_kernel(double m, double c, double never) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = double(threadIdx.x + k) * 1e-3;
#pragma unroll 1
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == never) g_probe_sink = s;
}

}  // namespace

extern "C" int qcd_probe_fp64_rate(double* flops_per_s, void* stream) {
  if (!flops_per_s) return qcd::set_last_error(QCD_ERR_INVALID_ARG, "flops_per_s is null");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp64_fma_kernel, kThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    return qcd::set_last_error(QCD_ERR_CUDA, "device query for the FP64 probe failed");
  }
  const int blocks = sms * std::max(1, per_sm) * 4;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return qcd::set_last_error(QCD_ERR_CUDA, "cudaEventCreate failed");
  }
  float best = 1e30f;
  cudaError_t err = cudaSuccess;
  for (int rep = 0; rep < 6 && err == cudaSuccess; ++rep) {  // first launch is a warm-up
    cudaEventRecord(e0, st);
    fp64_fma_kernel<<<blocks, kThreads, 0, st>>>(0.999999, 1e-6, -1.0);
    cudaEventRecord(e1, st);
    err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    float ms = 0.f;
    if (err == cudaSuccess && rep > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess)
    return qcd::set_last_error(QCD_ERR_CUDA, cudaGetErrorString(err));
  const double flops = 2.0 * kChains * double(kIters) * double(blocks) * kThreads;
  *flops_per_s = flops / (double(best) * 1e-3);
  return QCD_OK;
}
