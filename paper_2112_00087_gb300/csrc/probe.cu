// Measurement aid: the device's FP64 fused multiply-add rate, timed with CUDA events. On GB300
// the FP64 pipe, not HBM, bounds the complex double-precision products (a complex multiply-add
// is four FP64 FMAs), so the rooflines of the FP64 kernels are quoted against this measured rate.
//
// Every thread runs 8 independent FMA chains a_k <- a_k * m + c (|m| < 1, so the values stay
// bounded) for `iters` steps; the grid holds 16 blocks of 256 threads per SM, enough resident
// warps to cover the pipe's latency. The chains' sum is stored so nothing is optimised away.
#include <cuda_runtime.h>

#include "common.cuh"

namespace helm {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 16;
constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(kProbeThreads) fp64_fma_probe(double* out, int iters, double m, double c) {
  double a[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = 1e-3 * (threadIdx.x + 1) + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += a[k];
  out[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

}  // namespace
}  // namespace helm

extern "C" helm_status helm_probe_fp64_fma(int32_t iters, double* fma_per_s, void* stream) {
  using namespace helm;
  if (iters <= 0 || !fma_per_s) return set_error(HELM_ERR_ARG, "helm_probe_fp64_fma: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 1;
  HELM_CUDA(cudaGetDevice(&dev));
  HELM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = nsm * kProbeBlocksPerSm;
  double* out = nullptr;
  helm_status st = dev_alloc(&out, (size_t)blocks * kProbeThreads);
  if (st != HELM_OK) return st;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fp64_fma_probe<<<blocks, kProbeThreads, 0, s>>>(out, 16, 0.999999, 1e-7);  // warm-up
  cudaEventRecord(e0, s);
  fp64_fma_probe<<<blocks, kProbeThreads, 0, s>>>(out, iters, 0.999999, 1e-7);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return cuda_error(e, "helm_probe_fp64_fma");
  *fma_per_s = (double)blocks * kProbeThreads * (double)iters * kProbeChains / (ms * 1e-3);
  return HELM_OK;
}
