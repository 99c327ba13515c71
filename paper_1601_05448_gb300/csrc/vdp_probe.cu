// vdp_probe.cu -- vdp_probe_fp64: the FP64 FMA throughput of the current GPU, measured.
//
// The FP64 stencil sweeps of the solver are bound by the FP64 pipe, not by HBM, so their roofline
// needs the pipe's peak.  This probe measures it with the instruction those sweeps spend their
// time on: every thread advances kChains independent FMA chains a = a * b + c (independent so the
// pipe, not the FMA latency, sets the rate) for `iters` steps, over a grid of 8 blocks of 256
// threads per SM; CUDA events on the caller's stream time the launch.  FLOPs = 2 per FMA.
#include <cuda_runtime.h>

#include "vdp.h"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;

__device__ double g_probe_sink;  // keeps the chains alive; written only on an impossible value

__global__ void __launch_bounds__(kThreads) k_probe_fp64(int iters, double b, double c) {
  double a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = 1.0 + 1e-3 * (threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == -1.0) g_probe_sink = s;  // never true for |b| < 1, c > 0: the stores stay out
}

}  // namespace

extern "C" int vdp_probe_fp64(void* stream, double* tflops) {
  if (!tflops) return VDP_EINVAL;
  *tflops = 0.0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return VDP_ECUDA;
  const int blocks = 8 * sms, iters = 2048;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return VDP_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return VDP_ECUDA;
  }
  float best = 0.f;
  int status = VDP_OK;
  for (int rep = 0; rep < 4 && status == VDP_OK; ++rep) {  // the first launch warms up
    cudaEventRecord(e0, s);
    k_probe_fp64<<<blocks, kThreads, 0, s>>>(iters, 0.999999, 1e-6);
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        cudaGetLastError() != cudaSuccess) {
      status = VDP_ECUDA;
      break;
    }
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != VDP_OK || best <= 0.f) return status == VDP_OK ? VDP_ECUDA : status;
  const double flops = 2.0 * kChains * (double)iters * blocks * kThreads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return VDP_OK;
}
