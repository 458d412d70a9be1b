// rrmhd_probe.cu -- throughput probe of the FP64 pipe.
//
// The path's cell and face kernels are bound by the FP64 pipe (no dense
// contraction, and HBM under 1 % busy), so their roofline denominator is the rate
// at which this GPU retires FP64 instructions.  This probe measures it: every
// thread runs eight independent chains of DFMA (so the pipe, not the ~latency of
// one chain, is the limit), 64 warps per SM on every SM, timed with CUDA events on
// the caller's stream.  The count is thread-level FP64 instructions, the unit of
// the ncu counters sm__sass_thread_inst_executed_op_d{add,mul,fma}.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/rrmhd.h"

namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;   // 2048 threads per SM
constexpr int kChains = 8;
constexpr int kUnroll = 16;       // DFMA per chain per loop trip

__device__ double g_fp64_probe_sink;

__global__ void __launch_bounds__(kThreads, kBlocksPerSM) k_fp64_probe(int iters, double seed) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = seed + (double)(threadIdx.x + k);
  const double m = 0.9999999999, c = 1e-12;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < kUnroll; ++r)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = __fma_rn(a[k], m, c);
  }
  double t = a[0];
#pragma unroll
  for (int k = 1; k < kChains; ++k) t = __dadd_rn(t, a[k]);
  if (t == -1.0) g_fp64_probe_sink = t;  // never true; keeps the chains live
}

// One warp, one dependent DFMA chain per thread: the latency of a dependent FP64
// instruction when nothing else hides it (the regime of a grid too small to fill the SMs).
__global__ void __launch_bounds__(32) k_fp64_latency(int iters, double seed) {
  double a = seed + (double)threadIdx.x;
  const double m = 0.9999999999, c = 1e-12;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < kUnroll; ++r) a = __fma_rn(a, m, c);
  }
  if (a == -1.0) g_fp64_probe_sink = a;
}

// Runs the probe with `iters` trips; returns its duration in ms (or -1 on error).
float timed(cudaStream_t s, int blocks, int iters) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1.f;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return -1.f;
  }
  float ms = -1.f;
  cudaEventRecord(e0, s);
  k_fp64_probe<<<blocks, kThreads, 0, s>>>(iters, 1.0);
  cudaEventRecord(e1, s);
  if (cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess)
    cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

}  // namespace

extern "C" rrmhd_status rrmhd_probe_fp64(void* cuda_stream, double target_ms, double* inst_per_s) {
  if (!inst_per_s || !(target_ms > 0.0) || target_ms > 10000.0) return RRMHD_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return RRMHD_ECUDA;
  const int blocks = sms * kBlocksPerSM;
  // calibrate: a short run (also the warm-up), then scale the trip count to target_ms
  const int calib = 64;
  const float ms0 = timed(s, blocks, calib);
  if (!(ms0 > 0.f)) return RRMHD_ECUDA;
  const double scale = target_ms / ms0;
  const int iters = (int)std::min(1.0e7, std::max((double)calib, calib * scale));
  double best = 0.0;
  for (int r = 0; r < 3; ++r) {
    const float ms = timed(s, blocks, iters);
    if (!(ms > 0.f)) return RRMHD_ECUDA;
    const double inst = (double)blocks * kThreads * ((double)iters * kChains * kUnroll + (kChains - 1));
    best = std::max(best, inst / (ms * 1e-3));
  }
  *inst_per_s = best;
  return RRMHD_OK;
}

extern "C" rrmhd_status rrmhd_probe_fp64_latency(void* cuda_stream, double* ns_per_inst) {
  if (!ns_per_inst) return RRMHD_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int iters = 4096;  // 65536 dependent DFMA per thread
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return RRMHD_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return RRMHD_ECUDA;
  }
  float best = -1.f;
  rrmhd_status rc = RRMHD_OK;
  for (int r = 0; r < 3 && rc == RRMHD_OK; ++r) {
    cudaEventRecord(e0, s);
    k_fp64_latency<<<1, 32, 0, s>>>(iters, 1.0);
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      rc = RRMHD_ECUDA;
    else if (best < 0.f || ms < best)
      best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != RRMHD_OK) return rc;
  *ns_per_inst = (double)best * 1e6 / ((double)iters * kUnroll);
  return RRMHD_OK;
}
