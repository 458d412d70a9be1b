// rrmhd_noalloc.cu -- CFL time step of one grid without any device allocation.
//
// For callers that cannot allocate device memory on their own: a host program
// whose GPU memory is owned by its own pool or fixed arena, reserved at start-up,
// cannot let a library call cudaMalloc behind its back.  Such callers pass their
// inputs and outputs; the reduction's scratch lives in a fixed array that is
// part of this library's image on every GPU that loads it, until the process
// exits.
//
// Same arithmetic as the context path (k_signal + k_begin_step): per cell
// s = sum_d lambda_d / dx_d, dt = cfl / max s, with the FP64 order of
// physics_f64.cuh (--fmad=false), so both return the same bits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/rrmhd.h"
#include "physics_f64.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kCellsPerThread = 32;
constexpr int kMaxBlocks = RRMHD_NOALLOC_MAX_CELLS / (kThreads * kCellsPerThread);
static_assert((long long)kMaxBlocks * kThreads * kCellsPerThread == RRMHD_NOALLOC_MAX_CELLS,
              "capacity must be a whole number of blocks");

// Scratch shared by every call on a device: one partial maximum per block and the
// arrival counter of the last-block reduction (the counter must start at zero).
struct Scratch {
  double partial[kMaxBlocks];
  unsigned int arrived;
};
static __device__ __align__(256) Scratch g_cfl_scratch;

constexpr int kMaxDevices = 64;
Scratch* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu[kMaxDevices];

// Device address of g_cfl_scratch on the current device.  The first successful
// lookup is kept for the life of the process; a failed one (for instance a first
// call made during stream capture) is not, and the next call looks it up again.
cudaError_t scratch_on_current_device(Scratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu[dev]);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_cfl_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<Scratch*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

struct GridArgs {
  int ndim;
  double dx[3];
  int64_t ncells;
};

__device__ __forceinline__ double cell_speed_sum(const rr::Params& P, const GridArgs& g,
                                                 const double* __restrict__ V, int64_t c) {
  double v[rr::NV];
#pragma unroll
  for (int k = 0; k < rr::NV; ++k) v[k] = V[k * g.ncells + c];
  double s = rr::signal_speed(P, 0, v) / g.dx[0];
  for (int d = 1; d < g.ndim; ++d) s = s + rr::signal_speed(P, d, v) / g.dx[d];
  return s;
}

// A NaN speed wins the maximum (the context path fails such a step as well).
__device__ __forceinline__ double max_nan(double a, double b) {
  if (a != a) return a;
  if (b != b) return b;
  return a > b ? a : b;
}

// One launch: every block reduces its cells into partial[block]; the block that
// arrives last reduces the partials, writes dt = cfl / max and resets the counter.
__global__ void __launch_bounds__(kThreads) k_cfl_noalloc(rr::Params P, GridArgs g,
                                                          const double* __restrict__ V,
                                                          double* dt_out, Scratch* scr) {
  __shared__ double red[kThreads];
  __shared__ bool last;
  double m = 0.0;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  for (int64_t c = (int64_t)blockIdx.x * kThreads + threadIdx.x; c < g.ncells; c += stride)
    m = max_nan(m, cell_speed_sum(P, g, V, c));
  red[threadIdx.x] = m;
  __syncthreads();
  for (int h = kThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] = max_nan(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    scr->partial[blockIdx.x] = red[0];
    __threadfence();
    last = (atomicAdd(&scr->arrived, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double mm = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kThreads)
    mm = max_nan(mm, ((volatile double*)scr->partial)[b]);
  red[threadIdx.x] = mm;
  __syncthreads();
  for (int h = kThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] = max_nan(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *dt_out = P.cfl / red[0];
    scr->arrived = 0u;
  }
}

}  // namespace

extern "C" rrmhd_status rrmhd_cfl_dt_noalloc(const rrmhd_grid* grid, const rrmhd_opts* opts,
                                             const double* V, double* dt, void* cuda_stream) {
  if (!grid || !opts || !V || !dt) return RRMHD_EINVAL;
  const rrmhd_grid& gr = *grid;
  if (gr.ndim < 1 || gr.ndim > 3 || !(opts->gamma > 1.0) || !(opts->cfl > 0.0)) return RRMHD_EINVAL;
  int64_t n = 1;
  for (int d = 0; d < 3; ++d) {
    if (gr.n[d] < 1 || (d >= gr.ndim && gr.n[d] != 1)) return RRMHD_EINVAL;
    if (d < gr.ndim && !(gr.dx[d] > 0.0)) return RRMHD_EINVAL;
    n *= gr.n[d];
  }
  if (n > RRMHD_NOALLOC_MAX_CELLS) return RRMHD_ECAPACITY;

  Scratch* scr = nullptr;
  if (scratch_on_current_device(&scr) != cudaSuccess) return RRMHD_ECUDA;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // start from a zero arrival counter whatever an earlier call left behind
  if (cudaMemsetAsync(&scr->arrived, 0, sizeof(unsigned int), s) != cudaSuccess) return RRMHD_ECUDA;

  rr::Params P{};
  P.gamma = opts->gamma;
  P.cfl = opts->cfl;
  P.gfac = opts->gamma / (opts->gamma - 1.0);
  P.gm1g = (opts->gamma - 1.0) / opts->gamma;
  GridArgs g;
  g.ndim = gr.ndim;
  g.ncells = n;
  for (int d = 0; d < 3; ++d) g.dx[d] = d < gr.ndim ? gr.dx[d] : 1.0;
  const int64_t per_block = (int64_t)kThreads * kCellsPerThread;
  const int blocks = (int)((n + per_block - 1) / per_block);
  k_cfl_noalloc<<<blocks, kThreads, 0, s>>>(P, g, V, dt, scr);
  return cudaGetLastError() == cudaSuccess ? RRMHD_OK : RRMHD_ECUDA;
}
