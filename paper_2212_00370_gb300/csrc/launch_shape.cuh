// launch_shape.cuh -- how the faces and cells kernels spread their work items
// over threads (the shapes the autotuner chooses among).  Integer logic only.
//
//  grid schedule (block BS, PT items per thread): block b covers items
//    [b*BS*PT, (b+1)*BS*PT); thread t of the block takes b*BS*PT + j*BS + t for
//    j < PT, so the threads of a warp always read consecutive items;
//  persistent schedule: a resident grid (SMs x resident blocks per SM); every
//    warp takes chunks of 32 consecutive items from a device counter until none
//    are left, so warps that met cheap items take more chunks.  The counter is
//    zeroed on the stream before the launch.
// Every item is processed exactly once either way, so results do not depend on
// the shape.
#pragma once
#include <cstdint>

namespace rr {

template <int BS, int PT, class F>
__device__ __forceinline__ void grid_items(int64_t n, F&& f) {
  const int64_t base = (int64_t)blockIdx.x * (BS * PT) + threadIdx.x;
#pragma unroll
  for (int j = 0; j < PT; ++j) {
    const int64_t t = base + (int64_t)j * BS;
    if (t < n) f(t);
  }
}

template <class F>
__device__ __forceinline__ void persistent_items(int64_t n, unsigned long long* counter, F&& f) {
  const int lane = threadIdx.x & 31;
  while (true) {
    unsigned long long base = 0;
    __syncwarp();
    if (lane == 0) base = atomicAdd(counter, 32ull);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= (unsigned long long)n) break;
    const int64_t t = (int64_t)base + lane;
    if (t < n) f(t);
  }
}

// The shapes that are compiled: block size x items per thread (grid schedule) and
// block size (persistent schedule).
// Blocks of 8 and 16 threads (grid schedule, one item per thread) spread a small
// grid over more SMs with partial warps.
#define RR_GRID_SHAPES(X) \
  X(8, 1) X(16, 1) X(32, 1) X(32, 2) X(64, 1) X(64, 2) X(128, 1) X(128, 2) X(256, 1) X(256, 2)
#define RR_PERSISTENT_BLOCKS(X) X(32) X(64) X(128) X(256)

inline bool shape_ok(int block, int per_thread, int persistent) {
  const bool bs = block == 32 || block == 64 || block == 128 || block == 256;
  if (persistent) return bs && per_thread == 1 && persistent == 1;
  if (block == 8 || block == 16) return per_thread == 1 && persistent == 0;
  return bs && (per_thread == 1 || per_thread == 2) && persistent == 0;
}

}  // namespace rr
