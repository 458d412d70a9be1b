// batch_index.cuh -- integer index helpers of the packed batch layout (batch.h),
// shared by the FP64 and FP32-bulk kernels.  No floating-point arithmetic.
#pragma once
#include "batch.h"

namespace rr {
namespace idx {

// largest i in [lo, hi) with off[i] <= g  (off non-decreasing, off[lo] <= g)
static __device__ __forceinline__ int find_inst(const int64_t* off, int lo, int hi, int64_t g) {
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= g)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

static __device__ __forceinline__ int map_idx(int c, int n, int bc) {
  if (bc == 1) {
    const int m = c % n;
    return m < 0 ? m + n : m;
  }
  return c < 0 ? 0 : (c >= n ? n - 1 : c);
}

static __device__ __forceinline__ void load12(const double* __restrict__ A, int64_t stride, int64_t c,
                                       double* x) {
#pragma unroll
  for (int k = 0; k < NV; ++k) x[k] = __ldg(A + k * stride + c);
}

// Warp-level maximum of the CFL signal-speed bits onto the instances' smax words.
// Every lane of the warp calls it (inst = -1 for a lane with nothing to add); blocks
// are whole warps.  Cells of an instance are contiguous, so lanes with the same inst
// form runs: a segmented max over each run reaches its first lane, which issues the
// run's one atomicMax.  The bits of non-negative doubles order like their values
// (a NaN above every number), and a maximum does not depend on the order it is
// taken in, so smax ends as with one atomicMax per cell.
static __device__ __forceinline__ void warp_smax(unsigned long long* smax, int inst,
                                                 unsigned long long v) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long ov = __shfl_down_sync(full, v, off);
    const int oi = __shfl_down_sync(full, inst, off);
    if (lane + off < 32 && oi == inst && ov > v) v = ov;
  }
  const int pi = __shfl_up_sync(full, inst, 1);
  if (inst >= 0 && (lane == 0 || pi != inst)) atomicMax(smax + inst, v);
}

static __device__ __forceinline__ bool inst_active(const Batch& b, int i) {
  return b.st.status[i] == 0 && b.st.dt[i] > 0.0;
}

static __device__ __forceinline__ int64_t lane_faces(const Batch& b) {
  return b.f_count[0] + b.f_count[1] + b.f_count[2];
}

// Global face index of the t-th face of the launch's face ranges.
static __device__ __forceinline__ int64_t lane_face(const Batch& b, int64_t t) {
  if (t < b.f_count[0]) return b.f_begin[0] + t;
  t -= b.f_count[0];
  if (t < b.f_count[1]) return b.f_begin[1] + t;
  return b.f_begin[2] + (t - b.f_count[1]);
}

struct FacePos {
  int d, i, pos[3];
  InstDesc I;
};

static __device__ __forceinline__ FacePos face_pos(const Batch& b, int64_t g) {
  FacePos q;
  q.d = (g >= b.dir_base[2]) ? 2 : (g >= b.dir_base[1] ? 1 : 0);
  const int64_t gl = g - b.dir_base[q.d];
  const int64_t* off = b.face_off + (int64_t)q.d * (b.n_inst + 1);
  q.i = find_inst(off, b.i_begin, b.i_end, gl);
  q.I = b.inst[q.i];
  const int64_t lf = gl - off[q.i];
  const int m0 = q.I.n[0] + (q.d == 0);
  const int m1 = q.I.n[1] + (q.d == 1);
  q.pos[0] = (int)(lf % m0);
  const int64_t r = lf / m0;
  q.pos[1] = (int)(r % m1);
  q.pos[2] = (int)(r / m1);
  return q;
}

// Edge t of the launch's edge ranges (constrained transport): direction e,
// instance, position (edge dims m_d = n_d + 1 for d != e, d < ndim).
struct EdgePos {
  int e, i, pos[3];
  int64_t g;  // global edge index
  InstDesc I;
};

static __device__ __forceinline__ int64_t lane_edges(const Batch& b) {
  return b.e_count[0] + b.e_count[1] + b.e_count[2];
}

static __device__ __forceinline__ EdgePos edge_pos(const Batch& b, int64_t t) {
  EdgePos q;
  q.e = 0;
  while (q.e < 2 && t >= b.e_count[q.e]) {
    t -= b.e_count[q.e];
    ++q.e;
  }
  q.g = b.e_begin[q.e] + t;
  const int64_t g = q.g - b.edge_base[q.e];
  const int64_t* off = b.edge_off + (int64_t)q.e * (b.n_inst + 1);
  q.i = find_inst(off, b.i_begin, b.i_end, g);
  q.I = b.inst[q.i];
  const int64_t le = g - off[q.i];
  int m[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) m[d] = q.I.n[d] + ((d != q.e && d < q.I.ndim) ? 1 : 0);
  q.pos[0] = (int)(le % m[0]);
  const int64_t r = le / m[0];
  q.pos[1] = (int)(r % m[1]);
  q.pos[2] = (int)(r / m[1]);
  return q;
}

// Global index of the face of direction d at p (p[d] the face index along d, the
// other entries cell indices mapped through the boundaries).
static __device__ __forceinline__ int64_t face_gidx(const Batch& b, const InstDesc& I, int d,
                                                   const int p[3]) {
  int q[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) q[e] = (e == d) ? p[e] : map_idx(p[e], I.n[e], I.bc[e]);
  const int m0 = I.n[0] + (d == 0), m1 = I.n[1] + (d == 1);
  return b.dir_base[d] + I.face_off[d] + ((int64_t)q[2] * m1 + q[1]) * m0 + q[0];
}

// Global index of the cell at p (mapped through the boundaries).
static __device__ __forceinline__ int64_t cell_gidx(const InstDesc& I, const int p[3]) {
  int q[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) q[e] = map_idx(p[e], I.n[e], I.bc[e]);
  return I.cell_off + ((int64_t)q[2] * I.n[1] + q[1]) * I.n[0] + q[0];
}

// Whether instance I has edges along e (constrained transport).
static __device__ __forceinline__ bool has_edges(const InstDesc& I, int e) {
  return I.ndim == 3 || (I.ndim == 2 && e == 2);
}

// Global index of the edge along e at q (edge dims n_d + 1 for d != e, d < ndim).
static __device__ __forceinline__ int64_t edge_gidx(const Batch& b, const InstDesc& I, int e,
                                                   const int q[3]) {
  int m[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) m[d] = I.n[d] + ((d != e && d < I.ndim) ? 1 : 0);
  return b.edge_base[e] + I.edge_off[e] + ((int64_t)q[2] * m[1] + q[1]) * m[0] + q[0];
}

struct CellPos {
  int i;       // instance
  int p[3];    // position in the instance's grid
  InstDesc I;
};

static __device__ __forceinline__ CellPos cell_pos(const Batch& b, int64_t c) {
  CellPos q;
  q.i = find_inst(b.cell_off, b.i_begin, b.i_end, c);
  q.I = b.inst[q.i];
  const int64_t lc = c - q.I.cell_off;
  q.p[0] = (int)(lc % q.I.n[0]);
  const int64_t r = lc / q.I.n[0];
  q.p[1] = (int)(r % q.I.n[1]);
  q.p[2] = (int)(r / q.I.n[1]);
  return q;
}


}  // namespace idx
}  // namespace rr
