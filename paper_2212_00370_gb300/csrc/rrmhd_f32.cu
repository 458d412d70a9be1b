// rrmhd_f32.cu -- kernels of the FP32-bulk form of one IMEX-RK3 stage.
//
// Faces (PLM, fluxes, PVM-int-8 with tangent products, the Rusanov fallback) and
// the flux difference run in FP32; con2prim of the cells, the implicit
// radiation-matter solve and the accumulation of U stay in FP64 (the same solver
// as the FP64 path, compiled here with fused multiply-add; the iteration's
// approximate matrix is kept, solved and updated in FP32, while its residual, iterate
// and convergence tests stay FP64).  Same launch structure and lanes as rrmhd_f64.cu.
#include <cuda_runtime.h>

#include "batch.h"
#include "batch_index.cuh"
#include "launch_shape.cuh"
#include "physics_tangent.cuh"
#include "scheme_f64.cuh"

namespace rr {

namespace {
using namespace idx;

constexpr int kFaceThreads = 128;
constexpr int kCellThreads = 128;

// Resident warps per SM the cell kernels are compiled for (a register bound of
// 65536 / (32 x warps) per thread).  12 warps (168 registers; the solver's stack grows
// from 1.5 to 1.9 KB) hide more of the FP64 dependency latency than the 8 that 255
// registers allow: +2 % zone-updates/s on C1 in the live step, measured under three
// cell shapes; 16 warps (128 registers) gained nothing.
#ifndef RR_F32_CELL_WARPS
#define RR_F32_CELL_WARPS 12
#endif
// Blocks per SM for a warp target W (at most 32 resident blocks per SM: partial-warp
// blocks of 8 threads keep no bound).
#define RR_F32_BLOCKS(W, BS) ((((W) * 32 + (BS) - 1) / (BS)) > 32 ? 32 : (((W) * 32 + (BS) - 1) / (BS)))
#define RR_F32_CELL_BLOCKS(BS) RR_F32_BLOCKS(RR_F32_CELL_WARPS, BS)
// The FP32 face kernels (127 registers unbounded) at 24 warps per SM (85 registers):
// 8 % shorter face launches.
#ifndef RR_F32_FACE_WARPS
#define RR_F32_FACE_WARPS 24
#endif
#define RR_F32_FACE_BLOCKS(BS) RR_F32_BLOCKS(RR_F32_FACE_WARPS, BS)

__device__ __forceinline__ rrt::PT<float> p32_of(const Params& P) {
  rrt::PT<float> q;
  q.gamma = (float)P.gamma;
  q.gfac = (float)P.gfac;
  q.gm1g = (float)P.gm1g;
  q.recon = P.recon;
  q.beta_mode = P.beta_mode;
  q.c2p_maxit = P.c2p_maxit;
  q.pvm_k = P.pvm_k;
  return q;
}

__device__ __forceinline__ void load12f(const double* __restrict__ A, int64_t stride, int64_t c,
                                        float* x) {
#pragma unroll
  for (int k = 0; k < NV; ++k) x[k] = (float)__ldg(A + k * stride + c);
}

// Face t of the launch's face ranges, in FP32.
static __device__ __noinline__ void face_item_f32(const StageArgs& a, int64_t t) {
  const Batch& b = a.b;
  const int64_t g = lane_face(b, t);
  const FacePos fp = face_pos(b, g);
  if (a.check_active && !inst_active(b, fp.i)) return;
  const InstDesc& I = fp.I;
  const int d = fp.d;
  const int f = fp.pos[d];
  int64_t cidx[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    int q[3] = {fp.pos[0], fp.pos[1], fp.pos[2]};
    q[d] = map_idx(f - 2 + s, I.n[d], I.bc[d]);
    cidx[s] = I.cell_off + ((int64_t)q[2] * I.n[1] + q[1]) * I.n[0] + q[0];
  }
  const rrt::PT<float> P = p32_of(a.P);
  const int64_t N = b.ncells;
  float VL[NV], VR[NV];
  {
    float w0[NV], w1[NV], w2[NV], tmp[NV];
    load12f(a.Vs, N, cidx[0], w0);
    load12f(a.Vs, N, cidx[1], w1);
    load12f(a.Vs, N, cidx[2], w2);
    rrt::reconstruct<float>(P.recon, w0, w1, w2, tmp, VL);
    load12f(a.Vs, N, cidx[3], w0);
    rrt::reconstruct<float>(P.recon, w1, w2, w0, VR, tmp);
  }
  const float dxd = (float)I.dx[d];
  if (a.ct && I.ndim >= 2) {  // constrained transport: the staggered normal field
    const float bn = (float)a.bs[g];
    VL[5 + d] = bn;
    VR[5 + d] = bn;
  }
  const float tauL = (float)(__ldg(a.Us + cidx[1]) * (__ldg(a.kappa + cidx[1]) + __ldg(a.sigma + cidx[1]))) * dxd;
  const float tauR = (float)(__ldg(a.Us + cidx[2]) * (__ldg(a.kappa + cidx[2]) + __ldg(a.sigma + cidx[2]))) * dxd;
  float F[NV];
  if (a.P.solver == 1)
    rrt::radhll_flux<float>(P, d, VL, VR, tauL, tauR, F);
  else
    rrt::pvm_flux<float>(P, d, VL, VR, tauL, tauR, F);
  const int64_t o = g - a.out_base;
#pragma unroll
  for (int k = 0; k < NV; ++k) a.Fhat32[k * a.fstride + o] = F[k];
}

// U* with the flux difference in FP32, accumulated into FP64; FP64 implicit solve.
__device__ __forceinline__ int cell_update_f32(const StageArgs& a, int64_t c, const CellPos& q,
                                               double* Un, double* Vn) {
  const Batch& b = a.b;
  const InstDesc& I = q.I;
  const double dt = b.st.dt[q.i];
  float dtdx[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) dtdx[d] = (float)(dt / I.dx[d]);
  int64_t fl[3], fr[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int m0 = I.n[0] + (d == 0);
    const int m1 = I.n[1] + (d == 1);
    const int64_t base = b.dir_base[d] + b.face_off[(int64_t)d * (b.n_inst + 1) + q.i];
    fl[d] = base + ((int64_t)q.p[2] * m1 + q.p[1]) * m0 + q.p[0];
    int r[3] = {q.p[0], q.p[1], q.p[2]};
    r[d] += 1;
    fr[d] = base + ((int64_t)r[2] * m1 + r[1]) * m0 + r[0];
  }
  double ca = 0.0, cb = 1.0, cw = 1.0;
  if (a.stage == 2) {
    ca = 0.75;
    cb = 0.25;
    cw = 0.25;
  } else if (a.stage == 3) {
    ca = 1.0 / 3.0;
    cb = 2.0 / 3.0;
    cw = 2.0 / 3.0;
  }
  const int64_t N = b.ncells;
  const int64_t FS = a.fstride;
  double Ust[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    float acc = (a.Fhat32[k * FS + fr[0]] - a.Fhat32[k * FS + fl[0]]) * dtdx[0];
    for (int d = 1; d < I.ndim; ++d) acc += (a.Fhat32[k * FS + fr[d]] - a.Fhat32[k * FS + fl[d]]) * dtdx[d];
    const double us = a.Us[k * N + c];
    Ust[k] = (a.stage == 1) ? us - (double)acc : ca * a.U0[k * N + c] + cb * (us - (double)acc);
  }
  if (a.ct && I.ndim >= 2)  // constrained transport: B_d is the mean of the two faces (FP64)
    for (int d = 0; d < I.ndim; ++d) Ust[5 + d] = 0.5 * (a.bout[fl[d]] + a.bout[fr[d]]);
  double vs[NV];
  load12(a.Vs, N, c, vs);
  double jc[17];
#pragma unroll
  for (int k = 0; k < 17; ++k) jc[k] = a.jc[k * N + c];
  const int rc = implicit_cell<FormBulk>(a.P, a.kappa[c], a.sigma[c], cw * dt, Ust, prim_Z(a.P, vs), Un, Vn, jc);
#pragma unroll
  for (int k = 0; k < 17; ++k) a.jc[k * N + c] = jc[k];
  return rc;
}

__device__ __forceinline__ void store_cell(const StageArgs& a, int64_t c, const double* Un,
                                           const double* Vn) {
  const int64_t N = a.b.ncells;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    a.Uout[k * N + c] = Un[k];
    a.Vout[k * N + c] = Vn[k];
  }
}

static __device__ __noinline__ void cell_item_f32(const StageArgs& a, int64_t c) {
  const CellPos q = cell_pos(a.b, c);
  if (!inst_active(a.b, q.i)) return;
  double Un[NV], Vn[NV];
  const int rc = cell_update_f32(a, c, q, Un, Vn);
  if (a.cell_status) a.cell_status[c] = rc;
  const bool retry = fallback_retry(rc);
  a.bad[c] = retry ? 1 : 0;
  if (retry) {
    if (a.flagged) atomicAdd(a.flagged + 1, 1u);
    return;
  }
  if (rc != ST_OK) {
    atomicCAS(a.b.st.status + q.i, 0, rc);
    if (a.b.st.bad_cell) atomicMin(a.b.st.bad_cell + q.i, (long long)c);
    return;
  }
  store_cell(a, c, Un, Vn);
}

template <int BS, int PT>
__global__ void __launch_bounds__(BS, RR_F32_FACE_BLOCKS(BS)) k_faces_f32(StageArgs a) {
  grid_items<BS, PT>(lane_faces(a.b), [&](int64_t t) { face_item_f32(a, t); });
}

template <int BS>
__global__ void __launch_bounds__(BS, RR_F32_FACE_BLOCKS(BS)) k_faces_f32_persistent(StageArgs a) {
  persistent_items(lane_faces(a.b), a.work, [&](int64_t t) { face_item_f32(a, t); });
}

template <int BS, int PT>
__global__ void __launch_bounds__(BS, RR_F32_CELL_BLOCKS(BS)) k_cells_f32(StageArgs a) {
  grid_items<BS, PT>(a.b.c_end - a.b.c_begin, [&](int64_t t) { cell_item_f32(a, a.b.c_begin + t); });
}

template <int BS>
__global__ void __launch_bounds__(BS, RR_F32_CELL_BLOCKS(BS)) k_cells_f32_persistent(StageArgs a) {
  persistent_items(a.b.c_end - a.b.c_begin, a.work + 1,
                   [&](int64_t t) { cell_item_f32(a, a.b.c_begin + t); });
}

__global__ void __launch_bounds__(kFaceThreads) k_fallback_faces_f32(StageArgs a) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const Batch& b = a.b;
  if (t >= lane_faces(b) || (a.flagged && a.flagged[a.fb_pass] == 0)) return;
  const int64_t g = lane_face(b, t);
  const FacePos fp = face_pos(b, g);
  if (!inst_active(b, fp.i)) return;
  const InstDesc& I = fp.I;
  const int d = fp.d;
  int ql[3] = {fp.pos[0], fp.pos[1], fp.pos[2]}, qr[3] = {fp.pos[0], fp.pos[1], fp.pos[2]};
  ql[d] = map_idx(fp.pos[d] - 1, I.n[d], I.bc[d]);
  qr[d] = map_idx(fp.pos[d], I.n[d], I.bc[d]);
  const int64_t cl = I.cell_off + ((int64_t)ql[2] * I.n[1] + ql[1]) * I.n[0] + ql[0];
  const int64_t cr = I.cell_off + ((int64_t)qr[2] * I.n[1] + qr[1]) * I.n[0] + qr[0];
  if (a.bad[cl] != a.fb_pass && a.bad[cr] != a.fb_pass) return;
  float vl[NV], vr[NV], F[NV];
  load12f(a.Vs, b.ncells, cl, vl);
  load12f(a.Vs, b.ncells, cr, vr);
  rrt::llf_flux<float>(p32_of(a.P), d, vl, vr, F);
  // (constrained transport: the magnetic components enter the edge EMFs)
#pragma unroll
  for (int k = 0; k < NV; ++k) a.Fhat32[k * a.fstride + g] = F[k];
}

// One cell of a fallback pass; in the last pass of stage 3, inst and s receive the
// cell's instance and CFL signal speed (left at -1 where the cell adds none).
__device__ __forceinline__ void fallback_cell_f32(const StageArgs& a, int64_t c, int& inst,
                                                  double& s) {
  const Batch& b = a.b;
  const CellPos q = cell_pos(b, c);
  const int pass = a.fb_pass;
  const bool last = pass == kFallbackPasses;
  const bool none = a.flagged && a.flagged[pass] == 0;  // no cell flagged in this pass
  if (none && !(a.stage == 3 && last)) return;
  if (!inst_active(b, q.i)) {
    if (a.stage == 3 && last) {
      double u[NV], v[NV];
      load12(a.U0, b.ncells, c, u);
      load12(a.V0, b.ncells, c, v);
      store_cell(a, c, u, v);
    }
    return;
  }
  const InstDesc& I = q.I;
  bool hit = !none && a.bad[c] == pass;
  if (!none && !hit && a.ct && I.ndim >= 2) {
    // constrained transport: the face field changes on every face that meets a
    // flagged cell's edges, so the whole 3x3(x3) block around it is updated again
    const int lo2 = I.ndim == 3 ? -1 : 0, hi2 = I.ndim == 3 ? 1 : 0;
    for (int dk = lo2; dk <= hi2 && !hit; ++dk)
      for (int dj = -1; dj <= 1 && !hit; ++dj)
        for (int di = -1; di <= 1 && !hit; ++di) {
          const int p[3] = {q.p[0] + di, q.p[1] + dj, q.p[2] + dk};
          bool in = true;
          int r[3];
          for (int d = 0; d < 3; ++d) {
            if ((p[d] < 0 || p[d] >= I.n[d]) && I.bc[d] != 1) in = false;  // outflow ghost cell
            r[d] = map_idx(p[d], I.n[d], I.bc[d]);
          }
          if (in && a.bad[I.cell_off + ((int64_t)r[2] * I.n[1] + r[1]) * I.n[0] + r[0]] == pass) hit = true;
        }
  }
  for (int d = 0; d < I.ndim && !hit && !none; ++d) {
    for (int e = -1; e <= 1; e += 2) {
      const int pd = q.p[d] + e;
      if ((pd < 0 || pd >= I.n[d]) && I.bc[d] != 1) continue;
      int r[3] = {q.p[0], q.p[1], q.p[2]};
      r[d] = map_idx(pd, I.n[d], I.bc[d]);
      if (a.bad[I.cell_off + ((int64_t)r[2] * I.n[1] + r[1]) * I.n[0] + r[0]] == pass) hit = true;
    }
  }
  double Vn[NV];
  if (hit) {
    double Un[NV];
    const int rc = cell_update_f32(a, c, q, Un, Vn);
    if (a.cell_status) a.cell_status[c] = rc;
    if (fallback_retry(rc) && a.bad[c] == 0 && !last) {
      a.bad[c] = (uint8_t)(pass + 1);  // its faces go first-order in the next pass
      if (a.flagged) atomicAdd(a.flagged + pass + 1, 1u);
      return;
    }
    if (rc != ST_OK) {
      atomicCAS(b.st.status + q.i, 0, rc);
      if (b.st.bad_cell) atomicMin(b.st.bad_cell + q.i, (long long)c);
      return;
    }
    store_cell(a, c, Un, Vn);
  } else if (a.stage == 3 && last) {
    load12(a.Vout, b.ncells, c, Vn);
  }
  if (a.stage == 3 && last) {
    s = signal_speed(a.P, 0, Vn) / I.dx[0];
    for (int d = 1; d < I.ndim; ++d) s = s + signal_speed(a.P, d, Vn) / I.dx[d];
    inst = q.i;
  }
}

__global__ void __launch_bounds__(kCellThreads) k_fallback_cells_f32(StageArgs a) {
  const int64_t c = a.b.c_begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int inst = -1;
  double s = 0.0;
  if (c < a.b.c_end) fallback_cell_f32(a, c, inst, s);
  // the CFL maximum of the next step (launch-uniform condition: every lane gets here)
  if (a.stage == 3 && a.fb_pass == kFallbackPasses)
    warp_smax(a.b.st.smax, inst, (unsigned long long)__double_as_longlong(s));
}

__global__ void k_widen(const float* __restrict__ F32, int64_t fs32, int64_t f_begin, int64_t n,
                        double* __restrict__ F) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
#pragma unroll
  for (int k = 0; k < NV; ++k) F[k * n + t] = (double)F32[k * fs32 + f_begin + t];
}

inline unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// Resident blocks per SM of the persistent kernels ([0] faces, [1] cells; by
// block size index 0..3), resolved by prepare_launch_shapes().
int g_resident[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
int g_sms = 0;

inline int bs_index(int B) { return B == 32 ? 0 : B == 64 ? 1 : B == 128 ? 2 : 3; }

inline unsigned persistent_grid(int64_t n, int B, int kind) {
  const int per_sm = g_resident[kind][bs_index(B)] > 0 ? g_resident[kind][bs_index(B)] : 1;
  const int64_t resident = (int64_t)(g_sms > 0 ? g_sms : 1) * per_sm;
  const int64_t needed = (n + B - 1) / B;
  return (unsigned)(needed < resident ? needed : resident);
}

}  // namespace

bool prepare_launch_shapes_f32() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
  bool ok = true;
#define X(B)                                                                                    \
  ok = ok && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_resident[0][bs_index(B)],         \
                                                          k_faces_f32_persistent<B>, B, 0) == cudaSuccess; \
  ok = ok && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_resident[1][bs_index(B)],         \
                                                          k_cells_f32_persistent<B>, B, 0) == cudaSuccess;
  RR_PERSISTENT_BLOCKS(X)
#undef X
  return ok;
}

void launch_faces_f32(const StageArgs& a, const LaunchShape& sh, cudaStream_t s) {
  const int64_t n = a.b.f_count[0] + a.b.f_count[1] + a.b.f_count[2];
  if (n <= 0) return;
  if (sh.persistent) {
    cudaMemsetAsync(a.work, 0, sizeof(unsigned long long), s);
#define X(B) \
    if (sh.block == B) { k_faces_f32_persistent<B><<<persistent_grid(n, B, 0), B, 0, s>>>(a); return; }
    RR_PERSISTENT_BLOCKS(X)
#undef X
  }
#define X(B, T) \
  if (sh.block == B && sh.per_thread == T) { k_faces_f32<B, T><<<grid_for(n, B * T), B, 0, s>>>(a); return; }
  RR_GRID_SHAPES(X)
#undef X
}

void launch_cells_f32(const StageArgs& a, const LaunchShape& sh, cudaStream_t s) {
  const int64_t n = a.b.c_end - a.b.c_begin;
  if (n <= 0) return;
  if (sh.persistent) {
    cudaMemsetAsync(a.work + 1, 0, sizeof(unsigned long long), s);
#define X(B) \
    if (sh.block == B) { k_cells_f32_persistent<B><<<persistent_grid(n, B, 1), B, 0, s>>>(a); return; }
    RR_PERSISTENT_BLOCKS(X)
#undef X
  }
#define X(B, T) \
  if (sh.block == B && sh.per_thread == T) { k_cells_f32<B, T><<<grid_for(n, B * T), B, 0, s>>>(a); return; }
  RR_GRID_SHAPES(X)
#undef X
}

void launch_fallback_f32(const StageArgs& a, cudaStream_t s) {
  const int64_t nf = a.b.f_count[0] + a.b.f_count[1] + a.b.f_count[2];
  const int64_t nc = a.b.c_end - a.b.c_begin;
  if (nf > 0) k_fallback_faces_f32<<<grid_for(nf, kFaceThreads), kFaceThreads, 0, s>>>(a);
  if (a.ct) {
    launch_emf_f64(a, s);
    launch_bface_f64(a, s);
  }
  if (nc > 0) k_fallback_cells_f32<<<grid_for(nc, kCellThreads), kCellThreads, 0, s>>>(a);
}

void launch_widen_f32(const float* F32, int64_t fstride32, int64_t f_begin, int64_t n, double* F,
                      cudaStream_t s) {
  if (n > 0) k_widen<<<grid_for(n, 256), 256, 0, s>>>(F32, fstride32, f_begin, n, F);
}

}  // namespace rr
