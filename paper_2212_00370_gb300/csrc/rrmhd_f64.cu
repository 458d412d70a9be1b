// rrmhd_f64.cu -- FP64 kernels of one IMEX-RK3 stage over a batch of instances
// (arXiv:2212.00370, Secs. 3.1-3.3).  Compiled with --fmad=false: see the
// arithmetic contract in physics_f64.cuh.
//
// A stage is two launches over packed work lists, so ragged batches keep every
// lane busy:
//   k_faces : one thread per face (all directions, all instances): stencil of
//             4 cells along the face normal through the boundary map, PLM +
//             fallback, PVM-int-8 flux -> Fhat.
//   k_cells : one thread per cell: flux difference and RK combination, then
//             the implicit radiation-matter solve -> U^(s), V^(s); stage 3 also
//             reduces the next CFL signal speed per instance.
// The path is FP64-pipe bound (tens of thousands of FP64 instructions per cell
// and a few hundred bytes of traffic), so the layout favours full warps and low
// register pressure over shared-memory staging.
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
// Resident warps per SM requested from the register allocator for the face and cell
// kernels (launch-bounds tuning knobs): 0 leaves the registers unbounded (255 per
// thread, 8 warps per SM); W > 0 asks for W warps per SM in blocks of BS threads (at
// most 32 resident blocks per SM).
#ifndef RR_F64_FACE_WARPS
#define RR_F64_FACE_WARPS 0
#endif
#ifndef RR_F64_CELL_WARPS
#define RR_F64_CELL_WARPS 0
#endif
#define RR_F64_BLOCKS(W, BS) \
  ((W) == 0 ? 1 : ((((W) * 32 + (BS) - 1) / (BS)) > 32 ? 32 : (((W) * 32 + (BS) - 1) / (BS))))

// PVM flux with exact tangent products A w (the FP64 tangent variant): the same
// reconstruction, central fluxes, con2prim of U_m and beta as pvm_flux, only the
// A^2 products differ (dual numbers instead of Eq. utilde's flux differences).
__device__ __forceinline__ int pvm_flux_tangent(const Params& P, int d, const double* VL,
                                                const double* VR, double tauL, double tauR,
                                                double* Fhat) {
  double Um[NV], U0[NV], Ul[NV];
  double ZL, ZR;
  {
    double UL[NV], UR[NV], FL[NV], FR[NV];
    prim2con(P, VL, UL);
    prim2con(P, VR, UR);
    flux(P, d, VL, UL, FL);
    flux(P, d, VR, UR, FR);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      U0[k] = UR[k] - UL[k];
      Um[k] = 0.5 * (UL[k] + UR[k]);
      Fhat[k] = 0.5 * (FL[k] + FR[k]);
    }
    ZL = prim_Z(P, VL);
    ZR = prim_Z(P, VR);
  }
  const double Zg = 0.5 * (ZL + ZR);
  double beta = 1.0;
  if (P.beta_mode) {
    double t = tauL > tauR ? tauL : tauR;
    if (t < 1.0) t = 1.0;
    beta = 1.0 / t;
  }
  int fail = 1;
  double Vm[NV], Zm = 0.0;
  if (con2prim(P, Um, Zg, Vm, &Zm) == ST_OK) {
    rrt::PT<double> Q;
    Q.gamma = P.gamma;
    Q.gfac = P.gfac;
    Q.gm1g = P.gm1g;
    Q.recon = P.recon;
    Q.beta_mode = P.beta_mode;
    Q.c2p_maxit = P.c2p_maxit;
    Q.pvm_k = P.pvm_k;
    // W' = Z - D at the root and the residual's derivative there
    const rrt::C2PIn<double> c = rrt::c2p_in(Um);
    rrt::C2PPt<double> e;
    const double xm = Zm - Um[0];
    rrt::c2p_eval(c, P.gm1g, xm, e);
    if (e.ok && rrt::pvm_viscosity(Q, d, Um, xm, e.df, U0, Ul)) fail = 0;
  }
  if (fail) {
#pragma unroll
    for (int k = 0; k < NV; ++k) Ul[k] = U0[k];
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const double bk = (P.beta_mode == 2 && k < 8) ? 1.0 : beta;  // beta_mode 2: radiation only
    Fhat[k] = Fhat[k] - 0.5 * (bk * Ul[k]);
  }
  return fail;
}

// Face t of the launch's face ranges: stencil, PLM + fallback, PVM-int flux.
static __device__ __noinline__ void face_item(const StageArgs& a, int64_t t) {
  const Batch& b = a.b;
  const int64_t g = lane_face(b, t);
  const FacePos fp = face_pos(b, g);
  if (a.check_active && !inst_active(b, fp.i)) return;
  const InstDesc& I = fp.I;
  const int d = fp.d;
  const int* pos = fp.pos;
  const int f = pos[d];
  int64_t cidx[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    int q[3] = {pos[0], pos[1], pos[2]};
    q[d] = map_idx(f - 2 + s, I.n[d], I.bc[d]);
    cidx[s] = I.cell_off + ((int64_t)q[2] * I.n[1] + q[1]) * I.n[0] + q[0];
  }
  const int64_t N = b.ncells;
  double VL[NV], VR[NV];
  {
    double w0[NV], w1[NV], w2[NV], tmp[NV];
    load12(a.Vs, N, cidx[0], w0);
    load12(a.Vs, N, cidx[1], w1);
    load12(a.Vs, N, cidx[2], w2);
    reconstruct(a.P.recon, w0, w1, w2, tmp, VL);  // cell f-1: its right face
    load12(a.Vs, N, cidx[3], w0);
    reconstruct(a.P.recon, w1, w2, w0, VR, tmp);  // cell f: its left face
  }
  if (a.ct && I.ndim >= 2) {  // constrained transport: the staggered normal field
    const double bn = a.bs[g];
    VL[5 + d] = bn;
    VR[5 + d] = bn;
  }
  const double dxd = I.dx[d];
  const double tauL = (__ldg(a.Us + cidx[1]) * (__ldg(a.kappa + cidx[1]) + __ldg(a.sigma + cidx[1]))) * dxd;
  const double tauR = (__ldg(a.Us + cidx[2]) * (__ldg(a.kappa + cidx[2]) + __ldg(a.sigma + cidx[2]))) * dxd;
  double F[NV];
  if (a.P.solver == 1)
    radhll_flux(a.P, d, VL, VR, tauL, tauR, F);
  else if (a.P.pvm_products)
    pvm_flux_tangent(a.P, d, VL, VR, tauL, tauR, F);
  else
    pvm_flux(a.P, d, VL, VR, tauL, tauR, F);
  const int64_t o = g - a.out_base;
#pragma unroll
  for (int k = 0; k < NV; ++k) a.Fhat[k * a.fstride + o] = F[k];
}

// U* of cell c from its face fluxes (flux difference and RK combination,
// Sec. 3.1), then the implicit solve (Sec. 3.3); returns a Status.
__device__ __forceinline__ int cell_update(const StageArgs& a, int64_t c, const CellPos& q,
                                           double* Un, double* Vn) {
  const Batch& b = a.b;
  const InstDesc& I = q.I;
  const double dt = b.st.dt[q.i];
  double dtdx[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) dtdx[d] = dt / I.dx[d];
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
  const double hdt = cw * dt;
  const int64_t N = b.ncells;
  const int64_t FS = a.fstride;
  double Ust[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double acc = (a.Fhat[k * FS + fr[0]] - a.Fhat[k * FS + fl[0]]) * dtdx[0];
    for (int d = 1; d < I.ndim; ++d)
      acc = acc + (a.Fhat[k * FS + fr[d]] - a.Fhat[k * FS + fl[d]]) * dtdx[d];
    const double us = a.Us[k * N + c];
    if (a.stage == 1)
      Ust[k] = us - acc;
    else
      Ust[k] = ca * a.U0[k * N + c] + cb * (us - acc);
  }
  if (a.ct && I.ndim >= 2)  // constrained transport: B_d is the mean of the two faces
    for (int d = 0; d < I.ndim; ++d) Ust[5 + d] = 0.5 * (a.bout[fl[d]] + a.bout[fr[d]]);
  double vs[NV];
  load12(a.Vs, N, c, vs);
  const double Zg = prim_Z(a.P, vs);
  double jc[17];
#pragma unroll
  for (int k = 0; k < 17; ++k) jc[k] = a.jc[k * N + c];
  const int rc = implicit_cell(a.P, a.kappa[c], a.sigma[c], hdt, Ust, Zg, Un, Vn, jc);
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

// Pass 1: every cell.  A cell whose U* is inadmissible is only flagged.
static __device__ __noinline__ void cell_item(const StageArgs& a, int64_t c) {
  const CellPos q = cell_pos(a.b, c);
  if (!inst_active(a.b, q.i)) return;
  double Un[NV], Vn[NV];
  const int rc = cell_update(a, c, q, Un, Vn);
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
__global__ void __launch_bounds__(BS, RR_F64_BLOCKS(RR_F64_FACE_WARPS, BS)) k_faces(StageArgs a) {
  grid_items<BS, PT>(lane_faces(a.b), [&](int64_t t) { face_item(a, t); });
}

template <int BS>
__global__ void __launch_bounds__(BS, RR_F64_BLOCKS(RR_F64_FACE_WARPS, BS)) k_faces_persistent(StageArgs a) {
  persistent_items(lane_faces(a.b), a.work, [&](int64_t t) { face_item(a, t); });
}

template <int BS, int PT>
__global__ void __launch_bounds__(BS, RR_F64_BLOCKS(RR_F64_CELL_WARPS, BS)) k_cells(StageArgs a) {
  grid_items<BS, PT>(a.b.c_end - a.b.c_begin, [&](int64_t t) { cell_item(a, a.b.c_begin + t); });
}

template <int BS>
__global__ void __launch_bounds__(BS, RR_F64_BLOCKS(RR_F64_CELL_WARPS, BS)) k_cells_persistent(StageArgs a) {
  persistent_items(a.b.c_end - a.b.c_begin, a.work + 1,
                   [&](int64_t t) { cell_item(a, a.b.c_begin + t); });
}

// Admissibility fallback, pass a.fb_pass, faces: first-order Rusanov flux at
// every face next to a cell flagged in this pass.
__global__ void __launch_bounds__(kFaceThreads) k_fallback_faces(StageArgs a) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const Batch& b = a.b;
  if (t >= lane_faces(b) || (a.flagged && a.flagged[a.fb_pass] == 0)) return;
  const int64_t g = lane_face(b, t);
  const FacePos fp = face_pos(b, g);
  if (!inst_active(b, fp.i)) return;
  const InstDesc& I = fp.I;
  const int d = fp.d;
  const int* pos = fp.pos;
  int ql[3] = {pos[0], pos[1], pos[2]}, qr[3] = {pos[0], pos[1], pos[2]};
  ql[d] = map_idx(pos[d] - 1, I.n[d], I.bc[d]);
  qr[d] = map_idx(pos[d], I.n[d], I.bc[d]);
  const int64_t cl = I.cell_off + ((int64_t)ql[2] * I.n[1] + ql[1]) * I.n[0] + ql[0];
  const int64_t cr = I.cell_off + ((int64_t)qr[2] * I.n[1] + qr[1]) * I.n[0] + qr[0];
  if (a.bad[cl] != a.fb_pass && a.bad[cr] != a.fb_pass) return;
  double vl[NV], vr[NV], F[NV];
  load12(a.Vs, b.ncells, cl, vl);
  load12(a.Vs, b.ncells, cr, vr);
  llf_flux(a.P, d, vl, vr, F);
  // (constrained transport: the magnetic components enter the edge EMFs)
#pragma unroll
  for (int k = 0; k < NV; ++k) a.Fhat[k * a.fstride + g] = F[k];
}

// Admissibility fallback, pass a.fb_pass, cells: update again every cell with a
// face changed in this pass (flagged in it, or sharing a face with such a cell).
// A cell that still has no admissible update and was never flagged is flagged
// for the next pass; in the last pass it fails its instance.  The last pass of
// stage 3 also reduces the next CFL signal speed of every cell and carries
// inactive instances over.
// One cell of a fallback pass; in the last pass of stage 3, inst and s receive the
// cell's instance and CFL signal speed (left at -1 where the cell adds none).
__device__ __forceinline__ void fallback_cell(const StageArgs& a, int64_t c, int& inst, double& s) {
  const Batch& b = a.b;
  const CellPos q = cell_pos(b, c);
  const int pass = a.fb_pass;
  const bool last = pass == kFallbackPasses;
  const bool none = a.flagged && a.flagged[pass] == 0;  // no cell flagged in this pass
  if (none && !(a.stage == 3 && last)) return;
  if (!inst_active(b, q.i)) {
    // finished or failed instance: carry its start-of-step state into the
    // step's output buffers (a failed instance stays at its last good state)
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
      if ((pd < 0 || pd >= I.n[d]) && I.bc[d] != 1) continue;  // outflow ghost face
      int r[3] = {q.p[0], q.p[1], q.p[2]};
      r[d] = map_idx(pd, I.n[d], I.bc[d]);
      if (a.bad[I.cell_off + ((int64_t)r[2] * I.n[1] + r[1]) * I.n[0] + r[0]] == pass) hit = true;
    }
  }
  double Vn[NV];
  if (hit) {
    double Un[NV];
    const int rc = cell_update(a, c, q, Un, Vn);
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

__global__ void __launch_bounds__(kCellThreads, RR_F64_BLOCKS(RR_F64_CELL_WARPS, kCellThreads)) k_fallback_cells(StageArgs a) {
  const int64_t c = a.b.c_begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int inst = -1;
  double s = 0.0;
  if (c < a.b.c_end) fallback_cell(a, c, inst, s);
  // the CFL maximum of the next step (launch-uniform condition: every lane gets here)
  if (a.stage == 3 && a.fb_pass == kFallbackPasses)
    warp_smax(a.b.st.smax, inst, (unsigned long long)__double_as_longlong(s));
}

// ------------------------------------------------------------ constrained transport
// CT-contact edge EMF (Gardiner & Stone 2005, Eqs. 41 and 50), E_e at the edge
// between cells (ia-1, ia) along a and (ib-1, ib) along b, e = a x b cyclic:
// the mean of the four face EMFs (-F^a(B_b) at a-faces, +F^b(B_a) at b-faces)
// plus the half-cell differences to the cell-centre E_ref = v_b B_a - v_a B_b,
// each taken from the side the face mass flux comes from.
__device__ __forceinline__ double ct_upwind(double f, double lo, double hi) {
  if (f > 0.0) return lo;
  if (f < 0.0) return hi;
  return 0.5 * (lo + hi);
}

template <class FT>
__device__ __forceinline__ double fhat(const StageArgs& a, int64_t i);
template <>
__device__ __forceinline__ double fhat<double>(const StageArgs& a, int64_t i) { return a.Fhat[i]; }
template <>
__device__ __forceinline__ double fhat<float>(const StageArgs& a, int64_t i) {
  return (double)a.Fhat32[i];
}

// FT: the precision the face fluxes are stored in (FP64, or FP32 in FP32-bulk);
// the EMFs and the face field are FP64 either way.
template <class FT>
__global__ void __launch_bounds__(kFaceThreads) k_emf(StageArgs a) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const Batch& b = a.b;
  if (t >= lane_edges(b)) return;
  if (a.fb_pass > 0 && a.flagged && a.flagged[a.fb_pass] == 0) return;  // fallback pass: nothing flagged
  const EdgePos q = edge_pos(b, t);
  if (!inst_active(b, q.i)) return;
  const InstDesc& I = q.I;
  const int A = (q.e + 1) % 3, Bd = (q.e + 2) % 3;
  int pa0[3] = {q.pos[0], q.pos[1], q.pos[2]}, pa1[3] = {q.pos[0], q.pos[1], q.pos[2]};
  pa0[Bd] -= 1;
  const int64_t fa0 = face_gidx(b, I, A, pa0), fa1 = face_gidx(b, I, A, pa1);
  int pb0[3] = {q.pos[0], q.pos[1], q.pos[2]}, pb1[3] = {q.pos[0], q.pos[1], q.pos[2]};
  pb0[A] -= 1;
  const int64_t fb0 = face_gidx(b, I, Bd, pb0), fb1 = face_gidx(b, I, Bd, pb1);
  const int64_t FS = a.fstride;
  const double Ea0 = -fhat<FT>(a, (5 + Bd) * FS + fa0), Ea1 = -fhat<FT>(a, (5 + Bd) * FS + fa1);
  const double Eb0 = fhat<FT>(a, (5 + A) * FS + fb0), Eb1 = fhat<FT>(a, (5 + A) * FS + fb1);
  const double ma0 = fhat<FT>(a, fa0), ma1 = fhat<FT>(a, fa1);
  const double mb0 = fhat<FT>(a, fb0), mb1 = fhat<FT>(a, fb1);
  const int64_t N = b.ncells;
  double Er[2][2];
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      int p[3] = {q.pos[0], q.pos[1], q.pos[2]};
      p[A] += s - 1;
      p[Bd] += r - 1;
      const int64_t c = cell_gidx(I, p);
      const double va = a.Vs[(1 + A) * N + c], vb = a.Vs[(1 + Bd) * N + c];
      const double Ba = a.Vs[(5 + A) * N + c], Bb = a.Vs[(5 + Bd) * N + c];
      Er[s][r] = vb * Ba - va * Bb;
    }
  const double Lb = ct_upwind(ma0, Eb0 - Er[0][0], Eb1 - Er[1][0]);
  const double Ub = ct_upwind(ma1, Er[0][1] - Eb0, Er[1][1] - Eb1);
  const double La = ct_upwind(mb0, Ea0 - Er[0][0], Ea1 - Er[0][1]);
  const double Ra = ct_upwind(mb1, Er[1][0] - Ea0, Er[1][1] - Ea1);
  a.emf[q.g] = 0.25 * (((Ea0 + Ea1) + Eb0) + Eb1) + 0.25 * (Lb - Ub) + 0.25 * (La - Ra);
}

// Face-field stage update: b_out = a b0 + c (b_s - dt (curl E)_d), with
// (curl E)_d = dE_{d+2}/dx_{d+1} - dE_{d+1}/dx_{d+2} (cyclic) and the stage weights of
// U.  An inactive instance carries its step-start field in stage 3.
__global__ void __launch_bounds__(kFaceThreads) k_bface(StageArgs a) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const Batch& b = a.b;
  if (t >= lane_faces(b)) return;
  if (a.fb_pass > 0 && a.flagged && a.flagged[a.fb_pass] == 0) return;  // fallback pass: nothing flagged
  const int64_t g = lane_face(b, t);
  const FacePos fp = face_pos(b, g);
  const InstDesc& I = fp.I;
  if (I.ndim < 2) return;
  if (!inst_active(b, fp.i)) {
    if (a.stage == 3) a.bout[g] = a.b0[g];
    return;
  }
  const int d = fp.d, p1 = (d + 1) % 3, p2 = (d + 2) % 3;
  const double dt = b.st.dt[fp.i];
  double curl = 0.0;
  if (has_edges(I, p2)) {
    int q0[3] = {fp.pos[0], fp.pos[1], fp.pos[2]}, q1[3] = {fp.pos[0], fp.pos[1], fp.pos[2]};
    q1[p1] += 1;
    curl = curl + (a.emf[edge_gidx(b, I, p2, q1)] - a.emf[edge_gidx(b, I, p2, q0)]) / I.dx[p1];
  }
  if (has_edges(I, p1)) {
    int q0[3] = {fp.pos[0], fp.pos[1], fp.pos[2]}, q1[3] = {fp.pos[0], fp.pos[1], fp.pos[2]};
    q1[p2] += 1;
    curl = curl - (a.emf[edge_gidx(b, I, p1, q1)] - a.emf[edge_gidx(b, I, p1, q0)]) / I.dx[p2];
  }
  double ca = 0.0, cb = 1.0;
  if (a.stage == 2) {
    ca = 0.75;
    cb = 0.25;
  } else if (a.stage == 3) {
    ca = 1.0 / 3.0;
    cb = 2.0 / 3.0;
  }
  const double upd = a.bs[g] - dt * curl;
  a.bout[g] = (a.stage == 1) ? upd : ca * a.b0[g] + cb * upd;
}

// Set-up: face field from cell-centred B (mean of the two cells next to a face).
__global__ void k_faces_from_cells(Batch b, const double* __restrict__ V, double* bface) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= lane_faces(b)) return;
  const int64_t g = lane_face(b, t);
  const FacePos fp = face_pos(b, g);
  const InstDesc& I = fp.I;
  if (I.ndim < 2) return;
  int pl[3] = {fp.pos[0], fp.pos[1], fp.pos[2]}, pr[3] = {fp.pos[0], fp.pos[1], fp.pos[2]};
  pl[fp.d] -= 1;
  const int64_t N = b.ncells;
  const double bl = V[(5 + fp.d) * N + cell_gidx(I, pl)];
  const double br = V[(5 + fp.d) * N + cell_gidx(I, pr)];
  bface[g] = 0.5 * (bl + br);
}

// Set-up: periodic duplicate faces (index n_d) take the value of face 0.
__global__ void k_ct_canonical(Batch b, double* bface) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= lane_faces(b)) return;
  const int64_t g = lane_face(b, t);
  const FacePos fp = face_pos(b, g);
  const InstDesc& I = fp.I;
  if (I.ndim < 2 || I.bc[fp.d] != 1 || fp.pos[fp.d] != I.n[fp.d]) return;
  int p[3] = {fp.pos[0], fp.pos[1], fp.pos[2]};
  p[fp.d] = 0;
  bface[g] = bface[face_gidx(b, I, fp.d, p)];
}

// Set-up: cell-centred B_d (d < ndim) of V from the face means.
__global__ void k_cells_from_faces(Batch b, const double* __restrict__ bface, double* V) {
  const int64_t c = b.c_begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= b.c_end) return;
  const CellPos q = cell_pos(b, c);
  const InstDesc& I = q.I;
  if (I.ndim < 2) return;
  const int64_t N = b.ncells;
  for (int d = 0; d < I.ndim; ++d) {
    int pl[3] = {q.p[0], q.p[1], q.p[2]}, pr[3] = {q.p[0], q.p[1], q.p[2]};
    pr[d] += 1;
    V[(5 + d) * N + c] = 0.5 * (bface[face_gidx(b, I, d, pl)] + bface[face_gidx(b, I, d, pr)]);
  }
}

__global__ void k_signal(Params P, Batch b, const double* __restrict__ V) {
  const int64_t c = b.c_begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int i = -1;
  double s = 0.0;
  if (c < b.c_end) {
    i = find_inst(b.cell_off, b.i_begin, b.i_end, c);
    const InstDesc I = b.inst[i];
    double v[NV];
    load12(V, b.ncells, c, v);
    s = signal_speed(P, 0, v) / I.dx[0];
    for (int d = 1; d < I.ndim; ++d) s = s + signal_speed(P, d, v) / I.dx[d];
  }
  warp_smax(b.st.smax, i, (unsigned long long)__double_as_longlong(s));
}

// dt = CFL / max_cells sum_d lambda_d/dx_d, clipped to land on t_end.
__global__ void k_begin_step(Params P, Batch b) {
  const int i = b.i_begin + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= b.i_end) return;
  const double t = b.st.t[i], te = b.st.t_end[i];
  double dt = 0.0;
  if (b.st.status[i] == 0 && t < te) {
    const double smax = __longlong_as_double((long long)b.st.smax[i]);
    dt = P.cfl / smax;
    if (b.st.dt_max && dt > *b.st.dt_max) dt = *b.st.dt_max;
    if (t + dt > te) dt = te - t;
    if (!(dt > 0.0)) {  // NaN or non-positive speed bound
      dt = 0.0;
      b.st.status[i] = ST_UNPHYS;
    }
  }
  b.st.dt[i] = dt;
  b.st.smax[i] = 0ull;
}

// U -= (F_right - F_left) (dt_weight / dx_dir) at every cell (Eq. explicit, one
// direction); the FP64 operation order of the stage's flux difference.  FP32 fluxes
// (FP32-bulk) are differenced in FP32, as the FP32-bulk stage does.
__global__ void k_flux_accumulate(Batch b, int dir, double dt_weight, const double* __restrict__ F64,
                                  const float* __restrict__ F32, int64_t fstride, int64_t out_base,
                                  double* U) {
  const int64_t c = b.c_begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= b.c_end) return;
  const CellPos q = cell_pos(b, c);
  const InstDesc& I = q.I;
  if (dir >= I.ndim) return;  // no faces normal to dir
  const int m0 = I.n[0] + (dir == 0);
  const int m1 = I.n[1] + (dir == 1);
  const int64_t base = b.dir_base[dir] + b.face_off[(int64_t)dir * (b.n_inst + 1) + q.i];
  int r[3] = {q.p[0], q.p[1], q.p[2]};
  const int64_t fl = base + ((int64_t)r[2] * m1 + r[1]) * m0 + r[0] - out_base;
  r[dir] += 1;
  const int64_t fr = base + ((int64_t)r[2] * m1 + r[1]) * m0 + r[0] - out_base;
  const int64_t N = b.ncells;
  if (F32) {
    const float dtdx = (float)(dt_weight / I.dx[dir]);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const float acc = (F32[k * fstride + fr] - F32[k * fstride + fl]) * dtdx;
      U[k * N + c] = U[k * N + c] - (double)acc;
    }
  } else {
    const double dtdx = dt_weight / I.dx[dir];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double acc = (F64[k * fstride + fr] - F64[k * fstride + fl]) * dtdx;
      U[k * N + c] = U[k * N + c] - acc;
    }
  }
}

__global__ void k_fill_i64(long long* p, int64_t n, long long v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

__global__ void k_set_f64(double* p, double v) { *p = v; }

__global__ void k_end_step(Batch b) {
  const int i = b.i_begin + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= b.i_end) return;
  if (b.st.status[i] == 0 && b.st.dt[i] > 0.0) b.st.t[i] = b.st.t[i] + b.st.dt[i];
}

__global__ void k_prim2con(Params P, const double* __restrict__ V, double* __restrict__ U,
                           int64_t n) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double v[NV], u[NV];
  load12(V, n, c, v);
  prim2con(P, v, u);
#pragma unroll
  for (int k = 0; k < NV; ++k) U[k * n + c] = u[k];
}

__global__ void k_prim_Z(Params P, const double* __restrict__ V, double* __restrict__ Z,
                         int64_t n) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double v[NV];
  load12(V, n, c, v);
  Z[c] = prim_Z(P, v);
}

__global__ void k_con2prim(Params P, const double* __restrict__ U, const double* __restrict__ Zg,
                           double* __restrict__ V, int32_t* __restrict__ status, int64_t n) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double u[NV], v[NV];
  load12(U, n, c, u);
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = 0.0;
  const int rc = con2prim(P, u, Zg ? Zg[c] : 0.0, v, nullptr);
  if (status) status[c] = rc;
#pragma unroll
  for (int k = 0; k < NV; ++k) V[k * n + c] = v[k];
}

__global__ void k_implicit(Params P, Batch b, double hdt, const double* __restrict__ Us,
                           const double* __restrict__ Zg, const double* __restrict__ kappa,
                           const double* __restrict__ sigma, double* __restrict__ U,
                           double* __restrict__ V, int32_t* __restrict__ status) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = b.ncells;
  if (c >= n) return;
  double us[NV], un[NV], vn[NV];
  load12(Us, n, c, us);
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    un[k] = 0.0;
    vn[k] = 0.0;
  }
  const int rc = implicit_cell(P, kappa[c], sigma[c], hdt, us, Zg ? Zg[c] : 0.0, un, vn);
  if (status) status[c] = rc;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    U[k * n + c] = un[k];
    V[k * n + c] = vn[k];
  }
}

inline unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// Resident blocks per SM of the persistent kernels ([0] faces, [1] cells; by
// block size index 0..3), resolved by prepare_launch_shapes().
int g_resident[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
int g_sms = 0;

inline int bs_index(int B) { return B == 32 ? 0 : B == 64 ? 1 : B == 128 ? 2 : 3; }

// Blocks of a persistent launch: the resident grid, or fewer when n is small.
inline unsigned persistent_grid(int64_t n, int B, int kind) {
  const int per_sm = g_resident[kind][bs_index(B)] > 0 ? g_resident[kind][bs_index(B)] : 1;
  const int64_t resident = (int64_t)(g_sms > 0 ? g_sms : 1) * per_sm;
  const int64_t needed = (n + B - 1) / B;
  return (unsigned)(needed < resident ? needed : resident);
}

}  // namespace

bool prepare_launch_shapes_f64() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
  bool ok = true;
#define X(B)                                                                                   \
  ok = ok && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_resident[0][bs_index(B)],        \
                                                          k_faces_persistent<B>, B, 0) == cudaSuccess; \
  ok = ok && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_resident[1][bs_index(B)],        \
                                                          k_cells_persistent<B>, B, 0) == cudaSuccess;
  RR_PERSISTENT_BLOCKS(X)
#undef X
  return ok;
}

void launch_faces_f64(const StageArgs& a, const LaunchShape& sh, cudaStream_t s) {
  const int64_t n = a.b.f_count[0] + a.b.f_count[1] + a.b.f_count[2];
  if (n <= 0) return;
  if (sh.persistent) {
    cudaMemsetAsync(a.work, 0, sizeof(unsigned long long), s);
#define X(B) \
    if (sh.block == B) { k_faces_persistent<B><<<persistent_grid(n, B, 0), B, 0, s>>>(a); return; }
    RR_PERSISTENT_BLOCKS(X)
#undef X
  }
#define X(B, T) \
  if (sh.block == B && sh.per_thread == T) { k_faces<B, T><<<grid_for(n, B * T), B, 0, s>>>(a); return; }
  RR_GRID_SHAPES(X)
#undef X
}

void launch_cells_f64(const StageArgs& a, const LaunchShape& sh, cudaStream_t s) {
  const int64_t n = a.b.c_end - a.b.c_begin;
  if (n <= 0) return;
  if (sh.persistent) {
    cudaMemsetAsync(a.work + 1, 0, sizeof(unsigned long long), s);
#define X(B) \
    if (sh.block == B) { k_cells_persistent<B><<<persistent_grid(n, B, 1), B, 0, s>>>(a); return; }
    RR_PERSISTENT_BLOCKS(X)
#undef X
  }
#define X(B, T) \
  if (sh.block == B && sh.per_thread == T) { k_cells<B, T><<<grid_for(n, B * T), B, 0, s>>>(a); return; }
  RR_GRID_SHAPES(X)
#undef X
}

void launch_fallback_f64(const StageArgs& a, cudaStream_t s) {
  const int64_t nf = a.b.f_count[0] + a.b.f_count[1] + a.b.f_count[2];
  const int64_t nc = a.b.c_end - a.b.c_begin;
  if (nf > 0) k_fallback_faces<<<grid_for(nf, kFaceThreads), kFaceThreads, 0, s>>>(a);
  if (a.ct) {
    launch_emf_f64(a, s);
    launch_bface_f64(a, s);
  }
  if (nc > 0) k_fallback_cells<<<grid_for(nc, kCellThreads), kCellThreads, 0, s>>>(a);
}

void launch_emf_f64(const StageArgs& a, cudaStream_t s) {
  const int64_t n = a.b.e_count[0] + a.b.e_count[1] + a.b.e_count[2];
  if (n <= 0) return;
  if (a.fp32_fluxes)
    k_emf<float><<<grid_for(n, kFaceThreads), kFaceThreads, 0, s>>>(a);
  else
    k_emf<double><<<grid_for(n, kFaceThreads), kFaceThreads, 0, s>>>(a);
}

void launch_bface_f64(const StageArgs& a, cudaStream_t s) {
  const int64_t n = a.b.f_count[0] + a.b.f_count[1] + a.b.f_count[2];
  if (n > 0) k_bface<<<grid_for(n, kFaceThreads), kFaceThreads, 0, s>>>(a);
}

void launch_faces_from_cells_f64(const Batch& b, const double* V, double* bface, cudaStream_t s) {
  const int64_t n = b.f_count[0] + b.f_count[1] + b.f_count[2];
  if (n > 0) k_faces_from_cells<<<grid_for(n, 128), 128, 0, s>>>(b, V, bface);
}

void launch_ct_canonical_f64(const Batch& b, double* bface, cudaStream_t s) {
  const int64_t n = b.f_count[0] + b.f_count[1] + b.f_count[2];
  if (n > 0) k_ct_canonical<<<grid_for(n, 128), 128, 0, s>>>(b, bface);
}

void launch_cells_from_faces_f64(const Batch& b, const double* bface, double* V, cudaStream_t s) {
  const int64_t n = b.c_end - b.c_begin;
  if (n > 0) k_cells_from_faces<<<grid_for(n, 128), 128, 0, s>>>(b, bface, V);
}

void launch_signal_f64(const Params& P, const Batch& b, const double* V, cudaStream_t s) {
  const int64_t n = b.c_end - b.c_begin;
  if (n <= 0) return;
  k_signal<<<grid_for(n, 128), 128, 0, s>>>(P, b, V);
}

void launch_flux_accumulate(const Batch& b, int dir, double dt_weight, const double* F64,
                            const float* F32, int64_t fstride, int64_t out_base, double* U,
                            cudaStream_t s) {
  const int64_t n = b.c_end - b.c_begin;
  if (n > 0) k_flux_accumulate<<<grid_for(n, 128), 128, 0, s>>>(b, dir, dt_weight, F64, F32, fstride, out_base, U);
}

void launch_fill_i64(long long* p, int64_t n, long long v, cudaStream_t s) {
  if (n > 0) k_fill_i64<<<grid_for(n, 256), 256, 0, s>>>(p, n, v);
}

void launch_set_f64(double* p, double v, cudaStream_t s) { k_set_f64<<<1, 1, 0, s>>>(p, v); }

void launch_begin_step(const Params& P, const Batch& b, cudaStream_t s) {
  const int n = b.i_end - b.i_begin;
  if (n <= 0) return;
  k_begin_step<<<grid_for(n, 128), 128, 0, s>>>(P, b);
}

void launch_end_step(const Batch& b, cudaStream_t s) {
  const int n = b.i_end - b.i_begin;
  if (n <= 0) return;
  k_end_step<<<grid_for(n, 128), 128, 0, s>>>(b);
}

void launch_prim2con_f64(const Params& P, const double* V, double* U, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  k_prim2con<<<grid_for(n, 256), 256, 0, s>>>(P, V, U, n);
}

void launch_prim_Z_f64(const Params& P, const double* V, double* Z, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  k_prim_Z<<<grid_for(n, 256), 256, 0, s>>>(P, V, Z, n);
}

void launch_con2prim_f64(const Params& P, const double* U, const double* Zg, double* V,
                         int32_t* status, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  k_con2prim<<<grid_for(n, 128), 128, 0, s>>>(P, U, Zg, V, status, n);
}

void launch_implicit_f64(const Params& P, const Batch& b, double hdt, const double* Us,
                         const double* Zg, const double* kappa, const double* sigma, double* U,
                         double* V, int32_t* status, cudaStream_t s) {
  if (b.ncells <= 0) return;
  k_implicit<<<grid_for(b.ncells, kCellThreads), kCellThreads, 0, s>>>(P, b, hdt, Us, Zg, kappa,
                                                                       sigma, U, V, status);
}

}  // namespace rr
