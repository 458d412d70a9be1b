// engine.h -- host-side plumbing shared by the context API and the serving loop:
// validation of grids and options, the packed layout of a list of grids, the
// device buffers of a batch, the stage arguments, and the enqueueing of one
// IMEX-RK3 step (Sec. 3.1) of a contiguous range of instances.  Internal to
// librrmhd.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include "../../include/rrmhd.h"
#include "batch.h"
#include "launch_shape.cuh"

namespace rr {

inline Params make_params(const rrmhd_opts& o) {
  Params P;
  P.gamma = o.gamma;
  P.a_rad = o.a_rad;
  P.cfl = o.cfl;
  P.pvm_eps = o.pvm_eps;
  P.recon = o.recon;
  P.beta_mode = o.beta_mode;
  P.c2p_maxit = o.c2p_maxit;
  P.imp_maxit = o.imp_maxit;
  P.imp_tol = o.imp_tol;
  P.pvm_k = o.pvm_k;
  P.pvm_products = o.pvm_products;
  P.solver = o.solver;
  P.gfac = o.gamma / (o.gamma - 1.0);
  P.gm1g = (o.gamma - 1.0) / o.gamma;
  return P;
}

inline bool opts_ok(const rrmhd_opts& o) {
  return o.gamma > 1.0 && o.a_rad >= 0.0 && o.cfl > 0.0 && o.pvm_eps > 0.0 && o.recon >= 0 &&
         o.beta_mode >= 0 && o.beta_mode <= 2 &&
         o.recon <= 3 && o.c2p_maxit >= 1 && o.imp_maxit >= 1 && o.imp_tol > 0.0 &&
         (o.precision == RRMHD_FP64 || o.precision == RRMHD_FP32_BULK) && o.lanes >= 1 &&
         (o.pvm_k == 3 || o.pvm_k == 4) && (o.pvm_products == 0 || o.pvm_products == 1) &&
         (o.solver == RRMHD_SOLVER_PVM || o.solver == RRMHD_SOLVER_RADHLL) &&
         (o.ct == 0 || o.ct == 1) && o.closure == RRMHD_CLOSURE_M1;
}

inline bool grid_ok(const rrmhd_grid& g, std::string& why) {
  if (g.ndim < 1 || g.ndim > 3) {
    why = "ndim must be 1, 2 or 3";
    return false;
  }
  for (int d = 0; d < 3; ++d) {
    if (g.n[d] < 1) {
      why = "n[d] must be >= 1";
      return false;
    }
    if (d >= g.ndim && g.n[d] != 1) {
      why = "unused directions must have n = 1";
      return false;
    }
    if (d < g.ndim && !(g.dx[d] > 0.0)) {
      why = "dx must be > 0";
      return false;
    }
    if (g.bc[d] != RRMHD_BC_OUTFLOW && g.bc[d] != RRMHD_BC_PERIODIC) {
      why = "bc must be RRMHD_BC_OUTFLOW or RRMHD_BC_PERIODIC";
      return false;
    }
  }
  if ((int64_t)g.n[0] * g.n[1] * g.n[2] > (int64_t)1 << 34) {
    why = "grid too large";
    return false;
  }
  return true;
}

inline int64_t grid_cells(const rrmhd_grid& g) { return (int64_t)g.n[0] * g.n[1] * g.n[2]; }

// Faces normal to direction d of a grid (0 for unused directions).
inline int64_t grid_faces(const rrmhd_grid& g, int d) {
  if (d >= g.ndim) return 0;
  int64_t m[3] = {g.n[0], g.n[1], g.n[2]};
  m[d] += 1;
  return m[0] * m[1] * m[2];
}

inline int64_t grid_faces(const rrmhd_grid& g) {
  return grid_faces(g, 0) + grid_faces(g, 1) + grid_faces(g, 2);
}

// Edges along e of a grid for constrained transport: 2D grids have edges along z
// only, 3D grids along all three; 1D grids none.
inline int64_t grid_edges(const rrmhd_grid& g, int e) {
  if (g.ndim < 2 || (g.ndim == 2 && e != 2)) return 0;
  int64_t c = 1;
  for (int d = 0; d < 3; ++d) c *= g.n[d] + ((d != e && d < g.ndim) ? 1 : 0);
  return c;
}

// Packed layout of a list of instances: cells back to back, faces direction-major
// with per-instance blocks (batch.h).
struct Layout {
  int n_inst = 0;
  std::vector<InstDesc> inst;
  std::vector<int64_t> cell_off;  // [n_inst + 1]
  std::vector<int64_t> face_off;  // [3][n_inst + 1], prefix sums within each direction
  std::vector<int64_t> edge_off;  // [3][n_inst + 1], prefix sums within each edge direction
  int64_t ncells = 0, nfaces = 0, nedges = 0;
  int64_t dir_base[4] = {0, 0, 0, 0};
  int64_t edge_base[4] = {0, 0, 0, 0};
};

inline Layout make_layout(const rrmhd_grid* grids, int n_inst) {
  Layout L;
  L.n_inst = n_inst;
  L.inst.resize(n_inst);
  L.cell_off.assign(n_inst + 1, 0);
  L.face_off.assign(3 * (size_t)(n_inst + 1), 0);
  L.edge_off.assign(3 * (size_t)(n_inst + 1), 0);
  for (int i = 0; i < n_inst; ++i) {
    const rrmhd_grid& g = grids[i];
    InstDesc& I = L.inst[i];
    I.ndim = g.ndim;
    for (int d = 0; d < 3; ++d) {
      I.n[d] = g.n[d];
      I.bc[d] = g.bc[d];
      I.dx[d] = d < g.ndim ? g.dx[d] : 1.0;
    }
    I.cell_off = L.cell_off[i];
    L.cell_off[i + 1] = L.cell_off[i] + grid_cells(g);
    for (int d = 0; d < 3; ++d) {
      int64_t* fo = &L.face_off[(size_t)d * (n_inst + 1)];
      I.face_off[d] = fo[i];
      fo[i + 1] = fo[i] + grid_faces(g, d);
      int64_t* eo = &L.edge_off[(size_t)d * (n_inst + 1)];
      I.edge_off[d] = eo[i];
      eo[i + 1] = eo[i] + grid_edges(g, d);
    }
  }
  L.ncells = L.cell_off[n_inst];
  for (int d = 0; d < 3; ++d)
    L.dir_base[d + 1] = L.dir_base[d] + L.face_off[(size_t)d * (n_inst + 1) + n_inst];
  L.nfaces = L.dir_base[3];
  for (int d = 0; d < 3; ++d)
    L.edge_base[d + 1] = L.edge_base[d] + L.edge_off[(size_t)d * (n_inst + 1) + n_inst];
  L.nedges = L.edge_base[3];
  return L;
}

// Contiguous instance ranges [first, second) of about equal cell count.
inline std::vector<std::pair<int, int>> lane_ranges(const std::vector<int64_t>& cell_off,
                                                    int n_inst, int lanes) {
  std::vector<std::pair<int, int>> r;
  if (n_inst <= 0) return r;
  const int L = std::min(lanes, n_inst);
  const int64_t ncells = cell_off[n_inst];
  int i0 = 0;
  for (int l = 0; l < L; ++l) {
    int i1 = n_inst;
    if (l < L - 1) {
      const int64_t target = (ncells * (l + 1)) / L;
      i1 = i0 + 1;
      while (i1 < n_inst - (L - 1 - l) && cell_off[i1] < target) ++i1;
    }
    r.emplace_back(i0, i1);
    i0 = i1;
  }
  return r;
}

// Device buffers of a batch.  The state lives in (U0,V0) or (Ua,Va); (Ub,Vb)
// holds stage 2.  Plane strides are the batch's ncells (cells) and nfaces (Fhat).
struct DeviceBufs {
  double *U0 = nullptr, *Ua = nullptr, *Ub = nullptr;
  double *V0 = nullptr, *Va = nullptr, *Vb = nullptr;
  double *kappa = nullptr, *sigma = nullptr;
  double* Fhat = nullptr;  // [12][nfaces] FP64, or [12][nfaces] FP32 in the FP32-bulk form
  uint8_t* bad = nullptr;  // admissibility-fallback flags, one per cell
  double* jc = nullptr;    // per-cell Jacobian cache of the implicit solve, [17][ncells]
  // constrained transport: staggered face field sets (with U0/V0, Ua/Va, Ub/Vb), EMFs
  double *bf0 = nullptr, *bfa = nullptr, *bfb = nullptr, *emf = nullptr;
  // per instance
  InstDesc* inst = nullptr;
  int64_t* cell_off = nullptr;
  int64_t* face_off = nullptr;  // [3][n_inst + 1]
  int64_t* edge_off = nullptr;  // [3][n_inst + 1]
  double *t = nullptr, *t_end = nullptr, *dt = nullptr;
  unsigned long long* smax = nullptr;
  int* status = nullptr;
  double* dt_max = nullptr;        // [1] (contexts)
  long long* bad_cell = nullptr;   // [n_inst] (contexts)
};

// Batch of instances [i0, i1) of a layout whose tables live in B.
inline Batch make_batch(const Layout& L, const DeviceBufs& B, int i0, int i1) {
  Batch b;
  b.n_inst = L.n_inst;
  b.ncells = L.ncells;
  b.nfaces = L.nfaces;
  for (int d = 0; d < 4; ++d) b.dir_base[d] = L.dir_base[d];
  b.inst = B.inst;
  b.cell_off = B.cell_off;
  b.face_off = B.face_off;
  b.edge_off = B.edge_off;
  for (int d = 0; d < 4; ++d) b.edge_base[d] = L.edge_base[d];
  b.st.t = B.t;
  b.st.t_end = B.t_end;
  b.st.dt = B.dt;
  b.st.smax = B.smax;
  b.st.status = B.status;
  b.st.dt_max = B.dt_max;
  b.st.bad_cell = B.bad_cell;
  b.i_begin = i0;
  b.i_end = i1;
  b.c_begin = L.cell_off[i0];
  b.c_end = L.cell_off[i1];
  for (int d = 0; d < 3; ++d) {
    const int64_t* fo = &L.face_off[(size_t)d * (L.n_inst + 1)];
    b.f_begin[d] = L.dir_base[d] + fo[i0];
    b.f_count[d] = fo[i1] - fo[i0];
    const int64_t* eo = &L.edge_off[(size_t)d * (L.n_inst + 1)];
    b.e_begin[d] = L.edge_base[d] + eo[i0];
    b.e_count[d] = eo[i1] - eo[i0];
  }
  return b;
}

inline StageArgs stage_args(const Params& P, const DeviceBufs& B, const Batch& b, int stage,
                            const double* U0, const double* V0, const double* Us,
                            const double* Vs, double* Uout, double* Vout,
                            LaneCounters* cnt = nullptr) {
  StageArgs a;
  a.P = P;
  a.b = b;
  a.stage = stage;
  a.U0 = U0;
  a.V0 = V0;
  a.Us = Us;
  a.Vs = Vs;
  a.kappa = B.kappa;
  a.sigma = B.sigma;
  a.Fhat = B.Fhat;
  a.Fhat32 = reinterpret_cast<float*>(B.Fhat);  // FP32-bulk: same buffer, FP32 entries
  a.fstride = b.nfaces;
  a.out_base = 0;
  a.check_active = 1;
  a.Uout = Uout;
  a.Vout = Vout;
  a.cell_status = nullptr;
  a.bad = B.bad;
  a.fb_pass = 0;  // the main path; launch_fallback sets its passes
  a.flagged = (cnt && stage >= 1) ? cnt->flagged[stage - 1] : nullptr;
  a.jc = B.jc;
  a.work = cnt ? cnt->work : nullptr;
  a.ct = 0;
  a.fp32_fluxes = 0;
  a.b0 = a.bs = nullptr;
  a.bout = nullptr;
  a.emf = B.emf;
  return a;
}

inline void launch_faces(int precision, const StageArgs& a, const LaunchShape& sh, cudaStream_t s) {
  if (precision == RRMHD_FP32_BULK)
    launch_faces_f32(a, sh, s);
  else
    launch_faces_f64(a, sh, s);
}

inline void launch_cells(int precision, const StageArgs& a, const LaunchShape& sh, cudaStream_t s) {
  if (precision == RRMHD_FP32_BULK)
    launch_cells_f32(a, sh, s);
  else
    launch_cells_f64(a, sh, s);
}

// Every pass of the admissibility fallback; a pass with no flagged cell costs
// two short launches that return at once.
inline void launch_fallback(int precision, const StageArgs& a, cudaStream_t s) {
  StageArgs f = a;
  for (f.fb_pass = 1; f.fb_pass <= kFallbackPasses; ++f.fb_pass) {
    if (precision == RRMHD_FP32_BULK)
      launch_fallback_f32(f, s);
    else
      launch_fallback_f64(f, s);
  }
}

// Kernel launches of one step on one lane.
// (constrained transport: EMFs and face field in the main path and in every pass)
inline int launches_per_step(int ct) {
  return 2 + 3 * (2 + 2 * kFallbackPasses + (ct ? 2 + 2 * kFallbackPasses : 0));
}

// The launch groups of one stage in the given precision and shapes: faces, then
// (constrained transport) edge EMFs and the face-field update, cells, fallback.
inline void launch_stage(int precision, const Tuning& tu, const StageArgs& a, cudaStream_t s) {
  launch_faces(precision, a, tu.faces, s);
  if (a.ct) {
    launch_emf_f64(a, s);
    launch_bface_f64(a, s);
  }
  launch_cells(precision, a, tu.cells, s);
  launch_fallback(precision, a, s);
}

inline Tuning default_tuning() { return Tuning{}; }

inline bool tuning_ok(const Tuning& t) {
  return shape_ok(t.faces.block, t.faces.per_thread, t.faces.persistent) &&
         shape_ok(t.cells.block, t.cells.per_thread, t.cells.persistent);
}

// One IMEX-RK3 step of the instances of b, from the state in buffer set
// A = S[cur] into B = S[1-cur], with C = (Ub,Vb) for stage 2:
// stage 1 A -> B, stage 2 (B; A) -> C, stage 3 (C; A) -> B.  No stage writes its
// inputs, so the admissibility fallback can re-read them.  Launches: begin,
// 3 x {faces, [emf, bface,] cells, kFallbackPasses x {fallback faces, [emf,
// bface,] fallback cells}}, end (launches_per_step).  The flag counters are
// zeroed by a memset.
// cnt: this stream's counters (persistent shapes, fallback passes).
// ct: constrained transport on (the face-field sets rotate with the state).
inline void enqueue_step(const Params& P, int precision, const Tuning& tu, const DeviceBufs& B,
                         const Batch& b, int cur, LaneCounters* cnt, cudaStream_t s,
                         int ct = 0) {
  double* AU = cur ? B.Ua : B.U0;
  double* AV = cur ? B.Va : B.V0;
  double* BU = cur ? B.U0 : B.Ua;
  double* BV = cur ? B.V0 : B.Va;
  double* Ab = cur ? B.bfa : B.bf0;
  double* Bb = cur ? B.bf0 : B.bfa;
  launch_begin_step(P, b, s);
  cudaMemsetAsync(cnt->flagged, 0, sizeof(cnt->flagged), s);
  StageArgs s1 = stage_args(P, B, b, 1, AU, AV, AU, AV, BU, BV, cnt);
  StageArgs s2 = stage_args(P, B, b, 2, AU, AV, BU, BV, B.Ub, B.Vb, cnt);
  StageArgs s3 = stage_args(P, B, b, 3, AU, AV, B.Ub, B.Vb, BU, BV, cnt);
  if (ct) {
    s1.ct = s2.ct = s3.ct = 1;
    s1.fp32_fluxes = s2.fp32_fluxes = s3.fp32_fluxes = (precision == RRMHD_FP32_BULK);
    s1.b0 = s2.b0 = s3.b0 = Ab;
    s1.bs = Ab;
    s1.bout = Bb;
    s2.bs = Bb;
    s2.bout = B.bfb;
    s3.bs = B.bfb;
    s3.bout = Bb;
  }
  for (const StageArgs* a : {&s1, &s2, &s3}) launch_stage(precision, tu, *a, s);
  launch_end_step(b, s);
}



}  // namespace rr
