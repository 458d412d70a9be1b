// rrmhd_api.cu -- C ABI of librrmhd (declared in include/rrmhd.h): context and
// batch tables, device state, CUDA-graph stepping, host-buffer entry.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "../../include/rrmhd.h"
#include "batch.h"

using rr::Batch;
using rr::InstDesc;
using rr::Params;
using rr::StageArgs;

struct Lane {
  Batch b;                      // the lane's instance / cell / face ranges
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // one per value of rrmhd_ctx::cur
};

struct rrmhd_ctx {
  rrmhd_opts opts;
  Params P;
  cudaStream_t stream = nullptr;      // caller's stream (work is enqueued here)
  cudaStream_t cap_stream = nullptr;  // private stream used only to capture the step graph
  int n_inst = 0;
  std::vector<InstDesc> inst;
  std::vector<int64_t> cell_off;
  std::vector<int64_t> face_off;  // [3][n_inst+1]
  int64_t ncells = 0, nfaces = 0;
  int64_t dir_base[4] = {0, 0, 0, 0};
  // device
  InstDesc* d_inst = nullptr;
  int64_t* d_cell_off = nullptr;
  int64_t* d_face_off = nullptr;
  double *U0 = nullptr, *Ua = nullptr, *Ub = nullptr;
  double *V0 = nullptr, *Va = nullptr, *Vb = nullptr;
  double *kappa = nullptr, *sigma = nullptr, *Fhat = nullptr;
  uint8_t* bad = nullptr;  // admissibility-fallback flags, one per cell
  double* jc = nullptr;    // per-cell Jacobian cache of the implicit solve, [17][ncells]
  int cur = 0;             // the state lives in (U0,V0) when 0, in (Ua,Va) when 1
  double *t = nullptr, *t_end = nullptr, *dt = nullptr;
  unsigned long long* smax = nullptr;
  int* status = nullptr;
  std::vector<Lane> lanes;
  cudaEvent_t fork = nullptr;
  std::string err;
};

namespace {

double* cur_U(const rrmhd_ctx* c) { return c->cur ? c->Ua : c->U0; }
double* cur_V(const rrmhd_ctx* c) { return c->cur ? c->Va : c->V0; }

rrmhd_status set_err(const rrmhd_ctx* c, rrmhd_status s, const std::string& msg) {
  if (c) const_cast<rrmhd_ctx*>(c)->err = msg;
  return s;
}

rrmhd_status cuda_check(const rrmhd_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return RRMHD_OK;
  return set_err(c, e == cudaErrorMemoryAllocation ? RRMHD_ENOMEM : RRMHD_ECUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

#define RR_CUDA(ctx, expr)                                     \
  do {                                                         \
    rrmhd_status _s = cuda_check((ctx), (expr), #expr);        \
    if (_s != RRMHD_OK) return _s;                             \
  } while (0)

Params make_params(const rrmhd_opts& o) {
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
  P.gfac = o.gamma / (o.gamma - 1.0);
  P.gm1g = (o.gamma - 1.0) / o.gamma;
  return P;
}

Batch batch_of(const rrmhd_ctx* c) {
  Batch b;
  b.n_inst = c->n_inst;
  b.ncells = c->ncells;
  b.nfaces = c->nfaces;
  for (int d = 0; d < 4; ++d) b.dir_base[d] = c->dir_base[d];
  b.inst = c->d_inst;
  b.cell_off = c->d_cell_off;
  b.face_off = c->d_face_off;
  b.st.t = c->t;
  b.st.t_end = c->t_end;
  b.st.dt = c->dt;
  b.st.smax = c->smax;
  b.st.status = c->status;
  b.i_begin = 0;
  b.i_end = c->n_inst;
  b.c_begin = 0;
  b.c_end = c->ncells;
  for (int d = 0; d < 3; ++d) {
    b.f_begin[d] = c->dir_base[d];
    b.f_count[d] = c->dir_base[d + 1] - c->dir_base[d];
  }
  return b;
}

// Batch restricted to instances [i0, i1).
Batch sub_batch(const rrmhd_ctx* c, int i0, int i1) {
  Batch b = batch_of(c);
  b.i_begin = i0;
  b.i_end = i1;
  b.c_begin = c->cell_off[i0];
  b.c_end = c->cell_off[i1];
  for (int d = 0; d < 3; ++d) {
    const int64_t* fo = &c->face_off[(size_t)d * (c->n_inst + 1)];
    b.f_begin[d] = c->dir_base[d] + fo[i0];
    b.f_count[d] = fo[i1] - fo[i0];
  }
  return b;
}

StageArgs stage_args(const rrmhd_ctx* c, const Batch& b, int stage, const double* U0,
                     const double* V0, const double* Us, const double* Vs, double* Uout,
                     double* Vout) {
  StageArgs a;
  a.P = c->P;
  a.b = b;
  a.stage = stage;
  a.U0 = U0;
  a.V0 = V0;
  a.Us = Us;
  a.Vs = Vs;
  a.kappa = c->kappa;
  a.sigma = c->sigma;
  a.Fhat = c->Fhat;
  a.Fhat32 = reinterpret_cast<float*>(c->Fhat);  // FP32-bulk: same buffer, FP32 entries
  a.fstride = c->nfaces;
  a.out_base = 0;
  a.check_active = 1;
  a.Uout = Uout;
  a.Vout = Vout;
  a.cell_status = nullptr;
  a.bad = c->bad;
  a.jc = c->jc;
  return a;
}

// The three launch groups of one stage in the context's precision.
void launch_stage(const rrmhd_ctx* c, const StageArgs& a, cudaStream_t s) {
  if (c->opts.precision == RRMHD_FP32_BULK) {
    rr::launch_faces_f32(a, s);
    rr::launch_cells_f32(a, s);
    rr::launch_fallback_f32(a, s);
  } else {
    rr::launch_faces_f64(a, s);
    rr::launch_cells_f64(a, s);
    rr::launch_fallback_f64(a, s);
  }
}

// One IMEX-RK3 step of the instances of b, from the state in buffer set
// A = S[cur] into B = S[1-cur], with C = (Ub,Vb) for stage 2:
// stage 1 A -> B, stage 2 (B; A) -> C, stage 3 (C; A) -> B.  No stage writes its
// inputs, so the admissibility fallback can re-read them.  Launches: begin,
// 3 x {faces, cells, fallback faces, fallback cells}, end.
void enqueue_step(const rrmhd_ctx* c, const Batch& b, int cur, cudaStream_t s) {
  double* AU = cur ? c->Ua : c->U0;
  double* AV = cur ? c->Va : c->V0;
  double* BU = cur ? c->U0 : c->Ua;
  double* BV = cur ? c->V0 : c->Va;
  rr::launch_begin_step(c->P, b, s);
  const StageArgs s1 = stage_args(c, b, 1, AU, AV, AU, AV, BU, BV);
  const StageArgs s2 = stage_args(c, b, 2, AU, AV, BU, BV, c->Ub, c->Vb);
  const StageArgs s3 = stage_args(c, b, 3, AU, AV, c->Ub, c->Vb, BU, BV);
  for (const StageArgs* a : {&s1, &s2, &s3}) launch_stage(c, *a, s);
  rr::launch_end_step(b, s);
}

bool grid_ok(const rrmhd_grid& g, std::string& why) {
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

template <class T>
rrmhd_status dalloc(rrmhd_ctx* c, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cuda_check(c, cudaMalloc((void**)p, count * sizeof(T)), "cudaMalloc");
}

}  // namespace

extern "C" {

void rrmhd_default_opts(rrmhd_opts* o) {
  if (!o) return;
  o->gamma = 5.0 / 3.0;
  o->a_rad = 1.0;
  o->cfl = 0.4;
  o->pvm_eps = 1e-8;
  o->recon = RRMHD_RECON_VANLEER;
  o->beta_mode = 1;
  o->precision = RRMHD_FP64;
  o->c2p_maxit = 60;
  o->imp_maxit = 50;
  o->imp_tol = 1e-10;
  o->lanes = 8;
}

void rrmhd_destroy(rrmhd_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  for (Lane& L : c->lanes) {
    if (L.stream) cudaStreamSynchronize(L.stream);
    for (cudaGraphExec_t g : L.graph)
      if (g) cudaGraphExecDestroy(g);
    if (L.done) cudaEventDestroy(L.done);
    if (L.stream) cudaStreamDestroy(L.stream);
  }
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  void* bufs[] = {c->d_inst, c->d_cell_off, c->d_face_off, c->U0, c->Ua, c->Ub, c->V0,
                  c->Va,     c->Vb,         c->kappa,      c->sigma, c->Fhat, c->t, c->t_end,
                  c->dt,     c->smax,       c->status, c->bad,   c->jc};
  for (void* p : bufs)
    if (p) cudaFree(p);
  delete c;
}

rrmhd_status rrmhd_create(int n_inst, const rrmhd_grid* grids, const rrmhd_opts* opts,
                          void* cuda_stream, rrmhd_ctx** out) {
  if (!out) return RRMHD_EINVAL;
  *out = nullptr;
  if (n_inst < 1 || !grids || !opts) return RRMHD_EINVAL;
  const rrmhd_opts& o = *opts;
  if (!(o.gamma > 1.0) || !(o.a_rad >= 0.0) || !(o.cfl > 0.0) || !(o.pvm_eps > 0.0) ||
      o.recon < 0 || o.recon > 3 || o.c2p_maxit < 1 || o.imp_maxit < 1 || !(o.imp_tol > 0.0) ||
      (o.precision != RRMHD_FP64 && o.precision != RRMHD_FP32_BULK) || o.lanes < 1)
    return RRMHD_EINVAL;
  std::string why;
  for (int i = 0; i < n_inst; ++i)
    if (!grid_ok(grids[i], why)) return RRMHD_EINVAL;

  rrmhd_ctx* c = new rrmhd_ctx();
  c->opts = o;
  c->P = make_params(o);
  c->stream = (cudaStream_t)cuda_stream;
  c->n_inst = n_inst;
  c->inst.resize(n_inst);
  c->cell_off.assign(n_inst + 1, 0);
  c->face_off.assign(3 * (size_t)(n_inst + 1), 0);
  for (int i = 0; i < n_inst; ++i) {
    const rrmhd_grid& g = grids[i];
    InstDesc& I = c->inst[i];
    I.ndim = g.ndim;
    for (int d = 0; d < 3; ++d) {
      I.n[d] = g.n[d];
      I.bc[d] = g.bc[d];
      I.dx[d] = d < g.ndim ? g.dx[d] : 1.0;
    }
    const int64_t nc = (int64_t)g.n[0] * g.n[1] * g.n[2];
    I.cell_off = c->cell_off[i];
    c->cell_off[i + 1] = c->cell_off[i] + nc;
    for (int d = 0; d < 3; ++d) {
      int64_t nf = 0;
      if (d < g.ndim) {
        int m[3] = {g.n[0], g.n[1], g.n[2]};
        m[d] += 1;
        nf = (int64_t)m[0] * m[1] * m[2];
      }
      int64_t* fo = &c->face_off[(size_t)d * (n_inst + 1)];
      I.face_off[d] = fo[i];
      fo[i + 1] = fo[i] + nf;
    }
  }
  c->ncells = c->cell_off[n_inst];
  for (int d = 0; d < 3; ++d)
    c->dir_base[d + 1] = c->dir_base[d] + c->face_off[(size_t)d * (n_inst + 1) + n_inst];
  c->nfaces = c->dir_base[3];

  rrmhd_status s = RRMHD_OK;
  const size_t N12 = (size_t)12 * c->ncells;
  auto A = [&](rrmhd_status r) {
    if (s == RRMHD_OK) s = r;
  };
  A(dalloc(c, &c->d_inst, n_inst));
  A(dalloc(c, &c->d_cell_off, n_inst + 1));
  A(dalloc(c, &c->d_face_off, 3 * (size_t)(n_inst + 1)));
  for (double** p : {&c->U0, &c->Ua, &c->Ub, &c->V0, &c->Va, &c->Vb}) A(dalloc(c, p, N12));
  A(dalloc(c, &c->kappa, c->ncells));
  A(dalloc(c, &c->sigma, c->ncells));
  A(dalloc(c, &c->Fhat, (size_t)12 * c->nfaces));
  A(dalloc(c, &c->t, n_inst));
  A(dalloc(c, &c->t_end, n_inst));
  A(dalloc(c, &c->dt, n_inst));
  A(dalloc(c, &c->smax, n_inst));
  A(dalloc(c, &c->status, n_inst));
  A(dalloc(c, &c->bad, (size_t)c->ncells));
  A(dalloc(c, &c->jc, (size_t)17 * c->ncells));
  if (s == RRMHD_OK) {
    cudaStream_t st = c->stream;
    A(cuda_check(c, cudaMemcpyAsync(c->d_inst, c->inst.data(), sizeof(InstDesc) * n_inst,
                                    cudaMemcpyHostToDevice, st), "upload"));
    A(cuda_check(c, cudaMemcpyAsync(c->d_cell_off, c->cell_off.data(),
                                    sizeof(int64_t) * (n_inst + 1), cudaMemcpyHostToDevice, st),
                 "upload"));
    A(cuda_check(c, cudaMemcpyAsync(c->d_face_off, c->face_off.data(),
                                    sizeof(int64_t) * 3 * (n_inst + 1), cudaMemcpyHostToDevice, st),
                 "upload"));
    std::vector<double> zeros(n_inst, 0.0), inf(n_inst, std::numeric_limits<double>::infinity());
    A(cuda_check(c, cudaMemcpyAsync(c->t, zeros.data(), sizeof(double) * n_inst,
                                    cudaMemcpyHostToDevice, st), "upload"));
    A(cuda_check(c, cudaMemcpyAsync(c->t_end, inf.data(), sizeof(double) * n_inst,
                                    cudaMemcpyHostToDevice, st), "upload"));
    A(cuda_check(c, cudaMemsetAsync(c->dt, 0, sizeof(double) * n_inst, st), "memset"));
    A(cuda_check(c, cudaMemsetAsync(c->smax, 0, sizeof(unsigned long long) * n_inst, st), "memset"));
    A(cuda_check(c, cudaMemsetAsync(c->status, 0, sizeof(int) * n_inst, st), "memset"));
    A(cuda_check(c, cudaMemsetAsync(c->kappa, 0, sizeof(double) * c->ncells, st), "memset"));
    A(cuda_check(c, cudaMemsetAsync(c->sigma, 0, sizeof(double) * c->ncells, st), "memset"));
    A(cuda_check(c, cudaMemsetAsync(c->U0, 0, sizeof(double) * N12, st), "memset"));
    A(cuda_check(c, cudaMemsetAsync(c->V0, 0, sizeof(double) * N12, st), "memset"));
    A(cuda_check(c, cudaMemsetAsync(c->bad, 0, (size_t)c->ncells, st), "memset"));
    A(cuda_check(c, cudaMemsetAsync(c->jc, 0, sizeof(double) * 17 * c->ncells, st), "memset"));
    A(cuda_check(c, cudaStreamSynchronize(st), "sync"));  // host vectors go out of scope
  }
  if (s == RRMHD_OK) {
    // lanes: contiguous instance ranges of about equal cell count
    const int L = std::min(o.lanes, n_inst);
    int i0 = 0;
    for (int l = 0; l < L && s == RRMHD_OK; ++l) {
      int i1 = n_inst;
      if (l < L - 1) {
        const int64_t target = (c->ncells * (l + 1)) / L;
        i1 = i0 + 1;
        while (i1 < n_inst - (L - 1 - l) && c->cell_off[i1] < target) ++i1;
      }
      Lane lane;
      lane.b = sub_batch(c, i0, i1);
      A(cuda_check(c, cudaStreamCreateWithFlags(&lane.stream, cudaStreamNonBlocking), "stream"));
      A(cuda_check(c, cudaEventCreateWithFlags(&lane.done, cudaEventDisableTiming), "event"));
      c->lanes.push_back(lane);
      i0 = i1;
    }
    A(cuda_check(c, cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming), "event"));
  }
  if (s != RRMHD_OK) {
    rrmhd_destroy(c);
    return s;
  }
  *out = c;
  return RRMHD_OK;
}

int rrmhd_num_instances(const rrmhd_ctx* c) { return c ? c->n_inst : 0; }
int64_t rrmhd_num_cells(const rrmhd_ctx* c) { return c ? c->ncells : 0; }
int64_t rrmhd_num_faces(const rrmhd_ctx* c, int dir) {
  if (!c || dir < 0 || dir > 2) return 0;
  return c->dir_base[dir + 1] - c->dir_base[dir];
}

rrmhd_status rrmhd_cell_offsets(const rrmhd_ctx* c, int64_t* off) {
  if (!c || !off) return RRMHD_EINVAL;
  std::memcpy(off, c->cell_off.data(), sizeof(int64_t) * (c->n_inst + 1));
  return RRMHD_OK;
}

rrmhd_status rrmhd_face_offsets(const rrmhd_ctx* c, int dir, int64_t* off) {
  if (!c || !off || dir < 0 || dir > 2) return RRMHD_EINVAL;
  std::memcpy(off, &c->face_off[(size_t)dir * (c->n_inst + 1)], sizeof(int64_t) * (c->n_inst + 1));
  return RRMHD_OK;
}

rrmhd_status rrmhd_set_opacity(rrmhd_ctx* c, const double* kappa, const double* sigma) {
  if (!c || !kappa || !sigma) return set_err(c, RRMHD_EINVAL, "null argument");
  RR_CUDA(c, cudaMemcpyAsync(c->kappa, kappa, sizeof(double) * c->ncells, cudaMemcpyDeviceToDevice,
                             c->stream));
  RR_CUDA(c, cudaMemcpyAsync(c->sigma, sigma, sizeof(double) * c->ncells, cudaMemcpyDeviceToDevice,
                             c->stream));
  return RRMHD_OK;
}

static rrmhd_status refresh_state(rrmhd_ctx* c) {
  const Batch b = batch_of(c);
  rr::launch_prim2con_f64(c->P, cur_V(c), cur_U(c), c->ncells, c->stream);
  RR_CUDA(c, cudaMemsetAsync(c->smax, 0, sizeof(unsigned long long) * c->n_inst, c->stream));
  RR_CUDA(c, cudaMemsetAsync(c->status, 0, sizeof(int) * c->n_inst, c->stream));
  RR_CUDA(c, cudaMemsetAsync(c->dt, 0, sizeof(double) * c->n_inst, c->stream));
  // a new state starts with an empty Jacobian cache (validity plane)
  RR_CUDA(c, cudaMemsetAsync(c->jc + (size_t)16 * c->ncells, 0, sizeof(double) * c->ncells, c->stream));
  rr::launch_signal_f64(c->P, b, cur_V(c), c->stream);
  RR_CUDA(c, cudaGetLastError());
  return RRMHD_OK;
}

rrmhd_status rrmhd_set_state(rrmhd_ctx* c, const double* V) {
  if (!c || !V) return set_err(c, RRMHD_EINVAL, "null argument");
  RR_CUDA(c, cudaMemcpyAsync(cur_V(c), V, sizeof(double) * 12 * c->ncells,
                             cudaMemcpyDeviceToDevice, c->stream));
  return refresh_state(c);
}

rrmhd_status rrmhd_get_state(const rrmhd_ctx* c, double* U, double* V) {
  if (!c) return RRMHD_EINVAL;
  if (U)
    RR_CUDA(c, cudaMemcpyAsync(U, cur_U(c), sizeof(double) * 12 * c->ncells,
                               cudaMemcpyDeviceToDevice, c->stream));
  if (V)
    RR_CUDA(c, cudaMemcpyAsync(V, cur_V(c), sizeof(double) * 12 * c->ncells,
                               cudaMemcpyDeviceToDevice, c->stream));
  return RRMHD_OK;
}

rrmhd_status rrmhd_set_times(rrmhd_ctx* c, const double* t, const double* t_end) {
  if (!c || !t || !t_end) return set_err(c, RRMHD_EINVAL, "null argument");
  RR_CUDA(c, cudaMemcpyAsync(c->t, t, sizeof(double) * c->n_inst, cudaMemcpyHostToDevice, c->stream));
  RR_CUDA(c, cudaMemcpyAsync(c->t_end, t_end, sizeof(double) * c->n_inst, cudaMemcpyHostToDevice,
                             c->stream));
  RR_CUDA(c, cudaStreamSynchronize(c->stream));  // pageable host sources
  RR_CUDA(c, cudaMemsetAsync(c->smax, 0, sizeof(unsigned long long) * c->n_inst, c->stream));
  rr::launch_signal_f64(c->P, batch_of(c), cur_V(c), c->stream);
  RR_CUDA(c, cudaGetLastError());
  return RRMHD_OK;
}

rrmhd_status rrmhd_get_times(const rrmhd_ctx* c, double* t, double* dt_last) {
  if (!c) return RRMHD_EINVAL;
  if (t) RR_CUDA(c, cudaMemcpyAsync(t, c->t, sizeof(double) * c->n_inst, cudaMemcpyDeviceToHost, c->stream));
  if (dt_last)
    RR_CUDA(c, cudaMemcpyAsync(dt_last, c->dt, sizeof(double) * c->n_inst, cudaMemcpyDeviceToHost,
                               c->stream));
  RR_CUDA(c, cudaStreamSynchronize(c->stream));
  return RRMHD_OK;
}

rrmhd_status rrmhd_get_inst_status(const rrmhd_ctx* c, int32_t* status) {
  if (!c || !status) return RRMHD_EINVAL;
  RR_CUDA(c, cudaMemcpyAsync(status, c->status, sizeof(int) * c->n_inst, cudaMemcpyDeviceToHost,
                             c->stream));
  RR_CUDA(c, cudaStreamSynchronize(c->stream));
  return RRMHD_OK;
}

static rrmhd_status build_step_graph(rrmhd_ctx* c, Lane& L, int cur) {
  if (L.graph[cur]) return RRMHD_OK;
  if (!c->cap_stream)
    RR_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  RR_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  enqueue_step(c, L.b, cur, c->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_check(c, e, "cudaStreamEndCapture");
  }
  e = cudaGraphInstantiate(&L.graph[cur], g, 0);
  cudaGraphDestroy(g);
  return cuda_check(c, e, "cudaGraphInstantiate");
}

// Each step: the lanes fork from the caller's stream, run their step graph
// concurrently on their own streams, and join back into it.
rrmhd_status rrmhd_imex_step(rrmhd_ctx* c, int nsteps) {
  if (!c || nsteps < 0) return set_err(c, RRMHD_EINVAL, "bad argument");
  for (int k = 0; k < nsteps; ++k) {
    RR_CUDA(c, cudaEventRecord(c->fork, c->stream));
    for (Lane& L : c->lanes) {
      rrmhd_status s = build_step_graph(c, L, c->cur);
      if (s != RRMHD_OK) return s;
      RR_CUDA(c, cudaStreamWaitEvent(L.stream, c->fork, 0));
      RR_CUDA(c, cudaGraphLaunch(L.graph[c->cur], L.stream));
      RR_CUDA(c, cudaEventRecord(L.done, L.stream));
    }
    for (Lane& L : c->lanes) RR_CUDA(c, cudaStreamWaitEvent(c->stream, L.done, 0));
    c->cur ^= 1;
  }
  return RRMHD_OK;
}

rrmhd_status rrmhd_imex_step_host(rrmhd_ctx* c, const double* V_in, double* V_out, int nsteps) {
  if (!c || !V_in || !V_out || nsteps < 0) return set_err(c, RRMHD_EINVAL, "bad argument");
  const size_t bytes = sizeof(double) * 12 * c->ncells;
  RR_CUDA(c, cudaMemcpyAsync(cur_V(c), V_in, bytes, cudaMemcpyHostToDevice, c->stream));
  rrmhd_status s = refresh_state(c);
  if (s != RRMHD_OK) return s;
  s = rrmhd_imex_step(c, nsteps);
  if (s != RRMHD_OK) return s;
  RR_CUDA(c, cudaMemcpyAsync(V_out, cur_V(c), bytes, cudaMemcpyDeviceToHost, c->stream));
  RR_CUDA(c, cudaStreamSynchronize(c->stream));
  return RRMHD_OK;
}

rrmhd_status rrmhd_prim2con(rrmhd_ctx* c, const double* V, double* U, int64_t n) {
  if (!c || !V || !U || n < 0) return set_err(c, RRMHD_EINVAL, "bad argument");
  rr::launch_prim2con_f64(c->P, V, U, n, c->stream);
  RR_CUDA(c, cudaGetLastError());
  return RRMHD_OK;
}

rrmhd_status rrmhd_prim_z(rrmhd_ctx* c, const double* V, double* Z, int64_t n) {
  if (!c || !V || !Z || n < 0) return set_err(c, RRMHD_EINVAL, "bad argument");
  rr::launch_prim_Z_f64(c->P, V, Z, n, c->stream);
  RR_CUDA(c, cudaGetLastError());
  return RRMHD_OK;
}

rrmhd_status rrmhd_con2prim(rrmhd_ctx* c, const double* U, const double* Zguess, double* V,
                            int32_t* status, int64_t n) {
  if (!c || !U || !V || n < 0) return set_err(c, RRMHD_EINVAL, "bad argument");
  rr::launch_con2prim_f64(c->P, U, Zguess, V, status, n, c->stream);
  RR_CUDA(c, cudaGetLastError());
  return RRMHD_OK;
}

rrmhd_status rrmhd_flux_sweep(rrmhd_ctx* c, int dir, double* Fhat) {
  if (!c || !Fhat || dir < 0 || dir > 2) return set_err(c, RRMHD_EINVAL, "bad argument");
  Batch b = batch_of(c);
  for (int d = 0; d < 3; ++d) b.f_count[d] = (d == dir) ? b.f_count[d] : 0;
  StageArgs a = stage_args(c, b, 0, cur_U(c), cur_V(c), cur_U(c), cur_V(c), nullptr, nullptr);
  a.check_active = 0;
  const int64_t nd = c->dir_base[dir + 1] - c->dir_base[dir];
  if (c->opts.precision == RRMHD_FP32_BULK) {
    // FP32 fluxes into the context's face buffer, widened into the caller's array
    rr::launch_faces_f32(a, c->stream);
    rr::launch_widen_f32(a.Fhat32, c->nfaces, c->dir_base[dir], nd, Fhat, c->stream);
  } else {
    a.Fhat = Fhat;
    a.fstride = nd;
    a.out_base = c->dir_base[dir];
    rr::launch_faces_f64(a, c->stream);
  }
  RR_CUDA(c, cudaGetLastError());
  return RRMHD_OK;
}

rrmhd_status rrmhd_implicit_source(rrmhd_ctx* c, double hdt, const double* Ustar,
                                   const double* Zguess, double* U, double* V, int32_t* status) {
  if (!c || !Ustar || !U || !V || !(hdt >= 0.0)) return set_err(c, RRMHD_EINVAL, "bad argument");
  rr::launch_implicit_f64(c->P, batch_of(c), hdt, Ustar, Zguess, c->kappa, c->sigma, U, V, status,
                          c->stream);
  RR_CUDA(c, cudaGetLastError());
  return RRMHD_OK;
}

int rrmhd_launches_per_step(const rrmhd_ctx* c) {
  return c ? (int)c->lanes.size() * (2 + 3 * 4) : 0;
}

rrmhd_status rrmhd_profile_step(rrmhd_ctx* c, double* ms) {
  if (!c || !ms) return set_err(c, RRMHD_EINVAL, "bad argument");
  const int cur = c->cur;
  const Batch b = batch_of(c);
  double* AU = cur ? c->Ua : c->U0;
  double* AV = cur ? c->Va : c->V0;
  double* BU = cur ? c->U0 : c->Ua;
  double* BV = cur ? c->V0 : c->Va;
  const StageArgs st[3] = {stage_args(c, b, 1, AU, AV, AU, AV, BU, BV),
                           stage_args(c, b, 2, AU, AV, BU, BV, c->Ub, c->Vb),
                           stage_args(c, b, 3, AU, AV, c->Ub, c->Vb, BU, BV)};
  cudaEvent_t ev[14];
  for (auto& e : ev) RR_CUDA(c, cudaEventCreate(&e));
  cudaStream_t s = c->stream;
  int k = 0;
  cudaEventRecord(ev[k++], s);
  rr::launch_begin_step(c->P, b, s);
  cudaEventRecord(ev[k++], s);
  const bool f32 = c->opts.precision == RRMHD_FP32_BULK;
  for (int i = 0; i < 3; ++i) {
    if (f32) rr::launch_faces_f32(st[i], s); else rr::launch_faces_f64(st[i], s);
    cudaEventRecord(ev[k++], s);
    if (f32) rr::launch_cells_f32(st[i], s); else rr::launch_cells_f64(st[i], s);
    cudaEventRecord(ev[k++], s);
    if (f32) rr::launch_fallback_f32(st[i], s); else rr::launch_fallback_f64(st[i], s);
    cudaEventRecord(ev[k++], s);
  }
  rr::launch_end_step(b, s);
  cudaEventRecord(ev[k++], s);
  rrmhd_status rc = cuda_check(c, cudaEventSynchronize(ev[k - 1]), "profile");
  if (rc == RRMHD_OK) {
    float t;
    for (int q = 0; q < 4; ++q) ms[q] = 0.0;
    cudaEventElapsedTime(&t, ev[0], ev[1]);
    ms[3] += t;
    for (int i = 0; i < 3; ++i) {
      const int o = 1 + 3 * i;
      cudaEventElapsedTime(&t, ev[o], ev[o + 1]);
      ms[0] += t;
      cudaEventElapsedTime(&t, ev[o + 1], ev[o + 2]);
      ms[1] += t;
      cudaEventElapsedTime(&t, ev[o + 2], ev[o + 3]);
      ms[2] += t;
    }
    cudaEventElapsedTime(&t, ev[10], ev[11]);
    ms[3] += t;
    c->cur ^= 1;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  return rc;
}

const char* rrmhd_last_error(const rrmhd_ctx* c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"
