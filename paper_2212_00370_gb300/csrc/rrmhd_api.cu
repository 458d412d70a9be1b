// rrmhd_api.cu -- C ABI of librrmhd (declared in include/rrmhd.h): context and
// batch tables, device state, CUDA-graph stepping, host-buffer entry.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "../../include/rrmhd.h"
#include "batch.h"
#include "engine.h"

using rr::Batch;
using rr::InstDesc;
using rr::Params;
using rr::StageArgs;

struct Lane {
  Batch b;                      // the lane's instance / cell / face ranges
  rr::LaneCounters* cnt = nullptr;  // the lane's counters (persistent shapes, fallback passes)
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // one per value of rrmhd_ctx::cur
};

// Sets *flag when the two arrays differ in any bit (host-buffer entry: is the
// incoming state the context's own?).
__global__ void k_differs(const unsigned long long* __restrict__ a,
                          const unsigned long long* __restrict__ b, int64_t n, int* flag) {
  int diff = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    diff |= (a[i] != b[i]);
  if (__syncthreads_or(diff) && threadIdx.x == 0) atomicOr(flag, 1);
}

struct rrmhd_ctx {
  rrmhd_opts opts;
  Params P;
  cudaStream_t stream = nullptr;      // caller's stream (work is enqueued here)
  cudaStream_t cap_stream = nullptr;  // private stream used only to capture the step graph
  rr::Layout L;                       // packed layout of the instances
  rr::DeviceBufs B;                   // device state and tables
  int cur = 0;                        // the state lives in (U0,V0) when 0, in (Ua,Va) when 1
  rr::Tuning tune;                    // launch shapes
  rr::LaneCounters* work = nullptr;   // counters: one set per lane, then one for whole-batch calls
  std::vector<Lane> lanes;
  cudaEvent_t fork = nullptr;
  int* d_flag = nullptr;  // one device int (host-buffer entry)
  int* h_flag = nullptr;  // pinned mirror
  unsigned char ckpt_head[256] = {};  // source of the last checkpoint's header copy
  std::string err;
};

namespace {

double* cur_U(const rrmhd_ctx* c) { return c->cur ? c->B.Ua : c->B.U0; }
double* cur_b(const rrmhd_ctx* c) { return c->cur ? c->B.bfa : c->B.bf0; }
double* cur_V(const rrmhd_ctx* c) { return c->cur ? c->B.Va : c->B.V0; }

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

Batch batch_of(const rrmhd_ctx* c) { return rr::make_batch(c->L, c->B, 0, c->L.n_inst); }

StageArgs stage_args(const rrmhd_ctx* c, const Batch& b, int stage, const double* U0,
                     const double* V0, const double* Us, const double* Vs, double* Uout,
                     double* Vout) {
  return rr::stage_args(c->P, c->B, b, stage, U0, V0, Us, Vs, Uout, Vout);
}

template <class T>
rrmhd_status dalloc(rrmhd_ctx* c, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cuda_check(c, cudaMalloc((void**)p, count * sizeof(T)), "cudaMalloc");
}

void destroy_lanes(rrmhd_ctx* c) {
  for (Lane& L : c->lanes) {
    if (L.stream) cudaStreamSynchronize(L.stream);
    for (cudaGraphExec_t g : L.graph)
      if (g) cudaGraphExecDestroy(g);
    if (L.done) cudaEventDestroy(L.done);
    if (L.stream) cudaStreamDestroy(L.stream);
  }
  c->lanes.clear();
  if (c->work) cudaFree(c->work);
  c->work = nullptr;
}

// Splits the instances into n lanes of about equal cell count, each with its own
// stream, completion event and chunk counters.
rrmhd_status build_lanes(rrmhd_ctx* c, int n) {
  destroy_lanes(c);
  const auto ranges = rr::lane_ranges(c->L.cell_off, c->L.n_inst, n);
  const size_t nw = ranges.size() + 1;
  RR_CUDA(c, cudaMalloc((void**)&c->work, sizeof(rr::LaneCounters) * nw));
  RR_CUDA(c, cudaMemset(c->work, 0, sizeof(rr::LaneCounters) * nw));
  for (size_t l = 0; l < ranges.size(); ++l) {
    Lane lane;
    lane.b = rr::make_batch(c->L, c->B, ranges[l].first, ranges[l].second);
    lane.cnt = c->work + l;
    c->lanes.push_back(lane);
    Lane& L = c->lanes.back();
    RR_CUDA(c, cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking));
    RR_CUDA(c, cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming));
  }
  return RRMHD_OK;
}

// Counters of the whole-batch launches (flux sweep, profiled step).
rr::LaneCounters* batch_work(const rrmhd_ctx* c) { return c->work + c->lanes.size(); }

}  // namespace

namespace rr {
bool prepare_launch_shapes() {
  static std::once_flag once;
  static bool ok = false;
  std::call_once(once, [] { ok = prepare_launch_shapes_f64() && prepare_launch_shapes_f32(); });
  return ok;
}
}  // namespace rr

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
  o->pvm_k = 3;
  o->pvm_products = 0;
  o->solver = RRMHD_SOLVER_PVM;
  o->ct = 0;
  o->closure = RRMHD_CLOSURE_M1;
}

void rrmhd_destroy(rrmhd_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  destroy_lanes(c);
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->d_flag) cudaFree(c->d_flag);
  if (c->h_flag) cudaFreeHost(c->h_flag);
  const rr::DeviceBufs& B = c->B;
  void* bufs[] = {B.inst, B.cell_off, B.face_off, B.U0,  B.Ua,    B.Ub,   B.V0,
                  B.Va,   B.Vb,       B.kappa,    B.sigma, B.Fhat, B.t,    B.t_end,
                  B.dt,   B.smax,     B.status,   B.bad, B.jc,   B.edge_off, B.bf0,
                  B.bfa,  B.bfb,      B.emf,      B.dt_max, B.bad_cell};
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
  if (!rr::opts_ok(o)) return RRMHD_EINVAL;
  std::string why;
  for (int i = 0; i < n_inst; ++i)
    if (!rr::grid_ok(grids[i], why)) return RRMHD_EINVAL;
  if (!rr::prepare_launch_shapes()) return RRMHD_ECUDA;

  rrmhd_ctx* c = new rrmhd_ctx();
  c->opts = o;
  c->P = rr::make_params(o);
  c->stream = (cudaStream_t)cuda_stream;
  c->L = rr::make_layout(grids, n_inst);
  const rr::Layout& L = c->L;
  rr::DeviceBufs& B = c->B;

  rrmhd_status s = RRMHD_OK;
  const size_t N12 = (size_t)12 * L.ncells;
  auto A = [&](rrmhd_status r) {
    if (s == RRMHD_OK) s = r;
  };
  A(dalloc(c, &B.inst, n_inst));
  A(dalloc(c, &B.cell_off, n_inst + 1));
  A(dalloc(c, &B.face_off, 3 * (size_t)(n_inst + 1)));
  A(dalloc(c, &B.edge_off, 3 * (size_t)(n_inst + 1)));
  A(dalloc(c, &c->d_flag, 1));
  A(cuda_check(c, cudaMallocHost((void**)&c->h_flag, sizeof(int)), "cudaMallocHost"));
  if (o.ct) {
    for (double** p : {&B.bf0, &B.bfa, &B.bfb}) A(dalloc(c, p, (size_t)L.nfaces));
    A(dalloc(c, &B.emf, (size_t)L.nedges));
  }
  for (double** p : {&B.U0, &B.Ua, &B.Ub, &B.V0, &B.Va, &B.Vb}) A(dalloc(c, p, N12));
  A(dalloc(c, &B.kappa, L.ncells));
  A(dalloc(c, &B.sigma, L.ncells));
  A(dalloc(c, &B.Fhat, (size_t)12 * L.nfaces));
  A(dalloc(c, &B.t, n_inst));
  A(dalloc(c, &B.t_end, n_inst));
  A(dalloc(c, &B.dt, n_inst));
  A(dalloc(c, &B.smax, n_inst));
  A(dalloc(c, &B.status, n_inst));
  A(dalloc(c, &B.dt_max, 1));
  A(dalloc(c, &B.bad_cell, n_inst));
  A(dalloc(c, &B.bad, (size_t)L.ncells));
  A(dalloc(c, &B.jc, (size_t)17 * L.ncells));
  if (s == RRMHD_OK) {
    cudaStream_t st = c->stream;
    A(cuda_check(c, cudaMemcpyAsync(B.inst, L.inst.data(), sizeof(InstDesc) * n_inst,
                                    cudaMemcpyHostToDevice, st), "upload"));
    A(cuda_check(c, cudaMemcpyAsync(B.cell_off, L.cell_off.data(),
                                    sizeof(int64_t) * (n_inst + 1), cudaMemcpyHostToDevice, st),
                 "upload"));
    A(cuda_check(c, cudaMemcpyAsync(B.face_off, L.face_off.data(),
                                    sizeof(int64_t) * 3 * (n_inst + 1), cudaMemcpyHostToDevice, st),
                 "upload"));
    A(cuda_check(c, cudaMemcpyAsync(B.edge_off, L.edge_off.data(),
                                    sizeof(int64_t) * 3 * (n_inst + 1), cudaMemcpyHostToDevice, st),
                 "upload"));
    if (o.ct)
      for (double* p : {B.bf0, B.bfa, B.bfb})
        A(cuda_check(c, cudaMemsetAsync(p, 0, sizeof(double) * (L.nfaces ? L.nfaces : 1), st), "memset"));
    std::vector<double> zeros(n_inst, 0.0), inf(n_inst, std::numeric_limits<double>::infinity());
    A(cuda_check(c, cudaMemcpyAsync(B.t, zeros.data(), sizeof(double) * n_inst,
                                    cudaMemcpyHostToDevice, st), "upload"));
    A(cuda_check(c, cudaMemcpyAsync(B.t_end, inf.data(), sizeof(double) * n_inst,
                                    cudaMemcpyHostToDevice, st), "upload"));
    A(cuda_check(c, cudaMemsetAsync(B.dt, 0, sizeof(double) * n_inst, st), "memset"));
    A(cuda_check(c, cudaMemsetAsync(B.smax, 0, sizeof(unsigned long long) * n_inst, st), "memset"));
    A(cuda_check(c, cudaMemsetAsync(B.status, 0, sizeof(int) * n_inst, st), "memset"));
    rr::launch_set_f64(B.dt_max, std::numeric_limits<double>::infinity(), st);
    rr::launch_fill_i64(B.bad_cell, n_inst, std::numeric_limits<long long>::max(), st);
    A(cuda_check(c, cudaGetLastError(), "set-up kernels"));
    A(cuda_check(c, cudaMemsetAsync(B.kappa, 0, sizeof(double) * L.ncells, st), "memset"));
    A(cuda_check(c, cudaMemsetAsync(B.sigma, 0, sizeof(double) * L.ncells, st), "memset"));
    A(cuda_check(c, cudaMemsetAsync(B.U0, 0, sizeof(double) * N12, st), "memset"));
    A(cuda_check(c, cudaMemsetAsync(B.V0, 0, sizeof(double) * N12, st), "memset"));
    A(cuda_check(c, cudaMemsetAsync(B.bad, 0, (size_t)L.ncells, st), "memset"));
    A(cuda_check(c, cudaMemsetAsync(B.jc, 0, sizeof(double) * 17 * L.ncells, st), "memset"));
    A(cuda_check(c, cudaStreamSynchronize(st), "sync"));  // host vectors go out of scope
  }
  if (s == RRMHD_OK) {
    c->tune = rr::default_tuning();
    A(build_lanes(c, o.lanes));
    A(cuda_check(c, cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming), "event"));
  }
  if (s != RRMHD_OK) {
    rrmhd_destroy(c);
    return s;
  }
  *out = c;
  return RRMHD_OK;
}

int rrmhd_num_instances(const rrmhd_ctx* c) { return c ? c->L.n_inst : 0; }
int64_t rrmhd_num_cells(const rrmhd_ctx* c) { return c ? c->L.ncells : 0; }
int64_t rrmhd_num_faces(const rrmhd_ctx* c, int dir) {
  if (!c || dir < 0 || dir > 2) return 0;
  return c->L.dir_base[dir + 1] - c->L.dir_base[dir];
}

rrmhd_status rrmhd_cell_offsets(const rrmhd_ctx* c, int64_t* off) {
  if (!c || !off) return RRMHD_EINVAL;
  std::memcpy(off, c->L.cell_off.data(), sizeof(int64_t) * (c->L.n_inst + 1));
  return RRMHD_OK;
}

rrmhd_status rrmhd_face_offsets(const rrmhd_ctx* c, int dir, int64_t* off) {
  if (!c || !off || dir < 0 || dir > 2) return RRMHD_EINVAL;
  std::memcpy(off, &c->L.face_off[(size_t)dir * (c->L.n_inst + 1)], sizeof(int64_t) * (c->L.n_inst + 1));
  return RRMHD_OK;
}

rrmhd_status rrmhd_set_opacity(rrmhd_ctx* c, const double* kappa, const double* sigma) {
  if (!c || !kappa || !sigma) return set_err(c, RRMHD_EINVAL, "null argument");
  RR_CUDA(c, cudaMemcpyAsync(c->B.kappa, kappa, sizeof(double) * c->L.ncells, cudaMemcpyDeviceToDevice,
                             c->stream));
  RR_CUDA(c, cudaMemcpyAsync(c->B.sigma, sigma, sizeof(double) * c->L.ncells, cudaMemcpyDeviceToDevice,
                             c->stream));
  return RRMHD_OK;
}

static rrmhd_status refresh_state(rrmhd_ctx* c) {
  const Batch b = batch_of(c);
  rr::launch_prim2con_f64(c->P, cur_V(c), cur_U(c), c->L.ncells, c->stream);
  RR_CUDA(c, cudaMemsetAsync(c->B.smax, 0, sizeof(unsigned long long) * c->L.n_inst, c->stream));
  RR_CUDA(c, cudaMemsetAsync(c->B.status, 0, sizeof(int) * c->L.n_inst, c->stream));
  rr::launch_fill_i64(c->B.bad_cell, c->L.n_inst, std::numeric_limits<long long>::max(), c->stream);
  RR_CUDA(c, cudaMemsetAsync(c->B.dt, 0, sizeof(double) * c->L.n_inst, c->stream));
  // a new state starts with an empty Jacobian cache (validity plane)
  RR_CUDA(c, cudaMemsetAsync(c->B.jc + (size_t)16 * c->L.ncells, 0, sizeof(double) * c->L.ncells, c->stream));
  rr::launch_signal_f64(c->P, b, cur_V(c), c->stream);
  RR_CUDA(c, cudaGetLastError());
  return RRMHD_OK;
}

// Constrained transport: periodic duplicate faces made equal, then the
// cell-centred B of the current state set to the face means.
static rrmhd_status ct_sync_cells(rrmhd_ctx* c) {
  const Batch b = batch_of(c);
  rr::launch_ct_canonical_f64(b, cur_b(c), c->stream);
  rr::launch_cells_from_faces_f64(b, cur_b(c), cur_V(c), c->stream);
  RR_CUDA(c, cudaGetLastError());
  return RRMHD_OK;
}

rrmhd_status rrmhd_set_state(rrmhd_ctx* c, const double* V) {
  if (!c || !V) return set_err(c, RRMHD_EINVAL, "null argument");
  RR_CUDA(c, cudaMemcpyAsync(cur_V(c), V, sizeof(double) * 12 * c->L.ncells,
                             cudaMemcpyDeviceToDevice, c->stream));
  if (c->opts.ct) {
    rr::launch_faces_from_cells_f64(batch_of(c), cur_V(c), cur_b(c), c->stream);
    rrmhd_status s = ct_sync_cells(c);
    if (s != RRMHD_OK) return s;
  }
  return refresh_state(c);
}

rrmhd_status rrmhd_set_face_field(rrmhd_ctx* c, const double* b) {
  if (!c || !b) return set_err(c, RRMHD_EINVAL, "null argument");
  if (!c->opts.ct) return set_err(c, RRMHD_EINVAL, "constrained transport is off (opts.ct)");
  RR_CUDA(c, cudaMemcpyAsync(cur_b(c), b, sizeof(double) * c->L.nfaces, cudaMemcpyDeviceToDevice,
                             c->stream));
  rrmhd_status s = ct_sync_cells(c);
  if (s != RRMHD_OK) return s;
  return refresh_state(c);
}

rrmhd_status rrmhd_get_face_field(const rrmhd_ctx* c, double* b) {
  if (!c || !b) return RRMHD_EINVAL;
  if (!c->opts.ct) return set_err(c, RRMHD_EINVAL, "constrained transport is off (opts.ct)");
  RR_CUDA(c, cudaMemcpyAsync(b, cur_b(c), sizeof(double) * c->L.nfaces, cudaMemcpyDeviceToDevice,
                             c->stream));
  return RRMHD_OK;
}

rrmhd_status rrmhd_get_state(const rrmhd_ctx* c, double* U, double* V) {
  if (!c) return RRMHD_EINVAL;
  if (U)
    RR_CUDA(c, cudaMemcpyAsync(U, cur_U(c), sizeof(double) * 12 * c->L.ncells,
                               cudaMemcpyDeviceToDevice, c->stream));
  if (V)
    RR_CUDA(c, cudaMemcpyAsync(V, cur_V(c), sizeof(double) * 12 * c->L.ncells,
                               cudaMemcpyDeviceToDevice, c->stream));
  return RRMHD_OK;
}

rrmhd_status rrmhd_set_times(rrmhd_ctx* c, const double* t, const double* t_end) {
  if (!c || !t || !t_end) return set_err(c, RRMHD_EINVAL, "null argument");
  RR_CUDA(c, cudaMemcpyAsync(c->B.t, t, sizeof(double) * c->L.n_inst, cudaMemcpyHostToDevice, c->stream));
  RR_CUDA(c, cudaMemcpyAsync(c->B.t_end, t_end, sizeof(double) * c->L.n_inst, cudaMemcpyHostToDevice,
                             c->stream));
  RR_CUDA(c, cudaStreamSynchronize(c->stream));  // pageable host sources
  RR_CUDA(c, cudaMemsetAsync(c->B.smax, 0, sizeof(unsigned long long) * c->L.n_inst, c->stream));
  rr::launch_signal_f64(c->P, batch_of(c), cur_V(c), c->stream);
  RR_CUDA(c, cudaGetLastError());
  return RRMHD_OK;
}

rrmhd_status rrmhd_get_times(const rrmhd_ctx* c, double* t, double* dt_last) {
  if (!c) return RRMHD_EINVAL;
  if (t) RR_CUDA(c, cudaMemcpyAsync(t, c->B.t, sizeof(double) * c->L.n_inst, cudaMemcpyDeviceToHost, c->stream));
  if (dt_last)
    RR_CUDA(c, cudaMemcpyAsync(dt_last, c->B.dt, sizeof(double) * c->L.n_inst, cudaMemcpyDeviceToHost,
                               c->stream));
  RR_CUDA(c, cudaStreamSynchronize(c->stream));
  return RRMHD_OK;
}

rrmhd_status rrmhd_get_inst_status(const rrmhd_ctx* c, int32_t* status) {
  if (!c || !status) return RRMHD_EINVAL;
  RR_CUDA(c, cudaMemcpyAsync(status, c->B.status, sizeof(int) * c->L.n_inst, cudaMemcpyDeviceToHost,
                             c->stream));
  RR_CUDA(c, cudaStreamSynchronize(c->stream));
  return RRMHD_OK;
}

static rrmhd_status build_step_graph(rrmhd_ctx* c, Lane& L, int cur) {
  if (L.graph[cur]) return RRMHD_OK;
  if (!c->cap_stream)
    RR_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  RR_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  rr::enqueue_step(c->P, c->opts.precision, c->tune, c->B, L.b, cur, L.cnt, c->cap_stream,
                   c->opts.ct);
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

// The lanes fork from the caller's stream, run their nsteps step graphs back to
// back on their own streams, and join back into it once.  A lane touches only its
// own instances, cells, faces, edges and counters, so the lanes need no join
// between steps: a lane held up by a slow implicit solve in one step catches up
// while the others run ahead, and the results are those of nsteps single steps.
rrmhd_status rrmhd_imex_step(rrmhd_ctx* c, int nsteps) {
  if (!c || nsteps < 0) return set_err(c, RRMHD_EINVAL, "bad argument");
  if (nsteps == 0) return RRMHD_OK;
  for (Lane& L : c->lanes)
    for (int p = 0; p < (nsteps > 1 ? 2 : 1); ++p) {
      rrmhd_status s = build_step_graph(c, L, c->cur ^ p);
      if (s != RRMHD_OK) return s;
    }
  RR_CUDA(c, cudaEventRecord(c->fork, c->stream));
  for (Lane& L : c->lanes) RR_CUDA(c, cudaStreamWaitEvent(L.stream, c->fork, 0));
  // submitted step by step across the lanes: streams that share a hardware queue
  // then hold each other up by one step at most
  for (int k = 0; k < nsteps; ++k)
    for (Lane& L : c->lanes) RR_CUDA(c, cudaGraphLaunch(L.graph[c->cur ^ (k & 1)], L.stream));
  for (Lane& L : c->lanes) {
    RR_CUDA(c, cudaEventRecord(L.done, L.stream));
    RR_CUDA(c, cudaStreamWaitEvent(c->stream, L.done, 0));
  }
  c->cur ^= nsteps & 1;
  return RRMHD_OK;
}

rrmhd_status rrmhd_imex_step_dt(rrmhd_ctx* c, double dt_max, double* dt_taken) {
  if (!c || !(dt_max > 0.0)) return set_err(c, RRMHD_EINVAL, "bad argument");
  rr::launch_set_f64(c->B.dt_max, dt_max, c->stream);
  RR_CUDA(c, cudaGetLastError());
  rrmhd_status s = rrmhd_imex_step(c, 1);
  rr::launch_set_f64(c->B.dt_max, std::numeric_limits<double>::infinity(), c->stream);
  RR_CUDA(c, cudaGetLastError());
  if (s != RRMHD_OK) return s;
  return dt_taken ? rrmhd_get_times(c, nullptr, dt_taken) : RRMHD_OK;
}

// ---------------------------------------------------------------- checkpoints
// Layout: a 256-byte header, then every part below at a 256-byte-aligned offset.
namespace {

struct CkptHeader {
  char magic[8];  // "RRMHDCK1"
  int32_t precision, ct, n_inst, pad;
  int64_t ncells, nfaces, bytes;
};

struct CkptPart {
  void* dev;
  size_t bytes;
};

std::vector<CkptPart> ckpt_parts(const rrmhd_ctx* c) {
  const size_t N = (size_t)c->L.ncells, n = (size_t)c->L.n_inst;
  const rr::DeviceBufs& B = c->B;
  std::vector<CkptPart> p = {{cur_U(c), 96 * N},   {cur_V(c), 96 * N},   {B.kappa, 8 * N},
                             {B.sigma, 8 * N},     {B.jc, 136 * N},      {B.t, 8 * n},
                             {B.t_end, 8 * n},     {B.dt, 8 * n},        {B.smax, 8 * n},
                             {B.status, 4 * n},    {B.bad_cell, 8 * n}};
  if (c->opts.ct) p.push_back({cur_b(c), 8 * (size_t)c->L.nfaces});
  return p;
}

size_t ckpt_align(size_t x) { return (x + 255) & ~(size_t)255; }

CkptHeader ckpt_header(const rrmhd_ctx* c) {
  CkptHeader h{};
  std::memcpy(h.magic, "RRMHDCK1", 8);
  h.precision = c->opts.precision;
  h.ct = c->opts.ct;
  h.n_inst = c->L.n_inst;
  h.ncells = c->L.ncells;
  h.nfaces = c->L.nfaces;
  h.bytes = (int64_t)rrmhd_checkpoint_bytes(c);
  return h;
}

}  // namespace

size_t rrmhd_checkpoint_bytes(const rrmhd_ctx* c) {
  if (!c) return 0;
  size_t s = 256;
  for (const CkptPart& q : ckpt_parts(c)) s += ckpt_align(q.bytes);
  return s;
}

rrmhd_status rrmhd_checkpoint_save(rrmhd_ctx* c, void* buf) {
  if (!c || !buf) return set_err(c, RRMHD_EINVAL, "bad argument");
  const CkptHeader h = ckpt_header(c);
  std::memcpy(c->ckpt_head, &h, sizeof(h));
  char* dst = static_cast<char*>(buf);
  RR_CUDA(c, cudaMemcpyAsync(dst, c->ckpt_head, sizeof(h), cudaMemcpyDefault, c->stream));
  size_t off = 256;
  for (const CkptPart& q : ckpt_parts(c)) {
    RR_CUDA(c, cudaMemcpyAsync(dst + off, q.dev, q.bytes, cudaMemcpyDefault, c->stream));
    off += ckpt_align(q.bytes);
  }
  return RRMHD_OK;
}

rrmhd_status rrmhd_checkpoint_restore(rrmhd_ctx* c, const void* buf) {
  if (!c || !buf) return set_err(c, RRMHD_EINVAL, "bad argument");
  CkptHeader h{};
  const char* src = static_cast<const char*>(buf);
  RR_CUDA(c, cudaMemcpyAsync(&h, src, sizeof(h), cudaMemcpyDefault, c->stream));
  RR_CUDA(c, cudaStreamSynchronize(c->stream));
  const CkptHeader want = ckpt_header(c);
  if (std::memcmp(h.magic, want.magic, 8) != 0 || h.precision != want.precision ||
      h.ct != want.ct || h.n_inst != want.n_inst || h.ncells != want.ncells ||
      h.nfaces != want.nfaces || h.bytes != want.bytes)
    return set_err(c, RRMHD_EINVAL, "checkpoint: written by a context of another layout or form");
  size_t off = 256;
  for (const CkptPart& q : ckpt_parts(c)) {
    RR_CUDA(c, cudaMemcpyAsync(q.dev, src + off, q.bytes, cudaMemcpyDefault, c->stream));
    off += ckpt_align(q.bytes);
  }
  return RRMHD_OK;
}

rrmhd_status rrmhd_get_first_bad_cell(const rrmhd_ctx* c, int64_t* cell) {
  if (!c || !cell) return RRMHD_EINVAL;
  std::vector<long long> h(c->L.n_inst);
  RR_CUDA(c, cudaMemcpyAsync(h.data(), c->B.bad_cell, sizeof(long long) * c->L.n_inst,
                             cudaMemcpyDeviceToHost, c->stream));
  RR_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int i = 0; i < c->L.n_inst; ++i)
    cell[i] = h[i] == std::numeric_limits<long long>::max() ? -1 : (int64_t)h[i];
  return RRMHD_OK;
}

rrmhd_status rrmhd_imex_step_host(rrmhd_ctx* c, const double* V_in, double* V_out, int nsteps) {
  if (!c || !V_in || !V_out || nsteps < 0) return set_err(c, RRMHD_EINVAL, "bad argument");
  const int64_t n = (int64_t)12 * c->L.ncells;
  const size_t bytes = sizeof(double) * n;
  // V_in to the scratch set, then: the context's own state (a continuing run) or a new one?
  RR_CUDA(c, cudaMemcpyAsync(c->B.Vb, V_in, bytes, cudaMemcpyHostToDevice, c->stream));
  RR_CUDA(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream));
  k_differs<<<1216, 256, 0, c->stream>>>(reinterpret_cast<const unsigned long long*>(c->B.Vb),
                                         reinterpret_cast<const unsigned long long*>(cur_V(c)), n,
                                         c->d_flag);
  RR_CUDA(c, cudaGetLastError());
  RR_CUDA(c, cudaMemcpyAsync(c->h_flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  RR_CUDA(c, cudaStreamSynchronize(c->stream));
  rrmhd_status s = RRMHD_OK;
  if (*c->h_flag) {  // a new state: as rrmhd_set_state
    RR_CUDA(c, cudaMemcpyAsync(cur_V(c), c->B.Vb, bytes, cudaMemcpyDeviceToDevice, c->stream));
    s = refresh_state(c);
    if (s != RRMHD_OK) return s;
  }
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
  a.work = batch_work(c)->work;
  if (c->opts.ct) {
    a.ct = 1;
    a.fp32_fluxes = c->opts.precision == RRMHD_FP32_BULK;
    a.bs = cur_b(c);
  }
  const int64_t nd = c->L.dir_base[dir + 1] - c->L.dir_base[dir];
  if (c->opts.precision == RRMHD_FP32_BULK) {
    // FP32 fluxes into the context's face buffer, widened into the caller's array
    rr::launch_faces_f32(a, c->tune.faces, c->stream);
    rr::launch_widen_f32(a.Fhat32, c->L.nfaces, c->L.dir_base[dir], nd, Fhat, c->stream);
  } else {
    a.Fhat = Fhat;
    a.fstride = nd;
    a.out_base = c->L.dir_base[dir];
    rr::launch_faces_f64(a, c->tune.faces, c->stream);
  }
  RR_CUDA(c, cudaGetLastError());
  return RRMHD_OK;
}

rrmhd_status rrmhd_flux_accumulate(rrmhd_ctx* c, int dir, double dt_weight, double* U) {
  if (!c || !U || dir < 0 || dir > 2 || !(dt_weight >= 0.0))
    return set_err(c, RRMHD_EINVAL, "bad argument");
  Batch b = batch_of(c);
  for (int d = 0; d < 3; ++d) b.f_count[d] = (d == dir) ? b.f_count[d] : 0;
  StageArgs a = stage_args(c, b, 0, cur_U(c), cur_V(c), cur_U(c), cur_V(c), nullptr, nullptr);
  a.check_active = 0;
  a.work = batch_work(c)->work;
  if (c->opts.ct) {
    a.ct = 1;
    a.fp32_fluxes = c->opts.precision == RRMHD_FP32_BULK;
    a.bs = cur_b(c);
  }
  const int64_t nd = c->L.dir_base[dir + 1] - c->L.dir_base[dir];
  if (c->opts.precision == RRMHD_FP32_BULK) {
    // FP32 fluxes in the context's face buffer (columns = global face index)
    rr::launch_faces_f32(a, c->tune.faces, c->stream);
    rr::launch_flux_accumulate(batch_of(c), dir, dt_weight, nullptr, a.Fhat32, a.fstride, 0, U,
                               c->stream);
  } else {
    a.Fhat = c->B.Fhat;
    a.fstride = nd;
    a.out_base = c->L.dir_base[dir];
    rr::launch_faces_f64(a, c->tune.faces, c->stream);
    rr::launch_flux_accumulate(batch_of(c), dir, dt_weight, c->B.Fhat, nullptr, nd,
                               c->L.dir_base[dir], U, c->stream);
  }
  RR_CUDA(c, cudaGetLastError());
  return RRMHD_OK;
}

rrmhd_status rrmhd_implicit_source(rrmhd_ctx* c, double hdt, const double* Ustar,
                                   const double* Zguess, double* U, double* V, int32_t* status) {
  if (!c || !Ustar || !U || !V || !(hdt >= 0.0)) return set_err(c, RRMHD_EINVAL, "bad argument");
  rr::launch_implicit_f64(c->P, batch_of(c), hdt, Ustar, Zguess, c->B.kappa, c->B.sigma, U, V, status,
                          c->stream);
  RR_CUDA(c, cudaGetLastError());
  return RRMHD_OK;
}

int rrmhd_launches_per_step(const rrmhd_ctx* c) {
  return c ? (int)c->lanes.size() * rr::launches_per_step(c->opts.ct) : 0;
}

rrmhd_status rrmhd_profile_step(rrmhd_ctx* c, double* ms) {
  if (!c || !ms) return set_err(c, RRMHD_EINVAL, "bad argument");
  const int cur = c->cur;
  const Batch b = batch_of(c);
  double* AU = cur ? c->B.Ua : c->B.U0;
  double* AV = cur ? c->B.Va : c->B.V0;
  double* BU = cur ? c->B.U0 : c->B.Ua;
  double* BV = cur ? c->B.V0 : c->B.Va;
  rr::LaneCounters* w = batch_work(c);
  StageArgs st[3] = {rr::stage_args(c->P, c->B, b, 1, AU, AV, AU, AV, BU, BV, w),
                     rr::stage_args(c->P, c->B, b, 2, AU, AV, BU, BV, c->B.Ub, c->B.Vb, w),
                     rr::stage_args(c->P, c->B, b, 3, AU, AV, c->B.Ub, c->B.Vb, BU, BV, w)};
  if (c->opts.ct) {
    double* Ab = cur ? c->B.bfa : c->B.bf0;
    double* Bb = cur ? c->B.bf0 : c->B.bfa;
    for (StageArgs& x : st) {
      x.ct = 1;
      x.fp32_fluxes = c->opts.precision == RRMHD_FP32_BULK;
      x.b0 = Ab;
    }
    st[0].bs = Ab;
    st[0].bout = Bb;
    st[1].bs = Bb;
    st[1].bout = c->B.bfb;
    st[2].bs = c->B.bfb;
    st[2].bout = Bb;
  }
  cudaEvent_t ev[14];
  for (auto& e : ev) RR_CUDA(c, cudaEventCreate(&e));
  cudaStream_t s = c->stream;
  int k = 0;
  cudaEventRecord(ev[k++], s);
  rr::launch_begin_step(c->P, b, s);
  RR_CUDA(c, cudaMemsetAsync(w->flagged, 0, sizeof(w->flagged), s));
  cudaEventRecord(ev[k++], s);
  const int pr = c->opts.precision;
  for (int i = 0; i < 3; ++i) {
    rr::launch_faces(pr, st[i], c->tune.faces, s);
    if (st[i].ct) {
      rr::launch_emf_f64(st[i], s);
      rr::launch_bface_f64(st[i], s);
    }
    cudaEventRecord(ev[k++], s);
    rr::launch_cells(pr, st[i], c->tune.cells, s);
    cudaEventRecord(ev[k++], s);
    rr::launch_fallback(pr, st[i], s);
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

static rr::Tuning tuning_from(const rrmhd_tuning& t) {
  rr::Tuning tu;
  tu.faces = {t.face_block, t.face_per_thread, t.face_persistent};
  tu.cells = {t.cell_block, t.cell_per_thread, t.cell_persistent};
  return tu;
}

static rrmhd_tuning tuning_to(const rr::Tuning& tu, int lanes) {
  rrmhd_tuning t;
  t.face_block = tu.faces.block;
  t.face_per_thread = tu.faces.per_thread;
  t.face_persistent = tu.faces.persistent;
  t.cell_block = tu.cells.block;
  t.cell_per_thread = tu.cells.per_thread;
  t.cell_persistent = tu.cells.persistent;
  t.lanes = lanes;
  return t;
}

rrmhd_status rrmhd_get_tuning(const rrmhd_ctx* c, rrmhd_tuning* t) {
  if (!c || !t) return RRMHD_EINVAL;
  *t = tuning_to(c->tune, c->opts.lanes);
  return RRMHD_OK;
}

rrmhd_status rrmhd_set_tuning(rrmhd_ctx* c, const rrmhd_tuning* t) {
  if (!c || !t) return set_err(c, RRMHD_EINVAL, "null argument");
  const rr::Tuning tu = tuning_from(*t);
  if (!rr::tuning_ok(tu) || t->lanes < 1) return set_err(c, RRMHD_EINVAL, "unsupported launch shape");
  RR_CUDA(c, cudaStreamSynchronize(c->stream));
  c->tune = tu;
  c->opts.lanes = t->lanes;
  return build_lanes(c, t->lanes);  // new lanes, no step graphs yet
}

rrmhd_status rrmhd_autotune(rrmhd_ctx* c, int repeats, rrmhd_tuning* best, double* best_ms) {
  if (!c || repeats < 1) return set_err(c, RRMHD_EINVAL, "bad argument");
  const int n = c->L.n_inst;
  const size_t N12 = (size_t)12 * c->L.ncells, NJ = (size_t)17 * c->L.ncells;
  double *sU = nullptr, *sV = nullptr, *sJ = nullptr, *sT = nullptr, *sDt = nullptr;
  unsigned long long* sM = nullptr;
  int* sS = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto release = [&] {
    for (void* p : {(void*)sU, (void*)sV, (void*)sJ, (void*)sT, (void*)sDt, (void*)sM, (void*)sS})
      if (p) cudaFree(p);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (cudaMalloc((void**)&sU, 8 * N12) != cudaSuccess || cudaMalloc((void**)&sV, 8 * N12) != cudaSuccess ||
      cudaMalloc((void**)&sJ, 8 * NJ) != cudaSuccess || cudaMalloc((void**)&sT, 8 * n) != cudaSuccess ||
      cudaMalloc((void**)&sDt, 8 * n) != cudaSuccess || cudaMalloc((void**)&sM, 8 * n) != cudaSuccess ||
      cudaMalloc((void**)&sS, sizeof(int) * n) != cudaSuccess) {
    cudaGetLastError();
    release();
    return set_err(c, RRMHD_ENOMEM, "autotune: no memory for the saved state");
  }
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaStream_t st = c->stream;
  const int cur0 = c->cur;
  const rr::DeviceBufs& B = c->B;
  auto copy_state = [&](bool save) -> cudaError_t {
    double* U = cur0 ? B.Ua : B.U0;
    double* V = cur0 ? B.Va : B.V0;
    struct P { void* live; void* saved; size_t bytes; } parts[] = {
        {U, sU, 8 * N12}, {V, sV, 8 * N12}, {B.jc, sJ, 8 * NJ}, {B.t, sT, 8 * (size_t)n},
        {B.dt, sDt, 8 * (size_t)n}, {B.smax, sM, 8 * (size_t)n}, {B.status, sS, sizeof(int) * n}};
    for (const P& q : parts) {
      cudaError_t e = save ? cudaMemcpyAsync(q.saved, q.live, q.bytes, cudaMemcpyDeviceToDevice, st)
                           : cudaMemcpyAsync(q.live, q.saved, q.bytes, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return e;
    }
    if (!save) c->cur = cur0;
    return cudaSuccess;
  };
  rrmhd_status rc = cuda_check(c, copy_state(true), "autotune save");
  // best step time (ms) of a candidate over `repeats` steps, each from the saved state
  // (the fastest repeat is the least disturbed by other work on the device)
  auto trial = [&](const rrmhd_tuning& cand, double& ms) -> rrmhd_status {
    rrmhd_status r = rrmhd_set_tuning(c, &cand);
    if (r != RRMHD_OK) return r;
    RR_CUDA(c, copy_state(false));
    r = rrmhd_imex_step(c, 1);  // warm: builds the step graphs, loads the kernels
    if (r != RRMHD_OK) return r;
    std::vector<float> v;
    for (int k = 0; k < repeats; ++k) {
      RR_CUDA(c, copy_state(false));
      RR_CUDA(c, cudaEventRecord(e0, st));
      r = rrmhd_imex_step(c, 1);
      if (r != RRMHD_OK) return r;
      RR_CUDA(c, cudaEventRecord(e1, st));
      RR_CUDA(c, cudaEventSynchronize(e1));
      float x = 0.f;
      RR_CUDA(c, cudaEventElapsedTime(&x, e0, e1));
      v.push_back(x);
    }
    ms = *std::min_element(v.begin(), v.end());
    return RRMHD_OK;
  };
  rrmhd_tuning cur_best = tuning_to(c->tune, c->opts.lanes);
  double cur_ms = 0.0;
  if (rc == RRMHD_OK) rc = trial(cur_best, cur_ms);
  auto consider = [&](const rrmhd_tuning& cand) {
    if (rc != RRMHD_OK) return;
    double ms = 0.0;
    rc = trial(cand, ms);
    if (rc == RRMHD_OK && ms < cur_ms) {
      cur_ms = ms;
      cur_best = cand;
    }
  };
  const int blocks[6] = {8, 16, 32, 64, 128, 256};
  // 1. cell shapes
  for (int persistent = 0; persistent <= 1; ++persistent)
    for (int bsz : blocks)
      for (int pt = 1; pt <= (persistent ? 1 : 2); ++pt) {
        if (!rr::shape_ok(bsz, pt, persistent)) continue;
        rrmhd_tuning t = cur_best;
        t.cell_block = bsz;
        t.cell_per_thread = pt;
        t.cell_persistent = persistent;
        consider(t);
      }
  // 2. face shapes
  for (int persistent = 0; persistent <= 1; ++persistent)
    for (int bsz : blocks)
      for (int pt = 1; pt <= (persistent ? 1 : 2); ++pt) {
        if (!rr::shape_ok(bsz, pt, persistent)) continue;
        rrmhd_tuning t = cur_best;
        t.face_block = bsz;
        t.face_per_thread = pt;
        t.face_persistent = persistent;
        consider(t);
      }
  // 3. lanes
  for (int lanes : {1, 2, 4, 8, 16, 32}) {
    if (lanes > n) break;
    rrmhd_tuning t = cur_best;
    t.lanes = lanes;
    consider(t);
  }
  if (rc == RRMHD_OK) rc = rrmhd_set_tuning(c, &cur_best);
  if (rc == RRMHD_OK) rc = cuda_check(c, copy_state(false), "autotune restore");
  if (rc == RRMHD_OK) rc = cuda_check(c, cudaStreamSynchronize(st), "autotune sync");
  release();
  if (rc != RRMHD_OK) return rc;
  if (best) *best = cur_best;
  if (best_ms) *best_ms = cur_ms;
  return RRMHD_OK;
}

const char* rrmhd_last_error(const rrmhd_ctx* c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"
