// rrmhd_server.cu -- serving loop: continuous batching of independent solve
// requests on one GPU (declared in include/rrmhd.h).  The paper has no
// counterpart; each request is advanced by the same IMEX-RK3 step as a context.
//
// One engine thread owns all device work.  Its loop:
//   1. admit waiting requests in arrival order while they fit the resident bounds;
//   2. when the resident set changed: repack it into one contiguous batch
//      (survivors first, in their old order, then the new requests) by gather
//      kernels from the current buffers into the spare ones (cells, and with
//      constrained transport the staggered face field), upload the new
//      requests' primitives and compute their face field (constrained
//      transport), conserved state and signal speeds;
//   3. one IMEX step of every resident request (lanes on their own streams);
//   4. read back t, status and the next CFL maximum of every resident request,
//      copy out the finished ones and complete them.
// Compiled with --fmad=false: the admission computes U = prim2con(V) with the
// same operation order as the context path, so a request's result does not
// depend on how it was admitted.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <limits>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/rrmhd.h"
#include "batch.h"
#include "batch_index.cuh"
#include "engine.h"
#include "physics_f64.cuh"

namespace {

using rr::Batch;
using rr::InstDesc;
using rr::Params;

// Bytes the server holds per resident cell: six 12-plane state buffers, two
// copies of kappa, sigma and the 17-plane Jacobian cache, one fallback flag.
constexpr int64_t kBytesPerCell = 6 * 12 * 8 + 2 * (1 + 1 + 17) * 8 + 1;
// Per unit of face capacity: the 12-plane flux buffer; with constrained
// transport also the three staggered face-field sets and two edge EMFs (a
// request takes max(faces, edges / 2) units, so the edges fit in twice the
// face capacity).
inline int64_t bytes_per_face(int ct) { return 12 * 8 + (ct ? (3 + 2) * 8 : 0); }
// Face capacity per cell capacity: covers 2D grids of any size (2(n+1)/n faces
// per cell for n >= 40); 3D requests are bounded by the faces they need.
constexpr double kFacesPerCell = 2.05;
constexpr int kDefaultSlots = 4096;
constexpr int kThreads = 256;

inline unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// ---- kernels -------------------------------------------------------------

// One group of planes moved by the gather: planes of `src` with stride n_old to
// planes of `dst` with stride n_new.
struct PlaneGroup {
  const double* src;
  double* dst;
  int planes;
};

struct FaceGatherArgs {
  int n_inst;                        // survivors
  int n_all;                         // instances of the new layout
  const int64_t* new_off;            // [3][n_all + 1] face offsets of the new layout
  const int64_t* src_off;            // [3][n_inst] survivors' face offsets in the old layout
  int64_t new_base[3], old_base[3];  // direction bases of the two layouts
  int64_t cnt[3];                    // survivors' faces per direction
  const double* src;
  double* dst;
};

struct GatherArgs {
  int n_inst;              // survivors
  const int64_t* new_off;  // [n_inst + 1] their cell offsets in the new layout
  const int64_t* src_off;  // [n_inst] their cell offsets in the old layout
  int64_t n_old, n_new;    // plane strides
  PlaneGroup g[5];
};

// Survivors' cells to their new positions: c (new) <- src_off[i] + (c - new_off[i]).
__global__ void __launch_bounds__(kThreads) k_gather(GatherArgs a) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.new_off[a.n_inst]) return;
  const int i = rr::idx::find_inst(a.new_off, 0, a.n_inst, c);
  const int64_t s = a.src_off[i] + (c - a.new_off[i]);
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const PlaneGroup& G = a.g[q];
    for (int k = 0; k < G.planes; ++k) G.dst[k * a.n_new + c] = G.src[k * a.n_old + s];
  }
}

// Survivors' staggered face field to the new layout, direction by direction.
__global__ void __launch_bounds__(kThreads) k_gather_faces(FaceGatherArgs a) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int d = 0;
  while (d < 3 && t >= a.cnt[d]) {
    t -= a.cnt[d];
    ++d;
  }
  if (d == 3) return;
  const int64_t* no = a.new_off + (int64_t)d * (a.n_all + 1);
  const int i = rr::idx::find_inst(no, 0, a.n_inst, t);
  a.dst[a.new_base[d] + t] = a.src[a.old_base[d] + a.src_off[(int64_t)d * a.n_inst + i] + (t - no[i])];
}

// New requests' cells [c0, c1): U = prim2con(V) (Eq. eqU) and an empty Jacobian cache.
__global__ void __launch_bounds__(kThreads) k_admit(Params P, const double* __restrict__ V,
                                                     double* __restrict__ U, double* __restrict__ jc,
                                                     int64_t n, int64_t c0, int64_t c1) {
  const int64_t c = c0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= c1) return;
  double v[rr::NV], u[rr::NV];
  rr::idx::load12(V, n, c, v);
  rr::prim2con(P, v, u);
#pragma unroll
  for (int k = 0; k < rr::NV; ++k) U[k * n + c] = u[k];
  for (int k = 0; k < 17; ++k) jc[k * n + c] = 0.0;
}

// ---- host side -----------------------------------------------------------

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id = 0;
  rrmhd_grid grid{};
  int64_t cells = 0;
  int64_t faces = 0;  // face-capacity units: faces, or max(faces, edges / 2) with constrained transport
  std::vector<double> V, kappa, sigma;  // host copies of the inputs
  double t_end = 0.0;
  double* out = nullptr;                // caller's host buffer
  rrmhd_result res{};
  // resident bookkeeping (engine thread only)
  int64_t off = 0;  // cell offset in the current layout
  int slot = 0;     // instance index in the current layout
  double t = 0.0;
  unsigned long long smax = 0ull;
  int status = 0;
};

struct LaneRt {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
};

}  // namespace

struct rrmhd_server {
  rrmhd_opts opts{};
  Params P{};
  int device = 0;
  Clock::time_point t0;
  int64_t cap_cells = 0, cap_faces = 0;  // allocated capacity
  int64_t max_cells = 0;                 // admission bound on resident cells
  int cap_slots = 0;

  // device buffers (capacity-sized); B points at the live copies
  rr::DeviceBufs B;
  double *kap[2] = {nullptr, nullptr}, *sig[2] = {nullptr, nullptr}, *jcb[2] = {nullptr, nullptr};
  int64_t* d_src_off = nullptr;
  int64_t* d_src_foff = nullptr;       // [3][slots] survivors' old face offsets (constrained transport)
  rr::LaneCounters* work = nullptr;    // counters, one set per lane
  rr::Tuning tune;                     // launch shapes
  int kc = 0;   // live copy of kappa / sigma / jc
  int cur = 0;  // the state lives in (U0,V0) when 0, in (Ua,Va) when 1
  cudaStream_t stream = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<LaneRt> lanes;
  // pinned mirrors of the per-instance arrays
  double *h_t = nullptr, *h_tend = nullptr;
  unsigned long long* h_smax = nullptr;
  int* h_status = nullptr;

  // engine-thread state
  rr::Layout L;
  std::vector<std::unique_ptr<Request>> res;  // resident, in layout order
  bool dirty = false;                         // the resident set changed since the last repack

  // shared state (mu)
  std::mutex mu;
  std::condition_variable cv_work, cv_idle;
  std::deque<std::unique_ptr<Request>> waiting;
  std::vector<rrmhd_result> done;
  int64_t next_id = 1;
  bool stop = false;
  bool failed = false;
  int64_t n_resident = 0, resident_cells = 0, resident_faces = 0;  // admitted, not completed
  std::string err;
  rrmhd_server_stats st{};
  std::thread engine;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

bool set_failed(rrmhd_server* s, const std::string& msg) {
  std::lock_guard<std::mutex> lk(s->mu);
  s->failed = true;
  if (s->err.empty()) s->err = msg;
  return false;
}

#define SRV_CUDA(srv, expr)                                                                   \
  do {                                                                                        \
    cudaError_t _e = (expr);                                                                  \
    if (_e != cudaSuccess) return set_failed((srv), std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

// Repacks the resident set: survivors are s->res[0, n_surv) (at their offsets in
// the current layout), new requests follow.
bool relayout(rrmhd_server* s, int n_surv) {
  const int n = (int)s->res.size();
  std::vector<rrmhd_grid> grids(n);
  std::vector<int64_t> src_off(n_surv);
  for (int i = 0; i < n; ++i) grids[i] = s->res[i]->grid;
  for (int i = 0; i < n_surv; ++i) src_off[i] = s->res[i]->off;
  const int64_t n_old = s->L.ncells;
  const int ct = s->opts.ct;
  std::vector<int64_t> src_foff(3 * (size_t)n_surv);
  int64_t old_base[3];
  for (int d = 0; d < 3; ++d) {
    old_base[d] = s->L.dir_base[d];
    for (int i = 0; i < n_surv; ++i)
      src_foff[(size_t)d * n_surv + i] = s->L.face_off[(size_t)d * (s->L.n_inst + 1) + s->res[i]->slot];
  }
  s->L = rr::make_layout(grids.data(), n);
  const rr::Layout& L = s->L;
  rr::DeviceBufs& B = s->B;
  cudaStream_t st = s->stream;
  for (int i = 0; i < n; ++i) {
    s->res[i]->off = L.cell_off[i];
    s->res[i]->slot = i;
  }
  if (n == 0) return true;

  // tables of the new layout (the previous step has completed: the stream is idle)
  SRV_CUDA(s, cudaMemcpyAsync(B.inst, L.inst.data(), sizeof(InstDesc) * n, cudaMemcpyHostToDevice, st));
  SRV_CUDA(s, cudaMemcpyAsync(B.cell_off, L.cell_off.data(), sizeof(int64_t) * (n + 1),
                              cudaMemcpyHostToDevice, st));
  SRV_CUDA(s, cudaMemcpyAsync(B.face_off, L.face_off.data(), sizeof(int64_t) * 3 * (n + 1),
                              cudaMemcpyHostToDevice, st));
  SRV_CUDA(s, cudaMemcpyAsync(B.edge_off, L.edge_off.data(), sizeof(int64_t) * 3 * (n + 1),
                              cudaMemcpyHostToDevice, st));
  for (int i = 0; i < n; ++i) {
    const Request& r = *s->res[i];
    s->h_t[i] = r.t;
    s->h_tend[i] = r.t_end;
    s->h_smax[i] = r.smax;
    s->h_status[i] = r.status;
  }
  SRV_CUDA(s, cudaMemcpyAsync(B.t, s->h_t, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  SRV_CUDA(s, cudaMemcpyAsync(B.t_end, s->h_tend, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  SRV_CUDA(s, cudaMemcpyAsync(B.smax, s->h_smax, sizeof(unsigned long long) * n,
                              cudaMemcpyHostToDevice, st));
  SRV_CUDA(s, cudaMemcpyAsync(B.status, s->h_status, sizeof(int) * n, cudaMemcpyHostToDevice, st));

  // survivors: current buffers -> spare buffers at the new stride
  double* Ucur = s->cur ? B.Ua : B.U0;
  double* Vcur = s->cur ? B.Va : B.V0;
  double* Unew = s->cur ? B.U0 : B.Ua;
  double* Vnew = s->cur ? B.V0 : B.Va;
  const int ko = s->kc, kn = 1 - s->kc;
  if (n_surv > 0) {
    SRV_CUDA(s, cudaMemcpyAsync(s->d_src_off, src_off.data(), sizeof(int64_t) * n_surv,
                                cudaMemcpyHostToDevice, st));
    GatherArgs a;
    a.n_inst = n_surv;
    a.new_off = B.cell_off;
    a.src_off = s->d_src_off;
    a.n_old = n_old;
    a.n_new = L.ncells;
    a.g[0] = {Ucur, Unew, 12};
    a.g[1] = {Vcur, Vnew, 12};
    a.g[2] = {s->kap[ko], s->kap[kn], 1};
    a.g[3] = {s->sig[ko], s->sig[kn], 1};
    a.g[4] = {s->jcb[ko], s->jcb[kn], 17};
    k_gather<<<grid_for(L.cell_off[n_surv], kThreads), kThreads, 0, st>>>(a);
    SRV_CUDA(s, cudaGetLastError());
    if (ct) {
      SRV_CUDA(s, cudaMemcpyAsync(s->d_src_foff, src_foff.data(), sizeof(int64_t) * 3 * n_surv,
                                  cudaMemcpyHostToDevice, st));
      FaceGatherArgs f;
      f.n_inst = n_surv;
      f.n_all = n;
      f.new_off = B.face_off;
      f.src_off = s->d_src_foff;
      int64_t total = 0;
      for (int d = 0; d < 3; ++d) {
        f.new_base[d] = L.dir_base[d];
        f.old_base[d] = old_base[d];
        f.cnt[d] = L.face_off[(size_t)d * (n + 1) + n_surv];
        total += f.cnt[d];
      }
      f.src = s->cur ? B.bfa : B.bf0;
      f.dst = s->cur ? B.bf0 : B.bfa;
      if (total > 0) k_gather_faces<<<grid_for(total, kThreads), kThreads, 0, st>>>(f);
      SRV_CUDA(s, cudaGetLastError());
    }
  }
  // new requests: primitives and opacities from the host, then U, cache, speeds
  for (int i = n_surv; i < n; ++i) {
    const Request& r = *s->res[i];
    const int64_t off = L.cell_off[i];
    const size_t w = sizeof(double) * r.cells;
    for (int k = 0; k < 12; ++k)  // one copy per plane (plane pitches may exceed 2D-copy limits)
      SRV_CUDA(s, cudaMemcpyAsync(Vnew + k * L.ncells + off, r.V.data() + k * r.cells, w,
                                  cudaMemcpyHostToDevice, st));
    SRV_CUDA(s, cudaMemcpyAsync(s->kap[kn] + off, r.kappa.data(), w, cudaMemcpyHostToDevice, st));
    SRV_CUDA(s, cudaMemcpyAsync(s->sig[kn] + off, r.sigma.data(), w, cudaMemcpyHostToDevice, st));
  }
  s->cur ^= 1;
  s->kc = kn;
  B.kappa = s->kap[kn];
  B.sigma = s->sig[kn];
  B.jc = s->jcb[kn];
  if (n_surv < n) {
    const int64_t c0 = L.cell_off[n_surv], c1 = L.ncells;
    const Batch nb = rr::make_batch(L, B, n_surv, n);
    if (ct) {  // as a context's set_state: faces from the cells, duplicates, cells from the faces
      double* bnew = s->cur ? B.bfa : B.bf0;  // s->cur already names the new buffers
      rr::launch_faces_from_cells_f64(nb, Vnew, bnew, st);
      rr::launch_ct_canonical_f64(nb, bnew, st);
      rr::launch_cells_from_faces_f64(nb, bnew, Vnew, st);
      SRV_CUDA(s, cudaGetLastError());
    }
    k_admit<<<grid_for(c1 - c0, kThreads), kThreads, 0, st>>>(s->P, Vnew, Unew, B.jc, L.ncells, c0, c1);
    SRV_CUDA(s, cudaGetLastError());
    rr::launch_signal_f64(s->P, nb, Vnew, st);
    SRV_CUDA(s, cudaGetLastError());
  }
  SRV_CUDA(s, cudaStreamSynchronize(st));  // the host copies of the inputs may now go
  // the inputs are no longer needed on the host
  for (int i = n_surv; i < n; ++i) {
    Request& r = *s->res[i];
    std::vector<double>().swap(r.V);
    std::vector<double>().swap(r.kappa);
    std::vector<double>().swap(r.sigma);
  }
  return true;
}

// One IMEX step of every resident request, then the finished ones leave
// s->res (into `finished`, outputs copied) and the survivors keep their offsets.
bool step(rrmhd_server* s, std::vector<rrmhd_result>& finished, int64_t& zone_updates,
          double& busy) {
  const rr::Layout& L = s->L;
  const int n = L.n_inst;
  cudaStream_t st = s->stream;
  const double t_start = s->now();
  SRV_CUDA(s, cudaEventRecord(s->fork, st));
  const auto ranges = rr::lane_ranges(L.cell_off, n, (int)s->lanes.size());
  for (size_t l = 0; l < ranges.size(); ++l) {
    const LaneRt& ln = s->lanes[l];
    SRV_CUDA(s, cudaStreamWaitEvent(ln.stream, s->fork, 0));
    rr::enqueue_step(s->P, s->opts.precision, s->tune, s->B,
                     rr::make_batch(L, s->B, ranges[l].first, ranges[l].second), s->cur,
                     s->work + l, ln.stream, s->opts.ct);
    SRV_CUDA(s, cudaGetLastError());
    SRV_CUDA(s, cudaEventRecord(ln.done, ln.stream));
  }
  for (size_t l = 0; l < ranges.size(); ++l) SRV_CUDA(s, cudaStreamWaitEvent(st, s->lanes[l].done, 0));
  s->cur ^= 1;
  SRV_CUDA(s, cudaMemcpyAsync(s->h_t, s->B.t, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  SRV_CUDA(s, cudaMemcpyAsync(s->h_status, s->B.status, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
  SRV_CUDA(s, cudaMemcpyAsync(s->h_smax, s->B.smax, sizeof(unsigned long long) * n,
                              cudaMemcpyDeviceToHost, st));
  SRV_CUDA(s, cudaStreamSynchronize(st));

  zone_updates = 0;
  bool any_done = false;
  for (int i = 0; i < n; ++i) {
    Request& r = *s->res[i];
    const bool was_active = r.status == 0 && r.t < r.t_end;
    r.status = s->h_status[i];
    r.smax = s->h_smax[i];
    if (was_active && r.status == 0) {
      r.t = s->h_t[i];
      r.res.steps += 1;
      zone_updates += r.cells;
    }
    if (r.status != 0 || !(r.t < r.t_end)) any_done = true;
  }
  if (any_done) {
    const double* Vcur = s->cur ? s->B.Va : s->B.V0;
    for (int i = 0; i < n; ++i) {
      Request& r = *s->res[i];
      if (r.status == 0 && r.t < r.t_end) continue;
      const size_t w = sizeof(double) * r.cells;
      for (int k = 0; k < 12; ++k)
        SRV_CUDA(s, cudaMemcpyAsync(r.out + k * r.cells, Vcur + k * L.ncells + L.cell_off[i], w,
                                    cudaMemcpyDeviceToHost, st));
    }
    SRV_CUDA(s, cudaStreamSynchronize(st));
    const double t_done = s->now();
    std::vector<std::unique_ptr<Request>> keep;
    for (int i = 0; i < n; ++i) {
      std::unique_ptr<Request>& r = s->res[i];
      if (r->status == 0 && r->t < r->t_end) {
        keep.push_back(std::move(r));
        continue;
      }
      r->res.status = r->status;
      r->res.t = r->t;
      r->res.done_s = t_done;
      finished.push_back(r->res);
    }
    s->res = std::move(keep);
    s->dirty = true;
  }
  busy = s->now() - t_start;
  return true;
}

// Fails every request still held (after an engine error).
void fail_all(rrmhd_server* s) {
  std::lock_guard<std::mutex> lk(s->mu);
  const double t = s->now();
  auto fail = [&](Request& r) {
    r.res.status = RRMHD_ECUDA;
    r.res.t = r.t;
    r.res.done_s = t;
    s->done.push_back(r.res);
    s->st.completed += 1;
    s->st.failed += 1;
  };
  for (auto& r : s->res) fail(*r);
  for (auto& r : s->waiting) fail(*r);
  s->res.clear();
  s->waiting.clear();
  s->n_resident = s->resident_cells = s->resident_faces = 0;
  s->cv_idle.notify_all();
}

void engine_loop(rrmhd_server* s) {
  if (cudaSetDevice(s->device) != cudaSuccess) {
    set_failed(s, "cudaSetDevice failed on the engine thread");
    fail_all(s);
    return;
  }
  std::vector<rrmhd_result> finished;
  while (true) {
    std::vector<std::unique_ptr<Request>> adm;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || !s->waiting.empty() || !s->res.empty(); });
      if (s->stop) return;
      // admission in arrival order within the resident bounds
      std::vector<int64_t> cells, faces;
      for (const auto& r : s->waiting) {
        cells.push_back(r->cells);
        faces.push_back(r->faces);
      }
      const int k = rrmhd_server_admission(
          cells.data(), faces.data(), (int)cells.size(), s->max_cells - s->resident_cells,
          s->cap_faces - s->resident_faces, s->cap_slots - (int)s->n_resident);
      const double t = s->now();
      for (int j = 0; j < k; ++j) {
        std::unique_ptr<Request> r = std::move(s->waiting.front());
        s->waiting.pop_front();
        r->res.admit_s = t;
        s->n_resident += 1;
        s->resident_cells += r->cells;
        s->resident_faces += r->faces;
        adm.push_back(std::move(r));
      }
      s->st.admitted += k;
      s->st.peak_resident_cells = std::max(s->st.peak_resident_cells, s->resident_cells);
    }
    if (!adm.empty() || s->dirty) {
      const int n_surv = (int)s->res.size();
      for (auto& r : adm) s->res.push_back(std::move(r));
      if (!relayout(s, n_surv)) {
        fail_all(s);
        return;
      }
      s->dirty = false;
      std::lock_guard<std::mutex> lk(s->mu);
      s->st.relayouts += 1;
    }
    if (s->res.empty()) continue;
    finished.clear();
    int64_t zu = 0;
    double busy = 0.0;
    if (!step(s, finished, zu, busy)) {
      fail_all(s);
      return;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.steps += 1;
    s->st.zone_updates += zu;
    s->st.busy_s += busy;
    for (const rrmhd_result& r : finished) {
      s->done.push_back(r);
      s->st.completed += 1;
      if (r.status != RRMHD_OK) s->st.failed += 1;
      s->n_resident -= 1;
      s->resident_cells -= r.cells;
    }
    s->resident_faces = 0;
    for (const auto& r : s->res) s->resident_faces += r->faces;
    if (s->waiting.empty() && s->n_resident == 0) s->cv_idle.notify_all();
  }
}

void free_server(rrmhd_server* s) {
  for (LaneRt& l : s->lanes) {
    if (l.stream) cudaStreamDestroy(l.stream);
    if (l.done) cudaEventDestroy(l.done);
  }
  if (s->fork) cudaEventDestroy(s->fork);
  if (s->stream) cudaStreamDestroy(s->stream);
  rr::DeviceBufs& B = s->B;
  void* bufs[] = {B.inst,    B.cell_off, B.face_off, B.edge_off,  B.U0,          B.Ua,
                  B.Ub,      B.V0,       B.Va,       B.Vb,        B.Fhat,        B.bad,
                  B.bf0,     B.bfa,      B.bfb,      B.emf,       B.t,           B.t_end,
                  B.dt,      B.smax,     B.status,   s->kap[0],   s->kap[1],     s->sig[0],
                  s->sig[1], s->jcb[0],  s->jcb[1],  s->d_src_off, s->d_src_foff, s->work};
  for (void* p : bufs)
    if (p) cudaFree(p);
  void* hbufs[] = {s->h_t, s->h_tend, s->h_smax, s->h_status};
  for (void* p : hbufs)
    if (p) cudaFreeHost(p);
  delete s;
}

}  // namespace

extern "C" {

int rrmhd_server_admission(const int64_t* cells, const int64_t* faces, int n_waiting,
                           int64_t free_cells, int64_t free_faces, int free_slots) {
  if (!cells || !faces) return 0;
  int k = 0;
  while (k < n_waiting && k < free_slots && cells[k] <= free_cells && faces[k] <= free_faces) {
    free_cells -= cells[k];
    free_faces -= faces[k];
    ++k;
  }
  return k;
}

rrmhd_status rrmhd_server_create(const rrmhd_opts* opts, const rrmhd_server_config* cfg,
                                 rrmhd_server** out) {
  if (!out) return RRMHD_EINVAL;
  *out = nullptr;
  if (!opts || !rr::opts_ok(*opts)) return RRMHD_EINVAL;
  rrmhd_server_config c{};
  if (cfg) c = *cfg;
  if (c.mem_bytes < 0 || c.max_resident_cells < 0 || c.max_resident < 0) return RRMHD_EINVAL;
  const rrmhd_tuning& tu = c.tuning;
  const bool tuned = tu.face_block || tu.cell_block || tu.lanes;
  rr::Tuning tune = rr::default_tuning();
  int lanes = opts->lanes;
  if (tuned) {
    tune.faces = {tu.face_block, tu.face_per_thread, tu.face_persistent};
    tune.cells = {tu.cell_block, tu.cell_per_thread, tu.cell_persistent};
    lanes = tu.lanes;
    if (!rr::tuning_ok(tune) || lanes < 1) return RRMHD_EINVAL;
  }
  if (!rr::prepare_launch_shapes()) return RRMHD_ECUDA;

  rrmhd_server* s = new rrmhd_server();
  s->opts = *opts;
  s->opts.lanes = lanes;
  s->tune = tune;
  s->P = rr::make_params(*opts);
  s->t0 = Clock::now();
  auto fail = [&](rrmhd_status st) {
    free_server(s);
    return st;
  };
  if (cudaGetDevice(&s->device) != cudaSuccess) return fail(RRMHD_ECUDA);
  int64_t mem = c.mem_bytes;
  if (mem == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return fail(RRMHD_ECUDA);
    mem = (int64_t)(fr / 2);
  }
  s->cap_slots = c.max_resident > 0 ? c.max_resident : kDefaultSlots;
  s->cap_cells = (int64_t)(mem / (kBytesPerCell + kFacesPerCell * bytes_per_face(opts->ct)));
  if (c.max_resident_cells > 0) s->cap_cells = std::min(s->cap_cells, c.max_resident_cells);
  if (s->cap_cells < 1) return fail(RRMHD_EINVAL);
  s->cap_faces = (int64_t)(kFacesPerCell * (double)s->cap_cells) + 64;
  s->max_cells = s->cap_cells;

  const int64_t C = s->cap_cells, F = s->cap_faces, I = s->cap_slots;
  rr::DeviceBufs& B = s->B;
  bool ok = true;
  auto A = [&](void** p, size_t bytes) {
    if (ok && cudaMalloc(p, bytes) != cudaSuccess) ok = false;
  };
  for (double** p : {&B.U0, &B.Ua, &B.Ub, &B.V0, &B.Va, &B.Vb}) A((void**)p, sizeof(double) * 12 * C);
  for (int k = 0; k < 2; ++k) {
    A((void**)&s->kap[k], sizeof(double) * C);
    A((void**)&s->sig[k], sizeof(double) * C);
    A((void**)&s->jcb[k], sizeof(double) * 17 * C);
  }
  A((void**)&B.Fhat, sizeof(double) * 12 * F);
  A((void**)&B.bad, (size_t)C);
  A((void**)&B.inst, sizeof(InstDesc) * I);
  A((void**)&B.cell_off, sizeof(int64_t) * (I + 1));
  A((void**)&B.face_off, sizeof(int64_t) * 3 * (I + 1));
  A((void**)&B.edge_off, sizeof(int64_t) * 3 * (I + 1));
  if (opts->ct) {
    for (double** p : {&B.bf0, &B.bfa, &B.bfb}) A((void**)p, sizeof(double) * F);
    A((void**)&B.emf, sizeof(double) * 2 * F);
    A((void**)&s->d_src_foff, sizeof(int64_t) * 3 * I);
  }
  A((void**)&B.t, sizeof(double) * I);
  A((void**)&B.t_end, sizeof(double) * I);
  A((void**)&B.dt, sizeof(double) * I);
  A((void**)&B.smax, sizeof(unsigned long long) * I);
  A((void**)&B.status, sizeof(int) * I);
  A((void**)&s->d_src_off, sizeof(int64_t) * I);
  A((void**)&s->work, sizeof(rr::LaneCounters) * lanes);
  if (!ok) {
    cudaGetLastError();  // clear the allocation error
    return fail(RRMHD_ENOMEM);
  }
  if (cudaMallocHost((void**)&s->h_t, sizeof(double) * I) != cudaSuccess ||
      cudaMallocHost((void**)&s->h_tend, sizeof(double) * I) != cudaSuccess ||
      cudaMallocHost((void**)&s->h_smax, sizeof(unsigned long long) * I) != cudaSuccess ||
      cudaMallocHost((void**)&s->h_status, sizeof(int) * I) != cudaSuccess)
    return fail(RRMHD_ENOMEM);
  B.kappa = s->kap[0];
  B.sigma = s->sig[0];
  B.jc = s->jcb[0];
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming) != cudaSuccess)
    return fail(RRMHD_ECUDA);
  s->lanes.resize(lanes);
  for (LaneRt& l : s->lanes)
    if (cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&l.done, cudaEventDisableTiming) != cudaSuccess)
      return fail(RRMHD_ECUDA);
  // the fallback flags are written before they are read in every stage; zero once
  if (cudaMemset(B.bad, 0, (size_t)C) != cudaSuccess) return fail(RRMHD_ECUDA);
  s->st.cap_cells = s->cap_cells;
  s->st.cap_faces = s->cap_faces;
  s->engine = std::thread(engine_loop, s);
  *out = s;
  return RRMHD_OK;
}

rrmhd_status rrmhd_server_submit(rrmhd_server* s, const rrmhd_grid* grid, const double* V,
                                 const double* kappa, const double* sigma, double t_end,
                                 double* V_out, int64_t* id) {
  if (!s || !grid || !V || !kappa || !sigma || !V_out || !id) return RRMHD_EINVAL;
  std::string why;
  if (!rr::grid_ok(*grid, why) || t_end != t_end) return RRMHD_EINVAL;
  auto r = std::make_unique<Request>();
  r->grid = *grid;
  r->cells = rr::grid_cells(*grid);
  r->faces = rr::grid_faces(*grid);
  if (s->opts.ct) {
    int64_t edges = 0;
    for (int e = 0; e < 3; ++e) edges += rr::grid_edges(*grid, e);
    r->faces = std::max(r->faces, (edges + 1) / 2);
  }
  if (r->cells > s->max_cells || r->faces > s->cap_faces) return RRMHD_ECAPACITY;
  r->V.assign(V, V + 12 * r->cells);
  r->kappa.assign(kappa, kappa + r->cells);
  r->sigma.assign(sigma, sigma + r->cells);
  r->t_end = t_end;
  r->out = V_out;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->failed) return RRMHD_ECUDA;
  r->id = s->next_id++;
  r->res.id = r->id;
  r->res.cells = r->cells;
  r->res.submit_s = s->now();
  *id = r->id;
  s->waiting.push_back(std::move(r));
  s->st.submitted += 1;
  s->cv_work.notify_one();
  return RRMHD_OK;
}

int rrmhd_server_poll(rrmhd_server* s, rrmhd_result* out, int max) {
  if (!s || !out || max <= 0) return 0;
  std::lock_guard<std::mutex> lk(s->mu);
  const int k = std::min<int>(max, (int)s->done.size());
  std::copy(s->done.begin(), s->done.begin() + k, out);
  s->done.erase(s->done.begin(), s->done.begin() + k);
  return k;
}

rrmhd_status rrmhd_server_wait_idle(rrmhd_server* s, double timeout_s) {
  if (!s || !(timeout_s >= 0.0)) return RRMHD_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  const bool idle = s->cv_idle.wait_for(
      lk, std::chrono::duration<double>(timeout_s),
      [&] { return s->failed || (s->waiting.empty() && s->n_resident == 0); });
  if (s->failed) return RRMHD_ECUDA;
  return idle ? RRMHD_OK : RRMHD_ETIMEOUT;
}

rrmhd_status rrmhd_server_get_stats(rrmhd_server* s, rrmhd_server_stats* st) {
  if (!s || !st) return RRMHD_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *st = s->st;
  st->resident = s->n_resident;
  st->resident_cells = s->resident_cells;
  st->pending = (int64_t)s->waiting.size();
  return RRMHD_OK;
}

const char* rrmhd_server_last_error(rrmhd_server* s) {
  if (!s) return "null server";
  std::lock_guard<std::mutex> lk(s->mu);
  return s->err.c_str();
}

void rrmhd_server_destroy(rrmhd_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->engine.joinable()) s->engine.join();
  if (s->stream) cudaStreamSynchronize(s->stream);
  free_server(s);
}

}  // extern "C"
