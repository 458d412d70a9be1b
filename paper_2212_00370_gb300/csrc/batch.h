// batch.h -- device layout of a batch of independent instances (ragged 1D, 2D
// and 3D grids) and the launchers of the stage kernels.  Internal to librrmhd.
//
// Layout (all device, structure of arrays):
//   cells  : instance i owns cells [cell_off[i], cell_off[i+1]) of every plane,
//            row-major with x fastest;  U, V planes are [12][ncells].
//   faces  : direction-major; faces normal to d of instance i are
//            [dir_base[d] + face_off[d][i], ... + nfaces(i,d)), each instance's
//            block row-major over (n + e_d) with x fastest;  Fhat is [12][nfaces].
//   edges  : (constrained transport, 2D/3D instances) direction-major like the
//            faces; edges along e of instance i are [edge_base[e] + edge_off[e][i],
//            ...), row-major over m_d = n_d + 1 for the directions d != e in use
//            (2D: edges along z only).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "physics_f64.cuh"

namespace rr {

struct InstDesc {
  int ndim;
  int n[3];
  int bc[3];  // 0 outflow, 1 periodic (both sides of the direction)
  double dx[3];
  int64_t cell_off;
  int64_t face_off[3];  // within the direction's block
  int64_t edge_off[3];  // within the edge direction's block (constrained transport)
};

// Per-instance time-stepping state (device arrays of length n_inst).
struct InstState {
  double* t;
  double* t_end;
  double* dt;
  unsigned long long* smax;  // max_cells sum_d lambda_d/dx_d, as the bits of a non-negative double
  int* status;               // 0 ok, else the first failing Status
  const double* dt_max;      // [1] cap on every instance's dt (+inf: none), or null
  long long* bad_cell;       // lowest index of a cell whose failure froze the instance
                             // (LLONG_MAX: none), or null
};

struct Batch {
  int n_inst;
  int64_t ncells;
  int64_t nfaces;
  int64_t dir_base[4];       // faces of direction d: [dir_base[d], dir_base[d+1])
  const InstDesc* inst;      // [n_inst]
  const int64_t* cell_off;   // [n_inst + 1]
  const int64_t* face_off;   // [3][n_inst + 1] (prefix sums within each direction)
  const int64_t* edge_off;   // [3][n_inst + 1] (constrained transport)
  int64_t edge_base[4];      // edges along e: [edge_base[e], edge_base[e+1])
  InstState st;
  // the part of the batch a launch covers (a lane: contiguous instances)
  int i_begin, i_end;        // instances
  int64_t c_begin, c_end;    // cells
  int64_t f_begin[3];        // faces of direction d: [f_begin[d], f_begin[d] + f_count[d])
  int64_t f_count[3];
  int64_t e_begin[3];        // edges along e: [e_begin[e], e_begin[e] + e_count[e])
  int64_t e_count[3];
};

// Passes of the admissibility fallback: a cell that a pass updates again and
// that still has no admissible update flags its own faces for the next pass.
constexpr int kFallbackPasses = 3;

// Device counters of one lane: the chunk counters of its persistent launches and,
// per stage, how many cells each fallback pass flagged (a pass with none returns
// at once).  Zeroed on the lane's stream by the step that uses them.
struct LaneCounters {
  unsigned long long work[2];
  unsigned int flagged[3][kFallbackPasses + 1];
};

struct StageArgs {
  Params P;
  Batch b;
  int stage;               // 1, 2, 3
  const double* U0;        // U^(0) (state at the start of the step)
  const double* V0;        // V^(0)
  const double* Us;        // U^(s-1)
  const double* Vs;        // V^(s-1)
  const double* kappa;
  const double* sigma;
  double* Fhat;            // [12][fstride]; face g is stored at column g - out_base
  float* Fhat32;           // FP32-bulk form: same layout in FP32
  int64_t fstride;
  int64_t out_base;
  int check_active;        // skip instances that are finished or failed
  double* Uout;            // must not alias U0, Us, Vs (the fallback pass re-reads them)
  double* Vout;
  int32_t* cell_status;    // optional per-cell status
  uint8_t* bad;            // [ncells] fallback flags: p > 0 = flagged in pass p, 0 = not flagged
  int fb_pass;             // the admissibility-fallback pass a fallback launch runs, 1..kFallbackPasses
                           // (0: the main path)
  unsigned int* flagged;   // [kFallbackPasses + 1]: cells flagged with value p in this stage, or null
  double* jc;              // [17][ncells] per-cell Jacobian cache of the implicit solve
  unsigned long long* work;  // [2] chunk counters of persistent face / cell launches
  // constrained transport (2D/3D instances when ct != 0): the staggered normal
  // field per face (one value per face, the face layout) at the step start (b0),
  // the stage input (bs) and output (bout); the edge EMFs of the stage.
  int ct;
  int fp32_fluxes;  // the face fluxes are the FP32 ones (FP32-bulk form)
  const double* b0;
  const double* bs;
  double* bout;
  double* emf;
};

// How a kernel spreads its work items over threads (launch_shape.cuh).
struct LaunchShape {
  int block = 128;      // threads per block: 32, 64, 128, 256
  int per_thread = 1;   // items per thread of the grid schedule: 1, 2
  int persistent = 0;   // 1: resident grid, warps take 32-item chunks from a counter
};

struct Tuning {
  LaunchShape faces, cells;
};

// FP64 path (bit-compatible with the oracle's arithmetic order).  A persistent
// shape needs a.work zeroed on the stream before the launch (the launchers do it).
void launch_faces_f64(const StageArgs& a, const LaunchShape& sh, cudaStream_t s);
void launch_cells_f64(const StageArgs& a, const LaunchShape& sh, cudaStream_t s);
// one pass of the admissibility fallback (a.fb_pass): its faces, then (constrained
// transport) the EMFs and the face field again, then its cells
void launch_fallback_f64(const StageArgs& a, cudaStream_t s);
void launch_signal_f64(const Params& P, const Batch& b, const double* V, cudaStream_t s);
// constrained transport: edge EMFs (CT-contact) and the face-field stage update
void launch_emf_f64(const StageArgs& a, cudaStream_t s);
void launch_bface_f64(const StageArgs& a, cudaStream_t s);
// face field <-> cell-centred B (set-up), and periodic duplicate faces made equal
void launch_faces_from_cells_f64(const Batch& b, const double* V, double* bface, cudaStream_t s);
void launch_cells_from_faces_f64(const Batch& b, const double* bface, double* V, cudaStream_t s);
void launch_ct_canonical_f64(const Batch& b, double* bface, cudaStream_t s);

// FP32-bulk form: FP32 faces (tangent PVM products), FP64 cells
void launch_faces_f32(const StageArgs& a, const LaunchShape& sh, cudaStream_t s);
void launch_cells_f32(const StageArgs& a, const LaunchShape& sh, cudaStream_t s);
void launch_fallback_f32(const StageArgs& a, cudaStream_t s);
void launch_widen_f32(const float* F32, int64_t fstride32, int64_t f_begin, int64_t n, double* F,
                      cudaStream_t s);
// Resolves the resident-grid sizes of the persistent kernels (occupancy queries);
// call once per device before any stream capture.  Returns false on a CUDA error.
bool prepare_launch_shapes();
bool prepare_launch_shapes_f64();
bool prepare_launch_shapes_f32();
void launch_begin_step(const Params& P, const Batch& b, cudaStream_t s);
// U -= dt_weight / dx_dir (F_right - F_left) at every cell of the batch from the face
// fluxes of direction dir (F64 stride fstride, or the FP32 ones when F32 is not null)
void launch_flux_accumulate(const Batch& b, int dir, double dt_weight, const double* F64,
                            const float* F32, int64_t fstride, int64_t out_base, double* U,
                            cudaStream_t s);
void launch_fill_i64(long long* p, int64_t n, long long v, cudaStream_t s);
void launch_set_f64(double* p, double v, cudaStream_t s);
void launch_end_step(const Batch& b, cudaStream_t s);
void launch_prim2con_f64(const Params& P, const double* V, double* U, int64_t n, cudaStream_t s);
void launch_con2prim_f64(const Params& P, const double* U, const double* Zg, double* V,
                         int32_t* status, int64_t n, cudaStream_t s);
void launch_prim_Z_f64(const Params& P, const double* V, double* Z, int64_t n, cudaStream_t s);
void launch_implicit_f64(const Params& P, const Batch& b, double hdt, const double* Us,
                         const double* Zg, const double* kappa, const double* sigma, double* U,
                         double* V, int32_t* status, cudaStream_t s);

}  // namespace rr
