/*
 * rrmhd.h -- C ABI of the GB300 (sm_103a) finite-volume IMEX update of gray-M1
 * relativistic radiation magnetohydrodynamics with the PVM-int-8 Jacobian-free
 * Riemann solver (Lopez-Miralles, Marti & Perucho 2022, arXiv:2212.00370).
 *
 * The system (Sec. 2.1, Eq. eq0) is  d_t U + d_i F^i = S  with twelve
 * conserved variables (Eq. eqU) and primitives, both structure-of-arrays:
 *   U = (D, S^x, S^y, S^z, tau_e, B^x, B^y, B^z, E_r, F_r^x, F_r^y, F_r^z)
 *   V = (rho, v^x, v^y, v^z, p, B^x, B^y, B^z, E_r, F_r^x, F_r^y, F_r^z)
 * in code units c = 1, T = p/rho, 4 pi B = a_R T^4 (Sec. 2.1).
 *
 * A context holds a BATCH of independent instances (a single problem is a batch
 * of one).  Each instance is a 1D, 2D or 3D Cartesian grid with its own cell
 * sizes, boundaries, opacities, time, end time and time step.  Fields of all
 * instances are packed: instance i owns cells [off[i], off[i+1]) of every
 * plane (rrmhd_cell_offsets), each grid row-major with x fastest, and a field
 * of the context is double[12][ncells] (plane k at k*ncells).
 *
 * Conventions for every entry point:
 *  - Pointers are DEVICE pointers (CUDA global memory) unless marked "host".
 *    The caller owns them; the library never frees or retains them.
 *  - Work is enqueued on the CUDA stream given to rrmhd_create and is
 *    asynchronous unless the function returns host data.
 *  - Errors are returned as rrmhd_status, never by trap or exception; the text
 *    of the last error is available from rrmhd_last_error.  Argument errors
 *    return RRMHD_EINVAL before any work is enqueued.  Per-cell numerical
 *    failures (no con2prim root, no implicit solution) freeze the instance they
 *    occur in and are reported per instance by rrmhd_get_inst_status.
 *  - FP64 arithmetic follows one fixed IEEE operation order (no fused
 *    multiply-add), so results are reproducible bit for bit.
 */
#ifndef RRMHD_H
#define RRMHD_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RRMHD_OK = 0,
    RRMHD_EC2P = 1,       /* con2prim found no admissible root                  */
    RRMHD_EIMPLICIT = 2,  /* implicit radiation-matter solve did not converge   */
    RRMHD_EUNPHYS = 3,    /* inadmissible state (D <= 0, E_r <= 0, NaN speeds)  */
    RRMHD_EINVAL = 10,    /* invalid argument                                   */
    RRMHD_ENOMEM = 11,    /* device allocation failed                           */
    RRMHD_ECUDA = 12,     /* CUDA runtime error                                 */
    RRMHD_ECAPACITY = 13, /* input larger than a fixed capacity (alloc-free scratch, server budget) */
    RRMHD_ETIMEOUT = 14   /* a server still had work when the wait ran out           */
} rrmhd_status;

enum { RRMHD_RECON_GODUNOV = 0, RRMHD_RECON_MINMOD = 1, RRMHD_RECON_MC = 2, RRMHD_RECON_VANLEER = 3 };
enum { RRMHD_BC_OUTFLOW = 0, RRMHD_BC_PERIODIC = 1 };
enum { RRMHD_FP64 = 0, RRMHD_FP32_BULK = 1 };
enum { RRMHD_SOLVER_PVM = 0, RRMHD_SOLVER_RADHLL = 1 };
enum { RRMHD_CLOSURE_M1 = 0 };  /* the gray M1 closure, Eq. xi (Sec. 2.2) */

/* One instance's grid.  Unused directions: n = 1, dx = 1.  bc applies to both
 * sides of a direction: outflow copies the edge cell into the two ghost layers
 * that PLM needs, periodic wraps (Sec. 4 test set-ups). */
typedef struct {
    int    ndim;   /* 1, 2 or 3                    */
    int    n[3];   /* cells per direction (>= 1)   */
    double dx[3];  /* cell size per direction (> 0) */
    int    bc[3];  /* RRMHD_BC_* per direction     */
} rrmhd_grid;

/* Scheme options shared by all instances of a context. */
typedef struct {
    double gamma;      /* ideal-gas adiabatic index, Eq. eos (> 1)                       */
    double a_rad;      /* radiation constant a_R, 4 pi B = a_R T^4 (>= 0)                 */
    double cfl;        /* Courant number of dt = cfl / max sum_d lambda_d/dx_d            */
    double pvm_eps;    /* epsilon of the nested flux differences, Sec. 3.2.2 (1e-8)        */
    int    recon;      /* RRMHD_RECON_* (Sec. 3.2); VanLeer is the paper's default         */
    int    beta_mode;  /* 1: beta = min(1/tau_L, 1/tau_R, 1) (Eq. beta); 0: beta = 1;
                          2: Eq. beta on the radiation components (E_r, F_r) of the PVM
                          viscosity and beta = 1 on the magnetofluid ones (a variant: the
                          paper leaves other choices of beta open, Sec. 5)             */
    int    precision;  /* RRMHD_FP64 (reproducible) or RRMHD_FP32_BULK                     */
    int    c2p_maxit;  /* Newton iterations allowed in con2prim (60)                       */
    int    imp_maxit;  /* iterations allowed in one implicit Newton solve (50)             */
    double imp_tol;    /* implicit convergence: full Newton step <= imp_tol * E_r (1e-10)  */
    int    lanes;      /* independent sub-batches stepped on their own streams (8); the
                          instances are split into contiguous ranges of about equal cell
                          count, so one range's slow cells overlap the others' work     */
    int    pvm_k;      /* PVM-int-n with n = 2^pvm_k (Eq. iterat): 3 = PVM-int-8, the paper's
                          solver (4 A^2 products per face, default); 4 = PVM-int-16 (8)  */
    int    pvm_products; /* how the FP64 form takes the Jacobian products A w of the PVM
                          viscosity: 0 = nested flux differences with eps = pvm_eps, the
                          paper's (Eq. utilde; default; bit-reproducible against the
                          reference arithmetic); 1 = exact tangent (dual-number) products,
                          the root of con2prim differentiated by the implicit-function
                          theorem: no Newton iteration per product.  The FP32-bulk form
                          always uses tangent products (eps is below FP32 resolution). */
    int    solver;     /* RRMHD_SOLVER_PVM (Sec. 3.2.2, default) or RRMHD_SOLVER_RADHLL: the
                          radiative HLL of Sec. 3.2.1, HLL per block with the fast-
                          magnetosonic speeds for the magnetofluid and lambda_r1/lambda_r3
                          (Eqs. lam1-lam3) for the radiation, the latter capped at
                          4/(3 tau) (Eq. limits) when beta_mode = 1 or 2                 */
    int    ct;         /* 1: constrained transport of the magnetic field on 2D/3D instances
                          (CT-contact EMFs of Gardiner & Stone 2005, the scheme the paper's
                          multi-D runs use, Sec. 4): the normal field lives on the faces,
                          cell-centred B is the mean of the two faces, and the discrete
                          divergence is kept to round-off.  In the FP32-bulk form the EMFs
                          are formed in FP64 from the FP32 fluxes.  0: cell-centred B
                          updated by its fluxes (default).                               */
    int    closure;    /* the radiation closure: RRMHD_CLOSURE_M1 (Sec. 2.2, Eq. xi), the
                          one the paper uses and the only one built (EINVAL otherwise)   */
} rrmhd_opts;

typedef struct rrmhd_ctx rrmhd_ctx;

/* Fills o with the paper's defaults (gamma 5/3, a_R 1, CFL 0.4, eps 1e-8, VanLeer,
 * beta on, FP64).  o: host. */
void rrmhd_default_opts(rrmhd_opts* o);

/* Creates a context for n_inst instances (grids: host array of n_inst) on the
 * given CUDA stream (cudaStream_t, NULL = legacy default stream) of the current
 * device, and allocates its device state.  Opacities default to 0, times to
 * t = 0, t_end = +inf.  The problem statement is Sec. 2 (Eqs. eq0-xi).
 * Returns EINVAL for bad grids/options, ENOMEM if allocation fails. */
rrmhd_status rrmhd_create(int n_inst, const rrmhd_grid* grids, const rrmhd_opts* opts,
                          void* cuda_stream, rrmhd_ctx** out);

/* Releases the context and its device memory (synchronises its stream). */
void rrmhd_destroy(rrmhd_ctx* ctx);

/* Number of instances / cells of all instances / faces normal to dir (0..2). */
int     rrmhd_num_instances(const rrmhd_ctx* ctx);
int64_t rrmhd_num_cells(const rrmhd_ctx* ctx);
int64_t rrmhd_num_faces(const rrmhd_ctx* ctx, int dir);

/* Cell offsets of the packed layout: off (host, n_inst+1). */
rrmhd_status rrmhd_cell_offsets(const rrmhd_ctx* ctx, int64_t* off);

/* Face offsets of direction dir: instance i owns faces [off[i], off[i+1]) of a
 * flux array of that direction, each block row-major over (n + e_dir). off: host,
 * n_inst+1. */
rrmhd_status rrmhd_face_offsets(const rrmhd_ctx* ctx, int dir, int64_t* off);

/* Absorption kappa and scattering sigma_s (comoving, per unit mass; Eqs. g0, gi)
 * per cell: kappa, sigma: double[ncells].  Copied into the context. */
rrmhd_status rrmhd_set_opacity(rrmhd_ctx* ctx, const double* kappa, const double* sigma);

/* Sets the state from primitives V: double[12][ncells] (copied); computes U by
 * Eq. eqU and the CFL signal speeds. */
rrmhd_status rrmhd_set_state(rrmhd_ctx* ctx, const double* V);

/* Copies the current conserved (U) and/or primitive (V) state out:
 * double[12][ncells] each; either may be NULL. */
rrmhd_status rrmhd_get_state(const rrmhd_ctx* ctx, double* U, double* V);

/* Checkpoints.  A checkpoint holds everything that determines the context's future
 * steps apart from its grids, options and launch shapes: U and V, kappa and sigma,
 * the per-cell Jacobian cache of the implicit solve (Sec. 3.3), the staggered face
 * field (ct = 1), and per instance t, t_end, the last dt, the CFL signal maximum, the
 * status and the first bad cell.  Restoring it, into the same context or into
 * another one created with the same grids and options (any launch shapes), and
 * stepping on gives bit for bit the results of the run that wrote it, which a
 * restart through rrmhd_set_state (Jacobian cache emptied) does not.
 * rrmhd_checkpoint_bytes: the size of the buffer (0 for a NULL context).
 * rrmhd_checkpoint_save: writes into buf, caller-owned device or host memory of that
 *   size (pinned host memory keeps the copy asynchronous); enqueued on the context's
 *   stream, so synchronise before reading a host buffer.
 * rrmhd_checkpoint_restore: reads buf (device or host); synchronises the stream to
 *   read the header first; RRMHD_EINVAL if the checkpoint was written by a context
 *   of another layout (instances, cells, faces), precision or ct setting. */
size_t       rrmhd_checkpoint_bytes(const rrmhd_ctx* ctx);
rrmhd_status rrmhd_checkpoint_save(rrmhd_ctx* ctx, void* buf);
rrmhd_status rrmhd_checkpoint_restore(rrmhd_ctx* ctx, const void* buf);

/* Per-instance current time and end time (host, n_inst each); an instance
 * stops once t reaches t_end (the last step is clipped to land on it). */
rrmhd_status rrmhd_set_times(rrmhd_ctx* ctx, const double* t, const double* t_end);

/* Per-instance time and the size of the last step taken (host, n_inst each;
 * either may be NULL).  Synchronises the stream. */
rrmhd_status rrmhd_get_times(const rrmhd_ctx* ctx, double* t, double* dt_last);

/* Per-instance status (host int32[n_inst]): 0 ok, else the rrmhd_status of the
 * first cell failure.  Failed instances are frozen.  Synchronises the stream. */
rrmhd_status rrmhd_get_inst_status(const rrmhd_ctx* ctx, int32_t* status);

/* Advances every live instance by nsteps IMEX-RK3 steps (Sec. 3.1): each
 * step takes dt = cfl / max sum_d lambda_d/dx_d (clipped to t_end) and runs
 * three stages of {PLM + PVM-int-8 flux at every face (Sec. 3.2), flux
 * difference and RK combination (Eq. explicit), implicit radiation-matter solve
 * (Sec. 3.3)} with implicit weights 1, 1/4, 2/3.  A cell whose update has no
 * admissible state (no con2prim root, or no converged implicit solve) gets the
 * first-order Rusanov flux at its faces and is updated again with its neighbours,
 * in up to three passes (a neighbour that then fails is flagged in turn); only a
 * failure after that freezes the instance.  Enqueued as one CUDA graph per step
 * and lane; the lanes (independent instance ranges) run their nsteps steps back
 * to back and join the context's stream once, so one call of nsteps steps gives
 * the same results as nsteps calls of one step, and can take less time.  Returns
 * without synchronising. */
rrmhd_status rrmhd_imex_step(rrmhd_ctx* ctx, int nsteps);

/* One step as rrmhd_imex_step takes it, with every instance's dt capped:
 * dt = min(cfl / max sum_d lambda_d/dx_d, dt_max), then clipped to t_end.  dt_max
 * (> 0; +inf: no cap) applies to this call only.  dt_taken (host double[n_inst],
 * may be NULL) receives each instance's dt (0 for an instance that did not step);
 * with it the call synchronises the stream.  EINVAL for dt_max <= 0 or NaN. */
rrmhd_status rrmhd_imex_step_dt(rrmhd_ctx* ctx, double dt_max, double* dt_taken);

/* Per instance (host int64[n_inst]): the packed index of the lowest-numbered cell
 * whose failure (no con2prim root, no implicit solution, after the admissibility
 * fallback) froze the instance, or -1 if none did (also for an instance frozen by
 * a NaN or non-positive time step, which no single cell causes).  Reset by
 * rrmhd_set_state.  Synchronises the stream. */
rrmhd_status rrmhd_get_first_bad_cell(const rrmhd_ctx* ctx, int64_t* cell);

/* Same as rrmhd_imex_step, from and to HOST buffers: copies V_in (host
 * double[12][ncells], pinned memory recommended) to the device, takes nsteps steps
 * and copies the primitives back to V_out (host).  Synchronous.  If V_in equals
 * the context's current primitives bit for bit (a run that continues from the last
 * V_out), the run continues exactly as rrmhd_imex_step would: the per-cell
 * implicit-solver history, statuses and CFL speeds are kept.  Otherwise V_in becomes
 * the state as with rrmhd_set_state. */
rrmhd_status rrmhd_imex_step_host(rrmhd_ctx* ctx, const double* V_in, double* V_out, int nsteps);

/* Pointwise Eq. eqU on caller buffers: V, U double[12][n]. */
rrmhd_status rrmhd_prim2con(rrmhd_ctx* ctx, const double* V, double* U, int64_t n);

/* Pointwise con2prim (the inversion Sec. 3.2.2 step 2 refers to; Newton-Raphson
 * of Mignone & McKinney 2007 in W' = rho h W^2 - D): U double[12][n] -> V
 * double[12][n]; Zguess double[n] (rho h W^2 warm start) or NULL; status
 * int32[n] (0 ok, RRMHD_EC2P, RRMHD_EUNPHYS) or NULL.  V is zero where it fails. */
rrmhd_status rrmhd_con2prim(rrmhd_ctx* ctx, const double* U, const double* Zguess, double* V,
                            int32_t* status, int64_t n);

/* Numerical flux (Eqs. generalflux, beta; Sec. 3.2.2 steps 1-7) at every face
 * normal to dir of every instance, from the context's current primitives:
 * PLM reconstruction with the Godunov fallback (Sec. 3.2), then
 * F^ = (F_L + F_R)/2 - beta p_3(A) (U_R - U_L)/2 with p_3 the degree-8 internal
 * approximation of |x| (Eq. iterat), A^2 products by nested flux differences.
 * Fhat: double[12][num_faces(dir)] laid out as rrmhd_face_offsets(dir). */
rrmhd_status rrmhd_flux_sweep(rrmhd_ctx* ctx, int dir, double* Fhat);

/* The flux sweep accumulated into a state (Eq. explicit, one direction): computes the
 * numerical flux at every face normal to dir from the context's current primitives,
 * as rrmhd_flux_sweep does, and updates U (double[12][ncells], the caller's, e.g. a
 * copy of the context's U) in place:
 *   U -= dt_weight / dx_dir (F^_{i+1/2} - F^_{i-1/2})
 * at every cell of every instance (instances with fewer than dir+1 dimensions are
 * left unchanged).  The FP64 form uses the FP64 operation order of the stage's flux
 * difference; the FP32-bulk form differences its FP32 fluxes in FP32.  dt_weight >= 0.
 * Uses the context's face buffer (not thread-safe against a concurrent step). */
rrmhd_status rrmhd_flux_accumulate(rrmhd_ctx* ctx, int dir, double dt_weight, double* U);

/* Implicit radiation-matter step of every cell (Sec. 3.3, Eqs. timeadv, totale,
 * totalm): solves E_r = E* - h G^0, F_r = F* - h G^i (Eqs. g0, gi) with
 * tau_e + E_r and S + F_r conserved and the matter recovered by con2prim.
 * hdt: the implicit weight times dt.  Ustar: double[12][ncells] (U*);
 * Zguess: double[ncells] warm start or NULL; opacities from the context.
 * U, V: double[12][ncells] results; status: int32[ncells] or NULL. */
rrmhd_status rrmhd_implicit_source(rrmhd_ctx* ctx, double hdt, const double* Ustar,
                                   const double* Zguess, double* U, double* V, int32_t* status);

/* One IMEX-RK3 step exactly as rrmhd_imex_step takes it, but launched without
 * the CUDA graph and with CUDA events recorded on the context's stream between
 * launch groups; synchronises.  ms (host, 4): total device time of
 * [0] the 3 face-flux launches, [1] the 3 cell-update launches,
 * [2] the 18 admissibility-fallback launches (3 passes of faces and cells in
 * each stage), [3] the 2 per-instance time-step launches. */
rrmhd_status rrmhd_profile_step(rrmhd_ctx* ctx, double* ms);

/* Kernel launches one rrmhd_imex_step step enqueues (for launch accounting). */
int rrmhd_launches_per_step(const rrmhd_ctx* ctx);

/* ---- Launch shapes and the autotuner (no counterpart in the paper) ----------
 * How the face and cell kernels spread their work over threads, and into how many
 * concurrent lanes a context splits its instances.  Shapes never change results:
 * every face and cell is computed once, by the same arithmetic, whatever the
 * shape (bit-identical output).
 *   *_block        threads per block: 32, 64, 128 or 256; also 8 or 16 for the
 *                  grid schedule with one item per thread (partial warps: a small
 *                  grid spread over more SMs)
 *   *_per_thread   faces or cells per thread of the grid schedule: 1 or 2
 *   *_persistent   1: a resident grid (SMs x resident blocks per SM) whose warps take
 *                  chunks of 32 consecutive items from a counter until none are
 *                  left (per_thread must be 1); 0: one thread per item(s)
 *   lanes          >= 1; see rrmhd_opts.lanes
 * Defaults: 128 threads, 1 item per thread, grid schedule, opts.lanes. */
typedef struct {
    int face_block, face_per_thread, face_persistent;
    int cell_block, cell_per_thread, cell_persistent;
    int lanes;
} rrmhd_tuning;

/* The context's current shapes (host out). */
rrmhd_status rrmhd_get_tuning(const rrmhd_ctx* ctx, rrmhd_tuning* t);

/* Sets the shapes (host in); EINVAL for a shape that is not compiled.  Synchronises
 * the context's stream; the next step rebuilds its CUDA graphs. */
rrmhd_status rrmhd_set_tuning(rrmhd_ctx* ctx, const rrmhd_tuning* t);

/* Chooses the shapes for this context's batch by timing real steps from its
 * current state: coordinate descent over the cell shapes, then the face shapes,
 * then the lane count; each candidate is timed over `repeats` steps (CUDA events
 * on the context's stream, the fastest counts), each taken from the same saved state.  The
 * state, times and statuses are restored afterwards, so the context continues as
 * if no step had been taken; the fastest shapes are kept.  best (host, may be
 * NULL) receives them, best_ms (host, may be NULL) their best step time.  Allocates
 * a copy of the state for the duration of the call (ENOMEM if that fails). */
rrmhd_status rrmhd_autotune(rrmhd_ctx* ctx, int repeats, rrmhd_tuning* best, double* best_ms);

/* Staggered magnetic field of a context with opts.ct = 1: one value per face, the
 * component normal to the face, in the face layout of the fluxes (directions 0, 1, 2
 * one after the other, num_faces(dir) each; 1D instances' faces are unused).
 * rrmhd_set_state starts it from the cell-centred B (mean of the two cells next to
 * each face).  rrmhd_set_face_field replaces it (a divergence-free field should come
 * from a discrete vector potential); in periodic directions the faces at index 0 and
 * n are the same face, and face 0's value is kept for both.  Either call then resets
 * the cell-centred B of the state to the face means and recomputes U.  b: device
 * double[sum_dir num_faces(dir)].  EINVAL if opts.ct is 0. */
rrmhd_status rrmhd_set_face_field(rrmhd_ctx* ctx, const double* b);
rrmhd_status rrmhd_get_face_field(const rrmhd_ctx* ctx, double* b);

/* rho h W^2 of primitives: V double[12][n] -> Z double[n] (con2prim warm starts). */
rrmhd_status rrmhd_prim_z(rrmhd_ctx* ctx, const double* V, double* Z, int64_t n);

/* ---- FP64 throughput probe (not a step of the method) ------------------------
 * The cell and face kernels are bound by the FP64 pipe; this measures that pipe's
 * rate on the current device, the denominator of their roofline.  Every thread of
 * 8 blocks of 256 per SM runs eight independent DFMA chains (the pipe, not one
 * chain's latency, is the limit); a short run calibrates the trip count so that one
 * run takes about target_ms (host, ms, in (0, 10000]); the best of three runs, timed
 * with CUDA events on cuda_stream (NULL = legacy default), is returned in
 * *inst_per_s (host): thread-level FP64 instructions per second, the unit of the
 * ncu counters sm__sass_thread_inst_executed_op_d{add,mul,fma}.  Synchronises the
 * stream.  EINVAL for a bad argument, ECUDA if a launch or event fails. */
rrmhd_status rrmhd_probe_fp64(void* cuda_stream, double target_ms, double* inst_per_s);

/* Latency of a dependent FP64 instruction: one warp, one chain of 65,536 dependent
 * DFMA per thread, best of three runs timed with CUDA events on cuda_stream; *ns_per_inst
 * (host) receives nanoseconds per instruction.  This is what bounds a grid too small
 * to put several warps on every SM.  Synchronises the stream.  EINVAL for a NULL
 * output, ECUDA if a launch or event fails. */
rrmhd_status rrmhd_probe_fp64_latency(void* cuda_stream, double* ns_per_inst);

/* ---- Alloc-free entry point (no counterpart in the paper) ----------------
 * For callers that cannot allocate device memory themselves, e.g. a host program
 * whose GPU memory is all owned by its own pool or fixed arena, reserved at
 * start-up, so that no library may call cudaMalloc on its path.  It computes the
 * CFL time step of one grid, dt = cfl / max_cells sum_d lambda_d / dx_d: the same
 * signal speeds and the same value, bit for bit, as the time step
 * rrmhd_imex_step takes from that state (before any clipping to t_end).
 * grid: host, one 1D/2D/3D grid; opts: host (gamma and cfl are used); V: device
 * double[12][ncells] primitives; dt: device double[1] output; cuda_stream: the
 * stream to enqueue on (NULL = legacy default).  No device memory is allocated
 * or freed: the reduction's scratch is a fixed array inside this library
 * (about 32 KB), present on every GPU that loads the library until the process
 * exits.  It holds up to RRMHD_NOALLOC_MAX_CELLS cells; larger grids return
 * RRMHD_ECAPACITY before any work is enqueued.  The first call on a device looks
 * up the scratch's device address and keeps it for the life of the process; make
 * that first call before any stream capture (a lookup that fails returns ECUDA
 * and is tried again by the next call).  All calls on a device share the one scratch array
 * (each call first resets the part that must start at zero): calls that overlap
 * on the GPU -- on different streams, or from different host threads without
 * ordering -- race and return wrong values.  A NaN signal speed gives dt = NaN.
 * Returns EINVAL for bad arguments, ECUDA if the set-up or launch fails. */
#define RRMHD_NOALLOC_MAX_CELLS 33554432
rrmhd_status rrmhd_cfl_dt_noalloc(const rrmhd_grid* grid, const rrmhd_opts* opts, const double* V,
                                  double* dt, void* cuda_stream);

/* ---- Serving loop (no counterpart in the paper) ------------------------------
 * A server accepts solve requests -- one 1D, 2D or 3D grid with its primitive state,
 * opacities and end time each -- at any moment, from any host thread, and runs them
 * to completion on the current device with continuous batching.
 *  - Every request in the resident set is advanced by one IMEX-RK3 step per server
 *    step, with its own time step and end time, exactly as in a context: its result
 *    does not depend on which other requests share the device with it.
 *  - Between steps, finished requests (t = t_end, or a failure) leave.  Their
 *    primitives are copied to the caller's buffer.  Waiting requests are admitted in
 *    arrival order while they fit the resident bounds (cells, faces and slots, from
 *    the memory budget).  The resident state is then repacked into one contiguous
 *    batch: gather kernels, no host round trip.
 *  - With opts.ct, 2D and 3D requests use constrained transport (Sec. 4) as in a
 *    context: the staggered face field is built from the request's cell-centred B
 *    at admission and moves with it in every repack.  The output holds the
 *    cell-centred primitives (B = the face means).
 *  - One host thread per server (the engine) does all device work, on its own
 *    streams, split into `opts.lanes` concurrent sub-batches.
 * Times are seconds of the host's steady clock since rrmhd_server_create. */
typedef struct rrmhd_server rrmhd_server;

typedef struct {
    int64_t mem_bytes;           /* device memory for resident state; 0: half the free memory */
    int64_t max_resident_cells;  /* admission bound on the cells stepped together (it bounds
                                    the step time); 0: what mem_bytes holds              */
    int     max_resident;        /* admission bound on resident requests (slots); 0: 4096 */
    rrmhd_tuning tuning;         /* launch shapes and lanes; all zero: the defaults       */
} rrmhd_server_config;

typedef struct {
    int64_t id;          /* as returned by rrmhd_server_submit                          */
    int32_t status;      /* RRMHD_OK, or the instance's failure (then the output is its
                            last good state)                                          */
    int32_t steps;       /* IMEX steps taken                                            */
    int64_t cells;       /* cells of the request's grid                                 */
    double  t;           /* time reached (= t_end when status is RRMHD_OK)              */
    double  submit_s;    /* arrival                                                     */
    double  admit_s;     /* entry into the resident set                                 */
    double  done_s;      /* output written; time to solution = done_s - submit_s        */
} rrmhd_result;

typedef struct {
    int64_t submitted, admitted, completed, failed;
    int64_t steps;                 /* server steps (one IMEX step of every resident request) */
    int64_t zone_updates;          /* cells x steps of the resident requests that advanced    */
    int64_t relayouts;             /* times the resident set changed                         */
    int64_t resident, resident_cells, peak_resident_cells, pending;
    int64_t cap_cells, cap_faces;  /* resident bounds derived from the configuration         */
    double  busy_s;                /* host wall time spent inside server steps               */
} rrmhd_server_stats;

/* Creates a server on the current device and starts its engine thread.
 * opts: host, shared by every request (gamma, precision, lanes, ...); cfg: host or
 * NULL for the defaults.  Device memory for the resident bounds is allocated here,
 * once: about 1.1 KB per resident cell (1.2 KB with opts.ct).  Returns EINVAL for
 * bad options, ENOMEM if the allocation fails. */
rrmhd_status rrmhd_server_create(const rrmhd_opts* opts, const rrmhd_server_config* cfg,
                                 rrmhd_server** out);

/* Queues one request.  grid: host; V: host double[12][ncells] primitives, kappa,
 * sigma: host double[ncells] (copied before the call returns); t_end: end time
 * (the request starts at t = 0).  V_out: host double[12][ncells] that receives the
 * final primitives.  It is owned by the caller and must stay valid until
 * rrmhd_server_poll has returned the request's result.  id: host, receives the
 * request's id.  Thread-safe.  Returns EINVAL for a bad grid or NULL buffers,
 * ECAPACITY for a grid larger than the resident bounds (it could never be
 * admitted), ECUDA once the engine has failed. */
rrmhd_status rrmhd_server_submit(rrmhd_server* srv, const rrmhd_grid* grid, const double* V,
                                 const double* kappa, const double* sigma, double t_end,
                                 double* V_out, int64_t* id);

/* Moves up to max results of completed requests into out (host), in completion
 * order; returns how many.  Thread-safe. */
int rrmhd_server_poll(rrmhd_server* srv, rrmhd_result* out, int max);

/* Blocks until no request is waiting or resident, or until timeout_s seconds have
 * passed (RRMHD_ETIMEOUT).  Returns ECUDA if the engine failed. */
rrmhd_status rrmhd_server_wait_idle(rrmhd_server* srv, double timeout_s);

/* Counters of the server so far (host). */
rrmhd_status rrmhd_server_get_stats(rrmhd_server* srv, rrmhd_server_stats* st);

/* The admission rule on its own (host only, no device work): given the cells and
 * faces of the waiting requests in arrival order (host arrays of n_waiting), the
 * free cells, faces and slots of the resident set, returns how many requests
 * from the head of the queue are admitted.  Arrival order is kept: a request that
 * does not fit blocks the ones behind it. */
int rrmhd_server_admission(const int64_t* cells, const int64_t* faces, int n_waiting,
                           int64_t free_cells, int64_t free_faces, int free_slots);

/* Text of the server's last error (static storage owned by srv). */
const char* rrmhd_server_last_error(rrmhd_server* srv);

/* Stops the engine thread (after its current step), drops waiting requests and
 * releases the device memory. */
void rrmhd_server_destroy(rrmhd_server* srv);

/* Text of the last error of this context (static storage owned by ctx). */
const char* rrmhd_last_error(const rrmhd_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
