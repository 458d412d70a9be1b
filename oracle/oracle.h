/*
 * oracle.h -- plain FP64 CPU oracle for the gray-M1 relativistic radiation MHD
 * finite-volume IMEX update with the PVM-int-8 Jacobian-free flux
 * (Lopez-Miralles, Marti & Perucho 2022, arXiv:2212.00370).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the reference that the CUDA path
 * is checked against.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load it; the product path never does.  It shares
 * no code with the CUDA path.
 *
 * Everything is IEEE double, evaluated in the order the source spells out
 * (build with -ffp-contract=off so that no multiply-add is fused).  Only
 * +, -, *, / and sqrt are used on the numerical path, so every value is
 * determined bit-for-bit by the expression order.
 *
 * Variable order (Sec. 2.1, Eq. eqU):
 *   U = (D, S^x, S^y, S^z, tau_e, B^x, B^y, B^z, E_r, F_r^x, F_r^y, F_r^z)
 *   V = (rho, v^x, v^y, v^z, p, B^x, B^y, B^z, E_r, F_r^x, F_r^y, F_r^z)
 * Grid fields are structure-of-arrays [12][nz][ny][nx], x fastest.
 */
#ifndef RRMHD_ORACLE_H
#define RRMHD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_NV 12

enum { OR_RECON_GODUNOV = 0, OR_RECON_MINMOD = 1, OR_RECON_MC = 2, OR_RECON_VANLEER = 3 };
enum { OR_BC_OUTFLOW = 0, OR_BC_PERIODIC = 1 };
enum { OR_IMP_NEWTON = 0, OR_IMP_PICARD = 1, OR_IMP_MATTER = 2 };
enum { OR_SOLVER_PVM = 0, OR_SOLVER_RADHLL = 1 };

/* status codes (per call) */
enum {
    OR_OK = 0,
    OR_EC2P = 1,       /* con2prim found no admissible root            */
    OR_EIMPLICIT = 2,  /* implicit radiation-matter solve failed       */
    OR_EUNPHYS = 3     /* input state not admissible (D<=0, E_r<=0 ...) */
};

typedef struct {
    double gamma;      /* ideal-gas adiabatic index (Eq. eos)                       */
    double a_rad;      /* radiation constant: 4 pi B = a_R T^4, T = p/rho (Sec. 2.1) */
    double cfl;        /* Courant number                                           */
    double pvm_eps;    /* epsilon of the nested flux differences (Sec. 3.2.2, 1e-8) */
    int    recon;      /* OR_RECON_*                                               */
    int    beta_mode;  /* 1: beta = min(1/tau_L, 1/tau_R, 1) (Eq. beta); 0: beta=1;
                          2: Eq. beta on the radiation components, 1 on the others   */
    int    imp_mode;   /* OR_IMP_NEWTON (default), OR_IMP_PICARD (paper's C matrix), or
                          OR_IMP_MATTER (the matter-primitive iteration alone) */
    int    pvm_k;      /* PVM-int-n with n = 2^k (Eq. iterat): 3 (PVM-int-8), 4 (-16) */
    int    solver;     /* OR_SOLVER_PVM (Sec. 3.2.2) or OR_SOLVER_RADHLL (Sec. 3.2.1)  */
    int    c2p_maxit;  /* Newton iterations allowed in con2prim                    */
    int    imp_maxit;  /* outer iterations allowed in the implicit solve           */
    double imp_tol;    /* implicit convergence: max|dX| <= imp_tol * E_r           */
    /* derived constants, filled by or_params_init */
    double gfac;       /* gamma/(gamma-1) */
    double gm1g;       /* (gamma-1)/gamma */
} or_params;

/* counters of the algorithm's work, summed over a call (may be NULL) */
typedef struct {
    int64_t c2p_calls, c2p_iters, c2p_fail;
    int64_t flux_evals, pvm_faces, pvm_fallback;
    int64_t imp_cells, imp_iters, imp_resid, imp_jac, imp_fail;
    int64_t imp_matter;        /* solves in the matter primitives */
    int64_t imp_resid_max;     /* most residual evaluations of one cell's solve */
    int64_t fallback_cells;    /* cell updates repeated by the admissibility fallback */
    int64_t fallback_flagged;  /* cells flagged by it after its first pass */
    int64_t imp_polish;        /* polishing corrections of converged implicit solves */
} or_stats;

void or_params_init(or_params* P);

/* ---- point functions (physics.c) ---- */
void   or_prim2con(const or_params* P, const double V[12], double U[12]);
double or_prim_Z(const or_params* P, const double V[12]);   /* rho h W^2 */
void   or_flux(const or_params* P, int dir, const double V[12], const double U[12], double F[12]);
void   or_m1_pressure(double E, const double F[3], double Pr[3][3]);
double or_eddington_factor(double f);
int    or_con2prim(const or_params* P, const double U[12], double Zguess,
                   double V[12], double* Zout, or_stats* st);
double or_signal_speed(const or_params* P, int dir, const double V[12]);
void   or_four_force(double kappa, double sigma, double rho, const double u[3], double W,
                     double BP, double E, const double F[3], const double Pr[3][3], double G[4]);

/* ---- scheme (scheme.c) ---- */
double or_limiter(int recon, double dL, double dR);
int    or_pvm_coefficients(int k, double alpha[9]);   /* Horner-order coefficients of p_k */
void   or_reconstruct(const or_params* P, const double Vm1[12], const double V0[12],
                      const double Vp1[12], double Vminus[12], double Vplus[12], int* fallback);
int    or_pvm_flux(const or_params* P, int dir, const double VL[12], const double VR[12],
                   double tauL, double tauR, double Fhat[12], double U4[12], or_stats* st);
void   or_llf_flux(const or_params* P, int dir, const double VL[12], const double VR[12],
                   double Fhat[12]);
void   or_radhll_flux(const or_params* P, int dir, const double VL[12], const double VR[12],
                      double tauL, double tauR, double Fhat[12]);
void   or_mhd_speeds(const or_params* P, int dir, const double V[12], double* lm, double* lp);
void   or_rad_speeds(int dir, const double V[12], double* l1, double* l3);

/* ---- implicit step (implicit.c) ---- */
int  or_implicit(const or_params* P, double kappa, double sigma, double hdt,
                 const double Ustar[12], double Zguess, double U[12], double V[12], or_stats* st);
int  or_implicit_c(const or_params* P, double kappa, double sigma, double hdt,
                   const double Ustar[12], double Zguess, double U[12], double V[12], double* jc,
                   or_stats* st);
void or_picard_matrix(double kappa, double sigma, double hdt, double rho, const double u[3],
                      double W, double BP, const double Dr[3][3],
                      const double Ustar_r[4], double C[4][4], double rhs[4]);
int  or_solve4(double A[4][4], double b[4], double x[4]);

/* ---- grids (grid.c) ---- */
typedef struct {
    int    ndim;
    int    n[3];
    double dx[3];
    int    bc[3];
} or_grid;

double or_grid_dt(const or_params* P, const or_grid* g, const double* V);
int    or_grid_face_flux(const or_params* P, const or_grid* g, int dir, const double* U,
                         const double* V, const double* kappa, const double* sigma,
                         double* Fhat, or_stats* st);
int    or_grid_stage(const or_params* P, const or_grid* g, int stage, double dt,
                     const double* U0, const double* Us, const double* Vs,
                     const double* kappa, const double* sigma,
                     double* Uout, double* Vout, int32_t* cell_status, or_stats* st);
int    or_grid_step(const or_params* P, const or_grid* g, double dt, double* U, double* V,
                    const double* kappa, const double* sigma, or_stats* st);
int    or_grid_stage_c(const or_params* P, const or_grid* g, int stage, double dt,
                       const double* U0, const double* Us, const double* Vs,
                       const double* kappa, const double* sigma,
                       double* Uout, double* Vout, int32_t* cell_status, double* jcache,
                       or_stats* st);
int    or_grid_step_c(const or_params* P, const or_grid* g, double dt, double* U, double* V,
                      const double* kappa, const double* sigma, double* jcache, or_stats* st);
int    or_grid_run(const or_params* P, const or_grid* g, double t0, double t_end, int max_steps,
                   double* U, double* V, const double* kappa, const double* sigma,
                   double* t_out, int* steps_out, or_stats* st);

/* ---- constrained transport (ct.c; grid.c *_ct, *_b variants) ---- */
int    or_grid_face_flux_b(const or_params* P, const or_grid* g, int dir, const double* U,
                           const double* V, const double* kappa, const double* sigma,
                           const double* bdir, double* Fhat, or_stats* st);
int    or_grid_stage_ct(const or_params* P, const or_grid* g, int stage, double dt,
                        const double* U0, const double* Us, const double* Vs,
                        const double* kappa, const double* sigma,
                        const double* b0, const double* bs, double* bout,
                        double* Uout, double* Vout, int32_t* cell_status, double* jcache,
                        or_stats* st);
int    or_grid_step_ct(const or_params* P, const or_grid* g, double dt, double* U, double* V,
                       double* bface, const double* kappa, const double* sigma, double* jcache,
                       or_stats* st);
int    or_grid_run_ct(const or_params* P, const or_grid* g, double t0, double t_end, int max_steps,
                      double* U, double* V, double* bface, const double* kappa, const double* sigma,
                      double* t_out, int* steps_out, or_stats* st);
int64_t or_ct_face_base(const or_grid* g, int d);
int64_t or_ct_nfaces(const or_grid* g);
void   or_ct_faces_from_cells(const or_grid* g, const double* V, double* bface);
void   or_ct_cells_from_faces(const or_grid* g, const double* bface, double* U, double* V);
void   or_ct_div(const or_grid* g, const double* bface, double* div);
void   or_ct_canonical(const or_grid* g, double* bface);
void   or_ct_stage(const or_grid* g, int stage, double dt, double* const Fh[3], const double* V,
                   const double* b0, const double* bs, double* bout);

/* ---- vectorised helpers for the Python wrapper (physics.c) ---- */
void or_prim2con_n(const or_params* P, int64_t n, const double* V, double* U);
void or_con2prim_n(const or_params* P, int64_t n, const double* U, const double* Zg,
                   double* V, double* Z, int32_t* status, or_stats* st);
void or_flux_n(const or_params* P, int dir, int64_t n, const double* V, const double* U, double* F);
void or_signal_speed_n(const or_params* P, int dir, int64_t n, const double* V, double* lam);
void or_prim_Z_n(const or_params* P, int64_t n, const double* V, double* Z);
void or_pvm_flux_n(const or_params* P, int dir, int64_t n, const double* VL, const double* VR,
                   const double* tauL, const double* tauR, double* Fhat, double* U4,
                   int32_t* status, or_stats* st);
void or_implicit_n(const or_params* P, int64_t n, const double* kappa, const double* sigma,
                   double hdt, const double* Ustar, const double* Zg, double* U, double* V,
                   int32_t* status, or_stats* st);
void or_implicit_cn(const or_params* P, int64_t n, const double* kappa, const double* sigma,
                    double hdt, const double* Ustar, const double* Zg, double* U, double* V,
                    double* jcache, int32_t* status, or_stats* st);

#ifdef __cplusplus
}
#endif
#endif
