/*
 * grid.c -- finite-volume IMEX-RK3 update of one 1D/2D/3D Cartesian grid.
 * TEST INFRASTRUCTURE ONLY (the oracle; see oracle.h).
 *
 * Paper: Eq. full (conservative update), Eq. explicit (hyperbolic part,
 * read with its missing dt: U* = U - dt/dx (F_{i+1/2} - F_{i-1/2})), the RK3
 * IMEX stages of Sec. 3.1 with implicit weights 1, 1/4, 2/3, and
 * Sec. 3.3 for the implicit part.  Multi-dimensional grids sum the
 * directional flux differences in every stage (unsplit method of lines).
 * Boundaries: outflow (copy of the edge cell) or periodic, through index
 * mapping of the two ghost layers that PLM needs.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static int map_idx(int c, int n, int bc)
{
    if (bc == OR_BC_PERIODIC) {
        int m = c % n;
        return m < 0 ? m + n : m;
    }
    return c < 0 ? 0 : (c >= n ? n - 1 : c);
}

static int64_t ncells(const or_grid* g) { return (int64_t)g->n[0] * g->n[1] * g->n[2]; }

static int64_t lin(const or_grid* g, int i, int j, int k)
{
    return ((int64_t)k * g->n[1] + j) * g->n[0] + i;
}

static void load(const double* A, int64_t N, int64_t c, double* x)
{
    for (int q = 0; q < 12; q++) x[q] = A[q * N + c];
}

/* dt = CFL / max_cells sum_d lambda_d / dx_d (signal speeds of or_signal_speed) */
double or_grid_dt(const or_params* P, const or_grid* g, const double* V)
{
    int64_t N = ncells(g);
    double smax = 0.0;
    int bad = 0;
    for (int64_t c = 0; c < N; c++) {
        double v[12];
        load(V, N, c, v);
        double s = or_signal_speed(P, 0, v) / g->dx[0];
        for (int d = 1; d < g->ndim; d++) s = s + or_signal_speed(P, d, v) / g->dx[d];
        if (s != s) bad = 1;   /* NaN speed: inadmissible cell */
        if (s > smax) smax = s;
    }
    if (bad) return NAN;
    return P->cfl / smax;
}

static void face_dims(const or_grid* g, int dir, int m[3])
{
    m[0] = g->n[0];
    m[1] = g->n[1];
    m[2] = g->n[2];
    m[dir] += 1;
}

/* Numerical flux at every face normal to dir.  Face (i,j,k) of direction d
 * lies between cells with index i_d - 1 and i_d along d; faces are stored
 * [12][m2][m1][m0] with m = n + e_d. */
int or_grid_face_flux(const or_params* P, const or_grid* g, int dir, const double* U,
                      const double* V, const double* kappa, const double* sigma,
                      double* Fhat, or_stats* st)
{
    return or_grid_face_flux_b(P, g, dir, U, V, kappa, sigma, 0, Fhat, st);
}

/* Same, with the normal field component of both face states taken from the
 * staggered field bdir (the faces of direction dir; constrained transport) when
 * bdir is not NULL. */
int or_grid_face_flux_b(const or_params* P, const or_grid* g, int dir, const double* U,
                        const double* V, const double* kappa, const double* sigma,
                        const double* bdir, double* Fhat, or_stats* st)
{
    int64_t N = ncells(g);
    int m[3];
    face_dims(g, dir, m);
    int64_t NF = (int64_t)m[0] * m[1] * m[2];
    int nd = g->n[dir], bc = g->bc[dir];
    int nfb = 0;
    for (int k = 0; k < m[2]; k++)
        for (int j = 0; j < m[1]; j++)
            for (int i = 0; i < m[0]; i++) {
                int pos[3] = {i, j, k};
                int f = pos[dir];
                int64_t cidx[4];
                for (int s = 0; s < 4; s++) {
                    int q[3] = {i, j, k};
                    q[dir] = map_idx(f - 2 + s, nd, bc);
                    cidx[s] = lin(g, q[0], q[1], q[2]);
                }
                double w[4][12], Vm[12], Vp[12], VL[12], VR[12], F[12];
                for (int s = 0; s < 4; s++) load(V, N, cidx[s], w[s]);
                or_reconstruct(P, w[0], w[1], w[2], Vm, VL, 0); /* cell f-1: right face */
                or_reconstruct(P, w[1], w[2], w[3], VR, Vp, 0); /* cell f:   left face  */
                double tauL = (U[cidx[1]] * (kappa[cidx[1]] + sigma[cidx[1]])) * g->dx[dir];
                double tauR = (U[cidx[2]] * (kappa[cidx[2]] + sigma[cidx[2]])) * g->dx[dir];
                if (bdir) {
                    double bn = bdir[((int64_t)k * m[1] + j) * m[0] + i];
                    VL[5 + dir] = bn;
                    VR[5 + dir] = bn;
                }
                if (P->solver == OR_SOLVER_RADHLL)
                    or_radhll_flux(P, dir, VL, VR, tauL, tauR, F);
                else
                    nfb += or_pvm_flux(P, dir, VL, VR, tauL, tauR, F, 0, st);
                int64_t fi = ((int64_t)k * m[1] + j) * m[0] + i;
                for (int q = 0; q < 12; q++) Fhat[q * NF + fi] = F[q];
            }
    return nfb;
}

typedef struct {
    const or_params* P;
    const or_grid* g;
    int stage;
    double dt, a, b, hdt, dtdx[3];
    double* Fh[3];
    int m[3][3];
    const double *U0, *Us, *Vs, *kappa, *sigma;
    double* jc;   /* per-cell Jacobian cache, [17][N] planes, or NULL */
    const double* bface;   /* the stage's new staggered field (constrained transport), or NULL */
} stage_ctx;

/* U* of one cell from its face fluxes, then the implicit solve (Sec. 3.3). */
static int cell_update(const stage_ctx* s, int i, int j, int k, double Un[12], double Vn[12],
                       or_stats* st)
{
    const or_grid* g = s->g;
    int64_t N = ncells(g);
    int64_t c = lin(g, i, j, k);
    int64_t fl[3], fr[3], NF[3];
    for (int d = 0; d < g->ndim; d++) {
        int p[3] = {i, j, k};
        NF[d] = (int64_t)s->m[d][0] * s->m[d][1] * s->m[d][2];
        fl[d] = ((int64_t)p[2] * s->m[d][1] + p[1]) * s->m[d][0] + p[0];
        p[d] += 1;
        fr[d] = ((int64_t)p[2] * s->m[d][1] + p[1]) * s->m[d][0] + p[0];
    }
    double Ust[12], vs[12];
    for (int q = 0; q < 12; q++) {
        double acc = (s->Fh[0][q * NF[0] + fr[0]] - s->Fh[0][q * NF[0] + fl[0]]) * s->dtdx[0];
        for (int d = 1; d < g->ndim; d++)
            acc = acc + (s->Fh[d][q * NF[d] + fr[d]] - s->Fh[d][q * NF[d] + fl[d]]) * s->dtdx[d];
        if (s->stage == 1)
            Ust[q] = s->Us[q * N + c] - acc;
        else
            Ust[q] = s->a * s->U0[q * N + c] + s->b * (s->Us[q * N + c] - acc);
    }
    if (s->bface)   /* constrained transport: B_d is the mean of the two staggered faces */
        for (int d = 0; d < g->ndim; d++) {
            int64_t base = or_ct_face_base(g, d);
            Ust[5 + d] = 0.5 * (s->bface[base + fl[d]] + s->bface[base + fr[d]]);
        }
    load(s->Vs, N, c, vs);
    double Zg = or_prim_Z(s->P, vs);
    if (!s->jc) return or_implicit(s->P, s->kappa[c], s->sigma[c], s->hdt, Ust, Zg, Un, Vn, st);
    double jc[17];
    for (int q = 0; q < 17; q++) jc[q] = s->jc[q * N + c];
    int rc = or_implicit_c(s->P, s->kappa[c], s->sigma[c], s->hdt, Ust, Zg, Un, Vn, jc, st);
    for (int q = 0; q < 17; q++) s->jc[q * N + c] = jc[q];
    return rc;
}

/* A cell update the admissibility fallback retries with first-order faces: no
 * admissible explicit state, or no converged implicit solve from it. */
static int retry(int rc) { return rc == OR_EC2P || rc == OR_EUNPHYS || rc == OR_EIMPLICIT; }

/* Passes of the admissibility fallback. */
#define OR_FALLBACK_PASSES 3

/* One IMEX-RK3 stage (Sec. 3.1):
 *   stage 1: U* = U^(0) + dt L(U^(0)),                         U^(1) = U* + dt S
 *   stage 2: U* = 3/4 U^(0) + 1/4 (U^(1) + dt L(U^(1))),       U^(2) = U* + dt/4 S
 *   stage 3: U* = 1/3 U^(0) + 2/3 (U^(2) + dt L(U^(2))),       U^(3) = U* + 2dt/3 S
 * with dt L = -sum_d dt/dx_d (F_{+} - F_{-}) and the source solved implicitly
 * at the new stage state.
 * Admissibility fallback (a posteriori, conservative), in passes: cells whose U*
 * has no con2prim root, or whose implicit solve does not converge, are flagged;
 * in pass p every face adjacent to a cell flagged in pass p gets the first-order
 * lambda_max = 1 Rusanov flux of the cell-centre states (or_llf_flux), and every
 * cell touching such a face is updated again.  A re-updated cell that still fails
 * and was never flagged is flagged for pass p + 1; a failure in the last pass,
 * or of a cell already flagged, counts as failed.  Uout/Vout must not alias the
 * inputs. */
int or_grid_stage_c(const or_params* P, const or_grid* g, int stage, double dt,
                    const double* U0, const double* Us, const double* Vs,
                    const double* kappa, const double* sigma,
                    double* Uout, double* Vout, int32_t* cell_status, double* jcache, or_stats* st)
{
    return or_grid_stage_ct(P, g, stage, dt, U0, Us, Vs, kappa, sigma, 0, 0, 0, Uout, Vout,
                            cell_status, jcache, st);
}

/* One stage with constrained transport when b0 is not NULL (2D/3D): the face
 * fluxes take the normal field from bs, the staggered field advances to bout
 * (ct.c), and the cell-centred B of U* is the mean of bout's faces.  The
 * admissibility fallback's Rusanov fluxes enter the edge EMFs as well, and bout
 * is recomputed after each of its passes. */
int or_grid_stage_ct(const or_params* P, const or_grid* g, int stage, double dt,
                     const double* U0, const double* Us, const double* Vs,
                     const double* kappa, const double* sigma,
                     const double* b0, const double* bs, double* bout,
                     double* Uout, double* Vout, int32_t* cell_status, double* jcache, or_stats* st)
{
    int64_t N = ncells(g);
    const int ct = b0 && g->ndim >= 2;
    stage_ctx s;
    s.jc = jcache;
    s.bface = ct ? bout : 0;
    s.P = P;
    s.g = g;
    s.stage = stage;
    s.dt = dt;
    s.U0 = U0;
    s.Us = Us;
    s.Vs = Vs;
    s.kappa = kappa;
    s.sigma = sigma;
    s.Fh[0] = s.Fh[1] = s.Fh[2] = 0;
    for (int d = 0; d < g->ndim; d++) {
        face_dims(g, d, s.m[d]);
        s.Fh[d] = (double*)malloc(sizeof(double) * 12 * (size_t)s.m[d][0] * s.m[d][1] * s.m[d][2]);
        or_grid_face_flux_b(P, g, d, Us, Vs, kappa, sigma, ct ? bs + or_ct_face_base(g, d) : 0,
                            s.Fh[d], st);
    }
    if (ct) or_ct_stage(g, stage, dt, s.Fh, Vs, b0, bs, bout);
    s.a = 0.0;
    s.b = 1.0;
    double w = 1.0;
    if (stage == 2) { s.a = 0.75; s.b = 0.25; w = 0.25; }
    if (stage == 3) { s.a = 1.0 / 3.0; s.b = 2.0 / 3.0; w = 2.0 / 3.0; }
    s.hdt = w * dt;
    for (int d = 0; d < 3; d++) s.dtdx[d] = dt / g->dx[d];

    /* bad[c] = p: the cell was flagged in pass p of the fallback (0: not flagged) */
    unsigned char* bad = (unsigned char*)calloc((size_t)N, 1);
    int nfail = 0, nbad = 0;
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++) {
                int64_t c = lin(g, i, j, k);
                double Un[12], Vn[12];
                int rc = cell_update(&s, i, j, k, Un, Vn, st);
                if (cell_status) cell_status[c] = rc;
                if (retry(rc)) {
                    bad[c] = 1;
                    nbad++;
                } else if (rc != OR_OK) {
                    nfail++;
                }
                for (int q = 0; q < 12; q++) {
                    Uout[q * N + c] = Un[q];
                    Vout[q * N + c] = Vn[q];
                }
            }

    for (int pass = 1; nbad && pass <= OR_FALLBACK_PASSES; pass++) {
        nbad = 0;
        /* Rusanov fluxes at every face next to a cell flagged in this pass */
        for (int d = 0; d < g->ndim; d++) {
            int64_t NF = (int64_t)s.m[d][0] * s.m[d][1] * s.m[d][2];
            for (int k = 0; k < s.m[d][2]; k++)
                for (int j = 0; j < s.m[d][1]; j++)
                    for (int i = 0; i < s.m[d][0]; i++) {
                        int pos[3] = {i, j, k}, ql[3] = {i, j, k}, qr[3] = {i, j, k};
                        ql[d] = map_idx(pos[d] - 1, g->n[d], g->bc[d]);
                        qr[d] = map_idx(pos[d], g->n[d], g->bc[d]);
                        int64_t cl = lin(g, ql[0], ql[1], ql[2]), cr = lin(g, qr[0], qr[1], qr[2]);
                        if (bad[cl] != pass && bad[cr] != pass) continue;
                        double vl[12], vr[12], F[12];
                        load(Vs, N, cl, vl);
                        load(Vs, N, cr, vr);
                        or_llf_flux(P, d, vl, vr, F);
                        int64_t fi = ((int64_t)k * s.m[d][1] + j) * s.m[d][0] + i;
                        for (int q = 0; q < 12; q++) s.Fh[d][q * NF + fi] = F[q];
                    }
        }
        /* constrained transport: the edge EMFs of those faces go first-order too,
         * and the stage's face field is recomputed from the new fluxes */
        if (ct) or_ct_stage(g, stage, dt, s.Fh, Vs, b0, bs, bout);
        /* update again every cell with a changed face: flagged in this pass or
         * next to such a cell (with constrained transport, every cell of the
         * 3x3(x3) block around it: the face field changes on all faces that meet
         * the flagged cell's edges).  A cell that still fails, and was never
         * flagged, is flagged for the next pass; in the last pass it fails. */
        for (int k = 0; k < g->n[2]; k++)
            for (int j = 0; j < g->n[1]; j++)
                for (int i = 0; i < g->n[0]; i++) {
                    int64_t c = lin(g, i, j, k);
                    int hit = bad[c] == pass;
                    if (ct) {
                        int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
                        for (int d = 0; d < g->ndim; d++) { lo[d] = -1; hi[d] = 1; }
                        for (int dk = lo[2]; dk <= hi[2] && !hit; dk++)
                            for (int dj = lo[1]; dj <= hi[1] && !hit; dj++)
                                for (int di = lo[0]; di <= hi[0] && !hit; di++) {
                                    int p[3] = {i + di, j + dj, k + dk}, q[3], in = 1;
                                    for (int d = 0; d < 3; d++) {
                                        /* an outflow ghost cell is not a neighbour */
                                        if ((p[d] < 0 || p[d] >= g->n[d]) && g->bc[d] != OR_BC_PERIODIC) in = 0;
                                        q[d] = map_idx(p[d], g->n[d], g->bc[d]);
                                    }
                                    if (in && bad[lin(g, q[0], q[1], q[2])] == pass) hit = 1;
                                }
                    }
                    for (int d = 0; d < g->ndim && !hit; d++)
                        for (int e = -1; e <= 1; e += 2) {
                            int q[3] = {i, j, k};
                            int pd = q[d] + e;
                            q[d] = map_idx(pd, g->n[d], g->bc[d]);
                            /* an outflow ghost face is not shared with a neighbour */
                            if (pd < 0 || pd >= g->n[d]) {
                                if (g->bc[d] != OR_BC_PERIODIC) continue;
                            }
                            if (bad[lin(g, q[0], q[1], q[2])] == pass) hit = 1;
                        }
                    if (!hit) continue;
                    if (st) st->fallback_cells++;
                    double Un[12], Vn[12];
                    int rc = cell_update(&s, i, j, k, Un, Vn, st);
                    if (cell_status) cell_status[c] = rc;
                    if (retry(rc) && !bad[c] && pass < OR_FALLBACK_PASSES) {
                        bad[c] = (unsigned char)(pass + 1);
                        nbad++;
                        if (st) st->fallback_flagged++;
                    } else if (rc != OR_OK) {
                        nfail++;
                    }
                    for (int q = 0; q < 12; q++) {
                        Uout[q * N + c] = Un[q];
                        Vout[q * N + c] = Vn[q];
                    }
                }
    }
    free(bad);
    for (int d = 0; d < g->ndim; d++) free(s.Fh[d]);
    return nfail;
}

int or_grid_stage(const or_params* P, const or_grid* g, int stage, double dt,
                  const double* U0, const double* Us, const double* Vs,
                  const double* kappa, const double* sigma,
                  double* Uout, double* Vout, int32_t* cell_status, or_stats* st)
{
    return or_grid_stage_c(P, g, stage, dt, U0, Us, Vs, kappa, sigma, Uout, Vout, cell_status, 0, st);
}

/* One full IMEX-RK3 step of size dt; U and V are updated in place.  jcache: the
 * per-cell Jacobian cache carried from step to step ([17][N], zero = empty), or NULL. */
int or_grid_step_c(const or_params* P, const or_grid* g, double dt, double* U, double* V,
                   const double* kappa, const double* sigma, double* jcache, or_stats* st)
{
    return or_grid_step_ct(P, g, dt, U, V, 0, kappa, sigma, jcache, st);
}

/* One step; bface (constrained transport, 2D/3D, may be NULL) is advanced in
 * place with U and V. */
int or_grid_step_ct(const or_params* P, const or_grid* g, double dt, double* U, double* V,
                    double* bface, const double* kappa, const double* sigma, double* jcache,
                    or_stats* st)
{
    int64_t N = ncells(g);
    size_t bytes = sizeof(double) * 12 * (size_t)N;
    double* U1 = (double*)malloc(bytes);
    double* V1 = (double*)malloc(bytes);
    double* U2 = (double*)malloc(bytes);
    double* V2 = (double*)malloc(bytes);
    const int ct = bface && g->ndim >= 2;
    size_t fb = ct ? sizeof(double) * (size_t)or_ct_nfaces(g) : 0;
    double* b1 = ct ? (double*)malloc(fb) : 0;
    double* b2 = ct ? (double*)malloc(fb) : 0;
    const double* b0 = ct ? bface : 0;
    if (ct) or_ct_canonical(g, bface);
    int nfail = 0;
    nfail += or_grid_stage_ct(P, g, 1, dt, U, U, V, kappa, sigma, b0, b0, b1, U1, V1, 0, jcache, st);
    if (!nfail)
        nfail += or_grid_stage_ct(P, g, 2, dt, U, U1, V1, kappa, sigma, b0, b1, b2, U2, V2, 0, jcache, st);
    if (!nfail)
        nfail += or_grid_stage_ct(P, g, 3, dt, U, U2, V2, kappa, sigma, b0, b2, b1, U1, V1, 0, jcache, st);
    if (!nfail) {
        memcpy(U, U1, bytes);
        memcpy(V, V1, bytes);
        if (ct) memcpy(bface, b1, fb);
    }
    free(U1);
    free(V1);
    free(U2);
    free(V2);
    free(b1);
    free(b2);
    return nfail;
}

int or_grid_step(const or_params* P, const or_grid* g, double dt, double* U, double* V,
                 const double* kappa, const double* sigma, or_stats* st)
{
    return or_grid_step_c(P, g, dt, U, V, kappa, sigma, 0, st);
}

/* Advance from t0 to t_end (the last step is clipped to land on t_end), at
 * most max_steps steps, with a per-cell Jacobian cache that starts empty.
 * Returns the number of failed cells (0 on success). */
int or_grid_run(const or_params* P, const or_grid* g, double t0, double t_end, int max_steps,
                double* U, double* V, const double* kappa, const double* sigma,
                double* t_out, int* steps_out, or_stats* st)
{
    return or_grid_run_ct(P, g, t0, t_end, max_steps, U, V, 0, kappa, sigma, t_out, steps_out, st);
}

int or_grid_run_ct(const or_params* P, const or_grid* g, double t0, double t_end, int max_steps,
                   double* U, double* V, double* bface, const double* kappa, const double* sigma,
                   double* t_out, int* steps_out, or_stats* st)
{
    double t = t0;
    int s = 0, nfail = 0;
    double* jc = (double*)calloc((size_t)17 * ncells(g), sizeof(double));
    while (t < t_end && s < max_steps) {
        double dt = or_grid_dt(P, g, V);
        if (t + dt > t_end) dt = t_end - t;
        if (!(dt > 0.0)) {   /* NaN or non-positive: no admissible step */
            nfail = 1;
            break;
        }
        nfail = or_grid_step_ct(P, g, dt, U, V, bface, kappa, sigma, jc, st);
        if (nfail) break;
        t = t + dt;
        s++;
    }
    free(jc);
    if (t_out) *t_out = t;
    if (steps_out) *steps_out = s;
    return nfail;
}
