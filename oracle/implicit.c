/*
 * implicit.c -- per-cell implicit radiation-matter step of the IMEX scheme
 * (Sec. 3.3, Eqs. timeadv, totale, totalm).  TEST INFRASTRUCTURE ONLY
 * (the oracle; see oracle.h).
 *
 * The cell solves, for X = (E_r, F_r^i),
 *     R(X) = X - X* + h G(X, V(X)) = 0,            h = (stage weight) dt,
 * since S_r = (-G^0, -G^i) (Eq. sourceterms).  The magnetofluid follows from
 * the conserved totals (Eqs. totale, totalm):
 *     tau_e = tau_{e,t} - E_r,  S = S_t - F_r,  D and B unchanged,
 * and V(X) is the con2prim of that state (Sec. 3.3 step 5).
 *
 * Default (OR_IMP_NEWTON): Newton's method on R with a forward-difference
 * Jacobian.  The paper's iteration (OR_IMP_PICARD) freezes the matter and the
 * Eddington tensor in the matrix C^(m) of Sec. 3.3 step 2; it is kept as an
 * option.  The Picard form diverges once the radiation heat capacity term
 * 4 a_R T^3 h kappa (gamma-1)/rho exceeds about one, which the stiff
 * workloads reach, hence Newton by default.
 *
 * Where the radiation carries nearly all the energy, the matter is a small
 * difference of X and the totals, and the iteration on X loses it.  The same
 * equations are then solved for the matter primitives Y = (p, u^i) instead,
 * with X(Y) the totals minus the matter (the MHD-field iteration of Melon
 * Fuksman & Mignone 2019, the paper's reference for the IMEX M1 scheme).
 */
#include <math.h>
#include "oracle.h"

#define IMP_LADDER 6   /* continuation fallback starts at h / 2^6 */

typedef struct {
    const or_params* P;
    double kappa, sigma, hdt;
    double D, St[3], taut, B[3];
    double Xs[4];
    or_stats* st;
} imp_ctx;

static void matter_state(const imp_ctx* c, const double X[4], double Um[12])
{
    Um[0] = c->D;
    Um[1] = c->St[0] - X[1];
    Um[2] = c->St[1] - X[2];
    Um[3] = c->St[2] - X[3];
    Um[4] = c->taut - X[0];
    Um[5] = c->B[0];
    Um[6] = c->B[1];
    Um[7] = c->B[2];
    Um[8] = X[0];
    Um[9] = X[1];
    Um[10] = X[2];
    Um[11] = X[3];
}

/* R(X); also returns the primitives of the matter state at X. */
static int imp_residual(imp_ctx* c, const double X[4], double Zg, double R[4],
                        double V[12], double* Z)
{
    double Um[12];
    if (c->st) c->st->imp_resid++;
    if (!(X[0] > 0.0)) return 1;
    matter_state(c, X, Um);
    if (or_con2prim(c->P, Um, Zg, V, Z, c->st) != OR_OK) return 1;
    double v2 = (V[1] * V[1] + V[2] * V[2]) + V[3] * V[3];
    double W = 1.0 / sqrt(1.0 - v2);
    double u[3] = {W * V[1], W * V[2], W * V[3]};
    double T = V[4] / V[0];                       /* T = p/rho in code units */
    double BP = c->P->a_rad * ((T * T) * (T * T)); /* 4 pi B = a_R T^4 */
    double Pr[3][3], G[4];
    or_m1_pressure(X[0], X + 1, Pr);
    or_four_force(c->kappa, c->sigma, V[0], u, W, BP, X[0], X + 1, Pr, G);
    for (int i = 0; i < 4; i++) R[i] = (X[i] - c->Xs[i]) + c->hdt * G[i];
    return 0;
}

/* The residual as a function of the matter primitives Y = (p, u^i): rho = D/W,
 * W = sqrt(1 + u.u), v = u/W, B fixed; X = (tau_t - tau_e(Y), S_t - S(Y)).
 * Returns X and the primitives (matter from Y, radiation X) as well. */
static int imp_residual_m(imp_ctx* c, const double Y[4], double R[4], double X[4], double V[12])
{
    if (c->st) c->st->imp_resid++;
    if (!(Y[0] > 0.0)) return 1;
    double W = sqrt(1.0 + ((Y[1] * Y[1] + Y[2] * Y[2]) + Y[3] * Y[3]));
    double Um[12];
    V[0] = c->D / W;
    for (int i = 0; i < 3; i++) {
        V[1 + i] = Y[1 + i] / W;
        V[5 + i] = c->B[i];
        V[9 + i] = 0.0;
    }
    V[4] = Y[0];
    V[8] = 0.0;
    or_prim2con(c->P, V, Um);
    X[0] = c->taut - Um[4];
    for (int i = 0; i < 3; i++) X[1 + i] = c->St[i] - Um[1 + i];
    if (!(X[0] > 0.0)) return 1;
    for (int i = 0; i < 4; i++) V[8 + i] = X[i];
    double T = Y[0] / V[0];
    double BP = c->P->a_rad * ((T * T) * (T * T));
    double Pr[3][3], G[4];
    or_m1_pressure(X[0], X + 1, Pr);
    or_four_force(c->kappa, c->sigma, V[0], Y + 1, W, BP, X[0], X + 1, Pr, G);
    for (int i = 0; i < 4; i++) R[i] = (X[i] - c->Xs[i]) + c->hdt * G[i];
    return 0;
}

/* Gaussian elimination with partial pivoting; A and b are overwritten. */
int or_solve4(double A[4][4], double b[4], double x[4])
{
    for (int col = 0; col < 4; col++) {
        int piv = col;
        for (int r = col + 1; r < 4; r++)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (A[piv][col] == 0.0) return 1;
        if (piv != col) {
            for (int k = 0; k < 4; k++) {
                double t = A[col][k];
                A[col][k] = A[piv][k];
                A[piv][k] = t;
            }
            double t = b[col];
            b[col] = b[piv];
            b[piv] = t;
        }
        for (int r = col + 1; r < 4; r++) {
            double f = A[r][col] / A[col][col];
            for (int k = col + 1; k < 4; k++) A[r][k] = A[r][k] - f * A[col][k];
            b[r] = b[r] - f * b[col];
        }
    }
    for (int r = 3; r >= 0; r--) {
        double s = b[r];
        for (int k = r + 1; k < 4; k++) s = s - A[r][k] * x[k];
        x[r] = s / A[r][r];
    }
    return 0;
}

/* Matrix C^(m) and right-hand side of Sec. 3.3 steps 2-3, i.e. the linear
 * system R(X) = C X - rhs = 0 obtained with the matter (rho, W, u, 4piB) and
 * the Eddington tensor D_r frozen.  The block C_{i+1,j+1} is derived from
 * Eqs. g0 and gi: delta_j^i + h rho W [(kappa+sigma) delta_j^i + 2 sigma u^i u_j]
 * (the printed minus sign in front of h would make absorption amplify F_r).
 * W^2 - 1 = u^2 and 2W^2 - 1 = 2u^2 + 1. */
void or_picard_matrix(double kappa, double sigma, double hdt, double rho, const double u[3],
                      double W, double BP, const double Dr[3][3],
                      const double Xs[4], double C[4][4], double rhs[4])
{
    double u2 = (u[0] * u[0] + u[1] * u[1]) + u[2] * u[2];
    double Du[3];
    for (int i = 0; i < 3; i++) Du[i] = (Dr[i][0] * u[0] + Dr[i][1] * u[1]) + Dr[i][2] * u[2];
    double uDu = (u[0] * Du[0] + u[1] * Du[1]) + u[2] * Du[2];
    double ks = kappa + sigma;
    C[0][0] = 1.0 - hdt * ((rho * W) * (-kappa + sigma * (u2 + uDu)));
    for (int j = 0; j < 3; j++)
        C[0][1 + j] = -hdt * ((rho * u[j]) * (kappa - sigma * (2.0 * u2 + 1.0)));
    for (int i = 0; i < 3; i++) {
        C[1 + i][0] = -hdt * (rho * (ks * Du[i] + (sigma * u[i]) * ((W * W) + uDu)));
        for (int j = 0; j < 3; j++) {
            double t = hdt * ((rho * W) * ((i == j ? ks : 0.0) + (2.0 * sigma) * (u[i] * u[j])));
            C[1 + i][1 + j] = (i == j ? 1.0 : 0.0) + t;
        }
    }
    rhs[0] = Xs[0] + hdt * (((rho * W) * kappa) * BP);
    for (int i = 0; i < 3; i++) rhs[1 + i] = Xs[1 + i] + hdt * (((rho * u[i]) * kappa) * BP);
}

static void eddington_tensor(double E, const double F[3], double Dr[3][3])
{
    double F2 = (F[0] * F[0] + F[1] * F[1]) + F[2] * F[2];
    double f2 = F2 / (E * E);
    if (f2 > 1.0) f2 = 1.0;
    double xi = (3.0 + 4.0 * f2) / (5.0 + 2.0 * sqrt(4.0 - 3.0 * f2));
    double a = 0.5 * (1.0 - xi);
    double c = (F2 > 0.0) ? (0.5 * (3.0 * xi - 1.0)) / F2 : 0.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) Dr[i][j] = c * (F[i] * F[j]) + (i == j ? a : 0.0);
}

static int picard(imp_ctx* c, double X[4], double V[12], double* Z)
{
    const or_params* P = c->P;
    for (int m = 1; m <= P->imp_maxit; m++) {
        double v2 = (V[1] * V[1] + V[2] * V[2]) + V[3] * V[3];
        double W = 1.0 / sqrt(1.0 - v2);
        double u[3] = {W * V[1], W * V[2], W * V[3]};
        double T = V[4] / V[0];
        double BP = P->a_rad * ((T * T) * (T * T));
        double Dr[3][3], C[4][4], rhs[4], Xn[4], Um[12];
        eddington_tensor(X[0], X + 1, Dr);
        or_picard_matrix(c->kappa, c->sigma, c->hdt, V[0], u, W, BP, Dr, c->Xs, C, rhs);
        if (or_solve4(C, rhs, Xn)) return 1;
        if (c->st) c->st->imp_iters++;
        double dmax = 0.0;
        for (int i = 0; i < 4; i++) {
            double d = fabs(Xn[i] - X[i]);
            if (d > dmax) dmax = d;
            X[i] = Xn[i];
        }
        if (!(X[0] > 0.0)) return 1;
        matter_state(c, X, Um);
        if (or_con2prim(P, Um, *Z, V, Z, c->st) != OR_OK) return 1;
        if (dmax <= P->imp_tol * X[0]) return 0;
    }
    return 1;
}

/* C^(m) at the current iterate, from its matter primitives V and Eddington tensor */
static void picard_jacobian(const imp_ctx* c, const double X[4], const double V[12], double J[4][4])
{
    double v2 = (V[1] * V[1] + V[2] * V[2]) + V[3] * V[3];
    double W = 1.0 / sqrt(1.0 - v2);
    double u[3] = {W * V[1], W * V[2], W * V[3]};
    double Dr[3][3], rhs[4];
    eddington_tensor(X[0], X + 1, Dr);
    or_picard_matrix(c->kappa, c->sigma, c->hdt, V[0], u, W, 0.0, Dr, c->Xs, J, rhs);
}

/* Forward-difference Jacobian of R at X (step 1e-7 E_r; a backward step where
 * the forward one leaves the admissible set).  Returns 1 if neither is admissible. */
static int fd_jacobian(imp_ctx* c, const double X[4], const double R[4], double Z, double J[4][4])
{
    double h = 1e-7 * X[0];
    for (int j = 0; j < 4; j++) {
        double Xp[4] = {X[0], X[1], X[2], X[3]};
        double Rp[4], Vp[12], Zp;
        Xp[j] = X[j] + h;
        if (imp_residual(c, Xp, Z, Rp, Vp, &Zp)) {
            Xp[j] = X[j] - h;
            if (imp_residual(c, Xp, Z, Rp, Vp, &Zp)) return 1;
        }
        double dXj = Xp[j] - X[j];
        for (int i = 0; i < 4; i++) J[i][j] = (Rp[i] - R[i]) / dXj;
    }
    return 0;
}

#define IMP_POLISH_TOL 1e-14  /* polished root: last correction <= 1e-14 E_r */
#define IMP_POLISH_MAX 6      /* at most six polishing corrections           */

/* Polish of a converged iterate.  Convergence at imp_tol leaves an error of about
 * the last step times the matrix's contraction, and that contraction depends on
 * how the iterate was reached (the first matrix, the Broyden history, the cell's
 * cache): left there, the result would be a function of the solver's path rather
 * than of the state.  It is refined here towards the root of R itself: corrections
 * dX = -J^-1 R(X), each accepted without line search, J updated by Broyden's
 * formula after each, until a correction is <= 1e-14 E_r.  A correction that does
 * not halve the previous one means the rounding floor of R is reached: the polish
 * stops there without taking it.  last is the size of the converged step.  X, R,
 * V and Z are updated in place and stay those of the last accepted iterate. */
static void polish(imp_ctx* c, double J[4][4], double X[4], double R[4], double V[12], double* Z,
                   double last)
{
    double prev = last;
    for (int p = 0; p < IMP_POLISH_MAX; p++) {
        double A[4][4], b[4], dX[4];
        for (int i = 0; i < 4; i++) {
            b[i] = -R[i];
            for (int j = 0; j < 4; j++) A[i][j] = J[i][j];
        }
        if (or_solve4(A, b, dX)) return;
        double d = 0.0;
        for (int i = 0; i < 4; i++) d = fabs(dX[i]) > d ? fabs(dX[i]) : d;
        if (d <= IMP_POLISH_TOL * X[0]) return;
        if (p > 0 && d > 0.5 * prev) return;
        double Xn[4], Rn[4], Vn[12], Zn = *Z;
        for (int i = 0; i < 4; i++) Xn[i] = X[i] + dX[i];
        if (imp_residual(c, Xn, *Z, Rn, Vn, &Zn)) return;
        if (c->st) c->st->imp_polish++;
        {
            double s2 = ((dX[0] * dX[0] + dX[1] * dX[1]) + dX[2] * dX[2]) + dX[3] * dX[3];
            for (int i = 0; i < 4; i++) {
                double Jd = ((J[i][0] * dX[0] + J[i][1] * dX[1]) + J[i][2] * dX[2]) + J[i][3] * dX[3];
                double q = ((Rn[i] - R[i]) - Jd) / s2;
                for (int j = 0; j < 4; j++) J[i][j] = J[i][j] + q * dX[j];
            }
        }
        for (int i = 0; i < 4; i++) {
            X[i] = Xn[i];
            R[i] = Rn[i];
        }
        for (int k = 0; k < 12; k++) V[k] = Vn[k];
        *Z = Zn;
        prev = d;
    }
}

/* Quasi-Newton iteration on R(X) = 0.
 * The first matrix is the paper's C^(m) (the Jacobian with matter and Eddington
 * tensor frozen), so the first iterate is the iteration of Sec. 3.3.  Each
 * accepted step then updates the matrix by Broyden's rank-one formula
 * J += (dR - J dX) dX^T / (dX.dX), which learns the matter coupling (T^4,
 * recoil) the frozen matrix leaves out.  When successive steps contract by less
 * than 2x, or a step gives no descent, the matrix is replaced by a
 * forward-difference Jacobian (step 1e-7 E_r).  Every step is damped by a
 * backtracking line search on |R|^2 (Armijo 1e-4); converged when the full step
 * is <= imp_tol * E_r. */
static int newton(imp_ctx* c, double X[4], double R[4], double V[12], double* Z,
                  const double* Min, double* Mout)
{
    const or_params* P = c->P;
    double J[4][4];
    int need_fd = 0;      /* replace J by a forward-difference Jacobian          */
    int fresh_fd = 0;     /* J is an FD Jacobian at the current X, not updated   */
    int first = 1;        /* J is the initial matrix (C^(m) or the cached one)   */
    double prev = -1.0;
    if (Min) {
        /* the cell's matrix from its previous solve: J = I + h M */
        for (int i = 0; i < 4; i++)
            for (int j = 0; j < 4; j++) J[i][j] = (i == j ? 1.0 : 0.0) + c->hdt * Min[4 * i + j];
    } else {
        picard_jacobian(c, X, V, J);
    }
    for (int m = 1; m <= P->imp_maxit; m++) {
        if (need_fd) {
            if (fd_jacobian(c, X, R, *Z, J)) return 1;
            need_fd = 0;
            fresh_fd = 1;
            first = 0;
            if (c->st) c->st->imp_jac++;
        }
        double A[4][4], b[4], dX[4];
        for (int i = 0; i < 4; i++) {
            b[i] = -R[i];
            for (int j = 0; j < 4; j++) A[i][j] = J[i][j];
        }
        if (or_solve4(A, b, dX)) {
            if (!fresh_fd) { need_fd = 1; continue; }
            return 1;
        }
        if (c->st) c->st->imp_iters++;

        /* converged when the full step is below tolerance: take it and stop */
        double dfull = 0.0;
        for (int i = 0; i < 4; i++) dfull = fabs(dX[i]) > dfull ? fabs(dX[i]) : dfull;
        double Xn[4], Rn[4], Vn[12], Zn = *Z;
        if (dfull <= P->imp_tol * X[0]) {
            for (int i = 0; i < 4; i++) Xn[i] = X[i] + dX[i];
            if (imp_residual(c, Xn, *Z, Rn, Vn, &Zn)) return 1;
            for (int i = 0; i < 4; i++) {
                X[i] = Xn[i];
                R[i] = Rn[i];
            }
            for (int k = 0; k < 12; k++) V[k] = Vn[k];
            *Z = Zn;
            if (Mout)
                for (int i = 0; i < 4; i++)
                    for (int j = 0; j < 4; j++)
                        Mout[4 * i + j] = (J[i][j] - (i == j ? 1.0 : 0.0)) / c->hdt;
            polish(c, J, X, R, V, Z, dfull);
            return 0;
        }
        /* backtracking line search: halve the step, at most ten times, until the
         * matter state is admissible and |R|^2 decreases (the initial frozen-matter
         * matrix gets four halvings before the full Jacobian replaces it).  A
         * direction that needs more is not worth following: the matrix is replaced,
         * or the continuation in h and the matter form take over. */
        double r0 = ((R[0] * R[0] + R[1] * R[1]) + R[2] * R[2]) + R[3] * R[3];
        double lam = 1.0;
        int ok = 0;
        for (int k = 0; k < 10; k++) {
            for (int i = 0; i < 4; i++) Xn[i] = X[i] + dX[i];
            if (!imp_residual(c, Xn, *Z, Rn, Vn, &Zn)) {
                double r1 = ((Rn[0] * Rn[0] + Rn[1] * Rn[1]) + Rn[2] * Rn[2]) + Rn[3] * Rn[3];
                if (r1 <= (1.0 - 1e-4 * lam) * r0) { ok = 1; break; }
            }
            for (int i = 0; i < 4; i++) dX[i] = 0.5 * dX[i];
            lam = 0.5 * lam;
            if (first && k == 3) break;
        }
        if (!ok) {
            if (!fresh_fd) { need_fd = 1; continue; }
            return 1;
        }
        double dmax = 0.0;
        for (int i = 0; i < 4; i++) {
            double d = fabs(dX[i]);
            if (d > dmax) dmax = d;
        }
        /* Broyden update with the accepted step dX and residual change */
        {
            double dR[4];
            for (int i = 0; i < 4; i++) dR[i] = Rn[i] - R[i];
            double s2 = ((dX[0] * dX[0] + dX[1] * dX[1]) + dX[2] * dX[2]) + dX[3] * dX[3];
            for (int i = 0; i < 4; i++) {
                double Jd = ((J[i][0] * dX[0] + J[i][1] * dX[1]) + J[i][2] * dX[2]) + J[i][3] * dX[3];
                double q = (dR[i] - Jd) / s2;
                for (int j = 0; j < 4; j++) J[i][j] = J[i][j] + q * dX[j];
            }
            fresh_fd = 0;
            first = 0;
        }
        for (int i = 0; i < 4; i++) {
            X[i] = Xn[i];
            R[i] = Rn[i];
        }
        for (int k = 0; k < 12; k++) V[k] = Vn[k];
        *Z = Zn;
        /* slow contraction: replace J by the full Jacobian at the new point */
        if (prev >= 0.0 && dmax > 0.5 * prev) need_fd = 1;
        prev = dmax;
    }
    return 1;
}

/* Newton's method on R(Y) = 0 in the matter primitives, from Y: a forward-difference
 * Jacobian at every iterate (steps 1e-7 of the scales p and 1 + |u|), backtracking on
 * |R|^2 as in the iteration on X; converged when every component of the full step is
 * <= 100 imp_tol times its scale.  (R keeps the rounding of the radiation-sized terms,
 * which the Jacobian, condition ~1e3 where this form is used, carries into Y; the
 * bound is still far below the matter accuracy of the iteration on X there.)  On
 * success Y, X and V hold the solution. */
static int newton_m(imp_ctx* c, double Y[4], double X[4], double V[12])
{
    const or_params* P = c->P;
    double R[4];
    if (imp_residual_m(c, Y, R, X, V)) return 1;
    for (int m = 1; m <= P->imp_maxit; m++) {
        double su = 1.0 + sqrt((Y[1] * Y[1] + Y[2] * Y[2]) + Y[3] * Y[3]);
        double sc[4] = {Y[0], su, su, su};
        double J[4][4];
        for (int j = 0; j < 4; j++) {
            double Yp[4] = {Y[0], Y[1], Y[2], Y[3]};
            double Rp[4], Xp[4], Vp[12];
            Yp[j] = Y[j] + 1e-7 * sc[j];
            if (imp_residual_m(c, Yp, Rp, Xp, Vp)) {
                Yp[j] = Y[j] - 1e-7 * sc[j];
                if (imp_residual_m(c, Yp, Rp, Xp, Vp)) return 1;
            }
            double dYj = Yp[j] - Y[j];
            for (int i = 0; i < 4; i++) J[i][j] = (Rp[i] - R[i]) / dYj;
        }
        if (c->st) c->st->imp_jac++;
        double b[4], dY[4];
        for (int i = 0; i < 4; i++) b[i] = -R[i];
        if (or_solve4(J, b, dY)) return 1;
        if (c->st) c->st->imp_iters++;
        int conv = 1;
        for (int i = 0; i < 4; i++)
            if (fabs(dY[i]) > (100.0 * P->imp_tol) * sc[i]) conv = 0;
        double Yn[4], Rn[4], Xn[4], Vn[12];
        if (conv) {
            for (int i = 0; i < 4; i++) Yn[i] = Y[i] + dY[i];
            if (imp_residual_m(c, Yn, Rn, Xn, Vn)) return 1;
            for (int i = 0; i < 4; i++) {
                Y[i] = Yn[i];
                X[i] = Xn[i];
            }
            for (int k = 0; k < 12; k++) V[k] = Vn[k];
            return 0;
        }
        double r0 = ((R[0] * R[0] + R[1] * R[1]) + R[2] * R[2]) + R[3] * R[3];
        double lam = 1.0;
        int ok = 0;
        for (int k = 0; k < 40; k++) {
            for (int i = 0; i < 4; i++) Yn[i] = Y[i] + dY[i];
            if (!imp_residual_m(c, Yn, Rn, Xn, Vn)) {
                double r1 = ((Rn[0] * Rn[0] + Rn[1] * Rn[1]) + Rn[2] * Rn[2]) + Rn[3] * Rn[3];
                if (r1 <= (1.0 - 1e-4 * lam) * r0) { ok = 1; break; }
            }
            for (int i = 0; i < 4; i++) dY[i] = 0.5 * dY[i];
            lam = 0.5 * lam;
        }
        if (!ok) return 1;
        for (int i = 0; i < 4; i++) {
            Y[i] = Yn[i];
            R[i] = Rn[i];
            X[i] = Xn[i];
        }
        for (int k = 0; k < 12; k++) V[k] = Vn[k];
    }
    return 1;
}

/* The matter-primitive solve from the matter state of U* (primitives Vs). */
static int solve_matter(imp_ctx* c, const double Vs[12], double X[4], double V[12])
{
    if (c->st) c->st->imp_matter++;
    double v2 = (Vs[1] * Vs[1] + Vs[2] * Vs[2]) + Vs[3] * Vs[3];
    double W = 1.0 / sqrt(1.0 - v2);
    double Y[4] = {Vs[4], W * Vs[1], W * Vs[2], W * Vs[3]};
    return newton_m(c, Y, X, V);
}

/* jc (may be NULL): the cell's Jacobian cache, 16 entries of M = (J - I)/h from its
 * last converged solve and a validity flag jc[16].  A valid entry is the first
 * matrix of the quasi-Newton iteration instead of C^(m); the converged matrix is
 * stored back (the flag is cleared when the solve fails).  M does not depend on h,
 * so it carries over between stages of different weight.  Flag 2 records that the
 * last solve needed the matter primitives; the next one starts there.
 * Order: [flag 2: matter solve]; iteration on X (cache or C^(m)); continuation in
 * h on X; matter solve (unless it was the first attempt). */
static int implicit_cell(const or_params* P, double kappa, double sigma, double hdt,
                         const double Ustar[12], double Zguess, double U[12], double V[12],
                         double* jc, or_stats* st)
{
    if (st) st->imp_cells++;
    if ((kappa == 0.0 && sigma == 0.0) || hdt == 0.0) {
        for (int k = 0; k < 12; k++) U[k] = Ustar[k];
        int rc = or_con2prim(P, Ustar, Zguess, V, 0, st);
        if (rc != OR_OK && st) st->imp_fail++;
        return rc;
    }
    imp_ctx c;
    c.P = P;
    c.kappa = kappa;
    c.sigma = sigma;
    c.hdt = hdt;
    c.st = st;
    c.D = Ustar[0];
    c.taut = Ustar[4] + Ustar[8];
    for (int j = 0; j < 3; j++) {
        c.St[j] = Ustar[1 + j] + Ustar[9 + j];
        c.B[j] = Ustar[5 + j];
    }
    for (int i = 0; i < 4; i++) c.Xs[i] = Ustar[8 + i];

    double X[4] = {c.Xs[0], c.Xs[1], c.Xs[2], c.Xs[3]};
    double R[4], Z = Zguess;
    int fail = imp_residual(&c, X, Zguess, R, V, &Z);
    if (fail) {
        /* the explicit state U* itself is inadmissible (no con2prim root or E_r <= 0) */
        if (st) st->imp_fail++;
        return OR_EC2P;
    }
    if (P->imp_mode == OR_IMP_PICARD) {
        fail = picard(&c, X, V, &Z);
    } else if (P->imp_mode == OR_IMP_MATTER) {
        double Vs[12];
        for (int k = 0; k < 12; k++) Vs[k] = V[k];
        fail = solve_matter(&c, Vs, X, V);
    } else {
        double Mnew[16], Vs[12];
        for (int k = 0; k < 12; k++) Vs[k] = V[k];
        if (jc && jc[16] == 2.0) {
            /* the cell's last solve needed the matter primitives: start there */
            if (!solve_matter(&c, Vs, X, V)) {
                matter_state(&c, X, U);
                return OR_OK;
            }
            for (int i = 0; i < 4; i++) X[i] = c.Xs[i];
            for (int k = 0; k < 12; k++) V[k] = Vs[k];
            Z = Zguess;
            imp_residual(&c, X, Z, R, V, &Z);
        }
        int tried_m = jc && jc[16] == 2.0;
        fail = newton(&c, X, R, V, &Z, (jc && jc[16] == 1.0) ? jc : 0, Mnew);
        if (fail) {
            /* continuation in the implicit weight: solve with h/64, h/32, ..., h,
             * each from the previous solution (the solution moves continuously
             * away from X* as h grows, and Newton stays in its basin) */
            for (int i = 0; i < 4; i++) X[i] = c.Xs[i];
            Z = Zguess;
            fail = 0;
            for (int j = IMP_LADDER; j >= 0 && !fail; j--) {
                c.hdt = hdt / (double)(1 << j);
                fail = imp_residual(&c, X, Z, R, V, &Z);
                if (!fail) fail = newton(&c, X, R, V, &Z, 0, Mnew);
            }
            c.hdt = hdt;
        }
        int matter = 0;
        if (fail && !tried_m) {
            fail = solve_matter(&c, Vs, X, V);
            matter = !fail;
        }
        if (jc) {
            for (int k = 0; k < 16; k++) jc[k] = (fail || matter) ? 0.0 : Mnew[k];
            jc[16] = fail ? 0.0 : (matter ? 2.0 : 1.0);
        }
    }
    if (fail) {
        if (st) st->imp_fail++;
        return OR_EIMPLICIT;
    }
    matter_state(&c, X, U);
    return OR_OK;
}

int or_implicit_c(const or_params* P, double kappa, double sigma, double hdt,
                  const double Ustar[12], double Zguess, double U[12], double V[12], double* jc,
                  or_stats* st)
{
    int64_t r0 = st ? st->imp_resid : 0;
    int rc = implicit_cell(P, kappa, sigma, hdt, Ustar, Zguess, U, V, jc, st);
    if (st && st->imp_resid - r0 > st->imp_resid_max) st->imp_resid_max = st->imp_resid - r0;
    return rc;
}

int or_implicit(const or_params* P, double kappa, double sigma, double hdt,
                const double Ustar[12], double Zguess, double U[12], double V[12], or_stats* st)
{
    return or_implicit_c(P, kappa, sigma, hdt, Ustar, Zguess, U, V, 0, st);
}

void or_implicit_n(const or_params* P, int64_t n, const double* kappa, const double* sigma,
                   double hdt, const double* Ustar, const double* Zg, double* U, double* V,
                   int32_t* status, or_stats* st)
{
    for (int64_t i = 0; i < n; i++) {
        double us[12], u[12] = {0}, v[12] = {0};
        for (int k = 0; k < 12; k++) us[k] = Ustar[k * n + i];
        status[i] = or_implicit(P, kappa[i], sigma[i], hdt, us, Zg ? Zg[i] : 0.0, u, v, st);
        for (int k = 0; k < 12; k++) {
            U[k * n + i] = u[k];
            V[k * n + i] = v[k];
        }
    }
}

/* or_implicit_n with a per-cell Jacobian cache jcache ([17][n] planes, zero =
 * empty), read and written back as or_implicit_c does for one cell. */
void or_implicit_cn(const or_params* P, int64_t n, const double* kappa, const double* sigma,
                    double hdt, const double* Ustar, const double* Zg, double* U, double* V,
                    double* jcache, int32_t* status, or_stats* st)
{
    for (int64_t i = 0; i < n; i++) {
        double us[12], u[12] = {0}, v[12] = {0}, jc[17];
        for (int k = 0; k < 12; k++) us[k] = Ustar[k * n + i];
        for (int k = 0; k < 17; k++) jc[k] = jcache[k * n + i];
        status[i] = or_implicit_c(P, kappa[i], sigma[i], hdt, us, Zg ? Zg[i] : 0.0, u, v, jc, st);
        for (int k = 0; k < 17; k++) jcache[k * n + i] = jc[k];
        for (int k = 0; k < 12; k++) {
            U[k * n + i] = u[k];
            V[k * n + i] = v[k];
        }
    }
}
