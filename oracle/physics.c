/*
 * physics.c -- point functions of one state: equation of state, prim2con,
 * physical fluxes, the M1 closure, con2prim, signal speeds and the radiation
 * four-force.  TEST INFRASTRUCTURE ONLY (the oracle; see oracle.h).
 *
 * Paper: Lopez-Miralles, Marti & Perucho 2022 (arXiv:2212.00370), Sec. 2.
 * Units: c = 1; a factor 1/sqrt(4 pi) is absorbed in B (Sec. 2.1, footnote).
 */
#include <math.h>
#include "oracle.h"

void or_params_init(or_params* P)
{
    P->gfac = P->gamma / (P->gamma - 1.0);
    P->gm1g = (P->gamma - 1.0) / P->gamma;
}

/* Auxiliary quantities of a primitive state (Sec. 2.1, text after Eq. eqF):
 *   W   = 1/sqrt(1 - v^2)                     Lorentz factor
 *   b^0 = W (v.B),  b^i = B^i/W + v^i b^0      magnetic four-vector
 *   |b|^2 = b^mu b_mu = B^2/W^2 + (v.B)^2      (identity from the two lines above)
 *   rho h = rho (1 + eps) + p = rho + gamma/(gamma-1) p   (Eq. eos)
 *   h* = h + |b|^2/rho,  p* = p + |b|^2/2
 * The paper prints h* with "gamma/rho" where p/rho is meant (reading noted in
 * the design notes); rho h* = rho h + |b|^2 is used here. */
typedef struct {
    double v2, iW, W, vB, B2, b0, b[3], bsq, rhoh, ptot;
} aux_t;

static void aux_of(const or_params* P, const double* V, aux_t* a)
{
    double vx = V[1], vy = V[2], vz = V[3];
    double Bx = V[5], By = V[6], Bz = V[7];
    a->v2 = (vx * vx + vy * vy) + vz * vz;
    a->iW = sqrt(1.0 - a->v2);          /* 1/W */
    a->W = 1.0 / a->iW;
    a->vB = (vx * Bx + vy * By) + vz * Bz;
    a->B2 = (Bx * Bx + By * By) + Bz * Bz;
    a->b0 = a->W * a->vB;
    a->b[0] = Bx * a->iW + vx * a->b0;
    a->b[1] = By * a->iW + vy * a->b0;
    a->b[2] = Bz * a->iW + vz * a->b0;
    a->bsq = a->B2 * (a->iW * a->iW) + a->vB * a->vB;
    a->rhoh = V[0] + P->gfac * V[4];
    a->ptot = V[4] + 0.5 * a->bsq;
}

double or_prim_Z(const or_params* P, const double V[12])
{
    aux_t a;
    aux_of(P, V, &a);
    return a.rhoh * (a.W * a.W);
}

/* Eq. eqU.  D = rho W;  S^j = rho h* W^2 v^j - b^0 b^j;
 * tau_e = rho h* W^2 - p* - (b^0)^2 - rho W.
 * rho W^2 - rho W = D (W - 1) = D u^2/(W + 1) with u^2 = W^2 v^2 = W^2 - 1,
 * which keeps tau_e free of the cancellation of the printed form. */
void or_prim2con(const or_params* P, const double V[12], double U[12])
{
    aux_t a;
    aux_of(P, V, &a);
    double W2 = a.W * a.W;
    double D = V[0] * a.W;
    double rhohs_W2 = (a.rhoh + a.bsq) * W2;
    U[0] = D;
    U[1] = rhohs_W2 * V[1] - a.b0 * a.b[0];
    U[2] = rhohs_W2 * V[2] - a.b0 * a.b[1];
    U[3] = rhohs_W2 * V[3] - a.b0 * a.b[2];
    {
        double u2 = W2 * a.v2;
        double e1 = D * (u2 / (a.W + 1.0));
        double e2 = (P->gfac * V[4] + a.bsq) * W2;
        U[4] = (e1 + e2) - (a.ptot + a.b0 * a.b0);
    }
    for (int k = 5; k < 12; k++) U[k] = V[k];
}

/* M1 closure (Sec. 2.2): f = |F_r|/E_r, xi(f) = (3 + 4 f^2)/(5 + 2 sqrt(4 - 3 f^2)),
 * D^{ij} = (1 - xi)/2 delta^{ij} + (3 xi - 1)/2 n^i n^j,  P_r^{ij} = D^{ij} E_r.
 * f is clamped to [0,1]; with F_r = 0 the n n term is dropped (3 xi - 1 = 0 at f = 0). */
double or_eddington_factor(double f)
{
    double f2 = f * f;
    if (f2 > 1.0) f2 = 1.0;
    return (3.0 + 4.0 * f2) / (5.0 + 2.0 * sqrt(4.0 - 3.0 * f2));
}

void or_m1_pressure(double E, const double F[3], double Pr[3][3])
{
    double F2 = (F[0] * F[0] + F[1] * F[1]) + F[2] * F[2];
    double f2 = F2 / (E * E);
    if (f2 > 1.0) f2 = 1.0;
    double xi = (3.0 + 4.0 * f2) / (5.0 + 2.0 * sqrt(4.0 - 3.0 * f2));
    double a = (0.5 * (1.0 - xi)) * E;
    double c = 0.0;
    if (F2 > 0.0) c = ((0.5 * (3.0 * xi - 1.0)) * E) / F2;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double t = c * (F[i] * F[j]);
            Pr[i][j] = (i == j) ? t + a : t;
        }
}

/* Physical flux along direction d (Eq. eqF), written with the conserved
 * variables of the same state:
 *   rho h* W^2 v^d v^j + p* delta^{dj} - b^d b^j = S^j v^d - b^j B^d/W + p* delta^{dj}
 *   rho h* W^2 v^d - b^0 b^d - rho W v^d        = (tau_e + p*) v^d - b^0 B^d/W
 * (both follow from Eq. eqU and b^d = B^d/W + v^d b^0). */
void or_flux(const or_params* P, int d, const double V[12], const double U[12], double F[12])
{
    aux_t a;
    aux_of(P, V, &a);
    double vd = V[1 + d];
    double Bd = V[5 + d];
    double BdW = Bd * a.iW;
    F[0] = U[0] * vd;
    for (int j = 0; j < 3; j++) {
        double t = U[1 + j] * vd - a.b[j] * BdW;
        F[1 + j] = (j == d) ? t + a.ptot : t;
    }
    F[4] = (U[4] + a.ptot) * vd - a.b0 * BdW;
    for (int j = 0; j < 3; j++)
        F[5 + j] = (j == d) ? 0.0 : vd * V[5 + j] - Bd * V[1 + j];
    F[8] = V[9 + d];
    {
        double Fr[3] = {V[9], V[10], V[11]};
        double Pr[3][3];
        or_m1_pressure(V[8], Fr, Pr);
        F[9] = Pr[d][0];
        F[10] = Pr[d][1];
        F[11] = Pr[d][2];
    }
}

/* ------------------------------------------------------------------------
 * con2prim.  The paper defers the inversion to its companion code paper
 * (Sec. 3.2.2 step 2).  This is the published one-dimensional Newton-Raphson
 * scheme of Mignone & McKinney (2007, MNRAS 378, 1118) for the ideal-gas law,
 * iterating on W' = Z - D with Z = rho h W^2:
 *   v^2(Z) = (S^2 Z^2 + (S.B)^2 (2Z + B^2)) / (Z^2 (Z + B^2)^2)
 *   p(W')  = (gamma-1)/gamma [ W' (1 - v^2) - D v^2/(W + 1) ]
 *   f(W')  = W' - p + B^2 (1 + v^2)/2 - (S.B)^2/(2 Z^2) - tau_e = 0
 *   v^i    = (S^i + (S.B) B^i / Z) / (Z + B^2),   rho = D / W.
 * Stopping rule: the iteration stops at the Newton step with |dW'| <= 1e-10 W'
 * (the step is taken).  In Newton's quadratic regime the error left is of
 * order (1e-10 W')^2 / W', below rounding, so the nested flux differences of
 * the PVM flux, which differentiate con2prim at the 1e-8 level, see a
 * recovery exact to rounding.
 * A step that leaves the admissible region (W' <= 0 or v^2 >= 1) is halved.
 * ---------------------------------------------------------------------- */
typedef struct {
    double D, S[3], tau, B[3], S2, B2, SB, SB2, gm1g;
} c2p_in;

typedef struct {
    int ok;
    double x, Z, iZ, iZB, v2, W, p, f, df;
} c2p_pt;

static void c2p_eval(const c2p_in* c, double x, c2p_pt* e)
{
    e->x = x;
    e->ok = 0;
    if (!(x > 0.0)) return;
    double Z = x + c->D;
    double ZB = Z + c->B2;
    double iZ = 1.0 / Z;
    double iZB = 1.0 / ZB;
    double iZ2 = iZ * iZ;
    double v2 = (c->S2 + c->SB2 * ((2.0 * Z + c->B2) * iZ2)) * (iZB * iZB);
    if (!(v2 < 1.0)) return;
    double omv2 = 1.0 - v2;
    double W = 1.0 / sqrt(omv2);
    double p = c->gm1g * (x * omv2 - c->D * (v2 / (W + 1.0)));
    double f = ((x - p) + (0.5 * c->B2) * (1.0 + v2)) - ((0.5 * c->SB2) * iZ2 + c->tau);
    /* derivatives (Mignone & McKinney 2007, Sec. 3.2) */
    double dv2 = (-2.0 * (iZB * iZB * iZB)) *
                 (c->S2 + c->SB2 * (((3.0 * Z + 3.0 * c->B2) * Z + c->B2 * c->B2) * (iZ2 * iZ)));
    double dp = c->gm1g * (omv2 + dv2 * ((0.5 * c->D) * W - Z));
    double df = ((1.0 - dp) + (0.5 * c->B2) * dv2) + c->SB2 * (iZ2 * iZ);
    e->Z = Z;
    e->iZ = iZ;
    e->iZB = iZB;
    e->v2 = v2;
    e->W = W;
    e->p = p;
    e->f = f;
    e->df = df;
    e->ok = 1;
}

int or_con2prim(const or_params* P, const double U[12], double Zguess,
                double V[12], double* Zout, or_stats* st)
{
    c2p_in c;
    c.D = U[0];
    c.S[0] = U[1]; c.S[1] = U[2]; c.S[2] = U[3];
    c.tau = U[4];
    c.B[0] = U[5]; c.B[1] = U[6]; c.B[2] = U[7];
    c.S2 = (c.S[0] * c.S[0] + c.S[1] * c.S[1]) + c.S[2] * c.S[2];
    c.B2 = (c.B[0] * c.B[0] + c.B[1] * c.B[1]) + c.B[2] * c.B[2];
    c.SB = (c.S[0] * c.B[0] + c.S[1] * c.B[1]) + c.S[2] * c.B[2];
    c.SB2 = c.SB * c.SB;
    c.gm1g = P->gm1g;
    if (st) st->c2p_calls++;
    if (!(c.D > 0.0) || !(U[8] > 0.0)) {
        if (st) st->c2p_fail++;
        return OR_EUNPHYS;
    }

    /* admissible starting point: the guess, else tau_e (or D), doubled until v^2 < 1 */
    double x = Zguess - c.D;
    if (!(x > 0.0)) x = (c.tau > 0.0) ? c.tau : c.D;
    c2p_pt e;
    c2p_eval(&c, x, &e);
    for (int k = 0; k < 200 && !e.ok; k++) {
        x = 2.0 * x;
        c2p_eval(&c, x, &e);
    }
    if (!e.ok) {
        if (st) st->c2p_fail++;
        return OR_EC2P;
    }

    int conv = 0;
    for (int it = 1; it <= P->c2p_maxit; it++) {
        double dx = -e.f / e.df;
        c2p_pt en;
        c2p_eval(&c, x + dx, &en);
        for (int k = 0; k < 60 && !en.ok; k++) {
            dx = 0.5 * dx;
            c2p_eval(&c, x + dx, &en);
        }
        if (st) st->c2p_iters++;
        if (!en.ok) break;
        x = en.x;
        e = en;
        if (fabs(dx) <= 1e-10 * x) { conv = 1; break; }
    }
    if (!conv || !(e.p > 0.0)) {
        if (st) st->c2p_fail++;
        return OR_EC2P;
    }
    {
        double rho = c.D / e.W;
        double SBiZ = c.SB * e.iZ;
        V[0] = rho;
        V[1] = (c.S[0] + SBiZ * c.B[0]) * e.iZB;
        V[2] = (c.S[1] + SBiZ * c.B[1]) * e.iZB;
        V[3] = (c.S[2] + SBiZ * c.B[2]) * e.iZB;
        V[4] = e.p;
        for (int k = 5; k < 12; k++) V[k] = U[k];
    }
    if (Zout) *Zout = e.Z;
    return OR_OK;
}

/* Largest |signal speed| of a cell along direction d, capped at 1 (c = 1).
 * Magnetofluid: the fast-magnetosonic estimate of Del Zanna et al. (2007, ECHO),
 *   a^2 = c_s^2 + c_a^2 - c_s^2 c_a^2, c_s^2 = gamma p/(rho h), c_a^2 = |b|^2/(rho h + |b|^2),
 *   lambda = [v^d (1 - a^2) +- sqrt(a^2 (1 - v^2)(1 - v^2 a^2 - (v^d)^2 (1 - a^2)))]/(1 - v^2 a^2).
 * Radiation: lambda_r1, lambda_r3 of Eqs. lam1-lam3 with theta the angle between F_r
 * and the sweep direction. */
/* Signed fast-magnetosonic speed estimates lm <= lp of one state along d (the
 * Del Zanna et al. 2007 expressions above). */
void or_mhd_speeds(const or_params* P, int d, const double V[12], double* lm, double* lp)
{
    aux_t a;
    aux_of(P, V, &a);
    double cs2 = (P->gamma * V[4]) / a.rhoh;
    double ca2 = a.bsq / (a.rhoh + a.bsq);
    double a2 = (cs2 + ca2) - cs2 * ca2;
    double vd = V[1 + d];
    double den = 1.0 - a.v2 * a2;
    double disc = (a2 * (1.0 - a.v2)) * (den - (vd * vd) * (1.0 - a2));
    if (disc < 0.0) disc = 0.0;
    double sq = sqrt(disc);
    *lp = (vd * (1.0 - a2) + sq) / den;
    *lm = (vd * (1.0 - a2) - sq) / den;
}

/* Outer radiation eigenvalues lambda_r1 <= lambda_r3 of Eqs. lam1-lam3, theta the
 * angle between F_r and the direction d (cos theta = 0 when F_r = 0). */
void or_rad_speeds(int d, const double V[12], double* l1, double* l3)
{
    double E = V[8];
    double F2 = (V[9] * V[9] + V[10] * V[10]) + V[11] * V[11];
    double Fn = sqrt(F2);
    double f = Fn / E;
    if (f > 1.0) f = 1.0;
    double cth = (Fn > 0.0) ? V[9 + d] / Fn : 0.0;
    double f2 = f * f;
    double s = sqrt(4.0 - 3.0 * f2);
    double arg = (2.0 / 3.0) * ((4.0 - 3.0 * f2) - s) + (2.0 * (cth * cth)) * ((2.0 - f2) - s);
    if (arg < 0.0) arg = 0.0;
    double zeta = sqrt(arg);
    *l1 = (f * cth - zeta) / s;
    *l3 = (f * cth + zeta) / s;
}

double or_signal_speed(const or_params* P, int d, const double V[12])
{
    double lm, lp, l1, l3;
    or_mhd_speeds(P, d, V, &lm, &lp);
    double lf = fabs(lp) > fabs(lm) ? fabs(lp) : fabs(lm);
    or_rad_speeds(d, V, &l1, &l3);
    double lr = fabs(l1) > fabs(l3) ? fabs(l1) : fabs(l3);

    double lam = lf > lr ? lf : lr;
    if (lam > 1.0) lam = 1.0;
    return lam;
}

/* Radiation four-force in the laboratory frame, gray body (Eqs. g0, gi):
 *   G^0 = -rho kappa (4piB W - W E_r + u_i F^i)
 *         - rho sigma [W (W^2-1) E_r + W u_i u_j P^{ij} - (2W^2-1) u_i F^i]
 *   G^i = -4piB rho kappa u^i + rho (kappa+sigma)(W F^i - u_j P^{ij})
 *         - rho sigma u^i (W^2 E_r - 2 W u_j F^j + u_j u_k P^{jk})
 * with u^i = W v^i, W^2 - 1 = u^2, 2W^2 - 1 = 2u^2 + 1 and BP = 4 pi B = a_R T^4. */
void or_four_force(double kappa, double sigma, double rho, const double u[3], double W,
                   double BP, double E, const double F[3], const double Pr[3][3], double G[4])
{
    double u2 = (u[0] * u[0] + u[1] * u[1]) + u[2] * u[2];
    double uF = (u[0] * F[0] + u[1] * F[1]) + u[2] * F[2];
    double Pu[3];
    for (int i = 0; i < 3; i++) Pu[i] = (Pr[i][0] * u[0] + Pr[i][1] * u[1]) + Pr[i][2] * u[2];
    double uPu = (u[0] * Pu[0] + u[1] * Pu[1]) + u[2] * Pu[2];
    double rk = rho * kappa;
    double rs = rho * sigma;
    G[0] = -(rk * (W * (BP - E) + uF)) - rs * (((W * u2) * E + W * uPu) - (2.0 * u2 + 1.0) * uF);
    double q = ((W * W) * E - (2.0 * W) * uF) + uPu;
    for (int i = 0; i < 3; i++)
        G[1 + i] = ((-(BP * rk)) * u[i] + (rk + rs) * (W * F[i] - Pu[i])) - (rs * u[i]) * q;
}

/* ---------------- vectorised wrappers (SoA, stride n) ---------------- */
static void gather(const double* A, int64_t n, int64_t i, double* x)
{
    for (int k = 0; k < 12; k++) x[k] = A[k * n + i];
}
static void scatter(double* A, int64_t n, int64_t i, const double* x)
{
    for (int k = 0; k < 12; k++) A[k * n + i] = x[k];
}

void or_prim2con_n(const or_params* P, int64_t n, const double* V, double* U)
{
    for (int64_t i = 0; i < n; i++) {
        double v[12], u[12];
        gather(V, n, i, v);
        or_prim2con(P, v, u);
        scatter(U, n, i, u);
    }
}

void or_prim_Z_n(const or_params* P, int64_t n, const double* V, double* Z)
{
    for (int64_t i = 0; i < n; i++) {
        double v[12];
        gather(V, n, i, v);
        Z[i] = or_prim_Z(P, v);
    }
}

void or_con2prim_n(const or_params* P, int64_t n, const double* U, const double* Zg,
                   double* V, double* Z, int32_t* status, or_stats* st)
{
    for (int64_t i = 0; i < n; i++) {
        double u[12], v[12] = {0};
        double z = 0.0;
        gather(U, n, i, u);
        status[i] = or_con2prim(P, u, Zg ? Zg[i] : 0.0, v, &z, st);
        scatter(V, n, i, v);
        if (Z) Z[i] = z;
    }
}

void or_flux_n(const or_params* P, int dir, int64_t n, const double* V, const double* U, double* F)
{
    for (int64_t i = 0; i < n; i++) {
        double v[12], u[12], f[12];
        gather(V, n, i, v);
        gather(U, n, i, u);
        or_flux(P, dir, v, u, f);
        scatter(F, n, i, f);
    }
}

void or_signal_speed_n(const or_params* P, int dir, int64_t n, const double* V, double* lam)
{
    for (int64_t i = 0; i < n; i++) {
        double v[12];
        gather(V, n, i, v);
        lam[i] = or_signal_speed(P, dir, v);
    }
}
