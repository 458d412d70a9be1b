/*
 * scheme.c -- explicit step of one interface: piecewise-linear reconstruction
 * of the primitives with the Godunov fallback, and the PVM-int-8 Jacobian-free
 * numerical flux.  TEST INFRASTRUCTURE ONLY (the oracle; see oracle.h).
 *
 * Paper: Sec. 3.2 (reconstruct-solve-update) and Sec. 3.2.2 (PVM solver,
 * Eqs. generalflux, iterat, utilde, beta).
 */
#include <math.h>
#include "oracle.h"

/* Slope limiters of the PLM reconstruction (Sec. 3.2): MinMod (Roe 1986),
 * MC (van Leer 1977) and VanLeer (van Leer 1974).  dL = V_i - V_{i-1},
 * dR = V_{i+1} - V_i; zero slope at extrema. */
double or_limiter(int recon, double dL, double dR)
{
    if (recon == OR_RECON_GODUNOV) return 0.0;
    if (!(dL * dR > 0.0)) return 0.0;
    if (recon == OR_RECON_MINMOD) return fabs(dL) < fabs(dR) ? dL : dR;
    if (recon == OR_RECON_MC) {
        double m = 2.0 * fabs(dL);
        double r = 2.0 * fabs(dR);
        double c = fabs(0.5 * (dL + dR));
        if (r < m) m = r;
        if (c < m) m = c;
        return dL > 0.0 ? m : -m;
    }
    /* VanLeer: harmonic mean 2 dL dR/(dL + dR) */
    return ((2.0 * dL) * dR) / (dL + dR);
}

/* Face values of cell i from its neighbours: Vminus at x_{i-1/2}, Vplus at
 * x_{i+1/2}.  If either face value is superluminal (|v|^2 >= 1) or violates
 * |F_r| <= E_r, the cell falls back to zeroth order (Sec. 3.2, Godunov
 * reconstruction for non-physical reconstructed states). */
void or_reconstruct(const or_params* P, const double Vm1[12], const double V0[12],
                    const double Vp1[12], double Vminus[12], double Vplus[12], int* fallback)
{
    for (int k = 0; k < 12; k++) {
        double s = or_limiter(P->recon, V0[k] - Vm1[k], Vp1[k] - V0[k]);
        Vplus[k] = V0[k] + 0.5 * s;
        Vminus[k] = V0[k] - 0.5 * s;
    }
    int bad = 0;
    const double* faces[2] = {Vminus, Vplus};
    for (int q = 0; q < 2; q++) {
        const double* w = faces[q];
        double v2 = (w[1] * w[1] + w[2] * w[2]) + w[3] * w[3];
        double F2 = (w[9] * w[9] + w[10] * w[10]) + w[11] * w[11];
        if (!(v2 < 1.0) || F2 > w[8] * w[8]) bad = 1;
    }
    if (bad)
        for (int k = 0; k < 12; k++) {
            Vplus[k] = V0[k];
            Vminus[k] = V0[k];
        }
    if (fallback) *fallback = bad;
}

/* Coefficients of the internal approximation p_k of |x| on [-1,1] built by
 * Eq. iterat: p_0 = 1, p_k = (2 p_{k-1} - p_{k-1}^2 + x^2)/2, a polynomial of
 * degree m = 2^(k-1) in y = x^2.  alpha[0..m] are its coefficients in Horner
 * order (highest degree first): p_k = (...(alpha_0 y + alpha_1) y + ...) y + alpha_m.
 * For k = 3 these are the printed -1/128, 3/32, -23/64, 31/32, 39/128.  All
 * coefficients are dyadic rationals, exact in double for k <= 4.  Returns m,
 * or 0 for k outside 1..4. */
int or_pvm_coefficients(int k, double alpha[9])
{
    if (k < 1 || k > 4) return 0;
    double c[17] = {1.0};   /* ascending powers of y; p_0 = 1 */
    int deg = 0;
    for (int j = 1; j <= k; j++) {
        double sq[17] = {0.0};
        for (int a = 0; a <= deg; a++)
            for (int b = 0; b <= deg; b++) sq[a + b] += c[a] * c[b];
        int nd = 2 * deg > 1 ? 2 * deg : 1;
        double nc[17] = {0.0};
        for (int a = 0; a <= nd; a++) {
            double v = -sq[a];
            if (a <= deg) v += 2.0 * c[a];
            if (a == 1) v += 1.0;
            nc[a] = 0.5 * v;
        }
        for (int a = 0; a <= nd; a++) c[a] = nc[a];
        deg = nd;
    }
    for (int a = 0; a <= deg; a++) alpha[a] = c[deg - a];
    return deg;
}

typedef struct {
    const or_params* P;
    int dir;
    double Um[12], Fm[12], Zm;
    or_stats* st;
} pvm_ctx;

/* Jacobian-free product A(U_m)^2 w (Sec. 3.2.2 steps 3-5, Eq. utilde):
 *   U_eps  = U_m + eps w                 -> V_eps = c2p(U_eps),  F(U_eps)
 *   U~_eps = U_m + F(U_eps) - F(U_m)     -> V~_eps = c2p(U~_eps), F(U~_eps)
 *   A^2 w  ~ (F(U~_eps) - F(U_m)) / eps                                      */
static int a2_product(pvm_ctx* c, const double w[12], double out[12])
{
    const or_params* P = c->P;
    double Ue[12], Ve[12], Fe[12], Ut[12], Vt[12], Ft[12];
    for (int k = 0; k < 12; k++) Ue[k] = c->Um[k] + P->pvm_eps * w[k];
    if (or_con2prim(P, Ue, c->Zm, Ve, 0, c->st) != OR_OK) return 1;
    or_flux(P, c->dir, Ve, Ue, Fe);
    for (int k = 0; k < 12; k++) Ut[k] = c->Um[k] + (Fe[k] - c->Fm[k]);
    if (or_con2prim(P, Ut, c->Zm, Vt, 0, c->st) != OR_OK) return 1;
    or_flux(P, c->dir, Vt, Ut, Ft);
    if (c->st) c->st->flux_evals += 2;
    for (int k = 0; k < 12; k++) out[k] = (Ft[k] - c->Fm[k]) / P->pvm_eps;
    return 0;
}

/* PVM-int-n numerical flux at one interface (Sec. 3.2.2, steps 1-7), n = 2^k:
 *   F^ = (F_L + F_R)/2 - beta U_{m}/2,  U_{m} ~ p_k(A(U_m)) (U_R - U_L),
 * with lambda_max = 1 and the Horner recursion in A^2 (m = 2^(k-1) products)
 *   U_1 = a0 A^2 U_0 + a1 U_0,  U_{l+1} = A^2 U_l + a_{l+1} U_0  (l = 1..m-1).
 * k = 3 (PVM-int-8) is the paper's solver: four products, U_4 = U_{k+1}.  k = 4
 * (PVM-int-16) is the variant the paper reports testing.
 * and beta = min{1/tau_L, 1/tau_R, 1} (Eq. beta), tau = rho W (kappa + sigma) dx
 * at the two cell centres adjacent to the face (beta_mode 1), applied to the radiation
 * components only (beta_mode 2, a variant: the paper leaves other choices of beta
 * open), or beta = 1 (beta_mode 0).
 * If a con2prim inside the viscosity term fails, the face uses Q = I
 * (U_{k+1} = U_0, the lambda_max = 1 Rusanov flux) and returns 1. */
int or_pvm_flux(const or_params* P, int dir, const double VL[12], const double VR[12],
                double tauL, double tauR, double Fhat[12], double U4out[12], or_stats* st)
{
    double UL[12], UR[12], FL[12], FR[12], U0[12], Vm[12];
    pvm_ctx c;
    c.P = P;
    c.dir = dir;
    c.st = st;
    or_prim2con(P, VL, UL);
    or_prim2con(P, VR, UR);
    or_flux(P, dir, VL, UL, FL);
    or_flux(P, dir, VR, UR, FR);
    if (st) { st->flux_evals += 2; st->pvm_faces++; }
    for (int k = 0; k < 12; k++) {
        U0[k] = UR[k] - UL[k];
        c.Um[k] = 0.5 * (UL[k] + UR[k]);
    }
    double Zg = 0.5 * (or_prim_Z(P, VL) + or_prim_Z(P, VR));

    double beta = 1.0;
    if (P->beta_mode) {
        double t = tauL > tauR ? tauL : tauR;
        if (t < 1.0) t = 1.0;
        beta = 1.0 / t;
    }

    double alpha[9];
    const int m = or_pvm_coefficients(P->pvm_k, alpha);   /* A^2 products needed */
    double Ul[12], Y[12];
    int fail = 0;
    if (m == 0 || or_con2prim(P, c.Um, Zg, Vm, &c.Zm, st) != OR_OK) {
        fail = 1;
    } else {
        or_flux(P, dir, Vm, c.Um, c.Fm);
        if (st) st->flux_evals++;
        for (int k = 0; k < 12; k++) Ul[k] = U0[k];
        for (int l = 0; l < m && !fail; l++) {
            if (a2_product(&c, Ul, Y)) { fail = 1; break; }
            if (l == 0)
                for (int k = 0; k < 12; k++) Ul[k] = alpha[0] * Y[k] + alpha[1] * U0[k];
            else
                for (int k = 0; k < 12; k++) Ul[k] = Y[k] + alpha[l + 1] * U0[k];
        }
    }
    if (fail) {
        for (int k = 0; k < 12; k++) Ul[k] = U0[k];
        if (st) st->pvm_fallback++;
    }
    /* beta_mode 2: beta damps the radiation block (E_r, F_r) only; the magnetofluid
     * block keeps beta = 1 */
    for (int k = 0; k < 12; k++) {
        double bk = (P->beta_mode == 2 && k < 8) ? 1.0 : beta;
        Fhat[k] = 0.5 * (FL[k] + FR[k]) - 0.5 * (bk * Ul[k]);
    }
    if (U4out)
        for (int k = 0; k < 12; k++) U4out[k] = Ul[k];
    return fail;
}

/* First-order local Lax-Friedrichs (Rusanov) flux with lambda_max = 1, i.e.
 * Q = I in Eq. generalflux, from the cell-centre states of the two cells
 * adjacent to the face.  Used only by the admissibility fallback. */
void or_llf_flux(const or_params* P, int dir, const double VL[12], const double VR[12],
                 double Fhat[12])
{
    double UL[12], UR[12], FL[12], FR[12];
    or_prim2con(P, VL, UL);
    or_prim2con(P, VR, UR);
    or_flux(P, dir, VL, UL, FL);
    or_flux(P, dir, VR, UR, FR);
    for (int k = 0; k < 12; k++) Fhat[k] = 0.5 * (FL[k] + FR[k]) - 0.5 * (UR[k] - UL[k]);
}

/* HLL flux (Sec. 3.2.1) of components [k0, k1) with wave speeds sL <= sR:
 *   F_L if sL > 0;  F_R if sR < 0;  else (sR F_L - sL F_R + sR sL (U_R - U_L))/(sR - sL).
 * A degenerate fan (sR == sL == 0) takes the central flux. */
static void hll_block(int k0, int k1, double sL, double sR, const double* UL, const double* UR,
                      const double* FL, const double* FR, double* F)
{
    for (int k = k0; k < k1; k++) {
        if (sL > 0.0)
            F[k] = FL[k];
        else if (sR < 0.0)
            F[k] = FR[k];
        else if (sR > sL)
            F[k] = ((sR * FL[k] - sL * FR[k]) + (sR * sL) * (UR[k] - UL[k])) / (sR - sL);
        else
            F[k] = 0.5 * (FL[k] + FR[k]);
    }
}

/* Radiative HLL flux (Sec. 3.2.1): the magnetofluid block (D, S, tau, B) with the
 * fast-magnetosonic speeds of the two reconstructed states, sL = min(lm_L, lm_R),
 * sR = max(lp_L, lp_R); the radiation block (E_r, F_r) with the outer radiation
 * eigenvalues rL = min(l1_L, l1_R), rR = max(l3_L, l3_R), limited in optically
 * thick cells by Eq. limits, rL >= -4/(3 tau), rR <= 4/(3 tau), with tau the
 * larger optical depth of the two cells next to the face (beta_mode = 1). */
void or_radhll_flux(const or_params* P, int dir, const double VL[12], const double VR[12],
                    double tauL, double tauR, double Fhat[12])
{
    double UL[12], UR[12], FL[12], FR[12];
    or_prim2con(P, VL, UL);
    or_prim2con(P, VR, UR);
    or_flux(P, dir, VL, UL, FL);
    or_flux(P, dir, VR, UR, FR);
    double lmL, lpL, lmR, lpR, r1L, r3L, r1R, r3R;
    or_mhd_speeds(P, dir, VL, &lmL, &lpL);
    or_mhd_speeds(P, dir, VR, &lmR, &lpR);
    or_rad_speeds(dir, VL, &r1L, &r3L);
    or_rad_speeds(dir, VR, &r1R, &r3R);
    double sL = lmL < lmR ? lmL : lmR;
    double sR = lpL > lpR ? lpL : lpR;
    double rL = r1L < r1R ? r1L : r1R;
    double rR = r3L > r3R ? r3L : r3R;
    double t = tauL > tauR ? tauL : tauR;
    if (P->beta_mode && t > 0.0) {
        double lim = 4.0 / (3.0 * t);
        if (rL < -lim) rL = -lim;
        if (rR > lim) rR = lim;
    }
    hll_block(0, 8, sL, sR, UL, UR, FL, FR, Fhat);
    hll_block(8, 12, rL, rR, UL, UR, FL, FR, Fhat);
}

void or_pvm_flux_n(const or_params* P, int dir, int64_t n, const double* VL, const double* VR,
                   const double* tauL, const double* tauR, double* Fhat, double* U4,
                   int32_t* status, or_stats* st)
{
    for (int64_t i = 0; i < n; i++) {
        double vl[12], vr[12], f[12], u4[12];
        for (int k = 0; k < 12; k++) {
            vl[k] = VL[k * n + i];
            vr[k] = VR[k * n + i];
        }
        status[i] = or_pvm_flux(P, dir, vl, vr, tauL[i], tauR[i], f, u4, st);
        for (int k = 0; k < 12; k++) {
            Fhat[k * n + i] = f[k];
            if (U4) U4[k * n + i] = u4[k];
        }
    }
}
