// physics_f64.cuh -- FP64 device functions of the gray-M1 relativistic radiation
// MHD update (Lopez-Miralles, Marti & Perucho 2022, arXiv:2212.00370).
//
// Arithmetic contract of the FP64 path: every value is produced by IEEE
// +, -, *, /, sqrt in the association order written here, and the translation
// unit is compiled with --fmad=false, so the results are a pure function of the
// inputs.  The nested flux differences of the PVM viscosity divide rounding
// noise by eps = 1e-8, so a one-ulp change anywhere upstream shows up at the
// 1e-8 level; this order is therefore part of the specification of the path.
//
// Variable order (Sec. 2.1, Eq. eqU):
//   U = (D, S^x, S^y, S^z, tau_e, B^x, B^y, B^z, E_r, F^x, F^y, F^z)
//   V = (rho, v^x, v^y, v^z, p,   B^x, B^y, B^z, E_r, F^x, F^y, F^z)
#pragma once
#include <cstdint>

namespace rr {

constexpr int NV = 12;

enum Status : int {
  ST_OK = 0,
  ST_C2P = 1,       // con2prim found no admissible root
  ST_IMPLICIT = 2,  // implicit radiation-matter solve failed
  ST_UNPHYS = 3,    // inadmissible conserved state (D <= 0 or E_r <= 0)
};

// A cell update the admissibility fallback retries with first-order faces: no
// admissible explicit state, or no converged implicit solve from it.
__host__ __device__ inline bool fallback_retry(int rc) {
  return rc == ST_C2P || rc == ST_IMPLICIT || rc == ST_UNPHYS;
}

enum Recon : int { RECON_GODUNOV = 0, RECON_MINMOD = 1, RECON_MC = 2, RECON_VANLEER = 3 };

// Scheme constants shared by every kernel of a context (passed by value).
struct Params {
  double gamma, a_rad, cfl, pvm_eps;
  int recon, beta_mode, c2p_maxit, imp_maxit;
  int pvm_k;  // PVM-int-2^k: 3 (PVM-int-8) or 4 (PVM-int-16)
  int pvm_products;  // FP64 A w products: 0 nested flux differences (Eq. utilde), 1 tangent
  int solver;        // 0 PVM-int (Sec. 3.2.2), 1 radiative HLL (Sec. 3.2.1)
  double imp_tol;
  double gfac;  // gamma/(gamma-1)
  double gm1g;  // (gamma-1)/gamma
};

// ---------------------------------------------------------------- aux state
// W = 1/sqrt(1-v^2), b^0 = W v.B, b^i = B^i/W + v^i b^0, |b|^2 = B^2/W^2 + (v.B)^2,
// rho h = rho + gamma/(gamma-1) p, p* = p + |b|^2/2   (Sec. 2.1).
struct Aux {
  double v2, iW, W, vB, B2, b0, b[3], bsq, rhoh, ptot;
};

__device__ __forceinline__ void aux_of(const Params& P, const double* V, Aux& a) {
  const double vx = V[1], vy = V[2], vz = V[3];
  const double Bx = V[5], By = V[6], Bz = V[7];
  a.v2 = (vx * vx + vy * vy) + vz * vz;
  a.iW = sqrt(1.0 - a.v2);
  a.W = 1.0 / a.iW;
  a.vB = (vx * Bx + vy * By) + vz * Bz;
  a.B2 = (Bx * Bx + By * By) + Bz * Bz;
  a.b0 = a.W * a.vB;
  a.b[0] = Bx * a.iW + vx * a.b0;
  a.b[1] = By * a.iW + vy * a.b0;
  a.b[2] = Bz * a.iW + vz * a.b0;
  a.bsq = a.B2 * (a.iW * a.iW) + a.vB * a.vB;
  a.rhoh = V[0] + P.gfac * V[4];
  a.ptot = V[4] + 0.5 * a.bsq;
}

// rho h W^2: the con2prim unknown Z of a primitive state (warm starts).
__device__ __forceinline__ double prim_Z(const Params& P, const double* V) {
  Aux a;
  aux_of(P, V, a);
  return a.rhoh * (a.W * a.W);
}

// Eq. eqU, with rho W^2 - rho W = D u^2/(W+1) (u^2 = W^2 v^2).
__device__ __forceinline__ void prim2con(const Params& P, const double* V, double* U) {
  Aux a;
  aux_of(P, V, a);
  const double W2 = a.W * a.W;
  const double D = V[0] * a.W;
  const double hw = (a.rhoh + a.bsq) * W2;
  U[0] = D;
  U[1] = hw * V[1] - a.b0 * a.b[0];
  U[2] = hw * V[2] - a.b0 * a.b[1];
  U[3] = hw * V[3] - a.b0 * a.b[2];
  const double u2 = W2 * a.v2;
  const double e1 = D * (u2 / (a.W + 1.0));
  const double e2 = (P.gfac * V[4] + a.bsq) * W2;
  U[4] = (e1 + e2) - (a.ptot + a.b0 * a.b0);
#pragma unroll
  for (int k = 5; k < NV; ++k) U[k] = V[k];
}

// ------------------------------------------------------------- M1 closure
// xi(f) = (3 + 4f^2)/(5 + 2 sqrt(4 - 3f^2)), P = [(1-xi)/2 delta + (3xi-1)/2 n n] E
// (Sec. 2.2, Eq. xi); f clamped to 1; no n n term when F_r = 0.
struct M1 {
  double a, c;  // P_ij = c F_i F_j (+ a on the diagonal)
};

__device__ __forceinline__ M1 m1_coef(double E, double Fx, double Fy, double Fz) {
  const double F2 = (Fx * Fx + Fy * Fy) + Fz * Fz;
  double f2 = F2 / (E * E);
  if (f2 > 1.0) f2 = 1.0;
  const double xi = (3.0 + 4.0 * f2) / (5.0 + 2.0 * sqrt(4.0 - 3.0 * f2));
  M1 m;
  m.a = (0.5 * (1.0 - xi)) * E;
  m.c = 0.0;
  if (F2 > 0.0) m.c = ((0.5 * (3.0 * xi - 1.0)) * E) / F2;
  return m;
}

__device__ __forceinline__ double m1_P(const M1& m, const double* F, int i, int j) {
  const double t = m.c * (F[i] * F[j]);
  return (i == j) ? t + m.a : t;
}

// Eddington tensor D_r = P_r/E_r (coefficients without the E_r factor).
__device__ __forceinline__ void eddington(double E, const double* F, double Dr[3][3]) {
  const double F2 = (F[0] * F[0] + F[1] * F[1]) + F[2] * F[2];
  double f2 = F2 / (E * E);
  if (f2 > 1.0) f2 = 1.0;
  const double xi = (3.0 + 4.0 * f2) / (5.0 + 2.0 * sqrt(4.0 - 3.0 * f2));
  const double a = 0.5 * (1.0 - xi);
  const double c = (F2 > 0.0) ? (0.5 * (3.0 * xi - 1.0)) / F2 : 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Dr[i][j] = c * (F[i] * F[j]) + (i == j ? a : 0.0);
}

// ------------------------------------------------------------- fluxes
// Eq. eqF along direction d, using the conserved variables of the same state:
//   momentum  S^j v^d - b^j B^d/W + p* delta^{dj}
//   energy    (tau_e + p*) v^d - b^0 B^d/W
//   induction v^d B^j - B^d v^j;  radiation F^d, P^{dj}.
__device__ __forceinline__ void flux(const Params& P, int d, const double* V, const double* U,
                                     double* F) {
  Aux a;
  aux_of(P, V, a);
  const double vd = V[1 + d];
  const double Bd = V[5 + d];
  const double BdW = Bd * a.iW;
  F[0] = U[0] * vd;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const double t = U[1 + j] * vd - a.b[j] * BdW;
    F[1 + j] = (j == d) ? t + a.ptot : t;
  }
  F[4] = (U[4] + a.ptot) * vd - a.b0 * BdW;
#pragma unroll
  for (int j = 0; j < 3; ++j) F[5 + j] = (j == d) ? 0.0 : vd * V[5 + j] - Bd * V[1 + j];
  F[8] = V[9 + d];
  const M1 m = m1_coef(V[8], V[9], V[10], V[11]);
  const double* Fr = V + 9;
#pragma unroll
  for (int j = 0; j < 3; ++j) F[9 + j] = m1_P(m, Fr, d, j);
}

// ------------------------------------------------------------- con2prim
// One-dimensional Newton-Raphson in W' = Z - D, Z = rho h W^2, for the
// ideal-gas law (Mignone & McKinney 2007); after |dW'| <= 1e-10 W' exactly one
// more step is taken; steps leaving W' > 0, v^2 < 1 are halved.
struct C2PIn {
  double D, S[3], tau, B[3], S2, B2, SB, SB2, gm1g;
};
struct C2PPt {
  int ok;
  double x, Z, iZ, iZB, v2, W, p, f, df;
};

// FAST (the FP32-bulk form's cells): 1/Z and 1/(Z+B^2) from one division, W from
// rsqrt; the same values to a few ulps.  Otherwise the operation order above.
template <bool FAST = false>
__device__ __forceinline__ void c2p_eval(const C2PIn& c, double x, C2PPt& e) {
  e.x = x;
  e.ok = 0;
  if (!(x > 0.0)) return;
  const double Z = x + c.D;
  const double ZB = Z + c.B2;
  double iZ, iZB;
  if constexpr (FAST) {
    const double q = 1.0 / (Z * ZB);
    iZ = ZB * q;
    iZB = Z * q;
  } else {
    iZ = 1.0 / Z;
    iZB = 1.0 / ZB;
  }
  const double iZ2 = iZ * iZ;
  const double v2 = (c.S2 + c.SB2 * ((2.0 * Z + c.B2) * iZ2)) * (iZB * iZB);
  if (!(v2 < 1.0)) return;
  const double omv2 = 1.0 - v2;
  double W;
  if constexpr (FAST)
    W = rsqrt(omv2);
  else
    W = 1.0 / sqrt(omv2);
  const double p = c.gm1g * (x * omv2 - c.D * (v2 / (W + 1.0)));
  const double f = ((x - p) + (0.5 * c.B2) * (1.0 + v2)) - ((0.5 * c.SB2) * iZ2 + c.tau);
  const double dv2 = (-2.0 * ((iZB * iZB) * iZB)) *
                     (c.S2 + c.SB2 * (((3.0 * Z + 3.0 * c.B2) * Z + c.B2 * c.B2) * (iZ2 * iZ)));
  const double dp = c.gm1g * (omv2 + dv2 * ((0.5 * c.D) * W - Z));
  const double df = ((1.0 - dp) + (0.5 * c.B2) * dv2) + c.SB2 * (iZ2 * iZ);
  e.Z = Z;
  e.iZ = iZ;
  e.iZB = iZB;
  e.v2 = v2;
  e.W = W;
  e.p = p;
  e.f = f;
  e.df = df;
  e.ok = 1;
}

// Returns a Status; V, *Zout and *Wout (the Lorentz factor; may be null) are written
// only on success.
// Stopping rule: the iteration stops at the Newton step with |dx| <= 1e-10 x (the
// step is taken).  In Newton's quadratic regime the error left is of order
// (1e-10 x)^2 / x, below rounding, so the PVM's finite-difference products, which
// differentiate con2prim at the 1e-8 level, see a recovery exact to rounding.
template <bool FAST = false>
static __device__ __noinline__ int con2prim(const Params& P, const double* U, double Zguess,
                                            double* V, double* Zout, double* Wout = nullptr) {
  C2PIn c;
  c.D = U[0];
  c.S[0] = U[1];
  c.S[1] = U[2];
  c.S[2] = U[3];
  c.tau = U[4];
  c.B[0] = U[5];
  c.B[1] = U[6];
  c.B[2] = U[7];
  c.S2 = (c.S[0] * c.S[0] + c.S[1] * c.S[1]) + c.S[2] * c.S[2];
  c.B2 = (c.B[0] * c.B[0] + c.B[1] * c.B[1]) + c.B[2] * c.B[2];
  c.SB = (c.S[0] * c.B[0] + c.S[1] * c.B[1]) + c.S[2] * c.B[2];
  c.SB2 = c.SB * c.SB;
  c.gm1g = P.gm1g;
  if (!(c.D > 0.0) || !(U[8] > 0.0)) return ST_UNPHYS;

  double x = Zguess - c.D;
  if (!(x > 0.0)) x = (c.tau > 0.0) ? c.tau : c.D;
  C2PPt e;
  c2p_eval<FAST>(c, x, e);
  for (int k = 0; k < 200 && !e.ok; ++k) {
    x = 2.0 * x;
    c2p_eval<FAST>(c, x, e);
  }
  if (!e.ok) return ST_C2P;

  int conv = 0;
  for (int it = 1; it <= P.c2p_maxit; ++it) {
    double dx;
    if constexpr (FAST) {  // inexact Newton: an FP32 reciprocal of df (~6e-8 relative)
      const float d32 = (float)e.df;
      dx = (fabsf(d32) > 1e-30f && fabsf(d32) < 1e30f) ? -e.f * (double)__frcp_rn(d32)
                                                        : -e.f / e.df;
    } else {
      dx = -e.f / e.df;
    }
    C2PPt en;
    c2p_eval<FAST>(c, x + dx, en);
    for (int k = 0; k < 60 && !en.ok; ++k) {
      dx = 0.5 * dx;
      c2p_eval<FAST>(c, x + dx, en);
    }
    if (!en.ok) break;
    x = en.x;
    e = en;
    if (fabs(dx) <= 1e-10 * x) {
      conv = 1;
      break;
    }
  }
  if (!conv || !(e.p > 0.0)) return ST_C2P;
  const double rho = FAST ? c.D * ((1.0 - e.v2) * e.W) : c.D / e.W;  // D/W = D (1 - v^2) W
  const double SBiZ = c.SB * e.iZ;
  V[0] = rho;
  V[1] = (c.S[0] + SBiZ * c.B[0]) * e.iZB;
  V[2] = (c.S[1] + SBiZ * c.B[1]) * e.iZB;
  V[3] = (c.S[2] + SBiZ * c.B[2]) * e.iZB;
  V[4] = e.p;
#pragma unroll
  for (int k = 5; k < NV; ++k) V[k] = U[k];
  if (Zout) *Zout = e.Z;
  if (Wout) *Wout = e.W;
  return ST_OK;
}

// ------------------------------------------------------------- signal speed
// max |lambda| along d, capped at 1: fast-magnetosonic estimate (Del Zanna et
// al. 2007) and the radiation eigenvalues lambda_r1, lambda_r3 (Eqs. lam1-lam3).
// Signed fast-magnetosonic speed estimates lm <= lp along d (Del Zanna et al. 2007).
__device__ __forceinline__ void mhd_speeds(const Params& P, int d, const double* V, double& lm,
                                           double& lp) {
  Aux a;
  aux_of(P, V, a);
  const double cs2 = (P.gamma * V[4]) / a.rhoh;
  const double ca2 = a.bsq / (a.rhoh + a.bsq);
  const double a2 = (cs2 + ca2) - cs2 * ca2;
  const double vd = V[1 + d];
  const double den = 1.0 - a.v2 * a2;
  double disc = (a2 * (1.0 - a.v2)) * (den - (vd * vd) * (1.0 - a2));
  if (disc < 0.0) disc = 0.0;
  const double sq = sqrt(disc);
  lp = (vd * (1.0 - a2) + sq) / den;
  lm = (vd * (1.0 - a2) - sq) / den;
}

// Outer radiation eigenvalues l1 <= l3 (Eqs. lam1-lam3), theta between F_r and d.
__device__ __forceinline__ void rad_speeds(int d, const double* V, double& l1, double& l3) {
  const double E = V[8];
  const double F2 = (V[9] * V[9] + V[10] * V[10]) + V[11] * V[11];
  const double Fn = sqrt(F2);
  double f = Fn / E;
  if (f > 1.0) f = 1.0;
  const double cth = (Fn > 0.0) ? V[9 + d] / Fn : 0.0;
  const double f2 = f * f;
  const double s = sqrt(4.0 - 3.0 * f2);
  double arg = (2.0 / 3.0) * ((4.0 - 3.0 * f2) - s) + (2.0 * (cth * cth)) * ((2.0 - f2) - s);
  if (arg < 0.0) arg = 0.0;
  const double zeta = sqrt(arg);
  l1 = (f * cth - zeta) / s;
  l3 = (f * cth + zeta) / s;
}

__device__ __forceinline__ double signal_speed(const Params& P, int d, const double* V) {
  double lm, lp, l1, l3;
  mhd_speeds(P, d, V, lm, lp);
  const double lf = fabs(lp) > fabs(lm) ? fabs(lp) : fabs(lm);
  rad_speeds(d, V, l1, l3);
  const double lr = fabs(l1) > fabs(l3) ? fabs(l1) : fabs(l3);
  double lam = lf > lr ? lf : lr;
  if (lam > 1.0) lam = 1.0;
  return lam;
}

// ------------------------------------------------------------- four-force
// Eqs. g0, gi with u^i = W v^i, W^2 - 1 = u^2, 2W^2 - 1 = 2u^2 + 1, BP = a_R T^4.
__device__ __forceinline__ void four_force(double kappa, double sigma, double rho,
                                           const double* u, double W, double BP, double E,
                                           const double* F, const double Pr[3][3],
                                           double* G) {
  const double u2 = (u[0] * u[0] + u[1] * u[1]) + u[2] * u[2];
  const double uF = (u[0] * F[0] + u[1] * F[1]) + u[2] * F[2];
  double Pu[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) Pu[i] = (Pr[i][0] * u[0] + Pr[i][1] * u[1]) + Pr[i][2] * u[2];
  const double uPu = (u[0] * Pu[0] + u[1] * Pu[1]) + u[2] * Pu[2];
  const double rk = rho * kappa;
  const double rs = rho * sigma;
  G[0] = -(rk * (W * (BP - E) + uF)) - rs * (((W * u2) * E + W * uPu) - (2.0 * u2 + 1.0) * uF);
  const double q = ((W * W) * E - (2.0 * W) * uF) + uPu;
#pragma unroll
  for (int i = 0; i < 3; ++i)
    G[1 + i] = ((-(BP * rk)) * u[i] + (rk + rs) * (W * F[i] - Pu[i])) - (rs * u[i]) * q;
}

}  // namespace rr
