// scheme_f64.cuh -- FP64 interface and cell operators: PLM reconstruction with
// the Godunov fallback, the PVM-int-8 Jacobian-free numerical flux, and the
// implicit radiation-matter solve of one cell (arXiv:2212.00370, Secs. 3.2-3.3).
// Same arithmetic contract as physics_f64.cuh.
#pragma once
#include "physics_f64.cuh"

namespace rr {

// ------------------------------------------------------------ reconstruction
// Slope limiters of Sec. 3.2 (MinMod, MC, VanLeer); zero slope at extrema.
__device__ __forceinline__ double limiter(int recon, double dL, double dR) {
  if (recon == RECON_GODUNOV) return 0.0;
  if (!(dL * dR > 0.0)) return 0.0;
  if (recon == RECON_MINMOD) return fabs(dL) < fabs(dR) ? dL : dR;
  if (recon == RECON_MC) {
    double m = 2.0 * fabs(dL);
    const double r = 2.0 * fabs(dR);
    const double c = fabs(0.5 * (dL + dR));
    if (r < m) m = r;
    if (c < m) m = c;
    return dL > 0.0 ? m : -m;
  }
  return ((2.0 * dL) * dR) / (dL + dR);
}

// Face values of the middle cell: vm at its left face, vp at its right face.
// Either face with |v|^2 >= 1 or |F_r| > E_r sends the cell to first order.
__device__ __forceinline__ void reconstruct(int recon, const double* w0, const double* w1,
                                            const double* w2, double* vm, double* vp) {
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const double s = limiter(recon, w1[k] - w0[k], w2[k] - w1[k]);
    vp[k] = w1[k] + 0.5 * s;
    vm[k] = w1[k] - 0.5 * s;
  }
  const double v2m = (vm[1] * vm[1] + vm[2] * vm[2]) + vm[3] * vm[3];
  const double F2m = (vm[9] * vm[9] + vm[10] * vm[10]) + vm[11] * vm[11];
  const double v2p = (vp[1] * vp[1] + vp[2] * vp[2]) + vp[3] * vp[3];
  const double F2p = (vp[9] * vp[9] + vp[10] * vp[10]) + vp[11] * vp[11];
  const bool bad = !(v2m < 1.0) || F2m > vm[8] * vm[8] || !(v2p < 1.0) || F2p > vp[8] * vp[8];
  if (bad) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      vp[k] = w1[k];
      vm[k] = w1[k];
    }
  }
}

// ------------------------------------------------------------ PVM-int-8 / -16
// Horner coefficients (in x^2, highest degree first) of the internal
// approximations of |x| built by Eq. iterat: k = 3 gives p_3 of degree 8 (the
// printed alpha_0..alpha_4), k = 4 gives p_4 of degree 16 (nine dyadic rationals,
// p_4 = (2 p_3 - p_3^2 + x^2)/2 expanded).
__device__ __constant__ const double PVM_ALPHA[5] = {-1.0 / 128.0, 3.0 / 32.0, -23.0 / 64.0,
                                                     31.0 / 32.0, 39.0 / 128.0};
__device__ __constant__ const double PVM16_ALPHA[9] = {
    -1.0 / 32768.0, 3.0 / 4096.0,     -59.0 / 8192.0, 169.0 / 4096.0, -2635.0 / 16384.0,
    1693.0 / 4096.0, -5891.0 / 8192.0, 4807.0 / 4096.0, 8463.0 / 32768.0};

__device__ __forceinline__ double pvm_alpha(int k, int j) {
  return k == 4 ? PVM16_ALPHA[j] : PVM_ALPHA[j];
}

// A(U_m)^2 w by two nested flux differences (Sec. 3.2.2 steps 3-5, Eq. utilde).
// Returns false if a recovery fails.
__device__ __forceinline__ bool a2_product(const Params& P, int d, const double* Um,
                                           const double* Fm, double Zm, const double* w,
                                           double* out) {
  double Ue[NV], Ve[NV], Fe[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) Ue[k] = Um[k] + P.pvm_eps * w[k];
  if (con2prim(P, Ue, Zm, Ve, nullptr) != ST_OK) return false;
  flux(P, d, Ve, Ue, Fe);
  // reuse Ue/Ve for U~_eps = U_m + F(U_eps) - F(U_m)
#pragma unroll
  for (int k = 0; k < NV; ++k) Ue[k] = Um[k] + (Fe[k] - Fm[k]);
  if (con2prim(P, Ue, Zm, Ve, nullptr) != ST_OK) return false;
  flux(P, d, Ve, Ue, Fe);
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = (Fe[k] - Fm[k]) / P.pvm_eps;
  return true;
}

// F^ = (F_L + F_R)/2 - beta p_k(A(U_m)) (U_R - U_L)/2  (Eqs. generalflux, beta),
// m = 2^(k-1) A^2 products in Horner order (k = 3: PVM-int-8, 4: PVM-int-16);
// Q = I (lambda_max = 1 Rusanov) if a recovery inside the viscosity term fails.
// Returns 1 on that fallback, 0 otherwise.
__device__ __forceinline__ int pvm_flux(const Params& P, int d, const double* VL,
                                        const double* VR, double tauL, double tauR,
                                        double* Fhat) {
  double Um[NV], U0[NV], Fm[NV], Ul[NV];
  double ZL, ZR;
  {
    double UL[NV], UR[NV], FL[NV], FR[NV];
    prim2con(P, VL, UL);
    prim2con(P, VR, UR);
    flux(P, d, VL, UL, FL);
    flux(P, d, VR, UR, FR);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      U0[k] = UR[k] - UL[k];
      Um[k] = 0.5 * (UL[k] + UR[k]);
      Fhat[k] = 0.5 * (FL[k] + FR[k]);  // central part; viscosity subtracted below
    }
    ZL = prim_Z(P, VL);
    ZR = prim_Z(P, VR);
  }
  const double Zg = 0.5 * (ZL + ZR);
  double beta = 1.0;
  if (P.beta_mode) {
    double t = tauL > tauR ? tauL : tauR;
    if (t < 1.0) t = 1.0;
    beta = 1.0 / t;
  }
  int fail = 0;
  double Zm = 0.0;
  {
    double Vm[NV];
    if (con2prim(P, Um, Zg, Vm, &Zm) != ST_OK) {
      fail = 1;
    } else {
      flux(P, d, Vm, Um, Fm);
    }
  }
  if (!fail) {
#pragma unroll
    for (int k = 0; k < NV; ++k) Ul[k] = U0[k];
    const int m = P.pvm_k == 4 ? 8 : 4;
    for (int l = 0; l < m; ++l) {
      double Y[NV];
      if (!a2_product(P, d, Um, Fm, Zm, Ul, Y)) {
        fail = 1;
        break;
      }
      if (l == 0) {
        const double a0 = pvm_alpha(P.pvm_k, 0), a1 = pvm_alpha(P.pvm_k, 1);
#pragma unroll
        for (int k = 0; k < NV; ++k) Ul[k] = a0 * Y[k] + a1 * U0[k];
      } else {
        const double al = pvm_alpha(P.pvm_k, l + 1);
#pragma unroll
        for (int k = 0; k < NV; ++k) Ul[k] = Y[k] + al * U0[k];
      }
    }
  }
  if (fail) {
#pragma unroll
    for (int k = 0; k < NV; ++k) Ul[k] = U0[k];
  }
  // beta_mode 2: Eq. beta on the radiation block only (beta = 1 on the magnetofluid)
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const double bk = (P.beta_mode == 2 && k < 8) ? 1.0 : beta;
    Fhat[k] = Fhat[k] - 0.5 * (bk * Ul[k]);
  }
  return fail;
}

// HLL flux of components [k0, k1) with wave speeds sL <= sR (Sec. 3.2.1); a
// degenerate fan (sR == sL == 0) takes the central flux.
__device__ __forceinline__ void hll_block(int k0, int k1, double sL, double sR, const double* UL,
                                          const double* UR, const double* FL, const double* FR,
                                          double* F) {
  for (int k = k0; k < k1; ++k) {
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

// Radiative HLL (Sec. 3.2.1): magnetofluid block with the fast-magnetosonic speeds
// of the two states, radiation block with lambda_r1/lambda_r3, limited by Eq. limits
// to 4/(3 tau) (tau the larger of the two cells' optical depths) when beta_mode.
__device__ __forceinline__ void radhll_flux(const Params& P, int d, const double* VL,
                                            const double* VR, double tauL, double tauR,
                                            double* Fhat) {
  double UL[NV], UR[NV], FL[NV], FR[NV];
  prim2con(P, VL, UL);
  prim2con(P, VR, UR);
  flux(P, d, VL, UL, FL);
  flux(P, d, VR, UR, FR);
  double lmL, lpL, lmR, lpR, r1L, r3L, r1R, r3R;
  mhd_speeds(P, d, VL, lmL, lpL);
  mhd_speeds(P, d, VR, lmR, lpR);
  rad_speeds(d, VL, r1L, r3L);
  rad_speeds(d, VR, r1R, r3R);
  const double sL = lmL < lmR ? lmL : lmR;
  const double sR = lpL > lpR ? lpL : lpR;
  double rL = r1L < r1R ? r1L : r1R;
  double rR = r3L > r3R ? r3L : r3R;
  const double t = tauL > tauR ? tauL : tauR;
  if (P.beta_mode && t > 0.0) {
    const double lim = 4.0 / (3.0 * t);
    if (rL < -lim) rL = -lim;
    if (rR > lim) rR = lim;
  }
  hll_block(0, 8, sL, sR, UL, UR, FL, FR, Fhat);
  hll_block(8, 12, rL, rR, UL, UR, FL, FR, Fhat);
}

// First-order Rusanov flux with lambda_max = 1 (Q = I in Eq. generalflux) from
// the cell-centre states; used only by the admissibility fallback.
__device__ __forceinline__ void llf_flux(const Params& P, int d, const double* VL,
                                         const double* VR, double* Fhat) {
  double UL[NV], UR[NV], FL[NV], FR[NV];
  prim2con(P, VL, UL);
  prim2con(P, VR, UR);
  flux(P, d, VL, UL, FL);
  flux(P, d, VR, UR, FR);
#pragma unroll
  for (int k = 0; k < NV; ++k) Fhat[k] = 0.5 * (FL[k] + FR[k]) - 0.5 * (UR[k] - UL[k]);
}

// ------------------------------------------------------------ implicit step
// Per cell, solve R(X) = X - X* + h G(X, V(X)) = 0 for X = (E_r, F_r), with the
// magnetofluid from the conserved totals tau_t = tau* + E*, S_t = S* + F*
// (Eqs. timeadv, totale, totalm) and V(X) its con2prim (Sec. 3.3 step 5).
struct ImpCell {
  double kappa, sigma, hdt;
  double D, St[3], taut, B[3], Xs[4];
  double iD;  // 1/D (the FP32-bulk form's residual)
};

// Forms of the cell solver.  FormF64: the FP64 form, in the oracle's operation order
// (bit parity).  FormBulk: the FP32-bulk form, whose faces carry FP32 rounding (~1e-7
// relative), so its cells may spend less FP64 work where that changes no digit the
// form keeps: the iteration matrix in FP32 (newton_dir); a residual that takes W from
// con2prim's root and T = p W / D (a square root and two divisions fewer, the same
// values to rounding); con2prim<true>: evaluations with 1/Z and 1/(Z+B^2) from one
// division and W from rsqrt, Newton steps with an FP32 reciprocal of the derivative,
// rho = D (1 - v^2) W (the same root to a few ulps); and the polish of the converged
// root only where the radiation energy exceeds 100x the matter energy.  The
// polish moves the root by ~1e-11 E_r; the matter (tau_e = tau_t - E_r, S = S_t - F_r)
// takes that error relative to its own size, ~1e-11 E_r / tau_e: below 1e-9 unless the
// radiation dominates, where it would reach the 1e-5 level (the 2D blast, E_r ~ 1e6
// tau_e) and the polish is kept.
struct FormF64 {
  using Mat = double;
  static constexpr bool kReuseW = false;
  static constexpr bool kFastC2P = false;
  __device__ static bool polish(const ImpCell&, const double*) { return true; }
};
struct FormBulk {
  using Mat = float;
  static constexpr bool kReuseW = true;
  static constexpr bool kFastC2P = true;
  __device__ static bool polish(const ImpCell& c, const double* X) {
    return X[0] > 100.0 * (c.taut - X[0]);
  }
};

__device__ __forceinline__ void matter_state(const ImpCell& c, const double* X, double* Um) {
  Um[0] = c.D;
  Um[1] = c.St[0] - X[1];
  Um[2] = c.St[1] - X[2];
  Um[3] = c.St[2] - X[3];
  Um[4] = c.taut - X[0];
  Um[5] = c.B[0];
  Um[6] = c.B[1];
  Um[7] = c.B[2];
  Um[8] = X[0];
  Um[9] = X[1];
  Um[10] = X[2];
  Um[11] = X[3];
}

// Returns false if X is inadmissible (E_r <= 0 or no con2prim root).
template <class F>
static __device__ __noinline__ bool imp_residual(const Params& P, const ImpCell& c, const double* X,
                                                 double Zg, double* R, double* V, double* Z) {
  if (!(X[0] > 0.0)) return false;
  double Um[NV];
  matter_state(c, X, Um);
  double W, T;
  if constexpr (F::kReuseW) {  // W of con2prim's root; T = p / rho = p W / D
    if (con2prim<F::kFastC2P>(P, Um, Zg, V, Z, &W) != ST_OK) return false;
    T = V[4] * (W * c.iD);
  } else {
    if (con2prim(P, Um, Zg, V, Z) != ST_OK) return false;
    const double v2 = (V[1] * V[1] + V[2] * V[2]) + V[3] * V[3];
    W = 1.0 / sqrt(1.0 - v2);
    T = V[4] / V[0];
  }
  const M1 m = m1_coef(X[0], X[1], X[2], X[3]);
  const double u[3] = {W * V[1], W * V[2], W * V[3]};
  const double BP = P.a_rad * ((T * T) * (T * T));
  double Pr[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Pr[i][j] = m1_P(m, X + 1, i, j);
  double G[4];
  four_force(c.kappa, c.sigma, V[0], u, W, BP, X[0], X + 1, Pr, G);
#pragma unroll
  for (int i = 0; i < 4; ++i) R[i] = (X[i] - c.Xs[i]) + c.hdt * G[i];
  return true;
}

// Gaussian elimination with partial pivoting (A, b overwritten); false if singular.
// T: double (the FP64 form and the matter form), or float for the matrix of the
// FP32-bulk form's iteration on X.
template <class T>
__device__ __forceinline__ bool solve4(T A[4][4], T b[4], T x[4]) {
#pragma unroll
  for (int col = 0; col < 4; ++col) {
    int piv = col;
#pragma unroll
    for (int r = col + 1; r < 4; ++r)
      if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
    if (A[piv][col] == T(0)) return false;
    if (piv != col) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const T t = A[col][k];
        A[col][k] = A[piv][k];
        A[piv][k] = t;
      }
      const T t = b[col];
      b[col] = b[piv];
      b[piv] = t;
    }
#pragma unroll
    for (int r = col + 1; r < 4; ++r) {
      const T f = A[r][col] / A[col][col];
#pragma unroll
      for (int k = col + 1; k < 4; ++k) A[r][k] = A[r][k] - f * A[col][k];
      b[r] = b[r] - f * b[col];
    }
  }
#pragma unroll
  for (int r = 3; r >= 0; --r) {
    T s = b[r];
#pragma unroll
    for (int k = r + 1; k < 4; ++k) s = s - A[r][k] * x[k];
    x[r] = s / A[r][r];
  }
  return true;
}

// C^(m) of Sec. 3.3 step 2 (matter and Eddington tensor frozen), with the
// C_{i+1,j+1} sign derived from Eqs. g0/gi: delta + h rho W[(k+s) delta + 2 s u u].
__device__ __forceinline__ void picard_matrix(const ImpCell& c, const double* X,
                                              const double* V, double J[4][4]) {
  const double v2 = (V[1] * V[1] + V[2] * V[2]) + V[3] * V[3];
  const double W = 1.0 / sqrt(1.0 - v2);
  const double u[3] = {W * V[1], W * V[2], W * V[3]};
  const double rho = V[0];
  double Dr[3][3];
  eddington(X[0], X + 1, Dr);
  const double u2 = (u[0] * u[0] + u[1] * u[1]) + u[2] * u[2];
  double Du[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) Du[i] = (Dr[i][0] * u[0] + Dr[i][1] * u[1]) + Dr[i][2] * u[2];
  const double uDu = (u[0] * Du[0] + u[1] * Du[1]) + u[2] * Du[2];
  const double ks = c.kappa + c.sigma;
  const double h = c.hdt;
  J[0][0] = 1.0 - h * ((rho * W) * (-c.kappa + c.sigma * (u2 + uDu)));
#pragma unroll
  for (int j = 0; j < 3; ++j)
    J[0][1 + j] = -h * ((rho * u[j]) * (c.kappa - c.sigma * (2.0 * u2 + 1.0)));
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    J[1 + i][0] = -h * (rho * (ks * Du[i] + (c.sigma * u[i]) * ((W * W) + uDu)));
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double t = h * ((rho * W) * ((i == j ? ks : 0.0) + (2.0 * c.sigma) * (u[i] * u[j])));
      J[1 + i][1 + j] = (i == j ? 1.0 : 0.0) + t;
    }
  }
}

// The iteration on X keeps its matrix J (an approximation of dR/dX: C^(m), the
// cell's cache, Broyden updates, forward differences) in JT = F::Mat.  JT = double is
// the FP64 form.  JT = float is the FP32-bulk form: the residual R, the iterate X and
// every convergence test stay FP64, so the root is the FP64 root; only the Newton
// direction is solved, and the matrix updated, in FP32.  A direction with a relative
// error of ~1e-7 cond(J) is an inexact quasi-Newton step whose error the next FP64
// residual corrects, as the Broyden matrix's own (larger) error is.

// Newton direction dX = -J^-1 R: solved in JT, returned in double; false if singular.
template <class JT>
__device__ __forceinline__ bool newton_dir(const JT J[4][4], const double* R, double* dX) {
  JT A[4][4], b[4], x[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    b[i] = (JT)(-R[i]);
#pragma unroll
    for (int j = 0; j < 4; ++j) A[i][j] = J[i][j];
  }
  if (!solve4(A, b, x)) return false;
#pragma unroll
  for (int i = 0; i < 4; ++i) dX[i] = (double)x[i];
  return true;
}

// Broyden's rank-one update with the accepted step dX and residual change Rn - R:
// J += (dR - J dX) dX^T / (dX . dX), in JT.
template <class JT>
__device__ __forceinline__ void broyden(JT J[4][4], const double* dXd, const double* R,
                                        const double* Rn) {
  JT dX[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) dX[i] = (JT)dXd[i];
  const JT s2 = ((dX[0] * dX[0] + dX[1] * dX[1]) + dX[2] * dX[2]) + dX[3] * dX[3];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const JT dRi = (JT)(Rn[i] - R[i]);
    const JT Jd = ((J[i][0] * dX[0] + J[i][1] * dX[1]) + J[i][2] * dX[2]) + J[i][3] * dX[3];
    const JT q = (dRi - Jd) / s2;
#pragma unroll
    for (int j = 0; j < 4; ++j) J[i][j] = J[i][j] + q * dX[j];
  }
}

// Forward-difference Jacobian of R at X (step 1e-7 E_r; a backward step where the
// forward one leaves the admissible set).  False if neither is admissible.
template <class F>
static __device__ __noinline__ bool fd_jacobian(const Params& P, const ImpCell& c, const double* X,
                                                const double* R, double Z, typename F::Mat J[4][4]) {
  using JT = typename F::Mat;
  const double h = 1e-7 * X[0];
  for (int j = 0; j < 4; ++j) {
    double Xp[4] = {X[0], X[1], X[2], X[3]};
    double Rp[4], Vp[NV], Zp;
    Xp[j] = X[j] + h;
    if (!imp_residual<F>(P, c, Xp, Z, Rp, Vp, &Zp)) {
      Xp[j] = X[j] - h;
      if (!imp_residual<F>(P, c, Xp, Z, Rp, Vp, &Zp)) return false;
    }
    const double dXj = Xp[j] - X[j];
#pragma unroll
    for (int i = 0; i < 4; ++i) J[i][j] = (JT)((Rp[i] - R[i]) / dXj);
  }
  return true;
}

constexpr double IMP_POLISH_TOL = 1e-14;  // polished root: last correction <= 1e-14 E_r
constexpr int IMP_POLISH_MAX = 6;         // at most six polishing corrections

// Polish of a converged iterate.  Stopping at imp_tol leaves an error of about the
// last step times the matrix's contraction, which depends on how the iterate was
// reached (first matrix, Broyden history, the cell's cache).  The iterate is refined
// towards the root of R itself, so that the result is a function of the cell's state:
// corrections dX = -J^-1 R(X), accepted without line search, J updated by Broyden's
// formula after each, until a correction is <= 1e-14 E_r.  A correction that does not
// halve the previous one means the rounding floor of R is reached: the polish stops
// there without taking it.  last is the size of the converged step.  X, R, V and Z
// stay those of the last accepted iterate.
template <class F>
static __device__ __noinline__ void imp_polish(const Params& P, const ImpCell& c, typename F::Mat J[4][4],
                                               double* X, double* R, double* V, double* Z,
                                               double last) {
  double prev = last;
  for (int p = 0; p < IMP_POLISH_MAX; ++p) {
    double dX[4];
    if (!newton_dir(J, R, dX)) return;
    double d = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) d = fabs(dX[i]) > d ? fabs(dX[i]) : d;
    if (d <= IMP_POLISH_TOL * X[0]) return;
    if (p > 0 && d > 0.5 * prev) return;
    double Xn[4], Rn[4], Vn[NV], Zn = *Z;
#pragma unroll
    for (int i = 0; i < 4; ++i) Xn[i] = X[i] + dX[i];
    if (!imp_residual<F>(P, c, Xn, *Z, Rn, Vn, &Zn)) return;
    broyden(J, dX, R, Rn);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      X[i] = Xn[i];
      R[i] = Rn[i];
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) V[k] = Vn[k];
    *Z = Zn;
    prev = d;
  }
}

// Quasi-Newton iteration on R(X) = 0: first matrix C^(m) (the paper's
// frozen-matter iteration), Broyden rank-one update after every accepted step,
// forward-difference Jacobian (step 1e-7 E_r) when successive steps contract by
// less than 2x or no descent is found; Armijo backtracking on |R|^2 (at most ten
// halvings); converged
// when the full step is <= imp_tol * E_r, then polished (imp_polish).  Returns true
// on convergence.
template <class F>
static __device__ __noinline__ bool imp_newton(const Params& P, const ImpCell& c, double* X, double* R,
                                               double* V, double* Z, const double* Min, double* Mout) {
  using JT = typename F::Mat;
  JT J[4][4];
  int need_fd = 0, fresh_fd = 0, first = 1;
  double prev = -1.0;
  if (Min) {  // the cell's matrix from its previous solve: J = I + h M
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) J[i][j] = (JT)((i == j ? 1.0 : 0.0) + c.hdt * Min[4 * i + j]);
  } else {
    double Jd[4][4];
    picard_matrix(c, X, V, Jd);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) J[i][j] = (JT)Jd[i][j];
  }
  for (int m = 1; m <= P.imp_maxit; ++m) {
    if (need_fd) {
      if (!fd_jacobian<F>(P, c, X, R, *Z, J)) return false;
      need_fd = 0;
      fresh_fd = 1;
      first = 0;
    }
    double dX[4];
    if (!newton_dir(J, R, dX)) {
      if (!fresh_fd) {
        need_fd = 1;
        continue;
      }
      return false;
    }

    double dfull = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) dfull = fabs(dX[i]) > dfull ? fabs(dX[i]) : dfull;
    double Xn[4], Rn[4], Vn[NV], Zn = *Z;
    if (dfull <= P.imp_tol * X[0]) {
#pragma unroll
      for (int i = 0; i < 4; ++i) Xn[i] = X[i] + dX[i];
      if (!imp_residual<F>(P, c, Xn, *Z, Rn, Vn, &Zn)) return false;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        X[i] = Xn[i];
        R[i] = Rn[i];
      }
#pragma unroll
      for (int k = 0; k < NV; ++k) V[k] = Vn[k];
      *Z = Zn;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          Mout[4 * i + j] = ((double)J[i][j] - (i == j ? 1.0 : 0.0)) / c.hdt;
      if (F::polish(c, X)) imp_polish<F>(P, c, J, X, R, V, Z, dfull);
      return true;
    }
    const double r0 = ((R[0] * R[0] + R[1] * R[1]) + R[2] * R[2]) + R[3] * R[3];
    double lam = 1.0;
    int ok = 0;
    for (int k = 0; k < 10; ++k) {  // at most ten halvings
#pragma unroll
      for (int i = 0; i < 4; ++i) Xn[i] = X[i] + dX[i];
      if (imp_residual<F>(P, c, Xn, *Z, Rn, Vn, &Zn)) {
        const double r1 = ((Rn[0] * Rn[0] + Rn[1] * Rn[1]) + Rn[2] * Rn[2]) + Rn[3] * Rn[3];
        if (r1 <= (1.0 - 1e-4 * lam) * r0) {
          ok = 1;
          break;
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) dX[i] = 0.5 * dX[i];
      lam = 0.5 * lam;
      if (first && k == 3) break;
    }
    if (!ok) {
      if (!fresh_fd) {
        need_fd = 1;
        continue;
      }
      return false;
    }
    double dmax = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const double dd = fabs(dX[i]);
      if (dd > dmax) dmax = dd;
    }
    broyden(J, dX, R, Rn);
    fresh_fd = 0;
    first = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      X[i] = Xn[i];
      R[i] = Rn[i];
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) V[k] = Vn[k];
    *Z = Zn;
    if (prev >= 0.0 && dmax > 0.5 * prev) need_fd = 1;
    prev = dmax;
  }
  return false;
}

constexpr int IMP_LADDER = 6;  // continuation fallback starts at h / 2^6

// The same residual as a function of the matter primitives Y = (p, u^i):
// rho = D/W, W = sqrt(1 + u.u), v = u/W, B fixed, X = (tau_t - tau_e(Y), S_t - S(Y)).
// Where the radiation carries nearly all the energy the matter is a small
// difference of X and the totals, and the iteration on X loses it; this form
// keeps it (the MHD-field iteration of Melon Fuksman & Mignone 2019).  Also
// returns X and the primitives (matter from Y, radiation X).
static __device__ __noinline__ bool imp_residual_m(const Params& P, const ImpCell& c,
                                                   const double* Y, double* R, double* X,
                                                   double* V) {
  if (!(Y[0] > 0.0)) return false;
  const double W = sqrt(1.0 + ((Y[1] * Y[1] + Y[2] * Y[2]) + Y[3] * Y[3]));
  double Um[NV];
  V[0] = c.D / W;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    V[1 + i] = Y[1 + i] / W;
    V[5 + i] = c.B[i];
    V[9 + i] = 0.0;
  }
  V[4] = Y[0];
  V[8] = 0.0;
  prim2con(P, V, Um);
  X[0] = c.taut - Um[4];
#pragma unroll
  for (int i = 0; i < 3; ++i) X[1 + i] = c.St[i] - Um[1 + i];
  if (!(X[0] > 0.0)) return false;
#pragma unroll
  for (int i = 0; i < 4; ++i) V[8 + i] = X[i];
  const double T = Y[0] / V[0];
  const double BP = P.a_rad * ((T * T) * (T * T));
  const M1 m = m1_coef(X[0], X[1], X[2], X[3]);
  double Pr[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Pr[i][j] = m1_P(m, X + 1, i, j);
  double G[4];
  four_force(c.kappa, c.sigma, V[0], Y + 1, W, BP, X[0], X + 1, Pr, G);
#pragma unroll
  for (int i = 0; i < 4; ++i) R[i] = (X[i] - c.Xs[i]) + c.hdt * G[i];
  return true;
}

// Newton's method on R(Y) = 0 from Y: forward-difference Jacobian at every iterate
// (steps 1e-7 of the scales p and 1 + |u|), backtracking on |R|^2; converged when
// every component of the full step is <= 100 imp_tol times its scale (R keeps the
// rounding of the radiation-sized terms, which the Jacobian carries into Y).
static __device__ __noinline__ bool imp_newton_m(const Params& P, const ImpCell& c, double* Y,
                                                 double* X, double* V) {
  double R[4];
  if (!imp_residual_m(P, c, Y, R, X, V)) return false;
  for (int m = 1; m <= P.imp_maxit; ++m) {
    const double su = 1.0 + sqrt((Y[1] * Y[1] + Y[2] * Y[2]) + Y[3] * Y[3]);
    const double sc[4] = {Y[0], su, su, su};
    double J[4][4];
    for (int j = 0; j < 4; ++j) {
      double Yp[4] = {Y[0], Y[1], Y[2], Y[3]};
      double Rp[4], Xp[4], Vp[NV];
      Yp[j] = Y[j] + 1e-7 * sc[j];
      if (!imp_residual_m(P, c, Yp, Rp, Xp, Vp)) {
        Yp[j] = Y[j] - 1e-7 * sc[j];
        if (!imp_residual_m(P, c, Yp, Rp, Xp, Vp)) return false;
      }
      const double dYj = Yp[j] - Y[j];
#pragma unroll
      for (int i = 0; i < 4; ++i) J[i][j] = (Rp[i] - R[i]) / dYj;
    }
    double b[4], dY[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) b[i] = -R[i];
    if (!solve4(J, b, dY)) return false;
    bool conv = true;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (fabs(dY[i]) > (100.0 * P.imp_tol) * sc[i]) conv = false;
    double Yn[4], Rn[4], Xn[4], Vn[NV];
    if (conv) {
#pragma unroll
      for (int i = 0; i < 4; ++i) Yn[i] = Y[i] + dY[i];
      if (!imp_residual_m(P, c, Yn, Rn, Xn, Vn)) return false;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        Y[i] = Yn[i];
        X[i] = Xn[i];
      }
#pragma unroll
      for (int k = 0; k < NV; ++k) V[k] = Vn[k];
      return true;
    }
    const double r0 = ((R[0] * R[0] + R[1] * R[1]) + R[2] * R[2]) + R[3] * R[3];
    double lam = 1.0;
    bool ok = false;
    for (int k = 0; k < 40; ++k) {
#pragma unroll
      for (int i = 0; i < 4; ++i) Yn[i] = Y[i] + dY[i];
      if (imp_residual_m(P, c, Yn, Rn, Xn, Vn)) {
        const double r1 = ((Rn[0] * Rn[0] + Rn[1] * Rn[1]) + Rn[2] * Rn[2]) + Rn[3] * Rn[3];
        if (r1 <= (1.0 - 1e-4 * lam) * r0) {
          ok = true;
          break;
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) dY[i] = 0.5 * dY[i];
      lam = 0.5 * lam;
    }
    if (!ok) return false;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      Y[i] = Yn[i];
      R[i] = Rn[i];
      X[i] = Xn[i];
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) V[k] = Vn[k];
  }
  return false;
}

// The matter-primitive solve from the matter state of U* (primitives Vs).
__device__ __forceinline__ bool solve_matter(const Params& P, const ImpCell& c, const double* Vs,
                                             double* X, double* V) {
  const double v2 = (Vs[1] * Vs[1] + Vs[2] * Vs[2]) + Vs[3] * Vs[3];
  const double W = 1.0 / sqrt(1.0 - v2);
  double Y[4] = {Vs[4], W * Vs[1], W * Vs[2], W * Vs[3]};
  return imp_newton_m(P, c, Y, X, V);
}

// Implicit step of one cell (Sec. 3.3).  Writes U and V on success; returns a Status.
// jc (may be null): the cell's Jacobian cache, M = (J - I)/h of its last converged
// solve (16 entries) and a flag jc[16]; with flag 1 M replaces C^(m) as the first
// matrix, and the converged matrix is stored back (cleared on failure).  Flag 2: the
// last solve needed the matter primitives, and the next one starts there.  Order:
// [flag 2: matter solve]; iteration on X; continuation in h on X; matter solve
// (unless it was the first attempt).
template <class F = FormF64>
__device__ __forceinline__ int implicit_cell(const Params& P, double kappa, double sigma,
                                             double hdt, const double* Us, double Zguess,
                                             double* U, double* V, double* jc = nullptr) {
  if ((kappa == 0.0 && sigma == 0.0) || hdt == 0.0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) U[k] = Us[k];
    return con2prim(P, Us, Zguess, V, nullptr);
  }
  ImpCell c;
  c.kappa = kappa;
  c.sigma = sigma;
  c.hdt = hdt;
  c.D = Us[0];
  c.taut = Us[4] + Us[8];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    c.St[j] = Us[1 + j] + Us[9 + j];
    c.B[j] = Us[5 + j];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) c.Xs[i] = Us[8 + i];
  double X[4] = {c.Xs[0], c.Xs[1], c.Xs[2], c.Xs[3]};
  double R[4], Z = Zguess;
  // no admissible matter state at X*: the explicit update U* itself is inadmissible
  if constexpr (F::kReuseW) c.iD = 1.0 / c.D;
  if (!imp_residual<F>(P, c, X, Zguess, R, V, &Z)) return ST_C2P;
  double Mnew[16], Vs[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) Vs[k] = V[k];
  const bool tried_m = jc && jc[16] == 2.0;
  if (tried_m) {
    if (solve_matter(P, c, Vs, X, V)) {
      matter_state(c, X, U);
      return ST_OK;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) X[i] = c.Xs[i];
#pragma unroll
    for (int k = 0; k < NV; ++k) V[k] = Vs[k];
    Z = Zguess;
    imp_residual<F>(P, c, X, Z, R, V, &Z);
  }
  bool ok = imp_newton<F>(P, c, X, R, V, &Z, (jc && jc[16] == 1.0) ? jc : nullptr, Mnew);
  if (!ok) {
#pragma unroll
    for (int i = 0; i < 4; ++i) X[i] = c.Xs[i];
    Z = Zguess;
    ok = true;
    for (int j = IMP_LADDER; j >= 0 && ok; --j) {
      c.hdt = hdt / (double)(1 << j);
      ok = imp_residual<F>(P, c, X, Z, R, V, &Z);
      if (ok) ok = imp_newton<F>(P, c, X, R, V, &Z, nullptr, Mnew);
    }
    c.hdt = hdt;
  }
  bool matter = false;
  if (!ok && !tried_m) {
    ok = solve_matter(P, c, Vs, X, V);
    matter = ok;
  }
  if (jc) {
#pragma unroll
    for (int k = 0; k < 16; ++k) jc[k] = (ok && !matter) ? Mnew[k] : 0.0;
    jc[16] = ok ? (matter ? 2.0 : 1.0) : 0.0;
  }
  if (!ok) return ST_IMPLICIT;
  matter_state(c, X, U);
  return ST_OK;
}

}  // namespace rr
