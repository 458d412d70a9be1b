// physics_tangent.cuh -- face operators with TANGENT (forward-mode dual-number)
// Jacobian products for the PVM-int viscosity (arXiv:2212.00370, Sec. 3.2.2),
// templated on the scalar type S (float for the FP32-bulk form, double for the
// FP64 tangent variant): prim2con, fluxes, M1 closure, con2prim, reconstruction
// and the PVM-int flux.
//
// The paper forms A w by finite differences with eps = 1e-8 (Eq. utilde), which
// is below FP32 resolution (U_m + eps w == U_m).  Here A w = d/dt F(c2p(U_m + t w))
// at t = 0 is computed exactly: the derivative of the con2prim root follows from
// the implicit-function theorem, dW' = -(df/dU . w)/(df/dW'), using the root of
// the single con2prim of U_m, then V and F are evaluated in dual numbers.
// A^2 w = A(A w).  No Newton iteration runs per product.
#pragma once
#include <cstdint>

namespace rrt {

constexpr int NV = 12;

template <class S>
struct PT {
  S gamma, gfac, gm1g;
  int recon, beta_mode, c2p_maxit, pvm_k;
};

// ------------------------------------------------------------- scalar helpers
__device__ __forceinline__ float tsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double tsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float tabs(float a) { return fabsf(a); }
__device__ __forceinline__ double tabs(double a) { return fabs(a); }
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float tmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double tmin(double a, double b) { return fmin(a, b); }
// relative step below which the con2prim Newton takes its one last step
template <class S> __device__ __forceinline__ S c2p_tol();
template <> __device__ __forceinline__ float c2p_tol<float>() { return 1e-5f; }
template <> __device__ __forceinline__ double c2p_tol<double>() { return 1e-10; }

// ------------------------------------------------------------- dual numbers
template <class S>
struct Dual {
  S v, d;
};
template <class S> __device__ __forceinline__ Dual<S> mk(S v, S d = S(0)) { return Dual<S>{v, d}; }
template <class S> __device__ __forceinline__ Dual<S> operator+(Dual<S> a, Dual<S> b) { return {a.v + b.v, a.d + b.d}; }
template <class S> __device__ __forceinline__ Dual<S> operator-(Dual<S> a, Dual<S> b) { return {a.v - b.v, a.d - b.d}; }
template <class S> __device__ __forceinline__ Dual<S> operator-(Dual<S> a) { return {-a.v, -a.d}; }
template <class S> __device__ __forceinline__ Dual<S> operator*(Dual<S> a, Dual<S> b) {
  return {a.v * b.v, a.d * b.v + a.v * b.d};
}
template <class S> __device__ __forceinline__ Dual<S> operator/(Dual<S> a, Dual<S> b) {
  const S q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
// mixed with plain numbers (literals are float constants, exact in double too)
template <class S, class R> __device__ __forceinline__ Dual<S> operator+(Dual<S> a, R b) { return {a.v + S(b), a.d}; }
template <class S, class R> __device__ __forceinline__ Dual<S> operator+(R a, Dual<S> b) { return {S(a) + b.v, b.d}; }
template <class S, class R> __device__ __forceinline__ Dual<S> operator-(Dual<S> a, R b) { return {a.v - S(b), a.d}; }
template <class S, class R> __device__ __forceinline__ Dual<S> operator-(R a, Dual<S> b) { return {S(a) - b.v, -b.d}; }
template <class S, class R> __device__ __forceinline__ Dual<S> operator*(Dual<S> a, R b) { return {a.v * S(b), a.d * S(b)}; }
template <class S, class R> __device__ __forceinline__ Dual<S> operator*(R a, Dual<S> b) { return {S(a) * b.v, S(a) * b.d}; }
template <class S, class R> __device__ __forceinline__ Dual<S> operator/(Dual<S> a, R b) { return {a.v / S(b), a.d / S(b)}; }
template <class S, class R> __device__ __forceinline__ Dual<S> operator/(R a, Dual<S> b) {
  const S q = S(a) / b.v;
  return {q, -q * b.d / b.v};
}
__device__ __forceinline__ float val(float a) { return a; }
__device__ __forceinline__ double val(double a) { return a; }
template <class S> __device__ __forceinline__ S val(Dual<S> a) { return a.v; }
template <class S> __device__ __forceinline__ Dual<S> tsqrt(Dual<S> a) {
  const S s = tsqrt(a.v);
  return {s, a.d * (S(0.5) / s)};
}
// the scalar type of T (S itself, or the S of Dual<S>)
template <class T> struct scalar_of { using type = T; };
template <class S> struct scalar_of<Dual<S>> { using type = S; };
template <class T> __device__ __forceinline__ T cst(double c) { return T(c); }
template <> __device__ __forceinline__ Dual<float> cst<Dual<float>>(double c) { return mk(float(c)); }
template <> __device__ __forceinline__ Dual<double> cst<Dual<double>>(double c) { return mk(c); }

// ------------------------------------------------------------- state functions
template <class T>
struct Aux {
  T v2, iW, W, vB, B2, b0, b[3], bsq, rhoh, ptot;
};

template <class S, class T>
__device__ __forceinline__ void aux_of(const PT<S>& P, const T* V, Aux<T>& a) {
  a.v2 = V[1] * V[1] + V[2] * V[2] + V[3] * V[3];
  a.iW = tsqrt(1.f - a.v2);
  a.W = 1.f / a.iW;
  a.vB = V[1] * V[5] + V[2] * V[6] + V[3] * V[7];
  a.B2 = V[5] * V[5] + V[6] * V[6] + V[7] * V[7];
  a.b0 = a.W * a.vB;
#pragma unroll
  for (int j = 0; j < 3; ++j) a.b[j] = V[5 + j] * a.iW + V[1 + j] * a.b0;
  a.bsq = a.B2 * (a.iW * a.iW) + a.vB * a.vB;
  a.rhoh = V[0] + P.gfac * V[4];
  a.ptot = V[4] + 0.5f * a.bsq;
}

// Eq. eqU
template <class S, class T>
__device__ __forceinline__ void prim2con(const PT<S>& P, const T* V, T* U) {
  Aux<T> a;
  aux_of(P, V, a);
  const T W2 = a.W * a.W;
  const T D = V[0] * a.W;
  const T hw = (a.rhoh + a.bsq) * W2;
  U[0] = D;
#pragma unroll
  for (int j = 0; j < 3; ++j) U[1 + j] = hw * V[1 + j] - a.b0 * a.b[j];
  U[4] = D * ((W2 * a.v2) / (a.W + 1.f)) + (P.gfac * V[4] + a.bsq) * W2 - (a.ptot + a.b0 * a.b0);
#pragma unroll
  for (int k = 5; k < NV; ++k) U[k] = V[k];
}

template <class S, class T>
__device__ __forceinline__ T prim_Z(const PT<S>& P, const T* V) {
  Aux<T> a;
  aux_of(P, V, a);
  return a.rhoh * (a.W * a.W);
}

// Eq. eqF along d with the M1 closure (Sec. 2.2).
template <class S, class T>
__device__ __forceinline__ void flux(const PT<S>& P, int d, const T* V, const T* U, T* F) {
  Aux<T> a;
  aux_of(P, V, a);
  const T vd = V[1 + d];
  const T Bd = V[5 + d];
  const T BdW = Bd * a.iW;
  F[0] = U[0] * vd;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const T t = U[1 + j] * vd - a.b[j] * BdW;
    F[1 + j] = (j == d) ? t + a.ptot : t;
  }
  F[4] = (U[4] + a.ptot) * vd - a.b0 * BdW;
#pragma unroll
  for (int j = 0; j < 3; ++j) F[5 + j] = (j == d) ? cst<T>(0.0) : vd * V[5 + j] - Bd * V[1 + j];
  F[8] = V[9 + d];
  const T E = V[8];
  const T F2 = V[9] * V[9] + V[10] * V[10] + V[11] * V[11];
  T f2 = F2 / (E * E);
  const bool clamped = val(f2) > S(1);
  if (clamped) f2 = cst<T>(1.0);
  const T s = tsqrt(4.f - 3.f * f2);
  const T xi = (3.f + 4.f * f2) / (5.f + 2.f * s);
  const T am = (0.5f * (1.f - xi)) * E;
  // P^ij = am delta_ij + cm F_i F_j with cm = E (3 xi - 1) / (2 F^2).  Since
  // 3 xi - 1 = 6 f^2 / (2 + s) exactly (s^2 = 4 - 3 f^2), cm = 3 / (E (2 + s)): no
  // cancellation of 3 xi - 1 near f = 0 and no 1/|F|^2.  In FP32 the literal form
  // leaves ~1e-7 of rounding in 3 xi - 1; divided by F^2 << E^2 that puts a
  // spurious eigenvalue far above the speed of light into the tangent Jacobian,
  // outside the range where the PVM polynomial approximates |x|.
  const T cm = clamped ? (3.f * E) / ((2.f + s) * F2) : 3.f / (E * (2.f + s));
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const T t = cm * (V[9 + d] * V[9 + j]);
    F[9 + j] = (j == d) ? t + am : t;
  }
}

// ------------------------------------------------------------- con2prim (Mignone & McKinney 2007)
template <class T>
struct C2PIn {
  T D, S[3], tau, B[3], S2, B2, SB, SB2;
};
template <class T>
__device__ __forceinline__ C2PIn<T> c2p_in(const T* U) {
  C2PIn<T> c;
  c.D = U[0];
  c.tau = U[4];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    c.S[j] = U[1 + j];
    c.B[j] = U[5 + j];
  }
  c.S2 = c.S[0] * c.S[0] + c.S[1] * c.S[1] + c.S[2] * c.S[2];
  c.B2 = c.B[0] * c.B[0] + c.B[1] * c.B[1] + c.B[2] * c.B[2];
  c.SB = c.S[0] * c.B[0] + c.S[1] * c.B[1] + c.S[2] * c.B[2];
  c.SB2 = c.SB * c.SB;
  return c;
}

template <class T>
struct C2PPt {
  bool ok;
  T Z, iZ, iZB, v2, W, p, f;
  typename scalar_of<T>::type df;
};

// residual f(W') and, for real arguments, its derivative
template <class S, class T>
__device__ __forceinline__ void c2p_eval(const C2PIn<T>& c, S gm1g, T x, C2PPt<T>& e) {
  e.ok = false;
  if (!(val(x) > S(0))) return;
  const T Z = x + c.D;
  const T ZB = Z + c.B2;
  const T iZ = 1.f / Z;
  const T iZB = 1.f / ZB;
  const T iZ2 = iZ * iZ;
  const T v2 = (c.S2 + c.SB2 * ((2.f * Z + c.B2) * iZ2)) * (iZB * iZB);
  if (!(val(v2) < S(1))) return;
  const T omv2 = 1.f - v2;
  const T W = 1.f / tsqrt(omv2);
  const T p = gm1g * (x * omv2 - c.D * (v2 / (W + 1.f)));
  e.f = (x - p) + (0.5f * c.B2) * (1.f + v2) - ((0.5f * c.SB2) * iZ2 + c.tau);
  const S Zr = val(Z), B2r = val(c.B2), iZBr = val(iZB), iZ2r = val(iZ2), iZr = val(iZ);
  const S dv2 = (S(-2) * iZBr * iZBr * iZBr) *
                (val(c.S2) + val(c.SB2) * ((S(3) * Zr + S(3) * B2r) * Zr + B2r * B2r) * (iZ2r * iZr));
  const S dp = gm1g * (val(omv2) + dv2 * ((S(0.5) * val(c.D)) * val(W) - Zr));
  e.df = (S(1) - dp) + (S(0.5) * B2r) * dv2 + val(c.SB2) * (iZ2r * iZr);
  e.Z = Z;
  e.iZ = iZ;
  e.iZB = iZB;
  e.v2 = v2;
  e.W = W;
  e.p = p;
  e.ok = true;
}

template <class T>
__device__ __forceinline__ void c2p_recover(const C2PIn<T>& c, const C2PPt<T>& e, const T* U, T* V) {
  V[0] = c.D / e.W;
  const T SBiZ = c.SB * e.iZ;
#pragma unroll
  for (int j = 0; j < 3; ++j) V[1 + j] = (c.S[j] + SBiZ * c.B[j]) * e.iZB;
  V[4] = e.p;
#pragma unroll
  for (int k = 5; k < NV; ++k) V[k] = U[k];
}

// Newton in W'; returns the root (x_out) and the residual's derivative there, or false.
template <class S>
__device__ __forceinline__ bool c2p_solve(const PT<S>& P, const C2PIn<S>& c, S Zguess, S& x_out,
                                          C2PPt<S>& e) {
  if (!(c.D > S(0))) return false;
  S x = Zguess - c.D;
  if (!(x > S(0))) x = (c.tau > S(0)) ? c.tau : c.D;
  c2p_eval(c, P.gm1g, x, e);
  for (int k = 0; k < 100 && !e.ok; ++k) {
    x = S(2) * x;
    c2p_eval(c, P.gm1g, x, e);
  }
  if (!e.ok) return false;
  int final_step = 0;
  for (int it = 1; it <= P.c2p_maxit; ++it) {
    S dx = -e.f / e.df;
    C2PPt<S> en;
    c2p_eval(c, P.gm1g, x + dx, en);
    for (int k = 0; k < 40 && !en.ok; ++k) {
      dx = S(0.5) * dx;
      c2p_eval(c, P.gm1g, x + dx, en);
    }
    if (!en.ok) return false;
    x = x + dx;
    e = en;
    if (final_step) {
      x_out = x;
      return e.p > S(0);
    }
    if (tabs(dx) <= c2p_tol<S>() * x) final_step = 1;
  }
  return false;
}

// ------------------------------------------------------------- reconstruction
template <class S>
__device__ __forceinline__ S limiter(int recon, S dL, S dR) {
  if (recon == 0) return S(0);
  if (!(dL * dR > S(0))) return S(0);
  if (recon == 1) return tabs(dL) < tabs(dR) ? dL : dR;
  if (recon == 2) {
    const S m = tmin(tmin(S(2) * tabs(dL), S(2) * tabs(dR)), tabs(S(0.5) * (dL + dR)));
    return dL > S(0) ? m : -m;
  }
  return (S(2) * dL * dR) / (dL + dR);
}

template <class S>
__device__ __forceinline__ void reconstruct(int recon, const S* w0, const S* w1, const S* w2,
                                            S* vm, S* vp) {
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const S s = limiter(recon, w1[k] - w0[k], w2[k] - w1[k]);
    vp[k] = w1[k] + S(0.5) * s;
    vm[k] = w1[k] - S(0.5) * s;
  }
  const bool bad = !(vm[1] * vm[1] + vm[2] * vm[2] + vm[3] * vm[3] < S(1)) ||
                   vm[9] * vm[9] + vm[10] * vm[10] + vm[11] * vm[11] > vm[8] * vm[8] ||
                   !(vp[1] * vp[1] + vp[2] * vp[2] + vp[3] * vp[3] < S(1)) ||
                   vp[9] * vp[9] + vp[10] * vp[10] + vp[11] * vp[11] > vp[8] * vp[8];
  if (bad) {
#pragma unroll
    for (int k = 0; k < NV; ++k) vp[k] = vm[k] = w1[k];
  }
}

// ------------------------------------------------------------- PVM-int, tangent products
// A w at U_m: the con2prim root x_m of U_m (derivative fx there) is differentiated
// by the implicit-function theorem, then V and F are evaluated in dual numbers.
template <class S>
__device__ __forceinline__ bool a_product(const PT<S>& P, int d, const S* Um, S xm, S fx,
                                          const S* w, S* out) {
  Dual<S> U[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) U[k] = mk(Um[k], w[k]);
  const C2PIn<Dual<S>> c = c2p_in(U);
  C2PPt<Dual<S>> e;
  c2p_eval(c, P.gm1g, mk(xm), e);
  if (!e.ok) return false;
  const S dx = -e.f.d / fx;
  c2p_eval(c, P.gm1g, mk(xm, dx), e);
  if (!e.ok) return false;
  Dual<S> V[NV], F[NV];
  c2p_recover(c, e, U, V);
  flux(P, d, V, U, F);
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = F[k].d;
  return true;
}

// Horner coefficients of p_3 (PVM-int-8) and p_4 (PVM-int-16) from Eq. iterat
template <class S>
__device__ __forceinline__ S pvm_coef(int k, int j) {
  if (k == 4) {
    switch (j) {
      case 0: return S(-1.0 / 32768.0);
      case 1: return S(3.0 / 4096.0);
      case 2: return S(-59.0 / 8192.0);
      case 3: return S(169.0 / 4096.0);
      case 4: return S(-2635.0 / 16384.0);
      case 5: return S(1693.0 / 4096.0);
      case 6: return S(-5891.0 / 8192.0);
      case 7: return S(4807.0 / 4096.0);
      default: return S(8463.0 / 32768.0);
    }
  }
  switch (j) {
    case 0: return S(-1.0 / 128.0);
    case 1: return S(3.0 / 32.0);
    case 2: return S(-23.0 / 64.0);
    case 3: return S(31.0 / 32.0);
    default: return S(39.0 / 128.0);
  }
}

// U_m = p_k(A(U_m)) U0 by tangent products (m = 2^(k-1) A^2 products in Horner
// order).  xm, fx: the con2prim root of U_m and the residual's derivative there.
// Returns false if a product fails (the caller then takes Q = I).
template <class S>
__device__ __forceinline__ bool pvm_viscosity(const PT<S>& P, int d, const S* Um, S xm, S fx,
                                              const S* U0, S* Ul) {
  const int m = P.pvm_k == 4 ? 8 : 4;
#pragma unroll
  for (int k = 0; k < NV; ++k) Ul[k] = U0[k];
  for (int l = 0; l < m; ++l) {
    S Y1[NV], Y[NV];
    if (!a_product(P, d, Um, xm, fx, Ul, Y1) || !a_product(P, d, Um, xm, fx, Y1, Y)) return false;
    const S a0 = (l == 0) ? pvm_coef<S>(P.pvm_k, 0) : S(1);
    const S a1 = pvm_coef<S>(P.pvm_k, l + 1);
#pragma unroll
    for (int k = 0; k < NV; ++k) Ul[k] = a0 * Y[k] + a1 * U0[k];
  }
  return true;
}

// F^ = (F_L + F_R)/2 - beta p_k(A(U_m)) (U_R - U_L)/2 (Eqs. generalflux, iterat, beta)
// with the same Horner order in A^2 as the FP64 path; Q = I if U_m has no root.
template <class S>
__device__ __forceinline__ int pvm_flux(const PT<S>& P, int d, const S* VL, const S* VR, S tauL,
                                        S tauR, S* Fhat) {
  S U0[NV], Um[NV];
  S Zg;
  {
    S UL[NV], UR[NV], FL[NV], FR[NV];
    prim2con(P, VL, UL);
    prim2con(P, VR, UR);
    flux(P, d, VL, UL, FL);
    flux(P, d, VR, UR, FR);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      U0[k] = UR[k] - UL[k];
      Um[k] = S(0.5) * (UL[k] + UR[k]);
      Fhat[k] = S(0.5) * (FL[k] + FR[k]);
    }
    Zg = S(0.5) * (prim_Z(P, VL) + prim_Z(P, VR));
  }
  S beta = S(1);
  if (P.beta_mode) beta = S(1) / tmax(tmax(tauL, tauR), S(1));
  S Ul[NV];
  int fail = 1;
  const C2PIn<S> cm = c2p_in(Um);
  S xm;
  C2PPt<S> em;
  if (c2p_solve(P, cm, Zg, xm, em)) fail = pvm_viscosity(P, d, Um, xm, em.df, U0, Ul) ? 0 : 1;
  if (fail) {
#pragma unroll
    for (int k = 0; k < NV; ++k) Ul[k] = U0[k];
  }
#pragma unroll
  for (int k = 0; k < NV; ++k)
    Fhat[k] -= S(0.5) * (((P.beta_mode == 2 && k < 8) ? S(1) : beta) * Ul[k]);  // 2: radiation only
  return fail;
}

// Signed fast-magnetosonic speed estimates (Del Zanna et al. 2007) and the outer
// radiation eigenvalues (Eqs. lam1-lam3) of one state along d.
template <class S>
__device__ __forceinline__ void mhd_speeds(const PT<S>& P, int d, const S* V, S& lm, S& lp) {
  Aux<S> a;
  aux_of(P, V, a);
  const S cs2 = (P.gamma * V[4]) / a.rhoh;
  const S ca2 = a.bsq / (a.rhoh + a.bsq);
  const S a2 = (cs2 + ca2) - cs2 * ca2;
  const S vd = V[1 + d];
  const S den = S(1) - a.v2 * a2;
  S disc = (a2 * (S(1) - a.v2)) * (den - (vd * vd) * (S(1) - a2));
  if (disc < S(0)) disc = S(0);
  const S sq = tsqrt(disc);
  lp = (vd * (S(1) - a2) + sq) / den;
  lm = (vd * (S(1) - a2) - sq) / den;
}

template <class S>
__device__ __forceinline__ void rad_speeds(int d, const S* V, S& l1, S& l3) {
  const S E = V[8];
  const S Fn = tsqrt(V[9] * V[9] + V[10] * V[10] + V[11] * V[11]);
  S f = Fn / E;
  if (f > S(1)) f = S(1);
  const S cth = (Fn > S(0)) ? V[9 + d] / Fn : S(0);
  const S f2 = f * f;
  const S s = tsqrt(S(4) - S(3) * f2);
  S arg = S(2.0 / 3.0) * ((S(4) - S(3) * f2) - s) + (S(2) * (cth * cth)) * ((S(2) - f2) - s);
  if (arg < S(0)) arg = S(0);
  const S zeta = tsqrt(arg);
  l1 = (f * cth - zeta) / s;
  l3 = (f * cth + zeta) / s;
}

// Radiative HLL (Sec. 3.2.1), as in the FP64 path.
template <class S>
__device__ __forceinline__ void radhll_flux(const PT<S>& P, int d, const S* VL, const S* VR, S tauL,
                                            S tauR, S* Fhat) {
  S UL[NV], UR[NV], FL[NV], FR[NV];
  prim2con(P, VL, UL);
  prim2con(P, VR, UR);
  flux(P, d, VL, UL, FL);
  flux(P, d, VR, UR, FR);
  S lmL, lpL, lmR, lpR, r1L, r3L, r1R, r3R;
  mhd_speeds(P, d, VL, lmL, lpL);
  mhd_speeds(P, d, VR, lmR, lpR);
  rad_speeds(d, VL, r1L, r3L);
  rad_speeds(d, VR, r1R, r3R);
  const S sL = tmin(lmL, lmR), sR = tmax(lpL, lpR);
  S rL = tmin(r1L, r1R), rR = tmax(r3L, r3R);
  const S t = tmax(tauL, tauR);
  if (P.beta_mode && t > S(0)) {
    const S lim = S(4) / (S(3) * t);
    rL = tmax(rL, -lim);
    rR = tmin(rR, lim);
  }
  for (int k = 0; k < NV; ++k) {
    const S lo = k < 8 ? sL : rL, hi = k < 8 ? sR : rR;
    if (lo > S(0))
      Fhat[k] = FL[k];
    else if (hi < S(0))
      Fhat[k] = FR[k];
    else if (hi > lo)
      Fhat[k] = ((hi * FL[k] - lo * FR[k]) + (hi * lo) * (UR[k] - UL[k])) / (hi - lo);
    else
      Fhat[k] = S(0.5) * (FL[k] + FR[k]);
  }
}

template <class S>
__device__ __forceinline__ void llf_flux(const PT<S>& P, int d, const S* VL, const S* VR, S* Fhat) {
  S UL[NV], UR[NV], FL[NV], FR[NV];
  prim2con(P, VL, UL);
  prim2con(P, VR, UR);
  flux(P, d, VL, UL, FL);
  flux(P, d, VR, UR, FR);
#pragma unroll
  for (int k = 0; k < NV; ++k) Fhat[k] = S(0.5) * (FL[k] + FR[k]) - S(0.5) * (UR[k] - UL[k]);
}

}  // namespace rrt
