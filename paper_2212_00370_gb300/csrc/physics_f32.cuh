// physics_f32.cuh -- FP32 face operators of the FP32-bulk form: reconstruction,
// prim2con, fluxes, M1 closure, con2prim and the PVM-int-8 flux with TANGENT
// (forward-mode dual-number) Jacobian products (arXiv:2212.00370, Sec. 3.2.2).
//
// The paper forms A w by finite differences with eps = 1e-8 (Eq. utilde), which
// is below FP32 resolution (U_m + eps w == U_m).  Here A w = d/dt F(c2p(U_m + t w))
// at t = 0 is computed exactly in FP32: the derivative of the con2prim root
// follows from the implicit-function theorem, dW' = -(df/dU . w)/(df/dW'), using
// the root of the single FP32 con2prim of U_m, then V and F are evaluated in dual
// numbers.  A^2 w = A(A w).  No Newton iteration runs per product.
#pragma once
#include <cstdint>

namespace rr32 {

constexpr int NV = 12;

struct P32 {
  float gamma, gfac, gm1g;
  int recon, beta_mode, c2p_maxit;
};

// ------------------------------------------------------------- dual numbers
struct Dual {
  float v, d;
};
__device__ __forceinline__ Dual mk(float v, float d = 0.f) { return Dual{v, d}; }
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const float q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ Dual operator+(Dual a, float b) { return {a.v + b, a.d}; }
__device__ __forceinline__ Dual operator+(float a, Dual b) { return {a + b.v, b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, float b) { return {a.v - b, a.d}; }
__device__ __forceinline__ Dual operator-(float a, Dual b) { return {a - b.v, -b.d}; }
__device__ __forceinline__ Dual operator*(Dual a, float b) { return {a.v * b, a.d * b}; }
__device__ __forceinline__ Dual operator*(float a, Dual b) { return {a * b.v, a * b.d}; }
__device__ __forceinline__ Dual operator/(Dual a, float b) { return {a.v / b, a.d / b}; }
__device__ __forceinline__ Dual operator/(float a, Dual b) {
  const float q = a / b.v;
  return {q, -q * b.d / b.v};
}
__device__ __forceinline__ float val(float a) { return a; }
__device__ __forceinline__ float val(Dual a) { return a.v; }
__device__ __forceinline__ float tsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ Dual tsqrt(Dual a) {
  const float s = sqrtf(a.v);
  return {s, a.d * (0.5f / s)};
}
template <class T> __device__ __forceinline__ T cst(float c) { return T(c); }
template <> __device__ __forceinline__ Dual cst<Dual>(float c) { return mk(c); }

// ------------------------------------------------------------- state functions
template <class T>
struct Aux {
  T v2, iW, W, vB, B2, b0, b[3], bsq, rhoh, ptot;
};

template <class T>
__device__ __forceinline__ void aux_of(const P32& P, const T* V, Aux<T>& a) {
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
template <class T>
__device__ __forceinline__ void prim2con(const P32& P, const T* V, T* U) {
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

template <class T>
__device__ __forceinline__ T prim_Z(const P32& P, const T* V) {
  Aux<T> a;
  aux_of(P, V, a);
  return a.rhoh * (a.W * a.W);
}

// Eq. eqF along d with the M1 closure (Sec. 2.2), as in the FP64 path.
template <class T>
__device__ __forceinline__ void flux(const P32& P, int d, const T* V, const T* U, T* F) {
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
  for (int j = 0; j < 3; ++j) F[5 + j] = (j == d) ? cst<T>(0.f) : vd * V[5 + j] - Bd * V[1 + j];
  F[8] = V[9 + d];
  const T E = V[8];
  const T F2 = V[9] * V[9] + V[10] * V[10] + V[11] * V[11];
  T f2 = F2 / (E * E);
  const bool clamped = val(f2) > 1.f;
  if (clamped) f2 = cst<T>(1.f);
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
  float df;
};

// residual f(W') and, for real arguments, its derivative
template <class T>
__device__ __forceinline__ void c2p_eval(const C2PIn<T>& c, float gm1g, T x, C2PPt<T>& e) {
  e.ok = false;
  if (!(val(x) > 0.f)) return;
  const T Z = x + c.D;
  const T ZB = Z + c.B2;
  const T iZ = 1.f / Z;
  const T iZB = 1.f / ZB;
  const T iZ2 = iZ * iZ;
  const T v2 = (c.S2 + c.SB2 * ((2.f * Z + c.B2) * iZ2)) * (iZB * iZB);
  if (!(val(v2) < 1.f)) return;
  const T omv2 = 1.f - v2;
  const T W = 1.f / tsqrt(omv2);
  const T p = gm1g * (x * omv2 - c.D * (v2 / (W + 1.f)));
  e.f = (x - p) + (0.5f * c.B2) * (1.f + v2) - ((0.5f * c.SB2) * iZ2 + c.tau);
  const float Zr = val(Z), B2r = val(c.B2), iZBr = val(iZB), iZ2r = val(iZ2), iZr = val(iZ);
  const float dv2 = (-2.f * iZBr * iZBr * iZBr) *
                    (val(c.S2) + val(c.SB2) * ((3.f * Zr + 3.f * B2r) * Zr + B2r * B2r) * (iZ2r * iZr));
  const float dp = gm1g * (val(omv2) + dv2 * ((0.5f * val(c.D)) * val(W) - Zr));
  e.df = (1.f - dp) + (0.5f * B2r) * dv2 + val(c.SB2) * (iZ2r * iZr);
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

// FP32 Newton; returns the root W' (x) and df/dW' there, or false.
__device__ __forceinline__ bool c2p_solve(const P32& P, const C2PIn<float>& c, float Zguess,
                                          float& x_out, C2PPt<float>& e) {
  if (!(c.D > 0.f)) return false;
  float x = Zguess - c.D;
  if (!(x > 0.f)) x = (c.tau > 0.f) ? c.tau : c.D;
  c2p_eval(c, P.gm1g, x, e);
  for (int k = 0; k < 100 && !e.ok; ++k) {
    x = 2.f * x;
    c2p_eval(c, P.gm1g, x, e);
  }
  if (!e.ok) return false;
  int final_step = 0;
  for (int it = 1; it <= P.c2p_maxit; ++it) {
    float dx = -e.f / e.df;
    C2PPt<float> en;
    c2p_eval(c, P.gm1g, x + dx, en);
    for (int k = 0; k < 40 && !en.ok; ++k) {
      dx = 0.5f * dx;
      c2p_eval(c, P.gm1g, x + dx, en);
    }
    if (!en.ok) return false;
    x = x + dx;
    e = en;
    if (final_step) {
      x_out = x;
      return e.p > 0.f;
    }
    if (fabsf(dx) <= 1e-5f * x) final_step = 1;
  }
  return false;
}

// ------------------------------------------------------------- reconstruction
__device__ __forceinline__ float limiter(int recon, float dL, float dR) {
  if (recon == 0) return 0.f;
  if (!(dL * dR > 0.f)) return 0.f;
  if (recon == 1) return fabsf(dL) < fabsf(dR) ? dL : dR;
  if (recon == 2) {
    const float m = fminf(fminf(2.f * fabsf(dL), 2.f * fabsf(dR)), fabsf(0.5f * (dL + dR)));
    return dL > 0.f ? m : -m;
  }
  return (2.f * dL * dR) / (dL + dR);
}

__device__ __forceinline__ void reconstruct(int recon, const float* w0, const float* w1,
                                            const float* w2, float* vm, float* vp) {
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const float s = limiter(recon, w1[k] - w0[k], w2[k] - w1[k]);
    vp[k] = w1[k] + 0.5f * s;
    vm[k] = w1[k] - 0.5f * s;
  }
  const bool bad = !(vm[1] * vm[1] + vm[2] * vm[2] + vm[3] * vm[3] < 1.f) ||
                   vm[9] * vm[9] + vm[10] * vm[10] + vm[11] * vm[11] > vm[8] * vm[8] ||
                   !(vp[1] * vp[1] + vp[2] * vp[2] + vp[3] * vp[3] < 1.f) ||
                   vp[9] * vp[9] + vp[10] * vp[10] + vp[11] * vp[11] > vp[8] * vp[8];
  if (bad) {
#pragma unroll
    for (int k = 0; k < NV; ++k) vp[k] = vm[k] = w1[k];
  }
}

// ------------------------------------------------------------- PVM-int-8, tangent products
// A w at U_m: the con2prim root x_m of U_m (derivative fx there) is differentiated
// by the implicit-function theorem, then V and F are evaluated in dual numbers.
__device__ __forceinline__ bool a_product(const P32& P, int d, const float* Um, float xm, float fx,
                                          const float* w, float* out) {
  Dual U[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) U[k] = mk(Um[k], w[k]);
  const C2PIn<Dual> c = c2p_in(U);
  C2PPt<Dual> e;
  c2p_eval(c, P.gm1g, mk(xm), e);
  if (!e.ok) return false;
  const float dx = -e.f.d / fx;
  c2p_eval(c, P.gm1g, mk(xm, dx), e);
  if (!e.ok) return false;
  Dual V[NV], F[NV];
  c2p_recover(c, e, U, V);
  flux(P, d, V, U, F);
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = F[k].d;
  return true;
}

// F^ = (F_L + F_R)/2 - beta p_3(A(U_m)) (U_R - U_L)/2 (Eqs. generalflux, iterat, beta)
// with the same Horner order in A^2 as the FP64 path; Q = I if U_m has no FP32 root.
__device__ __forceinline__ int pvm_flux(const P32& P, int d, const float* VL, const float* VR,
                                        float tauL, float tauR, float* Fhat) {
  const float alpha[5] = {-1.f / 128.f, 3.f / 32.f, -23.f / 64.f, 31.f / 32.f, 39.f / 128.f};
  float U0[NV], Um[NV];
  float Zg;
  {
    float UL[NV], UR[NV], FL[NV], FR[NV];
    prim2con(P, VL, UL);
    prim2con(P, VR, UR);
    flux(P, d, VL, UL, FL);
    flux(P, d, VR, UR, FR);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      U0[k] = UR[k] - UL[k];
      Um[k] = 0.5f * (UL[k] + UR[k]);
      Fhat[k] = 0.5f * (FL[k] + FR[k]);
    }
    Zg = 0.5f * (prim_Z(P, VL) + prim_Z(P, VR));
  }
  float beta = 1.f;
  if (P.beta_mode) beta = 1.f / fmaxf(fmaxf(tauL, tauR), 1.f);
  float Ul[NV];
  int fail = 1;
  const C2PIn<float> cm = c2p_in(Um);
  float xm;
  C2PPt<float> em;
  if (c2p_solve(P, cm, Zg, xm, em)) {
    fail = 0;
#pragma unroll
    for (int k = 0; k < NV; ++k) Ul[k] = U0[k];
    for (int l = 0; l < 4 && !fail; ++l) {
      float Y1[NV], Y[NV];
      if (!a_product(P, d, Um, xm, em.df, Ul, Y1) || !a_product(P, d, Um, xm, em.df, Y1, Y)) {
        fail = 1;
        break;
      }
      const float a0 = (l == 0) ? alpha[0] : 1.f;
      const float a1 = alpha[l + 1];
#pragma unroll
      for (int k = 0; k < NV; ++k) Ul[k] = a0 * Y[k] + a1 * U0[k];
    }
  }
  if (fail) {
#pragma unroll
    for (int k = 0; k < NV; ++k) Ul[k] = U0[k];
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) Fhat[k] -= 0.5f * (beta * Ul[k]);
  return fail;
}

__device__ __forceinline__ void llf_flux(const P32& P, int d, const float* VL, const float* VR,
                                         float* Fhat) {
  float UL[NV], UR[NV], FL[NV], FR[NV];
  prim2con(P, VL, UL);
  prim2con(P, VR, UR);
  flux(P, d, VL, UL, FL);
  flux(P, d, VR, UR, FR);
#pragma unroll
  for (int k = 0; k < NV; ++k) Fhat[k] = 0.5f * (FL[k] + FR[k]) - 0.5f * (UR[k] - UL[k]);
}

}  // namespace rr32
