// Pair-mass arithmetic (and its adjoint) shared by the elementwise kernels (mass.cu) and the
// jagged-event kernels (jagged.cu, jagged_bwd.cu), so that both give the same bits for the same
// two particles.
//
// GenVectorX (Sec. 4.1, Fig. 1) forms mass((pt1,eta1,phi1,m1) + (pt2,eta2,phi2,m2)).  The plain
// form sqrt(E^2 - |P|^2) cancels catastrophically for light, collinear pairs; this uses
//   m^2 = m1^2 + m2^2 + 2 (m1^2 P2^2 + m2^2 P1^2 + m1^2 m2^2) / (E1 E2 + P1 P2)
//             + 4 pt1 pt2 (sinh^2(d_eta/2) + sin^2(d_phi/2)),
// P_i = pt_i cosh(eta_i) = |p_i|, E_i = sqrt(P_i^2 + m_i^2).  It follows from
//   E1 E2 - P1 P2 = (E1^2 E2^2 - P1^2 P2^2) / (E1 E2 + P1 P2),
//   P1 P2 - p1.p2 = pt1 pt2 (cosh d_eta - cos d_phi) = 2 pt1 pt2 (sinh^2(d_eta/2) + sin^2(d_phi/2)),
// and has only non-negative terms for pt >= 0, so its relative error is a few ulps.
#pragma once

#include "common.cuh"

namespace gvx {

constexpr double kPi = 3.141592653589793116;        // pi rounded to double (below pi)
constexpr double kPiLo = 1.2246467991473531772e-16;  // pi - kPi
constexpr float kPiF = 3.14159274101257324f;         // pi rounded to float (above pi)
constexpr float kPiLoF = -8.74227765734758577e-8f;   // pi - kPiF

// Half of the azimuthal difference, reduced so that sin^2 of it keeps full relative accuracy.
// For canonical angles (|phi| <= pi) with |d_phi| > pi, sin^2(d_phi/2) = sin^2(y/2) with
// y = 2 pi - |d_phi| = (pi - |phi1|) + (pi - |phi2|): each bracket is exact (Sterbenz) or a
// sum of non-negative numbers, so y carries no cancellation error even when it is tiny.
// *sign is set so that sin(d_phi) = *sign * 2 sin(h) cos(h) for the returned h (the wrapped
// half-angle y/2 has sin(d_phi) = -sign(d_phi) sin(y)).
template <typename T>
__device__ __forceinline__ T half_dphi(T phi1, T phi2, T *sign = nullptr) {
  const T pi = sizeof(T) == 8 ? (T)kPi : (T)kPiF;
  const T pi_lo = sizeof(T) == 8 ? (T)kPiLo : (T)kPiLoF;
  T d = phi1 - phi2;
  T a1 = fabs(phi1), a2 = fabs(phi2);
  if (fabs(d) > pi && a1 <= pi && a2 <= pi) {
    if (sign) *sign = d > (T)0 ? (T)-1 : (T)1;
    return (T)0.5 * (((pi - a1) + (pi - a2)) + (T)2 * pi_lo);
  }
  if (sign) *sign = (T)1;
  return (T)0.5 * d;
}

__device__ __forceinline__ double cosh_(double x) { return cosh(x); }
__device__ __forceinline__ float cosh_(float x) { return coshf(x); }
__device__ __forceinline__ double sinh_(double x) { return sinh(x); }
__device__ __forceinline__ float sinh_(float x) { return sinhf(x); }
__device__ __forceinline__ double sin_(double x) { return sin(x); }
__device__ __forceinline__ float sin_(float x) { return sinf(x); }
__device__ __forceinline__ double cos_(double x) { return cos(x); }
__device__ __forceinline__ float cos_(float x) { return cosf(x); }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }

// Per-leg quantities: m as given, q = m^2, P = |p|, E.
template <typename T>
struct Leg {
  T pt, eta, phi, m, q, P, E;
};

template <typename T>
__device__ __forceinline__ Leg<T> make_leg(V4<T> v) {
  Leg<T> l;
  l.pt = v.x;
  l.eta = v.y;
  l.phi = v.z;
  l.m = v.w;
  l.q = v.w * v.w;
  l.P = v.x * cosh_(v.y);
  l.E = sqrt_(fma(l.P, l.P, l.q));
  return l;
}

// Per-pair quantities shared by the forward and the adjoint.
template <typename T>
struct PairTerms {
  T se, sp, S, m2;
};

template <typename T>
__device__ __forceinline__ PairTerms<T> pair_terms(const Leg<T> &a, const Leg<T> &b) {
  PairTerms<T> t;
  T den = fma(a.E, b.E, a.P * b.P);
  T num = fma(a.q, b.P * b.P, fma(b.q, a.P * a.P, a.q * b.q));
  T tm = den > (T)0 ? (T)2 * num / den : (T)0;
  t.se = sinh_((T)0.5 * (a.eta - b.eta));
  t.sp = sin_(half_dphi(a.phi, b.phi));
  t.S = fma(t.se, t.se, t.sp * t.sp);
  T ta = (T)4 * a.pt * b.pt * t.S;
  t.m2 = a.q + b.q + tm + ta;
  return t;
}

// Adjoint of the pair mass.  With S = sinh^2(d_eta/2) + sin^2(d_phi/2) and
//   X = (P1^2 m2^2 - P2^2 m1^2) / ((P1 E2 + P2 E1) E1)      (= P1 E2/E1 - P2, without cancellation)
// the derivatives of m^2 with respect to leg 1 are
//   d/dpt1  = 4 pt2 S + 2 cosh(eta1) X
//   d/deta1 = 2 pt1 (pt2 sinh(d_eta) + sinh(eta1) X)
//   d/dphi1 = 2 pt1 pt2 sin(d_phi)
//   d/dm1   = 2 m1 (E1 + E2) / E1
// and leg 2 follows by exchanging the legs (d_eta, d_phi change sign).  dm = d(m^2) / (2 m);
// where m = 0 the gradient is 0.  A massless leg has E = pt cosh(eta), and at pt = 0 its
// one-sided (pt >= 0) derivatives are used: X -> m_o^2 / (E_o + P_o), d/dm = 0.
template <typename T>
__device__ __forceinline__ V4<T> leg_grad(const Leg<T> &s, const Leg<T> &o, T S, T sdeta, T sdphi,
                                          T scale) {
  // X = P_s E_o / E_s - P_o.  Its denominator vanishes (with E_s > 0) only when P_o = 0 and
  // either E_o = 0 (the other leg is the zero vector) or P_s = 0 (both legs at rest); X = 0 there.
  T X;
  if (s.E > (T)0) {
    T den = (s.P * o.E + o.P * s.E) * s.E;
    X = den > (T)0 ? (s.P * s.P * o.q - o.P * o.P * s.q) / den : (T)0;
  } else {
    X = (o.E + o.P) > (T)0 ? o.q / (o.E + o.P) : (T)0;
  }
  T ch = cosh_(s.eta), sh = sinh_(s.eta);
  V4<T> g;
  g.x = scale * ((T)4 * o.pt * S + (T)2 * ch * X);
  g.y = scale * ((T)2 * s.pt * (o.pt * sdeta + sh * X));
  g.z = scale * ((T)2 * s.pt * o.pt * sdphi);
  g.w = s.E > (T)0 ? scale * ((T)2 * s.m * (s.E + o.E) / s.E) : (T)0;
  return g;
}

// g * dm/d(pt, eta, phi, m) of leg a (g1) and leg b (g2), in the working precision T.
template <typename T>
__device__ __forceinline__ void pair_mass_grad(V4<T> x, V4<T> y, T g, V4<T> &g1, V4<T> &g2) {
  Leg<T> la = make_leg(x), lb = make_leg(y);
  PairTerms<T> t = pair_terms(la, lb);
  T m = sqrt_(t.m2);
  g1 = {0, 0, 0, 0};
  g2 = {0, 0, 0, 0};
  if (m > (T)0) {
    T scale = g / ((T)2 * m);
    // sinh(d_eta) = 2 sinh(d_eta/2) cosh(d_eta/2); sin(d_phi) = 2 sin(d_phi/2) cos(d_phi/2)
    T ce = sqrt_((T)1 + t.se * t.se);
    T sgn;
    T cp = cos_(half_dphi(la.phi, lb.phi, &sgn));
    T sdeta = (T)2 * t.se * ce, sdphi = sgn * (T)2 * t.sp * cp;
    g1 = leg_grad(la, lb, t.S, sdeta, sdphi, scale);
    g2 = leg_grad(lb, la, t.S, -sdeta, -sdphi, scale);
  }
}

}  // namespace gvx
