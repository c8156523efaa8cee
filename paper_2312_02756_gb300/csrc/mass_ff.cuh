// Pair mass in float-float (the FP64 invariant-mass kernels' fast path).
//
// Same identity as pair_math.cuh (all terms non-negative), evaluated in ff on the FP32 pipe:
//   m^2 = m1^2 + m2^2 + 2 (m1^2 E2^2 + m2^2 P1^2) / (E1 E2 + P1 P2)
//             + 4 pt1 pt2 (sinh^2(d_eta/2) + sin^2(d_phi/2)),
// with E1 E2 = sqrt((P1^2 + m1^2)(P2^2 + m2^2)) (one square root).  d_eta and d_phi are formed
// exactly from the doubles (ffm::diff), and for |d_phi| > pi the half-angle is taken from
// y = (pi - |phi1|) + (pi - |phi2|), whose brackets are exact differences too.
//
// Domain of the fast path (anything else returns false and the caller uses the FP64 path):
// finite inputs, pt >= 0, |eta| < 16, |phi| <= pi (rounded to double), and pt and m, scaled by
// the power of two 2^-s that brings the largest of them into [1, 2), either 0 or >= 2^-30; the
// scaled m^2 must come out >= 2^-80 (or exactly 0).  Over that domain every intermediate that
// matters stays inside the normal float range (E^2 <= 2^47, products >= 2^-120), and anything
// flushed to zero is below 2^-46 of the result.
#pragma once

#include "ff.cuh"

namespace gvx {
namespace ffm {

constexpr uint64_t kPiBits = 0x400921FB54442D18ull;  // pi rounded to double (below pi)
constexpr float kTwoPiLo = 2.4492935982947064e-16f;   // 2 (pi - that double)

// Leg data in ff: pt and m scaled by 2^-s; P = pt cosh(eta); q = m^2; E2 = P^2 + q.
struct LegFF {
  ff pt, q, P, P2, E2;
};

GVX_HD LegFF leg_ff(double pt, double eta, double m, int s, const Tables &T, bool *ok) {
  LegFF l;
  l.pt = from_double(pt, ok, s);
  ff mf = from_double(m, ok, s);
  ff ch = cosh(from_double(eta, ok), T);
  l.q = sqr(mf);
  l.P = mul(l.pt, ch);
  l.P2 = sqr(l.P);
  l.E2 = add_same(l.P2, l.q);
  return l;
}

// Half of the azimuthal difference reduced to [0, pi/2], for sin^2 of it.
GVX_HD ff half_dphi_ff(double phi1, double phi2, const Tables &T, bool *ok) {
  ff d = diff(phi1, phi2, ok);
  if (d.hi < 0.0f) d = neg(d);
  bool wrap = d.hi > T.pi.hi || (d.hi == T.pi.hi && d.lo > T.pi.lo);
  if (wrap) {
    // 2 pi - |d| = (pi_d - |phi1|) + (pi_d - |phi2|) + 2 (pi - pi_d)
    const double pid = u2d(kPiBits);
    double a1 = u2d(d2u(phi1) & 0x7fffffffffffffffull), a2 = u2d(d2u(phi2) & 0x7fffffffffffffffull);
    d = add_same(diff(pid, a1, ok), diff(pid, a2, ok));
    d = add_same_f(d, kTwoPiLo);
  }
  return scale(d, 0.5f);
}

// Fast-path domain test on the raw bits; s receives the scaling exponent.
GVX_HD bool mass_ff_domain(double pt1, double eta1, double phi1, double m1, double pt2, double eta2,
                           double phi2, double m2, int *s) {
  const uint64_t mag = 0x7fffffffffffffffull;
  uint64_t upt1 = d2u(pt1), upt2 = d2u(pt2);
  if ((upt1 | upt2) >> 63) return false;  // pt < 0 (or -0: handled by the FP64 path)
  // |eta| < 16: biased exponent <= 1026
  if (((d2u(eta1) & mag) >> 52) > 1026 || ((d2u(eta2) & mag) >> 52) > 1026) return false;
  if ((d2u(phi1) & mag) > kPiBits || (d2u(phi2) & mag) > kPiBits) return false;
  int e1 = dexp(pt1), e2 = dexp(pt2), e3 = dexp(m1), e4 = dexp(m2);
  int emax = e1 > e2 ? e1 : e2;
  emax = emax > e3 ? emax : e3;
  emax = emax > e4 ? emax : e4;
  if (emax == 0 || emax >= 0x7ff) return false;  // all zero, or Inf/NaN
  // every nonzero scaled magnitude >= 2^-30
  if ((e1 && emax - e1 > 30) || (e2 && emax - e2 > 30) || (e3 && emax - e3 > 30) ||
      (e4 && emax - e4 > 30))
    return false;
  *s = emax - 1023;
  return true;
}

// Returns false (and leaves *out untouched) outside the fast-path domain.
GVX_HD bool pair_mass_ff(double pt1, double eta1, double phi1, double m1, double pt2, double eta2,
                         double phi2, double m2, const Tables &T, double *out) {
  int s;
  if (!mass_ff_domain(pt1, eta1, phi1, m1, pt2, eta2, phi2, m2, &s)) return false;
  bool ok = true;
  LegFF a = leg_ff(pt1, eta1, m1, s, T, &ok);
  LegFF b = leg_ff(pt2, eta2, m2, s, T, &ok);
  // 2 (E1 E2 - P1 P2) = 2 (m1^2 E2^2 + m2^2 P1^2) / (E1 E2 + P1 P2)
  ff den = add_same(sqrt(mul(a.E2, b.E2)), mul(a.P, b.P));
  ff num = add_same(mul(a.q, b.E2), mul(b.q, a.P2));
  ff tm = den.hi > 0.0f ? scale(div(num, den), 2.0f) : make(0.0f);
  // 4 pt1 pt2 (sinh^2(d_eta/2) + sin^2(d_phi/2))
  ff se = sinh(scale(diff(eta1, eta2, &ok), 0.5f), T);
  ff sp = sin_q1(half_dphi_ff(phi1, phi2, T, &ok), T);
  ff ta = scale(mul(mul(a.pt, b.pt), add_same(sqr(se), sqr(sp))), 4.0f);
  ff m2s = add_same(add_same(add_same(a.q, b.q), tm), ta);
  if (!ok || (m2s.hi < 8.27180613e-25f && m2s.hi != 0.0f)) return false;  // 2^-80
  *out = to_double(sqrt(m2s), s);
  return true;
}

}  // namespace ffm
}  // namespace gvx
