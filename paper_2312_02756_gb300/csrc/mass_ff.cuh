// Pair mass in float-float (the FP64 invariant-mass kernels' fast path).
//
// Same identity as pair_math.cuh (all terms non-negative), evaluated in ff on the FP32 pipe:
//   m^2 = m1^2 + m2^2 + 2 (m1^2 E2^2 + m2^2 P1^2) / (E1 E2 + P1 P2)
//             + 4 pt1 pt2 (sinh^2(d_eta/2) + sin^2(d_phi/2)),
// with E1 E2 = sqrt((P1^2 + m1^2)(P2^2 + m2^2)) (one square root).  d_eta and d_phi are FP64
// differences (exact where they cancel), and for |d_phi| > pi the half-angle is taken from
// y = (pi - |phi1|) + (pi - |phi2|), whose brackets are exact differences too.  Five FP64
// operations per pair in all (the three differences, the wrap brackets, the final add).
//
// Domain of the fast path (anything else returns false and the caller uses the FP64 path):
// finite inputs, pt >= 0, |eta| < 16, |phi| <= pi (rounded to double), and pt and m, scaled by
// the power of two 2^-s that brings the largest of them into [1, 2), either 0 or >= 2^-30; the
// scaled m^2 must come out >= 2^-80 (or exactly 0).  Over that domain every intermediate that
// matters stays inside the normal float range (E^2 <= 2^47, products >= 2^-120), and anything
// flushed to zero is below 2^-46 of the result.
#pragma once

#include "ff_tables.cuh"

namespace gvx {
namespace ffm {

constexpr uint32_t kPiHiWord = 0x400921FBu;  // pi rounded to double (below pi): 0x400921FB54442D18
constexpr uint32_t kPiLoWord = 0x54442D18u;
constexpr float kTwoPiLo = 2.4492935982947064e-16f;  // 2 (pi - that double)

// |d| <= pi rounded to double, on the bits
GVX_HD bool within_pi(double d) {
  uint32_t h = dhi(d) & 0x7fffffffu;
  return h < kPiHiWord || (h == kPiHiWord && dlo(d) <= kPiLoWord);
}

// Fast-path domain test on the raw bits; s receives the scaling exponent.
GVX_HD bool mass_ff_domain(double pt1, double eta1, double phi1, double m1, double pt2, double eta2,
                           double phi2, double m2, int *s) {
  if ((dhi(pt1) | dhi(pt2)) >> 31) return false;  // pt < 0 (or -0: handled by the FP64 path)
  // |eta| < 16: biased exponent <= 1026
  if (((dhi(eta1) >> 20) & 0x7ffu) > 1026u || ((dhi(eta2) >> 20) & 0x7ffu) > 1026u) return false;
  if (!within_pi(phi1) || !within_pi(phi2)) return false;
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

// Half of the azimuthal difference reduced to [0, pi/2], for sin^2 of it.  d = phi1 - phi2 in
// FP64 is exact where it can cancel (Sterbenz); for |d| > pi the half-angle comes from
// y = (pi_d - |phi1|) + (pi_d - |phi2|) + 2 (pi - pi_d), whose brackets are exact FP64
// differences (|phi| >= pi/2 there) or sums without cancellation.
GVX_HD ff half_dphi_ff(double phi1, double phi2, bool *ok) {
  double d = phi1 - phi2;
  if (within_pi(d)) return scale(from_double(fabs(d), ok), 0.5f);
  const double pid = hilo2d(kPiHiWord, kPiLoWord);
  ff y = add_same(from_double(pid - fabs(phi1), ok), from_double(pid - fabs(phi2), ok));
  y = add_small(y, make(kTwoPiLo));
  return scale(y, 0.5f);
}

// Returns false (and leaves *out untouched) outside the fast-path domain.
GVX_HD bool pair_mass_ff(double pt1, double eta1, double phi1, double m1, double pt2, double eta2,
                         double phi2, double m2, const TabRef &T, double *out) {
  int s;
  if (!mass_ff_domain(pt1, eta1, phi1, m1, pt2, eta2, phi2, m2, &s)) return false;
  bool ok = true;
  ff pa = from_double(pt1, &ok, s), pb = from_double(pt2, &ok, s);
  ff qa = sqr(from_double(m1, &ok, s)), qb = sqr(from_double(m2, &ok, s));
  ff Pa = mul(pa, cosh_t(from_double(eta1, &ok), T));
  ff Pb = mul(pb, cosh_t(from_double(eta2, &ok), T));
  ff P2a = sqr(Pa), P2b = sqr(Pb);
  ff E2a = add_same(P2a, qa), E2b = add_same(P2b, qb);
  // 2 (E1 E2 - P1 P2) = 2 (m1^2 E2^2 + m2^2 P1^2) / (E1 E2 + P1 P2)
  ff den = add_same(sqrt(mul(E2a, E2b)), mul(Pa, Pb));
  ff num = add_same(mul(qa, E2b), mul(qb, P2a));
  ff tm = den.hi > 0.0f ? scale(div(num, den), 2.0f) : make(0.0f);
  // 4 pt1 pt2 (sinh^2(d_eta/2) + sin^2(d_phi/2)); d_eta in FP64 is exact where it cancels
  ff se = sinh_t(scale(from_double(eta1 - eta2, &ok), 0.5f), T);
  ff sp = sin_t(half_dphi_ff(phi1, phi2, &ok), T);
  ff ta = scale(mul(mul(pa, pb), add_same(sqr(se), sqr(sp))), 4.0f);
  ff m2s = renorm(add_same(add_same(add_same(qa, qb), tm), ta));
  if (!ok || (m2s.hi < 8.27180613e-25f && m2s.hi != 0.0f)) return false;  // 2^-80
  *out = to_double(sqrt(m2s), s);
  return true;
}

}  // namespace ffm
}  // namespace gvx
