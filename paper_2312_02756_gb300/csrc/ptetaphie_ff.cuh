// Pair mass of PtEtaPhiE legs in float-float (the fast path of the PtEtaPhiE mass kernel; the
// mass of Sec. 4.1 on the (pt, eta, phi, E) system of Sec. 3.1).
//
// The PtEtaPhiM identity of mass_ff.cuh holds for any q_i = E_i^2 - P_i^2 (P_i = pt_i cosh eta_i):
//   m^2 = q1 + q2 + 2 (q1 E2^2 + q2 P1^2) / (E1 E2 + P1 P2) + 4 pt1 pt2 (sinh^2(d_eta/2) + sin^2(d_phi/2)),
// because E1^2 E2^2 - P1^2 P2^2 = q1 E2^2 + q2 P1^2 + q1 q2 with E_i^2 = P_i^2 + q_i.  Here E_i is
// stored, so q_i is the difference E_i^2 - P_i^2 of a stored number and a computed one: in
// float-float its absolute error is ~2^-47 E_i^2, and the result is accurate normwise, within
// 2^-40 (M1 + M2)^2 in m|m| with M_i = max(E_i, P_i) -- the contract of the PtEtaPhiE masses.
// The legs are the LegFF of mass_ff.cuh (pt, P, q, E^2 at the pair's power-of-two scale) and the
// pair arithmetic is pair_m2_ff itself.  Outside the domain (the PtEtaPhiM one with E in the
// place of m, and E >= 0), and for a pair whose m^2 falls below 2^-80 of the scale (spacelike
// sums included), the functions return false and the caller takes the FP64 route.
#pragma once

#include "mass_ff.cuh"
#include "mass_ff2.cuh"

namespace gvx {
namespace ffm {

// One PtEtaPhiE leg at the scale 2^-s: pt, P = pt cosh(eta), q = E^2 - P^2, E^2.
GVX_HD LegFF make_leg_e_ff(double pt, double eta, double E, int s, const TabRef &T) {
  LegFF l;
  l.pt = from_double_ranged(pt, s);
  l.E2 = sqr(from_double_ranged(E, s));
  l.P = mul(l.pt, cosh_t(from_double_ranged(eta, 0), T));  // |eta| < 16
  l.q = add(l.E2, neg(sqr(l.P)));
  return l;
}

GVX_HD bool pair_mass_e_ff(double pt1, double eta1, double phi1, double E1, double pt2,
                           double eta2, double phi2, double E2, const TabRef &T, double *out) {
  if ((dhi(E1) | dhi(E2)) >> 31) return false;  // a negative (or -0) energy
  int s;
  if (!mass_ff_domain(pt1, eta1, phi1, E1, pt2, eta2, phi2, E2, &s)) return false;
  bool ok = true;
  const LegFF a = make_leg_e_ff(pt1, eta1, E1, s, T);
  const LegFF b = make_leg_e_ff(pt2, eta2, E2, s, T);
  return finish_mass(pair_m2_ff(a, b, eta1, eta2, phi1, phi2, T, &ok), s, ok, out);
}

// add of ff.cuh per lane (accurate under cancellation)
GVX_HD ff2 add(const ff2 &x, const ff2 &y) {
  ff2 s = two_sum2(x.hi, y.hi);
  const ff2 t = two_sum2(x.lo, y.lo);
  s = fast_two_sum2(s.hi, add2(s.lo, t.hi));
  return fast_two_sum2(s.hi, add2(s.lo, t.lo));
}

// pair_mass_e_ff with both legs (make_leg_e_ff) in one sequence of paired FP32 operations
// (mass_ff2.cuh; lane x leg 1, lane y leg 2): the same bits, the same domain.
GVX_HD bool pair_mass_e_ff_lp(double pt1, double eta1, double phi1, double e1, double pt2,
                              double eta2, double phi2, double e2, const TabRef &T, double *out) {
  if ((dhi(e1) | dhi(e2)) >> 31) return false;  // a negative (or -0) energy
  int s;
  if (!mass_ff_domain(pt1, eta1, phi1, e1, pt2, eta2, phi2, e2, &s)) return false;
  const ff2 pt = pack(from_double_ranged(pt1, s), from_double_ranged(pt2, s));
  const ff2 E2 = sqr(pack(from_double_ranged(e1, s), from_double_ranged(e2, s)));
  const ff2 eta = pack(from_double_ranged(eta1, 0), from_double_ranged(eta2, 0));
  const ff2 P = mul(pt, cosh_t(eta, T));
  const ff2 q = add(E2, neg(sqr(P)));
  const LegFF a{lane_x(pt), lane_x(P), lane_x(q), lane_x(E2)};
  const LegFF b{lane_y(pt), lane_y(P), lane_y(q), lane_y(E2)};
  bool ok = true;
  const ff m2s = pair_m2_ff(a, b, eta1, eta2, phi1, phi2, T, &ok);
  return finish_mass(m2s, s, ok, out);
}

}  // namespace ffm
}  // namespace gvx
