// The legs of the float-float pair-mass gradient (leg_grad_prep of mass_ff.cuh) on paired FP32
// instructions, lane x leg 1, lane y leg 2, as mass_ff2.cuh does for the pair mass: pt, m, m^2,
// sinh(eta) and cosh(eta) from the tables, P, E^2 and E = sqrt(E^2) of both legs in one
// sequence that repeats the scalar operations step for step (the same bits per lane).  The
// pair part (pair_grad_legs) stays scalar.
#pragma once

#include "mass_ff2.cuh"

namespace gvx {
namespace ffm {

// sinh and cosh per lane (sinhcosh_t of ff_tables.cuh); |x| < 16.
GVX_HD void sinhcosh_t(const ff2 &xin, const TabRef &T, ff2 *sh, ff2 *ch) {
  const f2 sg = mk2(xin.hi.x < 0.0f ? -1.0f : 1.0f, xin.hi.y < 0.0f ? -1.0f : 1.0f);
  const ff2 x = {mul2(xin.hi, sg), mul2(xin.lo, sg)};  // |x|
  const HypParts2 h = hyp_parts2(x, kExpInvC, kExpC0, kExpC1, kExpC2);
  const gvx_f4 tx = T.exp[h.jx], ty = T.exp[h.jy];
  const f2 pk = mk2(pow2f(h.kx), pow2f(h.ky)), mk = mk2(pow2f(-h.kx), pow2f(-h.ky));
  const ff2 a = {mul2(mk2(tx.x, ty.x), pk), mul2(mk2(tx.y, ty.y), pk)};
  const ff2 b = {mul2(mk2(tx.z, ty.z), mk), mul2(mk2(tx.w, ty.w), mk)};
  const ff2 S = scale(add_same(add_same(fast_two_sum2(pk, neg2(mk)), a), b), bc2(0.5f));
  ff2 tn = fast_two_sum2(bc2(1.0f), mk2(-tx.z, -ty.z));
  tn.lo = sub2(tn.lo, mk2(tx.w, ty.w));
  const ff2 C = add_same(S, scale(tn, mk));
  const ff2 s = add_same(mul(S, h.E), mul(C, h.O));
  *sh = {mul2(s.hi, sg), mul2(s.lo, sg)};
  *ch = add_same(mul(C, h.E), mul(S, h.O));
}

// sqrt per lane (sqrt of ff.cuh); a lane whose hi is not positive gives 0.
GVX_HD ff2 sqrt(const ff2 &x) {
  const f2 r0 = mk2(frsqrt_approx(x.hi.x), frsqrt_approx(x.hi.y));
  const f2 rs = fma2(mul2(bc2(0.5f), r0), fma2(neg2(x.hi), mul2(r0, r0), bc2(1.0f)), r0);
  const f2 s = mul2(x.hi, rs);
  const ff2 p = two_prod2(s, s);
  const f2 r = add2(sub2(sub2(x.hi, p.hi), p.lo), x.lo);
  ff2 o = fast_two_sum2(s, mul2(mul2(r, rs), bc2(0.5f)));
  if (!(x.hi.x > 0.0f)) o.hi.x = o.lo.x = 0.0f;
  if (!(x.hi.y > 0.0f)) o.hi.y = o.lo.y = 0.0f;
  return o;
}

GVX_HD LegGradFF lane_leg(const ff2 &pt, const ff2 &q, const ff2 &m, const ff2 &P, const ff2 &E2,
                          const ff2 &E, const ff2 &sh, const ff2 &ch, bool y) {
  LegGradFF l;
  l.pt = y ? lane_y(pt) : lane_x(pt);
  l.q = y ? lane_y(q) : lane_x(q);
  l.m = y ? lane_y(m) : lane_x(m);
  l.P = y ? lane_y(P) : lane_x(P);
  l.E2 = y ? lane_y(E2) : lane_x(E2);
  l.E = y ? lane_y(E) : lane_x(E);
  l.sh = y ? lane_y(sh) : lane_x(sh);
  l.ch = y ? lane_y(ch) : lane_x(ch);
  return l;
}

// pair_mass_grad_ff with both legs prepared in one paired sequence: the same bits, the same
// domain; false when the pair leaves the fast path.
GVX_HD bool pair_mass_grad_ff_lp(double pt1, double eta1, double phi1, double m1, double pt2,
                                 double eta2, double phi2, double m2, double gm, const TabRef &T,
                                 double *out) {
  int s;
  if (!mass_ff_domain(pt1, eta1, phi1, m1, pt2, eta2, phi2, m2, &s)) return false;
  bool ok = true;
  const ff2 pt = pack(from_double_ranged(pt1, s), from_double_ranged(pt2, s));
  const ff2 m = pack(from_double_ranged(m1, s), from_double_ranged(m2, s));
  const ff2 q = sqr(m);
  ff2 sh, ch;
  sinhcosh_t(pack(from_double(eta1, &ok), from_double(eta2, &ok)), T, &sh, &ch);
  const ff2 P = mul(pt, ch);
  const ff2 E2 = add_same(sqr(P), q);
  const ff2 E = sqrt(E2);
  const LegGradFF a = lane_leg(pt, q, m, P, E2, E, sh, ch, false);
  const LegGradFF b = lane_leg(pt, q, m, P, E2, E, sh, ch, true);
  return ok && pair_grad_legs(a, b, eta1, eta2, phi1, phi2, gm, s, T, out);
}

}  // namespace ffm
}  // namespace gvx
