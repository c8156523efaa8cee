// The legs of the float-float pair mass (mass_ff.cuh) on Blackwell's paired FP32 instructions
// (ff2.cuh).  Lane x carries leg 1 of a pair, lane y leg 2:
// pt, m^2, P = pt cosh(eta) and E^2 = P^2 + m^2 of both legs -- the table-driven cosh included --
// run as one paired sequence, which repeats the scalar operations of ff.cuh, ff_tables.cuh and
// make_leg_ff step for step, so each lane holds the scalar leg's bits (negations and subtractions
// are exact paired multiplies and FMAs: x - y = fma(y, -1, x)).  The pair arithmetic that follows
// is the scalar pair_m2_ff.  The integer parts -- the conversions from double and the table
// indices -- stay per lane.
//
// Pairing stops at the legs because packing values from different registers into a lane pair
// costs moves: pairing the pair-level steps too (or two whole pairs per thread) executed fewer
// instructions but ran slower on GB300 (more moves, or more registers and fewer resident warps).
#pragma once

#include "ff2.cuh"
#include "mass_ff.cuh"

namespace gvx {
namespace ffm {

// round_shift per lane: the integer n of each lane; returns nf.
GVX_HD f2 round_shift2(f2 x, int *nx, int *ny) {
  const f2 t = add2(x, bc2(12582912.0f));
  *nx = (int32_t)(f2u(t.x) - 0x4B400000u);
  *ny = (int32_t)(f2u(t.y) - 0x4B400000u);
  return sub2(t, bc2(12582912.0f));
}
GVX_HD ff2 reduce2(const ff2 &x, f2 nf, float c0, float c1, float c2) {
  const f2 r1 = fma2(nf, bc2(-c0), x.hi);  // -nf c0 + x.hi
  const ff2 p = two_prod2(nf, bc2(c1));
  const ff2 s = two_sum2(r1, neg2(p.hi));
  return two_sum2(s.hi, add2(sub2(s.lo, p.lo), sub2(x.lo, mul2(nf, bc2(c2)))));
}

struct HypParts2 {
  ff2 E, O;
  int jx, jy, kx, ky;
};
GVX_HD HypParts2 hyp_parts2(const ff2 &x, float inv_c, float c0, float c1, float c2) {
  HypParts2 h;
  int nx, ny;
  const f2 nf = round_shift2(mul2(x.hi, bc2(inv_c)), &nx, &ny);
  const ff2 r = reduce2(x, nf, c0, c1, c2);
  const f2 t = fma2(r.hi, r.hi, mul2(add2(r.hi, r.hi), r.lo));
  h.E = fast_two_sum2(bc2(1.0f), mul2(t, bc2(0.5f)));
  const ff2 o = two_sum2(r.hi, mul2(mul2(r.hi, t), bc2(0.16666667f)));
  h.O = {o.hi, add2(o.lo, r.lo)};
  h.jx = nx & 1023;
  h.kx = nx >> 10;
  h.jy = ny & 1023;
  h.ky = ny >> 10;
  return h;
}
GVX_HD ff2 add_eo(const ff2 &E, const ff2 &O) {
  const ff2 s = fast_two_sum2(E.hi, O.hi);
  return {s.hi, add2(s.lo, add2(E.lo, O.lo))};
}

// cosh per lane (cosh_t of ff_tables.cuh); |x| < 16.
GVX_HD ff2 cosh_t(const ff2 &xin, const TabRef &T) {
  const f2 sg = mk2(xin.hi.x < 0.0f ? -1.0f : 1.0f, xin.hi.y < 0.0f ? -1.0f : 1.0f);
  const ff2 x = {mul2(xin.hi, sg), mul2(xin.lo, sg)};  // |x|
  const HypParts2 h = hyp_parts2(x, kExpInvC, kExpC0, kExpC1, kExpC2);
  const gvx_f4 tx = T.exp[h.jx], ty = T.exp[h.jy];
  ff2 tp = fast_two_sum2(bc2(1.0f), mk2(tx.x, ty.x));
  tp.lo = add2(tp.lo, mk2(tx.y, ty.y));
  ff2 tn = fast_two_sum2(bc2(1.0f), mk2(-tx.z, -ty.z));
  tn.lo = sub2(tn.lo, mk2(tx.w, ty.w));
  const ff2 ep = scale(mul(tp, add_eo(h.E, h.O)), mk2(pow2f(h.kx - 1), pow2f(h.ky - 1)));
  const ff2 en = scale(mul(tn, add_eo(h.E, neg(h.O))), mk2(pow2f(-h.kx - 1), pow2f(-h.ky - 1)));
  return add_same(ep, en);
}

// pair_mass_ff with both legs (make_leg_ff) in one paired sequence: the same bits, the same
// domain; false outside the fast-path domain.
GVX_HD bool pair_mass_ff_lp(double pt1, double eta1, double phi1, double m1, double pt2,
                            double eta2, double phi2, double m2, const TabRef &T, double *out) {
  int s;
  if (!mass_ff_domain(pt1, eta1, phi1, m1, pt2, eta2, phi2, m2, &s)) return false;
  const ff2 eta = pack(from_double_ranged(eta1, 0), from_double_ranged(eta2, 0));
  const ff2 pt = pack(from_double_ranged(pt1, s), from_double_ranged(pt2, s));
  const ff2 q = sqr(pack(from_double_ranged(m1, s), from_double_ranged(m2, s)));
  const ff2 P = mul(pt, cosh_t(eta, T));
  const ff2 E2 = add_same(sqr(P), q);
  const LegFF a{lane_x(pt), lane_x(P), lane_x(q), lane_x(E2)};
  const LegFF b{lane_y(pt), lane_y(P), lane_y(q), lane_y(E2)};
  bool ok = true;
  const ff m2s = pair_m2_ff(a, b, eta1, eta2, phi1, phi2, T, &ok);
  return finish_mass(m2s, s, ok, out);
}

}  // namespace ffm
}  // namespace gvx
