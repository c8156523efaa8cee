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
// the power of two 2^-s that brings the largest of them into [1, 2), either 0 or >= 2^-30 (the
// largest above 2^-993, so no denormal passes); the scaled m^2 must come out >= 2^-80 (or
// exactly 0).  Over that domain every intermediate that
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

// Exponent used to scale a leg: the larger biased exponent of pt and m (0 when both are 0).
GVX_HD int leg_exponent(double pt, double m) {
  int e1 = dexp(pt), e3 = dexp(m);
  return e1 > e3 ? e1 : e3;
}

// Whether a scale exponent (biased) admits the fast path: not all zero, finite, and large enough
// (> 2^-993) that a nonzero denormal pt or m always fails the 2^-30 test below.
GVX_HD bool scale_exponent_ok(int emax) { return emax > 30 && emax < 0x7ff; }

// Whether one leg is inside the fast-path domain for the scale exponent emax (biased, passing
// scale_exponent_ok).  pt and m are then 0 or scaled into [2^-30, 2), so they convert to ff with
// from_double_ranged.
GVX_HD bool leg_in_domain(double pt, double eta, double phi, double m, int emax) {
  if (dhi(pt) >> 31) return false;                              // pt < 0 (or -0)
  if (((dhi(eta) >> 20) & 0x7ffu) > 1026u) return false;        // |eta| >= 16, NaN, Inf
  if (!within_pi(phi)) return false;                            // |phi| > pi, NaN
  int ep = dexp(pt), em = dexp(m);
  if (ep >= 0x7ff || em >= 0x7ff) return false;                 // Inf/NaN
  const bool pt_nz = (dhi(pt) | dlo(pt)) != 0u;
  const bool m_nz = ((dhi(m) & 0x7fffffffu) | dlo(m)) != 0u;
  if ((pt_nz && emax - ep > 30) || (m_nz && emax - em > 30)) return false;
  return true;
}

// Fast-path domain test on the raw bits; s receives the scaling exponent.
GVX_HD bool mass_ff_domain(double pt1, double eta1, double phi1, double m1, double pt2, double eta2,
                           double phi2, double m2, int *s) {
  int ea = leg_exponent(pt1, m1), eb = leg_exponent(pt2, m2);
  int emax = ea > eb ? ea : eb;
  if (!scale_exponent_ok(emax)) return false;  // all zero, tiny, or Inf/NaN
  if (!leg_in_domain(pt1, eta1, phi1, m1, emax) || !leg_in_domain(pt2, eta2, phi2, m2, emax))
    return false;
  *s = emax - 1023;
  return true;
}

// Half of the azimuthal difference reduced to [0, pi/2], for sin^2 of it.  d = phi1 - phi2 in
// FP64 is exact where it can cancel (Sterbenz); for |d| > pi the half-angle comes from
// y = (pi_d - |phi1|) + (pi_d - |phi2|) + 2 (pi - pi_d), whose brackets are exact FP64
// differences (|phi| >= pi/2 there) and whose sum has no cancellation.  Both candidates are
// formed and one is selected (no divergent branch); *wrapped tells which.
GVX_HD ff half_dphi_ff(double phi1, double phi2, bool *ok, bool *wrapped = nullptr) {
  const double d = fabs(phi1 - phi2);
  const double pid = hilo2d(kPiHiWord, kPiLoWord);
  const double y = (pid - fabs(phi1)) + (pid - fabs(phi2));
  const bool w = !within_pi(d);
  if (wrapped) *wrapped = w;
  ff h = from_double_ranged(w ? y : d, 0);  // 0 <= d, y <= 2 pi; below 2^-74 counts as 0
  h = add_small(h, make(w ? kTwoPiLo : 0.0f));
  return scale(h, 0.5f);
}

// One leg in ff, pt and m scaled by 2^-s: pt, P = pt cosh(eta), q = m^2, E2 = P^2 + q.
struct LegFF {
  ff pt, P, q, E2;
};

GVX_HD LegFF make_leg_ff(double pt, double eta, double m, int s, const TabRef &T, bool *ok) {
  LegFF l;
  l.pt = from_double_ranged(pt, s);
  l.q = sqr(from_double_ranged(m, s));
  l.P = mul(l.pt, cosh_t(from_double_ranged(eta, 0), T));  // |eta| < 16
  l.E2 = add_same(sqr(l.P), l.q);
  return l;
}

// Scaled m^2 of a pair of legs (renormalized).  eta and phi are the legs' unscaled angles.
GVX_HD ff pair_m2_ff(const LegFF &a, const LegFF &b, double eta1, double eta2, double phi1,
                     double phi2, const TabRef &T, bool *ok) {
  // 2 (E1 E2 - P1 P2) = 2 (m1^2 E2^2 + m2^2 P1^2) / (E1 E2 + P1 P2)
  ff den = add_same(sqrt(mul(a.E2, b.E2)), mul(a.P, b.P));
  ff num = add_same(mul(a.q, b.E2), mul(b.q, sqr(a.P)));
  ff tm = den.hi > 0.0f ? scale(div(num, den), 2.0f) : make(0.0f);
  // 4 pt1 pt2 (sinh^2(d_eta/2) + sin^2(d_phi/2)); d_eta in FP64 is exact where it cancels
  ff se = sinh_t(scale(from_double_ranged(eta1 - eta2, 0), 0.5f), T);
  ff sp = sin_t(half_dphi_ff(phi1, phi2, ok), T);
  ff ta = scale(mul(mul(a.pt, b.pt), add_same(sqr(se), sqr(sp))), 4.0f);
  return renorm(add_same(add_same(add_same(a.q, b.q), tm), ta));
}

// sqrt of a scaled m^2 as a double; false when m^2 fell below 2^-80 (where flushed terms could
// matter) or an operand left the float range.
GVX_HD bool finish_mass(ff m2s, int s, bool ok, double *out) {
  if (!ok || (m2s.hi < 8.27180613e-25f && m2s.hi != 0.0f)) return false;  // 2^-80
  *out = to_double(sqrt(m2s), s);
  return true;
}

// Returns false (and leaves *out untouched) outside the fast-path domain.
GVX_HD bool pair_mass_ff(double pt1, double eta1, double phi1, double m1, double pt2, double eta2,
                         double phi2, double m2, const TabRef &T, double *out) {
  int s;
  if (!mass_ff_domain(pt1, eta1, phi1, m1, pt2, eta2, phi2, m2, &s)) return false;
  bool ok = true;
  LegFF a = make_leg_ff(pt1, eta1, m1, s, T, &ok);
  LegFF b = make_leg_ff(pt2, eta2, m2, s, T, &ok);
  return finish_mass(pair_m2_ff(a, b, eta1, eta2, phi1, phi2, T, &ok), s, ok, out);
}

// Gradient of the pair mass, gm * dm/d(pt, eta, phi, m) of both legs, in ff.  With the scaled
// legs, S = sinh^2(d_eta/2) + sin^2(d_phi/2) and
//   X_s = (P_s^2 m_o^2 - P_o^2 m_s^2) / ((P_s E_o + P_o E_s) E_s)       (= P_s E_o/E_s - P_o)
// the derivatives of m^2 for leg s (o = the other leg) are
//   d/dpt_s = 4 pt_o S + 2 cosh(eta_s) X_s,      d/deta_s = 2 pt_s (pt_o sinh(d_eta_so) + sinh(eta_s) X_s),
//   d/dphi_s = 2 pt_s pt_o sin(d_phi_so),         d/dm_s = 2 m_s (E_s + E_o) / E_s,
// and dm = d(m^2) / (2 m).  Readings as in the FP64 kernel: zero where m = 0; for a leg with
// E_s = 0 the one-sided limit X_s = m_o^2 / (E_o + P_o); X_s = 0 where its denominator vanishes.
// Returns false outside the fast-path domain (the caller then uses the FP64 evaluation).
struct LegGradFF {
  ff pt, q, m, P, E2, E, sh, ch;
};

GVX_HD LegGradFF leg_grad_prep(double pt, double eta, double m, int s, const TabRef &T, bool *ok) {
  LegGradFF l;
  l.pt = from_double_ranged(pt, s);
  l.m = from_double_ranged(m, s);
  l.q = sqr(l.m);
  sinhcosh_t(from_double(eta, ok), T, &l.sh, &l.ch);
  l.P = mul(l.pt, l.ch);
  l.E2 = add_same(sqr(l.P), l.q);
  l.E = sqrt(l.E2);
  return l;
}

GVX_HD ff leg_x(const LegGradFF &s, const LegGradFF &o) {
  if (s.E.hi > 0.0f) {
    ff den = mul(add_same(mul(s.P, o.E), mul(o.P, s.E)), s.E);
    if (!(den.hi > 0.0f)) return make(0.0f);
    return div(add(mul(sqr(s.P), o.q), neg(mul(sqr(o.P), s.q))), den);
  }
  ff eo = add_same(o.E, o.P);
  return eo.hi > 0.0f ? div(o.q, eo) : make(0.0f);
}

// Pair-level terms of the gradient: c = gm / (2 m) (times 2^s), S, sinh(d_eta), sin(d_phi).
struct PairGradFF {
  ff c, S, sdeta, sdphi;
};

// The pair part of the gradient from two legs prepared at a common scale 2^-s (leg_grad_prep);
// eta and phi are the legs' unscaled angles.  Returns 0 when the pair leaves the fast path (an
// operand outside its range, or m^2 below 2^-80 of the scale), 1 when m = 0 (zero gradient),
// 2 with the terms in *pg.
GVX_HD int pair_grad_terms(const LegGradFF &a, const LegGradFF &b, double eta1, double eta2,
                           double phi1, double phi2, double gm, const TabRef &T, PairGradFF *pg) {
  bool ok = true;
  ff den = add_same(mul(a.E, b.E), mul(a.P, b.P));
  ff num = add_same(mul(a.q, b.E2), mul(b.q, sqr(a.P)));
  ff tm = den.hi > 0.0f ? scale(div(num, den), 2.0f) : make(0.0f);
  ff se, ce;
  sinhcosh_t(scale(from_double(eta1 - eta2, &ok), 0.5f), T, &se, &ce);
  bool wrapped;
  ff sp, cp;
  const double dphi = phi1 - phi2;
  sincos_q1_t(half_dphi_ff(phi1, phi2, &ok, &wrapped), T, &sp, &cp);
  ff S = add_same(sqr(se), sqr(sp));
  ff m2s = renorm(add_same(add_same(add_same(a.q, b.q), tm), scale(mul(mul(a.pt, b.pt), S), 4.0f)));
  if (!ok || (m2s.hi < 8.27180613e-25f && m2s.hi != 0.0f)) return 0;  // 2^-80
  if (!(m2s.hi > 0.0f)) return 1;
  ff g = from_double(gm, &ok);
  if (!ok) return 0;
  pg->c = div(g, scale(sqrt(m2s), 2.0f));  // gm / (2 m), scaled by 2^s
  pg->S = S;
  // sinh(d_eta) = 2 sinh(d_eta/2) cosh(d_eta/2);  sin(d_phi) = +-2 sin(h) cos(h), with the sign
  // of phi1 - phi2 (its sign bit: no FP64 comparison) and reversed for the wrapped half-angle
  pg->sdeta = scale(mul(se, ce), 2.0f);
  pg->sdphi = scale(mul(sp, cp), 2.0f);
  const bool dneg = (dhi(dphi) >> 31) != 0u;
  if (dneg != wrapped) pg->sdphi = neg(pg->sdphi);
  return 2;
}

// gm dm/d(pt, eta, phi, m) of leg x against leg o as ff, before the final scaling: components 0
// and 3 are the values, components 1 and 2 the values times 2^-s.  sde, sdp: sinh(eta_x - eta_o)
// and sin(phi_x - phi_o).
GVX_HD void leg_grad_terms(const LegGradFF &x, const LegGradFF &o, const PairGradFF &pg, ff sde,
                           ff sdp, ff *out) {
  ff X = leg_x(x, o);
  ff d_pt = add(scale(mul(o.pt, pg.S), 4.0f), scale(mul(x.ch, X), 2.0f));
  ff d_eta = scale(mul(x.pt, add(mul(o.pt, sde), mul(x.sh, X))), 2.0f);
  ff d_phi = scale(mul(mul(x.pt, o.pt), sdp), 2.0f);
  ff d_m = x.E.hi > 0.0f ? scale(div(mul(x.m, add_same(x.E, o.E)), x.E), 2.0f) : make(0.0f);
  out[0] = mul(pg.c, d_pt);
  out[1] = mul(pg.c, d_eta);
  out[2] = mul(pg.c, d_phi);
  out[3] = mul(pg.c, d_m);
}

// leg_grad_terms to doubles.
GVX_HD void leg_grad_out(const ff *t, int s, double *out) {
  out[0] = to_double(renorm(t[0]));
  out[1] = to_double(renorm(t[1]), s);
  out[2] = to_double(renorm(t[2]), s);
  out[3] = to_double(renorm(t[3]));
}

// The gradient of both legs from two legs prepared at a common scale 2^-s: leg a into out[0..3],
// leg b into out[4..7].  False when the pair leaves the fast path.
GVX_HD bool pair_grad_legs(const LegGradFF &a, const LegGradFF &b, double eta1, double eta2,
                           double phi1, double phi2, double gm, int s, const TabRef &T,
                           double *out) {
  PairGradFF pg;
  const int r = pair_grad_terms(a, b, eta1, eta2, phi1, phi2, gm, T, &pg);
  if (r == 0) return false;
  if (r == 1) {
    for (int k = 0; k < 8; k++) out[k] = 0.0;
    return true;
  }
  ff t[4];
  leg_grad_terms(a, b, pg, pg.sdeta, pg.sdphi, t);
  leg_grad_out(t, s, out);
  leg_grad_terms(b, a, pg, neg(pg.sdeta), neg(pg.sdphi), t);
  leg_grad_out(t, s, out + 4);
  return true;
}

// out[0..3] leg a (pt, eta, phi, m), out[4..7] leg b.
GVX_HD bool pair_mass_grad_ff(double pt1, double eta1, double phi1, double m1, double pt2,
                              double eta2, double phi2, double m2, double gm, const TabRef &T,
                              double *out) {
  int s;
  if (!mass_ff_domain(pt1, eta1, phi1, m1, pt2, eta2, phi2, m2, &s)) return false;
  bool ok = true;
  LegGradFF a = leg_grad_prep(pt1, eta1, m1, s, T, &ok);
  LegGradFF b = leg_grad_prep(pt2, eta2, m2, s, T, &ok);
  return ok && pair_grad_legs(a, b, eta1, eta2, phi1, phi2, gm, s, T, out);
}

}  // namespace ffm
}  // namespace gvx
