// Adjoint of the FP64 pair mass in light-cone form (the fast path of the FP64 mass_bwd kernel).
//
// With F = m^2 = (D1 + D2)(Y1 + Y2) + 4 pt1 pt2 S (mass_lc.cuh), D = E - P, Y = E + P,
// P_i = pt_i cosh(eta_i), E_i = sqrt(P_i^2 + m_i^2), S = sinh^2(d_eta/2) + sin^2(d_phi/2), the
// derivative of (sum D)(sum Y) is 2 (E1 + E2) dE - 2 (P1 + P2) dP, and for leg i against the
// other leg o
//   G_i = (E1 + E2) P_i / E_i - (P1 + P2) = (D_o Y_i - Y_o D_i) / (2 E_i),
//   dF/dpt_i  = 2 cosh(eta_i) G_i + 4 pt_o S,
//   dF/deta_i = 2 pt_i sinh(eta_i) G_i +- 2 pt1 pt2 sinh(d_eta),
//   dF/dphi_i = +- 2 pt1 pt2 sin(d_phi),
//   dF/dm_i   = 2 (E1 + E2) m_i / E_i,
// (+ for leg 1, - for leg 2; d_eta = eta1 - eta2, d_phi = phi1 - phi2), and dm/dx = dF/dx / (2m).
// sinh(d_eta) and sin(d_phi) are 2 sinh(h) cosh(h) and 2 sin(h) cos(h) of the half-angles that
// the forward already reduces.  The two legs run as the lanes of paired FP32 instructions.
// Where m = 0 the gradient is 0 (m is not differentiable there); with the forward's masses given
// (m_saved) that is where the forward returned 0.
//
// Fast-path domain: the forward's (mass_lc.cuh), and in addition 2^-60 <= |gm| <= 2^60 (or
// gm = 0), and a saved mass either 0 or at least 2^-40 of the pair's scale.  Anything else
// returns false and the caller takes the FP64 formulas.
#pragma once

#include "mass_lc.cuh"

namespace gvx {
namespace ffm {

// x + y of any signs: TwoSum of the leading parts, no renormalization (under cancellation the
// result keeps an absolute error of ~2^-48 of the operands).
template <class F>
GVX_HD F lc_sum(const F &x, const F &y) {
  const auto s = vadd(x.hi, y.hi);
  const auto bb = vsub(s, x.hi);
  const auto e = vadd(vsub(x.hi, vsub(s, bb)), vsub(y.hi, bb));
  return {s, vadd(e, vadd(x.lo, y.lo))};
}

GVX_HD float sign_of(double d) { return (dhi(d) >> 31) ? -1.0f : 1.0f; }

// The angular terms of a pair for its adjoint: *S = sinh^2(|d_eta|/2) + sin^2(|d_phi|/2) and
// *sd = (2 sinh(d_eta), 2 sin(d_phi)) = 4 (sinh, sin)(cosh, cos) of the half-angles, signed like
// d_eta = eta1 - eta2 and d_phi = phi1 - phi2 (both FP64 differences, as in the forward).  False
// when |d_phi|/2 is within 2^-7 of pi (the caller takes the FP64 formulas).
GVX_HD bool lc_pair_angles(double eta1, double eta2, double phi1, double phi2, const LcTab &T,
                           ff *S, ff2 *sd) {
  const double de = eta1 - eta2, dp = phi1 - phi2;
  const uint32_t hde = dhi(de) & 0x7fffffffu, hdp = dhi(dp) & 0x7fffffffu;
  const CvtParts cp = cvt_parts(hdp, dlo(dp), kRebaseHalf);
  const ff2 xa = cvt2(cvt_parts(hde, dlo(de), kRebaseHalf), cp);
  const int32_t e3 = (int32_t)(cp.hb & 0x7f800000u) - (int32_t)(46u << 23);
  const uint32_t el3 = (uint32_t)(e3 > 0 ? e3 : 0);
  const float lo3 = fsub(u2f(el3 | ((dlo(dp) & 63u) << 17)), u2f(el3));
  uint32_t nj[2];
  ff2 r = lc_reduce(xa, nj);
  r.lo = add2(r.lo, mk2(0.0f, lo3));
  const gvx_f4 th = ldtab(&T.hyp[umin32(nj[0], GVX_HYP_N)]);
  const gvx_f4 ts = ldtab(&T.sin[umin32(nj[1], GVX_SIN_N)]);
  const ff2 A = {mk2(th.z, ts.x), mk2(th.w, ts.y)};    // (sinh, sin) of the table point
  const ff2 B = {mk2(th.x, ts.z), mk2(th.y, ts.w)};    // (cosh, cos)
  const ff2 Bn = {mk2(th.z, -ts.x), mk2(th.w, -ts.y)};  // (sinh, -sin)
  const TabPoly<f2> tp = tab_poly(r, mk2(0.5f, -0.5f));
  const ff2 w = tab_comb(A, B, r, tp);        // (sinh |d_eta|/2, sin |d_phi|/2)
  const ff2 wc = tab_comb_any(B, Bn, r, tp);  // (cosh |d_eta|/2, cos |d_phi|/2)
  const ff2 w2 = lc_sqr(w);
  *S = lc_add(lane_x(w2), lane_y(w2));
  *sd = lc_scale(lc_mul(w, wc), mk2(4.0f * sign_of(de), 4.0f * sign_of(dp)));
  return nj[1] - 802u > 4u;
}

// gm dm/d(pt, eta, phi, m) of both legs: out[0..3] leg 1, out[4..7] leg 2.  has_ms: ms is the
// forward's mass of this pair.  False outside the fast-path domain (out untouched).
GVX_HD bool pair_mass_grad_lc(double pt1, double eta1, double phi1, double m1, double pt2,
                              double eta2, double phi2, double m2, double gm, bool has_ms,
                              double ms, const LcTab &T, double *out) {
  // -- the forward's domain and scale --
  const uint32_t hp1 = dhi(pt1), hp2 = dhi(pt2);
  const uint32_t hm1 = dhi(m1) & 0x7fffffffu, hm2 = dhi(m2) & 0x7fffffffu;
  const uint32_t wmax = umax32(umax32(hp1, hm1), umax32(hp2, hm2));
  const uint32_t ew = wmax & 0x7ff00000u;
  const uint32_t vmin_ = umin32(umin32(hp1 - 0x100000u, hm1 - 0x100000u),
                                umin32(hp2 - 0x100000u, hm2 - 0x100000u));
  const uint32_t he1 = dhi(eta1) & 0x7fffffffu, he2 = dhi(eta2) & 0x7fffffffu;
  const uint32_t hf1 = dhi(phi1) & 0x7fffffffu, hf2 = dhi(phi2) & 0x7fffffffu;
  const uint32_t hg = dhi(gm) & 0x7fffffffu, hms = dhi(ms) & 0x7fffffffu;
  // |gm| in [2^-60, 2^60] or 0 (high-word exponent field 963..1083, or the word 0 of +-0)
  const bool g_ok = hg - (963u << 20) < (121u << 20) || (hg | dlo(gm)) == 0u;
  bool ok = wmax - (200u << 20) < (1700u << 20) && vmin_ >= ew - (41u << 20) &&
            umin32(umax32(hp1, hm1), umax32(hp2, hm2)) >= 0x100000u &&
            umax32(he1, he2) < 0x40200000u && umax32(hf1, hf2) < 0x400C0000u && g_ok &&
            (!has_ms || (hms | dlo(ms)) == 0u || hms >= ew - (40u << 20));
  if (!ok) return false;
  if ((hg | dlo(gm)) == 0u || (has_ms && (hms | dlo(ms)) == 0u)) {
    for (int k = 0; k < 8; k++) out[k] = 0.0;
    return true;
  }
  const uint32_t rb = ew - (127u << 20);

  // -- angular terms --
  ff S;
  ff2 sd;
  if (!lc_pair_angles(eta1, eta2, phi1, phi2, T, &S, &sd)) return false;

  // -- the legs (lane x: leg 1, lane y: leg 2) --
  const ff2 pt = cvt2(cvt_parts(hp1, dlo(pt1), rb), cvt_parts(hp2, dlo(pt2), rb));
  const ff2 mm = cvt2(cvt_parts(hm1, dlo(m1), rb), cvt_parts(hm2, dlo(m2), rb));
  const ff2 x = cvt2(cvt_parts_normal(umax32(he1, 0x3E100000u), dlo(eta1), kRebaseOne),
                     cvt_parts_normal(umax32(he2, 0x3E100000u), dlo(eta2), kRebaseOne));
  ff2 sh, ch;
  const LcLeg<ff2> L = lc_leg(pt, mm, x, T.hyp, &sh, &ch);

  // -- the pair: m, c = gm / (2 m) --
  const ff pt1f = lane_x(pt), pt2f = lane_y(pt);
  const ff p12 = lc_mul(pt1f, pt2f);
  ff m;
  if (has_ms) {
    m = cvt1(cvt_parts(hms, dlo(ms), rb));
  } else {
    const ff ta = lc_mul(p12, S);
    const ff m2s = lc_add(lc_mul(lc_add(lane_x(L.D), lane_y(L.D)), lc_add(lane_x(L.Y), lane_y(L.Y))),
                          ff{fmul(ta.hi, 4.0f), fmul(ta.lo, 4.0f)});
    if (m2s.hi == 0.0f) {
      for (int k = 0; k < 8; k++) out[k] = 0.0;
      return true;
    }
    if (m2s.hi < 8.27180613e-25f) return false;  // 2^-80
    m = lc_sqrt_refined(m2s);
  }
  const ff g = cvt1(cvt_parts(hg, dlo(gm), kRebaseOne));
  const ff c = lc_scale(lc_div(g, ff{fmul(m.hi, 2.0f), fmul(m.lo, 2.0f)}), sign_of(gm));

  // -- the gradient terms, scaled: G2 = 2 G = (N, -N) / E, N = D2 Y1 - Y2 D1 --
  const ff N = lc_sum(lc_mul(lane_y(L.D), lane_x(L.Y)), lc_scale(lc_mul(lane_y(L.Y), lane_x(L.D)), -1.0f));
  const ff2 invE = lc_div(ff2{bc2(1.0f), bc2(0.0f)}, L.E);
  const ff2 G2 = lc_mul(ff2{mk2(N.hi, -N.hi), mk2(N.lo, -N.lo)}, invE);
  const ff2 Sb = {bc2(S.hi), bc2(S.lo)};
  const ff2 pto = {mk2(pt.hi.y, pt.hi.x), mk2(pt.lo.y, pt.lo.x)};
  const ff2 dpt = lc_sum(lc_mul(ch, G2), lc_scale(lc_mul(pto, Sb), bc2(4.0f)));
  const ff2 p12b = {bc2(p12.hi), bc2(p12.lo)};
  const ff sde = lane_x(sd), sdp = lane_y(sd);
  const ff2 sdeb = {mk2(sde.hi, -sde.hi), mk2(sde.lo, -sde.lo)};   // +- 2 sinh d_eta
  const ff2 sdpb = {mk2(sdp.hi, -sdp.hi), mk2(sdp.lo, -sdp.lo)};   // +- 2 sin d_phi
  const ff2 deta = lc_sum(lc_scale(lc_mul(lc_mul(pt, sh), G2), mk2(sign_of(eta1), sign_of(eta2))),
                          lc_mul(p12b, sdeb));
  const ff2 dphi = lc_mul(p12b, sdpb);
  const ff2 SE = lc_add(L.E, ff2{mk2(L.E.hi.y, L.E.hi.x), mk2(L.E.lo.y, L.E.lo.x)});  // E1 + E2
  const ff2 dm = lc_scale(lc_mul(lc_mul(mm, invE), SE), mk2(2.0f * sign_of(m1), 2.0f * sign_of(m2)));
  const ff2 cb = {bc2(c.hi), bc2(c.lo)};
  // pt and m gradients carry no unit, eta and phi gradients the unit of m (2^s)
  const ff2 o_pt = lc_mul(cb, dpt), o_eta = lc_mul(cb, deta), o_phi = lc_mul(cb, dphi),
            o_m = lc_mul(cb, dm);
  constexpr uint32_t e0 = 896u << 20;
  out[0] = lc_to_double(lane_x(o_pt), e0);
  out[1] = lc_to_double(lane_x(o_eta), rb);
  out[2] = lc_to_double(lane_x(o_phi), rb);
  out[3] = lc_to_double(lane_x(o_m), e0);
  out[4] = lc_to_double(lane_y(o_pt), e0);
  out[5] = lc_to_double(lane_y(o_eta), rb);
  out[6] = lc_to_double(lane_y(o_phi), rb);
  out[7] = lc_to_double(lane_y(o_m), e0);
  return true;
}

}  // namespace ffm
}  // namespace gvx
