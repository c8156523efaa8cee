// Pair mass of PtEtaPhiE legs in light-cone form (the fast path of the FP64 PtEtaPhiE mass
// kernel; the mass of Sec. 4.1 on the (pt, eta, phi, E) system of Sec. 3.1).
//
// With P_i = pt_i cosh(eta_i) and the stored energy E_i, Y_i = E_i + P_i and D_i = E_i - P_i, the
// mass of the summed vector is
//   m^2 = (D1 + D2)(Y1 + Y2) + 4 pt1 pt2 S,   S = sinh^2(|d_eta|/2) + sin^2(|d_phi|/2),
// the identity of mass_lc.cuh with D_i = m_i^2 / Y_i replaced by the difference itself (for
// PtEtaPhiE legs m_i^2 = E_i^2 - P_i^2 is not a stored number).  D_i is a float-float difference
// of a stored number and a computed one, with an absolute error of ~2^-46 (E_i + P_i); the
// result is therefore accurate normwise, within 2^-40 (M1 + M2)^2 in m|m| with
// M_i = max(E_i, P_i) -- the contract of the PtEtaPhiE masses.  The two legs run as the lanes of
// paired FP32 instructions.
//
// Domain (anything else returns false and the caller takes the other route): pt >= 0 and E >= 0,
// |eta| < 8, |phi| < 3.5, the common power-of-two scale of pt and E with exponent field
// 200..1899, each nonzero pt and E at least 2^-40 of the scale, no leg with pt = E = 0,
// |d_phi|/2 not within 2^-7 of pi, and a scaled m^2 of at least 2^-80 (spacelike sums and masses
// lost in the float-float differences included).
#pragma once

#include "mass_lc.cuh"

namespace gvx {
namespace ffm {

GVX_HD bool pair_mass_e_lc(double pt1, double eta1, double phi1, double e1, double pt2,
                           double eta2, double phi2, double e2, const LcTab &T, double *out) {
  const uint32_t hp1 = dhi(pt1), hp2 = dhi(pt2), hE1 = dhi(e1), hE2 = dhi(e2);
  const uint32_t wmax = umax32(umax32(hp1, hE1), umax32(hp2, hE2));  // the sign bits count too
  const uint32_t ew = wmax & 0x7ff00000u;
  const uint32_t vmin_ = umin32(umin32(hp1 - 0x100000u, hE1 - 0x100000u),
                                umin32(hp2 - 0x100000u, hE2 - 0x100000u));
  const uint32_t he1 = dhi(eta1) & 0x7fffffffu, he2 = dhi(eta2) & 0x7fffffffu;
  const uint32_t hf1 = dhi(phi1) & 0x7fffffffu, hf2 = dhi(phi2) & 0x7fffffffu;
  // wmax below 2^31 keeps out negative pt and E; vmin_ (unsigned, zeros wrap around) requires
  // every nonzero pt and E within 2^-40 of the scale
  if (!(wmax - (200u << 20) < (1700u << 20) && vmin_ >= ew - (41u << 20) &&
        umin32(umax32(hp1, hE1), umax32(hp2, hE2)) >= 0x100000u &&
        umax32(he1, he2) < 0x40200000u && umax32(hf1, hf2) < 0x400C0000u))
    return false;
  ff S;
  if (!lc_pair_S(eta1, eta2, phi1, phi2, T, &S)) return false;
  const uint32_t rb = ew - (127u << 20);
  const ff2 pt = cvt2(cvt_parts(hp1, dlo(pt1), rb), cvt_parts(hp2, dlo(pt2), rb));
  const ff2 E = cvt2(cvt_parts(hE1, dlo(e1), rb), cvt_parts(hE2, dlo(e2), rb));
  const ff2 x = cvt2(cvt_parts_normal(umax32(he1, 0x3E100000u), dlo(eta1), kRebaseOne),
                     cvt_parts_normal(umax32(he2, 0x3E100000u), dlo(eta2), kRebaseOne));
  // cosh |eta| from the table (the reduction of lc_leg)
  uint32_t n[2];
  const ff2 r = lc_reduce(x, n);
  ff2 C, Sh;
  tab_load(T.hyp, GVX_HYP_N, n, &C, &Sh);
  const ff2 ch = tab_comb(C, Sh, r, tab_poly(r, bc2(0.5f)));
  const ff2 P = lc_mul(pt, ch);
  const ff2 Y = lc_add(E, P);
  const ff2 D = add_same(E, ff2{neg2(P.hi), neg2(P.lo)});  // E - P, either sign
  const ff sD = add_same(lane_x(D), lane_y(D)), sY = lc_add(lane_x(Y), lane_y(Y));
  const ff ta = lc_mul(lc_mul(lane_x(pt), lane_y(pt)), S);
  const ff m2s = add_same(lc_mul(sD, sY), ff{fmul(ta.hi, 4.0f), fmul(ta.lo, 4.0f)});
  if (!(m2s.hi >= 8.27180613e-25f)) return false;  // below 2^-80 (or negative)
  *out = lc_mass_out(m2s, ew);
  return true;
}

}  // namespace ffm
}  // namespace gvx
