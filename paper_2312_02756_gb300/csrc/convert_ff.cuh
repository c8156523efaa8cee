// Conversion of one 4-vector to PxPyPzE (Sec. 3.1: vectors are templated on their coordinate
// system, and every system maps to the Cartesian one):
//   PtEtaPhiM: px = pt cos(phi), py = pt sin(phi), pz = pt sinh(eta), E = sqrt((pt cosh eta)^2 + m^2);
//   PtEtaPhiE: the same momentum, E as stored;
//   PxPyPzM:   the momentum as stored, E = sqrt(|p|^2 + m^2).
// The FP64 fast path evaluates these in float-float (the values scaled by a power of two) and
// rounds each component to double once: every component is within 2^-43 max(|E|, |p|) of the
// exact conversion of the stored values.  Outside its domain the functions return false and the
// caller converts in FP64.
#pragma once

#include "mass_ff.cuh"
#include "mass_lc.cuh"

namespace gvx {
namespace ffm {

// (pt, eta, phi, w) -> (px, py, pz, E), w being E when e_stored, else the mass, with the
// light-cone tables (mass_lc.cuh): one paired reduction of (|eta|, |phi|) gives (sinh, sin) and (cosh, cos) from the two tables
// at step 2^-8, the products with pt run on paired FP32 lanes, and each component returns to
// double by its bits and one FP64 addition.  The input conversions keep 47 bits and small eta
// exactly (sinh(eta) ~ eta), so every component is within 2^-43 max(|E|, |p|) of the exact
// conversion.  Domain: pt >= 0, |eta| < 8, |phi| < 3.5, the scale (pt, or the larger of pt and
// |m|) with exponent field 200..1899, a finite stored E; false otherwise (the caller converts in
// FP64).
GVX_HD bool ptetaphi_to_cart_lc(double pt, double eta, double phi, double w, bool e_stored,
                                const LcTab &T, double *out) {
  const uint32_t hp = dhi(pt), hw = dhi(w) & 0x7fffffffu;
  const uint32_t he = dhi(eta) & 0x7fffffffu, hf = dhi(phi) & 0x7fffffffu;
  const uint32_t wmax = e_stored ? hp : umax32(hp, hw);  // a negative pt fails the range check
  const uint32_t ew = wmax & 0x7ff00000u;
  if (!(wmax - (200u << 20) < (1700u << 20) && he < 0x40200000u && hf < 0x400C0000u &&
        (!e_stored || hw < 0x7ff00000u)))
    return false;
  const uint32_t rb = ew - (127u << 20);
  // lanes (|eta|, |phi|): (sinh, sin) and (cosh, cos)
  const ff2 xa = cvt2(cvt_parts(he, dlo(eta), kRebaseOne), cvt_parts(hf, dlo(phi), kRebaseOne));
  uint32_t nj[2];
  const ff2 r = lc_reduce(xa, nj);
  const gvx_f4 th = ldtab(&T.hyp[umin32(nj[0], GVX_HYP_N)]);
  const gvx_f4 ts = ldtab(&T.sin[umin32(nj[1], GVX_SIN_N)]);
  const ff2 A = {mk2(th.z, ts.x), mk2(th.w, ts.y)};    // (sinh, sin) of the table point
  const ff2 B = {mk2(th.x, ts.z), mk2(th.y, ts.w)};    // (cosh, cos)
  const ff2 Bn = {mk2(th.z, -ts.x), mk2(th.w, -ts.y)};  // (sinh, -sin)
  const TabPoly<f2> tp = tab_poly(r, mk2(0.5f, -0.5f));
  // both with TwoSum (any order of the terms): near |phi| = pi the table's sin is as small as
  // cos times the remainder
  const ff2 w1 = tab_comb_any(A, B, r, tp);    // (sinh |eta|, sin |phi|)
  const ff2 wc = tab_comb_any(B, Bn, r, tp);   // (cosh |eta|, cos |phi|)
  const ff ptf = cvt1(cvt_parts(hp, dlo(pt), rb));
  const ff2 ptb = {bc2(ptf.hi), bc2(ptf.lo)};
  const ff2 pzy = lc_mul(ptb, w1);  // (pt sinh |eta|, pt sin |phi|)
  const ff2 Px = lc_mul(ptb, wc);   // (pt cosh |eta| = P, pt cos phi)
  const float seta = (dhi(eta) >> 31) ? -1.0f : 1.0f, sphi = (dhi(phi) >> 31) ? -1.0f : 1.0f;
  out[0] = lc_to_double(lane_y(Px), rb);
  out[1] = lc_to_double(lc_scale(lane_y(pzy), sphi), rb);
  out[2] = lc_to_double(lc_scale(lane_x(pzy), seta), rb);
  if (e_stored) {
    out[3] = w;
  } else {
    const ff mm = cvt1(cvt_parts(hw, dlo(w), rb));
    const ff P = lane_x(Px);
    out[3] = lc_to_double(lc_sqrt_refined(lc_add(lc_sqr(P), lc_sqr(mm))), rb);
  }
  return true;
}

// (px, py, pz, m) -> (px, py, pz, E).
GVX_HD bool pxpypzm_to_cart(const double *x, double *out) {
  int emax = 0;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const int e = dexp(x[k]);
    emax = e > emax ? e : emax;
  }
  if (!scale_exponent_ok(emax)) return false;
  const int s = emax - 1023;
  ff acc = sqr(from_double_ranged(x[0], s));
#pragma unroll
  for (int k = 1; k < 4; k++) acc = add_same(acc, sqr(from_double_ranged(x[k], s)));
  out[0] = x[0];
  out[1] = x[1];
  out[2] = x[2];
  out[3] = to_double(ffm::sqrt(acc), s);
  return true;
}

}  // namespace ffm
}  // namespace gvx
