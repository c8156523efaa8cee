// Conversion of one 4-vector to PxPyPzE (Sec. 3.1: vectors are templated on their coordinate
// system, and every system maps to the Cartesian one):
//   PtEtaPhiM: px = pt cos(phi), py = pt sin(phi), pz = pt sinh(eta), E = sqrt((pt cosh eta)^2 + m^2);
//   PtEtaPhiE: the same momentum, E as stored;
//   PxPyPzM:   the momentum as stored, E = sqrt(|p|^2 + m^2).
// The FP64 fast path evaluates these in float-float (table-driven sin/cos and sinh/cosh of
// ff_tables.cuh, the values scaled by a power of two) and rounds each component to double once:
// every component is within 2^-43 max(|E|, |p|) of the exact conversion of the stored values.
// Outside its domain (pt < 0, |eta| >= 16, |phi| > pi, a non-finite value, a scale beyond the
// float-float range) the functions return false and the caller converts in FP64.
#pragma once

#include "mass_ff.cuh"

namespace gvx {
namespace ffm {

// (pt, eta, phi, w) -> (px, py, pz, E): w is E when e_stored, else the mass.
GVX_HD bool ptetaphi_to_cart(double pt, double eta, double phi, double w, bool e_stored,
                             const TabRef &T, double *out) {
  if (dhi(pt) >> 31) return false;                        // pt < 0 (or -0)
  if (((dhi(eta) >> 20) & 0x7ffu) > 1026u) return false;  // |eta| >= 16, NaN, Inf
  if (!within_pi(phi)) return false;                      // |phi| > pi, NaN
  const int emax = e_stored ? dexp(pt) : leg_exponent(pt, w);
  if (!scale_exponent_ok(emax)) return false;  // zero, tiny or non-finite scale
  if (e_stored && dexp(w) == 0x7ff) return false;
  const int s = emax - 1023;
  bool ok = true;
  const ff ptf = from_double_ranged(pt, s);
  ff sn, cs, sh, ch;
  sincos_t(phi, T, &sn, &cs, &ok);
  sinhcosh_t(from_double_ranged(eta, 0), T, &sh, &ch);  // |eta| < 16
  out[0] = to_double(renorm(mul(ptf, cs)), s);
  out[1] = to_double(renorm(mul(ptf, sn)), s);
  out[2] = to_double(renorm(mul(ptf, sh)), s);
  if (e_stored) {
    out[3] = w;
  } else {
    const ff P = mul(ptf, ch);
    out[3] = to_double(ffm::sqrt(add_same(sqr(P), sqr(from_double_ranged(w, s)))), s);
  }
  return ok;
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
