// FP64 Lorentz boost with part of its arithmetic in float-float (the FP64 boost kernels' fast
// path).
//
// With gamma = 1/s, s = sqrt(1 - b2), w = gamma/(1 + gamma) = 1/(1 + s) and
// k = gamma^2/(1 + gamma) = gamma w:
//   t = E + beta.p,  E' = gamma t,  p' = p + f beta,  f = k beta.p + gamma E = k t + w E.
// In the last form both terms are >= 0 for physical vectors (E >= |p|), so f carries no
// cancellation and ff precision is enough for it.  The output's condition number is
// C = (E + |beta| |p|) / t (t cancels when beta points against p at high |beta|; C reaches ~200
// for |beta| <= 0.99), so t, the one step whose rounding C amplifies, stays in FP64, as do
// E' = gamma t (exact for beta = 0) and the multiply-adds p_k + f beta_k.  1 - b2 is exact in
// 64-bit fixed point; s, gamma, w, k and f are formed in ff on the FP32 pipe, and gamma and f
// return to double with integer operations.  That leaves seven FP64 operations per vector
// (t 3, E' 1, p' 3); the normwise error vs E' stays below a few 2^-53 C plus a few 2^-47.
//
// Domain (anything else returns false and the caller uses the FP64 evaluation): 1 - b2 >= 2^-16
// (|beta| <= 0.9999924, gamma <= 256), finite inputs, and the vector's largest component
// magnitude in [2^-823, 2^1013), which keeps every scaled intermediate and both outputs inside
// the normal ranges of float and double.  Scaled values below 2^-74 count as 0 in the ff steps.
#pragma once

#include "ff.cuh"

namespace gvx {
namespace ffm {

// The velocity's part, computed once per beta.
struct BetaFF {
  ff w, k;    // 1/(1 + s) and gamma/(1 + s), s = sqrt(1 - b2)
  double g;   // gamma
  bool ok;    // |beta| inside the domain
};

GVX_HD BetaFF beta_ff(double bx, double by, double bz) {
  BetaFF B;
  bool ok = true;
  const ff omb = one_minus_sq3(bx, by, bz, &ok);
  const ff s = sqrt(omb);
  const ff g = recip(s);
  B.w = recip(add_same(make(1.0f), s));
  B.k = mul(g, B.w);
  B.g = ok ? to_double_int(g, 0) : 0.0;
  B.ok = ok;
  return B;
}

GVX_HD int max_exponent4(double a, double b, double c, double d) {
  int ea = dexp(a), eb = dexp(b), ec = dexp(c), ed = dexp(d);
  ea = ea > eb ? ea : eb;
  ec = ec > ed ? ec : ed;
  return ea > ec ? ea : ec;
}

// L(beta) (px, py, pz, E) into out[0..3] (PxPyPzE); false outside the domain.
GVX_HD bool boost_ff(const BetaFF &B, double bx, double by, double bz, double px, double py,
                     double pz, double E, double *out) {
  const int e = max_exponent4(px, py, pz, E);
  if (!B.ok || e < 200 || e > 2035) return false;
  const int s = e - 1023;  // components scaled into magnitudes below 2
  const double t = fma(bx, px, fma(by, py, fma(bz, pz, E)));
  const ff f = add(mul(B.k, from_double_ranged(t, s)), mul(B.w, from_double_ranged(E, s)));
  const double fd = to_double_int(f, s);
  out[0] = fma(fd, bx, px);
  out[1] = fma(fd, by, py);
  out[2] = fma(fd, bz, pz);
  out[3] = B.g * t;
  return true;
}

}  // namespace ffm
}  // namespace gvx
