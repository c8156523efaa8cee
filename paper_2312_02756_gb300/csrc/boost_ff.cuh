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
// return to double with integer operations (lc_to_double_int of mass_lc.cuh: truncation below
// one ulp).  That leaves seven FP64 operations per vector
// (t 3, E' 1, p' 3); the normwise error vs E' stays below a few 2^-53 C plus a few 2^-47.
//
// Domain (anything else returns false and the caller uses the FP64 evaluation): 1 - b2 >= 2^-16
// (|beta| <= 0.9999924, gamma <= 256), finite inputs, and the vector's largest component
// magnitude in [2^-823, 2^1013), which keeps every scaled intermediate and both outputs inside
// the normal ranges of float and double.  Scaled values below 2^-74 count as 0 in the ff steps.
#pragma once

#include "ff.cuh"
#include "mass_lc.cuh"

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
  B.g = ok ? lc_to_double_int(renorm(g), 896u << 20) : 0.0;
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
  const double fd = lc_to_double_int(f, (uint32_t)(896 + s) << 20);
  out[0] = fma(fd, bx, px);
  out[1] = fma(fd, by, py);
  out[2] = fma(fd, bz, pz);
  out[3] = B.g * t;
  return true;
}

// ---- adjoint ------------------------------------------------------------------------------
// grad_v = L grad_out (L is symmetric) and, with gb = beta.grad_p, tg = gE + gb,
// k' = dk/dgamma = gamma (gamma + 2)/(gamma + 1)^2 (so k' - 1 = -(s w)^2):
//   grad_beta = A beta + B p + f grad_p,
//   A = gamma^3 [gb (t + (k' - 1) bp) + gE t],   B = k gb + gamma gE,   f = k t + w E.
// t = E + bp and tg = gE + gb are FP64 (the sums that can cancel); bp = t - E, gb = tg - gE,
// A, B, f and the boost of grad_out are formed in ff from the scaled inputs and return to double
// by integer operations; the combinations of grad_beta with beta, p and grad_p are FP64
// multiply-adds (they can cancel by more than ff would resolve): 15 FP64 operations per vector.

struct BetaBwdFF {
  ff gf, w, k, kpm1, g3;  // gamma, 1/(1 + s), gamma w, k' - 1, gamma^3
  bool ok;
};

GVX_HD BetaBwdFF beta_bwd_ff(double bx, double by, double bz) {
  BetaBwdFF B;
  bool ok = true;
  const ff omb = one_minus_sq3(bx, by, bz, &ok);
  const ff s = sqrt(omb);
  const ff g = recip(s);
  B.gf = g;
  B.w = recip(add_same(make(1.0f), s));
  B.k = mul(g, B.w);
  B.kpm1 = neg(sqr(mul(s, B.w)));
  B.g3 = mul(sqr(g), g);
  B.ok = ok;
  return B;
}

// Both adjoint outputs for one vector p (px, py, pz, E) and upstream gradient q (the same
// layout); false outside the domain: beta as for boost_ff, each of p and q with its largest
// magnitude in [2^-823, 2^1013) (q may also be exactly zero), and their scales together within
// [2^-800, 2^900].
GVX_HD bool boost_bwd_ff(const BetaBwdFF &B, double bx, double by, double bz, const double *p,
                         const double *q, double *gv, double *gbeta) {
  if (!B.ok) return false;
  const int ev = max_exponent4(p[0], p[1], p[2], p[3]);
  const int eq = max_exponent4(q[0], q[1], q[2], q[3]);
  if (ev < 200 || ev > 2035) return false;
  if (eq == 0 && ((dhi(q[0]) | dlo(q[0]) | dhi(q[1]) | dlo(q[1]) | dhi(q[2]) | dlo(q[2]) |
                   dhi(q[3]) | dlo(q[3])) & 0x7fffffffu) == 0u &&
      ((dlo(q[0]) | dlo(q[1]) | dlo(q[2]) | dlo(q[3])) == 0u)) {
    for (int c = 0; c < 4; c++) gv[c] = 0.0;  // a zero upstream gradient gives zero gradients
    for (int c = 0; c < 3; c++) gbeta[c] = 0.0;
    return true;
  }
  if (eq < 200 || eq > 2035 || ev + eq - 2046 < -800 || ev + eq - 2046 > 900) return false;
  const int sv = ev - 1023, sq = eq - 1023;
  // the two sums that can cancel, in FP64 as in the forward; beta.p and beta.grad_p follow from
  // them in ff (t - E is exact up to t's own rounding, which stays at the FP64 level)
  const double t = fma(bx, p[0], fma(by, p[1], fma(bz, p[2], p[3])));
  const double tg = fma(bx, q[0], fma(by, q[1], fma(bz, q[2], q[3])));
  const ff T = from_double_ranged(t, sv), En = from_double_ranged(p[3], sv);
  const ff BP = add(T, neg(En));
  const ff TG = from_double_ranged(tg, sq), GE = from_double_ranged(q[3], sq);
  const ff GB = add(TG, neg(GE));
  const uint32_t rv = (uint32_t)(896 + sv) << 20, rq = (uint32_t)(896 + sq) << 20;
  const double f = lc_to_double_int(add(mul(B.k, T), mul(B.w, En)), rv);
  const ff FQ = add(mul(B.k, TG), mul(B.w, GE));
  const ff A = mul(B.g3, add(mul(GB, add(T, mul(B.kpm1, BP))), mul(GE, T)));
  const double a = lc_to_double_int(renorm(A), (uint32_t)(896 + sv + sq) << 20);
  const double bq = lc_to_double_int(add(mul(B.k, GB), mul(B.gf, GE)), rq);
  // grad_v = L grad_out in ff (its terms cancel by at most the condition of L, gamma (1 + |beta|)):
  // q_k + fq beta_k and gamma tg, returned to double by integer operations
  {
    // 47-bit inputs suffice here (the terms cancel by at most the condition of L): the light-cone
    // conversions of q_k and beta_k, signs applied on the bits; outputs assembled by integer
    // operations
    const auto cv = [](double d, uint32_t rb) {
      const ff m = cvt1(cvt_parts(dhi(d) & 0x7fffffffu, dlo(d), rb));
      return (dhi(d) >> 31) ? ff{-m.hi, -m.lo} : m;
    };
    gv[0] = lc_to_double_int(renorm(add(cv(q[0], rq), mul(FQ, cv(bx, kRebaseOne)))), rq);
    gv[1] = lc_to_double_int(renorm(add(cv(q[1], rq), mul(FQ, cv(by, kRebaseOne)))), rq);
    gv[2] = lc_to_double_int(renorm(add(cv(q[2], rq), mul(FQ, cv(bz, kRebaseOne)))), rq);
    gv[3] = lc_to_double_int(renorm(mul(B.gf, TG)), rq);
  }
  gbeta[0] = fma(a, bx, fma(bq, p[0], f * q[0]));
  gbeta[1] = fma(a, by, fma(bq, p[1], f * q[1]));
  gbeta[2] = fma(a, bz, fma(bq, p[2], f * q[2]));
  return true;
}

}  // namespace ffm
}  // namespace gvx
