// Table-driven float-float elementary functions.  The tables (gvx_tables.inc) are generated at
// build time by gen_tables.py; kernels copy them to shared memory and pass a TabRef.
#pragma once

#include "ff.cuh"

#if defined(__CUDACC__)
#define GVX_TABLE static __device__
#else
#define GVX_TABLE static
#endif

namespace gvx {
namespace ffm {

#include "gvx_tables.inc"

struct TabRef {
  const gvx_f4 *exp;   // kExpTab: {tm1.hi, tm1.lo, um1.hi, um1.lo}
  const gvx_f4 *trig;  // kTrigTab: {sin.hi, sin.lo, cos.hi, cos.lo}
};

// cosh(x) for |x| < 16:  (2^(n/N) (E + O) + 2^(-n/N) (E - O)) / 2 with n = N k + j,
// 2^(j/N) = 1 + tm1[j] and 2^(-j/N) = 1 - um1[j]  (N = 1024).
GVX_HD ff cosh_t(ff x, const TabRef &T) {
  if (x.hi < 0.0f) x = neg(x);
  HypParts h = hyp_parts(x, kExpInvC, kExpC0, kExpC1, kExpC2);
  gvx_f4 t = T.exp[h.j];
  ff tp = fast_two_sum(1.0f, t.x);
  tp.lo = fadd(tp.lo, t.y);
  ff tn = fast_two_sum(1.0f, -t.z);
  tn.lo = fsub(tn.lo, t.w);
  ff ep = scale(mul(tp, add_eo(h.E, h.O)), pow2f(h.k - 1));
  ff en = scale(mul(tn, add_eo(h.E, neg(h.O))), pow2f(-h.k - 1));
  return add_same(ep, en);
}

// The sums sin(jd) cos r + cos(jd) sin r and sinh(nc) cosh r + cosh(nc) sinh r below can have
// terms of opposite sign, but the second term is at most about half the first (j, n >= 1) or the
// first is 0 (j = n = 0), so they cancel at most threefold and add_same keeps ff precision.

// sinh(x) for |x| < 16, with full relative accuracy also for tiny |x|:
//   sinh(n c + r) = S E + C O,  S = sinh(n c) = ((2^k - 2^-k) + 2^k tm1[j] + 2^-k um1[j]) / 2
//   (every term >= 0), C = cosh(n c) = S + 2^-k (1 - um1[j]).
GVX_HD ff sinh_t(ff x, const TabRef &T) {
  bool negx = x.hi < 0.0f;
  if (negx) x = neg(x);
  HypParts h = hyp_parts(x, kExpInvC, kExpC0, kExpC1, kExpC2);
  gvx_f4 t = T.exp[h.j];
  float pk = pow2f(h.k), mk = pow2f(-h.k);
  ff a = {fmul(t.x, pk), fmul(t.y, pk)};
  ff b = {fmul(t.z, mk), fmul(t.w, mk)};
  ff S = scale(add_same(add_same(fast_two_sum(pk, -mk), a), b), 0.5f);
  ff tn = fast_two_sum(1.0f, -t.z);
  tn.lo = fsub(tn.lo, t.w);
  ff C = add_same(S, scale(tn, mk));
  ff s = add_same(mul(S, h.E), mul(C, h.O));  // opposite signs cancel at most 3x
  return negx ? neg(s) : s;
}

// sin(h) for 0 <= h <= pi/2 (+ a few ulps):  sin(j d + r) = sin(j d) cos r + cos(j d) sin r,
//   d = pi/2048, |r| <= d/2,  cos r = 1 - r^2/2 + r^4/24,  sin r = r - r^3/6.
GVX_HD ff sin_t(ff h, const TabRef &T) {
  int j;
  float jf = round_shift(fmul(h.hi, kTrigInvD), &j);
  if (j > GVX_TRIG_N) {
    j = GVX_TRIG_N;
    jf = (float)GVX_TRIG_N;
  }
  if (j < 0) {
    j = 0;
    jf = 0.0f;
  }
  ff r = reduce(h, jf, kTrigD0, kTrigD1, kTrigD2);
  ff r2 = two_prod(r.hi, r.hi);
  r2.lo = ffma(fadd(r.hi, r.hi), r.lo, r2.lo);
  ff cr = fast_two_sum(1.0f, fmul(r2.hi, -0.5f));
  cr.lo = fadd(cr.lo, ffma(r2.lo, -0.5f, fmul(fmul(r2.hi, r2.hi), 0.041666668f)));
  ff sr = two_sum(r.hi, fmul(fmul(r.hi, r2.hi), -0.16666667f));
  sr.lo = fadd(sr.lo, r.lo);
  gvx_f4 t = T.trig[j];
  return add_same(mul(ff{t.x, t.y}, cr), mul(ff{t.z, t.w}, sr));  // cancels at most 3x
}

// sinh(x) and cosh(x) together (one reduction), |x| < 16.
GVX_HD void sinhcosh_t(ff x, const TabRef &T, ff *sh, ff *ch) {
  bool negx = x.hi < 0.0f;
  if (negx) x = neg(x);
  HypParts h = hyp_parts(x, kExpInvC, kExpC0, kExpC1, kExpC2);
  gvx_f4 t = T.exp[h.j];
  float pk = pow2f(h.k), mk = pow2f(-h.k);
  ff a = {fmul(t.x, pk), fmul(t.y, pk)};
  ff b = {fmul(t.z, mk), fmul(t.w, mk)};
  ff S = scale(add_same(add_same(fast_two_sum(pk, -mk), a), b), 0.5f);
  ff tn = fast_two_sum(1.0f, -t.z);
  tn.lo = fsub(tn.lo, t.w);
  ff C = add_same(S, scale(tn, mk));
  ff s = add_same(mul(S, h.E), mul(C, h.O));  // opposite signs cancel at most 3x
  *sh = negx ? neg(s) : s;
  *ch = add_same(mul(C, h.E), mul(S, h.O));
}

// sin(h) and cos(h) for 0 <= h <= pi/2 (+ a few ulps), relative accuracy ~2^-46 for both.
GVX_HD void sincos_q1_t(ff h, const TabRef &T, ff *sn, ff *cs) {
  int j;
  float jf = round_shift(fmul(h.hi, kTrigInvD), &j);
  if (j > GVX_TRIG_N) {
    j = GVX_TRIG_N;
    jf = (float)GVX_TRIG_N;
  }
  if (j < 0) {
    j = 0;
    jf = 0.0f;
  }
  ff r = reduce(h, jf, kTrigD0, kTrigD1, kTrigD2);
  ff r2 = two_prod(r.hi, r.hi);
  r2.lo = ffma(fadd(r.hi, r.hi), r.lo, r2.lo);
  ff cr = fast_two_sum(1.0f, fmul(r2.hi, -0.5f));
  cr.lo = fadd(cr.lo, ffma(r2.lo, -0.5f, fmul(fmul(r2.hi, r2.hi), 0.041666668f)));
  ff sr = two_sum(r.hi, fmul(fmul(r.hi, r2.hi), -0.16666667f));
  sr.lo = fadd(sr.lo, r.lo);
  gvx_f4 t = T.trig[j];
  ff sj = {t.x, t.y}, cj = {t.z, t.w};
  *sn = add_same(mul(sj, cr), mul(cj, sr));
  *cs = add(mul(cj, cr), neg(mul(sj, sr)));
}

// sin(phi) and cos(phi) for |phi| <= pi (+ a few ulps), absolute error ~2^-47: the first
// quadrant through the table, the second through pi - |phi|.
GVX_HD void sincos_t(double phi, const TabRef &T, ff *sn, ff *cs, bool *ok) {
  ff a = from_double(fabs(phi), ok);
  bool q2 = a.hi > 1.57079637f;
  if (q2) a = add(ff{kPiHi, kPiLo}, neg(a));
  int j;
  float jf = round_shift(fmul(a.hi, kTrigInvD), &j);
  if (j > GVX_TRIG_N) {
    j = GVX_TRIG_N;
    jf = (float)GVX_TRIG_N;
  }
  if (j < 0) {
    j = 0;
    jf = 0.0f;
  }
  ff r = reduce(a, jf, kTrigD0, kTrigD1, kTrigD2);
  ff r2 = two_prod(r.hi, r.hi);
  r2.lo = ffma(fadd(r.hi, r.hi), r.lo, r2.lo);
  ff cr = fast_two_sum(1.0f, fmul(r2.hi, -0.5f));
  cr.lo = fadd(cr.lo, ffma(r2.lo, -0.5f, fmul(fmul(r2.hi, r2.hi), 0.041666668f)));
  ff sr = two_sum(r.hi, fmul(fmul(r.hi, r2.hi), -0.16666667f));
  sr.lo = fadd(sr.lo, r.lo);
  gvx_f4 t = T.trig[j];
  ff sj = {t.x, t.y}, cj = {t.z, t.w};
  ff s = add_same(mul(sj, cr), mul(cj, sr));
  ff c = add(mul(cj, cr), neg(mul(sj, sr)));
  *sn = (dhi(phi) >> 31) ? neg(s) : s;
  *cs = q2 ? neg(c) : c;
}

#if defined(__CUDACC__)
// Copy both tables (32 KB) into shared memory; every thread of the CTA takes part.
__device__ __forceinline__ TabRef stage_tables(gvx_f4 *s_exp, gvx_f4 *s_trig) {
  for (int k = threadIdx.x; k < GVX_EXP_N; k += blockDim.x) s_exp[k] = kExpTab[k];
  for (int k = threadIdx.x; k <= GVX_TRIG_N; k += blockDim.x) s_trig[k] = kTrigTab[k];
  __syncthreads();
  return TabRef{s_exp, s_trig};
}
#endif

}  // namespace ffm
}  // namespace gvx
