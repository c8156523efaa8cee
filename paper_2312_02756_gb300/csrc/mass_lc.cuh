// Pair mass in float-float through light-cone components: the fast path of the FP64
// invariant-mass kernel (GenVectorX, Sec. 4.1, Fig. 1: per index, the mass of v1 + v2).
//
// With P_i = |p_i| = pt_i cosh(eta_i), E_i = sqrt(P_i^2 + m_i^2) and, per leg, the light-cone
// components Y_i = E_i + P_i and D_i = E_i - P_i = m_i^2 / Y_i (a quotient: no cancellation),
//   m^2 = (E1 + E2)^2 - |p1 + p2|^2 = (E1 + E2)^2 - (P1 + P2)^2 + 2 (P1 P2 - p1.p2)
//       = (D1 + D2)(Y1 + Y2) + 4 pt1 pt2 (sinh^2(d_eta/2) + sin^2(d_phi/2)),
// because P1 P2 - p1.p2 = pt1 pt2 (cosh d_eta - cos d_phi).  Every factor and term is
// non-negative for pt >= 0, so the relative error of m^2 is that of its ingredients, whatever
// the cancellation in E^2 - |p|^2.
//
// Arithmetic: float-float (ff, ff.cuh) on the FP32 pipe, the two legs of a pair as the lanes of
// Blackwell's paired FP32 instructions (ff2.cuh), and sinh(|d_eta|/2) with sin(|d_phi|/2) as the
// two lanes of one paired evaluation.  Three FP64 operations per pair: the two angle differences
// (exact where they cancel) and the final add that forms the double.
//
// Transcendentals: tables at the power-of-two step h = 2^-8 (kHypTab: cosh, sinh of n h;
// kSinTab: sin, cos of j h; generated by gen_tables.py; 47 KB, read through L1), so that x = n h + r, |r| <= h/2, is an
// exact float operation, and f(x) = A Ce(r) + B So(r) with the table pair (A, B),
// Ce = 1 + s r^2/2 + r^4/24 and So = r + s r^3/6 + r^5/120 (s = +1 hyperbolic, -1 circular;
// the next terms are below 2^-54 relative).
//
// Conversions from double are integer bit operations (cvt_parts): the leading 24 bits of the
// significand (truncated) become hi, the next 23 bits lo, so hi + lo is the double to within
// 2^-46 relative; the exponent is rebased by one subtraction, which also applies the pair's
// common power-of-two scale of pt and m (the largest brought into [1, 2)).
//
// Fast-path domain (anything else returns false and the caller takes the FP64 formulas):
//  - pt >= 0 (not -0), |eta| < 8, |phi| < 3.5, all inputs finite, neither leg a zero vector
//    (pt = m = 0);
//  - the pair's scale 2^e of pt and m with 2^-823 <= 2^e < 2^877, and every nonzero pt and m
//    at least 2^-40 of it (denormal inputs count as zero: below 2^-199 of the scale);
//  - |d_phi| not within 2^-6 of 2 pi (there the FP64 rounding of phi1 - phi2 would matter);
//  - the scaled m^2 either 0 or >= 2^-80, so that every term flushed below the float range is
//    under 2^-46 of it.
// Error over the domain: below 2^-42 relative in m (host tests against the binary128 oracle,
// with the hardware approximations' worst-case error modelled on the host).
#pragma once

#include "ff2.cuh"
#include "ff_tables.cuh"

namespace gvx {
namespace ffm {

// The tables are read where they are (global memory on the device) through the read-only data
// path: at 47 KB they stay resident in each SM's L1, so they take no shared memory.
struct LcTab {
  const gvx_f4 *hyp;  // kHypTab: {cosh.hi, cosh.lo, sinh.hi, sinh.lo} of n 2^-8
  const gvx_f4 *sin;  // kSinTab: {sin.hi, sin.lo, cos.hi, cos.lo} of j 2^-8
};

GVX_HD gvx_f4 ldtab(const gvx_f4 *p) {
#if defined(__CUDA_ARCH__)
  return __ldg(p);
#else
  return *p;
#endif
}

GVX_HD uint32_t umax32(uint32_t a, uint32_t b) { return a > b ? a : b; }
GVX_HD uint32_t umin32(uint32_t a, uint32_t b) { return a < b ? a : b; }

// (hi:lo << 3) >> 32: the top word of a double shifted left by three bits.
GVX_HD uint32_t funnel_l3(uint32_t lo, uint32_t hi) {
#if defined(__CUDA_ARCH__)
  return __funnelshift_l(lo, hi, 3);
#else
  return (hi << 3) | (lo >> 29);
#endif
}

// Hardware approximations (MUFU): 1/a and 1/sqrt(a) with a relative error below 2^-22.9.  The
// host build models that worst case (the result moved by +-2^-23 relative, the sign taken from
// the input's bits), so that the host tests bound the device's error rather than a correctly
// rounded one's.
GVX_HD float rcp_mufu(float a) {
#if defined(__CUDA_ARCH__)
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
#else
  const double e = (f2u(a) & 1u) ? 1.0 + 0x1p-23 : 1.0 - 0x1p-23;
  return (float)(e / (double)a);
#endif
}
GVX_HD float rsqrt_mufu(float a) {
#if defined(__CUDA_ARCH__)
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
#else
  const double e = (f2u(a) & 2u) ? 1.0 + 0x1p-23 : 1.0 - 0x1p-23;
  return (float)(e / ::sqrt((double)a));
#endif
}
GVX_HD float fmax_(float a, float b) { return a > b ? a : b; }

// ---- conversion from the words of a double ---------------------------------------------------

// Exponent rebase of a double's high word: R(E) = (E - 127) << 20 for the double's biased
// exponent E that becomes the float exponent 127 (1.0).
constexpr uint32_t kRebaseOne = 896u << 20;   // E = 1023: the value itself
constexpr uint32_t kRebaseHalf = 897u << 20;  // E = 1024: half the value

// hi bits and the two words whose float difference is lo (paired later with one subtraction).
struct CvtParts {
  uint32_t hb, ab, bb;
};

// |d| * 2^(1023 - E) as float-float from the words of d (wh without its sign bit, wl), E given
// by rb = R(E): the exponent is rebased in the high word and clamped at 0 (signed), then hi =
// the leading 24 significand bits (a funnel shift by 3) and lo = u2f(ab) - u2f(bb) the next 23
// (lo in [0, ulp(hi))).  A value whose rebased exponent would be <= 0 (a zero, a denormal, or
// below 2^-126 after rebasing) becomes hi = a float below 2^-146 and lo = 0 or a denormal:
// zero to the arithmetic that follows.  Requires the rebased exponent of a value that matters
// in [24, 254].
GVX_HD CvtParts cvt_parts(uint32_t wh, uint32_t wl, uint32_t rb) {
  const int32_t w = (int32_t)(wh - rb);
  const uint32_t hb = funnel_l3(wl, (uint32_t)(w > 0 ? w : 0));
  const int32_t e = (int32_t)(hb & 0x7f800000u) - (int32_t)(23u << 23);
  const uint32_t el = (uint32_t)(e > 0 ? e : 0);
  return {hb, el | ((wl >> 6) & 0x7fffffu), el};
}

// cvt_parts for a value known to rebase to an exponent in [24, 254] (|eta| raised to >= 2^-30):
// no clamps.
GVX_HD CvtParts cvt_parts_normal(uint32_t wh, uint32_t wl, uint32_t rb) {
  const uint32_t hb = funnel_l3(wl, wh - rb);
  const uint32_t el = (hb & 0x7f800000u) - (23u << 23);
  return {hb, el | ((wl >> 6) & 0x7fffffu), el};
}

GVX_HD ff2 cvt2(const CvtParts &a, const CvtParts &b) {
  ff2 r;
  r.hi = mk2(u2f(a.hb), u2f(b.hb));
  r.lo = sub2(mk2(u2f(a.ab), u2f(b.ab)), mk2(u2f(a.bb), u2f(b.bb)));
  return r;
}
GVX_HD ff cvt1(const CvtParts &a) { return {u2f(a.hb), fsub(u2f(a.ab), u2f(a.bb))}; }

// ---- lane-generic float-float steps ---------------------------------------------------------
// Each step is written once for V = float (one value) and V = f2 (two values as the lanes of
// Blackwell's paired FP32 instructions).  A lane of the paired form rounds exactly as the scalar
// form (a - b and -a are single correctly rounded or exact operations either way), so the
// jagged kernel's per-particle terms (scalar) have the bits of the elementwise kernel's two
// legs (paired).  Results may be unnormalized: |lo| up to ~2 ulp(hi).

GVX_HD float fmin_(float a, float b) { return a < b ? a : b; }
GVX_HD float vadd(float a, float b) { return fadd(a, b); }
GVX_HD f2 vadd(f2 a, f2 b) { return add2(a, b); }
GVX_HD float vmul(float a, float b) { return fmul(a, b); }
GVX_HD f2 vmul(f2 a, f2 b) { return mul2(a, b); }
GVX_HD float vfma(float a, float b, float c) { return ffma(a, b, c); }
GVX_HD f2 vfma(f2 a, f2 b, f2 c) { return fma2(a, b, c); }
GVX_HD float vsub(float a, float b) { return fsub(a, b); }
GVX_HD f2 vsub(f2 a, f2 b) { return sub2(a, b); }
GVX_HD float vneg(float a) { return -a; }
GVX_HD f2 vneg(f2 a) { return neg2(a); }
GVX_HD float vmax(float a, float b) { return fmax_(a, b); }
GVX_HD f2 vmax(f2 a, f2 b) { return mk2(fmax_(a.x, b.x), fmax_(a.y, b.y)); }
GVX_HD float vmin(float a, float b) { return fmin_(a, b); }
GVX_HD f2 vmin(f2 a, f2 b) { return mk2(fmin_(a.x, b.x), fmin_(a.y, b.y)); }
GVX_HD float vrsqrt(float a) { return rsqrt_mufu(a); }
GVX_HD f2 vrsqrt(f2 a) { return mk2(rsqrt_mufu(a.x), rsqrt_mufu(a.y)); }
GVX_HD float vrcp(float a) { return rcp_mufu(a); }
GVX_HD f2 vrcp(f2 a) { return mk2(rcp_mufu(a.x), rcp_mufu(a.y)); }
GVX_HD float vbc(float c, float) { return c; }
GVX_HD f2 vbc(float c, f2) { return bc2(c); }

template <class F>
using lane_t = decltype(F::hi);

template <class F>
GVX_HD F lc_sqr(const F &x) {
  const auto p = vmul(x.hi, x.hi);
  const auto e = vfma(x.hi, x.hi, vneg(p));
  return {p, vfma(vadd(x.hi, x.hi), x.lo, e)};
}
template <class F>
GVX_HD F lc_mul(const F &x, const F &y) {
  const auto p = vmul(x.hi, y.hi);
  const auto e = vfma(x.hi, y.hi, vneg(p));
  return {p, vfma(x.lo, y.hi, vfma(x.hi, y.lo, e))};
}
// x times a power of two or a sign (exact)
template <class F>
GVX_HD F lc_scale(const F &x, lane_t<F> k) {
  return {vmul(x.hi, k), vmul(x.lo, k)};
}
// x + y for x, y >= 0: Fast2Sum of the leading parts ordered by max/min (exact for non-negative
// operands; the comparisons run on the integer ALU, leaving the FMA pipes three operations).
template <class F>
GVX_HD F lc_add(const F &x, const F &y) {
  const auto a = vmax(x.hi, y.hi), b = vmin(x.hi, y.hi);
  const auto s = vadd(a, b);
  return {s, vadd(vsub(b, vsub(s, a)), vadd(x.lo, y.lo))};
}
// sqrt(x), x.hi > 0: s = x.hi rs with the approximate reciprocal square root rs, corrected
// once from the float-float residual x - s^2.  With rs within 2^-22.9 relative, the corrected root is
// within ~1.5 (2^-22.9)^2 = 2^-45.2 relative (the correction removes the first-order error).
template <class F>
GVX_HD F lc_sqrt(const F &x) {
  using V = lane_t<F>;
  const V rs = vrsqrt(x.hi);
  const V s = vmul(x.hi, rs);
  const V pp = vmul(s, s);
  const V pe = vfma(s, s, vneg(pp));
  const V res = vadd(vsub(vsub(x.hi, pp), pe), x.lo);
  return {s, vmul(res, vmul(rs, vbc(0.5f, V{})))};
}
// q / y, y.hi > 0: q1 = q.hi / y.hi from the approximate reciprocal, one correction from the
// float-float remainder.
template <class F>
GVX_HD F lc_div(const F &q, const F &y) {
  using V = lane_t<F>;
  const V ry = vrcp(y.hi);
  const V q1 = vmul(q.hi, ry);
  const V r0 = vfma(vneg(q1), y.hi, q.hi);
  const V r1 = vfma(vneg(q1), y.lo, vadd(r0, q.lo));
  return {q1, vmul(r1, ry)};
}
// The output's square root, x.hi > 0: rs refined by one Newton step first, so that the mass
// itself carries no error from the approximation.
GVX_HD ff lc_sqrt_refined(ff x) {
  float rs = rsqrt_mufu(x.hi);
  rs = ffma(fmul(rs, 0.5f), ffma(-x.hi, fmul(rs, rs), 1.0f), rs);
  const float s = fmul(x.hi, rs);
  const float pp = fmul(s, s);
  const float pe = ffma(s, s, -pp);
  const float res = fadd(fsub(fsub(x.hi, pp), pe), x.lo);
  return {s, fmul(res, fmul(rs, 0.5f))};
}

// ---- table-driven functions ----------------------------------------------------------------

// The Taylor parts at the reduced argument r (|r| <= 2^-9, r.lo small against r.hi), hs = s/2
// (s = +1 hyperbolic, -1 circular): Ce = 1 + p + c with p = s r.hi^2/2 rounded and c the rest
// (its rounding error, s r.hi r.lo, r^4/24); So = r.hi + so with so = r.lo + r (s r^2/6 +
// r^4/120) = r.lo + r.hi p (1/3 + p/30).
template <class V>
struct TabPoly {
  V p, c, so;
};
template <class F>
GVX_HD TabPoly<lane_t<F>> tab_poly(const F &r, lane_t<F> hs) {
  using V = lane_t<F>;
  const V h = vmul(r.hi, hs);          // s r.hi / 2 (exact)
  const V p = vmul(r.hi, h);           // s r.hi^2 / 2, rounded
  const V pe = vfma(r.hi, h, vneg(p));  // its rounding error (exact)
  V c = vfma(vadd(h, h), r.lo, pe);    // + s r.hi r.lo
  c = vfma(p, vmul(p, vbc(0.16666667f, V{})), c);  // + r^4 / 24 = p^2 / 6
  const V t = vmul(p, vfma(p, vbc(0.033333335f, V{}), vbc(0.33333334f, V{})));
  return {p, c, vfma(r.hi, t, r.lo)};
}
// A Ce + B So.  The three leading terms A.hi, B.hi r.hi and A.hi p are summed with exact
// two-products and Fast2Sum, which needs |A.hi| >= |B.hi r.hi| (or A = 0) and the first sum above
// A.hi p: true for cosh (A = cosh >= 1), for sinh at n >= 1 (tanh(n h) > h/2) and at n = 0
// (A = 0), and for sin(|d_phi|/2) at j = 0 and wherever |sin(j h)| >= 3 h/2 (every j outside
// the band around pi that the pair mass leaves to FP64).  The rest is collected in one float
// (each term below 2^-22 of the result).
template <class F>
GVX_HD F tab_comb(const F &A, const F &B, const F &r, const TabPoly<lane_t<F>> &q) {
  using V = lane_t<F>;
  const V a1 = vmul(A.hi, q.p);
  const V a1e = vfma(A.hi, q.p, vneg(a1));
  const V b1 = vmul(B.hi, r.hi);
  const V b1e = vfma(B.hi, r.hi, vneg(b1));
  const V s1 = vadd(A.hi, b1);
  const V e1 = vsub(b1, vsub(s1, A.hi));
  const V s2 = vadd(s1, a1);
  const V e2 = vsub(a1, vsub(s2, s1));
  V lo = vfma(A.hi, q.c, a1e);
  lo = vfma(B.hi, q.so, lo);
  lo = vfma(B.lo, r.hi, lo);
  lo = vfma(A.lo, q.p, lo);
  lo = vadd(lo, A.lo);
  lo = vadd(lo, b1e);
  lo = vadd(lo, vadd(e1, e2));
  return {s2, lo};
}
// The same without an ordering of A.hi and B.hi r.hi (TwoSum for the first sum): sin and cos
// of an arbitrary angle in [0, 3.5].
template <class F>
GVX_HD F tab_comb_any(const F &A, const F &B, const F &r, const TabPoly<lane_t<F>> &q) {
  using V = lane_t<F>;
  const V a1 = vmul(A.hi, q.p);
  const V a1e = vfma(A.hi, q.p, vneg(a1));
  const V b1 = vmul(B.hi, r.hi);
  const V b1e = vfma(B.hi, r.hi, vneg(b1));
  const V s1 = vadd(A.hi, b1);
  const V bb = vsub(s1, A.hi);
  const V e1 = vadd(vsub(A.hi, vsub(s1, bb)), vsub(b1, bb));
  const V s2 = vadd(s1, a1);
  const V bb2 = vsub(s2, s1);
  const V e2 = vadd(vsub(s1, vsub(s2, bb2)), vsub(a1, bb2));
  V lo = vfma(A.hi, q.c, a1e);
  lo = vfma(B.hi, q.so, lo);
  lo = vfma(B.lo, r.hi, lo);
  lo = vfma(A.lo, q.p, lo);
  lo = vadd(lo, A.lo);
  lo = vadd(lo, b1e);
  lo = vadd(lo, vadd(e1, e2));
  return {s2, lo};
}
template <class F>
GVX_HD F tab_eval(const F &A, const F &B, const F &r, lane_t<F> hs) {
  return tab_comb(A, B, r, tab_poly(r, hs));
}

constexpr float kLcMagic = 12582912.0f;   // 1.5 * 2^23: adding it rounds to an integer
constexpr uint32_t kLcMagicBits = 0x4B400000u;
constexpr float kLcStep = 0.00390625f;    // 2^-8
constexpr float kLcInvStep = 256.0f;

GVX_HD void lane_idx(float t, uint32_t *n) { n[0] = f2u(t) - kLcMagicBits; }
GVX_HD void lane_idx(f2 t, uint32_t *n) {
  n[0] = f2u(t.x) - kLcMagicBits;
  n[1] = f2u(t.y) - kLcMagicBits;
}

// x = n 2^-8 + r per lane, x >= 0 with x.lo in [0, ulp(x.hi)) (as the conversions give it): n is
// the nearest integer of 256 x.hi, x.hi - n 2^-8 is exact, and Fast2Sum adds x.lo (whenever that
// difference is nonzero it is at least ulp(x.hi) > x.lo).  n is returned unclamped.
template <class F>
GVX_HD F lc_reduce(const F &x, uint32_t *n) {
  using V = lane_t<F>;
  const V t = vfma(x.hi, vbc(kLcInvStep, V{}), vbc(kLcMagic, V{}));
  lane_idx(t, n);
  const V ra = vfma(vsub(t, vbc(kLcMagic, V{})), vbc(-kLcStep, V{}), x.hi);
  const V rh = vadd(ra, x.lo);
  return {rh, vsub(x.lo, vsub(rh, ra))};
}

// Table entries per lane, the index clamped for lanes outside the domain (NaN, |x| > 8), whose
// result is discarded.  first = components (x, y) of the entry, second = (z, w).
GVX_HD void tab_load(const gvx_f4 *tab, uint32_t nmax, const uint32_t *n, ff *first, ff *second) {
  const gvx_f4 t = ldtab(&tab[umin32(n[0], nmax)]);
  *first = {t.x, t.y};
  *second = {t.z, t.w};
}
GVX_HD void tab_load(const gvx_f4 *tab, uint32_t nmax, const uint32_t *n, ff2 *first, ff2 *second) {
  const gvx_f4 tx = ldtab(&tab[umin32(n[0], nmax)]);
  const gvx_f4 ty = ldtab(&tab[umin32(n[1], nmax)]);
  *first = {mk2(tx.x, ty.x), mk2(tx.y, ty.y)};
  *second = {mk2(tx.z, ty.z), mk2(tx.w, ty.w)};
}

// The light-cone terms of one leg or two (lanes), pt and m scaled to the pair's (or event's)
// power of two, x = |eta| < 8: P = pt cosh(eta), E = sqrt(P^2 + m^2), Y = E + P, D = m^2 / Y.
template <class F>
struct LcLeg {
  F P, E, Y, D;
};
// With sh (chp) given, also *sh = sinh(x) (*chp = cosh(x)), from the same reduction and entry.
template <class F>
GVX_HD LcLeg<F> lc_leg(const F &pt, const F &mm, const F &x, const gvx_f4 *hyp, F *sh = nullptr,
                       F *chp = nullptr) {
  using V = lane_t<F>;
  uint32_t n[2];
  const F r = lc_reduce(x, n);
  F C, Sh;
  tab_load(hyp, GVX_HYP_N, n, &C, &Sh);
  const TabPoly<V> tp = tab_poly(r, vbc(0.5f, V{}));
  const F ch = tab_comb(C, Sh, r, tp);
  if (sh) *sh = tab_comb(Sh, C, r, tp);
  if (chp) *chp = ch;
  const F q = lc_sqr(mm);
  LcLeg<F> l;
  l.P = lc_mul(pt, ch);
  l.E = lc_sqrt(lc_add(lc_sqr(l.P), q));
  l.Y = lc_add(l.E, l.P);
  l.D = lc_div(q, l.Y);
  return l;
}

// sin and cos of x in [0, 3.5] (x.lo in [0, ulp(x.hi))), absolute error ~2^-46.
GVX_HD void sincos_lc(const ff &x, const gvx_f4 *sintab, ff *sn, ff *cs) {
  uint32_t j[1];
  const ff r = lc_reduce(x, j);
  ff Sj, Cj;
  tab_load(sintab, GVX_SIN_N, j, &Sj, &Cj);
  const TabPoly<float> tp = tab_poly(r, -0.5f);
  *sn = tab_comb_any(Sj, Cj, r, tp);
  *cs = tab_comb_any(Cj, ff{-Sj.hi, -Sj.lo}, r, tp);
}

// ---- the pair ------------------------------------------------------------------------------

// The angular factor of a pair, S = sinh^2(|d_eta|/2) + sin^2(|d_phi|/2), from its raw angles,
// the two half-angle functions as the lanes of one paired table evaluation.  False when
// |d_phi|/2 is within 2^-7 of pi (there the FP64 rounding of phi1 - phi2 matters).
GVX_HD bool lc_pair_S(double eta1, double eta2, double phi1, double phi2, const LcTab &T, ff *S) {
  const double de = eta1 - eta2, dp = phi1 - phi2;  // FP64: exact where the legs are close
  const uint32_t hde = dhi(de) & 0x7fffffffu, hdp = dhi(dp) & 0x7fffffffu;
  const CvtParts cp = cvt_parts(hdp, dlo(dp), kRebaseHalf);
  const ff2 xa = cvt2(cvt_parts(hde, dlo(de), kRebaseHalf), cp);
  // |d_phi|/2 needs its last 6 bits too (at |d_phi| ~ 2 pi, sin is taken near pi where the
  // reduction's remainder r is small): lo3 = those bits as a float (0 or a denormal when
  // |d_phi|/2 is below 2^-80)
  const int32_t e3 = (int32_t)(cp.hb & 0x7f800000u) - (int32_t)(46u << 23);
  const uint32_t el3 = (uint32_t)(e3 > 0 ? e3 : 0);
  const float lo3 = fsub(u2f(el3 | ((dlo(dp) & 63u) << 17)), u2f(el3));
  uint32_t nj[2];
  ff2 r = lc_reduce(xa, nj);
  r.lo = add2(r.lo, mk2(0.0f, lo3));
  const gvx_f4 th = ldtab(&T.hyp[umin32(nj[0], GVX_HYP_N)]);
  const gvx_f4 ts = ldtab(&T.sin[umin32(nj[1], GVX_SIN_N)]);
  const ff2 A = {mk2(th.z, ts.x), mk2(th.w, ts.y)};
  const ff2 B = {mk2(th.x, ts.z), mk2(th.y, ts.w)};
  const ff2 w = lc_sqr(tab_eval(A, B, r, mk2(0.5f, -0.5f)));
  *S = lc_add(lane_x(w), lane_y(w));
  return nj[1] - 802u > 4u;  // |d_phi|/2 within 2^-7 of pi
}

// The scaled m^2 = (D1 + D2)(Y1 + Y2) + 4 pt1 pt2 S from the legs' scaled pt, Y and D; false
// when it is nonzero and below 2^-80 (where terms flushed below the float range could matter).
GVX_HD bool lc_pair_m2(ff pt1, ff pt2, ff Y1, ff Y2, ff D1, ff D2, ff S, ff *m2s) {
  const ff ta = lc_mul(lc_mul(pt1, pt2), S);
  *m2s = lc_add(lc_mul(lc_add(D1, D2), lc_add(Y1, Y2)), ff{fmul(ta.hi, 4.0f), fmul(ta.lo, 4.0f)});
  return m2s->hi >= 8.27180613e-25f || m2s->hi == 0.0f;  // 2^-80
}

// The scaled float-float m^2 of a pair and the scale exponent field; false outside the
// fast-path domain (then *m2s and *emax_w are meaningless).
GVX_HD bool pair_m2_lc(double pt1, double eta1, double phi1, double m1, double pt2, double eta2,
                       double phi2, double m2, const LcTab &T, ff *m2s, uint32_t *emax_w) {
  // -- domain and the common scale of pt and m (high words; pt's sign bit fails the range) --
  const uint32_t hp1 = dhi(pt1), hp2 = dhi(pt2);
  const uint32_t hm1 = dhi(m1) & 0x7fffffffu, hm2 = dhi(m2) & 0x7fffffffu;
  const uint32_t wmax = umax32(umax32(hp1, hm1), umax32(hp2, hm2));
  const uint32_t ew = wmax & 0x7ff00000u;
  // every nonzero value's exponent >= emax - 40 (exponent field 0 counts as zero)
  const uint32_t vmin_ = umin32(umin32(hp1 - 0x100000u, hm1 - 0x100000u),
                                umin32(hp2 - 0x100000u, hm2 - 0x100000u));
  const uint32_t he1 = dhi(eta1) & 0x7fffffffu, he2 = dhi(eta2) & 0x7fffffffu;
  const uint32_t hf1 = dhi(phi1) & 0x7fffffffu, hf2 = dhi(phi2) & 0x7fffffffu;
  const bool ok = wmax - (200u << 20) < (1700u << 20) && vmin_ >= ew - (41u << 20) &&
                  umin32(umax32(hp1, hm1), umax32(hp2, hm2)) >= 0x100000u &&  // no zero leg
                  umax32(he1, he2) < 0x40200000u && umax32(hf1, hf2) < 0x400C0000u;
  *emax_w = ew;
  // -- the angular factor first: the raw angles are then dead during the legs --
  ff S;
  const bool oks = lc_pair_S(eta1, eta2, phi1, phi2, T, &S);
  // -- the legs (lane x: leg 1, lane y: leg 2), pt and m scaled by 2^(1023 - emax) --
  const uint32_t rb = ew - (127u << 20);
  const ff2 pt = cvt2(cvt_parts(hp1, dlo(pt1), rb), cvt_parts(hp2, dlo(pt2), rb));
  const ff2 mm = cvt2(cvt_parts(hm1, dlo(m1), rb), cvt_parts(hm2, dlo(m2), rb));
  // |eta| below 2^-30 is raised to [2^-30, 2^-29): cosh changes by less than 2^-58
  const ff2 x = cvt2(cvt_parts_normal(umax32(he1, 0x3E100000u), dlo(eta1), kRebaseOne),
                     cvt_parts_normal(umax32(he2, 0x3E100000u), dlo(eta2), kRebaseOne));
  const LcLeg<ff2> L = lc_leg(pt, mm, x, T.hyp);
  return lc_pair_m2(lane_x(pt), lane_y(pt), lane_x(L.Y), lane_y(L.Y), lane_x(L.D), lane_y(L.D),
                    S, m2s) && ok && oks;
}

// m = sqrt(m2s) * 2^(e - 1023), e the scale's exponent (field ew = e << 20), as a double: the
// leading float placed by bits, the trailing one likewise (or 0 when it is zero, denormal or
// below 2^-60 of the leading one), one FP64 add.  The domain keeps the exponents in range.
// ff times 2^shift -> double: hi and lo each moved exactly to double by their bits (integer
// operations), then one FP64 addition (one rounding of the exact sum).  eoff = (896 + shift) << 20
// moves the float exponent field to the double one.  hi normal or 0; a denormal lo counts as 0;
// the result must lie in the normal range of double.
GVX_HD double lc_to_double(const ff &x, uint32_t eoff) {
  const uint32_t hb = f2u(x.hi), lb = f2u(x.lo);
  const uint32_t ah = hb & 0x7fffffffu, al = lb & 0x7fffffffu;
  const double dh = hilo2d(ah >= 0x800000u ? ((ah >> 3) + eoff) | (hb & 0x80000000u) : 0u, hb << 29);
  const double dl = hilo2d(al >= 0x800000u ? ((al >> 3) + eoff) | (lb & 0x80000000u) : 0u, lb << 29);
  return dh + dl;
}

GVX_HD double lc_mass_out(ff m2s, uint32_t ew) {
  if (m2s.hi == 0.0f) return 0.0;
  const ff m = lc_sqrt_refined(m2s);
  const uint32_t eoff = ew - (127u << 20);  // float exponent f -> double exponent f + e - 127
  const uint32_t hb = f2u(m.hi), lb = f2u(m.lo), lm = lb & 0x7fffffffu;
  const double dh = hilo2d((hb >> 3) + eoff, hb << 29);
  const double dl = lm + (60u << 23) >= hb
                        ? hilo2d(((lm >> 3) + eoff) | (lb & 0x80000000u), lm << 29)
                        : 0.0;
  return dh + dl;
}

// A normalized ff (|lo| at most half an ulp of hi; hi normal or 0) times 2^shift -> double with
// integer operations only (no FP64 instruction): hi exactly plus lo truncated to hi's double ulp,
// an error below one ulp of the result.  eoff = (896 + shift) << 20 moves the float exponent
// field to the double one.  With hi a power of two and lo of the other sign the result lies in
// the binade below, whose ulp is half hi's: lo is then taken to one more bit.  A denormal lo
// counts as 0.  The result must lie in the normal range of double; a zero or denormal hi gives 0.
GVX_HD double lc_to_double_int(const ff &x, uint32_t eoff) {
  const uint32_t hb = f2u(x.hi), lb = f2u(x.lo);
  const uint32_t ah = hb & 0x7fffffffu, al = lb & 0x7fffffffu;
  const uint32_t sub = (hb ^ lb) >> 31;
  const uint32_t fix = sub & (uint32_t)((ah & 0x7fffffu) == 0u);
  // lo in units of hi's double ulp (of the ulp below for fix): (ml 2^6) 2^-(eh - el - 23 - fix)
  const uint32_t ml = al >= 0x800000u ? ((al & 0x7fffffu) | 0x800000u) : 0u;
  const uint32_t sh = umin32((ah >> 23) - (al >> 23) - 23u - fix, 31u);
  const uint32_t L = (ml << 6) >> sh;
  const uint64_t base = ((uint64_t)((((ah >> 3) + eoff) | (hb & 0x80000000u))) << 32) |
                        (uint64_t)(hb << 29);
  const uint64_t r = sub ? base - L : base + L;
  return ah >= 0x800000u ? u2d(r) : 0.0;
}

// lc_mass_out without its FP64 addition: the refined root renormalized (Fast2Sum) and assembled
// by lc_to_double_int (truncation below one ulp of the double).  For kernels whose FP64 pipe is
// the scarce one (the jagged pair masses).
GVX_HD double lc_mass_out_int(ff m2s, uint32_t ew) {
  if (m2s.hi == 0.0f) return 0.0;
  const ff m = lc_sqrt_refined(m2s);
  return lc_to_double_int(fast_two_sum(m.hi, m.lo), ew - (127u << 20));
}

// Returns false (and leaves *out untouched) outside the fast-path domain.
GVX_HD bool pair_mass_lc(double pt1, double eta1, double phi1, double m1, double pt2, double eta2,
                         double phi2, double m2, const LcTab &T, double *out) {
  ff m2s;
  uint32_t ew;
  if (!pair_m2_lc(pt1, eta1, phi1, m1, pt2, eta2, phi2, m2, T, &m2s, &ew)) return false;
  *out = lc_mass_out(m2s, ew);
  return true;
}


}  // namespace ffm
}  // namespace gvx
