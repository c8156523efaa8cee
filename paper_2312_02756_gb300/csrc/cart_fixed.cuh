// Pair mass of PxPyPzE legs in exact fixed-point integer arithmetic: the fast path of the
// Cartesian-input mass kernels (the mass kernel of Sec. 4.1 on the PxPyPzE system of Sec. 3.1).
//
// The plain definition m^2 = (E1 + E2)^2 - (px1 + px2)^2 - (py1 + py2)^2 - (pz1 + pz2)^2 cancels
// catastrophically in floating point for light, collinear pairs.  Here the eight components are
// scaled by the power of two 2^-sc that brings the largest magnitude into [1, 2) and truncated to
// integers in units of 2^-83 (magnitudes below 2^84, three 32-bit words), so the four component
// sums are exact.  Each sum is squared from 32-bit limb products (IMADs) and kept, truncated, in
// units of 2^-102; the signed total fits a 128-bit integer.  The only errors are the
// truncations: in scaled units |error of m^2| < 4 (2 * 4 * 2^-82 + 3 * 2^-102) < 2^-76.9.  The
// result is kept when |m^2| >= 2^-31 (scaled), i.e. with relative error below 2^-45.9; it is then
// rounded to float-float (47 bits), its square root taken in float-float, and scaled back: the
// relative error of m is below 2^-44.  Integer and FP32 pipes only, plus one FP64 add for the
// final rounding (none for FP32 output).
//
// Outside the fast path (a non-finite component, a scale exponent outside [-900, 900] for double
// or [-100, 100] for float input, or |m^2| below the threshold, zero included) the functions
// return false and the caller evaluates the cancellation-free FP64 form.
#pragma once

#include "ff.cuh"
#include "mass_ff2.cuh"

namespace gvx {
namespace cfix {

using ffm::ff;
typedef unsigned __int128 u128;
typedef __int128 i128;

constexpr int kFrac = 83;                 // input units: 2^-83 of the scale
constexpr int kM2Units = 2 * kFrac - 64;   // m^2 units: 2^-102
constexpr int kMinLead = kM2Units - 31;    // |m^2| >= 2^-31: leading bit at or above 71

GVX_HD uint32_t mul32hi(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// a * b for a < 2^32, as a 128-bit integer (two 32 x 32 -> 64 products).
GVX_HD u128 mul32x64(uint32_t a, uint64_t b) {
  const uint64_t lo = (uint64_t)a * (uint32_t)b;
  const uint64_t hi = (uint64_t)a * (uint32_t)(b >> 32);
  return ((u128)hi << 32) + lo;
}

// Biased exponent field and integer significand of a double or a float (0 for zero and
// denormals, whose magnitude is far below the resolution wherever the scale passes).
struct Decoded {
  uint64_t sig;
  int e;
  bool neg;
};

GVX_HD Decoded decode(double x) {
  const uint32_t wh = ffm::dhi(x), wl = ffm::dlo(x);
  const int e = (int)((wh >> 20) & 0x7ffu);
  return {((uint64_t)((wh & 0xfffffu) | 0x100000u) << 32) | wl, e, (wh >> 31) != 0};
}

GVX_HD Decoded decode(float x) {
  const uint32_t u = ffm::f2u(x);
  const int e = (int)((u >> 23) & 0xffu);
  return {(uint64_t)((u & 0x7fffffu) | 0x800000u), e, (u >> 31) != 0};
}

// Format constants: kSig = significand bits - 1 (the exponent of the integer significand's top
// bit), kBias, kMaxE (the Inf/NaN exponent), kScaleLim (allowed |scale exponent|).
template <typename T>
struct Fmt;
template <>
struct Fmt<double> {
  static constexpr int kSig = 52, kBias = 1023, kMaxE = 0x7ff, kScaleLim = 900;
};
template <>
struct Fmt<float> {
  static constexpr int kSig = 23, kBias = 127, kMaxE = 0xff, kScaleLim = 100;
};

// |x| * 2^(kFrac - sc), truncated, for the largest biased exponent emax of the pair (sc = emax -
// bias, so |x| 2^-sc < 2): x = sig * 2^(e - bias - kSig), so the significand moves left by
// k = e - emax + kFrac - kSig (at most 31 for double, 60 for float) or right by -k.
template <typename T>
GVX_HD u128 align(const Decoded &d, int emax) {
  const int k = d.e == 0 ? -64 : d.e - emax + kFrac - Fmt<T>::kSig;
  if (k < 0) return (u128)(k > -64 ? d.sig >> -k : 0);
  if (sizeof(T) == 8) {  // k <= 31: the low 64 bits and the top word separately
    const uint32_t top = k ? (uint32_t)(d.sig >> 32) >> (32 - k) : 0u;
    return ((u128)top << 64) | (uint64_t)(d.sig << k);
  }
  return (u128)d.sig << k;  // float: a 24-bit significand, k <= 60
}

// |a +- b| for magnitudes a, b < 2^84 with signs na, nb: their sum or their difference.
GVX_HD u128 abs_sum(u128 a, bool na, u128 b, bool nb) {
  if (na == nb) return a + b;
  return a >= b ? a - b : b - a;
}

// floor-ish(U^2 / 2^64) for U < 2^85, within 3 units: with U = h 2^64 + l1 2^32 + l0,
// U^2 / 2^64 = h^2 2^64 + 2 h (l1 2^32 + l0) + l1^2 + 2 l1 l0 / 2^32 + l0^2 / 2^64, the last term
// dropped and the one before it truncated.
GVX_HD u128 square_shift64(u128 U) {
  const uint32_t h = (uint32_t)(U >> 64), l1 = (uint32_t)((uint64_t)U >> 32), l0 = (uint32_t)U;
  return ((u128)((uint64_t)h * h) << 64) + mul32x64(2u * h, (uint64_t)U) +
         ((uint64_t)l1 * l1 + 2ull * mul32hi(l1, l0));
}

// The scaled m^2 (units 2^-102) of two PxPyPzE legs and the scale exponent sc; false when a
// component is not finite or sc is out of range.
template <typename T>
GVX_HD bool m2_fixed(const T *a, const T *b, i128 *m2, int *sc) {
  Decoded d[8];
  int emax = 0;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    d[k] = decode(a[k]);
    d[k + 4] = decode(b[k]);
  }
#pragma unroll
  for (int k = 0; k < 8; k++) emax = d[k].e > emax ? d[k].e : emax;
  const int s = emax - Fmt<T>::kBias;
  if (emax == Fmt<T>::kMaxE || s < -Fmt<T>::kScaleLim || s > Fmt<T>::kScaleLim) return false;
  u128 pos = 0, neg = 0;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const u128 q = square_shift64(
        abs_sum(align<T>(d[k], emax), d[k].neg, align<T>(d[k + 4], emax), d[k + 4].neg));
    if (k == 3) pos = q;  // components 0..2 are p, 3 is E
    else neg += q;
  }
  *m2 = (i128)pos - (i128)neg;
  *sc = s;
  return true;
}

// |q| * 2^-102 as ff, truncated to 47 bits, for q with its leading bit p in [71, 107].
GVX_HD ff fixed_to_ff(u128 q, int p) {
  const uint64_t t = (uint64_t)(q >> (p - 46));  // 47 bits, leading 1 at bit 46
  const uint32_t top = (uint32_t)(t >> 23);       // leading 1 at bit 23 (implicit in hi)
  const uint32_t rest = (uint32_t)t & 0x7fffffu;
  const uint32_t eh = (uint32_t)(p - kM2Units + 127);  // biased exponent of hi: 2^(p - 102)
  const float hi = ffm::u2f((eh << 23) | (top & 0x7fffffu));
  const uint32_t base = (eh - 23u) << 23;  // 2^(p - 125): the rest has weight 2^(p - 148)
  return {hi, ffm::fsub(ffm::u2f(base | rest), ffm::u2f(base))};
}

// sqrt(|m^2|) in ff (scaled) with the sign of m^2; false below the threshold.
GVX_HD bool mass_scaled(i128 m2, ff *m, bool *neg) {
  *neg = m2 < 0;
  const u128 q = *neg ? (u128)(-m2) : (u128)m2;
  const uint64_t top = (uint64_t)(q >> 64);
  if (top < ((uint64_t)1 << (kMinLead - 64))) return false;
#if defined(__CUDA_ARCH__)
  const int p = 127 - __clzll((long long)top);
#else
  const int p = 127 - __builtin_clzll(top);
#endif
  *m = ffm::sqrt(fixed_to_ff(q, p));
  return true;
}

// Pair mass of two FP64 PxPyPzE legs (m = -sqrt(-m^2) for a spacelike sum); false outside the
// fast path.
GVX_HD bool mass_pxpypze(const double *a, const double *b, double *out) {
  i128 m2;
  int sc;
  ff m;
  bool neg;
  if (!m2_fixed<double>(a, b, &m2, &sc) || !mass_scaled(m2, &m, &neg)) return false;
  const double r = ffm::to_double(m, sc);
  *out = neg ? -r : r;
  return true;
}

// The same for FP32 legs, rounded once to float (hi + lo in one float add, then an exact
// power-of-two scaling: the scaled mass lies in [2^-16, 2^3) and |sc| <= 100).
GVX_HD bool mass_pxpypze(const float *a, const float *b, float *out) {
  i128 m2;
  int sc;
  ff m;
  bool neg;
  if (!m2_fixed<float>(a, b, &m2, &sc) || !mass_scaled(m2, &m, &neg)) return false;
  const float r = ffm::fmul(ffm::fadd(m.hi, m.lo), ffm::pow2f(sc));
  *out = neg ? -r : r;
  return true;
}

// ---- PxPyPzM legs ----------------------------------------------------------------------------
// With the mass stored, E_i = sqrt(P_i^2 + m_i^2) is not a stored number, and
//   m^2 = m1^2 + m2^2 + 2 (E1 E2 - p1.p2),
//   E1 E2 - p1.p2 = (|p1 x p2|^2 + m1^2 P2^2 + m2^2 P1^2 + m1^2 m2^2) / (E1 E2 + p1.p2)   (p1.p2 > 0)
//                 = E1 E2 + |p1.p2|                                                        (otherwise),
// the numerator being E1^2 E2^2 - (p1.p2)^2 by Lagrange's identity.  Every term is non-negative
// and the only cancelling quantities are the components of p1 x p2: those come from the
// fixed-point limb products (components truncated to units of 2^-83 of their leg's scale, the
// products kept to units of 2^-102 of 2^(s1 + s2)); P_i^2, m_i^2 and p1.p2 (which only ever
// enters next to E1 E2) are float-float arithmetic on the scaled components, like the rest.
// Each leg has its own power-of-two scale 2^s_i: an absolute error in m_i^2 reaches m^2
// multiplied by about E_o / E_i, so the resolution must follow each leg.  In units of the larger
// leg's squared scale H the fixed-point errors stay below 2^-76; the result is kept when
// m^2 >= 2^-31 H, so its relative error (with the float-float steps) is below 2^-43.
// Domain: both legs finite with scale exponents within half the format's limit and at most 60
// apart.

// (A B) / 2^64 for magnitudes A, B < 2^85, within 4 units: with A = ah 2^64 + a1 2^32 + a0,
// A B / 2^64 = ah bh 2^64 + ah (b1 2^32 + b0) + bh (a1 2^32 + a0) + a1 b1 + (a1 b0 + a0 b1) / 2^32
// + a0 b0 / 2^64, the last term dropped and the one before it truncated term by term.
GVX_HD u128 mul_shift64(u128 A, u128 B) {
  const uint32_t ah = (uint32_t)(A >> 64), a1 = (uint32_t)((uint64_t)A >> 32), a0 = (uint32_t)A;
  const uint32_t bh = (uint32_t)(B >> 64), b1 = (uint32_t)((uint64_t)B >> 32), b0 = (uint32_t)B;
  return ((u128)((uint64_t)ah * bh) << 64) + mul32x64(ah, (uint64_t)B) + mul32x64(bh, (uint64_t)A) +
         ((uint64_t)a1 * b1 + mul32hi(a1, b0) + mul32hi(a0, b1));
}

// |q| * 2^-102 as ff (truncated to 47 bits), for any q < 2^112; 0 gives 0.
GVX_HD ff fixed_to_ff_any(u128 q) {
  const uint64_t hi64 = (uint64_t)(q >> 64), lo64 = (uint64_t)q;
  if ((hi64 | lo64) == 0) return {0.0f, 0.0f};
#if defined(__CUDA_ARCH__)
  const int p = hi64 ? 127 - __clzll((long long)hi64) : 63 - __clzll((long long)lo64);
#else
  const int p = hi64 ? 127 - __builtin_clzll(hi64) : 63 - __builtin_clzll(lo64);
#endif
  const uint64_t t = p >= 46 ? (uint64_t)(q >> (p - 46)) : lo64 << (46 - p);
  const uint32_t top = (uint32_t)(t >> 23), rest = (uint32_t)t & 0x7fffffu;
  const uint32_t eh = (uint32_t)(p - kM2Units + 127);  // >= 25
  const float hi = ffm::u2f((eh << 23) | (top & 0x7fffffu));
  const uint32_t base = (eh - 23u) << 23;
  return {hi, ffm::fsub(ffm::u2f(base | rest), ffm::u2f(base))};
}

// x 2^-s as ff: a double through the ranged conversion (below 2^-74 counts as 0), a float exactly.
GVX_HD ff scaled_ff(double x, int s) { return ffm::from_double_ranged(x, s); }
GVX_HD ff scaled_ff(float x, int s) { return {ffm::fmul(x, ffm::pow2f(-s)), 0.0f}; }

// |component of p1 x p2| = |s_a A - s_b B| for the magnitudes A, B of the two products.
GVX_HD ff cross_component(u128 A, bool na, u128 B, bool nb) {
  return fixed_to_ff_any(abs_sum(A, na, B, !nb));
}

// The scaled mass sqrt(m^2 / 2^(2 e)) in ff and the exponent e of the pair mass of two PxPyPzM
// legs; false outside the fast path.
template <typename T>
GVX_HD bool mass_pxpypzm_scaled(const T *a, const T *b, ff *m, int *e_out) {
  Decoded d[8];
  int e1 = 0, e2 = 0;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    d[k] = decode(a[k]);
    d[k + 4] = decode(b[k]);
    e1 = d[k].e > e1 ? d[k].e : e1;
    e2 = d[k + 4].e > e2 ? d[k + 4].e : e2;
  }
  const int s1 = e1 - Fmt<T>::kBias, s2 = e2 - Fmt<T>::kBias;
  const int lim = Fmt<T>::kScaleLim / 2;
  if (e1 == Fmt<T>::kMaxE || e2 == Fmt<T>::kMaxE || s1 < -lim || s1 > lim || s2 < -lim || s2 > lim ||
      s1 - s2 > 60 || s2 - s1 > 60)
    return false;
  using namespace ffm;
  // |p1 x p2| components from exact limb products (scale 2^(s1 + s2))
  u128 A[3], B[3];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    A[k] = align<T>(d[k], e1);
    B[k] = align<T>(d[k + 4], e2);
  }
  const ff cx = cross_component(mul_shift64(A[1], B[2]), d[1].neg != d[6].neg,
                                mul_shift64(A[2], B[1]), d[2].neg != d[5].neg);
  const ff cy = cross_component(mul_shift64(A[2], B[0]), d[2].neg != d[4].neg,
                                mul_shift64(A[0], B[2]), d[0].neg != d[6].neg);
  const ff cz = cross_component(mul_shift64(A[0], B[1]), d[0].neg != d[5].neg,
                                mul_shift64(A[1], B[0]), d[1].neg != d[4].neg);
  // the rest in ff on the scaled components; the per-leg quantities |p_i|^2, m_i^2 and E_i^2
  // of both legs on paired FP32 operations (mass_ff2.cuh: lane x leg 1, lane y leg 2, each lane
  // the scalar operations' bits)
  ff2 v[4];
#pragma unroll
  for (int k = 0; k < 4; k++) v[k] = pack(scaled_ff(a[k], s1), scaled_ff(b[k], s2));
  const ff2 PP = add_same(add_same(sqr(v[0]), sqr(v[1])), sqr(v[2]));
  const ff2 qq = sqr(v[3]);
  const ff2 EE = add_same(PP, qq);
  const ff P1 = lane_x(PP), P2 = lane_y(PP), q1 = lane_x(qq), q2 = lane_y(qq);
  const ff dot = add(add(mul(lane_x(v[0]), lane_y(v[0])), mul(lane_x(v[1]), lane_y(v[1]))),
                     mul(lane_x(v[2]), lane_y(v[2])));
  const ff E1E2 = ffm::sqrt(mul(lane_x(EE), lane_y(EE)));  // scale 2^(s1 + s2)
  ff T2;
  if (dot.hi > 0.0f) {
    const ff c2 = add_same(add_same(sqr(cx), sqr(cy)), sqr(cz));
    const ff N = add_same(add_same(c2, mul(q1, P2)), add_same(mul(q2, P1), mul(q1, q2)));
    T2 = scale(div(N, add_same(E1E2, dot)), 2.0f);
  } else {
    T2 = scale(add_same(E1E2, neg(dot)), 2.0f);
  }
  // m^2 / 2^(s1 + s2) = q1 2^(s1 - s2) + q2 2^(s2 - s1) + 2 T; an odd s1 + s2 moves one factor 2
  // inside the root
  const int odd = (s1 + s2) & 1;
  const ff m2 = renorm(add_same(add_same(scale(q1, pow2f(s1 - s2 + odd)), scale(q2, pow2f(s2 - s1 + odd))),
                                scale(T2, odd ? 2.0f : 1.0f)));
  // threshold: m^2 >= 2^-31 2^(2 max(s1, s2)), i.e. the scaled value >= 2^(|s1 - s2| - 31 + odd)
  const int gap = s1 > s2 ? s1 - s2 : s2 - s1;
  if (!(m2.hi >= pow2f(gap - 31 + odd))) return false;
  *m = ffm::sqrt(m2);
  *e_out = (s1 + s2 - odd) / 2;
  return true;
}

GVX_HD bool mass_pxpypzm(const double *a, const double *b, double *out) {
  ff m;
  int e;
  if (!mass_pxpypzm_scaled(a, b, &m, &e)) return false;
  *out = ffm::to_double(m, e);
  return true;
}

GVX_HD bool mass_pxpypzm(const float *a, const float *b, float *out) {
  ff m;
  int e;
  if (!mass_pxpypzm_scaled(a, b, &m, &e)) return false;
  *out = ffm::fmul(ffm::fadd(m.hi, m.lo), ffm::pow2f(e));
  return true;
}

}  // namespace cfix
}  // namespace gvx
