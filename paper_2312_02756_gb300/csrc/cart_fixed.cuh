// Pair mass of PxPyPzE legs in exact fixed-point integer arithmetic: the fast path of the
// Cartesian-input mass kernels (the mass kernel of Sec. 4.1 on the PxPyPzE system of Sec. 3.1).
//
// The plain definition m^2 = (E1 + E2)^2 - (px1 + px2)^2 - (py1 + py2)^2 - (pz1 + pz2)^2 cancels
// catastrophically in floating point for light, collinear pairs.  Here the eight components are
// scaled by the power of two 2^-s that brings the largest magnitude into [1, 2) and truncated to
// signed integers in units of 2^-90 (magnitudes below 2^91), so the four component sums are
// exact.  Each sum is squared with 64-bit limb products and kept, truncated, in units of 2^-116;
// the signed total fits a 128-bit integer.  The only errors are the two truncations: in scaled
// units |error of m^2| < 4 (2 * 2 * 2 * 2^-90 + 2^-116) < 2^-84.  The result is kept when
// |m^2| >= 2^-38 (scaled), i.e. with relative error below 2^-46; it is rounded to float-float (47
// bits), its square root taken in float-float, and scaled back: the relative error of m is
// below 2^-44.  Integer and FP32 pipes only, plus one FP64 add for the final rounding (none for
// FP32 output).
//
// Outside the fast path (a non-finite component, a scale exponent outside [-900, 900] for double
// or [-100, 100] for float input, or |m^2| below the threshold, zero included) the functions
// return false and the caller evaluates the cancellation-free FP64 form.
#pragma once

#include "ff.cuh"

namespace gvx {
namespace cfix {

using ffm::ff;
typedef unsigned __int128 u128;
typedef __int128 i128;

constexpr int kFrac = 90;                // input units: 2^-90 of the scale
constexpr int kM2Units = 2 * kFrac - 64;  // m^2 units: 2^-116
constexpr int kMinLead = kM2Units - 38;   // |m^2| >= 2^-38: leading bit at or above 78

GVX_HD uint64_t mul64hi(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((u128)a * b) >> 64);
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

// x * 2^(kFrac - sc), truncated toward zero, for the largest biased exponent emax of the pair
// (sc = emax - bias, so |x| 2^-sc < 2).  x = sig * 2^(e - bias - kSig), hence the shift
// k = e - emax + kFrac - kSig <= kFrac - kSig.
template <typename T>
GVX_HD i128 to_fixed(const Decoded &d, int emax) {
  const int k = d.e - emax + kFrac - Fmt<T>::kSig;
  u128 v;
  if (d.e == 0 || k <= -(Fmt<T>::kSig + 1)) {
    v = 0;
  } else if (k >= 0) {
    v = (u128)d.sig << k;
  } else {
    v = (u128)(d.sig >> -k);
  }
  return d.neg ? -(i128)v : (i128)v;
}

// floor(S^2 / 2^64) for |S| < 2^92: with |S| = h 2^64 + l (h < 2^28),
// S^2 / 2^64 = h^2 2^64 + 2 h l + l^2 / 2^64.
GVX_HD u128 square_shift64(i128 S) {
  const u128 U = S < 0 ? (u128)(-S) : (u128)S;
  const uint32_t h = (uint32_t)(U >> 64);
  const uint64_t l = (uint64_t)U;
  return ((u128)((uint64_t)h * h) << 64) + (mul32x64(h, l) << 1) + mul64hi(l, l);
}

// The scaled m^2 (units 2^-116) of two PxPyPzE legs and the scale exponent sc; false when a
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
  i128 acc = 0;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const i128 S = to_fixed<T>(d[k], emax) + to_fixed<T>(d[k + 4], emax);
    const u128 q = square_shift64(S);
    acc = k == 3 ? acc + (i128)q : acc - (i128)q;  // components 0..2 are p, 3 is E
  }
  *m2 = acc;
  *sc = s;
  return true;
}

// |q| * 2^-116 as ff, truncated to 47 bits, for q with its leading bit p in [78, 121].
GVX_HD ff fixed_to_ff(u128 q, int p) {
  const uint64_t t = (uint64_t)(q >> (p - 46));  // 47 bits, leading 1 at bit 46
  const uint32_t top = (uint32_t)(t >> 23);       // leading 1 at bit 23 (implicit in hi)
  const uint32_t rest = (uint32_t)t & 0x7fffffu;
  const uint32_t eh = (uint32_t)(p - kM2Units + 127);  // biased exponent of hi: 2^(p - 116)
  const float hi = ffm::u2f((eh << 23) | (top & 0x7fffffu));
  const uint32_t base = (eh - 23u) << 23;  // 2^(p - 139): the rest has weight 2^(p - 162)
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
// power-of-two scaling: the scaled mass lies in [2^-19, 2^3) and |sc| <= 100).
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

}  // namespace cfix
}  // namespace gvx
