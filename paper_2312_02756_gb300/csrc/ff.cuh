// Float-float ("double-float") arithmetic: the FP64 kernels' arithmetic on the FP32 pipe.
//
// A GB300 SM issues 128 FP32 FMAs per clock but only ~1.6 FP64 operations, so an FP64 kernel
// that keeps its transcendentals on the FP64 pipe runs ~20x slower than the memory system.  An
// ff value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2 (48 significand
// bits, relative precision ~2^-47 per operation), built from the error-free transformations
// TwoSum / Fast2Sum (Knuth; Dekker) and TwoProduct via FMA.  Conversions between double and ff,
// and exact differences of doubles, are done with integer bit manipulation (the F2F conversion
// instructions run on the FP64 pipe).  Range: the exponent range of float; callers scale their
// inputs and route anything outside the documented ranges to an FP64 path.
//
// The functions here are __host__ __device__ so the test suite can also run them on the CPU.
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define GVX_HD __host__ __device__ __forceinline__
#else
#define GVX_HD static inline
#endif

namespace gvx {
namespace ffm {

struct ff {
  float hi, lo;
};

// ---- single roundings that must not be contracted into FMAs ------------------------------

GVX_HD float fadd(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
GVX_HD float fsub(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
GVX_HD float fmul(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
GVX_HD float ffma(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(a, b, c);
#else
  return fmaf(a, b, c);
#endif
}
// a / b to within a couple of ulps (the callers correct the quotient in ff).
GVX_HD float fdiv_approx(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fdividef(a, b);
#else
  return a / b;
#endif
}
// 1/sqrt(a) to within a couple of ulps, a > 0.
GVX_HD float frsqrt_approx(float a) {
#if defined(__CUDA_ARCH__)
  return rsqrtf(a);
#else
  return 1.0f / sqrtf(a);
#endif
}

GVX_HD uint32_t f2u(float f) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(f);
#else
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
#endif
}
GVX_HD float u2f(uint32_t u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}
GVX_HD uint64_t d2u(double d) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t u;
  memcpy(&u, &d, 8);
  return u;
#endif
}
GVX_HD double u2d(uint64_t u) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)u);
#else
  double d;
  memcpy(&d, &u, 8);
  return d;
#endif
}
GVX_HD float i2f(int32_t i) {
#if defined(__CUDA_ARCH__)
  return __int2float_rn(i);
#else
  return (float)i;
#endif
}
GVX_HD int clz64(uint64_t x) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

// 2^k as a float, -126 <= k <= 127.
GVX_HD float pow2f(int k) { return u2f((uint32_t)(k + 127) << 23); }

// ---- error-free transformations -----------------------------------------------------------

GVX_HD ff two_sum(float a, float b) {
  float s = fadd(a, b);
  float bb = fsub(s, a);
  float e = fadd(fsub(a, fsub(s, bb)), fsub(b, bb));
  return {s, e};
}
// requires exponent(a) >= exponent(b) (e.g. |a| >= |b|)
GVX_HD ff fast_two_sum(float a, float b) {
  float s = fadd(a, b);
  return {s, fsub(b, fsub(s, a))};
}
GVX_HD ff two_prod(float a, float b) {
  float p = fmul(a, b);
  return {p, ffma(a, b, -p)};
}

// ---- ff arithmetic --------------------------------------------------------------------------

GVX_HD ff make(float x) { return {x, 0.0f}; }
GVX_HD ff neg(ff x) { return {-x.hi, -x.lo}; }
// exact scaling by a power of two
GVX_HD ff scale(ff x, float p2) { return {fmul(x.hi, p2), fmul(x.lo, p2)}; }

// x + y, accurate also under cancellation (relative error ~2^-47 of the result)
GVX_HD ff add(ff x, ff y) {
  ff s = two_sum(x.hi, y.hi);
  ff t = two_sum(x.lo, y.lo);
  s = fast_two_sum(s.hi, fadd(s.lo, t.hi));
  return fast_two_sum(s.hi, fadd(s.lo, t.lo));
}
// x + y for operands of the same sign (no cancellation): cheaper, same accuracy there
GVX_HD ff add_same(ff x, ff y) {
  ff s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, fadd(s.lo, fadd(x.lo, y.lo)));
}
// ff + float of the same sign
GVX_HD ff add_same_f(ff x, float y) {
  ff s = two_sum(x.hi, y);
  return fast_two_sum(s.hi, fadd(s.lo, x.lo));
}
GVX_HD ff mul(ff x, ff y) {
  ff p = two_prod(x.hi, y.hi);
  float e = ffma(x.hi, y.lo, p.lo);
  e = ffma(x.lo, y.hi, e);
  return fast_two_sum(p.hi, e);
}
GVX_HD ff mul_f(ff x, float f) {
  ff p = two_prod(x.hi, f);
  return fast_two_sum(p.hi, ffma(x.lo, f, p.lo));
}
GVX_HD ff sqr(ff x) {
  ff p = two_prod(x.hi, x.hi);
  return fast_two_sum(p.hi, ffma(fadd(x.hi, x.hi), x.lo, p.lo));
}
// x / y, y != 0: approximate quotient q1, then two corrections from ff remainders.
GVX_HD ff div(ff x, ff y) {
  float q1 = fdiv_approx(x.hi, y.hi);
  ff r = add(x, neg(mul_f(y, q1)));
  ff q = fast_two_sum(q1, fdiv_approx(r.hi, y.hi));
  ff r2 = add(x, neg(mul(y, q)));
  return fast_two_sum(q.hi, fadd(q.lo, fdiv_approx(r2.hi, y.hi)));
}
// sqrt(x), x >= 0: s = x.hi * rsqrt(x.hi), then one correction with the ff residual x - s^2.
GVX_HD ff sqrt(ff x) {
  if (!(x.hi > 0.0f)) return {0.0f, 0.0f};
  float rs = frsqrt_approx(x.hi);
  float s = fmul(x.hi, rs);
  ff p = two_prod(s, s);
  ff r = add(x, neg(p));
  float c = fmul(fmul(r.hi, rs), 0.5f);
  ff y = fast_two_sum(s, c);
  // second correction (the first leaves ~2^-45 when rsqrt is off by 2 ulps)
  ff r2 = add(x, neg(sqr(y)));
  return fast_two_sum(y.hi, fadd(y.lo, fmul(fmul(r2.hi, rs), 0.5f)));
}

// ---- conversions ----------------------------------------------------------------------------

// d * 2^-shift -> ff.  hi = the value rounded to 24 bits (integer rounding of the fraction),
// lo = the rounded remainder.  *ok is cleared unless d is 0 or the scaled magnitude lies in
// [2^-74, 2^126) (so that lo is a normal float and hi cannot overflow); NaN/Inf clear it too.
GVX_HD ff from_double(double d, bool *ok, int shift = 0) {
  uint64_t b = d2u(d);
  uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  int e = (int)((b >> 52) & 0x7ff);
  uint64_t frac = b & 0xfffffffffffffull;
  if (e == 0) {
    if (frac != 0) *ok = false;
    return {u2f(sign), 0.0f};
  }
  if (e == 0x7ff) *ok = false;
  int ef = e - 1023 + 127 - shift;  // float biased exponent of hi
  if (ef < 53 || ef > 252) {
    *ok = false;
    ef = 127;
  }
  uint32_t top = (uint32_t)(frac >> 29);
  uint32_t rbit = (uint32_t)(frac >> 28) & 1u;
  uint32_t hib = (sign | ((uint32_t)ef << 23) | top) + rbit;  // a carry moves into the exponent
  int32_t rem = (int32_t)(uint32_t)(frac & 0x1fffffffu) - (int32_t)(rbit << 29);
  float lo = fmul(i2f(rem), pow2f(ef - 127 - 52));
  return {u2f(hib), sign ? -lo : lo};
}

// Biased exponent field of a double (0 for zero and denormals).
GVX_HD int dexp(double d) { return (int)((d2u(d) >> 52) & 0x7ff); }

// f * 2^shift -> double exactly, by bits (denormal floats flushed to zero; Inf/NaN kept).
GVX_HD double f2d_bits(float f, int shift = 0) {
  uint32_t u = f2u(f);
  uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  uint32_t ef = (u >> 23) & 0xffu;
  if (ef == 0) return u2d(sign);
  uint64_t ed = ef == 0xffu ? 0x7ffull : (uint64_t)((int)ef - 127 + 1023 + shift);
  return u2d(sign | (ed << 52) | ((uint64_t)(u & 0x7fffffu) << 29));
}

// ff * 2^shift -> double: one rounding (one FP64 add).
GVX_HD double to_double(ff x, int shift = 0) { return f2d_bits(x.hi, shift) + f2d_bits(x.lo, shift); }

// Signed integer D times 2^p as ff (|D| < 2^62), rounding only in lo.
GVX_HD ff from_scaled_int(int64_t D, int p, bool *ok) {
  if (D == 0) return {0.0f, 0.0f};
  uint32_t sign = D < 0 ? 0x80000000u : 0u;
  uint64_t a = D < 0 ? (uint64_t)(-D) : (uint64_t)D;
  int lead = 63 - clz64(a);  // position of the leading 1
  int sh = lead > 23 ? lead - 23 : 0;
  uint32_t m = (uint32_t)(a >> sh);  // 24 significant bits (fewer when lead < 23)
  uint64_t rem = a - ((uint64_t)m << sh);
  int ehi = lead + p;  // exponent of hi
  if (p < -126 || ehi > 126) {
    *ok = false;
    p = 0;
    ehi = lead;
  }
  float hi;
  if (lead >= 23) {
    hi = u2f(sign | ((uint32_t)((ehi + 127) & 0xff) << 23) | (m & 0x7fffffu));
  } else {
    hi = fmul(i2f((int32_t)m), pow2f(p > 127 ? 127 : p));
    if (sign) hi = -hi;
  }
  // rem < 2^sh <= 2^39: split so the int -> float conversion sees at most 31 bits
  float lo = 0.0f;
  if (rem) {
    int rs = sh > 31 ? sh - 31 : 0;
    lo = fmul(i2f((int32_t)(rem >> rs)), pow2f(p + rs));
    if (sign) lo = -lo;
  }
  return {hi, lo};
}

// Exact a - b for doubles whose exponents differ by at most one (the range where the
// difference can cancel): integer subtraction of the aligned significands.  Otherwise the
// ff difference of the converted operands, which keeps relative accuracy there.
GVX_HD ff diff(double a, double b, bool *ok) {
  uint64_t ua = d2u(a), ub = d2u(b);
  int ea = (int)((ua >> 52) & 0x7ff), eb = (int)((ub >> 52) & 0x7ff);
  bool same_sign = ((ua ^ ub) >> 63) == 0;
  int de = ea - eb;
  if (same_sign && ea != 0 && eb != 0 && de >= -1 && de <= 1 && ea != 0x7ff && eb != 0x7ff) {
    int emin = ea < eb ? ea : eb;
    int64_t ma = (int64_t)((ua & 0xfffffffffffffull) | (1ull << 52)) << (ea - emin);
    int64_t mb = (int64_t)((ub & 0xfffffffffffffull) | (1ull << 52)) << (eb - emin);
    int64_t D = ma - mb;
    if (ua >> 63) D = -D;
    return from_scaled_int(D, emin - 1075, ok);
  }
  ff fa = from_double(a, ok), fb = from_double(b, ok);
  return add(fa, neg(fb));
}

// ---- tables for the elementary functions ------------------------------------------------------

// exp family: c = ln2/64, n = 64 k + j;  tm1[j] = 2^(j/64) - 1,  um1[j] = 1 - 2^(-j/64).
// trig: d = pi/256;  sn[j] = sin(j d), cs[j] = cos(j d), j = 0..128.
// Reduction constants (Cody & Waite): c = hc[0] + hc[1] + hc[2] with hc[0] carrying 11
// significant bits (so n hc[0] is exact for |n| < 2^13); d = tc[0] + tc[1] + tc[2] with tc[0]
// carrying 16 bits.  pi = pi_ff + (remainder below 2^-48).
struct Tables {
  ff tm1[64];
  ff um1[64];
  ff sn[129];
  ff cs[129];
  float hc[3];
  float tc[3];
  float inv_c;  // 1/c
  float inv_d;  // 1/d
  ff third6;    // 1/6
  ff pi;
};

// Host construction of the tables in long double (64- or 113-bit significand).
#if defined(__CUDACC__)
#define GVX_HOST __host__
#else
#define GVX_HOST
#endif
GVX_HOST static inline ff ff_of_ld(long double x) {
  float hi = (float)x;
  float lo = (float)(x - (long double)hi);
  return {hi, lo};
}
GVX_HOST static inline float trunc_bits(long double x, int bits) {
  int e;
  long double m = frexpl(x, &e);  // x = m 2^e, 0.5 <= |m| < 1
  long double t = truncl(ldexpl(m, bits));
  return (float)ldexpl(t, e - bits);
}
GVX_HOST static inline void build_tables(Tables *T) {
  const long double ln2 = logl(2.0L);
  const long double pi = acosl(-1.0L);
  const long double c = ln2 / 64;
  const long double d = pi / 256;
  for (int j = 0; j < 64; j++) {
    T->tm1[j] = ff_of_ld(expm1l((long double)j * c));
    T->um1[j] = ff_of_ld(-expm1l(-(long double)j * c));
  }
  for (int j = 0; j <= 128; j++) {
    T->sn[j] = ff_of_ld(sinl((long double)j * d));
    T->cs[j] = ff_of_ld(cosl((long double)j * d));
  }
  T->hc[0] = trunc_bits(c, 11);
  T->hc[1] = (float)(c - T->hc[0]);
  T->hc[2] = (float)(c - T->hc[0] - (long double)T->hc[1]);
  T->tc[0] = trunc_bits(d, 16);
  T->tc[1] = (float)(d - T->tc[0]);
  T->tc[2] = (float)(d - T->tc[0] - (long double)T->tc[1]);
  T->inv_c = (float)(1.0L / c);
  T->inv_d = (float)(1.0L / d);
  T->third6 = ff_of_ld(1.0L / 6);
  T->pi = ff_of_ld(pi);
}

// ---- elementary functions -------------------------------------------------------------------

// Round-to-nearest integer of x (|x| < 2^22) with two FP32 adds (the 1.5 * 2^23 shift).
GVX_HD float round_shift(float x, int *n) {
  const float magic = 12582912.0f;
  float t = fadd(x, magic);
  *n = (int32_t)(f2u(t) - 0x4B400000u);
  return fsub(t, magic);
}

// r = x - nf (c0 + c1 + c2) as ff, with nf c0 exact and x.hi - nf c0 exact.
GVX_HD ff reduce(ff x, float nf, const float *c) {
  float r1 = ffma(-nf, c[0], x.hi);
  ff p = two_prod(nf, c[1]);
  ff s = two_sum(r1, -p.hi);
  float lo = fadd(fsub(s.lo, p.lo), fsub(x.lo, fmul(nf, c[2])));
  return two_sum(s.hi, lo);
}

// Even and odd Taylor parts of exp(r) for |r| <= ln2/128:
//   E = 1 + r^2/2 + r^4/24 (r^6/720 < 4e-17 dropped),  O = r + r^3/6 + r^5/120.
GVX_HD void exp_parts(ff r, const Tables &T, ff *E, ff *O) {
  ff r2 = sqr(r);
  float r4 = fmul(r2.hi, r2.hi);
  ff e = fast_two_sum(1.0f, fmul(r2.hi, 0.5f));
  *E = fast_two_sum(e.hi, fadd(e.lo, ffma(r2.lo, 0.5f, fmul(r4, 0.041666668f))));
  ff r3 = mul(r, r2);
  ff r3_6 = mul(r3, T.third6);
  float r5_120 = fmul(fmul(r3.hi, r2.hi), 0.008333334f);
  *O = add_same(r, add_same_f(r3_6, r5_120));
}

// cosh(x) for ff x with |x| <= 40:  (2^(n/64) (E + O) + 2^(-n/64) (E - O)) / 2, n = 64 k + j,
//   2^(j/64) = 1 + tm1[j],  2^(-j/64) = 1 - um1[j].
GVX_HD ff cosh(ff x, const Tables &T) {
  if (x.hi < 0.0f) x = neg(x);
  int n;
  float nf = round_shift(fmul(x.hi, T.inv_c), &n);
  ff r = reduce(x, nf, T.hc);
  ff E, O;
  exp_parts(r, T, &E, &O);
  int j = n & 63, k = n >> 6;
  ff tp = fast_two_sum(1.0f, T.tm1[j].hi);
  tp.lo = fadd(tp.lo, T.tm1[j].lo);
  ff tn = fast_two_sum(1.0f, -T.um1[j].hi);
  tn.lo = fsub(tn.lo, T.um1[j].lo);
  ff ep = scale(mul(tp, add_same(E, O)), pow2f(k - 1));
  ff en = scale(mul(tn, add(E, neg(O))), pow2f(-k - 1));
  return add_same(ep, en);
}

// sinh(x) for ff x with |x| <= 40, accurate to ~2^-46 relative also for tiny |x|:
//   sinh(n c + r) = S_n E(r) + C_n O(r),
//   S_n = ((2^k - 2^-k) + 2^k tm1[j] + 2^-k um1[j]) / 2        (all terms >= 0)
//   C_n = ((2^k + 2^-k) + 2^k tm1[j] - 2^-k um1[j]) / 2        (>= 1)
GVX_HD ff sinh(ff x, const Tables &T) {
  bool negx = x.hi < 0.0f;
  if (negx) x = neg(x);
  int n;
  float nf = round_shift(fmul(x.hi, T.inv_c), &n);
  ff r = reduce(x, nf, T.hc);
  ff E, O;
  exp_parts(r, T, &E, &O);
  int j = n & 63, k = n >> 6;
  float pk = pow2f(k), mk = pow2f(-k);
  ff a = scale(T.tm1[j], pk), b = scale(T.um1[j], mk);
  ff S = scale(add_same(add_same(fast_two_sum(pk, -mk), a), b), 0.5f);
  ff C = scale(add(add_same(fast_two_sum(pk, mk), a), neg(b)), 0.5f);
  ff s = add(mul(S, E), mul(C, O));
  return negx ? neg(s) : s;
}

// sin(h) for ff h with 0 <= h <= pi/2 (+ a few ulps):  sin(j d + r) = sn[j] cos r + cs[j] sin r,
//   cos r = 1 - r^2/2 + r^4/24,  sin r = r - r^3/6 + r^5/120,  |r| <= pi/512.
GVX_HD ff sin_q1(ff h, const Tables &T) {
  int j;
  float jf = round_shift(fmul(h.hi, T.inv_d), &j);
  if (j > 128) {
    j = 128;
    jf = 128.0f;
  }
  if (j < 0) {
    j = 0;
    jf = 0.0f;
  }
  ff r = reduce(h, jf, T.tc);
  ff r2 = sqr(r);
  float r4 = fmul(r2.hi, r2.hi);
  ff cr = fast_two_sum(1.0f, -fmul(r2.hi, 0.5f));
  cr = fast_two_sum(cr.hi, fadd(cr.lo, ffma(-r2.lo, 0.5f, fmul(r4, 0.041666668f))));
  ff r3 = mul(r, r2);
  ff r3_6 = mul(r3, T.third6);
  float r5_120 = fmul(fmul(r3.hi, r2.hi), 0.008333334f);
  ff sr = add(r, neg(add_same_f(r3_6, -r5_120)));
  return add(mul(T.sn[j], cr), mul(T.cs[j], sr));
}

}  // namespace ffm
}  // namespace gvx
