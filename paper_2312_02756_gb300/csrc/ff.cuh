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
GVX_HD uint32_t dhi(double d) {
#if defined(__CUDA_ARCH__)
  return (uint32_t)__double2hiint(d);
#else
  return (uint32_t)(d2u(d) >> 32);
#endif
}
GVX_HD uint32_t dlo(double d) {
#if defined(__CUDA_ARCH__)
  return (uint32_t)__double2loint(d);
#else
  return (uint32_t)d2u(d);
#endif
}
GVX_HD double hilo2d(uint32_t hi, uint32_t lo) {
#if defined(__CUDA_ARCH__)
  return __hiloint2double((int)hi, (int)lo);
#else
  return u2d(((uint64_t)hi << 32) | lo);
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
// Results of add/mul may be left unnormalized (|lo| up to ~2^-22 |hi|): every consumer below
// reads hi and lo separately, so the value hi + lo keeps its precision; renorm() restores
// |lo| <= ulp(hi)/2 where a comparison or a conversion needs it.

GVX_HD ff make(float x) { return {x, 0.0f}; }
GVX_HD ff neg(ff x) { return {-x.hi, -x.lo}; }
GVX_HD ff renorm(ff x) { return fast_two_sum(x.hi, x.lo); }
// exact scaling by a power of two
GVX_HD ff scale(ff x, float p2) { return {fmul(x.hi, p2), fmul(x.lo, p2)}; }

// x + y, accurate also under cancellation (relative error ~2^-47 of the result)
GVX_HD ff add(ff x, ff y) {
  ff s = two_sum(x.hi, y.hi);
  ff t = two_sum(x.lo, y.lo);
  s = fast_two_sum(s.hi, fadd(s.lo, t.hi));
  return fast_two_sum(s.hi, fadd(s.lo, t.lo));
}
// x + y for operands of the same sign (no cancellation)
GVX_HD ff add_same(ff x, ff y) {
  ff s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, fadd(s.lo, fadd(x.lo, y.lo)));
}
// x + y where |y| <= |x| / 2^10 or so (a small correction): no renormalization of the result
GVX_HD ff add_small(ff x, ff y) {
  ff s = fast_two_sum(x.hi, y.hi);
  return {s.hi, fadd(s.lo, fadd(x.lo, y.lo))};
}
GVX_HD ff mul(ff x, ff y) {
  ff p = two_prod(x.hi, y.hi);
  return {p.hi, ffma(x.lo, y.hi, ffma(x.hi, y.lo, p.lo))};
}
GVX_HD ff mul_f(ff x, float f) {
  ff p = two_prod(x.hi, f);
  return {p.hi, ffma(x.lo, f, p.lo)};
}
GVX_HD ff sqr(ff x) {
  ff p = two_prod(x.hi, x.hi);
  return {p.hi, ffma(fadd(x.hi, x.hi), x.lo, p.lo)};
}
// 1/a to within 1 ulp: hardware approximation and one Newton step.
GVX_HD float frcp(float a) {
  float r = fdiv_approx(1.0f, a);
  return ffma(r, ffma(-a, r, 1.0f), r);
}
// 1/sqrt(a) to within ~1 ulp, a > 0: hardware approximation and one Newton step.
GVX_HD float frsq(float a) {
  float r = frsqrt_approx(a);
  return ffma(fmul(0.5f, r), ffma(-a, fmul(r, r), 1.0f), r);
}
// x / y, y != 0: q1 = x.hi / y.hi to ~1 ulp, one correction from the ff remainder.
GVX_HD ff div(ff x, ff y) {
  float ry = frcp(y.hi);
  float q1 = fmul(x.hi, ry);
  ff p = two_prod(q1, y.hi);
  float r = fadd(fsub(fsub(x.hi, p.hi), p.lo), ffma(-q1, y.lo, x.lo));
  return fast_two_sum(q1, fmul(r, ry));
}
// sqrt(x), x >= 0: s = x.hi / sqrt(x.hi) to ~1 ulp, one correction from the ff residual.
GVX_HD ff sqrt(ff x) {
  if (!(x.hi > 0.0f)) return {0.0f, 0.0f};
  float rs = frsq(x.hi);
  float s = fmul(x.hi, rs);
  ff p = two_prod(s, s);
  float r = fadd(fsub(fsub(x.hi, p.hi), p.lo), x.lo);
  return fast_two_sum(s, fmul(fmul(r, rs), 0.5f));
}
// 1/x, x != 0
GVX_HD ff recip(ff x) {
  float y = frcp(x.hi);
  ff p = two_prod(y, x.hi);
  float e = fsub(fsub(1.0f, p.hi), ffma(y, x.lo, p.lo));
  return fast_two_sum(y, fmul(y, e));
}

// ---- conversions ----------------------------------------------------------------------------

// d * 2^-shift -> ff, from the two 32-bit words of d.  hi = the value rounded to 24 bits (integer
// rounding of the fraction), lo = the rounded remainder.  *ok is cleared unless d is 0 or the
// scaled magnitude lies in [2^-74, 2^126) (so that lo is a normal float and hi cannot overflow);
// NaN and Inf clear it too.
GVX_HD ff from_double(double d, bool *ok, int shift = 0) {
  uint32_t wh = dhi(d), wl = dlo(d);
  uint32_t sign = wh & 0x80000000u;
  int e = (int)((wh >> 20) & 0x7ffu);
  if (e == 0) {
    if ((wh & 0xfffffu) | wl) *ok = false;
    return {u2f(sign), 0.0f};
  }
  int ef = e - 896 - shift;  // float biased exponent of hi
  if (ef < 53 || ef > 252) {
    *ok = false;
    ef = 127;
  }
  uint32_t top = ((wh & 0xfffffu) << 3) | (wl >> 29);
  uint32_t rbit = (wl >> 28) & 1u;
  uint32_t hib = (sign | ((uint32_t)ef << 23) | top) + rbit;  // a carry moves into the exponent
  int32_t rem = (int32_t)(wl & 0x1fffffffu) - (int32_t)(rbit << 29);
  float lo = fmul(i2f(rem), pow2f(ef - 179));
  return {u2f(hib), sign ? -lo : lo};
}

// from_double without the range checks, for a d whose scaled magnitude is known to be below
// 2^126: zeros, denormals and values that scale below 2^-74 give a signed zero.  Bitwise the same
// result as from_double wherever that leaves *ok set.
GVX_HD ff from_double_ranged(double d, int shift) {
  uint32_t wh = dhi(d), wl = dlo(d);
  uint32_t sign = wh & 0x80000000u;
  int e = (int)((wh >> 20) & 0x7ffu);
  int ef = e - 896 - shift;
  uint32_t top = ((wh & 0xfffffu) << 3) | (wl >> 29);
  uint32_t rbit = (wl >> 28) & 1u;
  uint32_t hib = (sign | ((uint32_t)ef << 23) | top) + rbit;
  int32_t rem = (int32_t)(wl & 0x1fffffffu) - (int32_t)(rbit << 29);
  float lo = fmul(i2f(rem), pow2f(ef - 179));
  ff r = {u2f(hib), sign ? -lo : lo};
  return (e != 0 && ef >= 53) ? r : ff{u2f(sign), 0.0f};
}

// Biased exponent field of a double (0 for zero and denormals).
GVX_HD int dexp(double d) { return (int)((dhi(d) >> 20) & 0x7ffu); }

// f * 2^shift -> double exactly, by bits (denormal floats flushed to zero; Inf/NaN kept).
GVX_HD double f2d_bits(float f, int shift = 0) {
  uint32_t u = f2u(f);
  uint32_t sign = u & 0x80000000u;
  uint32_t ef = (u >> 23) & 0xffu;
  if (ef == 0) return hilo2d(sign, 0u);
  uint32_t ed = ef == 0xffu ? 0x7ffu : (uint32_t)((int)ef + 896 + shift);
  return hilo2d(sign | (ed << 20) | ((u & 0x7fffffu) >> 3), (u & 7u) << 29);
}

// ff * 2^shift -> double: one rounding (one FP64 add).
GVX_HD double to_double(ff x, int shift = 0) {
  return f2d_bits(x.hi, shift) + f2d_bits(x.lo, shift);
}

// ff * 2^shift -> double with integer operations only (no FP64 instruction): the exact sum
// hi + lo truncated to 53 bits, an error below 2 ulps of the result.  Requires hi normal or 0,
// |lo| <= 2^-21 |hi| (true of every normalized ff: add, renorm, recip, sqrt), and a result
// inside the normal range of double.  A denormal lo counts as 0.
GVX_HD double to_double_int(ff x, int shift) {
  const uint32_t uh = f2u(x.hi), ul = f2u(x.lo);
  const int eh = (int)((uh >> 23) & 0xffu), el = (int)((ul >> 23) & 0xffu);
  const uint32_t mh = (uh & 0x7fffffu) | 0x800000u;
  const uint32_t ml = el ? ((ul & 0x7fffffu) | 0x800000u) : 0u;
  // lo in units of ulp(hi as a double) = 2^-29 ulp(hi as a float); |L| < 2^32
  const int sft = el - eh + 29;
  const uint32_t L = sft >= 0 ? ml << sft : (sft > -24 ? ml >> -sft : 0u);
  const uint64_t M = (uint64_t)mh << 29;
  uint64_t S = ((uh ^ ul) >> 31) ? M - L : M + L;  // in (2^52 - 2^32, 2^53 + 2^32)
  int ed = eh + 896 + shift;
  if (S >> 53) {
    S >>= 1;
    ed += 1;
  } else if (!(S >> 52)) {
    S <<= 1;
    ed -= 1;
  }
  const uint64_t bits = ((uint64_t)(uh >> 31) << 63) | ((uint64_t)ed << 52) |
                        (S & 0xfffffffffffffull);
  return eh ? u2d(bits) : f2d_bits(x.lo, shift);
}

// Non-negative integer D times 2^p as ff (D < 2^63), rounding only in lo.
GVX_HD ff from_scaled_int(uint64_t D, int p, bool *ok) {
  if (D == 0) return {0.0f, 0.0f};
  int lead = 63 - clz64(D);  // position of the leading 1
  int sh = lead > 23 ? lead - 23 : 0;
  uint32_t m = (uint32_t)(D >> sh);  // 24 significant bits (fewer when lead < 23)
  uint64_t rem = D - ((uint64_t)m << sh);
  int ehi = lead + p;  // exponent of hi
  if (p < -126 || p > 100 || ehi > 126) {
    *ok = false;
    return {0.0f, 0.0f};
  }
  float hi = lead >= 23 ? u2f(((uint32_t)(ehi + 127) << 23) | (m & 0x7fffffu))
                        : fmul(i2f((int32_t)m), pow2f(p));
  float lo = 0.0f;
  if (rem) {
    int rs = sh > 31 ? sh - 31 : 0;  // at most 31 bits into the int -> float conversion
    lo = fmul(i2f((int32_t)(rem >> rs)), pow2f(p + rs));
  }
  return {hi, lo};
}

GVX_HD uint64_t umulhi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// 1 - (bx^2 + by^2 + bz^2) for doubles with |b| < 1, in 64-bit fixed point (unit 2^-62): each
// square is the top 64 bits of the 106-bit square of the significand, truncated, so the result
// is exact to 3 * 2^-62.  *ok is cleared when the result is below 2^-16 (|beta| > 0.9999924) or
// any component is not finite / not below 1 in magnitude.
GVX_HD ff one_minus_sq3(double bx, double by, double bz, bool *ok) {
  const double c[3] = {bx, by, bz};
  uint64_t sum = 0;
  for (int k = 0; k < 3; k++) {
    uint32_t wh = dhi(c[k]), wl = dlo(c[k]);
    int eb = (int)((wh >> 20) & 0x7ffu);
    if (eb == 0) continue;  // zero (denormals count as zero: < 2^-1022)
    int e = eb - 1023;      // |b| in [2^e, 2^(e+1))
    if (e >= 0) {
      *ok = false;
      return make(0.0f);
    }
    uint64_t m = ((((uint64_t)(wh & 0xfffffu) | 0x100000u) << 32) | wl) << 11;
    uint64_t hi = umulhi64(m, m);  // floor(M^2 2^22 / 2^64); the square is hi 2^(2e - 62)
    int sh = -2 * e;               // >= 2
    sum += sh < 64 ? hi >> sh : 0;
  }
  const uint64_t one = 1ull << 62;
  if (sum >= one - (one >> 16)) {  // 1 - b2 < 2^-16
    *ok = false;
    return make(0.0f);
  }
  return from_scaled_int(one - sum, -62, ok);
}

// ---- elementary functions (tables in ff_tables.cuh) ------------------------------------------

#if defined(__CUDACC__)
typedef float4 gvx_f4;
#else
struct alignas(16) gvx_f4 {
  float x, y, z, w;
};
#endif

// Round-to-nearest integer of x (|x| < 2^22) with two FP32 adds (the 1.5 * 2^23 shift).
GVX_HD float round_shift(float x, int *n) {
  const float magic = 12582912.0f;
  float t = fadd(x, magic);
  *n = (int32_t)(f2u(t) - 0x4B400000u);
  return fsub(t, magic);
}

// r = x - nf (c0 + c1 + c2) as ff, with nf c0 exact and x.hi - nf c0 exact.
GVX_HD ff reduce(ff x, float nf, float c0, float c1, float c2) {
  float r1 = ffma(-nf, c0, x.hi);
  ff p = two_prod(nf, c1);
  ff s = two_sum(r1, -p.hi);
  return two_sum(s.hi, fadd(fsub(s.lo, p.lo), fsub(x.lo, fmul(nf, c2))));
}

// Hyperbolic reduction for x >= 0 with x < 16: x = n c + r, |r| <= c/2 = ln2/2048, and the even
// and odd Taylor parts of exp(r): E = 1 + r^2/2 (r^4/24 < 6e-16 dropped), O = r + r^3/6.
struct HypParts {
  ff E, O;
  int j, k;  // n = 1024 k + j
};
GVX_HD HypParts hyp_parts(ff x, float inv_c, float c0, float c1, float c2) {
  HypParts h;
  int n;
  float nf = round_shift(fmul(x.hi, inv_c), &n);
  ff r = reduce(x, nf, c0, c1, c2);
  float t = ffma(r.hi, r.hi, fmul(fadd(r.hi, r.hi), r.lo));  // r^2
  h.E = fast_two_sum(1.0f, fmul(t, 0.5f));
  ff o = two_sum(r.hi, fmul(fmul(r.hi, t), 0.16666667f));
  h.O = {o.hi, fadd(o.lo, r.lo)};
  h.j = n & 1023;
  h.k = n >> 10;
  return h;
}

// E +- O as ff (|O| <= 4e-4, E ~ 1: no cancellation)
GVX_HD ff add_eo(ff E, ff O) {
  ff s = fast_two_sum(E.hi, O.hi);
  return {s.hi, fadd(s.lo, fadd(E.lo, O.lo))};
}

}  // namespace ffm
}  // namespace gvx
