// Paired float-float arithmetic on Blackwell's paired FP32 instructions (FADD2 / FMUL2 / FFMA2:
// one instruction, two independent operations, each rounded exactly as the scalar __fadd_rn /
// __fmul_rn / __fmaf_rn).  An ff2 holds two float-float numbers, one per lane; every operation
// below repeats the scalar one of ff.cuh step for step, so each lane gets the scalar operation's
// bits (negations and subtractions are exact paired multiplies and FMAs: x - y = fma(y, -1, x)).
// On the host the paired instructions are emulated lane by lane with the same roundings.
#pragma once

#include "ff.cuh"

namespace gvx {
namespace ffm {

#if defined(__CUDACC__)
typedef float2 f2;
#else
struct f2 {
  float x, y;
};
#endif

GVX_HD f2 mk2(float a, float b) {
  f2 r;
  r.x = a;
  r.y = b;
  return r;
}
GVX_HD f2 bc2(float a) { return mk2(a, a); }
GVX_HD f2 add2(f2 a, f2 b) {
#if defined(__CUDA_ARCH__)
  return __fadd2_rn(a, b);
#else
  return mk2(fadd(a.x, b.x), fadd(a.y, b.y));
#endif
}
GVX_HD f2 mul2(f2 a, f2 b) {
#if defined(__CUDA_ARCH__)
  return __fmul2_rn(a, b);
#else
  return mk2(fmul(a.x, b.x), fmul(a.y, b.y));
#endif
}
GVX_HD f2 fma2(f2 a, f2 b, f2 c) {
#if defined(__CUDA_ARCH__)
  return __ffma2_rn(a, b, c);
#else
  return mk2(ffma(a.x, b.x, c.x), ffma(a.y, b.y, c.y));
#endif
}
GVX_HD f2 sub2(f2 a, f2 b) { return fma2(b, bc2(-1.0f), a); }  // a - b, one rounding
GVX_HD f2 neg2(f2 a) { return mul2(a, bc2(-1.0f)); }

struct alignas(16) ff2 {
  f2 hi, lo;
};

GVX_HD ff2 pack(ff a, ff b) { return {mk2(a.hi, b.hi), mk2(a.lo, b.lo)}; }
GVX_HD ff lane_x(const ff2 &v) { return {v.hi.x, v.lo.x}; }
GVX_HD ff lane_y(const ff2 &v) { return {v.hi.y, v.lo.y}; }

GVX_HD ff2 two_sum2(f2 a, f2 b) {
  const f2 s = add2(a, b);
  const f2 bb = sub2(s, a);
  return {s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}
GVX_HD ff2 fast_two_sum2(f2 a, f2 b) {
  const f2 s = add2(a, b);
  return {s, sub2(b, sub2(s, a))};
}
GVX_HD ff2 two_prod2(f2 a, f2 b) {
  const f2 p = mul2(a, b);
  return {p, fma2(a, b, neg2(p))};
}
GVX_HD ff2 neg(const ff2 &x) { return {neg2(x.hi), neg2(x.lo)}; }
GVX_HD ff2 scale(const ff2 &x, f2 p2) { return {mul2(x.hi, p2), mul2(x.lo, p2)}; }
GVX_HD ff2 add_same(const ff2 &x, const ff2 &y) {
  const ff2 s = two_sum2(x.hi, y.hi);
  return fast_two_sum2(s.hi, add2(s.lo, add2(x.lo, y.lo)));
}
GVX_HD ff2 mul(const ff2 &x, const ff2 &y) {
  const ff2 p = two_prod2(x.hi, y.hi);
  return {p.hi, fma2(x.lo, y.hi, fma2(x.hi, y.lo, p.lo))};
}
GVX_HD ff2 sqr(const ff2 &x) {
  const ff2 p = two_prod2(x.hi, x.hi);
  return {p.hi, fma2(add2(x.hi, x.hi), x.lo, p.lo)};
}

}  // namespace ffm
}  // namespace gvx
