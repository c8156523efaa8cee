// A general Lorentz transformation out = L v in float-float: the fast path of the FP64
// gvx_lorentz_apply for one 4x4 matrix shared by every vector (Sec. 4.1: a transformation is a
// 4x4 matrix applied to each vector of an array).
//
// Sixteen FP64 FMAs per vector would keep the FP64 pipe busy about three times longer than the
// memory system needs to stream the vectors, so the row sums run on the FP32 pipe:
//   * each row i of L is scaled by the power of two 2^-r_i that brings its largest entry into
//     [1, 2), each vector by the 2^-s that does the same for its largest component, and the
//     scaled values are converted to ff (entries or components below 2^-74 of that largest one
//     count as 0);
//   * the four products of a row are formed by TwoProduct with the cross terms of the low parts,
//     their high parts added by TwoSum, and the low parts and the TwoSum errors collected in
//     one float;
//   * the result, hi + lo scaled by 2^(r_i + s), is rounded to double by one FP64 add (each
//     float moved into a double exactly by integer operations).
// Error of each component: below 2^-42 sum_j |L_ij v_j| + 2^-70 max_j |L_ij| max_j |v_j| (the
// second term covers what the conversions flush to zero).
//
// Domain: L finite, each row either all zero or with a scale exponent r_i in [-400, 400]; each
// vector finite with its scale exponent s in [-400, 400].  A matrix outside it sends the whole
// launch to the FP64 FMA chains; a vector outside it takes them for that vector alone.
#pragma once

#include "ff.cuh"

namespace gvx {
namespace ffm {

constexpr int kApplyScaleLim = 400;

struct LorentzFF {
  ff l[16];  // row-major, row i scaled by 2^-r[i]
  int r[4];  // unbiased row scale exponents (0 for a zero row)
  bool ok;
};

GVX_HD LorentzFF lorentz_ff(const double *L) {
  LorentzFF M;
  M.ok = true;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    int emax = 0;
    bool nz = false;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int e = dexp(L[4 * i + j]);
      emax = e > emax ? e : emax;
      nz = nz || ((dhi(L[4 * i + j]) & 0x7fffffffu) | dlo(L[4 * i + j])) != 0u;
    }
    const int r = emax - 1023;
    // a zero row is exact; a row of denormals alone, or one out of range, is not handled
    if (nz && (r < -kApplyScaleLim || r > kApplyScaleLim)) M.ok = false;
    M.r[i] = nz ? r : 0;
#pragma unroll
    for (int j = 0; j < 4; j++) M.l[4 * i + j] = from_double_ranged(L[4 * i + j], M.r[i]);
  }
  return M;
}

// f * 2^(shift) as a double, exactly, for k = (896 + shift) << 20 and a float f that is 0 or
// normal: the float's exponent and fraction move into the double's fields by one add on the
// high word.  A denormal f counts as 0.
GVX_HD double f2d_rebias(float f, uint32_t k) {
  const uint32_t u = f2u(f);
  if ((u & 0x7f800000u) == 0u) return 0.0;
  return hilo2d((((u & 0x7fffffffu) >> 3) + k) | (u & 0x80000000u), u << 29);
}

// sum_j l[j] x[j] for ff l, x: the high parts' products by TwoProduct and TwoSum, everything
// else collected in one float.  Returned unnormalized (the caller rounds hi + lo once).
GVX_HD ff dot4_ff(const ff *l, const ff *x) {
  ff p = two_prod(l[0].hi, x[0].hi);
  float s = p.hi;
  float e = ffma(l[0].lo, x[0].hi, ffma(l[0].hi, x[0].lo, p.lo));
#pragma unroll
  for (int j = 1; j < 4; j++) {
    p = two_prod(l[j].hi, x[j].hi);
    const ff t = two_sum(s, p.hi);
    s = t.hi;
    e = fadd(e, fadd(t.lo, ffma(l[j].lo, x[j].hi, ffma(l[j].hi, x[j].lo, p.lo))));
  }
  return {s, e};
}

// out = L v for one vector, with the scaled ff matrix l (row-major) and its row scale exponents
// r from lorentz_ff; false (out untouched) outside the domain.
GVX_HD bool apply_ff(const ff *l, const int *r, const double *v, double *out) {
  int emax = 0;
#pragma unroll
  for (int j = 0; j < 4; j++) {
    const int e = dexp(v[j]);
    emax = e > emax ? e : emax;
  }
  const int s = emax - 1023;
  if (s < -kApplyScaleLim || s > kApplyScaleLim) return false;  // also Inf/NaN and all-zero
  ff x[4];
#pragma unroll
  for (int j = 0; j < 4; j++) x[j] = from_double_ranged(v[j], s);
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const ff y = dot4_ff(l + 4 * i, x);
    const uint32_t k = (uint32_t)(896 + r[i] + s) << 20;  // float -> double exponent rebias
    out[i] = f2d_rebias(y.hi, k) + f2d_rebias(y.lo, k);
  }
  return true;
}

}  // namespace ffm
}  // namespace gvx
