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
//     one float; rows 0 and 1, and rows 2 and 3, run together on paired FP32 instructions
//     (ff2.cuh: each lane the scalar operations' bits), the matrix kept with those rows
//     interleaved so that one 16-byte load gives both rows' entries of a column;
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
#include "ff2.cuh"

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

// The scaled matrix with its rows paired: lp[4 p + j] holds column j of rows 2p (lane x) and
// 2p + 1 (lane y).
GVX_HD void pair_rows(const LorentzFF &M, ff2 *lp) {
#pragma unroll
  for (int p = 0; p < 2; p++)
#pragma unroll
    for (int j = 0; j < 4; j++) lp[4 * p + j] = pack(M.l[8 * p + j], M.l[8 * p + 4 + j]);
}

// sum_j l[j] x[j] of two rows at once (lanes), for ff x: the high parts' products by TwoProduct
// and TwoSum, everything else collected in one float per lane.  Returned unnormalized (the
// caller rounds hi + lo once).
GVX_HD ff2 dot4_ff2(const ff2 *l, const ff *x) {
  f2 xh = bc2(x[0].hi), xl = bc2(x[0].lo);
  ff2 p = two_prod2(l[0].hi, xh);
  f2 s = p.hi;
  f2 e = fma2(l[0].lo, xh, fma2(l[0].hi, xl, p.lo));
#pragma unroll
  for (int j = 1; j < 4; j++) {
    xh = bc2(x[j].hi);
    xl = bc2(x[j].lo);
    p = two_prod2(l[j].hi, xh);
    const ff2 t = two_sum2(s, p.hi);
    s = t.hi;
    e = add2(e, add2(t.lo, fma2(l[j].lo, xh, fma2(l[j].hi, xl, p.lo))));
  }
  return {s, e};
}

// out = L v for one vector, with the row-paired scaled matrix lp (pair_rows) and the row scale
// exponents r of lorentz_ff; false (out untouched) outside the domain.
GVX_HD bool apply_ff(const ff2 *lp, const int *r, const double *v, double *out) {
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
  for (int p = 0; p < 2; p++) {
    const ff2 y = dot4_ff2(lp + 4 * p, x);
    const uint32_t k0 = (uint32_t)(896 + r[2 * p] + s) << 20;  // float -> double exponent rebias
    const uint32_t k1 = (uint32_t)(896 + r[2 * p + 1] + s) << 20;
    out[2 * p] = f2d_rebias(y.hi.x, k0) + f2d_rebias(y.lo.x, k0);
    out[2 * p + 1] = f2d_rebias(y.hi.y, k1) + f2d_rebias(y.lo.y, k1);
  }
  return true;
}

}  // namespace ffm
}  // namespace gvx
