// Pair mass of Cartesian legs (PxPyPzE or PxPyPzM), cancellation-free (the mass kernels of
// Sec. 4.1 on the other 4-D coordinate systems of Sec. 3.1), in the working precision T.
//
// With P_i = |p_i|, q_i = m_i^2 (= E_i^2 - P_i^2 for PxPyPzE legs) and E_i^2 = P_i^2 + q_i:
//   m^2 = q1 + q2 + 2 T1 + 2 T2,
//   T1 = E1 E2 - P1 P2 = (q1 P2^2 + q2 P1^2 + q1 q2) / (E1 E2 + P1 P2),
//   T2 = P1 P2 - p1.p2 = |p1 x p2|^2 / (P1 P2 + p1.p2)   when p1.p2 > 0,
//                      = P1 P2 + |p1.p2|                 otherwise,
// every term >= 0 for q_i >= 0 (for PxPyPzE legs E1 E2 is the product of the stored energies, so
// the identities hold for any stored values).  The two steps that cancel are made (nearly)
// exact: the cross product p1 x p2 by Kahan's FMA form of a b - c d (within 1.5 ulp of each
// component), and for PxPyPzE legs q = E^2 - px^2 - py^2 - pz^2 from exact FMA squares and an
// error-free running sum.  Everything else adds, multiplies, divides or takes roots of
// non-negative numbers, so the relative error of m is a few ulps (a leg stored with E < |p| makes
// its q negative, and sums of mixed sign then carry their own conditioning).  A spacelike sum
// gives -sqrt of |m^2| (GenVector's convention).
#pragma once

#include <math.h>

#if defined(__CUDACC__)
#define GVX_CHD __host__ __device__ __forceinline__
#else
#define GVX_CHD static inline
#endif

namespace gvx {
namespace cart {

GVX_CHD double root(double x) { return sqrt(x); }
GVX_CHD float root(float x) { return sqrtf(x); }

// a b - c d within 1.5 ulp (Kahan: the rounding error of c d is recovered by an FMA).
template <typename T>
GVX_CHD T diff_of_products(T a, T b, T c, T d) {
  const T w = c * d;
  const T e = fma(-c, d, w);  // w - c d, exactly
  return fma(a, b, -w) + e;
}

// E^2 - (x^2 + y^2 + z^2): every square split exactly (FMA), the terms added by TwoSum, then the
// collected error terms -- within a few ulps of the result even when it is 1e-20 of E^2.
template <typename T>
GVX_CHD T q_from_energy(T E, T x, T y, T z) {
  const T h[4] = {E * E, -(x * x), -(y * y), -(z * z)};
  const T l[4] = {fma(E, E, -h[0]), -fma(x, x, h[1]), -fma(y, y, h[2]), -fma(z, z, h[3])};
  T s = h[0], err = (T)0;
  for (int k = 1; k < 4; k++) {
    const T t = s + h[k];
    const T bb = t - s;
    err += (s - (t - bb)) + (h[k] - bb);
    s = t;
  }
  return s + (err + ((l[0] + l[1]) + (l[2] + l[3])));
}

// coords 0: legs are (px, py, pz, E); coords 1: (px, py, pz, m).
template <typename T>
GVX_CHD T mass(const T *a, const T *b, int coords) {
  const T P1 = fma(a[0], a[0], fma(a[1], a[1], a[2] * a[2]));
  const T P2 = fma(b[0], b[0], fma(b[1], b[1], b[2] * b[2]));
  const T q1 = coords == 0 ? q_from_energy(a[3], a[0], a[1], a[2]) : a[3] * a[3];
  const T q2 = coords == 0 ? q_from_energy(b[3], b[0], b[1], b[2]) : b[3] * b[3];
  const T d = fma(a[0], b[0], fma(a[1], b[1], a[2] * b[2]));
  const T cx = diff_of_products(a[1], b[2], a[2], b[1]);
  const T cy = diff_of_products(a[2], b[0], a[0], b[2]);
  const T cz = diff_of_products(a[0], b[1], a[1], b[0]);
  const T c2 = fma(cx, cx, fma(cy, cy, cz * cz));
  const T PP = root(P1) * root(P2);
  const T EE = coords == 0 ? a[3] * b[3] : root(P1 + q1) * root(P2 + q2);
  const T den1 = EE + PP;
  const T T1 = den1 > (T)0 ? (fma(q1, P2, q2 * P1) + q1 * q2) / den1 : (T)0;
  const T T2 = d > (T)0 ? c2 / (PP + d) : PP - d;
  const T m2 = q1 + q2 + (T)2 * (T1 + T2);
  return m2 >= (T)0 ? root(m2) : -root(-m2);
}

}  // namespace cart
}  // namespace gvx
