// Other 4-D coordinate systems and general Lorentz transformations (GenVectorX Sec. 3.1: vectors
// are templated on their coordinate system; Sec. 4.1: transformations are 4x4 matrices applied
// to every vector of an array).
//
// gvx_invariant_mass_cart: pair masses of Cartesian legs, PxPyPzE or PxPyPzM, through the
// fixed-point evaluations of cart_fixed.cuh (integer and FP32 pipes); the rare pairs outside
// their domain take the cancellation-free FP64 form of cart_mass.cuh (an FMA-exact cross product
// and E^2 - |p|^2), on the FP64 pipe for both storage precisions.
//
// gvx_to_pxpypze: PtEtaPhiM, PtEtaPhiE or PxPyPzM vectors to PxPyPzE (convert_ff.cuh in FP64 with
// the light-cone tables, the float functions in FP32).  PtEtaPhiE pair masses: in FP64 the light-cone form of
// ptetaphie_lc.cuh; otherwise both legs converted the same way and the exact fixed-point mass of
// the converted legs.
//
// gvx_lorentz_apply: out = L v for a row-major 4x4 matrix L, shared or one per vector.  One
// shared FP64 matrix takes the float-float row sums of apply_ff.cuh; a matrix per vector (whose
// own 128 bytes make the launch memory-bound) and FP32 take four FMA chains per vector in the
// working precision.
#include <cuda_runtime.h>

#include "apply_ff.cuh"
#include "convert_ff.cuh"
#include "ptetaphie_lc.cuh"
#include "cart_fixed.cuh"
#include "cart_mass.cuh"
#include "common.cuh"
#include "pair_math.cuh"

namespace gvx {
namespace {

template <typename T, int LA, int LB, int COORDS>
__global__ void __launch_bounds__(256) mass_cart_kernel(Lv a, Lv b, T *__restrict__ m, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const V4<T> x = ld4<T, LA>(a, i), y = ld4<T, LB>(b, i);
    T r;
    bool fast = false;
    {
      const T ta[4] = {x.x, x.y, x.z, x.w}, tb[4] = {y.x, y.y, y.z, y.w};
      fast = COORDS == 0 ? cfix::mass_pxpypze(ta, tb, &r) : cfix::mass_pxpypzm(ta, tb, &r);
    }
    if (!fast) {
      // FP32 legs are evaluated in FP64 (exact upcasts): a float E next to a float |p| leaves q
      // as rounding noise of either sign, and only FP64 carries the sums of mixed sign that follow
      const double pa[4] = {x.x, x.y, x.z, x.w}, pb[4] = {y.x, y.y, y.z, y.w};
      r = (T)cart::mass(pa, pb, COORDS);
    }
    st_s(m + i, r);
  }
}

// out = L v by four FMA chains in the working precision.
template <typename T>
__device__ __forceinline__ V4<T> apply_fma(const T *l, const V4<T> &x) {
  V4<T> o;
  o.x = fma(l[0], x.x, fma(l[1], x.y, fma(l[2], x.z, l[3] * x.w)));
  o.y = fma(l[4], x.x, fma(l[5], x.y, fma(l[6], x.z, l[7] * x.w)));
  o.z = fma(l[8], x.x, fma(l[9], x.y, fma(l[10], x.z, l[11] * x.w)));
  o.w = fma(l[12], x.x, fma(l[13], x.y, fma(l[14], x.z, l[15] * x.w)));
  return o;
}

template <typename T, int LV, int LO, bool SHARED>
__global__ void __launch_bounds__(256, 4) lorentz_apply_kernel(const T *__restrict__ L, Lv v, LvOut out,
                                                            int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if constexpr (SHARED && sizeof(T) == 8) {
    // one matrix for every vector: the float-float row sums of apply_ff.cuh (the scaled matrix
    // in shared memory, read by broadcast), FP64 FMA chains for a matrix or a vector outside
    // their domain (the raw matrix also in shared memory, read only there, so that it holds no
    // registers)
    __shared__ ffm::ff2 s_l[8];  // rows paired (pair_rows): one 16-byte load per column
    __shared__ double s_raw[16];
    __shared__ int s_r[4];
    __shared__ int s_ok;
    if (threadIdx.x < 16) s_raw[threadIdx.x] = L[threadIdx.x];
    if (threadIdx.x == 0) {
      double l0[16];
      for (int k = 0; k < 16; k++) l0[k] = L[k];
      const ffm::LorentzFF M = ffm::lorentz_ff(l0);
      ffm::pair_rows(M, s_l);
      for (int k = 0; k < 4; k++) s_r[k] = M.r[k];
      s_ok = M.ok;
    }
    __syncthreads();
    const bool ok = s_ok != 0;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    V4<T> xn = {0, 0, 0, 0};
    if (i < n) xn = ld4<T, LV>(v, i);
    for (; i < n; i += stride) {
      // the next vector's loads go out before this one's arithmetic: two vectors in flight
      const V4<T> x = xn;
      if (i + stride < n) xn = ld4<T, LV>(v, i + stride);
      const double xv[4] = {x.x, x.y, x.z, x.w};
      double o[4];
      V4<T> r;
      if (ok && ffm::apply_ff(s_l, s_r, xv, o)) {
        r = {o[0], o[1], o[2], o[3]};
      } else {
        r = apply_fma(s_raw, x);
      }
      st4<T, LO>(out, i, r);
    }
  } else {
    T l0[16];
    if (SHARED) {
#pragma unroll
      for (int k = 0; k < 16; k++) l0[k] = L[k];
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      const V4<T> x = ld4<T, LV>(v, i);
      T l[16];
      if (SHARED) {
#pragma unroll
        for (int k = 0; k < 16; k++) l[k] = l0[k];
      } else if constexpr (sizeof(T) == 8) {  // 16-byte loads of the vector's own matrix
        const double2 *q = reinterpret_cast<const double2 *>(L) + 8 * i;
#pragma unroll
        for (int k = 0; k < 8; k++) {
          const double2 t = __ldcs(q + k);
          l[2 * k] = t.x;
          l[2 * k + 1] = t.y;
        }
      } else {
        const float4 *q = reinterpret_cast<const float4 *>(L) + 4 * i;
#pragma unroll
        for (int k = 0; k < 4; k++) {
          const float4 t = __ldcs(q + k);
          l[4 * k] = t.x;
          l[4 * k + 1] = t.y;
          l[4 * k + 2] = t.z;
          l[4 * k + 3] = t.w;
        }
      }
      st4<T, LO>(out, i, apply_fma(l, x));
    }
  }
}

// One leg to PxPyPzE in FP64 (the float-float path, FP64 outside its domain); coords as in
// gvx_coords.
__device__ __forceinline__ void to_cart_f64(const V4<double> &x, int coords, const ffm::LcTab &T,
                                            double *o) {
  if (coords == GVX_PXPYPZM) {
    const double xv[4] = {x.x, x.y, x.z, x.w};
    if (!ffm::pxpypzm_to_cart(xv, o)) {
      o[0] = x.x;
      o[1] = x.y;
      o[2] = x.z;
      o[3] = sqrt(fma(x.x, x.x, fma(x.y, x.y, fma(x.z, x.z, x.w * x.w))));
    }
    return;
  }
  const bool e_stored = coords == GVX_PTETAPHIE;
  if (!ffm::ptetaphi_to_cart_lc(x.x, x.y, x.z, x.w, e_stored, T, o)) {
    double sn, cs;
    sincos(x.z, &sn, &cs);
    o[0] = x.x * cs;
    o[1] = x.x * sn;
    o[2] = x.x * sinh(x.y);
    o[3] = e_stored ? x.w : hypot(x.x * cosh(x.y), x.w);
  }
}

// The same in FP32 with CUDA's float functions.
__device__ __forceinline__ void to_cart_f32(const V4<float> &x, int coords, float *o) {
  if (coords == GVX_PXPYPZM) {
    o[0] = x.x;
    o[1] = x.y;
    o[2] = x.z;
    o[3] = norm4df(x.x, x.y, x.z, x.w);
    return;
  }
  float sn, cs;
  sincosf(x.z, &sn, &cs);
  o[0] = x.x * cs;
  o[1] = x.x * sn;
  o[2] = x.x * sinhf(x.y);
  o[3] = coords == GVX_PTETAPHIE ? x.w : hypotf(x.x * coshf(x.y), x.w);
}

template <typename T, int LV, int LO, int COORDS>
__global__ void __launch_bounds__(256) to_pxpypze_kernel(Lv v, LvOut out, int64_t n) {
  const ffm::LcTab T_{ffm::kHypTab, ffm::kSinTab};  // read through L1
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  V4<T> xn = {0, 0, 0, 0};
  if (i < n) xn = ld4<T, LV>(v, i);
  for (; i < n; i += stride) {
    const V4<T> x = xn;  // the next vector's loads go out before this one's arithmetic
    if (i + stride < n) xn = ld4<T, LV>(v, i + stride);
    T o[4];
    if constexpr (sizeof(T) == 8) {
      to_cart_f64(x, COORDS, T_, o);
    } else {
      to_cart_f32(x, COORDS, o);
    }
    st4<T, LO>(out, i, V4<T>{o[0], o[1], o[2], o[3]});
  }
}

// FP32 PtEtaPhiE pair mass in the form of the FP32 PtEtaPhiM one (pair_math.cuh pair_terms), the
// mass of v1 + v2 (Sec. 4.1): with P_i = pt_i cosh(eta_i), the stored E_i,
// m_i^2 = (E_i - P_i)(E_i + P_i), Q = E_1 E_2 - P_1 P_2 and S = sinh^2(d_eta/2) + sin^2(d_phi/2),
//   m^2 = m_1^2 + m_2^2 + 2 Q + 4 pt_1 pt_2 S     (P_1 P_2 - p_1.p_2 = 2 pt_1 pt_2 S).
// Every term is bounded by (M_1 + M_2)^2, M_i = max(|E_i|, |P_i|), and carries a few ulps of it,
// so the error in m|m| stays within ~8 u (M_1 + M_2)^2 (u = 2^-24).  A spacelike sum gives
// -sqrt(-m^2).  False when m^2 is not finite (the caller takes the exact route).
__device__ __forceinline__ bool pair_mass_e_f32(const V4<float> &x, const V4<float> &y, float *r) {
  const float P1 = x.x * coshf(x.y), P2 = y.x * coshf(y.y);
  const float q1 = (x.w - P1) * (x.w + P1), q2 = (y.w - P2) * (y.w + P2);
  const float Q = fmaf(x.w, y.w, -P1 * P2);
  const float se = sinhf(0.5f * (x.y - y.y));
  const float sp = sinf(half_dphi(x.z, y.z));
  const float S = fmaf(se, se, sp * sp);
  const float m2 = fmaf(4.0f * x.x * y.x, S, fmaf(2.0f, Q, q1 + q2));
  if (!isfinite(m2)) return false;
  *r = m2 >= 0.0f ? sqrtf(m2) : -sqrtf(-m2);
  return true;
}

__device__ __forceinline__ float pair_mass_e_f32_any(const V4<float> &x, const V4<float> &y) {
  float r;
  if (pair_mass_e_f32(x, y, &r)) return r;
  float ca[4], cb[4];
  to_cart_f32(x, GVX_PTETAPHIE, ca);
  to_cart_f32(y, GVX_PTETAPHIE, cb);
  if (!cfix::mass_pxpypze(ca, cb, &r)) {
    const double pa[4] = {ca[0], ca[1], ca[2], ca[3]}, pb[4] = {cb[0], cb[1], cb[2], cb[3]};
    r = (float)cart::mass(pa, pb, 0);
  }
  return r;
}

// FP32 PtEtaPhiE pair masses: HBM-bound, so each thread loads kUnrollE pairs (strided by the grid)
// before it computes any of them, to keep more loads in flight per SM.
constexpr int kUnrollE = 4;

template <int LA, int LB>
__global__ void __launch_bounds__(256) mass_ptetaphie_f32_kernel(Lv a, Lv b, float *__restrict__ m,
                                                                 int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (kUnrollE - 1) * stride < n; i += kUnrollE * stride) {
    V4<float> x[kUnrollE], y[kUnrollE];
#pragma unroll
    for (int u = 0; u < kUnrollE; u++) {
      x[u] = ld4<float, LA>(a, i + u * stride);
      y[u] = ld4<float, LB>(b, i + u * stride);
    }
#pragma unroll
    for (int u = 0; u < kUnrollE; u++) st_s(m + i + u * stride, pair_mass_e_f32_any(x[u], y[u]));
  }
  for (; i < n; i += stride) st_s(m + i, pair_mass_e_f32_any(ld4<float, LA>(a, i), ld4<float, LB>(b, i)));
}

// Pair masses of PtEtaPhiE legs in FP64: the light-cone form of ptetaphie_lc.cuh; outside its
// domain both legs converted as above, then the exact fixed-point mass of the converted legs
// (cart_fixed.cuh), the FP64 form outside that one's domain.  (FP32: mass_ptetaphie_f32_kernel.)
template <typename T, int LA, int LB>
__global__ void __launch_bounds__(256, 4) mass_ptetaphie_kernel(Lv a, Lv b, T *__restrict__ m, int64_t n) {
  // the light-cone tables of the fast path and of the conversion route, read through L1
  const ffm::LcTab L{ffm::kHypTab, ffm::kSinTab};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const V4<T> x = ld4<T, LA>(a, i), y = ld4<T, LB>(b, i);
    T ca[4], cb[4], r;
    if constexpr (sizeof(T) == 8) {
      double rf;
      if (ffm::pair_mass_e_lc(x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w, L, &rf)) {
        st_s(m + i, rf);  // the light-cone form, legs paired (ptetaphie_lc.cuh)
        continue;
      }
      to_cart_f64(x, GVX_PTETAPHIE, L, ca);
      to_cart_f64(y, GVX_PTETAPHIE, L, cb);
    } else {
      to_cart_f32(x, GVX_PTETAPHIE, ca);
      to_cart_f32(y, GVX_PTETAPHIE, cb);
    }
    if (!cfix::mass_pxpypze(ca, cb, &r)) {
      const double pa[4] = {ca[0], ca[1], ca[2], ca[3]}, pb[4] = {cb[0], cb[1], cb[2], cb[3]};
      r = (T)cart::mass(pa, pb, 0);
    }
    st_s(m + i, r);
  }
}

template <typename T, int COORDS>
cudaError_t launch_cart_t(const Lv &a, const Lv &b, T *m, int64_t n, cudaStream_t s) {
  const int threads = 256;
  if (a.layout == GVX_SOA && b.layout == GVX_SOA) {
    constexpr auto k = mass_cart_kernel<T, GVX_SOA, GVX_SOA, COORDS>;
    k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(a, b, m, n);
  } else if (a.layout == GVX_SOA) {
    constexpr auto k = mass_cart_kernel<T, GVX_SOA, GVX_AOS, COORDS>;
    k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(a, b, m, n);
  } else if (b.layout == GVX_SOA) {
    constexpr auto k = mass_cart_kernel<T, GVX_AOS, GVX_SOA, COORDS>;
    k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(a, b, m, n);
  } else {
    constexpr auto k = mass_cart_kernel<T, GVX_AOS, GVX_AOS, COORDS>;
    k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(a, b, m, n);
  }
  return cudaGetLastError();
}

template <typename T, bool SHARED>
cudaError_t launch_apply_t(const T *L, const Lv &v, const LvOut &out, int64_t n, cudaStream_t s) {
  const int threads = 256;
  if (v.layout == GVX_SOA && out.layout == GVX_SOA) {
    constexpr auto k = lorentz_apply_kernel<T, GVX_SOA, GVX_SOA, SHARED>;
    k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(L, v, out, n);
  } else if (v.layout == GVX_SOA) {
    constexpr auto k = lorentz_apply_kernel<T, GVX_SOA, GVX_AOS, SHARED>;
    k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(L, v, out, n);
  } else if (out.layout == GVX_SOA) {
    constexpr auto k = lorentz_apply_kernel<T, GVX_AOS, GVX_SOA, SHARED>;
    k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(L, v, out, n);
  } else {
    constexpr auto k = lorentz_apply_kernel<T, GVX_AOS, GVX_AOS, SHARED>;
    k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(L, v, out, n);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ptetaphie_t(const Lv &a, const Lv &b, T *m, int64_t n, cudaStream_t s) {
  const int threads = 256;
  if constexpr (sizeof(T) == 4) {
    if (a.layout == GVX_SOA && b.layout == GVX_SOA) {
      constexpr auto k = mass_ptetaphie_f32_kernel<GVX_SOA, GVX_SOA>;
      k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(a, b, m, n);
    } else if (a.layout == GVX_SOA) {
      constexpr auto k = mass_ptetaphie_f32_kernel<GVX_SOA, GVX_AOS>;
      k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(a, b, m, n);
    } else if (b.layout == GVX_SOA) {
      constexpr auto k = mass_ptetaphie_f32_kernel<GVX_AOS, GVX_SOA>;
      k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(a, b, m, n);
    } else {
      constexpr auto k = mass_ptetaphie_f32_kernel<GVX_AOS, GVX_AOS>;
      k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(a, b, m, n);
    }
    return cudaGetLastError();
  }
  if (a.layout == GVX_SOA && b.layout == GVX_SOA) {
    constexpr auto k = mass_ptetaphie_kernel<T, GVX_SOA, GVX_SOA>;
    k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(a, b, m, n);
  } else if (a.layout == GVX_SOA) {
    constexpr auto k = mass_ptetaphie_kernel<T, GVX_SOA, GVX_AOS>;
    k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(a, b, m, n);
  } else if (b.layout == GVX_SOA) {
    constexpr auto k = mass_ptetaphie_kernel<T, GVX_AOS, GVX_SOA>;
    k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(a, b, m, n);
  } else {
    constexpr auto k = mass_ptetaphie_kernel<T, GVX_AOS, GVX_AOS>;
    k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(a, b, m, n);
  }
  return cudaGetLastError();
}

template <typename T, int COORDS>
cudaError_t launch_convert_t(const Lv &v, const LvOut &out, int64_t n, cudaStream_t s) {
  const int threads = 256;
  if (v.layout == GVX_SOA && out.layout == GVX_SOA) {
    constexpr auto k = to_pxpypze_kernel<T, GVX_SOA, GVX_SOA, COORDS>;
    k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(v, out, n);
  } else if (v.layout == GVX_SOA) {
    constexpr auto k = to_pxpypze_kernel<T, GVX_SOA, GVX_AOS, COORDS>;
    k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(v, out, n);
  } else if (out.layout == GVX_SOA) {
    constexpr auto k = to_pxpypze_kernel<T, GVX_AOS, GVX_SOA, COORDS>;
    k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(v, out, n);
  } else {
    constexpr auto k = to_pxpypze_kernel<T, GVX_AOS, GVX_AOS, COORDS>;
    k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(v, out, n);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_convert_c(const Lv &v, const LvOut &out, int64_t n, int coords, cudaStream_t s) {
  if (coords == GVX_PTETAPHIM) return launch_convert_t<T, GVX_PTETAPHIM>(v, out, n, s);
  if (coords == GVX_PTETAPHIE) return launch_convert_t<T, GVX_PTETAPHIE>(v, out, n, s);
  return launch_convert_t<T, GVX_PXPYPZM>(v, out, n, s);
}

}  // namespace

cudaError_t launch_to_pxpypze(const Lv &v, const LvOut &out, int64_t n, int coords, int dtype,
                              cudaStream_t s) {
  return dtype == GVX_F64 ? launch_convert_c<double>(v, out, n, coords, s)
                          : launch_convert_c<float>(v, out, n, coords, s);
}

cudaError_t launch_mass_cart(const Lv &a, const Lv &b, void *m, int64_t n, int coords, int dtype,
                             cudaStream_t s) {
  if (coords == GVX_PTETAPHIE)
    return dtype == GVX_F64 ? launch_ptetaphie_t<double>(a, b, (double *)m, n, s)
                            : launch_ptetaphie_t<float>(a, b, (float *)m, n, s);
  if (dtype == GVX_F64)
    return coords == GVX_PXPYPZE ? launch_cart_t<double, 0>(a, b, (double *)m, n, s)
                                 : launch_cart_t<double, 1>(a, b, (double *)m, n, s);
  return coords == GVX_PXPYPZE ? launch_cart_t<float, 0>(a, b, (float *)m, n, s)
                               : launch_cart_t<float, 1>(a, b, (float *)m, n, s);
}

cudaError_t launch_lorentz_apply(const void *L, int64_t l_stride, const Lv &v, const LvOut &out,
                                 int64_t n, int dtype, cudaStream_t s) {
  if (dtype == GVX_F64)
    return l_stride == 0 ? launch_apply_t<double, true>((const double *)L, v, out, n, s)
                         : launch_apply_t<double, false>((const double *)L, v, out, n, s);
  return l_stride == 0 ? launch_apply_t<float, true>((const float *)L, v, out, n, s)
                       : launch_apply_t<float, false>((const float *)L, v, out, n, s);
}

}  // namespace gvx
