// Device-side helpers shared by the kernel translation units: layout-aware loads and stores of
// 4-vectors and velocities, and the launch-shape rule.
#pragma once

#include <stdint.h>

#include "gvx_internal.h"

namespace gvx {

template <typename T>
struct V4 {
  T x, y, z, w;
};
template <typename T>
struct V3 {
  T x, y, z;
};

// Streaming (evict-first) loads: every input element is read exactly once.
__device__ __forceinline__ double ld_s(const double *p) { return __ldcs(p); }
__device__ __forceinline__ float ld_s(const float *p) { return __ldcs(p); }
__device__ __forceinline__ void st_s(double *p, double v) { __stcs(p, v); }
__device__ __forceinline__ void st_s(float *p, float v) { __stcs(p, v); }

template <typename T, int LAYOUT>
__device__ __forceinline__ V4<T> ld4(const Lv &v, int64_t i) {
  if constexpr (LAYOUT == GVX_SOA) {
    return {ld_s((const T *)v.c[0] + i), ld_s((const T *)v.c[1] + i), ld_s((const T *)v.c[2] + i),
            ld_s((const T *)v.c[3] + i)};
  } else if constexpr (sizeof(T) == 8) {
    const double2 *p = (const double2 *)v.c[0] + 2 * i;
    double2 a = __ldcs(p), b = __ldcs(p + 1);
    return {a.x, a.y, b.x, b.y};
  } else {
    float4 a = __ldcs((const float4 *)v.c[0] + i);
    return {a.x, a.y, a.z, a.w};
  }
}

template <typename T, int LAYOUT>
__device__ __forceinline__ void st4(const LvOut &v, int64_t i, V4<T> x) {
  if constexpr (LAYOUT == GVX_SOA) {
    st_s((T *)v.c[0] + i, x.x);
    st_s((T *)v.c[1] + i, x.y);
    st_s((T *)v.c[2] + i, x.z);
    st_s((T *)v.c[3] + i, x.w);
  } else if constexpr (sizeof(T) == 8) {
    double2 *p = (double2 *)v.c[0] + 2 * i;
    __stcs(p, make_double2(x.x, x.y));
    __stcs(p + 1, make_double2(x.z, x.w));
  } else {
    __stcs((float4 *)v.c[0] + i, make_float4(x.x, x.y, x.z, x.w));
  }
}

// The same load through the read-only path with normal caching, for data that other threads
// read again soon (partners of a particle in an event).
template <int LAYOUT>
__device__ __forceinline__ V4<double> ld4c(const Lv &v, int64_t i) {
  if constexpr (LAYOUT == GVX_SOA) {
    return {__ldg((const double *)v.c[0] + i), __ldg((const double *)v.c[1] + i),
            __ldg((const double *)v.c[2] + i), __ldg((const double *)v.c[3] + i)};
  } else {
    const double2 *p = (const double2 *)v.c[0] + 2 * i;
    double2 a = __ldg(p), b = __ldg(p + 1);
    return {a.x, a.y, b.x, b.y};
  }
}

// Velocities: SoA c[0..2] or packed triples at c[0].  `i` is already multiplied by the stride.
template <typename T, int LAYOUT>
__device__ __forceinline__ V3<T> ld3(const Lv &v, int64_t i) {
  if constexpr (LAYOUT == GVX_SOA) {
    return {ld_s((const T *)v.c[0] + i), ld_s((const T *)v.c[1] + i), ld_s((const T *)v.c[2] + i)};
  } else {
    const T *p = (const T *)v.c[0] + 3 * i;
    return {ld_s(p), ld_s(p + 1), ld_s(p + 2)};
  }
}

template <typename T, int LAYOUT>
__device__ __forceinline__ void st3(const LvOut &v, int64_t i, V3<T> x) {
  if constexpr (LAYOUT == GVX_SOA) {
    st_s((T *)v.c[0] + i, x.x);
    st_s((T *)v.c[1] + i, x.y);
    st_s((T *)v.c[2] + i, x.z);
  } else {
    T *p = (T *)v.c[0] + 3 * i;
    st_s(p, x.x);
    st_s(p + 1, x.y);
    st_s(p + 2, x.z);
  }
}

// Grid for a grid-stride elementwise kernel: enough CTAs to fill every SM `per_sm` times,
// never more than the work needs.
inline unsigned grid_for(int64_t n, int threads, int per_sm) {
  int64_t need = (n + threads - 1) / threads;
  int64_t cap = (int64_t)num_sms() * per_sm;
  int64_t g = need < cap ? need : cap;
  return (unsigned)(g < 1 ? 1 : g);
}

// CTAs per resident slot for grid-stride kernels.  With several times more CTAs than fit at once,
// the hardware block scheduler hands the work out in smaller pieces and evens out SMs that run
// ahead or behind; on GB300 a grid of exactly one resident wave finished 9-10% later than eight
// waves on the FP64 mass and boost kernels (and sixteen waves gained nothing more).
constexpr int kWaves = 8;

// Grid for a grid-stride kernel: kWaves times the CTAs that can be resident at once (occupancy
// query, cached per kernel by the caller's static), never more than the work (n elements,
// per_block per CTA and pass; 0 means one per thread).
template <typename Kernel>
inline unsigned balanced_grid(Kernel k, int threads, size_t smem, int64_t n, int *cache,
                              int64_t per_block = 0, int waves = kWaves) {
  if (*cache <= 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    *cache = per_sm;
  }
  if (per_block <= 0) per_block = threads;
  int64_t need = (n + per_block - 1) / per_block;
  int64_t cap = (int64_t)num_sms() * *cache * waves;
  int64_t g = need < cap ? need : cap;
  return (unsigned)(g < 1 ? 1 : g);
}

// balanced_grid for one kernel instantiation, its occupancy cached per device.
template <auto Kernel>
inline unsigned balanced_grid_of(int threads, size_t smem, int64_t n, int64_t per_block = 0,
                                 int waves = kWaves) {
  static int occ[64];
  int dev = 0;
  cudaGetDevice(&dev);
  return balanced_grid(Kernel, threads, smem, n, &occ[dev & 63], per_block, waves);
}

// Record a device-detected error (the first one since the last read wins).
__device__ __forceinline__ void raise_status(int32_t *word, int32_t code) {
  atomicCAS(word, 0, code);
}

// Explicit index checks at the computed indices of the jagged kernels (partners, pair slots,
// pair gradients, particles).  In a build with GVX_DEBUG_BOUNDS defined a failed check records
// GVX_ERR_BOUNDS and the caller skips the access; otherwise the checks compile to nothing.
#ifdef GVX_DEBUG_BOUNDS
__device__ __forceinline__ bool in_bounds(int64_t i, int64_t n, int32_t *status) {
  if (i >= 0 && i < n) return true;
  raise_status(status, GVX_ERR_BOUNDS);
  return false;
}
#define GVX_IN_BOUNDS(i, n, status) ::gvx::in_bounds((int64_t)(i), (int64_t)(n), (status))
#else
#define GVX_IN_BOUNDS(i, n, status) true
#endif

}  // namespace gvx
