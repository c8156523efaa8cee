// Lorentz boost of PxPyPzE vectors and its adjoint (GenVectorX, Sec. 4.1: ApplyBoost applies a
// 4x4 Lorentz matrix to every vector of an array).
//
// The symmetric matrix L(beta) is applied without being formed:
//   gamma = 1/sqrt(1 - b2),  bp = beta.p,  E' = gamma (E + bp),
//   p' = p + f beta,  f = k bp + gamma E = E' - w bp,   k = gamma^2/(1 + gamma),  w = gamma/(1 + gamma).
// The form f = E' - w bp keeps gamma out of the part of f that cancels when a vector is boosted
// towards its rest frame (p' -> 0): an error in gamma then scales E' only, and only w's error is
// amplified.  1 - b2 is formed from exact squares and error-free sums, so gamma keeps the
// working precision as |beta| -> 1 instead of losing log10(1/(1 - b2)) digits.
//
// FP64: the fast path (boost_ff.cuh) forms gamma and f = k (E + bp) + w E in float-float on the
// FP32 pipe and keeps seven FP64 operations per vector; vectors outside its domain take the FP64
// evaluation below, with the compensated 1 - b2.
#include <cuda_runtime.h>

#include "boost_ff.cuh"
#include "common.cuh"
#include "ff.cuh"

namespace gvx {
namespace {

template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T &s, T &e) {
  s = a + b;
  T bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// 1 - (bx^2 + by^2 + bz^2), correctly rounded up to a few ulps of the result.
template <typename T>
__device__ __forceinline__ T one_minus_b2(V3<T> b) {
  T px = b.x * b.x, py = b.y * b.y, pz = b.z * b.z;
  T lo = -((fma(b.x, b.x, -px) + fma(b.y, b.y, -py)) + fma(b.z, b.z, -pz));
  T r, e1, e2, e3;
  two_sum((T)1, -px, r, e1);
  two_sum(r, -py, r, e2);
  two_sum(r, -pz, r, e3);
  return r + (lo + ((e1 + e2) + e3));
}

__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_(float x) { return 1.0f / sqrtf(x); }

template <typename T>
struct BoostCoef {
  T g, w;
  bool ok;
};

template <typename T>
__device__ __forceinline__ BoostCoef<T> boost_coef(V3<T> b) {
  BoostCoef<T> c;
  T omb = one_minus_b2(b);
  c.ok = omb > (T)0;
  c.g = rsqrt_(omb);
  c.w = c.g / ((T)1 + c.g);
  return c;
}

template <typename T>
__device__ __forceinline__ V4<T> apply_boost(V3<T> b, BoostCoef<T> c, V4<T> v) {
  if (!c.ok) {
    const T nan = (T)NAN;
    return {nan, nan, nan, nan};
  }
  T bp = fma(b.x, v.x, fma(b.y, v.y, b.z * v.z));
  T ep = c.g * (v.w + bp);
  T f = fma(-c.w, bp, ep);
  return {fma(f, b.x, v.x), fma(f, b.y, v.y), fma(f, b.z, v.z), ep};
}

template <typename T, int LV, int LBETA, int LOUT, bool SHARED>
__global__ void __launch_bounds__(256) boost_kernel(Lv v, Lv beta, LvOut out, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  V3<T> b0;
  if (SHARED) b0 = ld3<T, LBETA>(beta, 0);
  if constexpr (sizeof(T) == 8) {
    ffm::BetaFF B0;
    if (SHARED) B0 = ffm::beta_ff(b0.x, b0.y, b0.z);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      V4<T> x = ld4<T, LV>(v, i);
      V3<T> b = SHARED ? b0 : ld3<T, LBETA>(beta, i);
      const ffm::BetaFF B = SHARED ? B0 : ffm::beta_ff(b.x, b.y, b.z);
      double o[4];
      V4<T> r;
      if (ffm::boost_ff(B, b.x, b.y, b.z, x.x, x.y, x.z, x.w, o))
        r = {o[0], o[1], o[2], o[3]};
      else
        r = apply_boost(b, boost_coef(b), x);
      st4<T, LOUT>(out, i, r);
    }
  } else {
    // FP32: memory-bound, so each thread loads kUnroll vectors (strided by the grid) before it
    // computes any of them, to keep more loads in flight per SM.
    constexpr int kUnroll = 4;
    BoostCoef<T> c0;
    if (SHARED) c0 = boost_coef(b0);
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + (kUnroll - 1) * stride < n; i += kUnroll * stride) {
      V4<T> x[kUnroll];
      V3<T> b[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; u++) {
        x[u] = ld4<T, LV>(v, i + u * stride);
        b[u] = SHARED ? b0 : ld3<T, LBETA>(beta, i + u * stride);
      }
#pragma unroll
      for (int u = 0; u < kUnroll; u++)
        st4<T, LOUT>(out, i + u * stride, apply_boost(b[u], SHARED ? c0 : boost_coef(b[u]), x[u]));
    }
    for (; i < n; i += stride) {
      V4<T> x = ld4<T, LV>(v, i);
      V3<T> b = SHARED ? b0 : ld3<T, LBETA>(beta, i);
      st4<T, LOUT>(out, i, apply_boost(b, SHARED ? c0 : boost_coef(b), x));
    }
  }
}

// Adjoint.  grad_v = L grad_out (L symmetric: the same boost applied to grad_out).  With
// gb = beta . grad_p, k' = dk/dgamma = gamma (gamma + 2)/(gamma + 1)^2, f = k bp + gamma E:
//   grad_beta = gamma^3 [gb (k' bp + E) + gE (E + bp)] beta + (k gb + gamma gE) p + f grad_p.
// This is the FP32 evaluation and the FP64 one outside the float-float domain (there gamma, k,
// k' = (1 + 2 s)/(1 + s)^2 and gamma^3, s = 1/gamma = sqrt(1 - b2), come from float-float
// arithmetic and the multiply-adds stay in FP64); FP64 inputs inside it take boost_bwd_ff
// (boost_ff.cuh), which keeps 15 FP64 operations per vector.
template <typename T>
struct BoostCoefBwd {
  BoostCoef<T> c;
  T k, kp, g3;
};

template <typename T>
__device__ __forceinline__ BoostCoefBwd<T> boost_coef_bwd(V3<T> b) {
  if constexpr (sizeof(T) == 8) {
    bool ok = true;
    ffm::ff omb = ffm::one_minus_sq3(b.x, b.y, b.z, &ok);
    if (ok) {
      ffm::ff s = ffm::sqrt(omb);
      ffm::ff g = ffm::recip(s);
      ffm::ff w = ffm::recip(ffm::add_same(ffm::make(1.0f), s));
      ffm::ff k = ffm::mul(g, w);
      ffm::ff kp = ffm::mul(ffm::add_same(ffm::make(1.0f), ffm::scale(s, 2.0f)), ffm::sqr(w));
      ffm::ff g3 = ffm::mul(ffm::sqr(g), g);
      BoostCoefBwd<T> r;
      r.c = {ffm::to_double(ffm::renorm(g)), ffm::to_double(ffm::renorm(w)), true};
      r.k = ffm::to_double(ffm::renorm(k));
      r.kp = ffm::to_double(ffm::renorm(kp));
      r.g3 = ffm::to_double(ffm::renorm(g3));
      return r;
    }
  }
  BoostCoefBwd<T> r;
  r.c = boost_coef(b);
  r.k = r.c.g * r.c.w;
  T gp1 = r.c.g + (T)1;
  r.kp = r.c.g * (r.c.g + (T)2) / (gp1 * gp1);
  r.g3 = r.c.g * r.c.g * r.c.g;
  return r;
}

template <typename T>
__device__ __forceinline__ void boost_grads(V3<T> b, BoostCoefBwd<T> cb, V4<T> v, V4<T> g,
                                            V4<T> &gv, V3<T> &gbeta) {
  const BoostCoef<T> &c = cb.c;
  if (!c.ok) {
    const T nan = (T)NAN;
    gv = {nan, nan, nan, nan};
    gbeta = {nan, nan, nan};
    return;
  }
  gv = apply_boost(b, c, g);
  T bp = fma(b.x, v.x, fma(b.y, v.y, b.z * v.z));
  T gb = fma(b.x, g.x, fma(b.y, g.y, b.z * g.z));
  T f = fma(-c.w, bp, c.g * (v.w + bp));
  T kp = cb.kp;
  T g3 = cb.g3;
  T A = g3 * fma(gb, fma(kp, bp, v.w), g.w * (v.w + bp));
  T B = fma(cb.k, gb, c.g * g.w);
  gbeta.x = fma(A, b.x, fma(B, v.x, f * g.x));
  gbeta.y = fma(A, b.y, fma(B, v.y, f * g.y));
  gbeta.z = fma(A, b.z, fma(B, v.z, f * g.z));
}

// Both adjoint outputs for one vector: the float-float path (boost_ff.cuh) for FP64 inputs in its
// domain, the FP64 (or FP32) formulas above otherwise.
template <typename T>
__device__ __forceinline__ void boost_grads_any(V3<T> b, const ffm::BetaBwdFF &B,
                                                const BoostCoefBwd<T> *cb, V4<T> x, V4<T> g,
                                                V4<T> &ogv, V3<T> &ogb) {
  if constexpr (sizeof(T) == 8) {
    const double p[4] = {x.x, x.y, x.z, x.w}, q[4] = {g.x, g.y, g.z, g.w};
    double o[4], ob[3];
    if (ffm::boost_bwd_ff(B, b.x, b.y, b.z, p, q, o, ob)) {
      ogv = {o[0], o[1], o[2], o[3]};
      ogb = {ob[0], ob[1], ob[2]};
      return;
    }
  }
  boost_grads(b, cb ? *cb : boost_coef_bwd(b), x, g, ogv, ogb);
}

template <typename T>
__device__ __forceinline__ ffm::BetaBwdFF beta_bwd_any(V3<T> b) {
  if constexpr (sizeof(T) == 8) return ffm::beta_bwd_ff(b.x, b.y, b.z);
  ffm::BetaBwdFF B;
  B.ok = false;
  return B;
}

template <typename T, int LV, int LBETA, int LG, int LGV, int LGB>
__global__ void __launch_bounds__(256) boost_bwd_kernel(Lv v, Lv beta, Lv gout, LvOut gv,
                                                        LvOut gbeta, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    V4<T> x = ld4<T, LV>(v, i);
    V3<T> b = ld3<T, LBETA>(beta, i);
    V4<T> g = ld4<T, LG>(gout, i);
    V4<T> ogv;
    V3<T> ogb;
    boost_grads_any(b, beta_bwd_any(b), (const BoostCoefBwd<T> *)nullptr, x, g, ogv, ogb);
    st4<T, LGV>(gv, i, ogv);
    st3<T, LGB>(gbeta, i, ogb);
  }
}

// Shared velocity: grad_beta is a sum over all vectors.  Each CTA writes its partial sum (in
// double) to ws[3 * blockIdx.x + k]; a second one-CTA kernel adds the partials in a fixed order,
// so the result does not depend on scheduling.
constexpr int kBwdThreads = 256;

template <typename T, int LV, int LBETA, int LG, int LGV>
__global__ void __launch_bounds__(kBwdThreads) boost_bwd_shared_kernel(Lv v, Lv beta, Lv gout,
                                                                       LvOut gv, double *ws,
                                                                       int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  V3<T> b = ld3<T, LBETA>(beta, 0);
  const BoostCoefBwd<T> c = boost_coef_bwd(b);
  const ffm::BetaBwdFF B = beta_bwd_any(b);
  double acc[3] = {0, 0, 0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    V4<T> x = ld4<T, LV>(v, i);
    V4<T> g = ld4<T, LG>(gout, i);
    V4<T> ogv;
    V3<T> ogb;
    boost_grads_any(b, B, &c, x, g, ogv, ogb);
    st4<T, LGV>(gv, i, ogv);
    acc[0] += (double)ogb.x;
    acc[1] += (double)ogb.y;
    acc[2] += (double)ogb.z;
  }
  __shared__ double red[3][kBwdThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 3; k++) {
    double s = acc[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[k][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0;
    for (int w = 0; w < kBwdThreads / 32; w++) s += red[threadIdx.x][w];
    ws[3 * blockIdx.x + threadIdx.x] = s;
  }
}

template <typename T, int LGB>
__global__ void __launch_bounds__(kBwdThreads) reduce_partials_kernel(const double *ws, int parts,
                                                                      LvOut gbeta) {
  __shared__ double red[3][kBwdThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 3; k++) {
    double s = 0;
    for (int p = threadIdx.x; p < parts; p += blockDim.x) s += ws[3 * p + k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[k][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s[3] = {0, 0, 0};
    for (int k = 0; k < 3; k++)
      for (int w = 0; w < kBwdThreads / 32; w++) s[k] += red[k][w];
    st3<T, LGB>(gbeta, 0, V3<T>{(T)s[0], (T)s[1], (T)s[2]});
  }
}

constexpr int kSoA = GVX_SOA, kAoS = GVX_AOS;

// Runtime layout flags -> template instantiation.
template <typename F>
void dispatch2(int l0, int l1, F &&f) {
  if (l0 == kSoA && l1 == kSoA) f(std::integral_constant<int, kSoA>{}, std::integral_constant<int, kSoA>{});
  else if (l0 == kSoA) f(std::integral_constant<int, kSoA>{}, std::integral_constant<int, kAoS>{});
  else if (l1 == kSoA) f(std::integral_constant<int, kAoS>{}, std::integral_constant<int, kSoA>{});
  else f(std::integral_constant<int, kAoS>{}, std::integral_constant<int, kAoS>{});
}

template <typename T>
cudaError_t launch_boost_t(const Lv &v, const Lv &beta, int64_t stride, const LvOut &out,
                           int64_t n, cudaStream_t s) {
  const int threads = 256;
  dispatch2(v.layout, out.layout, [&](auto LV, auto LO) {
    dispatch2(beta.layout, kSoA, [&](auto LB, auto) {
      if (stride == 0) {
        constexpr auto k = boost_kernel<T, LV, LB, LO, true>;
        k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(v, beta, out, n);
      } else {
        constexpr auto k = boost_kernel<T, LV, LB, LO, false>;
        k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(v, beta, out, n);
      }
    });
  });
  return cudaGetLastError();
}

unsigned bwd_shared_grid(int64_t n) { return grid_for(n, kBwdThreads, 4); }

template <typename T>
cudaError_t launch_boost_bwd_t(const Lv &v, const Lv &beta, int64_t stride, const Lv &gout,
                               const LvOut &gv, const LvOut &gbeta, int64_t n, void *ws,
                               cudaStream_t s) {
  if (stride == 0) {
    unsigned grid = bwd_shared_grid(n);
    double *w = (double *)ws;
    dispatch2(v.layout, gout.layout, [&](auto LV, auto LG) {
      dispatch2(beta.layout, gv.layout, [&](auto LB, auto LGV) {
        boost_bwd_shared_kernel<T, LV, LB, LG, LGV><<<grid, kBwdThreads, 0, s>>>(v, beta, gout, gv,
                                                                                w, n);
      });
    });
    if (gbeta.layout == kSoA)
      reduce_partials_kernel<T, kSoA><<<1, kBwdThreads, 0, s>>>(w, (int)grid, gbeta);
    else
      reduce_partials_kernel<T, kAoS><<<1, kBwdThreads, 0, s>>>(w, (int)grid, gbeta);
    return cudaGetLastError();
  }
  const int threads = 256;
  dispatch2(v.layout, gout.layout, [&](auto LV, auto LG) {
    dispatch2(beta.layout, gv.layout, [&](auto LB, auto LGV) {
      if (gbeta.layout == kSoA) {
        constexpr auto k = boost_bwd_kernel<T, LV, LB, LG, LGV, kSoA>;
        k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(v, beta, gout, gv, gbeta, n);
      } else {
        constexpr auto k = boost_bwd_kernel<T, LV, LB, LG, LGV, kAoS>;
        k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(v, beta, gout, gv, gbeta, n);
      }
    });
  });
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_boost(const Lv &v, const Lv &beta, int64_t beta_stride, const LvOut &out,
                         int64_t n, int dtype, cudaStream_t s) {
  return dtype == GVX_F64 ? launch_boost_t<double>(v, beta, beta_stride, out, n, s)
                          : launch_boost_t<float>(v, beta, beta_stride, out, n, s);
}

size_t boost_bwd_workspace(int64_t n, int64_t beta_stride, int dtype) {
  (void)dtype;
  if (beta_stride != 0 || n == 0) return 0;
  return (size_t)bwd_shared_grid(n) * 3 * sizeof(double);
}

cudaError_t launch_boost_bwd(const Lv &v, const Lv &beta, int64_t beta_stride, const Lv &gout,
                             const LvOut &gv, const LvOut &gbeta, int64_t n, int dtype, void *ws,
                             cudaStream_t s) {
  return dtype == GVX_F64
             ? launch_boost_bwd_t<double>(v, beta, beta_stride, gout, gv, gbeta, n, ws, s)
             : launch_boost_bwd_t<float>(v, beta, beta_stride, gout, gv, gbeta, n, ws, s);
}

}  // namespace gvx
