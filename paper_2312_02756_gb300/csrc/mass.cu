// Invariant mass of pairs of PtEtaPhiM vectors and its adjoint (GenVectorX, Sec. 4.1, Fig. 1:
// per index, the two vectors are added and the mass of the sum is stored).
//
// The plain form sqrt(E^2 - |P|^2) cancels catastrophically for light, collinear pairs.  Both
// precisions use the identity (all terms >= 0 for pt >= 0)
//   m^2 = m1^2 + m2^2 + 2 (m1^2 P2^2 + m2^2 P1^2 + m1^2 m2^2) / (E1 E2 + P1 P2)
//             + 4 pt1 pt2 (sinh^2(d_eta/2) + sin^2(d_phi/2)),
// with P_i = pt_i cosh(eta_i) = |p_i| and E_i = sqrt(P_i^2 + m_i^2): a relative error of a few
// ulps whatever the cancellation in the plain form.
//
// FP64 forward: float-float on the FP32 pipe -- a GB300 SM retires ~64x more FP32 than FP64
// operations -- through the light-cone form of the same mass (mass_lc.cuh): with D = E - P and
// Y = E + P per leg, m^2 = (D1 + D2)(Y1 + Y2) + 4 pt1 pt2 (sinh^2(d_eta/2) + sin^2(d_phi/2)),
// again all terms non-negative.  The FP64 evaluation is kept for the rare lanes outside the
// float-float domain (|eta| >= 8, extreme scale ratios, |d_phi| near 2 pi).
#include <cuda_runtime.h>

#include "common.cuh"
#include "mass_lc.cuh"
#include "mass_lc_grad.cuh"
#include "pair_math.cuh"

namespace gvx {
namespace {

// FP32: memory-bound, so each thread loads kUnroll pairs (strided by the grid) before it
// computes any of them, to keep more loads in flight per SM.
constexpr int kUnroll = 4;

// Grid of the FP64 kernels: 32 times the resident CTAs (small CTAs and many waves even out the
// SMs' progress).
constexpr int kMassWaves = 32;

template <typename T, int LA, int LB>
__global__ void __launch_bounds__(256) mass_kernel(Lv a, Lv b, T *__restrict__ m, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (kUnroll - 1) * stride < n; i += kUnroll * stride) {
    V4<T> x[kUnroll], y[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
      x[u] = ld4<T, LA>(a, i + u * stride);
      y[u] = ld4<T, LB>(b, i + u * stride);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; u++)
      st_s(m + i + u * stride, sqrt_(pair_terms(make_leg(x[u]), make_leg(y[u])).m2));
  }
  for (; i < n; i += stride) {
    Leg<T> la = make_leg(ld4<T, LA>(a, i));
    Leg<T> lb = make_leg(ld4<T, LB>(b, i));
    st_s(m + i, sqrt_(pair_terms(la, lb).m2));
  }
}

// One FP64 pair: the light-cone float-float fast path (mass_lc.cuh), the FP64 formulas for a
// lane outside its domain.
__device__ __forceinline__ double pair_mass_f64(const V4<double> &x, const V4<double> &y,
                                                const ffm::LcTab &T) {
  double out;
  if (!ffm::pair_mass_lc(x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w, T, &out))
    out = sqrt(pair_terms(make_leg(x), make_leg(y)).m2);
  return out;
}

// FP64 forward: grid-stride, one pair per thread and step; 64 registers, eight CTAs of 128
// threads per SM, a grid of 32 times the resident CTAs (small CTAs and many waves even out the
// SMs' progress: 2-3% faster than four CTAs of 256 and 8 waves on GB300).  For a leg in SoA layout (four separate arrays), lanes 0..7 of each warp
// first ask L2 to prefetch the warp's next 32 elements of each array (one 128-byte line per
// lane), so that the next step's eight loads find them in L2 rather than in HBM.
template <int LA, int LB>
__global__ void __launch_bounds__(128, 8) mass_f64_kernel(Lv a, Lv b, double *__restrict__ m, int64_t n) {
  const ffm::LcTab T{ffm::kHypTab, ffm::kSinTab};
  const int lane = threadIdx.x & 31;
  const int leg = (lane >> 2) & 1;  // lanes 0-3: leg a's arrays, 4-7: leg b's
  const bool soa = leg ? LB == GVX_SOA : LA == GVX_SOA;
  // the lane's array by selects (an index into the parameters would copy them to local memory)
  const void *pa = (lane & 2) ? ((lane & 1) ? a.c[3] : a.c[2]) : ((lane & 1) ? a.c[1] : a.c[0]);
  const void *pb = (lane & 2) ? ((lane & 1) ? b.c[3] : b.c[2]) : ((lane & 1) ? b.c[1] : b.c[0]);
  const char *pbase = (const char *)(leg ? pb : pa) + 128 * ((lane >> 3) & 1);
  const bool prefetch = soa && lane < 16;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int64_t next = i - lane + stride;  // the warp's first element of the next step
    if (prefetch && next + 32 <= n) asm volatile("prefetch.global.L2 [%0];" ::"l"(pbase + 8 * next));
    st_s(m + i, pair_mass_f64(ld4<double, LA>(a, i), ld4<double, LB>(b, i), T));
  }
}

// cosh and sinh of x in FP32 from one exponential: (e + 1/e)/2 and (e - 1/e)/2, e = exp(|x|);
// below |x| = 1/4 sinh from its Taylor series to x^7 (the difference would lose relative digits).
__device__ __forceinline__ void hyp_pair_f32(float x, float *ch, float *sh) {
  const float ax = fabsf(x), e = expf(ax), r = 1.0f / e;
  *ch = 0.5f * (e + r);
  const float x2 = ax * ax;
  const float taylor = ax * fmaf(x2, fmaf(x2, fmaf(x2, 1.0f / 5040.0f, 1.0f / 120.0f), 1.0f / 6.0f), 1.0f);
  *sh = copysignf(ax < 0.25f ? taylor : 0.5f * (e - r), x);
}

// The FP32 pair-mass adjoint: the formulas of pair_mass_grad (pair_math.cuh) with each leg's
// cosh and sinh from one exponential, the half-angle terms of d_eta from another, sin and cos of
// the azimuthal half-angle from one sincosf, and the forward's mass where it is given.
__device__ __forceinline__ void pair_mass_grad_f32(const V4<float> &x, const V4<float> &y, float g,
                                                   bool has_ms, float ms, V4<float> &g1,
                                                   V4<float> &g2) {
  g1 = {0.0f, 0.0f, 0.0f, 0.0f};
  g2 = {0.0f, 0.0f, 0.0f, 0.0f};
  float ch1, sh1, ch2, sh2, ce, se, sp, cp, sgn;
  hyp_pair_f32(x.y, &ch1, &sh1);
  hyp_pair_f32(y.y, &ch2, &sh2);
  hyp_pair_f32(0.5f * (x.y - y.y), &ce, &se);
  sincosf(half_dphi(x.z, y.z, &sgn), &sp, &cp);
  const float q1 = x.w * x.w, q2 = y.w * y.w;
  const float P1 = x.x * ch1, P2 = y.x * ch2;
  const float E1 = sqrtf(fmaf(P1, P1, q1)), E2 = sqrtf(fmaf(P2, P2, q2));
  const float S = fmaf(se, se, sp * sp);
  float m;
  if (has_ms) {
    m = ms;
  } else {
    const float den = fmaf(E1, E2, P1 * P2);
    const float num = fmaf(q1, P2 * P2, fmaf(q2, P1 * P1, q1 * q2));
    const float tm = den > 0.0f ? 2.0f * num / den : 0.0f;
    m = sqrtf(q1 + q2 + tm + 4.0f * x.x * y.x * S);
  }
  if (!(m > 0.0f)) return;
  const float scale = g / (2.0f * m);
  const float sdeta = 2.0f * se * ce, sdphi = sgn * 2.0f * sp * cp;
  // X_s = P_s E_o / E_s - P_o without cancellation (pair_math.cuh leg_grad)
  const auto leg = [&](float pts, float ms_, float Ps, float Es, float qs, float chs, float shs,
                       float pto, float Po, float Eo, float qo, float sde, float sdp) {
    float X;
    if (Es > 0.0f) {
      const float den = (Ps * Eo + Po * Es) * Es;
      X = den > 0.0f ? (Ps * Ps * qo - Po * Po * qs) / den : 0.0f;
    } else {
      X = (Eo + Po) > 0.0f ? qo / (Eo + Po) : 0.0f;
    }
    V4<float> r;
    r.x = scale * (4.0f * pto * S + 2.0f * chs * X);
    r.y = scale * (2.0f * pts * (pto * sde + shs * X));
    r.z = scale * (2.0f * pts * pto * sdp);
    r.w = Es > 0.0f ? scale * (2.0f * ms_ * (Es + Eo) / Es) : 0.0f;
    return r;
  };
  g1 = leg(x.x, x.w, P1, E1, q1, ch1, sh1, y.x, P2, E2, q2, sdeta, sdphi);
  g2 = leg(y.x, y.w, P2, E2, q2, ch2, sh2, x.x, P1, E1, q1, -sdeta, -sdphi);
}

// Where the forward's saved mass ms[i] is 0 the gradient is 0 (the convention of the adjoint),
// so that forward and adjoint agree even where a recomputed mass would round away from 0.
template <typename T, int LA, int LB, int LGA, int LGB>
__global__ void __launch_bounds__(256) mass_bwd_kernel(Lv a, Lv b, const T *__restrict__ ms,
                                                       const T *__restrict__ gm, LvOut ga, LvOut gb,
                                                       int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    V4<T> g1 = {0, 0, 0, 0}, g2 = {0, 0, 0, 0};
    static_assert(sizeof(T) == 4, "the FP64 adjoint is mass_bwd_f64_kernel");
    const float msv = ms ? ld_s(ms + i) : 1.0f;
    if (msv != 0.0f)
      pair_mass_grad_f32(ld4<T, LA>(a, i), ld4<T, LB>(b, i), ld_s(gm + i), ms != nullptr, msv, g1, g2);
    st4<T, LGA>(ga, i, g1);
    st4<T, LGB>(gb, i, g2);
  }
}

template <int LA, int LB>
void launch_mass_f64_l(const Lv &a, const Lv &b, double *m, int64_t n, cudaStream_t s) {
  const int threads = 128;
  mass_f64_kernel<LA, LB><<<balanced_grid_of<mass_f64_kernel<LA, LB>>(threads, 0, n, 0, kMassWaves),
                            threads, 0, s>>>(a, b, m, n);
}

cudaError_t launch_mass_f64(const Lv &a, const Lv &b, void *m, int64_t n, cudaStream_t s) {
  double *mo = (double *)m;
  if (a.layout == GVX_SOA && b.layout == GVX_SOA)
    launch_mass_f64_l<GVX_SOA, GVX_SOA>(a, b, mo, n, s);
  else if (a.layout == GVX_SOA)
    launch_mass_f64_l<GVX_SOA, GVX_AOS>(a, b, mo, n, s);
  else if (b.layout == GVX_SOA)
    launch_mass_f64_l<GVX_AOS, GVX_SOA>(a, b, mo, n, s);
  else
    launch_mass_f64_l<GVX_AOS, GVX_AOS>(a, b, mo, n, s);
  return cudaGetLastError();
}

// FP64 adjoint: the light-cone float-float evaluation (mass_lc_grad.cuh; the two legs on paired
// FP32 instructions, the forward's saved masses used where given) with the FP64 formulas kept for
// lanes outside its domain.
template <int LA, int LB, int LGA, int LGB>
__global__ void __launch_bounds__(128, 6) mass_bwd_f64_kernel(Lv a, Lv b, const double *__restrict__ ms,
                                                           const double *__restrict__ gm,
                                                           LvOut ga, LvOut gb, int64_t n) {
  const ffm::LcTab T{ffm::kHypTab, ffm::kSinTab};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    V4<double> x = ld4<double, LA>(a, i);
    V4<double> y = ld4<double, LB>(b, i);
    double g = ld_s(gm + i);
    double o[8];
    V4<double> g1, g2;
    const double msv = ms ? ld_s(ms + i) : 0.0;
    if (ffm::pair_mass_grad_lc(x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w, g, ms != nullptr, msv, T, o)) {
      g1 = {o[0], o[1], o[2], o[3]};
      g2 = {o[4], o[5], o[6], o[7]};
    } else if (ms && msv == 0.0) {
      g1 = {0, 0, 0, 0};
      g2 = {0, 0, 0, 0};
    } else {
      pair_mass_grad(x, y, g, g1, g2);
    }
    st4<double, LGA>(ga, i, g1);
    st4<double, LGB>(gb, i, g2);
  }
}

template <typename T>
cudaError_t launch_mass_t(const Lv &a, const Lv &b, void *m, int64_t n, cudaStream_t s) {
  const int threads = 256;
  T *mo = (T *)m;
  if (a.layout == GVX_SOA && b.layout == GVX_SOA)
    mass_kernel<T, GVX_SOA, GVX_SOA>
        <<<balanced_grid_of<mass_kernel<T, GVX_SOA, GVX_SOA>>(threads, 0, n), threads, 0, s>>>(a, b, mo, n);
  else if (a.layout == GVX_SOA)
    mass_kernel<T, GVX_SOA, GVX_AOS>
        <<<balanced_grid_of<mass_kernel<T, GVX_SOA, GVX_AOS>>(threads, 0, n), threads, 0, s>>>(a, b, mo, n);
  else if (b.layout == GVX_SOA)
    mass_kernel<T, GVX_AOS, GVX_SOA>
        <<<balanced_grid_of<mass_kernel<T, GVX_AOS, GVX_SOA>>(threads, 0, n), threads, 0, s>>>(a, b, mo, n);
  else
    mass_kernel<T, GVX_AOS, GVX_AOS>
        <<<balanced_grid_of<mass_kernel<T, GVX_AOS, GVX_AOS>>(threads, 0, n), threads, 0, s>>>(a, b, mo, n);
  return cudaGetLastError();
}

template <typename T, int LA, int LB, int LGA, int LGB>
void launch_bwd_one(int threads, const Lv &a, const Lv &b, const T *ms, const T *gm,
                    const LvOut &ga, const LvOut &gb, int64_t n, cudaStream_t s) {
  if constexpr (sizeof(T) == 8) {
    constexpr auto k = mass_bwd_f64_kernel<LA, LB, LGA, LGB>;
    constexpr int t64 = 128;  // the FP64 kernel's launch bounds
    k<<<balanced_grid_of<k>(t64, 0, n, 0, kMassWaves), t64, 0, s>>>(a, b, ms, gm, ga, gb, n);
  } else {
    constexpr auto k = mass_bwd_kernel<T, LA, LB, LGA, LGB>;
    k<<<balanced_grid_of<k>(threads, 0, n), threads, 0, s>>>(a, b, ms, gm, ga, gb, n);
  }
}

template <typename T, int LA, int LB>
void launch_bwd_out(int threads, const Lv &a, const Lv &b, const T *ms, const T *gm,
                    const LvOut &ga, const LvOut &gb, int64_t n, cudaStream_t s) {
  if (ga.layout == GVX_SOA && gb.layout == GVX_SOA)
    launch_bwd_one<T, LA, LB, GVX_SOA, GVX_SOA>(threads, a, b, ms, gm, ga, gb, n, s);
  else if (ga.layout == GVX_SOA)
    launch_bwd_one<T, LA, LB, GVX_SOA, GVX_AOS>(threads, a, b, ms, gm, ga, gb, n, s);
  else if (gb.layout == GVX_SOA)
    launch_bwd_one<T, LA, LB, GVX_AOS, GVX_SOA>(threads, a, b, ms, gm, ga, gb, n, s);
  else
    launch_bwd_one<T, LA, LB, GVX_AOS, GVX_AOS>(threads, a, b, ms, gm, ga, gb, n, s);
}

template <typename T>
cudaError_t launch_mass_bwd_t(const Lv &a, const Lv &b, const void *ms, const void *gm,
                              const LvOut &ga, const LvOut &gb, int64_t n, cudaStream_t s) {
  const int threads = 256;
  const T *g = (const T *)gm, *msv = (const T *)ms;
  if (a.layout == GVX_SOA && b.layout == GVX_SOA)
    launch_bwd_out<T, GVX_SOA, GVX_SOA>(threads, a, b, msv, g, ga, gb, n, s);
  else if (a.layout == GVX_SOA)
    launch_bwd_out<T, GVX_SOA, GVX_AOS>(threads, a, b, msv, g, ga, gb, n, s);
  else if (b.layout == GVX_SOA)
    launch_bwd_out<T, GVX_AOS, GVX_SOA>(threads, a, b, msv, g, ga, gb, n, s);
  else
    launch_bwd_out<T, GVX_AOS, GVX_AOS>(threads, a, b, msv, g, ga, gb, n, s);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mass(const Lv &a, const Lv &b, void *m, int64_t n, int dtype, cudaStream_t s) {
  return dtype == GVX_F64 ? launch_mass_f64(a, b, m, n, s) : launch_mass_t<float>(a, b, m, n, s);
}

cudaError_t launch_mass_bwd(const Lv &a, const Lv &b, const void *ms, const void *gm,
                            const LvOut &ga, const LvOut &gb, int64_t n, int dtype, cudaStream_t s) {
  return dtype == GVX_F64 ? launch_mass_bwd_t<double>(a, b, ms, gm, ga, gb, n, s)
                          : launch_mass_bwd_t<float>(a, b, ms, gm, ga, gb, n, s);
}

}  // namespace gvx
