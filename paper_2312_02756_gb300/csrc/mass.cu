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
// FP64 forward: the identity is evaluated in float-float on the FP32 pipe (mass_ff.cuh) -- a
// GB300 SM retires ~80x more FP32 than FP64 operations -- with the FP64 evaluation kept for the
// rare lanes outside the float-float domain (huge |eta|, extreme scale ratios).
#include <cuda_runtime.h>

#include "common.cuh"
#include "mass_ff.cuh"
#include "pair_math.cuh"

namespace gvx {
namespace {

// FP32: memory-bound, so each thread loads kUnroll pairs (strided by the grid) before it
// computes any of them, to keep more loads in flight per SM.
constexpr int kUnroll = 4;

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

template <int LA, int LB>
__global__ void __launch_bounds__(256) mass_f64_kernel(Lv a, Lv b, double *__restrict__ m, int64_t n) {
  __shared__ ffm::gvx_f4 s_exp[GVX_EXP_N];
  __shared__ ffm::gvx_f4 s_trig[GVX_TRIG_N + 1];
  const ffm::TabRef T = ffm::stage_tables(s_exp, s_trig);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    V4<double> x = ld4<double, LA>(a, i);
    V4<double> y = ld4<double, LB>(b, i);
    double out;
    if (!ffm::pair_mass_ff(x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w, T, &out))
      out = sqrt(pair_terms(make_leg(x), make_leg(y)).m2);
    st_s(m + i, out);
  }
}

// Adjoint.  With S = sinh^2(d_eta/2) + sin^2(d_phi/2) and
//   X = (P1^2 m2^2 - P2^2 m1^2) / ((P1 E2 + P2 E1) E1)      (= P1 E2/E1 - P2, without cancellation)
// the derivatives of m^2 with respect to leg 1 are
//   d/dpt1  = 4 pt2 S + 2 cosh(eta1) X
//   d/deta1 = 2 pt1 (pt2 sinh(d_eta) + sinh(eta1) X)
//   d/dphi1 = 2 pt1 pt2 sin(d_phi)
//   d/dm1   = 2 m1 (E1 + E2) / E1
// and leg 2 follows by exchanging the legs (d_eta, d_phi change sign).  dm = d(m^2) / (2 m);
// where m = 0 the gradient is 0.  A massless leg has E = pt cosh(eta), and at pt = 0 its
// one-sided (pt >= 0) derivatives are used: X -> m_o^2 / (E_o + P_o), d/dm = 0.
template <typename T>
__device__ __forceinline__ V4<T> leg_grad(const Leg<T> &s, const Leg<T> &o, T S, T sdeta, T sdphi,
                                          T scale) {
  // X = P_s E_o / E_s - P_o.  Its denominator vanishes (with E_s > 0) only when P_o = 0 and
  // either E_o = 0 (the other leg is the zero vector) or P_s = 0 (both legs at rest); X = 0 there.
  T X;
  if (s.E > (T)0) {
    T den = (s.P * o.E + o.P * s.E) * s.E;
    X = den > (T)0 ? (s.P * s.P * o.q - o.P * o.P * s.q) / den : (T)0;
  } else {
    X = (o.E + o.P) > (T)0 ? o.q / (o.E + o.P) : (T)0;
  }
  T ch = cosh_(s.eta), sh = sinh_(s.eta);
  V4<T> g;
  g.x = scale * ((T)4 * o.pt * S + (T)2 * ch * X);
  g.y = scale * ((T)2 * s.pt * (o.pt * sdeta + sh * X));
  g.z = scale * ((T)2 * s.pt * o.pt * sdphi);
  g.w = s.E > (T)0 ? scale * ((T)2 * s.m * (s.E + o.E) / s.E) : (T)0;
  return g;
}

template <typename T, int LA, int LB, int LGA, int LGB>
__global__ void __launch_bounds__(256) mass_bwd_kernel(Lv a, Lv b, const T *__restrict__ gm,
                                                       LvOut ga, LvOut gb, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    Leg<T> la = make_leg(ld4<T, LA>(a, i));
    Leg<T> lb = make_leg(ld4<T, LB>(b, i));
    T g = ld_s(gm + i);
    PairTerms<T> t = pair_terms(la, lb);
    T m = sqrt_(t.m2);
    V4<T> g1 = {0, 0, 0, 0}, g2 = {0, 0, 0, 0};
    if (m > (T)0) {
      T scale = g / ((T)2 * m);
      // sinh(d_eta) = 2 sinh(d_eta/2) cosh(d_eta/2); sin(d_phi) = 2 sin(d_phi/2) cos(d_phi/2)
      T ce = sqrt_((T)1 + t.se * t.se);
      T sgn;
      T cp = cos_(half_dphi(la.phi, lb.phi, &sgn));
      T sdeta = (T)2 * t.se * ce, sdphi = sgn * (T)2 * t.sp * cp;
      g1 = leg_grad(la, lb, t.S, sdeta, sdphi, scale);
      g2 = leg_grad(lb, la, t.S, -sdeta, -sdphi, scale);
    }
    st4<T, LGA>(ga, i, g1);
    st4<T, LGB>(gb, i, g2);
  }
}

template <int LA, int LB>
void launch_mass_f64_l(const Lv &a, const Lv &b, double *m, int64_t n, cudaStream_t s) {
  static int occ[64];
  const int threads = 256;
  int dev = 0;
  cudaGetDevice(&dev);
  unsigned grid = resident_grid(mass_f64_kernel<LA, LB>, threads, 0, n, &occ[dev & 63]);
  mass_f64_kernel<LA, LB><<<grid, threads, 0, s>>>(a, b, m, n);
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

// FP64 adjoint: float-float evaluation (mass_ff.cuh, pair_mass_grad_ff) with the FP64 formulas
// kept for lanes outside its domain.
template <int LA, int LB, int LGA, int LGB>
__global__ void __launch_bounds__(256) mass_bwd_f64_kernel(Lv a, Lv b, const double *__restrict__ gm,
                                                           LvOut ga, LvOut gb, int64_t n) {
  __shared__ ffm::gvx_f4 s_exp[GVX_EXP_N];
  __shared__ ffm::gvx_f4 s_trig[GVX_TRIG_N + 1];
  const ffm::TabRef T = ffm::stage_tables(s_exp, s_trig);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    V4<double> x = ld4<double, LA>(a, i);
    V4<double> y = ld4<double, LB>(b, i);
    double g = ld_s(gm + i);
    double o[8];
    V4<double> g1, g2;
    if (ffm::pair_mass_grad_ff(x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w, g, T, o)) {
      g1 = {o[0], o[1], o[2], o[3]};
      g2 = {o[4], o[5], o[6], o[7]};
    } else {
      Leg<double> la = make_leg(x), lb = make_leg(y);
      PairTerms<double> t = pair_terms(la, lb);
      double m = sqrt(t.m2);
      g1 = {0, 0, 0, 0};
      g2 = {0, 0, 0, 0};
      if (m > 0.0) {
        double scale = g / (2.0 * m);
        double ce = sqrt(1.0 + t.se * t.se);
        double sgn;
        double cp = cos(half_dphi(la.phi, lb.phi, &sgn));
        double sdeta = 2.0 * t.se * ce, sdphi = sgn * 2.0 * t.sp * cp;
        g1 = leg_grad(la, lb, t.S, sdeta, sdphi, scale);
        g2 = leg_grad(lb, la, t.S, -sdeta, -sdphi, scale);
      }
    }
    st4<double, LGA>(ga, i, g1);
    st4<double, LGB>(gb, i, g2);
  }
}

template <typename T>
cudaError_t launch_mass_t(const Lv &a, const Lv &b, void *m, int64_t n, cudaStream_t s) {
  const int threads = 256;
  unsigned grid = grid_for(n, threads, 8);
  T *mo = (T *)m;
  if (a.layout == GVX_SOA && b.layout == GVX_SOA)
    mass_kernel<T, GVX_SOA, GVX_SOA><<<grid, threads, 0, s>>>(a, b, mo, n);
  else if (a.layout == GVX_SOA)
    mass_kernel<T, GVX_SOA, GVX_AOS><<<grid, threads, 0, s>>>(a, b, mo, n);
  else if (b.layout == GVX_SOA)
    mass_kernel<T, GVX_AOS, GVX_SOA><<<grid, threads, 0, s>>>(a, b, mo, n);
  else
    mass_kernel<T, GVX_AOS, GVX_AOS><<<grid, threads, 0, s>>>(a, b, mo, n);
  return cudaGetLastError();
}

template <typename T, int LA, int LB, int LGA, int LGB>
void launch_bwd_one(unsigned grid, int threads, const Lv &a, const Lv &b, const T *gm,
                    const LvOut &ga, const LvOut &gb, int64_t n, cudaStream_t s) {
  if constexpr (sizeof(T) == 8) {
    static int occ[64];
    int dev = 0;
    cudaGetDevice(&dev);
    unsigned g = resident_grid(mass_bwd_f64_kernel<LA, LB, LGA, LGB>, threads, 0, n, &occ[dev & 63]);
    mass_bwd_f64_kernel<LA, LB, LGA, LGB><<<g, threads, 0, s>>>(a, b, gm, ga, gb, n);
  } else {
    mass_bwd_kernel<T, LA, LB, LGA, LGB><<<grid, threads, 0, s>>>(a, b, gm, ga, gb, n);
  }
}

template <typename T, int LA, int LB>
void launch_bwd_out(unsigned grid, int threads, const Lv &a, const Lv &b, const T *gm,
                    const LvOut &ga, const LvOut &gb, int64_t n, cudaStream_t s) {
  if (ga.layout == GVX_SOA && gb.layout == GVX_SOA)
    launch_bwd_one<T, LA, LB, GVX_SOA, GVX_SOA>(grid, threads, a, b, gm, ga, gb, n, s);
  else if (ga.layout == GVX_SOA)
    launch_bwd_one<T, LA, LB, GVX_SOA, GVX_AOS>(grid, threads, a, b, gm, ga, gb, n, s);
  else if (gb.layout == GVX_SOA)
    launch_bwd_one<T, LA, LB, GVX_AOS, GVX_SOA>(grid, threads, a, b, gm, ga, gb, n, s);
  else
    launch_bwd_one<T, LA, LB, GVX_AOS, GVX_AOS>(grid, threads, a, b, gm, ga, gb, n, s);
}

template <typename T>
cudaError_t launch_mass_bwd_t(const Lv &a, const Lv &b, const void *gm, const LvOut &ga,
                              const LvOut &gb, int64_t n, cudaStream_t s) {
  const int threads = 256;
  unsigned grid = grid_for(n, threads, 8);
  const T *g = (const T *)gm;
  if (a.layout == GVX_SOA && b.layout == GVX_SOA)
    launch_bwd_out<T, GVX_SOA, GVX_SOA>(grid, threads, a, b, g, ga, gb, n, s);
  else if (a.layout == GVX_SOA)
    launch_bwd_out<T, GVX_SOA, GVX_AOS>(grid, threads, a, b, g, ga, gb, n, s);
  else if (b.layout == GVX_SOA)
    launch_bwd_out<T, GVX_AOS, GVX_SOA>(grid, threads, a, b, g, ga, gb, n, s);
  else
    launch_bwd_out<T, GVX_AOS, GVX_AOS>(grid, threads, a, b, g, ga, gb, n, s);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mass(const Lv &a, const Lv &b, void *m, int64_t n, int dtype, cudaStream_t s) {
  return dtype == GVX_F64 ? launch_mass_f64(a, b, m, n, s) : launch_mass_t<float>(a, b, m, n, s);
}

cudaError_t launch_mass_bwd(const Lv &a, const Lv &b, const void *gm, const LvOut &ga,
                            const LvOut &gb, int64_t n, int dtype, cudaStream_t s) {
  return dtype == GVX_F64 ? launch_mass_bwd_t<double>(a, b, gm, ga, gb, n, s)
                          : launch_mass_bwd_t<float>(a, b, gm, ga, gb, n, s);
}

}  // namespace gvx
