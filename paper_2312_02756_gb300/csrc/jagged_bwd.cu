// Adjoint of the jagged-event pair masses and event sums (the per-event combinatorics of the
// RDataFrame analyses that GenVectorX names as its next target, Sec. 6, differentiated; the pair
// mass is that of Sec. 4.1, Fig. 1).
//
// For particle i of event e, with the upstream gradients gm of the packed pair masses and gs of
// the event sums (PxPyPzE):
//   grad_i = sum over j != i of gm[pair(i, j)] dm(p_i, p_j)/dp_i  +  J_i^T gs[e],
// J_i = d(px, py, pz, E)/d(pt, eta, phi, m) of the particle.
//
// One thread per particle accumulates its own gradient over its partners in a fixed order, so the
// result does not depend on scheduling and no atomics are needed.  Each pair is therefore
// evaluated twice (once from each side).  CTAs take tiles of kTE consecutive events (grid-stride
// over tiles); the pair gradient is the float-float one of the elementwise FP64 adjoint
// (mass_ff.cuh) with the FP64 formulas for pairs outside its domain; the Jacobian rows come from
// the float-float sin/cos/sinh/cosh tables and are combined in FP64.  The pair offsets are those
// the forward call wrote; each tile checks them (and the offsets) against the event sizes and the
// pair count before it reads any pair gradient, and records GVX_ERR_OFFSETS for a tile that does
// not match (its particles' gradients are then not written).
#include <cuda_runtime.h>

#include "common.cuh"
#include "mass_ff.cuh"
#include "pair_math.cuh"

namespace gvx {
namespace {

constexpr int kTE = 32;    // events per tile
constexpr int kNT = 256;   // threads per CTA

struct BArgs {
  Lv p;
  const int64_t *off, *pair_off;
  int64_t n_events, n_particles, n_pairs;
  const double *gpm;
  Lv gsum;
  bool has_gsum;
  LvOut grad;
  int32_t *status;
};

// J^T gs for one particle: gs = (gx, gy, gz, gE) against the rows
//   px: (cos phi, 0, -pt sin phi, 0)       py: (sin phi, 0, pt cos phi, 0)
//   pz: (sinh eta, pt cosh eta, 0, 0)      E:  (pt cosh^2 eta, pt^2 cosh eta sinh eta, 0, m) / E,
// and for a massless particle (E = pt cosh eta) the E row (cosh eta, pt sinh eta, 0, 0).
__device__ __forceinline__ V4<double> sum_part(V4<double> x, V4<double> gs, const ffm::TabRef &T) {
  const double pt = x.x, eta = x.y, phi = x.z, m = x.w;
  double c, s, sh, ch;
  bool ok = ((ffm::dhi(eta) >> 20) & 0x7ffu) <= 1026u;  // |eta| < 16 for the tables
  if (ok) {
    ffm::ff sn, cs, fsh, fch;
    ffm::sincos_t(phi, T, &sn, &cs, &ok);
    ffm::sinhcosh_t(ffm::from_double(eta, &ok), T, &fsh, &fch);
    c = ffm::to_double(cs);
    s = ffm::to_double(sn);
    sh = ffm::to_double(fsh);
    ch = ffm::to_double(fch);
  }
  if (!ok) {
    sincos(phi, &s, &c);
    sh = sinh(eta);
    ch = cosh(eta);
  }
  double eE0, eE1, eE3;  // E row: d/dpt, d/deta, d/dm
  if (m == 0.0) {
    eE0 = ch;
    eE1 = pt * sh;
    eE3 = 0.0;
  } else {
    const double P = pt * ch;
    const double E = sqrt(fma(P, P, m * m));
    eE0 = P * ch / E;
    eE1 = P * pt * sh / E;
    eE3 = m / E;
  }
  V4<double> g;
  g.x = fma(gs.x, c, fma(gs.y, s, fma(gs.z, sh, gs.w * eE0)));
  g.y = fma(gs.z, pt * ch, gs.w * eE1);
  g.z = pt * fma(gs.y, c, -gs.x * s);
  g.w = gs.w * eE3;
  return g;
}

template <int LP, int LS, int LG>
__global__ void __launch_bounds__(kNT) event_pairs_bwd_kernel(BArgs A) {
  __shared__ ffm::gvx_f4 s_exp[GVX_EXP_N];
  __shared__ ffm::gvx_f4 s_trig[GVX_TRIG_N + 1];
  __shared__ int64_t s_off[kTE + 1], s_poff[kTE + 1];
  __shared__ int s_bad;
  const ffm::TabRef T = ffm::stage_tables(s_exp, s_trig);
  const int64_t n_tiles = (A.n_events + kTE - 1) / kTE;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t e0 = tile * kTE;
    const int ne = (int)(A.n_events - e0 < kTE ? A.n_events - e0 : kTE);
    __syncthreads();  // the previous tile is done with s_off / s_poff
    if (threadIdx.x == 0) s_bad = 0;
    if (threadIdx.x <= ne) {
      s_off[threadIdx.x] = A.off[e0 + threadIdx.x];
      s_poff[threadIdx.x] = A.pair_off[e0 + threadIdx.x];
    }
    __syncthreads();
    if (threadIdx.x < ne) {
      const int64_t a = s_off[threadIdx.x], b = s_off[threadIdx.x + 1], n = b - a;
      const int64_t pa = s_poff[threadIdx.x], pb = s_poff[threadIdx.x + 1];
      bool bad = a < 0 || n < 0 || b > A.n_particles || n > (1ll << 31) || pa < 0 ||
                 pb > A.n_pairs || pb - pa != n * (n - 1) / 2;
      if (e0 + threadIdx.x == 0 && (a != 0 || pa != 0)) bad = true;
      if (bad) s_bad = 1;
    }
    __syncthreads();
    if (s_bad) {
      if (threadIdx.x == 0) raise_status(A.status, GVX_ERR_OFFSETS);
      continue;
    }
    const int64_t pbeg = s_off[0], np = s_off[ne] - pbeg;
    for (int64_t k = threadIdx.x; k < np; k += kNT) {
      const int64_t i = pbeg + k;
      int lo = 0, hi = ne - 1;  // the event: the last e with s_off[e] <= i
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_off[mid] <= i) lo = mid; else hi = mid - 1;
      }
      const int e = lo;
      const int64_t base = s_off[e], n = s_off[e + 1] - base, li = i - base;
      const V4<double> x = ld4c<LP>(A.p, i);
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      for (int64_t lj = 0; lj < n; lj++) {
        if (lj == li) continue;
        const int64_t r = li < lj ? li : lj, q = li < lj ? lj : li;
        const double g = __ldg(A.gpm + s_poff[e] + r * n - r * (r + 1) / 2 + (q - r - 1));
        const V4<double> y = ld4c<LP>(A.p, base + lj);
        double o[8];
        if (!ffm::pair_mass_grad_ff(x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w, g, T, o)) {
          V4<double> g1, g2;
          pair_mass_grad(x, y, g, g1, g2);
          o[0] = g1.x;
          o[1] = g1.y;
          o[2] = g1.z;
          o[3] = g1.w;
        }
        acc[0] += o[0];
        acc[1] += o[1];
        acc[2] += o[2];
        acc[3] += o[3];
      }
      if (A.has_gsum) {
        const V4<double> gsv = ld4c<LS>(A.gsum, e0 + e);
        const V4<double> sp = sum_part(x, gsv, T);
        acc[0] += sp.x;
        acc[1] += sp.y;
        acc[2] += sp.z;
        acc[3] += sp.w;
      }
      st4<double, LG>(A.grad, i, V4<double>{acc[0], acc[1], acc[2], acc[3]});
    }
  }
}

template <int LP, int LS, int LG>
cudaError_t launch_l(const BArgs &A, cudaStream_t s) {
  constexpr auto k = event_pairs_bwd_kernel<LP, LS, LG>;
  const int64_t n_tiles = (A.n_events + kTE - 1) / kTE;
  const unsigned grid = balanced_grid_of<k>(kNT, 0, n_tiles, 1);  // one tile per CTA and pass
  k<<<grid, kNT, 0, s>>>(A);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_event_pairs_bwd(const Lv &p, const int64_t *off, const int64_t *pair_off,
                                   int64_t n_events, int64_t n_particles, const double *gpm,
                                   int64_t n_pairs, const Lv *gsum, const LvOut &grad,
                                   cudaStream_t s) {
  BArgs A;
  A.p = p;
  A.off = off;
  A.pair_off = pair_off;
  A.n_events = n_events;
  A.n_particles = n_particles;
  A.n_pairs = n_pairs;
  A.gpm = gpm;
  A.has_gsum = gsum != nullptr;
  A.gsum = gsum ? *gsum : Lv{{nullptr, nullptr, nullptr, nullptr}, GVX_SOA};
  A.grad = grad;
  A.status = device_status_word();
  const int lp = p.layout, ls = A.gsum.layout, lg = grad.layout;
  if (lp == GVX_SOA) {
    if (ls == GVX_SOA) return lg == GVX_SOA ? launch_l<GVX_SOA, GVX_SOA, GVX_SOA>(A, s)
                                            : launch_l<GVX_SOA, GVX_SOA, GVX_AOS>(A, s);
    return lg == GVX_SOA ? launch_l<GVX_SOA, GVX_AOS, GVX_SOA>(A, s)
                         : launch_l<GVX_SOA, GVX_AOS, GVX_AOS>(A, s);
  }
  if (ls == GVX_SOA) return lg == GVX_SOA ? launch_l<GVX_AOS, GVX_SOA, GVX_SOA>(A, s)
                                          : launch_l<GVX_AOS, GVX_SOA, GVX_AOS>(A, s);
  return lg == GVX_SOA ? launch_l<GVX_AOS, GVX_AOS, GVX_SOA>(A, s)
                       : launch_l<GVX_AOS, GVX_AOS, GVX_AOS>(A, s);
}

}  // namespace gvx
