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
// result does not depend on scheduling and no atomics are needed; each pair is therefore
// evaluated from both sides, but each side computes only its own leg's gradient.  CTAs take tiles
// of kTE consecutive events (grid-stride over tiles) and stage them in sub-batches of whole
// events of at most kNT particles: per particle once, its raw values, the event's scale and the
// float-float leg terms (mass_ff.cuh, leg_grad_prep) go to shared memory, and its event-sum part
// (the Jacobian rows from the float-float tables) starts a float-float accumulator.  After one
// barrier every particle walks its partners with the float-float pair gradient
// (pair_grad_terms, leg_grad_terms), adding to that accumulator at the event's scale, and
// converts it to double once at the end; pairs outside the float-float domain use the FP64
// formulas and a separate FP64 accumulator.  (The FP64 pipe is the scarce one: per directed pair
// this leaves the FP64 differences of the angles only.)
// An event with more than kNT particles is handled alone, straight from global memory.  The
// pair offsets are those the forward call wrote; each tile checks them (and the offsets) against
// the event sizes and the pair count before it reads any pair gradient, and records
// GVX_ERR_OFFSETS for a tile that does not match (its particles' gradients are then not written).
#include <cuda_runtime.h>

#include "common.cuh"
#include "mass_ff.cuh"
#include "pair_math.cuh"

namespace gvx {
namespace {

constexpr int kTE = 28;    // events per tile (about 224 particles at the benchmark multiplicity)
constexpr int kNT = 256;   // threads per CTA, and particles staged per sub-batch
constexpr int kNoFast = -100000;  // scale marker of a particle outside the float-float domain
// per staged particle: pt, eta, phi, m (doubles), the ff leg terms, leg exponent and scale (ints)
constexpr size_t kDynSmem = (size_t)kNT * (4 * sizeof(double) + sizeof(ffm::LegGradFF) + 2 * sizeof(int));

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

// gm-weighted gradient of particle i's leg over its partners in one event, everything read from
// global memory (the path of events too large to stage).
// The same J^T gs for a particle on the float-float path, from its prepared leg (scaled by 2^-sc)
// and returned in the accumulator convention of leg_grad_terms (components 1 and 2 times 2^-sc).
// False when an upstream component is outside the ff range (the caller then uses sum_part).
__device__ __forceinline__ bool sum_part_ff(const ffm::LegGradFF &L, double phi, V4<double> gs,
                                            const ffm::TabRef &T, ffm::ff *out) {
  using namespace ffm;
  bool ok = true;
  ff sn, cs;
  sincos_t(phi, T, &sn, &cs, &ok);
  const ff gx = from_double(gs.x, &ok), gy = from_double(gs.y, &ok);
  const ff gz = from_double(gs.z, &ok), gE = from_double(gs.w, &ok);
  if (!ok) return false;
  ff e0, e1, e3;  // E row: d/dpt, d/deta (times 2^-sc), d/dm
  if (L.m.hi == 0.0f) {
    e0 = L.ch;
    e1 = mul(L.pt, L.sh);
    e3 = make(0.0f);
  } else {
    const ff rE = recip(L.E);
    e0 = mul(mul(L.P, L.ch), rE);
    e1 = mul(mul(L.P, mul(L.pt, L.sh)), rE);
    e3 = mul(L.m, rE);
  }
  out[0] = add(add(mul(gx, cs), mul(gy, sn)), add(mul(gz, L.sh), mul(gE, e0)));
  out[1] = add(mul(gz, L.P), mul(gE, e1));
  out[2] = mul(L.pt, add(mul(gy, cs), neg(mul(gx, sn))));
  out[3] = mul(gE, e3);
  return true;
}

template <int LP>
__device__ __forceinline__ void partners_from_global(const BArgs &A, const ffm::TabRef &T,
                                                     int64_t i, int64_t base, int64_t n,
                                                     int64_t pair0, double *acc) {
  const V4<double> x = ld4c<LP>(A.p, i);
  const int64_t li = i - base;
  for (int64_t lj = 0; lj < n; lj++) {
    if (lj == li) continue;
    const int64_t r = li < lj ? li : lj, q = li < lj ? lj : li;
    const double g = __ldg(A.gpm + pair0 + r * n - r * (r + 1) / 2 + (q - r - 1));
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
    for (int c = 0; c < 4; c++) acc[c] += o[c];
  }
}

template <int LP, int LS, int LG>
__global__ void __launch_bounds__(kNT, 3) event_pairs_bwd_kernel(BArgs A) {
  extern __shared__ double s_dyn[];
  double *s_pt = s_dyn, *s_eta = s_pt + kNT, *s_phi = s_eta + kNT, *s_m = s_phi + kNT;
  ffm::LegGradFF *s_leg = reinterpret_cast<ffm::LegGradFF *>(s_m + kNT);
  int *s_ex = reinterpret_cast<int *>(s_leg + kNT), *s_fs = s_ex + kNT;
  __shared__ ffm::gvx_f4 s_exp[GVX_EXP_N];
  __shared__ ffm::gvx_f4 s_trig[GVX_TRIG_N + 1];
  __shared__ int64_t s_off[kTE + 1], s_poff[kTE + 1];
  __shared__ int s_order[kTE], s_start[kTE];
  __shared__ int s_bad;
  const ffm::TabRef T = ffm::stage_tables(s_exp, s_trig);
  const int64_t n_tiles = (A.n_events + kTE - 1) / kTE;
  const int k = threadIdx.x;  // the particle this thread stages in every sub-batch
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t e0 = tile * kTE;
    const int ne = (int)(A.n_events - e0 < kTE ? A.n_events - e0 : kTE);
    __syncthreads();  // the previous tile is done with the shared arrays
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
    int sb = 0;
    while (sb < ne) {
      const int64_t pbeg = s_off[sb];
      const bool fits =
          threadIdx.x >= sb && threadIdx.x < ne && s_off[threadIdx.x + 1] - pbeg <= kNT;
      const int sbe = sb + __syncthreads_count(fits);
      if (sbe == sb) {  // one event larger than a sub-batch
        const int64_t n = s_off[sb + 1] - pbeg;
        for (int64_t t = threadIdx.x; t < n; t += kNT) {
          double acc[4] = {0.0, 0.0, 0.0, 0.0};
          const V4<double> x = ld4c<LP>(A.p, pbeg + t);
          if (A.has_gsum) {
            const V4<double> sp = sum_part(x, ld4c<LS>(A.gsum, e0 + sb), T);
            acc[0] = sp.x;
            acc[1] = sp.y;
            acc[2] = sp.z;
            acc[3] = sp.w;
          }
          partners_from_global<LP>(A, T, pbeg + t, pbeg, n, s_poff[sb], acc);
          st4<double, LG>(A.grad, pbeg + t, V4<double>{acc[0], acc[1], acc[2], acc[3]});
        }
        sb++;
        __syncthreads();
        continue;
      }
      const int np = (int)(s_off[sbe] - pbeg);
      // (a) raw particles and their leg exponents
      V4<double> x = {0.0, 0.0, 0.0, 0.0};
      if (k < np) {
        x = ld4c<LP>(A.p, pbeg + k);
        s_pt[k] = x.x;
        s_eta[k] = x.y;
        s_phi[k] = x.z;
        s_m[k] = x.w;
        s_ex[k] = ffm::leg_exponent(x.x, x.w);
      }
      __syncthreads();
      // (b) the particle's event and scale and its ff leg terms; and the order of phase (c):
      // events by decreasing size, so that the partner loops of a warp have similar lengths
      if (k < np) {
        int e = sb, hi = sbe - 1;  // the particle's event: the last e with s_off[e] <= pbeg + k
        while (e < hi) {
          const int mid = (e + hi + 1) >> 1;
          if (s_off[mid] <= pbeg + k) e = mid;
          else hi = mid - 1;
        }
        int emax = 0;
        for (int t = (int)(s_off[e] - pbeg); t < (int)(s_off[e + 1] - pbeg); t++)
          emax = s_ex[t] > emax ? s_ex[t] : emax;
        int sc = kNoFast;
        if (ffm::scale_exponent_ok(emax) && ffm::leg_in_domain(x.x, x.y, x.z, x.w, emax)) {
          bool ok = true;
          const ffm::LegGradFF L = ffm::leg_grad_prep(x.x, x.y, x.w, emax - 1023, T, &ok);
          if (ok) {
            sc = emax - 1023;
            s_leg[k] = L;
          }
        }
        s_fs[k] = sc;
      }
      const int ns = sbe - sb;
      if (threadIdx.x < ns) {  // rank of event sb + threadIdx.x: larger first, ties by position
        const int me = sb + threadIdx.x;
        const int64_t nme = s_off[me + 1] - s_off[me];
        int rank = 0;
        int64_t before = 0;  // particles of the events ranked ahead
        for (int o = sb; o < sbe; o++) {
          const int64_t no = s_off[o + 1] - s_off[o];
          if (no > nme || (no == nme && o < me)) {
            rank++;
            before += no;
          }
        }
        s_order[rank] = me;
        s_start[rank] = (int)before;
      }
      __syncthreads();
      // (c) one particle per thread in that order: its event-sum part, then its partners in
      // order; fast-path terms accumulate in ff at the event's scale
      if (k < np) {
        int r = 0, hi = ns - 1;  // the sorted event holding thread position k
        while (r < hi) {
          const int mid = (r + hi + 1) >> 1;
          if (s_start[mid] <= k) r = mid;
          else hi = mid - 1;
        }
        const int e = s_order[r];
        const int b0 = (int)(s_off[e] - pbeg);
        const int li32 = k - s_start[r];
        const int p = b0 + li32;  // the particle this thread now takes
        const V4<double> xp = {s_pt[p], s_eta[p], s_phi[p], s_m[p]};
        const int sc = s_fs[p];
        ffm::ff acc_f[4] = {ffm::make(0.0f), ffm::make(0.0f), ffm::make(0.0f), ffm::make(0.0f)};
        double acc[4] = {0.0, 0.0, 0.0, 0.0};  // FP64 contributions (off the fast path)
        if (A.has_gsum) {
          const V4<double> gsv = ld4c<LS>(A.gsum, e0 + e);
          if (sc == kNoFast || !sum_part_ff(s_leg[p], xp.z, gsv, T, acc_f)) {
            const V4<double> sp = sum_part(xp, gsv, T);
            acc[0] = sp.x;
            acc[1] = sp.y;
            acc[2] = sp.z;
            acc[3] = sp.w;
          }
        }
        const int64_t n = s_off[e + 1] - s_off[e], li = li32, pair0 = s_poff[e];
        for (int64_t lj = 0; lj < n; lj++) {
          if (lj == li) continue;
          const int64_t rr = li < lj ? li : lj, q = li < lj ? lj : li;
          const double g = __ldg(A.gpm + pair0 + rr * n - rr * (rr + 1) / 2 + (q - rr - 1));
          const int j = b0 + (int)lj;
          int done = 0;
          if (sc != kNoFast && s_fs[j] != kNoFast) {
            const ffm::LegGradFF &a = s_leg[p], &b = s_leg[j];
            ffm::PairGradFF pg;
            done = ffm::pair_grad_terms(a, b, xp.y, s_eta[j], xp.z, s_phi[j], g, T, &pg);
            if (done == 2) {
              ffm::ff t[4];
              ffm::leg_grad_terms(a, b, pg, pg.sdeta, pg.sdphi, t);
              for (int c = 0; c < 4; c++) acc_f[c] = ffm::add(acc_f[c], t[c]);
            }
          }
          if (!done) {
            V4<double> g1, g2;
            pair_mass_grad(xp, V4<double>{s_pt[j], s_eta[j], s_phi[j], s_m[j]}, g, g1, g2);
            acc[0] += g1.x;
            acc[1] += g1.y;
            acc[2] += g1.z;
            acc[3] += g1.w;
          }
        }
        double out[4] = {0.0, 0.0, 0.0, 0.0};
        if (sc != kNoFast) ffm::leg_grad_out(acc_f, sc, out);
        st4<double, LG>(A.grad, pbeg + p,
                        V4<double>{out[0] + acc[0], out[1] + acc[1], out[2] + acc[2], out[3] + acc[3]});
      }
      __syncthreads();  // before the next sub-batch overwrites the staged particles
      sb = sbe;
    }
  }
}

template <int LP, int LS, int LG>
cudaError_t launch_l(const BArgs &A, cudaStream_t s) {
  constexpr auto k = event_pairs_bwd_kernel<LP, LS, LG>;
  cudaError_t err =
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDynSmem);
  if (err != cudaSuccess) return err;
  const int64_t n_tiles = (A.n_events + kTE - 1) / kTE;
  const unsigned grid = balanced_grid_of<k>(kNT, kDynSmem, n_tiles, 1);  // one tile per CTA and pass
  k<<<grid, kNT, kDynSmem, s>>>(A);
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
