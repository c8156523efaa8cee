// Adjoint of the jagged-event pair masses and event sums (the per-event combinatorics of the
// RDataFrame analyses that GenVectorX names as its next target, Sec. 6, differentiated; the pair
// mass is that of Sec. 4.1, Fig. 1).
//
// For particle i of event e, with the upstream gradients gm of the packed pair masses and gs of
// the event sums (PxPyPzE):
//   grad_i = sum over j != i of gm[pair(i, j)] dm(p_i, p_j)/dp_i  +  J_i^T gs[e],
// J_i = d(px, py, pz, E)/d(pt, eta, phi, m) of the particle.
//
// Pair part in light-cone form (mass_lc_grad.cuh): with Y = E + P, D = E - P = m^2/Y,
// F = m^2 = (D_i + D_j)(Y_i + Y_j) + 4 pt_i pt_j S and c_ij = gm_ij / (2 m_ij),
//   dm/dpt_i  = (cosh eta_i / E_i) (Y_i A1 - D_i A2) + 4 A5,
//   dm/deta_i = (pt_i sinh eta_i / E_i) (Y_i A1 - D_i A2) + pt_i A6,
//   dm/dphi_i = pt_i A7,
//   dm/dm_i   = (2 m_i / E_i) (E_i A3 + A4),
// summed over the partners j through seven accumulators (float-float sums whose absolute error
// stays within ~2^-47 of the summed magnitudes)
//   A1 = sum c D_j,  A2 = sum c Y_j,  A3 = sum c,  A4 = sum c E_j,  A5 = sum c pt_j S_ij,
//   A6 = sum c pt_j 2 sinh(eta_i - eta_j),  A7 = sum c pt_j 2 sin(phi_i - phi_j),
// so that a pair costs its angular terms and its mass once and each direction seven float-float
// multiply-accumulates (paired FP32 lanes where two share a factor).
//
// CTAs take tiles of kTE consecutive events (grid-stride over tiles) and stage them in
// sub-batches of whole events of at most kNT particles and kPC pairs: (a) the raw particles, and
// the order of the sub-batch's events by decreasing size (so that the lanes of a warp walk
// partner loops of similar length); (b) per particle, by the thread that will take it in (d),
// its event's scale and light-cone terms (at the event's scale, as the forward kernel stages
// them) and its event-sum part J^T gs (float-float, in double in the thread's own shared-memory
// slot); (c) one thread per pair: the pair's angular terms, m and c once, stored per pair as
// c, c S and c (2 sinh d_eta, 2 sin d_phi); (d) one thread per particle walks its partners in a
// fixed order, adding the seven sums from the pair slots and the partners' staged terms, and
// assembles and converts its gradient -- so the result does not depend on scheduling and no
// atomic operation touches it.  Pairs outside the float-float domain (either particle outside the
// forward's domain at the event scale, |d_phi|/2 within 2^-7 of pi, a scaled m^2 below 2^-80,
// |gm| outside [2^-60, 2^20]) are marked in (c) and take the FP64 formulas; so does an event-sum
// part whose gs lies outside the float-float range, and an event with more than kNT particles or
// kPC pairs is handled alone, straight from global memory, with the elementwise kernels' pair
// adjoint.  These rare FP64 paths run in a second launch of the same kernel (FIX = true): the
// first launch contains no function call (a call site costs the staged path ~12% in spills at
// 96 registers), skips them and appends each tile that met one to a list in the caller's
// workspace; the second launch takes only the listed tiles (none: it returns at once), repeats
// their staging and classification and adds, per particle, the FP64 contributions to the
// gradient the first launch wrote (big events it writes whole).  The pair offsets are
// those the forward call wrote; each tile checks them (and the offsets) against the event sizes
// and the pair count before it reads any pair gradient, and records GVX_ERR_OFFSETS for a tile
// that does not match (its particles' gradients are then not written).
#include <cuda_runtime.h>

#include <limits.h>

#include "common.cuh"
#include "mass_lc_grad.cuh"
#include "pair_index.cuh"
#include "pair_math.cuh"

namespace gvx {
namespace {

constexpr int kTE = 14;    // events per tile (about 112 particles at the benchmark multiplicity)
constexpr int kNT = 128;   // threads per CTA, and particles staged per sub-batch
constexpr int kPC = 640;   // pairs staged per sub-batch (the events of a sub-batch average ~450)
constexpr int kNoFast = INT_MIN;  // scale marker of a particle outside the float-float domain
constexpr uint32_t kSlowPair = 0x7fc00000u;  // the bits of c.hi marking a pair for FP64
// Workspace: the count of listed tiles (zeroed by the call before the first launch), then from
// byte kWsList the list of tiles (int64) the FIX launch takes, at most one entry per tile.
constexpr size_t kWsList = 256;
// per staged particle: pt, eta, phi, m and the FP64 accumulator (doubles); (pt, Y), (D, E),
// (cosh, sinh) (float4) and m (float2); the larger high word of pt and |m|, and its event's scale
// field or kNoFast (ints); per staged pair: (c, c S) and (c 2 sinh d_eta, c 2 sin d_phi) (float4)
constexpr size_t kDynSmem =
    (size_t)kNT * (4 * sizeof(double) + sizeof(double4) + 3 * sizeof(float4) + sizeof(float2) +
                   2 * sizeof(int)) +
    (size_t)kPC * 2 * sizeof(float4);

struct BArgs {
  Lv p;
  const int64_t *off, *pair_off;
  int64_t n_events, n_particles, n_pairs;
  const double *gpm;
  Lv gsum;
  bool has_gsum;
  LvOut grad;
  int32_t *status;
  unsigned long long *fix_count;  // workspace: tiles listed for the FIX launch
  int64_t *fix_tiles;             // workspace: their indices
};

// J^T gs in FP64 for one particle: gs = (gx, gy, gz, gE) against the rows
//   px: (cos phi, 0, -pt sin phi, 0)       py: (sin phi, 0, pt cos phi, 0)
//   pz: (sinh eta, pt cosh eta, 0, 0)      E:  (P cosh eta, P pt sinh eta, 0, m) / E,
// P = pt cosh eta; for a massless particle (E = P) the E row is (cosh eta, pt sinh eta, 0, 0).
__device__ __noinline__ V4<double> sum_part(V4<double> x, V4<double> gs) {
  const double pt = x.x, eta = x.y, phi = x.z, m = x.w;
  double s, c;
  sincos(phi, &s, &c);
  const double sh = sinh(eta), ch = cosh(eta);
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

// The same J^T gs in float-float from the particle's staged light-cone terms (scaled by 2^-s:
// pt, P, E, m; cosh and sinh of |eta|), gs converted at its own scale 2^sg; returned in double.
// False when gs has a nonzero component outside [2^-300, 2^300] (the caller then uses sum_part).
__device__ __forceinline__ bool sum_part_lc(ffm::ff pt, ffm::ff E, ffm::ff mm, ffm::ff ch,
                                            ffm::ff sh, double eta, double phi, double m,
                                            uint32_t eoff_s, V4<double> gs, const ffm::LcTab &T,
                                            V4<double> *out) {
  using namespace ffm;
  const uint32_t h0 = dhi(gs.x) & 0x7fffffffu, h1 = dhi(gs.y) & 0x7fffffffu;
  const uint32_t h2 = dhi(gs.z) & 0x7fffffffu, h3 = dhi(gs.w) & 0x7fffffffu;
  const uint32_t hmax = umax32(umax32(h0, h1), umax32(h2, h3));
  if (hmax == 0u && (dlo(gs.x) | dlo(gs.y) | dlo(gs.z) | dlo(gs.w)) == 0u) {
    *out = V4<double>{0.0, 0.0, 0.0, 0.0};
    return true;
  }
  if (hmax - (723u << 20) >= (600u << 20)) return false;  // scale field 723..1322
  const uint32_t ewg = hmax & 0x7ff00000u, rbg = ewg - (127u << 20);
  const ff gx = cvt1(cvt_parts(h0, dlo(gs.x), rbg)), gy = cvt1(cvt_parts(h1, dlo(gs.y), rbg));
  const ff gz = cvt1(cvt_parts(h2, dlo(gs.z), rbg)), gE = cvt1(cvt_parts(h3, dlo(gs.w), rbg));
  const float sx = sign_of(gs.x), sy = sign_of(gs.y), sz = sign_of(gs.z), sE = sign_of(gs.w);
  const float seta = sign_of(eta), sphi = sign_of(phi), sm = sign_of(m);
  ff sn, cs;  // sin and cos of |phi|
  sincos_lc(cvt1(cvt_parts(dhi(phi) & 0x7fffffffu, dlo(phi), kRebaseOne)), T.sin, &sn, &cs);
  const ff P = lc_mul(pt, ch);
  const ff rE = lc_div(ff{1.0f, 0.0f}, E);
  const ff e0 = lc_mul(lc_mul(P, ch), rE);           // dE/dpt
  const ff e1 = lc_mul(lc_mul(P, lc_mul(pt, sh)), rE);  // |dE/deta| (times 2^-s)
  const ff e3 = lc_mul(mm, rE);                       // |dE/dm|
  // signed products (the sign of a product of signed values, on the hi and lo parts)
  const auto sp = [](const ff &a, const ff &b, float sgn) { return lc_scale(lc_mul(a, b), sgn); };
  const ff dpt = add_same(add_same(sp(gx, cs, sx), sp(gy, sn, sy * sphi)),
                     add_same(sp(gz, sh, sz * seta), sp(gE, e0, sE)));
  const ff deta = add_same(sp(gz, P, sz), sp(gE, e1, sE * seta));
  const ff dphi = lc_mul(pt, add_same(sp(gy, cs, sy), sp(gx, sn, -sx * sphi)));
  const ff dm = sp(gE, e3, sE * sm);
  const uint32_t eoff_g = ewg - (127u << 20);       // 2^sg
  const uint32_t eoff_gs = eoff_g + eoff_s - (896u << 20);  // 2^(sg + s)
  *out = V4<double>{lc_to_double(dpt, eoff_g), lc_to_double(deta, eoff_gs),
                    lc_to_double(dphi, eoff_gs), lc_to_double(dm, eoff_g)};
  return true;
}

// gm-weighted gradient of particle i's leg over its partners in one event, everything read from
// global memory (the path of events too large to stage).
template <int LP>
__device__ __forceinline__ void partners_from_global(const BArgs &A, const ffm::LcTab &T,
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
    if (!ffm::pair_mass_grad_lc(x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w, g, false, 0.0, T, o)) {
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

// An event with more than kNT particles (rare): its particles in strides of the CTA, each
// against all its partners from global memory.  Out of line, so that its registers do not count
// against the staged path's.
template <int LP, int LS, int LG>
__device__ __noinline__ void big_event(const BArgs &A, const ffm::LcTab &T, int64_t e, int64_t pbeg,
                                       int64_t n, int64_t pair0) {
  for (int64_t t = threadIdx.x; t < n; t += kNT) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const V4<double> x = ld4c<LP>(A.p, pbeg + t);
    if (A.has_gsum) {
      const V4<double> sp = sum_part(x, ld4c<LS>(A.gsum, e));
      acc[0] = sp.x;
      acc[1] = sp.y;
      acc[2] = sp.z;
      acc[3] = sp.w;
    }
    partners_from_global<LP>(A, T, pbeg + t, pbeg, n, pair0, acc);
    st4<double, LG>(A.grad, pbeg + t, V4<double>{acc[0], acc[1], acc[2], acc[3]});
  }
}

// One pair outside the float-float domain: its FP64 gradient of the first leg added to *slot.
__device__ __noinline__ void slow_pair_add(V4<double> x, V4<double> y, double g, double4 *slot) {
  V4<double> g1, g2;
  pair_mass_grad(x, y, g, g1, g2);
  double4 a = *slot;
  a.x += g1.x;
  a.y += g1.y;
  a.z += g1.z;
  a.w += g1.w;
  *slot = a;
}

__device__ __forceinline__ float4 pack4(const ffm::ff &a, const ffm::ff &b) {
  return make_float4(a.hi, a.lo, b.hi, b.lo);
}

template <int LP, int LS, int LG, bool FIX>
__global__ void __launch_bounds__(kNT, 5) event_pairs_bwd_kernel(BArgs A) {
  bool fix = false;  // FIX == false: this thread met an FP64 path in the current tile
  using ffm::ff;
  using ffm::ff2;
  extern __shared__ double s_dyn[];
  double *s_pt = s_dyn, *s_eta = s_pt + kNT, *s_phi = s_eta + kNT, *s_m = s_phi + kNT;
  double4 *s_acc = reinterpret_cast<double4 *>(s_m + kNT);  // FP64 part of each gradient
  float4 *s_pY = reinterpret_cast<float4 *>(s_acc + kNT);   // (pt, Y)
  float4 *s_DE = s_pY + kNT;                                // (D, E)
  float4 *s_cs = s_DE + kNT;                                // (cosh, sinh) of |eta|
  float2 *s_mm = reinterpret_cast<float2 *>(s_cs + kNT);    // |m|
  int *s_sc = reinterpret_cast<int *>(s_mm + kNT), *s_fs = s_sc + kNT;
  float4 *s_w0 = reinterpret_cast<float4 *>(s_fs + kNT);  // per pair: (c, c S)
  float4 *s_w1 = s_w0 + kPC;                              // (c 2 sinh d_eta, c 2 sin d_phi)
  __shared__ int64_t s_off[kTE + 1], s_poff[kTE + 1];
  __shared__ int s_order[kTE], s_start[kTE];
  __shared__ int s_bad;
  const ffm::LcTab T{ffm::kHypTab, ffm::kSinTab};
  const int64_t n_tiles = (A.n_events + kTE - 1) / kTE;
  // the first launch: every tile; the FIX launch: the listed ones (written by the first launch)
  const int64_t n_iter = FIX ? (int64_t)*(volatile unsigned long long *)A.fix_count : n_tiles;
  const int k = threadIdx.x;
  for (int64_t it = blockIdx.x; it < n_iter; it += gridDim.x) {
    int64_t tile = it;
    if constexpr (FIX) {
      tile = A.fix_tiles[it];
      if (!GVX_IN_BOUNDS(tile, n_tiles, A.status)) continue;
    }
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
      const bool fits = threadIdx.x >= sb && threadIdx.x < ne &&
                        s_off[threadIdx.x + 1] - pbeg <= kNT &&
                        s_poff[threadIdx.x + 1] - s_poff[sb] <= kPC;
      const int sbe = sb + __syncthreads_count(fits);
      if (sbe == sb) {  // one event larger than a sub-batch (particles or pairs)
        if constexpr (FIX) big_event<LP, LS, LG>(A, T, e0 + sb, pbeg, s_off[sb + 1] - pbeg, s_poff[sb]);
        else fix = true;
        sb++;
        __syncthreads();
        continue;
      }
      const int np = (int)(s_off[sbe] - pbeg);
      const int ns = sbe - sb;
      // (a) raw particles, the larger high word of pt and |m|; the events' order
      if (k < np && GVX_IN_BOUNDS(pbeg + k, A.n_particles, A.status)) {
        const V4<double> x = ld4c<LP>(A.p, pbeg + k);
        s_pt[k] = x.x;
        s_eta[k] = x.y;
        s_phi[k] = x.z;
        s_m[k] = x.w;
        s_sc[k] = (int)ffm::umax32(ffm::dhi(x.x), ffm::dhi(x.w) & 0x7fffffffu);
      }
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
      // the particle this thread takes in (b) and (c): thread k holds position k of the sorted
      // events
      int e = 0, b0 = 0, li = 0, p = 0;
      if (k < np) {
        int r = 0, hi = ns - 1;
        while (r < hi) {
          const int mid = (r + hi + 1) >> 1;
          if (s_start[mid] <= k) r = mid;
          else hi = mid - 1;
        }
        e = s_order[r];
        b0 = (int)(s_off[e] - pbeg);
        li = k - s_start[r];
        p = b0 + li;
      }
      const int n = k < np ? (int)(s_off[e + 1] - s_off[e]) : 0;
      // (b) the particle's event scale, domain and light-cone terms
      int sc = kNoFast;
      if (k < np) {
        uint32_t wmax = 0;
        for (int t = b0; t < b0 + n; t++) wmax = ffm::umax32((uint32_t)s_sc[t], wmax);
        const double pt = s_pt[p], eta = s_eta[p], phi = s_phi[p], m = s_m[p];
        const uint32_t ew = wmax & 0x7ff00000u;
        const uint32_t hp = ffm::dhi(pt), hm = ffm::dhi(m) & 0x7fffffffu;
        const uint32_t he = ffm::dhi(eta) & 0x7fffffffu, hf = ffm::dhi(phi) & 0x7fffffffu;
        if (wmax - (200u << 20) < (1700u << 20) &&
            ffm::umin32(hp - 0x100000u, hm - 0x100000u) >= ew - (41u << 20) &&
            ffm::umax32(hp, hm) >= 0x100000u && he < 0x40200000u && hf < 0x400C0000u) {
          const uint32_t rb = ew - (127u << 20);
          const ff pt_i = ffm::cvt1(ffm::cvt_parts(hp, ffm::dlo(pt), rb));
          const ff mmf = ffm::cvt1(ffm::cvt_parts(hm, ffm::dlo(m), rb));
          const ff xe = ffm::cvt1(ffm::cvt_parts_normal(ffm::umax32(he, 0x3E100000u),
                                                        ffm::dlo(eta), ffm::kRebaseOne));
          ff sh, ch;
          const ffm::LcLeg<ff> L = ffm::lc_leg(pt_i, mmf, xe, T.hyp, &sh, &ch);
          s_pY[p] = pack4(pt_i, L.Y);
          s_DE[p] = pack4(L.D, L.E);
          s_cs[p] = pack4(ch, sh);
          s_mm[p] = make_float2(mmf.hi, mmf.lo);
          sc = (int)ew;
        }
        s_fs[p] = sc;
        // the event-sum part starts the particle's FP64 slot
        V4<double> sp = {0.0, 0.0, 0.0, 0.0};
        if (A.has_gsum) {
          const V4<double> gsv = ld4c<LS>(A.gsum, e0 + e);
          const V4<double> xp = {pt, eta, phi, m};
          bool done = false;
          if (sc != kNoFast) {
            const float4 pY = s_pY[p], DE = s_DE[p], cs = s_cs[p];
            const float2 mm2 = s_mm[p];
            done = sum_part_lc(ff{pY.x, pY.y}, ff{DE.z, DE.w}, ff{mm2.x, mm2.y}, ff{cs.x, cs.y},
                               ff{cs.z, cs.w}, eta, phi, m, (uint32_t)sc - (127u << 20), gsv, T, &sp);
          }
          if constexpr (FIX) {  // only what the first launch left out
            sp = done ? V4<double>{0.0, 0.0, 0.0, 0.0} : sum_part(xp, gsv);
          } else if (!done) {
            fix = true;
          }
        }
        s_acc[p] = make_double4(sp.x, sp.y, sp.z, sp.w);
      }
      __syncthreads();
      // (c) pair-parallel: each pair's angular terms, m and c = gm / (2m) once, into the pair's
      // slot (the sd terms for the orientation (i, j), i < j); a pair outside the float-float
      // domain gets the marker kSlowPair
      const int64_t q0 = s_poff[sb];
      const int npq = (int)(s_poff[sbe] - q0);
      for (int q = threadIdx.x; q < npq; q += kNT) {
        int lo = sb, hi = sbe - 1;  // the pair's event: the last with s_poff[ev] <= q0 + q
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_poff[mid] <= q0 + q) lo = mid;
          else hi = mid - 1;
        }
        int64_t i, j;
        decode_pair(q0 + q - s_poff[lo], s_off[lo + 1] - s_off[lo], i, j);
        const int ia = (int)(s_off[lo] - pbeg + i), ib = (int)(s_off[lo] - pbeg + j);
        if (!(GVX_IN_BOUNDS(ia, np, A.status) && GVX_IN_BOUNDS(ib, np, A.status) &&
              GVX_IN_BOUNDS(q, kPC, A.status) && GVX_IN_BOUNDS(q0 + q, A.n_pairs, A.status)))
          continue;
        const double g = __ldg(A.gpm + q0 + q);
        const uint32_t hg = ffm::dhi(g) & 0x7fffffffu;
        float4 w0 = make_float4(__uint_as_float(kSlowPair), 0.0f, 0.0f, 0.0f);
        float4 w1 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (s_fs[ia] != kNoFast && s_fs[ib] != kNoFast) {
          if ((hg | ffm::dlo(g)) == 0u) {
            w0 = w1;  // gm = 0: no contribution
          } else if (hg - (963u << 20) < (81u << 20)) {  // |gm| in [2^-60, 2^20]
            ff S;
            ff2 sd;
            const bool oka = ffm::lc_pair_angles(s_eta[ia], s_eta[ib], s_phi[ia], s_phi[ib], T, &S, &sd);
            const float4 pa = s_pY[ia], pb = s_pY[ib], da = s_DE[ia], db = s_DE[ib];
            ff m2s;
            const bool okm = ffm::lc_pair_m2(ff{pa.x, pa.y}, ff{pb.x, pb.y}, ff{pa.z, pa.w},
                                             ff{pb.z, pb.w}, ff{da.x, da.y}, ff{db.x, db.y}, S, &m2s);
            if (oka && okm) {
              w0 = w1;  // m = 0: the gradient is 0
              if (m2s.hi != 0.0f) {
                const ff m = ffm::lc_sqrt_refined(m2s);
                const ff gf = ffm::cvt1(ffm::cvt_parts(hg, ffm::dlo(g), ffm::kRebaseOne));
                const ff c = ffm::lc_scale(ffm::lc_div(gf, ff{ffm::fmul(m.hi, 2.0f), ffm::fmul(m.lo, 2.0f)}),
                                           ffm::sign_of(g));
                const ff cS = ffm::lc_mul(c, S);
                const ff2 csd = ffm::lc_mul(ff2{ffm::bc2(c.hi), ffm::bc2(c.lo)}, sd);
                w0 = make_float4(c.hi, c.lo, cS.hi, cS.lo);
                w1 = make_float4(csd.hi.x, csd.lo.x, csd.hi.y, csd.lo.y);
              }
            }
          }
        }
        s_w0[q] = w0;
        s_w1[q] = w1;
      }
      __syncthreads();
      // (d) per particle, its partners in order: seven float-float sums from the pair slots, the
      // FP64 formulas for marked pairs; then the pair part and the conversion
      if (k < np) {
        const int slot0 = (int)(s_poff[e] - q0);  // the event's first pair slot
        ff2 A12 = {ffm::bc2(0.0f), ffm::bc2(0.0f)};  // (A1, A2)
        ff2 A34 = A12, A56 = A12;                    // (A3, A4), (A5, A6)
        ff A7 = {0.0f, 0.0f};
        // packed index of pair (min(li, j), max(li, j)): for j < li it is j n - j(j+1)/2 + li - j - 1
        // (step n - j - 2), for j > li it is li n - li(li+1)/2 + j - li - 1 (step 1)
        int idx = li - 1;  // the index for j = 0 (when li > 0)
        for (int j = 0; j < n; j++) {
          if (j == li) {
            idx = li * n - li * (li + 1) / 2;  // the index for j = li + 1
            continue;
          }
          const int pidx = idx;
          idx += j < li ? n - j - 2 : 1;
          const int q = b0 + j;
          if (!(GVX_IN_BOUNDS(slot0 + pidx, npq, A.status) && GVX_IN_BOUNDS(q, np, A.status)))
            continue;
          const float4 w0 = s_w0[slot0 + pidx], w1 = s_w1[slot0 + pidx];
          if constexpr (FIX) {  // the marked pairs only, into this thread's own slot
            if (__float_as_uint(w0.x) == kSlowPair)
              slow_pair_add(V4<double>{s_pt[p], s_eta[p], s_phi[p], s_m[p]},
                            V4<double>{s_pt[q], s_eta[q], s_phi[q], s_m[q]},
                            __ldg(A.gpm + s_poff[e] + pidx), s_acc + p);
            continue;
          }
          if (__float_as_uint(w0.x) == kSlowPair) {  // left to the FIX launch
            fix = true;
            continue;
          }
          const float sg = j > li ? 1.0f : -1.0f;  // the slot's sd terms are for (min, max)
          const float4 pY = s_pY[q], DE = s_DE[q];
          const ff c = {w0.x, w0.y};
          const ff2 cb = {ffm::bc2(c.hi), ffm::bc2(c.lo)};
          A12 = ffm::add_same(A12, ffm::lc_mul(cb, ff2{ffm::mk2(DE.x, pY.z), ffm::mk2(DE.y, pY.w)}));
          const ff cE = ffm::lc_mul(c, ff{DE.z, DE.w});
          A34 = ffm::add_same(A34, ff2{ffm::mk2(c.hi, cE.hi), ffm::mk2(c.lo, cE.lo)});
          const ff2 ptb = {ffm::bc2(pY.x), ffm::bc2(pY.y)};
          A56 = ffm::add_same(A56, ffm::lc_mul(ptb, ff2{ffm::mk2(w0.z, sg * w1.x), ffm::mk2(w0.w, sg * w1.y)}));
          A7 = ffm::add_same(A7, ffm::lc_mul(ff{pY.x, pY.y}, ff{sg * w1.z, sg * w1.w}));
        }
        // the pair part from the accumulators, plus the FP64 slot (event-sum part, slow pairs)
        const double4 a = s_acc[p];
        double out[4] = {a.x, a.y, a.z, a.w};
        if constexpr (FIX) {
          if (a.x != 0.0 || a.y != 0.0 || a.z != 0.0 || a.w != 0.0) {
            // the first launch's value (plain coherent loads: this launch writes the array)
            const V4<double> w = ld4<double, LG>(Lv{{A.grad.c[0], A.grad.c[1], A.grad.c[2], A.grad.c[3]},
                                                    A.grad.layout}, pbeg + p);
            st4<double, LG>(A.grad, pbeg + p, V4<double>{w.x + out[0], w.y + out[1], w.z + out[2], w.w + out[3]});
          }
        } else if (sc != kNoFast) {
          const float4 DE = s_DE[p], cs = s_cs[p];
          const float2 mm2 = s_mm[p];
          const ff E_i = {DE.z, DE.w}, ch = {cs.x, cs.y}, sh = {cs.z, cs.w}, mm = {mm2.x, mm2.y};
          const uint32_t eoff_s = (uint32_t)sc - (127u << 20);  // 2^s
          const float4 pYi = s_pY[p];
          const ff pt_i = {pYi.x, pYi.y}, Y_i = {pYi.z, pYi.w}, D_i = {DE.x, DE.y};
          const ff2 yd = ffm::lc_mul(ff2{ffm::mk2(Y_i.hi, D_i.hi), ffm::mk2(Y_i.lo, D_i.lo)}, A12);
          const ff G = ffm::add_same(ffm::lane_x(yd), ffm::lc_scale(ffm::lane_y(yd), -1.0f));  // Y A1 - D A2
          const ff rE = ffm::lc_div(ff{1.0f, 0.0f}, E_i);
          const float seta = ffm::sign_of(s_eta[p]), sm = ffm::sign_of(s_m[p]);
          const ff dpt = ffm::add_same(ffm::lc_mul(ffm::lc_mul(ch, rE), G),
                                       ff{ffm::fmul(ffm::lane_x(A56).hi, 4.0f), ffm::fmul(ffm::lane_x(A56).lo, 4.0f)});
          const ff deta = ffm::add_same(ffm::lc_scale(ffm::lc_mul(ffm::lc_mul(ffm::lc_mul(pt_i, sh), rE), G), seta),
                                        ffm::lc_mul(pt_i, ffm::lane_y(A56)));
          const ff dphi = ffm::lc_mul(pt_i, A7);
          const ff dm = ffm::lc_scale(ffm::lc_mul(ffm::lc_mul(mm, rE),
                                                  ffm::add_same(ffm::lc_mul(E_i, ffm::lane_x(A34)), ffm::lane_y(A34))),
                                      2.0f * sm);
          constexpr uint32_t kUnscaled = 896u << 20;
          out[0] += ffm::lc_to_double(dpt, kUnscaled);
          out[1] += ffm::lc_to_double(deta, eoff_s);
          out[2] += ffm::lc_to_double(dphi, eoff_s);
          out[3] += ffm::lc_to_double(dm, kUnscaled);
        }
        if constexpr (!FIX) st4<double, LG>(A.grad, pbeg + p, V4<double>{out[0], out[1], out[2], out[3]});
      }
      __syncthreads();  // before the next sub-batch overwrites the staged particles
      sb = sbe;
    }
    if constexpr (!FIX) {  // list the tile for the FIX launch if any thread met an FP64 path
      if (__syncthreads_or(fix) && threadIdx.x == 0) {
        const unsigned long long q = atomicAdd(A.fix_count, 1ull);  // < n_tiles: one per tile
        if (GVX_IN_BOUNDS(q, n_tiles, A.status)) A.fix_tiles[q] = tile;
      }
      fix = false;
    }
  }
}

template <int LP, int LS, int LG, bool FIX>
cudaError_t launch_one(const BArgs &A, cudaStream_t s) {
  constexpr auto k = event_pairs_bwd_kernel<LP, LS, LG, FIX>;
  cudaError_t err =
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDynSmem);
  if (err != cudaSuccess) return err;
  const int64_t n_tiles = (A.n_events + kTE - 1) / kTE;
  const unsigned grid = balanced_grid_of<k>(kNT, kDynSmem, n_tiles, 1);  // one tile per CTA and pass
  k<<<grid, kNT, kDynSmem, s>>>(A);
  return cudaGetLastError();
}

// The list count zeroed, the staged launch, then the FIX launch (which has nothing to do unless
// the first listed tiles).
template <int LP, int LS, int LG>
cudaError_t launch_l(const BArgs &A, cudaStream_t s) {
  cudaError_t err = cudaMemsetAsync(A.fix_count, 0, sizeof(unsigned long long), s);
  if (err != cudaSuccess) return err;
  err = launch_one<LP, LS, LG, false>(A, s);
  if (err != cudaSuccess) return err;
  return launch_one<LP, LS, LG, true>(A, s);
}

}  // namespace

size_t event_pairs_bwd_workspace(int64_t n_events) {
  return kWsList + (size_t)((n_events + kTE - 1) / kTE) * sizeof(int64_t);
}

cudaError_t launch_event_pairs_bwd(const Lv &p, const int64_t *off, const int64_t *pair_off,
                                   int64_t n_events, int64_t n_particles, const double *gpm,
                                   int64_t n_pairs, const Lv *gsum, const LvOut &grad, void *ws,
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
  A.fix_count = (unsigned long long *)ws;
  A.fix_tiles = (int64_t *)((char *)ws + kWsList);
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
