// Fused per-event analysis step: particle selection, a histogram of the pair masses of the
// selected particles, and per event the selected pair whose mass is closest to a target (the
// RDataFrame-style use of the per-event combinatorics that GenVectorX names as its next target,
// Sec. 6; the pair mass is that of Sec. 4.1, Fig. 1).  No pair mass is written to memory.
//
// CTAs take tiles of kTE consecutive events (grid-stride) and stage them in sub-batches of whole
// events of at most kNT particles.  Per sub-batch:
//   (a) one thread per particle: load, cuts, and a block scan of the selection flags that gives
//       every selected particle its place in a compacted list;
//   (b) one thread per selected particle: the scale of its event (the largest high word of pt
//       and |m| over the event's selected particles) and its light-cone terms (pt, Y = E + P,
//       D = m^2 / Y in float-float at that scale, as the jagged kernel stages them), stored at
//       its compacted place;
//       one thread per event: its number of selected pairs, and a block scan of those;
//   (c) one thread per selected pair (in rounds of kRound): its packed index k in the order of
//       gvx_event_pair_masses, its mass with the light-cone pair step of the FP64 mass kernels
//       (mass_lc.cuh; FP64 formulas outside its domain), its histogram slot (shared-memory integer
//       atomics, so the totals do not depend on the order) and its |m - target| in shared
//       memory; then one thread per event walks its pairs of the round in order and keeps the
//       first smallest |m - target| -- exact, and the smaller k on ties.
// Events of more than kNT particles are handled alone by the whole block, every pair from global
// memory, with a block reduction of (|m - target|, k).  At the end each CTA adds its histogram
// to the caller's counts.
#include <cuda_runtime.h>

#include <limits.h>
#include <math.h>

#include "common.cuh"
#include "mass_lc.cuh"
#include "pair_index.cuh"
#include "pair_math.cuh"

namespace gvx {
namespace {

constexpr int kTE = 64;       // events per tile
constexpr int kNT = 256;      // threads per CTA, and particles per sub-batch
constexpr int kRound = 512;   // selected pairs evaluated per round
constexpr int kNoFast = INT_MIN;  // scale marker of a particle outside the float-float domain
// dynamic shared memory, first part: per compacted particle (pt, Y) and D, eta, phi, scale and
// original position; per sub-batch particle its scale word and scan value; per round of pairs
// |m - t|, m and k
constexpr size_t kDynFixed =
    (size_t)kNT * (sizeof(float4) + sizeof(float2) + 2 * sizeof(double) + 4 * sizeof(int)) +
    sizeof(int) + (size_t)kRound * (2 * sizeof(double) + sizeof(long long));

struct SArgs {
  Lv p;
  const int64_t *off;
  int64_t n_events, n_particles;
  double pt_min, eta_max, lo, hi, inv_w, target;
  int n_bins;
  unsigned long long *counts;
  int64_t *best_k;
  double *best_m;
  int32_t *status;
};

__device__ __forceinline__ bool passes(double pt, double eta, const SArgs &A) {
  return pt >= A.pt_min && fabs(eta) <= A.eta_max;
}

// Histogram slot of a mass: 0 below lo, n_bins + 1 at or above hi (and NaN), else 1 + the bin
// floor((m - lo) * inv_w) clamped to the range (both operations rounded as written).
__device__ __forceinline__ int slot_of(double m, const SArgs &A) {
  if (m < A.lo) return 0;
  if (!(m < A.hi)) return A.n_bins + 1;
  long long b = __double2ll_rz(__dmul_rn(__dsub_rn(m, A.lo), A.inv_w));
  b = b < 0 ? 0 : b;
  b = b > A.n_bins - 1 ? A.n_bins - 1 : b;
  return (int)b + 1;
}

// The pair mass of two particles given by their raw values (elementwise fast path, FP64 fallback).
__device__ __forceinline__ double pair_mass_raw(V4<double> x, V4<double> y, const ffm::LcTab &T) {
  double m;
  if (!ffm::pair_mass_lc(x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w, T, &m))
    m = sqrt(pair_terms(make_leg(x), make_leg(y)).m2);
  return m;
}

// (d, k) before (d', k'): the smaller |m - target|, then the smaller k; k < 0 is "none".
__device__ __forceinline__ bool better(double d, long long k, double d0, long long k0) {
  return k >= 0 && (k0 < 0 || d < d0 || (d == d0 && k < k0));
}

// One event of more than kNT particles, by the whole block from global memory.
template <int LP>
__device__ void big_event_select(const SArgs &A, const ffm::LcTab &T, unsigned *s_hist,
                                 int64_t pb, int64_t n, double *best_d, long long *best_k,
                                 double *best_m, double *s_rd, long long *s_rk, double *s_rm) {
  double bd = INFINITY, bm = NAN;
  long long bk = -1;
  const long long npairs = (long long)n * (n - 1) / 2;
  for (long long k = threadIdx.x; k < npairs; k += kNT) {
    int64_t i, j;
    decode_pair_wide(k, n, i, j);
    const V4<double> x = ld4c<LP>(A.p, pb + i), y = ld4c<LP>(A.p, pb + j);
    if (!(passes(x.x, x.y, A) && passes(y.x, y.y, A))) continue;
    const double m = pair_mass_raw(x, y, T);
    atomicAdd(&s_hist[slot_of(m, A)], 1u);
    const double d = fabs(m - A.target);
    if (better(d, k, bd, bk)) {
      bd = d;
      bk = k;
      bm = m;
    }
  }
  s_rd[threadIdx.x] = bd;
  s_rk[threadIdx.x] = bk;
  s_rm[threadIdx.x] = bm;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int t = 0; t < kNT; t++)
      if (better(s_rd[t], s_rk[t], bd, bk) || t == 0) {
        bd = s_rd[t];
        bk = s_rk[t];
        bm = s_rm[t];
      }
    *best_d = bd;
    *best_k = bk;
    *best_m = bm;
  }
  __syncthreads();
}

template <int LP>
__global__ void __launch_bounds__(kNT, 3) pair_select_kernel(SArgs A) {
  extern __shared__ double s_dyn[];
  float4 *s_pY = reinterpret_cast<float4 *>(s_dyn);                    // by compacted place
  float2 *s_D = reinterpret_cast<float2 *>(s_pY + kNT);
  double *s_eta = reinterpret_cast<double *>(s_D + kNT), *s_phi = s_eta + kNT;
  double *s_d = s_phi + kNT, *s_m = s_d + kRound;                       // by pair of the round
  long long *s_k = reinterpret_cast<long long *>(s_m + kRound);
  int *s_fs = reinterpret_cast<int *>(s_k + kRound), *s_orig = s_fs + kNT;  // by compacted place
  int *s_ex = s_orig + kNT, *s_cs = s_ex + kNT;  // by particle of the sub-batch (s_cs: kNT + 1)
  unsigned *s_hist = reinterpret_cast<unsigned *>(s_cs + kNT + 1);
  __shared__ int64_t s_off[kTE + 1], s_pp[kTE + 1], s_warp[kNT / 32];
  __shared__ double s_bd[kTE], s_bm[kTE];
  __shared__ long long s_bk[kTE];
  __shared__ int s_bad;
  for (int s = threadIdx.x; s < A.n_bins + 2; s += kNT) s_hist[s] = 0u;
  const ffm::LcTab T{ffm::kHypTab, ffm::kSinTab};  // read through L1

  const int64_t n_tiles = (A.n_events + kTE - 1) / kTE;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t e0 = tile * kTE;
    const int ne = (int)(A.n_events - e0 < kTE ? A.n_events - e0 : kTE);
    __syncthreads();  // the previous tile is done with the shared arrays
    if (threadIdx.x == 0) s_bad = 0;
    if (threadIdx.x <= ne) s_off[threadIdx.x] = A.off[e0 + threadIdx.x];
    if (threadIdx.x < ne) {
      s_bd[threadIdx.x] = INFINITY;
      s_bk[threadIdx.x] = -1;
      s_bm[threadIdx.x] = NAN;
    }
    __syncthreads();
    if (threadIdx.x < ne) {
      const int64_t a = s_off[threadIdx.x], b = s_off[threadIdx.x + 1];
      bool bad = a < 0 || b < a || b > A.n_particles;
      if (e0 + threadIdx.x == 0 && a != 0) bad = true;
      if (e0 + threadIdx.x == A.n_events - 1 && b != A.n_particles) bad = true;
      if (bad) s_bad = 1;
    }
    __syncthreads();
    if (s_bad) {  // nothing of the tile is read; its events report no candidate
      if (threadIdx.x == 0) raise_status(A.status, GVX_ERR_OFFSETS);
      if (threadIdx.x < ne) {
        if (A.best_k) A.best_k[e0 + threadIdx.x] = -1;
        if (A.best_m) A.best_m[e0 + threadIdx.x] = NAN;
      }
      continue;
    }
    int sb = 0;
    while (sb < ne) {
      const int64_t pb = s_off[sb];
      const bool fits =
          threadIdx.x >= sb && threadIdx.x < ne && s_off[threadIdx.x + 1] - pb <= kNT;
      const int sbe = sb + __syncthreads_count(fits);
      if (sbe == sb) {  // one event larger than a sub-batch
        big_event_select<LP>(A, T, s_hist, pb, s_off[sb + 1] - pb, &s_bd[sb], &s_bk[sb],
                             &s_bm[sb], s_d, s_k, s_m);
        sb++;
        continue;
      }
      const int np = (int)(s_off[sbe] - pb), nev = sbe - sb;
      const int k = threadIdx.x;
      // (a) cuts and compaction
      V4<double> x = {0.0, 0.0, 0.0, 0.0};
      bool pass = false;
      if (k < np) {
        x = ld4<double, LP>(A.p, pb + k);
        pass = passes(x.x, x.y, A);
        s_ex[k] = pass ? (int)ffm::umax32(ffm::dhi(x.x), ffm::dhi(x.w) & 0x7fffffffu) : 0;
      }
      int64_t nsel;
      const int c = (int)block_excl_scan<kNT>(pass ? 1 : 0, s_warp, &nsel);  // ends synchronised
      if (k < np) s_cs[k] = c;
      if (k == 0) s_cs[np] = (int)nsel;
      // (b) legs of the selected particles; selected pairs per event
      if (pass) {
        int e = sb, hi = sbe - 1;  // the particle's event: the last e with s_off[e] <= pb + k
        while (e < hi) {
          const int mid = (e + hi + 1) >> 1;
          if (s_off[mid] <= pb + k) e = mid;
          else hi = mid - 1;
        }
        uint32_t wmax = 0;  // the event's scale word over its selected particles
        for (int t = (int)(s_off[e] - pb); t < (int)(s_off[e + 1] - pb); t++)
          wmax = ffm::umax32((uint32_t)s_ex[t], wmax);
        // the domain of the elementwise fast path (mass_lc.cuh), at the event's scale
        const uint32_t ew = wmax & 0x7ff00000u;
        const uint32_t hp = ffm::dhi(x.x), hm = ffm::dhi(x.w) & 0x7fffffffu;
        const uint32_t he = ffm::dhi(x.y) & 0x7fffffffu, hf = ffm::dhi(x.z) & 0x7fffffffu;
        int sc = kNoFast;
        if (wmax - (200u << 20) < (1700u << 20) &&
            ffm::umin32(hp - 0x100000u, hm - 0x100000u) >= ew - (41u << 20) &&
            ffm::umax32(hp, hm) >= 0x100000u && he < 0x40200000u && hf < 0x400C0000u) {
          const uint32_t rb = ew - (127u << 20);
          const ffm::ff ptf = ffm::cvt1(ffm::cvt_parts(hp, ffm::dlo(x.x), rb));
          const ffm::ff mmf = ffm::cvt1(ffm::cvt_parts(hm, ffm::dlo(x.w), rb));
          const ffm::ff xe = ffm::cvt1(ffm::cvt_parts_normal(ffm::umax32(he, 0x3E100000u),
                                                             ffm::dlo(x.y), ffm::kRebaseOne));
          const ffm::LcLeg<ffm::ff> L = ffm::lc_leg(ptf, mmf, xe, T.hyp);
          s_pY[c] = make_float4(ptf.hi, ptf.lo, L.Y.hi, L.Y.lo);
          s_D[c] = make_float2(L.D.hi, L.D.lo);
          sc = (int)ew;
        }
        s_fs[c] = sc;
        s_orig[c] = k;
        s_eta[c] = x.y;
        s_phi[c] = x.z;
      }
      __syncthreads();  // s_cs complete
      int64_t npairs_ev = 0;
      if (threadIdx.x < nev) {
        const int st = (int)(s_off[sb + threadIdx.x] - pb), en = (int)(s_off[sb + threadIdx.x + 1] - pb);
        const int64_t ns = s_cs[en] - s_cs[st];
        npairs_ev = ns * (ns - 1) / 2;
      }
      int64_t total;
      const int64_t pex = block_excl_scan<kNT>(npairs_ev, s_warp, &total);  // ends synchronised
      if (threadIdx.x < nev) s_pp[threadIdx.x] = pex;
      if (threadIdx.x == 0) s_pp[nev] = total;
      __syncthreads();
      // (c) the selected pairs, in rounds
      for (int64_t r0 = 0; r0 < total; r0 += kRound) {
        const int64_t r1 = total - r0 < kRound ? total : r0 + kRound;
        for (int64_t q = r0 + threadIdx.x; q < r1; q += kNT) {
          int e = 0, hi = nev - 1;  // the pair's event within the sub-batch
          while (e < hi) {
            const int mid = (e + hi + 1) >> 1;
            if (s_pp[mid] <= q) e = mid;
            else hi = mid - 1;
          }
          const int st = (int)(s_off[sb + e] - pb);
          const int64_t n = s_off[sb + e + 1] - s_off[sb + e];
          const int64_t ns = s_cs[st + (int)n] - s_cs[st];
          int64_t a, b;
          decode_pair(q - s_pp[e], ns, a, b);
          const int ci = s_cs[st] + (int)a, cj = s_cs[st] + (int)b;
          const int64_t i = s_orig[ci] - st, j = s_orig[cj] - st;  // positions in the event
          double m;
          bool done = false;
          const int sc = s_fs[ci];
          if (sc != kNoFast && s_fs[cj] != kNoFast) {
            ffm::ff S, m2s;
            const bool oks = ffm::lc_pair_S(s_eta[ci], s_eta[cj], s_phi[ci], s_phi[cj], T, &S);
            const float4 a4 = s_pY[ci], b4 = s_pY[cj];
            const float2 da = s_D[ci], db = s_D[cj];
            if (ffm::lc_pair_m2(ffm::ff{a4.x, a4.y}, ffm::ff{b4.x, b4.y}, ffm::ff{a4.z, a4.w},
                                ffm::ff{b4.z, b4.w}, ffm::ff{da.x, da.y}, ffm::ff{db.x, db.y}, S,
                                &m2s) && oks) {
              m = ffm::lc_mass_out_int(m2s, (uint32_t)sc);
              done = true;
            }
          }
          if (!done) m = pair_mass_raw(ld4c<LP>(A.p, pb + st + i), ld4c<LP>(A.p, pb + st + j), T);
          atomicAdd(&s_hist[slot_of(m, A)], 1u);
          s_d[q - r0] = fabs(m - A.target);
          s_m[q - r0] = m;
          s_k[q - r0] = i * n - i * (i + 1) / 2 + (j - i - 1);
        }
        __syncthreads();
        if (threadIdx.x < nev) {  // each event's pairs of the round, in order
          const int e = threadIdx.x;
          const int64_t q0 = s_pp[e] > r0 ? s_pp[e] : r0, q1 = s_pp[e + 1] < r1 ? s_pp[e + 1] : r1;
          double bd = s_bd[sb + e], bm = s_bm[sb + e];
          long long bk = s_bk[sb + e];
          for (int64_t q = q0; q < q1; q++)
            if (better(s_d[q - r0], s_k[q - r0], bd, bk)) {
              bd = s_d[q - r0];
              bk = s_k[q - r0];
              bm = s_m[q - r0];
            }
          s_bd[sb + e] = bd;
          s_bk[sb + e] = bk;
          s_bm[sb + e] = bm;
        }
        __syncthreads();
      }
      sb = sbe;
    }
    __syncthreads();
    if (threadIdx.x < ne) {
      if (A.best_k) A.best_k[e0 + threadIdx.x] = s_bk[threadIdx.x];
      if (A.best_m) A.best_m[e0 + threadIdx.x] = s_bk[threadIdx.x] >= 0 ? s_bm[threadIdx.x] : NAN;
    }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < A.n_bins + 2; s += kNT)
    if (s_hist[s]) atomicAdd(A.counts + s, (unsigned long long)s_hist[s]);
}

template <int LP>
cudaError_t launch_l(const SArgs &A, cudaStream_t s) {
  constexpr auto k = pair_select_kernel<LP>;
  const size_t smem = kDynFixed + (size_t)(A.n_bins + 2) * sizeof(unsigned);
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  const int64_t n_tiles = (A.n_events + kTE - 1) / kTE;
  k<<<balanced_grid_of<k>(kNT, smem, n_tiles, 1), kNT, smem, s>>>(A);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pair_select(const Lv &p, const int64_t *off, int64_t n_events,
                               int64_t n_particles, double pt_min, double eta_max, double lo,
                               double hi, int n_bins, double target, uint64_t *counts,
                               int64_t *best_k, double *best_m, cudaStream_t s) {
  SArgs A;
  A.p = p;
  A.off = off;
  A.n_events = n_events;
  A.n_particles = n_particles;
  A.pt_min = pt_min;
  A.eta_max = eta_max;
  A.lo = lo;
  A.hi = hi;
  A.inv_w = (double)n_bins / (hi - lo);
  A.target = target;
  A.n_bins = n_bins;
  A.counts = reinterpret_cast<unsigned long long *>(counts);
  A.best_k = best_k;
  A.best_m = best_m;
  A.status = device_status_word();
  return p.layout == GVX_SOA ? launch_l<GVX_SOA>(A, s) : launch_l<GVX_AOS>(A, s);
}

}  // namespace gvx
