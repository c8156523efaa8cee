// Fused per-event analysis step: particle selection, a histogram of the pair masses of the
// selected particles, and per event the selected pair whose mass is closest to a target (the
// RDataFrame-style use of the per-event combinatorics that GenVectorX names as its next target,
// Sec. 6; the pair mass is that of Sec. 4.1, Fig. 1).  No pair mass is written to memory.
//
// One warp per event, warps of a CTA on different events.  Events of at most kLegCap particles:
// the lanes load the particles, test the cuts, compact the selected ones in order (ballots),
// find their scale (warp max of their leg exponents), and cache their float-float legs in the
// warp's shared-memory slice; the lanes then walk the pairs of selected particles (their packed
// index k in the order of gvx_event_pair_masses follows from the original positions) with the
// float-float pair arithmetic of the FP64 mass kernel (the FP64 formulas outside its domain).  Each pair's slot goes to a per-CTA shared-memory histogram (integer atomics, so the
// totals do not depend on the order), and each lane keeps its best (|m - target|, k); a shuffle
// reduction picks the smallest |m - target|, then the smallest k.  Larger events take the same
// loop with every pair evaluated from global memory.  At the end each CTA adds its histogram to
// the caller's counts.
#include <cuda_runtime.h>

#include <math.h>

#include "common.cuh"
#include "mass_ff.cuh"
#include "pair_index.cuh"
#include "pair_math.cuh"

namespace gvx {
namespace {

constexpr int kNT = 256;
constexpr int kWarps = kNT / 32;
constexpr int kLegCap = 64;  // particles per event cached in shared memory
constexpr unsigned kPass = 1u, kFast = 2u;
// per warp: kLegCap legs (4 ff) + eta, phi (doubles) + flags
constexpr size_t kWarpSmem = (size_t)kLegCap * (sizeof(ffm::LegFF) + 2 * sizeof(double) + sizeof(unsigned));

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
__device__ __forceinline__ double pair_mass_raw(V4<double> x, V4<double> y, const ffm::TabRef &T) {
  double m;
  if (!ffm::pair_mass_ff(x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w, T, &m))
    m = sqrt(pair_terms(make_leg(x), make_leg(y)).m2);
  return m;
}

template <int LP>
__global__ void __launch_bounds__(kNT) pair_select_kernel(SArgs A) {
  extern __shared__ double s_dyn[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // dynamic shared memory: legs, eta, phi and flags of every warp's slice, then the histogram
  ffm::LegFF *legs = reinterpret_cast<ffm::LegFF *>(s_dyn);
  double *etas = reinterpret_cast<double *>(legs + kWarps * kLegCap);
  double *phis = etas + kWarps * kLegCap;
  unsigned *flags = reinterpret_cast<unsigned *>(phis + kWarps * kLegCap);
  unsigned *s_hist = flags + kWarps * kLegCap;
  ffm::LegFF *s_leg = legs + warp * kLegCap;
  double *s_eta = etas + warp * kLegCap, *s_phi = phis + warp * kLegCap;
  unsigned *s_flag = flags + warp * kLegCap;
  __shared__ ffm::gvx_f4 s_exp[GVX_EXP_N];
  __shared__ ffm::gvx_f4 s_trig[GVX_TRIG_N + 1];
  for (int s = threadIdx.x; s < A.n_bins + 2; s += kNT) s_hist[s] = 0u;
  const ffm::TabRef T = ffm::stage_tables(s_exp, s_trig);  // ends with a barrier

  const int64_t nw = (int64_t)gridDim.x * kWarps;
  for (int64_t e = (int64_t)blockIdx.x * kWarps + warp; e < A.n_events; e += nw) {
    const int64_t b0 = A.off[e], b1 = A.off[e + 1], n = b1 - b0;
    if (b0 < 0 || n < 0 || b1 > A.n_particles || (e == 0 && b0 != 0) ||
        (e == A.n_events - 1 && b1 != A.n_particles)) {
      if (lane == 0) {
        raise_status(A.status, GVX_ERR_OFFSETS);
        if (A.best_k) A.best_k[e] = -1;
        if (A.best_m) A.best_m[e] = NAN;
      }
      continue;
    }
    double bd = INFINITY, bm = NAN;  // this lane's best |m - target|, its mass and index
    long long bk = -1;
    const int64_t npairs = n * (n - 1) / 2;
    if (n <= kLegCap) {
      // particles: cuts, then the selected ones compacted in order (ballots), their scale (warp
      // max of their leg exponents) and their legs
      V4<double> x[2];
      unsigned sel[2];
      int ex = 0;
      for (int r = 0; r < 2; r++) {
        const int t = lane + 32 * r;
        x[r] = t < n ? ld4c<LP>(A.p, b0 + t) : V4<double>{0.0, 0.0, 0.0, 0.0};
        const bool pass = t < n && passes(x[r].x, x[r].y, A);
        sel[r] = __ballot_sync(0xffffffffu, pass);
        const int et = pass ? ffm::leg_exponent(x[r].x, x[r].w) : 0;
        ex = et > ex ? et : ex;
      }
      const int emax = __reduce_max_sync(0xffffffffu, ex);
      const int sc = emax - 1023;
      const int ns = __popc(sel[0]) + __popc(sel[1]);
      for (int r = 0; r < 2; r++) {
        const int t = lane + 32 * r;
        if ((sel[r] >> lane) & 1u) {
          const int c = (r ? __popc(sel[0]) : 0) + __popc(sel[r] & ((1u << lane) - 1u));
          s_eta[c] = x[r].y;
          s_phi[c] = x[r].z;
          unsigned f = kPass | ((unsigned)t << 8);  // the original position rides in the flags
          if (ffm::scale_exponent_ok(emax) &&
              ffm::leg_in_domain(x[r].x, x[r].y, x[r].z, x[r].w, emax)) {
            bool ok = true;
            s_leg[c] = ffm::make_leg_ff(x[r].x, x[r].y, x[r].w, sc, T, &ok);
            f |= kFast;
          }
          s_flag[c] = f;
        }
      }
      __syncwarp();
      const int64_t nsp = (int64_t)ns * (ns - 1) / 2;
      for (long long q = lane; q < nsp; q += 32) {
        int64_t ci, cj;
        decode_pair(q, ns, ci, cj);
        const unsigned fi = s_flag[ci], fj = s_flag[cj];
        const int64_t i = fi >> 8, j = fj >> 8;  // original positions, i < j
        const long long k = i * n - i * (i + 1) / 2 + (j - i - 1);
        double m;
        bool done = false;
        if (fi & fj & kFast) {
          bool ok = true;
          const ffm::ff m2 = ffm::pair_m2_ff(s_leg[ci], s_leg[cj], s_eta[ci], s_eta[cj],
                                              s_phi[ci], s_phi[cj], T, &ok);
          done = ffm::finish_mass(m2, sc, ok, &m);
        }
        if (!done) m = pair_mass_raw(ld4c<LP>(A.p, b0 + i), ld4c<LP>(A.p, b0 + j), T);
        atomicAdd(&s_hist[slot_of(m, A)], 1u);
        const double d = fabs(m - A.target);
        if (d < bd) {  // k grows along the lane's loop: an equal later pair keeps the first
          bd = d;
          bk = k;
          bm = m;
        }
      }
      __syncwarp();  // the slice is reused by the warp's next event
    } else {
      for (long long k = lane; k < npairs; k += 32) {
        int64_t i, j;
        decode_pair_wide(k, n, i, j);
        const V4<double> x = ld4c<LP>(A.p, b0 + i), y = ld4c<LP>(A.p, b0 + j);
        if (!(passes(x.x, x.y, A) && passes(y.x, y.y, A))) continue;
        const double m = pair_mass_raw(x, y, T);
        atomicAdd(&s_hist[slot_of(m, A)], 1u);
        const double d = fabs(m - A.target);
        if (d < bd) {
          bd = d;
          bk = k;
          bm = m;
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {  // smallest |m - target|, then smallest k
      const double od = __shfl_down_sync(0xffffffffu, bd, o);
      const long long ok = __shfl_down_sync(0xffffffffu, bk, o);
      const double om = __shfl_down_sync(0xffffffffu, bm, o);
      if (ok >= 0 && (bk < 0 || od < bd || (od == bd && ok < bk))) {
        bd = od;
        bk = ok;
        bm = om;
      }
    }
    if (lane == 0) {
      if (A.best_k) A.best_k[e] = bk;
      if (A.best_m) A.best_m[e] = bk >= 0 ? bm : NAN;
    }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < A.n_bins + 2; s += kNT)
    if (s_hist[s]) atomicAdd(A.counts + s, (unsigned long long)s_hist[s]);
}

template <int LP>
cudaError_t launch_l(const SArgs &A, cudaStream_t s) {
  constexpr auto k = pair_select_kernel<LP>;
  const size_t smem = kWarps * kWarpSmem + (size_t)(A.n_bins + 2) * sizeof(unsigned);
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kNT, smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  int64_t need = (A.n_events + kWarps - 1) / kWarps;
  int64_t cap = (int64_t)num_sms() * per_sm * kWaves;
  int64_t grid = need < cap ? need : cap;
  if (grid < 1) grid = 1;
  k<<<(unsigned)grid, kNT, smem, s>>>(A);
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
