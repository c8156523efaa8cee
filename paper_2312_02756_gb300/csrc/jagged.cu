// Jagged events: every in-event pair mass and every per-event summed 4-vector, in one
// persistent launch (the per-event combinatorics of the RDataFrame analyses that GenVectorX
// names as its next target, Sec. 6; the pair mass itself is that of Sec. 4.1, Fig. 1).
//
// Work unit: a tile of TE consecutive events.  CTAs take tiles in increasing order from an
// atomic counter and stay resident until the tiles run out.  Per tile:
//   1. load and validate offsets[e0 .. e0+TE];  n_e(n_e-1)/2 pairs per event, block scan;
//   2. decoupled look-back over the tile descriptors for the number of pairs before the tile
//      (bounded wait: a predecessor that never publishes makes the CTA record GVX_ERR_TIMEOUT
//      and go on);  write pair_offsets;
//   3. stage the tile's particles in shared memory in sub-batches of at most kCP particles:
//      per-particle terms once per particle (one thread each, which also finds its event's
//      scale) -- the float-float light-cone terms of the leg (pt, Y = E + P, D = m^2 / Y, scaled
//      by the event's power of two, bit for bit a lane of the elementwise FP64 kernel's legs) and
//      the Cartesian components for the sums, in float-float -- then, after one barrier, the
//      event sums (one thread per event and component, float-float at the event's scale and one
//      conversion per sum) and the pair masses (one thread per pair over the flattened pair range
//      of the sub-batch, coalesced stores) with the elementwise kernel's pair arithmetic
//      (mass_lc.cuh: lc_pair_m2; the output assembled by integer operations, so that a pair
//      costs two FP64 operations), falling back to FP64 for pairs outside its domain;
//   4. an event with more than kCP particles is handled alone, straight from global memory.
// Tile descriptors are 64-bit words: 2 flag bits (aggregate / inclusive prefix) + 62-bit value.
#include <cuda_runtime.h>

#include <type_traits>

#include <limits.h>

#include "common.cuh"
#include "mass_lc.cuh"
#include "pair_index.cuh"
#include "pair_math.cuh"

namespace gvx {
namespace {

// particles staged in shared memory per sub-batch
constexpr int kCP = 224;
// per particle: eta, phi, px, py, pz, E (doubles), pt, Y, D (float pairs), the particle's
// largest high word of pt and |m|, and its event's scale field or kNoFast (ints)
constexpr size_t kDynSmem = (size_t)kCP * (6 * sizeof(double) + 3 * sizeof(float2) + 2 * sizeof(int));
constexpr int kNoFast = INT_MIN;  // scale marker of a particle outside the float-float domain
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagInc = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // 1 s bound on a look-back wait
constexpr unsigned long long kMaxPolls = 1ull << 26;        // backstop if the timer stalls
constexpr size_t kWsHeader = 256;                           // tile counter, padded
constexpr int kMinTE = 64;

struct JArgs {
  Lv p;
  const int64_t *off;
  int64_t n_events, n_particles, n_tiles;
  int64_t *pair_off;
  double *pair_m;
  int64_t cap;
  LvOut sums;
  unsigned int *counter;
  unsigned long long *desc;
  int32_t *status;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// A float-float value kept in a double-sized shared-memory slot (its two floats' bits).
__device__ __forceinline__ void st_ff(double *slot, const ffm::ff &x) {
  *reinterpret_cast<float2 *>(slot) = make_float2(x.hi, x.lo);
}
__device__ __forceinline__ ffm::ff ld_ff(const double *slot) {
  const float2 v = *reinterpret_cast<const float2 *>(slot);
  return {v.x, v.y};
}

template <int NT, int LP, int LS>
__device__ void big_event(const JArgs &A, int64_t e, int64_t pbeg, int64_t n, int64_t out0,
                          double *s_red) {
  // event sum
  double acc[4] = {0, 0, 0, 0};
  for (int64_t k = threadIdx.x; k < n; k += NT) {
    V4<double> v = ld4<double, LP>(A.p, pbeg + k);
    double s, c;
    sincos(v.z, &s, &c);
    Leg<double> l = make_leg(v);
    acc[0] += v.x * c;
    acc[1] += v.x * s;
    acc[2] += v.x * sinh(v.y);
    acc[3] += l.E;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = 0; c < 4; c++) {
    double x = acc[c];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) s_red[c * (NT / 32) + warp] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[4] = {0, 0, 0, 0};
    for (int c = 0; c < 4; c++)
      for (int w = 0; w < NT / 32; w++) t[c] += s_red[c * (NT / 32) + w];
    st4<double, LS>(A.sums, e, V4<double>{t[0], t[1], t[2], t[3]});
  }
  __syncthreads();
  // pairs, each leg recomputed from global memory
  const int64_t npairs = n * (n - 1) / 2;
  bool over = false;
  for (int64_t k = threadIdx.x; k < npairs; k += NT) {
    int64_t i, j;
    decode_pair_wide(k, n, i, j);
    Leg<double> a = make_leg(ld4<double, LP>(A.p, pbeg + i));
    Leg<double> b = make_leg(ld4<double, LP>(A.p, pbeg + j));
    int64_t dst = out0 + k;
    if (dst < A.cap)
      st_s(A.pair_m + dst, sqrt(pair_terms(a, b).m2));
    else
      over = true;
  }
  if (__syncthreads_or(over) && threadIdx.x == 0) raise_status(A.status, GVX_ERR_CAPACITY);
}

template <int TE, int NT, int LP, int LS>
__global__ void __launch_bounds__(NT, 1024 / NT) event_pairs_kernel(JArgs A) {
  static_assert(TE <= NT && NT % 32 == 0, "one event per thread in the tile scan");
  extern __shared__ double s_dyn[];
  double *s_eta = s_dyn, *s_phi = s_eta + kCP, *s_px = s_phi + kCP, *s_py = s_px + kCP;
  double *s_pz = s_py + kCP, *s_E = s_pz + kCP;
  ffm::ff *s_pt = reinterpret_cast<ffm::ff *>(s_E + kCP), *s_Y = s_pt + kCP, *s_D = s_Y + kCP;
  int *s_sc = reinterpret_cast<int *>(s_D + kCP), *s_fs = s_sc + kCP;
  __shared__ int64_t s_off[TE + 1];
  __shared__ int64_t s_pp[TE + 1];
  __shared__ int64_t s_warp[NT / 32];
  __shared__ double s_red[4 * (NT / 32)];
  __shared__ int64_t s_base;
  __shared__ int64_t s_tile;
  const ffm::LcTab T{ffm::kHypTab, ffm::kSinTab};

  for (;;) {
    if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(A.counter, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= A.n_tiles) break;
    const int64_t e0 = tile * TE;
    const int ne = (int)((A.n_events - e0) < TE ? (A.n_events - e0) : TE);

    // 1. offsets, validation, pair counts, tile scan
    for (int k = threadIdx.x; k <= ne; k += NT) s_off[k] = A.off[e0 + k];
    __syncthreads();
    bool bad = false;
    if (threadIdx.x < ne) {
      int64_t lo = s_off[threadIdx.x], hi = s_off[threadIdx.x + 1];
      bad = lo < 0 || hi < lo || hi > A.n_particles;
    }
    if (threadIdx.x == 0) {
      if (tile == 0 && s_off[0] != 0) bad = true;
      if (tile == A.n_tiles - 1 && s_off[ne] != A.n_particles) bad = true;
    }
    const bool tile_bad = __syncthreads_or(bad);
    if (tile_bad) {  // treat every event of the tile as empty: nothing is read or written
      if (threadIdx.x == 0) raise_status(A.status, GVX_ERR_OFFSETS);
      __syncthreads();
      for (int k = threadIdx.x; k <= ne; k += NT) s_off[k] = 0;
      __syncthreads();
    }
    int64_t cnt = threadIdx.x < ne ? s_off[threadIdx.x + 1] - s_off[threadIdx.x] : 0;
    int64_t tile_total;
    int64_t excl = block_excl_scan<NT>(cnt * (cnt - 1) / 2, s_warp, &tile_total);
    if (threadIdx.x < ne) s_pp[threadIdx.x] = excl;
    if (threadIdx.x == 0) s_pp[ne] = tile_total;

    // 2. decoupled look-back
    if (threadIdx.x == 0) {
      int64_t prefix = 0;
      if (tile == 0) {
        st_relaxed(&A.desc[0], kFlagInc | (unsigned long long)tile_total);
      } else {
        st_relaxed(&A.desc[tile], kFlagAgg | (unsigned long long)tile_total);
        int64_t j = tile - 1;
        unsigned long long t0 = 0, polls = 0;
        while (j >= 0) {
          unsigned long long d = ld_relaxed(&A.desc[j]);
          unsigned long long f = d & ~kValMask;
          if (f == 0) {
            unsigned long long now = global_ns();
            if (t0 == 0) t0 = now;
            if (now - t0 > kWaitLimitNs || ++polls > kMaxPolls) {
              raise_status(A.status, GVX_ERR_TIMEOUT);
              break;
            }
            __nanosleep(64);
            continue;
          }
          prefix += (int64_t)(d & kValMask);
          if (f == kFlagInc) break;
          j--;
        }
        st_relaxed(&A.desc[tile], kFlagInc | (unsigned long long)(prefix + tile_total));
      }
      s_base = prefix;
    }
    __syncthreads();
    const int64_t base = s_base;
    if (threadIdx.x < ne) A.pair_off[e0 + threadIdx.x] = base + s_pp[threadIdx.x];
    if (tile == A.n_tiles - 1 && threadIdx.x == 0) A.pair_off[A.n_events] = base + tile_total;

    // 3./4. sub-batches of whole events that fit in shared memory
    int sb = 0;
    while (sb < ne) {
      const int64_t pb = s_off[sb];
      const bool fits = threadIdx.x >= sb && threadIdx.x < ne && s_off[threadIdx.x + 1] - pb <= kCP;
      const int sbe = sb + __syncthreads_count(fits);
      if (sbe == sb) {  // one event larger than the staging buffer
        const int64_t n = s_off[sb + 1] - pb;
        big_event<NT, LP, LS>(A, e0 + sb, pb, n, base + s_pp[sb], s_red);
        sb++;
        __syncthreads();
        continue;
      }
      const int np = (int)(s_off[sbe] - pb);
      // (a) raw particles; pt and m parked in the px/py slots, the larger high word of pt and
      // |m| in s_sc
      for (int k = threadIdx.x; k < np; k += NT) {
        if (!GVX_IN_BOUNDS(pb + k, A.n_particles, A.status)) continue;
        V4<double> v = ld4<double, LP>(A.p, pb + k);
        s_eta[k] = v.y;
        s_phi[k] = v.z;
        s_px[k] = v.x;
        s_py[k] = v.w;
        s_sc[k] = (int)ffm::umax32(ffm::dhi(v.x), ffm::dhi(v.w) & 0x7fffffffu);
      }
      __syncthreads();
      // (b) one thread per particle: its event's scale (the largest high word over the event,
      // from s_sc), whether the fast path takes it (the event's scale field goes to s_fs, so s_sc
      // stays intact for the other particles of the event), and its per-particle terms
      for (int k = threadIdx.x; k < np; k += NT) {
        int lo = sb, hi = sbe - 1;  // the particle's event: the last e with s_off[e] <= pb + k
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_off[mid] <= pb + k) lo = mid;
          else hi = mid - 1;
        }
        uint32_t wmax = 0;
        for (int t = (int)(s_off[lo] - pb); t < (int)(s_off[lo + 1] - pb); t++)
          wmax = ffm::umax32((uint32_t)s_sc[t], wmax);
        const double pt = s_px[k], eta = s_eta[k], phi = s_phi[k], m = s_py[k];
        // the domain of the elementwise fast path (mass_lc.cuh), at the event's scale
        const uint32_t ew = wmax & 0x7ff00000u;
        const uint32_t hp = ffm::dhi(pt), hm = ffm::dhi(m) & 0x7fffffffu;
        const uint32_t he = ffm::dhi(eta) & 0x7fffffffu, hf = ffm::dhi(phi) & 0x7fffffffu;
        int sc = wmax - (200u << 20) < (1700u << 20) &&
                         ffm::umin32(hp - 0x100000u, hm - 0x100000u) >= ew - (41u << 20) &&
                         ffm::umax32(hp, hm) >= 0x100000u && he < 0x40200000u && hf < 0x400C0000u
                     ? (int)ew
                     : kNoFast;
        if (sc != kNoFast) {
          const uint32_t rb = ew - (127u << 20);
          const ffm::ff ptf = ffm::cvt1(ffm::cvt_parts(hp, ffm::dlo(pt), rb));
          const ffm::ff mmf = ffm::cvt1(ffm::cvt_parts(hm, ffm::dlo(m), rb));
          const ffm::ff xe = ffm::cvt1(ffm::cvt_parts_normal(ffm::umax32(he, 0x3E100000u),
                                                             ffm::dlo(eta), ffm::kRebaseOne));
          ffm::ff sh, sn, cs;
          const ffm::LcLeg<ffm::ff> L = ffm::lc_leg(ptf, mmf, xe, T.hyp, &sh);
          ffm::sincos_lc(ffm::cvt1(ffm::cvt_parts(hf, ffm::dlo(phi), ffm::kRebaseOne)), T.sin, &sn, &cs);
          s_pt[k] = ptf;
          s_Y[k] = L.Y;
          s_D[k] = L.D;
          // the Cartesian components in float-float at the event's scale (summed per event in
          // float-float and converted once per event: no FP64 operation per particle)
          const float sphi = (ffm::dhi(phi) >> 31) ? -1.0f : 1.0f, seta = (ffm::dhi(eta) >> 31) ? -1.0f : 1.0f;
          st_ff(s_px + k, ffm::lc_mul(ptf, cs));
          st_ff(s_py + k, ffm::lc_scale(ffm::lc_mul(ptf, sn), sphi));
          st_ff(s_pz + k, ffm::lc_scale(ffm::lc_mul(ptf, sh), seta));
          st_ff(s_E + k, L.E);
        } else {  // FP64 evaluation
          double sphi, cphi;
          sincos(phi, &sphi, &cphi);
          s_px[k] = pt * cphi;
          s_py[k] = pt * sphi;
          s_pz[k] = pt * sinh(eta);
          s_E[k] = make_leg(V4<double>{pt, eta, phi, m}).E;
        }
        s_fs[k] = sc;
      }
      __syncthreads();
      // event sums: one thread per (event, component), taken by the last threads of the CTA (those
      // with one pair fewer in the pair loop's last round); float-float terms of the fast-path
      // particles summed in float-float at the event's scale, FP64 terms of the others in FP64
      for (int t = NT - 1 - (int)threadIdx.x; t < 4 * (sbe - sb); t += NT) {
        const int e = sb + (t >> 2), c = t & 3;
        const double *col = c == 0 ? s_px : c == 1 ? s_py : c == 2 ? s_pz : s_E;
        ffm::ff sf = {0.0f, 0.0f};
        double sd = 0.0;
        int sce = kNoFast;
        const int k1 = (int)(s_off[e + 1] - pb);
        for (int k = (int)(s_off[e] - pb); k < k1; k++) {
          if (s_fs[k] != kNoFast) {
            sf = ffm::add_same(sf, ld_ff(col + k));
            sce = s_fs[k];
          } else {
            sd += col[k];
          }
        }
        const double total = sce != kNoFast ? ffm::lc_to_double(sf, (uint32_t)sce - (127u << 20)) + sd : sd;
        double *dst = LS == GVX_SOA ? (double *)A.sums.c[c] + (e0 + e) : (double *)A.sums.c[0] + 4 * (e0 + e) + c;
        st_s(dst, total);
      }
      const int64_t q0 = s_pp[sb], q1 = s_pp[sbe];
      bool over = false;
      for (int64_t q = q0 + threadIdx.x; q < q1; q += NT) {
        int lo = sb, hi = sbe - 1;
        while (lo < hi) {
          int mid = (lo + hi + 1) >> 1;
          if (s_pp[mid] <= q) lo = mid;
          else hi = mid - 1;
        }
        const int64_t n = s_off[lo + 1] - s_off[lo];
        int64_t i, j;
        decode_pair(q - s_pp[lo], n, i, j);
        const int ia = (int)(s_off[lo] - pb + i), ib = (int)(s_off[lo] - pb + j);
        if (!(GVX_IN_BOUNDS(ia, np, A.status) && GVX_IN_BOUNDS(ib, np, A.status))) continue;
        double mass;
        bool done = false;
        const int sc = s_fs[ia];
        if (sc != kNoFast && s_fs[ib] != kNoFast) {
          ffm::ff S, m2s;
          const bool oks = ffm::lc_pair_S(s_eta[ia], s_eta[ib], s_phi[ia], s_phi[ib], T, &S);
          if (ffm::lc_pair_m2(s_pt[ia], s_pt[ib], s_Y[ia], s_Y[ib], s_D[ia], s_D[ib], S, &m2s) && oks) {
            mass = ffm::lc_mass_out_int(m2s, (uint32_t)sc);
            done = true;
          }
        }
        if (!done) {
          Leg<double> a = make_leg(ld4<double, LP>(A.p, pb + ia));
          Leg<double> b = make_leg(ld4<double, LP>(A.p, pb + ib));
          mass = sqrt(pair_terms(a, b).m2);
        }
        const int64_t dst = base + q;
        if (dst < A.cap)
          st_s(A.pair_m + dst, mass);
        else
          over = true;
      }
      if (__syncthreads_or(over) && threadIdx.x == 0) raise_status(A.status, GVX_ERR_CAPACITY);
      sb = sbe;
    }
    __syncthreads();
  }
}

// Tile shapes the autotuner chooses among: (events per tile, threads per CTA).
struct Shape {
  int te, nt;
};
constexpr Shape kShapes[] = {{64, 128}, {128, 128}, {128, 256}, {256, 256}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

template <int TE, int NT, int LP, int LS>
cudaError_t launch_shape(const JArgs &A0, bool skip_first_tile, cudaStream_t s) {
  auto kern = event_pairs_kernel<TE, NT, LP, LS>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kDynSmem);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, kDynSmem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  JArgs A = A0;
  A.n_tiles = (A.n_events + TE - 1) / TE;
  int64_t grid = (int64_t)num_sms() * per_sm;
  if (grid > A.n_tiles) grid = A.n_tiles;
  if (grid < 1) grid = 1;
  // tile counter + one descriptor per tile start at zero
  err = cudaMemsetAsync(A.counter, 0, kWsHeader + (size_t)A.n_tiles * 8, s);
  if (err != cudaSuccess) return err;
  if (skip_first_tile) {  // test hook: tile 0 is never taken, so its successors' waits time out
    err = cudaMemsetAsync(A.counter, 1, 1, s);
    if (err != cudaSuccess) return err;
  }
  kern<<<(unsigned)grid, NT, kDynSmem, s>>>(A);
  return cudaGetLastError();
}

template <int LP, int LS>
cudaError_t launch_any_shape(int shape, const JArgs &A, bool skip, cudaStream_t s) {
  switch (shape) {
    case 0: return launch_shape<64, 128, LP, LS>(A, skip, s);
    case 1: return launch_shape<128, 128, LP, LS>(A, skip, s);
    case 2: return launch_shape<128, 256, LP, LS>(A, skip, s);
    default: return launch_shape<256, 256, LP, LS>(A, skip, s);
  }
}

}  // namespace

int event_pairs_num_shapes() { return kNumShapes; }

void event_pairs_shape(int shape, int *te, int *nt) {
  if (shape < 0 || shape >= kNumShapes) shape = 0;
  *te = kShapes[shape].te;
  *nt = kShapes[shape].nt;
}

size_t event_pairs_workspace(int64_t n_events) {
  return kWsHeader + (size_t)((n_events + kMinTE - 1) / kMinTE) * 8;
}

cudaError_t launch_event_pairs_shape(int shape, const Lv &p, const int64_t *off, int64_t n_events,
                                     int64_t n_particles, int64_t *pair_off, double *pair_m,
                                     int64_t capacity, const LvOut &sums, void *ws,
                                     bool skip_first_tile, cudaStream_t s) {
  JArgs A;
  A.p = p;
  A.off = off;
  A.n_events = n_events;
  A.n_particles = n_particles;
  A.n_tiles = 0;
  A.pair_off = pair_off;
  A.pair_m = pair_m;
  A.cap = capacity;
  A.sums = sums;
  A.counter = (unsigned int *)ws;
  A.desc = (unsigned long long *)((char *)ws + kWsHeader);
  A.status = device_status_word();
  if (!A.status) return cudaErrorInvalidSymbol;
  const bool k = skip_first_tile;
  if (p.layout == GVX_SOA && sums.layout == GVX_SOA)
    return launch_any_shape<GVX_SOA, GVX_SOA>(shape, A, k, s);
  if (p.layout == GVX_SOA) return launch_any_shape<GVX_SOA, GVX_AOS>(shape, A, k, s);
  if (sums.layout == GVX_SOA) return launch_any_shape<GVX_AOS, GVX_SOA>(shape, A, k, s);
  return launch_any_shape<GVX_AOS, GVX_AOS>(shape, A, k, s);
}

}  // namespace gvx
