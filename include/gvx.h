/*
 * gvx -- Lorentz-vector kernels for one GB300 (sm_103a): C ABI.
 *
 * The operations follow GenVectorX (arXiv 2312.02756):
 *   - InvariantMasses (Sec. 4.1, Fig. 1): two arrays of Lorentz vectors in PtEtaPhiM
 *     coordinates; for each index i the vectors are added and the mass of the sum is stored.
 *   - ApplyBoost (Sec. 4.1): a Lorentz boost, held in the paper as a 4x4 matrix, applied to
 *     every vector of a PxPyPzE array.
 *   - The jagged per-event form (all pair masses and the summed 4-vector of each event) serves
 *     the RDataFrame-style analyses named as the next target in Sec. 6, and so does the fused
 *     per-event selection, pair-mass histogram and best candidate.
 *   - The other 4-D coordinate systems of Sec. 3.1 as inputs: pair masses of PxPyPzE, PxPyPzM
 *     and PtEtaPhiE legs, and the conversion of PtEtaPhiM, PtEtaPhiE and PxPyPzM vectors to
 *     PxPyPzE (the input of the boost); a general 4x4 Lorentz transformation (Sec. 4.1).
 *   - The *_bwd entry points are the adjoints (vector-Jacobian products) of the mass, the boost
 *     and the jagged form.
 *
 * Conventions shared by every entry point
 *   Memory:  every pointer is caller-owned memory that the GPU can address: device memory
 *            (cudaMalloc, torch, ...), or host memory the device maps (pinned / registered
 *            memory, and on systems with pageable-memory access any host memory) -- the kernels
 *            then stream it over the host link, which is how host buffers are processed without
 *            staging copies.  The library allocates no device memory; the few calls that need
 *            scratch take a caller-provided workspace and have a *_workspace size query.
 *   Streams: `stream` is a cudaStream_t passed as void*; NULL is the legacy default stream.
 *            Every call only enqueues work on `stream` and returns without synchronising
 *            (the autotuner, graph creation and gvx_device_status synchronise, as documented).
 *   Sizes:   element counts are int64_t; n = 0 is valid and launches nothing.
 *   Errors:  arguments are validated on the host before anything is enqueued; a failed check
 *            returns its gvx_status and enqueues nothing.  GVX_ERR_CUDA means a launch or a copy
 *            was refused by the CUDA runtime (cudaGetLastError is cleared and its code kept for
 *            gvx_last_cuda_error).  Conditions only the device can see (a jagged output that
 *            does not fit, a bounded wait that timed out) are recorded in a device status word
 *            read by gvx_device_status.
 *   Values:  the mass of a PtEtaPhiM vector enters only through m^2 (its sign is ignored); pt is
 *            a magnitude (pt >= 0; negative pt is outside the domain).  A velocity with
 *            |beta| >= 1 yields NaN in every output component of that vector.
 *
 * Layout of a Lorentz-vector array (gvx_lv):
 *   GVX_SOA: c[0..3] point to four separate arrays of n scalars (pt, eta, phi, m) or
 *            (px, py, pz, E); each must be aligned to its scalar size.
 *   GVX_AOS: c[0] points to n packed structs of four scalars in the same order (32 bytes per
 *            vector in FP64, 16 in FP32); c[0] must be aligned to the struct size.
 * Velocities (beta) use the same struct with three components: SoA c[0..2], or AoS with
 * n packed triples (24 / 12 bytes, aligned to the scalar size).
 */
#ifndef GVX_H
#define GVX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GVX_OK = 0,
  GVX_ERR_NULL = 1,       /* a required pointer is NULL */
  GVX_ERR_SIZE = 2,       /* a negative or unsupported size */
  GVX_ERR_DTYPE = 3,      /* dtype is not GVX_F64 or GVX_F32 */
  GVX_ERR_LAYOUT = 4,     /* layout is not GVX_SOA or GVX_AOS */
  GVX_ERR_ALIGN = 5,      /* a pointer is not aligned as its layout requires */
  GVX_ERR_OFFSETS = 6,    /* jagged offsets are malformed (device-detected) */
  GVX_ERR_WORKSPACE = 7,  /* workspace NULL or smaller than the size query returned */
  GVX_ERR_CUDA = 8,       /* the CUDA runtime refused a launch or copy */
  GVX_ERR_TIMEOUT = 9,    /* a bounded device-side wait gave up (device-detected) */
  GVX_ERR_CAPACITY = 10,  /* a jagged output is larger than its buffer (device-detected) */
  GVX_ERR_ARG = 11,       /* any other invalid argument */
  GVX_ERR_BOUNDS = 12     /* an index failed an explicit check of a GVX_DEBUG_BOUNDS build
                             (device-detected; the access was skipped) */
} gvx_status;

typedef enum { GVX_F64 = 0, GVX_F32 = 1 } gvx_dtype;
typedef enum { GVX_SOA = 0, GVX_AOS = 1 } gvx_layout;
/* 4-D coordinate systems of a Lorentz-vector array (the component order of an AoS struct or of
 * the four SoA arrays). */
typedef enum { GVX_PTETAPHIM = 0, GVX_PXPYPZE = 1, GVX_PXPYPZM = 2, GVX_PTETAPHIE = 3 } gvx_coords;

typedef struct {
  void *c[4];     /* see "Layout of a Lorentz-vector array" above */
  int32_t layout; /* gvx_layout */
} gvx_lv;

/* Library version, "major.minor.patch". */
const char *gvx_version(void);

/* Human-readable name of a status code (static storage; never NULL). */
const char *gvx_status_string(int32_t status);

/* The cudaError_t behind the last GVX_ERR_CUDA returned on this host thread (0 if none). */
int32_t gvx_last_cuda_error(void);

/*
 * Invariant mass of pairs (Sec. 4.1, Fig. 1: m[i] = (v1[i] + v2[i]).mass()).
 *   a, b:   n PtEtaPhiM vectors each (layouts may differ), scalars of `dtype`.
 *   m:      n outputs of `dtype`.  m[i] = sqrt(E^2 - |P|^2) of the summed vector, computed from
 *           non-negative terms only, so m[i] >= 0 and the result keeps its relative accuracy for
 *           light, collinear pairs.
 *   dtype:  GVX_F64 (relative error <= 1e-12 against the exact value) or GVX_F32 (FP32 in and
 *           out; error stated per output by the test suite).
 * Returns GVX_OK or a validation error; asynchronous on `stream`.
 */
gvx_status gvx_invariant_mass(const gvx_lv *a, const gvx_lv *b, void *m, int64_t n, int32_t dtype,
                              void *stream);

/*
 * Adjoint of gvx_invariant_mass: grad_a[i] = grad_m[i] * dm[i]/d(pt, eta, phi, m) of leg a, and
 * likewise grad_b.  grad_a and grad_b are written (not accumulated) in their own layouts.  Where
 * m[i] = 0 the gradient is 0 (m is not differentiable there).
 *   m_saved: NULL, or the n masses gvx_invariant_mass returned for the same a and b (device,
 *            `dtype`, aligned to its size).  When given, "m[i] = 0" means m_saved[i] = 0, so
 *            that the adjoint's zeros coincide with the forward's; the caller keeps it alive
 *            until the call has run.
 */
gvx_status gvx_invariant_mass_bwd(const gvx_lv *a, const gvx_lv *b, const void *m_saved,
                                  const void *grad_m, gvx_lv *grad_a, gvx_lv *grad_b, int64_t n,
                                  int32_t dtype, void *stream);

/*
 * Lorentz boost (Sec. 4.1 ApplyBoost): out[i] = L(beta_i) v[i] for PxPyPzE vectors, with
 *   gamma = 1/sqrt(1 - beta^2), E' = gamma (E + beta.p),
 *   p' = p + (gamma^2/(1 + gamma) (beta.p) + gamma E) beta
 * (the symmetric 4x4 matrix of the paper applied without being stored; "boost by +beta": a
 * vector at rest acquires velocity +beta).
 *   v, out:       n vectors (out may alias v only if it has the same layout and pointers).
 *   beta:         3-component velocity array (SoA c[0..2] or AoS triples).
 *   beta_stride:  1 = one velocity per vector; 0 = beta[0] applies to every vector.
 * In FP32, 1 - beta^2 is formed from exact products so that gamma keeps FP32 accuracy as
 * |beta| -> 1.
 */
gvx_status gvx_boost(const gvx_lv *v, const gvx_lv *beta, int64_t beta_stride, gvx_lv *out,
                     int64_t n, int32_t dtype, void *stream);

/*
 * Pair masses of legs in the other 4-D coordinate systems of Sec. 3.1 (the invariant mass of
 * Sec. 4.1): m[i] = mass(a[i] + b[i]) for coords GVX_PXPYPZE (components px, py, pz, E),
 * GVX_PXPYPZM (px, py, pz, m; E = sqrt(|p|^2 + m^2)) or GVX_PTETAPHIE (pt, eta, phi, E).  A spacelike sum gives -sqrt of
 * |E^2 - |P|^2| (GenVector's convention).  PxPyPzE: the definition evaluated exactly in
 * fixed-point integers (every component truncated to 2^-83 of the pair's largest), within 2^-44
 * relative; PxPyPzM: p1 x p2, p1.p2, |p_i|^2 and m_i^2 in fixed point at each leg's own scale and
 * the cancellation-free combination m1^2 + m2^2 + 2 (E1 E2 - p1.p2) in float-float, within 2^-43
 * relative.  Pairs whose |m^2| falls below 2^-31 of the larger leg's squared scale (a power of
 * two within 2x of its largest component), or outside the fixed-point range, take a
 * cancellation-free FP64 form (an FMA-exact cross product and E^2 - |p|^2): within 1e-12
 * relative for legs with E^2 >= |p|^2.  FP32 legs go through the same evaluations and are rounded
 * once.  PtEtaPhiE: in FP64 the PtEtaPhiM identity with q_i = E_i^2 - (pt_i cosh eta_i)^2 in
 * float-float; outside its domain (negative E, m^2 below 2^-80 of the scale, spacelike sums) and
 * in FP32, both legs converted to PxPyPzE as gvx_to_pxpypze does and the exact fixed-point mass of
 * the converted legs (the FP64 form outside that one's domain).  Since E_i^2 - |p_i|^2 is not a
 * stored number the error is stated normwise: |m|m| - m_ref|m_ref|| <= 2^-40 (M1 + M2)^2 with
 * M_i = max(|E_i|, pt_i cosh(eta_i)) (FP32: 2^-19).  Layouts and alignment as
 * gvx_invariant_mass; coords GVX_PTETAPHIM is gvx_invariant_mass itself.
 */
gvx_status gvx_invariant_mass_cart(const gvx_lv *a, const gvx_lv *b, void *m, int64_t n,
                                   int32_t coords, int32_t dtype, void *stream);

/*
 * Conversion to PxPyPzE (Sec. 3.1: every 4-D coordinate system maps to the Cartesian one), so that
 * gvx_boost and gvx_lorentz_apply take vectors given in any of them: out[i] = (px, py, pz, E) of
 * v[i] for coords GVX_PTETAPHIM (px = pt cos phi, py = pt sin phi, pz = pt sinh eta,
 * E = sqrt((pt cosh eta)^2 + m^2)), GVX_PTETAPHIE (the same momentum, E as stored) or GVX_PXPYPZM
 * (E = sqrt(|p|^2 + m^2)).  FP64: float-float with table-driven functions, each component within
 * 2^-43 max(|E|, |p|) of the exact conversion; pt < 0, |eta| >= 16, |phi| > pi, zero scales and
 * non-finite values take FP64 formulas.  FP32: CUDA's float functions.  Layouts as gvx_boost;
 * coords GVX_PXPYPZE is refused (GVX_ERR_ARG): there is nothing to convert.
 */
gvx_status gvx_to_pxpypze(const gvx_lv *v, gvx_lv *out, int64_t n, int32_t coords, int32_t dtype,
                          void *stream);

/*
 * A general 4-D Lorentz transformation (Sec. 4.1: 4x4 matrices applied to every vector of an
 * array): out[i] = L_i v[i] for PxPyPzE vectors, L row-major 4x4 in (x, y, z, t) order.
 * l_stride 0: L holds one matrix (16 scalars) for every vector; 1: L holds n matrices, 16
 * scalars each, contiguous.  No structure of L is assumed.  FP32, and FP64 with a matrix per
 * vector: four FMA chains per vector, within 4 u sum_k |L_rk v_k| per component (u the unit
 * roundoff).  FP64 with one shared matrix: float-float row sums (rows and vectors scaled by
 * powers of two), within 2^-42 sum_k |L_rk v_k| + 2^-70 max_k |L_rk| max_k |v_k| per component;
 * vectors (or a matrix) outside its range (scale exponents beyond +-400, zero vectors, Inf/NaN)
 * take the FMA chains.  L must be aligned to 16 bytes when l_stride is 1.
 */
gvx_status gvx_lorentz_apply(const void *L, int64_t l_stride, const gvx_lv *v, gvx_lv *out,
                             int64_t n, int32_t dtype, void *stream);

/* Bytes of workspace gvx_boost_bwd needs (0 unless beta_stride == 0). */
size_t gvx_boost_bwd_workspace(int64_t n, int64_t beta_stride, int32_t dtype);

/*
 * Adjoint of gvx_boost for the upstream gradient grad_out (n PxPyPzE-shaped vectors):
 *   grad_v[i]    = L(beta_i)^T grad_out[i]   (L is symmetric),
 *   grad_beta[i] = d <grad_out[i], L(beta_i) v[i]> / d beta_i.
 * beta_stride 0: grad_beta holds one velocity, the sum over i, reduced deterministically through
 * `workspace` (gvx_boost_bwd_workspace bytes; may be NULL when that is 0).
 */
gvx_status gvx_boost_bwd(const gvx_lv *v, const gvx_lv *beta, int64_t beta_stride,
                         const gvx_lv *grad_out, gvx_lv *grad_v, gvx_lv *grad_beta, int64_t n,
                         int32_t dtype, void *workspace, size_t workspace_bytes, void *stream);

/* Bytes of workspace gvx_event_pair_masses needs for n_events events. */
size_t gvx_event_pair_masses_workspace(int64_t n_events);

/*
 * Jagged events (FP64).  Event e owns PtEtaPhiM particles [offsets[e], offsets[e+1]).
 *   particles:     n_particles vectors (SoA or AoS, FP64).
 *   offsets:       n_events + 1 int64, offsets[0] = 0, non-decreasing, last = n_particles.
 *   pair_offsets:  out, n_events + 1 int64: exclusive running sum of n_e (n_e - 1)/2.
 *   pair_m:        out, the masses of all pairs i < j of every event, event after event, each
 *                  event's pairs in row-major order k(i,j) = i n - i(i+1)/2 + (j - i - 1).
 *   pair_capacity: length of pair_m; if the total is larger, nothing beyond it is written and
 *                  GVX_ERR_CAPACITY is recorded in the device status word.
 *   event_sum:     out, n_events PxPyPzE vectors (SoA or AoS): the sum of each event's particles.
 *   workspace:     gvx_event_pair_masses_workspace(n_events) bytes of device memory.
 * Events with more than 64 particles are supported (processed by a slower branch).  Malformed
 * offsets are detected on the device and recorded as GVX_ERR_OFFSETS.  One launch.
 */
gvx_status gvx_event_pair_masses(const gvx_lv *particles, const int64_t *offsets, int64_t n_events,
                                 int64_t n_particles, int64_t *pair_offsets, double *pair_m,
                                 int64_t pair_capacity, gvx_lv *event_sum, void *workspace,
                                 size_t workspace_bytes, void *stream);

/*
 * Adjoint of gvx_event_pair_masses (FP64): the gradient with respect to the particles of
 *   sum_k grad_pair_m[k] pair_m[k] + sum_e <grad_event_sum[e], event_sum[e]>,
 * i.e. for particle i of event e
 *   grad_particles[i] = sum over j != i of grad_pair_m[pair(i, j)] dm(p_i, p_j)/dp_i
 *                       + J_i^T grad_event_sum[e],
 * with J_i the Jacobian of the particle's (px, py, pz, E) with respect to (pt, eta, phi, m).
 * (The paper defines the forward quantities only, Sec. 4.1 Fig. 1 and Sec. 6; this is their
 * derivative, with the conventions of gvx_invariant_mass_bwd: zero where a pair mass is 0, the
 * one-sided pt >= 0 derivative of a massless particle.)
 *   particles:       n_particles PtEtaPhiM vectors (SoA or AoS), as given to the forward call.
 *   offsets:         the forward call's n_events + 1 event offsets.
 *   pair_offsets:    the n_events + 1 pair offsets the forward call wrote.
 *   grad_pair_m:     n_pairs upstream gradients, packed like pair_m (n_pairs = pair_offsets[n_events]).
 *   grad_event_sum:  n_events PxPyPzE upstream gradients (SoA or AoS), or NULL for zero.
 *   grad_particles:  out, n_particles PtEtaPhiM-shaped gradients (SoA or AoS).
 *   workspace:       gvx_event_pair_masses_bwd_workspace(n_events) bytes of device memory,
 *                    256-byte aligned (GVX_ERR_WORKSPACE when missing or smaller, GVX_ERR_ALIGN
 *                    when misaligned; not needed when n_events or n_particles is 0).  Its
 *                    contents are scratch; calls in flight at once need separate workspaces.
 * Deterministic (a fixed summation order per particle).  Offsets or pair offsets that do not
 * match the event sizes or n_pairs are detected on the device: GVX_ERR_OFFSETS is recorded in the
 * device status word and the gradients of the affected events are not written.  All pointers
 * are device (or GPU-addressable host) memory; nothing is allocated.  One 8-byte memset and two
 * launches: the staged float-float pass, which lists in the workspace the tiles of 14 events
 * that met a rare FP64 case (a pair or event-sum part outside the float-float domain, an event
 * of more than 128 particles or 640 pairs), then a pass over the listed tiles alone that adds
 * those contributions (with none listed it returns at once).
 */
gvx_status gvx_event_pair_masses_bwd(const gvx_lv *particles, const int64_t *offsets,
                                     const int64_t *pair_offsets, int64_t n_events,
                                     int64_t n_particles, const double *grad_pair_m,
                                     int64_t n_pairs, const gvx_lv *grad_event_sum,
                                     gvx_lv *grad_particles, void *workspace,
                                     size_t workspace_bytes, void *stream);

/* Bytes of workspace gvx_event_pair_masses_bwd needs for n_events events (0 for none). */
size_t gvx_event_pair_masses_bwd_workspace(int64_t n_events);

/*
 * Fused per-event analysis step (FP64): particle selection, a histogram of the pair masses of
 * the selected particles, and per event the selected pair closest to a target mass -- the use
 * of the per-event combinatorics in RDataFrame analyses that the paper names as its next target
 * (Sec. 6; it defines no such step, so the semantics are these).  No pair mass is stored.
 *   particles, offsets, n_events, n_particles: as gvx_event_pair_masses.
 *   pt_min, eta_max: a particle is selected when pt >= pt_min and |eta| <= eta_max.
 *   lo, hi, n_bins: n_bins equal bins over [lo, hi), 1 <= n_bins <= GVX_SELECT_MAX_BINS, lo < hi.
 *   counts: in/out, n_bins + 2 uint64 in device memory; the counts of this call are ADDED:
 *           counts[0] m < lo, counts[1 + b] bin b = floor((m - lo) * (n_bins / (hi - lo)))
 *           (double arithmetic, clamped to [0, n_bins - 1]), counts[n_bins + 1] m >= hi or NaN.
 *   target: the mass the best candidate is closest to.
 *   best_k: out, n_events int64 (or NULL): the packed pair index k(i, j) (the order of
 *           gvx_event_pair_masses) of the selected pair with the smallest |m - target|, the
 *           smaller k on ties; -1 when the event has no selected pair.
 *   best_m: out, n_events doubles (or NULL): that pair's mass, NaN when none.
 * Pair masses are computed as in gvx_event_pair_masses (within 1e-12 relative of the definition;
 * an event's scale comes from its selected particles, so the last bits may differ).  A mass
 * within that tolerance of a bin edge or of another candidate's |m - target| may therefore
 * land in the neighbouring bin or pick the other pair.  Malformed offsets
 * are detected on the device (GVX_ERR_OFFSETS; such an event reports no candidate).  One launch;
 * nothing is allocated.
 */
#define GVX_SELECT_MAX_BINS 4094
gvx_status gvx_event_pair_select(const gvx_lv *particles, const int64_t *offsets,
                                 int64_t n_events, int64_t n_particles, double pt_min,
                                 double eta_max, double lo, double hi, int32_t n_bins,
                                 double target, uint64_t *counts, int64_t *best_k, double *best_m,
                                 void *stream);

/*
 * gvx_event_pair_masses without a workspace argument, for callers that cannot allocate device
 * memory: code that runs where cudaMalloc is not allowed or not wanted -- inside a host callback
 * or a framework plugin that does not own the allocator, in a pipeline with a fixed memory budget
 * decided up front, or on a hot path where cudaMalloc's implicit device synchronisation would
 * stall other streams.  (The paper has no counterpart: its host functions allocate freely.)
 *
 * The scratch memory is a fixed array inside the library module, GVX_NOALLOC_MAX_EVENTS events
 * large (262,400 bytes); every GPU that loads the library keeps it until the process exits.
 * Arguments and results are those of gvx_event_pair_masses.  More than GVX_NOALLOC_MAX_EVENTS
 * events returns GVX_ERR_SIZE and launches nothing.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) and caches it per device; make that first call
 * before any stream capture, and make no call on a device after cudaDeviceReset of it (the
 * cached address belonged to the reset context).
 * All calls share the one array (each clears what it uses before its kernel): two calls that can
 * run at the same time on the GPU (unordered streams) race and give wrong results -- order them.
 * Nothing here calls cudaMalloc, cudaFree or an allocating library routine.
 */
#define GVX_NOALLOC_MAX_EVENTS (1 << 21)
gvx_status gvx_event_pair_masses_noalloc(const gvx_lv *particles, const int64_t *offsets,
                                         int64_t n_events, int64_t n_particles,
                                         int64_t *pair_offsets, double *pair_m,
                                         int64_t pair_capacity, gvx_lv *event_sum, void *stream);

/*
 * Tile shapes of the jagged kernel.  The kernel is compiled for gvx_event_pair_masses_num_shapes()
 * (events per tile, threads per CTA) shapes; which one a call uses is looked up per device and
 * per power-of-two bucket of n_events (a default shape until a bucket is tuned or set).
 */
int32_t gvx_event_pair_masses_num_shapes(void);
gvx_status gvx_event_pair_masses_shape(int32_t shape, int32_t *events_per_tile, int32_t *threads);
int32_t gvx_event_pair_masses_get_shape(int64_t n_events);
gvx_status gvx_event_pair_masses_set_shape(int64_t n_events, int32_t shape);

/*
 * Autotuner: runs gvx_event_pair_masses with every shape (one warm-up and `reps` timed runs
 * each, CUDA events on `stream`), records the fastest for the bucket of n_events on the current
 * device and returns it in *best_shape (mean time in *best_ms).  Synchronises `stream`; writes
 * the same outputs as gvx_event_pair_masses.
 */
gvx_status gvx_event_pair_masses_autotune(const gvx_lv *particles, const int64_t *offsets,
                                          int64_t n_events, int64_t n_particles,
                                          int64_t *pair_offsets, double *pair_m,
                                          int64_t pair_capacity, gvx_lv *event_sum,
                                          void *workspace, size_t workspace_bytes, int32_t reps,
                                          void *stream, int32_t *best_shape, float *best_ms);

/*
 * Captured form of gvx_event_pair_masses: the whole call (the workspace reset and the one
 * persistent kernel) recorded once into a CUDA graph for these exact pointers and sizes, with the
 * shape selected for n_events at creation.  gvx_graph_launch replays it on any stream (one graph
 * launch per call); the pointed-to buffers must stay valid until gvx_graph_destroy.  Creating the
 * graph runs the call once (synchronously, on a private stream).
 */
typedef struct gvx_graph_s *gvx_graph;
gvx_status gvx_event_pair_masses_graph_create(const gvx_lv *particles, const int64_t *offsets,
                                              int64_t n_events, int64_t n_particles,
                                              int64_t *pair_offsets, double *pair_m,
                                              int64_t pair_capacity, gvx_lv *event_sum,
                                              void *workspace, size_t workspace_bytes,
                                              gvx_graph *out);
gvx_status gvx_graph_launch(gvx_graph graph, void *stream);
gvx_status gvx_graph_destroy(gvx_graph graph);

/*
 * Test hook (fault injection on the host side of one launch).  While enabled on this host thread,
 * gvx_event_pair_masses starts its tile counter at 1: tile 0 is never processed, so the tiles
 * after it wait for a prefix that never comes, give up after their bounded wait (about 1 s),
 * record GVX_ERR_TIMEOUT and finish.  The outputs of such a call are not meaningful.
 */
void gvx_testing_skip_first_tile(int32_t enable);

/*
 * Synchronises `stream`, copies the device status word to *host_status (a gvx_status value:
 * GVX_OK, or the first device-detected error since the last call) and clears it.
 */
gvx_status gvx_device_status(void *stream, int32_t *host_status);

#ifdef __cplusplus
}
#endif

#endif /* GVX_H */
