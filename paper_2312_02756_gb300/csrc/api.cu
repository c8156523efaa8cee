// The C ABI (include/gvx.h): host-side validation, dispatch to the kernel translation units,
// the device status word, the jagged-kernel autotuner table and captured graphs.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "gvx.h"
#include "gvx_internal.h"

namespace gvx {
int event_pairs_num_shapes();
void event_pairs_shape(int shape, int *te, int *nt);
cudaError_t launch_event_pairs_shape(int shape, const Lv &p, const int64_t *off, int64_t n_events,
                                     int64_t n_particles, int64_t *pair_off, double *pair_m,
                                     int64_t capacity, const LvOut &sums, void *ws,
                                     bool skip_first_tile, cudaStream_t s);
}  // namespace gvx

namespace {

constexpr int kMaxDevices = 64;

// One status word per device, in the module's own device memory (no allocation needed).
__device__ int32_t g_device_status;

thread_local int32_t t_last_cuda_error = 0;
thread_local bool t_skip_first_tile = false;

gvx_status cuda_fail(cudaError_t e) {
  t_last_cuda_error = (int32_t)e;
  return GVX_ERR_CUDA;
}

gvx_status from_cuda(cudaError_t e) { return e == cudaSuccess ? GVX_OK : cuda_fail(e); }

int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return (d >= 0 && d < kMaxDevices) ? d : 0;
}

size_t scalar_size(int32_t dtype) { return dtype == GVX_F64 ? 8 : 4; }

bool valid_dtype(int32_t dtype) { return dtype == GVX_F64 || dtype == GVX_F32; }

// ncomp = 4 for Lorentz vectors, 3 for velocities.
gvx_status check_lv(const gvx_lv *v, int32_t dtype, int ncomp) {
  if (!v) return GVX_ERR_NULL;
  const size_t es = scalar_size(dtype);
  if (v->layout == GVX_SOA) {
    for (int k = 0; k < ncomp; k++) {
      if (!v->c[k]) return GVX_ERR_NULL;
      if ((uintptr_t)v->c[k] % es) return GVX_ERR_ALIGN;
    }
    return GVX_OK;
  }
  if (v->layout == GVX_AOS) {
    if (!v->c[0]) return GVX_ERR_NULL;
    const size_t al = ncomp == 4 ? 4 * es : es;
    if ((uintptr_t)v->c[0] % al) return GVX_ERR_ALIGN;
    return GVX_OK;
  }
  return GVX_ERR_LAYOUT;
}

#define GVX_TRY(expr)             \
  do {                            \
    gvx_status st_ = (expr);      \
    if (st_ != GVX_OK) return st_; \
  } while (0)

// Autotuned jagged shapes: per device, per log2(n_events) bucket; -1 = not tuned.
std::mutex g_shape_mu;
signed char g_shape[kMaxDevices][64];
bool g_shape_init = false;
constexpr int kDefaultShape = 1;

int bucket_of(int64_t n) {
  int b = 0;
  while (b < 63 && (1ll << (b + 1)) <= n) b++;
  return b;
}

int shape_for(int64_t n_events) {
  std::lock_guard<std::mutex> lk(g_shape_mu);
  if (!g_shape_init) {
    memset(g_shape, -1, sizeof(g_shape));
    g_shape_init = true;
  }
  int s = g_shape[current_device()][bucket_of(n_events)];
  return s < 0 ? kDefaultShape : s;
}

void set_shape(int64_t n_events, int shape) {
  std::lock_guard<std::mutex> lk(g_shape_mu);
  if (!g_shape_init) {
    memset(g_shape, -1, sizeof(g_shape));
    g_shape_init = true;
  }
  g_shape[current_device()][bucket_of(n_events)] = (signed char)shape;
}

struct JaggedCall {
  const gvx_lv *particles;
  const int64_t *offsets;
  int64_t n_events, n_particles;
  int64_t *pair_offsets;
  double *pair_m;
  int64_t pair_capacity;
  gvx_lv *event_sum;
  void *workspace;
  size_t workspace_bytes;
};

gvx_status check_jagged(const JaggedCall &c) {
  if (c.n_events < 0 || c.n_particles < 0 || c.pair_capacity < 0) return GVX_ERR_SIZE;
  if (!c.offsets || !c.pair_offsets) return GVX_ERR_NULL;
  if ((uintptr_t)c.offsets % 8 || (uintptr_t)c.pair_offsets % 8) return GVX_ERR_ALIGN;
  if (c.n_events == 0) return GVX_OK;
  GVX_TRY(check_lv(c.event_sum, GVX_F64, 4));
  if (c.n_particles > 0) GVX_TRY(check_lv(c.particles, GVX_F64, 4));
  if (c.pair_capacity > 0 && !c.pair_m) return GVX_ERR_NULL;
  if ((uintptr_t)c.pair_m % 8) return GVX_ERR_ALIGN;
  if (!c.workspace || c.workspace_bytes < gvx::event_pairs_workspace(c.n_events))
    return GVX_ERR_WORKSPACE;
  if ((uintptr_t)c.workspace % 256) return GVX_ERR_ALIGN;
  return GVX_OK;
}

gvx_status enqueue_jagged(const JaggedCall &c, int shape, cudaStream_t s) {
  if (c.n_events == 0) {
    // pair_offsets[0] = 0 is the whole output
    return from_cuda(cudaMemsetAsync(c.pair_offsets, 0, sizeof(int64_t), s));
  }
  gvx::Lv p = c.particles ? gvx::as_in(*c.particles) : gvx::Lv{{0, 0, 0, 0}, GVX_SOA};
  if (c.n_particles == 0) p.layout = c.particles ? c.particles->layout : GVX_SOA;
  return from_cuda(gvx::launch_event_pairs_shape(shape, p, c.offsets, c.n_events, c.n_particles,
                                                 c.pair_offsets, c.pair_m, c.pair_capacity,
                                                 gvx::as_out(*c.event_sum), c.workspace,
                                                 t_skip_first_tile, s));
}

}  // namespace

struct gvx_graph_s {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  int device;
};

namespace gvx {

int num_sms() {
  static int cache[kMaxDevices] = {0};
  int d = current_device();
  if (cache[d] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d);
    cache[d] = v > 0 ? v : 1;
  }
  return cache[d];
}

gvx_status status_from_cuda(cudaError_t e) { return from_cuda(e); }

int32_t *device_status_word() {
  static int32_t *cache[kMaxDevices] = {nullptr};
  int d = current_device();
  if (!cache[d]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_status) == cudaSuccess) cache[d] = (int32_t *)p;
  }
  return cache[d];
}

}  // namespace gvx

extern "C" {

const char *gvx_version(void) { return "0.1.0"; }

const char *gvx_status_string(int32_t s) {
  switch (s) {
    case GVX_OK: return "GVX_OK";
    case GVX_ERR_NULL: return "GVX_ERR_NULL: a required pointer is NULL";
    case GVX_ERR_SIZE: return "GVX_ERR_SIZE: negative or unsupported size";
    case GVX_ERR_DTYPE: return "GVX_ERR_DTYPE: dtype must be GVX_F64 or GVX_F32";
    case GVX_ERR_LAYOUT: return "GVX_ERR_LAYOUT: layout must be GVX_SOA or GVX_AOS";
    case GVX_ERR_ALIGN: return "GVX_ERR_ALIGN: pointer not aligned for its layout";
    case GVX_ERR_OFFSETS: return "GVX_ERR_OFFSETS: malformed jagged offsets";
    case GVX_ERR_WORKSPACE: return "GVX_ERR_WORKSPACE: workspace missing or too small";
    case GVX_ERR_CUDA: return "GVX_ERR_CUDA: the CUDA runtime refused a launch or copy";
    case GVX_ERR_TIMEOUT: return "GVX_ERR_TIMEOUT: a bounded device-side wait gave up";
    case GVX_ERR_CAPACITY: return "GVX_ERR_CAPACITY: jagged output larger than its buffer";
    case GVX_ERR_ARG: return "GVX_ERR_ARG: invalid argument";
    case GVX_ERR_BOUNDS: return "GVX_ERR_BOUNDS: an index failed a GVX_DEBUG_BOUNDS check";
    default: return "unknown gvx status";
  }
}

int32_t gvx_last_cuda_error(void) { return t_last_cuda_error; }

void gvx_testing_skip_first_tile(int32_t enable) { t_skip_first_tile = enable != 0; }

gvx_status gvx_invariant_mass(const gvx_lv *a, const gvx_lv *b, void *m, int64_t n, int32_t dtype,
                              void *stream) {
  GVX_NVTX_RANGE("gvx_invariant_mass");
  if (!valid_dtype(dtype)) return GVX_ERR_DTYPE;
  if (n < 0) return GVX_ERR_SIZE;
  if (n == 0) return GVX_OK;
  GVX_TRY(check_lv(a, dtype, 4));
  GVX_TRY(check_lv(b, dtype, 4));
  if (!m) return GVX_ERR_NULL;
  if ((uintptr_t)m % scalar_size(dtype)) return GVX_ERR_ALIGN;
  return from_cuda(
      gvx::launch_mass(gvx::as_in(*a), gvx::as_in(*b), m, n, dtype, (cudaStream_t)stream));
}

gvx_status gvx_invariant_mass_cart(const gvx_lv *a, const gvx_lv *b, void *m, int64_t n,
                                   int32_t coords, int32_t dtype, void *stream) {
  GVX_NVTX_RANGE("gvx_invariant_mass_cart");
  if (coords == GVX_PTETAPHIM) return gvx_invariant_mass(a, b, m, n, dtype, stream);
  if (coords != GVX_PXPYPZE && coords != GVX_PXPYPZM && coords != GVX_PTETAPHIE) return GVX_ERR_ARG;
  if (!valid_dtype(dtype)) return GVX_ERR_DTYPE;
  if (n < 0) return GVX_ERR_SIZE;
  if (n == 0) return GVX_OK;
  GVX_TRY(check_lv(a, dtype, 4));
  GVX_TRY(check_lv(b, dtype, 4));
  if (!m) return GVX_ERR_NULL;
  if ((uintptr_t)m % scalar_size(dtype)) return GVX_ERR_ALIGN;
  return from_cuda(gvx::launch_mass_cart(gvx::as_in(*a), gvx::as_in(*b), m, n, coords, dtype,
                                         (cudaStream_t)stream));
}

gvx_status gvx_to_pxpypze(const gvx_lv *v, gvx_lv *out, int64_t n, int32_t coords, int32_t dtype,
                          void *stream) {
  GVX_NVTX_RANGE("gvx_to_pxpypze");
  if (coords != GVX_PTETAPHIM && coords != GVX_PTETAPHIE && coords != GVX_PXPYPZM) return GVX_ERR_ARG;
  if (!valid_dtype(dtype)) return GVX_ERR_DTYPE;
  if (n < 0) return GVX_ERR_SIZE;
  if (n == 0) return GVX_OK;
  GVX_TRY(check_lv(v, dtype, 4));
  GVX_TRY(check_lv(out, dtype, 4));
  return from_cuda(gvx::launch_to_pxpypze(gvx::as_in(*v), gvx::as_out(*out), n, coords, dtype,
                                          (cudaStream_t)stream));
}

gvx_status gvx_lorentz_apply(const void *L, int64_t l_stride, const gvx_lv *v, gvx_lv *out,
                             int64_t n, int32_t dtype, void *stream) {
  GVX_NVTX_RANGE("gvx_lorentz_apply");
  if (!valid_dtype(dtype)) return GVX_ERR_DTYPE;
  if (n < 0) return GVX_ERR_SIZE;
  if (l_stride != 0 && l_stride != 1) return GVX_ERR_ARG;
  if (n == 0) return GVX_OK;
  if (!L) return GVX_ERR_NULL;
  if ((uintptr_t)L % (l_stride ? 16 : scalar_size(dtype))) return GVX_ERR_ALIGN;
  GVX_TRY(check_lv(v, dtype, 4));
  GVX_TRY(check_lv(out, dtype, 4));
  return from_cuda(gvx::launch_lorentz_apply(L, l_stride, gvx::as_in(*v), gvx::as_out(*out), n,
                                             dtype, (cudaStream_t)stream));
}

gvx_status gvx_invariant_mass_bwd(const gvx_lv *a, const gvx_lv *b, const void *m_saved,
                                  const void *grad_m, gvx_lv *grad_a, gvx_lv *grad_b, int64_t n,
                                  int32_t dtype, void *stream) {
  GVX_NVTX_RANGE("gvx_invariant_mass_bwd");
  if (!valid_dtype(dtype)) return GVX_ERR_DTYPE;
  if (n < 0) return GVX_ERR_SIZE;
  if (n == 0) return GVX_OK;
  GVX_TRY(check_lv(a, dtype, 4));
  GVX_TRY(check_lv(b, dtype, 4));
  GVX_TRY(check_lv(grad_a, dtype, 4));
  GVX_TRY(check_lv(grad_b, dtype, 4));
  if (!grad_m) return GVX_ERR_NULL;
  if ((uintptr_t)grad_m % scalar_size(dtype)) return GVX_ERR_ALIGN;
  if (m_saved && (uintptr_t)m_saved % scalar_size(dtype)) return GVX_ERR_ALIGN;
  return from_cuda(gvx::launch_mass_bwd(gvx::as_in(*a), gvx::as_in(*b), m_saved, grad_m,
                                        gvx::as_out(*grad_a), gvx::as_out(*grad_b), n, dtype,
                                        (cudaStream_t)stream));
}

gvx_status gvx_boost(const gvx_lv *v, const gvx_lv *beta, int64_t beta_stride, gvx_lv *out,
                     int64_t n, int32_t dtype, void *stream) {
  GVX_NVTX_RANGE("gvx_boost");
  if (!valid_dtype(dtype)) return GVX_ERR_DTYPE;
  if (n < 0) return GVX_ERR_SIZE;
  if (beta_stride != 0 && beta_stride != 1) return GVX_ERR_ARG;
  if (n == 0) return GVX_OK;
  GVX_TRY(check_lv(v, dtype, 4));
  GVX_TRY(check_lv(beta, dtype, 3));
  GVX_TRY(check_lv(out, dtype, 4));
  return from_cuda(gvx::launch_boost(gvx::as_in(*v), gvx::as_in(*beta), beta_stride,
                                     gvx::as_out(*out), n, dtype, (cudaStream_t)stream));
}

size_t gvx_boost_bwd_workspace(int64_t n, int64_t beta_stride, int32_t dtype) {
  if (n <= 0 || !valid_dtype(dtype)) return 0;
  return gvx::boost_bwd_workspace(n, beta_stride, dtype);
}

gvx_status gvx_boost_bwd(const gvx_lv *v, const gvx_lv *beta, int64_t beta_stride,
                         const gvx_lv *grad_out, gvx_lv *grad_v, gvx_lv *grad_beta, int64_t n,
                         int32_t dtype, void *workspace, size_t workspace_bytes, void *stream) {
  GVX_NVTX_RANGE("gvx_boost_bwd");
  if (!valid_dtype(dtype)) return GVX_ERR_DTYPE;
  if (n < 0) return GVX_ERR_SIZE;
  if (beta_stride != 0 && beta_stride != 1) return GVX_ERR_ARG;
  if (n == 0) return GVX_OK;
  GVX_TRY(check_lv(v, dtype, 4));
  GVX_TRY(check_lv(beta, dtype, 3));
  GVX_TRY(check_lv(grad_out, dtype, 4));
  GVX_TRY(check_lv(grad_v, dtype, 4));
  GVX_TRY(check_lv(grad_beta, dtype, 3));
  const size_t need = gvx::boost_bwd_workspace(n, beta_stride, dtype);
  if (need > 0 && (!workspace || workspace_bytes < need)) return GVX_ERR_WORKSPACE;
  if (need > 0 && (uintptr_t)workspace % 8) return GVX_ERR_ALIGN;
  return from_cuda(gvx::launch_boost_bwd(gvx::as_in(*v), gvx::as_in(*beta), beta_stride,
                                         gvx::as_in(*grad_out), gvx::as_out(*grad_v),
                                         gvx::as_out(*grad_beta), n, dtype, workspace,
                                         (cudaStream_t)stream));
}

size_t gvx_event_pair_masses_workspace(int64_t n_events) {
  return n_events <= 0 ? 0 : gvx::event_pairs_workspace(n_events);
}

gvx_status gvx_event_pair_masses(const gvx_lv *particles, const int64_t *offsets, int64_t n_events,
                                 int64_t n_particles, int64_t *pair_offsets, double *pair_m,
                                 int64_t pair_capacity, gvx_lv *event_sum, void *workspace,
                                 size_t workspace_bytes, void *stream) {
  GVX_NVTX_RANGE("gvx_event_pair_masses");
  JaggedCall c{particles, offsets, n_events, n_particles, pair_offsets, pair_m,
               pair_capacity, event_sum, workspace, workspace_bytes};
  GVX_TRY(check_jagged(c));
  return enqueue_jagged(c, shape_for(n_events), (cudaStream_t)stream);
}

size_t gvx_event_pair_masses_bwd_workspace(int64_t n_events) {
  return n_events <= 0 ? 0 : gvx::event_pairs_bwd_workspace(n_events);
}

gvx_status gvx_event_pair_masses_bwd(const gvx_lv *particles, const int64_t *offsets,
                                     const int64_t *pair_offsets, int64_t n_events,
                                     int64_t n_particles, const double *grad_pair_m,
                                     int64_t n_pairs, const gvx_lv *grad_event_sum,
                                     gvx_lv *grad_particles, void *workspace,
                                     size_t workspace_bytes, void *stream) {
  GVX_NVTX_RANGE("gvx_event_pair_masses_bwd");
  if (n_events < 0 || n_particles < 0 || n_pairs < 0) return GVX_ERR_SIZE;
  if (!offsets || !pair_offsets) return GVX_ERR_NULL;
  if ((uintptr_t)offsets % 8 || (uintptr_t)pair_offsets % 8) return GVX_ERR_ALIGN;
  if (n_events == 0 || n_particles == 0) return GVX_OK;  // no particle has a gradient
  if (!workspace || workspace_bytes < gvx::event_pairs_bwd_workspace(n_events))
    return GVX_ERR_WORKSPACE;
  if ((uintptr_t)workspace % 256) return GVX_ERR_ALIGN;
  GVX_TRY(check_lv(particles, GVX_F64, 4));
  GVX_TRY(check_lv(grad_particles, GVX_F64, 4));
  if (grad_event_sum) GVX_TRY(check_lv(grad_event_sum, GVX_F64, 4));
  if (n_pairs > 0 && !grad_pair_m) return GVX_ERR_NULL;
  if ((uintptr_t)grad_pair_m % 8) return GVX_ERR_ALIGN;
  gvx::Lv gs;
  if (grad_event_sum) gs = gvx::as_in(*grad_event_sum);
  return from_cuda(gvx::launch_event_pairs_bwd(gvx::as_in(*particles), offsets, pair_offsets,
                                               n_events, n_particles, grad_pair_m, n_pairs,
                                               grad_event_sum ? &gs : nullptr,
                                               gvx::as_out(*grad_particles), workspace,
                                               (cudaStream_t)stream));
}

gvx_status gvx_event_pair_select(const gvx_lv *particles, const int64_t *offsets,
                                 int64_t n_events, int64_t n_particles, double pt_min,
                                 double eta_max, double lo, double hi, int32_t n_bins,
                                 double target, uint64_t *counts, int64_t *best_k, double *best_m,
                                 void *stream) {
  GVX_NVTX_RANGE("gvx_event_pair_select");
  if (n_events < 0 || n_particles < 0) return GVX_ERR_SIZE;
  if (n_bins < 1 || n_bins > GVX_SELECT_MAX_BINS) return GVX_ERR_SIZE;
  if (!(hi > lo) || !(fabs(hi - lo) < INFINITY)) return GVX_ERR_ARG;
  if (!offsets || !counts) return GVX_ERR_NULL;
  if ((uintptr_t)offsets % 8 || (uintptr_t)counts % 8 || (uintptr_t)best_k % 8 ||
      (uintptr_t)best_m % 8)
    return GVX_ERR_ALIGN;
  if (n_events == 0) return GVX_OK;
  if (n_particles > 0) GVX_TRY(check_lv(particles, GVX_F64, 4));
  gvx::Lv p = particles ? gvx::as_in(*particles) : gvx::Lv{{0, 0, 0, 0}, GVX_SOA};
  return from_cuda(gvx::launch_pair_select(p, offsets, n_events, n_particles, pt_min, eta_max,
                                           lo, hi, n_bins, target, counts, best_k, best_m,
                                           (cudaStream_t)stream));
}

int32_t gvx_event_pair_masses_num_shapes(void) { return gvx::event_pairs_num_shapes(); }

gvx_status gvx_event_pair_masses_shape(int32_t shape, int32_t *events_per_tile,
                                       int32_t *threads) {
  if (shape < 0 || shape >= gvx::event_pairs_num_shapes()) return GVX_ERR_ARG;
  if (!events_per_tile || !threads) return GVX_ERR_NULL;
  int te, nt;
  gvx::event_pairs_shape(shape, &te, &nt);
  *events_per_tile = te;
  *threads = nt;
  return GVX_OK;
}

int32_t gvx_event_pair_masses_get_shape(int64_t n_events) { return shape_for(n_events); }

gvx_status gvx_event_pair_masses_set_shape(int64_t n_events, int32_t shape) {
  if (shape < 0 || shape >= gvx::event_pairs_num_shapes()) return GVX_ERR_ARG;
  set_shape(n_events, shape);
  return GVX_OK;
}

gvx_status gvx_event_pair_masses_autotune(const gvx_lv *particles, const int64_t *offsets,
                                          int64_t n_events, int64_t n_particles,
                                          int64_t *pair_offsets, double *pair_m,
                                          int64_t pair_capacity, gvx_lv *event_sum,
                                          void *workspace, size_t workspace_bytes, int32_t reps,
                                          void *stream, int32_t *best_shape, float *best_ms) {
  GVX_NVTX_RANGE("gvx_event_pair_masses_autotune");
  JaggedCall c{particles, offsets, n_events, n_particles, pair_offsets, pair_m,
               pair_capacity, event_sum, workspace, workspace_bytes};
  GVX_TRY(check_jagged(c));
  if (reps < 1) reps = 1;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(cudaGetLastError());
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(cudaGetLastError());
  }
  int best = -1;
  float best_t = 0;
  gvx_status st = GVX_OK;
  for (int shape = 0; shape < gvx::event_pairs_num_shapes() && st == GVX_OK; shape++) {
    st = enqueue_jagged(c, shape, s);  // warm-up
    float total = 0;
    for (int r = 0; r < reps && st == GVX_OK; r++) {
      cudaEventRecord(e0, s);
      st = enqueue_jagged(c, shape, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) st = cuda_fail(cudaGetLastError());
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      total += ms;
    }
    if (st == GVX_OK && (best < 0 || total / reps < best_t)) {
      best = shape;
      best_t = total / reps;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != GVX_OK) return st;
  set_shape(n_events, best);
  if (best_shape) *best_shape = best;
  if (best_ms) *best_ms = best_t;
  return GVX_OK;
}

gvx_status gvx_event_pair_masses_graph_create(const gvx_lv *particles, const int64_t *offsets,
                                              int64_t n_events, int64_t n_particles,
                                              int64_t *pair_offsets, double *pair_m,
                                              int64_t pair_capacity, gvx_lv *event_sum,
                                              void *workspace, size_t workspace_bytes,
                                              gvx_graph *out) {
  GVX_NVTX_RANGE("gvx_event_pair_masses_graph_create");
  if (!out) return GVX_ERR_NULL;
  *out = nullptr;
  JaggedCall c{particles, offsets, n_events, n_particles, pair_offsets, pair_m,
               pair_capacity, event_sum, workspace, workspace_bytes};
  GVX_TRY(check_jagged(c));
  const int shape = shape_for(n_events);
  // the function attributes and the status-word address are set up outside the capture
  if (!gvx::device_status_word()) return cuda_fail(cudaGetLastError());
  cudaStream_t cs;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e);
  gvx_status st = enqueue_jagged(c, shape, cs);  // first launch sets the kernel attributes
  if (st == GVX_OK) st = from_cuda(cudaStreamSynchronize(cs));
  cudaGraph_t g = nullptr;
  if (st == GVX_OK) st = from_cuda(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  if (st == GVX_OK) {
    gvx_status st2 = enqueue_jagged(c, shape, cs);
    cudaError_t ee = cudaStreamEndCapture(cs, &g);
    st = st2 != GVX_OK ? st2 : from_cuda(ee);
  }
  cudaGraphExec_t ex = nullptr;
  if (st == GVX_OK) st = from_cuda(cudaGraphInstantiate(&ex, g, 0));
  cudaStreamDestroy(cs);
  if (st != GVX_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  gvx_graph h = new gvx_graph_s{g, ex, current_device()};
  *out = h;
  return GVX_OK;
}

gvx_status gvx_graph_launch(gvx_graph g, void *stream) {
  GVX_NVTX_RANGE("gvx_graph_launch");
  if (!g) return GVX_ERR_NULL;
  return from_cuda(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
}

gvx_status gvx_graph_destroy(gvx_graph g) {
  if (!g) return GVX_OK;
  cudaGraphExecDestroy(g->exec);
  cudaGraphDestroy(g->graph);
  delete g;
  return GVX_OK;
}

gvx_status gvx_device_status(void *stream, int32_t *host_status) {
  if (!host_status) return GVX_ERR_NULL;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e);
  int32_t v = 0;
  e = cudaMemcpyFromSymbol(&v, g_device_status, sizeof(v));
  if (e != cudaSuccess) return cuda_fail(e);
  const int32_t zero = 0;
  e = cudaMemcpyToSymbol(g_device_status, &zero, sizeof(zero));
  if (e != cudaSuccess) return cuda_fail(e);
  *host_status = v;
  return GVX_OK;
}

}  // extern "C"
