// gvx_event_pair_masses_noalloc: the jagged-event kernel with its scratch memory in a fixed-size
// array that belongs to the library module, for callers that must not allocate device memory.
//
// The scratch (tile counter + look-back descriptors) lives in g_scratch below.  Host code never
// uses the name g_scratch as an address: the device address comes from cudaGetSymbolAddress,
// taken once per device (with that device current) by the first call on it and cached.  The
// cached address belongs to the context it was taken in: after cudaDeviceReset it is stale.
// Every call shares the one array; each call clears the part it uses before its kernel runs, so
// calls that overlap on the GPU (different streams, no ordering between them) race on it.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "gvx.h"
#include "gvx_internal.h"

namespace gvx {
cudaError_t launch_event_pairs_shape(int shape, const Lv &p, const int64_t *off, int64_t n_events,
                                     int64_t n_particles, int64_t *pair_off, double *pair_m,
                                     int64_t capacity, const LvOut &sums, void *ws,
                                     bool skip_first_tile, cudaStream_t s);
}  // namespace gvx

namespace {

// Scratch for GVX_NOALLOC_MAX_EVENTS events: 256 bytes of tile counter and one 8-byte descriptor
// per 64 events (the smallest tile), i.e. gvx_event_pair_masses_workspace(2^21) = 262,400 bytes.
constexpr int64_t kMaxEvents = GVX_NOALLOC_MAX_EVENTS;
constexpr size_t kScratchBytes = 256 + 8 * (size_t)((kMaxEvents + 63) / 64);

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices];

// Device address of g_scratch on the current device (set-up on the first call per device).
cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

gvx_status check_lv64(const gvx_lv *v) {
  if (!v) return GVX_ERR_NULL;
  if (v->layout == GVX_SOA) {
    for (int k = 0; k < 4; k++) {
      if (!v->c[k]) return GVX_ERR_NULL;
      if ((uintptr_t)v->c[k] % 8) return GVX_ERR_ALIGN;
    }
    return GVX_OK;
  }
  if (v->layout == GVX_AOS) {
    if (!v->c[0]) return GVX_ERR_NULL;
    return (uintptr_t)v->c[0] % 32 ? GVX_ERR_ALIGN : GVX_OK;
  }
  return GVX_ERR_LAYOUT;
}

}  // namespace

extern "C" gvx_status gvx_event_pair_masses_noalloc(const gvx_lv *particles,
                                                    const int64_t *offsets, int64_t n_events,
                                                    int64_t n_particles, int64_t *pair_offsets,
                                                    double *pair_m, int64_t pair_capacity,
                                                    gvx_lv *event_sum, void *stream) {
  GVX_NVTX_RANGE("gvx_event_pair_masses_noalloc");
  if (n_events < 0 || n_particles < 0 || pair_capacity < 0) return GVX_ERR_SIZE;
  if (n_events > kMaxEvents) return GVX_ERR_SIZE;  // beyond the fixed scratch
  if (!offsets || !pair_offsets) return GVX_ERR_NULL;
  if ((uintptr_t)offsets % 8 || (uintptr_t)pair_offsets % 8) return GVX_ERR_ALIGN;
  cudaStream_t s = (cudaStream_t)stream;
  if (n_events == 0) {
    return gvx::status_from_cuda(cudaMemsetAsync(pair_offsets, 0, sizeof(int64_t), s));
  }
  gvx_status st = check_lv64(event_sum);
  if (st != GVX_OK) return st;
  if (n_particles > 0 && (st = check_lv64(particles)) != GVX_OK) return st;
  if (pair_capacity > 0 && !pair_m) return GVX_ERR_NULL;
  if ((uintptr_t)pair_m % 8) return GVX_ERR_ALIGN;
  if (gvx::event_pairs_workspace(n_events) > kScratchBytes) return GVX_ERR_SIZE;
  void *ws = nullptr;
  cudaError_t e = scratch_address(&ws);
  if (e == cudaSuccess) {
    gvx::Lv p = particles ? gvx::as_in(*particles) : gvx::Lv{{0, 0, 0, 0}, GVX_SOA};
    e = gvx::launch_event_pairs_shape(gvx_event_pair_masses_get_shape(n_events), p, offsets,
                                      n_events, n_particles, pair_offsets, pair_m, pair_capacity,
                                      gvx::as_out(*event_sum), ws, false, s);
  }
  return gvx::status_from_cuda(e);
}
