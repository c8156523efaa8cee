// Internal interface between the C-ABI layer (api.cu) and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "gvx.h"

namespace gvx {

// Device-side view of one Lorentz-vector (or velocity) array.
struct Lv {
  const void *c[4];
  int32_t layout;  // GVX_SOA / GVX_AOS
};
struct LvOut {
  void *c[4];
  int32_t layout;
};

inline Lv as_in(const gvx_lv &v) { return Lv{{v.c[0], v.c[1], v.c[2], v.c[3]}, v.layout}; }
inline LvOut as_out(const gvx_lv &v) { return LvOut{{v.c[0], v.c[1], v.c[2], v.c[3]}, v.layout}; }

// Number of SMs of the current device (cached per device).
int num_sms();

// Device status word (one per device, in device memory owned by the library).
int32_t *device_status_word();

// GVX_OK for cudaSuccess; otherwise GVX_ERR_CUDA, with the error recorded for
// gvx_last_cuda_error on this host thread.
gvx_status status_from_cuda(cudaError_t e);

cudaError_t launch_mass(const Lv &a, const Lv &b, void *m, int64_t n, int dtype,
                        cudaStream_t s);
cudaError_t launch_mass_bwd(const Lv &a, const Lv &b, const void *ms, const void *gm,
                            const LvOut &ga, const LvOut &gb, int64_t n, int dtype, cudaStream_t s);
cudaError_t launch_boost(const Lv &v, const Lv &beta, int64_t beta_stride, const LvOut &out,
                         int64_t n, int dtype, cudaStream_t s);
size_t boost_bwd_workspace(int64_t n, int64_t beta_stride, int dtype);
cudaError_t launch_boost_bwd(const Lv &v, const Lv &beta, int64_t beta_stride, const Lv &gout,
                             const LvOut &gv, const LvOut &gbeta, int64_t n, int dtype,
                             void *ws, cudaStream_t s);
size_t event_pairs_workspace(int64_t n_events);
cudaError_t launch_to_pxpypze(const Lv &v, const LvOut &out, int64_t n, int coords, int dtype,
                              cudaStream_t s);
cudaError_t launch_mass_cart(const Lv &a, const Lv &b, void *m, int64_t n, int coords, int dtype,
                             cudaStream_t s);
cudaError_t launch_lorentz_apply(const void *L, int64_t l_stride, const Lv &v, const LvOut &out,
                                 int64_t n, int dtype, cudaStream_t s);
cudaError_t launch_pair_select(const Lv &p, const int64_t *off, int64_t n_events,
                               int64_t n_particles, double pt_min, double eta_max, double lo,
                               double hi, int n_bins, double target, uint64_t *counts,
                               int64_t *best_k, double *best_m, cudaStream_t s);
size_t event_pairs_bwd_workspace(int64_t n_events);
cudaError_t launch_event_pairs_bwd(const Lv &p, const int64_t *off, const int64_t *pair_off,
                                   int64_t n_events, int64_t n_particles, const double *gpm,
                                   int64_t n_pairs, const Lv *gsum, const LvOut &grad, void *ws,
                                   cudaStream_t s);

// One NVTX range per compute call of the ABI, named after it (visible in Nsight timelines;
// NVTX costs a pointer check when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace gvx

#define GVX_NVTX_RANGE(name) ::gvx::NvtxRange gvx_nvtx_range_(name)
