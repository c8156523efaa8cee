// Helpers shared by the jagged kernels: the row-major packing of the pairs of one event (the
// order the jagged outputs use) and a block-wide exclusive scan.
#pragma once

#include <stdint.h>

namespace gvx {

// Row-major index k of pair (i, j), i < j, among n particles: k = i n - i(i+1)/2 + (j - i - 1).
// Inverse: the largest i with start(i) = i (2n - i - 1)/2 <= k.  The estimate from the
// quadratic formula (in float: within one of the answer for the sizes staged in shared memory)
// is corrected by integer steps, so the result is exact for any n.
__device__ __forceinline__ void decode_pair(int64_t k, int64_t n, int64_t &i, int64_t &j) {
  float b = (float)(2 * n - 1);
  int64_t r = (int64_t)((b - sqrtf(fmaxf(b * b - 8.0f * (float)k, 0.0f))) * 0.5f);
  if (r < 0) r = 0;
  if (r > n - 2) r = n - 2;
  while (r > 0 && r * (2 * n - r - 1) / 2 > k) r--;
  while ((r + 1) * (2 * n - r - 2) / 2 <= k) r++;
  i = r;
  j = k - r * (2 * n - r - 1) / 2 + r + 1;
}

// The same decoding with a double-precision estimate, for events of any size.
__device__ __forceinline__ void decode_pair_wide(int64_t k, int64_t n, int64_t &i, int64_t &j) {
  double b = (double)(2 * n - 1);
  int64_t r = (int64_t)((b - sqrt(fmax(b * b - 8.0 * (double)k, 0.0))) * 0.5);
  if (r < 0) r = 0;
  if (r > n - 2) r = n - 2;
  while (r > 0 && r * (2 * n - r - 1) / 2 > k) r--;
  while ((r + 1) * (2 * n - r - 2) / 2 <= k) r++;
  i = r;
  j = k - r * (2 * n - r - 1) / 2 + r + 1;
}

// Exclusive scan of one int64 per thread; *total gets the block sum.  Ends synchronised.
template <int NT>
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *s_warp, int64_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < NT / 32 ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NT / 32) s_warp[lane] = w;
  }
  __syncthreads();
  int64_t excl = x - v + (warp > 0 ? s_warp[warp - 1] : 0);
  *total = s_warp[NT / 32 - 1];
  __syncthreads();
  return excl;
}

}  // namespace gvx
