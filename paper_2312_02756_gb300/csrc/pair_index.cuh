// Row-major packing of the pairs of one event (the order the jagged outputs use), shared by the
// jagged kernels.
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

}  // namespace gvx
