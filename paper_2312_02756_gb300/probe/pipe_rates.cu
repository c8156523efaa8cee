// Pipe-rate probe: the issue rates of the instruction kinds the FP64 kernels trade against each
// other (FP64 FMA/add on the FP64 pipe, FP32 FMA scalar and paired, integer multiply-add and
// logic, the special-function unit, int -> float conversion).  Each thread runs kChains
// independent dependency chains of one operation for `iters` steps; a launch fills every SM
// several times over.  Times are CUDA events around one launch (best of kRuns after a warm-up).
// Prints one JSON line: per kind, operations per second over the whole GPU.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kRuns = 5;

enum Kind { DFMA, DADD, FFMA, FFMA2, IMAD, LOP3, MUFU_RSQ, I2F, NKIND };
static const char *kName[NKIND] = {"dfma", "dadd", "ffma", "ffma2_pairs", "imad", "lop3",
                                   "mufu_rsq", "i2f"};
// operations counted per chain step (a paired FMA counts as two FP32 FMAs)
static const int kOpsPerStep[NKIND] = {1, 1, 1, 2, 1, 1, 1, 1};

template <int K>
__global__ void __launch_bounds__(kThreads) probe(int iters, float fa, float fb, uint32_t ua,
                                                  uint32_t ub, uint32_t uc, double *sink) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double dacc = 0.0;
  if constexpr (K == DFMA || K == DADD) {
    double x[kChains];
    for (int c = 0; c < kChains; c++) x[c] = 1.0 + 1e-3 * (t + c);
    const double a = 1.0 - 1e-12 * fa, b = 1e-9 * fb;
    for (int i = 0; i < iters; i++)
#pragma unroll
      for (int c = 0; c < kChains; c++) x[c] = K == DFMA ? fma(x[c], a, b) : x[c] + b;
    for (int c = 0; c < kChains; c++) dacc += x[c];
  } else if constexpr (K == FFMA || K == MUFU_RSQ) {
    float x[kChains];
    for (int c = 0; c < kChains; c++) x[c] = 1.0f + 1e-3f * (float)((t + c) & 255);
    for (int i = 0; i < iters; i++)
#pragma unroll
      for (int c = 0; c < kChains; c++) x[c] = K == FFMA ? __fmaf_rn(x[c], fa, fb) : rsqrtf(x[c]);
    for (int c = 0; c < kChains; c++) dacc += x[c];
  } else if constexpr (K == FFMA2) {
    float2 x[kChains];
    for (int c = 0; c < kChains; c++) x[c] = make_float2(1.0f + 1e-3f * c, 1.0f - 1e-3f * c);
    const float2 a = make_float2(fa, fa), b = make_float2(fb, fb);
    for (int i = 0; i < iters; i++)
#pragma unroll
      for (int c = 0; c < kChains; c++) x[c] = __ffma2_rn(x[c], a, b);
    for (int c = 0; c < kChains; c++) dacc += x[c].x + x[c].y;
  } else if constexpr (K == IMAD || K == LOP3) {
    uint32_t x[kChains];
    for (int c = 0; c < kChains; c++) x[c] = (uint32_t)t * 2654435761u + c;
    for (int i = 0; i < iters; i++)
#pragma unroll
      for (int c = 0; c < kChains; c++) x[c] = K == IMAD ? x[c] * ua + ub : ((x[c] & ua) ^ ub) | uc;
    for (int c = 0; c < kChains; c++) dacc += (double)x[c];
  } else {  // I2F: int -> float, the float's bits fed back as the next int (one logic op too)
    uint32_t x[kChains];
    for (int c = 0; c < kChains; c++) x[c] = (uint32_t)t + 977u * c;
    for (int i = 0; i < iters; i++)
#pragma unroll
      for (int c = 0; c < kChains; c++) x[c] = __float_as_uint(__int2float_rn((int)x[c])) ^ ua;
    for (int c = 0; c < kChains; c++) dacc += (double)x[c];
  }
  if (dacc == 12345.678) sink[t] = dacc;  // keeps the chains live
}

template <int K>
static float time_kind(int blocks, int iters, double *sink) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  probe<K><<<blocks, kThreads>>>(iters / 8, 0.999f, 1e-7f, 0x7fffffffu, 0x1234567u, 0x10u, sink);
  float best = 1e30f;
  for (int r = 0; r < kRuns; r++) {
    cudaEventRecord(e0);
    probe<K><<<blocks, kThreads>>>(iters, 0.999f, 1e-7f, 0x7fffffffu, 0x1234567u, 0x10u, sink);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

int main(int argc, char **argv) {
  int iters = argc > 1 ? atoi(argv[1]) : 4096;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, 0) != cudaSuccess) {
    fprintf(stderr, "no CUDA device\n");
    return 1;
  }
  const int blocks = prop.multiProcessorCount * 8;
  double *sink = nullptr;
  if (cudaMalloc(&sink, sizeof(double) * blocks * kThreads) != cudaSuccess) return 1;
  float ms[NKIND] = {time_kind<DFMA>(blocks, iters / 8, sink), time_kind<DADD>(blocks, iters / 8, sink),
                     time_kind<FFMA>(blocks, iters, sink),     time_kind<FFMA2>(blocks, iters, sink),
                     time_kind<IMAD>(blocks, iters, sink),     time_kind<LOP3>(blocks, iters, sink),
                     time_kind<MUFU_RSQ>(blocks, iters, sink), time_kind<I2F>(blocks, iters, sink)};
  const int it[NKIND] = {iters / 8, iters / 8, iters, iters, iters, iters, iters, iters};
  cudaError_t err = cudaDeviceSynchronize();
  printf("{\"device\": \"%s\", \"sms\": %d, \"blocks\": %d, \"threads\": %d, \"chains\": %d",
         prop.name, prop.multiProcessorCount, blocks, kThreads, kChains);
  for (int k = 0; k < NKIND; k++) {
    double ops = (double)blocks * kThreads * kChains * it[k] * kOpsPerStep[k];
    printf(", \"%s\": {\"ms\": %.4f, \"ops_per_s\": %.4e}", kName[k], ms[k], ops / (ms[k] * 1e-3));
  }
  printf(", \"cuda_error\": %d}\n", (int)err);
  cudaFree(sink);
  return err != cudaSuccess;
}
