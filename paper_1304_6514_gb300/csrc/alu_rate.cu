// Measured FMA throughput of this GPU's float64 and float32 pipes: the peak
// that the ALU-bound build kernels are reported against.  Every thread runs
// eight independent chains x <- fma(x, a, b) (a and b are launch arguments,
// so nothing folds); a persistent grid fills every SM with 2048 threads.
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace nvpit {

constexpr int kRateChains = 8;
constexpr int kRateUnroll = 4;
__device__ double g_rate_sink;

template <typename T>
__global__ void __launch_bounds__(256) alu_rate_kernel(T a, T b, int64_t iters) {
  T x[kRateChains];
#pragma unroll
  for (int i = 0; i < kRateChains; ++i) x[i] = (T)(threadIdx.x + 1 + i) * (T)1e-3;
  for (int64_t k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < kRateUnroll; ++u) {
#pragma unroll
      for (int i = 0; i < kRateChains; ++i) x[i] = fma(x[i], a, b);
    }
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < kRateChains; ++i) s += x[i];
  // never true for the values used (the chains converge to b / (1 - a) > 0),
  // but the compiler cannot know that: the chains stay live
  if (s == (T)-1.0) g_rate_sink = (double)s;
}

template <typename T>
static nv_status measure(int64_t iters, cudaStream_t s, double* flops_per_s) {
  int dev = 0, sms = 0, per_sm = 0;
  nv_status st = nv_cuda_check(cudaGetDevice(&dev), "current device");
  if (st != NV_OK) return st;
  st = nv_cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
  if (st != NV_OK) return st;
  st = nv_cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, alu_rate_kernel<T>, 256, 0),
                     "occupancy query");
  if (st != NV_OK) return st;
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  st = nv_cuda_check(cudaEventCreate(&e0), "event");
  if (st == NV_OK) st = nv_cuda_check(cudaEventCreate(&e1), "event");
  const T a = (T)0.999999, b = (T)1e-7;
  if (st == NV_OK) {
    alu_rate_kernel<T><<<grid, 256, 0, s>>>(a, b, iters / 4);    // warm-up (clocks ramp)
    st = nv_cuda_check(cudaGetLastError(), "rate kernel launch");
  }
  const int reps = 3;
  if (st == NV_OK) {
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r) alu_rate_kernel<T><<<grid, 256, 0, s>>>(a, b, iters);
    cudaEventRecord(e1, s);
    st = nv_cuda_check(cudaGetLastError(), "rate kernel launch");
  }
  if (st == NV_OK) st = nv_cuda_check(cudaEventSynchronize(e1), "rate kernel");
  float ms = 0.f;
  if (st == NV_OK) st = nv_cuda_check(cudaEventElapsedTime(&ms, e0, e1), "event time");
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st != NV_OK) return st;
  const double flop = 2.0 * kRateChains * kRateUnroll * (double)iters * grid * 256.0 * reps;
  *flops_per_s = flop / (ms * 1e-3);
  return NV_OK;
}

}  // namespace nvpit

extern "C" nv_status nv_alu_rate(int32_t prec, double* flops_per_s, void* stream) {
  if (!flops_per_s) return nv_fail(NV_EINVAL, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // about 20 ms per launch at the nominal rates (1.25 / 80 TFLOP/s)
  if (prec == NV_FP64) return nvpit::measure<double>(1250, s, flops_per_s);
  if (prec == NV_FP32) return nvpit::measure<float>(80000, s, flops_per_s);
  return nv_fail(NV_EINVAL, "precision must be NV_FP64 or NV_FP32");
}
