// Device-side building blocks shared by the kernels: right-hand sides, the
// fine schemes, the device status word and a bounded grid barrier.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace nvpit {

// ---------------------------------------------------------------------------
// Device status word: the first error recorded wins.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void record_status(int* status, int code) {
  atomicCAS(status, (int)NV_OK, code);
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier for a cooperative launch of G CTAs.  `target` = (round+1)*G.
// Every wait is bounded: after ~2^22 polls (>= 0.4 s with the back-off) the CTA
// records NV_ETIMEOUT and returns false, so no launch can hang the device.
__device__ __forceinline__ bool grid_barrier(unsigned* counter, unsigned target, int* status,
                                             int* smem_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(counter, 1u);
    int ok = 1;
    unsigned polls = 0;
    while (ld_acquire_u32(counter) < target) {
      if (++polls > (1u << 22)) {
        record_status(status, NV_ETIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(polls < 64 ? 32 : 100);
    }
    __threadfence();
    *smem_flag = ok;
  }
  __syncthreads();
  return *smem_flag != 0;
}

// Round a float32 to the nearest TF32 value (10 explicit mantissa bits, ties
// away from zero).  Tensor cores read TF32 operands by dropping the low 13
// bits; feeding them values that are already rounded keeps the operand error
// unbiased instead of always toward zero.
__device__ __forceinline__ float round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Right-hand-side parameters passed by value to kernels.
struct RhsParams {
  double p[NVPIT_MAX_PARAMS];
};

// ---------------------------------------------------------------------------
// Right-hand sides of the table workloads, f(c, y) with c a staged
// time-dependent coefficient (cos t for the cos-cubic problem).
// ---------------------------------------------------------------------------
template <typename T>
struct RhsLinearScalar {
  static constexpr int D = 1;
  static constexpr bool TIME_DEP = false;
  T lam;
  __device__ explicit RhsLinearScalar(const double* p) : lam((T)p[0]) {}
  __device__ __forceinline__ void operator()(T, const T* y, T* f) const { f[0] = lam * y[0]; }
};

template <typename T>
struct RhsSquare {
  static constexpr int D = 1;
  static constexpr bool TIME_DEP = false;
  __device__ explicit RhsSquare(const double*) {}
  __device__ __forceinline__ void operator()(T, const T* y, T* f) const { f[0] = y[0] * y[0]; }
};

template <typename T>
struct RhsCosCubic {  // y' = cos(t) y - y^3 = y (cos t - y^2)
  static constexpr int D = 1;
  static constexpr bool TIME_DEP = true;
  __device__ explicit RhsCosCubic(const double*) {}
  __device__ __forceinline__ void operator()(T c, const T* y, T* f) const {
    f[0] = y[0] * (c - y[0] * y[0]);
  }
};

template <typename T>
struct RhsVdp {  // x' = y, y' = mu (1 - x^2) y - x
  static constexpr int D = 2;
  static constexpr bool TIME_DEP = false;
  T mu;
  __device__ explicit RhsVdp(const double* p) : mu((T)p[0]) {}
  __device__ __forceinline__ void operator()(T, const T* y, T* f) const {
    f[0] = y[1];
    f[1] = mu * ((T)1 - y[0] * y[0]) * y[1] - y[0];
  }
};

template <typename T>
struct RhsChain3 {  // wall-m1-m2-m3-wall, tension k d + k3 d^3, damping c
  static constexpr int D = 6;
  static constexpr bool TIME_DEP = false;
  T k, k3, c;
  __device__ explicit RhsChain3(const double* p) : k((T)p[0]), k3((T)p[1]), c((T)p[2]) {}
  __device__ __forceinline__ T tension(T d) const { return d * (k + k3 * d * d); }
  __device__ __forceinline__ void operator()(T, const T* y, T* f) const {
    const T t0 = tension(y[0]), t1 = tension(y[1] - y[0]), t2 = tension(y[2] - y[1]);
    const T t3 = -tension(y[2]);
    f[0] = y[3];
    f[1] = y[4];
    f[2] = y[5];
    f[3] = -t0 + t1 - c * y[3];
    f[4] = -t1 + t2 - c * y[4];
    f[5] = -t2 + t3 - c * y[5];
  }
};

// ---------------------------------------------------------------------------
// Fine schemes for a D-dimensional state held in registers.
// c0, ch, c1: the time-dependent coefficient at t, t + h/2, t + h.
// ---------------------------------------------------------------------------
// State update y <- y + inc.  In float32 the update is compensated (Kahan):
// the rounding error of each addition is carried in c and fed back, so long
// recurrences of small increments keep float32 rounding instead of growing
// with the step count.  In float64 it is the plain sum.
template <typename T>
__device__ __forceinline__ void add_update(T& y, T inc, T& c) {
  if constexpr (sizeof(T) == 4) {
    const T yk = inc - c;
    const T t = y + yk;
    c = (t - y) - yk;
    y = t;
  } else {
    y = y + inc;
  }
}

template <class R, typename T>
__device__ __forceinline__ void euler_step(const R& rhs, T c0, T h, T* y, T* comp) {
  T f[R::D];
  rhs(c0, y, f);
#pragma unroll
  for (int d = 0; d < R::D; ++d) add_update(y[d], h * f[d], comp[d]);
}

template <class R, typename T>
__device__ __forceinline__ void rk4_step(const R& rhs, T c0, T ch, T c1, T h, T* y, T* comp) {
  T k[R::D], z[R::D], acc[R::D];
  const T hh = h * (T)0.5;
  rhs(c0, y, k);
#pragma unroll
  for (int d = 0; d < R::D; ++d) { acc[d] = k[d]; z[d] = y[d] + hh * k[d]; }
  rhs(ch, z, k);
#pragma unroll
  for (int d = 0; d < R::D; ++d) { acc[d] += (T)2 * k[d]; z[d] = y[d] + hh * k[d]; }
  rhs(ch, z, k);
#pragma unroll
  for (int d = 0; d < R::D; ++d) { acc[d] += (T)2 * k[d]; z[d] = y[d] + h * k[d]; }
  rhs(c1, z, k);
  const T h6 = h / (T)6;
#pragma unroll
  for (int d = 0; d < R::D; ++d) add_update(y[d], h6 * (acc[d] + k[d]), comp[d]);
}

}  // namespace nvpit
