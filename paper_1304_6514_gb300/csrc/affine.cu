// Exact affine slice maps for linear systems (eqs. lineardiscrete and
// linearreconstruct): per slice j, one solve from 0 with the forcing on gives
// b_j and d homogeneous solves from e_c give the columns of A_j.
//
// Heat equation kernels: one warp (or a group of lanes) integrates one basis
// column.  Lane l holds rows l*R .. l*R+R-1 of the d-vector (or of a window of
// it) in registers; the stencil reaches the neighbouring lanes by shuffles.
// No shared or global memory is touched until the column is written.
//
// Time-invariant homogeneous columns take the RK4 step as one nine-point
// stencil (or in Horner form, y <- y + hL(y + hL/2(y + hL/3(y + hL/4 y))):
// for y' = L y with constant L both are the classical RK4 step exactly, the
// degree-4 Taylor polynomial of hL applied to y), by default only over the
// rows each column's steps can reach.  The float64 forcing column takes the
// nine-point form plus the forcing's contribution along the sine eigenvector;
// the float32 one and every column of a time-dependent operator take the four
// RK4 stages literally.
#include <cuda_bf16.h>
#include <math.h>

#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "heat.cuh"

namespace nvpit {

// Store a lane-blocked column (lane l holds rows l*R .. l*R+R-1) so that each
// warp store covers 32 consecutive rows: the warp stages the column in its own
// shared-memory slot (lane stride R+1 to spread the banks) and reads row
// k*32+l back in lane l. Every store instruction then writes whole 32-byte
// sectors, where the blocked order left each sector partly written and the L2
// had to fill it from DRAM. buf holds 32*(R+1) values for this warp.
template <int R, bool TF32OUT, typename T>
__device__ __forceinline__ void store_column(const T* y, T* buf, T* col, int lane, int n) {
  __syncwarp();
#pragma unroll
  for (int i = 0; i < R; ++i) buf[lane * (R + 1) + i] = y[i];
  __syncwarp();
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int r = k * 32 + lane;
    const int src = r / R;
    const T v = buf[src * (R + 1) + (r - src * R)];
    if (r < n) {
      if constexpr (TF32OUT) col[r] = round_tf32(v);
      else col[r] = v;
    }
  }
}

// Per-warp staging slots of store_column for a CTA of at most 256 threads.
template <int R, typename T>
__device__ __forceinline__ T* column_stage() {
  __shared__ T stage[8 * 32 * (R + 1)];
  return stage + (threadIdx.x >> 5) * 32 * (R + 1);
}

// Homogeneous columns of a time-invariant operator (c = 1..d): Horner-form
// RK4 only, so a thread holds just y and v (2R values) and many warps fit.
template <typename T, int R, bool TF32OUT>
__global__ void __launch_bounds__(256, (sizeof(T) * R <= 64) ? 4 : 1) heat_horner_kernel(HeatArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int n = a.n, cols = n + 1;
  const int64_t total = (int64_t)a.S * n;
  const double dx = 1.0 / (double)(n + 1);
  const T cdx = (T)(a.kappa / (dx * dx));
  const T h = (T)a.h;
  T* out = reinterpret_cast<T*>(a.out);
  for (int64_t w = warp0; w < total; w += nwarps) {
    const int j = (int)(w / n);
    const int c = 1 + (int)(w - (int64_t)j * n);
    T y[R], v[R];
#pragma unroll
    for (int i = 0; i < R; ++i) y[i] = (lane * R + i == c - 1) ? (T)1 : (T)0;
    for (int64_t i = 0; i < a.m; ++i) heat_horner_step<R>(y, v, cdx, h, lane, n);
    store_column<R, TF32OUT>(y, column_stage<R, T>(), out + ((int64_t)j * cols + c) * n, lane, n);
  }
}

// Homogeneous columns of a time-invariant operator, the RK4 step as one
// nine-point stencil.  For y' = Ly with L = cdx [1,-2,1] the classical RK4
// step is y <- P(hL) y with P(z) = 1 + z + z^2/2 + z^3/6 + z^4/24, and the
// powers of the [1,-2,1] stencil ([1,-4,6,-4,1], ...) make P(hL) a symmetric
// stencil of half-width 4 with weights c_0..c_4, polynomials in a = h cdx.
// The Dirichlet ends hold exactly under odd reflection about the zero
// boundary value (y_{-1-k} = -y_{-1+k}), which L and so every power of L
// preserves.  Nine multiply-adds per point and step (four sums, one multiply,
// four FMAs) against twelve for the Horner stages.  Lane l holds rows
// l*R .. l*R+R-1; R >= 4 so the four-row halo comes from one neighbour lane,
// and n is a multiple of R so the right end falls on a lane boundary.
template <typename T, int R, bool TF32OUT>
__global__ void __launch_bounds__(256, (sizeof(T) * R <= 64 && R <= 8) ? 4 : 1) heat_poly9_kernel(HeatArgs a) {
  static_assert(R >= 4, "the halo must fit in one neighbour lane");
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int n = a.n, cols = n + 1;
  const int last = n / R - 1;                       // lane holding row n-1
  const int64_t total = (int64_t)a.S * n;
  const T c0 = poly9_weight<T>(a, 0), c1 = poly9_weight<T>(a, 1), c2 = poly9_weight<T>(a, 2),
          c3 = poly9_weight<T>(a, 3), c4 = poly9_weight<T>(a, 4);
  T* out = reinterpret_cast<T*>(a.out);
  for (int64_t w = warp0; w < total; w += nwarps) {
    const int j = (int)(w / n);
    const int c = 1 + (int)(w - (int64_t)j * n);
    T y[R];
#pragma unroll
    for (int i = 0; i < R; ++i) y[i] = (lane * R + i == c - 1) ? (T)1 : (T)0;
    for (int64_t step = 0; step < a.m; ++step) {
      T e[R + 8];                                   // rows lane*R-4 .. lane*R+R+3
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        e[q] = __shfl_up_sync(0xffffffffu, y[R - 4 + q], 1);
        e[R + 4 + q] = __shfl_down_sync(0xffffffffu, y[q], 1);
      }
      if (lane == 0) {                              // rows -4..-1 = -y2, -y1, -y0, 0
        e[0] = -y[2];
        e[1] = -y[1];
        e[2] = -y[0];
        e[3] = (T)0;
      }
      if (lane == last) {                           // rows n..n+3 = 0, -y_{n-1}, -y_{n-2}, -y_{n-3}
        e[R + 4] = (T)0;
        e[R + 5] = -y[R - 1];
        e[R + 6] = -y[R - 2];
        e[R + 7] = -y[R - 3];
      }
#pragma unroll
      for (int i = 0; i < R; ++i) e[i + 4] = y[i];
#pragma unroll
      for (int i = 0; i < R; ++i) {
        T acc = c4 * (e[i] + e[i + 8]);
        acc = fma(c3, e[i + 1] + e[i + 7], acc);
        acc = fma(c2, e[i + 2] + e[i + 6], acc);
        acc = fma(c1, e[i + 3] + e[i + 5], acc);
        y[i] = fma(c0, e[i + 4], acc);
      }
      if (lane > last) {                            // lanes past the last row stay zero
#pragma unroll
        for (int i = 0; i < R; ++i) y[i] = (T)0;
      }
    }
    store_column<R, TF32OUT>(y, column_stage<R, T>(), out + ((int64_t)j * cols + c) * n, lane, n);
  }
}

// One nine-point step of a window of G*R rows held by G lanes (R rows each):
// the halo comes from the neighbouring lanes of the group, and at the
// window's ends it is the odd reflection (lo_end / hi_end: the end of the
// window is the end of the domain) or zero (the window is cut inside the
// domain).  Same expression, operand for operand, as heat_poly9_kernel.
template <typename T, int G, int R>
__device__ __forceinline__ void window_step(T (&y)[R], int gl, bool lo_end, bool hi_end, T c0, T c1, T c2,
                                            T c3, T c4) {
  T e[R + 8];                                       // rows w0+gl*R-4 .. w0+gl*R+R+3
  if constexpr (G > 1) {                            // one lane per window: both ends are set below
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      e[k] = __shfl_up_sync(0xffffffffu, y[R - 4 + k], 1, G);
      e[R + 4 + k] = __shfl_down_sync(0xffffffffu, y[k], 1, G);
    }
  }
  if (gl == 0) {                                    // rows w0-4..w0-1
    e[0] = lo_end ? -y[2] : (T)0;
    e[1] = lo_end ? -y[1] : (T)0;
    e[2] = lo_end ? -y[0] : (T)0;
    e[3] = (T)0;
  }
  if (gl == G - 1) {                                // rows w0+W .. w0+W+3
    e[R + 4] = (T)0;
    e[R + 5] = hi_end ? -y[R - 1] : (T)0;
    e[R + 6] = hi_end ? -y[R - 2] : (T)0;
    e[R + 7] = hi_end ? -y[R - 3] : (T)0;
  }
#pragma unroll
  for (int i = 0; i < R; ++i) e[i + 4] = y[i];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    T acc = c4 * (e[i] + e[i + 8]);
    acc = fma(c3, e[i + 1] + e[i + 7], acc);
    acc = fma(c2, e[i + 2] + e[i + 6], acc);
    acc = fma(c1, e[i + 3] + e[i + 5], acc);
    y[i] = fma(c0, e[i + 4], acc);
  }
}

// Window origin of column c (1-based) for a window of W rows and reach 4m.
__device__ __forceinline__ int window_origin(int c, int reach, int n, int W) {
  return min(max(c - 1 - reach, 0), n - W);
}

// Window staging in shared memory: a column's W = G*R rows contiguous, in
// slots of G*(R+1) values per column (the same 32*(R+1) values per warp as a
// lane-blocked column), so that a row's offset in its window is its index in
// the slot.  Lane l = q*G + gl writes its rows gl*R .. gl*R+R-1 of column q at
// l*(R+1) - gl.
template <int G, int R>
__device__ __forceinline__ int window_slot(int lane) {
  return lane * (R + 1) - lane % G;
}

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  static constexpr int V = 4;
  __device__ static void store(float* p, const float* v) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct Vec16<double> {
  static constexpr int V = 2;
  __device__ static void store(double* p, const double* v) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
};

// Write the windows of 32/G columns (w*CPW .. w*CPW+CPW-1 of the flattened
// (slice, column) order), staged by window_slot, as full columns of n rows
// with zeros outside the windows: 16-byte stores of consecutive rows by
// consecutive lanes where the columns are 16-byte aligned (n a multiple of 4
// floats or 2 doubles), else one row per lane and store.
template <typename T, int G, int R, bool TF32OUT>
__device__ __forceinline__ void store_windows(const T* buf, T* out, int64_t first, int64_t total, int n,
                                              int reach, int lane) {
  constexpr int W = G * R, CPW = 32 / G, SW = G * (R + 1), V = Vec16<T>::V;
  const int cols = n + 1;
#pragma unroll 1
  for (int g = 0; g < CPW; ++g) {
    const int64_t id = first + g;
    if (id >= total) break;                         // warp-uniform
    const int jg = (int)(id / n);
    const int cg = 1 + (int)(id - (int64_t)jg * n);
    const int v0 = window_origin(cg, reach, n, W);
    T* col = out + ((int64_t)jg * cols + cg) * n;
    const T* win = buf + g * SW;
    if (n % V == 0) {
      for (int r0 = lane * V; r0 < n; r0 += 32 * V) {
        T v[V];
#pragma unroll
        for (int q = 0; q < V; ++q) {
          const int o = r0 + q - v0;
          v[q] = (unsigned)o < (unsigned)W ? win[o] : (T)0;
          if constexpr (TF32OUT) v[q] = round_tf32(v[q]);
        }
        Vec16<T>::store(col + r0, v);
      }
    } else {
      for (int r = lane; r < n; r += 32) {
        const int o = r - v0;
        const T v = (unsigned)o < (unsigned)W ? win[o] : (T)0;
        if constexpr (TF32OUT) col[r] = round_tf32(v);
        else col[r] = v;
      }
    }
  }
}

// The homogeneous columns again, each integrated over its domain of
// dependence only.  A nine-point step carries information four rows, so the
// column started from e_c is exactly zero outside rows c-1-4k .. c-1+4k after
// k steps.  A group of G lanes (R rows each, 32/G columns per warp) holds a
// window of W = G*R >= 8m+1 rows placed so that those rows of the last step
// lie inside it: w0 = clamp(c-1-4m, 0, n-W).  Where the window is cut inside
// the domain its halo reads zeros, the exact values there at every step that
// reads them (the column's reach before the last step is 4(m-1), the cut is
// 4m+1 rows away); where it meets an end of the domain the odd reflection
// applies as above.  Each entry in the window is the same floating-point
// expression as in heat_poly9_kernel (the inputs differ at most in the sign of
// a zero), so the maps agree bit for bit up to the sign of zero entries; the
// rows outside the window are written as zeros.  The work per column falls
// from n to W rows.
template <typename T, int G, int R, bool TF32OUT>
__global__ void __launch_bounds__(256, (sizeof(T) * R <= 64) ? 4 : 2) heat_window_kernel(HeatArgs a) {
  static_assert(R >= 4 && G >= 2 && 32 % G == 0, "R >= 4 rows per lane, G lanes dividing the warp");
  constexpr int W = G * R, CPW = 32 / G;
  const int lane = threadIdx.x & 31, gl = lane % G, q = lane / G;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int n = a.n;
  const int reach = (int)(4 * a.m);                 // launcher: 8m+1 <= W <= n
  const int64_t total = (int64_t)a.S * n;
  const T c0 = poly9_weight<T>(a, 0), c1 = poly9_weight<T>(a, 1), c2 = poly9_weight<T>(a, 2),
          c3 = poly9_weight<T>(a, 3), c4 = poly9_weight<T>(a, 4);
  T* out = reinterpret_cast<T*>(a.out);
  T* buf = column_stage<R, T>();
  for (int64_t w = warp0; w * CPW < total; w += nwarps) {
    const int64_t idx = w * CPW + q;                // this group's column; past the end: a dummy
    const int j = idx < total ? (int)(idx / n) : 0;
    const int c = idx < total ? 1 + (int)(idx - (int64_t)j * n) : 1;
    const int w0 = window_origin(c, reach, n, W);
    const bool lo_end = w0 == 0, hi_end = w0 + W == n;
    T y[R];
#pragma unroll
    for (int i = 0; i < R; ++i) y[i] = (w0 + gl * R + i == c - 1) ? (T)1 : (T)0;
    for (int64_t step = 0; step < a.m; ++step) window_step<T, G, R>(y, gl, lo_end, hi_end, c0, c1, c2, c3, c4);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < R; ++i) buf[window_slot<G, R>(lane) + i] = y[i];
    __syncwarp();
    store_windows<T, G, R, TF32OUT>(buf, out, w * CPW, total, n, reach, lane);
    __syncwarp();
  }
}

// Two windows per column: the column's reach grows by four rows a step, so
// the first m1 steps (8*m1+1 <= GA*R rows) run on windows of GA lanes, 32/GA
// columns per warp, and the remaining m - m1 steps on windows of GB = 2*GA
// lanes (8m+1 <= GB*R rows), the warp's columns in two rounds of 32/GB.  Between
// the phases each column's narrow window is staged in shared memory and read
// back into the wide one by row (the narrow window lies inside the wide one:
// both are clamped to the domain around the same row).  The steps are the
// same expressions as in heat_window_kernel, so the maps are the same.
template <typename T, int GA, int R, bool TF32OUT>
__global__ void __launch_bounds__(256, (sizeof(T) * R <= 64) ? 4 : 2) heat_window2_kernel(HeatArgs a, int m1) {
  constexpr int GB = 2 * GA, WA = GA * R, WB = GB * R, CPW = 32 / GA, CPB = 32 / GB;
  static_assert(R >= 4 && GA >= 2 && 32 % GB == 0, "R >= 4 rows per lane, 2*GA lanes dividing the warp");
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int n = a.n;
  const int reach1 = 4 * m1, reach = (int)(4 * a.m);   // launcher: 8*m1+1 <= WA, 8m+1 <= WB <= n
  const int64_t total = (int64_t)a.S * n;
  const T c0 = poly9_weight<T>(a, 0), c1 = poly9_weight<T>(a, 1), c2 = poly9_weight<T>(a, 2),
          c3 = poly9_weight<T>(a, 3), c4 = poly9_weight<T>(a, 4);
  T* out = reinterpret_cast<T*>(a.out);
  __shared__ T narrow_all[8 * 32 * (R + 1)];         // the narrow windows, lane*(R+1)+i
  T* narrow = narrow_all + (threadIdx.x >> 5) * 32 * (R + 1);
  T* buf = column_stage<R, T>();
  for (int64_t w = warp0; w * CPW < total; w += nwarps) {
    {                                               // phase 1: CPW columns, GA lanes each
      const int gl = lane % GA;
      const int64_t idx = w * CPW + lane / GA;
      const int j = idx < total ? (int)(idx / n) : 0;
      const int c = idx < total ? 1 + (int)(idx - (int64_t)j * n) : 1;
      const int w0 = window_origin(c, reach1, n, WA);
      T y[R];
#pragma unroll
      for (int i = 0; i < R; ++i) y[i] = (w0 + gl * R + i == c - 1) ? (T)1 : (T)0;
      for (int step = 0; step < m1; ++step)
        window_step<T, GA, R>(y, gl, w0 == 0, w0 + WA == n, c0, c1, c2, c3, c4);
      __syncwarp();
#pragma unroll
      for (int i = 0; i < R; ++i) narrow[window_slot<GA, R>(lane) + i] = y[i];
      __syncwarp();
    }
#pragma unroll 1
    for (int round = 0; round < CPW / CPB; ++round) { // phase 2: CPB columns at a time, GB lanes each
      const int gl = lane % GB, qa = round * CPB + lane / GB;   // the column's slot in phase 1
      const int64_t first = w * CPW + round * CPB;
      if (first >= total) break;                    // warp-uniform
      const int64_t idx = w * CPW + qa;
      const int j = idx < total ? (int)(idx / n) : 0;
      const int c = idx < total ? 1 + (int)(idx - (int64_t)j * n) : 1;
      const int wa = window_origin(c, reach1, n, WA), wb = window_origin(c, reach, n, WB);
      T y[R];
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const int o = wb + gl * R + i - wa;         // row's offset in the narrow window
        T v = (T)0;
        if (o >= 0 && o < WA) {
          v = narrow[qa * GA * (R + 1) + o];
        }
        y[i] = v;
      }
      for (int64_t step = m1; step < a.m; ++step)
        window_step<T, GB, R>(y, gl, wb == 0, wb + WB == n, c0, c1, c2, c3, c4);
      __syncwarp();
#pragma unroll
      for (int i = 0; i < R; ++i) buf[window_slot<GB, R>(lane) + i] = y[i];
      __syncwarp();
      store_windows<T, GB, R, TF32OUT>(buf, out, first, total, n, reach, lane);
      __syncwarp();
    }
  }
}

// Fill a wide window (origin wide0, G lanes of R rows, this lane's rows
// gl*R ..) from a narrow window of slot `slot` staged by GN lanes per column
// by window_slot (origin wn, WN rows); rows outside the narrow window are 0.
template <typename T, int GN, int R>
__device__ __forceinline__ void widen_window(T (&y)[R], const T* narrow, int slot, int wn, int WN, int wide0,
                                             int gl) {
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int o = wide0 + gl * R + i - wn;
    T v = (T)0;
    if (o >= 0 && o < WN) {
      v = narrow[slot * GN * (R + 1) + o];
    }
    y[i] = v;
  }
}

// Three windows per column, doubling the lanes each time: the first
// m1 = (G1*R-1)/8 steps on G1 lanes (32/G1 columns per warp), up to step
// m2 = (2*G1*R-1)/8 on 2*G1 lanes, the rest on 4*G1 lanes (8m+1 <= 4*G1*R).
// The narrow windows are staged in shared memory and widened by row as in
// heat_window2_kernel; with the column staging that is three buffers of
// 32*(R+1) values per warp, so the CTA has at most four warps.  The steps are
// the same expressions as in heat_window_kernel, so the maps are the same.
template <typename T, int G1, int R, bool TF32OUT>
__global__ void __launch_bounds__(128) heat_window3_kernel(HeatArgs a, int m1, int m2) {
  constexpr int G2 = 2 * G1, G3 = 4 * G1, W1 = G1 * R, W2 = G2 * R, W3 = G3 * R;
  constexpr int C1 = 32 / G1, C2 = 32 / G2, C3 = 32 / G3;
  static_assert(R >= 4 && G1 >= 1 && 32 % G3 == 0, "R >= 4 rows per lane, 4*G1 lanes dividing the warp");
  __shared__ T slots[4][3][32 * (R + 1)];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* b1 = slots[warp][0];
  T* b2 = slots[warp][1];
  T* stage = slots[warp][2];
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int n = a.n;
  const int reach1 = 4 * m1, reach2 = 4 * m2, reach = (int)(4 * a.m);   // launcher: 8m+1 <= W3 <= n
  const int64_t total = (int64_t)a.S * n;
  const T c0 = poly9_weight<T>(a, 0), c1 = poly9_weight<T>(a, 1), c2 = poly9_weight<T>(a, 2),
          c3 = poly9_weight<T>(a, 3), c4 = poly9_weight<T>(a, 4);
  T* out = reinterpret_cast<T*>(a.out);
  auto column = [&](int64_t idx) {              // (slice, column) of flattened index idx
    const int j = idx < total ? (int)(idx / n) : 0;
    return idx < total ? 1 + (int)(idx - (int64_t)j * n) : 1;
  };
  for (int64_t w = warp0; w * C1 < total; w += nwarps) {
    {                                           // phase 1: C1 columns, G1 lanes each
      const int gl = lane % G1;
      const int c = column(w * C1 + lane / G1);
      const int w0 = window_origin(c, reach1, n, W1);
      T y[R];
#pragma unroll
      for (int i = 0; i < R; ++i) y[i] = (w0 + gl * R + i == c - 1) ? (T)1 : (T)0;
      for (int step = 0; step < m1; ++step)
        window_step<T, G1, R>(y, gl, w0 == 0, w0 + W1 == n, c0, c1, c2, c3, c4);
      __syncwarp();
#pragma unroll
      for (int i = 0; i < R; ++i) b1[window_slot<G1, R>(lane) + i] = y[i];
      __syncwarp();
    }
#pragma unroll 1
    for (int r2 = 0; r2 < C1 / C2; ++r2) {      // phase 2: C2 columns at a time, G2 lanes each
      const int64_t first2 = w * C1 + r2 * C2;
      if (first2 >= total) break;               // warp-uniform
      {
        const int gl = lane % G2, q = r2 * C2 + lane / G2;   // slot in phase 1
        const int c = column(w * C1 + q);
        const int wa = window_origin(c, reach1, n, W1), wb = window_origin(c, reach2, n, W2);
        T y[R];
        widen_window<T, G1, R>(y, b1, q, wa, W1, wb, gl);
        for (int step = m1; step < m2; ++step)
          window_step<T, G2, R>(y, gl, wb == 0, wb + W2 == n, c0, c1, c2, c3, c4);
        __syncwarp();
#pragma unroll
        for (int i = 0; i < R; ++i) b2[window_slot<G2, R>(lane) + i] = y[i];
        __syncwarp();
      }
#pragma unroll 1
      for (int r3 = 0; r3 < C2 / C3; ++r3) {    // phase 3: C3 columns at a time, G3 lanes each
        const int64_t first3 = first2 + r3 * C3;
        if (first3 >= total) break;             // warp-uniform
        const int gl = lane % G3, q = r3 * C3 + lane / G3;   // slot in phase 2
        const int c = column(first2 + q);
        const int wb = window_origin(c, reach2, n, W2), wc = window_origin(c, reach, n, W3);
        T y[R];
        widen_window<T, G2, R>(y, b2, q, wb, W2, wc, gl);
        for (int64_t step = m2; step < a.m; ++step)
          window_step<T, G3, R>(y, gl, wc == 0, wc + W3 == n, c0, c1, c2, c3, c4);
        __syncwarp();
#pragma unroll
        for (int i = 0; i < R; ++i) stage[window_slot<G3, R>(lane) + i] = y[i];
        __syncwarp();
        store_windows<T, G3, R, TF32OUT>(stage, out, first3, total, n, reach, lane);
        __syncwarp();
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Packed float32 pairs.  The homogeneous heat columns are the same arithmetic
// in every slice (the operator does not depend on time), so the float32 build
// can carry column c of slices 2p and 2p+1 in the low and high halves of one
// 64-bit register and issue each stencil operation once for both: the
// Blackwell packed add / mul / fma on .f32x2 (round to nearest, no flush to
// zero), each half the IEEE operation of the scalar code, so every entry is
// the scalar kernel's bit for bit.  Half the arithmetic instructions per
// row-step; the shuffles and window-edge selects stay one per value.
typedef unsigned long long f32x2_t;

__device__ __forceinline__ f32x2_t f2_add(f32x2_t a, f32x2_t b) {
  f32x2_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2_t f2_mul(f32x2_t a, f32x2_t b) {
  f32x2_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2_t f2_fma(f32x2_t a, f32x2_t b, f32x2_t c) {   // a*b + c
  f32x2_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f32x2_t f2_splat(float x) {
  f32x2_t d;
  asm("mov.b64 %0, {%1, %1};" : "=l"(d) : "f"(x));
  return d;
}
__device__ __forceinline__ void f2_unpack(f32x2_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2_t f2_neg(f32x2_t a) { return a ^ 0x8000000080000000ull; }   // sign flips

// window_step on packed pairs: the same halo rules and the same expression.
template <int G, int R>
__device__ __forceinline__ void window_step_x2(f32x2_t (&y)[R], int gl, bool lo_end, bool hi_end, f32x2_t c0,
                                               f32x2_t c1, f32x2_t c2, f32x2_t c3, f32x2_t c4) {
  f32x2_t e[R + 8];
  if constexpr (G > 1) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      e[k] = __shfl_up_sync(0xffffffffu, y[R - 4 + k], 1, G);
      e[R + 4 + k] = __shfl_down_sync(0xffffffffu, y[k], 1, G);
    }
  }
  if (gl == 0) {
    e[0] = lo_end ? f2_neg(y[2]) : 0ull;
    e[1] = lo_end ? f2_neg(y[1]) : 0ull;
    e[2] = lo_end ? f2_neg(y[0]) : 0ull;
    e[3] = 0ull;
  }
  if (gl == G - 1) {
    e[R + 4] = 0ull;
    e[R + 5] = hi_end ? f2_neg(y[R - 1]) : 0ull;
    e[R + 6] = hi_end ? f2_neg(y[R - 2]) : 0ull;
    e[R + 7] = hi_end ? f2_neg(y[R - 3]) : 0ull;
  }
#pragma unroll
  for (int i = 0; i < R; ++i) e[i + 4] = y[i];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    f32x2_t acc = f2_mul(c4, f2_add(e[i], e[i + 8]));
    acc = f2_fma(c3, f2_add(e[i + 1], e[i + 7]), acc);
    acc = f2_fma(c2, f2_add(e[i + 2], e[i + 6]), acc);
    acc = f2_fma(c1, f2_add(e[i + 3], e[i + 5]), acc);
    y[i] = f2_fma(c0, e[i + 4], acc);
  }
}

// store_windows for packed pairs: pair index id = p*n + c-1 holds column c of
// slices 2p (low halves) and 2p+1 (high halves; absent when 2p+1 = S).
template <int G, int R, bool TF32OUT>
__device__ __forceinline__ void store_windows_x2(const f32x2_t* buf, float* out, int64_t first, int64_t total,
                                                 int n, int reach, int lane, int S) {
  constexpr int W = G * R, CPW = 32 / G, SW = G * (R + 1);
  const int cols = n + 1;
#pragma unroll 1
  for (int g = 0; g < CPW; ++g) {
    const int64_t id = first + g;
    if (id >= total) break;                         // warp-uniform
    const int jp = (int)(id / n);
    const int cg = 1 + (int)(id - (int64_t)jp * n);
    const int v0 = window_origin(cg, reach, n, W);
    const bool has_hi = 2 * jp + 1 < S;
    float* colA = out + ((int64_t)(2 * jp) * cols + cg) * n;
    float* colB = colA + (int64_t)cols * n;
    const f32x2_t* win = buf + g * SW;
    if (n % 4 == 0) {
      for (int r0 = lane * 4; r0 < n; r0 += 128) {
        float va[4], vb[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int o = r0 + q - v0;
          f2_unpack((unsigned)o < (unsigned)W ? win[o] : 0ull, va[q], vb[q]);
          if constexpr (TF32OUT) {
            va[q] = round_tf32(va[q]);
            vb[q] = round_tf32(vb[q]);
          }
        }
        *reinterpret_cast<float4*>(colA + r0) = make_float4(va[0], va[1], va[2], va[3]);
        if (has_hi) *reinterpret_cast<float4*>(colB + r0) = make_float4(vb[0], vb[1], vb[2], vb[3]);
      }
    } else {
      for (int r = lane; r < n; r += 32) {
        const int o = r - v0;
        float va, vb;
        f2_unpack((unsigned)o < (unsigned)W ? win[o] : 0ull, va, vb);
        if constexpr (TF32OUT) {
          va = round_tf32(va);
          vb = round_tf32(vb);
        }
        colA[r] = va;
        if (has_hi) colB[r] = vb;
      }
    }
  }
}

// heat_window3_kernel in float32 on packed slice pairs: the same three
// windows, phases and staging (shared memory of 8-byte pairs, dynamic: four
// warps x three buffers of 32*(R+1) pairs), over ceil(S/2)*n pair columns.
template <int G1, int R, bool TF32OUT>
__global__ void __launch_bounds__(128) heat_window3_x2_kernel(HeatArgs a, int m1, int m2) {
  constexpr int G2 = 2 * G1, G3 = 4 * G1, W1 = G1 * R, W2 = G2 * R, W3 = G3 * R;
  constexpr int C1 = 32 / G1, C2 = 32 / G2, C3 = 32 / G3;
  static_assert(R >= 4 && G1 >= 1 && 32 % G3 == 0, "R >= 4 rows per lane, 4*G1 lanes dividing the warp");
  extern __shared__ __align__(16) unsigned char x2_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  f32x2_t* b1 = reinterpret_cast<f32x2_t*>(x2_smem) + warp * 3 * 32 * (R + 1);
  f32x2_t* b2 = b1 + 32 * (R + 1);
  f32x2_t* stage = b2 + 32 * (R + 1);
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int n = a.n;
  const int reach1 = 4 * m1, reach2 = 4 * m2, reach = (int)(4 * a.m);   // launcher: 8m+1 <= W3 <= n
  const int64_t total = (int64_t)((a.S + 1) / 2) * n;                   // pair columns
  const f32x2_t c0 = f2_splat(poly9_weight<float>(a, 0)), c1 = f2_splat(poly9_weight<float>(a, 1)),
                c2 = f2_splat(poly9_weight<float>(a, 2)), c3 = f2_splat(poly9_weight<float>(a, 3)),
                c4 = f2_splat(poly9_weight<float>(a, 4));
  const f32x2_t one = f2_splat(1.0f);
  float* out = reinterpret_cast<float*>(a.out);
  auto column = [&](int64_t idx) {              // column of pair index idx
    const int jp = idx < total ? (int)(idx / n) : 0;
    return idx < total ? 1 + (int)(idx - (int64_t)jp * n) : 1;
  };
  for (int64_t w = warp0; w * C1 < total; w += nwarps) {
    {                                           // phase 1: C1 pair columns, G1 lanes each
      const int gl = lane % G1;
      const int c = column(w * C1 + lane / G1);
      const int w0 = window_origin(c, reach1, n, W1);
      f32x2_t y[R];
#pragma unroll
      for (int i = 0; i < R; ++i) y[i] = (w0 + gl * R + i == c - 1) ? one : 0ull;
      for (int step = 0; step < m1; ++step)
        window_step_x2<G1, R>(y, gl, w0 == 0, w0 + W1 == n, c0, c1, c2, c3, c4);
      __syncwarp();
#pragma unroll
      for (int i = 0; i < R; ++i) b1[window_slot<G1, R>(lane) + i] = y[i];
      __syncwarp();
    }
#pragma unroll 1
    for (int r2 = 0; r2 < C1 / C2; ++r2) {      // phase 2
      const int64_t first2 = w * C1 + r2 * C2;
      if (first2 >= total) break;               // warp-uniform
      {
        const int gl = lane % G2, q = r2 * C2 + lane / G2;
        const int c = column(w * C1 + q);
        const int wa = window_origin(c, reach1, n, W1), wb = window_origin(c, reach2, n, W2);
        f32x2_t y[R];
        widen_window<f32x2_t, G1, R>(y, b1, q, wa, W1, wb, gl);
        for (int step = m1; step < m2; ++step)
          window_step_x2<G2, R>(y, gl, wb == 0, wb + W2 == n, c0, c1, c2, c3, c4);
        __syncwarp();
#pragma unroll
        for (int i = 0; i < R; ++i) b2[window_slot<G2, R>(lane) + i] = y[i];
        __syncwarp();
      }
#pragma unroll 1
      for (int r3 = 0; r3 < C2 / C3; ++r3) {    // phase 3
        const int64_t first3 = first2 + r3 * C3;
        if (first3 >= total) break;             // warp-uniform
        const int gl = lane % G3, q = r3 * C3 + lane / G3;
        const int c = column(first2 + q);
        const int wb = window_origin(c, reach2, n, W2), wc = window_origin(c, reach, n, W3);
        f32x2_t y[R];
        widen_window<f32x2_t, G2, R>(y, b2, q, wb, W2, wc, gl);
        for (int64_t step = m2; step < a.m; ++step)
          window_step_x2<G3, R>(y, gl, wc == 0, wc + W3 == n, c0, c1, c2, c3, c4);
        __syncwarp();
#pragma unroll
        for (int i = 0; i < R; ++i) stage[window_slot<G3, R>(lane) + i] = y[i];
        __syncwarp();
        store_windows_x2<G3, R, TF32OUT>(stage, out, first3, total, n, reach, lane, a.S);
        __syncwarp();
      }
    }
  }
}

// Columns that take the four RK4 stages literally: the forcing column c = 0
// of every slice, and for a time-dependent operator every column.
template <typename T, int R>
__global__ void __launch_bounds__(256) heat_literal_kernel(HeatArgs a, int all_columns) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int n = a.n, cols = n + 1;
  const int per_slice = all_columns ? cols : 1;
  const int64_t total = (int64_t)a.S * per_slice;
  const double dx = 1.0 / (double)(n + 1);
  const T cdx = (T)(a.kappa / (dx * dx));
  T* out = reinterpret_cast<T*>(a.out);
  __shared__ double sxt[32 * R];
  forcing_table(sxt, min(n, 32 * R));
  for (int64_t w = warp0; w < total; w += nwarps) {
    const int j = (int)(w / per_slice);
    const int c = (int)(w - (int64_t)j * per_slice);
    const double Tj = __dadd_rn(a.t0, __dmul_rn((double)j, a.H));
    const bool forced = (c == 0);
    T y[R], z[R], acc[R], sx[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int r = lane * R + i;
      y[i] = (c >= 1 && r == c - 1) ? (T)1 : (T)0;
      sx[i] = (T)0;
    }
    if (forced) {
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const int r = lane * R + i;
        if (r < n) sx[i] = (T)sxt[r];
      }
    }
    HalfStepCoefs hc{};
    for (int64_t i = 0; i < a.m; ++i) {
      const int64_t i0 = i - (i % 15);
      if (i == i0) hc = half_step_coefs(a, Tj, i0, lane);
      heat_rk4_step<R>(y, z, acc, a.h, step_coefs<T>(hc, i, i0, cdx), sx, forced, lane, n);
    }
    store_column<R, false>(y, column_stage<R, T>(), out + ((int64_t)j * cols + c) * n, lane, n);
  }
}

// Serial fine solve of the heat equation: one warp, S*m literal RK4 steps.
template <int R>
__global__ void heat_serial_kernel(HeatArgs a, const double* y0, double* yT) {
  const int lane = threadIdx.x & 31;
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  const int n = a.n;
  const double dx = 1.0 / (double)(n + 1);
  const double cdx = a.kappa / (dx * dx);
  double y[R], z[R], acc[R], sx[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int r = lane * R + i;
    y[i] = r < n ? y0[r] : 0.0;
    sx[i] = r < n ? sin(M_PI * ((double)(r + 1) / (double)(n + 1))) : 0.0;
  }
  for (int j = 0; j < a.S; ++j) {
    const double Tj = __dadd_rn(a.t0, __dmul_rn((double)j, a.H));
    HalfStepCoefs hc{};
    for (int64_t i = 0; i < a.m; ++i) {
      const int64_t i0 = i - (i % 15);
      if (i == i0) hc = half_step_coefs(a, Tj, i0, lane);
      heat_rk4_step<R>(y, z, acc, a.h, step_coefs<double>(hc, i, i0, cdx), sx, true, lane, n);
    }
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int r = lane * R + i;
    if (r < n) yT[r] = y[i];
  }
}

// Defects of approximate boundary states for the float64 correction pass:
// d_j = g^j(lt_j) - lt_{j+1}, one warp per slice j integrating the full
// inhomogeneous right-hand side over slice j from lt_j with literal RK4
// stages in float64 (lt has S+1 rows of n, d has S rows).
// The forcing column b_j of float64 maps (time-invariant operator): the
// slice's forced solve from 0, in the nine-point form of the defects (the
// forcing lies along the sine eigenvector of the operator, so each RK4 step
// adds phi times that vector; the literal stages where the form does not
// apply), one warp per slice, stored like the homogeneous columns.
template <int R>
__global__ void __launch_bounds__(256) heat_forcing_kernel(HeatArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int n = a.n;
  double* out = reinterpret_cast<double*>(a.out);
  __shared__ double sxt[32 * R];
  forcing_table(sxt, min(n, 32 * R));
  for (int64_t j = warp0; j < a.S; j += nwarps) {
    double y[R];
#pragma unroll
    for (int i = 0; i < R; ++i) y[i] = 0.0;
    heat_forced_solve<R>(a, y, j, lane, sxt);
    store_column<R, false>(y, column_stage<R, double>(), out + j * (int64_t)(n + 1) * n, lane, n);
  }
}

template <int R>
__global__ void __launch_bounds__(256) heat_defect_kernel(HeatArgs a, const double* lt, double* d) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  __shared__ double sxt[32 * R];
  forcing_table(sxt, min(a.n, 32 * R));
  for (int64_t j = warp0; j < a.S; j += nwarps) heat_defect_slice<R>(a, lt, d, j, lane, sxt);
}

}  // namespace nvpit

using namespace nvpit;

static int rows_per_lane(int n) {
  const int r = (n + 31) / 32;
  if (r <= 1) return 1;
  if (r <= 2) return 2;
  if (r <= 4) return 4;
  if (r <= 8) return 8;
  if (r <= 16) return 16;
  return 0;
}

HeatArgs heat_args(const nv_maps* M) {
  HeatArgs a{};
  a.out = M->data;
  a.n = M->dim;
  a.S = M->S;
  a.m = M->m;
  a.t0 = M->t0;
  a.H = M->H;
  a.h = M->h;
  a.varcoef = M->rhs_kind == NV_RHS_HEAT1D_VARCOEF;
  a.kappa = (!a.varcoef && M->nparams > 0) ? M->params[0] : 1.0;
  a.amp = (!a.varcoef && M->nparams > 1) ? M->params[1] : 1.0;
  // P(hL) with L = cdx [1,-2,1]: sum over k of (h cdx)^k / k! times the k-th
  // power of the stencil, whose weights at offsets 0..4 are, for k = 1..4,
  // (-2, 1), (6, -4, 1), (-20, 15, -6, 1), (70, -56, 28, -8, 1)
  const double dx = 1.0 / (double)(a.n + 1);
  const double z = a.h * (a.kappa / (dx * dx));
  const double z2 = z * z / 2.0, z3 = z * z * z / 6.0, z4 = z * z * z * z / 24.0;
  a.poly9[0] = 1.0 - 2.0 * z + 6.0 * z2 - 20.0 * z3 + 70.0 * z4;
  a.poly9[1] = z - 4.0 * z2 + 15.0 * z3 - 56.0 * z4;
  a.poly9[2] = z2 - 6.0 * z3 + 28.0 * z4;
  a.poly9[3] = z3 - 8.0 * z4;
  a.poly9[4] = z4;
  // The step maps a constant (a smooth mode, to second order) to itself only
  // if c_0 + 2 (c_1 + .. + c_4) = 1 exactly; the rounded weights miss that by
  // about an ulp, and the smooth modes then grow or decay by that much every
  // step: over the 10 240 steps of the heat workload, 1e-12 (float64) and
  // 8e-5 (float32) relative drift.  So c_4, the smallest weight, takes up the
  // rounding residual of the sum, computed exactly: for the float32 weights
  // in double arithmetic (their sum needs < 40 bits), for the float64 ones
  // with error-free two-sums.  The drift then falls to 2e-15 and 6e-6.
  {
    float f[5];
    for (int k = 0; k < 5; ++k) f[k] = (float)a.poly9[k];
    const double tot = (double)f[0] + 2.0 * ((double)f[1] + (double)f[2] + (double)f[3] + (double)f[4]);
    f[4] = (float)((double)f[4] + 0.5 * (1.0 - tot));
    for (int k = 0; k < 5; ++k) a.poly9f[k] = f[k];
    // double: hi + lo = c_0 + 2 c_1 + .. + 2 c_4 exactly (Knuth's two-sum)
    double hi = a.poly9[0], lo = 0.0;
    for (int k = 1; k < 5; ++k) {
      const double b = 2.0 * a.poly9[k];
      const double sum = hi + b, bb = sum - hi;
      lo += (hi - (sum - bb)) + (b - bb);
      hi = sum;
    }
    a.poly9[4] += 0.5 * ((1.0 - hi) - lo);
  }
  return a;
}


template <typename T, int G, int R>
static nv_status launch_window_GR(const HeatArgs& a, int block, cudaStream_t s, bool tf32out) {
  const int64_t warps = ((int64_t)a.S * a.n + 32 / G - 1) / (32 / G);
  int grid = 0;
  nv_status st;
  if constexpr (sizeof(T) == 4) {
    if (tf32out) {
      st = persistent_grid(heat_window_kernel<T, G, R, true>, block, warps, &grid);
      if (st != NV_OK) return st;
      heat_window_kernel<T, G, R, true><<<grid, block, 0, s>>>(a);
      return nv_cuda_check(cudaGetLastError(), "heat_window_kernel launch");
    }
  }
  st = persistent_grid(heat_window_kernel<T, G, R, false>, block, warps, &grid);
  if (st != NV_OK) return st;
  heat_window_kernel<T, G, R, false><<<grid, block, 0, s>>>(a);
  return nv_cuda_check(cudaGetLastError(), "heat_window_kernel launch");
}

template <typename T, int GA, int R>
static nv_status launch_window2(const HeatArgs& a, int m1, int block, cudaStream_t s, bool tf32out) {
  const int64_t warps = ((int64_t)a.S * a.n + 32 / GA - 1) / (32 / GA);
  int grid = 0;
  nv_status st;
  if constexpr (sizeof(T) == 4) {
    if (tf32out) {
      st = persistent_grid(heat_window2_kernel<T, GA, R, true>, block, warps, &grid);
      if (st != NV_OK) return st;
      heat_window2_kernel<T, GA, R, true><<<grid, block, 0, s>>>(a, m1);
      return nv_cuda_check(cudaGetLastError(), "heat_window2_kernel launch");
    }
  }
  st = persistent_grid(heat_window2_kernel<T, GA, R, false>, block, warps, &grid);
  if (st != NV_OK) return st;
  heat_window2_kernel<T, GA, R, false><<<grid, block, 0, s>>>(a, m1);
  return nv_cuda_check(cudaGetLastError(), "heat_window2_kernel launch");
}

template <typename T, int G1, int R>
static nv_status launch_window3(const HeatArgs& a, int m1, int m2, cudaStream_t s, bool tf32out) {
  const int block = 128;                        // the kernel's shared memory holds four warps
  const int64_t warps = ((int64_t)a.S * a.n + 32 / G1 - 1) / (32 / G1);
  int grid = 0;
  nv_status st;
  if constexpr (sizeof(T) == 4) {
    if (tf32out) {
      st = persistent_grid(heat_window3_kernel<T, G1, R, true>, block, warps, &grid);
      if (st != NV_OK) return st;
      heat_window3_kernel<T, G1, R, true><<<grid, block, 0, s>>>(a, m1, m2);
      return nv_cuda_check(cudaGetLastError(), "heat_window3_kernel launch");
    }
  }
  st = persistent_grid(heat_window3_kernel<T, G1, R, false>, block, warps, &grid);
  if (st != NV_OK) return st;
  heat_window3_kernel<T, G1, R, false><<<grid, block, 0, s>>>(a, m1, m2);
  return nv_cuda_check(cudaGetLastError(), "heat_window3_kernel launch");
}

template <int G1, int R>
static nv_status launch_window3_x2(const HeatArgs& a, int m1, int m2, cudaStream_t s, bool tf32out) {
  const int block = 128;
  const size_t smem = sizeof(f32x2_t) * 4 * 3 * 32 * (R + 1);
  const int64_t warps = ((int64_t)((a.S + 1) / 2) * a.n + 32 / G1 - 1) / (32 / G1);
  int grid = 0;
  nv_status st;
  if (tf32out) {
    st = nv_cuda_check(cudaFuncSetAttribute(heat_window3_x2_kernel<G1, R, true>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                       "heat_window3_x2_kernel shared memory");
    if (st == NV_OK) st = persistent_grid(heat_window3_x2_kernel<G1, R, true>, block, warps, &grid, smem);
    if (st != NV_OK) return st;
    heat_window3_x2_kernel<G1, R, true><<<grid, block, smem, s>>>(a, m1, m2);
    return nv_cuda_check(cudaGetLastError(), "heat_window3_x2_kernel launch");
  }
  st = nv_cuda_check(cudaFuncSetAttribute(heat_window3_x2_kernel<G1, R, false>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                     "heat_window3_x2_kernel shared memory");
  if (st == NV_OK) st = persistent_grid(heat_window3_x2_kernel<G1, R, false>, block, warps, &grid, smem);
  if (st != NV_OK) return st;
  heat_window3_x2_kernel<G1, R, false><<<grid, block, smem, s>>>(a, m1, m2);
  return nv_cuda_check(cudaGetLastError(), "heat_window3_x2_kernel launch");
}

// Built window shapes: one window of G lanes x R rows (W = G*R >= 8m+1); two
// (GA x R for the first m1 = (GA*R-1)/8 steps, 2*GA x R for the rest); or
// three (G1, 2*G1, 4*G1 lanes of R rows, switching after m1 = (G1*R-1)/8 and
// m2 = (2*G1*R-1)/8 steps).  The launcher takes the built option with the
// fewest row-steps per column (m*W; m1*GA*R + (m-m1)*2*GA*R; and so on); a
// window as wide as n only when asked for, since the full-width kernel does
// the same work.  Form 3 takes single windows only, form 4 two-phase windows
// only, form 5 three-phase windows only, form 0 any.  NV_ENOTSUP, with no
// launch, when nothing fits.
// What a heat build launched for the homogeneous columns: the point-steps it
// integrates per column and the kernel, for nv_maps_info.
struct BuildInfo {
  int64_t work_per_column = 0;
  char kernel[64] = "";
};

template <typename T>
static const char* type_name() { return sizeof(T) == 8 ? "double" : "float"; }

static void note_build(BuildInfo* bi, int64_t work, const char* fmt, ...) {
  if (!bi) return;
  bi->work_per_column = work;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(bi->kernel, sizeof(bi->kernel), fmt, ap);
  va_end(ap);
}

static const int kWindow1[][2] = {{8, 4}, {8, 8}, {8, 11}, {16, 8}, {16, 11}, {32, 8}};
static const int kWindow2[][2] = {{4, 11}, {8, 8}};
// three windows of 22, 44 and 88 rows: two lanes of 11 rows for the first
// (float64), or one lane of 22 rows (float32, where the shuffles and the
// window edges, not the arithmetic, set the pace); key 17 picks for float32
static const int kWindow3[][2] = {{2, 11}, {1, 22}};

// float32 three-window build on packed slice pairs: nv_tune_set key 17 = 0
// (default: two lanes of 11 rows), 3 or 4
static bool heat_f32_packed() { return g_tune.heat_f32_lanes == 0 || g_tune.heat_f32_lanes >= 3; }

template <typename T>
static nv_status launch_heat_window(const HeatArgs& a, int block, cudaStream_t s, bool tf32out, int form,
                                    BuildInfo* bi) {
  int64_t best = INT64_MAX;
  int pick = -1, m1 = 0;
  int m2 = 0;
  if (form == 0 || form == 3) {
    for (int k = 0; k < 6; ++k) {
      const int W = kWindow1[k][0] * kWindow1[k][1];
      if (8 * a.m + 1 > W || W > a.n || (W == a.n && form != 3)) continue;
      if (a.m * W < best) best = a.m * W, pick = k;
    }
  }
  if (form == 0 || form == 4) {
    for (int k = 0; k < 2; ++k) {
      const int WA = kWindow2[k][0] * kWindow2[k][1], WB = 2 * WA, k1 = (WA - 1) / 8;
      if (8 * a.m + 1 > WB || WB > a.n || k1 >= a.m || (WB == a.n && form != 4)) continue;
      const int64_t cost = k1 * WA + (a.m - k1) * WB;
      if (cost < best) best = cost, pick = 6 + k, m1 = k1;
    }
  }
  if (form == 0 || form == 5) {
    const int lanes = g_tune.heat_f32_lanes;
    const int k3 = sizeof(T) == 4 && (lanes == 1 || lanes == 3) ? 1 : 0;
    for (int k = k3; k <= k3; ++k) {
      const int W1 = kWindow3[k][0] * kWindow3[k][1], W2 = 2 * W1, W3 = 4 * W1;
      const int k1 = (W1 - 1) / 8, k2 = (W2 - 1) / 8;
      if (8 * a.m + 1 > W3 || W3 > a.n || k2 >= a.m || k1 < 1 || (W3 == a.n && form != 5)) continue;
      const int64_t cost = k1 * W1 + (k2 - k1) * W2 + (a.m - k2) * W3;
      if (cost < best) best = cost, pick = 8 + k, m1 = k1, m2 = k2;
    }
  }
  const int t32 = tf32out ? 1 : 0;
  if (pick >= 0 && pick < 6)
    note_build(bi, best, "heat_window_kernel<%s,%d,%d,%d>", type_name<T>(), kWindow1[pick][0], kWindow1[pick][1], t32);
  else if (pick >= 6 && pick < 8)
    note_build(bi, best, "heat_window2_kernel<%s,%d,%d,%d>", type_name<T>(), kWindow2[pick - 6][0],
               kWindow2[pick - 6][1], t32);
  // float32 three windows on packed slice pairs (key 17 = 3 or 4) where S > 1
  const bool x2 = sizeof(T) == 4 && pick >= 8 && a.S > 1 && heat_f32_packed();
  if (x2)
    note_build(bi, best, "heat_window3_x2_kernel<%d,%d,%d>", kWindow3[pick - 8][0], kWindow3[pick - 8][1], t32);
  else if (pick >= 8)
    note_build(bi, best, "heat_window3_kernel<%s,%d,%d,%d>", type_name<T>(), kWindow3[pick - 8][0],
               kWindow3[pick - 8][1], t32);
  if (x2) return pick == 8 ? launch_window3_x2<2, 11>(a, m1, m2, s, tf32out)
                           : launch_window3_x2<1, 22>(a, m1, m2, s, tf32out);
  switch (pick) {
    case 0: return launch_window_GR<T, 8, 4>(a, block, s, tf32out);
    case 1: return launch_window_GR<T, 8, 8>(a, block, s, tf32out);
    case 2: return launch_window_GR<T, 8, 11>(a, block, s, tf32out);
    case 3: return launch_window_GR<T, 16, 8>(a, block, s, tf32out);
    case 4: return launch_window_GR<T, 16, 11>(a, block, s, tf32out);
    case 5: return launch_window_GR<T, 32, 8>(a, block, s, tf32out);
    case 6: return launch_window2<T, 4, 11>(a, m1, block, s, tf32out);
    case 7: return launch_window2<T, 8, 8>(a, m1, block, s, tf32out);
    case 8: return launch_window3<T, 2, 11>(a, m1, m2, s, tf32out);
    case 9:
      if constexpr (sizeof(T) == 4) return launch_window3<T, 1, 22>(a, m1, m2, s, tf32out);
      break;
    default: break;
  }
  if (form >= 3)
    return nv_fail(NV_ENOTSUP, "no built window holds 8m+1 = %lld rows within n = %d",
                   (long long)(8 * a.m + 1), a.n);
  return NV_ENOTSUP;
}

template <typename T, int R>
static nv_status launch_heat_forcing(const HeatArgs& a, int block, cudaStream_t s);
template <typename T, int R>
static nv_status launch_heat_homogeneous(const HeatArgs& a, int block, cudaStream_t s, bool tf32out,
                                         BuildInfo* bi);

// A library-owned non-blocking stream per device for work that runs beside a
// build on the caller's stream (created on first use, kept for the process;
// not valid after a cudaDeviceReset of that device).
static nv_status heat_side_stream(cudaStream_t* out) {
  static std::mutex mu;
  static cudaStream_t streams[64] = {};
  int dev = 0;
  nv_status st = nv_cuda_check(cudaGetDevice(&dev), "current device");
  if (st != NV_OK) return st;
  if (dev < 0 || dev >= 64) return nv_fail(NV_ENOTSUP, "device index %d too large", dev);
  std::lock_guard<std::mutex> lock(mu);
  if (!streams[dev]) {
    st = nv_cuda_check(cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking), "side stream");
    if (st != NV_OK) return st;
  }
  *out = streams[dev];
  return NV_OK;
}

template <typename T, int R>
static nv_status launch_heat_R(const HeatArgs& a, cudaStream_t s, bool tf32out, BuildInfo* bi) {
  const int warps_per_cta = g_tune.affine_warps > 0 ? g_tune.affine_warps : 8;
  const int block = 32 * warps_per_cta;
  int grid = 0;
  nv_status st;
  if (a.varcoef) {
    note_build(bi, (int64_t)a.n * a.m, "heat_literal_kernel<%s,%d>", type_name<T>(), R);
    st = persistent_grid(heat_literal_kernel<T, R>, block, (int64_t)a.S * (a.n + 1), &grid);
    if (st != NV_OK) return st;
    heat_literal_kernel<T, R><<<grid, block, 0, s>>>(a, 1);
    return nv_cuda_check(cudaGetLastError(), "heat_literal_kernel launch");
  }
  // The forcing columns (one forced solve per slice, latency-bound) run on a
  // second stream beside the homogeneous build, submitted after it so that
  // they take the SMs its last CTAs leave free.
  cudaStream_t side = nullptr;
  if ((st = heat_side_stream(&side)) != NV_OK) return st;
  cudaEvent_t fork = nullptr, join = nullptr;
  st = nv_cuda_check(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming), "fork event");
  if (st == NV_OK) st = nv_cuda_check(cudaEventCreateWithFlags(&join, cudaEventDisableTiming), "join event");
  if (st == NV_OK) st = nv_cuda_check(cudaEventRecord(fork, s), "fork record");
  if (st == NV_OK) st = launch_heat_homogeneous<T, R>(a, block, s, tf32out, bi);
  if (st == NV_OK) st = nv_cuda_check(cudaStreamWaitEvent(side, fork, 0), "fork wait");
  if (st == NV_OK) st = launch_heat_forcing<T, R>(a, block, side);
  if (st == NV_OK) st = nv_cuda_check(cudaEventRecord(join, side), "join record");
  if (st == NV_OK) st = nv_cuda_check(cudaStreamWaitEvent(s, join, 0), "join wait");
  if (fork) cudaEventDestroy(fork);
  if (join) cudaEventDestroy(join);
  return st;
}

template <typename T, int R>
static nv_status launch_heat_forcing(const HeatArgs& a, int block, cudaStream_t s) {
  int grid = 0;
  nv_status st;
  if constexpr (sizeof(T) == 8) {
    st = persistent_grid(heat_forcing_kernel<R>, block, (int64_t)a.S, &grid);
    if (st != NV_OK) return st;
    heat_forcing_kernel<R><<<grid, block, 0, s>>>(a);
    return nv_cuda_check(cudaGetLastError(), "heat_forcing_kernel launch");
  } else {
    st = persistent_grid(heat_literal_kernel<T, R>, block, (int64_t)a.S, &grid);
    if (st != NV_OK) return st;
    heat_literal_kernel<T, R><<<grid, block, 0, s>>>(a, 0);
    return nv_cuda_check(cudaGetLastError(), "heat_literal_kernel launch");
  }
}

// The homogeneous columns of a time-independent heat operator.
template <typename T, int R>
static nv_status launch_heat_homogeneous(const HeatArgs& a, int block, cudaStream_t s, bool tf32out,
                                         BuildInfo* bi) {
  const int t32 = tf32out ? 1 : 0;
  int grid = 0;
  nv_status st;
  const int form = g_tune.heat_step_form;
  if (form == 0 || form >= 3) {
    st = launch_heat_window<T>(a, block, s, tf32out, form, bi);
    if (st != NV_ENOTSUP || form != 0) return st;
  }
  if constexpr (R >= 4) {
    if (g_tune.heat_step_form != 1 && a.n % R == 0) {
      note_build(bi, (int64_t)a.n * a.m, "heat_poly9_kernel<%s,%d,%d>", type_name<T>(), R, t32);
      if constexpr (sizeof(T) == 4) {
        if (tf32out) {
          st = persistent_grid(heat_poly9_kernel<T, R, true>, block, (int64_t)a.S * a.n, &grid);
          if (st != NV_OK) return st;
          heat_poly9_kernel<T, R, true><<<grid, block, 0, s>>>(a);
          return nv_cuda_check(cudaGetLastError(), "heat_poly9_kernel launch");
        }
      }
      st = persistent_grid(heat_poly9_kernel<T, R, false>, block, (int64_t)a.S * a.n, &grid);
      if (st != NV_OK) return st;
      heat_poly9_kernel<T, R, false><<<grid, block, 0, s>>>(a);
      return nv_cuda_check(cudaGetLastError(), "heat_poly9_kernel launch");
    }
  }
  note_build(bi, (int64_t)a.n * a.m, "heat_horner_kernel<%s,%d,%d>", type_name<T>(), R, t32);
  if constexpr (sizeof(T) == 4) {
    if (tf32out) {
      st = persistent_grid(heat_horner_kernel<T, R, true>, block, (int64_t)a.S * a.n, &grid);
      if (st != NV_OK) return st;
      heat_horner_kernel<T, R, true><<<grid, block, 0, s>>>(a);
      return nv_cuda_check(cudaGetLastError(), "heat_horner_kernel launch");
    }
  }
  st = persistent_grid(heat_horner_kernel<T, R, false>, block, (int64_t)a.S * a.n, &grid);
  if (st != NV_OK) return st;
  heat_horner_kernel<T, R, false><<<grid, block, 0, s>>>(a);
  return nv_cuda_check(cudaGetLastError(), "heat_horner_kernel launch");
}

template <typename T>
static nv_status launch_heat_typed(const HeatArgs& a, int R, cudaStream_t s, bool tf32out, BuildInfo* bi) {
  switch (R) {
    case 1: return launch_heat_R<T, 1>(a, s, tf32out, bi);
    case 2: return launch_heat_R<T, 2>(a, s, tf32out, bi);
    case 4: return launch_heat_R<T, 4>(a, s, tf32out, bi);
    case 8: return launch_heat_R<T, 8>(a, s, tf32out, bi);
    case 16: return launch_heat_R<T, 16>(a, s, tf32out, bi);
    default: return nv_fail(NV_ENOTSUP, "heat equation dimension %d exceeds 512", a.n);
  }
}

nv_status launch_advdiff_build(nv_maps* M, cudaStream_t s);
nv_status launch_wave_build(const nv_maps* M, cudaStream_t s);

nv_status launch_affine_build(nv_maps* M, cudaStream_t s) {
  if (M->rhs_kind == NV_RHS_HEAT1D || M->rhs_kind == NV_RHS_HEAT1D_VARCOEF) {
    if (M->scheme != NV_RK4) return nv_fail(NV_ENOTSUP, "affine heat maps are built with RK4");
    const int R = rows_per_lane(M->dim);
    if (R == 0) return nv_fail(NV_ENOTSUP, "heat equation dimension %d exceeds 512", M->dim);
    const HeatArgs a = heat_args(M);
    // each RK4 step of the three-point operator widens a column's support by
    // four rows on each side (four stages), so A_j is zero off the band
    // |r - c| <= 4m
    M->band = M->m < (1 << 28) ? (int32_t)(4 * M->m + 1) : 0;
    BuildInfo bi;
    const nv_status st = M->prec == NV_FP64 ? launch_heat_typed<double>(a, R, s, false, &bi)
                                            : launch_heat_typed<float>(a, R, s, M->prec == NV_TF32_REFINE, &bi);
    // the forcing column (full width; every column for the variable-coefficient
    // equation, whose kernel records the work of one) and the homogeneous ones
    M->work_per_slice = (int64_t)M->dim * M->m + (int64_t)M->dim * bi.work_per_column;
    memcpy(M->build_kernel, bi.kernel, sizeof(M->build_kernel));
    return st;
  }
  if (M->rhs_kind == NV_RHS_ADVDIFF2D) return launch_advdiff_build(M, s);
  if (M->rhs_kind == NV_RHS_WAVE_CHEB) return launch_wave_build(M, s);
  return nv_fail(NV_ENOTSUP, "affine maps are not built for rhs kind %d", M->rhs_kind);
}

nv_status launch_serial_heat(const nv_maps* M, const double* y0, double* yT, cudaStream_t s) {
  const HeatArgs a = heat_args(M);
  switch (rows_per_lane(M->dim)) {
    case 1: heat_serial_kernel<1><<<1, 32, 0, s>>>(a, y0, yT); break;
    case 2: heat_serial_kernel<2><<<1, 32, 0, s>>>(a, y0, yT); break;
    case 4: heat_serial_kernel<4><<<1, 32, 0, s>>>(a, y0, yT); break;
    case 8: heat_serial_kernel<8><<<1, 32, 0, s>>>(a, y0, yT); break;
    case 16: heat_serial_kernel<16><<<1, 32, 0, s>>>(a, y0, yT); break;
    default: return nv_fail(NV_ENOTSUP, "heat equation dimension %d exceeds 512", M->dim);
  }
  return nv_cuda_check(cudaGetLastError(), "heat_serial_kernel launch");
}

nv_status launch_heat_defect(const nv_maps* M, const double* lam_tilde, double* d, cudaStream_t s) {
  if (M->rhs_kind != NV_RHS_HEAT1D && M->rhs_kind != NV_RHS_HEAT1D_VARCOEF)
    return nv_fail(NV_ENOTSUP, "float64 defects are built for the heat equations");
  const HeatArgs a = heat_args(M);
  const int block = 64;     // two warps per CTA: one slice per warp spread over all SMs
  int grid = 0;
  nv_status st;
#define NVPIT_DEFECT_CASE(RR)                                                                   \
  case RR:                                                                                     \
    st = persistent_grid(heat_defect_kernel<RR>, block, (int64_t)a.S, &grid);                  \
    if (st != NV_OK) return st;                                                                \
    heat_defect_kernel<RR><<<grid, block, 0, s>>>(a, lam_tilde, d);                            \
    break;
  switch (rows_per_lane(M->dim)) {
    NVPIT_DEFECT_CASE(1)
    NVPIT_DEFECT_CASE(2)
    NVPIT_DEFECT_CASE(4)
    NVPIT_DEFECT_CASE(8)
    NVPIT_DEFECT_CASE(16)
    default: return nv_fail(NV_ENOTSUP, "heat equation dimension %d exceeds 512", M->dim);
  }
#undef NVPIT_DEFECT_CASE
  return nv_cuda_check(cudaGetLastError(), "heat_defect_kernel launch");
}
