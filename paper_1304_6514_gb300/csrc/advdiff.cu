// Periodic 2-D advection-diffusion on the 64 x 64 grid (d = 4096): the affine
// map build (float64 strip kernel; float32 / bfloat16 block kernel, by default
// with the first steps on windows), the float64 defects of the refinement and
// the serial fine solve.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>

#include "common.cuh"

namespace nvpit {

// ---------------------------------------------------------------------------
// Periodic 2-D advection-diffusion on an nx x nx grid (nx = 64, d = 4096):
// L u = nu lap5(u) - ax D-x u - ay D-y u.  Float64 (the build, the serial
// solve, the correction defects): one CTA of 256 threads integrates one state
// (a basis column).  Thread t holds the strip iy = 16*(t/64) .. +15 at
// ix = t % 64 in registers: its y-neighbours are in the same thread except at
// the strip ends, its x-neighbours in lanes +-1 (warp shuffles) except at the
// warp's edge lanes; strip-end rows and edge-lane strips cross through
// double-buffered shared memory, one __syncthreads per stage.  RK4 runs in
// Horner form (time-invariant operator), the stage factor h/k folded into the
// five stencil weights.  The float32 build uses 8 x 8 blocks instead
// (advdiff_block_kernel below), where the FP32 pipe, not the FP64 one, is the
// limit and the strip layout's shuffles would be.
constexpr int kAdvNx = 64;
constexpr int kAdvRows = 16;     // rows per thread strip

struct AdvArgs {
  void* out;
  int S;
  int64_t m;
  double h;
  double w_xm, w_xp, w_ym, w_yp, w_0;   // L u = sum of weights times neighbours
  // stage weights (h/k) w_* for Horner stage k = 4..1 (index 4 - k), in both
  // precisions so the float32 kernel does no float64 arithmetic
  double cw64[4][5];
  float cw32[4][5];
};

template <typename T>
__device__ __forceinline__ const T* adv_weights(const AdvArgs& a, int stage);
template <>
__device__ __forceinline__ const double* adv_weights<double>(const AdvArgs& a, int stage) {
  return a.cw64[stage];
}
template <>
__device__ __forceinline__ const float* adv_weights<float>(const AdvArgs& a, int stage) {
  return a.cw32[stage];
}

// m Horner-form RK4 steps of one state held in the strip layout (thread t:
// rows iy0 .. iy0+15 at column ix); the shared halo buffers belong to the CTA.
template <typename T>
struct AdvStripSmem {
  T top[2][4][kAdvNx];          // first row of each strip block, per buffer
  T bot[2][4][kAdvNx];          // last row
  T edge[2][8][2][kAdvRows];    // per warp: strips of lanes 0 and 31
};

template <typename T>
__device__ __forceinline__ void adv_strip_integrate(const AdvArgs& a, T* y, AdvStripSmem<T>& sm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ix = tid % kAdvNx, blk = tid / kAdvNx;
  const int pw = warp ^ 1;            // the other warp of the same 64-wide row band
  T v[kAdvRows];
  int buf = 0;
  for (int64_t i = 0; i < a.m; ++i) {
#pragma unroll
    for (int r = 0; r < kAdvRows; ++r) v[r] = y[r];
#pragma unroll
    for (int kk = 4; kk >= 1; --kk) {
      const T* cw = adv_weights<T>(a, 4 - kk);
      const T cxm = cw[0], cxp = cw[1], cym = cw[2], cyp = cw[3], c0 = cw[4];
      sm.top[buf][blk][ix] = v[0];
      sm.bot[buf][blk][ix] = v[kAdvRows - 1];
      if (lane == 0 || lane == 31) {
#pragma unroll
        for (int r = 0; r < kAdvRows; ++r) sm.edge[buf][warp][lane == 31][r] = v[r];
      }
      __syncthreads();
      const T above = sm.bot[buf][(blk + 3) & 3][ix];     // row iy0 - 1 (periodic)
      const T below = sm.top[buf][(blk + 1) & 3][ix];     // row iy0 + 16
      T nv[kAdvRows];
#pragma unroll
      for (int r = 0; r < kAdvRows; ++r) {
        T xm = __shfl_up_sync(0xffffffffu, v[r], 1);
        T xp = __shfl_down_sync(0xffffffffu, v[r], 1);
        if (lane == 0) xm = sm.edge[buf][pw][1][r];        // ix - 1 lives in the other warp's lane 31
        if (lane == 31) xp = sm.edge[buf][pw][0][r];       // ix + 1 in its lane 0
        const T ym = r == 0 ? above : v[r - 1];
        const T yp = r == kAdvRows - 1 ? below : v[r + 1];
        T acc = fma(c0, v[r], y[r]);
        acc = fma(cxm, xm, acc);
        acc = fma(cxp, xp, acc);
        acc = fma(cym, ym, acc);
        nv[r] = fma(cyp, yp, acc);
      }
#pragma unroll
      for (int r = 0; r < kAdvRows; ++r) v[r] = nv[r];
      buf ^= 1;
    }
#pragma unroll
    for (int r = 0; r < kAdvRows; ++r) y[r] = v[r];
  }
  __syncthreads();   // the shared halos are reused by the next state
}

template <typename T>
__global__ void __launch_bounds__(256) advdiff_affine_kernel(AdvArgs a) {
  constexpr int n = kAdvNx * kAdvNx;
  __shared__ AdvStripSmem<T> sm;
  const int tid = threadIdx.x;
  const int ix = tid % kAdvNx, blk = tid / kAdvNx, iy0 = blk * kAdvRows;
  T* out = reinterpret_cast<T*>(a.out);
  const int64_t total = (int64_t)a.S * (n + 1);
  for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
    const int j = (int)(w / (n + 1));
    const int c = (int)(w - (int64_t)j * (n + 1));     // 0: solve from 0 (no forcing), else e_{c-1}
    T y[kAdvRows];
#pragma unroll
    for (int r = 0; r < kAdvRows; ++r) y[r] = ((c >= 1) && ((iy0 + r) * kAdvNx + ix == c - 1)) ? (T)1 : (T)0;
    adv_strip_integrate<T>(a, y, sm);
    T* col = out + ((int64_t)j * (n + 1) + c) * n;
#pragma unroll
    for (int r = 0; r < kAdvRows; ++r) col[(iy0 + r) * kAdvNx + ix] = y[r];
  }
}

// Float64 defects of approximate boundary states for the correction passes of
// NV_BF16_REFINE: d_j = g^j(lam_j) - lam_{j+1}, one CTA per slice integrating
// lam_j over slice j in float64 (the operator is time-invariant and unforced,
// so the Horner form is the RK4 step).  lam: (S+1) x n, d: S x n.
__global__ void __launch_bounds__(256) advdiff_defect_kernel(AdvArgs a, const double* lam, double* d) {
  constexpr int n = kAdvNx * kAdvNx;
  __shared__ AdvStripSmem<double> sm;
  const int tid = threadIdx.x;
  const int ix = tid % kAdvNx, blk = tid / kAdvNx, iy0 = blk * kAdvRows;
  for (int j = blockIdx.x; j < a.S; j += gridDim.x) {
    double y[kAdvRows];
#pragma unroll
    for (int r = 0; r < kAdvRows; ++r) y[r] = lam[(int64_t)j * n + (iy0 + r) * kAdvNx + ix];
    adv_strip_integrate<double>(a, y, sm);
#pragma unroll
    for (int r = 0; r < kAdvRows; ++r) {
      const int64_t o = (int64_t)(iy0 + r) * kAdvNx + ix;
      d[(int64_t)j * n + o] = y[r] - lam[(int64_t)(j + 1) * n + o];
    }
  }
}

// Float32 build with 8 x 8 blocks: one CTA of 64 threads integrates one basis
// column, thread (tx, ty) = (t % 8, t / 8) holding the grid block
// ix = 8 tx .. 8 tx + 7, iy = 8 ty .. 8 ty + 7 in registers. A stage exchanges
// only the block's four edges (32 values for 64 points, against two shuffles
// per point in the strip layout): each thread writes its edges to
// double-buffered shared memory as 128-bit stores, one __syncthreads, and
// reads its four neighbours' facing edges (periodic in both directions).
// The arithmetic per point and its order are those of advdiff_affine_kernel.
constexpr int kAdvB = 8;                       // block edge
constexpr int kAdvBlockThreads = (kAdvNx / kAdvB) * (kAdvNx / kAdvB);   // 64

// Column output of the float32 block build: float32, or bfloat16 bits rounded
// to nearest even (NV_BF16_REFINE), one 16-byte store per 4 / 8 values.
__device__ __forceinline__ void adv_store_row(float* dst, const float* v) {
  reinterpret_cast<float4*>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
  reinterpret_cast<float4*>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
}
__device__ __forceinline__ void adv_store_row(uint16_t* dst, const float* v) {
  uint32_t w[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);   // low half = v[2q]
    w[q] = *reinterpret_cast<const uint32_t*>(&p);
  }
  reinterpret_cast<uint4*>(dst)[0] = make_uint4(w[0], w[1], w[2], w[3]);
}

template <typename OutT>
__global__ void __launch_bounds__(kAdvBlockThreads, 4) advdiff_block_kernel(AdvArgs a) {
  constexpr int n = kAdvNx * kAdvNx;
  constexpr int TB = kAdvNx / kAdvB;           // 8 blocks per direction
  // edges[buffer][side][half][thread]: side 0 left column, 1 right column,
  // 2 top row, 3 bottom row; half h holds edge points 4h .. 4h+3
  __shared__ float4 edges[2][4][2][kAdvBlockThreads];
  const int t = threadIdx.x, tx = t % TB, ty = t / TB;
  const int ix0 = kAdvB * tx, iy0 = kAdvB * ty;
  const int t_left = ty * TB + (tx + TB - 1) % TB, t_right = ty * TB + (tx + 1) % TB;
  const int t_up = ((ty + TB - 1) % TB) * TB + tx, t_down = ((ty + 1) % TB) * TB + tx;
  OutT* out = reinterpret_cast<OutT*>(a.out);
  const int64_t total = (int64_t)a.S * (n + 1);
  int buf = 0;
  for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
    const int j = (int)(w / (n + 1));
    const int c = (int)(w - (int64_t)j * (n + 1));     // 0: solve from 0 (no forcing), else e_{c-1}
    float y[kAdvB][kAdvB], v[kAdvB][kAdvB];
#pragma unroll
    for (int r = 0; r < kAdvB; ++r)
#pragma unroll
      for (int q = 0; q < kAdvB; ++q) y[r][q] = ((iy0 + r) * kAdvNx + ix0 + q == c - 1) ? 1.f : 0.f;
    for (int64_t i = 0; i < a.m; ++i) {
#pragma unroll
      for (int r = 0; r < kAdvB; ++r)
#pragma unroll
        for (int q = 0; q < kAdvB; ++q) v[r][q] = y[r][q];
#pragma unroll
      for (int kk = 4; kk >= 1; --kk) {
        const float* cw = a.cw32[4 - kk];
        const float cxm = cw[0], cxp = cw[1], cym = cw[2], cyp = cw[3], c0 = cw[4];
        float4(*e)[2][kAdvBlockThreads] = edges[buf];
        e[0][0][t] = make_float4(v[0][0], v[1][0], v[2][0], v[3][0]);
        e[0][1][t] = make_float4(v[4][0], v[5][0], v[6][0], v[7][0]);
        e[1][0][t] = make_float4(v[0][7], v[1][7], v[2][7], v[3][7]);
        e[1][1][t] = make_float4(v[4][7], v[5][7], v[6][7], v[7][7]);
        e[2][0][t] = make_float4(v[0][0], v[0][1], v[0][2], v[0][3]);
        e[2][1][t] = make_float4(v[0][4], v[0][5], v[0][6], v[0][7]);
        e[3][0][t] = make_float4(v[7][0], v[7][1], v[7][2], v[7][3]);
        e[3][1][t] = make_float4(v[7][4], v[7][5], v[7][6], v[7][7]);
        __syncthreads();
        // x - 1 of column 0: the left block's right column; x + 1 of column 7:
        // the right block's left column; y - 1 of row 0: the upper block's
        // bottom row; y + 1 of row 7: the lower block's top row
        const float4 l0 = e[1][0][t_left], l1 = e[1][1][t_left];
        const float4 r0 = e[0][0][t_right], r1 = e[0][1][t_right];
        const float4 u0 = e[3][0][t_up], u1 = e[3][1][t_up];
        const float4 d0 = e[2][0][t_down], d1 = e[2][1][t_down];
        const float hl[kAdvB] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
        const float hr[kAdvB] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
        const float hu[kAdvB] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
        const float hd[kAdvB] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
        float prev[kAdvB];                     // row r - 1 before this stage
#pragma unroll
        for (int q = 0; q < kAdvB; ++q) prev[q] = hu[q];
#pragma unroll
        for (int r = 0; r < kAdvB; ++r) {
          float nrow[kAdvB];
#pragma unroll
          for (int q = 0; q < kAdvB; ++q) {
            const float xm = q == 0 ? hl[r] : v[r][q - 1];
            const float xp = q == kAdvB - 1 ? hr[r] : v[r][q + 1];
            const float yp = r == kAdvB - 1 ? hd[q] : v[r + 1][q];
            float acc = fmaf(c0, v[r][q], y[r][q]);
            acc = fmaf(cxm, xm, acc);
            acc = fmaf(cxp, xp, acc);
            acc = fmaf(cym, prev[q], acc);
            nrow[q] = fmaf(cyp, yp, acc);
          }
#pragma unroll
          for (int q = 0; q < kAdvB; ++q) {
            prev[q] = v[r][q];
            v[r][q] = nrow[q];
          }
        }
        buf ^= 1;
      }
#pragma unroll
      for (int r = 0; r < kAdvB; ++r)
#pragma unroll
        for (int q = 0; q < kAdvB; ++q) y[r][q] = v[r][q];
    }
    OutT* col = out + ((int64_t)j * (n + 1) + c) * n;
#pragma unroll
    for (int r = 0; r < kAdvB; ++r) adv_store_row(col + (iy0 + r) * kAdvNx + ix0, y[r]);
  }
}

// The float32 build with the first steps on windows.  The four Horner stages
// of a step on the five-point operator carry information one point each, so
// the column started from the unit point (cx, cy) is exactly zero outside
// |x - cx| + |y - cy| <= 4k (periodically) after k steps.  For the first
// m1 <= 3 steps (radius <= 12) each column is integrated on a window of 4 x 4
// blocks (32 x 32 points) whose block-aligned origin bx0 = floor((cx-12)/8)
// (mod 8) puts the radius-12 diamond inside it with the cut edges at least 13
// points from the centre: the zeros read there are the exact values at every
// stage that reads them (the reach before the last stage is 4*m1 - 1).  So
// the 64 threads of a CTA carry four columns through those steps, 16 threads
// (4 x 4 blocks of 8 x 8 points) each, then take the columns one after another
// through the remaining steps on the whole periodic grid, starting from the
// windows staged in shared memory.  One step loop serves both (its halo
// sources are set per segment; a missing neighbour reads a zero edge slot), so
// the unrolled stages appear once in the code.  Every point is the same
// floating-point expression as in advdiff_block_kernel (inputs differ at most
// in the sign of a zero), so the maps are the same; the point-steps per column
// fall from 4096 m to 1024 m1 + 4096 (m - m1).
template <typename OutT>
__global__ void __launch_bounds__(kAdvBlockThreads, 4) advdiff_window_kernel(AdvArgs a, int m1) {
  constexpr int n = kAdvNx * kAdvNx;
  constexpr int TB = kAdvNx / kAdvB;           // 8 blocks per direction
  constexpr int WB = 4;                        // window edge in blocks
  constexpr int CPC = kAdvBlockThreads / (WB * WB);   // columns per CTA in the windows
  constexpr int kZero = kAdvBlockThreads;      // edge slot that stays zero
  // edges[buffer][side][half][thread]: as advdiff_block_kernel, plus the zero slot
  __shared__ float4 edges[2][4][2][kAdvBlockThreads + 1];
  // the windows' blocks as 16 float4 each, one float4 of padding so that the
  // threads' slots fall on different banks
  constexpr int kSlot = kAdvB * kAdvB / 4 + 1;
  __shared__ float4 win[CPC][WB * WB][kSlot];
  const int t = threadIdx.x, tx = t % TB, ty = t / TB;
  const int g = t / (WB * WB), lt = t % (WB * WB), lx = lt % WB, ly = lt / WB;
  const int reach1 = 4 * m1;                   // launcher: 1 <= m1 <= 3, m1 <= m
  if (t < 16) edges[t >> 3][(t >> 1) & 3][t & 1][kZero] = make_float4(0.f, 0.f, 0.f, 0.f);
  OutT* out = reinterpret_cast<OutT*>(a.out);
  const int64_t total = (int64_t)a.S * (n + 1);
  int buf = 0;
  for (int64_t w = blockIdx.x; w * CPC < total; w += gridDim.x) {
#pragma unroll 1
    for (int seg = 0; seg <= CPC; ++seg) {     // 0: the windows; s >= 1: column s - 1 on the whole grid
      const bool windows = seg == 0;
      const int64_t idx = w * CPC + (windows ? g : seg - 1);
      if (!windows && idx >= total) break;     // uniform over the CTA
      const int j = idx < total ? (int)(idx / (n + 1)) : 0;
      const int c = idx < total ? (int)(idx - (int64_t)j * (n + 1)) : 0;   // 0: no unit point
      const int cx = c >= 1 ? (c - 1) % kAdvNx : reach1, cy = c >= 1 ? (c - 1) / kAdvNx : reach1;
      const int bx0 = ((cx - reach1 + kAdvNx) / kAdvB) % TB, by0 = ((cy - reach1 + kAdvNx) / kAdvB) % TB;
      int bx, by, n_left, n_right, n_up, n_down;
      if (windows) {                           // block (lx, ly) of this group's window
        bx = (bx0 + lx) % TB;
        by = (by0 + ly) % TB;
        n_left = lx > 0 ? t - 1 : kZero;
        n_right = lx < WB - 1 ? t + 1 : kZero;
        n_up = ly > 0 ? t - WB : kZero;
        n_down = ly < WB - 1 ? t + WB : kZero;
      } else {                                 // block (tx, ty) of the periodic grid
        bx = tx;
        by = ty;
        n_left = ty * TB + (tx + TB - 1) % TB;
        n_right = ty * TB + (tx + 1) % TB;
        n_up = ((ty + TB - 1) % TB) * TB + tx;
        n_down = ((ty + 1) % TB) * TB + tx;
      }
      const int ix0 = kAdvB * bx, iy0 = kAdvB * by;
      float y[kAdvB][kAdvB], v[kAdvB][kAdvB];
      if (windows) {
#pragma unroll
        for (int r = 0; r < kAdvB; ++r)
#pragma unroll
          for (int q = 0; q < kAdvB; ++q) y[r][q] = ((iy0 + r) * kAdvNx + ix0 + q == c - 1) ? 1.f : 0.f;
      } else {
        const int wx = (tx - bx0 + TB) % TB, wy = (ty - by0 + TB) % TB;   // block in the window
        const bool inside = wx < WB && wy < WB;
        const float4* src = win[seg - 1][inside ? wy * WB + wx : 0];
#pragma unroll
        for (int r = 0; r < kAdvB; ++r) {
          const float4 p0 = src[2 * r], p1 = src[2 * r + 1];
          y[r][0] = inside ? p0.x : 0.f;
          y[r][1] = inside ? p0.y : 0.f;
          y[r][2] = inside ? p0.z : 0.f;
          y[r][3] = inside ? p0.w : 0.f;
          y[r][4] = inside ? p1.x : 0.f;
          y[r][5] = inside ? p1.y : 0.f;
          y[r][6] = inside ? p1.z : 0.f;
          y[r][7] = inside ? p1.w : 0.f;
        }
      }
      const int64_t i1 = windows ? m1 : a.m;
      for (int64_t i = windows ? 0 : m1; i < i1; ++i) {
#pragma unroll
        for (int r = 0; r < kAdvB; ++r)
#pragma unroll
          for (int q = 0; q < kAdvB; ++q) v[r][q] = y[r][q];
#pragma unroll
        for (int kk = 4; kk >= 1; --kk) {
          const float* cw = a.cw32[4 - kk];
          const float cxm = cw[0], cxp = cw[1], cym = cw[2], cyp = cw[3], c0 = cw[4];
          float4(*e)[2][kAdvBlockThreads + 1] = edges[buf];
          e[0][0][t] = make_float4(v[0][0], v[1][0], v[2][0], v[3][0]);
          e[0][1][t] = make_float4(v[4][0], v[5][0], v[6][0], v[7][0]);
          e[1][0][t] = make_float4(v[0][7], v[1][7], v[2][7], v[3][7]);
          e[1][1][t] = make_float4(v[4][7], v[5][7], v[6][7], v[7][7]);
          e[2][0][t] = make_float4(v[0][0], v[0][1], v[0][2], v[0][3]);
          e[2][1][t] = make_float4(v[0][4], v[0][5], v[0][6], v[0][7]);
          e[3][0][t] = make_float4(v[7][0], v[7][1], v[7][2], v[7][3]);
          e[3][1][t] = make_float4(v[7][4], v[7][5], v[7][6], v[7][7]);
          __syncthreads();
          const float4 l0 = e[1][0][n_left], l1 = e[1][1][n_left];
          const float4 r0 = e[0][0][n_right], r1 = e[0][1][n_right];
          const float4 u0 = e[3][0][n_up], u1 = e[3][1][n_up];
          const float4 d0 = e[2][0][n_down], d1 = e[2][1][n_down];
          const float hl[kAdvB] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
          const float hr[kAdvB] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
          const float hu[kAdvB] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
          const float hd[kAdvB] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
          float prev[kAdvB];                   // row r - 1 before this stage
#pragma unroll
          for (int q = 0; q < kAdvB; ++q) prev[q] = hu[q];
#pragma unroll
          for (int r = 0; r < kAdvB; ++r) {
            float nrow[kAdvB];
#pragma unroll
            for (int q = 0; q < kAdvB; ++q) {
              const float xm = q == 0 ? hl[r] : v[r][q - 1];
              const float xp = q == kAdvB - 1 ? hr[r] : v[r][q + 1];
              const float yp = r == kAdvB - 1 ? hd[q] : v[r + 1][q];
              float acc = fmaf(c0, v[r][q], y[r][q]);
              acc = fmaf(cxm, xm, acc);
              acc = fmaf(cxp, xp, acc);
              acc = fmaf(cym, prev[q], acc);
              nrow[q] = fmaf(cyp, yp, acc);
            }
#pragma unroll
            for (int q = 0; q < kAdvB; ++q) {
              prev[q] = v[r][q];
              v[r][q] = nrow[q];
            }
          }
          buf ^= 1;
        }
#pragma unroll
        for (int r = 0; r < kAdvB; ++r)
#pragma unroll
          for (int q = 0; q < kAdvB; ++q) y[r][q] = v[r][q];
      }
      if (windows) {
#pragma unroll
        for (int r = 0; r < kAdvB; ++r) {
          win[g][lt][2 * r] = make_float4(y[r][0], y[r][1], y[r][2], y[r][3]);
          win[g][lt][2 * r + 1] = make_float4(y[r][4], y[r][5], y[r][6], y[r][7]);
        }
        __syncthreads();
      } else {
        OutT* col = out + ((int64_t)j * (n + 1) + c) * n;
#pragma unroll
        for (int r = 0; r < kAdvB; ++r) adv_store_row(col + (iy0 + r) * kAdvNx + ix0, y[r]);
      }
    }
    __syncthreads();                           // the windows are rewritten next
  }
}

// The float64 build with the first steps on windows, in the strip layout of
// advdiff_affine_kernel.  As in advdiff_window_kernel, after k steps the
// column from the unit point (cx, cy) is exactly zero outside the periodic
// diamond |x - cx| + |y - cy| <= 4k.  A window of rows cy - a .. cy - a + H - 1
// that holds the diamond after the last of its steps, k_e (a >= 4 k_e and
// H - 1 - a >= 4 k_e), also has its cut halo rows at distance >= 4 k_e, where
// every stage that reads them (the first 4 k_e) reads the exact zero; the
// same holds in x.  So:
//   phase 0  the first m1 <= 3 steps on the 32 x 32 window with origin
//            (cx - 16, cy - 16) (mod 64), four columns per CTA, 32/R warps each
//            (warp g (32/R) + s holds rows R s .. R s + R - 1 of column g's
//            window at window column x = lane; x-neighbours by shuffles, zero at
//            the window's side edges; the strips' facing rows through the
//            shared top / bottom rows, a zero slot at the window's top and
//            bottom edges);
//   ladder   then, column by column, each step i on the whole periodic width
//            but only the H(i) rows around cy, H(i) the least multiple of R
//            holding 8 (i + 1) + 1 rows (R = 8: 40, 48, 56 rows for steps 4, 5,
//            6; R = 16: 48 rows for steps 4 and 5), a = H/2, the strips of
//            the window active and the others idle (warp-uniform);
//   full     the remaining steps on the whole grid, in exactly
//            advdiff_affine_kernel's layout.
// Each phase starts from the previous one's window staged in shared memory
// (the 32 x 32 windows, or a 64 x 64 grid buffer), zeros outside it.  Every
// point is the same floating-point expression as in the whole-grid kernel, and
// the zeros are exact, so the maps are bit for bit the same; the point-steps
// per column fall from 4096 m to 1024 m1 + 64 (H(m1) + ... ) for the ladder
// steps + 4096 for each full step.
// Strip height R (rows per thread): 16 (256 threads), 8 (512) or 32 (128).
// Thread t's top / bottom row slot is t in every phase: row block b is threads
// 64 b .. 64 b + 63, window strip s of column g is warp g (32/R) + s.  Shared
// memory (dynamic): two buffers of 64 NB + 1 top and bottom rows (the last slot
// stays zero), the edge-lane strips of every warp, the four 32 x 32 windows,
// the 64 x 64 grid buffer of the ladder.
template <int R>
struct AdvWin64Shape {
  static constexpr int NB = kAdvNx / R;               // row blocks of the grid
  static constexpr int THREADS = kAdvNx * NB;         // 256, 512 or 128
  static constexpr int NW = THREADS / 32;
  static constexpr int WPC = 32 / R;                  // warps per window
  static constexpr int ROWS = kAdvNx * NB + 1;        // row slots per buffer, zero slot last
  static constexpr size_t SMEM = sizeof(double) * (2 * 2 * (size_t)ROWS + 2 * (size_t)NW * 2 * R +
                                                   4 * 32 * 32 + (size_t)kAdvNx * kAdvNx);
};

// Rows of the ladder window of step i (0-based): the least multiple of R
// holding 8 (i + 1) + 1 rows, at most the whole grid (host and device).
template <int R>
__host__ __device__ __forceinline__ int adv_ladder_rows(int64_t i) {
  const int64_t need = 8 * (i + 1) + 1;
  const int64_t h = (need + R - 1) / R * R;
  return h >= kAdvNx ? kAdvNx : (int)h;
}

template <int R>
__global__ void __launch_bounds__(AdvWin64Shape<R>::THREADS) advdiff_window64_kernel(AdvArgs a, int m1,
                                                                                     int ladder) {
  using Sh = AdvWin64Shape<R>;
  constexpr int n = kAdvNx * kAdvNx;
  constexpr int NB = Sh::NB, WPC = Sh::WPC, ROWS = Sh::ROWS, RING = kAdvNx * NB;
  constexpr int kZ = RING;                     // zero slot
  extern __shared__ __align__(16) double adv64_smem[];
  double* top = adv64_smem;                    // [2][ROWS]
  double* bot = top + 2 * ROWS;                // [2][ROWS]
  double* edge = bot + 2 * ROWS;               // [2][NW][2][R]
  double* win = edge + 2 * Sh::NW * 2 * R;     // [4][32][32]
  double* grid = win + 4 * 32 * 32;            // [64][64], the ladder's staging
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ix = tid % kAdvNx, blk = tid / kAdvNx;                   // grid strip layout
  const int g = warp / WPC, s = warp % WPC;                          // window layout
  const int pw = warp ^ 1;
  if (tid < 2) {
    top[tid * ROWS + kZ] = 0.0;
    bot[tid * ROWS + kZ] = 0.0;
  }
  double* out = reinterpret_cast<double*>(a.out);
  const int64_t total = (int64_t)a.S * (n + 1);
  int buf = 0;
  for (int64_t w = blockIdx.x; w * 4 < total; w += gridDim.x) {
    // One loop over the group's phases, so that the unrolled step body appears
    // once: gc = -1 is phase 0 (the four 32 x 32 windows), then each column gc
    // runs its ladder phases and its whole-grid phase.
    int gc = -1, sy = 0, sh = 0;       // sh = 0: the previous window is the column's 32 x 32 one
    int64_t i = 0;
#pragma unroll 1
    for (;;) {
      const bool p0 = gc < 0;
      const int64_t idx = w * 4 + (p0 ? g : gc);
      if (!p0 && idx >= total) break;  // uniform over the CTA
      const int j = idx < total ? (int)(idx / (n + 1)) : 0;
      const int c = idx < total ? (int)(idx - (int64_t)j * (n + 1)) : 0;   // 0: no unit point
      const int cx = c >= 1 ? (c - 1) % kAdvNx : 0, cy = c >= 1 ? (c - 1) / kAdvNx : 0;
      const int wx0 = (cx + kAdvNx - 16) % kAdvNx, wy0 = (cy + kAdvNx - 16) % kAdvNx;
      int H, wy, abv, blw;
      int64_t count;
      bool active, cut_x;
      double y[R];
      if (p0) {
        H = 32;
        wy = wy0;
        count = m1;
        active = true;
        cut_x = true;
        abv = s > 0 ? tid - 32 : kZ;
        blw = s < WPC - 1 ? tid + 32 : kZ;
        const int gx = (wx0 + lane) % kAdvNx;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int gy = (wy0 + R * s + r) % kAdvNx;
          y[r] = (c >= 1 && gy * kAdvNx + gx == c - 1) ? 1.0 : 0.0;
        }
      } else {
        H = (ladder && i < a.m) ? adv_ladder_rows<R>(i) : kAdvNx;
        int64_t iend = i;
        while (iend < a.m && (ladder ? adv_ladder_rows<R>(iend) : kAdvNx) == H) ++iend;
        count = iend - i;
        i = iend;
        const bool full = H == kAdvNx;
        wy = full ? 0 : (cy - H / 2 + kAdvNx) % kAdvNx;
        const int strips = H / R;
        active = blk < strips;
        cut_x = false;
        abv = full ? (tid + RING - kAdvNx) % RING : (blk > 0 ? tid - kAdvNx : kZ);
        blw = full ? (tid + kAdvNx) % RING : (blk < strips - 1 ? tid + kAdvNx : kZ);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int gy = (wy + R * blk + r) % kAdvNx;
          double v = 0.0;
          if (sh == 0) {
            const int wx = (ix - wx0 + kAdvNx) % kAdvNx, wyy = (gy - wy0 + kAdvNx) % kAdvNx;
            if (wx < 32 && wyy < 32) v = win[(gc * 32 + wyy) * 32 + wx];
          } else if ((gy - sy + kAdvNx) % kAdvNx < sh) {
            v = grid[gy * kAdvNx + ix];
          }
          y[r] = v;
        }
      }
      for (int64_t it = 0; it < count; ++it) {
        double v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = y[r];
#pragma unroll
        for (int kk = 4; kk >= 1; --kk) {
          const double* cw = a.cw64[4 - kk];
          const double cxm = cw[0], cxp = cw[1], cym = cw[2], cyp = cw[3], c0 = cw[4];
          double* topb = top + buf * ROWS;
          double* botb = bot + buf * ROWS;
          double* edgeb = edge + buf * Sh::NW * 2 * R;
          topb[tid] = v[0];
          botb[tid] = v[R - 1];
          if (lane == 0 || lane == 31) {
#pragma unroll
            for (int r = 0; r < R; ++r) edgeb[(warp * 2 + (lane == 31)) * R + r] = v[r];
          }
          __syncthreads();
          if (active) {                          // uniform over each warp
            const double above = botb[abv], below = topb[blw];
            double nv[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
              double xm = __shfl_up_sync(0xffffffffu, v[r], 1);
              double xp = __shfl_down_sync(0xffffffffu, v[r], 1);
              if (lane == 0) xm = cut_x ? 0.0 : edgeb[(pw * 2 + 1) * R + r];
              if (lane == 31) xp = cut_x ? 0.0 : edgeb[(pw * 2 + 0) * R + r];
              const double ym = r == 0 ? above : v[r - 1];
              const double yp = r == R - 1 ? below : v[r + 1];
              double acc = fma(c0, v[r], y[r]);
              acc = fma(cxm, xm, acc);
              acc = fma(cxp, xp, acc);
              acc = fma(cym, ym, acc);
              nv[r] = fma(cyp, yp, acc);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = nv[r];
          }
          buf ^= 1;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) y[r] = v[r];
      }
      if (p0) {
#pragma unroll
        for (int r = 0; r < R; ++r) win[(g * 32 + R * s + r) * 32 + lane] = y[r];
        __syncthreads();
        gc = 0;
        i = m1;
        sh = 0;
      } else if (H == kAdvNx) {
        double* col = out + ((int64_t)j * (n + 1) + c) * n;
#pragma unroll
        for (int r = 0; r < R; ++r) col[(R * blk + r) * kAdvNx + ix] = y[r];
        ++gc;
        if (gc == 4) break;
        i = m1;
        sh = 0;
      } else {
        // every thread loaded the previous window before this phase's first
        // block barrier (a ladder phase has at least one step)
        if (active) {
#pragma unroll
          for (int r = 0; r < R; ++r) grid[((wy + R * blk + r) % kAdvNx) * kAdvNx + ix] = y[r];
        }
        __syncthreads();
        sy = wy;
        sh = H;
      }
    }
    __syncthreads();                           // the windows are rewritten next
  }
}

template <int R>
static nv_status launch_adv_window64(const AdvArgs& a, int m1, int ladder, int64_t cols, cudaStream_t s) {
  using Sh = AdvWin64Shape<R>;
  nv_status st = nv_cuda_check(cudaFuncSetAttribute(advdiff_window64_kernel<R>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM),
                               "window kernel shared memory attribute");
  if (st != NV_OK) return st;
  int dev = 0, sms = 0, per_sm = 0;
  if ((st = nv_cuda_check(cudaGetDevice(&dev), "current device")) != NV_OK) return st;
  if ((st = nv_cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count")) != NV_OK)
    return st;
  if ((st = nv_cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, advdiff_window64_kernel<R>,
                                                                        Sh::THREADS, Sh::SMEM),
                          "occupancy query")) != NV_OK)
    return st;
  const int64_t work = (cols + 3) / 4;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(work, (int64_t)sms * std::max(per_sm, 1)));
  advdiff_window64_kernel<R><<<grid, Sh::THREADS, Sh::SMEM, s>>>(a, m1, ladder);
  return nv_cuda_check(cudaGetLastError(), "advdiff_window64_kernel launch");
}

// Serial fine solve of the advection-diffusion system (one CTA, S*m steps).
template <typename T>
__global__ void __launch_bounds__(256) advdiff_serial_kernel(AdvArgs a, const double* y0, double* yT) {
  __shared__ AdvStripSmem<T> sm;
  const int tid = threadIdx.x;
  const int ix = tid % kAdvNx, blk = tid / kAdvNx, iy0 = blk * kAdvRows;
  T y[kAdvRows];
#pragma unroll
  for (int r = 0; r < kAdvRows; ++r) y[r] = (T)y0[(iy0 + r) * kAdvNx + ix];
  AdvArgs all = a;
  all.m = (int64_t)a.S * a.m;                  // every slice's steps in one run
  adv_strip_integrate<T>(all, y, sm);
#pragma unroll
  for (int r = 0; r < kAdvRows; ++r) yT[(iy0 + r) * kAdvNx + ix] = (double)y[r];
}

}  // namespace nvpit

using namespace nvpit;

static AdvArgs adv_args(const nv_maps* M) {
  AdvArgs a{};
  a.out = M->data;
  a.S = M->S;
  a.m = M->m;
  a.h = M->h;
  const double nu = M->params[0], ax = M->params[1], ay = M->params[2];
  const double dx = 1.0 / kAdvNx;
  a.w_xm = nu / (dx * dx) + ax / dx;
  a.w_xp = nu / (dx * dx);
  a.w_ym = nu / (dx * dx) + ay / dx;
  a.w_yp = nu / (dx * dx);
  a.w_0 = -4.0 * nu / (dx * dx) - ax / dx - ay / dx;
  const double w[5] = {a.w_xm, a.w_xp, a.w_ym, a.w_yp, a.w_0};
  for (int st = 0; st < 4; ++st) {
    for (int q = 0; q < 5; ++q) {
      a.cw64[st][q] = (a.h / (4 - st)) * w[q];
      a.cw32[st][q] = (float)a.cw64[st][q];
    }
    // The periodic operator maps constants to zero (its weights sum to 0), so
    // the mean is conserved; the float32 stage weights rounded one by one sum
    // to about 1e-9 instead, and every stage then scales the mean by that (a
    // float32 fine integration of the 5 120 steps drifts by 1.4e-5 from the
    // float64 one that way, by 5e-7 without).  So the centre weight is minus
    // the exact sum of the other four, which must itself be a float32: the
    // sum of four float32 values is exact in double, and the last neighbour
    // weight moves by single ulps (at most a few) until that sum rounds to
    // float32 exactly.  (The composed float32 maps err by 8.6e-5 either way:
    // there the maps' own float32 entries and the chain's sums dominate.)
    float* c = a.cw32[st];
    const float base = c[3];
    for (int k = 0; k < 64; ++k) {
      const int d = (k + 1) / 2 * ((k & 1) ? 1 : -1);   // 0, +1, -1, +2, -2, ... ulps
      float c3 = base;
      for (int i = 0; i < (d > 0 ? d : -d); ++i) c3 = nextafterf(c3, d > 0 ? INFINITY : -INFINITY);
      const double s4 = (double)c[0] + (double)c[1] + (double)c[2] + (double)c3;
      if ((double)(float)s4 == s4) {
        c[3] = c3;
        c[4] = -(float)s4;
        break;
      }
    }
  }
  return a;
}

nv_status launch_advdiff_build(nv_maps* M, cudaStream_t s) {
  if (M->dim != kAdvNx * kAdvNx) return nv_fail(NV_ENOTSUP, "advection-diffusion is built for a 64 x 64 grid");
  if (M->scheme != NV_RK4) return nv_fail(NV_ENOTSUP, "affine maps are built with RK4");
  const AdvArgs a = adv_args(M);
  int grid = 0;
  nv_status st;
  const int64_t cols = (int64_t)M->S * (M->dim + 1);
  if (M->prec == NV_FP64) {
    // windows for the first min(m, 3) steps unless the whole-grid form is asked for
    const int m1 = g_tune.adv_build_form == 1 ? 0 : (int)std::min<int64_t>(M->m, 3);
    if (m1 > 0) {
      // strip height: 16 rows (256 threads) unless key 16 asks for 8 or 32;
      // the ladder of row windows after the first steps unless key 15 = 2
      const int R = g_tune.adv_fp64_rows == 8 || g_tune.adv_fp64_rows == 32 ? g_tune.adv_fp64_rows : 16;
      const int ladder = g_tune.adv_build_form == 2 ? 0 : 1;
      int64_t per_col = 1024 * (int64_t)m1;
      for (int64_t i = m1; i < M->m; ++i) {
        const int H = !ladder ? kAdvNx : R == 8 ? adv_ladder_rows<8>(i) : R == 16 ? adv_ladder_rows<16>(i)
                                                                            : adv_ladder_rows<32>(i);
        per_col += (int64_t)kAdvNx * H;
      }
      M->work_per_slice = (int64_t)(M->dim + 1) * per_col;
      snprintf(M->build_kernel, sizeof(M->build_kernel), "advdiff_window64_kernel<%d>", R);
      if (R == 32) return launch_adv_window64<32>(a, m1, ladder, cols, s);
      return R == 8 ? launch_adv_window64<8>(a, m1, ladder, cols, s) : launch_adv_window64<16>(a, m1, ladder, cols, s);
    } else {
      M->work_per_slice = (int64_t)(M->dim + 1) * M->dim * M->m;
      snprintf(M->build_kernel, sizeof(M->build_kernel), "advdiff_affine_kernel<double>");
      st = persistent_grid(advdiff_affine_kernel<double>, 256, cols * 8, &grid);
      if (st != NV_OK) return st;
      advdiff_affine_kernel<double><<<grid, 256, 0, s>>>(a);
    }
  } else {
    // columns start at j * (n + 1) * n values: 16-byte aligned for the
    // vector stores since n = 4096 and the map buffer is 256-byte aligned
    // windows for the first min(m, 3) steps unless the whole-grid form is asked for
    const int m1 = g_tune.adv_build_form == 1 ? 0 : (int)std::min<int64_t>(M->m, 3);
    const char* out_t = M->prec == NV_BF16_REFINE ? "uint16_t" : "float";
    M->work_per_slice = (int64_t)(M->dim + 1) * (1024 * m1 + (int64_t)M->dim * (M->m - m1));
    snprintf(M->build_kernel, sizeof(M->build_kernel), m1 > 0 ? "advdiff_window_kernel<%s>" : "advdiff_block_kernel<%s>",
             out_t);
    if (m1 > 0 && M->prec == NV_BF16_REFINE) {
      st = persistent_grid(advdiff_window_kernel<uint16_t>, kAdvBlockThreads, cols / 2 + 2, &grid);
      if (st != NV_OK) return st;
      advdiff_window_kernel<uint16_t><<<grid, kAdvBlockThreads, 0, s>>>(a, m1);
    } else if (m1 > 0) {
      st = persistent_grid(advdiff_window_kernel<float>, kAdvBlockThreads, cols / 2 + 2, &grid);
      if (st != NV_OK) return st;
      advdiff_window_kernel<float><<<grid, kAdvBlockThreads, 0, s>>>(a, m1);
    } else if (M->prec == NV_BF16_REFINE) {
      st = persistent_grid(advdiff_block_kernel<uint16_t>, kAdvBlockThreads, cols * 2, &grid);
      if (st != NV_OK) return st;
      advdiff_block_kernel<uint16_t><<<grid, kAdvBlockThreads, 0, s>>>(a);
    } else {
      st = persistent_grid(advdiff_block_kernel<float>, kAdvBlockThreads, cols * 2, &grid);
      if (st != NV_OK) return st;
      advdiff_block_kernel<float><<<grid, kAdvBlockThreads, 0, s>>>(a);
    }
  }
  return nv_cuda_check(cudaGetLastError(), "advdiff_affine_kernel launch");
}

nv_status launch_serial_advdiff(const nv_maps* M, const double* y0, double* yT, cudaStream_t s) {
  if (M->dim != kAdvNx * kAdvNx) return nv_fail(NV_ENOTSUP, "advection-diffusion is built for a 64 x 64 grid");
  const AdvArgs a = adv_args(M);
  advdiff_serial_kernel<double><<<1, 256, 0, s>>>(a, y0, yT);
  return nv_cuda_check(cudaGetLastError(), "advdiff_serial_kernel launch");
}

nv_status launch_advdiff_defect(const nv_maps* M, const double* lam, double* d, cudaStream_t s) {
  if (M->dim != kAdvNx * kAdvNx) return nv_fail(NV_ENOTSUP, "advection-diffusion is built for a 64 x 64 grid");
  const AdvArgs a = adv_args(M);
  int grid = 0;
  nv_status st = persistent_grid(advdiff_defect_kernel, 256, (int64_t)M->S * 8, &grid);
  if (st != NV_OK) return st;
  advdiff_defect_kernel<<<grid, 256, 0, s>>>(a, lam, d);
  return nv_cuda_check(cudaGetLastError(), "advdiff_defect_kernel launch");
}
