// Heat-equation device code shared by the map build (affine.cu) and the
// pipelined refinement (wavefront.cu): the argument block, the lane-blocked
// stencil stages and the literal RK4 step of u_t = a(t) u_xx + g(t) sin(pi x)
// (Sections 4.2 and 4.3: the forced and the variable-coefficient heat
// equations), and the float64 defect of one slice.
#pragma once

#include "common.cuh"

namespace nvpit {

struct HeatArgs {
  void* out;
  int n, S, rows_valid_full;
  int64_t m;
  double t0, H, h;
  double kappa, amp;     // NV_RHS_HEAT1D parameters
  int varcoef;           // NV_RHS_HEAT1D_VARCOEF
  double poly9[5];       // nine-point form of the RK4 step: weights c_0..c_4
};

// Neighbour values of a lane-blocked vector: left of row lane*R, right of row
// lane*R+R-1 (zero at the Dirichlet boundary and past the last row).
template <int R, typename T>
__device__ __forceinline__ void halos(const T* v, int lane, int n, T& left, T& right) {
  left = __shfl_up_sync(0xffffffffu, v[R - 1], 1);
  right = __shfl_down_sync(0xffffffffu, v[0], 1);
  if (lane == 0) left = (T)0;
  if (lane == 31 || (lane + 1) * R >= n) right = (T)0;
}

// One Horner-form RK4 step of y' = cdx * lap(y), lap the [1,-2,1] stencil.
template <int R, typename T>
__device__ __forceinline__ void heat_horner_step(T* y, T* v, T cdx, T h, int lane, int n) {
#pragma unroll
  for (int i = 0; i < R; ++i) v[i] = y[i];
#pragma unroll
  for (int kk = 4; kk >= 1; --kk) {
    const T ck = (h / (T)kk) * cdx;
    T prev, right;
    halos<R>(v, lane, n, prev, right);
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const T cur = v[i];
      const T nxt = (i + 1 < R) ? v[i + 1] : right;
      T s = prev + nxt;
      s = fma((T)-2, cur, s);
      v[i] = fma(ck, s, y[i]);
      prev = cur;
    }
    if ((lane + 1) * R > n) {  // padding rows stay zero
#pragma unroll
      for (int i = 0; i < R; ++i)
        if (lane * R + i >= n) v[i] = (T)0;
    }
  }
#pragma unroll
  for (int i = 0; i < R; ++i) y[i] = v[i];
}

// Right-hand side f(t, z) = a(t) cdx lap(z) + g(t) sx at one stage, folded into
// the stage updates of the literal RK4 step.
template <int R, typename T>
__device__ __forceinline__ void heat_stage(const T* y, T* z, T* acc, T a_cdx, T g, const T* sx,
                                           bool forced, T zc, T accw, bool first, int lane,
                                           int n) {
  T prev, right;
  halos<R>(z, lane, n, prev, right);
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const T cur = z[i];
    const T nxt = (i + 1 < R) ? z[i + 1] : right;
    T s = prev + nxt;
    s = fma((T)-2, cur, s);
    T k = a_cdx * s;
    if (forced) k = fma(g, sx[i], k);
    acc[i] = first ? k : fma(accw, k, acc[i]);
    z[i] = fma(zc, k, y[i]);
    prev = cur;
  }
  if ((lane + 1) * R > n) {
#pragma unroll
    for (int i = 0; i < R; ++i)
      if (lane * R + i >= n) z[i] = (T)0;
  }
}

__device__ __forceinline__ double heat_a(int varcoef, double t) {
  return varcoef ? 1.0 + 0.25 * sin(t) : 1.0;
}
// forcing amplitude g(t) multiplying sin(pi x)
__device__ __forceinline__ double heat_g(int varcoef, double amp, double t) {
  if (!varcoef) return amp * cos(t);
  const double a = 1.0 + 0.25 * sin(t);
  return -sin(t) + a * (M_PI * M_PI) * cos(t);
}

// Time-dependent coefficients of one literal RK4 step, at t, t+h/2, t+h:
// forcing amplitudes g and diffusion coefficients a(t) cdx.
template <typename T>
struct StageCoefs {
  T g0, gh, g1, a0, ah, a1;
};

// Coefficients of the steps i0 .. i0+15 of a slice starting at Tj: lane l
// evaluates the half-step time q = 2 i0 + l (l <= 30; l = 31 idles) once, and
// the steps read them by shuffle, so the trigonometric calls run once per
// warp instead of once per lane.
struct HalfStepCoefs {
  double g, a;
};

__device__ __forceinline__ HalfStepCoefs half_step_coefs(const HeatArgs& a, double Tj, int64_t i0,
                                                         int lane) {
  const int64_t q = 2 * i0 + lane;
  const int64_t i = q >> 1;
  double t = __dadd_rn(Tj, __dmul_rn((double)i, a.h));
  if (q & 1) t = __dadd_rn(t, 0.5 * a.h);
  HalfStepCoefs c;
  c.g = heat_g(a.varcoef, a.amp, t);
  c.a = heat_a(a.varcoef, t);
  return c;
}

template <typename T>
__device__ __forceinline__ StageCoefs<T> step_coefs(const HalfStepCoefs& hc, int64_t i, int64_t i0,
                                                    T cdx) {
  const int l = (int)(2 * (i - i0));
  StageCoefs<T> c;
  c.g0 = (T)__shfl_sync(0xffffffffu, hc.g, l);
  c.gh = (T)__shfl_sync(0xffffffffu, hc.g, l + 1);
  c.g1 = (T)__shfl_sync(0xffffffffu, hc.g, l + 2);
  c.a0 = (T)__shfl_sync(0xffffffffu, hc.a, l) * cdx;
  c.ah = (T)__shfl_sync(0xffffffffu, hc.a, l + 1) * cdx;
  c.a1 = (T)__shfl_sync(0xffffffffu, hc.a, l + 2) * cdx;
  return c;
}

// Literal RK4 step (stage times t, t+h/2, t+h) for the heat right-hand side.
template <int R, typename T>
__device__ __forceinline__ void heat_rk4_step(T* y, T* z, T* acc, double h, const StageCoefs<T>& c,
                                              const T* sx, bool forced, int lane, int n) {
  const T hh = (T)(0.5 * h), hT = (T)h;
  const T g0 = forced ? c.g0 : (T)0, gh = forced ? c.gh : (T)0, g1 = forced ? c.g1 : (T)0;
  const T a0 = c.a0, ah = c.ah, a1 = c.a1;
#pragma unroll
  for (int i = 0; i < R; ++i) z[i] = y[i];
  heat_stage<R>(y, z, acc, a0, g0, sx, forced, hh, (T)0, true, lane, n);
  heat_stage<R>(y, z, acc, ah, gh, sx, forced, hh, (T)2, false, lane, n);
  heat_stage<R>(y, z, acc, ah, gh, sx, forced, hT, (T)2, false, lane, n);
  // stage 4: k4 = f(t+h, z); y <- y + h/6 (acc + k4)
  {
    T prev, right;
    halos<R>(z, lane, n, prev, right);
    const T h6 = (T)(h / 6.0);
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const T cur = z[i];
      const T nxt = (i + 1 < R) ? z[i + 1] : right;
      T s = prev + nxt;
      s = fma((T)-2, cur, s);
      T k = a1 * s;
      if (forced) k = fma(g1, sx[i], k);
      y[i] = fma(h6, acc[i] + k, y[i]);
      prev = cur;
    }
    if ((lane + 1) * R > n) {
#pragma unroll
      for (int i = 0; i < R; ++i)
        if (lane * R + i >= n) y[i] = (T)0;
    }
  }
}

// Float64 defect of slice j (the residual correction the Conclusion
// proposes): d_j = g^j(lt_j) - lt_{j+1}, one literal RK4 fine solve of the
// forced equation from lt_j over the slice.  One warp; lane l holds rows
// l*R .. l*R+R-1.
template <int R>
__device__ __forceinline__ void heat_defect_slice(const HeatArgs& a, const double* lt, double* d, int64_t j,
                                                  int lane) {
  const int n = a.n;
  const double dx = 1.0 / (double)(n + 1);
  const double cdx = a.kappa / (dx * dx);
  const double Tj = __dadd_rn(a.t0, __dmul_rn((double)j, a.H));
  double y[R], z[R], acc[R], sx[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int r = lane * R + i;
    y[i] = r < n ? lt[j * n + r] : 0.0;
    sx[i] = r < n ? sin(M_PI * ((double)(r + 1) / (double)(n + 1))) : 0.0;
  }
  HalfStepCoefs hc{};
  for (int64_t i = 0; i < a.m; ++i) {
    const int64_t i0 = i - (i % 15);
    if (i == i0) hc = half_step_coefs(a, Tj, i0, lane);
    heat_rk4_step<R>(y, z, acc, a.h, step_coefs<double>(hc, i, i0, cdx), sx, true, lane, n);
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int r = lane * R + i;
    if (r < n) d[j * n + r] = y[i] - lt[(j + 1) * n + r];
  }
}

}  // namespace nvpit

// Host: the argument block of the heat kernels for maps M (affine.cu).
struct nv_maps;
nvpit::HeatArgs heat_args(const nv_maps* M);
