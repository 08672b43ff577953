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
  float poly9f[5];       // the same rounded to float32, with c_0 + 2 (c_1 + .. + c_4) = 1
};

template <typename T>
__device__ __forceinline__ T poly9_weight(const HeatArgs& a, int k);
template <>
__device__ __forceinline__ double poly9_weight<double>(const HeatArgs& a, int k) { return a.poly9[k]; }
template <>
__device__ __forceinline__ float poly9_weight<float>(const HeatArgs& a, int k) { return a.poly9f[k]; }

// Neighbour values of a lane-blocked vector: left of row lane*R, right of row
// lane*R+R-1 (zero at the Dirichlet boundary and past the last row).
template <int R, typename T>
__device__ __forceinline__ void halos(const T* v, int lane, int n, T& left, T& right) {
  left = __shfl_up_sync(0xffffffffu, v[R - 1], 1);
  right = __shfl_down_sync(0xffffffffu, v[0], 1);
  if (lane == 0) left = (T)0;
  if (lane == 31 || (lane + 1) * R >= n) right = (T)0;
}

// Halo policy of the literal RK4 step: one warp holds the whole vector (lane
// l: rows l*R .. l*R+R-1).
struct WarpHalo {
  int lane;
  __device__ int gl() const { return lane; }   // lane index within the whole vector
  template <int R, typename T>
  __device__ __forceinline__ void operator()(const T* v, int n, T& left, T& right) {
    halos<R>(v, lane, n, left, right);
  }
};

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
template <int R, typename T, typename H>
__device__ __forceinline__ void heat_stage(const T* y, T* z, T* acc, T a_cdx, T g, const T* sx,
                                           bool forced, T zc, T accw, bool first, H& halo,
                                           int n) {
  const int lane = halo.gl();
  T prev, right;
  halo.template operator()<R>(z, n, prev, right);
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
// Spatial shape of the forcing, sin(pi x_r) at x_r = (r+1)/(n+1): the same
// for every slice and column, so the kernels that integrate many forced
// columns tabulate it once per CTA (forcing_table) instead of per lane and
// column: float64 sines run at the FP64 rate.
__device__ __forceinline__ double forcing_shape(int r, int n) {
  return sin(M_PI * ((double)(r + 1) / (double)(n + 1)));
}

// Fill tab[0 .. n-1] with forcing_shape; every thread of the CTA must call it.
__device__ __forceinline__ void forcing_table(double* tab, int n) {
  for (int r = threadIdx.x; r < n; r += blockDim.x) tab[r] = forcing_shape(r, n);
  __syncthreads();
}

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
template <int R, typename T, typename H>
__device__ __forceinline__ void heat_rk4_step(T* y, T* z, T* acc, double h, const StageCoefs<T>& c,
                                              const T* sx, bool forced, H& halo, int n) {
  const int lane = halo.gl();
  const T hh = (T)(0.5 * h), hT = (T)h;
  const T g0 = forced ? c.g0 : (T)0, gh = forced ? c.gh : (T)0, g1 = forced ? c.g1 : (T)0;
  const T a0 = c.a0, ah = c.ah, a1 = c.a1;
#pragma unroll
  for (int i = 0; i < R; ++i) z[i] = y[i];
  heat_stage<R>(y, z, acc, a0, g0, sx, forced, hh, (T)0, true, halo, n);
  heat_stage<R>(y, z, acc, ah, gh, sx, forced, hh, (T)2, false, halo, n);
  heat_stage<R>(y, z, acc, ah, gh, sx, forced, hT, (T)2, false, halo, n);
  // stage 4: k4 = f(t+h, z); y <- y + h/6 (acc + k4)
  {
    T prev, right;
    halo.template operator()<R>(z, n, prev, right);
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

template <int R, typename T>
__device__ __forceinline__ void heat_rk4_step(T* y, T* z, T* acc, double h, const StageCoefs<T>& c,
                                              const T* sx, bool forced, int lane, int n) {
  WarpHalo halo{lane};
  heat_rk4_step<R>(y, z, acc, h, c, sx, forced, halo, n);
}

// One RK4 step of u' = a(t) cdx T u + g(t) s in nine-point form.  T (the
// [1,-2,1] stencil with zero ends) has s = sin(pi x) as an eigenvector, T s =
// lam s with lam = -4 sin^2(pi/(2(n+1))), and the step's operators a(.) cdx T
// all commute, so the classical RK4 step is exactly Q(T) u + phi s: Q the
// degree-4 polynomial of the four stages in T, with the stage multipliers u0,
// uh, u1 = h a(t) cdx at t, t+h/2, t+h, written as the weights c0..c4 of a
// symmetric nine-point stencil; phi the same four stages run on the forcing's
// coefficient along s.  (With a constant, Q is the Taylor polynomial of
// degree 4 of the build's nine-point form.)  The stencil is applied in
// difference form, y + sum_k c_k (y_{i-k} + y_{i+k} - 2 y_i): the weights
// c_1..c_4 act on second differences, as the literal stages do, so that
// rounding the weights cannot change the step's action on smooth vectors.
// (With c_0 = 1 - 2 (c_1 + .. + c_4) stored as a rounded weight of its own,
// the smooth mode's factor per step differs from the exact one by about an
// ulp, and over the 10 240 steps of the heat workload the fine solve drifts
// by 7e-13 from the literal stages; in difference form the two agree to
// 4e-16.)
struct Rk4Poly9 {
  double c1, c2, c3, c4, phi;
};

__device__ __forceinline__ Rk4Poly9 rk4_poly9(double h, double u0, double uh, double u1, double g0, double gh,
                                              double g1, double lam) {
  const double q1 = (u0 + 4.0 * uh + u1) / 6.0;
  const double q2 = uh * (u0 + uh + u1) / 6.0;
  const double q3 = uh * uh * (u0 + u1) / 12.0;
  const double q4 = u0 * uh * uh * u1 / 24.0;
  Rk4Poly9 p;
  p.c1 = q1 - 4.0 * q2 + 15.0 * q3 - 56.0 * q4;
  p.c2 = q2 - 6.0 * q3 + 28.0 * q4;
  p.c3 = q3 - 8.0 * q4;
  p.c4 = q4;
  const double k1 = g0;
  const double k2 = gh + 0.5 * uh * lam * k1;
  const double k3 = gh + 0.5 * uh * lam * k2;
  const double k4 = g1 + u1 * lam * k3;
  p.phi = h / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4);
  return p;
}

__device__ __forceinline__ double shfl_d(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// One RK4 fine solve of the forced equation over slice j, float64, from the
// state in y (one warp; lane l holds rows l*R .. l*R+R-1; rows past n - 1
// hold 0).  Where every lane holds 4 to 8 whole rows (4 <= R <= 8,
// n % R == 0) the steps take the nine-point form (13 instead of 24 float64
// operations per row and step: the stencil's weights and phi for steps
// i0 .. i0+14 are computed one step per lane and broadcast by shuffle);
// otherwise the literal stages.
template <int R>
__device__ __forceinline__ void heat_forced_solve(const HeatArgs& a, double (&y)[R], int64_t j, int lane,
                                                  const double* sxt = nullptr) {
  const int n = a.n;
  const double dx = 1.0 / (double)(n + 1);
  const double cdx = a.kappa / (dx * dx);
  const double Tj = __dadd_rn(a.t0, __dmul_rn((double)j, a.H));
  double sx[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int r = lane * R + i;
    sx[i] = r < n ? (sxt ? sxt[r] : forcing_shape(r, n)) : 0.0;
  }
  HalfStepCoefs hc{};
  // (R = 16, d > 256: the nine-point halo would not fit the registers)
  if (R >= 4 && R <= 8 && n % R == 0) {
    const int last = n / R - 1;                   // lane holding row n-1
    // 2 cos(pi/(n+1)) - 2 = -4 sin^2(pi/(2(n+1))), the second form without
    // the cancellation that would cost the first one ~1e-12 relative accuracy
    const double sh = sin(M_PI / (2.0 * (double)(n + 1)));
    const double lam = -4.0 * sh * sh;
    Rk4Poly9 pl{};
    for (int64_t i = 0; i < a.m; ++i) {
      const int64_t i0 = i - (i % 15);
      if (i == i0) {                              // lane l: step i0 + l (l < 15)
        hc = half_step_coefs(a, Tj, i0, lane);
        const int l2 = min(2 * lane, 28);
        const double g0 = shfl_d(hc.g, l2), gh = shfl_d(hc.g, l2 + 1), g1 = shfl_d(hc.g, l2 + 2);
        const double a0 = shfl_d(hc.a, l2), ah = shfl_d(hc.a, l2 + 1), a1 = shfl_d(hc.a, l2 + 2);
        pl = rk4_poly9(a.h, a.h * (a0 * cdx), a.h * (ah * cdx), a.h * (a1 * cdx), g0, gh, g1, lam);
      }
      const int src = (int)(i - i0);
      const double c1 = shfl_d(pl.c1, src), c2 = shfl_d(pl.c2, src);
      const double c3 = shfl_d(pl.c3, src), c4 = shfl_d(pl.c4, src), phi = shfl_d(pl.phi, src);
      double e[R + 8];                            // rows lane*R-4 .. lane*R+R+3
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        e[q] = __shfl_up_sync(0xffffffffu, y[R - 4 + q], 1);
        e[R + 4 + q] = __shfl_down_sync(0xffffffffu, y[q], 1);
      }
      if (lane == 0) {                            // rows -4..-1 = -y2, -y1, -y0, 0 (odd reflection)
        e[0] = -y[2];
        e[1] = -y[1];
        e[2] = -y[0];
        e[3] = 0.0;
      }
      if (lane == last) {                         // rows n..n+3 = 0, -y_{n-1}, -y_{n-2}, -y_{n-3}
        e[R + 4] = 0.0;
        e[R + 5] = -y[R - 1];
        e[R + 6] = -y[R - 2];
        e[R + 7] = -y[R - 3];
      }
#pragma unroll
      for (int i2 = 0; i2 < R; ++i2) e[i2 + 4] = y[i2];
#pragma unroll
      for (int i2 = 0; i2 < R; ++i2) {
        const double yc = e[i2 + 4];
        double acc = fma(phi, sx[i2], yc);
        acc = fma(c4, fma(-2.0, yc, e[i2] + e[i2 + 8]), acc);
        acc = fma(c3, fma(-2.0, yc, e[i2 + 1] + e[i2 + 7]), acc);
        acc = fma(c2, fma(-2.0, yc, e[i2 + 2] + e[i2 + 6]), acc);
        y[i2] = fma(c1, fma(-2.0, yc, e[i2 + 3] + e[i2 + 5]), acc);
      }
      if (lane > last) {
#pragma unroll
        for (int i2 = 0; i2 < R; ++i2) y[i2] = 0.0;
      }
    }
  } else {
    double z[R], acc[R];
    for (int64_t i = 0; i < a.m; ++i) {
      const int64_t i0 = i - (i % 15);
      if (i == i0) hc = half_step_coefs(a, Tj, i0, lane);
      heat_rk4_step<R>(y, z, acc, a.h, step_coefs<double>(hc, i, i0, cdx), sx, true, lane, n);
    }
  }
}

// Float64 defect of slice j (the residual correction the Conclusion
// proposes): d_j = g^j(lt_j) - lt_{j+1}, the forced solve from lt_j.
template <int R>
__device__ __forceinline__ void heat_defect_slice(const HeatArgs& a, const double* lt, double* d, int64_t j,
                                                  int lane, const double* sxt = nullptr) {
  const int n = a.n;
  double y[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int r = lane * R + i;
    y[i] = r < n ? lt[j * n + r] : 0.0;
  }
  heat_forced_solve<R>(a, y, j, lane, sxt);
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
