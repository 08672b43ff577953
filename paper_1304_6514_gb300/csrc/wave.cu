// Wave equation u_tt = u_xx on [-1, 1] (Section 5, eq. waveequation), Dirichlet
// ends, Chebyshev spectral differences on x_i = cos(i pi / M), leapfrog steps
//   u^{n+1} = 2 u^n - u^{n-1} + h^2 D2 u^n
// on the two-level state Y = (u^n, u^{n-1}) of dimension n = 2d, d = M - 1
// (the doubled initial-value space of Section 5).  The operator is dense and
// time-invariant and there is no forcing, so the affine map of a slice is the
// m-th power of the one-step matrix and b_j = 0.
//
// Build: a CTA keeps D2 (transposed, zero-padded to DP x DP) in shared memory
// and advances a tile of C basis columns through all m steps without leaving
// the chip: per step the tile's u^n (DP x C, shared) is multiplied by D2 in a
// register-blocked product (thread = 8 rows x CB columns, rows from D2 by
// vector loads, columns spread across the lanes), and the thread updates its
// own 8 x CB entries, whose u^{n-1} it holds in registers.  The final state is
// staged in shared memory and written column by column, coalesced.  Columns of
// all slices form one index space (global column g = j (n+1) + c lands at
// g * n in the column-major maps).
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace nvpit {

constexpr int kWaveMaxDP = 80;     // d = M - 1 <= 80

struct WaveArgs {
  void* out;          // S (n+1) columns of n values, precision T
  const double* d2t;  // DP x DP, d2t[k * DP + i] = D2[i][k], zero outside d x d
  int d, n, S;
  int64_t m;
  double h2;          // h^2
};

// D (Gauss-Lobatto differentiation, (M+1)^2) into scratch, one CTA per row:
// the off-diagonal entries, then the diagonal as minus the row's sum.
__global__ void wave_dmat_kernel(int M, double* D) {
  const int N = M + 1, i = blockIdx.x;
  __shared__ double xs[kWaveMaxDP + 3];
  for (int q = threadIdx.x; q < N; q += blockDim.x) xs[q] = cos((double)q * M_PI / (double)M);
  __syncthreads();
  const double ci = (i == 0 || i == M) ? 2.0 : 1.0;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    if (j == i) continue;
    const double cj = (j == 0 || j == M) ? 2.0 : 1.0;
    const double sign = ((i + j) & 1) ? -1.0 : 1.0;
    D[i * N + j] = (ci / cj) * sign / (xs[i] - xs[j]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {                               // rows sum to zero
    double s = 0.0;
    for (int j = 0; j < N; ++j)
      if (j != i) s += D[i * N + j];
    D[i * N + i] = -s;
  }
}

// The interior block of D D, transposed and zero-padded into d2t (DP x DP),
// one CTA per row k of d2t.
__global__ void wave_d2_kernel(int M, int DP, const double* D, double* d2t) {
  const int N = M + 1, d = M - 1, k = blockIdx.x;
  for (int i = threadIdx.x; i < DP; i += blockDim.x) {
    double v = 0.0;
    if (i < d && k < d) {
      for (int l = 0; l < N; ++l) v = fma(D[(i + 1) * N + l], D[l * N + (k + 1)], v);
    }
    d2t[k * DP + i] = v;
  }
}

template <typename T>
struct Vec8;
template <>
struct Vec8<float> {
  __device__ static void load(const float* p, float* a) {
    const float4 x = reinterpret_cast<const float4*>(p)[0], y = reinterpret_cast<const float4*>(p)[1];
    a[0] = x.x; a[1] = x.y; a[2] = x.z; a[3] = x.w; a[4] = y.x; a[5] = y.y; a[6] = y.z; a[7] = y.w;
  }
};
template <>
struct Vec8<double> {
  __device__ static void load(const double* p, double* a) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double2 x = reinterpret_cast<const double2*>(p)[q];
      a[2 * q] = x.x;
      a[2 * q + 1] = x.y;
    }
  }
};

template <typename T, int DP, int CB>
struct WaveTile {
  static constexpr int RB = 8;              // rows per thread
  static constexpr int TR = DP / RB;        // row groups = warps
  static constexpr int THREADS = TR * 32;
  static constexpr int C = 32 * CB;         // columns per tile
  static constexpr int LD = C + 1;          // padded row of the state tiles
  static constexpr size_t SMEM = sizeof(T) * ((size_t)DP * DP + 2 * (size_t)DP * LD);
};

template <typename T, int DP, int CB>
__global__ void __launch_bounds__(WaveTile<T, DP, CB>::THREADS, 1) wave_build_kernel(WaveArgs a) {
  using W = WaveTile<T, DP, CB>;
  constexpr int RB = W::RB, C = W::C, LD = W::LD;
  extern __shared__ __align__(16) unsigned char wave_smem[];
  T* d2s = reinterpret_cast<T*>(wave_smem);          // DP x DP, [k][i]
  T* U = d2s + DP * DP;                              // DP x LD, u^n of the tile
  T* UO = U + DP * LD;                               // DP x LD, staging of u^{n-1}
  const int tid = threadIdx.x, lane = tid & 31, r0 = (tid >> 5) * RB;
  const int d = a.d, n = a.n;
  const T h2 = (T)a.h2;
  for (int idx = tid; idx < DP * DP; idx += blockDim.x) d2s[idx] = (T)a.d2t[idx];
  T* out = reinterpret_cast<T*>(a.out);
  const int64_t total = (int64_t)a.S * (n + 1);
  const int64_t tiles = (total + C - 1) / C;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t g0 = tile * C;
    T u[RB][CB], uo[RB][CB];
#pragma unroll
    for (int cb = 0; cb < CB; ++cb) {
      const int col = lane + 32 * cb;
      const int64_t g = g0 + col;
      // basis index c of this column: 0 (the solve from 0), 1..d (u^n = e),
      // d+1..2d (u^{n-1} = e); past the last column: zeros
      const int c = g < total ? (int)(g % (n + 1)) : 0;
#pragma unroll
      for (int rb = 0; rb < RB; ++rb) {
        const int r = r0 + rb;
        u[rb][cb] = (c >= 1 && c <= d && r == c - 1) ? (T)1 : (T)0;
        uo[rb][cb] = (c > d && r == c - 1 - d) ? (T)1 : (T)0;
        U[r * LD + col] = u[rb][cb];
      }
    }
    __syncthreads();
    for (int64_t step = 0; step < a.m; ++step) {
      T acc[RB][CB];
#pragma unroll
      for (int rb = 0; rb < RB; ++rb)
#pragma unroll
        for (int cb = 0; cb < CB; ++cb) acc[rb][cb] = (T)0;
#pragma unroll 2
      for (int k = 0; k < d; ++k) {
        T av[RB], bv[CB];
        Vec8<T>::load(d2s + k * DP + r0, av);
#pragma unroll
        for (int cb = 0; cb < CB; ++cb) bv[cb] = U[k * LD + lane + 32 * cb];
#pragma unroll
        for (int rb = 0; rb < RB; ++rb)
#pragma unroll
          for (int cb = 0; cb < CB; ++cb) acc[rb][cb] = fma(av[rb], bv[cb], acc[rb][cb]);
      }
      __syncthreads();                                  // every read of u^n is done
#pragma unroll
      for (int rb = 0; rb < RB; ++rb)
#pragma unroll
        for (int cb = 0; cb < CB; ++cb) {
          const T un = fma(h2, acc[rb][cb], (T)2 * u[rb][cb] - uo[rb][cb]);
          uo[rb][cb] = u[rb][cb];
          u[rb][cb] = un;
          U[(r0 + rb) * LD + lane + 32 * cb] = un;
        }
      __syncthreads();
    }
#pragma unroll
    for (int rb = 0; rb < RB; ++rb)
#pragma unroll
      for (int cb = 0; cb < CB; ++cb) UO[(r0 + rb) * LD + lane + 32 * cb] = uo[rb][cb];
    __syncthreads();
    // column g holds (u^m, u^{m-1}): n = 2d contiguous values at g * n
    const int64_t cols = std::min<int64_t>(C, total - g0);
    for (int idx = tid; idx < cols * n; idx += blockDim.x) {
      const int col = idx / n, row = idx - col * n;
      out[(g0 + col) * n + row] = row < d ? U[row * LD + col] : UO[(row - d) * LD + col];
    }
    __syncthreads();                                    // U, UO are reused by the next tile
  }
}

// Serial leapfrog solve of S m steps from y0 = (u^0, u^{-1}), one CTA.
__global__ void wave_serial_kernel(WaveArgs a, int DP, int64_t steps, const double* y0, double* yT) {
  __shared__ double u[kWaveMaxDP], uo[kWaveMaxDP];
  const int d = a.d, i = threadIdx.x;
  if (i < d) {
    u[i] = y0[i];
    uo[i] = y0[d + i];
  }
  __syncthreads();
  for (int64_t s = 0; s < steps; ++s) {
    double un = 0.0;
    if (i < d) {
      double w = 0.0;
      for (int k = 0; k < d; ++k) w = fma(a.d2t[k * DP + i], u[k], w);
      un = fma(a.h2, w, 2.0 * u[i] - uo[i]);
    }
    __syncthreads();
    if (i < d) {
      uo[i] = u[i];
      u[i] = un;
    }
    __syncthreads();
  }
  if (i < d) {
    yT[i] = u[i];
    yT[d + i] = uo[i];
  }
}

// Float64 defects of approximate boundary states for the correction passes
// of NV_FP32_REFINE: d_j = g^j(lam_j) - lam_{j+1}, one CTA per slice running
// the m leapfrog steps of slice j from lam_j = (u^n, u^{n-1}) with the
// arithmetic of wave_serial_kernel.  lam: (S+1) x n, d: S x n.
__global__ void wave_defect_kernel(WaveArgs a, int DP, const double* lam, double* dout) {
  __shared__ double u[kWaveMaxDP], uo[kWaveMaxDP];
  const int d = a.d, n = a.n, i = threadIdx.x;
  for (int j = blockIdx.x; j < a.S; j += gridDim.x) {
    const double* l0 = lam + (int64_t)j * n;
    if (i < d) {
      u[i] = l0[i];
      uo[i] = l0[d + i];
    }
    __syncthreads();
    for (int64_t s = 0; s < a.m; ++s) {
      double un = 0.0;
      if (i < d) {
        double w = 0.0;
        for (int k = 0; k < d; ++k) w = fma(a.d2t[k * DP + i], u[k], w);
        un = fma(a.h2, w, 2.0 * u[i] - uo[i]);
      }
      __syncthreads();
      if (i < d) {
        uo[i] = u[i];
        u[i] = un;
      }
      __syncthreads();
    }
    if (i < d) {
      const double* l1 = lam + (int64_t)(j + 1) * n;
      dout[(int64_t)j * n + i] = u[i] - l1[i];
      dout[(int64_t)j * n + d + i] = uo[i] - l1[d + i];
    }
    __syncthreads();                                    // u, uo are reused by the next slice
  }
}

template <typename T, int DP, int CB>
static nv_status launch_wave_tiles(const WaveArgs& a, cudaStream_t s) {
  using W = WaveTile<T, DP, CB>;
  const void* fn = (const void*)wave_build_kernel<T, DP, CB>;
  nv_status st = nv_cuda_check(
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)W::SMEM), "wave smem attribute");
  if (st != NV_OK) return st;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  st = nv_cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wave_build_kernel<T, DP, CB>,
                                                                   W::THREADS, W::SMEM),
                     "wave occupancy");
  if (st != NV_OK) return st;
  const int64_t tiles = ((int64_t)a.S * (a.n + 1) + W::C - 1) / W::C;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sms * std::max(per_sm, 1)));
  wave_build_kernel<T, DP, CB><<<grid, W::THREADS, W::SMEM, s>>>(a);
  return nv_cuda_check(cudaGetLastError(), "wave_build_kernel launch");
}

}  // namespace nvpit

using namespace nvpit;

static int wave_dp(int d) { return d <= 40 ? 40 : kWaveMaxDP; }

// The operator occupies the maps' auxiliary region: (M+1)^2 doubles of D
// followed by DP^2 doubles of the transposed interior D2.
int64_t wave_aux_elems(int d) {
  const int M = d + 1, DP = wave_dp(d);
  return (int64_t)(M + 1) * (M + 1) + (int64_t)DP * DP;
}

static nv_status wave_operator(int d, double* aux, cudaStream_t s) {
  const int M = d + 1, DP = wave_dp(d);
  wave_dmat_kernel<<<M + 1, 128, 0, s>>>(M, aux);
  nv_status st = nv_cuda_check(cudaGetLastError(), "wave_dmat_kernel launch");
  if (st != NV_OK) return st;
  wave_d2_kernel<<<DP, 128, 0, s>>>(M, DP, aux, aux + (int64_t)(M + 1) * (M + 1));
  return nv_cuda_check(cudaGetLastError(), "wave_d2_kernel launch");
}

nv_status launch_wave_build(const nv_maps* M, cudaStream_t s) {
  const int n = M->dim, d = n / 2;
  if (d < 1 || d > kWaveMaxDP || n != 2 * d) return nv_fail(NV_ENOTSUP, "wave state dimension must be 2(M-1) <= 160");
  if (!M->aux) return nv_fail(NV_EINVAL, "wave maps have no operator storage");
  nv_status st = wave_operator(d, M->aux, s);
  if (st != NV_OK) return st;
  const int DP = wave_dp(d);
  WaveArgs a{};
  a.out = M->data;
  a.d2t = M->aux + (int64_t)(d + 2) * (d + 2);
  a.d = d;
  a.n = n;
  a.S = M->S;
  a.m = M->m;
  a.h2 = M->h * M->h;
  if (M->prec == NV_FP64)
    return DP == 40 ? launch_wave_tiles<double, 40, 2>(a, s) : launch_wave_tiles<double, 80, 2>(a, s);
  return DP == 40 ? launch_wave_tiles<float, 40, 4>(a, s) : launch_wave_tiles<float, 80, 4>(a, s);
}

nv_status launch_wave_defect(const nv_maps* M, const double* lam, double* d, cudaStream_t s) {
  const int n = M->dim, dd = n / 2;
  if (dd < 1 || dd > kWaveMaxDP || n != 2 * dd) return nv_fail(NV_ENOTSUP, "wave state dimension must be 2(M-1) <= 160");
  if (!M->aux) return nv_fail(NV_EINVAL, "wave maps have no operator storage");
  WaveArgs a{};
  a.d2t = M->aux + (int64_t)(dd + 2) * (dd + 2);
  a.d = dd;
  a.n = n;
  a.S = M->S;
  a.m = M->m;
  a.h2 = M->h * M->h;
  const int grid = (int)std::min<int64_t>(M->S, 4096);
  wave_defect_kernel<<<grid, 128, 0, s>>>(a, wave_dp(dd), lam, d);
  return nv_cuda_check(cudaGetLastError(), "wave_defect_kernel launch");
}

nv_status launch_serial_wave(const nv_maps* P, const double* y0, double* yT, cudaStream_t s) {
  const int n = P->dim, d = n / 2;
  if (d < 1 || d > kWaveMaxDP || n != 2 * d) return nv_fail(NV_ENOTSUP, "wave state dimension must be 2(M-1) <= 160");
  const int DP = wave_dp(d);
  double* aux = nullptr;
  nv_status st = nv_cuda_check(cudaMallocAsync((void**)&aux, sizeof(double) * wave_aux_elems(d), s),
                               "wave operator scratch");
  if (st != NV_OK) return st;
  st = wave_operator(d, aux, s);
  if (st == NV_OK) {
    WaveArgs a{};
    a.d2t = aux + (int64_t)(d + 2) * (d + 2);
    a.d = d;
    a.n = n;
    a.S = P->S;
    a.m = P->m;
    a.h2 = P->h * P->h;
    wave_serial_kernel<<<1, 128, 0, s>>>(a, DP, (int64_t)P->S * P->m, y0, yT);
    st = nv_cuda_check(cudaGetLastError(), "wave_serial_kernel launch");
  }
  nv_status st2 = nv_cuda_check(cudaFreeAsync(aux, s), "wave operator scratch free");
  return st != NV_OK ? st : st2;
}
