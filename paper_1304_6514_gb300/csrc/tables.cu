// Table maps (NV_MAP_PL1D, NV_MAP_BILINEAR2D): computation phase and
// communication phase of Figure "pseudocode" for low-dimensional problems.
//
//   coef_kernel         time-dependent right-hand-side coefficients per slice
//                       (cos t at every stage time), computed once and staged
//                       through shared memory by the integrator
//   table_build_kernel  one thread per (slice j, sample k): the fine scheme over
//                       [T_{j-1}, T_j] from xi_k, final state stored as the
//                       table value lambda_j^k (sample generated from indices)
//   table_chain_kernel  lambda_j = phi^j(lambda_{j-1}), sequential, float64
//   serial_table_kernel the serial fine solve (one thread)
#include <math.h>

#include "common.cuh"

namespace nvpit {

// Stage-time coefficients: Euler needs t_i = T_{j-1} + i h (i < m); RK4 needs
// t_i, t_i + h/2 and t_i + h, stored at half steps q = 0..2m.  Products and
// sums use explicit round-to-nearest so that the times equal the oracle's.
__global__ void coef_kernel(double* coef, int64_t per_slice, int S, double t0, double H, double h,
                            int rk4) {
  const int64_t total = per_slice * (int64_t)S;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = idx / per_slice, q = idx - j * per_slice;
    const double Tj = __dadd_rn(t0, __dmul_rn((double)j, H));
    double t;
    if (rk4) {
      const int64_t i = q >> 1;
      t = __dadd_rn(Tj, __dmul_rn((double)i, h));
      if (q & 1) t = __dadd_rn(t, 0.5 * h);
    } else {
      t = __dadd_rn(Tj, __dmul_rn((double)q, h));
    }
    coef[idx] = cos(t);
  }
}

struct TableArgs {
  void* out;
  const double* coef;
  int64_t coef_per_slice;
  int64_t m;
  int64_t samples;       // per slice
  int per_dim;
  double lo0, lo1, d0, d1;
  double h;
  double params[NVPIT_MAX_PARAMS];
};

constexpr int kChunkSteps = 2048;

template <class R, typename T, int RK4>
__global__ void __launch_bounds__(256) table_build_kernel(TableArgs a) {
  extern __shared__ unsigned char smem_raw[];
  T* cs = reinterpret_cast<T*>(smem_raw);
  const int j = blockIdx.y;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = k < a.samples;
  const R rhs(a.params);
  const T h = (T)a.h;

  T y[R::D], comp[R::D];
#pragma unroll
  for (int d = 0; d < R::D; ++d) y[d] = comp[d] = 0;
  if constexpr (R::D == 1) {
    y[0] = (T)__dadd_rn(a.lo0, __dmul_rn((double)k, a.d0));
  } else {
    const int p = (int)(k % a.per_dim), q = (int)(k / a.per_dim);
    y[0] = (T)__dadd_rn(a.lo0, __dmul_rn((double)p, a.d0));
    y[1] = (T)__dadd_rn(a.lo1, __dmul_rn((double)q, a.d1));
  }

  for (int64_t i0 = 0; i0 < a.m; i0 += kChunkSteps) {
    const int64_t i1 = min(a.m, i0 + (int64_t)kChunkSteps);
    if (R::TIME_DEP) {
      // stage this chunk's coefficients: Euler i0..i1-1, RK4 half steps 2 i0 .. 2 i1
      const int64_t q0 = RK4 ? 2 * i0 : i0;
      const int64_t nq = RK4 ? 2 * (i1 - i0) + 1 : (i1 - i0);
      const double* src = a.coef + (int64_t)j * a.coef_per_slice + q0;
      __syncthreads();
      for (int64_t q = threadIdx.x; q < nq; q += blockDim.x) cs[q] = (T)src[q];
      __syncthreads();
    }
    if (active) {
      if (RK4) {
        for (int64_t i = i0; i < i1; ++i) {
          const int64_t q = 2 * (i - i0);
          T c0 = 0, ch = 0, c1 = 0;
          if (R::TIME_DEP) { c0 = cs[q]; ch = cs[q + 1]; c1 = cs[q + 2]; }
          rk4_step(rhs, c0, ch, c1, h, y, comp);
        }
      } else {
        for (int64_t i = i0; i < i1; ++i) {
          T c0 = 0;
          if (R::TIME_DEP) c0 = cs[i - i0];
          euler_step(rhs, c0, h, y, comp);
        }
      }
    }
  }
  if (active) {
    T* out = reinterpret_cast<T*>(a.out);
    const int64_t base = ((int64_t)j * a.samples + k) * R::D;
#pragma unroll
    for (int d = 0; d < R::D; ++d) out[base + d] = y[d];
  }
}

// --------------------------------------------------------------------------
// Sequential composition of table maps, float64 (Figure "pseudocode",
// communication phase).  One thread walks the S slices.
// --------------------------------------------------------------------------
struct ChainArgs {
  const void* table;
  int S, per_dim, dim;
  double lo0, lo1, hi0, hi1, d0, d1;
  double r0, r1;    // 1 / d0, 1 / d1: the single thread's chain multiplies instead of
                    // dividing (an FP64 division is a long dependent sequence here)
  const double* y0;
  double* yT;
  double* lambdas;
  int* status;
  unsigned long long* oob;
  int oob_error;
  int64_t cached;   // > 0: the whole table (this many elements) is first copied to shared memory
};

// Table value at element i; p is a global or a shared-memory address.
template <typename T>
__device__ __forceinline__ double tload(const T* p, int64_t i) { return (double)p[i]; }

__device__ __forceinline__ int clamp_cell(double u, int cells) {
  // floor(u) clamped to [0, cells-1]; NaN maps to 0 (caught by the finite check)
  double f = floor(u);
  if (!(f >= 0.0)) return 0;
  if (f > (double)(cells - 1)) return cells - 1;
  return (int)f;
}

// One thread walks the S dependent lookups.  When the table fits in shared
// memory the CTA first copies it there, so each lookup waits on a shared load
// instead of a round trip to L2 / HBM.
template <typename T>
__global__ void table_chain_kernel(ChainArgs a) {
  extern __shared__ __align__(16) unsigned char tab_smem[];
  if (blockIdx.x != 0) return;
  const T* tab = reinterpret_cast<const T*>(a.table);
  if (a.cached > 0) {
    T* st = reinterpret_cast<T*>(tab_smem);
    for (int64_t i = threadIdx.x; i < a.cached; i += blockDim.x) st[i] = __ldg(tab + i);
    __syncthreads();
    tab = st;
  }
  if (threadIdx.x != 0) return;
  unsigned long long oob = 0;
  bool bad = false;
  if (a.dim == 1) {
    const int M = a.per_dim;
    double lam = a.y0[0];
    if (a.lambdas) a.lambdas[0] = lam;
    for (int j = 0; j < a.S; ++j) {
      const int s = clamp_cell((lam - a.lo0) * a.r0, M - 1);
      const double w = (lam - __dadd_rn(a.lo0, __dmul_rn((double)s, a.d0))) * a.r0;
      oob += (lam < a.lo0 || lam > a.hi0);
      const int64_t base = (int64_t)j * M + s;
      lam = (1.0 - w) * tload(tab, base) + w * tload(tab, base + 1);
      bad |= !isfinite(lam);
      if (a.lambdas) a.lambdas[j + 1] = lam;
    }
    a.yT[0] = lam;
  } else {
    const int P = a.per_dim;
    double x = a.y0[0], y = a.y0[1];
    if (a.lambdas) { a.lambdas[0] = x; a.lambdas[1] = y; }
    for (int j = 0; j < a.S; ++j) {
      const int p = clamp_cell((x - a.lo0) * a.r0, P - 1);
      const int q = clamp_cell((y - a.lo1) * a.r1, P - 1);
      const double wx = (x - __dadd_rn(a.lo0, __dmul_rn((double)p, a.d0))) * a.r0;
      const double wy = (y - __dadd_rn(a.lo1, __dmul_rn((double)q, a.d1))) * a.r1;
      oob += !(x >= a.lo0 && x <= a.hi0 && y >= a.lo1 && y <= a.hi1);
      const int64_t b00 = (((int64_t)j * P + q) * P + p) * 2;
      const int64_t b10 = b00 + 2;                 // (p+1, q)
      const int64_t b01 = b00 + 2 * (int64_t)P;    // (p, q+1)
      const int64_t b11 = b01 + 2;
      const double c00 = (1.0 - wx) * (1.0 - wy), c10 = wx * (1.0 - wy);
      const double c01 = (1.0 - wx) * wy, c11 = wx * wy;
      const double nx = c00 * tload(tab, b00) + c10 * tload(tab, b10) + c01 * tload(tab, b01) +
                        c11 * tload(tab, b11);
      const double ny = c00 * tload(tab, b00 + 1) + c10 * tload(tab, b10 + 1) +
                        c01 * tload(tab, b01 + 1) + c11 * tload(tab, b11 + 1);
      x = nx;
      y = ny;
      bad |= !(isfinite(x) && isfinite(y));
      if (a.lambdas) { a.lambdas[2 * (j + 1)] = x; a.lambdas[2 * (j + 1) + 1] = y; }
    }
    a.yT[0] = x;
    a.yT[1] = y;
  }
  if (oob) {
    atomicAdd(a.oob, oob);
    if (a.oob_error) record_status(a.status, NV_EDOMAIN);
  }
  if (bad) record_status(a.status, NV_EBADMAP);
}

// --------------------------------------------------------------------------
// Serial fine solve for the table right-hand sides (one thread, S*m steps,
// step i of slice j at T_{j-1} + i h, like the oracle).
// --------------------------------------------------------------------------
struct ParamPack {
  double p[NVPIT_MAX_PARAMS];
};

template <class R>
__global__ void serial_table_kernel(ParamPack pp, double t0, double H, double h, int S,
                                    int64_t m, int rk4, const double* y0, double* yT) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const R rhs(pp.p);
  double y[R::D], comp[R::D];
  for (int d = 0; d < R::D; ++d) { y[d] = y0[d]; comp[d] = 0.0; }
  for (int j = 0; j < S; ++j) {
    const double Tj = __dadd_rn(t0, __dmul_rn((double)j, H));
    for (int64_t i = 0; i < m; ++i) {
      const double t = __dadd_rn(Tj, __dmul_rn((double)i, h));
      if (rk4) {
        double c0 = 0, ch = 0, c1 = 0;
        if (R::TIME_DEP) { c0 = cos(t); ch = cos(__dadd_rn(t, 0.5 * h)); c1 = cos(__dadd_rn(t, h)); }
        rk4_step(rhs, c0, ch, c1, h, y, comp);
      } else {
        double c0 = 0;
        if (R::TIME_DEP) c0 = cos(t);
        euler_step(rhs, c0, h, y, comp);
      }
    }
  }
  for (int d = 0; d < R::D; ++d) yT[d] = y[d];
}

}  // namespace nvpit

using namespace nvpit;

nv_status launch_coef_tables(nv_maps* M, cudaStream_t s) {
  if (!M->coef) return NV_OK;
  const int64_t total = M->coef_per_slice * M->S;
  const int block = 256;
  const int grid = (int)std::min<int64_t>((total + block - 1) / block, 152 * 8);
  coef_kernel<<<grid, block, 0, s>>>(M->coef, M->coef_per_slice, M->S, M->t0, M->H, M->h,
                                     M->scheme == NV_RK4);
  return nv_cuda_check(cudaGetLastError(), "coef_kernel launch");
}

template <class R, typename T>
static nv_status launch_table_typed(nv_maps* M, cudaStream_t s, int block) {
  TableArgs a{};
  a.out = M->data;
  a.coef = M->coef;
  a.coef_per_slice = M->coef_per_slice;
  a.m = M->m;
  a.per_dim = M->per_dim;
  a.samples = (M->map == NV_MAP_PL1D) ? M->per_dim : (int64_t)M->per_dim * M->per_dim;
  a.lo0 = M->lo[0];
  a.lo1 = M->lo[1];
  a.d0 = (M->hi[0] - M->lo[0]) / (M->per_dim - 1);
  a.d1 = (M->hi[1] - M->lo[1]) / (M->per_dim - 1);
  a.h = M->h;
  for (int i = 0; i < NVPIT_MAX_PARAMS; ++i) a.params[i] = M->params[i];
  const dim3 grid((unsigned)((a.samples + block - 1) / block), (unsigned)M->S);
  const int rk4 = M->scheme == NV_RK4;
  const size_t smem = R::TIME_DEP ? sizeof(T) * (2 * kChunkSteps + 1) : 0;
  if (rk4)
    table_build_kernel<R, T, 1><<<grid, block, smem, s>>>(a);
  else
    table_build_kernel<R, T, 0><<<grid, block, smem, s>>>(a);
  return nv_cuda_check(cudaGetLastError(), "table_build_kernel launch");
}

template <typename T>
static nv_status launch_table_prec(nv_maps* M, cudaStream_t s, int block) {
  switch (M->rhs_kind) {
    case NV_RHS_LINEAR_SCALAR: return launch_table_typed<RhsLinearScalar<T>, T>(M, s, block);
    case NV_RHS_SQUARE: return launch_table_typed<RhsSquare<T>, T>(M, s, block);
    case NV_RHS_COS_CUBIC: return launch_table_typed<RhsCosCubic<T>, T>(M, s, block);
    case NV_RHS_VDP: return launch_table_typed<RhsVdp<T>, T>(M, s, block);
    default: return nv_fail(NV_ENOTSUP, "table maps are not built for rhs kind %d", M->rhs_kind);
  }
}

nv_status launch_table_build(nv_maps* M, cudaStream_t s, int block) {
  nv_status st = launch_coef_tables(M, s);
  if (st != NV_OK) return st;
  if (M->prec == NV_FP64) return launch_table_prec<double>(M, s, block);
  return launch_table_prec<float>(M, s, block);
}

nv_status launch_table_compose(const nv_maps* M, const double* y0, double* yT, double* lambdas,
                               cudaStream_t s) {
  ChainArgs a{};
  a.table = M->data;
  a.S = M->S;
  a.per_dim = M->per_dim;
  a.dim = M->dim;
  a.lo0 = M->lo[0];
  a.lo1 = M->lo[1];
  a.hi0 = M->hi[0];
  a.hi1 = M->hi[1];
  a.d0 = (M->hi[0] - M->lo[0]) / (M->per_dim - 1);
  a.d1 = (M->hi[1] - M->lo[1]) / (M->per_dim - 1);
  a.r0 = 1.0 / a.d0;
  a.r1 = a.d1 != 0.0 ? 1.0 / a.d1 : 0.0;
  a.y0 = y0;
  a.yT = yT;
  a.lambdas = lambdas;
  a.status = M->status;
  a.oob = M->oob;
  a.oob_error = M->oob_policy == NV_OOB_ERROR;
  const int64_t elems = M->elems_per_slice * (int64_t)M->S;
  const size_t bytes = (size_t)elems * (size_t)M->elem_bytes;
  const size_t kCacheMax = 200 * 1024;
  const void* fn = M->prec == NV_FP64 ? (const void*)table_chain_kernel<double>
                                      : (const void*)table_chain_kernel<float>;
  size_t smem = 0;
  int threads = 32;
  if (bytes <= kCacheMax) {
    a.cached = elems;
    smem = bytes;
    threads = 1024;
    if (smem > 48 * 1024) {
      nv_status st = nv_cuda_check(
          cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "table smem attribute");
      if (st != NV_OK) return st;
    }
  }
  if (M->prec == NV_FP64)
    table_chain_kernel<double><<<1, threads, smem, s>>>(a);
  else
    table_chain_kernel<float><<<1, threads, smem, s>>>(a);
  return nv_cuda_check(cudaGetLastError(), "table_chain_kernel launch");
}

nv_status launch_serial_table(int32_t rhs_kind, const double* params, double t0, double H,
                              double h, int32_t S, int64_t m, int32_t scheme, const double* y0,
                              double* yT, cudaStream_t s) {
  const int rk4 = scheme == NV_RK4;
  ParamPack pp{};
  for (int i = 0; i < NVPIT_MAX_PARAMS; ++i) pp.p[i] = params[i];
  switch (rhs_kind) {
    case NV_RHS_LINEAR_SCALAR:
      serial_table_kernel<RhsLinearScalar<double>><<<1, 32, 0, s>>>(pp, t0, H, h, S, m, rk4, y0, yT);
      break;
    case NV_RHS_SQUARE:
      serial_table_kernel<RhsSquare<double>><<<1, 32, 0, s>>>(pp, t0, H, h, S, m, rk4, y0, yT);
      break;
    case NV_RHS_COS_CUBIC:
      serial_table_kernel<RhsCosCubic<double>><<<1, 32, 0, s>>>(pp, t0, H, h, S, m, rk4, y0, yT);
      break;
    case NV_RHS_VDP:
      serial_table_kernel<RhsVdp<double>><<<1, 32, 0, s>>>(pp, t0, H, h, S, m, rk4, y0, yT);
      break;
    case NV_RHS_CHAIN3:
      serial_table_kernel<RhsChain3<double>><<<1, 32, 0, s>>>(pp, t0, H, h, S, m, rk4, y0, yT);
      break;
    default:
      return nv_fail(NV_ENOTSUP, "serial fine solve not built for rhs kind %d", rhs_kind);
  }
  return nv_cuda_check(cudaGetLastError(), "serial_table_kernel launch");
}
