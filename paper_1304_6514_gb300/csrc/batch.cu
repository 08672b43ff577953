// Batched independent instances: one persistent launch builds the table maps
// of B instances with uneven slice counts and horizons.
//
// Work items are (instance i, slice j) pairs.  Their cost is m_i steps for
// every sample, so the host orders them by decreasing m_i (longest processing
// time first) and the persistent CTAs pull them from a device counter: the
// long slices start first and the short ones fill the tail.  A CTA integrates
// all P^2 (or M) samples of its item, SPT samples per thread interleaved for
// instruction-level parallelism, with the instance parameters in registers.
// The composition walks each instance's slices in float64, one thread per
// instance.  nv_batch_run replays build + compose from a captured CUDA graph.
#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace nvpit {

struct InstDesc {
  double p[4];        // right-hand-side parameters
  double t0, H, h;
  int64_t m;          // fine steps per slice
  int64_t off;        // element offset of slice 0's table
  int32_t S;
  int32_t pad;
};

struct BatchBuildArgs {
  const InstDesc* inst;
  const int2* items;
  int nitems;
  unsigned* counter;
  void* out;
  int samples;          // per slice
  int per_dim, dim;
  double lo0, lo1, d0, d1;
};

// Largest CTA a variant with SPT samples per thread is compiled for.
__host__ __device__ constexpr int batch_bound(int spt) { return spt <= 1 ? 1024 : (spt == 2 ? 512 : 256); }

// Node coordinates lo + p d (float64, rounded to nearest, then to T) are the
// same for every item: a CTA computes them once into shared memory when the
// grid has at most kNodeCache nodes per axis, so the item loop does no float64
// work.
constexpr int kNodeCache = 1024;

template <class R, typename T, int SPT, int RK4>
__global__ void __launch_bounds__(batch_bound(SPT)) batch_build_kernel(BatchBuildArgs a) {
  __shared__ int item_s;
  __shared__ T nodes[R::D][kNodeCache];
  const int naxis = R::D == 1 ? a.samples : a.per_dim;
  const bool cached = naxis <= kNodeCache;
  if (cached)
    for (int i = threadIdx.x; i < naxis; i += blockDim.x) {
      nodes[0][i] = (T)__dadd_rn(a.lo0, __dmul_rn((double)i, a.d0));
      if constexpr (R::D == 2) nodes[1][i] = (T)__dadd_rn(a.lo1, __dmul_rn((double)i, a.d1));
    }
  T* out = reinterpret_cast<T*>(a.out);
  for (;;) {
    if (threadIdx.x == 0) item_s = (int)atomicAdd(a.counter, 1u);
    __syncthreads();
    const int it = item_s;
    __syncthreads();
    if (it >= a.nitems) return;
    const int2 w = a.items[it];
    const InstDesc d = a.inst[w.x];
    const int j = w.y;
    const R rhs(d.p);
    const T h = (T)d.h;
    T y[SPT][R::D], comp[SPT][R::D];
    bool act[SPT];
#pragma unroll
    for (int s = 0; s < SPT; ++s) {
      const int k = threadIdx.x + s * blockDim.x;
      act[s] = k < a.samples;
#pragma unroll
      for (int c = 0; c < R::D; ++c) y[s][c] = comp[s][c] = (T)0;
      if constexpr (R::D == 1) {
        if (act[s]) y[s][0] = cached ? nodes[0][k] : (T)__dadd_rn(a.lo0, __dmul_rn((double)k, a.d0));
      } else {
        const int p = k % a.per_dim, q = k / a.per_dim;
        if (act[s]) {
          y[s][0] = cached ? nodes[0][p] : (T)__dadd_rn(a.lo0, __dmul_rn((double)p, a.d0));
          y[s][1] = cached ? nodes[1][q] : (T)__dadd_rn(a.lo1, __dmul_rn((double)q, a.d1));
        }
      }
    }
    for (int64_t i = 0; i < d.m; ++i) {
#pragma unroll
      for (int s = 0; s < SPT; ++s) {
        if (RK4)
          rk4_step(rhs, (T)0, (T)0, (T)0, h, y[s], comp[s]);
        else
          euler_step(rhs, (T)0, h, y[s], comp[s]);
      }
    }
#pragma unroll
    for (int s = 0; s < SPT; ++s) {
      const int k = threadIdx.x + s * blockDim.x;
      if (!act[s]) continue;
      const int64_t base = d.off + ((int64_t)j * a.samples + k) * R::D;
#pragma unroll
      for (int c = 0; c < R::D; ++c) out[base + c] = y[s][c];
    }
  }
}

struct BatchComposeArgs {
  const InstDesc* inst;
  const void* tables;
  int B, dim, per_dim;
  double lo0, lo1, hi0, hi1, d0, d1;
  double r0, r1;   // 1 / d0, 1 / d1 (a division is a long dependent FP64 sequence)
  const double* y0;
  double* yT;
  int* status;
  unsigned long long* oob;
  int oob_error;
};

__device__ __forceinline__ int batch_cell(double u, int cells) {
  double f = floor(u);
  if (!(f >= 0.0)) return 0;
  if (f > (double)(cells - 1)) return cells - 1;
  return (int)f;
}

template <typename T>
__global__ void batch_compose_kernel(BatchComposeArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.B) return;
  const InstDesc d = a.inst[i];
  const T* tab = reinterpret_cast<const T*>(a.tables) + d.off;
  unsigned long long oob = 0;
  bool bad = false;
  if (a.dim == 1) {
    const int M = a.per_dim;
    double lam = a.y0[i];
    for (int j = 0; j < d.S; ++j) {
      const int s = batch_cell((lam - a.lo0) * a.r0, M - 1);
      const double w = (lam - __dadd_rn(a.lo0, __dmul_rn((double)s, a.d0))) * a.r0;
      oob += (lam < a.lo0 || lam > a.hi0);
      const int64_t b = (int64_t)j * M + s;
      lam = (1.0 - w) * (double)__ldg(tab + b) + w * (double)__ldg(tab + b + 1);
      bad |= !isfinite(lam);
    }
    a.yT[i] = lam;
  } else {
    const int P = a.per_dim;
    double x = a.y0[2 * i], y = a.y0[2 * i + 1];
    for (int j = 0; j < d.S; ++j) {
      const int p = batch_cell((x - a.lo0) * a.r0, P - 1);
      const int q = batch_cell((y - a.lo1) * a.r1, P - 1);
      const double wx = (x - __dadd_rn(a.lo0, __dmul_rn((double)p, a.d0))) * a.r0;
      const double wy = (y - __dadd_rn(a.lo1, __dmul_rn((double)q, a.d1))) * a.r1;
      oob += !(x >= a.lo0 && x <= a.hi0 && y >= a.lo1 && y <= a.hi1);
      const int64_t b00 = (((int64_t)j * P + q) * P + p) * 2;
      const int64_t b10 = b00 + 2, b01 = b00 + 2 * (int64_t)P, b11 = b01 + 2;
      const double c00 = (1.0 - wx) * (1.0 - wy), c10 = wx * (1.0 - wy);
      const double c01 = (1.0 - wx) * wy, c11 = wx * wy;
      const double nx = c00 * (double)__ldg(tab + b00) + c10 * (double)__ldg(tab + b10) +
                        c01 * (double)__ldg(tab + b01) + c11 * (double)__ldg(tab + b11);
      const double ny = c00 * (double)__ldg(tab + b00 + 1) + c10 * (double)__ldg(tab + b10 + 1) +
                        c01 * (double)__ldg(tab + b01 + 1) + c11 * (double)__ldg(tab + b11 + 1);
      x = nx;
      y = ny;
      bad |= !(isfinite(x) && isfinite(y));
    }
    a.yT[2 * i] = x;
    a.yT[2 * i + 1] = y;
  }
  if (oob) {
    atomicAdd(a.oob, oob);
    if (a.oob_error) record_status(a.status, NV_EDOMAIN);
  }
  if (bad) record_status(a.status, NV_EBADMAP);
}

}  // namespace nvpit

using namespace nvpit;

struct nv_batch {
  int32_t rhs_kind, dim, B, scheme, prec, map, per_dim, oob_policy;
  double lo[2], hi[2];
  int samples;                  // per slice
  int64_t elems_per_slice;
  int64_t total_slices, traj_steps, table_bytes;
  int elem_bytes;
  std::vector<InstDesc> host_inst;
  InstDesc* inst;               // device
  int2* items;                  // device
  void* tables;                 // device
  void* ws;                     // status (0), oob (8), counter (16)
  int* status;
  unsigned long long* oob;
  unsigned* counter;
  int threads;                  // CTA size of the build
  cudaGraphExec_t graph;
  const double* graph_y0;
  double* graph_yT;
  int device;
};

static std::mutex g_tune_mu;
static std::map<int, int> g_best_threads;   // device -> CTA size chosen by the autotuner

template <class R, typename T, int RK4>
static nv_status launch_batch_build_T(nv_batch* b, cudaStream_t s, int threads) {
  BatchBuildArgs a{};
  a.inst = b->inst;
  a.items = b->items;
  a.nitems = (int)b->total_slices;
  a.counter = b->counter;
  a.out = b->tables;
  a.samples = b->samples;
  a.per_dim = b->per_dim;
  a.dim = b->dim;
  a.lo0 = b->lo[0];
  a.lo1 = b->lo[1];
  a.d0 = (b->hi[0] - b->lo[0]) / (b->per_dim - 1);
  a.d1 = (b->hi[1] - b->lo[1]) / (b->per_dim - 1);
  const int spt = (b->samples + threads - 1) / threads;
  const void* fn = nullptr;
  int SPT = 0;
  switch (spt) {
    case 1: fn = (const void*)batch_build_kernel<R, T, 1, RK4>; SPT = 1; break;
    case 2: fn = (const void*)batch_build_kernel<R, T, 2, RK4>; SPT = 2; break;
    case 3: case 4: fn = (const void*)batch_build_kernel<R, T, 4, RK4>; SPT = 4; break;
    case 5: case 6: case 7: case 8: fn = (const void*)batch_build_kernel<R, T, 8, RK4>; SPT = 8; break;
    default: return nv_fail(NV_ENOTSUP, "more than 8 samples per thread (samples %d, CTA %d)",
                            b->samples, threads);
  }
  if (threads > batch_bound(SPT))
    return nv_fail(NV_ENOTSUP, "CTA of %d threads with %d samples per thread", threads, SPT);
  int sms = 152, dev = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  nv_status st = nv_cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0),
                               "batch occupancy");
  if (st != NV_OK) return st;
  if (per_sm < 1) return nv_fail(NV_ENOTSUP, "batch build does not fit %d threads per CTA", threads);
  const int64_t grid = std::min<int64_t>((int64_t)sms * per_sm, b->total_slices);
  if ((st = nv_cuda_check(cudaMemsetAsync(b->counter, 0, sizeof(unsigned), s), "queue reset")) != NV_OK)
    return st;
  void* args[] = {&a};
  return nv_cuda_check(cudaLaunchKernel(fn, dim3((unsigned)std::max<int64_t>(grid, 1)), dim3(threads), args, 0, s),
                       "batch_build_kernel launch");
}

static nv_status launch_batch_build(nv_batch* b, cudaStream_t s, int threads) {
  const bool rk4 = b->scheme == NV_RK4;
  const bool f64 = b->prec == NV_FP64;
#define NVPIT_BATCH_RHS(RHS)                                                            \
  if (f64) return rk4 ? launch_batch_build_T<RHS<double>, double, 1>(b, s, threads)     \
                      : launch_batch_build_T<RHS<double>, double, 0>(b, s, threads);    \
  return rk4 ? launch_batch_build_T<RHS<float>, float, 1>(b, s, threads)                \
             : launch_batch_build_T<RHS<float>, float, 0>(b, s, threads);
  switch (b->rhs_kind) {
    case NV_RHS_VDP: { NVPIT_BATCH_RHS(RhsVdp) }
    case NV_RHS_LINEAR_SCALAR: { NVPIT_BATCH_RHS(RhsLinearScalar) }
    case NV_RHS_SQUARE: { NVPIT_BATCH_RHS(RhsSquare) }
    default: return nv_fail(NV_ENOTSUP, "batched tables are built for autonomous rhs kinds 0, 1, 4");
  }
#undef NVPIT_BATCH_RHS
}

static nv_status launch_batch_compose(const nv_batch* b, const double* y0, double* yT, cudaStream_t s) {
  BatchComposeArgs a{};
  a.inst = b->inst;
  a.tables = b->tables;
  a.B = b->B;
  a.dim = b->dim;
  a.per_dim = b->per_dim;
  a.lo0 = b->lo[0];
  a.lo1 = b->lo[1];
  a.hi0 = b->hi[0];
  a.hi1 = b->hi[1];
  a.d0 = (b->hi[0] - b->lo[0]) / (b->per_dim - 1);
  a.d1 = (b->hi[1] - b->lo[1]) / (b->per_dim - 1);
  a.r0 = 1.0 / a.d0;
  a.r1 = a.d1 != 0.0 ? 1.0 / a.d1 : 0.0;
  a.y0 = y0;
  a.yT = yT;
  a.status = b->status;
  a.oob = b->oob;
  a.oob_error = b->oob_policy == NV_OOB_ERROR;
  const int block = 128;
  const int grid = (b->B + block - 1) / block;
  if (b->prec == NV_FP64)
    batch_compose_kernel<double><<<grid, block, 0, s>>>(a);
  else
    batch_compose_kernel<float><<<grid, block, 0, s>>>(a);
  return nv_cuda_check(cudaGetLastError(), "batch_compose_kernel launch");
}

static void free_batch(nv_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->inst) cudaFree(b->inst);
  if (b->items) cudaFree(b->items);
  if (b->tables) cudaFree(b->tables);
  if (b->ws) cudaFree(b->ws);
  delete b;
}

extern "C" nv_status nv_build_batch(int32_t rhs_kind, int32_t dim, int32_t B, const double* params,
                                    int32_t nparams, const double* t0, const double* T,
                                    const int32_t* S, const nv_samples* sm, const nv_steps* st,
                                    nv_batch** out, void* stream) {
  if (!out || !t0 || !T || !S || !sm || !st) return nv_fail(NV_EINVAL, "NULL argument");
  if (B < 1 || B > (1 << 24)) return nv_fail(NV_EINVAL, "B must be 1..2^24");
  if (nparams < 0 || nparams > 4 || (nparams > 0 && !params))
    return nv_fail(NV_EINVAL, "batched rhs takes 0..4 parameters per instance");
  if (rhs_kind == NV_RHS_VDP && (dim != 2 || nparams < 1))
    return nv_fail(NV_EINVAL, "Van der Pol instances have dim 2 and params {mu}");
  if ((rhs_kind == NV_RHS_LINEAR_SCALAR || rhs_kind == NV_RHS_SQUARE) && dim != 1)
    return nv_fail(NV_EINVAL, "scalar instances have dim 1");
  if (rhs_kind == NV_RHS_LINEAR_SCALAR && nparams < 1)
    return nv_fail(NV_EINVAL, "linear scalar instances need params {lambda}");
  if (rhs_kind != NV_RHS_VDP && rhs_kind != NV_RHS_LINEAR_SCALAR && rhs_kind != NV_RHS_SQUARE)
    return nv_fail(NV_ENOTSUP, "batched tables are built for autonomous rhs kinds 0, 1, 4");
  const int want_map = dim == 1 ? NV_MAP_PL1D : NV_MAP_BILINEAR2D;
  if (sm->map != want_map) return nv_fail(NV_EINVAL, "batched instances use PL1D (d=1) or BILINEAR2D (d=2)");
  if (sm->per_dim < 2 || sm->per_dim > 1024) return nv_fail(NV_EINVAL, "per_dim must be 2..1024");
  for (int i = 0; i < dim; ++i)
    if (!(sm->hi[i] > sm->lo[i])) return nv_fail(NV_EINVAL, "need lo < hi");
  if (sm->oob_policy != NV_OOB_EXTRAPOLATE && sm->oob_policy != NV_OOB_ERROR)
    return nv_fail(NV_EINVAL, "unknown out-of-range policy");
  if (st->scheme != NV_EULER && st->scheme != NV_RK4) return nv_fail(NV_EINVAL, "unknown scheme");
  if (st->prec != NV_FP64 && st->prec != NV_FP32) return nv_fail(NV_EINVAL, "batched tables are FP64 or FP32");

  nv_batch* b = new (std::nothrow) nv_batch();
  if (!b) return nv_fail(NV_ENOMEM, "host allocation of the batch");
  b->rhs_kind = rhs_kind;
  b->dim = dim;
  b->B = B;
  b->scheme = st->scheme;
  b->prec = st->prec;
  b->map = sm->map;
  b->per_dim = sm->per_dim;
  b->oob_policy = sm->oob_policy;
  for (int i = 0; i < 2; ++i) { b->lo[i] = sm->lo[i]; b->hi[i] = sm->hi[i]; }
  b->samples = dim == 1 ? sm->per_dim : sm->per_dim * sm->per_dim;
  b->elems_per_slice = (int64_t)b->samples * dim;
  b->elem_bytes = st->prec == NV_FP64 ? 8 : 4;
  b->host_inst.resize(B);
  int64_t off = 0, steps = 0;
  for (int i = 0; i < B; ++i) {
    InstDesc& d = b->host_inst[i];
    memset(&d, 0, sizeof(d));
    for (int k = 0; k < nparams; ++k) {
      if (!isfinite(params[(size_t)i * nparams + k])) { free_batch(b); return nv_fail(NV_EINVAL, "instance %d: parameter not finite", i); }
      d.p[k] = params[(size_t)i * nparams + k];
    }
    if (S[i] < 1) { free_batch(b); return nv_fail(NV_EINVAL, "instance %d: S < 1", i); }
    nv_status e = nv_plan_steps(t0[i], T[i], S[i], st->dt, st->steps_per_slice, &d.m, &d.h);
    if (e != NV_OK) { free_batch(b); return nv_fail(e, "instance %d: %s", i, nv_last_error()); }
    d.t0 = t0[i];
    d.H = (T[i] - t0[i]) / S[i];
    d.S = S[i];
    d.off = off;
    off += (int64_t)S[i] * b->elems_per_slice;
    steps += (int64_t)S[i] * d.m * b->samples;
  }
  b->traj_steps = steps;
  b->table_bytes = off * b->elem_bytes;
  // work items in decreasing cost (m_i), then instance and slice order
  std::vector<int> order(B);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return b->host_inst[x].m > b->host_inst[y].m; });
  std::vector<int2> items;
  items.reserve((size_t)(off / b->elems_per_slice));
  for (int i : order)
    for (int j = 0; j < b->host_inst[i].S; ++j) items.push_back(make_int2(i, j));
  b->total_slices = (int64_t)items.size();
  if (b->total_slices > INT32_MAX) { free_batch(b); return nv_fail(NV_EINVAL, "too many slices"); }

  nv_status e;
  cudaGetDevice(&b->device);
  if ((e = nv_cuda_check(cudaMalloc(&b->inst, sizeof(InstDesc) * B), "instance allocation")) != NV_OK ||
      (e = nv_cuda_check(cudaMalloc(&b->items, sizeof(int2) * items.size()), "work-queue allocation")) != NV_OK ||
      (e = nv_cuda_check(cudaMalloc(&b->tables, (size_t)b->table_bytes), "table allocation")) != NV_OK ||
      (e = nv_cuda_check(cudaMalloc(&b->ws, 256), "workspace allocation")) != NV_OK) {
    free_batch(b);
    return e;
  }
  b->status = static_cast<int*>(b->ws);
  b->oob = reinterpret_cast<unsigned long long*>(static_cast<char*>(b->ws) + 8);
  b->counter = reinterpret_cast<unsigned*>(static_cast<char*>(b->ws) + 16);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((e = nv_cuda_check(cudaMemcpyAsync(b->inst, b->host_inst.data(), sizeof(InstDesc) * B,
                                         cudaMemcpyHostToDevice, s), "instance upload")) != NV_OK ||
      (e = nv_cuda_check(cudaMemcpyAsync(b->items, items.data(), sizeof(int2) * items.size(),
                                         cudaMemcpyHostToDevice, s), "work-queue upload")) != NV_OK ||
      (e = nv_cuda_check(cudaMemsetAsync(b->ws, 0, 256, s), "workspace reset")) != NV_OK ||
      (e = nv_cuda_check(cudaStreamSynchronize(s), "batch set-up")) != NV_OK) {
    free_batch(b);
    return e;
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_best_threads.find(b->device);
    b->threads = it != g_best_threads.end() ? it->second : 256;
  }
  if ((e = launch_batch_build(b, s, b->threads)) != NV_OK) {
    free_batch(b);
    return e;
  }
  *out = b;
  return NV_OK;
}

extern "C" nv_status nv_batch_rebuild(nv_batch* b, void* stream) {
  if (!b) return nv_fail(NV_EINVAL, "batch is NULL");
  return launch_batch_build(b, static_cast<cudaStream_t>(stream), b->threads);
}

extern "C" nv_status nv_batch_compose(const nv_batch* b, const double* y0, double* yT, void* stream) {
  if (!b || !y0 || !yT) return nv_fail(NV_EINVAL, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  nv_status e = nv_cuda_check(cudaMemsetAsync(b->ws, 0, 16, s), "status reset");
  if (e != NV_OK) return e;
  return launch_batch_compose(b, y0, yT, s);
}

extern "C" nv_status nv_batch_run(nv_batch* b, const double* y0, double* yT, void* stream) {
  if (!b || !y0 || !yT) return nv_fail(NV_EINVAL, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  nv_status e;
  if (!b->graph || b->graph_y0 != y0 || b->graph_yT != yT) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    cudaStream_t cap;
    if ((e = nv_cuda_check(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream")) != NV_OK)
      return e;
    cudaGraph_t g = nullptr;
    e = nv_cuda_check(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (e == NV_OK) {
      nv_status e1 = launch_batch_build(b, cap, b->threads);
      nv_status e2 = e1 == NV_OK ? nv_cuda_check(cudaMemsetAsync(b->ws, 0, 16, cap), "status reset") : e1;
      nv_status e3 = e2 == NV_OK ? launch_batch_compose(b, y0, yT, cap) : e2;
      nv_status e4 = nv_cuda_check(cudaStreamEndCapture(cap, &g), "end capture");
      e = e3 != NV_OK ? e3 : e4;
    }
    if (e == NV_OK) e = nv_cuda_check(cudaGraphInstantiate(&b->graph, g, 0), "graph instantiate");
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (e != NV_OK) {
      b->graph = nullptr;
      return e;
    }
    b->graph_y0 = y0;
    b->graph_yT = yT;
  }
  return nv_cuda_check(cudaGraphLaunch(b->graph, s), "graph launch");
}

extern "C" nv_status nv_batch_autotune(nv_batch* b, void* stream, int32_t* best_threads) {
  if (!b) return nv_fail(NV_EINVAL, "batch is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  nv_status e = nv_cuda_check(cudaEventCreate(&e0), "event");
  if (e != NV_OK) return e;
  if ((e = nv_cuda_check(cudaEventCreate(&e1), "event")) != NV_OK) { cudaEventDestroy(e0); return e; }
  const int cands[] = {128, 256, 512, 1024};
  int best = b->threads;
  float best_ms = 1e30f;
  for (int c : cands) {
    if ((b->samples + c - 1) / c > 8 || c > 1024) continue;
    nv_status w = launch_batch_build(b, s, c);               // warm-up / feasibility
    if (w != NV_OK) continue;
    cudaEventRecord(e0, s);
    w = launch_batch_build(b, s, c);
    cudaEventRecord(e1, s);
    if (w != NV_OK) continue;
    if ((e = nv_cuda_check(cudaEventSynchronize(e1), "autotune timing")) != NV_OK) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) { best_ms = ms; best = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != NV_OK) return e;
  if (best != b->threads && b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  b->threads = best;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_best_threads[b->device] = best;
  }
  if (best_threads) *best_threads = best;
  return NV_OK;
}

extern "C" nv_status nv_batch_info(const nv_batch* b, int64_t* total_slices, int64_t* traj_steps,
                                   int64_t* table_bytes, int32_t* threads) {
  if (!b) return nv_fail(NV_EINVAL, "batch is NULL");
  if (total_slices) *total_slices = b->total_slices;
  if (traj_steps) *traj_steps = b->traj_steps;
  if (table_bytes) *table_bytes = b->table_bytes;
  if (threads) *threads = b->threads;
  return NV_OK;
}

extern "C" nv_status nv_batch_copy_out(const nv_batch* b, void* dst, int64_t bytes, void* stream) {
  if (!b || !dst) return nv_fail(NV_EINVAL, "NULL argument");
  if (bytes < 0 || bytes > b->table_bytes) return nv_fail(NV_EINVAL, "byte count exceeds the tables");
  return nv_cuda_check(cudaMemcpyAsync(dst, b->tables, (size_t)bytes, cudaMemcpyDefault,
                                       static_cast<cudaStream_t>(stream)), "batch copy-out");
}

extern "C" nv_status nv_batch_check(const nv_batch* b, void* stream, int64_t* oob_count) {
  if (!b) return nv_fail(NV_EINVAL, "batch is NULL");
  nv_status e = nv_cuda_check(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)), "synchronise");
  if (e != NV_OK) return e;
  struct { int status; int pad; unsigned long long oob; } h{};
  if ((e = nv_cuda_check(cudaMemcpy(&h, b->ws, sizeof(h), cudaMemcpyDeviceToHost), "status read")) != NV_OK)
    return e;
  if (oob_count) *oob_count = (int64_t)h.oob;
  if (h.status != NV_OK)
    return nv_fail((nv_status)h.status, h.status == NV_EDOMAIN ? "an evaluation left the sampled range"
                                                               : "a table value was not finite");
  return NV_OK;
}

extern "C" nv_status nv_batch_destroy(nv_batch* b) {
  if (!b) return NV_OK;
  cudaError_t ce = cudaDeviceSynchronize();
  free_batch(b);
  return nv_cuda_check(ce, "synchronise before destroy");
}
