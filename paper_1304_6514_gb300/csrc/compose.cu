// Communication phase for affine maps (Figure "pseudocode" with eq.
// linearreconstruct): lambda_j = A_j lambda_{j-1} + b_j, j = 1..S, float64.
//
// The chain is inherently sequential in j, so the kernel is a cooperative
// launch of G CTAs that stay resident for all S steps.  CTA g owns rows
// [g*rpc, (g+1)*rpc) of every product.  Per step it
//   1. issues the loads of its rows of [b_j | A_j] (independent of lambda),
//   2. waits at the grid barrier for lambda_{j-1},
//   3. stages lambda_{j-1} in shared memory, forms its rows, writes them.
// Maps are stored column-major d x (d+1) per slice with column 0 = b_j, so a
// warp's loads for one column are contiguous rows.  Each barrier wait is
// bounded and records NV_ETIMEOUT instead of hanging.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace nvpit {

struct AffineChainArgs {
  const void* maps;
  int n, S, rpc;
  const double* y0;
  double* yT;
  double* lambdas;
  double* xbuf;     // 2 * n
  unsigned* bar;
  int* status;
};

// Loads issued ahead of the barrier: up to kPre columns per thread.
constexpr int kPre = 16;

template <typename MT>
__global__ void __launch_bounds__(256) affine_chain_kernel(AffineChainArgs a) {
  extern __shared__ double sx[];  // n + 1 (sx[0] = 1 multiplies b_j)
  __shared__ int flag;
  __shared__ double red[256];
  const int n = a.n, rpc = a.rpc;
  const int tid = threadIdx.x;
  const int r = tid % rpc, cg = tid / rpc, ncg = blockDim.x / rpc;
  const int row = blockIdx.x * rpc + r;
  const bool active = (cg < ncg) && (row < n);
  const unsigned G = gridDim.x;
  const MT* maps = reinterpret_cast<const MT*>(a.maps);
  const int64_t slice_elems = (int64_t)n * (n + 1);

  if (blockIdx.x == 0 && a.lambdas)
    for (int i = tid; i < n; i += blockDim.x) a.lambdas[i] = a.y0[i];

  MT pre[kPre];
  auto prefetch = [&](int k) {
    const MT* A = maps + (int64_t)k * slice_elems;
#pragma unroll
    for (int q = 0; q < kPre; ++q) {
      const int c = cg + q * ncg;
      pre[q] = (active && c <= n) ? __ldcs(A + (int64_t)c * n + row) : (MT)0;
    }
  };
  prefetch(0);

  for (int k = 0; k < a.S; ++k) {
    const double* xin = (k == 0) ? a.y0 : a.xbuf + ((k - 1) & 1) * n;
    for (int i = tid; i < n; i += blockDim.x) sx[i + 1] = __ldcg(xin + i);
    if (tid == 0) sx[0] = 1.0;
    __syncthreads();
    double acc = 0.0;
    if (active) {
#pragma unroll
      for (int q = 0; q < kPre; ++q) {
        const int c = cg + q * ncg;
        if (c <= n) acc = fma((double)pre[q], sx[c], acc);
      }
      const MT* A = maps + (int64_t)k * slice_elems;
      for (int c = cg + kPre * ncg; c <= n; c += ncg)
        acc = fma((double)__ldcs(A + (int64_t)c * n + row), sx[c], acc);
    }
    red[tid] = acc;
    __syncthreads();
    if (tid < rpc && row < n) {
      double v = 0.0;
      for (int g = 0; g < ncg; ++g) v += red[g * rpc + tid];
      a.xbuf[(k & 1) * n + row] = v;
      if (a.lambdas) a.lambdas[(int64_t)(k + 1) * n + row] = v;
      if (k == a.S - 1) a.yT[row] = v;
    }
    if (k + 1 < a.S) {
      prefetch(k + 1);
      if (!grid_barrier(a.bar, (unsigned)(k + 1) * G, a.status, &flag)) return;
    }
  }
}

// Chain within one thread-block cluster (d <= 512): the C CTAs of a cluster
// own ceil(d/C) rows each and exchange lambda through distributed shared
// memory: after forming its rows, every CTA stores them into the next state
// buffer of all C CTAs, then the cluster's hardware barrier (release /
// acquire) orders the step.  No global-memory round trip, no spin loop.
// AT is the arithmetic type of the products: double for float64 maps, float
// for float32 maps (the float32 chain keeps its state in float).
template <typename MT, typename AT>
__global__ void __launch_bounds__(256) affine_chain_cluster_kernel(AffineChainArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank(), csize = cl.num_blocks();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = a.n, rpc = a.rpc, ld = n + 1;
  AT* xs = reinterpret_cast<AT*>(smem_raw);          // two buffers of n+1, xs[.][0] = 1
  AT* red = xs + 2 * ld;                              // blockDim partial sums
  const int tid = threadIdx.x;
  const int r = tid % rpc, cgi = tid / rpc, ncg = blockDim.x / rpc;
  const int row = (int)rank * rpc + r;
  const bool active = (cgi < ncg) && (row < n);
  const MT* maps = reinterpret_cast<const MT*>(a.maps);
  const int64_t slice_elems = (int64_t)n * (n + 1);

  for (int i = tid; i < n; i += blockDim.x) xs[1 + i] = (AT)a.y0[i];
  if (tid == 0) { xs[0] = (AT)1; xs[ld] = (AT)1; }
  if (rank == 0 && a.lambdas)
    for (int i = tid; i < n; i += blockDim.x) a.lambdas[i] = a.y0[i];

  MT pre[kPre];
  auto prefetch = [&](int k) {
    const MT* A = maps + (int64_t)k * slice_elems;
#pragma unroll
    for (int q = 0; q < kPre; ++q) {
      const int c = cgi + q * ncg;
      pre[q] = (active && c <= n) ? __ldcs(A + (int64_t)c * n + row) : (MT)0;
    }
  };
  prefetch(0);
  cl.sync();   // every CTA's buffer 0 is initialised before anyone writes buffer 1

  for (int k = 0; k < a.S; ++k) {
    const AT* x = xs + (k & 1) * ld;
    AT acc = 0;
    if (active) {
#pragma unroll
      for (int q = 0; q < kPre; ++q) {
        const int c = cgi + q * ncg;
        if (c <= n) acc = fma((AT)pre[q], x[c], acc);
      }
      const MT* A = maps + (int64_t)k * slice_elems;
      for (int c = cgi + kPre * ncg; c <= n; c += ncg)
        acc = fma((AT)__ldcs(A + (int64_t)c * n + row), x[c], acc);
    }
    red[tid] = acc;
    if (k + 1 < a.S) prefetch(k + 1);
    __syncthreads();
    if (tid < rpc && row < n) {
      AT v = 0;
      for (int g = 0; g < ncg; ++g) v += red[g * rpc + tid];
      const int nb = ((k + 1) & 1) * ld + 1 + row;
      for (unsigned p = 0; p < csize; ++p) cl.map_shared_rank(xs, p)[nb] = v;
      if (a.lambdas) a.lambdas[(int64_t)(k + 1) * n + row] = (double)v;
      if (k == a.S - 1) a.yT[row] = (double)v;
    }
    cl.sync();
  }
}

}  // namespace nvpit

using namespace nvpit;

// One cluster of up to 16 CTAs for d <= 512; returns NV_ENOTSUP if the device
// cannot hold such a cluster (the caller then takes the grid-wide chain).
static nv_status launch_affine_chain_cluster(const nv_maps* M, const double* y0, double* yT,
                                             double* lambdas, cudaStream_t s, int want_csize) {
  const int n = M->dim;
  const int block = 256;
  const bool f64 = M->prec == NV_FP64;
  const void* fn = f64 ? (const void*)affine_chain_cluster_kernel<double, double>
                       : (const void*)affine_chain_cluster_kernel<float, float>;
  const size_t esz = f64 ? sizeof(double) : sizeof(float);
  const size_t smem = esz * (2 * (size_t)(n + 1) + block);
  nv_status st = nv_cuda_check(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1),
                               "cluster size attribute");
  if (st != NV_OK) return st;
  for (int csize = want_csize > 0 ? want_csize : 16; csize >= 2; csize /= 2) {
    const int rpc = (n + csize - 1) / csize;
    if (rpc > block) break;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(csize);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      continue;
    }
    AffineChainArgs a{};
    a.maps = M->data;
    a.n = n;
    a.S = M->S;
    a.rpc = rpc;
    a.y0 = y0;
    a.yT = yT;
    a.lambdas = lambdas;
    a.status = M->status;
    void* args[] = {&a};
    return nv_cuda_check(cudaLaunchKernelExC(&cfg, fn, args), "affine_chain_cluster_kernel launch");
  }
  return nv_fail(NV_ENOTSUP, "no cluster configuration fits the chain");
}

nv_status launch_affine_chain(const nv_maps* M, const double* y0, double* yT, double* lambdas,
                              cudaStream_t s, int rows_per_cta) {
  const int n = M->dim;
  if (n <= 512 && g_tune.chain_cluster >= 0) {
    nv_status st = launch_affine_chain_cluster(M, y0, yT, lambdas, s, g_tune.chain_cluster);
    if (st != NV_ENOTSUP) return st;
  }
  const int block = 256;
  int rpc = rows_per_cta > 0 ? rows_per_cta : 16;
  rpc = std::min(rpc, block);
  while (block % rpc) --rpc;
  const int G = (n + rpc - 1) / rpc;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = sizeof(double) * (size_t)(n + 1);
  const void* fn = (M->prec == NV_FP64) ? (const void*)affine_chain_kernel<double>
                                        : (const void*)affine_chain_kernel<float>;
  if (smem > 48 * 1024) {
    nv_status st = nv_cuda_check(
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
        "chain smem attribute");
    if (st != NV_OK) return st;
  }
  nv_status st = nv_cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem),
                               "chain occupancy");
  if (st != NV_OK) return st;
  if ((int64_t)per_sm * sms < G)
    return nv_fail(NV_ENOTSUP, "chain needs %d resident CTAs, device holds %d", G, per_sm * sms);
  st = nv_cuda_check(cudaMemsetAsync(M->bar, 0, sizeof(unsigned), s), "barrier reset");
  if (st != NV_OK) return st;
  AffineChainArgs a{};
  a.maps = M->data;
  a.n = n;
  a.S = M->S;
  a.rpc = rpc;
  a.y0 = y0;
  a.yT = yT;
  a.lambdas = lambdas;
  a.xbuf = M->xbuf;
  a.bar = M->bar;
  a.status = M->status;
  void* args[] = {&a};
  return nv_cuda_check(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(block), args, smem, s),
                       "affine_chain_kernel cooperative launch");
}

nv_status launch_affine_chain_buffers(const void* maps, int prec, int n, int S, const double* y0,
                                      double* yT, double* lambdas, double* xbuf, unsigned* bar,
                                      int* status, cudaStream_t s, int rows_per_cta) {
  const int block = 256;
  int rpc = rows_per_cta > 0 ? rows_per_cta : 16;
  rpc = std::min(rpc, block);
  while (block % rpc) --rpc;
  const int G = (n + rpc - 1) / rpc;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = sizeof(double) * (size_t)(n + 1);
  const void* fn = (prec == NV_FP64) ? (const void*)affine_chain_kernel<double>
                                     : (const void*)affine_chain_kernel<float>;
  if (smem > 48 * 1024) {
    nv_status st = nv_cuda_check(
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
        "chain smem attribute");
    if (st != NV_OK) return st;
  }
  nv_status st = nv_cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem),
                               "chain occupancy");
  if (st != NV_OK) return st;
  if ((int64_t)per_sm * sms < G)
    return nv_fail(NV_ENOTSUP, "chain needs %d resident CTAs, device holds %d", G, per_sm * sms);
  AffineChainArgs a{};
  a.maps = maps;
  a.n = n;
  a.S = S;
  a.rpc = rpc;
  a.y0 = y0;
  a.yT = yT;
  a.lambdas = lambdas;
  a.xbuf = xbuf;
  a.bar = bar;
  a.status = status;
  void* args[] = {&a};
  return nv_cuda_check(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(block), args, smem, s),
                       "affine_chain_kernel cooperative launch");
}
