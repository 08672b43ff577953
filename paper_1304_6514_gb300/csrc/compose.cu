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
#include <cuda.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "chain.cuh"
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
  unsigned extra;   // barrier participants that never arrive (test hook; 0 in use)
  // tiled chain only (the float64 correction of NV_BF16_REFINE):
  const double* vadd;   // optional: v_j added to slice j's product (S x n)
  const double* base;   // optional: added to every state written (S+1 x n)
  int col0_off;         // 1: drop column 0 (b_j) of the maps
  int test_skip;        // ring chain test hook: CTA 0 never stores the partials of step test_skip - 1
};

// Loads issued ahead of the barrier: up to kPre columns per thread.
constexpr int kPre = 16;

template <typename MT, typename AT>
__global__ void __launch_bounds__(256) affine_chain_kernel(AffineChainArgs a) {
  extern __shared__ __align__(16) unsigned char sx_raw[];
  AT* sx = reinterpret_cast<AT*>(sx_raw);  // n + 1 (sx[0] = 1 multiplies b_j)
  __shared__ int flag;
  __shared__ AT red[256];
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
    for (int i = tid; i < n; i += blockDim.x) sx[i + 1] = (AT)__ldcg(xin + i);
    if (tid == 0) sx[0] = (AT)1;
    __syncthreads();
    AT acc = 0;
    if (active) {
#pragma unroll
      for (int q = 0; q < kPre; ++q) {
        const int c = cg + q * ncg;
        if (c <= n) acc = fma((AT)pre[q], sx[c], acc);
      }
      const MT* A = maps + (int64_t)k * slice_elems;
#pragma unroll 8
      for (int c = cg + kPre * ncg; c <= n; c += ncg)
        acc = fma((AT)__ldcs(A + (int64_t)c * n + row), sx[c], acc);
    }
    red[tid] = acc;
    __syncthreads();
    if (tid < rpc && row < n) {
      double v = 0.0;
      for (int g = 0; g < ncg; ++g) v += (double)red[g * rpc + tid];
      a.xbuf[(k & 1) * n + row] = v;
      if (a.lambdas) a.lambdas[(int64_t)(k + 1) * n + row] = v;
      if (k == a.S - 1) a.yT[row] = v;
    }
    if (k + 1 < a.S) {
      prefetch(k + 1);
      if (!grid_barrier(a.bar, (unsigned)(k + 1) * (G + a.extra), a.status, &flag)) return;
    }
  }
}

// Batched chains within thread-block clusters (d <= 512).  Cluster q runs
// chain q: x <- A_j x + v_j for the slices j of that chain, where A_j is a
// column-major d x d matrix and v_j a d-vector, both addressed by strides so
// that the same kernel walks the slice maps ([b_j | A_j] blocks), block-total
// matrices, or separate correction vectors.  The C CTAs of a cluster own
// ceil(d/C) rows each and exchange x through distributed shared memory:
// after forming its rows, every CTA stores them into the next state buffer of
// all C CTAs, then the cluster's hardware barrier (release / acquire) orders
// the step.  No global-memory round trip, no spin loop.  AT is the arithmetic
// type: double for float64 maps, float for float32 maps.

template <typename MT, typename AT>
__global__ void __launch_bounds__(256) affine_chains_kernel(ChainsArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank(), csize = cl.num_blocks();
  const int q = (int)(blockIdx.x / csize);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = a.n, rpc = a.rpc;
  AT* xs = reinterpret_cast<AT*>(smem_raw);           // two state buffers of n
  AT* red = xs + 2 * n;                                // blockDim partial sums
  const int tid = threadIdx.x;
  const int r = tid % rpc, cgi = tid / rpc, ncg = blockDim.x / rpc;
  const int row = (int)rank * rpc + r;
  const bool active = (cgi < ncg) && (row < n);
  const MT* Ab = reinterpret_cast<const MT*>(a.A);
  const int j0 = q * a.len;
  const int len = min(a.len, a.S - j0);

  const double* x0 = a.x0 ? a.x0 + (int64_t)q * a.x0_stride : nullptr;
  for (int i = tid; i < n; i += blockDim.x) xs[i] = x0 ? (AT)x0[i] : (AT)0;
  if (q == 0 && rank == 0 && a.write_state0 && a.states)
    for (int i = tid; i < n; i += blockDim.x)
      a.states[i] = (x0 ? x0[i] : 0.0) + (a.add ? a.add[i] : 0.0);

  // Loads of A_j are independent of x: they are issued two steps ahead into
  // two register sets, so HBM latency overlaps two cluster barriers.
  MT pa[kPre], pb[kPre];
  auto prefetch = [&](MT* pre, int k) {
    const MT* A = Ab + (int64_t)(j0 + k) * a.a_stride;
#pragma unroll
    for (int qq = 0; qq < kPre; ++qq) {
      const int c = cgi + qq * ncg;
      pre[qq] = (active && c < n) ? __ldcs(A + (int64_t)c * n + row) : (MT)0;
    }
  };
  auto step = [&](MT* pre, int k) {
    const int j = j0 + k;
    const AT* x = xs + (k & 1) * n;
    AT acc = 0;
    if (active) {
#pragma unroll
      for (int qq = 0; qq < kPre; ++qq) {
        const int c = cgi + qq * ncg;
        if (c < n) acc = fma((AT)pre[qq], x[c], acc);
      }
      const MT* A = Ab + (int64_t)j * a.a_stride;
      for (int c = cgi + kPre * ncg; c < n; c += ncg)
        acc = fma((AT)__ldcs(A + (int64_t)c * n + row), x[c], acc);
    }
    red[tid] = acc;
    if (k + 2 < len) prefetch(pre, k + 2);
    __syncthreads();
    if (tid < rpc && row < n) {
      AT s = 0;
      for (int g = 0; g < ncg; ++g) s += red[g * rpc + tid];
      AT vj = a.v_double ? (AT)(reinterpret_cast<const double*>(a.v)[(int64_t)j * a.v_stride + row])
                         : (AT)(reinterpret_cast<const MT*>(a.v)[(int64_t)j * a.v_stride + row]);
      s += vj;
      const int nb = ((k + 1) & 1) * n + row;
      for (unsigned p = 0; p < csize; ++p) cl.map_shared_rank(xs, p)[nb] = s;
      const int64_t o = (int64_t)(j + 1) * n + row;
      const double out = (double)s + (a.add ? a.add[o] : 0.0);
      if (a.states) a.states[o] = out;
      if (a.yT && j == a.S - 1) a.yT[row] = out;
      if (a.finals && k == len - 1) a.finals[(int64_t)q * n + row] = (double)s;
    }
    cl.sync();
  };
  if (len > 0) prefetch(pa, 0);
  if (len > 1) prefetch(pb, 1);
  cl.sync();   // every CTA's first buffer is initialised before anyone writes the second
  for (int k = 0; k < len; k += 2) {
    step(pa, k);
    if (k + 1 < len) step(pb, k + 1);
  }
}

template <typename MT, typename AT>
__global__ void __launch_bounds__(256) affine_chains_tma_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                ChainsArgs a, int* status) {
  cluster_chain_run<MT, AT>(&tmA, a, status, (int)(blockIdx.x / cg::this_cluster().num_blocks()),
                            ChainNoHooks{});
}

// acc[0..VEC) += (the VEC map entries in t) * xc, for one column of a tile:
// VEC consecutive rows of MT (bfloat16 as the high halves of float32 words).
template <typename MT, typename AT, int VEC, typename V>
__device__ __forceinline__ void tile_madd(AT* acc, const V& t, AT xc) {
  if constexpr (sizeof(MT) == 2) {
    const uint32_t w[2] = {t.x, t.y};
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      acc[2 * i] = fma((AT)__uint_as_float(w[i] << 16), xc, acc[2 * i]);
      acc[2 * i + 1] = fma((AT)__uint_as_float(w[i] & 0xffff0000u), xc, acc[2 * i + 1]);
    }
  } else if constexpr (VEC == 4) {
    acc[0] = fma((AT)t.x, xc, acc[0]);
    acc[1] = fma((AT)t.y, xc, acc[1]);
    acc[2] = fma((AT)t.z, xc, acc[2]);
    acc[3] = fma((AT)t.w, xc, acc[3]);
  } else {
    acc[0] = fma((AT)t.x, xc, acc[0]);
    acc[1] = fma((AT)t.y, xc, acc[1]);
  }
}

// Grid-wide chain for large d (d > 512, d a multiple of 4).  CTA (rb, cb)
// owns a tile of the slice map: rows [rb*RB, rb*RB + RB) of the column block
// [cb*cpc, (cb+1)*cpc) of [b_j | A_j].  A column of the tile is RB contiguous
// values (8 KB for float32), so the map streams in long runs; each thread reads
// VEC consecutive rows with one 16-byte (bfloat16: 8-byte) load per column.
// Step k stores the tile's partial row sums, one 16-byte store per thread, in
// the partial buffer k % 2 (a row of ncb values per state component), and one
// bounded grid barrier per step orders the steps.  Step k + 1 then sums, for
// its own column block only, the ncb partials of each state component it
// multiplies (ncb * cpc L2 reads per CTA) and the row-block-0 CTAs write those
// states out: no atomics, no buffer to clear, and a fixed summation order.
template <typename MT, typename AT>
__global__ void __launch_bounds__(512, 1) affine_chain_tile_kernel(AffineChainArgs a, int nrb, int cpc,
                                                                AT* part) {
  // MT: double, float, or uint16_t holding bfloat16 bits.  Rows per thread:
  // 2 (double), 4 (float, and bfloat16 as 8-byte loads: 8 rows per thread
  // would halve the column blocks' row count and double the partial sums
  // per state component)
  constexpr int VEC = sizeof(MT) == 2 ? 4 : 16 / (int)sizeof(MT);
  static_assert(VEC * sizeof(AT) == 16, "one 16-byte partial store per thread");
  using V = typename std::conditional<sizeof(MT) == 4, float4,
                                      typename std::conditional<sizeof(MT) == 8, double2, uint2>::type>::type;
  extern __shared__ __align__(16) unsigned char sxt_raw[];
  AT* sx = reinterpret_cast<AT*>(sxt_raw);    // the cpc state values of this column block
  AT* red = sx + ((cpc + 3) & ~3);            // max(blockDim.x, cpc) group sums
  __shared__ int flag;
  const int n = a.n;
  const int RB = VEC * blockDim.x;
  const int rb = blockIdx.x % nrb, cb = blockIdx.x / nrb;
  const int ncb = gridDim.x / nrb;
  const int tid = threadIdx.x;
  const int row0 = rb * RB + tid * VEC;
  const bool active = row0 < n;
  const int c0 = cb * cpc, c1 = min(n + 1, c0 + cpc);
  const int ncols = max(0, c1 - c0);
  const int ngrp = ncols > 0 ? max(1, (int)blockDim.x / ncols) : 1;
  const unsigned G = gridDim.x;
  const MT* maps = reinterpret_cast<const MT*>(a.maps);
  const int64_t slice_elems = (int64_t)n * (n + 1);
  if (blockIdx.x == 0 && a.lambdas)
    for (int i = tid; i < n; i += blockDim.x) a.lambdas[i] = a.y0[i] + (a.base ? a.base[i] : 0.0);
  const AT one = a.col0_off ? (AT)0 : (AT)1;

  // sx <- the state after kk steps for this block's columns, summed from the
  // partials of step kk - 1; CTAs of row block 0 write it out (+ base).
  auto gather = [&](int kk) {
    const AT* P = part + (size_t)((kk - 1) & 1) * ncb * n;
    for (int p = tid; p < ncols * ngrp; p += blockDim.x) {
      const int j = p % ncols, g = p / ncols;
      const int i = c0 + j - 1;   // state component multiplied by column c0 + j
      AT sum = 0;
      if (i >= 0)
        for (int b0 = g; b0 < ncb; b0 += 8 * ngrp) {
          AT v[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int b = b0 + q * ngrp;
            v[q] = b < ncb ? __ldcg(P + (size_t)b * n + i) : (AT)0;
          }
#pragma unroll
          for (int q = 0; q < 8; ++q) sum += v[q];
        }
      red[g * ncols + j] = sum;
    }
    __syncthreads();
    for (int j = tid; j < ncols; j += blockDim.x) {
      const int c = c0 + j;
      AT sum = 0;
      for (int g = 0; g < ngrp; ++g) sum += red[g * ncols + j];
      sx[j] = c == 0 ? one : sum;
      if (rb == 0 && c > 0) {
        const int64_t o = (int64_t)kk * n + c - 1;
        const double xv = (double)sum + (a.base ? a.base[o] : 0.0);
        if (a.lambdas) a.lambdas[o] = xv;
        if (kk == a.S && a.yT) a.yT[c - 1] = xv;
      }
    }
  };

  // batches of kBatch independent loads in flight per thread; the last batch
  // of a column block is predicated
  constexpr int kBatch = 16;
  V t[kBatch];
  auto load_batch = [&](const MT* A, int c) {
#pragma unroll
    for (int q = 0; q < kBatch; ++q)
      if (c + q < c1) t[q] = __ldg(reinterpret_cast<const V*>(A + (int64_t)(c + q) * n));
  };
  // the first batch of every step is loaded before the barrier that ends the
  // previous step (it does not depend on the state), so the map stream runs
  // while the grid waits
  if (active) load_batch(maps + row0, c0);
  for (int k = 0; k < a.S; ++k) {
    if (k == 0) {
      for (int c = c0 + tid; c < c1; c += blockDim.x) sx[c - c0] = c == 0 ? one : (AT)a.y0[c - 1];
    } else {
      gather(k);
    }
    __syncthreads();
    if (active) {
      AT acc[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) acc[v] = 0;
      const MT* A = maps + (int64_t)k * slice_elems + row0;
      for (int c = c0; c < c1; c += kBatch) {
        if (c != c0) load_batch(A, c);
#pragma unroll
        for (int q = 0; q < kBatch; ++q)
          if (c + q < c1) tile_madd<MT, AT, VEC>(acc, t[q], sx[c + q - c0]);
      }
      if (a.vadd && cb == 0) {
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] += (AT)a.vadd[(int64_t)k * n + row0 + v];
      }
      AT* dst = part + ((size_t)(k & 1) * ncb + cb) * n + row0;
      if constexpr (sizeof(AT) == 4)
        __stcg(reinterpret_cast<float4*>(dst), make_float4(acc[0], acc[1], acc[2], acc[3]));
      else
        __stcg(reinterpret_cast<double2*>(dst), make_double2(acc[0], acc[1]));
      if (k + 1 < a.S) load_batch(A + slice_elems, c0);
    }
    if (!grid_barrier(a.bar, (unsigned)(k + 1) * G, a.status, &flag)) return;
  }
  if (rb == 0) gather(a.S);
}

// The same tiled chain with the map stream decoupled from the arithmetic and
// no grid barrier.
//
// Stream: one producer lane copies the CTA's tile, column segments of RB rows,
// into a ring of kTileStages shared-memory stages with bulk asynchronous
// copies that complete on the stage's mbarrier; 16 consumer warps multiply
// each stage by the state and release it.  The producer's sequence of stages
// runs over all S steps without regard to the state, so while the consumers
// wait for the next state it keeps streaming the next map into the free
// stages.
//
// Exchange: each partial row sum is stored as one 64-bit word, a 32-bit
// payload (a float32, or one half of a float64) beside the 32-bit tag k + 1 of
// the step that produced it.  An aligned 64-bit store or load is single-copy
// atomic, so a reader that polls the words it needs until their tags read
// k + 1 has the values themselves: no fence, no counter, no barrier, and each
// CTA waits only for the partials its own columns multiply.  Step k writes
// buffer k % 3.  Overwriting it at step k + 3 is safe: a CTA at step t has
// read partials of step t - 1 from every column block of some row block,
// whose columns together span all n + 1 columns, so those CTAs had read the
// partials of step t - 2 from every CTA, i.e. every CTA had finished reading
// step t - 3's buffer.  The buffers are cleared before each launch so that no
// tag from an earlier launch matches.
//
// Consumers synchronise among themselves with named barrier 1; the producer
// warp joins no block-wide barrier after the set-up.  Every wait is bounded
// (1 s); a thread that gives up records NV_ETIMEOUT in the status word and
// sets the CTA's abort flag, after which no thread of the CTA waits again, the
// producer stops issuing and waits for its copies in flight, and the
// consumers run out their loops without waiting.
constexpr int kTileConsumers = 512;
constexpr int kTileStageBytes = 16 * 1024;
constexpr int kTileStages = 12;
constexpr int kTagBuffers = 3;

__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kTileConsumers) : "memory");
}

__device__ __forceinline__ void ring_release(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(cta_smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   cta_smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(cta_smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void st_tagged(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_tagged(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// 64-bit words per partial value: the value's 32-bit pieces, each with a tag.
template <typename AT>
constexpr int tag_words() { return (int)sizeof(AT) / 4; }

__device__ __forceinline__ void tag_pack(float x, uint32_t tag, unsigned long long* w) {
  w[0] = ((unsigned long long)tag << 32) | __float_as_uint(x);
}
__device__ __forceinline__ void tag_pack(double x, uint32_t tag, unsigned long long* w) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  w[0] = ((unsigned long long)tag << 32) | (u & 0xffffffffull);
  w[1] = ((unsigned long long)tag << 32) | (u >> 32);
}
__device__ __forceinline__ float tag_value(const unsigned long long* w, float*) {
  return __uint_as_float((uint32_t)w[0]);
}
__device__ __forceinline__ double tag_value(const unsigned long long* w, double*) {
  return __longlong_as_double((long long)((w[1] << 32) | (w[0] & 0xffffffffull)));
}

template <typename MT, typename AT>
__global__ void __launch_bounds__(kTileConsumers + 32, 1)
    affine_chain_ring_kernel(AffineChainArgs a, int nrb, int cpc, unsigned long long* part) {
  constexpr int VEC = sizeof(MT) == 2 ? 4 : 16 / (int)sizeof(MT);
  constexpr int W = tag_words<AT>();
  using V = typename std::conditional<sizeof(MT) == 4, float4,
                                      typename std::conditional<sizeof(MT) == 8, double2, uint2>::type>::type;
  constexpr int RB = VEC * kTileConsumers;                       // rows of a tile
  constexpr int CPS = kTileStageBytes / (RB * (int)sizeof(MT));  // columns per stage
  static_assert(CPS >= 1 && CPS * RB * (int)sizeof(MT) == kTileStageBytes, "whole columns per stage");
  extern __shared__ __align__(128) unsigned char ring_raw[];
  MT* ring = reinterpret_cast<MT*>(ring_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(ring_raw + kTileStages * kTileStageBytes);
  uint64_t* empty = full + kTileStages;
  AT* sx = reinterpret_cast<AT*>(empty + kTileStages);   // the cpc state values of this column block
  AT* red = sx + ((cpc + 3) & ~3);                        // max(kTileConsumers, cpc) group sums
  __shared__ volatile int s_abort;
  const int n = a.n;
  const int rb = blockIdx.x % nrb, cb = blockIdx.x / nrb;
  const int ncb = gridDim.x / nrb;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = rb * RB + tid * VEC;
  const bool active = tid < kTileConsumers && row0 < n;
  const int c0 = cb * cpc, c1 = min(n + 1, c0 + cpc);
  const int ncols = max(0, c1 - c0);
  const int nst = (ncols + CPS - 1) / CPS;                // stages per step
  const int rows = min(RB, n - rb * RB);
  const uint32_t seg_bytes = (uint32_t)rows * (uint32_t)sizeof(MT);
  const MT* maps = reinterpret_cast<const MT*>(a.maps);
  const int64_t slice_elems = (int64_t)n * (n + 1);
  const size_t buf_words = (size_t)ncb * n * W;
  if (tid == 0) {
    for (int i = 0; i < kTileStages; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(cta_smem_u32(&full[i])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(cta_smem_u32(&empty[i])),
                   "n"(kTileConsumers / 32)
                   : "memory");
    }
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == kTileConsumers / 32) {   // producer
    if (lane == 0 && nst > 0) {
      // stage g = (step k, stage st of the step) in ring slot g % kTileStages;
      // all cursors advance incrementally (no 64-bit divisions in this loop)
      const int64_t total = (int64_t)a.S * nst;
      const MT* tile0 = maps + (int64_t)c0 * n + (int64_t)rb * RB;   // step 0, stage 0
      const int64_t step_stride = slice_elems, stage_stride = (int64_t)CPS * n;
      auto stage_cols = [&](int st) { return min(CPS, ncols - st * CPS); };
      const MT* src = tile0;                 // stage g
      int st = 0, slot = 0;
      uint32_t parity = 1;                   // phase parity of the stage's previous use
      int64_t g = 0;
      for (; g < total && !s_abort; ++g) {
        if (g >= kTileStages) {   // wait until the consumers free this stage
          if (!ring_wait(&empty[slot], parity)) {
            record_status(a.status, NV_ETIMEOUT);
            s_abort = 1;
            break;
          }
        }
        const int cnt = stage_cols(st);
        arm_tx(&full[slot], (uint32_t)cnt * seg_bytes);
        MT* dst = ring + (size_t)slot * CPS * RB;
        for (int q = 0; q < cnt; ++q) bulk_load(dst + q * RB, src + (int64_t)q * n, seg_bytes, &full[slot]);
        if (++st == nst) {
          st = 0;
          src += step_stride - (int64_t)(nst - 1) * stage_stride;
        } else {
          src += stage_stride;
        }
        if (++slot == kTileStages) {
          slot = 0;
          parity ^= 1;
        }
      }
      // no copy may land in the shared memory of an exited CTA: wait for the
      // last stages issued (the consumers have already taken them unless a
      // wait gave up)
      for (int64_t gg = g > kTileStages ? g - kTileStages : 0; gg < g; ++gg)
        ring_wait(&full[gg % kTileStages], (uint32_t)((gg / kTileStages) & 1));
    }
    return;
  }

  // consumers: threads 0 .. kTileConsumers-1
  const int ngrp = ncols > 0 ? max(1, kTileConsumers / ncols) : 1;
  if (blockIdx.x == 0 && a.lambdas)
    for (int i = tid; i < n; i += kTileConsumers) a.lambdas[i] = a.y0[i] + (a.base ? a.base[i] : 0.0);
  const AT one = a.col0_off ? (AT)0 : (AT)1;
  // sx <- the state after kk steps for this block's columns.  First one
  // thread per source column block polls one sentinel word of that block (the
  // first state component this CTA needs) until its tag reads kk: a source
  // block's rows are stored together at the end of its step, so the rest is
  // then almost always there too, and polling one word per source keeps the
  // L2 traffic of the wait small.  Then thread (j, g) loads the partials of
  // column blocks g, g + ngrp, ... for state component c0 + j - 1, re-polls
  // any whose tag is not yet kk, and sums them in that order; CTAs of row
  // block 0 write the state out (+ base).
  const int i_sent = max(c0 - 1, 0);
  const bool needs_state = c1 - 1 > i_sent;
  auto gather = [&](int kk) {
    const unsigned long long* P = part + (size_t)((kk - 1) % kTagBuffers) * buf_words;
    auto poll = [&](const unsigned long long* p) {   // bounded; returns the word read last
      unsigned long long v = ld_tagged(p);
      uint64_t t0 = 0;
      while ((uint32_t)(v >> 32) != (uint32_t)kk && !s_abort) {
        uint64_t t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t0 == 0) {
          t0 = t;
        } else if (t - t0 > 1000000000ull) {
          record_status(a.status, NV_ETIMEOUT);
          s_abort = 1;
        }
        __nanosleep(20);
        v = ld_tagged(p);
      }
      return v;
    };
    if (needs_state)
      for (int b = tid; b < ncb; b += kTileConsumers) poll(P + ((size_t)b * n + i_sent) * W);
    consumers_sync();
    for (int p = tid; p < ncols * ngrp; p += kTileConsumers) {
      const int j = p % ncols, g = p / ncols;
      const int i = c0 + j - 1;   // state component multiplied by column c0 + j
      AT sum = 0;
      if (i >= 0)
        for (int b0 = g; b0 < ncb; b0 += 8 * ngrp) {
          unsigned long long v[8][W];
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (b0 + q * ngrp < ncb)
#pragma unroll
              for (int w = 0; w < W; ++w) v[q][w] = ld_tagged(P + ((size_t)(b0 + q * ngrp) * n + i) * W + w);
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (b0 + q * ngrp < ncb) {
#pragma unroll
              for (int w = 0; w < W; ++w)
                if ((uint32_t)(v[q][w] >> 32) != (uint32_t)kk)
                  v[q][w] = poll(P + ((size_t)(b0 + q * ngrp) * n + i) * W + w);
              sum += tag_value(v[q], (AT*)nullptr);
            }
        }
      red[g * ncols + j] = sum;
    }
    consumers_sync();
    for (int j = tid; j < ncols; j += kTileConsumers) {
      const int c = c0 + j;
      AT sum = 0;
      for (int g = 0; g < ngrp; ++g) sum += red[g * ncols + j];
      sx[j] = c == 0 ? one : sum;
      if (rb == 0 && c > 0) {
        const int64_t o = (int64_t)kk * n + c - 1;
        const double xv = (double)sum + (a.base ? a.base[o] : 0.0);
        if (a.lambdas) a.lambdas[o] = xv;
        if (kk == a.S && a.yT) a.yT[c - 1] = xv;
      }
    }
  };
  int cslot = 0;          // ring slot and phase parity of the next stage
  uint32_t cphase = 0;
  for (int k = 0; k < a.S; ++k) {
    if (k == 0) {
      for (int c = c0 + tid; c < c1; c += kTileConsumers) sx[c - c0] = c == 0 ? one : (AT)a.y0[c - 1];
    } else {
      gather(k);
    }
    consumers_sync();
    AT acc[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[v] = 0;
    for (int st = 0; st < nst; ++st) {
      const int slot = cslot;
      const uint32_t cpar = cphase;
      if (++cslot == kTileStages) {
        cslot = 0;
        cphase ^= 1;
      }
      bool ok = !s_abort;
      if (ok && !ring_wait(&full[slot], cpar)) {
        record_status(a.status, NV_ETIMEOUT);
        s_abort = 1;
        ok = false;
      }
      if (ok && active) {
        const MT* seg = ring + (size_t)slot * CPS * RB + tid * VEC;
#pragma unroll
        for (int q = 0; q < CPS; ++q) {
          if (st * CPS + q < ncols)
            tile_madd<MT, AT, VEC>(acc, *reinterpret_cast<const V*>(seg + q * RB), sx[st * CPS + q]);
        }
      }
      __syncwarp();
      if (lane == 0) ring_release(&empty[slot]);
    }
    if (active) {
      if (a.vadd && cb == 0) {
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] += (AT)a.vadd[(int64_t)k * n + row0 + v];
      }
      unsigned long long* dst = part + (size_t)(k % kTagBuffers) * buf_words + ((size_t)cb * n + row0) * W;
      if (!(a.test_skip == k + 1 && blockIdx.x == 0))
#pragma unroll
      for (int v = 0; v < VEC; ++v) {
        unsigned long long w[W];
        tag_pack(acc[v], (uint32_t)(k + 1), w);
#pragma unroll
        for (int q = 0; q < W; ++q) st_tagged(dst + v * W + q, w[q]);
      }
    }
  }
  if (rb == 0) gather(a.S);
}

}  // namespace nvpit

using namespace nvpit;

typedef CUresult (*EncodeTiledFnC)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                   CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                   CUtensorMapFloatOOBfill);

static nv_status chain_encode_fn(EncodeTiledFnC* out) {
  static std::mutex mu;
  static EncodeTiledFnC fn = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult qr;
    nv_status st = nv_cuda_check(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                                  cudaEnableDefault, &qr),
                                 "driver entry point cuTensorMapEncodeTiled");
    if (st != NV_OK) return st;
    if (qr != cudaDriverEntryPointSuccess || !p)
      return nv_fail(NV_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    fn = reinterpret_cast<EncodeTiledFnC>(p);
  }
  *out = fn;
  return NV_OK;
}

// Launch nchains clusters of up to `want_csize` CTAs (0 = as large as fits,
// up to 16); NV_ENOTSUP if no cluster shape fits the device.
// TMA-fed chains: 16-CTA clusters, 16 rows per CTA (d <= 256, d % 4 == 0,
// 16-byte aligned matrices and strides).  NV_ENOTSUP if the shape or device
// does not allow it (the caller then takes the register-prefetch kernel).
nv_status chain_tma_prepare(const ChainsArgs& args_in, bool f64, CUtensorMap* tmap, size_t* smem) {
  const int n = args_in.n;
  const int block = 256, rpc = kChainRpc;
  const size_t esz = f64 ? 8 : 4;
  if (n > 256 || n < 64 || n % 16 != 0) return NV_ENOTSUP;
  if (((uintptr_t)args_in.A % 16) || ((args_in.a_stride * esz) % 16)) return NV_ENOTSUP;
  const size_t vsz = args_in.v_double ? 8 : esz;
  if (((uintptr_t)args_in.v % 16) || ((args_in.v_stride * vsz) % 16)) return NV_ENOTSUP;
  if (args_in.add && ((uintptr_t)args_in.add % 16)) return NV_ENOTSUP;
  EncodeTiledFnC enc = nullptr;
  nv_status st = chain_encode_fn(&enc);
  if (st != NV_OK) return st;
  const cuuint64_t gdim[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)args_in.S};
  const cuuint64_t gstride[2] = {(cuuint64_t)n * esz, (cuuint64_t)args_in.a_stride * esz};
  const int wcols = chain_band_cols(n, args_in.band);
  const cuuint32_t box[3] = {(cuuint32_t)rpc, (cuuint32_t)wcols, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult cr = enc(tmap, f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                    const_cast<void*>(args_in.A), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return NV_ENOTSUP;
  *smem = esz * (size_t)kRing * rpc * wcols + 2 * 8 * (size_t)kRing * rpc + esz * (2 * (size_t)n + 2 * block) +
          8 * (kRing + 2) + 16;
  return NV_OK;
}

static nv_status launch_chains_tma(const ChainsArgs& args_in, bool f64, cudaStream_t s, int* status) {
  const int block = 256, csize = 16, rpc = kChainRpc;
  CUtensorMap tmap;
  size_t smem = 0;
  nv_status st = chain_tma_prepare(args_in, f64, &tmap, &smem);
  if (st != NV_OK) return st;
  const void* fn = f64 ? (const void*)affine_chains_tma_kernel<double, double>
                       : (const void*)affine_chains_tma_kernel<float, float>;
  if ((st = nv_cuda_check(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1),
                          "cluster size attribute")) != NV_OK)
    return st;
  if ((st = nv_cuda_check(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                          "chain smem attribute")) != NV_OK)
    return st;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(csize * args_in.nchains));
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
    return NV_ENOTSUP;
  }
  ChainsArgs a = args_in;
  a.rpc = rpc;
  void* args[] = {&tmap, &a, &status};
  return nv_cuda_check(cudaLaunchKernelExC(&cfg, fn, args), "affine_chains_tma_kernel launch");
}

nv_status launch_chains(const ChainsArgs& args_in, bool f64, cudaStream_t s, int want_csize) {
  const int n = args_in.n;
  const int block = 256;
  if (n > 512) return nv_fail(NV_ENOTSUP, "cluster chains need d <= 512");
  if (want_csize <= 0 || want_csize == 16) {
    nv_status st = launch_chains_tma(args_in, f64, s, args_in.status);
    if (st != NV_ENOTSUP) return st;
  }
  const void* fn = f64 ? (const void*)affine_chains_kernel<double, double>
                       : (const void*)affine_chains_kernel<float, float>;
  const size_t esz = f64 ? sizeof(double) : sizeof(float);
  const size_t smem = esz * (2 * (size_t)n + block);
  nv_status st = nv_cuda_check(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1),
                               "cluster size attribute");
  if (st != NV_OK) return st;
  for (int csize = want_csize > 0 ? want_csize : 16; csize >= 1; csize /= 2) {
    const int rpc = (n + csize - 1) / csize;
    if (rpc > block) break;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(csize * args_in.nchains));
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
    ChainsArgs a = args_in;
    a.rpc = rpc;
    void* args[] = {&a};
    return nv_cuda_check(cudaLaunchKernelExC(&cfg, fn, args), "affine_chains_kernel launch");
  }
  return nv_fail(NV_ENOTSUP, "no cluster configuration fits the chain");
}

static nv_status launch_affine_chain_cluster(const nv_maps* M, const double* y0, double* yT,
                                             double* lambdas, cudaStream_t s, int want_csize) {
  const int n = M->dim;
  const bool f64 = M->prec == NV_FP64;
  const size_t esz = f64 ? sizeof(double) : sizeof(float);
  ChainsArgs a{};
  a.n = n;
  a.nchains = 1;
  a.len = M->S;
  a.S = M->S;
  a.A = static_cast<const char*>(M->data) + esz * n;   // column 1 of slice 0's block
  a.a_stride = (int64_t)n * (n + 1);
  a.v = M->data;                                       // column 0 = b_j
  a.v_stride = (int64_t)n * (n + 1);
  a.x0 = y0;
  a.states = lambdas;
  a.yT = yT;
  a.write_state0 = 1;
  a.status = M->status;
  a.band = g_tune.chain_dense ? 0 : M->band;
  return launch_chains(a, f64, s, want_csize);
}

size_t tile_chain_ring_scratch(int n, int ncb, int value_bytes) {
  return (size_t)kTagBuffers * ncb * n * (value_bytes / 4) * sizeof(unsigned long long);
}

size_t tile_chain_scratch_bytes(int prec, int n, int sms) {
  const bool f64 = prec == NV_FP64;
  const int rb = f64 ? 2 * 512 : 4 * 512;   // rows per tile: VEC x 512 threads
  const int ncb = std::max(1, sms / ((n + rb - 1) / rb));
  const int esz = f64 ? 8 : 4;
  return std::max(tile_chain_ring_scratch(n, ncb, esz), (size_t)esz * 2 * ncb * n);
}

// Tiled grid-wide chain (d > 512, d % 4 == 0): one CTA per SM, row blocks of
// 2048 (float32, bfloat16) / 1024 (float64) rows, column blocks sized to fill
// the grid.  Tunable 9 selects the kernel (default: the register kernel for
// float32 maps, the bulk-copy ring for float64 and bfloat16 maps, whose
// columns must then be 16-byte aligned).
template <typename MT, typename AT>
static nv_status tile_chain(const nv_maps* M, const double* y0, double* yT, double* lambdas,
                            const TileChainExtra* ex, cudaStream_t s) {
  const int n = M->dim;
  const int block = 512;
  const int vec = sizeof(MT) == 2 ? 4 : 16 / (int)sizeof(MT);
  const int RB = vec * block;
  const int nrb = (n + RB - 1) / RB;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ncb = std::max(1, sms / nrb);
  const int cpc = (n + 1 + ncb - 1) / ncb;
  const int G = nrb * ncb;
  const size_t esz = sizeof(AT);
  const size_t state_smem = esz * ((size_t)((cpc + 3) & ~3) + (size_t)std::max(block, cpc));
  // the bulk-copy ring needs 16-byte aligned column segments
  // measured at d = 4096, S = 512: the ring is faster for float64 maps
  // (16.9 vs 19.4 ms) and bfloat16 maps (5.0 vs 5.2 ms), the register kernel
  // for float32 maps (6.8 vs 7.0 ms)
  const int form = g_tune.tile_chain_form != 0 ? g_tune.tile_chain_form : (sizeof(MT) == 4 ? 1 : 2);
  const bool ring = form == 2 && ((uintptr_t)M->data & 15) == 0 && ((size_t)n * sizeof(MT)) % 16 == 0;
  const void* fn = ring ? (const void*)affine_chain_ring_kernel<MT, AT>
                        : (const void*)affine_chain_tile_kernel<MT, AT>;
  const int threads = ring ? kTileConsumers + 32 : block;
  const size_t smem = ring ? (size_t)kTileStages * kTileStageBytes + 2 * kTileStages * sizeof(uint64_t) + state_smem
                           : state_smem;
  nv_status st;
  if (ring && (st = nv_cuda_check(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                                  "ring chain smem attribute")) != NV_OK)
    return st;
  int per_sm = 0;
  if ((st = nv_cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem),
                          "chain occupancy")) != NV_OK)
    return st;
  if ((int64_t)per_sm * sms < G)
    return nv_fail(NV_ENOTSUP, "chain needs %d resident CTAs, device holds %d", G, per_sm * sms);
  // the partial sums after the float64 chain vectors: two buffers of ncb x n
  // values (register kernel) or three of tagged 64-bit words (ring kernel)
  const size_t part_bytes = ring ? tile_chain_ring_scratch(n, ncb, (int)esz) : esz * 2 * (size_t)ncb * (size_t)n;
  if (M->ws_bytes < 256 + sizeof(double) * 2 * (size_t)n + 16 + part_bytes)
    return nv_fail(NV_ENOTSUP, "workspace too small for the tiled chain");
  void* xb = reinterpret_cast<char*>(M->xbuf) + sizeof(double) * 2 * (size_t)n;
  xb = reinterpret_cast<void*>(((uintptr_t)xb + 15) & ~(uintptr_t)15);
  if ((st = nv_cuda_check(cudaMemsetAsync(M->bar, 0, sizeof(unsigned), s), "barrier reset")) != NV_OK)
    return st;
  if (ring && (st = nv_cuda_check(cudaMemsetAsync(xb, 0, part_bytes, s), "tag reset")) != NV_OK) return st;
  AffineChainArgs a{};
  a.maps = M->data;
  a.n = n;
  a.S = M->S;
  a.rpc = 0;
  a.y0 = y0;
  a.yT = yT;
  a.lambdas = lambdas;
  a.xbuf = M->xbuf;
  a.bar = M->bar;
  a.status = M->status;
  if (ex) {
    a.vadd = ex->vadd;
    a.base = ex->base;
    a.col0_off = ex->col0_off;
  }
  a.test_skip = g_tune.test_skip_partials;
  int nrb_arg = nrb, cpc_arg = cpc;
  void* args[] = {&a, &nrb_arg, &cpc_arg, &xb};
  return nv_cuda_check(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(threads), args, smem, s),
                       "tiled chain cooperative launch");
}

nv_status launch_tile_chain(const nv_maps* M, const double* y0, double* yT, double* lambdas,
                            const TileChainExtra* ex, cudaStream_t s) {
  if (M->prec == NV_FP64) return tile_chain<double, double>(M, y0, yT, lambdas, ex, s);
  if (M->prec == NV_BF16_REFINE) {
    if (M->dim % 8) return nv_fail(NV_ENOTSUP, "bfloat16 chain needs d %% 8 == 0");
    return tile_chain<uint16_t, float>(M, y0, yT, lambdas, ex, s);
  }
  return tile_chain<float, float>(M, y0, yT, lambdas, ex, s);
}

nv_status launch_affine_chain(const nv_maps* M, const double* y0, double* yT, double* lambdas,
                              cudaStream_t s, int rows_per_cta) {
  const int n = M->dim;
  if (n <= 512 && g_tune.chain_cluster >= 0) {
    nv_status st = launch_affine_chain_cluster(M, y0, yT, lambdas, s, g_tune.chain_cluster);
    if (st != NV_ENOTSUP) return st;
  }
  if (n > 512 && n % 4 == 0) return launch_tile_chain(M, y0, yT, lambdas, nullptr, s);
  const int block = 256;
  int rpc = rows_per_cta > 0 ? rows_per_cta : 16;
  rpc = std::min(rpc, block);
  while (block % rpc) --rpc;
  const int G = (n + rpc - 1) / rpc;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = (M->prec == NV_FP64 ? sizeof(double) : sizeof(float)) * (size_t)(n + 1);
  const void* fn = (M->prec == NV_FP64) ? (const void*)affine_chain_kernel<double, double>
                                        : (const void*)affine_chain_kernel<float, float>;
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
  a.extra = (unsigned)g_tune.test_barrier_extra;
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
  nv_status st0 = nv_cuda_check(cudaGetDevice(&dev), "current device");
  if (st0 != NV_OK) return st0;
  st0 = nv_cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
  if (st0 != NV_OK) return st0;
  const size_t smem = sizeof(double) * (size_t)(n + 1);
  const void* fn = (prec == NV_FP64) ? (const void*)affine_chain_kernel<double, double>
                                     : (const void*)affine_chain_kernel<float, double>;
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
