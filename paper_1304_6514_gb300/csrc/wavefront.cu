// Pipelined float64 refinement of the heat-equation composition over float32
// maps (NV_FP32_REFINE, 64 <= d <= 256, d % 16 == 0).
//
// The residual correction the Conclusion proposes runs P passes after the
// approximate chain:
//   chain 0   lt0_{j+1} = A~_j lt0_j + b~_j              float32 maps, from y0
//   pass c    d^c_j    = g^j(lt^{c-1}_j) - lt^{c-1}_{j+1}  float64 fine solve
//             e_{j+1}  = A~_j e_j + d^c_j, e_0 = 0
//             lt^c_j   = lt^{c-1}_j + e_j
// Done one after another these are P + 1 chains of S dependent steps each.
// But d^c_j needs only the two states lt^{c-1}_j and lt^{c-1}_{j+1}, and step
// j of pass c's chain only d^c_j, so the chains can run concurrently, each a
// few slices behind the one it corrects, with the defects computed in
// between: the whole refinement then takes about one chain's time.
//
// One cooperative launch of 16-CTA clusters holds every role, so all of them
// are resident together (nothing else guarantees that blocks waiting on each
// other run at the same time):
//   clusters 0 .. P       chain c (the cluster chain of chain.cuh), which
//                         waits, before it prefetches slice j, for the flag
//                         of d^c_j, and counts its CTA in cnt[c][j+1] for
//                         each state it has stored (in batches);
//   clusters P+1 ..       defect workers: warp w takes work items w, w + W,
//                         ..., item i = slice i / P of pass 1 + i % P, waits
//                         until cnt[c-1][j] and cnt[c-1][j+1] are complete,
//                         computes d^c_j (heat_defect_slice) and sets its flag.
// Item i depends only on items below i (pass c, slice j needs pass c-1 up to
// slice j), and each warp takes its items in increasing order, so the lowest
// unfinished item can always run: no cycle of waits.  The arithmetic is the
// sequential refinement's, in the same order, so the results are identical.
//
// Every wait is bounded (1 s of globaltimer) and also ends when any CTA has
// set the shared abort word; a waiter that gives up records NV_ETIMEOUT.
#include <algorithm>

#include "chain.cuh"
#include "heat.cuh"

namespace nvpit {

constexpr int kWaveMaxChains = 4;      // approximate chain + up to 3 correction passes
constexpr int kWaveWorkerWarps = 4;    // defect warps per worker CTA: one per SM sub-partition

struct WavefrontArgs {
  ChainsArgs chain[kWaveMaxChains];
  const double* lt[kWaveMaxChains];    // states of chain c, (S+1) x n (c < nchains - 1)
  double* d[kWaveMaxChains];           // defects of pass c >= 1, S x n
  unsigned* cnt;                       // nchains x (S+1): CTAs that stored their rows of state j
  unsigned* dflag;                     // nchains x S: defect of pass c, slice j, stored
  unsigned* abort;                     // nonzero once any waiter gave up
  int nchains, S, owners;
  int withhold;                        // test hook: the flag of pass 1, slice withhold - 1 is never set (0: off)
  HeatArgs heat;
};

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool wave_wait(const unsigned* p, unsigned target, const WavefrontArgs& w) {
  uint64_t t0 = 0;
  while (ld_acquire_u32(p) < target) {
    if (*(volatile unsigned*)w.abort) return false;
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t0 == 0) {
      t0 = t;
    } else if (t - t0 > 1000000000ull) {
      record_status(w.chain[0].status, NV_ETIMEOUT);
      atomicExch(w.abort, 1u);
      return false;
    }
    __nanosleep(256);
  }
  return true;
}

// The hooks run in the chain's issuer thread, off the path of the products
// and the state exchange, and keep global-memory round trips rare: a chain
// acquires the defect flags kWaveBatch slices at a time (independent loads,
// one latency) into a shared cursor, and publishes its states once every
// kWaveBatch steps behind a single fence.  The few extra microseconds of lag
// this adds per pass are far below the lag of the defect solves.
constexpr int kWaveBatch = 32;

struct WaveHooks {
  static constexpr bool kTopBarrierFree = false;   // keep the step's first barrier (see chain.cuh)
  const WavefrontArgs* w;
  int c;
  int* ready;   // shared: defects of slices < *ready are known to be stored (the issuer)
  __device__ bool before_issue(int j) const {
    // (the abort word only speeds up giving up: read it once per batch)
    if (j % kWaveBatch == 0 && *(volatile unsigned*)w->abort) return false;
    if (c == 0 || j < *ready) return true;
    const unsigned* f = w->dflag + (size_t)c * w->S;
    // relaxed loads are independent (acquire loads would each wait for the
    // previous one); one fence then orders everything after them
    unsigned v[kWaveBatch];
#pragma unroll
    for (int q = 0; q < kWaveBatch; ++q) v[q] = j + q < w->S ? ld_relaxed_u32(f + j + q) : 0u;
    int r = 0;
    while (r < kWaveBatch && v[r] != 0u) ++r;
    if (r == 0) {
      if (!wave_wait(f + j, 1u, *w)) return false;
      r = 1;
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");   // acquire: the defects after their flags
    *ready = j + r;
    // the bulk copies that follow read d^c_j and lt^{c-1}_{j+1} in the async proxy
    asm volatile("fence.proxy.async.global;" ::: "memory");
    return true;
  }
  __device__ void stored(int i) const {   // states 1..i of this CTA's rows are stored
    if (i % kWaveBatch != 0 && i != w->S) return;
    asm volatile("fence.acq_rel.gpu;" ::: "memory");   // release: the rows before the counts
    unsigned* cnt = w->cnt + (size_t)c * (w->S + 1);
    for (int t = ((i - 1) / kWaveBatch) * kWaveBatch + 1; t <= i; ++t) atomicAdd(cnt + t, 1u);
  }
  __device__ bool before_state0() const {
    return c == 0 || wave_wait(w->cnt + (size_t)(c - 1) * (w->S + 1), (unsigned)w->owners, *w);
  }
  __device__ void after_state0() const {
    __threadfence();
    atomicAdd(w->cnt + (size_t)c * (w->S + 1), (unsigned)w->owners);
  }
};

template <int R>
__global__ void __launch_bounds__(256, 1) heat_wavefront_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                const __grid_constant__ WavefrontArgs w) {
  // the roles need 16-CTA clusters and at least one worker cluster; any
  // other launch shape records an error and returns at once (uniformly)
  if (cg::this_cluster().num_blocks() != 16 || gridDim.x % 16 != 0 || gridDim.x < 16u * (w.nchains + 1) ||
      blockDim.x != 256) {
    if (threadIdx.x == 0) {
      record_status(w.chain[0].status, NV_ECUDA);
      atomicExch(w.abort, 1u);
    }
    return;
  }
  const int cluster = (int)(blockIdx.x / 16);
  if (cluster < w.nchains) {
    __shared__ int ready;
    if (threadIdx.x == 0) ready = 0;   // then read and written by the chain's issuer only
    cluster_chain_run<float, float>(&tmA, w.chain[cluster], w.chain[cluster].status, 0,
                                    WaveHooks{&w, cluster, &ready});
    return;
  }
  // defect workers: kWaveWorkerWarps independent warps per CTA, one slice each
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp >= kWaveWorkerWarps) return;
  const int P = w.nchains - 1;
  const int64_t nw = (int64_t)(gridDim.x - 16 * w.nchains) * kWaveWorkerWarps;
  const int64_t wid = (int64_t)(blockIdx.x - 16 * w.nchains) * kWaveWorkerWarps + warp;
  for (int64_t it = wid; it < (int64_t)P * w.S; it += nw) {
    const int c = 1 + (int)(it % P);
    const int64_t j = it / P;
    const unsigned* cprev = w.cnt + (size_t)(c - 1) * (w.S + 1);
    const bool ok = wave_wait(cprev + j, (unsigned)w.owners, w) && wave_wait(cprev + j + 1, (unsigned)w.owners, w);
    if (!__all_sync(0xffffffffu, ok)) break;
    heat_defect_slice<R>(w.heat, w.lt[c - 1], w.d[c], j, lane);
    __syncwarp();
    if (lane == 0 && !(c == 1 && j + 1 == w.withhold)) {
      __threadfence();
      atomicExch(w.dflag + (size_t)c * w.S + j, 1u);
    }
  }
}

}  // namespace nvpit

using namespace nvpit;

size_t heat_wavefront_scratch_bytes(int n, int S, int passes) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  return al(sizeof(double) * (size_t)passes * (S + 1) * n) + al(sizeof(double) * (size_t)passes * S * n) +
         al(sizeof(unsigned) * ((size_t)(passes + 1) * (2 * (size_t)S + 1) + 1));
}

nv_status launch_heat_wavefront(nv_maps* M, const double* y0, double* yT, double* lambdas, int passes,
                                void* scratch, cudaStream_t s) {
  const int n = M->dim, S = M->S;
  if (passes < 1 || passes >= kWaveMaxChains || M->prec != NV_FP32_REFINE) return NV_ENOTSUP;
  if (M->rhs_kind != NV_RHS_HEAT1D && M->rhs_kind != NV_RHS_HEAT1D_VARCOEF) return NV_ENOTSUP;
  const int R = n <= 64 ? 2 : (n <= 128 ? 4 : 8);   // rows per lane of a defect warp
  if (R * 32 < n) return NV_ENOTSUP;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  char* p = static_cast<char*>(scratch);
  double* lt = reinterpret_cast<double*>(p);                    // passes state sets
  p += al(sizeof(double) * (size_t)passes * (S + 1) * n);
  double* dd = reinterpret_cast<double*>(p);                    // passes defect sets
  p += al(sizeof(double) * (size_t)passes * S * n);
  unsigned* flags = reinterpret_cast<unsigned*>(p);
  const size_t nflags = (size_t)(passes + 1) * (2 * (size_t)S + 1) + 1;

  WavefrontArgs w{};
  w.nchains = passes + 1;
  w.withhold = g_tune.test_withhold_defect;
  w.S = S;
  w.owners = n / kChainRpc;
  w.heat = heat_args(M);
  w.cnt = flags;
  w.dflag = flags + (size_t)(passes + 1) * (S + 1);
  w.abort = flags + nflags - 1;
  const float* maps = static_cast<const float*>(M->data);
  for (int c = 0; c <= passes; ++c) {
    ChainsArgs& a = w.chain[c];
    a.n = n;
    a.nchains = 1;
    a.len = S;
    a.S = S;
    a.rpc = kChainRpc;
    a.A = maps + n;                                   // columns 1..d of every slice
    a.a_stride = (int64_t)n * (n + 1);
    a.status = M->status;
    a.write_state0 = 1;
    a.band = g_tune.chain_dense ? 0 : M->band;
    const bool last = c == passes;
    double* states = last ? lambdas : lt + (size_t)c * (S + 1) * n;
    a.states = states;
    a.yT = last ? yT : nullptr;
    if (!last) w.lt[c] = states;
    if (c == 0) {
      a.v = maps;                                     // column 0: b_j
      a.v_stride = (int64_t)n * (n + 1);
      a.x0 = y0;
    } else {
      w.d[c] = dd + (size_t)(c - 1) * S * n;
      a.v = w.d[c];
      a.v_double = 1;
      a.v_stride = n;
      a.add = w.lt[c - 1];
    }
  }
  CUtensorMap tmap;
  size_t smem = 0;
  nv_status st = chain_tma_prepare(w.chain[passes > 0 ? 1 : 0], false, &tmap, &smem);
  if (st != NV_OK) return st;
  // more than half an SM's shared memory: one CTA per SM, so no defect team
  // shares an SM with a chain's CTA
  smem = std::max(smem, (size_t)116 * 1024);
  const void* fn = R == 2 ? (const void*)heat_wavefront_kernel<2>
                 : R == 4 ? (const void*)heat_wavefront_kernel<4>
                          : (const void*)heat_wavefront_kernel<8>;
  if ((st = nv_cuda_check(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1),
                          "cluster size attribute")) != NV_OK ||
      (st = nv_cuda_check(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                          "wavefront smem attribute")) != NV_OK)
    return st;
  cudaLaunchConfig_t cfg{};
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 16;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeCooperative;
  attr[1].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  cfg.gridDim = dim3(16);
  int maxc = 0;
  if (cudaOccupancyMaxActiveClusters(&maxc, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return NV_ENOTSUP;
  }
  if (maxc < w.nchains + 1) return NV_ENOTSUP;      // no room for a defect worker cluster
  cfg.gridDim = dim3((unsigned)(16 * maxc));
  if ((st = nv_cuda_check(cudaMemsetAsync(flags, 0, sizeof(unsigned) * nflags, s), "wavefront flags reset")) !=
      NV_OK)
    return st;
  void* args[] = {&tmap, &w};
  return nv_cuda_check(cudaLaunchKernelExC(&cfg, fn, args), "heat_wavefront_kernel cooperative launch");
}
