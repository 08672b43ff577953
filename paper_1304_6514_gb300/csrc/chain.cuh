// Chain of affine steps x_{k+1} = A_k x_k + v_k within one 16-CTA cluster
// (the communication phase of Figure "pseudocode", eq. linearreconstruct),
// shared by the composition (compose.cu) and the pipelined refinement
// (wavefront.cu).
#pragma once

#include <cooperative_groups.h>
#include <cuda.h>

#include "common.cuh"

namespace nvpit {

namespace cg = cooperative_groups;

// TMA-fed variant (64 <= d <= 256, d % 16 == 0; 16 CTAs x 16 rows): each
// CTA's rows of A_j (16 x d, one 3-D box) are copied by the tensor memory
// accelerator into a ring of kRing shared-memory stages, kRing - 1 slices
// ahead, completing on an mbarrier; the copies run in the async proxy, so no
// load sits on the dependency chain.  Stage layout: element (row r, column c)
// at c*16 + r.
//
// The new state is exchanged without a cluster barrier: the lane that owns a
// row stores it into the matching state buffer of every CTA of the cluster
// with st.async, which completes bytes on that CTA's state mbarrier, and a CTA
// starts step k+1 as soon as its own barrier has counted all d values of
// x_{k+1}.  Two state buffers alternate; buffer (k+2) & 1 is rewritten only
// by senders that already hold x_{k+1}, which every CTA sends after it has
// read x_k, so no CTA overwrites a state another is still reading.  The
// final state x_len is written to global memory only.  Every wait is bounded
// (1 s of globaltimer); a CTA that gives up records NV_ETIMEOUT, stops
// sending and leaves the loop, so the others give up at their next wait.
constexpr int kRing = 3;
constexpr int kChainRpc = 16;   // rows per CTA of the TMA chain
constexpr int kChainIssuer = 32; // the thread that issues the ring's copies (warp 1, lane 0)

__device__ __forceinline__ uint32_t cta_smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool ring_wait(uint64_t* bar, uint32_t parity) {
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.b32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(cta_smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > 1000000000ull) return false;
  }
}

// Wait for a phase completed by other CTAs' st.async: acquire at cluster scope.
__device__ __forceinline__ bool state_wait(uint64_t* bar, uint32_t parity) {
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2; "
        "selp.b32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(cta_smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > 1000000000ull) return false;
  }
}

__device__ __forceinline__ void arm_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(cta_smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ uint32_t cluster_addr(uint32_t local, unsigned rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}

// 16 bytes to another CTA's shared memory, completing on its mbarrier.
__device__ __forceinline__ void st_async16(uint32_t addr, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                           uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                   addr),
               "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(bar)
               : "memory");
}

// Eight consecutive row values (this lane's half of the CTA's 16 rows) as
// 32 (float) or 64 (double) bytes of 16-byte stores.
__device__ __forceinline__ void send_rows(const float* v, uint32_t addr, uint32_t bar) {
#pragma unroll
  for (int q = 0; q < 2; ++q)
    st_async16(addr + 16 * q, __float_as_uint(v[4 * q]), __float_as_uint(v[4 * q + 1]),
               __float_as_uint(v[4 * q + 2]), __float_as_uint(v[4 * q + 3]), bar);
}
__device__ __forceinline__ void send_rows(const double* v, uint32_t addr, uint32_t bar) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const unsigned long long u0 = __double_as_longlong(v[2 * q]), u1 = __double_as_longlong(v[2 * q + 1]);
    st_async16(addr + 16 * q, (uint32_t)u0, (uint32_t)(u0 >> 32), (uint32_t)u1, (uint32_t)(u1 >> 32), bar);
  }
}

// Hooks of cluster_chain_run.  before_issue(j): the issuer, before it copies
// slice j's map rows, v_j and add_{j+1} (false gives up); stored(i): the
// issuer, once this CTA's rows of states[1..i] are stored and ordered before
// it by a CTA barrier; before_state0 / after_state0: thread 0 of the CTA that
// writes states[0], around that write.
struct ChainNoHooks {
  static constexpr bool kTopBarrierFree = true;   // the step needs no barrier before its product
  __device__ bool before_issue(int) const { return true; }
  __device__ void stored(int) const {}
  __device__ bool before_state0() const { return true; }
  __device__ void after_state0() const {}
};

// Banded maps (ChainsArgs::band > 0): the 16 rows r0 .. r0+15 of a CTA meet
// nonzero entries only in columns r0-(band-1) .. r0+15+(band-1).  The CTA
// reads exactly those columns, r0-bw .. r0+15+bw with bw = band-1; each thread
// takes the window's columns whose global index is congruent to its column
// group modulo 16, in increasing order, so that the products are the dense
// chain's, less terms that are exactly zero.  chain_band_lo is bw, or 0 when
// that window is not narrower than d (the CTA then reads all d columns);
// chain_band_cols the columns read.
__host__ __device__ inline int chain_band_lo(int n, int band) {
  if (band <= 0) return 0;
  const int bw = band - 1;
  return kChainRpc + 2 * bw < n ? bw : 0;
}
__host__ __device__ inline int chain_band_cols(int n, int band) {
  const int bw = chain_band_lo(n, band);
  return bw > 0 ? kChainRpc + 2 * bw : n;
}

template <typename MT, typename AT, typename Hooks>
__device__ __forceinline__ void cluster_chain_run(const CUtensorMap* tmA, const ChainsArgs& a, int* status,
                                                  int q, const Hooks& hooks) {
  constexpr int rpc = kChainRpc;
  cg::cluster_group cl = cg::this_cluster();
  // The exchange addresses 16 peer CTAs of the cluster: a launch that is not
  // in 16-CTA clusters (whatever the cause) records an error and touches no
  // cluster address.  Uniform over the cluster, so no CTA waits for another.
  if (cl.num_blocks() != 16 || blockDim.x != 256) {
    if (threadIdx.x == 0) record_status(status, NV_ECUDA);
    return;
  }
  const unsigned rank = cl.block_rank();
  extern __shared__ __align__(128) unsigned char ring_smem[];
  const int n = a.n;
  const int wcols = chain_band_cols(n, a.band);                        // columns of A_j read
  const int bw = chain_band_lo(n, a.band);
  const int col0 = bw > 0 ? (int)rank * rpc - bw : 0;                  // the first (may be < 0)
  const int stage_elems = rpc * wcols;
  MT* ring = reinterpret_cast<MT*>(ring_smem);                          // kRing stages
  // per stage also rpc values of v_j and of add_{j+1}, as doubles (16-byte slots)
  double* vring = reinterpret_cast<double*>(ring + kRing * stage_elems);
  double* aring = vring + kRing * rpc;
  AT* xs = reinterpret_cast<AT*>(aring + kRing * rpc);                 // two state buffers
  AT* red = xs + 2 * n;                                                // per-warp row partials, x2
  uint64_t* full = reinterpret_cast<uint64_t*>(
      ((uintptr_t)(red + 2 * blockDim.x) + 7) & ~(uintptr_t)7);
  uint64_t* xbar = full + kRing;                                       // state buffers 0, 1
  __shared__ int abort_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int r = tid % rpc, cgi = tid / rpc, ncg = blockDim.x / rpc;
  const int my_row = (int)rank * rpc + (lane & (rpc - 1));              // row of a lane in warp 0
  const bool active = (int)rank * rpc + r < n;
  // CTAs past row n - 1 (d < 256) own no rows: they neither read nor send a
  // state and take no part in the exchange
  const unsigned owners = (unsigned)(n / rpc);
  const bool has_rows = rank < owners;
  const int j0 = q * a.len;
  const int len = min(a.len, a.S - j0);
  const int vsz = a.v_double ? 8 : (int)sizeof(MT);
  const uint32_t stage_bytes = (uint32_t)(stage_elems * sizeof(MT)) + (uint32_t)(rpc * vsz) +
                               (a.add ? (uint32_t)(rpc * 8) : 0u);
  // Banded maps: a CTA's columns are the rows of the CTAs within hops ranks,
  // so it receives the state rows of those CTAs only, and sends its own rows
  // to the same CTAs (the relation is symmetric, which keeps the ordering
  // argument of the state buffers below).  Dense: every CTA that owns rows.
  const int hops = (bw + rpc - 1) / rpc;
  const unsigned src_lo = bw > 0 ? (unsigned)max((int)rank - hops, 0) : 0u;
  const unsigned src_hi = bw > 0 ? min(rank + (unsigned)hops, owners - 1u) : owners - 1u;
  const uint32_t state_bytes = (uint32_t)((src_hi - src_lo + 1u) * rpc * sizeof(AT));

  if (tid == 0) {
    for (int i = 0; i < kRing + 2; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(cta_smem_u32(&full[i])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (has_rows && len >= 2) arm_tx(&xbar[1], state_bytes);   // x_1, sent during step 0
    if (has_rows && len >= 3) arm_tx(&xbar[0], state_bytes);   // x_2, sent during step 1
    abort_flag = 0;
  }
  __syncthreads();
  // One thread outside warp 0 (which sums, sends and stores each step's rows)
  // issues the copies, after the step's reduction barrier: the copy work
  // then overlaps warp 0's tail of the step instead of delaying the products.
  const bool issuer = tid == kChainIssuer;
  auto issue = [&](int k) {   // the issuer: copy this CTA's rows of A_{j0+k}
    if (!hooks.before_issue(j0 + k)) return false;
    const int st = k % kRing;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(cta_smem_u32(&full[st])),
                 "r"(stage_bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(cta_smem_u32(ring + st * stage_elems)),
        "l"(tmA), "r"((int)rank * rpc), "r"(col0), "r"(j0 + k), "r"(cta_smem_u32(&full[st]))
        : "memory");
    const char* vsrc = reinterpret_cast<const char*>(a.v) +
                       ((int64_t)(j0 + k) * a.v_stride + (int64_t)rank * rpc) * vsz;
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            cta_smem_u32(vring + st * rpc)),
        "l"(vsrc), "r"(rpc * vsz), "r"(cta_smem_u32(&full[st]))
        : "memory");
    if (a.add) {
      const double* asrc = a.add + (int64_t)(j0 + k + 1) * n + (int64_t)rank * rpc;
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              cta_smem_u32(aring + st * rpc)),
          "l"(asrc), "r"(rpc * 8), "r"(cta_smem_u32(&full[st]))
          : "memory");
    }
    return true;
  };
  int issued = 0;   // copies issued so far (the issuer)
  if (issuer && has_rows)
    for (; issued < min(kRing - 1, len); ++issued)
      if (!issue(issued)) {
        abort_flag = 1;
        break;
      }

  const double* x0 = a.x0 ? a.x0 + (int64_t)q * a.x0_stride : nullptr;
  for (int i = tid; i < n; i += blockDim.x) xs[i] = x0 ? (AT)x0[i] : (AT)0;
  if (q == 0 && rank == 0 && a.write_state0 && a.states) {
    if (tid == 0 && !hooks.before_state0()) abort_flag = 1;
    __syncthreads();
    if (!abort_flag) {
      for (int i = tid; i < n; i += blockDim.x)
        a.states[i] = (x0 ? x0[i] : 0.0) + (a.add ? a.add[i] : 0.0);
      __syncthreads();
      if (tid == 0) hooks.after_state0();
    }
  }
  cl.sync();   // barriers initialised and armed, x_0 in place, before any st.async

  // Sending: lane l of warp 0 stores rows 8 (l / 16) .. +7 of this CTA into
  // CTA p = l % 16; its remote addresses of both state buffers and barriers.
  const unsigned peer = (unsigned)(lane & 15);
  const int half_rows = (lane >> 4) * 8;
  const bool sender = warp == 0 && peer < owners && (bw == 0 || abs((int)peer - (int)rank) <= hops);
  uint32_t rx0 = 0u, rx1 = 0u, rb0 = 0u, rb1 = 0u;
  if (sender) {
    const uint32_t off = (uint32_t)(((int)rank * rpc + half_rows) * sizeof(AT));
    rx0 = cluster_addr(cta_smem_u32(xs), peer) + off;
    rx1 = cluster_addr(cta_smem_u32(xs + n), peer) + off;
    rb0 = cluster_addr(cta_smem_u32(&xbar[0]), peer);
    rb1 = cluster_addr(cta_smem_u32(&xbar[1]), peer);
  }

  // the window's columns inside 0 .. d-1 (those outside are the copy's zero
  // fill); this thread's first one: global index congruent to its group mod 16
  const int cb = max(0, -col0), ce = min(wcols, n - col0);
  const int cfirst = cb + ((cgi - col0 - cb) % ncg + ncg) % ncg;
  int consumed = len;
  for (int k = 0; has_rows && k < len; ++k) {
    const int j = j0 + k;
    const int st = k % kRing;
    bool ok = true;
    if (k >= 1) ok = state_wait(&xbar[k & 1], (uint32_t)(((k - 1) >> 1) & 1));
    if (ok) ok = ring_wait(&full[st], (uint32_t)((k / kRing) & 1));
    // No block barrier is needed here: every thread waits on the barriers of
    // what it reads itself.  (The reduction buffer alternates by step; a ring
    // slot is refilled only after the reduction barrier of the following step;
    // and state buffer k & 1 cannot receive x_{k+2} before this CTA has sent
    // its rows of x_{k+1}, which warp 0 does after that barrier, when every
    // warp here has read x_k.)  A failed wait is acted on at the reduction
    // barrier.  Measured on one GB300: without it a float32 step is 7 % faster,
    // a float64 step 1 % slower, and the pipelined refinement's chains, whose
    // issuer runs hooks after the reduction barrier, 4 % slower: so it stays
    // except for float32 chains without hooks.
    if (!ok) abort_flag = 1;
    if constexpr (!(Hooks::kTopBarrierFree && sizeof(AT) == 4)) __syncthreads();
    if (tid == 0 && k >= 1 && k + 2 <= len - 1) arm_tx(&xbar[k & 1], state_bytes);   // x_{k+2}
    const AT* x = xs + (k & 1) * n;
    const MT* Aj = ring + st * stage_elems;
    AT acc = 0;
    if (active)
      for (int c = cfirst; c < ce; c += ncg) acc = fma((AT)Aj[c * rpc + r], x[col0 + c], acc);
    // lanes l and l ^ 16 hold the same row (rpc = 16)
    acc += __shfl_xor_sync(0xffffffffu, acc, 16);
    AT* redk = red + (k & 1) * blockDim.x;
    if (lane < rpc) redk[warp * rpc + lane] = acc;
    __syncthreads();
    if (abort_flag) {
      consumed = k;
      break;
    }
    // stage k+2 into slot (k-1) % kRing, which every thread finished with in
    // step k-1
    if (issuer && issued < len) {
      if (issue(issued)) ++issued;
      else abort_flag = 1;                 // seen at the next step's barrier
    }
    // warp 0 stored its rows of states[j0 + k] in step k - 1, before this
    // step's reduction barrier
    if (issuer && k >= 1) hooks.stored(j0 + k);
    if (warp == 0) {
      const int rr = lane & (rpc - 1), half = lane >> 4;
      AT s = 0;
      for (int w = half * (nw >> 1); w < (half + 1) * (nw >> 1); ++w) s += redk[w * rpc + rr];
      s += __shfl_xor_sync(0xffffffffu, s, 16);
      const bool own = lane < rpc && my_row < n;
      if (own) {
        const AT vj = a.v_double ? (AT)vring[st * rpc + rr]
                                 : (AT)reinterpret_cast<const MT*>(vring + st * rpc)[rr];
        s += vj;
      }
      // x_{k+1} to every CTA that owns rows (not sent after the last step)
      if (k + 1 < len) {
        AT v8[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v8[i] = __shfl_sync(0xffffffffu, s, half_rows + i);
        const bool odd = (k + 1) & 1;
        if (sender) send_rows(v8, odd ? rx1 : rx0, odd ? rb1 : rb0);
      }
      if (own) {
        const int64_t o = (int64_t)(j + 1) * n + my_row;
        const double out = (double)s + (a.add ? aring[st * rpc + rr] : 0.0);
        if (a.states) a.states[o] = out;
        if (a.yT && j == a.S - 1) a.yT[my_row] = out;
        if (a.finals && k == len - 1) a.finals[(int64_t)q * n + my_row] = (double)s;
      }
    }
    // this step's reduction buffer is next written two steps on, after the
    // next reduction barrier, which warp 0 reaches only when it is done with it
  }
  __syncthreads();
  if (has_rows && !abort_flag && issuer && len >= 1) hooks.stored(j0 + len);
  if (abort_flag && issuer) {
    record_status(status, NV_ETIMEOUT);
    for (int kk = min(consumed, issued); kk < issued; ++kk)   // copies in flight (bounded waits)
      ring_wait(&full[kk % kRing], (uint32_t)((kk / kRing) & 1));
  }
  cl.sync();   // no CTA leaves while another may still address its shared memory
}

}  // namespace nvpit

// Host (compose.cu): NV_OK and the tensor map of the maps' rows and the
// dynamic shared memory of cluster_chain_run if the chain fits it (64 <= d <=
// 256, d % 16 == 0, 16-byte aligned operands), else NV_ENOTSUP.
nv_status chain_tma_prepare(const ChainsArgs& args, bool f64, CUtensorMap* tmap, size_t* smem);
