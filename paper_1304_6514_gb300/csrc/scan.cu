// Reduced-precision composition with float64 refinement (NV_TF32_REFINE).
//
// The communication phase of Figure "pseudocode" is a chain of S dependent
// affine steps.  Affine maps compose associatively, (A2,b2)o(A1,b1) =
// (A2 A1, A2 b1 + b2), so the chain can be cut into B blocks of L slices:
//   A  block totals   R_b = A_{bL+L-1} ... A_{bL}      tcgen05 TF32 GEMMs
//   B  block vectors  c_b = chain of block b from 0    batched cluster chains
//   C  block chain    Lam_b = R_b Lam_{b-1} + c_b      one cluster chain, B steps
//   D  block states   lt_j: chain of block b from Lam_{b-1}   batched chains
// and the sequential depth drops from S to 2L + B.  The float32 maps and the
// TF32 products carry ~1e-3 relative error, which one float64 residual
// correction removes (the parareal-style combination the Conclusion
// proposes, with the reduced-precision maps as the coarse propagator):
//   E  d_j = g^j(lt_j) - lt_{j+1}       float64 fine solve from lt_j per slice
//   F, G, H  the same block scheme on e_{j+1} = A_j e_j + d_j, e_0 = 0
//   lambda_j = lt_j + e_j.
//
// Block-total kernel (phase A): CTA (h, b) owns rows [128h, 128h+128) of the
// running suffix product R <- R A_j (j from the block's last slice down), so
// the row halves never exchange data.  R's rows stay in shared memory as the
// K-major A operand (128B-swizzled, 1024-byte atoms).  Each A_j is stored
// column-major in HBM, which is exactly the K-major layout of the B operand;
// TMA streams it in K-slabs of 32 (256 x 128 B boxes, SWIZZLE_128B) through a
// three-stage mbarrier ring (the most that fits beside the 128 KB A operand),
// one warp issuing the copies continuously across the products.  One thread
// of another warp issues tcgen05.mma (kind::tf32, M=128, N=256, K=8) into one
// of two 128 x 256 float32 accumulators in tensor memory, alternating by
// product; four warps read the finished one back with tcgen05.ld and write
// the next A operand slab by slab, each slab released to the MMAs on its own
// mbarrier, so the next product starts while the epilogue runs (or,
// after the last slice, the block total to global memory).  Every mbarrier
// wait is bounded (1 s of globaltimer), after which the kernel records
// NV_ETIMEOUT, waits (bounded) for its copies in flight, frees its tensor
// memory and returns.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "tc.cuh"

namespace nvpit {
namespace tc {

constexpr int kRows = 128;              // rows of R per CTA (UMMA M)
constexpr int kN = 256;                 // UMMA N (padded d)
constexpr int kSlab = 32;               // K per TMA box / swizzle atom (128 B of tf32)
constexpr int kSlabBytesA = kRows * 128;
constexpr int kSlabBytesB = kN * 128;
constexpr int kStages = 3;                // 128 KB A operand + 96 KB of B stages: 225 KB
constexpr int kMaxSlabs = 8;            // d <= 256
constexpr int kSmemA = kMaxSlabs * kSlabBytesA;          // 128 KB
constexpr int kSmemB = kStages * kSlabBytesB;            // 96 KB
constexpr int kSmemBytes = kSmemA + kSmemB + 256 + 1024; // + barriers + alignment slack

struct ScanArgs {
  int n, S, L, nblocks, nslabs;
  float* R;        // nblocks x n x n, column-major block totals
  int* status;
};

// Row m of the K-major A operand, 32 floats of slab s, 128B-swizzled.
__device__ __forceinline__ float4* arow_chunk(uint8_t* aop, int s, int m, int chunk) {
  return reinterpret_cast<float4*>(aop + s * kSlabBytesA + m * 128 + ((chunk ^ (m & 7)) << 4));
}

// Warp roles of the block-total kernel: warps 0-3 read the accumulator back
// (tcgen05.ld reaches TMEM lanes 32w .. 32w+31 from warp w) and write the
// next A operand or the block total; warp 4 streams the maps' K-slabs with
// TMA; warp 5 issues the MMAs.  The accumulator alternates between two TMEM
// buffers of 256 columns, so product k+1 accumulates into one while the
// epilogue of product k reads the other, and it reads A slab s as soon as the
// epilogue has written that slab (one mbarrier per slab): the epilogue and
// the B stream overlap the MMAs instead of following them.
constexpr int kEpiWarps = 4, kTmaWarp = 4, kMmaWarp = 5;
constexpr int kScanThreads = 32 * (kMmaWarp + 1);

__global__ void __launch_bounds__(kScanThreads, 1)
    scan_block_totals_kernel(const __grid_constant__ CUtensorMap tmB, ScanArgs a) {
  extern __shared__ unsigned char smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* aop = base;
  uint8_t* bst = base + kSmemA;
  uint64_t* full = reinterpret_cast<uint64_t*>(base + kSmemA + kSmemB);
  uint64_t* empty = full + kStages;
  uint64_t* done = empty + kStages;         // [2]: product into accumulator buffer b complete
  uint64_t* aready = done + 2;              // [kMaxSlabs]: the epilogue wrote A slab s
  uint64_t* tfree = aready + kMaxSlabs;     // [2]: the epilogue read accumulator buffer b
  uint64_t* fin = tfree + 2;                // every MMA issued has completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  __shared__ int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int h = blockIdx.x, blk = blockIdx.y;
  const int n = a.n, ns = a.nslabs;
  const int j0 = blk * a.L;
  const int len = min(a.L, a.S - j0);

  if (warp == 0) tmem_alloc(tmem_slot, 2 * kN);
  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&done[b], 1);
      mbar_init(&tfree[b], kEpiWarps);
    }
    for (int s = 0; s < kMaxSlabs; ++s) mbar_init(&aready[s], kEpiWarps);
    mbar_init(fin, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // A operand = rows [128h, 128h+128) of the identity (zero beyond d)
  if (warp < kEpiWarps) {
    const int m = tid;                      // one row per epilogue thread
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int s = 0; s < kMaxSlabs; ++s)
      for (int c = 0; c < 8; ++c) *arow_chunk(aop, s, m, c) = z;
    const int gm = kRows * h + m;
    if (gm < n) {
      const int s = gm / kSlab, kk = gm % kSlab;
      float* p = reinterpret_cast<float*>(arow_chunk(aop, s, m, kk >> 2));
      p[kk & 3] = 1.0f;
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const int total = len * ns;               // K-slabs of B over all products of this block
  volatile int* vabort = &abort_flag;
  int issued = 0;                           // the TMA lane: slabs whose copies were issued

  if (warp == kTmaWarp && lane == 0) {
    // slab g of the stream is slab s = g % ns of product k = g / ns (map j0 + len - 1 - k:
    // the suffix product runs from the block's last slice down)
    for (; issued < total && !*vabort; ++issued) {
      const int g = issued, st = g % kStages;
      if (g >= kStages && !mbar_wait(&empty[st], (uint32_t)(((g / kStages) - 1) & 1))) {
        *vabort = 1;
        break;
      }
      const int k = g / ns, s = g - k * ns;
      mbar_expect_tx(&full[st], kSlabBytesB);
      tma_load_3d(bst + st * kSlabBytesB, &tmB, &full[st], s * kSlab, 1, j0 + len - 1 - k);
    }
  } else if (warp == kMmaWarp && lane == 0) {
    const uint32_t idesc = idesc_tf32(kRows, kN);
    const uint32_t aop_addr = smem_u32(aop), bst_addr = smem_u32(bst);
    bool ok = true;
    int g = 0;
    for (int k = 0; k < len && ok; ++k) {
      const uint32_t d = tmem + (uint32_t)((k & 1) * kN);
      if (k >= 2) {                         // the epilogue of product k-2 has read buffer k & 1
        ok = mbar_wait(&tfree[k & 1], (uint32_t)(((k - 2) >> 1) & 1));
        if (!ok) break;
        fence_after();
      }
      for (int s = 0; s < ns; ++s, ++g) {
        const int st = g % kStages;
        ok = mbar_wait(&full[st], (uint32_t)((g / kStages) & 1));
        if (ok && k >= 1) ok = mbar_wait(&aready[s], (uint32_t)((k - 1) & 1));
        if (!ok || *vabort) {
          ok = false;
          break;
        }
        fence_after();
#pragma unroll
        for (int kk = 0; kk < kSlab / 8; ++kk) {
          const uint64_t ad = sdesc_k_sw128(aop_addr + s * kSlabBytesA + kk * 32);
          const uint64_t bd = sdesc_k_sw128(bst_addr + st * kSlabBytesB + kk * 32);
          mma_tf32(d, ad, bd, idesc, (s | kk) != 0);
        }
        mma_commit(&empty[st]);             // the stage is free once these MMAs are done
      }
      if (ok) mma_commit(&done[k & 1]);
    }
    if (!ok) *vabort = 1;
    mma_commit(fin);                        // completes with every MMA issued above
    mbar_wait(fin, 0);
  } else if (warp < kEpiWarps) {
    // warp w owns accumulator rows (TMEM lanes) 32w .. 32w+31
    const int m = warp * 32 + lane;
    const int gm = kRows * h + m;
    for (int k = 0; k < len; ++k) {
      if (!mbar_wait(&done[k & 1], (uint32_t)((k >> 1) & 1))) {
        *vabort = 1;
        break;
      }
      if (*vabort) break;
      fence_after();
      const uint32_t t = tmem + (uint32_t)((k & 1) * kN) + ((uint32_t)(warp * 32) << 16);
      const bool last = (k == len - 1);
      for (int s = 0; s < ns; ++s) {
        float v[32];
        tmem_ld32(t + (uint32_t)(s * kSlab), v);
        if (!last) {                          // slab s of the next product's A operand
#pragma unroll
          for (int c = 0; c < 8; ++c)
            *arow_chunk(aop, s, m, c) = make_float4(round_tf32(v[4 * c]), round_tf32(v[4 * c + 1]),
                                                    round_tf32(v[4 * c + 2]), round_tf32(v[4 * c + 3]));
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(&aready[s]);
        } else if (gm < n) {
          float* Rb = a.R + (int64_t)blk * n * n;
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int col = s * kSlab + i;
            if (col < n) Rb[(int64_t)col * n + gm] = v[i];
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tfree[k & 1]);   // the MMAs of product k+2 may overwrite it
    }
  }
  __syncthreads();
  if (*vabort) {
    if (tid == 0) record_status(a.status, NV_ETIMEOUT);
    if (warp == kTmaWarp && lane == 0)      // let copies in flight land (bounded)
      for (int g = max(0, issued - kStages); g < issued; ++g)
        mbar_wait(&full[g % kStages], (uint32_t)((g / kStages) & 1));
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 2 * kN);
}

}  // namespace tc
}  // namespace nvpit

using namespace nvpit;

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

static nv_status encode_fn(EncodeTiledFn* out) {
  static std::mutex mu;
  static EncodeTiledFn fn = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    nv_status st = nv_cuda_check(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                                  cudaEnableDefault, &q),
                                 "driver entry point cuTensorMapEncodeTiled");
    if (st != NV_OK) return st;
    if (q != cudaDriverEntryPointSuccess || !p)
      return nv_fail(NV_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  *out = fn;
  return NV_OK;
}

// Scratch of the refined composition, carved from one allocation.
struct ScanScratch {
  float* R;
  double *cvec, *lam, *lt, *lt2, *d, *cpr, *E;
};

static size_t scan_scratch_bytes(int n, int S, int B) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t b = al(sizeof(float) * (size_t)B * n * n);
  b += al(sizeof(double) * (size_t)B * n) * 2;         // cvec, cpr
  b += al(sizeof(double) * (size_t)(B + 1) * n) * 2;   // lam, E
  b += al(sizeof(double) * (size_t)(S + 1) * n) * 2;    // lt, lt2
  b += al(sizeof(double) * (size_t)S * n);              // d
  return b;
}

static ScanScratch carve(void* p, int n, int S, int B) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  char* c = static_cast<char*>(p);
  ScanScratch s;
  s.R = reinterpret_cast<float*>(c);
  c += al(sizeof(float) * (size_t)B * n * n);
  s.cvec = reinterpret_cast<double*>(c);
  c += al(sizeof(double) * (size_t)B * n);
  s.cpr = reinterpret_cast<double*>(c);
  c += al(sizeof(double) * (size_t)B * n);
  s.lam = reinterpret_cast<double*>(c);
  c += al(sizeof(double) * (size_t)(B + 1) * n);
  s.E = reinterpret_cast<double*>(c);
  c += al(sizeof(double) * (size_t)(B + 1) * n);
  s.lt = reinterpret_cast<double*>(c);
  c += al(sizeof(double) * (size_t)(S + 1) * n);
  s.lt2 = reinterpret_cast<double*>(c);
  c += al(sizeof(double) * (size_t)(S + 1) * n);
  s.d = reinterpret_cast<double*>(c);
  return s;
}


nv_status launch_scan_refine(nv_maps* M, const double* y0, double* yT, double* lambdas, cudaStream_t s) {
  const int n = M->dim, S = M->S;
  if (M->rhs_kind != NV_RHS_HEAT1D && M->rhs_kind != NV_RHS_HEAT1D_VARCOEF)
    return nv_fail(NV_ENOTSUP, "refined tensor-core composition is built for the heat equations");
  if (n > tc::kN || n % 4 != 0)
    return nv_fail(NV_ENOTSUP, "tensor-core scan needs d <= 256 and d a multiple of 4 (d = %d)", n);
  int L = g_tune.scan_block > 0 ? g_tune.scan_block : (int)lround(sqrt((double)S));
  L = std::max(1, std::min(L, S));
  const int B = (S + L - 1) / L;

  const size_t need = scan_scratch_bytes(n, S, B);
  if (M->scan_ws_bytes < need) {
    if (M->scan_ws) {
      cudaStreamSynchronize(s);
      cudaFree(M->scan_ws);
      M->scan_ws = nullptr;
      M->scan_ws_bytes = 0;
    }
    nv_status st = nv_cuda_check(cudaMalloc(&M->scan_ws, need), "scan scratch allocation");
    if (st != NV_OK) return st;
    M->scan_ws_bytes = need;
  }
  const ScanScratch sc = carve(M->scan_ws, n, S, B);

  // TMA view of the float32 maps: (row i: d, column c: d+1, slice j: S); a box
  // of 32 rows x 256 columns of one slice is one K-slab of A_j (columns 1..d).
  EncodeTiledFn enc = nullptr;
  nv_status st = encode_fn(&enc);
  if (st != NV_OK) return st;
  CUtensorMap tmap;
  const cuuint64_t gdim[3] = {(cuuint64_t)n, (cuuint64_t)(n + 1), (cuuint64_t)S};
  const cuuint64_t gstride[2] = {(cuuint64_t)n * 4, (cuuint64_t)n * (n + 1) * 4};
  const cuuint32_t box[3] = {(cuuint32_t)tc::kSlab, (cuuint32_t)tc::kN, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult cr = enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, M->data, gdim, gstride, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return nv_fail(NV_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);

  // A: block totals on the tensor cores
  tc::ScanArgs sa{};
  sa.n = n;
  sa.S = S;
  sa.L = L;
  sa.nblocks = B;
  sa.nslabs = (n + tc::kSlab - 1) / tc::kSlab;
  sa.R = sc.R;
  sa.status = M->status;
  st = nv_cuda_check(cudaFuncSetAttribute(tc::scan_block_totals_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes),
                     "scan smem attribute");
  if (st != NV_OK) return st;
  const int halves = (n + tc::kRows - 1) / tc::kRows;
  tc::scan_block_totals_kernel<<<dim3(halves, B), tc::kScanThreads, tc::kSmemBytes, s>>>(tmap, sa);
  st = nv_cuda_check(cudaGetLastError(), "scan_block_totals_kernel launch");
  if (st != NV_OK) return st;

  // 16-CTA clusters keep every thread's columns inside the prefetched set
  // (16 rows per CTA); clusters of different chains share SMs.
  const int cs_many = 16;
  const float* mapsf = static_cast<const float*>(M->data);
  const int64_t bs = (int64_t)n * (n + 1);

  ChainsArgs blockc{};            // chains over the slices of each block
  blockc.n = n;
  blockc.status = M->status;
  blockc.nchains = B;
  blockc.len = L;
  blockc.S = S;
  blockc.A = mapsf + n;
  blockc.a_stride = bs;

  ChainsArgs topc{};              // one chain over the block totals
  topc.n = n;
  topc.status = M->status;
  topc.nchains = 1;
  topc.len = B;
  topc.S = B;
  topc.A = sc.R;
  topc.a_stride = (int64_t)n * n;
  topc.v_double = 1;
  topc.v_stride = n;
  topc.write_state0 = 1;

  // B: block vectors from zero
  ChainsArgs cb = blockc;
  cb.v = mapsf;
  cb.v_stride = bs;
  cb.finals = sc.cvec;
  if ((st = launch_chains(cb, false, s, cs_many)) != NV_OK) return st;
  // C: Lam_b
  ChainsArgs cc = topc;
  cc.v = sc.cvec;
  cc.x0 = y0;
  cc.states = sc.lam;
  if ((st = launch_chains(cc, false, s, 16)) != NV_OK) return st;
  // D: approximate boundary states lt
  ChainsArgs cd = blockc;
  cd.v = mapsf;
  cd.v_stride = bs;
  cd.x0 = sc.lam;
  cd.x0_stride = n;
  cd.states = sc.lt;
  cd.write_state0 = 1;
  if ((st = launch_chains(cd, false, s, cs_many)) != NV_OK) return st;
  // E-H: float64 correction passes (tunable; 0 returns the unrefined states)
  // Default 3: on a constant-coefficient problem every slice map, and so every
  // TF32 block total, carries the same rounding error, which then adds up
  // coherently along the chain; each pass contracts the error by about
  // S * 2^-11 (~0.04 on the 1024-slice heat equation: 8.5e-2, 4.0e-3,
  // 1.3e-4, 3.1e-6 after 0..3 passes).
  const int passes = g_tune.refine_passes > 0 ? g_tune.refine_passes
                     : (g_tune.refine_passes < 0 ? 0 : 3);
  const double* cur = sc.lt;
  if (passes == 0) {
    if (lambdas &&
        (st = nv_cuda_check(cudaMemcpyAsync(lambdas, sc.lt, sizeof(double) * (size_t)(S + 1) * n,
                                            cudaMemcpyDeviceToDevice, s), "states copy")) != NV_OK)
      return st;
    return nv_cuda_check(cudaMemcpyAsync(yT, sc.lt + (size_t)S * n, sizeof(double) * n,
                                         cudaMemcpyDeviceToDevice, s), "final state copy");
  }
  for (int p = 0; p < passes; ++p) {
    const bool lastp = (p == passes - 1);
    double* out = lastp ? lambdas : (cur == sc.lt ? sc.lt2 : sc.lt);
    // E: float64 defects d_j = g^j(cur_j) - cur_{j+1}
    if ((st = launch_heat_defect(M, cur, sc.d, s)) != NV_OK) return st;
    // F: correction block vectors from zero
    ChainsArgs cf = blockc;
    cf.v = sc.d;
    cf.v_double = 1;
    cf.v_stride = n;
    cf.finals = sc.cpr;
    if ((st = launch_chains(cf, false, s, cs_many)) != NV_OK) return st;
    // G: correction at block ends
    ChainsArgs cgc = topc;
    cgc.v = sc.cpr;
    cgc.states = sc.E;
    if ((st = launch_chains(cgc, false, s, 16)) != NV_OK) return st;
    // H: e_j inside the blocks; lambda_j = cur_j + e_j
    ChainsArgs ch = blockc;
    ch.v = sc.d;
    ch.v_double = 1;
    ch.v_stride = n;
    ch.x0 = sc.E;
    ch.x0_stride = n;
    ch.states = out;
    ch.add = cur;
    ch.yT = lastp ? yT : nullptr;
    ch.write_state0 = 1;
    if ((st = launch_chains(ch, false, s, cs_many)) != NV_OK) return st;
    cur = out;
  }
  return NV_OK;
}
