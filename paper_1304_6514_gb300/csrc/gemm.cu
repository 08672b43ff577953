// BF16 tensor-core GEMM for the slice-conditioned MLP propagator:
//   D[M x 256] = A[M x K] . B[256 x K]^T  (both operands K-major, row-major in
//   HBM), float32 accumulation in tensor memory, fused epilogues.
//
// One CTA computes a 128 x 256 tile.  Thread 0 streams K-slabs of 64 bf16
// (128 B) of A (128 rows) and B (256 rows) with TMA (SWIZZLE_128B) through a
// four-stage mbarrier ring and issues tcgen05.mma (kind::f16, M=128, N=256,
// K=16); eight warps then read the accumulator back with tcgen05.ld, one
// accumulator row per thread (warps w and w+4 share the TMEM lane quarter
// w % 4 and take 128 columns each).  Split-K: blockIdx.y takes one K range and the
// epilogue accumulates with atomics.  Every wait is bounded (1 s); on timeout
// the kernel records NV_ETIMEOUT, waits (bounded) for its copies in flight,
// frees its tensor memory and returns.
//
// Epilogues (z = D + bias):
//   kAtomic   out32[m, n] += D                     (weight gradients, split-K)
//   kFwdTrain GELU'(z) saved (fp32, for the backward pass), h = GELU(z) stored
//             bf16 row-major and transposed (one erf serves both)
//   kBwd      dz = D * zin (zin = the saved GELU', row r / zdiv for row r of
//             D) stored bf16 row-major and, unless NULL, transposed; column
//             sums of dz added to dbias unless NULL
//   kFwdInfer h = GELU(z) stored bf16 row-major
#include <cuda_bf16.h>

#include <mutex>

#include "common.cuh"
#include "tc.cuh"

namespace nvpit {
namespace gemm {

constexpr int kBM = 128, kBN = 256, kBK = 64;
constexpr int kStages = 4;
constexpr int kStageA = kBM * 128;      // 16 KB
constexpr int kStageB = kBN * 128;      // 32 KB
constexpr int kSmem = kStages * (kStageA + kStageB) + 256 + 1024;

enum Mode { kAtomic = 0, kFwdTrain = 1, kBwd = 2, kFwdInfer = 3 };

struct Args {
  int M, K, k_per_split, mode;
  int zdiv;            // kBwd: row r of D takes zin row r / zdiv
  float* out32;
  const float* bias;
  float* zsave;
  const float* zin;
  __nv_bfloat16* out_bf;
  __nv_bfloat16* out_bfT;
  float* dbias;
  int* status;
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
// GELU(z) = z Phi(z) and GELU'(z) = Phi(z) + z phi(z), sharing Phi's erf
__device__ __forceinline__ float gelu_with_grad(float z, float* grad) {
  const float cdf = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
  *grad = cdf + z * 0.39894228040143268f * expf(-0.5f * z * z);
  return z * cdf;
}

constexpr int kThreads = 256;

// MODE: the epilogue (one instantiation each keeps the code per kernel small)
template <int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_bf16_tn_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, Args a) {
  using namespace tc;
  extern __shared__ unsigned char smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = base;
  uint8_t* sB = base + kStages * kStageA;
  uint64_t* full = reinterpret_cast<uint64_t*>(base + kStages * (kStageA + kStageB));
  uint64_t* empty = full + kStages;
  uint64_t* done = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kBM;
  const int k0 = blockIdx.y * a.k_per_split;
  const int k1 = min(a.K, k0 + a.k_per_split);
  const int nk = (k1 - k0) / kBK;

  if (warp == 0) tmem_alloc(tmem_slot, kBN);
  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (tid == 0) {
    const uint32_t idesc = idesc_bf16(kBM, kBN);
    uint32_t fph[kStages] = {0, 0, 0, 0}, eph[kStages] = {0, 0, 0, 0};
    int issued = 0;
    bool ok = true;
    for (; issued < min(kStages, nk); ++issued) {
      const int st = issued;
      mbar_expect_tx(&full[st], kStageA + kStageB);
      tma_load_2d(sA + st * kStageA, &tmA, &full[st], k0 + issued * kBK, m0);
      tma_load_2d(sB + st * kStageB, &tmB, &full[st], k0 + issued * kBK, 0);
    }
    for (int s = 0; s < nk && ok; ++s) {
      const int st = s % kStages;
      ok = mbar_wait(&full[st], fph[st]);
      fph[st] ^= 1;
      if (!ok) break;
      fence_after();
      const uint32_t aaddr = smem_u32(sA + st * kStageA), baddr = smem_u32(sB + st * kStageB);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk)
        mma_bf16(tmem, sdesc_k_sw128(aaddr + kk * 32), sdesc_k_sw128(baddr + kk * 32), idesc,
                 (s | kk) != 0);
      mma_commit(&empty[st]);
      if (issued < nk) {
        ok = mbar_wait(&empty[st], eph[st]);
        eph[st] ^= 1;
        if (!ok) break;
        mbar_expect_tx(&full[st], kStageA + kStageB);
        tma_load_2d(sA + st * kStageA, &tmA, &full[st], k0 + issued * kBK, m0);
        tma_load_2d(sB + st * kStageB, &tmB, &full[st], k0 + issued * kBK, 0);
        ++issued;
      }
    }
    if (ok) mma_commit(done);
    if (!ok) {
      abort_flag = 1;
      record_status(a.status, NV_ETIMEOUT);
      for (int s = 0; s < kStages; ++s) mbar_wait(&full[s], fph[s]);   // copies in flight (bounded)
    }
  }
  __syncthreads();
  if (!abort_flag && !tc::mbar_wait(done, 0)) abort_flag = 1;
  __syncthreads();
  if (!abort_flag) {
    fence_after();
    // After the last MMA has completed (done) the stage memory is free: each
    // warp transposes its 32 x 32 chunks there, so that row-major traffic
    // (float32 results, saved pre-activations, bf16 row-major copies, the
    // split-K accumulation) moves as 128-byte rows across the lanes instead of
    // one 1 KB-strided row per lane.  Tile t: 32 x 33 floats per warp (two per
    // warp for the training forward pass: 67.6 KB of the 192 KB of stages).
    float* t = reinterpret_cast<float*>(base) + warp * 32 * 33;
    const int quarter = warp & 3, half = warp >> 2;   // TMEM lanes 32q .. 32q+31, columns 128h ..
    const int m = quarter * 32 + lane;
    const int row = m0 + m;
    const int wrow0 = m0 + quarter * 32;               // first row of this warp
    const int nrows = max(0, min(32, a.M - wrow0));
    for (int c0 = half * (kBN / 2); c0 < (half + 1) * (kBN / 2); c0 += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, v);
      if constexpr (MODE == kAtomic) {
#pragma unroll
        for (int i = 0; i < 32; ++i) t[lane * 33 + i] = v[i];
        __syncwarp();
        #pragma unroll
        for (int r = 0; r < 32; ++r)
          if (r < nrows) atomicAdd(a.out32 + (int64_t)(wrow0 + r) * kBN + c0 + lane, t[r * 33 + lane]);
        __syncwarp();
      } else if constexpr (MODE == kFwdTrain || MODE == kFwdInfer) {
        // h and GELU'(z) go straight to two tiles (the second after all eight
        // warps' first tiles), so no second 32-value array stays live
        float* t2 = reinterpret_cast<float*>(base) + (kThreads / 32 + warp) * 32 * 33;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float z = v[i] + a.bias[c0 + i];
          float gp = 0.f;
          const float h = MODE == kFwdTrain ? gelu_with_grad(z, &gp) : gelu_f(z);
          const __nv_bfloat16 hb = __float2bfloat16(h);
          if (MODE == kFwdTrain && row < a.M && a.out_bfT) a.out_bfT[(int64_t)(c0 + i) * a.M + row] = hb;
          t[lane * 33 + i] = __bfloat162float(hb);      // exact: hb is a bf16 value
          if (MODE == kFwdTrain) t2[lane * 33 + i] = gp;
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < 32; ++r)
          if (r < nrows) {
            a.out_bf[(int64_t)(wrow0 + r) * kBN + c0 + lane] = __float2bfloat16(t[r * 33 + lane]);
            if (MODE == kFwdTrain) a.zsave[(int64_t)(wrow0 + r) * kBN + c0 + lane] = t2[r * 33 + lane];
          }
        __syncwarp();
      } else {   // kBwd: zin arrives by rows, dz leaves by rows and transposed
        // all 32 loads in flight before any is used (rows past M repeat the
        // last valid row; nrows >= 1 for every warp that has rows)
#pragma unroll
        for (int h = 0; h < 32; h += 16) {           // two batches of 16 keep the registers in bounds
          float zr[16];
#pragma unroll
          for (int r = 0; r < 16; ++r)
            zr[r] = a.zin[(int64_t)((wrow0 + min(h + r, nrows - 1)) / a.zdiv) * kBN + c0 + lane];
#pragma unroll
          for (int r = 0; r < 16; ++r) t[(h + r) * 33 + lane] = zr[r];
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float dz = row < a.M ? v[i] * t[lane * 33 + i] : 0.f;
          if (row < a.M && a.out_bfT) a.out_bfT[(int64_t)(c0 + i) * a.M + row] = __float2bfloat16(dz);
          v[i] = dz;
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 32; ++i) t[lane * 33 + i] = v[i];
        __syncwarp();
        // lane l: column c0 + l over the warp's 32 rows: bias gradient and the
        // row-major bf16 copy (rows past M hold dz = 0)
        float colsum = 0.f;
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const float dz = t[r * 33 + lane];
          colsum += dz;
          if (r < nrows) a.out_bf[(int64_t)(wrow0 + r) * kBN + c0 + lane] = __float2bfloat16(dz);
        }
        if (a.dbias) atomicAdd(a.dbias + c0 + lane, colsum);
        __syncwarp();
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kBN);
}

}  // namespace gemm
}  // namespace nvpit

using namespace nvpit;

typedef CUresult (*EncodeTiledFnG)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                   CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                   CUtensorMapFloatOOBfill);

static nv_status gemm_encode_fn(EncodeTiledFnG* out) {
  static std::mutex mu;
  static EncodeTiledFnG fn = nullptr;
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
    fn = reinterpret_cast<EncodeTiledFnG>(p);
  }
  *out = fn;
  return NV_OK;
}

// 2-D bf16 tensor map over a row-major [rows][K] matrix, box 64 x box_rows.
static nv_status bf16_map(CUtensorMap* map, const void* ptr, int rows, int K, int box_rows) {
  EncodeTiledFnG enc = nullptr;
  nv_status st = gemm_encode_fn(&enc);
  if (st != NV_OK) return st;
  const cuuint64_t gdim[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t gstride[1] = {(cuuint64_t)K * 2};
  const cuuint32_t box[2] = {(cuuint32_t)gemm::kBK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult cr = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), gdim, gstride, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return nv_fail(NV_ECUDA, "cuTensorMapEncodeTiled (bf16) failed (%d)", (int)cr);
  return NV_OK;
}

// Sets the kernel's shared-memory limit once (before any graph capture).
nv_status gemm_bf16_prepare() {
  const void* fns[] = {(const void*)gemm::gemm_bf16_tn_kernel<gemm::kAtomic>,
                       (const void*)gemm::gemm_bf16_tn_kernel<gemm::kFwdTrain>,
                       (const void*)gemm::gemm_bf16_tn_kernel<gemm::kBwd>,
                       (const void*)gemm::gemm_bf16_tn_kernel<gemm::kFwdInfer>};
  for (const void* f : fns) {
    nv_status st = nv_cuda_check(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, gemm::kSmem),
                                 "gemm smem attribute");
    if (st != NV_OK) return st;
  }
  return NV_OK;
}

// D[M x 256] = A[M x K] B[256 x K]^T with epilogue `mode`; splits > 1 divides K.
nv_status launch_gemm_bf16(const void* A, const void* B, int M, int K, int splits, int mode, float* out32,
                           const float* bias, float* zsave, const float* zin, void* out_bf, void* out_bfT,
                           float* dbias, int* status, cudaStream_t s, int zdiv) {
  if (M % gemm::kBM || K % gemm::kBK || splits < 1 || (K / gemm::kBK) % splits || zdiv < 1)
    return nv_fail(NV_EINVAL, "gemm shape M=%d K=%d splits=%d zdiv=%d not tiled", M, K, splits, zdiv);
  CUtensorMap ta, tb;
  nv_status st = bf16_map(&ta, A, M, K, gemm::kBM);
  if (st != NV_OK) return st;
  if ((st = bf16_map(&tb, B, gemm::kBN, K, gemm::kBN)) != NV_OK) return st;
  gemm::Args a{};
  a.M = M;
  a.K = K;
  a.k_per_split = K / splits;
  a.mode = mode;
  a.zdiv = zdiv;
  a.out32 = out32;
  a.bias = bias;
  a.zsave = zsave;
  a.zin = zin;
  a.out_bf = static_cast<__nv_bfloat16*>(out_bf);
  a.out_bfT = static_cast<__nv_bfloat16*>(out_bfT);
  a.dbias = dbias;
  a.status = status;
  const dim3 grid(M / gemm::kBM, splits);
  switch (mode) {
    case gemm::kAtomic: gemm::gemm_bf16_tn_kernel<gemm::kAtomic><<<grid, gemm::kThreads, gemm::kSmem, s>>>(ta, tb, a); break;
    case gemm::kFwdTrain: gemm::gemm_bf16_tn_kernel<gemm::kFwdTrain><<<grid, gemm::kThreads, gemm::kSmem, s>>>(ta, tb, a); break;
    case gemm::kBwd: gemm::gemm_bf16_tn_kernel<gemm::kBwd><<<grid, gemm::kThreads, gemm::kSmem, s>>>(ta, tb, a); break;
    case gemm::kFwdInfer: gemm::gemm_bf16_tn_kernel<gemm::kFwdInfer><<<grid, gemm::kThreads, gemm::kSmem, s>>>(ta, tb, a); break;
    default: return nv_fail(NV_EINVAL, "unknown gemm epilogue %d", mode);
  }
  return nv_cuda_check(cudaGetLastError(), "gemm_bf16_tn_kernel launch");
}
