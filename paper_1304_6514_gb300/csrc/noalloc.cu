// Allocation-free composition of affine slice maps.
//
// Some callers cannot allocate device memory at the moment they compose: a
// host application whose memory pool already owns the whole GPU and hands out
// nothing further, a real-time loop that must not pay for (or synchronise on)
// cudaMalloc/cudaFree, or a plug-in running inside another runtime that only
// lends it the buffers it was given.  nv_compose_affine_noalloc serves them:
// the chain's scratch (grid-barrier counter, status word and the two ping-pong
// state vectors) lives in one file-scope __device__ array of fixed size
// instead of the maps object's workspace.  Every GPU that loads this library
// holds that array (kNoallocScratchBytes, about 64 KiB) until the process exits.
#include <mutex>

#include "common.cuh"

namespace {

constexpr int kNoallocMaxDim = NVPIT_NOALLOC_MAX_DIM;
constexpr size_t kStateOffset = 256;  // status word at 0, barrier counter at 16
constexpr size_t kNoallocScratchBytes = kStateOffset + 2 * sizeof(double) * kNoallocMaxDim;

// The shared scratch.  Host code must not pass this symbol to a kernel: on the
// host it names a stand-in object, not device memory.  Its device address is
// looked up once per device with cudaGetSymbolAddress (noalloc_scratch below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device, looked up on the
// first call made with that device current and kept for the process: after a
// cudaDeviceReset of that device the kept address is stale, so the entry
// point must not be used on a device that was reset.
nv_status noalloc_scratch(void** out) {
  int dev = -1;
  nv_status st = nv_cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (st != NV_OK) return st;
  if (dev < 0 || dev >= kMaxDevices) return nv_fail(NV_ENOTSUP, "device index %d too large", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    st = nv_cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch),
                       "cudaGetSymbolAddress of the no-alloc scratch");
    if (st != NV_OK) return st;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return NV_OK;
}

}  // namespace

extern "C" nv_status nv_compose_affine_noalloc(const void* maps_dev, int32_t prec, int32_t dim,
                                               int32_t S, const double* y0_dev, double* yT_dev,
                                               double* lambdas_dev, int32_t* status_dev,
                                               void* stream) {
  if (!maps_dev || !y0_dev || !yT_dev) return nv_fail(NV_EINVAL, "maps, y0 and yT must not be NULL");
  if (prec != NV_FP64 && prec != NV_FP32)
    return nv_fail(NV_EINVAL, "no-alloc composition takes NV_FP64 or NV_FP32 maps");
  if (dim < 1 || dim > kNoallocMaxDim)
    return nv_fail(NV_EINVAL, "no-alloc composition supports 1 <= dim <= %d (got %d): its scratch "
                              "is a fixed-size static array", kNoallocMaxDim, dim);
  if (S < 1) return nv_fail(NV_EINVAL, "S must be >= 1");
  void* base = nullptr;
  nv_status st = noalloc_scratch(&base);
  if (st != NV_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* b = static_cast<char*>(base);
  int* status = reinterpret_cast<int*>(b);
  unsigned* bar = reinterpret_cast<unsigned*>(b + 16);
  double* xbuf = reinterpret_cast<double*>(b + kStateOffset);
  // The status word and the barrier counter must start at zero; the state
  // vectors are fully written before they are read.
  st = nv_cuda_check(cudaMemsetAsync(base, 0, kStateOffset, s), "no-alloc scratch reset");
  if (st != NV_OK) return st;
  // 16 rows per CTA, whatever nv_tune_set key 1 says: every dim up to the
  // limit then needs at most 256 resident CTAs
  st = launch_affine_chain_buffers(maps_dev, prec, dim, S, y0_dev, yT_dev, lambdas_dev, xbuf, bar,
                                   status, s, 16);
  if (st != NV_OK) return st;
  if (status_dev)
    st = nv_cuda_check(cudaMemcpyAsync(status_dev, status, sizeof(int32_t), cudaMemcpyDeviceToDevice, s),
                       "no-alloc status copy");
  return st;
}
