// Internal declarations shared by the translation units of libnvpit.so.
// Not part of the ABI: include/nvpit.h is.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/nvpit.h"

// Device status word values mirror nv_status.
#define NVPIT_MAX_PARAMS 8

struct nv_maps {
  // problem (Figure "pseudocode", Given)
  int32_t rhs_kind;
  int32_t dim;
  double params[NVPIT_MAX_PARAMS];
  int32_t nparams;
  double t0, T, H, h;
  int32_t S;
  int64_t m;
  int32_t scheme;
  // samples / map
  int32_t map;
  int32_t prec;
  int32_t per_dim;
  double lo[2], hi[2];
  int32_t oob_policy;
  // map storage (device)
  void* data;
  int64_t bytes;
  int64_t elems_per_slice;
  int32_t elem_bytes;
  // workspace (device), one allocation
  void* ws;
  size_t ws_bytes;
  int* status;                 // device status word (nv_status)
  unsigned long long* oob;     // evaluations outside Xi
  unsigned int* bar;           // grid-barrier counter
  double* xbuf;                // 2 * dim doubles (ping-pong chain state)
  double* coef;                // per-slice staged coefficients (may be NULL)
  int64_t coef_per_slice;
  double* aux;                 // operator storage (wave: D and D2), may be NULL
  int64_t aux_elems;
  // 0: dense maps; > 0: every A_j[r][c] with |r - c| >= band is exactly zero
  // (set by the build where the scheme fixes it; the chains then skip them)
  int32_t band;
  // what the last build ran: point-steps integrated per slice, main kernel
  int64_t work_per_slice;
  char build_kernel[64];
  // reduced-precision composition scratch (NV_TF32_REFINE), allocated lazily
  void* scan_ws;
  size_t scan_ws_bytes;
  int device;
};

// Error helpers (api.cu).  nv_fail records the message for nv_last_error().
nv_status nv_fail(nv_status code, const char* fmt, ...);
nv_status nv_cuda_check(cudaError_t e, const char* what);

// Launchers.  Each validates nothing (the API layer did), launches on `s`
// and returns NV_OK or NV_ECUDA.
nv_status launch_coef_tables(nv_maps* M, cudaStream_t s);
nv_status launch_table_build(nv_maps* M, cudaStream_t s, int block);
nv_status launch_affine_build(nv_maps* M, cudaStream_t s);
nv_status launch_table_compose(const nv_maps* M, const double* y0, double* yT, double* lambdas,
                               cudaStream_t s);
nv_status launch_affine_chain(const nv_maps* M, const double* y0, double* yT, double* lambdas,
                              cudaStream_t s, int rows_per_cta);
// Chain composition over caller-supplied buffers (used by the allocation-free
// entry point): maps in the AFFINE layout, prec NV_FP64 or NV_FP32, xbuf of
// 2*n doubles, bar and status zeroed by the caller before the launch.
nv_status launch_affine_chain_buffers(const void* maps, int prec, int n, int S, const double* y0,
                                      double* yT, double* lambdas, double* xbuf, unsigned* bar,
                                      int* status, cudaStream_t s, int rows_per_cta);
nv_status launch_serial_fine(int32_t rhs_kind, int32_t dim, const double* params, double t0,
                             double H, double h, int32_t S, int64_t m, int32_t scheme,
                             const double* y0, double* yT, cudaStream_t s);
nv_status launch_scan_refine(nv_maps* M, const double* y0, double* yT, double* lambdas,
                             cudaStream_t s);
nv_status launch_chain_refine(nv_maps* M, const double* y0, double* yT, double* lambdas,
                              cudaStream_t s);

// Tiled grid-wide chain (d > 512) over the maps' own storage, with the
// options of the float64 correction chain.
struct TileChainExtra {
  const double* vadd;   // v_j added to slice j's product (S x n), or NULL
  const double* base;   // added to every state written (S+1 x n), or NULL
  int col0_off;         // 1: drop column 0 (b_j) of the maps
};
// Bytes of the d > 512 chain's partial-sum scratch (in the maps workspace).
size_t tile_chain_ring_scratch(int n, int ncb, int value_bytes);
size_t tile_chain_scratch_bytes(int prec, int n, int sms);
// Pipelined refinement of the heat equations over float32 maps (wavefront.cu):
// chains and defects of all passes in one cooperative launch; NV_ENOTSUP when
// the shape or device does not fit it.  scratch: heat_wavefront_scratch_bytes.
size_t heat_wavefront_scratch_bytes(int n, int S, int passes);
nv_status launch_heat_wavefront(nv_maps* M, const double* y0, double* yT, double* lambdas, int passes,
                                void* scratch, cudaStream_t s);
nv_status launch_tile_chain(const nv_maps* M, const double* y0, double* yT, double* lambdas,
                            const TileChainExtra* ex, cudaStream_t s);
// float64 defects of the advection-diffusion maps: d_j = g^j(lam_j) - lam_{j+1}
nv_status launch_advdiff_defect(const nv_maps* M, const double* lam, double* d, cudaStream_t s);

// Batched cluster chains (compose.cu, affine_chains_kernel): chain q runs
// x <- A_j x + v_j over slices j = q*len .. min(S, (q+1)*len) - 1.
struct ChainsArgs {
  int n, nchains, len, S, rpc;
  const void* A;          // A_j = A + j * a_stride (elements of MT), column-major, ld n
  int64_t a_stride;
  const void* v;          // v_j = v + j * v_stride (elements of MT, or double if v_double)
  int64_t v_stride;
  int v_double;
  const double* x0;       // start of chain q: x0 + q * x0_stride; NULL = zero
  int64_t x0_stride;
  double* states;         // optional: states[(j+1)*n + i] = x after slice j (+ add)
  double* finals;         // optional: finals[q*n + i] = x at the end of chain q
  const double* add;      // optional: added to x when writing states / yT
  double* yT;             // optional: x after the last slice S-1 (+ add)
  int write_state0;       // chain 0 also writes states[0..n) = x0 (+ add)
  int* status;            // device status word (bounded waits record NV_ETIMEOUT)
  int band;               // 0 dense; > 0: A_j[r][c] == 0 whenever |r - c| >= band
};

nv_status launch_chains(const ChainsArgs& args, bool f64, cudaStream_t s, int want_csize);
nv_status launch_heat_defect(const nv_maps* M, const double* lam_tilde, double* d, cudaStream_t s);
// float64 defects of the wave maps (leapfrog from each approximate state)
nv_status launch_wave_defect(const nv_maps* M, const double* lam, double* d, cudaStream_t s);
// float64 correction passes NV_*_REFINE runs when nv_tune_set key 5 is 0
int default_refine_passes(const nv_maps* M);

// Tunables (set by nv_tune_set, read by the launchers).
struct nv_tunables {
  int table_block;         // threads per CTA for the table build
  int chain_rows_per_cta;  // rows of the chain GEMV owned by one CTA
  int affine_warps;        // warps per CTA in the affine build
  int chain_cluster;       // CTAs per cluster of the d <= 512 chain (0 auto, < 0 grid-wide)
  int scan_block;          // slices per block of the tensor-core scan (0 auto)
  int refine_passes;       // float64 correction passes of NV_TF32_REFINE (0 = 1, < 0 none)
  int heat_step_form;      // homogeneous heat columns: 0 auto, 1 Horner stages, 2 nine-point stencil, 3 / 4 / 5 one / two / three windows
  int test_barrier_extra;  // test hook: participants that never arrive at the row chain's grid barrier
  int mlp_wgrad_splits;    // split-K of the MLP weight-gradient GEMMs (0 auto)
  int tile_chain_form;     // d > 512 chain: 0 auto, 1 register batches, 2 bulk-copy ring
  int refine_schedule;     // heat NV_FP32_REFINE: 0 auto (pipelined), 1 sequential passes
  int test_withhold_defect;  // test hook: pipelined refinement never flags pass 1's defect of this slice + 1
  int test_skip_partials;    // test hook: the d > 512 ring chain's CTA 0 never stores step value - 1's partials
  int chain_dense;           // 1: the d <= 256 cluster chains read every column even of banded maps
  int adv_build_form;        // advection-diffusion build: 0 auto (windows first), 1 whole grid only
  int adv_fp64_rows;         // float64 advection-diffusion window build: rows per thread, 0 (= 16), 8 or 32
  int heat_f32_lanes;        // float32 heat three-window build: 0 auto, 1 / 2: one lane of 22 rows / two of 11,
                             // 3 / 4: the same with two slices per packed f32x2 register
  int learned_first_form;    // iteration 0 of nv_mlp_parareal: 0 auto, 1 per-slice tcgen05 forward, 2 fused sweep
  int learned_correction_form;  // nv_mlp_parareal corrections: 0 Jacobians of the learned composition,
                                // 1 tangent sweep, 2 Jacobians at each previous iterate
  int learned_f32_iters;        // nv_mlp_parareal: leading iterations with float32 fine solves (0: none)
};
extern nv_tunables g_tune;

// Grid of a persistent kernel: the CTAs that fit on every SM at once (from the
// occupancy of `kernel` with `block` threads), or fewer when work_warps warps
// need fewer.
template <typename K>
inline nv_status persistent_grid(K kernel, int block, int64_t work_warps, int* grid_out, size_t smem = 0) {
  int sms = 152, dev = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  nv_status st = nv_cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem),
                               "occupancy query");
  if (st != NV_OK) return st;
  int64_t grid = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
  grid = std::min<int64_t>(grid, (work_warps * 32 + block - 1) / block);
  *grid_out = (int)std::max<int64_t>(grid, 1);
  return NV_OK;
}
