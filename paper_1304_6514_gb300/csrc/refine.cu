// Reduced-precision composition with float64 refinement (NV_BF16_REFINE,
// NV_FP32_REFINE): the advection-diffusion system (d = 4096) over the tiled
// chain, the heat and wave equations (d <= 512) over the cluster chain.
//
// At d = 4096 the composition for one initial state is a chain of S
// matrix-vector products that reads every map once, so its time is the maps'
// bytes over HBM bandwidth; a tensor-core scan of the maps would cost
// 2 d^3 (S - 1) = 7e13 FLOP, far more.  Storing the maps in bfloat16 halves
// the bytes.  The bfloat16 rounding (2^-9 relative per entry) is then won back
// by the residual correction the Conclusion proposes, with the reduced maps
// as the coarse propagator:
//   lt_j   chain over the bfloat16 maps from y0 (float32 accumulation)
//   d_j  = g^j(lt_j) - lt_{j+1}         float64 fine solve per slice
//   e_0  = 0, e_{j+1} = At_j e_j + d_j  the same chain over the bfloat16 maps
//   lt_j <- lt_j + e_j                  written by the chain as it goes
// The error after a pass is sum_k At^(S-k) (At - A) e_(k-1): the maps'
// rounding accumulates along the chain in the modes the maps barely damp (the
// mean, which the periodic operator conserves, and the lowest Fourier modes,
// |lambda| ~ 0.9986 per slice).  With bfloat16 maps (2^-9) a pass contracts
// the error by roughly S / 1500 on the 64 x 64 problem (0.3 to 0.13 at
// S = 512), so the default number of passes grows with log S (six at
// S = 512, measured 8.5e-6); float32 maps (2^-24) need one pass at S = 512.
#include <algorithm>

#include "internal.h"

static nv_status ensure_scratch(nv_maps* M, size_t need, cudaStream_t s) {
  if (M->scan_ws_bytes >= need) return NV_OK;
  if (M->scan_ws) {
    cudaStreamSynchronize(s);
    cudaFree(M->scan_ws);
    M->scan_ws = nullptr;
    M->scan_ws_bytes = 0;
  }
  nv_status st = nv_cuda_check(cudaMalloc(&M->scan_ws, need), "refinement scratch allocation");
  if (st == NV_OK) M->scan_ws_bytes = need;
  return st;
}

// The heat equations and the wave equation (d <= 512): the same passes with
// the cluster chain (compose.cu), whose options carry d_j (v), the
// approximate states (add) and every state written; the defects come from
// the family's float64 defect kernel (heat: nine-point / literal RK4 stages;
// wave: leapfrog on the two-level state).
static nv_status cluster_chain_refine(nv_maps* M, const double* y0, double* yT, double* lambdas,
                                      double* lt, double* lt2, double* d, int passes, cudaStream_t s) {
  const bool wave = M->rhs_kind == NV_RHS_WAVE_CHEB;
  const int n = M->dim, S = M->S;
  const float* maps = static_cast<const float*>(M->data);
  ChainsArgs c{};
  c.n = n;
  c.nchains = 1;
  c.len = S;
  c.S = S;
  c.A = maps + n;                        // columns 1..d of each slice
  c.a_stride = (int64_t)n * (n + 1);
  c.status = M->status;
  c.write_state0 = 1;
  c.band = g_tune.chain_dense ? 0 : M->band;
  ChainsArgs approx = c;                 // lt: the chain over the float32 maps from y0
  approx.v = maps;                       // column 0, b_j
  approx.v_stride = (int64_t)n * (n + 1);
  approx.x0 = y0;
  approx.states = passes == 0 ? lambdas : lt;
  approx.yT = passes == 0 ? yT : nullptr;
  nv_status st = launch_chains(approx, false, s, 16);
  if (st != NV_OK || passes == 0) return st;
  double* cur = lt;
  for (int p = 0; p < passes; ++p) {
    const bool last = p == passes - 1;
    double* out = last ? lambdas : (cur == lt ? lt2 : lt);
    if ((st = wave ? launch_wave_defect(M, cur, d, s) : launch_heat_defect(M, cur, d, s)) != NV_OK) return st;
    ChainsArgs corr = c;                 // e_{j+1} = At_j e_j + d_j from e_0 = 0, written as cur + e
    corr.v = d;
    corr.v_double = 1;
    corr.v_stride = n;
    corr.add = cur;
    corr.states = out;
    corr.yT = last ? yT : nullptr;
    if ((st = launch_chains(corr, false, s, 16)) != NV_OK) return st;
    cur = out;
  }
  return NV_OK;
}

// Default number of float64 passes: one for float32 maps of the damped
// problems; two for the undamped wave equation, whose float32 map error
// (~3e-6 per map) composes coherently over all S slices, so that one pass
// only contracts its 6e-3 to about 1e-5; and for bfloat16 maps two passes
// up to 32 slices and one more for every doubling of S beyond (each pass
// contracts by roughly S / 1500 at the advection-diffusion problem).
int default_refine_passes(const nv_maps* M) {
  if (M->prec == NV_BF16_REFINE) {
    int p = 2;
    for (int64_t s = 32; s < M->S; s *= 2) ++p;
    return p;
  }
  return M->rhs_kind == NV_RHS_WAVE_CHEB ? 2 : 1;
}

nv_status launch_chain_refine(nv_maps* M, const double* y0, double* yT, double* lambdas, cudaStream_t s) {
  const bool heat = M->rhs_kind == NV_RHS_HEAT1D || M->rhs_kind == NV_RHS_HEAT1D_VARCOEF;
  const bool wave = M->rhs_kind == NV_RHS_WAVE_CHEB;
  if (M->rhs_kind != NV_RHS_ADVDIFF2D && !heat && !wave)
    return nv_fail(NV_ENOTSUP, "chain refinement is built for the heat, wave and advection-diffusion equations");
  const int n = M->dim, S = M->S;
  const int dflt = default_refine_passes(M);
  const int passes = g_tune.refine_passes > 0 ? g_tune.refine_passes : (g_tune.refine_passes < 0 ? 0 : dflt);
  const bool pipelined = heat && passes >= 1 && g_tune.refine_schedule != 1;
  const size_t states = (size_t)(S + 1) * n;
  // two state sets, the defects, one zero vector (or the pipelined passes' scratch)
  size_t need = sizeof(double) * (2 * states + (size_t)S * n + (size_t)n);
  if (pipelined) need = std::max(need, heat_wavefront_scratch_bytes(n, S, passes));
  nv_status st = ensure_scratch(M, need, s);
  if (st != NV_OK) return st;
  if (pipelined) {   // all passes in one launch where they fit, else one after another
    st = launch_heat_wavefront(M, y0, yT, lambdas, passes, M->scan_ws, s);
    if (st != NV_ENOTSUP) return st;
  }
  double* lt = static_cast<double*>(M->scan_ws);
  double* lt2 = lt + states;
  double* d = lt2 + states;
  if (heat || wave) return cluster_chain_refine(M, y0, yT, lambdas, lt, lt2, d, passes, s);
  double* zero = d + (size_t)S * n;
  if ((st = nv_cuda_check(cudaMemsetAsync(zero, 0, sizeof(double) * n, s), "zero state")) != NV_OK) return st;
  // approximate boundary states over the bfloat16 maps
  double* cur = lt;
  if ((st = launch_tile_chain(M, y0, passes == 0 ? yT : nullptr, passes == 0 && lambdas ? lambdas : cur,
                              nullptr, s)) != NV_OK)
    return st;
  if (passes == 0) return NV_OK;
  for (int p = 0; p < passes; ++p) {
    const bool last = p == passes - 1;
    double* out = last ? lambdas : (cur == lt ? lt2 : lt);
    if ((st = launch_advdiff_defect(M, cur, d, s)) != NV_OK) return st;
    TileChainExtra ex{};
    ex.vadd = d;
    ex.base = cur;
    ex.col0_off = 1;
    if ((st = launch_tile_chain(M, zero, last ? yT : nullptr, out, &ex, s)) != NV_OK) return st;
    cur = out;
  }
  return NV_OK;
}
