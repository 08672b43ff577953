// C ABI of libnvpit.so (include/nvpit.h): argument validation, step planning,
// device allocation, dispatch to the kernels, thread-local error messages.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>

#include "internal.h"

nv_status launch_serial_table(int32_t rhs_kind, const double* params, double t0, double H,
                              double h, int32_t S, int64_t m, int32_t scheme, const double* y0,
                              double* yT, cudaStream_t s);
nv_status launch_serial_heat(const nv_maps* M, const double* y0, double* yT, cudaStream_t s);
nv_status launch_serial_advdiff(const nv_maps* M, const double* y0, double* yT, cudaStream_t s);
nv_status launch_serial_wave(const nv_maps* M, const double* y0, double* yT, cudaStream_t s);
int64_t wave_aux_elems(int d);

nv_tunables g_tune = {};

static thread_local char g_err[512] = "";

nv_status nv_fail(nv_status code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

nv_status nv_cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return NV_OK;
  if (e == cudaErrorMemoryAllocation)
    return nv_fail(NV_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  return nv_fail(NV_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

extern "C" const char* nv_last_error(void) { return g_err; }
extern "C" int32_t nv_version(void) { return NVPIT_VERSION; }

extern "C" nv_status nv_plan_steps(double t0, double T, int32_t S, double dt,
                                   int64_t steps_per_slice, int64_t* m, double* h) {
  if (!(T > t0) || S < 1 || !isfinite(t0) || !isfinite(T))
    return nv_fail(NV_EINVAL, "need finite t0 < T and S >= 1");
  const double H = (T - t0) / S;
  int64_t mm;
  if (steps_per_slice > 0) {
    mm = steps_per_slice;
  } else {
    if (!(dt > 0.0) || !isfinite(dt)) return nv_fail(NV_EINVAL, "need dt > 0 or steps_per_slice > 0");
    const double ratio = H / dt - 1e-9;
    if (ratio > 1e15) return nv_fail(NV_EINVAL, "H/dt too large");
    mm = (int64_t)ceil(ratio);
    if (mm < 1) mm = 1;
  }
  if (m) *m = mm;
  if (h) *h = H / (double)mm;
  return NV_OK;
}

// ----------------------------------------------------------------- validation

static nv_status check_rhs(const nv_rhs* rhs, double* params, int32_t* nparams) {
  if (!rhs) return nv_fail(NV_EINVAL, "rhs is NULL");
  if (rhs->nparams < 0 || rhs->nparams > NVPIT_MAX_PARAMS || (rhs->nparams > 0 && !rhs->params))
    return nv_fail(NV_EINVAL, "rhs params: need 0..%d values and a non-NULL array", NVPIT_MAX_PARAMS);
  for (int i = 0; i < NVPIT_MAX_PARAMS; ++i) params[i] = 0.0;
  for (int i = 0; i < rhs->nparams; ++i) {
    if (!isfinite(rhs->params[i])) return nv_fail(NV_EINVAL, "rhs param %d is not finite", i);
    params[i] = rhs->params[i];
  }
  *nparams = rhs->nparams;
  const int d = rhs->dim;
  switch (rhs->kind) {
    case NV_RHS_LINEAR_SCALAR:
      if (rhs->nparams < 1) return nv_fail(NV_EINVAL, "linear scalar rhs needs params {lambda}");
      if (d != 1) return nv_fail(NV_EINVAL, "linear scalar rhs has dim 1");
      break;
    case NV_RHS_SQUARE:
    case NV_RHS_COS_CUBIC:
      if (d != 1) return nv_fail(NV_EINVAL, "scalar rhs has dim 1");
      break;
    case NV_RHS_VDP:
      if (d != 2) return nv_fail(NV_EINVAL, "Van der Pol rhs has dim 2");
      if (rhs->nparams < 1) return nv_fail(NV_EINVAL, "Van der Pol rhs needs params {mu}");
      break;
    case NV_RHS_CHAIN3:
      if (d != 6) return nv_fail(NV_EINVAL, "chain rhs has dim 6");
      if (rhs->nparams == 0) { params[0] = 1.0; params[1] = 0.5; params[2] = 0.05; *nparams = 3; }
      else if (rhs->nparams < 3) return nv_fail(NV_EINVAL, "chain rhs needs params {k, k3, c}");
      break;
    case NV_RHS_HEAT1D:
      if (d < 1 || d > 512) return nv_fail(NV_EINVAL, "heat rhs dim must be 1..512");
      if (rhs->nparams == 0) { params[0] = 1.0; params[1] = 1.0; *nparams = 2; }
      else if (rhs->nparams < 2) return nv_fail(NV_EINVAL, "heat rhs needs params {kappa, amp}");
      break;
    case NV_RHS_HEAT1D_VARCOEF:
      if (d < 1 || d > 512) return nv_fail(NV_EINVAL, "heat rhs dim must be 1..512");
      break;
    case NV_RHS_ADVDIFF2D: {
      const int nx = (int)lround(sqrt((double)d));
      if (d < 4 || nx * nx != d) return nv_fail(NV_EINVAL, "advection-diffusion dim must be nx*nx");
      if (rhs->nparams == 0) { params[0] = 0.01; params[1] = 1.0; params[2] = 0.5; *nparams = 3; }
      else if (rhs->nparams < 3) return nv_fail(NV_EINVAL, "advection-diffusion needs {nu, ax, ay}");
      break;
    }
    case NV_RHS_WAVE_CHEB: {
      if (d < 2 || d > 160 || d % 2) return nv_fail(NV_EINVAL, "wave rhs dim must be 2(M-1) with 2 <= M <= 81");
      if (rhs->nparams == 0) { params[0] = d / 2 + 1; *nparams = 1; }
      if (params[0] != (double)(d / 2 + 1)) return nv_fail(NV_EINVAL, "wave rhs: dim must be 2(M-1)");
      break;
    }
    default:
      return nv_fail(NV_EINVAL, "unknown rhs kind %d", rhs->kind);
  }
  return NV_OK;
}

static bool is_linear_kind(int k) {
  return k == NV_RHS_HEAT1D || k == NV_RHS_HEAT1D_VARCOEF || k == NV_RHS_ADVDIFF2D || k == NV_RHS_WAVE_CHEB;
}

// Leapfrog belongs to the two-level wave state and the wave state to leapfrog.
static nv_status check_scheme(int32_t kind, int32_t scheme) {
  if (scheme != NV_EULER && scheme != NV_RK4 && scheme != NV_LEAPFROG) return nv_fail(NV_EINVAL, "unknown scheme");
  if ((kind == NV_RHS_WAVE_CHEB) != (scheme == NV_LEAPFROG))
    return nv_fail(NV_EINVAL, "NV_LEAPFROG is the scheme of NV_RHS_WAVE_CHEB and only of it");
  return NV_OK;
}

static nv_status plan(const nv_rhs* rhs, double t0, double T, int32_t S, const nv_samples* sm,
                      const nv_steps* st, nv_maps* P) {
  memset(P, 0, sizeof(*P));
  nv_status e = check_rhs(rhs, P->params, &P->nparams);
  if (e != NV_OK) return e;
  if (!sm || !st) return nv_fail(NV_EINVAL, "samples and steps must not be NULL");
  if (S < 1 || S > (1 << 24)) return nv_fail(NV_EINVAL, "S must be 1..2^24");
  if ((e = check_scheme(rhs->kind, st->scheme)) != NV_OK) return e;
  if (st->prec < NV_FP64 || st->prec > NV_FP32_REFINE) return nv_fail(NV_EINVAL, "unknown precision");
  e = nv_plan_steps(t0, T, S, st->dt, st->steps_per_slice, &P->m, &P->h);
  if (e != NV_OK) return e;
  P->rhs_kind = rhs->kind;
  P->dim = rhs->dim;
  P->t0 = t0;
  P->T = T;
  P->S = S;
  P->H = (T - t0) / S;
  P->scheme = st->scheme;
  P->map = sm->map;
  P->prec = st->prec;
  P->per_dim = sm->per_dim;
  P->oob_policy = sm->oob_policy;
  for (int i = 0; i < 2; ++i) { P->lo[i] = sm->lo[i]; P->hi[i] = sm->hi[i]; }
  if (sm->oob_policy != NV_OOB_EXTRAPOLATE && sm->oob_policy != NV_OOB_ERROR)
    return nv_fail(NV_EINVAL, "unknown out-of-range policy");
  const int d = rhs->dim;
  switch (sm->map) {
    case NV_MAP_PL1D:
    case NV_MAP_BILINEAR2D: {
      const int want = sm->map == NV_MAP_PL1D ? 1 : 2;
      if (d != want) return nv_fail(NV_EINVAL, "map kind needs state dimension %d", want);
      if (sm->per_dim < 2 || sm->per_dim > (1 << 20))
        return nv_fail(NV_EINVAL, "per_dim must be 2..2^20");
      for (int i = 0; i < want; ++i)
        if (!(sm->hi[i] > sm->lo[i]) || !isfinite(sm->lo[i]) || !isfinite(sm->hi[i]))
          return nv_fail(NV_EINVAL, "need finite lo < hi in dimension %d", i);
      if (st->prec >= NV_TF32_REFINE) return nv_fail(NV_EINVAL, "reduced-precision refinement is for affine maps");
      if (is_linear_kind(rhs->kind)) return nv_fail(NV_EINVAL, "PDE right-hand sides use affine maps");
      if (rhs->kind == NV_RHS_CHAIN3) return nv_fail(NV_ENOTSUP, "6-D chain has no table map");
      P->elems_per_slice = (int64_t)sm->per_dim * (want == 2 ? sm->per_dim * 2 : 1);
      break;
    }
    case NV_MAP_AFFINE:
      if (!is_linear_kind(rhs->kind)) return nv_fail(NV_EINVAL, "affine maps need a linear rhs");
      if (st->prec == NV_BF16_REFINE && (rhs->kind != NV_RHS_ADVDIFF2D || d <= 512 || d % 8))
        return nv_fail(NV_ENOTSUP, "bfloat16 refinement is built for advection-diffusion with d > 512, d %% 8 == 0");
      if (st->prec == NV_FP32_REFINE &&
          !((rhs->kind == NV_RHS_ADVDIFF2D && d > 512 && d % 8 == 0) ||
            (rhs->kind == NV_RHS_HEAT1D || rhs->kind == NV_RHS_HEAT1D_VARCOEF) ||
            rhs->kind == NV_RHS_WAVE_CHEB))
        return nv_fail(NV_ENOTSUP, "float32 refinement is built for the heat, wave and advection-diffusion equations");
      if (rhs->kind == NV_RHS_WAVE_CHEB) {
        if (st->prec == NV_TF32_REFINE) return nv_fail(NV_ENOTSUP, "TF32 refinement is built for the heat equation");
        P->aux_elems = wave_aux_elems(d / 2);
      } else if (st->scheme != NV_RK4) {
        return nv_fail(NV_ENOTSUP, "affine maps are built with RK4");
      }
      P->elems_per_slice = (int64_t)d * (d + 1);
      break;
    default:
      return nv_fail(NV_EINVAL, "unknown map kind %d", sm->map);
  }
  P->elem_bytes = st->prec == NV_FP64 ? 8 : (st->prec == NV_BF16_REFINE ? 2 : 4);
  P->bytes = P->elems_per_slice * (int64_t)S * P->elem_bytes;
  if (rhs->kind == NV_RHS_COS_CUBIC) P->coef_per_slice = st->scheme == NV_RK4 ? 2 * P->m + 1 : P->m;
  return NV_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Map storage and workspace come from the device's stream-ordered pool on the
// build stream.  Once per device the pool keeps up to 1 GB of freed memory
// (instead of returning everything at each synchronisation), so a repeated
// nv_solve of a problem up to that size does not pay for fresh allocations;
// larger maps still go back to the driver when freed.
static nv_status pool_setup(int dev) {
  static std::mutex mu;
  static bool done[256] = {};
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 0 || dev >= 256 || done[dev]) return NV_OK;
  cudaMemPool_t pool;
  nv_status e = nv_cuda_check(cudaDeviceGetDefaultMemPool(&pool, dev), "default memory pool");
  if (e != NV_OK) return e;
  uint64_t keep = 1ull << 30;
  e = nv_cuda_check(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep), "pool threshold");
  if (e == NV_OK) done[dev] = true;
  return e;
}

static nv_status alloc_maps(nv_maps* P, cudaStream_t s) {
  nv_status e = nv_cuda_check(cudaGetDevice(&P->device), "cudaGetDevice");
  if (e != NV_OK) return e;
  if ((e = pool_setup(P->device)) != NV_OK) return e;
  e = nv_cuda_check(cudaMallocAsync(&P->data, (size_t)P->bytes, s), "map allocation");
  if (e != NV_OK) { P->data = nullptr; return e; }
  const size_t xoff = 256;
  // 2 float64 chain vectors + slack; for d > 512 also the tiled chain's
  // partial-sum scratch
  int sms = 0;
  if (P->dim > 512 &&
      (e = nv_cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device),
                         "SM count")) != NV_OK)
    return e;
  const size_t part_bytes = P->dim > 512 ? tile_chain_scratch_bytes(P->prec, P->dim, sms) : 0;
  const size_t coff = align256(xoff + sizeof(double) * 2 * (size_t)P->dim + 16 + part_bytes + 64);
  const size_t aoff = align256(coff + sizeof(double) * (size_t)(P->coef_per_slice * P->S));
  P->ws_bytes = aoff + sizeof(double) * (size_t)P->aux_elems;
  e = nv_cuda_check(cudaMallocAsync(&P->ws, P->ws_bytes, s), "workspace allocation");
  if (e != NV_OK) { cudaFreeAsync(P->data, s); P->data = nullptr; P->ws = nullptr; return e; }
  char* w = static_cast<char*>(P->ws);
  P->status = reinterpret_cast<int*>(w);
  P->oob = reinterpret_cast<unsigned long long*>(w + 8);
  P->bar = reinterpret_cast<unsigned*>(w + 16);
  P->xbuf = reinterpret_cast<double*>(w + xoff);
  P->coef = P->coef_per_slice ? reinterpret_cast<double*>(w + coff) : nullptr;
  P->aux = P->aux_elems ? reinterpret_cast<double*>(w + aoff) : nullptr;
  return nv_cuda_check(cudaMemsetAsync(P->ws, 0, 256, s), "workspace reset");
}

// Frees in the order of stream s (the caller has ordered s after all work
// on the maps).  The reduced-precision scratch is a plain allocation.
static void free_maps(nv_maps* P, cudaStream_t s) {
  if (!P) return;
  if (P->data) cudaFreeAsync(P->data, s);
  if (P->ws) cudaFreeAsync(P->ws, s);
  if (P->scan_ws) cudaFree(P->scan_ws);
  delete P;
}

// ----------------------------------------------------------------- entry points

extern "C" nv_status nv_build_propagators(const nv_rhs* rhs, double t0, double T, int32_t S,
                                          const nv_samples* samples, const nv_steps* steps,
                                          nv_maps** maps, void* stream) {
  if (!maps) return nv_fail(NV_EINVAL, "maps out-pointer is NULL");
  nv_maps P;
  nv_status e = plan(rhs, t0, T, S, samples, steps, &P);
  if (e != NV_OK) return e;
  nv_maps* M = *maps;
  if (M) {
    if (M->bytes != P.bytes || M->map != P.map || M->prec != P.prec || M->dim != P.dim ||
        M->S != P.S || M->coef_per_slice != P.coef_per_slice || M->aux_elems != P.aux_elems)
      return nv_fail(NV_EINVAL, "existing maps have different sizes; destroy them first");
    // keep storage and scratch, take the new problem description
    P.data = M->data; P.ws = M->ws; P.ws_bytes = M->ws_bytes; P.status = M->status;
    P.oob = M->oob; P.bar = M->bar; P.xbuf = M->xbuf; P.coef = M->coef; P.aux = M->aux;
    P.scan_ws = M->scan_ws; P.scan_ws_bytes = M->scan_ws_bytes; P.device = M->device;
    *M = P;
  } else {
    M = new (std::nothrow) nv_maps(P);
    if (!M) return nv_fail(NV_ENOMEM, "host allocation of the maps object");
    e = alloc_maps(M, static_cast<cudaStream_t>(stream));
    if (e != NV_OK) { free_maps(M, static_cast<cudaStream_t>(stream)); return e; }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (M->map == NV_MAP_AFFINE)
    e = launch_affine_build(M, s);
  else
    e = launch_table_build(M, s, g_tune.table_block > 0 ? g_tune.table_block : 64);
  if (e != NV_OK) {
    if (!*maps) free_maps(M, s);
    return e;
  }
  *maps = M;
  return NV_OK;
}

extern "C" nv_status nv_compose(const nv_maps* maps, const double* y0_dev, double* yT_dev,
                                double* lambdas_dev, void* stream) {
  if (!maps || !maps->data) return nv_fail(NV_EBADMAP, "maps are NULL or destroyed");
  if (!y0_dev || !yT_dev) return nv_fail(NV_EINVAL, "y0 and yT must not be NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  nv_status e = nv_cuda_check(cudaMemsetAsync(maps->ws, 0, 16, s), "status reset");
  if (e != NV_OK) return e;
  if (maps->map != NV_MAP_AFFINE) return launch_table_compose(maps, y0_dev, yT_dev, lambdas_dev, s);
  if (maps->prec == NV_TF32_REFINE)
    return launch_scan_refine(const_cast<nv_maps*>(maps), y0_dev, yT_dev, lambdas_dev, s);
  if (maps->prec == NV_BF16_REFINE || maps->prec == NV_FP32_REFINE)
    return launch_chain_refine(const_cast<nv_maps*>(maps), y0_dev, yT_dev, lambdas_dev, s);
  return launch_affine_chain(maps, y0_dev, yT_dev, lambdas_dev, s, g_tune.chain_rows_per_cta);
}

extern "C" nv_status nv_maps_destroy(nv_maps* maps) {
  if (!maps) return NV_OK;
  cudaError_t ce = cudaDeviceSynchronize();
  free_maps(maps, 0);
  return nv_cuda_check(ce, "synchronise before destroy");
}

extern "C" nv_status nv_solve(const nv_rhs* rhs, double t0, double T, int32_t S,
                              const nv_samples* samples, const nv_steps* steps,
                              const double* y0_dev, double* yT_dev, void* stream) {
  nv_maps* M = nullptr;
  nv_status e = nv_build_propagators(rhs, t0, T, S, samples, steps, &M, stream);
  if (e != NV_OK) return e;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  e = nv_compose(M, y0_dev, yT_dev, nullptr, stream);
  int st = NV_OK;
  nv_status e2 = NV_OK;
  if (e == NV_OK)
    e2 = nv_cuda_check(cudaMemcpyAsync(&st, M->status, sizeof(int), cudaMemcpyDeviceToHost, s), "status read");
  nv_status e3 = nv_cuda_check(cudaStreamSynchronize(s), "solve synchronise");
  if (e2 == NV_OK) e2 = e3;
  free_maps(M, s);
  if (e != NV_OK) return e;
  if (e2 != NV_OK) return e2;
  if (st != NV_OK) return nv_fail((nv_status)st, "device recorded status %d during solve", st);
  return NV_OK;
}

extern "C" nv_status nv_serial_fine(const nv_rhs* rhs, double t0, double T, int32_t S,
                                    const nv_steps* steps, const double* y0_dev, double* yT_dev,
                                    void* stream) {
  if (!steps || !y0_dev || !yT_dev) return nv_fail(NV_EINVAL, "NULL argument");
  nv_maps P;
  memset(&P, 0, sizeof(P));
  nv_status e = check_rhs(rhs, P.params, &P.nparams);
  if (e != NV_OK) return e;
  if (S < 1) return nv_fail(NV_EINVAL, "S must be >= 1");
  if ((e = check_scheme(rhs->kind, steps->scheme)) != NV_OK) return e;
  e = nv_plan_steps(t0, T, S, steps->dt, steps->steps_per_slice, &P.m, &P.h);
  if (e != NV_OK) return e;
  P.rhs_kind = rhs->kind;
  P.dim = rhs->dim;
  P.t0 = t0;
  P.T = T;
  P.S = S;
  P.H = (T - t0) / S;
  P.scheme = steps->scheme;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (rhs->kind == NV_RHS_HEAT1D || rhs->kind == NV_RHS_HEAT1D_VARCOEF) {
    if (steps->scheme != NV_RK4) return nv_fail(NV_ENOTSUP, "heat serial solve uses RK4");
    return launch_serial_heat(&P, y0_dev, yT_dev, s);
  }
  if (rhs->kind == NV_RHS_ADVDIFF2D) {
    if (steps->scheme != NV_RK4) return nv_fail(NV_ENOTSUP, "advection-diffusion serial solve uses RK4");
    return launch_serial_advdiff(&P, y0_dev, yT_dev, s);
  }
  if (rhs->kind == NV_RHS_WAVE_CHEB) return launch_serial_wave(&P, y0_dev, yT_dev, s);
  return launch_serial_table(rhs->kind, P.params, t0, P.H, P.h, S, P.m, steps->scheme, y0_dev,
                             yT_dev, s);
}

extern "C" nv_status nv_maps_info(const nv_maps* maps, nv_maps_desc* out) {
  if (!maps || !out) return nv_fail(NV_EINVAL, "NULL argument");
  out->map = maps->map;
  out->prec = maps->prec;
  out->scheme = maps->scheme;
  out->S = maps->S;
  out->dim = maps->dim;
  out->per_dim = maps->per_dim;
  out->steps_per_slice = maps->m;
  out->h = maps->h;
  out->elems_per_slice = maps->elems_per_slice;
  out->bytes = maps->bytes;
  out->elem_bytes = maps->elem_bytes;
  out->band = maps->band;
  out->work_per_slice = maps->work_per_slice;
  memcpy(out->build_kernel, maps->build_kernel, sizeof(out->build_kernel));
  out->build_kernel[sizeof(out->build_kernel) - 1] = '\0';
  return NV_OK;
}

extern "C" nv_status nv_maps_copy_out(const nv_maps* maps, void* dst, int64_t bytes, void* stream) {
  if (!maps || !dst) return nv_fail(NV_EINVAL, "NULL argument");
  if (bytes < 0 || bytes > maps->bytes) return nv_fail(NV_EINVAL, "byte count exceeds the maps");
  return nv_cuda_check(cudaMemcpyAsync(dst, maps->data, (size_t)bytes, cudaMemcpyDefault,
                                       static_cast<cudaStream_t>(stream)),
                       "maps copy-out");
}

extern "C" nv_status nv_maps_copy_range(const nv_maps* maps, void* dst, int64_t offset, int64_t bytes,
                                        void* stream) {
  if (!maps || !dst) return nv_fail(NV_EINVAL, "NULL argument");
  if (offset < 0 || bytes < 0 || offset > maps->bytes || bytes > maps->bytes - offset)
    return nv_fail(NV_EINVAL, "range leaves the maps");
  return nv_cuda_check(cudaMemcpyAsync(dst, static_cast<const char*>(maps->data) + offset, (size_t)bytes,
                                       cudaMemcpyDefault, static_cast<cudaStream_t>(stream)),
                       "maps range copy");
}

extern "C" nv_status nv_maps_check(const nv_maps* maps, void* stream, int64_t* oob_count) {
  if (!maps) return nv_fail(NV_EINVAL, "maps is NULL");
  nv_status e = nv_cuda_check(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)), "synchronise");
  if (e != NV_OK) return e;
  struct { int status; int pad; unsigned long long oob; } h{};
  e = nv_cuda_check(cudaMemcpy(&h, maps->ws, sizeof(h), cudaMemcpyDeviceToHost), "status read");
  if (e != NV_OK) return e;
  if (oob_count) *oob_count = (int64_t)h.oob;
  if (h.status != NV_OK) {
    const char* what = h.status == NV_ETIMEOUT ? "a bounded device wait gave up"
                       : h.status == NV_EDOMAIN ? "an evaluation left the sampled range"
                       : h.status == NV_EBADMAP ? "a map value was not finite"
                                                : "device error";
    return nv_fail((nv_status)h.status, "%s", what);
  }
  return NV_OK;
}

extern "C" nv_status nv_tune_set(int32_t key, int32_t value) {
  switch (key) {
    case 0: g_tune.table_block = value; break;
    case 1: g_tune.chain_rows_per_cta = value; break;
    case 2: g_tune.affine_warps = value; break;
    case 3: g_tune.chain_cluster = value; break;
    case 4: g_tune.scan_block = value; break;
    case 5: g_tune.refine_passes = value; break;
    case 6:
      if (value < 0 || value > 5) return nv_fail(NV_EINVAL, "heat step form is 0..5");
      g_tune.heat_step_form = value;
      break;
    case 7:
      if (value < 0 || value > 4) return nv_fail(NV_EINVAL, "phantom barrier participants are 0..4");
      g_tune.test_barrier_extra = value;
      break;
    case 8:
      if (value < 0 || value > 16 || (value & (value - 1))) return nv_fail(NV_EINVAL, "split-K is 0 (auto) or 1, 2, 4, 8, 16");
      g_tune.mlp_wgrad_splits = value;
      break;
    case 9:
      if (value < 0 || value > 2) return nv_fail(NV_EINVAL, "tiled chain form is 0, 1 or 2");
      g_tune.tile_chain_form = value;
      break;
    case 10:
      if (value < 0 || value > 1) return nv_fail(NV_EINVAL, "refinement schedule is 0 or 1");
      g_tune.refine_schedule = value;
      break;
    case 12:
      if (value < 0) return nv_fail(NV_EINVAL, "withheld slice is 0 (off) or slice + 1");
      g_tune.test_withhold_defect = value;
      break;
    case 13:
      if (value < 0) return nv_fail(NV_EINVAL, "skipped step is 0 (off) or step + 1");
      g_tune.test_skip_partials = value;
      break;
    case 14:
      if (value < 0 || value > 1) return nv_fail(NV_EINVAL, "chain band use is 0 or 1");
      g_tune.chain_dense = value;
      break;
    case 15:
      if (value < 0 || value > 2) return nv_fail(NV_EINVAL, "advection-diffusion build form is 0, 1 or 2");
      g_tune.adv_build_form = value;
      break;
    case 17:
      if (value < 0 || value > 4) return nv_fail(NV_EINVAL, "float32 heat window form is 0..4");
      g_tune.heat_f32_lanes = value;
      break;
    case 18:
      if (value < 0 || value > 2) return nv_fail(NV_EINVAL, "learned iteration-0 form is 0, 1 or 2");
      g_tune.learned_first_form = value;
      break;
    case 19:
      if (value < 0 || value > 2) return nv_fail(NV_EINVAL, "learned correction form is 0, 1 or 2");
      g_tune.learned_correction_form = value;
      break;
    case 20:
      if (value < 0 || value > 1000) return nv_fail(NV_EINVAL, "float32 learned iterations are 0..1000");
      g_tune.learned_f32_iters = value;
      break;
    case 16:
      if (value != 0 && value != 8 && value != 16 && value != 32)
        return nv_fail(NV_EINVAL, "strip height is 0 (16), 8, 16 or 32");
      g_tune.adv_fp64_rows = value;
      break;
    default: return nv_fail(NV_EINVAL, "unknown tunable %d", key);
  }
  return NV_OK;
}
