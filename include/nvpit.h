/*
 * nvpit.h - Nievergelt parallel-in-time propagators on GB300 (sm_103a).
 *
 * C ABI of the library libnvpit.so.  The calls follow the paper's statement of
 * the problem (Barker, "A minimal communication approach to parallel time
 * integration", Figure "pseudocode"): given an initial value problem
 * y' = f(t, y), a sample Xi_h of the initial value space, a final time T and a
 * number of time slices S,
 *   - the computation phase builds, for every slice [T_{j-1}, T_j], a map
 *     phi^j from initial to final states (nv_build_propagators), and
 *   - the communication phase composes the maps, lambda_j = phi^j(lambda_{j-1})
 *     (nv_compose).
 *
 * Conventions shared by every call
 *   - Pointers named *_dev are CUDA device pointers on the current device;
 *     everything else is host memory.  The caller owns every buffer it passes.
 *   - Maps (nv_maps) are library-owned device memory, created by
 *     nv_build_propagators and released by nv_maps_destroy.
 *   - Every call is asynchronous on the CUDA stream given as `stream`
 *     (a cudaStream_t; NULL = legacy default stream) unless it says otherwise.
 *   - No C++ exception and no exit() crosses this ABI.  Every call returns an
 *     nv_status; nv_last_error() gives the message of the calling thread's
 *     last failure.  CUDA launch/runtime errors map to NV_ECUDA.
 *   - Errors found on the device (a bounded wait that gave up, an evaluation
 *     outside Xi under NV_OOB_ERROR) are recorded in a device status word of the
 *     maps object and returned by nv_maps_check after it synchronises.
 *   - Time slices: T_j = t0 + j (T - t0)/S (Figure "pseudocode", Initialize).
 *     Fine steps per slice: m = steps_per_slice if > 0, else ceil(H/dt) with
 *     H = (T - t0)/S (a guard of 1e-9 keeps integer ratios exact), step size
 *     h = H/m, step i of slice j starts at T_{j-1} + i h.
 */
#ifndef NVPIT_H
#define NVPIT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NVPIT_VERSION 1

typedef enum {
  NV_OK = 0,
  NV_EINVAL = 1,    /* an argument is invalid; nothing was launched        */
  NV_ENOMEM = 2,    /* a device allocation failed                           */
  NV_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed          */
  NV_EDOMAIN = 4,   /* an evaluation left Xi under NV_OOB_ERROR             */
  NV_EBADMAP = 5,   /* maps missing, of the wrong kind, or holding NaN/Inf  */
  NV_ETIMEOUT = 6,  /* a bounded device-side wait gave up                   */
  NV_ENOTSUP = 7    /* valid request this build does not implement          */
} nv_status;

/* Right-hand sides f(t, y) compiled into the library.  `dim` must match. */
typedef enum {
  NV_RHS_LINEAR_SCALAR = 0,   /* y' = p0 y;                         dim 1, params {p0}            */
  NV_RHS_SQUARE = 1,          /* y' = y^2 (Section 3, eq. scalarmodel); dim 1                   */
  NV_RHS_COS_CUBIC = 2,       /* y' = cos(t) y - y^3;               dim 1                         */
  NV_RHS_HEAT1D = 3,          /* u_t = k u_xx + a sin(pi x) cos t, Dirichlet 0, central
                                 differences, x_i = i/(n+1);        dim n, params {k, a} (1, 1)  */
  NV_RHS_VDP = 4,             /* x' = y, y' = mu (1 - x^2) y - x;   dim 2, params {mu}            */
  NV_RHS_CHAIN3 = 5,          /* wall-m1-m2-m3-wall, tension k d + k3 d^3, damping c;
                                 state (x1,x2,x3,v1,v2,v3);         dim 6, params {k, k3, c}      */
  NV_RHS_ADVDIFF2D = 6,       /* u_t = nu lap5(u) - (ax D-x u + ay D-y u), periodic nx*nx grid,
                                 spacing 1/nx, index iy*nx+ix;      dim nx*nx, params {nu, ax, ay} */
  NV_RHS_HEAT1D_VARCOEF = 7,  /* Section 5, eq. heatequation: u_t = (1 + sin(t)/4) u_xx + b(t,x),
                                 b making cos(t) sin(pi x) exact;   dim n                         */
  NV_RHS_WAVE_CHEB = 8        /* Section 5, eq. waveequation: u_tt = u_xx on [-1,1], u(+-1) = 0,
                                 Chebyshev spectral D2 on x_i = cos(i pi/M), interior d = M-1
                                 points; state (u^n, u^{n-1}) (the doubled initial-value space
                                 of Section 5);                    dim 2(M-1) <= 160, params {M}
                                 (optional: M = dim/2 + 1); scheme NV_LEAPFROG only            */
} nv_rhs_kind;

typedef struct {
  int32_t kind;            /* nv_rhs_kind                                   */
  int32_t dim;             /* state dimension d                             */
  const double* params;    /* host array of nparams values (may be NULL)    */
  int32_t nparams;
} nv_rhs;

/* NV_LEAPFROG: u^{n+1} = 2u^n - u^{n-1} + h^2 D2 u^n on the two-level state of
   NV_RHS_WAVE_CHEB (Section 5: "explicit second-order leapfrog"); one step
   advances (u^n, u^{n-1}) to (u^{n+1}, u^n).  The state at a slice boundary
   T_j is (u(T_j), u(T_j - h)) with the planned h = H/m.                      */
typedef enum { NV_EULER = 0, NV_RK4 = 1, NV_LEAPFROG = 2 } nv_scheme;

typedef enum {
  NV_MAP_PL1D = 0,         /* d = 1: piecewise-linear table on M equispaced nodes      */
  NV_MAP_BILINEAR2D = 1,   /* d = 2: bilinear table on a P x P equispaced grid         */
  NV_MAP_AFFINE = 2        /* linear systems: y_end = A_j y0 + b_j from d+1 basis solves */
} nv_map_kind;

typedef enum {
  NV_FP64 = 0,             /* integrate and store in float64                           */
  NV_FP32 = 1,             /* integrate and store in float32                           */
  NV_TF32_REFINE = 2,      /* affine only: maps integrated in float32 and stored rounded
                              to TF32 (float32 containers, 11 significant bits; the
                              forcing column b_j keeps float32), composition on tcgen05
                              tensor cores in TF32 with float32 accumulation, then
                              float64 residual-correction passes (three by default).
                              Heat equations, d <= 256, d % 4 == 0                        */
  NV_BF16_REFINE = 3,      /* affine only: maps integrated in float32 and stored rounded
                              to bfloat16 (half the bytes of float32), composed by the
                              HBM-bound chain with float32 accumulation, then float64
                              residual-correction passes whose chains reuse the
                              bfloat16 maps.  Advection-diffusion, d > 512, d % 8 == 0.
                              The maps' rounding compounds along the chain in the
                              slowly decaying modes, so a pass contracts the error by
                              roughly S / 1500 on the 64 x 64 problem: the default is
                              two passes up to S = 32 and one more per doubling of S
                              (six at S = 512)                                          */
  NV_FP32_REFINE = 4       /* affine only: float32 maps and float32 chain as NV_FP32,
                              then float64 residual-correction passes (default one;
                              two for the undamped wave equation).  Heat equations,
                              wave equation, advection-diffusion with d > 512          */
} nv_precision;

typedef enum { NV_OOB_EXTRAPOLATE = 0, NV_OOB_ERROR = 1 } nv_oob_policy;

/* Xi_h (Section 3: "sample points inside Xi to get a discrete set Xi_h").
 * PL1D: nodes lo[0] + k (hi[0]-lo[0])/(per_dim-1), k = 0..per_dim-1.
 * BILINEAR2D: grid (lo[0] + p dx, lo[1] + q dy), p, q = 0..per_dim-1.
 * AFFINE: the d+1 basis {0 (with forcing), e_1..e_d (homogeneous)} of eq.
 *   linearreconstruct; per_dim, lo, hi are ignored.
 * Evaluation outside [lo, hi] extends the edge segment/cell (EXTRAPOLATE, and
 * is counted) or additionally records NV_EDOMAIN (ERROR). */
typedef struct {
  int32_t map;             /* nv_map_kind     */
  int32_t per_dim;
  double lo[2];
  double hi[2];
  int32_t oob_policy;      /* nv_oob_policy   */
} nv_samples;

typedef struct {
  int32_t scheme;          /* nv_scheme                              */
  double dt;               /* target fine step (used when steps == 0) */
  int64_t steps_per_slice; /* m; 0 => ceil(H/dt)                      */
  int32_t prec;            /* nv_precision                           */
} nv_steps;

typedef struct nv_maps nv_maps;   /* opaque, library-owned */

/* Layout description of built maps (nv_maps_info).
 *   PL1D        data[j*M + k]                        (value from node k, slice j)
 *   BILINEAR2D  data[((j*P + q)*P + p)*2 + c]        (component c from node (p, q))
 *   AFFINE      data[j*d*(d+1) + col*d + i]          column-major d x (d+1) per slice:
 *               col 0 = b_j, col c >= 1 = A_j e_c  (eq. linearreconstruct)
 * Element type: double for NV_FP64, float otherwise. */
typedef struct {
  int32_t map, prec, scheme, S, dim, per_dim;
  int64_t steps_per_slice;
  double h;                /* fine step size                 */
  int64_t elems_per_slice;
  int64_t bytes;           /* total bytes of map data        */
  int32_t elem_bytes;      /* 8 (double) or 4 (float)        */
  int32_t band;            /* AFFINE: 0 dense; > 0: A_j[r][c] == 0 whenever |r - c| >= band */
  int64_t work_per_slice;  /* point-steps the last build integrated per slice: rows times fine
                              steps, summed over the slice's columns (a windowed build counts
                              the rows it integrates); 0 where not recorded */
  char build_kernel[64];   /* the last build's main kernel, "" where not recorded */
} nv_maps_desc;

/* Computation phase (Figure "pseudocode"; eqs. lineardiscrete and
 * linearreconstruct for NV_MAP_AFFINE).  For every slice j and every sample
 * xi_k, integrates the fine scheme over [T_{j-1}, T_j] from xi_k and stores
 * the final states as the slice map.
 * If *maps is non-NULL it must come from an earlier call with the same sizes,
 * map kind and precision; its storage is reused and nothing is allocated.
 * Otherwise a new object is allocated and returned in *maps.
 * All work is ordered on `stream`.  The heat equations' forcing columns run
 * on a library-owned second stream of the device, forked from and joined back
 * to `stream` by events; that stream is created on first use and kept, so it
 * is not valid after a cudaDeviceReset of the device.
 * Returns NV_EINVAL for inconsistent arguments (nothing launched), NV_ENOMEM,
 * NV_ENOTSUP for map/rhs combinations not built, NV_ECUDA on launch failure. */
nv_status nv_build_propagators(const nv_rhs* rhs, double t0, double T, int32_t S,
                               const nv_samples* samples, const nv_steps* steps,
                               nv_maps** maps, void* stream);

/* Communication phase (Figure "pseudocode"): lambda_0 = y0,
 * lambda_j = phi^j(lambda_{j-1}), j = 1..S, evaluated in float64.
 *   y0_dev       d doubles (input)
 *   yT_dev       d doubles (output, lambda_S)
 *   lambdas_dev  (S+1) x d doubles (output, may be NULL): every boundary state.
 * Tables: one sequential chain of S lookups.  AFFINE NV_FP64 / NV_FP32: a
 * chain of S matrix-vector products on all SMs (cooperative launch, bounded
 * grid barrier; NV_ETIMEOUT is recorded if a barrier wait gives up).
 * AFFINE NV_TF32_REFINE: blocked scan of the affine maps on tcgen05 tensor
 * cores, then float64 residual-correction passes with float64 fine solves
 * from the approximate boundary states.  AFFINE NV_BF16_REFINE: the chain over
 * the bfloat16 maps, then float64 correction passes (fine solves from the
 * approximate boundary states, the correction chained over the same maps);
 * AFFINE NV_FP32_REFINE: the same over float32 maps.
 * Buffers must not overlap. */
nv_status nv_compose(const nv_maps* maps, const double* y0_dev, double* yT_dev,
                     double* lambdas_dev, void* stream);

/* Build followed by compose (Figure "pseudocode" end to end).  Allocates and
 * frees its own maps; y0_dev / yT_dev as in nv_compose.  Synchronises the
 * stream before freeing, so it returns after the result is written. */
nv_status nv_solve(const nv_rhs* rhs, double t0, double T, int32_t S,
                   const nv_samples* samples, const nv_steps* steps,
                   const double* y0_dev, double* yT_dev, void* stream);

/* Serial fine solve over all slices from y0 with the same step size and step
 * times as the slices: the "plain" reference the method is measured against
 * (Section 4, Theorem).  One thread per component group; latency-bound. */
nv_status nv_serial_fine(const nv_rhs* rhs, double t0, double T, int32_t S,
                         const nv_steps* steps, const double* y0_dev, double* yT_dev,
                         void* stream);

/* Releases maps (NULL is accepted).  Synchronises the device first. */
nv_status nv_maps_destroy(nv_maps* maps);

/* Describes built maps (host-side, no synchronisation). */
nv_status nv_maps_info(const nv_maps* maps, nv_maps_desc* out);

/* Copies the map data (nv_maps_desc.bytes bytes, layout above) to dst, a host
 * or device pointer, asynchronously on `stream`. */
nv_status nv_maps_copy_out(const nv_maps* maps, void* dst, int64_t bytes, void* stream);

/* Copies `bytes` bytes of map data starting `offset` bytes into the maps to
 * dst (host or device), asynchronously on `stream`; NV_EINVAL if the range
 * leaves the maps. */
nv_status nv_maps_copy_range(const nv_maps* maps, void* dst, int64_t offset, int64_t bytes,
                             void* stream);

/* Synchronises `stream`, then returns the device status recorded by this
 * maps object's kernels (NV_OK, NV_EDOMAIN, NV_ETIMEOUT) and, if oob_count is
 * non-NULL, the number of evaluations outside Xi since the last compose. */
nv_status nv_maps_check(const nv_maps* maps, void* stream, int64_t* oob_count);

/* Message of the calling thread's last failure ("" if none).  Valid until the
 * thread's next failing call. */
const char* nv_last_error(void);

/* NVPIT_VERSION of the built library. */
int32_t nv_version(void);

/* ---------------------------------------------------------------------------
 * Batched independent instances (the "great deal more parallelism" of the
 * Conclusion: every (instance, slice, sample) trajectory is independent).
 * B instances of one right-hand side family, each with its own parameters,
 * interval [t0_i, T_i] and slice count S_i, share the sample grid and the
 * step rule.  The computation phase of all instances runs in ONE persistent
 * launch: CTAs pull (instance, slice) work items from a device queue ordered
 * by decreasing cost (longest-processing-time first).  Table maps only
 * (NV_MAP_PL1D for d = 1, NV_MAP_BILINEAR2D for d = 2); composition in float64.
 * Tables of instance i start at element offset sum_{i'<i} S_i' * E, E the
 * elements per slice (M or 2 P^2), and follow the nv_maps_desc layout.
 * ------------------------------------------------------------------------- */
typedef struct nv_batch nv_batch;   /* opaque, library-owned */

/* Builds the tables of every instance.  params: B x nparams host array (row
 * i = parameters of instance i); t0, T, S: host arrays of B values.  Allocates
 * the batch object (tables, instance descriptors, work queue) and launches
 * the persistent build on `stream`.  NV_EINVAL for inconsistent arguments. */
nv_status nv_build_batch(int32_t rhs_kind, int32_t dim, int32_t B, const double* params,
                         int32_t nparams, const double* t0, const double* T, const int32_t* S,
                         const nv_samples* samples, const nv_steps* steps, nv_batch** out,
                         void* stream);

/* Rebuilds the tables of an existing batch (same instances) on `stream`. */
nv_status nv_batch_rebuild(nv_batch* batch, void* stream);

/* Composes every instance: yT[i] = phi^{S_i}_i( ... phi^1_i(y0[i])), float64.
 * y0_dev, yT_dev: B x dim doubles (device). */
nv_status nv_batch_compose(const nv_batch* batch, const double* y0_dev, double* yT_dev,
                           void* stream);

/* Build + compose replayed from a CUDA graph captured on the first call with
 * these buffers (re-captured when the buffers change).  Launches on `stream`. */
nv_status nv_batch_run(nv_batch* batch, const double* y0_dev, double* yT_dev, void* stream);

/* Times the persistent build for each candidate CTA shape (threads per CTA
 * 128/256/512/1024 at full occupancy) on this batch with CUDA events, keeps
 * the fastest for this batch and as the default for the device, and returns
 * it in best_threads (may be NULL).  Synchronises `stream`. */
nv_status nv_batch_autotune(nv_batch* batch, void* stream, int32_t* best_threads);

/* Sizes: total slices (work items), trajectory-steps of one build, bytes of
 * tables, and the CTA size in use. */
nv_status nv_batch_info(const nv_batch* batch, int64_t* total_slices, int64_t* traj_steps,
                        int64_t* table_bytes, int32_t* threads);

/* Copies the tables (table_bytes bytes) to a host or device pointer. */
nv_status nv_batch_copy_out(const nv_batch* batch, void* dst, int64_t bytes, void* stream);

/* Synchronises, returns the recorded device status and the out-of-range count. */
nv_status nv_batch_check(const nv_batch* batch, void* stream, int64_t* oob_count);

/* Releases the batch (NULL accepted); synchronises the device first. */
nv_status nv_batch_destroy(nv_batch* batch);

/* ---------------------------------------------------------------------------
 * Learned propagator for high-dimensional nonlinear problems (Section 4: a
 * uniform table with l points per axis costs l^r solves).  The method's own
 * computation phase produces training pairs; a slice-conditioned MLP
 * (x = (y0/sx, T_{j-1}/T) -> 256 -> 256 -> 256 -> (y_end - y0)/sd, GELU)
 * trained on the GPU with bf16 tensor-core forward/backward stands in for the
 * table; float64 fine integration checks it and replaces it on slices whose
 * validation error is too large.  Built for the 3-mass chain (NV_RHS_CHAIN3).
 * ------------------------------------------------------------------------- */
typedef struct nv_mlp nv_mlp;   /* opaque, library-owned */

/* Training pairs: for slice j and sample k, xi = lo + (hi-lo) u with u the
 * SplitMix64 outputs (j*M + k)*6 + c (c = 0..5) of `seed` (top 53 bits), and
 * g^j(xi) from the fine scheme.  y0_dev, yend_dev: S x M x 6 values, float for
 * NV_FP32 (Kahan-compensated updates), double for NV_FP64. */
nv_status nv_build_pairs(const nv_rhs* rhs, double t0, double T, int32_t S, const nv_steps* steps,
                         int64_t M, uint64_t seed, double lo, double hi, void* y0_dev, void* yend_dev,
                         void* stream);

/* Fine integration of `count` states (y_dev, count x 6 doubles, in place)
 * over slices j0 .. j0+nslices-1, one thread per state: in float64 for
 * steps->prec = NV_FP64 (the reference and the fallback), in float32 with
 * Kahan-compensated updates for NV_FP32 (the plain float32 method); other
 * precisions return NV_EINVAL. */
nv_status nv_propagate(const nv_rhs* rhs, double t0, double T, int32_t S, const nv_steps* steps,
                       int32_t j0, int32_t nslices, int64_t count, double* y_dev, void* stream);

/* Creates the network with weights drawn from SplitMix64(seed), uniform in
 * +-1/sqrt(fan_in).  Synchronous. */
nv_status nv_mlp_create(uint64_t seed, nv_mlp** out);
nv_status nv_mlp_destroy(nv_mlp* mlp);

/* Input scale sx and output scale sd (6 positive doubles each, host). */
nv_status nv_mlp_set_scales(nv_mlp* mlp, const double* sx, const double* sd);

/* Parameter vector (float32, layout in mlp.cu): count in *count; copied to
 * host if host != NULL.  nv_mlp_set_params writes it back.  Synchronous. */
nv_status nv_mlp_params(nv_mlp* mlp, float* host, int64_t* count);
nv_status nv_mlp_set_params(nv_mlp* mlp, const float* host);

/* Gradients of the half mean-squared loss on one batch: X_dev B x 8 floats
 * (features, column 7 zero), Y_dev B x 8 floats (targets, columns 6, 7 zero),
 * grads_dev receives the parameter-vector gradient.  B multiple of 128.
 * Synchronous. */
nv_status nv_mlp_grads(nv_mlp* mlp, const float* X_dev, const float* Y_dev, int32_t B, float* grads_dev,
                       double* loss, void* stream);

/* `steps` Adam steps (lr) on batches of B pairs drawn from the S x M float32
 * pairs (S*M a power of two), replayed from a captured CUDA graph.  Returns
 * the last batch's loss.  Synchronous. */
nv_status nv_mlp_train(nv_mlp* mlp, const float* y0_dev, const float* yend_dev, int32_t S, int64_t M,
                       int64_t steps, int32_t B, double lr, void* stream, double* last_loss);

/* Per-slice relative error ||y0 + sd*MLP - y_end|| / ||y_end|| over Mv float64
 * validation pairs per slice (S x Mv x 6 doubles each); err_host: S doubles.
 * Mv multiple of 128.  Synchronous. */
nv_status nv_mlp_validate(nv_mlp* mlp, const double* y0_dev, const double* yend_dev, int32_t S,
                          int64_t Mv, double* err_host, void* stream);

/* Composition with the learned map for `count` initial states (multiple of
 * 128; y0_dev, yT_dev: count x 6 doubles): slice j advances
 * lambda += sd*MLP(lambda/sx, j/S), or, where fallback[j] != 0 (host array of
 * S flags, may be NULL), integrates the slice in float64. */
nv_status nv_mlp_compose(nv_mlp* mlp, const nv_rhs* rhs, double t0, double T, int32_t S,
                         const nv_steps* steps, const int32_t* fallback, int64_t count,
                         const double* y0_dev, double* yT_dev, void* stream);

/* The learned map as the coarse propagator of a float64 residual correction
 * (the combination with parareal the Conclusion proposes), for nonlinear
 * problems.  Iteration 0 is the learned composition
 * lambda_{j+1} = G_j(lambda_j), G_j(y) = y + sd*MLP(y/sx, j/S): by default,
 * while count <= 32 x (SMs / 2), every state's chain in one launch with
 * float32 activations (the network's bf16 weights), else, or with
 * nv_tune_set key 18 = 1, slice by slice through nv_mlp_compose's path
 * (bf16 activations between the layers), then bit for bit its states.  Iteration k >= 1:
 *   d_j = F_j(lambda_j) - lambda_{j+1}      float64 fine solve per slice, for
 *                                           every slice and state at once
 *   e_0 = 0, e_{j+1} = J_j e_j + d_j        J_j the network's Jacobian (6 x 6)
 *                                           at slice j's state of the learned
 *                                           composition, computed once for all
 *                                           iterations (nv_tune_set key 19 has
 *                                           the other forms)
 *   lambda_{j+1} <- lambda_{j+1} + e_{j+1}  written by the chain as it goes
 * i.e. a simplified Newton step on the multiple-shooting equations
 * lambda_{j+1} = F_j(lambda_j), with the learned Jacobian in place of F_j's.
 * After k iterations the first k boundary states equal the float64 fine
 * solution's; the iterates converge to the float64 fine integration of every
 * state (the correction is relative, so the bf16 rounding of the network does
 * not set a floor).
 *   count        states, a positive multiple of 128
 *   y0_dev       count x 6 doubles (input); yT_dev count x 6 (output)
 *   lambdas_dev  (S+1) x count x 6 doubles (output, may be NULL): every
 *                boundary state of the last iterate
 * steps->prec must be NV_FP64.  The network owns the boundary states, defects
 * and Jacobians ((2 S + 1) count 6 doubles, S count 36 floats, and the
 * scratch of one chunk of at most 65536 (slice, state) items, about 0.7 GB):
 * the first call for a (count, S)
 * synchronises `stream` and allocates them, and the first call for a schedule
 * (count, S, iters, steps, rhs parameters) captures the whole schedule into a
 * CUDA graph, later calls replay it (at small counts the learned composition's
 * kernels are launch-bound when issued one by one); make those first calls
 * outside any stream capture.  Calls on one network must not overlap.  NV_EINVAL for a bad
 * count, iters < 0 or another precision; NV_ENOTSUP for a right-hand side other
 * than the 3-mass chain. */
nv_status nv_mlp_parareal(nv_mlp* mlp, const nv_rhs* rhs, double t0, double T, int32_t S,
                          const nv_steps* steps, int32_t iters, int64_t count, const double* y0_dev,
                          double* yT_dev, double* lambdas_dev, void* stream);

/* Largest state dimension nv_compose_affine_noalloc accepts. */
#define NVPIT_NOALLOC_MAX_DIM 4096

/* Affine composition that allocates nothing (the paper has no counterpart:
 * this serves callers, not the method).  For callers that cannot allocate
 * device memory when they compose - an application whose memory pool already
 * owns the GPU, a real-time loop that must not pay for or synchronise on
 * cudaMalloc/cudaFree, a plug-in that may only use the buffers it is lent.
 * Computes the same chain as nv_compose for NV_MAP_AFFINE maps, float64:
 *   maps_dev     S blocks of dim x (dim+1) values in the AFFINE layout of
 *                nv_maps_desc (column 0 = b_j), double for NV_FP64, float for
 *                NV_FP32 (input, caller-owned device memory)
 *   y0_dev       dim doubles (input); yT_dev dim doubles (output, lambda_S)
 *   lambdas_dev  (S+1) x dim doubles (output, may be NULL)
 *   status_dev   one int32 (output, may be NULL): the device status of this
 *                call (NV_OK or NV_ETIMEOUT), written on `stream`
 * Scratch: a fixed static __device__ array of about 64 KiB per GPU that loads
 * the library, held until the process exits; it serves 1 <= dim <=
 * NVPIT_NOALLOC_MAX_DIM, larger dim returns NV_EINVAL.  The first call on a
 * device looks up that array's device address with cudaGetSymbolAddress (make
 * that first call before any stream capture on that device) and keeps it for
 * the process, so the entry point must not be used on a device after
 * cudaDeviceReset.  All calls share
 * the array: calls that overlap on the GPU (other streams, other threads)
 * race and give wrong results; order them on one stream or synchronise.
 * Each call runs the chain with 16 rows per CTA (nv_tune_set key 1 does not
 * apply): a cooperative grid of ceil(dim/16) CTAs, NV_ENOTSUP if the device
 * cannot hold them all at once (a GB300 holds them for every dim up to the
 * limit); NV_ECUDA if a CUDA call fails.
 * Calls no cudaMalloc, cudaFree or allocating library routine. */
nv_status nv_compose_affine_noalloc(const void* maps_dev, int32_t prec, int32_t dim, int32_t S,
                                    const double* y0_dev, double* yT_dev, double* lambdas_dev,
                                    int32_t* status_dev, void* stream);

/* Launch-shape tunables, process-wide (host only; set by the autotuner).
 *   key 0: threads per CTA of the table build (32..256, default 64)
 *   key 1: rows of each chain product owned by one CTA (default 16)
 *   key 2: warps per CTA of the affine build (default 8)
 *   key 3: CTAs per cluster of the d <= 512 chain (default 0 = largest that
 *          fits, up to 16; a negative value selects the grid-wide chain)
 *   key 4: slices per block of the NV_TF32_REFINE scan (default round(sqrt(S)))
 *   key 5: float64 correction passes of NV_TF32_REFINE / NV_BF16_REFINE /
 *          NV_FP32_REFINE (default 0 = three / 2 + ceil(log2(S/32)) for S > 32, else
 *          two / one, two for the wave equation; a negative value
 *          returns the unrefined reduced-precision states)
 *   key 6: form of the RK4 step for the homogeneous heat columns: 0 auto (the
 *          windowed nine-point stencil where a built window fits, else the
 *          full-width nine-point stencil where every lane holds >= 4 whole
 *          rows, else Horner stages), 1 Horner stages, 2 full-width nine-point
 *          stencil where it applies, 3 one window per column, 4 two windows
 *          per column (a narrow one for the first steps, a wide one for the
 *          rest), 5 three windows.  Forms 3, 4 and 5 make the build return
 *          NV_ENOTSUP when no built window of that kind holds the 8m+1 rows
 *          within n.  All are
 *          the classical RK4 step of y' = Ly exactly; Horner and nine-point
 *          differ in rounding only, and a windowed stencil integrates each
 *          column only over the rows its steps can reach (they are exactly
 *          zero elsewhere), with the same nonzero entries as the full-width
 *          stencil bit for bit.
 *   key 7: test hook, 0..4 (default 0): participants that never arrive, added to the
 *          grid barrier of the cooperative row chain (selected by key 3 < 0).  Every
 *          CTA then gives up at its first bounded wait (~0.4 s), records NV_ETIMEOUT
 *          in the maps' status word (read by nv_maps_check) and returns; the
 *          context stays usable.  The paper has no counterpart.
 *   key 8: split-K of the learned propagator's weight-gradient GEMMs (K = the
 *          batch): 0 auto, or 1, 2, 4, 8, 16
 *   key 9: kernel of the d > 512 chain: 0 auto (1 for float32 maps, 2 for
 *          float64 and bfloat16 maps), 1 loads into registers in batches with
 *          a grid barrier per step, 2 a shared-memory ring fed by bulk
 *          asynchronous copies with a barrier-free tagged exchange of the
 *          partial sums.  Same arithmetic in the same order: the results are
 *          identical.
 *   key 10: schedule of the float64 correction passes of NV_FP32_REFINE on the
 *          heat equations: 0 auto (pipelined: the approximate chain, every
 *          pass's defects and correction chain run concurrently in one
 *          cooperative launch, each a few slices behind the one it corrects,
 *          where 64 <= d <= 256, d % 16 == 0 and at most 3 passes), 1 the
 *          passes one after another.  Same arithmetic: identical results.
 *   key 12: test hook, >= 0 (default 0): in the pipelined refinement the
 *          defect of slice value - 1 of the first pass is computed but its
 *          flag is never set, so the correction chain's bounded wait for it
 *          runs out (~1 s): NV_ETIMEOUT is recorded in the maps' status word
 *          (read by nv_maps_check), every role of the launch gives up, and
 *          the context stays usable.  The paper has no counterpart.
 *   key 13: test hook, >= 0 (default 0): the d > 512 ring chain's first CTA
 *          never stores its partial sums of step value - 1, so the CTAs that
 *          need them give up after their bounded wait (~1 s) and record
 *          NV_ETIMEOUT; the others run out their loops; the context stays
 *          usable.  The paper has no counterpart.
 *   key 14: 0 (default) or 1: with 1 the d <= 256 cluster chains read every
 *          column of banded maps (those of the heat equations, zero off
 *          |r - c| <= 4m) instead of the band around each CTA's rows; the
 *          results are the same bit for bit.
 *   key 15: 0 (default), 1 or 2: with 1 the float64 / float32 / bfloat16
 *          advection-diffusion build integrates every column on the whole grid
 *          for all m steps; by default the first min(m, 3) steps run on
 *          32 x 32 windows around each column's unit point (the points those
 *          steps cannot reach are exactly zero), and the float64 build then
 *          runs the next steps on the whole width but only the rows they can
 *          reach (a ladder of 48-row windows for steps 4 and 5 at 16-row
 *          strips; 40, 48, 56 rows for steps 4-6 at 8-row strips); 2 keeps
 *          the 32 x 32 windows without the ladder.  The same maps bit for bit.
 *   key 16: 0 (default, = 16), 8, 16 or 32: rows of the grid each thread holds
 *          in the float64 advection-diffusion window build (16: 256-thread
 *          CTAs, 8: 512-thread CTAs, 32: 128-thread CTAs); the same maps bit
 *          for bit.
 *   key 17: 0..4: form of the float32 heat build's three windows (22, 44,
 *          88 rows): 1 one lane of 22 rows per column (then 2 and 4), 2 two
 *          lanes of 11 rows (then 4 and 8, the float64 shape), 3 and 4 the
 *          same shapes with column c of two slices in the two halves of each
 *          register, every stencil operation one packed f32x2 instruction for
 *          both (S > 1); 0 (default) = 4.  The same maps bit for bit.
 *   key 18: 0 (default), 1 or 2: iteration 0 of nv_mlp_parareal: 0 the
 *          fused one-launch sweep while count <= 32 x (SMs / 2), else the
 *          per-slice path of nv_mlp_compose; 1 always that per-slice path;
 *          2 always the sweep.  The two differ in the rounding of the
 *          network's activations (bf16 between layers on the per-slice path,
 *          float32 in the sweep); the corrected iterates converge to the same
 *          float64 fine solution either way.
 *   key 19: 0 (default), 1 or 2: the corrections of nv_mlp_parareal.  0: the
 *          network's Jacobians at the learned composition (iteration 0's
 *          states), for every slice and state at once (reverse mode through
 *          tcgen05 GEMMs, bf16 adjoints), computed once and used by every
 *          iteration's 6 x 6 correction chain; 2: the same Jacobians
 *          recomputed at each previous iterate; 1: the tangent of the
 *          network at the iterate as the chain corrects it, every state's
 *          chain in one launch across all slices (float32).  All converge to
 *          the same float64 fine solution.
 *   key 20: 0..1000 (default 0): the first `value` iterations of
 *          nv_mlp_parareal compute their defects with float32 fine solves
 *          (Kahan-compensated updates from the float32-rounded states), the
 *          rest with float64 ones.  The float32 iterations converge towards
 *          the float32 fine solution, about 1e-6 from the float64 one, at a
 *          fraction of the float64 solves' cost; the float64 iterations then
 *          continue to the float64 fine solution.  The leading boundary states
 *          are exact only for the float64 iterations.
 * A value of 0 restores the default (and <= 0 for keys 0-2).  Returns NV_EINVAL for an unknown key
 * or an out-of-range value of keys 6, 7, 8, 9, 10, 12, 13, 14, 15, 16, 17, 18, 19 and 20. */
nv_status nv_tune_set(int32_t key, int32_t value);

/* Measured fused multiply-add throughput of the current device's float64
 * (prec = NV_FP64) or float32 (NV_FP32) pipe, in FLOP/s (FMA = 2): the peak
 * the ALU-bound map builds are reported against.  The paper has no
 * counterpart (a measurement helper).  Launches a persistent grid of eight
 * independent FMA chains per thread on `stream`, about 20 ms per launch at the
 * nominal rates (one warm-up and three timed launches), and synchronises the
 * stream.  Writes *flops_per_s; NV_EINVAL for another precision or a NULL
 * pointer, NV_ECUDA if a launch fails.  Allocates no device memory. */
nv_status nv_alu_rate(int32_t prec, double* flops_per_s, void* stream);

/* Fine steps per slice and step size by the rule stated above (host only). */
nv_status nv_plan_steps(double t0, double T, int32_t S, double dt, int64_t steps_per_slice,
                        int64_t* m, double* h);

#ifdef __cplusplus
}
#endif
#endif /* NVPIT_H */
