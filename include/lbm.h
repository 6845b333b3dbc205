/*
 * lbm.h -- C-ABI of liblbm.so, a GB300 (sm_103a) solver for the pressure-based D2Q8
 * multiple-relaxation-time lattice Boltzmann model of incompressible porous flow of
 * Liu & He, "Multiple-relaxation-time lattice Boltzmann modeling of incompressible flows in
 * porous media" (arXiv 1311.7239), with the D2Q5 temperature equation of its Appendix B.
 *
 * Conventions (all entry points):
 *   - Every function returns LBM_OK (0) or a negative LBM_E* code; none throws or aborts.
 *     lbm_strerror() names a code; lbm_last_error() gives the message of the last failure
 *     on the calling thread.
 *   - Fields are row-major [ny][nx] (x fastest), row y = 0 at the bottom wall side; population
 *     arrays are [q][ny][nx] with q in the paper's order (i = 1..8 of Eq. 7 stored as 0..7;
 *     D2Q5 i = 0..4 of Eq. B.3).
 *   - Pointers passed in may be device memory of the context's GPU or host memory (pinned or
 *     pageable); the library detects which.  Caller memory is never freed or retained: inputs
 *     are copied in, outputs are written before the call's work on the context stream ends.
 *   - Work is enqueued on the context's CUDA stream (lbm_config.stream, or a stream the
 *     library creates when that is NULL).  Calls with host outputs, lbm_sync, lbm_residual and
 *     lbm_nusselt wait for the stream; the others return once the work is enqueued.
 *   - A context is used by one host thread at a time.
 */
#ifndef LBM_H
#define LBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_ABI_VERSION 2u

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

/* status codes */
#define LBM_OK 0
#define LBM_EINVAL (-1)    /* bad argument or configuration */
#define LBM_ENOMEM (-2)    /* device or host allocation failed */
#define LBM_ECUDA (-3)     /* a CUDA runtime call failed */
#define LBM_EUNSTABLE (-4) /* a step produced a non-finite velocity (reported at the next sync) */
#define LBM_ETIMEOUT (-5)  /* a bounded device-side wait gave up */
#define LBM_EABI (-6)      /* lbm_config.abi_version differs from LBM_ABI_VERSION */
#define LBM_ESTATE (-7)    /* call not valid in the context's current state */

/* population storage (all arithmetic is FP32; storage holds f - f_rest, see lbm_config) */
#define LBM_FP32 0u
#define LBM_FP16_DEV 1u
#define LBM_BF16_DEV 2u

/* boundary kinds of the x sides (left/right) and y sides (bottom/top) */
#define LBM_PERIODIC 0u
#define LBM_WALL 1u     /* halfway bounce-back, optionally moving (u_wall) */
#define LBM_PRESSURE 2u /* x sides only: pressure columns by non-equilibrium extrapolation */
#define LBM_NEE 3u      /* walls on the outermost nodes, treated by non-equilibrium extrapolation (the
                         * paper's scheme, Sec. 3): f_b = f_eq(p_nb, u_w) + f_nb - f_eq(p_nb, u_nb), nb
                         * the node inward along the normal; walls at distance nx - 1 / ny - 1; a
                         * temperature wall node takes g_eq(T_w or T_nb, u_w) + g_nb - g_eq(T_nb, u_nb);
                         * needs nx, ny >= 3 (lbm_adjoint: >= 4 across an extrapolated side pair) */

/* population streaming (lbm_config.streaming) */
#define LBM_STREAM_AB 0u      /* two population buffers: the step pulls from one into the other */
#define LBM_STREAM_INPLACE 1u /* one buffer, updated in place ("esoteric pull": every cell writes back into the
                               * slots it read, each slot receiving the opposite population; populations
                               * leaving through a wall are parked in one ghost row below and above and one
                               * ghost column right of the lattice).  Same arithmetic and results as
                               * LBM_STREAM_AB with half the population memory.  All sides; with LBM_NEE or
                               * LBM_PRESSURE sides each step first computes the boundary nodes' states
                               * (one small extra launch; 4 (8 or 13) (nx + ny) bytes kept), since a
                               * boundary node reads a neighbour that the step overwrites.  lbm_adjoint
                               * runs on two A-B buffers of its workspace; batches: LBM_PERIODIC and
                               * LBM_WALL sides only.  The last step of each
                               * lbm_step call records the velocity of its collisions, u(t-1) for
                               * lbm_residual (8 B per cell kept and written once per call), unless
                               * LBM_OPT_NO_RESIDUAL_RECORD is set.  Limit:
                               * 8 ((ny + 2) pitch + ny + 2) <= 2^32 elements, pitch = nx rounded up to 128
                               * (about 23000 x 23000). */
/* lbm_config.options bits */
#define LBM_OPT_NO_RESIDUAL_RECORD 1u /* in-place contexts: keep no u(t-1) record (lbm_residual returns LBM_ESTATE) */

/* wall indices of u_wall / T_wall */
#define LBM_LEFT 0
#define LBM_RIGHT 1
#define LBM_BOTTOM 2
#define LBM_TOP 3

/*
 * Problem description.  Symbols follow the paper: phi porosity, K permeability, nu the fluid
 * viscosity upsilon, J = upsilon_e / upsilon (Eq. 5), rho0 the mean density, s_e and s_q the
 * rates of Eq. 13 (1.1 and 1.2 in Sec. 3), a the external acceleration of Eq. 3.
 * The viscous rate is s_v = 1/tau_v with J nu = c_s^2 (tau_v - 1/2) (Eq. 21).
 */
typedef struct lbm_config {
  uint32_t abi_version; /* = LBM_ABI_VERSION */
  uint32_t nx, ny;      /* lattice size, 2..65535 each */
  uint32_t precision;   /* LBM_FP32 | LBM_FP16_DEV | LBM_BF16_DEV */
  uint32_t bc_x, bc_y;  /* LBM_PERIODIC | LBM_WALL | LBM_NEE (| LBM_PRESSURE for bc_x) */
  int32_t forchheimer;  /* 1: F_phi = 1.75 / sqrt(150 phi^3) (Eq. 4); 0: F_phi = 0 (Brinkman) */
  int32_t thermal;      /* 1: couple the D2Q5 temperature equation (Appendix B, Sec. 3.4) */
  double nu, J, rho0, s_e, s_q;
  double ax, ay;        /* uniform external acceleration a (Eq. 3) */
  double phi, K;        /* uniform medium, used until lbm_set_medium gives per-cell fields */
  double u_wall[4][2];  /* wall velocities (left, right, bottom, top); a moving lid is u_wall[LBM_TOP] */
  double p_in, p_out;   /* pressures of the x = 0 and x = nx-1 columns when bc_x == LBM_PRESSURE */
  double p_rest;        /* reference phi*p of the stored deviations: f_rest,i = 3 w_i p_rest (Eq. 22, u = 0) */
  int32_t dev_scale_log2; /* FP16 storage holds (f - f_rest) * 2^dev_scale_log2 (away from FP16 subnormals);
                             FP32 and BF16 store f - f_rest unscaled */
  /* temperature equation (used when thermal == 1) */
  double tau_T;         /* zeta_1 = zeta_2 = 1/tau_T (Eq. B.7) */
  double zeta3, zeta4;  /* remaining rates (1.1 in Sec. 3.4) */
  double sigma;         /* thermal capacity ratio (Eq. B.1) */
  double g_beta, T0;    /* buoyancy a = g_beta (T - T0) j (Sec. 3.4); T0 is also the stored reference */
  double T_wall[4];     /* wall temperature (anti-bounce-back), NaN = adiabatic (bounce-back) */
  void* stream;         /* cudaStream_t to use, or NULL */
  uint32_t streaming;   /* LBM_STREAM_AB (default) | LBM_STREAM_INPLACE */
  uint32_t options;     /* LBM_OPT_* bits, 0 by default */
} lbm_config;

typedef struct lbm_ctx lbm_ctx;

/* Fill *cfg with the paper's defaults (Sec. 3): J = 1, rho0 = 1, s_e = 1.1, s_q = 1.2,
 * zeta3 = zeta4 = 1.1, sigma = 1, periodic x, walls in y, FP32, phi = 1, K = 1e30, p_rest = 1,
 * dev_scale_log2 = 10, adiabatic walls. */
LBM_API void lbm_config_defaults(lbm_config* cfg);

/* sizeof(lbm_config) as compiled into the library, for bindings to check their layout. */
LBM_API uint32_t lbm_config_size(void);

/* Create a context on the current CUDA device: allocates two population buffers (A-B
 * streaming; one with LBM_STREAM_INPLACE), the medium fields and, if thermal, the temperature
 * buffers in the same number.  The state is
 * initialised as by lbm_init_equilibrium(ctx, 1, 0, 0, 0).  EABI / EINVAL / ENOMEM / ECUDA. */
LBM_API int lbm_create(const lbm_config* cfg, lbm_ctx** out);

/* Release everything the context owns.  NULL is accepted. */
LBM_API void lbm_destroy(lbm_ctx* ctx);

/* Per-cell porosity eps (phi of Eq. 3) and permeability K, float32 [ny][nx], copied in.
 * Either may be NULL to keep a uniform value (cfg.phi / cfg.K).  Requires 0 < eps <= 1 and
 * K > 0 (checked on the device; EINVAL).  Does not change the populations. */
LBM_API int lbm_set_medium(lbm_ctx* ctx, const float* eps, const float* K);
/* Per-cell viscosity ratio J = upsilon_e / upsilon (Eq. 5), float32 [ny][nx], e.g. J > 1 in a porous
 * layer and 1 in free fluid (Sec. 3.2): the viscous rate becomes s_v = 1 / (1/2 + J nu / c_s^2)
 * per cell (Eq. 21), while the Darcy drag of Eq. 3 keeps the fluid viscosity nu.  NULL returns to
 * the uniform cfg.J.  Switches the context to per-cell medium fields (8 B + 4 B per cell read per
 * step).  Requires J > 0 (EINVAL); waits for the stream. */
LBM_API int lbm_set_viscosity_ratio(lbm_ctx* ctx, const float* J);
/* The same with log K given instead of K (K = exp(logK) per cell; the parameterisation of the
 * adjoint's gradient). */
LBM_API int lbm_set_medium_log(lbm_ctx* ctx, const float* eps, const float* logK);

/* Set the populations to the equilibrium f_eq(p, u; phi) of Eq. 22 (= M^-1 m_eq, Eqs. 8, 11) with
 * u = (ux0, uy0) and p = p0 (phi_p_uniform == 0, the initial state of Sec. 3.1) or p = p0/phi
 * (phi_p_uniform == 1: uniform phi p, the rest state of a medium with varying porosity).
 * Resets the step counter.  lbm_init_temperature sets g to the equilibrium of Eq. B.6 at
 * T = T_init, u = 0 (thermal contexts only; ESTATE otherwise). */
LBM_API int lbm_init_equilibrium(lbm_ctx* ctx, double p0, double ux0, double uy0, int phi_p_uniform);
LBM_API int lbm_init_temperature(lbm_ctx* ctx, double T_init);

/* Advance n >= 0 time steps of Eq. 6 (collision Eq. 14, streaming Eq. 15) and, if thermal,
 * of Eq. B.2 with the buoyancy coupling.  Runs of 32 steps or more replay a CUDA graph of 32
 * steps, captured on first use from a private stream (so a context on the legacy default stream
 * works too); lbm_set_medium discards the captured graphs. */
LBM_API int lbm_step(lbm_ctx* ctx, int n);

/* Replace the wall velocities u_wall[4][2] (left, right, bottom, top; float32, host or device)
 * for the following steps -- e.g. a time-dependent lid.  The copy is enqueued on the stream. */
LBM_API int lbm_set_walls(lbm_ctx* ctx, const float* u_wall);

/* (p, ux, uy, T) of one cell of the current state into out[4] (T = 0 without a temperature
 * field), by the same rules as lbm_macros.  Host outputs wait for the stream. */
LBM_API int lbm_probe(lbm_ctx* ctx, int x, int y, float* out);
/* lbm_probe without the wait: the read of the cell is enqueued on the stream and the call returns;
 * out[4] holds the values once the stream has passed this point (lbm_sync, or an event the caller
 * records on the stream after the call and waits for).  Host out should be page-locked (pinned):
 * the copy into pageable memory is staged by the driver and may wait.  A loop that steps, probes
 * and reads the previous step's probe keeps the GPU busy while the host reads. */
LBM_API int lbm_probe_async(lbm_ctx* ctx, int x, int y, float* out);

/* Macroscopic fields of the current state (pre-collision populations f(x, t)): pressure p
 * (Eq. 20), velocity u (Eqs. 18-19) and, if thermal, temperature T = sum g.  Outputs are
 * float32 [ny][nx]; any may be NULL. */
LBM_API int lbm_macros(lbm_ctx* ctx, float* p, float* ux, float* uy, float* T);

/* Export / import the current pre-collision populations f(x, t) as float32 [8][ny][nx]
 * (g: [5][ny][nx]).  On import, columns recomputed by a pressure boundary are replaced at
 * the next step. */
LBM_API int lbm_get_populations(lbm_ctx* ctx, float* f, float* g);
LBM_API int lbm_set_populations(lbm_ctx* ctx, const float* f, const float* g);

/* Steady-state residual r = ||u(t) - u(t-1)||_2 / ||u(t)||_2 over all cells, summed in FP64
 * on the device (needs one step since the last initialisation or import; ESTATE before that).
 * In-place contexts take u(t-1) from the velocity the last step of the last lbm_step call
 * recorded (ESTATE with LBM_OPT_NO_RESIDUAL_RECORD).  Waits for the stream. */
LBM_API int lbm_residual(lbm_ctx* ctx, double* r);

/* Allocation-free residual, for callers that must not allocate device memory (a service that
 * sizes one memory pool at start-up, a host whose framework owns all device memory through its
 * own allocator, a real-time loop that cannot afford the device-wide synchronisation of
 * cudaMalloc/cudaFree).  The paper has no counterpart: this is the residual above, computed from
 * two velocity fields the caller holds instead of from a context.
 *   ux, uy, ux_prev, uy_prev: device float32 arrays of n cells (any layout, the same for all four);
 *   r: device or host double receiving ||u - u_prev||_2 / ||u||_2 (sums in FP64; 0 if u = 0);
 *      managed memory counts as device memory: r is then written asynchronously on the stream,
 *      and the caller synchronises the stream before reading it on the host;
 *   stream: cudaStream_t to run on (NULL = the default stream).
 * Limits: 1 <= n <= 67108864 (2^26, an 8192 x 8192 lattice); larger n is EINVAL.  The partial
 * sums use a fixed 64 KB array in device memory that liblbm.so reserves on every GPU that loads
 * it, until the process exits; no call allocates or frees anything.  The first call on a device
 * looks up that array's address (once per device, with the device current); make that first
 * call before any stream capture.  All calls share the one array and each call overwrites it, so
 * calls whose work overlaps on the GPU (different streams, or different host threads) race and
 * must be serialised by the caller.  With a host r the call waits for the stream. */
LBM_API int lbm_residual_noalloc(const float* ux, const float* uy, const float* ux_prev, const float* uy_prev, int64_t n,
                                 double* r, void* stream);

/* loss kinds of lbm_adjoint */
#define LBM_LOSS_OUTLET_FLUX 0     /* L = sum_y u_x(nx-1, y) of the final state */
#define LBM_LOSS_VELOCITY_MISFIT 1 /* L = 1/2 sum |u - u*|^2 over all cells of the final state */

/* Discrete adjoint of T flow steps (collision Eq. 14, streaming Eq. 15, pressure columns and
 * extrapolated wall nodes) from the current initial state (call right after lbm_init_equilibrium;
 * ESTATE otherwise, and for thermal contexts; EINVAL for an LBM_NEE side pair fewer than 4 nodes
 * apart; an in-place context runs the sweep on two A-B state buffers of the workspace and takes the
 * final state back into its own layout): runs the T steps -- the context ends at step T, as after lbm_step(ctx, T) -- and
 * returns the loss and its gradient with respect to the per-cell log K and eps (phi) fields,
 * including their effect on the initial equilibrium (Eq. 22).  Memory: checkpoints of the
 * post-collision state every ceil(sqrt(T)) steps, two segments of ceil(sqrt(T)) states (the
 * states of one segment are recomputed, on a second stream of lower priority, while the adjoint
 * steps of the next run on a stream of higher priority), two FP32 adjoint states and the gradient
 * sums (FP32 partial sums over at most 64 steps, folded into FP64 totals) form a workspace that
 * stays allocated after the call, so that repeated calls (an optimisation loop) allocate nothing;
 * it is counted by lbm_memory_bytes and freed by lbm_release_workspace or lbm_destroy.  The
 * forward work is about 2 T steps.
 *   target_ux, target_uy: float32 [ny][nx] (misfit loss only; host or device).
 *   grad_logK, grad_eps: double [ny][nx] outputs (host or device; NULL skips); loss: double.
 * Waits for the stream. */
LBM_API int lbm_adjoint(lbm_ctx* ctx, int T, int loss_kind, const float* target_ux, const float* target_uy, double* grad_logK,
                        double* grad_eps, double* loss);

/* lbm_adjoint under the name used in the method's interface description (same arguments, same
 * behaviour): the adjoint of the stream-collide step applied over T steps. */
LBM_API int lbm_adjoint_step(lbm_ctx* ctx, int T, int loss_kind, const float* target_ux, const float* target_uy,
                             double* grad_logK, double* grad_eps, double* loss);

/* Frees the workspace that lbm_adjoint keeps between calls (no-op if there is none); the next
 * lbm_adjoint allocates it again.  Waits for the stream.  Not in the paper: memory management. */
LBM_API int lbm_release_workspace(lbm_ctx* ctx);

/* Average Nusselt number of a wall with a prescribed temperature (side = LBM_LEFT or
 * LBM_RIGHT): Nu = (L / (T_hot - T_cold)) * mean_y(-+ dT/dx at the wall).  Halfway walls
 * (LBM_WALL): L = nx, dT/dx from the parabola through the wall value and the two nearest cells;
 * wall nodes (LBM_NEE): L = nx - 1, dT/dx = (-3 T_0 + 4 T_1 - T_2) / 2, over the rows 1..ny-2
 * when the bottom/top walls are wall nodes too (they own the corners).  FP64 sum.  Waits. */
LBM_API int lbm_nusselt(lbm_ctx* ctx, int side, double* nu);

/* ---------------------------------------------------------------------------------------------
 * Batched ensembles: n independent isothermal lattices, each with its own lbm_config (size,
 * boundaries, parameters, medium; one storage precision for all), advanced together by one
 * launch per time step over the concatenated work items of all lattices (one CTA per item, CTAs
 * of a few items, or a persistent grid: lbm_batch_set_launch, lbm_batch_tune), with
 * runs of 32 steps replayed as a captured CUDA graph.  The batch runs on cfgs[0].stream (NULL:
 * a stream of its own).  Every lattice keeps per-cell medium fields (8 B per cell).  All lattices
 * use one streaming form: LBM_STREAM_AB (two population pools), or LBM_STREAM_INPLACE (one pool,
 * periodic and halfway-wall sides, launch shape 128 threads per CTA and one CTA per work item).
 * ------------------------------------------------------------------------------------------- */
typedef struct lbm_batch lbm_batch;

/* Create the batch and initialise every lattice to the equilibrium at p = 1, u = 0. */
LBM_API int lbm_batch_create(const lbm_config* cfgs, int n, lbm_batch** out);
/* lbm_batch_create under the name used in the method's interface description (same arguments,
 * same behaviour). */
LBM_API int lbm_create_batch(const lbm_config* cfgs, int n, lbm_batch** out);
LBM_API void lbm_batch_destroy(lbm_batch* b);
/* Medium of lattice d (as lbm_set_medium; waits for the stream). */
LBM_API int lbm_batch_set_medium(lbm_batch* b, int d, const float* eps, const float* K);
/* Equilibrium initial state of lattice d (d = -1: all), as lbm_init_equilibrium. */
LBM_API int lbm_batch_init_equilibrium(lbm_batch* b, int d, double p0, double ux0, double uy0, int phi_p_uniform);
/* Advance every lattice by n steps with the batched kernel (one launch per step for the batch). */
LBM_API int lbm_batch_step(lbm_batch* b, int n);
/* The same n steps run lattice by lattice with the single-lattice kernel (for comparison). */
LBM_API int lbm_batch_step_each(lbm_batch* b, int n);
/* Launch shape of the batched kernel: threads per CTA (64, 128, 256) and CTAs per SM: 0 = one CTA
 * per work item (a lattice table of 4 bytes per item is kept on the device), 1..32 = a persistent
 * grid of SMs x k CTAs, k lowered to the kernel's occupancy limit so that every CTA is resident.
 * In-place batches take (128, 0) only (EINVAL otherwise). */
LBM_API int lbm_batch_set_launch(lbm_batch* b, int threads_per_cta, int ctas_per_sm);
LBM_API int lbm_batch_get_launch(const lbm_batch* b, int* threads_per_cta, int* ctas_per_sm);
/* Work items per CTA when ctas_per_sm = 0: 1 (the default) = one CTA per work item; 2, 4 or 8 = CTAs
 * of that many consecutive work items of the concatenated list (4 x items_per_cta cells per thread;
 * ceil(items / items_per_cta) CTAs walking their ranges as the persistent form does, the lattice
 * table not needed).  In-place batches take 1 only (EINVAL otherwise).  The work-item tables are
 * rebuilt. */
LBM_API int lbm_batch_set_items_per_cta(lbm_batch* b, int items_per_cta);
LBM_API int lbm_batch_get_items_per_cta(const lbm_batch* b, int* items_per_cta);
/* Tiling of each lattice into work items of one CTA (A-B batches; in-place batches keep their own
 * tiling and accept LBM_TILING_FLAT only, EINVAL otherwise):
 *   LBM_TILING_ROWS  rows of work items: a row of G four-cell groups takes ceil(G / threads) items,
 *                    or several short rows share one;
 *   LBM_TILING_FLAT  the lattice's groups in row-major order, `threads` consecutive groups per item
 *                    (an item may end one row and start the next; only the last item is ragged).
 * The default is LBM_TILING_FLAT.  The work-item tables are rebuilt for the current launch shape. */
#define LBM_TILING_ROWS 0
#define LBM_TILING_FLAT 1
LBM_API int lbm_batch_set_tiling(lbm_batch* b, int tiling);
LBM_API int lbm_batch_get_tiling(const lbm_batch* b, int* tiling);
/* Time `steps` steps for every launch shape (threads per CTA 64 / 128 / 256; one CTA per work item,
 * CTAs of 2 or 4 work items, persistent grids of 1..16 CTAs per SM) and tiling on a copy of the
 * current state, keep the fastest, restore the state; outputs may be NULL (the chosen tiling and
 * work items per CTA: lbm_batch_get_tiling, lbm_batch_get_items_per_cta).  Waits for the stream. */
LBM_API int lbm_batch_tune(lbm_batch* b, int steps, int* threads_per_cta, int* ctas_per_sm, float* ms_per_step);
/* Read-outs of lattice d (float32 [ny_d][nx_d] / [8][ny_d][nx_d], host or device). */
LBM_API int lbm_batch_macros(lbm_batch* b, int d, float* p, float* ux, float* uy);
LBM_API int lbm_batch_get_populations(lbm_batch* b, int d, float* f);
/* Total cells, steps taken since the last full initialisation, device bytes held. */
LBM_API int lbm_batch_info(const lbm_batch* b, int64_t* cells, int64_t* steps, uint64_t* bytes);
/* Wait for the batch's stream and report a deferred error. */
LBM_API int lbm_batch_sync(lbm_batch* b);

/* Checkpoint / resume: write the context's state (both population buffers -- in-place contexts:
 * the one buffer and the u(t-1) record --, temperature populations, medium, step counters,
 * configuration) to a file, and read it back into a context of the same size, precision, thermal
 * mode, streaming form and record option; stepping after lbm_load continues bitwise as the saved
 * context would have.  Both wait for the stream.  EINVAL on I/O or format errors. */
LBM_API int lbm_save(lbm_ctx* ctx, const char* path);
LBM_API int lbm_load(lbm_ctx* ctx, const char* path);

/* Wait for the context stream and report a deferred error (EUNSTABLE, ECUDA). */
LBM_API int lbm_sync(lbm_ctx* ctx);

/* Number of steps taken since the last initialisation. */
LBM_API int lbm_step_count(const lbm_ctx* ctx, int64_t* steps);

/* Device byte count of the context's allocations (populations, medium, scratch). */
LBM_API int lbm_memory_bytes(const lbm_ctx* ctx, uint64_t* bytes);

LBM_API const char* lbm_strerror(int code);
LBM_API const char* lbm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
