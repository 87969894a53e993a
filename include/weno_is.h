/*
 * weno_is.h -- C ABI of the GB300 (sm_103a) library for the L2-norm
 * regularized incremental-stencil WENO scheme of Zhu & Hu (arXiv 1908.02464)
 * applied to the compressible Euler equations.
 *
 * The library computes, on one GPU, the semi-discrete right-hand side
 *     dU_j/dt = - sum_d (F^_{j+1/2} - F^_{j-1/2}) / dx_d          (Eq. goveq5)
 * with the characteristic-wise numerical flux of Sec. 2.4 (Roe average,
 * eigensystem, projection Eq. eqchara, local Lax-Friedrichs splitting
 * Eq. flxuspliting, reconstruction Eq. reconstruction/reconstruction1,
 * back-projection Eq. reconstruction2), the regularized weights Eq. eq8-r
 * with the L2 error terms Eq. eq18, the detector and regularization
 * parameter Eq. eq27-29 and the hybrid switch to the optimal linear upwind
 * scheme Eq. eqhy/linearupwind/eq31; and advances it with the third-order
 * TVD Runge-Kutta scheme at a CFL-limited time step (Sec. 4).
 *
 * Conventions for every entry point:
 *   - Every call returns a weno_status; nothing aborts or throws across the
 *     ABI.  Errors raised on the device (non-physical state) are latched in a
 *     status word and reported by the next call that synchronizes.
 *   - State arrays are structure-of-arrays, interior cells only, C order
 *     [nvar][nz][ny][nx] (nvar = dim + 2: rho, rho*u_x, [rho*u_y], [rho*u_z],
 *     E).  The element type is double for WENO_FP64 and float for WENO_FP32
 *     and WENO_MIXED.
 *   - Pointers passed in are borrowed; the library copies what it keeps.
 *     Device pointers must be allocated on the context's device and be
 *     naturally aligned.
 *   - All device work is issued on the stream given to weno_create (the
 *     legacy default stream when NULL).  A context is not thread-safe.
 */
#ifndef WENO_IS_H
#define WENO_IS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WENO_OK = 0,
    WENO_ERR_INVALID_ARG = 1,   /* bad pointer, size, code or combination      */
    WENO_ERR_CUDA = 2,          /* a CUDA runtime call failed (see last_error) */
    WENO_ERR_NONPHYSICAL = 3,   /* rho <= 0, p <= 0 or a non-finite value      */
    WENO_ERR_TIMEOUT = 4,       /* a bounded device wait ran out               */
    WENO_ERR_UNSUPPORTED = 5    /* valid request that this build does not do   */
} weno_status;

typedef enum {
    WENO_FP64 = 0,   /* all arithmetic and storage in double                    */
    WENO_FP32 = 1,   /* float storage and arithmetic; time step, time and the
                        conserved totals in double                             */
    WENO_MIXED = 2   /* as FP32, with the detector's fifth difference
                        (Eq. eq28), which decides the hybrid switch, formed
                        as exact nested float differences                      */
} weno_precision;

/* boundary codes, one per side and direction (ghost cells, three layers).
   The double Mach codes are accepted only on the y boundaries and the jet
   only on the x boundaries of a 2D or 3D grid (weno_create returns
   WENO_ERR_INVALID_ARG otherwise). */
enum {
    WENO_BC_TRANSMISSIVE = 0, /* copy of the nearest interior cell                    */
    WENO_BC_REFLECT = 1,      /* mirror image, normal momentum negated                */
    WENO_BC_PERIODIC = 2,     /* wrap-around                                          */
    WENO_BC_INFLOW = 3,       /* fixed conservative state bc_state[0]                 */
    WENO_BC_DMR_BOTTOM = 4,   /* y-low of the double Mach reflection (Sec. 4.5):
                                 bc_state[0] for x < 1/6, reflecting wall otherwise */
    WENO_BC_DMR_TOP = 5,      /* y-high of the double Mach reflection: bc_state[0]
                                 for x < 1/6 + (1 + 20 t)/sqrt(3), bc_state[1] else */
    WENO_BC_JET = 6           /* x-low inflow jet (Sec. 4.7): bc_state[0] where
                                 y < 0.05, bc_state[1] elsewhere                   */
};

/* Uniform cell-centred grid x_i = lo + (i + 1/2) dx (Sec. 2.1, x_j = j dx). */
typedef struct {
    int dim;                 /* 1, 2 or 3                                    */
    int n[3];                /* interior cells per direction (unused = 1)    */
    double lo[3], hi[3];     /* domain bounds                                */
    int bc_lo[3], bc_hi[3];  /* WENO_BC_* per side                           */
    double bc_state[2][5];   /* conservative states used by INFLOW and DMR   */
} weno_grid;

/* Constants of the method.  Defaults (weno_default_params) are the paper's:
 * gamma 1.4, CFL 0.5 (Sec. 4), eps 1e-20 (Eq. eq8), c 1 (Eq. eq29),
 * C 1 and alpha 3 (Eq. eq31), L 1 (characteristic length of Eq. eq31). */
typedef struct {
    double gamma;
    double cfl;
    double eps;        /* epsilon of Eq. eq8-r                                  */
    double c_lambda;   /* c of Eq. eq29: lambda = c sigma^s                      */
    double C_thr;      /* C of Eq. eq31                                          */
    double L_char;     /* L of Eq. eq31                                          */
    int alpha_thr;     /* alpha of Eq. eq31 (integer power)                      */
    int hybrid;        /* 0: WENO everywhere; 1: linear upwind scheme on faces
                          where sigma^s < eps_h for all s (Eq. eqhy, the
                          method); 2: also per field on the other faces (the
                          optimal linear weights for each field with
                          sigma^s < eps_h)                                      */
    int precision;     /* weno_precision                                         */
    int weights;       /* 0 regularized (Eq. eq8-r, the method), 1 WENO-IS
                          (Eq. eq8), 2 WENO-IS of Wang et al. (Eq. eq14-15),
                          3 optimal linear weights d_k                          */
    int splitting;     /* 0 local LF over the six stencil cells, 1 global LF
                          over the domain, 2 Roe (Eq. flxuspliting)              */
} weno_params;

typedef struct weno_ctx weno_ctx;

/* Fill *p with the paper's constants, WENO_FP64, the regularized weights and
 * LLF splitting. */
weno_status weno_default_params(weno_params* p);

/* Create a context on the current CUDA device.  Allocates the state buffers
 * (three rotating RK states and, for dim >= 2, one RHS accumulator, each with
 * three ghost layers), the device scalars and the reduction scratch.
 * stream: a cudaStream_t cast to void* (NULL = legacy default stream).
 * Errors: WENO_ERR_INVALID_ARG for dim outside 1..3, n < 1, a domain with
 * hi <= lo, an unknown BC code, a periodic side paired with a non-periodic
 * one, n < 3 in a periodic direction, or an unknown precision;
 * WENO_ERR_CUDA when allocation fails.  On error *out is NULL. */
weno_status weno_create(const weno_grid* grid, const weno_params* params, void* stream,
                        weno_ctx** out);

/* Release every device allocation of the context; NULL is accepted. */
void weno_destroy(weno_ctx* ctx);

/* Copy a state into the context and set the time to t (steps counter and
 * device status are reset).  U: interior-only array (see conventions), host
 * memory when on_device = 0, device memory otherwise.  Page-locked, mapped
 * host memory (cudaHostAlloc, or registered with the mapped flag) is read
 * directly by the layout kernel; pageable host memory goes through a device
 * copy.  Synchronizes the context's stream. */
weno_status weno_set_state(weno_ctx* ctx, const void* U, int on_device, double t);

/* Copy the current state out (same layout) and, if t is not NULL, the time.
 * Page-locked, mapped host memory is written directly by the layout kernel.
 * Synchronizes the context's stream. */
weno_status weno_get_state(weno_ctx* ctx, void* U, int on_device, double* t);

/* Semi-discrete right-hand side dU/dt (Eq. goveq5 summed over directions) of
 * the interior-only device array U_dev, with ghost cells filled at time t.
 * dUdt_dev: interior-only device array of the same shape, overwritten; it
 * must not overlap U_dev (WENO_ERR_INVALID_ARG if the two are the same
 * array).  The sweeps read U_dev and write dUdt_dev in place, with no copy
 * into the context's padded layout (the ghost cells are computed from the
 * boundary conditions while the tiles are staged).  The context's own state
 * is not touched.  Asynchronous on the context's stream; returns
 * WENO_ERR_CUDA if a launch fails. */
weno_status weno_rhs(weno_ctx* ctx, const void* U_dev, void* dUdt_dev, double t);

/* Vector-Jacobian product of the semi-discrete operator (the adjoint of
 * weno_rhs; the paper does not differentiate its scheme):
 *     gU = (d RHS / d U)^T w   at U = U_dev, ghost cells filled at time t.
 * The hybrid flag of each face (Eq. eqhy) and the stencil cell attaining
 * each LLF maximum (Eq. flxuspliting) are held at their values for U_dev
 * (first index on ties): the result is the derivative of the active smooth
 * piece.  The backward pass recomputes every forward quantity (Roe state,
 * detector, projections, nonlinear weights); nothing is stored between
 * calls.  Ghost-cell contributions are mapped back through the boundary
 * conditions (fixed inflow states receive none).  U_dev, w_dev, gU_dev:
 * interior-only device arrays of the state's shape and element type, read
 * and written in place (the tiles compute U's ghost cells while staging;
 * the cotangent is zero on ghost cells); gU_dev must not overlap U_dev or
 * w_dev (WENO_ERR_INVALID_ARG if it is one of them).  Deterministic (no
 * atomics).  Asynchronous; WENO_ERR_CUDA if a launch or the first call's
 * allocation of the per-line ghost-gradient buffer fails;
 * WENO_ERR_UNSUPPORTED unless the context uses the regularized weights with
 * LLF splitting and hybrid 0 or 1. */
weno_status weno_rhs_vjp(weno_ctx* ctx, const void* U_dev, const void* w_dev, void* gU_dev, double t);

/* Per-face hybrid flags of U_dev at time t: 1 where the linear upwind scheme
 * is used (Eq. eqhy, sigma_{j+1/2} = 1), 0 where the regularized WENO-IS flux
 * is used.  flags_dev: uint8 device array holding, for each direction d in
 * order, the faces of shape [nz][ny][nx] with n_d + 1 entries along d (face
 * i - 1/2 lies between cells i - 1 and i).  Asynchronous. */
weno_status weno_face_flags(weno_ctx* ctx, const void* U_dev, double t, uint8_t* flags_dev);

/* One TVD RK3 step of the context's state.  dt = CFL / max_cells
 * sum_d (|u_d| + c) / dx_d, clipped so that t + dt <= t_end (time reaches
 * t_end exactly on the clipped step).  Writes the dt taken (0 when t >= t_end)
 * to *dt_taken if not NULL.  Synchronizes.  On a non-physical stage state
 * returns WENO_ERR_NONPHYSICAL and leaves state and time at the last good
 * step. */
weno_status weno_step(weno_ctx* ctx, double t_end, double* dt_taken);

/* Up to max_steps steps towards t_end, replayed from CUDA graphs in chunks
 * (the host reads the device time and status once per chunk).  *steps_taken
 * receives the number of completed steps.  Errors as weno_step. */
weno_status weno_advance(weno_ctx* ctx, double t_end, int max_steps, int* steps_taken);

/* Asynchronous stepping: enqueue nsteps RK3 steps (CUDA-graph replays)
 * towards t_end on the context's stream and return without synchronizing.
 * Steps that would pass t_end, and every step after a non-physical stage,
 * do nothing on the device; the next synchronizing call (weno_get_time,
 * weno_get_state, weno_step, ...) reads the true time, step count and
 * status.  Errors: WENO_ERR_CUDA if capture or a launch fails. */
weno_status weno_enqueue_steps(weno_ctx* ctx, double t_end, int nsteps);

/* Measurement helper (no counterpart in the paper): times `reps` launches of
 * the sweep kernel of every direction on the current state (ghosts filled at
 * the current time; the sweeps write the RHS accumulator only, the state is
 * not changed), each launch bracketed by CUDA events on the context's stream.
 * If flush_dev is not NULL, flush_bytes of it are overwritten before every
 * launch (to evict L2).  ms[d] receives the mean launch time of direction d,
 * weno_faces[d] (if not NULL) the number of faces of one launch that took
 * the WENO flux.  Synchronizes. */
weno_status weno_time_sweeps(weno_ctx* ctx, int reps, void* flush_dev, size_t flush_bytes, double* ms,
                             unsigned long long* weno_faces);

/* Tile autotuner (no counterpart in the paper): for every sweep direction,
 * times each compiled tile shape `reps` times on the current state and keeps
 * the fastest for this context.  Shapes (variant: lines x cells per CTA):
 * 0: 2x63, 1: 8x15, 2: 4x31, 3: 1x127, 4: 1x95, 5: flat, 123 consecutive
 * faces of the line-after-line face sequence (a tile may end one line and
 * start the next; lines shorter than 122 cells take variant 3), 6: flat
 * with 251 faces on 256 threads (lines shorter than 250 take 3), 7: FP32
 * and mixed sweeps across x (y, z) by marching warps, one lane per line
 * along a segment of 12 (2D) or 18 (3D) cells with the six-cell stencil
 * in registers (FP32 along x takes 3, FP64 takes 5).  Defaults: FP64 5 in
 * every direction except along y in 3D (2); FP32 and mixed 3 along x, 1
 * across, 7 across when lines x segments reach four rounds of 16 warps on
 * every SM.
 * variants[3] (if not NULL) receives the choice per direction.
 * The state is not changed; the step graphs are rebuilt on next use.
 * Synchronizes. */
weno_status weno_autotune(weno_ctx* ctx, int reps, int* variants);

/* Pin the tile shape of every sweep direction (variants[d] in 0..7, see
 * weno_autotune; ignored in 1D).  Results do not depend on the tile shape:
 * every face is computed by the same arithmetic.  WENO_ERR_INVALID_ARG for
 * an unknown variant. */
weno_status weno_set_tiles(weno_ctx* ctx, const int* variants);

/* Conserved totals sum_cells U dV per variable (nvar doubles, host memory),
 * accumulated in double.  Synchronizes. */
weno_status weno_conserved_totals(weno_ctx* ctx, double* totals);

/* ------------------------------------------------------------------------
 * Batched 1D problems (many independent shock tubes of uneven sizes).
 * Each instance i is a 1D Euler problem on [lo[i], hi[i]] with n[i] cells,
 * advanced from t = 0 to t_end[i] with its own CFL step (same scheme and
 * constants as weno_params), in one persistent launch replayed from a CUDA
 * graph: every CTA takes the next instance from a work queue ordered
 * largest first and runs its whole RK3 loop (Sec. 4) on its own.
 * ---------------------------------------------------------------------- */
typedef struct {
    int count;              /* number of instances (>= 1)                      */
    const int* n;           /* host [count]: cells of each instance (>= 3)     */
    const double* lo;       /* host [count]                                    */
    const double* hi;       /* host [count]                                    */
    const double* t_end;    /* host [count]: end time of each instance         */
    int bc_lo, bc_hi;       /* WENO_BC_TRANSMISSIVE, _REFLECT or _PERIODIC     */
    int max_steps;          /* per-instance step limit, 0 = none               */
} weno_batch_desc;

typedef struct weno_batch weno_batch;

/* Create a batch: copies the description, orders the instances largest
 * first, allocates three ghosted work arrays per instance.  States are passed
 * to weno_batch_run as one device array holding the instances back to back,
 * instance i as [3][n[i]] (rho, rho u, E) starting at element 3 sum_{j<i} n[j]
 * (double for WENO_FP64, float otherwise).  Errors: WENO_ERR_INVALID_ARG for
 * an empty batch, n < 3, hi <= lo, negative t_end, other boundary codes or an
 * unknown precision; WENO_ERR_CUDA if allocation fails. */
weno_status weno_batch_create(const weno_batch_desc* desc, const weno_params* params, void* stream,
                              weno_batch** out);

/* Advance every instance of U_dev (in place: initial states in, states at
 * their t_end out) in one graph-replayed persistent launch.  Asynchronous;
 * read the per-instance outcome with weno_batch_results. */
weno_status weno_batch_run(weno_batch* batch, void* U_dev);

/* Per-instance results of the last run (host arrays of count entries, each
 * may be NULL): status (0 ok, WENO_ERR_NONPHYSICAL: the instance stopped at
 * its last admissible step), completed steps and reached time.
 * Synchronizes; returns WENO_ERR_NONPHYSICAL if any instance failed. */
weno_status weno_batch_results(weno_batch* batch, int* status, long long* steps, double* t);

/* Autotuner (no counterpart in the paper): times trial runs for each CTA
 * size (64, 128, 256 threads: tiles of 63, 127, 255 faces) and residency
 * (all that fit, 4 or 2 CTAs per SM) and keeps the fastest.  U_dev is not
 * modified.  The trials start from a scratch copy of U_dev advanced with
 * the current configuration to half of each instance's end time: the cost
 * of a step changes as the waves spread, and trials from the initial states
 * rank the configurations unlike full runs do.  This pass costs about half
 * a run and allocates the scratch state and a t_end array for the call.  In
 * a trial run instance i takes ceil(trial_steps N_i / N_max) steps (at least
 * one): a full run's step count grows with the cell count, so the trial
 * keeps the full run's work per instance, growing like N_i^2, and with it
 * the load balance of the schedule.  choice[0] = tile variant, choice[1] =
 * CTAs launched.  The per-instance results afterwards are those of the last
 * trial.  Synchronizes. */
weno_status weno_batch_autotune(weno_batch* batch, const void* U_dev, int trial_steps, int* choice);

/* Fixes the configuration without timing (no counterpart in the paper):
 * variant 0, 1, 2 = 128-, 64-, 256-thread CTAs (tiles of 127, 63, 255
 * faces); blocks_per_sm = resident CTAs per SM, 0 = as many as fit (values
 * above that are lowered to it).  *blocks (may be NULL) receives the CTAs a
 * run launches: min(count, residency x SMs).  WENO_ERR_INVALID_ARG for a
 * variant outside 0..2 or a negative blocks_per_sm. */
weno_status weno_batch_set_config(weno_batch* batch, int variant, int blocks_per_sm, int* blocks);

/* Number of faces computed with the WENO (non-linear) flux by the batch's
 * runs (autotuner trial runs included) since creation or the last call with
 * reset != 0; a face counts once per RK stage.  Synchronizes. */
weno_status weno_batch_weno_face_count(weno_batch* batch, unsigned long long* count, int reset);

void weno_batch_destroy(weno_batch* batch);
const char* weno_batch_last_error(const weno_batch* batch);

/* ------------------------------------------------------------------------
 * Batched 2D problems (many independent 2D boxes of uneven sizes).
 * Instance i is a 2D Euler problem on [lo_x[i], hi_x[i]] x [lo_y[i], hi_y[i]]
 * with nx[i] x ny[i] cells, advanced from t = 0 to t_end[i] with its own CFL
 * step (dt = CFL / max (|u| + c)/dx + (|v| + c)/dy, Sec. 4) by the same
 * dimension-by-dimension scheme as weno_step (Sec. 2.4, Eq. goveq5), in one
 * persistent launch replayed from a CUDA graph: every CTA takes the next
 * instance from a work queue ordered by nx ny max(nx, ny) (cells x steps),
 * largest first, and runs its whole RK3 loop on its own.  Each stage is the
 * y sweep (flux divergence into an accumulator) followed by the x sweep
 * (its divergence plus the RK3 combination), as in the grid solver, whose
 * results the batch reproduces bit for bit.
 * ---------------------------------------------------------------------- */
typedef struct {
    int count;              /* number of instances (>= 1)                      */
    const int* nx;          /* host [count]: cells along x (>= 3)              */
    const int* ny;          /* host [count]: cells along y (>= 3)              */
    const double* lo_x;     /* host [count]                                    */
    const double* hi_x;
    const double* lo_y;
    const double* hi_y;
    const double* t_end;    /* host [count]: end time of each instance         */
    int bc_lo[2], bc_hi[2]; /* per direction (x, y): WENO_BC_TRANSMISSIVE, _REFLECT or _PERIODIC */
    int max_steps;          /* per-instance step limit, 0 = none               */
} weno_batch2d_desc;

/* Create a 2D batch: the returned handle takes weno_batch_run, _results,
 * _autotune, _set_config (variants 0..2: x / y tiles of 4x31 / 8x15 and 2x63
 * / 4x31 on 128 threads, 2x31 / 4x15 on 64 threads), _weno_face_count and
 * _destroy like a 1D batch.  States are one device array holding the
 * instances back to back, instance i as [4][ny[i]][nx[i]] (rho, rho u, rho v,
 * E; x fastest) starting at element 4 sum_{j<i} nx[j] ny[j] (double for
 * WENO_FP64, float otherwise).  Allocates four work arrays of the batch's
 * size.  Errors: WENO_ERR_INVALID_ARG for an empty batch, nx or ny < 3,
 * hi <= lo, negative t_end, other boundary codes, unpaired periodic
 * boundaries or an unknown precision; WENO_ERR_UNSUPPORTED for global
 * Lax-Friedrichs splitting; WENO_ERR_CUDA if allocation fails. */
weno_status weno_batch2d_create(const weno_batch2d_desc* desc, const weno_params* params, void* stream,
                                weno_batch** out);

/* One-call form: create, run, collect per-instance status (host array of
 * count ints, may be NULL), destroy. */
weno_status weno_batch_solve(const weno_batch_desc* desc, const weno_params* params, void* stream, void* U_dev,
                             int* per_instance);

/* Allocation-free conserved totals (the paper has no counterpart; this is a
 * service for callers that cannot allocate device memory where they need
 * the totals: applications whose device memory belongs to their own pool or
 * allocator, and time-stepping loops with a fixed memory budget that must
 * neither allocate nor take the device-wide synchronization cudaMalloc can
 * imply).  Same sums as weno_conserved_totals, for a state the caller owns
 * and without a context; nothing is allocated.
 *   dim, n[dim], dx[dim]: grid (cells per direction, spacing); the result is
 *       sum_cells U dV with dV = prod dx.
 *   precision: element type of U_dev (double for WENO_FP64, float else).
 *   U_dev: device array, interior cells only, [nvar][nz][ny][nx], nvar = dim+2.
 *   totals_dev: device array of nvar doubles, overwritten.
 *   stream: cudaStream_t cast to void* (NULL = legacy default stream).
 * The per-block partial sums live in one file-scope device array of 640 KiB
 * (16384 blocks x 5 variables, 4096 cells per block) that every GPU loading
 * the library keeps until the process exits; grids of more than 67,108,864
 * cells are rejected with WENO_ERR_INVALID_ARG, as are a bad dim, n < 1, an
 * unknown precision or a NULL pointer.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device
 * current, and so does every later call made outside stream capture (the
 * address changes if the device is reset); make the first call before any
 * stream capture.  Each call
 * overwrites the partial sums it uses before reading them, but all calls on a
 * device share the one array: calls that overlap on the GPU (different
 * streams without ordering) race.  Asynchronous; WENO_ERR_CUDA if the
 * address lookup or a launch fails. */
weno_status weno_conserved_totals_noalloc(int dim, const int* n, const double* dx, int precision,
                                          const void* U_dev, double* totals_dev, void* stream);

/* Number of faces computed with the WENO (non-linear) flux since the last
 * call with reset != 0, over every sweep launched by weno_rhs, weno_step
 * and weno_advance.  Synchronizes. */
weno_status weno_weno_face_count(weno_ctx* ctx, unsigned long long* count, int reset);

/* Time and completed steps of the context (host copies; synchronizes). */
weno_status weno_get_time(weno_ctx* ctx, double* t, long long* steps);

/* Human-readable text of the last error of ctx (or of the last failed
 * weno_create when ctx is NULL).  Valid until the next call on ctx. */
const char* weno_last_error(const weno_ctx* ctx);

/* Measurement helper (no counterpart in the paper): peak fused multiply-add
 * throughput of the current device in FLOP/s for precision 0 = double,
 * 1 = float, from a dependent-chain kernel that fills every SM.  Writes the
 * rate to *flops and the kernel time in seconds to *seconds.  Synchronizes. */
weno_status weno_measure_fma_peak(int precision, double* flops, double* seconds);

/* Diagnostic (no counterpart in the paper): evaluates, for n doubles x_dev[i]
 * on the device, the refined reciprocal and reciprocal square root that the
 * FP64 sweeps use (Roe average, sound speeds, weight denominator of Eq.
 * eq8-r) next to CUDA's correctly rounded 1.0 / x and its rsqrt(x), so that
 * tests can bound their errors.  out_dev (device, 4 n doubles, caller-owned)
 * receives [rcp_newton(x) | 1/x | rsqrt_refined(x) | rsqrt(x)].  n < 0, or
 * null pointers with n > 0: WENO_ERR_INVALID_ARG.  Synchronizes the device. */
weno_status weno_arith_selftest(const double* x_dev, long long n, double* out_dev);

#ifdef __cplusplus
}
#endif
#endif /* WENO_IS_H */
