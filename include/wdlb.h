/*
 * wdlb.h - C ABI of the GB300 Weighted Density Lattice Boltzmann (WDLB)
 * library: the per-timestep lattice update of Marini Bettolo Marconi &
 * Melchionna, "Weighted density Lattice Boltzmann approach to fluids under
 * confinement" (arXiv:1304.7880), run as sm_103a CUDA kernels.
 *
 * One call of wdlb_step advances the five-step algorithm of Sec. 5 (Numerical
 * results) by one or more time steps on one lattice ("pore"):
 *   fields   smeared density nbar (Sec. 3, Fischer-Methfessel prescription),
 *            C = n (F^mf + F^viscous) (Sec. 3, Eq. campoc) and the SMDB field
 *            A (Eq. campod), as sums over the contact shell |e| ~ sigma;
 *   collide  BGK relaxation (Eq. relaxationtime) plus the hydrodynamic
 *            projection with force n g + C and the A-term (Eq. SMDB,
 *            Eq. eq:dufty2), second-order (trapezoidal) in time;
 *   stream   D3Q19 (Sec. 5), periodic in x and y (and z without walls),
 *            half-way bounce-back on the smooth walls z = 0 and z = nz-1.
 *
 * Units: lattice units, spacing = time step = mass = 1, k_B T = 1/3.
 * Layout of every per-node array exchanged through this header: node index
 * i = x + nx*(y + ny*z); vector fields are three consecutive arrays of N
 * values (x components, then y, then z), N = nx*ny*nz.
 *
 * Threading: a context may be used by one host thread at a time.  All device
 * work of a context is issued on its stream (wdlb_options.stream); calls that
 * return host data synchronise that stream.
 *
 * Errors: every call returns a wdlb_status; wdlb_last_error(ctx) gives a
 * message.  No call aborts the process.  A kernel that detects a non-physical
 * state (packing fraction of the smeared density >= 1, non-finite or
 * non-positive density) records it in a device status word; the next call
 * that synchronises returns WDLB_ERR_UNSTABLE.
 */
#ifndef WDLB_H
#define WDLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wdlb_ctx wdlb_ctx; /* opaque; owned by the library */

typedef enum {
    WDLB_OK = 0,
    WDLB_ERR_ARG = 1,      /* invalid argument; nothing was changed             */
    WDLB_ERR_OOM = 2,      /* device allocation failed or workspace too small   */
    WDLB_ERR_CUDA = 3,     /* a CUDA call failed; message in wdlb_last_error.
                              Also: in the bounds-checked build
                              (libwdlb_checked.so), a kernel index outside its
                              array (the access was skipped)                    */
    WDLB_ERR_UNSTABLE = 4, /* smeared packing fraction >= 1 or non-finite state */
    WDLB_ERR_TIMEOUT = 5,  /* a bounded wait ran out, or a served request hit its
                              step cap before its steady-state tolerance        */
    WDLB_ERR_STATE = 6     /* call out of order (e.g. step before init)         */
} wdlb_status;

typedef struct {
    int32_t nx, ny, nz;
} wdlb_lattice;

enum { WDLB_WALLS_NONE = 0, WDLB_WALLS_Z = 1 };
/* Contact value g2(sigma+) of the homogeneous hard-sphere fluid at packing
 * fraction chi = pi n sigma^3 / 6 (Sec. 3 leaves it open):
 * Carnahan-Starling (1 - chi/2)/(1 - chi)^3, Percus-Yevick (1 + chi/2)/(1 - chi)^2,
 * or 1 (test closure). */
enum { WDLB_CLOSURE_CS = 0, WDLB_CLOSURE_PY = 1, WDLB_CLOSURE_ONE = 2 };
/* Relaxation frequency: constant 1/tau, or (Sec. 4, omega0 proportional to
 * n g2) tau(r) - 1/2 = (tau - 1/2) n_ref g2(n_ref) / (nbar(r) g2(nbar(r))),
 * clamped to tau >= 0.501. */
enum { WDLB_OMEGA_CONST = 0, WDLB_OMEGA_NBAR = 1 };
/* Population storage: plain FP64 (FP64 arithmetic), FP32 deviation from the
 * node's rest state w_q s(r) (FP32 arithmetic), FP16 relative deviation
 * f_q / (w_q s(r)) - 1 (FP32 arithmetic).  FP16 is accepted for periodic boxes
 * only (WDLB_WALLS_NONE; with walls wdlb_create, wdlb_workspace_size and
 * wdlb_batch_add return WDLB_ERR_ARG): in a driven slit its 10-bit deviations
 * leave steady-state u_x errors of 2 to 15 %, and it is no faster than FP32,
 * whose step is bound by arithmetic, not by HBM. */
enum { WDLB_STORE_F64 = 0, WDLB_STORE_F32 = 1, WDLB_STORE_F16 = 2 };
/* Quadrature of the integral over khat in Eq. campoc (the paper leaves the
 * discrete form open):
 *   FULL     every lattice vector with (sigma-1/2)^2 < |e|^2 <= (sigma+1/2)^2
 *            and one uniform weight w, sigma^2 sum_e w e_z^2/|e| = 4 pi sigma^3/3
 *            (the discrete virial coefficient is b = 2 pi sigma^3/3 exactly);
 *   COMPACT  two or three orbits of the cubic group inside that shell, one
 *            weight per orbit, fixed by the same virial condition, by
 *            sum_e w_e khat_x^2 e_z^2 = 4 pi sigma^2/15 (the continuum value of
 *            the moment behind the collisional viscosity) and by
 *            sum_e w_e khat_z^2 e_z^2 = 3 sum_e w_e khat_x^2 e_z^2 (isotropic
 *            fourth moment), every weight positive; of all such unions the one
 *            with the fewest vectors (26 to 42 for sigma 3 to 8, against 98 to
 *            762), then the smallest sum of (|e|^2 - sigma^2)^2, then the first
 *            in orbit order (|e|^2, then sorted components).  No such union
 *            exists below sigma = 1.55 or for 2.25 <= sigma <= 2.3: wdlb_create
 *            then fails with WDLB_ERR_ARG.  The compact shell changes the
 *            discrete equations (not the equation of state or the long-wave
 *            shear viscosity, which it reproduces at the continuum values). */
enum { WDLB_SHELL_FULL = 0, WDLB_SHELL_COMPACT = 1 };

typedef struct {
    int32_t closure;          /* WDLB_CLOSURE_*, default CS                          */
    int32_t omega_mode;       /* WDLB_OMEGA_*, default CONST                         */
    int32_t storage;          /* WDLB_STORE_*, default F32                           */
    int32_t interactions;     /* 1: fields C and A on (default); 0: plain BGK + g    */
    double k_cross;           /* K: the A-term carries K * traceless(A) in its second
                                 moment; 2 reproduces Eq. extrapressure (default)    */
    double n_ref;             /* reference density (storage offset, NBAR mode);
                                 0: mean fluid density of the initial state          */
    void *workspace;          /* caller-owned device buffer of at least
                                 wdlb_workspace_size bytes, 256-byte aligned, valid
                                 until wdlb_destroy; NULL: the library allocates     */
    uint64_t workspace_bytes; /* size of workspace                                   */
    void *stream;             /* cudaStream_t for all work; NULL: the library creates
                                 (and destroys) its own non-blocking stream          */
    int32_t tile;             /* shape of the shared-memory tiled shell kernel (FP32
                                 and FP16 storage, CS closure, sigma 3, 4 or 6):
                                 -1 (default) chosen by the autotuner, 0 8x8x8 bricks
                                 on 256 threads, 1 8x8x8 on 512 threads, 2 8x8x4 on
                                 256 threads (WDLB_TILE_*)                          */
    int32_t autotune;         /* with tile = -1: 1 (default) time the tile variants on
                                 a scratch lattice the first time a (storage, sigma,
                                 walls, nz, shell rule) key is seen; 0 use the
                                 built-in table                                     */
    int32_t shell_rule;       /* WDLB_SHELL_*, default FULL                          */
    int32_t staging;          /* how the tiled shell kernel stages its field tile:
                                 WDLB_STAGING_AUTO (default) one TMA box per array
                                 for bricks whose tile needs no periodic wrap, where
                                 the halo allows it (sigma 4, nx a multiple of 4),
                                 per-node cp.async copies elsewhere;
                                 WDLB_STAGING_CP_ASYNC per-node copies everywhere.
                                 Both give bitwise the same tile                     */
    int32_t wait_limit;       /* polls of the TMA tile's wait before the kernel gives
                                 up, reports WDLB_ERR_TIMEOUT and skips the brick
                                 (0: the default, about a million tries, each of
                                 which may suspend the thread briefly in
                                 hardware).  Negative values are for tests of that
                                 path: the kernel then issues no copy and waits on
                                 a barrier that nothing completes, for -wait_limit
                                 polls; the step's results are then not meaningful */
    int32_t persistent;       /* batches: 0 (default) one launch per phase (moments,
                                 smeared density, shell) for all pores, replayed from
                                 CUDA graphs; 1 one persistent kernel per
                                 wdlb_batch_step call in which each pore's phases
                                 follow one another without device-wide barriers
                                 (used where every pore runs the tiled sigma-4 kernel
                                 on 8 x 8 x 4 bricks, else the default).  Both give
                                 bitwise the same results                            */
    int32_t collision;        /* arithmetic of the collision and push (step 3 of
                                 Sec. 5, Eq. SMDB) with FP32 storage:
                                 WDLB_COLLISION_FP32 (default) FP32; with walls
                                 the momentum of its changes along the walls is
                                 summed in double-word arithmetic and restored
                                 (FP32 roundings otherwise lose momentum, and in
                                 a driven slit, where each step changes it by a
                                 fraction ~ nu/H^2 of itself, bias the steady
                                 flow by up to ~6e-5 of max|u_x| at H = 159;
                                 restored, ~5e-6);
                                 WDLB_COLLISION_DW the whole collision in
                                 double-word pairs of floats (~48-bit
                                 significands on the FP32 units), the result
                                 rounded to FP32 once, at the store (~5e-6 too).
                                 Lattices with walls and FP32 storage only
                                 (WDLB_ERR_ARG otherwise; periodic boxes meet
                                 1e-5 in FP32)                                   */
} wdlb_options;
enum { WDLB_STAGING_AUTO = 0, WDLB_STAGING_CP_ASYNC = 1 };
enum { WDLB_COLLISION_FP32 = 0, WDLB_COLLISION_DW = 1 };

enum { WDLB_TILE_AUTO = -1, WDLB_TILE_8x8x8 = 0, WDLB_TILE_8x8x8_WIDE = 1, WDLB_TILE_8x8x4 = 2 };

/* Fill *opt with the defaults above.  opt must not be NULL. */
void wdlb_default_options(wdlb_options *opt);

/* Device bytes the context needs for this lattice and options (populations
 * double-buffered, field arrays, staging and reduction scratch).  No GPU call. */
wdlb_status wdlb_workspace_size(wdlb_lattice lat, double sigma, int32_t walls,
                                const wdlb_options *opt, uint64_t *bytes);

/* Create a context for one lattice (Sec. 5: cubic lattice, D3Q19).
 *   lat    nx, ny >= 1; nz >= 3 with walls, >= 1 without; N < 2^31.
 *   sigma  hard-sphere diameter in lattice units, 1 <= sigma <= 8.
 *   walls  WDLB_WALLS_NONE (periodic box) or WDLB_WALLS_Z (slit: solid planes
 *          z = 0 and z = nz-1, fluid in between; hydrodynamic width nz - 2).
 *   tau    BGK relaxation time, tau > 0.5 (omega0 = 1/tau of Eq. relaxationtime).
 *   g      external acceleration F/m of Eq. uno (3 doubles, host memory).
 *   opt    options or NULL for defaults.
 * On success *out owns the device memory (or uses opt->workspace).  The state
 * is undefined until wdlb_init_fields. */
wdlb_status wdlb_create(wdlb_lattice lat, double sigma, int32_t walls, double tau,
                        const double g[3], const wdlb_options *opt, wdlb_ctx **out);

/* Step 1 of the algorithm of Sec. 5: populations set to the discrete local
 * equilibrium of density n and velocity u (host arrays of N and 3N doubles;
 * u may be NULL for rest).  Density at solid nodes is ignored.  Synchronous. */
wdlb_status wdlb_init_fields(wdlb_ctx *ctx, const double *n, const double *u);

/* Same with device arrays (d_n: N doubles, d_u: 3N doubles or NULL), enqueued
 * on the context stream. */
wdlb_status wdlb_init_fields_device(wdlb_ctx *ctx, const double *d_n, const double *d_u);

/* Steps 2-5 of the algorithm of Sec. 5, nsteps >= 0 times.  Asynchronous on
 * the context stream (captured in a CUDA graph for repeated step counts). */
wdlb_status wdlb_step(wdlb_ctx *ctx, int64_t nsteps);

/* Step 4 of Sec. 5 / Eq. colonna: density n (N doubles) and field velocity v
 * (3N doubles) of the current populations into host arrays (either may be
 * NULL).  v is the velocity the next step's fields use: the lagged
 * linear-implicit predictor of the second-order velocity u = (j + F/2)/n,
 *   (1 + H) v = j/n + g/2 + C_prev/(2n) + H v_prev,
 *   H = (kappa beta / 6) t_prev,  t = sum_e w g2 n(r+e),  kappa = 2,
 *   beta = 2 sigma^2 sqrt(kT/pi),
 * equal to u at a steady state.  Solid nodes report 0.  Synchronous. */
wdlb_status wdlb_moments(wdlb_ctx *ctx, double *n, double *u);

/* Same into device arrays, enqueued on the context stream. */
wdlb_status wdlb_moments_device(wdlb_ctx *ctx, double *d_n, double *d_u);

/* Intermediate fields of the current state (step 2 of Sec. 5), host arrays,
 * any may be NULL: nbar (N), C (3N, Eq. campoc), A (6N: xx, yy, zz, xy, xz, yz,
 * Eq. campod, before removing its trace), u (3N, the collision velocity
 * (j + F/2)/n with F = n g + C).  Does not advance the state.  Synchronous;
 * allocates temporary device memory for its FP64 outputs. */
wdlb_status wdlb_fields(wdlb_ctx *ctx, double *nbar, double *C, double *A, double *u);

/* Energy-equation fields of Sec. 3 on a prescribed temperature field, from
 * the current state (its n, field velocity v and smeared density, with the
 * shell quadrature and contact values of C and A):
 *   Q    (N)  = T n sigma^2 sum_e w g2 n(r+e) [-khat.(v(r+e)-v(r))/2
 *                                             + sqrt(T/pi) (T(r+e)-T(r))/T]   (Eq. campob1)
 *   B    (3N) = -2 T n sigma^2 sum_e w khat g2 n(r+e) (T(r+e)-T(r))           (Eq. campos)
 *   FT   (3N) = -(sigma^2/2) sum_e w khat g2 n(r+e) (T(r+e)-T(r))             (Eq. thermalforce)
 * T: N doubles on the host, k_B T per node in lattice units (m = 1), finite
 * and positive on fluid nodes (values on solid planes are ignored); outputs
 * are host arrays (any may be NULL), zero on solid nodes, computed in FP64
 * from the state's storage precision.  The time step itself is isothermal
 * (Sec. 5: k_B T = 1/3 in C and A) and no temperature is evolved; this
 * evaluates the fields of the paper's energy equation on a given T.  Does not
 * advance the state.  Synchronous; allocates temporary device memory.
 * WDLB_ERR_ARG on a NULL T or a non-positive or non-finite T on a fluid node;
 * WDLB_ERR_STATE before init. */
wdlb_status wdlb_thermal_fields(wdlb_ctx *ctx, const double *T, double *Q, double *B, double *FT);

/* Populations f_q of the current state as FP64 (19N doubles, q-major, in the
 * order of wdlb_velocity_set), solid nodes 0.  Synchronous. */
wdlb_status wdlb_get_populations(wdlb_ctx *ctx, double *f);

/* Checkpoint and resume (no counterpart in the paper).  The state of an
 * initialised context is its populations as stored, the per-node storage
 * scale, the field velocity of the last moments pass (the predictor's v_prev,
 * with n - n_off), C_prev, t_prev, the reference density and the step count;
 * restoring it continues the run bit for bit.  The buffer is an opaque host
 * blob of wdlb_state_bytes bytes, caller-owned, valid for a context with the
 * same lattice, walls, sigma, tau, storage and shell rule (WDLB_ERR_ARG
 * otherwise, and for a buffer that is too small or not a saved state).
 * Synchronous. */
wdlb_status wdlb_state_bytes(const wdlb_ctx *ctx, uint64_t *bytes);
wdlb_status wdlb_save_state(wdlb_ctx *ctx, void *host, uint64_t bytes);
wdlb_status wdlb_load_state(wdlb_ctx *ctx, const void *host, uint64_t bytes);

/* Pore-averaged quantities (abstract: pore-averaged properties), reduced in
 * FP64 on the device over fluid nodes: mean density, mean u_x, flux
 * sum(n u_x)/(nx ny), mass sum(n), eta_eff = <n> g_x H^2 / (12 <u_x>) with
 * H = nz - 2 (NaN without walls), the last steady-state residual (NaN if none)
 * and the step count.  Synchronous. */
typedef struct {
    double mean_n, mean_ux, flux_x, mass, eta_eff, residual;
    int64_t steps;
} wdlb_pore_stats;
wdlb_status wdlb_pore_average(wdlb_ctx *ctx, wdlb_pore_stats *out);

/* Steady-state driver: step in blocks of check_every (>= 1) steps; after each
 * block compute in FP64 the relative change per step of the pore flux
 * Q = sum(n u_x) over fluid nodes, r = |Q(t) - Q(t - check_every)| /
 * (check_every |Q(t)|), and stop when r < tol or after max_steps.  (A max-norm
 * change of u_x stalls near 2e-7 in FP32: rounding jitter next to the walls;
 * the flux averages it out.)  *steps_done and *residual (either may be NULL)
 * report the outcome. */
wdlb_status wdlb_run_steady(wdlb_ctx *ctx, double tol, int32_t check_every, int64_t max_steps,
                            int64_t *steps_done, double *residual);

/* Library tables, host only, no GPU needed.
 * wdlb_velocity_set: the 19 D3Q19 velocities (c: 57 int32, q-major) and
 * weights (w: 19 doubles) in the library's population order.
 * wdlb_stencil: which = 0 the smeared-density ball {b : |b|^2 <= (sigma/2)^2},
 * which = 1 the contact shell {e : (sigma-1/2)^2 < |e|^2 <= (sigma+1/2)^2};
 * writes up to cap vectors (3 int32 each) into vecs (may be NULL), the full
 * count into *count, and for the shell the uniform quadrature weight w with
 * sigma^2 sum_e w (e_z^2/|e|) = 4 pi sigma^3 / 3 into *weight (may be NULL). */
wdlb_status wdlb_velocity_set(int32_t *c, double *w);
wdlb_status wdlb_stencil(double sigma, int32_t which, int32_t *vecs, int32_t cap,
                         int32_t *count, double *weight);
/* The contact shell of a quadrature rule (WDLB_SHELL_*) with the weight of
 * every vector: writes up to cap vectors (3 int32 each, +e and -e adjacent)
 * into vecs and their weights into weights (either may be NULL) and the full
 * count into *count.  WDLB_ERR_ARG if sigma is outside [1, 8], the rule is
 * unknown or it has no shell at this sigma.  Host only, no GPU needed. */
wdlb_status wdlb_shell_table(double sigma, int32_t rule, int32_t *vecs, double *weights, int32_t cap,
                             int32_t *count);

/* Advance nsteps (>= 1) like wdlb_step, but launch the three kernels of each
 * step one by one with CUDA events around each on the context stream, and
 * write the mean device time per launch in milliseconds: ms[0] moments and
 * field velocity, ms[1] smeared density, ms[2] shell sums + collision +
 * streaming.  Synchronous. */
wdlb_status wdlb_profile_step(wdlb_ctx *ctx, int64_t nsteps, double ms[3]);

/* ---- Tile autotuner (no counterpart in the paper: a launch-shape choice) --
 *
 * The tiled shell kernel comes in three shapes (WDLB_TILE_*).  Which one is
 * fastest depends on sigma (shared memory per block, hence blocks per SM) and
 * on nz (z padding of the bricks in thin slits).  Contexts created with
 * tile = -1 take the shape from a process-wide table keyed by (storage,
 * sigma, walls, nz, shell rule).  A missing key is filled by timing every shape on a
 * scratch lattice of that key (nz as given, a square cross-section of about
 * 2^20 / nz nodes so that the kernel fills the GPU as a batch does; uniform
 * density; six steps after two warm-up steps) when autotune = 1, else from a
 * built-in table.  Every shape computes the same arithmetic per node; alone
 * and batched lattices of one key share the table entry, so they run the
 * same kernel.  Thread-safe; the table lives until wdlb_autotune_reset. */

/* Time every tile shape for this key now (replacing its table entry).
 * *best: the fastest shape; ms[3]: milliseconds per time step of each shape's
 * shell kernel (NaN for a shape that cannot run); either may be NULL.
 * WDLB_ERR_ARG if the tiled kernel does not apply to these arguments. */
wdlb_status wdlb_autotune(wdlb_lattice lat, double sigma, int32_t walls, const wdlb_options *opt,
                          int32_t *best, double ms[3]);

/* The shell kernel a context runs: *tiled 1 for the tiled kernel (then
 * *tile is its shape), 0 for the per-node kernel (*tile = -1). */
wdlb_status wdlb_tile_info(const wdlb_ctx *ctx, int32_t *tiled, int32_t *tile);

/* How the context's tiled shell kernel stages its field tile: *tma 1 if
 * bricks whose tile needs no periodic wrap load it as one TMA box per array
 * (sigma 4, FP32/FP16 storage, nx a multiple of 4, staging WDLB_STAGING_AUTO),
 * 0 if every brick copies it node by node.  No counterpart in the paper. */
wdlb_status wdlb_staging_info(const wdlb_ctx *ctx, int32_t *tma);

/* Forget every autotuned entry (later contexts probe again). */
void wdlb_autotune_reset(void);

/* ---- Batches of independent lattices (continuous batching) --------------
 * Many pores of different sizes stepped together: each phase of a time step
 * is one kernel launch for all pores of the batch (one shell launch per group
 * of pores with the same sigma, geometry and tile shape), replayed from a
 * CUDA graph.
 * The kernels are those of the single-lattice path, so a pore's result is the
 * same alone and in a batch.  Pores are admitted by device-memory footprint
 * into a pool of fixed size and removed when done; admission, removal and
 * stepping may interleave freely (continuous batching).
 *
 * opt: options shared by all pores (closure, omega mode, storage,
 * interactions, K); opt->workspace, if set, is the pool (caller-owned,
 * 256-byte aligned, >= pool_bytes), else the library allocates pool_bytes;
 * opt->stream as for wdlb_create.  The batch also allocates small device
 * tables (parameters and work lists of its slots). */
typedef struct wdlb_batch wdlb_batch;
typedef struct {
    wdlb_lattice lat;
    double sigma;
    int32_t walls;
    double tau;
    double g[3];
} wdlb_pore_desc;

wdlb_status wdlb_batch_create(const wdlb_options *opt, uint64_t pool_bytes, int32_t max_pores,
                              wdlb_batch **out);
/* Pool bytes one pore of this description occupies. */
wdlb_status wdlb_batch_pore_bytes(const wdlb_batch *b, const wdlb_pore_desc *d, uint64_t *bytes);
/* Admit a pore with initial fields n (N doubles), u (3N doubles or NULL) on the
 * host (step 1 of Sec. 5); *slot receives its slot.  WDLB_ERR_OOM if no slot
 * or not enough contiguous pool memory is free (nothing changed). */
wdlb_status wdlb_batch_add(wdlb_batch *b, const wdlb_pore_desc *d, const double *n, const double *u,
                           int32_t *slot);
/* Release a pore and its pool memory. */
wdlb_status wdlb_batch_remove(wdlb_batch *b, int32_t slot);
/* Steps 2-5 of the algorithm of Sec. 5 for every pore, nsteps times (async). */
wdlb_status wdlb_batch_step(wdlb_batch *b, int64_t nsteps);
/* nsteps time steps of every pore of the batch, launched kernel by kernel
 * (moments, smeared density, every shell group) with CUDA events around each
 * phase on the batch stream; ms[0..2] = average device time per step of each
 * phase.  Same kernels, order and results as wdlb_batch_step; blocks until done.
 * For measurement (no counterpart in the paper). */
wdlb_status wdlb_batch_profile_step(wdlb_batch *b, int64_t nsteps, double ms[3]);
/* Per slot (array of max_pores): the FP64 steady-state residual of
 * wdlb_run_steady, |Q - Q(previous call)| / (interval |Q|) with Q the pore flux
 * (+inf at a pore's first call, NaN for empty slots), and the slot status
 * (WDLB_OK, WDLB_ERR_UNSTABLE, WDLB_ERR_CUDA for the checked build's index
 * flag, -1 empty); either array may be NULL.
 * Synchronous. */
wdlb_status wdlb_batch_residuals(wdlb_batch *b, int32_t interval, double *res, int32_t *status);
/* The context of a slot (owned by the batch): use it for wdlb_moments,
 * wdlb_pore_average, wdlb_fields, wdlb_get_populations; do not step or
 * destroy it.  NULL for an empty slot. */
wdlb_ctx *wdlb_batch_context(wdlb_batch *b, int32_t slot);
int32_t wdlb_batch_active(const wdlb_batch *b);
uint64_t wdlb_batch_free_bytes(const wdlb_batch *b);
int64_t wdlb_batch_launch_count(const wdlb_batch *b);
const char *wdlb_batch_last_error(const wdlb_batch *b);
void wdlb_batch_destroy(wdlb_batch *b);

/* ---- Serving: continuous batching of steady-state solves ----------------
 * Requests (a pore, its initial fields and a steady-state tolerance) arrive
 * at any time from any thread.  A worker thread of the server admits queued
 * requests into a batch while the HBM budget (the batch pool) has room, steps
 * all admitted pores together in blocks of check_every steps, tests each
 * pore's FP64 residual (as wdlb_run_steady) after every block, and retires
 * converged pores (status WDLB_OK), pores that reach max_steps
 * (WDLB_ERR_TIMEOUT) or become non-physical (WDLB_ERR_UNSTABLE); a pore larger
 * than the whole budget is rejected (WDLB_ERR_OOM).  Each request's result is
 * the same as solving it alone with wdlb_run_steady(tol, check_every). */
typedef struct wdlb_server wdlb_server;
typedef struct {
    wdlb_pore_desc desc;
    const double *n, *u;      /* initial fields (host; copied by submit; u may be NULL) */
    double tol;               /* steady-state tolerance (> 0)                        */
    int64_t max_steps;        /* give up after this many steps (>= 1)                */
    double *out_n, *out_u;    /* optional host buffers (N, 3N doubles) for the final
                                 moments; valid until the result is polled           */
} wdlb_request;
typedef struct {
    int64_t id;
    int32_t status;
    int64_t steps;
    double residual;
    double submit_s, start_s, finish_s;   /* server clock (seconds since creation) */
    wdlb_pore_stats stats;
} wdlb_result;
typedef struct {
    int64_t submitted, admitted, completed, queued, active;
    uint64_t pool_free;
    int64_t launches;
    double clock_s;
    int64_t node_steps;       /* lattice-node updates executed so far */
    double gpu_step_s;        /* device time of the worker's blocks of time steps
                                 (CUDA events on the batch's stream; the rest of
                                 clock_s is admission, residual tests, retiring
                                 and idle time)                                   */
} wdlb_server_stats;

/* opt as for wdlb_batch_create, except that opt->autotune is taken as 0: the
 * worker thread never runs a tile probe, its pores take the autotuner's table
 * as it stands (call wdlb_autotune first to probe keys); hbm_budget: pool
 * bytes for admitted pores; max_active: slots; check_every: steps between
 * residual tests.  Starts the worker thread on the current device. */
wdlb_status wdlb_server_create(const wdlb_options *opt, uint64_t hbm_budget, int32_t max_active,
                               int32_t check_every, wdlb_server **out);
/* Queue a request (thread-safe, returns at once); *id identifies its result. */
wdlb_status wdlb_server_submit(wdlb_server *s, const wdlb_request *r, int64_t *id);
/* Move up to cap finished results into out; returns how many. */
int32_t wdlb_server_poll(wdlb_server *s, wdlb_result *out, int32_t cap);
/* Counters of the server (thread-safe).  active, pool_free and launches are
 * the batch's values as the worker thread last published them (after each
 * admission round and each block of steps); the worker owns the batch, and
 * this call never reads it. */
wdlb_status wdlb_server_info(wdlb_server *s, wdlb_server_stats *info);
/* Stop the worker (unfinished requests are dropped) and free everything. */
void wdlb_server_destroy(wdlb_server *s);

/* ---- Fields without any device allocation --------------------------------
 * No counterpart in the paper: an entry point for callers that cannot
 * allocate device memory (code that runs inside another framework's memory
 * pool, plugin hosts that forbid cudaMalloc, processes whose device footprint
 * must not grow after start-up).  It computes what wdlb_fields computes for a
 * state at rest with respect to its own history -- the smeared density nbar,
 * C (Eq. campoc) and A (Eq. campod) with the neighbours' velocity u -- from
 * device arrays n (N doubles) and u (3N doubles), into device arrays nbar (N,
 * may be NULL), C (3N) and A (6N: xx, yy, zz, xy, xz, yz), FP32 arithmetic,
 * with the full contact shell (WDLB_SHELL_FULL).  Solid nodes (walls) report 0.
 *
 * Its scratch is one file-scope __device__ array of fixed size (about 5 MiB:
 * the field arrays for WDLB_STATIC_MAX_NODES nodes, the stencil tables and a
 * reduction slot) that every GPU which loads the library holds until the
 * process exits; the call allocates and frees nothing.  Lattices with more
 * than WDLB_STATIC_MAX_NODES nodes, or sigma outside [1, 8], are rejected with
 * WDLB_ERR_ARG.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) on the current device and keeps it for the
 * later calls on that device.  The kept address belongs to the device's
 * current context: after a cudaDeviceReset it is no longer valid.  All work is enqueued on `stream` (a
 * cudaStream_t, NULL = legacy default stream); the stencil tables are copied
 * from pageable host memory.  The call then waits for its work on `stream` to
 * finish and reads back the status word its kernels set in the array:
 *   WDLB_OK            nbar, C and A are written;
 *   WDLB_ERR_UNSTABLE  the state is not physical: a smeared packing fraction
 *                      >= 1, a negative or non-finite density or a non-finite
 *                      velocity at a fluid node (the outputs are not meaningful);
 *   WDLB_ERR_CUDA      a CUDA call failed, or (bounds-checked build only) a
 *                      kernel index left its array and the access was skipped.
 * Every call shares the one array and the array keeps the last call's
 * contents (the status word is cleared at the start of each call): calls that
 * overlap on the GPU (other streams, other host threads) race on it and must
 * be serialised by the caller. */
#define WDLB_STATIC_MAX_NODES 262144
wdlb_status wdlb_fields_static(wdlb_lattice lat, double sigma, int32_t walls, int32_t closure,
                               const double *d_n, const double *d_u, double *d_nbar, double *d_C,
                               double *d_A, void *stream);

/* Number of kernels this context has launched so far (a graph replay counts
 * the kernels it contains). */
int64_t wdlb_launch_count(const wdlb_ctx *ctx);

/* Human-readable message of the last error of ctx ("" if none; ctx may be NULL
 * for errors of wdlb_create). */
const char *wdlb_last_error(const wdlb_ctx *ctx);

/* Release the context and its device memory (not a caller workspace).
 * NULL-safe.  Synchronises the context stream first. */
void wdlb_destroy(wdlb_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* WDLB_H */
