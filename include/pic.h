/*
 * pic.h -- C ABI of the GB300 (sm_103a) electromagnetic particle-in-cell
 * timestep library.
 *
 * One timestep (Fonseca et al., Sec. 2 and Sec. 5.2 steps i-v):
 *   gather E and B at each particle with order-p B-spline weights, each
 *   component at its own Yee location (Sec. 5.1, Sec. 5.2 step ii);
 *   relativistic Boris push of u = gamma*beta (Sec. 2, Sec. 5.2 step iii);
 *   position update on an integer cell index plus an FP32 offset from the
 *   cell's lower vertex (Sec. 5.1);
 *   charge-conserving current deposit on the straight segment (Sec. 5.2,
 *   Esirkepov's decomposition);
 *   Yee FDTD update B(1/2) -> E -> B(1/2) (Sec. 2; Sec. 3: a local field
 *   solver).
 * Normalised units, c = 1: dE/dt = curl B - J, dB/dt = -curl E, div E = rho.
 * Lengths in c/omega, fields in m c omega / e, charge and mass in units of
 * the electron's magnitude.  A particle's weight w is a density (n / ppc):
 * rho(node) = sum q w S(x - node).
 *
 * Layout conventions shared by every call:
 *   axis 0 is the fastest in memory; field arrays are component arrays of
 *   n0*n1*n2 FP32 values, idx = i + n0*(j + n1*k) (n2 = 1 in 2D);
 *   Yee locations in cells: Ex (1/2,0,0) Ey (0,1/2,0) Ez (0,0,1/2)
 *   Bx (0,1/2,1/2) By (1/2,0,1/2) Bz (1/2,1/2,0); in 2D the third axis is
 *   absent and Ez, Jz sit on nodes;
 *   the last axis is the propagation axis of the laser and of the moving
 *   window; it may be open (Mur fields, absorbing particles); the other axes
 *   are periodic;
 *   particle arrays are component-major: cell[dim][n], off[dim][n],
 *   u[3][n], w[n], id[n].
 *
 * Ownership: the library owns all device memory, allocated at pic_create /
 * first load through the caller's allocator when one is given (else
 * cudaMalloc).  Host pointers passed in are borrowed for the duration of the
 * call only.  The CUDA stream is borrowed; every device operation of a
 * handle is ordered on it.  One handle is used by one host thread at a time.
 *
 * Errors: every int-returning call returns PIC_OK (0) or a negative PIC_E*
 * code and never aborts.  Conditions detected on the device (capacity
 * overflow, a bounded wait that gave up) are latched in a device status word
 * and returned by the next pic_sync / pic_diagnostics / read call.
 */
#ifndef PIC_GB300_H
#define PIC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_ABI_VERSION 1

/* exported entry points (the library is built with hidden visibility) */
#if defined(__GNUC__)
#define PIC_API __attribute__((visibility("default")))
#else
#define PIC_API
#endif

#define PIC_OK 0
#define PIC_EINVAL (-1)    /* bad argument or configuration (Courant >= 1, bad order, bits) */
#define PIC_ENOMEM (-2)    /* allocation failed */
#define PIC_ECUDA (-3)     /* a CUDA runtime call failed */
#define PIC_EOVERFLOW (-4) /* particle capacity exceeded (no trap; work dropped and latched) */
#define PIC_ETIMEOUT (-5)  /* a bounded device wait gave up */
#define PIC_ESTATE (-6)    /* call not valid in the handle's current state */

#define PIC_BC_PERIODIC 0
#define PIC_BC_OPEN 1 /* last axis only: first-order Mur fields, absorbing particles */

/* field selectors for pic_read_fields / pic_write_fields */
#define PIC_EX 0
#define PIC_EY 1
#define PIC_EZ 2
#define PIC_BX 3
#define PIC_BY 4
#define PIC_BZ 5
#define PIC_JX 6
#define PIC_JY 7
#define PIC_JZ 8
#define PIC_RHO 9 /* charge density of the particles (computed on read) */

/* Grid: dim = 2 or 3; n cells per axis (n[2] ignored in 2D); d cell sizes;
 * dt must satisfy the Yee Courant condition dt * sqrt(sum 1/d^2) < 1
 * (Sec. 2: the time step is set by the Courant limit of the field
 * solver).  bc_last: PIC_BC_PERIODIC or PIC_BC_OPEN. */
typedef struct {
    int32_t dim;
    int32_t n[3];
    double d[3];
    double dt;
    int32_t bc_last;
    int32_t reserved;
} pic_grid;

/* One mobile species (immobile neutralising ions are implied: the initial
 * electron charge is the background).  ppc and the density profile are used
 * for plasma injected by the moving window: ppc[a] particles per axis at
 * offsets (m + 1/2)/ppc[a], cold, weight density(z_lab)/prod(ppc).
 * density(z) is piecewise linear through n_knots equally spaced knots over
 * [profile_z0, profile_z1] (clamped outside), or the constant `density` when
 * n_knots == 0.  per_particle_weight = 1 makes pic_load_particles require w;
 * otherwise every particle carries weight w_const. */
typedef struct {
    double q, m;
    int32_t ppc[3];
    int32_t per_particle_weight;
    double w_const;
    double density;
    const double *profile_knots;
    int32_t n_knots;
    int32_t reserved;
    double profile_z0, profile_z1;
} pic_species;

/* Laser antenna (Sec. 2 laser driver): one-way plane source at node `plane`
 * of the last axis, polarised along `pol_axis` (0 in 2D), travelling towards
 * +last axis: E_inc = a0 exp(-r^2/waist^2) exp(-2 ln2 (xi - t_peak)^2/fwhm^2)
 * cos(omega0 (xi - t_peak)), xi = t - (z - z_plane), r from the box axis.
 * Active until the moving window first shifts. */
typedef struct {
    int32_t enabled;
    int32_t pol_axis;
    int32_t plane;
    int32_t reserved;
    double a0, omega0, waist, fwhm, t_peak;
} pic_laser;

/* Moving window along the last axis (Sec. 2): once t >= t_start the box
 * shifts one cell back whenever velocity * (t - t_start) passes the next
 * multiple of d[last]; the new front layer is injected with plasma. */
typedef struct {
    int32_t enabled;
    int32_t reserved;
    double velocity, t_start;
} pic_window;

/* Allocator hooks (e.g. the PyTorch caching allocator).  alloc returns a
 * device pointer of at least `bytes` (16-byte aligned) or NULL. */
typedef void *(*pic_alloc_fn)(size_t bytes, void *ctx);
typedef void (*pic_free_fn)(void *ptr, void *ctx);

/* Tuning: tile[a] cells per tile per axis (powers of two, 0 = default);
 * sort_interval: steps between tile sorts under the fixed policy (0 =
 * default, 4), the longest interval under the adaptive one (0 = default,
 * 32); sort_policy: 0 = adaptive (default): each step the device sorts a
 * run when sort_interval steps have passed since its last sort or when its
 * push has sent, summed over the steps since that sort, at least 1/65536 of
 * its particles down the slow path from their tiles (particles outside their
 * tile's staged region, each of which stalls its warp; the unsorted tail that
 * the moving window injects is not counted); 1 = fixed: every sort_interval
 * steps.  The adjoint form always uses the fixed schedule (every
 * sort_interval steps, default 4), so that a recomputed segment repeats the
 * forward run's sorts.  drift: cells a
 * particle may stray outside its tile between sorts and still use the
 * staged fast path (-1 = default); block: threads per tile CTA, 128, 256, 384
 * or 512 (0 = default);
 * persistent: 0 = default (persistent for batches, one CTA per tile
 * otherwise), 1 = one persistent grid whose CTAs take tiles from a device
 * work queue, largest runs first, 2 = one CTA per tile.
 * Compiled (tile, drift) pairs: 2D 16x16 with drift 1, 2 (default) or 3,
 * 8x8 with 1, 32x32 with 2; 3D 8x8x8 with 1 (default) or 2, 8x8x4 with 1; any other pair
 * is PIC_EINVAL.  Shape order 4: 2D 16x16 with drift 2, 3D 8x8x8 with drift 1 only.
 * use_graph: capture each step kind in a CUDA graph and replay it.
 * sort_sub: sub-buckets per tile in the sort, 0 = default (1 = none),
 * else a power of two <= 32 (with sort_rows = 0 or 2): slot i of a tile's
 * particles goes to sub-bucket i mod sort_sub, so that the particles one
 * warp pushes together come from different cells.
 * tma: 1 = stage the 3D field tile with the tensor-memory accelerator (the
 * entry 8x8x8 with drift 1, whose tile rows are then 16-byte aligned TMA
 * box rows), 0 = default (plain loads into the bank-padded tile).
 * adjoint_keep: checkpoint segments whose per-step records the forward run
 * keeps, so that the reverse sweep recomputes only the others: 0 = default
 * (as many as 75 % of the free device memory holds), -1 = none (every
 * segment recomputed), n = at most n.
 * stream_zero_tiles: 0 = default (1), 1 = each step, classify the tiles on
 * the device: a tile whose staged field region is all +0 (E = B = 0 at every
 * particle, as ahead of a laser front) is advanced by a streaming kernel
 * without shared-memory tiles, the others by the staged kernel; 2 = every
 * tile through the staged kernel.
 * deposit: 0 = default: Esirkepov's decomposition on the whole straight move;
 * 1 = virtual trajectories (Sec. 5.2 step iv): the move is cut where it
 * crosses a boundary between the grid points nearest the particle (half-
 * integer positions for even orders, cell faces for odd ones) and each piece
 * is deposited on its own; for linear shapes this is Villasenor and
 * Buneman's scheme.  Compiled for the default tile of each dimension, orders
 * 1-3, without TMA staging (otherwise PIC_EINVAL).
 * j_layout: 0 = default: the current as three component arrays; 1 = one
 * array of four-component nodes (x, y, z, unused; Sec. 5.1), each tile's
 * current added to it by one 16-byte vector atomic per node.  Reads of
 * PIC_JX..PIC_JZ return the same values either way.
 * sort_rows: 0 = default (1 unless sort_sub > 1), 1 = the sort groups each
 * tile's particles by row of cells along x (their y and z cell in the
 * tile), so that the particles one warp pushes together lie in one or two
 * rows and share field-tile addresses; 2 = no order inside a tile.  Only the
 * assignment of particles to threads changes.
 * quiet_tiles (with stream_zero_tiles on): the field update and the J reset
 * skip the tiles whose E, B and J stay +0 through the step (no fields within
 * twice a tile's deposit reach after the last step, no slow-path deposit in
 * reach, no antenna plane in reach) and walk the others as a list: 0 =
 * default (on for handles of at least 2^22 cells), 1 = on, 2 = off.  The
 * result is the same either way. */
typedef struct {
    int32_t tile[3];
    int32_t sort_interval;
    int32_t drift;
    int32_t block;
    int32_t use_graph;
    int32_t persistent;
    int32_t sort_sub;
    int32_t tma;
    int32_t adjoint_keep;
    int32_t sort_policy;
    int32_t stream_zero_tiles;
    int32_t deposit;
    int32_t j_layout;
    int32_t sort_rows;
    int32_t quiet_tiles;
} pic_tuning;

typedef struct {
    int32_t abi_version; /* PIC_ABI_VERSION */
    int32_t shape_order; /* B-spline order 1, 2, 3 or 4 (Table 3 varies it); order 4 with
                            the default tile and drift of each dimension, no TMA staging
                            and no adjoint form */
    pic_grid grid;
    int32_t n_species;   /* must be 1 */
    int32_t track_ids;   /* 1: keep a per-particle int32 id through sorts: the n loaded
                            particles 0 .. n-1 in load order, the k-th window shift's
                            layer of m particles n + (k-1) m + j (-1 past 2^31 - 1) */
    const pic_species *species;
    pic_laser laser;
    pic_window window;
    uint64_t seed;
    int64_t capacity;    /* particle slots, allocated by pic_create (two buffers; PIC_ENOMEM
                            there if they do not fit); 0 = 1.25x the first load + injection
                            room, allocated by the first pic_load_particles */
    pic_tuning tuning;
    pic_alloc_fn alloc;  /* NULL: cudaMalloc */
    pic_free_fn free;
    void *alloc_ctx;
    void *stream;        /* cudaStream_t, borrowed; NULL = default stream */
} pic_config;

typedef struct {
    int64_t step;
    double time;
    int64_t shifts;        /* moving-window shifts so far */
    double W_E, W_B;       /* 1/2 sum E^2 V, 1/2 sum B^2 V at integer time */
    double W_kin;          /* V sum w m (gamma - 1), gamma from u^{n-1/2} */
    double gauss_resid;    /* max|div E - (rho - rho_0)| / max|rho_0| */
    int64_t n_particles;   /* live particles */
    double imbalance;      /* max / mean particles per occupied tile (Sec. 3) */
    int64_t slow_path;     /* particles outside their tile's staged region, last step */
    int32_t status;        /* latched device status (PIC_OK or a PIC_E* code) */
    int32_t sorts;         /* tile sorts so far */
    int64_t streamed;      /* particle slots advanced by the zero-field tile kernel, all steps so far */
    int64_t live_tiles;    /* non-empty tiles advanced by the staged kernel, all steps so far (with
                              the zero-field tiles streamed; 0 otherwise) */
} pic_diag;

typedef struct pic_s pic_t;

/* Validate `cfg`, allocate grid and state, zero the fields.  *out receives
 * the handle.  Errors: PIC_EINVAL (Courant, order, dims not encodable in the
 * packed cell index, unsupported species count), PIC_ENOMEM, PIC_ECUDA. */
PIC_API int pic_create(const pic_config *cfg, pic_t **out);

/* Batched form: n independent runs of equal dim and shape order advanced
 * together, each kernel phase covering every run's tiles in one launch.
 * The other calls address run 0 until pic_select_run chooses another. */
PIC_API int pic_create_batch(const pic_config *cfgs, int32_t n, pic_t **out);
PIC_API int pic_select_run(pic_t *h, int32_t run);
PIC_API int32_t pic_num_runs(const pic_t *h);

/* Append n particles of `species` (0) to the current run.  cell[dim][n]:
 * cell index per axis in [0, n_a); off[dim][n]: FP32 offset in [0, 1) from
 * the cell's lower vertex (Sec. 5.1); u[3][n]: gamma*beta; w[n]: weights
 * (required iff per_particle_weight, else ignored and may be NULL).  Host
 * pointers.  Particles are sorted into tiles before the next step.
 * Errors: PIC_EINVAL (index out of range), PIC_EOVERFLOW (capacity), PIC_ESTATE
 * (after the first step). */
PIC_API int pic_load_particles(pic_t *h, int32_t species, int64_t n, const int32_t *cell, const float *off,
                       const float *u, const float *w);

/* Enqueue nsteps timesteps of every run on the handle's stream; returns
 * without waiting.  Device-side conditions are latched (see pic_sync). */
PIC_API int pic_step(pic_t *h, int32_t nsteps);

/* Wait for the handle's stream and return the latched device status. */
PIC_API int pic_sync(pic_t *h);

/* Copy field `which` of the current run into dst (n_elems >= n0*n1*n2),
 * ordered in the window frame (index 0 of the last axis = rear of the
 * window).  on_device: dst is a device pointer (else host).  PIC_RHO is the
 * current particles' charge density.  Synchronises the stream. */
PIC_API int pic_read_fields(pic_t *h, int32_t which, float *dst, size_t n_elems, int32_t on_device);

/* Overwrite field `which` (E or B components only) of the current run from
 * src (window-frame order, n_elems = n0*n1*n2); on_device as above. */
PIC_API int pic_write_fields(pic_t *h, int32_t which, const float *src, size_t n_elems, int32_t on_device);

/* Copy the live particles of the current run to host arrays: cell[dim][cap],
 * off[dim][cap], u[3][cap], w[cap], id[cap] (id only with track_ids; any
 * pointer may be NULL to skip it).  Cell indices are in the window frame.
 * *n receives the count; PIC_EOVERFLOW if it exceeds cap (nothing copied). */
PIC_API int pic_read_particles(pic_t *h, int32_t species, int32_t *cell, float *off, float *u, float *w,
                       int32_t *id, int64_t cap, int64_t *n);

/* Compute diagnostics of the current run (synchronises the stream). */
PIC_API int pic_diagnostics(pic_t *h, pic_diag *out);

/* Phase timing with CUDA events recorded on the handle's stream around each
 * phase of every step (steps then run without graph replay).
 * pic_profile_begin(h, max_steps) arms it for up to max_steps steps;
 * pic_profile_end(h, ms, n_phases, launches) synchronises and writes the
 * summed milliseconds of each phase into ms[0..n_phases) in the order
 * PIC_PH_* below, and the number of kernels the profiled steps launched into
 * *launches. */
#define PIC_PH_SORT 0
#define PIC_PH_ZERO_J 1
#define PIC_PH_PUSH 2
#define PIC_PH_YEE_B1 3
#define PIC_PH_YEE_E 4 /* includes the Mur save/apply */
#define PIC_PH_YEE_B2 5
#define PIC_PH_WINDOW 6 /* end-of-step bookkeeping, window shift and injection */
#define PIC_PH_PUSH_ZERO 7 /* the zero-field tiles' streaming kernel: a part of PIC_PH_PUSH */
#define PIC_NUM_PHASES 8
PIC_API int pic_profile_begin(pic_t *h, int32_t max_steps);
PIC_API int pic_profile_end(pic_t *h, double *ms, int32_t n_phases, int64_t *launches);

/* ---- adjoint form --------------------------------------------------------
 * Gradients of a final-state objective through the timestep, by the
 * discrete adjoint (reverse mode of the FP32 forward arithmetic) with step
 * checkpointing and segment recomputation.  Objective (a smooth "trailing
 * window" of the last axis, positions in window-frame cells):
 *   L = sum w K sigma / sum w sigma,  K = m (gamma - 1),
 *   sigma(z) = logistic((z - z_lo)/width) * logistic((z_hi - z)/width).
 * Requirements: a single run, track_ids = 1, per_particle_weight = 1, shape
 * order 1-3 with the default deposit, particles loaded, no step taken yet.
 * With a moving window the gradient includes the plasma the window injects
 * (its weights follow the density knots at the lab position of injection);
 * the forward run's ids then also number the injected particles: the k-th
 * shift's layer (k = 1, 2, ...) gets ids n + (k - 1) m .. n + k m - 1, n the
 * loaded particles, m the particles of one layer. */
typedef struct {
    double z_lo, z_hi, width;
} pic_objective;

/* Arm the reverse mode for a forward run of total_steps steps: allocates the
 * adjoint arrays, ceil(total/checkpoint_every) checkpoints (particle state and
 * E, B) and one segment of per-step records; the following pic_step calls
 * save a checkpoint every checkpoint_every steps (copied between step graph
 * replays; the recomputation inside pic_adjoint_backward runs without graphs
 * because it records each step). */
PIC_API int pic_adjoint_begin(pic_t *h, int32_t total_steps, int32_t checkpoint_every);

/* Checkpoint segments whose records the forward run keeps (see
 * pic_tuning.adjoint_keep), after pic_adjoint_begin; negative on error. */
PIC_API int pic_adjoint_kept(pic_t *h);

/* L of the current state (no adjoint). */
PIC_API int pic_objective_value(pic_t *h, const pic_objective *obj, double *L);

/* After exactly total_steps forward steps: L, dL/da0 (laser amplitude),
 * dL/dknots[n_knots] (the piecewise-linear density profile of pic_species:
 * w = density(z at load or injection) / prod(ppc)) and dL/dw[n] for the ids
 * of the n loaded particles (host arrays; any output may be NULL).  The handle is left in a recomputed
 * intermediate state and cannot be stepped further (PIC_ESTATE). */
PIC_API int pic_adjoint_backward(pic_t *h, const pic_objective *obj, double *L, double *dL_da0, double *dL_dknots,
                                 int32_t n_knots, double *dL_dw);

/* Transpose of the field part of one step (B half, E, B half, with the
 * open-end Mur updates and the antenna) applied in place to
 * lam[6][n0*n1*n2] = (lamEx, lamEy, lamEz, lamBx, lamBy, lamBz) (host, window
 * frame); lam_j[3][...] (host, may be NULL) receives the adjoint of the
 * current.  t is the time at the start of the step.  A building block of
 * pic_adjoint_backward, exposed for transpose (dot-product) checks. */
PIC_API int pic_adjoint_fields(pic_t *h, float *lam, float *lam_j, double t);

/* Transpose of the particle part of one step (Sec. 5.2 steps i-v: gather,
 * Boris push, move, charge-conserving deposit) at the handle's current
 * state: the map (E, B, x, u, w) -> (x', u', J) that the next pic_step's
 * particle phase would apply, linearised at the particles and fields the
 * handle holds now, transposed and applied to the adjoints of its outputs.
 * In (by particle id, n ids): lam_x[dim][n] of the new positions (cells),
 * lam_u[3][n] of the new momenta; lam_j[3][n0*n1*n2] of the deposited
 * current (the order of pic_read_fields).  Out, overwritten: lam_x, lam_u
 * (of the old positions and momenta), lam_w[n] (of the weights) and
 * lam_f[6][n0*n1*n2] (of Ex..Bz).  Host arrays.  Requirements as for the
 * adjoint form (one run, track_ids, per_particle_weight, orders 1-3, no
 * moving window); n is the number of particles loaded.  A building block of
 * pic_adjoint_backward, exposed for transpose (dot-product) checks; it
 * allocates its scratch arrays for the call. */
PIC_API int pic_adjoint_particles(pic_t *h, float *lam_x, float *lam_u, const float *lam_j, double *lam_w,
                                  float *lam_f, int64_t n);

/* Charge density without any device allocation, for callers that cannot
 * allocate device memory (a host framework that passes the library only its
 * own buffers, a memory budget that forbids new allocations, a loop that
 * must not allocate once running).  The paper has no counterpart; it is the
 * same charge density as pic_read_fields(PIC_RHO),
 * rho(node) = sum q w S(x - node) with periodic wrap on every axis, computed
 * for the n particles given here.
 *   grid: dim, n (cells per axis; d, dt and bc_last are ignored);
 *   cell[dim][n] (int32), off[dim][n] (FP32 in [0,1)), w[n] (FP32, or NULL
 *   to use w_const for every particle) and rho[n0*n1*n2] (FP32 output) are
 *   device pointers owned by the caller; stream is a cudaStream_t (NULL =
 *   default stream); the call is asynchronous on it.
 * The FP64 accumulation grid is a static device array of PIC_STATIC_MAX_CELLS
 * cells (16 MiB), held by every GPU that loads the library until the
 * process exits; larger grids return PIC_EINVAL.  It is cleared at the start
 * of every call.  All calls on a device share the array, so calls that
 * overlap on the GPU (different streams, threads or handles) race and must
 * be ordered by the caller.  The first call on a device looks up the
 * array's device address (with that device current), so make that first
 * call before any CUDA stream capture; after cudaDeviceReset the next call
 * looks it up again in the new context.  Host threads may call
 * concurrently (the address lookup is locked).  No cudaMalloc, cudaFree or other
 * allocating routine is called.  Errors: PIC_EINVAL (arguments, grid too
 * large), PIC_ECUDA (launch failure). */
#define PIC_STATIC_MAX_CELLS (1ll << 21)
PIC_API int pic_charge_density_static(const pic_grid *grid, int32_t shape_order, double q, double w_const,
                                      int64_t n, const int32_t *cell, const float *off, const float *w, float *rho,
                                      void *stream);

/* Release everything (waits for the stream first).  NULL is ignored. */
PIC_API void pic_destroy(pic_t *h);

/* Static description of a status code. */
PIC_API const char *pic_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* PIC_GB300_H */
