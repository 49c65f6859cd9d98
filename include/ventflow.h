/*
 * ventflow.h -- C ABI of the GB300 incompressible-flow time step of DNSLABIB
 * (Korhonen, Laitinen, Ersavas Isitman, Jimenez, Vuorinen: "A GPU-accelerated computational fluid dynamics
 * solver for assessing shear-driven indoor airflow and virus transmission by scale-resolved simulations",
 * arXiv 2204.02107).
 *
 * One grid is a uniform periodic Cartesian box of nx*ny*nz cells (cell centres x_i = i*lx/nx, ...).  A time step
 * (Sec. 2.1-2.2) is:
 *   1. classic RK4 of u, v, w and the passive scalar c: skew-symmetric central convection, central diffusion,
 *      relaxation forcing S (u_set - u) / tau_f, body force b; every stage right-hand side is multiplied by the
 *      binary mask beta (Eqs. 2-4), no pressure term inside the stages;
 *   2. the divergence r = D u* by central differences;
 *   3. n iterations of  L p^{k+1} = D((1 - beta) G p^k) + r / dt  (Eq. 9), each a forward 3D FFT, a division by
 *      the eigenvalues of L = D o G, lambda = -sum_j sin^2(2 pi k_j / n_j) / h_j^2 (zero on the eight null
 *      modes), and an inverse 3D FFT; p^0 is the previous step's pressure.  p is the pressure divided by
 *      density: the paper's Eq. 8 has no dt, so its p is dt times this one;
 *   4. the projection u = beta (u* - dt G p) (Eq. 8);
 *   5. the sixth-order filter q <- beta (q + pi^-6 sum_j S6_j q), S6 = (1,-6,15,-20,15,-6,1), on u, v, w, c (Eq. 6);
 *   6. optional FP64 reductions (energy, divergence, scalar inventory, 64-bin histogram) (Sec. 3.3).
 *
 * Memory layout: every field is one array of nx*ny*nz values, x fastest: index = x + nx*(y + ny*z).
 * Precision: VF_FP64 computes everything in double; VF_FP32_MIXED keeps fields, stencils and FFTs in float and
 * accumulates every reduction to double precision or better (per-thread compensated float sums, float-float
 * pairs across threads and CTAs, converted to double once at the end; FP64 grids sum in double throughout).
 *
 * Errors: every call returns VF_OK (0) or a negative VF_E* code.  A failing call on a grid records a message
 * (vf_last_error) and, for CUDA failures, a sticky status that later calls on that grid return.  Calls never
 * throw.  Device kernels never trap: bounded waits and checks report through status words read by the host.
 *
 * Ownership: the caller owns every buffer it passes; the library copies from it (stream-ordered) before the call
 * returns and never keeps the pointer.  The library owns all device memory it allocates for a grid, through the
 * optional allocator callback, until vf_destroy.
 *
 * Threading: a grid may be used from one host thread at a time.
 */
#ifndef VENTFLOW_H
#define VENTFLOW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------------------------- */
#define VF_OK 0
#define VF_EINVAL (-1)      /* bad argument (null pointer, bad enum, non-positive length, ...) */
#define VF_ESIZE (-2)       /* grid size not even, < 8, with a prime factor other than 2, 3, 5, or over 2^30 cells */
#define VF_ENOMEM (-3)      /* allocation failed, or a batch is over its memory budget */
#define VF_ECUDA (-4)       /* a CUDA runtime call failed (sticky for the grid) */
#define VF_ESTATE (-5)      /* call not valid in the current state (e.g. step before set_mask) */
#define VF_ENONFINITE (-6)  /* a reduction found a NaN or Inf in the fields */
#define VF_ETIMEOUT (-7)    /* a bounded device wait expired */

typedef enum { VF_FP64 = 0, VF_FP32_MIXED = 1 } vf_precision;
typedef enum { VF_U = 0, VF_V = 1, VF_W = 2, VF_C = 3, VF_P = 4 } vf_field;
typedef enum { VF_HOST = 0, VF_DEVICE = 1 } vf_mem;

/* Optional device allocator.  alloc returns a device pointer of at least `bytes` (256-byte aligned) usable on
 * `stream` (a cudaStream_t), or NULL on failure; free releases it.  NULL allocator -> cudaMallocAsync/FreeAsync. */
typedef struct vf_allocator {
    void* (*alloc)(size_t bytes, void* stream, void* ctx);
    void (*free)(void* ptr, void* stream, void* ctx);
    void* ctx;
} vf_allocator;

/* Grid description (Sec. 2.4: the case parameters).  Fill with vf_grid_desc_default, then override. */
typedef struct vf_grid_desc {
    int32_t nx, ny, nz;          /* cells per axis: each even, >= 8, of the form 2^a 3^b 5^c; nx*ny*nz <= 2^30 */
    double lx, ly, lz;           /* box lengths [m]; h_j = l_j / n_j */
    double nu;                   /* kinematic viscosity [m^2/s] */
    double alpha_c;              /* scalar diffusivity [m^2/s]; < 0 -> nu */
    double dt;                   /* fixed time step [s], > 0 */
    double tau_f;                /* forcing relaxation time [s]; <= 0 -> dt */
    double body_force[3];        /* b [m/s^2] */
    int32_t n_pressure_iters;    /* iterations of Eq. 9 per step (paper: 4); grids without solid cells use 1,
                                    which gives the same result because (1 - beta) G p vanishes */
    int32_t filter;              /* 1: apply the Eq. 6 filter after the projection; 0: skip it */
    int32_t precision;           /* vf_precision */
    int32_t history_capacity;    /* number of per-step reduction records kept on the device (ring buffer) */
    void* cuda_stream;           /* cudaStream_t the grid works on; NULL -> a stream the grid creates */
    const vf_allocator* alloc;   /* NULL -> cudaMallocAsync */
    double courant_max;          /* > 0: dynamic time step (Sec. 2.4, AdjustDt: the user sets the maximum Courant
                                    number).  Before every step dt = min(dt, courant_max / sigma) with
                                    sigma = max over cells of sum_j |u_j| / h_j of the current state (dt itself
                                    while the fluid is at rest), chosen on the device; p/rho needs no rescale.
                                    0: fixed dt.  tau_f <= 0 follows the current dt. */
} vf_grid_desc;

/* FP64 reductions of one state (Sec. 3.3 diagnostics).  dV = hx*hy*hz.  Room cells are those flagged by
 * vf_set_region (default: all fluid cells). */
typedef struct vf_reduce {
    double t;                    /* simulated time of the state [s] */
    int64_t step;                /* steps taken to reach it */
    double ke;                   /* 1/2 sum dV |u|^2 */
    double div_max;              /* max |D u|: records taken by vf_step use the velocity right after the
                                    projection (before the filter), vf_reductions the current velocity */
    double div_l2;               /* sqrt(sum dV (D u)^2), same velocity as div_max */
    double u_max;                /* max over cells and components of |u_i| */
    double c_total;              /* sum dV c over all cells */
    double c_room;               /* sum dV c over room cells */
    double c2_room;              /* sum dV c^2 over room cells */
    double v_room;               /* sum dV over room cells */
    int64_t hist[64];            /* room cells with c in [b/64, (b+1)/64) (c == 1 in bin 63) */
    int64_t hist_under;          /* room cells with c < 0 */
    int64_t hist_over;           /* room cells with c > 1 */
    double dt;                   /* time step that produced the state (the grid's dt for vf_reductions) */
    /* Scalar budget of the step that produced the state (Eqs. 3-4 in flux form, the room inventory of
     * Sec. 3.3), in units of c m^3; records taken by vf_step only (vf_reductions leaves them 0).  Each stage
     * term is the RK4-weighted sum dt sum_s b_s X_s over the four stage states s.  With c_total and c_room of
     * the previous record they close: c_total' = c_total + budget_forcing - budget_mask_loss and
     * c_room' = c_room + budget_forcing_room - budget_outflow + budget_filter_room. */
    double budget_forcing;       /* X_s = sum over fluid cells dV S (c_set - c_s) / tau_f */
    double budget_forcing_room;  /* the same over the room cells */
    double budget_outflow;       /* X_s = scalar flux out of the room through its faces to non-room fluid cells
                                    (convective minus diffusive face flux of Eq. 3 times the face area) */
    double budget_mask_loss;     /* scalar the filter puts into solid cells, removed again by the re-mask */
    double budget_filter_room;   /* change of the room inventory by the filter (Eq. 6) */
} vf_reduce;

typedef struct vf_grid vf_grid;

/* ---- grid lifecycle ------------------------------------------------------------------------------------- */

/* Fill *d with defaults (the case parameters of Sec. 2.4; nu of air, Tab. 3): 64^3 unit box, nu = 1.6e-5,
 * alpha_c = nu, dt = 1e-3, tau_f = dt, no body force,
 * 4 pressure iterations, filter on, FP32_MIXED, 4096 history records, own stream, default allocator. */
int vf_grid_desc_default(vf_grid_desc* d);

/* Validate *d, allocate every device buffer of the grid on the current CUDA device, build the FFT twiddle and
 * eigenvalue tables (Sec. 2.2) and zero all fields.  The mask starts as all-fluid with no forcing region; the
 * grid is ready to step once vf_set_mask has been called.  *out receives the handle (NULL on failure). */
int vf_create_grid(const vf_grid_desc* d, vf_grid** out);

/* Release everything the grid owns (waits for its stream first).  NULL is accepted.  (Resource handling: no
 * counterpart in the paper.) */
int vf_destroy(vf_grid* g);

/* ---- inputs (Sec. 2.1: beta, S, u_set, c_set; Sec. 3.3: the room region) ----------------------------------- */

/* The binary mask beta of Sec. 2.1 (Eq. 4): nx*ny*nz bytes in `mem`, nonzero = fluid, 0 = solid.  Fields are
 * re-masked (set to zero in solids). */
int vf_set_mask(vf_grid* g, const uint8_t* beta, int mem);

/* S: nx*ny*nz bytes, nonzero = forcing region (cells outside the fluid are ignored); u_set[3] and c_set are the
 * targets of the relaxation terms S (u_set - u) / tau_f and S (c_set - c) / tau_f (Eqs. 2-3).  S may be NULL to
 * keep the current region and only change the set point. */
int vf_set_inflow(vf_grid* g, const uint8_t* S, const double u_set[3], double c_set, int mem);

/* Smooth forcing region of Eq. 5 (the paper's general inlet model): on every cell centre x_j = i h_j
 *   S = prod_j (1 - tanh(B_j [d_j / (W_j/2) - (W_j/2) / d_j])) / 2,
 * d_j the periodic (minimum-image) distance from x_j to center[j], each factor 1 where d_j = 0 (its limit).
 * center [m], width W [m] (> 0) and sharpness B (> 0) per axis (x, y, z).  Replaces the forcing region and sets
 * the targets u_set, c_set; S is evaluated in double on the device and stored in the grid's precision. */
int vf_set_inflow_tanh(vf_grid* g, const double center[3], const double width[3], const double sharpness[3],
                       const double u_set[3], double c_set);

/* Smooth forcing region from values: S is nx*ny*nz values in [0, 1] (double if is_fp64, else float) in `mem`
 * (for example a sum of Eq. 5 windows).  Replaces the forcing region and sets u_set, c_set.  vf_set_inflow with a
 * non-NULL S returns to a binary region. */
int vf_set_inflow_values(vf_grid* g, const void* S, int is_fp64, const double u_set[3], double c_set, int mem);

/* Forcing with per-cell targets (Eqs. 2-3 with u_set and c_set varying in space, e.g. the parabolic inflow profile
 * of the cube-in-channel case, Sec. 3.1.2): S is nx*ny*nz values in [0, 1]; targets is 4 arrays of nx*ny*nz
 * values one after the other (u_set, v_set, w_set, c_set); double if is_fp64, else float; in `mem`.  The targets
 * take 4 values per cell of device memory, allocated on the first call (beyond vf_grid_bytes).  vf_set_inflow,
 * vf_set_inflow_tanh and vf_set_inflow_values return to constant targets. */
int vf_set_inflow_field(vf_grid* g, const void* S, const void* targets, int is_fp64, int mem);

/* The room whose CO2 inventory, volume and concentration distribution Sec. 3.3 evaluates: room is nx*ny*nz bytes
 * in `mem`, nonzero = counted in c_room, c2_room, v_room and the histogram. */
int vf_set_region(vf_grid* g, const uint8_t* room, int mem);

/* Overwrite one field of the state of Sec. 2.1 (u, v, w, c, p) from nx*ny*nz values (double if is_fp64, else
 * float) in `mem`.  VF_P takes the pressure
 * divided by density p/rho (the warm start of the next pressure solve); u, v, w, c are multiplied by beta on the
 * way in. */
int vf_set_field(vf_grid* g, int field, const void* src, int is_fp64, int mem);

/* Set the simulated time and step counter of the current state (with vf_set_field, restores a saved state; no
 * counterpart in the paper, which only writes its fields out, Sec. 2.4). */
int vf_set_time(vf_grid* g, double t, int64_t step);

/* ---- stepping -------------------------------------------------------------------------------------------- */

/* Enqueue n time steps (Sec. 2.1-2.2, steps 1-6 above) on the grid's stream and return without waiting.  Every
 * `reduce_every`-th step (counted from step 0; 0 = never) also records the reductions of the new state into the
 * device history.  Steps replay a captured CUDA graph of one step unless the environment variable VF_NO_GRAPH is
 * set. */
int vf_step(vf_grid* g, int64_t n, int32_t reduce_every);

/* Wait for all work enqueued on the grid (no counterpart in the paper). */
int vf_sync(vf_grid* g);

/* ---- outputs --------------------------------------------------------------------------------------------- */

/* Copy one field of the state of Sec. 2.1 (nx*ny*nz values, double if as_fp64 else float) into dst in `mem`,
 * after all enqueued steps.
 * VF_P is the pressure divided by density, p/rho [m^2/s^2]; the library stores exactly this value, so reading
 * and writing it back restores the state bit for bit. */
int vf_read_field(vf_grid* g, int field, void* dst, int as_fp64, int mem);

/* Compute the reductions (the Sec. 3.3 diagnostics of vf_reduce) of the current state (waits).  Returns
 * VF_ENONFINITE if a field holds NaN/Inf. */
int vf_reductions(vf_grid* g, vf_reduce* out);

/* Copy the per-step reduction records (Sec. 3.3 time series) taken by vf_step (oldest first, at most
 * max_records of the most recent)
 * into out[]; *count receives the number copied.  Waits for enqueued steps. */
int vf_history(vf_grid* g, vf_reduce* out, int64_t max_records, int64_t* count);

/* Forget the recorded history (of the Sec. 3.3 time series). */
int vf_clear_history(vf_grid* g);

/* Immersed-boundary force on a solid region (the drag of the cube-in-channel case, Sec. 3.1.2).  region: nx*ny*nz
 * bytes in `mem`, nonzero = part of the region (kept until the next call). */
int vf_set_force_region(vf_grid* g, const uint8_t* region, int mem);

/* force[3] = dV sum over the region of the unmasked right-hand side of Eq. 2 of the current state,
 * -convection + nu diffusion + S (u_set - u) / tau_f + b - grad(p/rho), in FP64 [m^4/s^2, i.e. N per kg/m^3 of
 * density]: the rate at which the mask removes momentum there, the force the fluid exerts on the body.  Waits. */
int vf_region_force(vf_grid* g, double force[3]);

/* Simulated time, step count, cell count and bytes of device memory held by the grid (bookkeeping: no
 * counterpart in the paper).  With a dynamic time step the
 * time is read from the device (waits for the enqueued steps). */
int vf_info(const vf_grid* g, double* t, int64_t* step, int64_t* cells, int64_t* device_bytes);

/* Solve L p = f once with the grid's FFT Poisson solver (Sec. 2.2, one pass of step 3 above): forward 3D FFT,
 * division by lambda (null modes -> 0), inverse 3D FFT.  f and p are device arrays of nx*ny*nz values in the
 * grid's precision (double for VF_FP64, float otherwise); they may alias.  Uses the grid's spectrum buffer as
 * scratch; stream-ordered on the grid's stream, returns without waiting. */
int vf_poisson_solve(vf_grid* g, const void* f, void* p);

/* ---- launch tiles and the autotuner ---------------------------------------------------------------------- */

/* Launch shapes of this implementation (the paper has no counterpart).
 * zc_*: planes one CTA of a stencil kernel marches along z, per kernel family.  A chunk changes no field value;
 * with the filter on, the divergence norm is summed per filter warp, so its last bits follow zc_filter (with the
 * filter off, every reduction follows it).  Each chunk lies in [VF_ZCHUNK_MIN, VF_ZCHUNK_MAX].
 * fft_*: radix schedule of the generic mixed-radix FFT passes (Sec. 2.2's FFTs) along the x half length nx/2, y
 * and z: an index into vf_fft_schedules' candidates for that length, 0 = the default.  Every schedule computes the
 * same transforms in another rounding order, so fields agree to rounding (not bitwise) across schedules.  Grids
 * whose FFT takes the register path (vf_fft_path) keep the indices but do not use them. */
#define VF_ZCHUNK_MIN 4
#define VF_ZCHUNK_MAX 64
typedef struct vf_tiles {
    int32_t zc_stage;    /* the four RK4 stage kernels */
    int32_t zc_div;      /* divergence */
    int32_t zc_project;  /* projection */
    int32_t zc_filter;   /* filter and its divergence records (also the standalone reductions) */
    int32_t fft_x;       /* radix schedule of the nx/2-point x transforms */
    int32_t fft_y;       /* of the ny-point y transforms */
    int32_t fft_z;       /* of the nz-point z transforms */
} vf_tiles;

/* The tiles a grid launches with.  A new grid takes the process-wide tile cache's entry for its (nx, ny, nz,
 * precision) if there is one, else (4, 32, 8, 16, 0, 0, 0): the z-chunks the autotuner chose for a 256 x 128 x 128
 * room on GB300 and the default FFT schedules. */
int vf_get_tiles(const vf_grid* g, vf_tiles* out);

/* Which passes the grid's pressure solve (Sec. 2.2's FFTs) runs, chosen at vf_create_grid from the lengths and the
 * precision: VF_FFT_GENERIC (the mixed-radix passes), VF_FFT_REGISTER_PLANE (register-resident transforms, the
 * (y, z) plane of each kx in one CTA) or VF_FFT_REGISTER_TILE (register transforms, y passes and z tiles).  The
 * register path takes lengths nx/2, ny, nz each 16 G (G = 1, 2, 4, 8, 16), and in FP32 also 36, 40, 48, 60, 72,
 * 80 or 96 (then ny = nz, the plane kernel only).  VF_EINVAL for a NULL argument.  Host only. */
#define VF_FFT_GENERIC 0
#define VF_FFT_REGISTER_PLANE 1
#define VF_FFT_REGISTER_TILE 2
int vf_fft_path(const vf_grid* g, int32_t* path);

/* Set a grid's tiles (VF_EINVAL if a chunk is out of range or an FFT index is not a candidate of its length; the
 * grid is unchanged then).  Takes effect at the next vf_step (the step graph is captured again).  Waits. */
int vf_set_tiles(vf_grid* g, const vf_tiles* t);

/* Radix schedule `index` of the generic FFT passes for a transform of length n (an implementation choice; the paper
 * has no counterpart beyond its use of the FFT in Sec. 2.2): writes its radices (each 2, 3, 4, 5, 8 or 16, product
 * n, applied in this order) to radices[0 .. count-1] and returns count; returns 0 when index is past the last
 * candidate (or n is not 2-3-5 smooth), VF_EINVAL for a NULL radices, index < 0 or max_radices too small (16
 * always suffices).  Candidate 0 is the default: as few power-of-two passes as possible, then the 3s and
 * 5s; the others (at most 8 in all) split the power-of-two part into radix-16, radix-8 or radix-4 passes (radix-2
 * too when it is at most 8), or run the default's small radices first, with the odd factors last or first.  Host
 * only. */
int vf_fft_schedules(int32_t n, int32_t index, int32_t* radices, int32_t max_radices);

/* Autotuner: time every chunk in {4, 8, 16, 32} for each kernel family on this grid's own arrays (reps launches
 * each after one warm-up, CUDA events on the grid's stream, the least mean time wins); then, for a grid on the
 * generic FFT path, every candidate radix schedule of each axis in turn (x, then y, then z, the others held at their
 * best so far), timed as one Poisson solve (FFT, 1/lambda, inverse FFT) of a scratch array.  Sets the winners on the
 * grid, stores them in the tile cache under the grid's (nx, ny, nz, precision) and copies them to *chosen (may be
 * NULL).  Only scratch arrays are written: the state, the pressure, the history and the step count are unchanged
 * (the next steps may differ from an untuned grid's in the last bits if another FFT schedule won).  Waits; reps in
 * [1, 1000].  Other work on the GPU at the same time perturbs the timings. */
int vf_autotune(vf_grid* g, int32_t reps, vf_tiles* chosen);

/* Tile cache: look up (1 found and *out set, 0 not found), or forget every entry. */
int vf_tile_cache_lookup(int32_t nx, int32_t ny, int32_t nz, int32_t precision, vf_tiles* out);
int vf_tile_cache_clear(void);

/* Tile cache contents, so that tuned tiles can be saved and restored across processes (host only, no device
 * work): the number of entries; entry i in (nx, ny, nz, precision) order, key[4] = {nx, ny, nz, precision} and its
 * tiles (VF_EINVAL for i out of range or a NULL pointer); and storing tiles under a key as vf_autotune does,
 * replacing an entry (VF_EINVAL for a chunk out of range, an unknown precision or an FFT index that is not a
 * candidate of its axis length; VF_ESIZE for sizes vf_create_grid rejects).  Grids created afterwards take the
 * stored tiles. */
int64_t vf_tile_cache_size(void);
int vf_tile_cache_entry(int64_t i, int32_t key[4], vf_tiles* out);
int vf_tile_cache_insert(int32_t nx, int32_t ny, int32_t nz, int32_t precision, const vf_tiles* t);

/* ---- batched rooms and continuous batching (many rooms advanced together) --------------------------------- */
/* The paper runs one case at a time; batching and serving many rooms has no counterpart there.  Each room's step is
 * the step of Sec. 2.1-2.2 exactly as vf_step runs it. */

/* Device bytes vf_create_grid will allocate for a description (used for admission by memory budget). */
int64_t vf_grid_bytes(const vf_grid_desc* d);

typedef struct vf_batch vf_batch;
typedef struct vf_batch_desc {
    int32_t max_slots;           /* rooms held at once */
    int64_t hbm_budget_bytes;    /* admission limit: sum of vf_grid_bytes of the rooms held */
    int32_t reduce_every;        /* record each room's reductions every k batch steps (0 = never) */
    void* cuda_stream;           /* stream the batch graph runs on; NULL -> a stream the batch creates */
    int32_t autotune;            /* > 0: a room whose (nx, ny, nz, precision) has no tile-cache entry is autotuned
                                    with this many reps when admitted (the batch stream is drained first, so the
                                    timings see an idle GPU); 0: rooms take the cached or default tiles */
} vf_batch_desc;

/* Empty batch.  One batch step advances every running room by one time step through a single CUDA graph launch
 * with independent lanes of rooms (the lanes' kernels run concurrently; the rooms of a lane one after another, as
 * many lanes as keep the Poisson working set of the rooms in flight within L2, at least 8; the environment
 * variable VF_BATCH_LANES, read when the graph is captured, sets the count, 0 = one lane per room); a room's
 * arithmetic is the same as alone, so its fields are bitwise identical alone and in any mix. */
int vf_batch_create(const vf_batch_desc* d, vf_batch** out);
int vf_batch_destroy(vf_batch* b);

/* Admit a room into a free slot: a grid is created from *gd (its cuda_stream is ignored), given the mask beta, the
 * forcing region S (may be NULL) with set points u_set, c_set, the room region (may be NULL: all fluid cells) and
 * the initial scalar c0 (may be NULL: zero; nx*ny*nz values, double if c0_is_fp64), all in `mem`; it will run
 * `steps` steps.  *slot receives the slot.  VF_ENOMEM when no slot is free or its vf_grid_bytes would exceed the
 * budget (nothing is allocated then). */
int vf_batch_add(vf_batch* b, const vf_grid_desc* gd, const uint8_t* beta, const uint8_t* S, const uint8_t* room,
                 const double u_set[3], double c_set, const void* c0, int c0_is_fp64, int64_t steps, int mem,
                 int32_t* slot);

/* Enqueue up to n batch steps (async).  Every running room advances by min(n, its remaining steps); the steps are
 * launched in chunks that end when a room reaches its target, which then stops and is reported by vf_batch_poll. */
int vf_batch_step(vf_batch* b, int64_t n);
int vf_batch_sync(vf_batch* b);

/* Wait for enqueued steps; write up to max_slots finished slots to done_slots, their total to *n_done. */
int vf_batch_poll(vf_batch* b, int32_t* done_slots, int32_t max_slots, int32_t* n_done);

/* The grid of a slot (NULL if empty): read its fields and history with the vf_grid calls after vf_batch_poll.  The
 * batch's step graph holds the slot's launch shapes: do not change them through this handle (vf_set_tiles,
 * vf_autotune) while the slot is in the batch. */
vf_grid* vf_batch_grid(vf_batch* b, int32_t slot);

/* Free a slot and its memory (waits for enqueued steps). */
int vf_batch_remove(vf_batch* b, int32_t slot);

/* Running and finished rooms, bytes held and batch steps taken. */
int vf_batch_info(const vf_batch* b, int32_t* active, int32_t* done, int64_t* bytes_in_use, int64_t* batch_steps);
const char* vf_batch_last_error(const vf_batch* b);

/* ---- Poisson solve without device allocation --------------------------------------------------------------- */

/* The paper has no counterpart of this call; it exists for callers that cannot allocate device memory (code that
 * runs where cudaMalloc is forbidden or unavailable, e.g. inside an allocator or a framework that owns every
 * device allocation).  It computes the same solve as vf_poisson_solve -- L p = f with the forward 3D FFT,
 * division by lambda (null modes -> 0) and inverse 3D FFT -- without a grid handle and without allocating:
 * its scratch (half spectrum and FFT / eigenvalue tables) is one file-scope device array of 33 MiB that every
 * GPU loading the library holds until the process exits.
 *   nx, ny, nz, lx, ly, lz: sizes and box lengths as in vf_grid_desc;  precision: VF_FP64 (f, p are double) or
 *   VF_FP32_MIXED (float);  f, p: caller-owned device arrays of nx*ny*nz values (may alias);  stream: a
 *   cudaStream_t or NULL.  Returns after p is written.
 * Limits: nx*ny*nz <= vf_poisson_noalloc_max_cells(precision) (4,194,304 in FP64, 8,388,608 in FP32), every
 * FFT length (nx/2 + 1, ny, nz) <= 1024, and ny, nz <= 581 in FP64 or <= 592 in FP32 (the y and z passes keep
 * three tiles and a twiddle table of the longer axis in one CTA's shared memory); larger sizes return VF_ESIZE.
 * The first call on a device looks up the array's device address (once per device, with that device current);
 * make that first call before any stream capture.  Every call reuses the same array and leaves its contents
 * behind; calls that overlap on the GPU (several streams or threads at once) race on it. */
int vf_poisson_solve_noalloc(int32_t nx, int32_t ny, int32_t nz, double lx, double ly, double lz,
                             int32_t precision, const void* f, void* p, void* stream);

/* Largest nx*ny*nz that vf_poisson_solve_noalloc accepts in the given precision (0 for a bad precision). */
int64_t vf_poisson_noalloc_max_cells(int32_t precision);

/* ---- Lagrangian particles (Sec. 2.3) --------------------------------------------------------------------- */

/* Replace the grid's particles by n particles (n = 0 removes them), one-way coupled: after every step each
 * airborne particle moves with du_p/dt = (C_d / tau_p)(u_f - u_p) + g, tau_p = rho_p d^2 / (18 rho_f nu),
 * C_d = 1 + Re_p^(2/3) / 6, Re_p = |u_f - u_p| d / nu, by implicit Euler with C_d from the relative velocity at the
 * start of the step (u_p' = (u_p + a u_f + dt g) / (1 + a), a = dt C_d / tau_p; x_p' = x_p + dt u_p'), u_f the
 * new fluid velocity interpolated trilinearly between cell centres.  Positions wrap periodically; a particle
 * whose nearest cell becomes solid is deposited (stays put with zero velocity).
 * pos, vel: n x 3 doubles (x, y, z of each particle) [m], [m/s]; size: n doubles d [m] (the paper's sedimentation
 * times hold for d the diameter); rho_p, rho_f [kg/m^3]; gravity[3] [m/s^2].  Host arrays, copied.  The
 * particle arrays (n x 64 bytes) are device memory of the grid beyond vf_grid_bytes. */
int vf_particles_set(vf_grid* g, int64_t n, const double* pos, const double* vel, const double* size, double rho_p,
                     double rho_f, const double gravity[3]);

/* Copy the particles to host arrays after the enqueued steps (waits): pos, vel n x 3 doubles, deposited n ints
 * (1 = deposited); any of them may be NULL. */
int vf_particles_read(vf_grid* g, double* pos, double* vel, int32_t* deposited);

/* Number of particles of the grid (Sec. 2.3). */
int vf_particles_count(const vf_grid* g, int64_t* n);

/* ---- measurement ----------------------------------------------------------------------------------------- */

/* Kernel phases of one step, in launch order (measurement: no counterpart in the paper). */
#define VF_PHASE_STAGE1 0       /* RK4 stage 1: k1, acc = q + dt/6 k1, q2 = q + dt/2 k1 */
#define VF_PHASE_STAGE2 1       /* RK4 stage 2 */
#define VF_PHASE_STAGE3 2       /* RK4 stage 3 */
#define VF_PHASE_STAGE4 3       /* RK4 stage 4: q* = acc + dt/6 k4 */
#define VF_PHASE_DIV 4          /* r = D u* / dt */
#define VF_PHASE_FFT_X_FWD 5    /* real-to-complex FFT along x of the Eq. 9 right-hand side */
#define VF_PHASE_FFT_Y_FWD 6    /* FFT along y */
#define VF_PHASE_FFT_Z_SOLVE 7  /* FFT along z, division by lambda, inverse FFT along z */
#define VF_PHASE_FFT_Y_INV 8    /* inverse FFT along y */
#define VF_PHASE_FFT_X_INV 9    /* complex-to-real inverse FFT along x -> p */
#define VF_PHASE_PROJECT 10     /* u = beta (u* - dt G p) */
#define VF_PHASE_FILTER 11      /* Eq. 6 filter (with the reductions: also the divergence of its input) */
#define VF_PHASE_REDUCE 12      /* FP64 reductions of the step's final state */
#define VF_PHASE_POISSON_RHS 13 /* Eq. 9 correction D((1 - beta) G p) at the cells next to solids */
#define VF_PHASE_FFT_YZ_SOLVE 14 /* per-kx plane: y, z FFTs, division by lambda, inverse z, y FFTs */
#define VF_PHASE_ADJUST_DT 15   /* dynamic time step: dt from the Courant rate of the current state */
#define VF_PHASE_PARTICLES 16   /* Lagrangian particles (Sec. 2.3) in the new velocity */
#define VF_N_PHASES 17

/* Run n steps like vf_step but with direct launches bracketed by CUDA events on the grid's stream; adds the
 * elapsed milliseconds of every phase to phase_ms[VF_N_PHASES] and its launch count to launches[VF_N_PHASES]
 * (both caller-owned, not cleared).  Waits for completion. */
int vf_profile_steps(vf_grid* g, int64_t n, int32_t reduce_every, double* phase_ms, int64_t* launches);

/* Measurement helper (no counterpart in the paper): the device's FP64 fused multiply-add rate in GFLOP/s (2 flops
 * per FMA), from eight independent FMA chains per thread on every SM, timed with CUDA events.  The FP64 form of the
 * step is bound by this rate on GB300. */
int vf_measure_fp64_rate(double* gflops);

/* Name of a phase id ("stage1", "fft_z_solve", ...), or "unknown". */
const char* vf_phase_name(int phase);

/* ---- status ---------------------------------------------------------------------------------------------- */
/* Status and binding helpers (no counterpart in the paper). */

const char* vf_status_string(int status);

/* Byte sizes of the ABI structs as this library was compiled: out[0] vf_grid_desc, out[1] vf_reduce,
 * out[2] vf_batch_desc, out[3] vf_tiles (for bindings to check their layouts). */
int vf_abi_sizes(int64_t out[4]);
const char* vf_last_error(const vf_grid* g);

/* ---- host-side ventilation metrics (Sec. 3.3.2, 3.4), from a reduction series -------------------------------- */

/* ACH [1/h] from the least-squares slope of ln c(t) (fresh air c = 0; the decay of Sec. 3.3.2 with C1 = 0):
 * ACH = -3600 d ln c / dt, t in seconds. */
int vf_ach_log_slope(const double* t_seconds, const double* c_mean, int64_t n, double* ach_per_hour);

/* Three-parameter fit c(t) = C0 exp(-ACH t) + C1 (Sec. 3.3.2): ACH [1/h], C0, C1. */
int vf_ach_fit3(const double* t_seconds, const double* c_mean, int64_t n, double* ach_per_hour, double* c0,
                double* c1);

/* Time-dependent Wells-Riley (Eqs. 17-18): dose Q(t) = (C0 p / ACH)(1 - exp(-ACH t)) and P = 1 - exp(-Q).
 * c0 [quanta/m^3], breathing p [m^3/h], ach [1/h] (0 allowed), t [h]. */
int vf_wells_riley(double c0, double breathing_m3_h, double ach_per_hour, double t_hours, double* dose,
                   double* probability);

#ifdef __cplusplus
}
#endif

#endif /* VENTFLOW_H */
