/*
 * lbm.h - C ABI of the GB300 D3Q19 lattice Boltzmann library (liblbm.so).
 *
 * The library runs the data-parallel hot path of the patch/block lattice
 * Boltzmann scheme of Feichtinger et al. on one GPU: the fused pull
 * stream-and-collide sweep (Sec. 2.1, Eq. (1)-(2); GPU kernel design of
 * Sec. 3.2) with half-way bounce-back and moving walls read from a per-cell
 * flag field (Sec. 2.1), and the ghost-layer exchange between the Blocks of
 * one Patch (Sec. 4.2, Sec. 4.4), done entirely in device memory.
 *
 * Conventions shared by every entry point
 *  - Every function returns an lbm_status (0 = LBM_OK); no C++ exception
 *    crosses this boundary.  lbm_last_error() gives a readable message.
 *  - The library owns all device memory of a context (allocated through the
 *    allocator installed with lbm_set_allocator, cudaMalloc by default) and
 *    enqueues all work on the context's stream (lbm_params.stream, or a
 *    stream it creates).  The caller owns every host buffer and every device
 *    buffer it passes in.
 *  - "host" pointers are ordinary CPU memory (pageable or pinned); "device"
 *    pointers are CUDA device memory of the current device.  Entry points
 *    taking host pointers synchronise the context stream before returning;
 *    entry points taking device pointers (suffix _device) only enqueue.
 *  - A context is used by one host thread at a time.
 *  - Cell fields are laid out with x fastest: cell (x,y,z) of a domain of
 *    nx*ny*nz interior cells has index c = (z*ny + y)*nx + x.  PDF arrays
 *    are direction-major: f[q*N + c].  Velocity arrays are component-major:
 *    u[a*N + c].  For a batch context the instances are concatenated in
 *    order, each with its own N_k and this layout inside its slice
 *    (PDF slice 19*N_k values, velocity slice 3*N_k values).
 *
 * D3Q19 directions (Sec. 2.1: 19 PDFs per cell, weights 1/3, 1/18, 1/36):
 *    q :  0   1   2   3   4   5   6   7   8   9  10  11  12  13  14  15  16  17  18
 *   ex :  0  +1  -1   0   0   0   0  +1  -1  +1  -1  +1  -1  +1  -1   0   0   0   0
 *   ey :  0   0   0  +1  -1   0   0  +1  -1  -1  +1   0   0   0   0  +1  -1  +1  -1
 *   ez :  0   0   0   0   0  +1  -1   0   0   0   0  +1  -1  -1  +1  +1  -1  -1  +1
 * opposite(q) = q+1 for odd q, q-1 for even q > 0, and 0 for q = 0.
 *
 * PDFs are exchanged in their shifted form f~_q = f_q - w_q rho0 (Sec. 2.1),
 * so a fluid at rest with density rho0 has f~ = 0.  The stored state after a
 * step holds post-collision values; rho = rho0 + sum_q f~_q and
 * u = (sum_q e_q f~_q - F/2)/rho0 recover the density and velocity that the
 * last collision of each cell used.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_Q 19

/* Status codes. */
typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = -1,    /* an argument is out of its documented range */
    LBM_ENOMEM = -2,    /* the allocator returned NULL */
    LBM_ECUDA = -3,     /* a CUDA call failed (message in lbm_last_error) */
    LBM_ETIMEOUT = -4,  /* a bounded device-side wait gave up */
    LBM_ENUMERIC = -5   /* a NaN or Inf was found where the call checks for it */
} lbm_status;

/* Per-cell flag values (one uint8 per interior cell).  LBM_PRESSURE (not in
 * the paper, which leaves further boundary conditions on the GPU to future
 * work, Sec. 6): a pressure boundary; a population that would stream into it returns by
 * anti-bounce-back with the velocity correction,
 *   f~_ibar(x) = -f~*_i(x) + 2 w_i [(rho_b - rho0) + rho0 (4.5 (e_i.u_b)^2 - 1.5 u_b.u_b)],
 * which holds the density rho_b halfway between x and the boundary node;
 * u_b is the velocity of x's last collision, (sum_j e_j f~*_j(x) - F/2) / rho0
 * from its stored populations.  A velocity inlet is an LBM_MOVING face with
 * wall_u the inlet velocity (Ladd bounce-back). */
enum { LBM_FLUID = 0, LBM_NOSLIP = 1, LBM_MOVING = 2, LBM_PRESSURE = 3 };
/* Collision operators: single relaxation time of Eq. (1), or two relaxation times. */
enum { LBM_BGK = 0, LBM_TRT = 1 };
/* PDF storage formats.  Arithmetic is FP32 for the first three and FP64 for
 * LBM_F64.  F16S/BF16S store the shifted PDF f~ (times storage_scale) in
 * IEEE half / bfloat16, rounded to nearest even. */
enum { LBM_F32 = 0, LBM_F16S = 1, LBM_BF16S = 2, LBM_F64 = 3 };

typedef struct {
    int collision;        /* LBM_BGK (default) or LBM_TRT */
    double magic;         /* TRT Lambda = (tau - 1/2)(1/omega_minus - 1/2); default 3/16 */
    double rho0;          /* reference density; default 1 */
    double force[3];      /* body force density F (Guo forcing); default 0 */
    double wall_u[3];     /* velocity of every LBM_MOVING wall or cell; default 0 */
    int periodic[3];      /* 1 = periodic along x / y / z; default 0 */
    int face_bc[6];       /* wall kind beyond the -x,+x,-y,+y,-z,+z faces of a
                             non-periodic axis: LBM_NOSLIP (default), LBM_MOVING or
                             LBM_PRESSURE.
                             Edge and corner cells of the wall shell shared by two
                             walls rest (LBM_NOSLIP). */
    int storage;          /* LBM_F32 (default), LBM_F16S, LBM_BF16S, LBM_F64 */
    double storage_scale; /* power of two multiplying f~ in F16S/BF16S storage; default 1 */
    void *stream;         /* cudaStream_t to enqueue on; NULL = the library creates one */
    int tile[3];          /* sweep tile: threads along x (a multiple of 32), rows along
                             y, z slices, one cell per thread; {0,0,0} = the library's
                             default: two cells per thread where every Block width is even
                             (FP32 / 16-bit storage; row tiles of 64 x 4 x 2 cells where the
                             widths are multiples of 64, else runs of 256 cells), otherwise
                             row tiles, or runs of 256 cells where a width is not a multiple
                             of 32 (lbm_autotune may change any of these) */
    int graph_steps;      /* steps per captured CUDA graph; 0 = automatic, -1 = no graphs */
    int kernel;           /* LBM_KERNEL_AUTO (default): the register sweep, with the
                             TMA-staged sweep prepared where the Patch allows it so
                             that lbm_autotune can choose it; LBM_KERNEL_REGISTER;
                             LBM_KERNEL_TMA (LBM_EINVAL at create when not applicable) */
    int debug_flags;      /* 0; LBM_DEBUG_DROP_STAGE makes the TMA sweep skip one staged
                             load so its bounded waits expire (failure-path tests) */
    double rho_b;         /* density of every LBM_PRESSURE boundary; 0 (default) = rho0 */
    int streaming;        /* LBM_STREAM_TWO_GRID (default): the pull of Sec. 3.2 from one
                             PDF array into a second; LBM_STREAM_AA: one array updated in
                             place (AA access pattern, half the PDF memory, the same bytes
                             per cell update).  Steps alternate between a local step (each
                             cell reads its own PDFs and writes them back into the opposite
                             slots) and a step that pulls from and pushes to the neighbours;
                             every even number of steps the array is in the natural layout
                             and, with F32 storage, bitwise equal to the two-array state.
                             At an odd time every query reads a gathered copy (a transient
                             second array).  Single Patches only (not lbm_batch_create), the
                             register sweep, one cell per thread; lbm_residual is not
                             available (no previous state is kept: lbm_run_to_residual uses
                             a velocity snapshot one step before each check instead). */
    int layout;           /* LBM_LAYOUT_BLOCKS (default): every cell of every Block stored
                             (Sec. 3.2); LBM_LAYOUT_SPARSE: only fluid cells, as a list with
                             18 neighbour indices per cell (periodic images and Block faces
                             resolved in the table, no ghost exchange): 19 x 4 x 2 + 18 x 4
                             = 224 B per fluid-cell update (FP32) against at most 153 B
                             per cell (sectors of only solid cells are not touched); with
                             FP32 sphere packings it measured faster below ~40% fluid
                             cells.  The same results as the
                             Block layout (FP32 bitwise).  Single Patches with two-array
                             streaming, no curved walls. */
} lbm_params;

enum { LBM_KERNEL_AUTO = 0, LBM_KERNEL_REGISTER = 1, LBM_KERNEL_TMA = 2 };
enum { LBM_STREAM_TWO_GRID = 0, LBM_STREAM_AA = 1 };
enum { LBM_LAYOUT_BLOCKS = 0, LBM_LAYOUT_SPARSE = 1 };
enum { LBM_DEBUG_DROP_STAGE = 1 };

typedef struct lbm_ctx lbm_ctx;

/* Fills *p with the defaults listed above. */
void lbm_default_params(lbm_params *p);

/*
 * lbm_create - one Patch (Sec. 4.2) of dims[0]*dims[1]*dims[2] interior
 * cells split into a Cartesian grid of Blocks of block_dims cells each.
 *   dims, block_dims : host int[3]; dims[a] must be a positive multiple of
 *                      block_dims[a] (else LBM_EINVAL).
 *   tau              : relaxation time, > 1/2 (else LBM_EINVAL); omega = 1/tau.
 *   flags            : host uint8[nx*ny*nz] with LBM_FLUID/NOSLIP/MOVING/PRESSURE, x fastest,
 *                      copied; NULL = all fluid.
 *   p                : host, may be NULL for defaults.
 *   out              : receives the context; NULL on failure.
 * Every Block carries a one-cell ghost shell.  Along periodic axes the
 * ghost cells are images of the opposite boundary (filled by the exchange);
 * beyond non-periodic faces they are walls of kind face_bc.  The state starts
 * at rest: f~ = 0 in every cell (Sec. 2.1 initialisation).
 */
int lbm_create(const int dims[3], const int block_dims[3], double tau, const uint8_t *flags,
               const lbm_params *p, lbm_ctx **out);

/*
 * lbm_batch_create - n independent instances (each one single-Block Patch)
 * in one context, advanced together by one sweep launch per step.
 *   dims  : host int[n*3], the interior size of each instance.
 *   tau   : host double[n], one relaxation time per instance (> 1/2).
 *   flags : host array of n pointers to uint8[nx_k*ny_k*nz_k]; the array or
 *           any entry may be NULL (all fluid).
 *   p     : boundary kinds, force, storage etc. shared by all instances.
 */
int lbm_batch_create(int n, const int *dims, const double *tau, const uint8_t *const *flags,
                     const lbm_params *p, lbm_ctx **out);

/* Releases every resource of the context (NULL is ignored). */
void lbm_destroy(lbm_ctx *ctx);

/*
 * lbm_step - advance n >= 0 time steps.  Each step is one Sweep (Sec. 4):
 * the communication step (ghost exchange in device memory) then the work
 * step (fused pull stream + bounce-back + collide, Eq. (1)).  Enqueued on
 * the context stream; device errors surface at the next synchronising call.
 */
int lbm_step(lbm_ctx *ctx, int n);

/* Blocks until all enqueued work of the context has finished.  Returns
 * LBM_ETIMEOUT if a bounded device-side wait of a TMA sweep gave up since the
 * last check (the state is then undefined; reset it with lbm_set_pdfs or
 * lbm_init_equilibrium). */
int lbm_synchronize(lbm_ctx *ctx);

/*
 * lbm_macroscopic - density and velocity of every interior cell of the
 * current state (Sec. 2.1 moments): rho = rho0 + sum f~, u = (sum e f~ - F/2)/rho0.
 * Solid cells report rho0 and 0.  rho: float[N], u: float[3*N].
 * The host variant synchronises; the _device variant writes caller-owned
 * device arrays asynchronously on the context stream.
 */
int lbm_macroscopic(lbm_ctx *ctx, float *rho, float *u);
int lbm_macroscopic_device(lbm_ctx *ctx, float *rho, float *u);

/*
 * lbm_get_pdfs / lbm_set_pdfs - the shifted PDFs f~ of the current state as
 * host double[19*N] (checkpoint / restart and parity interface).  Solid
 * cells read as 0; values written into solid cells are ignored.  With
 * F16S/BF16S storage, set rounds to the storage format.
 */
int lbm_get_pdfs(lbm_ctx *ctx, double *f);
int lbm_set_pdfs(lbm_ctx *ctx, const double *f);

/*
 * lbm_get_pdfs_device / lbm_set_pdfs_device - the same on a caller-owned
 * device double[19*N] in the same layout, enqueued on the context stream
 * (no host copy).  A state read from one context can be set into another of
 * the same geometry and a different storage format: the hand-over from
 * shifted 16-bit to FP32 storage is exact (every 16-bit value divided by a
 * power-of-two scale is an FP32 value).
 */
int lbm_get_pdfs_device(lbm_ctx *ctx, double *f);
int lbm_set_pdfs_device(lbm_ctx *ctx, const double *f);

/*
 * lbm_init_equilibrium - sets every fluid cell to f~eq(rho - rho0, u) of
 * Eq. (2) (warm start from given fields).  rho: float[N], u: float[3*N].
 */
int lbm_init_equilibrium(lbm_ctx *ctx, const float *rho, const float *u);
int lbm_init_equilibrium_device(lbm_ctx *ctx, const float *rho, const float *u);

/*
 * lbm_invariants - FP64 sums over fluid cells of the current state:
 * mass = sum (rho0 + sum f~), momentum = sum (sum e f~ - F/2), and the number
 * of cells holding a NaN or Inf (nonfinite may be NULL).  Host outputs.
 * per_instance != NULL receives 5 doubles per instance
 * {mass, mom_x, mom_y, mom_z, nonfinite}.  Deterministic for a given context.
 */
int lbm_invariants(lbm_ctx *ctx, double *mass, double mom[3], double *nonfinite,
                   double *per_instance);

/*
 * lbm_residual - one-step velocity residual r = ||u_n - u_{n-1}||_2 / ||u_n||_2
 * over fluid cells (FP64), between the current state and the one before the
 * last step.  r = 0 when both norms vanish.  per_instance != NULL receives one
 * residual per instance.  LBM_EINVAL if no step has been taken since the
 * state was last set.
 */
int lbm_residual(lbm_ctx *ctx, double *r, double *per_instance);

/*
 * lbm_run_to_residual - steps in chunks of check_every until the residual
 * falls below tol or max_steps is reached.  *steps receives the steps taken
 * and *r the last residual.  Returns LBM_ENUMERIC if a NaN appears.
 */
int lbm_run_to_residual(lbm_ctx *ctx, double tol, int check_every, long long max_steps,
                        long long *steps, double *r);

/*
 * lbm_set_forces - per-instance body force: force[3*k + a] is component a of
 * the force density of instance k (replaces lbm_params.force for every
 * instance; the Guo source and the moment shift use it).  Synchronises.
 * LBM_EINVAL for a non-finite value.
 */
int lbm_set_forces(lbm_ctx *ctx, const double *force);

/*
 * lbm_impose_velocity_device - in every fluid cell adds
 * f~eq(drho, u_target) - f~eq(drho, u_now) (Eq. (2)), so that the velocity of
 * the moments becomes u_target (device float[3*N], macroscopic layout) while
 * the density and the non-equilibrium part are kept.  Asynchronous.
 *
 * lbm_init_consistent_device - lbm_init_equilibrium_device(rho, u), then
 * `iterations` rounds of one time step followed by
 * lbm_impose_velocity_device(u): the density and the non-equilibrium part
 * relax to values consistent with the prescribed velocity (Mei et al.'s
 * consistent initial conditions), so a warm start from a known velocity
 * field does not begin with the transient of a bare equilibrium.
 */
int lbm_impose_velocity_device(lbm_ctx *ctx, const float *u);
int lbm_init_consistent_device(lbm_ctx *ctx, const float *rho, const float *u, int iterations);

/*
 * lbm_snapshot_velocity - stores the current velocity field (library-owned
 * device copy, float32).  lbm_residual_vs_snapshot - the change per step
 * since then, r = ||u - u_snap||_2 / (steps_since ||u||_2) over fluid cells
 * (FP64 sums; per_instance may be NULL; NaN for an instance holding a
 * non-finite value).  Over an even number of steps this residual is blind to
 * period-2 oscillations, which the one-step residual is not: bounce-back on
 * obstacles in a periodic channel excites an undamped staggered (period-2)
 * mode of the D3Q19 scheme, on which the one-step residual stalls while the
 * flow itself is steady.  LBM_EINVAL before the first snapshot.
 */
int lbm_snapshot_velocity(lbm_ctx *ctx);
int lbm_residual_vs_snapshot(lbm_ctx *ctx, int steps_since, double *r, double *per_instance);

/*
 * lbm_run_to_residual_each - steps a batch in chunks of check_every until
 * every instance's own residual falls below tol or max_steps is reached: the
 * one-step residual of lbm_residual (interval = 0) or the change per step
 * over the chunk (interval = 1, check_every even; lbm_residual_vs_snapshot).  An instance that has converged is frozen: its
 * state is kept (in both buffers) and the sweep skips it, so the remaining
 * work shrinks as instances converge.  steps[k] receives the steps after
 * which instance k first met tol (a multiple of check_every), or -1; res[k]
 * (res may be NULL) its residual then, or its last residual.  Afterwards the
 * context sweeps every instance again.  LBM_ENUMERIC if a residual is NaN;
 * LBM_EINVAL for in-place streaming and the fluid-cell list (single Patches:
 * lbm_run_to_residual).
 */
int lbm_run_to_residual_each(lbm_ctx *ctx, double tol, int check_every, int interval, long long max_steps,
                             long long *steps, double *res);

/*
 * lbm_set_wall_distances - curved resting walls (not in the paper, which
 * leaves further boundary conditions to future work, Sec. 6): linear
 * interpolated bounce-back (Bouzidi, Firdaouss and Lallemand, 2001) on the
 * listed links; every other wall link stays half-way bounce-back.
 *   n      : number of links (0 clears all distances).
 *   cells  : host int64[n], fluid cell of each link in the concatenated cell
 *            numbering of lbm_get_pdfs (instance base + x + nx (y + ny z)).
 *   dirs   : host int[n], the pull direction i (1..18) whose source x - e_i
 *            is a resting wall (LBM_NOSLIP cell or face).
 *   q      : host double[n] in (0, 1], the wall's position x - q e_i along the
 *            link (1/2: half-way).  The pull becomes
 *              q <  1/2: 2q f*_ibar(x) + (1 - 2q) f*_ibar(x + e_i)
 *                        (half-way where x + e_i is not fluid)
 *              q >= 1/2: f*_ibar(x) / (2q) + (1 - 1/(2q)) f*_i(x)
 *            with ibar = opp(i) and f* the stored post-collision state.
 * Replaces the previous set.  The sweeps that carry it are the register
 * sweeps (a context on the TMA sweep switches to them).  LBM_EINVAL for an
 * index, direction or distance out of range, a cell that is not fluid or a
 * source that is not a resting wall (no distance is then set), and for
 * in-place streaming.
 */
int lbm_set_wall_distances(lbm_ctx *ctx, long long n, const long long *cells, const int *dirs, const double *q);

/* Sizes of a context. */
typedef struct {
    long long cells;          /* interior cells over all Blocks / instances */
    long long fluid_cells;    /* interior fluid cells */
    long long stored_cells;   /* cells per PDF buffer including ghost shells and padding */
    int blocks;               /* Blocks (patch) or instances (batch) */
    int instances;
    int storage;
    int bytes_per_pdf;
    long long exchange_pdfs;  /* PDFs copied by one ghost exchange */
    long long device_bytes;   /* device memory held by the context */
    int tile[3];              /* sweep tile in use */
    long long tiles;          /* sweep work items (CTAs) per step */
    int kernel;               /* LBM_KERNEL_REGISTER or LBM_KERNEL_TMA in use */
    int sweep_ctas;           /* CTAs of one sweep launch */
    int stages;               /* pipeline depth of the TMA sweep (0 for the register sweep) */
    int flat;                 /* > 0: the register sweep runs each Block as runs of this many
                                 consecutive cells per CTA (tile[] is then {flat, 1, 1}) */
    int mask;                 /* 1: the register sweep treats near-wall cells through
                                 precomputed link masks under a warp vote */
    int pair;                 /* 1: the register sweep updates two neighbouring cells per
                                 thread (tile[0] then counts threads, each covering 2 cells) */
    int streaming;            /* LBM_STREAM_TWO_GRID or LBM_STREAM_AA */
    int aa_phase;             /* in place: 1 after an odd number of steps (swapped layout) */
    int layout;               /* LBM_LAYOUT_BLOCKS or LBM_LAYOUT_SPARSE */
    long long list_cells;     /* fluid cells in the list (LBM_LAYOUT_SPARSE) */
} lbm_info;
int lbm_get_info(lbm_ctx *ctx, lbm_info *info);

/*
 * Timing of individual launches, for roofline accounting.  While enabled,
 * lbm_step launches without graphs and records a CUDA event pair around
 * every exchange and sweep launch on the context stream.  lbm_profile_read
 * synchronises, returns the accumulated device times in milliseconds and
 * the launch counts, and clears them.
 */
typedef struct {
    double sweep_ms;
    long long sweep_launches;
    double exchange_ms;
    long long exchange_launches;
} lbm_profile;
int lbm_profile_enable(lbm_ctx *ctx, int on);
int lbm_profile_read(lbm_ctx *ctx, lbm_profile *out);

/*
 * lbm_autotune - times each candidate sweep configuration (row tiles, runs
 * of consecutive cells, persistent grids, register budgets, the TMA sweep
 * where it applies) on the context's own data (sweeps from the current state
 * into the scratch buffer, which leaves the simulation state unchanged; in
 * place, pairs of steps with the state saved before and restored after, so
 * that it needs a transient second array and fails with LBM_ENOMEM where
 * that does not fit) and keeps the fastest.  cache_path (may be
 * NULL) names a JSON-lines file: a matching entry is reused instead of
 * timing, a new result is appended.  best (may be NULL) receives the tile.
 */
int lbm_autotune(lbm_ctx *ctx, const char *cache_path, int best[3]);

/*
 * lbm_get_sweep_config / lbm_set_sweep_config - the sweep configuration that
 * lbm_autotune chooses, as 8 ints {kind, tx, ty, tz, grid, minb, zchunk,
 * mask}: kind 0 = register sweep over row tiles of tx x ty cells and tz z
 * slices (tx a multiple of 32, tx*ty <= 256); 1 = TMA-staged sweep (only where
 * it applies) with zchunk z slices per work item; 2 = register sweep over
 * runs of tx consecutive cells (32..256, a multiple of 32); 3 and 4 = kinds 0
 * and 2 with two neighbouring cells per thread (tx threads cover 2 tx cells;
 * even Block widths, FP32 / F16S / BF16S storage); grid = CTAs of a
 * persistent launch (0 = one per work item); minb = 3 or 4 resident CTAs per
 * SM the register budget allows (FP64 storage always uses 2), or 5 (48
 * registers) for the one-cell register sweep (kinds 0 and 2) of two-array
 * Block layouts, whose Patches with pressure boundaries or curved walls run
 * the budget-4 kernels instead; mask = 1 treats
 * near-wall cells through precomputed link masks under a warp vote.  Every
 * configuration gives bitwise identical results.  In-place streaming takes
 * kinds 0, 2, 3 and 4 with mask 0 (its tuning saves and restores the state
 * around the timed steps, a transient second array); the fluid-cell list
 * uses only grid and minb.  LBM_EINVAL for an invalid or inapplicable
 * configuration (the context is then unchanged).
 */
int lbm_get_sweep_config(lbm_ctx *ctx, int cfg[8]);
int lbm_set_sweep_config(lbm_ctx *ctx, const int cfg[8]);

/* Device memory hooks: alloc(bytes, stream, user) returns a device pointer or
 * NULL; release(ptr, bytes, stream, user) frees it.  Passing NULL restores
 * cudaMalloc/cudaFree.  Applies to contexts created afterwards. */
typedef void *(*lbm_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*lbm_free_fn)(void *ptr, size_t bytes, void *stream, void *user);
int lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn release, void *user);

/* The direction table above: e int[57] (q-major triples), w double[19],
 * opp int[19].  Host only, needs no GPU. */
int lbm_directions(int *e, double *w, int *opp);

/*
 * lbm_invariants_noalloc - the FP64 sums of lbm_invariants for callers that
 * cannot allocate device memory.  The paper has no counterpart; it exists for
 * callers that run where cudaMalloc is not allowed or not safe: inside a
 * framework's allocator callback (a new allocation would re-enter it), or
 * when a caching allocator already holds all device memory (cudaMalloc
 * fails).
 *   f       : device, float[19*n_cells], shifted PDFs, direction-major
 *             (f[q*n_cells + c]); caller-owned.
 *   flags   : device, uint8[n_cells] (LBM_FLUID = 0 is summed), or NULL = all fluid.
 *   rho0, force : as in lbm_params; mass = sum (rho0 + sum f~),
 *             momentum = sum (sum e f~ - F/2) over fluid cells.
 *   out     : device-accessible double[5] = {mass, mom_x, mom_y, mom_z, nonfinite}.
 *   stream  : cudaStream_t to enqueue on (NULL = legacy default stream).
 * Allocates nothing: partial sums go to a fixed file-scope device array of
 * 2 MiB (32768 partials of 2048 cells), which every GPU that loads the
 * library holds until the process exits.  n_cells above 67108864 returns
 * LBM_EINVAL.  The first call on a device looks the array up with
 * cudaGetSymbolAddress; make that first call before any stream capture.
 * Every call reuses the same array, so calls that overlap on the GPU (other
 * streams, other threads) race; every slot a call reads it writes first.
 * Asynchronous: out is valid once the stream has reached the call.
 */
int lbm_invariants_noalloc(const float *f, const uint8_t *flags, long long n_cells, double rho0,
                           const double force[3], double *out, void *stream);

/* Message of the last failure on ctx, or of the calling thread's last failed
 * lbm_create / lbm_batch_create when ctx is NULL.  Never NULL. */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Library version string, e.g. "lbm 0.1 sm_103a". */
const char *lbm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
