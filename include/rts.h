/*
 * rts.h - C ABI of librts: regional time stepping (RTS) for WCSPH and PCISPH on one
 * GB300 GPU (sm_103a).
 *
 * Method: Goswami & Batty, "Asynchronous Liquids: Regional Time Stepping for Faster SPH
 * and PCISPH".  The library advances fluid particles among static boundary particles.
 * Particles are binned into a uniform block grid (Section 3); every filled block takes
 * a time-step level from the maximum velocity and force of its particles (Section 3.1,
 * Eq. 1-3), smoothed at region borders (R_min, Section 4.2); WCSPH evaluates density,
 * pressure and forces only for the particles whose true step ends at the current base
 * substep and integrates everyone with the Serna predictor-corrector (Section 4.1,
 * Algorithm 1); PCISPH assigns density-correction iterations per region and refreshes
 * neighbourhoods asynchronously (Section 5, Algorithms 2 and 3).
 *
 * Conventions shared by every entry point:
 *  - Pointers to particle arrays may be host or device pointers (unified addressing
 *    resolves them); they are borrowed for the duration of the call and copied.
 *    Vectors are n x 3 floats (x, y, z), contiguous, in the caller's particle order.
 *  - All work is enqueued on the CUDA stream given to rts_init (borrowed; 0 = legacy
 *    default stream).  Calls that return data to the caller synchronise that stream.
 *    Dependent kernels of a call are launched with programmatic dependencies: each is
 *    scheduled while the work before it drains but waits for that work to complete
 *    before its first memory access, so stream order holds for the caller's own work on
 *    the same stream as for any other launch.
 *  - Every call returns an rts_status and never throws or aborts.  Argument errors are
 *    returned at once.  Errors found on the device (particle outside the grid, block
 *    over capacity, PCISPH non-convergence) are recorded in a device status word and
 *    returned by the next call that synchronises (rts_sync, rts_advance, rts_get_*).
 *    Such an error is sticky: later stepping calls return RTS_ERR_STATE until
 *    rts_set_state installs a new state.  rts_last_error gives a message.
 *  - The context owns all its device memory (allocated in rts_init, freed by
 *    rts_destroy).  Internally particles are kept in block order; rts_get_state
 *    returns the caller's order.
 */
#ifndef RTS_H
#define RTS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rts_status {
  RTS_OK = 0,
  RTS_ERR_ARG = 1,            /* invalid argument (returned before any work)            */
  RTS_ERR_DOMAIN = 2,         /* a particle left the block grid, or a NaN position       */
  RTS_ERR_CUDA = 3,           /* a CUDA runtime call failed                              */
  RTS_ERR_OOM = 4,            /* device allocation failed                                */
  RTS_ERR_CAPACITY = 5,       /* a block exceeded max_per_block, or a neighbour list
                                 exceeded max_neighbors                                  */
  RTS_ERR_NOT_CONVERGED = 6,  /* PCISPH: a minor step hit max_iters (state is advanced)  */
  RTS_ERR_TIMEOUT = 7,        /* a bounded device wait gave up                           */
  RTS_ERR_STATE = 8,          /* an earlier device error is pending; call rts_set_state  */
  RTS_ERR_INTERNAL = 9        /* a device-side consistency check failed (an index read from
                                 memory was out of range; the access was skipped)          */
} rts_status;

enum { RTS_WCSPH = 0, RTS_PCISPH = 1 };

/* mode: regional time stepping (the paper's method), or a global comparator in which
 * every particle is active every step: adaptive (the finest level that Eq. 1-3 give for
 * the whole fluid) or constant (dt_b). */
enum { RTS_MODE_REGIONAL = 0, RTS_MODE_GLOBAL_ADAPTIVE = 1, RTS_MODE_GLOBAL_CONSTANT = 2 };

/* Parameters (Sections 3-6).  Lengths in metres, times in seconds, SI throughout. */
typedef struct rts_params {
  int32_t scheme;            /* RTS_WCSPH or RTS_PCISPH                                   */
  int32_t mode;              /* RTS_MODE_*                                                */
  int32_t force_level;       /* -1: classify blocks; >= 0: every filled block takes this
                                level (test hook: 0 reproduces global stepping at dt_b)   */
  float spacing;             /* s, initial particle spacing                               */
  float support_r;           /* r, kernel support radius (= 2h of the cubic spline)       */
  float block_edge;          /* block edge: r for WCSPH (Section 3), 2.2 s for PCISPH
                                (Section 5.6); must be >= support_r                       */
  float domain_min[3];       /* grid origin                                               */
  int32_t grid_dim[3];       /* blocks per axis; the grid spans domain_min + dim * edge   */
  float rho0, c_s, gamma, visc_alpha;   /* rest density, sound speed, Tait exponent,
                                           artificial viscosity alpha                    */
  float gravity[3];
  float lambda_v, lambda_f, alpha;      /* Eq. 1, Eq. 2, Eq. 3 coefficients               */
  int32_t n_levels;          /* number of levels (<= 8)                                    */
  int32_t level_mult[8];     /* dt of level L = level_mult[L] * dt_b (increasing)          */
  float beta[8];             /* beta of level L in Eq. 3 (beta[0] = +inf)                  */
  float dt_b;                /* base (smallest) step                                       */
  int32_t max_per_block;     /* block capacity (fluid particles per block), <= 1024        */
  /* PCISPH (Section 5) */
  int32_t n_minor;           /* minor steps per major step (N = 4)                         */
  float eta;                 /* allowed density error (relative), 0.01                     */
  float eta_T;               /* average-error threshold for global extra iterations        */
  int32_t max_iters;         /* iteration cap per minor step                               */
  int32_t max_global_iters;  /* global iterations after which major steps are shortened    */
  int32_t max_local_iters;   /* local iterations before reverting to global                */
  int32_t expand_layers;     /* dilation of regions 1 and 2 (4 blocks)                     */
  int32_t r1_search_rings;   /* neighbour search rings for region 1 (2)                    */
  int32_t clean_majors;      /* clean major steps before the major step is restored (10)   */
  int32_t short_minor;       /* minor steps of a shortened major step (2)                  */
  int32_t sched[4][8];       /* correction iterations of region n in minor step j          */
  int32_t refresh[8];        /* neighbourhood validity of region n, in minor steps         */
  int32_t max_neighbors;     /* PCISPH neighbour list capacity per particle                */
  /* Container (the paper gives no boundary handling beyond static boundary particles):
     with wall_project = 1 a fluid particle that crosses a face of the box
     [wall_lo, wall_hi] after a position update is put back on that face and loses its
     velocity component into it (non-penetration); 0: off.                            */
  int32_t wall_project;
  float wall_lo[3], wall_hi[3];
  /* WCSPH activity clock.  0: Algorithm 1 as stated: a particle that computes takes
     validity = its level's multiplier, so particles of one block drift out of phase.
     1: level-aligned variant: validity = mult - (k mod mult), so every particle of level
     L computes at the substeps k that are multiples of mult[L] (plus pre-emptions).   */
  int32_t level_clock;
  /* Tait stiffness B; 0 derives it from the sound speed, B = c_s^2 rho0 / gamma (the
     viscosity keeps using c_s).  A separate value lets B be varied on its own.        */
  float tait_B;
  /* 0: the Tait pressure is clamped at zero (free-surface particles do not attract);
     1: negative pressure is kept (the equation of state is then smooth everywhere).  */
  int32_t tait_no_clamp;
  /* Ablations of the paper's choices (off by default).  serna_off = 1: the Section 4.1
     correction is skipped (an evaluated particle keeps its predicted position and
     velocity; its held acceleration is still replaced), the paper's Fig. 3 comparison.
     r2_search_rings: neighbour search rings of PCISPH region 2 (0 or 1 = one ring; the
     paper searches two rings for region 1 only).                                      */
  int32_t serna_off;
  int32_t r2_search_rings;
  /* Re-sorting with the level-aligned clock (level_clock = 1, WCSPH, regional).  S =
     stale_bins > 1: a substep whose index is not a multiple of S keeps the particle
     order of the last sort instead of sorting again.  Classification and activity use
     every particle's current block as always; the density pass searches, around each
     group of evaluated particles, the sorted blocks widened by the largest distance a
     particle has left its sorted block since that sort, so the neighbour sets are
     exactly those of a fresh sort (only the order of summation differs).  With S = 2
     the kept substeps are those at which only the finest level is due.  0 or 1: sort
     every substep.  A particle that moves half a block or more between sorts is
     reported as RTS_ERR_INTERNAL (check 8): lower stale_bins for such flows.             */
  int32_t stale_bins;
} rts_params;

/* Counters accumulated over one rts_advance call. */
typedef struct rts_stats {
  int64_t substeps;          /* base substeps (dt_b) advanced                              */
  int64_t steps;             /* calls of the step kernel sequence (global steps may span
                                several substeps)                                          */
  int64_t particle_evals;    /* particles whose density and acceleration were evaluated   */
  int64_t pair_interactions; /* neighbour pairs (d < r) of those evaluations               */
  int64_t active_blocks;     /* sum over steps of blocks with an evaluated particle        */
  int64_t level_count[8];    /* fluid particles per level at the end of the call           */
  int64_t candidate_tests;   /* candidates in the evaluated particles' 27-block stencils   */
  int64_t tests_performed;   /* distance tests after culling the stencil to each group's
                                bounding box (WCSPH)                                       */
  int64_t pcisph_iterations; /* density-correction iterations                              */
  int64_t pcisph_local_iterations;
  int64_t pcisph_global_restarts;
  double t_sim;              /* simulated time at the end of the call                      */
} rts_stats;

typedef struct rts_ctx rts_ctx;

/* Create a context.  x, v: n_fluid x 3 positions and velocities; xb: n_boundary x 3
 * static boundary positions.  The state starts unprimed: accelerations, validity and
 * levels are zero, and the first stepping call first evaluates every particle at the
 * current time (Section 4.1 needs an acceleration to predict with).
 * Errors: RTS_ERR_ARG (bad sizes or parameters), RTS_ERR_OOM, RTS_ERR_CUDA,
 * RTS_ERR_DOMAIN (a boundary particle outside the grid). */
rts_status rts_init(const rts_params* params, int32_t n_fluid, const float* x, const float* v,
                    int32_t n_boundary, const float* xb, void* cuda_stream, rts_ctx** out);

/* Section 3: bin the fluid particles at their current positions into the block grid
 * (sorted by block, then by the caller's particle index). */
rts_status rts_bin(rts_ctx* ctx);

/* Section 3.1 and 4.2: block maxima of |v| and |a|, level per filled block from
 * Eq. 1-3, then the R_min smoothing (or force_level).  Uses the current bins. */
rts_status rts_classify_blocks(rts_ctx* ctx);

/* Evaluate density, pressure and acceleration of every fluid particle at the current
 * state, without advancing time (the priming evaluation of the Serna scheme): bins,
 * classifies, sets every particle's level and validity from its block, the held
 * acceleration to the new one and the last-evaluation substep to the current one. */
rts_status rts_evaluate(rts_ctx* ctx);

/* One WCSPH base substep dt_b (Algorithm 1, Section 4.1): predict all particles, bin,
 * classify, decrement validity and pre-empt on a level change, evaluate the active
 * particles against every particle's predicted state, correct the active particles.
 * In a global mode, one global step of mult * dt_b instead (see rts_advance). */
rts_status rts_wcsph_substep(rts_ctx* ctx);

/* One PCISPH minor step dt_b (Algorithm 2 with Algorithm 3 for density correction).
 * Region assignment, grid and neighbourhood refresh happen at major-step starts.  In a
 * global mode, one plain PCISPH step of mult * dt_b for every particle instead (mult from
 * the whole fluid's maxima, or 1), with a fresh grid and fresh neighbourhoods. */
rts_status rts_pcisph_step(rts_ctx* ctx);

/* Advance to simulated time t_sim (rounded to whole base substeps) with the context's
 * scheme and mode; synchronises.  out may be NULL. */
rts_status rts_advance(rts_ctx* ctx, double t_sim, rts_stats* out);

/* Copy the state out in the caller's order.  Any pointer may be NULL.  x, v, a are
 * n x 3; level, validity, klast, nbr are n int32; compute is n bytes (1 = evaluated by
 * the last step).  a is the held acceleration; nbr the neighbour count (excluding the
 * particle itself) at the last evaluation.  Synchronises. */
rts_status rts_get_state(rts_ctx* ctx, float* x, float* v, float* a, float* rho, float* p,
                         int32_t* level, int32_t* validity, int32_t* klast, int32_t* nbr,
                         uint8_t* compute);

/* Install a state (caller's order).  x, v required; the others may be NULL (then zero,
 * rho0 for rho).  k: completed base substeps; primed: 0 = evaluate before the next
 * step.  Clears a pending device error. */
rts_status rts_set_state(rts_ctx* ctx, const float* x, const float* v, const float* a,
                         const float* rho, const float* p, const int32_t* level,
                         const int32_t* validity, const int32_t* klast, int64_t k,
                         int32_t primed);

/* Bins of the last rts_bin / step: key (block id of each particle, caller's order),
 * perm (caller's index of the particle at each sorted position), cstart (n_blocks + 1
 * exclusive prefix of the block counts).  Any pointer may be NULL.  Synchronises. */
rts_status rts_get_bins(rts_ctx* ctx, int32_t* key, int32_t* perm, int32_t* cstart);

/* Block levels of the last classification (n_blocks int32, -1 = no fluid): raw from
 * Eq. 1-3, level after R_min smoothing.  For a PCISPH context, level is the region
 * field of the current major step (R_min, region expansion, pre-emption).
 * Any pointer may be NULL.  Synchronises. */
rts_status rts_get_blocks(rts_ctx* ctx, int32_t* raw, int32_t* level);

/* Phases timed by the optional profiler (CUDA events on the context's stream).  The
 * paper's Table 2 buckets map as: neighbour = BIN (+ the neighbour walk inside DENSITY
 * and FORCE); physics = DENSITY + FORCE + CORRECT; RTS = CLASSIFY + ACTIVITY. */
enum {
  RTS_PHASE_BIN = 0,       /* predict + block key + counting sort + gather              */
  RTS_PHASE_CLASSIFY = 1,  /* block maxima, Eq. 1-3 levels, R_min (+ PCISPH regions)     */
  RTS_PHASE_ACTIVITY = 2,  /* validity, pre-emption, active-block work list             */
  RTS_PHASE_DENSITY = 3,   /* WCSPH density / PCISPH neighbour lists                     */
  RTS_PHASE_FORCE = 4,     /* WCSPH forces / PCISPH non-pressure forces                  */
  RTS_PHASE_CORRECT = 5,   /* Serna correction / PCISPH integration                      */
  RTS_PHASE_ITERATE = 6,   /* PCISPH density-correction iterations                       */
  RTS_PHASE_OTHER = 7,     /* global maxima, statistics, caller-order I/O                */
  RTS_NUM_PHASES = 8
};

typedef struct rts_profile {
  double ms[RTS_NUM_PHASES];         /* device time of the timed instances of each phase   */
  int64_t launches[RTS_NUM_PHASES];  /* kernel launches per phase                          */
  int64_t kernels;                   /* all kernel launches of this library                */
  int64_t timed[RTS_NUM_PHASES];     /* phase instances that were timed                    */
  int64_t passes[RTS_NUM_PHASES];    /* phase instances (a sorted density pass launches
                                        two kernels, of which one returns at once)         */
} rts_profile;

/* Per-phase event timing: 0 off; 1 every phase instance; 2 every 7th instance of the
 * density and of the force pass only (a sample whose stride is prime to the level
 * cycles: the lightest way to time the neighbour kernels inside a long run; the
 * average duration is ms / timed).  Launch counts are always kept.  RTS_ERR_ARG for
 * other values. */
rts_status rts_profile_enable(rts_ctx* ctx, int32_t on);

/* Read the accumulated profile (synchronises); reset != 0 clears it afterwards. */
rts_status rts_profile_read(rts_ctx* ctx, rts_profile* out, int32_t reset);

/* Statistics of the last PCISPH minor step (Algorithm 3). */
typedef struct rts_pcisph_info {
  int32_t iterations;        /* density-correction iterations                         */
  int32_t global_iterations; /* iterations in which every region had a turn          */
  int32_t local_iterations;  /* iterations on S_e only (Section 5.5)                  */
  int32_t reverts;           /* local runs that failed and restored the pressures    */
  int32_t not_converged;     /* 1 if max_iters was reached                           */
  int32_t minor;             /* minor step the next call will take                   */
  int32_t n_minor_current;   /* minor steps of the current major step (N or short)   */
  int32_t clean_majors;      /* shortened major steps without an overrun so far      */
  double err_max, err_avg;   /* maximum and average relative compression error       */
} rts_pcisph_info;

rts_status rts_pcisph_last(rts_ctx* ctx, rts_pcisph_info* out);

/* PCISPH state in the caller's order: ap (n x 3) pressure acceleration of the last minor
 * step, err (n) latest relative compression error max(0, rho* - rho0) / rho0, in_se (n)
 * membership of S_e.  Any pointer may be NULL.  Synchronises. */
rts_status rts_get_pcisph_state(rts_ctx* ctx, float* ap, float* err, uint8_t* in_se);

/* Neighbour lists of the last evaluation, caller's order: counts (n); idx (n x cap,
 * may be NULL) with fluid j as j and boundary particle b as n + b (caller indices).
 * WCSPH: valid for the particles the last step evaluated; PCISPH: the lists in use.
 * RTS_ERR_CAPACITY if a list is longer than cap.  Synchronises. */
rts_status rts_get_neighbors(rts_ctx* ctx, int32_t* counts, int32_t* idx, int32_t cap);

/* Wait for the stream; return a pending device error, if any. */
rts_status rts_sync(rts_ctx* ctx);

/* Allocation-free binning.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory - hosts that reserve the whole GPU at
 * start-up (a later cudaMalloc would fail), loops with a latency budget that an
 * allocation's implicit synchronisation would break, and plugin hosts that own all
 * device memory.  It computes what rts_bin followed by rts_get_bins gives (block of
 * each particle, particles ordered by block then index, block starts) with no context
 * and no allocation: its working memory is a fixed array of about 5 MB compiled into
 * the library, present on every device that loads the library until the process
 * exits.
 *   x: n x 3 floats, key: n, perm: n, cstart: nblocks + 1, all in device memory;
 *   n <= RTS_NOALLOC_MAX_PARTICLES and grid_dim[0]*grid_dim[1]*grid_dim[2] <=
 *   RTS_NOALLOC_MAX_BLOCKS, else RTS_ERR_ARG (nothing is launched).
 * Only the block grid fields of params are read.  The call synchronises the stream and
 * returns RTS_ERR_DOMAIN if a particle lies outside the grid (key, perm and cstart are
 * then unspecified), RTS_ERR_CAPACITY if a block holds more than
 * RTS_NOALLOC_MAX_PER_BLOCK particles (the in-block order by index is found by a scan of
 * the block, quadratic in its occupancy, so the cap bounds a call's work), and
 * RTS_ERR_CUDA, with nothing launched, if a CUDA error from earlier work was pending on
 * the calling thread (it is cleared and named in rts_last_error(NULL)).  A failed call
 * leaves nothing behind: the next call starts from cleared counters.  The first call on a
 * device looks up the array's device address (once per device); make that first call
 * before any stream capture.  Every call shares the one array: calls whose work can
 * overlap on the GPU (other streams, other host threads) race and must be serialised. */
#define RTS_NOALLOC_MAX_PARTICLES 262144
#define RTS_NOALLOC_MAX_BLOCKS 524288
#define RTS_NOALLOC_MAX_PER_BLOCK 4096
rts_status rts_bin_noalloc(const rts_params* params, int32_t n, const float* x, int32_t* key,
                           int32_t* perm, int32_t* cstart, void* cuda_stream);

int64_t rts_num_blocks(const rts_ctx* ctx);
int64_t rts_substep_index(const rts_ctx* ctx);   /* completed base substeps */
const char* rts_last_error(const rts_ctx* ctx);  /* never NULL; ctx may be NULL */
rts_status rts_destroy(rts_ctx* ctx);            /* NULL is a no-op */

/* -------------------------------------------------------- batched scenes --- */
/* Many independent RTS-PCISPH scenes (Section 5, Algorithms 2 and 3) advanced together.
 * The paper treats one scene; batching is this library's addition.  Each scene keeps its
 * own block grid, container and density-correction control: every scene runs the
 * iterations, S_e / R_ob sets, local runs and reverts of Algorithm 3 on its own errors,
 * exactly as it would alone.  The scenes share the parameters (physics, dt_b, regions,
 * schedule) and the major-step clock: when any scene exceeds max_global_iters the batch
 * shortens its major step (Section 5.5).  One launch of each pass serves all scenes;
 * the iterations of a minor step run as one CUDA graph (a while node driven by the
 * device-side control) over a work queue of the scenes still iterating.
 *
 * The context is an ordinary rts_ctx: rts_pcisph_step / rts_advance step every scene by
 * one minor step / to t_sim; rts_get_state, rts_set_state, rts_get_pcisph_state,
 * rts_get_neighbors, rts_sync, rts_destroy work on the concatenation of the scenes in
 * the caller's order (scene 0's particles first).  rts_get_bins / rts_get_blocks return
 * the stacked grid (rts_batch_layout gives each scene's place in it).  In rts_stats,
 * pcisph_iterations counts scene-iterations (the sum over scenes); rts_pcisph_last
 * reports the iterations the batch ran in its last minor step (the largest scene count),
 * the largest global and local counts and the largest error of any scene. */
typedef struct rts_scene {
  int32_t n_fluid;           /* fluid particles of the scene (consecutive in x, v)        */
  int32_t n_boundary;        /* boundary particles of the scene (consecutive in xb)       */
  float domain_min[3];       /* origin of the scene's block grid, in its own coordinates  */
  int32_t grid_dim[3];       /* blocks per axis of the scene's grid, each in [1, 4096]    */
  float wall_lo[3], wall_hi[3];  /* the scene's container (when params->wall_project)    */
} rts_scene;

/* params: shared parameters (scheme RTS_PCISPH, mode RTS_MODE_REGIONAL; domain_min,
 * grid_dim, wall_lo and wall_hi are taken from each scene instead).  scenes: n_scenes
 * descriptions, 1 <= n_scenes <= 1024.  x, v: all scenes' fluid particles concatenated
 * (sum of n_fluid x 3); xb: all boundary particles concatenated.  Pointers as for
 * rts_init (host or device, copied).  The scenes are stacked along z in one grid with
 * max(expand_layers, r1_search_rings, r2_search_rings, 1) empty block layers between two
 * scenes.
 * Errors: RTS_ERR_ARG, RTS_ERR_OOM, RTS_ERR_CUDA, RTS_ERR_DOMAIN (a boundary particle
 * outside its scene's grid). */
rts_status rts_batch_init(const rts_params* params, int32_t n_scenes, const rts_scene* scenes,
                          const float* x, const float* v, const float* xb, void* cuda_stream,
                          rts_ctx** out);

/* Algorithm 3 statistics of one scene in the last minor step (iterations, global, local,
 * reverts, not_converged, err_max, err_avg are the scene's; minor, n_minor_current and
 * clean_majors the batch's).  Reads what the last step copied back: no synchronisation.
 * RTS_ERR_ARG for a context that is not a batch or a scene out of range. */
rts_status rts_batch_scene_info(rts_ctx* ctx, int32_t scene, rts_pcisph_info* out);

/* Placement of the scenes: grid_dim (3) of the stacked grid; z0 (n_scenes + 1) first z
 * layer of each scene (z0[n_scenes] = the grid's layers); fluid_base and boundary_base
 * (n_scenes + 1) first particle of each scene in the concatenated arrays.  A block
 * (bx, by, bz) of scene s is the stacked block ((bz + z0[s]) * ny + by) * nx + bx.
 * Any pointer may be NULL. */
rts_status rts_batch_layout(const rts_ctx* ctx, int32_t* grid_dim, int32_t* z0,
                            int32_t* fluid_base, int32_t* boundary_base);

/* Launch shape of the iteration passes: threads per CTA of the persistent work-queue
 * kernels (a multiple of 32 in [64, 1024]); tile, particles per queue item (a multiple
 * of 32 in [32, 8192]); use_graph 1 runs the iterations as a captured CUDA graph, 0 from
 * the host (one round trip per iteration).  The results do not depend on any of these.
 * Defaults: 256, 128, 1.  RTS_ERR_ARG otherwise. */
rts_status rts_batch_set_launch(rts_ctx* ctx, int32_t threads, int32_t tile, int32_t use_graph);
rts_status rts_batch_get_launch(const rts_ctx* ctx, int32_t* threads, int32_t* tile,
                                int32_t* use_graph, int64_t* iterations_run);

/* Autotuner: times one full iteration (every particle of every scene participating) for
 * threads in {128, 256, 512} x tile in {32, 64, 128, 256, 512}, reps timed runs each after a
 * warm-up, on the current state, which it restores afterwards; keeps the fastest shape
 * and returns it with its time per iteration (ms).  Needs the neighbour lists of a
 * previous step (RTS_ERR_STATE before the first step).  Synchronises. */
rts_status rts_batch_autotune(rts_ctx* ctx, int32_t reps, int32_t* threads, int32_t* tile,
                              float* ms_per_iteration);

/* ------------------------------------------------ differentiable rollout --- */
/* No counterpart in the paper: a WCSPH rollout under global constant stepping at dt_b
 * (every particle active every step; the Serna predictor-corrector of Section 4.1 and the
 * same physics, boundary particles and container as the regional path) with its
 * hand-written adjoint, for gradients of a loss of the final state with respect to the
 * initial velocities, the Tait stiffness B and the viscosity coefficient alpha.  The
 * priming evaluation a_0 = A(x_0, v_0) starts the rollout; after n_steps steps it returns
 * x_T and rho_T = rho(x_T) (summation density at x_T).  Particles keep the caller's order.
 * The backward pass stores (x, v, a) every ckpt_every steps during the forward pass and
 * recomputes each segment (its evaluation points, neighbour lists and container masks)
 * before reversing it. */
typedef struct rts_diff rts_diff;

/* params: as for rts_init (scheme RTS_WCSPH; mode, levels and c_s's role in B are ignored:
 * B and alpha are given per forward call; the viscosity uses c_s).  x0: n_fluid x 3 initial
 * positions; xb: n_boundary x 3 static boundary positions (host or device, copied).
 * Device memory grows with n_fluid x max_neighbors x ckpt_every.
 * Errors: RTS_ERR_ARG, RTS_ERR_OOM, RTS_ERR_CUDA, RTS_ERR_DOMAIN (a boundary particle
 * outside the grid); the message is rts_last_error(NULL). */
rts_status rts_diff_create(const rts_params* params, int32_t n_fluid, const float* x0,
                           int32_t n_boundary, const float* xb, int32_t n_steps,
                           int32_t ckpt_every, void* cuda_stream, rts_diff** out);

/* Run the rollout from (x0, v0) with stiffness tait_B and viscosity visc_alpha.  v0:
 * n x 3 (host or device); x_out (n x 3) and rho_out (n) may be NULL.  Synchronises.
 * Errors: RTS_ERR_ARG, RTS_ERR_DOMAIN (a particle left the grid), RTS_ERR_CAPACITY (a
 * neighbour list exceeded max_neighbors), RTS_ERR_CUDA; sticky (RTS_ERR_STATE after). */
rts_status rts_diff_forward(rts_diff* d, const float* v0, float tait_B, float visc_alpha,
                            float* x_out, float* rho_out);

/* Gradients for the adjoints gx = dL/dx_T (n x 3) and grho = dL/drho_T (n) of the last
 * forward (either may be NULL for zero): gv0 = dL/dv0 (n x 3, host or device), *gB =
 * dL/dB and *galpha = dL/dalpha (host doubles, may be NULL).  Synchronises; the forward
 * must be run again before the next backward.  Errors: RTS_ERR_STATE (no forward),
 * RTS_ERR_ARG, RTS_ERR_CUDA. */
rts_status rts_diff_backward(rts_diff* d, const float* gx, const float* grho, float* gv0,
                             double* gB, double* galpha);

const char* rts_diff_last_error(const rts_diff* d);
void rts_diff_destroy(rts_diff* d);

#ifdef __cplusplus
}
#endif
#endif
