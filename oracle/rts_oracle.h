/*
 * rts_oracle.h - FP64 CPU oracle for regional time stepping (RTS) of WCSPH and PCISPH.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously correct restatement of
 * Goswami & Batty, "Asynchronous Liquids: Regional Time Stepping for Faster SPH and
 * PCISPH", written from the paper.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table or
 * constant with the CUDA library; both receive the same seeded inputs.
 *
 * All arithmetic is IEEE double with round-to-nearest and no contraction
 * (built with -ffp-contract=off).  Arrays are in the caller's (user) order:
 * positions, velocities and accelerations are n x 3 doubles.  Discrete decisions
 * (block index, neighbour predicate, level thresholds) are evaluated exactly on the
 * stored values, which parity tests fill from FP32 inputs.
 *
 * Parity status per function is given next to each declaration:
 *   pinned   - checked by a -m "not gpu" test against a value fixed independently
 *              of this code (closed form, brute force, invariant, special case)
 *   parity unpinned - no independent pin exists (the paper is silent or the figure
 *              that defines it is missing); self-consistency checks only.
 */
#ifndef RTS_ORACLE_H
#define RTS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_DOMAIN = 2, ORC_ERR_CAPACITY = 5,
       ORC_ERR_NOT_CONVERGED = 6 };

typedef struct orc_params {
  int32_t scheme;          /* 0 WCSPH, 1 PCISPH */
  int32_t mode;            /* 0 regional, 1 global adaptive, 2 global constant */
  int32_t force_level;     /* -1 classify; >= 0 every filled block takes this level */
  double s, r, edge;       /* spacing, kernel support radius (= 2h), block edge */
  double origin[3];
  int32_t dim[3];
  double rho0, c_s, gamma, visc_alpha;
  double g[3];
  double lambda_v, lambda_f, alpha;
  int32_t n_levels;
  int32_t mult[8];         /* dt_L = mult[L] * dt_b */
  double beta[8];          /* beta for level L (beta[0] = inf) */
  double dt_b;
  int32_t max_per_block;
  /* PCISPH */
  int32_t n_minor;
  double eta, eta_T;
  int32_t max_iters, max_global_iters, max_local_iters;
  int32_t expand_layers, r1_rings, clean_majors, short_minor;
  int32_t sched[4][8];     /* correction iterations per region per minor step */
  int32_t refresh[8];      /* neighbourhood validity per region, minor steps */
  int32_t max_neighbors;
  /* Container box: with wall_project = 1 a particle beyond a face after a position
   * update is put back on the face and its velocity component into it is dropped. */
  int32_t wall_project;
  double wall_lo[3], wall_hi[3];
  /* WCSPH activity clock: 0 validity = level multiplier (Algorithm 1); 1 validity up to
   * the next multiple of the multiplier (level-aligned variant). */
  int32_t level_clock;
  double tait_B;           /* Tait stiffness; 0: c_s^2 rho0 / gamma */
  int32_t tait_no_clamp;   /* 1: negative Tait pressure kept */
  /* Ablations.  serna_off = 1: the Section 4.1 correction is not applied (an evaluated
   * particle keeps its predicted position and velocity; the held acceleration is still
   * replaced).  r2_rings: neighbour search rings of region 2 (PCISPH), 0 or 1 = one. */
  int32_t serna_off;
  int32_t r2_rings;
} orc_params;

/* WCSPH state in user order. */
typedef struct orc_wstate {
  int32_t n, nb;
  double *x, *v, *a;       /* 3n each; a = held acceleration of the last evaluation */
  double *rho, *p;         /* n */
  int32_t *klast;          /* n: substep index of the last evaluation */
  int32_t *validity;       /* n */
  int32_t *level;          /* n: particle level (-1 = none yet) */
  uint8_t *compute;        /* n: output - particle evaluated in the last call */
  int32_t *nbr;            /* n: neighbours (excluding self) at the last evaluation */
  const double *xb;        /* 3nb static boundary positions */
  int32_t *block_level;    /* B: output - level per block (-1 = no fluid) */
  int64_t k;               /* completed base substeps */
  int32_t primed;
} orc_wstate;

/* Threads used by the OpenMP loops (omp_get_max_threads). */
int orc_num_threads(void);

/* Cubic-spline (M4) kernel in 3D, support 2h [pinned: normalisation, symmetry]. */
double orc_kernel_W(double d, double h);
double orc_kernel_dW(double d, double h);   /* dW/dd */

/* Block grid (Section 3) [pinned: brute-force key/sort check]. */
int orc_block_key(const orc_params* P, const double* x3, int32_t* key);
int orc_bin(const orc_params* P, int32_t n, const double* x, int32_t* key,
            int32_t* perm, int32_t* cstart);

/* Neighbour sets N(i) = { j != i : |x_i - x_j|^2 < r^2 }; fluid j as j, boundary b
 * as n + b.  offsets has n + 1 entries; idx may be NULL to count only.
 * [pinned: grid search equals brute force] */
int64_t orc_neighbors_brute(int32_t n, const double* x, int32_t nb, const double* xb,
                            double r, int32_t* offsets, int32_t* idx);
int64_t orc_neighbors_grid(const orc_params* P, int32_t n, const double* x, int32_t nb,
                           const double* xb, int32_t rings, int32_t* offsets, int32_t* idx);

/* WCSPH density + Tait pressure, and accelerations, for particles with mask[i] != 0
 * (mask NULL = all) [pinned: rest-lattice density, momentum, hydrostatic column]. */
int orc_wcsph_density(const orc_params* P, int32_t n, const double* x, int32_t nb,
                      const double* xb, const uint8_t* mask, double* rho, double* p,
                      int32_t* nbr);
int orc_wcsph_accel(const orc_params* P, int32_t n, const double* x, const double* v,
                    const double* rho, const double* p, int32_t nb, const double* xb,
                    const uint8_t* mask, double* a_out);
/* The Tait equation of state exactly as the density pass applies it (test entry).
 * [pinned: p(rho0) = 0, dp/drho(rho0) = c_s^2, d2p/drho2(rho0) = (gamma - 1) c_s^2 / rho0,
 * the clamp] */
double orc_tait(const orc_params* P, double rho);

/* Level thresholds of Eq. 1-3 per level [pinned: closed-form table]. */
void orc_level_thresholds(const orc_params* P, double* vthr2, double* athr2, int32_t* eq1);

/* Block levels: Eq. 1-3 per filled block, then the R_min smoothing (Section 4.2).
 * raw may be NULL.  [pinned: hand-built level fields] */
int orc_classify_wcsph(const orc_params* P, int32_t n, const double* x, const double* v,
                       const double* a, int32_t* raw, int32_t* level);

/* Regional time stepping for WCSPH (Algorithm 1 with the Serna predictor-corrector of
 * Section 4.1).  evaluate = priming pass at the current time; substep = one dt_b.
 * [pinned: interpolation identity, forced-finest equals global stepping] */
int orc_wcsph_evaluate(const orc_params* P, orc_wstate* S);
int orc_wcsph_substep(const orc_params* P, orc_wstate* S);
/* Global stepping comparator: one step of mult * dt_b with every particle active.
 * The multiplier is the finest level over all particles (mode 1) or 1 (mode 2),
 * capped at max_mult.  [pinned: hydrostatic column, harmonic convergence] */
int orc_wcsph_global_step(const orc_params* P, orc_wstate* S, int32_t max_mult,
                          int32_t* mult_used);

/* ------------------------------------------------------------------ PCISPH --- */

/* PCISPH state in user order (Sections 5.2-5.6, Algorithms 2 and 3). */
typedef struct orc_pstate {
  int32_t n, nb;
  double *x, *v;           /* 3n */
  double *anp;             /* 3n: non-pressure acceleration (viscosity + gravity), held */
  double *ap;              /* 3n: pressure acceleration of the current minor step */
  double *p, *rho, *err;   /* n: pressure, latest predicted density, latest relative error */
  int32_t *level;          /* n: region index (0 = R_1 ... 3 = R_4) */
  int32_t *validity;       /* n: minor steps until the neighbourhood expires */
  uint8_t *compute;        /* n: neighbourhood / non-pressure forces refreshed this step */
  int32_t *nbr_cnt;        /* n */
  int32_t *nbr_idx;        /* n * cap: fluid j as j, boundary b as n + b */
  int32_t cap;
  const double *xb;        /* 3nb */
  int32_t *pblock;         /* n: block of each particle at the major-step start */
  int32_t *cs, *pm;        /* grid of the major-step start: B + 1, n */
  int32_t *bcs, *bpm;      /* static boundary grid: B + 1, nb */
  int32_t *block_level;    /* B: region of each block (-1 = no fluid) */
  int32_t *block_raw;      /* B: region from Eq. 2-3 before smoothing and expansion */
  uint8_t *block_ob;       /* B: observed blocks (R_ob) of the last iteration */
  double *p_backup;        /* n: pressures before local iterations began */
  uint8_t *in_se;          /* n: particle in S_e */
  int32_t minor;           /* minor step within the major step */
  int32_t n_minor_cur;     /* minor steps of the current major step (N or shortened) */
  int32_t clean;           /* consecutive major steps without > max_global_iters */
  int32_t shorten_now;     /* this major step exceeded max_global_iters */
  int64_t k;               /* minor steps done */
  /* statistics of the last minor step */
  int32_t iters, global_iters, local_iters, reverts, not_converged;
  double err_max, err_avg;
  int64_t total_iters, total_local, total_restarts;
} orc_pstate;

/* Solenthaler-Pajarola pressure scaling: delta = 1 / (beta sum |grad W|^2) on a prototype
 * particle with a full cubic lattice of spacing s, beta = 2 (dt_b m / rho0)^2.
 * [pinned: closed-form lattice sum] */
double orc_pcisph_delta(const orc_params* P);

/* Regions: Eq. 2-3 (alpha = 1, no Eq. 1), R_min smoothing, expansion of R_1 then R_2 by
 * expand_layers blocks (Section 5.5).  [pinned: hand-built fields] */
int orc_classify_pcisph(const orc_params* P, int32_t n, const double* x, const double* v,
                        const double* a, int32_t* raw, int32_t* level);

/* Observed blocks: filled blocks not in R_e bordering R_e or a smaller region
 * (Section 5.4, Figure 4 c-d).  in_re: B flags.  [pinned: hand-built fields] */
void orc_observed_blocks(const orc_params* P, const int32_t* block_level, const uint8_t* in_re,
                         uint8_t* ob);

/* One minor step of Algorithm 2 with Algorithm 3 (major-step start included).
 * Returns ORC_ERR_NOT_CONVERGED (state advanced) when a minor step hits max_iters.
 * [parity unpinned for the correction schedule, which is reconstructed; pinned: rest
 * lattice at rest, forced-R_1 equals plain PCISPH, delta] */
int orc_pcisph_step(const orc_params* P, orc_pstate* S);

/* Plain PCISPH (Solenthaler & Pajarola) for comparison: every particle refreshes its
 * neighbourhood from a fresh grid, >= 3 global iterations until max error <= eta.
 * Shares the state layout; uses dt_b. */
int orc_pcisph_plain_step(const orc_params* P, orc_pstate* S);

/* Global comparators for PCISPH: plain PCISPH with one step of mult * dt_b, mult from the
 * finest region Eq. 2-3 give for the whole fluid (mode 1) or 1 (mode 2), capped at
 * max_mult; delta follows the step.  Mode 1 rejects a step whose correction reaches
 * max_iters and retries it with half the multiplier.  [pinned: mode 2 is plain PCISPH] */
int orc_pcisph_global_step(const orc_params* P, orc_pstate* S, int32_t max_mult,
                           int32_t* mult_used);

/* Test entries: the pressure acceleration (given p and predicted densities rho) and the
 * non-pressure acceleration (viscosity + gravity, given v) exactly as Algorithms 2-3
 * apply them, for every fluid particle, over one-ring neighbourhoods searched at x.
 * [pinned: linear-pressure lattice closed form, half-space closed forms, rigid motion] */
int orc_pcisph_pressure_accel(const orc_params* P, int32_t n, const double* x,
                              const double* p, const double* rho, int32_t nb,
                              const double* xb, double* a_out);
int orc_pcisph_nonpressure_accel(const orc_params* P, int32_t n, const double* x,
                                 const double* v, int32_t nb, const double* xb,
                                 double* a_out);

#ifdef __cplusplus
}
#endif
#endif
