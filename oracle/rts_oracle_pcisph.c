/*
 * rts_oracle_pcisph.c - FP64 CPU oracle, PCISPH part (TEST INFRASTRUCTURE ONLY).
 *
 * Plain restatement of regional time stepping for PCISPH: Algorithm 2 (major and minor
 * steps, region determination with expansion, observed blocks, validity-driven
 * neighbourhood refresh) and Algorithm 3 (DensityCorrectionRTS), with the Sections
 * 5.3-5.6 rules.  The predictive-corrective core follows Solenthaler & Pajarola (cited by
 * the paper): predict v*, x*; predicted density; p += delta (rho* - rho0)+; pressure
 * force with predicted densities.  Readings where the paper is silent or the defining
 * figure (the schedule, Figure 5) is missing:
 *   - schedule: iterations per region and minor step come from params (sched); row r of
 *     minor step j gives a turn to region n iff r <= sched[n][j];
 *   - an iteration is global when every region has a turn;
 *   - the standard 3 iterations come first; after every later non-converged iteration,
 *     average error >= eta_T -> one more global iteration (all regions), otherwise a local
 *     one (S_e only); more than max_local_iters consecutive local iterations -> revert
 *     the pressures to their values before the local run and stay global;
 *   - converged iff the maximum latest relative compression error <= eta; S_e = particles
 *     with error > eta / 2; errors are compression only, max(0, rho* - rho0) / rho0;
 *   - non-pressure forces (artificial viscosity with rho0, gravity) are refreshed only for
 *     particles whose neighbourhood is refreshed (Algorithm 2);
 *   - neighbourhoods are searched around the particle's block of the major-step start
 *     (1 ring, 2 for R_1) with current positions; the grid is kept for the major step;
 *   - pre-emption: after integration, a particle whose own velocity and acceleration need
 *     a smaller region lowers its block and the 26 neighbouring blocks to that region;
 *     their particles refresh at the next minor step;
 *   - boundary particles add mass m to the density sum and have no pressure of their own.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle_internal.h"
#include "rts_oracle.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------ delta (S&P) --- */

double orc_pcisph_delta(const orc_params* P) {
  double h = 0.5 * P->r, s = P->s, m = orci_particle_mass(P);
  double sum_g[3] = {0, 0, 0}, sum_gg = 0.0;
  int R = (int)ceil(P->r / s) + 1;
  for (int i = -R; i <= R; ++i)
    for (int j = -R; j <= R; ++j)
      for (int k = -R; k <= R; ++k) {
        if (!i && !j && !k) continue;
        double xij[3] = {-(double)i * s, -(double)j * s, -(double)k * s};
        double d2 = xij[0] * xij[0] + xij[1] * xij[1] + xij[2] * xij[2];
        if (!(d2 < P->r * P->r)) continue;
        double d = sqrt(d2);
        double f = orc_kernel_dW(d, h) / d;
        double g[3] = {f * xij[0], f * xij[1], f * xij[2]};
        for (int c = 0; c < 3; ++c) sum_g[c] += g[c];
        sum_gg += g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
      }
  double beta = 2.0 * (P->dt_b * m / P->rho0) * (P->dt_b * m / P->rho0);
  double denom = -(sum_g[0] * sum_g[0] + sum_g[1] * sum_g[1] + sum_g[2] * sum_g[2]) - sum_gg;
  return -1.0 / (beta * denom);
}

/* --------------------------------------------------------------- regions --- */

static int region_max_dilate(const orc_params* P, const int32_t* in, int32_t* out, int target,
                             int layers) {
  /* blocks within Chebyshev distance <= layers of a block with region <= target take
   * min(current, target); filled blocks only (in[b] >= 0) */
  int32_t B = orci_n_blocks(P);
  memcpy(out, in, sizeof(int32_t) * (size_t)B);
  for (int bz = 0; bz < P->dim[2]; ++bz)
    for (int by = 0; by < P->dim[1]; ++by)
      for (int bx = 0; bx < P->dim[0]; ++bx) {
        int32_t b = orci_block_lin(P, bx, by, bz);
        if (in[b] < 0 || in[b] <= target) continue;
        int hit = 0;
        for (int dz = -layers; dz <= layers && !hit; ++dz)
          for (int dy = -layers; dy <= layers && !hit; ++dy)
            for (int dx = -layers; dx <= layers && !hit; ++dx) {
              int cx = bx + dx, cy = by + dy, cz = bz + dz;
              if (cx < 0 || cy < 0 || cz < 0 || cx >= P->dim[0] || cy >= P->dim[1] ||
                  cz >= P->dim[2])
                continue;
              int32_t L = in[orci_block_lin(P, cx, cy, cz)];
              if (L >= 0 && L <= target) hit = 1;
            }
        if (hit) out[b] = target;
      }
  return 0;
}

/* Section 3.1 with alpha = 1 and no Eq. 1, R_min (Section 4.2), then Section 5.5: expand
 * R_1 and R_2 by expand_layers blocks. */
int orc_classify_pcisph(const orc_params* P, int32_t n, const double* x, const double* v,
                        const double* a, int32_t* raw, int32_t* level) {
  int32_t B = orci_n_blocks(P);
  int st = orci_raw_levels(P, n, x, v, a, raw);
  if (st) return st;
  if (P->force_level >= 0) {
    for (int32_t b = 0; b < B; ++b) level[b] = raw[b] < 0 ? -1 : P->force_level;
    return ORC_OK;
  }
  int32_t* t1 = (int32_t*)malloc(sizeof(int32_t) * (size_t)B);
  int32_t* t2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)B);
  orci_rmin_smooth(P, raw, t1);
  region_max_dilate(P, t1, t2, 0, P->expand_layers);
  region_max_dilate(P, t2, level, 1, P->expand_layers);
  free(t1);
  free(t2);
  return ORC_OK;
}

/* R_ob: filled blocks outside R_e with a 26-neighbour in R_e or of a smaller region. */
void orc_observed_blocks(const orc_params* P, const int32_t* lev, const uint8_t* in_re,
                         uint8_t* ob) {
  for (int bz = 0; bz < P->dim[2]; ++bz)
    for (int by = 0; by < P->dim[1]; ++by)
      for (int bx = 0; bx < P->dim[0]; ++bx) {
        int32_t b = orci_block_lin(P, bx, by, bz);
        uint8_t o = 0;
        if (lev[b] >= 0 && !(in_re && in_re[b])) {
          for (int dz = -1; dz <= 1 && !o; ++dz)
            for (int dy = -1; dy <= 1 && !o; ++dy)
              for (int dx = -1; dx <= 1 && !o; ++dx) {
                if (!dx && !dy && !dz) continue;
                int cx = bx + dx, cy = by + dy, cz = bz + dz;
                if (cx < 0 || cy < 0 || cz < 0 || cx >= P->dim[0] || cy >= P->dim[1] ||
                    cz >= P->dim[2])
                  continue;
                int32_t c = orci_block_lin(P, cx, cy, cz);
                if (lev[c] < 0) continue;
                if ((in_re && in_re[c]) || lev[c] < lev[b]) o = 1;
              }
        }
        ob[b] = o;
      }
}

/* ------------------------------------------------------------ PCISPH core --- */

typedef struct {
  ogrid G;  /* views of the state's grid arrays */
} pgrid;

static void view_grid(const orc_params* P, orc_pstate* S, ogrid* G) {
  G->B = orci_n_blocks(P);
  G->key = S->pblock;
  G->cs = S->cs;
  G->pm = S->pm;
  G->bcs = S->bcs;
  G->bpm = S->bpm;
  G->bkey = NULL;
}

static const double* pos_of(const orc_pstate* S, const double* xs, int32_t j) {
  return j < S->n ? xs + 3 * (int64_t)j : S->xb + 3 * (int64_t)(j - S->n);
}

/* Neighbourhood N_i around the particle's major-start block (rings 1, or 2 for R_1; the
 * r2_rings ablation searches R_2 with more rings as well). */
static int refresh_list(const orc_params* P, orc_pstate* S, const ogrid* G, int32_t i,
                        int32_t* buf) {
  int32_t b = S->pblock[i];
  int c[3] = {b % P->dim[0], (b / P->dim[0]) % P->dim[1], b / (P->dim[0] * P->dim[1])};
  int rings = S->level[i] == 0 ? P->r1_rings : (S->level[i] == 1 && P->r2_rings > 1 ? P->r2_rings : 1);
  int cnt = orci_nbr_list(P, G, S->n, S->x, S->xb, i, c, rings, P->r * P->r, buf, NBR_CAP);
  if (cnt < 0 || cnt > S->cap) return ORC_ERR_CAPACITY;
  memcpy(S->nbr_idx + (int64_t)i * S->cap, buf, sizeof(int32_t) * (size_t)cnt);
  S->nbr_cnt[i] = cnt;
  return ORC_OK;
}

/* Non-pressure acceleration: gravity + artificial viscosity (nu = 2 alpha h c / (2 rho0))
 * over the neighbourhood; boundary neighbours have zero velocity. */
static void nonpressure(const orc_params* P, orc_pstate* S, int32_t i) {
  double h = 0.5 * P->r, m = orci_particle_mass(P);
  double nu = 2.0 * P->visc_alpha * h * P->c_s / (2.0 * P->rho0);
  const double* xi = S->x + 3 * (int64_t)i;
  const double* vi = S->v + 3 * (int64_t)i;
  double a[3] = {P->g[0], P->g[1], P->g[2]};
  for (int q = 0; q < S->nbr_cnt[i]; ++q) {
    int32_t j = S->nbr_idx[(int64_t)i * S->cap + q];
    const double* xj = pos_of(S, S->x, j);
    double vj[3] = {0, 0, 0};
    if (j < S->n) memcpy(vj, S->v + 3 * (int64_t)j, sizeof vj);
    double xij[3] = {xi[0] - xj[0], xi[1] - xj[1], xi[2] - xj[2]};
    double d2 = xij[0] * xij[0] + xij[1] * xij[1] + xij[2] * xij[2];
    if (!(d2 > 0.0)) continue;
    double d = sqrt(d2);
    double vx = (vi[0] - vj[0]) * xij[0] + (vi[1] - vj[1]) * xij[1] + (vi[2] - vj[2]) * xij[2];
    if (vx >= 0.0) continue;
    double Pi = -nu * vx / (d2 + 0.01 * h * h);
    double f = orc_kernel_dW(d, h) / d;
    for (int k = 0; k < 3; ++k) a[k] -= m * Pi * f * xij[k];
  }
  memcpy(S->anp + 3 * (int64_t)i, a, sizeof a);
}

/* Predicted density over the neighbourhood at the predicted positions xs (boundary
 * particles at rest). */
static double predicted_density(const orc_params* P, const orc_pstate* S, const double* xs,
                                int32_t i) {
  double h = 0.5 * P->r, m = orci_particle_mass(P);
  const double* xi = xs + 3 * (int64_t)i;
  double rho = m * orc_kernel_W(0.0, h);
  for (int q = 0; q < S->nbr_cnt[i]; ++q) {
    const double* xj = pos_of(S, xs, S->nbr_idx[(int64_t)i * S->cap + q]);
    double dx = xi[0] - xj[0], dy = xi[1] - xj[1], dz = xi[2] - xj[2];
    rho += m * orc_kernel_W(sqrt(dx * dx + dy * dy + dz * dz), h);
  }
  return rho;
}

/* Pressure acceleration -m sum (p_i / rho_i*^2 + p_j / rho_j*^2) grad W(x*_ij). */
static void pressure_accel(const orc_params* P, orc_pstate* S, const double* xs, int32_t i) {
  double h = 0.5 * P->r, m = orci_particle_mass(P);
  const double* xi = xs + 3 * (int64_t)i;
  double ci = S->p[i] / (S->rho[i] * S->rho[i]);
  double a[3] = {0, 0, 0};
  for (int q = 0; q < S->nbr_cnt[i]; ++q) {
    int32_t j = S->nbr_idx[(int64_t)i * S->cap + q];
    const double* xj = pos_of(S, xs, j);
    double cj = j < S->n ? S->p[j] / (S->rho[j] * S->rho[j]) : 0.0;
    double xij[3] = {xi[0] - xj[0], xi[1] - xj[1], xi[2] - xj[2]};
    double d2 = xij[0] * xij[0] + xij[1] * xij[1] + xij[2] * xij[2];
    if (!(d2 > 0.0)) continue;
    double d = sqrt(d2);
    double f = orc_kernel_dW(d, h) / d;
    for (int k = 0; k < 3; ++k) a[k] -= m * (ci + cj) * f * xij[k];
  }
  memcpy(S->ap + 3 * (int64_t)i, a, sizeof a);
}

/* Test entries: a state holding only what pressure_accel / nonpressure read, with the
 * one-ring neighbourhoods of every particle searched at x. */
static int accel_state(const orc_params* P, int32_t n, const double* x, const double* v,
                       const double* p, const double* rho, int32_t nb, const double* xb,
                       orc_pstate* S, ogrid* G) {
  memset(S, 0, sizeof(*S));
  S->n = n;
  S->nb = nb;
  S->x = (double*)x;
  S->v = (double*)v;
  S->p = (double*)p;
  S->rho = (double*)rho;
  S->xb = xb;
  S->cap = NBR_CAP;
  S->nbr_cnt = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
  S->nbr_idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1) * NBR_CAP);
  S->ap = (double*)calloc(3 * (size_t)(n > 0 ? n : 1), sizeof(double));
  S->anp = (double*)calloc(3 * (size_t)(n > 0 ? n : 1), sizeof(double));
  int st = orci_grid_build(P, n, x, nb, xb, G);
  for (int32_t i = 0; i < n && !st; ++i) {
    int c[3];
    st = orci_block_coords(P, x + 3 * (int64_t)i, c);
    if (st) break;
    int cnt = orci_nbr_list(P, G, n, x, xb, i, c, 1, P->r * P->r,
                            S->nbr_idx + (int64_t)i * NBR_CAP, NBR_CAP);
    if (cnt < 0) st = ORC_ERR_CAPACITY;
    else S->nbr_cnt[i] = cnt;
  }
  return st;
}

static void accel_state_free(orc_pstate* S, ogrid* G) {
  free(S->nbr_cnt);
  free(S->nbr_idx);
  free(S->ap);
  free(S->anp);
  orci_grid_free(G);
}

int orc_pcisph_pressure_accel(const orc_params* P, int32_t n, const double* x,
                              const double* p, const double* rho, int32_t nb,
                              const double* xb, double* a_out) {
  orc_pstate S;
  ogrid G;
  int st = accel_state(P, n, x, NULL, p, rho, nb, xb, &S, &G);
  if (!st) {
    for (int32_t i = 0; i < n; ++i) pressure_accel(P, &S, x, i);
    memcpy(a_out, S.ap, sizeof(double) * 3 * (size_t)n);
  }
  accel_state_free(&S, &G);
  return st;
}

int orc_pcisph_nonpressure_accel(const orc_params* P, int32_t n, const double* x,
                                 const double* v, int32_t nb, const double* xb,
                                 double* a_out) {
  orc_pstate S;
  ogrid G;
  int st = accel_state(P, n, x, v, NULL, NULL, nb, xb, &S, &G);
  if (!st) {
    for (int32_t i = 0; i < n; ++i) nonpressure(P, &S, i);
    memcpy(a_out, S.anp, sizeof(double) * 3 * (size_t)n);
  }
  accel_state_free(&S, &G);
  return st;
}

/* ------------------------------------------------------ major-step start --- */

static int major_start(const orc_params* P, orc_pstate* S) {
  int32_t n = S->n, B = orci_n_blocks(P);
  /* grid of the major step (Section 5.6: built once per major step) */
  int st = orc_bin(P, n, S->x, S->pblock, S->pm, S->cs);
  if (st) return st;
  /* regions from the held total acceleration */
  double* a = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  for (int64_t q = 0; q < 3 * (int64_t)n; ++q) a[q] = S->anp[q] + S->ap[q];
  st = orc_classify_pcisph(P, n, S->x, S->v, a, S->block_raw, S->block_level);
  free(a);
  if (st) return st;
  (void)B;
  for (int32_t i = 0; i < n; ++i) {
    int32_t L = S->block_level[S->pblock[i]];
    S->level[i] = L;
    S->validity[i] = P->refresh[L];
    S->compute[i] = 1;
  }
  S->shorten_now = 0;
  return ORC_OK;
}

/* Section 5.6: a particle needing a smaller region lowers its block and its 26 neighbours. */
static void preempt(const orc_params* P, orc_pstate* S) {
  int32_t n = S->n, B = orci_n_blocks(P);
  double vthr2[8], athr2[8];
  int32_t eq1[8];
  orc_level_thresholds(P, vthr2, athr2, eq1);
  int32_t* newlev = (int32_t*)malloc(sizeof(int32_t) * (size_t)B);
  memcpy(newlev, S->block_level, sizeof(int32_t) * (size_t)B);
  for (int32_t i = 0; i < n; ++i) {
    double a[3] = {S->anp[3 * i] + S->ap[3 * i], S->anp[3 * i + 1] + S->ap[3 * i + 1],
                   S->anp[3 * i + 2] + S->ap[3 * i + 2]};
    int32_t L = orci_pick_level(P, vthr2, athr2, eq1, orci_norm2(S->v + 3 * (int64_t)i),
                                orci_norm2(a));
    if (P->force_level >= 0) L = P->force_level;
    if (L >= S->level[i]) continue;
    int32_t b = S->pblock[i];
    int bx = b % P->dim[0], by = (b / P->dim[0]) % P->dim[1], bz = b / (P->dim[0] * P->dim[1]);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int cx = bx + dx, cy = by + dy, cz = bz + dz;
          if (cx < 0 || cy < 0 || cz < 0 || cx >= P->dim[0] || cy >= P->dim[1] || cz >= P->dim[2])
            continue;
          int32_t c = orci_block_lin(P, cx, cy, cz);
          if (newlev[c] >= 0 && L < newlev[c]) newlev[c] = L;
        }
  }
  for (int32_t i = 0; i < n; ++i) {
    int32_t L = newlev[S->pblock[i]];
    if (L < S->level[i]) {
      S->level[i] = L;
      S->validity[i] = P->refresh[L];
      S->compute[i] = 1;
    }
  }
  memcpy(S->block_level, newlev, sizeof(int32_t) * (size_t)B);
  free(newlev);
}

/* ---------------------------------------------------------- Algorithm 3 --- */

enum { MODE_SCHED = 0, MODE_GLOBAL = 1, MODE_LOCAL = 2 };

static int density_correction(const orc_params* P, orc_pstate* S, int j) {
  int32_t n = S->n, B = orci_n_blocks(P);
  double dt = P->dt_b, delta = orc_pcisph_delta(P);
  double* xs = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  uint8_t* in_re = (uint8_t*)calloc((size_t)B, 1);
  uint8_t* part = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
  uint8_t* turn = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
  int min_sched = 1 << 30;
  for (int r = 0; r < P->n_levels && r < 4; ++r)
    if (P->sched[r][j] < min_sched) min_sched = P->sched[r][j];
  memset(S->in_se, 0, (size_t)n);
  orc_observed_blocks(P, S->block_level, NULL, S->block_ob);
  int min_iter = 3, done = 0, row = 1, mode = MODE_SCHED, local_run = 0, stay_global = 0;
  int status = ORC_OK;
  S->iters = S->global_iters = S->local_iters = S->reverts = S->not_converged = 0;
  for (;;) {
    int all_turn = mode == MODE_GLOBAL || (mode == MODE_SCHED && row <= min_sched);
    for (int32_t i = 0; i < n; ++i)
      turn[i] = mode == MODE_GLOBAL || (mode == MODE_SCHED && row <= P->sched[S->level[i]][j]);
    /* predict v*, x* (all) */
    for (int32_t i = 0; i < n; ++i)
      for (int k = 0; k < 3; ++k) {
        double vs = S->v[3 * i + k] + dt * (S->anp[3 * i + k] + S->ap[3 * i + k]);
        xs[3 * i + k] = S->x[3 * i + k] + dt * vs;
      }
    /* predicted density, error, pressure for turn, S_e, S_ob */
    for (int32_t i = 0; i < n; ++i) {
      part[i] = turn[i] || S->in_se[i] || S->block_ob[S->pblock[i]];
      if (!part[i]) continue;
      double rho = predicted_density(P, S, xs, i);
      double comp = rho - P->rho0 > 0.0 ? rho - P->rho0 : 0.0;
      S->rho[i] = rho;
      S->err[i] = comp / P->rho0;
      S->p[i] += delta * comp;
    }
    /* update S_e (error above eta / 2), R_e, R_ob */
    memset(in_re, 0, (size_t)B);
    for (int32_t i = 0; i < n; ++i) {
      S->in_se[i] = S->err[i] > 0.5 * P->eta;
      if (S->in_se[i]) in_re[S->pblock[i]] = 1;
    }
    orc_observed_blocks(P, S->block_level, in_re, S->block_ob);
    /* pressure force for turn and S_e */
    for (int32_t i = 0; i < n; ++i)
      if (turn[i] || S->in_se[i]) pressure_accel(P, S, xs, i);
    ++done;
    if (all_turn) ++S->global_iters;
    if (mode == MODE_LOCAL) ++S->local_iters;
    double emax = 0.0, esum = 0.0;
    for (int32_t i = 0; i < n; ++i) {
      if (S->err[i] > emax) emax = S->err[i];
      esum += S->err[i];
    }
    S->err_max = emax;
    S->err_avg = n > 0 ? esum / n : 0.0;
    int converged = emax <= P->eta;
    if (done >= min_iter && converged) break;
    if (done >= P->max_iters) {
      status = ORC_ERR_NOT_CONVERGED;
      S->not_converged = 1;
      break;
    }
    if (done < 3) {
      ++row;  /* the standard schedule rows */
      continue;
    }
    /* extra iterations (Section 5.5) */
    min_iter = done + 1;
    if (stay_global || S->err_avg >= P->eta_T) {
      mode = MODE_GLOBAL;
      local_run = 0;
    } else {
      if (mode != MODE_LOCAL) {
        memcpy(S->p_backup, S->p, sizeof(double) * (size_t)n);
        local_run = 0;
      }
      mode = MODE_LOCAL;
      if (++local_run > P->max_local_iters) {
        memcpy(S->p, S->p_backup, sizeof(double) * (size_t)n);
        ++S->reverts;
        mode = MODE_GLOBAL;
        stay_global = 1;
        local_run = 0;
      }
    }
  }
  S->iters = done;
  S->total_iters += done;
  S->total_local += S->local_iters;
  S->total_restarts += S->reverts;
  free(xs);
  free(in_re);
  free(part);
  free(turn);
  return status;
}

/* ---------------------------------------------------------- Algorithm 2 --- */

int orc_pcisph_step(const orc_params* P, orc_pstate* S) {
  int32_t n = S->n;
  int st;
  if (S->n_minor_cur <= 0) S->n_minor_cur = P->n_minor;
  if (S->minor == 0 && (st = major_start(P, S))) return st;
  int j = S->minor;
  ogrid G;
  view_grid(P, S, &G);
  int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * NBR_CAP);
  st = ORC_OK;
  for (int32_t i = 0; i < n && !st; ++i)
    if (S->compute[i]) st = refresh_list(P, S, &G, i, buf);
  free(buf);
  if (st) return st;
  for (int32_t i = 0; i < n; ++i)
    if (S->compute[i]) nonpressure(P, S, i);
  for (int32_t i = 0; i < n; ++i) {
    S->p[i] = 0.0;
    S->ap[3 * i] = S->ap[3 * i + 1] = S->ap[3 * i + 2] = 0.0;
  }
  int cst = density_correction(P, S, j);
  /* integrate: v += dt (a_np + a_p), x += dt v */
  for (int32_t i = 0; i < n; ++i) {
    for (int k = 0; k < 3; ++k) {
      S->v[3 * i + k] += P->dt_b * (S->anp[3 * i + k] + S->ap[3 * i + k]);
      S->x[3 * i + k] += P->dt_b * S->v[3 * i + k];
    }
    orci_wall_project(P, S->x + 3 * i, S->v + 3 * i);
  }
  if (S->global_iters > P->max_global_iters) S->shorten_now = 1;
  int last = (j + 1 >= S->n_minor_cur) || S->shorten_now;
  for (int32_t i = 0; i < n; ++i) {
    S->validity[i] -= 1;
    if (S->validity[i] <= 0) {
      S->compute[i] = 1;
      S->validity[i] = P->refresh[S->level[i]];
    } else {
      S->compute[i] = 0;
    }
  }
  if (!last) preempt(P, S);
  S->k += 1;
  if (last) {
    /* major step ends: shortened major steps after an overrun, restored after
     * clean_majors clean ones (Section 5.5) */
    if (S->shorten_now) {
      S->n_minor_cur = P->short_minor;
      S->clean = 0;
    } else if (S->n_minor_cur != P->n_minor) {
      if (++S->clean >= P->clean_majors) {
        S->n_minor_cur = P->n_minor;
        S->clean = 0;
      }
    }
    S->minor = 0;
  } else {
    S->minor = j + 1;
  }
  return cst;
}

/* Plain PCISPH: fresh grid and neighbourhoods every step, non-pressure forces for all,
 * >= 3 global iterations until the maximum error is <= eta (or max_iters). */
int orc_pcisph_plain_step(const orc_params* P, orc_pstate* S) {
  int32_t n = S->n;
  double dt = P->dt_b, delta = orc_pcisph_delta(P);
  int st = orc_bin(P, n, S->x, S->pblock, S->pm, S->cs);
  if (st) return st;
  ogrid G;
  view_grid(P, S, &G);
  int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * NBR_CAP);
  for (int32_t i = 0; i < n; ++i) {
    int32_t b = S->pblock[i];
    int c[3] = {b % P->dim[0], (b / P->dim[0]) % P->dim[1], b / (P->dim[0] * P->dim[1])};
    int cnt = orci_nbr_list(P, &G, n, S->x, S->xb, i, c, 1, P->r * P->r, buf, NBR_CAP);
    if (cnt < 0 || cnt > S->cap) {
      free(buf);
      return ORC_ERR_CAPACITY;
    }
    memcpy(S->nbr_idx + (int64_t)i * S->cap, buf, sizeof(int32_t) * (size_t)cnt);
    S->nbr_cnt[i] = cnt;
  }
  free(buf);
  for (int32_t i = 0; i < n; ++i) {
    nonpressure(P, S, i);
    S->p[i] = 0.0;
    S->ap[3 * i] = S->ap[3 * i + 1] = S->ap[3 * i + 2] = 0.0;
  }
  double* xs = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  int it = 0, status = ORC_OK;
  for (;;) {
    for (int32_t i = 0; i < n; ++i)
      for (int k = 0; k < 3; ++k) {
        double vs = S->v[3 * i + k] + dt * (S->anp[3 * i + k] + S->ap[3 * i + k]);
        xs[3 * i + k] = S->x[3 * i + k] + dt * vs;
      }
    for (int32_t i = 0; i < n; ++i) {
      double rho = predicted_density(P, S, xs, i);
      double comp = rho - P->rho0 > 0.0 ? rho - P->rho0 : 0.0;
      S->rho[i] = rho;
      S->err[i] = comp / P->rho0;
      S->p[i] += delta * comp;
    }
    for (int32_t i = 0; i < n; ++i) pressure_accel(P, S, xs, i);
    ++it;
    double emax = 0.0;
    for (int32_t i = 0; i < n; ++i)
      if (S->err[i] > emax) emax = S->err[i];
    S->err_max = emax;
    if (it >= 3 && emax <= P->eta) break;
    if (it >= P->max_iters) {
      status = ORC_ERR_NOT_CONVERGED;
      break;
    }
  }
  free(xs);
  for (int32_t i = 0; i < n; ++i) {
    for (int k = 0; k < 3; ++k) {
      S->v[3 * i + k] += dt * (S->anp[3 * i + k] + S->ap[3 * i + k]);
      S->x[3 * i + k] += dt * S->v[3 * i + k];
    }
    orci_wall_project(P, S->x + 3 * i, S->v + 3 * i);
  }
  S->iters = it;
  S->k += 1;
  return status;
}

int orc_pcisph_global_step(const orc_params* P, orc_pstate* S, int32_t max_mult,
                           int32_t* mult_used) {
  int32_t L = 0;
  if (P->mode != 2) {
    double vthr2[8], athr2[8];
    int32_t eq1[8];
    orc_level_thresholds(P, vthr2, athr2, eq1);
    double vmax2 = 0.0, amax2 = 0.0;
    for (int32_t i = 0; i < S->n; ++i) {
      double a[3] = {S->anp[3 * i] + S->ap[3 * i], S->anp[3 * i + 1] + S->ap[3 * i + 1],
                     S->anp[3 * i + 2] + S->ap[3 * i + 2]};
      double v2 = orci_norm2(S->v + 3 * (int64_t)i), a2 = orci_norm2(a);
      if (v2 > vmax2) vmax2 = v2;
      if (a2 > amax2) amax2 = a2;
    }
    L = orci_pick_level(P, vthr2, athr2, eq1, vmax2, amax2);
  }
  int32_t m = P->mult[L];
  if (m > max_mult) m = max_mult;
  if (m < 1) m = 1;
  /* a step whose correction does not converge is rejected and retried with half the
   * multiplier (density-error feedback of an adaptive global step) */
  int32_t n = S->n;
  size_t v3 = sizeof(double) * 3 * (size_t)(n > 0 ? n : 1);
  double* x0 = (double*)malloc(v3);
  double* v0 = (double*)malloc(v3);
  memcpy(x0, S->x, v3);
  memcpy(v0, S->v, v3);
  int64_t k0 = S->k;
  int st;
  for (;;) {
    orc_params Q = *P;
    Q.dt_b = (double)m * P->dt_b;
    st = orc_pcisph_plain_step(&Q, S);
    if (st != ORC_ERR_NOT_CONVERGED || m == 1 || P->mode == 2) break;
    memcpy(S->x, x0, v3);
    memcpy(S->v, v0, v3);
    m = m / 2 > 1 ? m / 2 : 1;
  }
  free(x0);
  free(v0);
  S->k = k0 + m;
  for (int32_t i = 0; i < S->n; ++i) S->level[i] = L;
  if (mult_used) *mult_used = m;
  return st;
}
