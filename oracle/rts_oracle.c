/*
 * rts_oracle.c - FP64 CPU oracle, WCSPH part (TEST INFRASTRUCTURE ONLY).
 *
 * Plain restatement of the paper's WCSPH regional time stepping: the block grid
 * (Section 3), the time-step criteria Eq. 1-3 and the R_min smoothing (Sections 3.1,
 * 4.2), the Serna predictor-corrector (Section 4.1) and Algorithm 1.  The SPH physics
 * the paper cites without restating (Becker & Teschner WCSPH: cubic spline,
 * summation density, Tait equation of state, artificial viscosity) follows the
 * textbook definitions.  Readings of points where the paper is silent:
 *   - kernel support r = 2h with h = s, block edge = r (Section 3: r ~ 2s);
 *   - negative pressure clamped to 0; static boundary particles carry mass m in the
 *     density sum, zero velocity and no pressure of their own, so the pressure force
 *     they exert is the exact gradient of the fluid's internal energy
 *     (-m p_i / rho_i^2 grad W); the artificial viscosity uses rho_b = rho_i.
 *     (Mirroring p_b = p_i doubles that force, is not energy consistent and was
 *     seen to drive an instability at the tank's edges and corners.)
 *   - substep loop rotated so the correction uses the acceleration evaluated at
 *     the corrected time level (the equations of Section 4.1);
 *   - pre-emption on any change of the block's level (Algorithm 1);
 *   - R_min: one Jacobi pass of the minimum over the 26 neighbouring filled blocks.
 * No blocking, fusion or reordering beyond the paper's own block grid.
 */
#include "rts_oracle.h"
#include "oracle_internal.h"

#include <math.h>
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads the oracle's OpenMP loops use (1 without OpenMP). */
int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}



/* ---------------------------------------------------------------- kernel --- */

/* Cubic spline W(q) = sigma (1 - 1.5 q^2 + 0.75 q^3), q < 1; sigma/4 (2 - q)^3,
 * 1 <= q < 2; sigma = 1 / (pi h^3), q = d / h. */
double orc_kernel_W(double d, double h) {
  double q = d / h;
  double sigma = 1.0 / (M_PI * h * h * h);
  if (q < 1.0) return sigma * (1.0 - 1.5 * q * q + 0.75 * q * q * q);
  if (q < 2.0) {
    double t = 2.0 - q;
    return sigma * 0.25 * t * t * t;
  }
  return 0.0;
}

/* dW/dd of the cubic spline. */
double orc_kernel_dW(double d, double h) {
  double q = d / h;
  double sigma = 1.0 / (M_PI * h * h * h);
  if (q < 1.0) return sigma * (-3.0 * q + 2.25 * q * q) / h;
  if (q < 2.0) {
    double t = 2.0 - q;
    return -0.75 * sigma * t * t / h;
  }
  return 0.0;
}

/* ------------------------------------------------------------ block grid --- */

int orci_block_coords(const orc_params* P, const double* x, int c[3]) {
  for (int d = 0; d < 3; ++d) {
    double t = (x[d] - P->origin[d]) / P->edge;
    double f = floor(t);
    if (!(f >= 0.0 && f < (double)P->dim[d])) return ORC_ERR_DOMAIN;
    c[d] = (int)f;
  }
  return ORC_OK;
}

int32_t orci_block_lin(const orc_params* P, int bx, int by, int bz) {
  return ((int32_t)bz * P->dim[1] + by) * P->dim[0] + bx;
}

int32_t orci_n_blocks(const orc_params* P) {
  return P->dim[0] * P->dim[1] * P->dim[2];
}

/* Section 3: each particle lies in exactly one block of a uniform virtual grid. */
int orc_block_key(const orc_params* P, const double* x3, int32_t* key) {
  int c[3];
  int st = orci_block_coords(P, x3, c);
  if (st) return st;
  *key = orci_block_lin(P, c[0], c[1], c[2]);
  return ORC_OK;
}

/* Particles ordered by block, ties by index; cstart[b]..cstart[b+1] lists block b. */
int orc_bin(const orc_params* P, int32_t n, const double* x, int32_t* key, int32_t* perm,
            int32_t* cstart) {
  int32_t B = orci_n_blocks(P);
  for (int32_t i = 0; i < n; ++i) {
    int st = orc_block_key(P, x + 3 * (int64_t)i, &key[i]);
    if (st) return st;
  }
  memset(cstart, 0, sizeof(int32_t) * ((size_t)B + 1));
  for (int32_t i = 0; i < n; ++i) cstart[key[i] + 1]++;
  for (int32_t b = 0; b < B; ++b) cstart[b + 1] += cstart[b];
  int32_t* fill = (int32_t*)malloc(sizeof(int32_t) * (size_t)B);
  memcpy(fill, cstart, sizeof(int32_t) * (size_t)B);
  for (int32_t i = 0; i < n; ++i) perm[fill[key[i]]++] = i;
  free(fill);
  return ORC_OK;
}

void orci_grid_free(ogrid* G) {
  free(G->key); free(G->cs); free(G->pm);
  free(G->bkey); free(G->bcs); free(G->bpm);
  memset(G, 0, sizeof(*G));
}

int orci_grid_build(const orc_params* P, int32_t n, const double* x, int32_t nb,
                      const double* xb, ogrid* G) {
  memset(G, 0, sizeof(*G));
  G->B = orci_n_blocks(P);
  G->key = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  G->pm = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  G->cs = (int32_t*)malloc(sizeof(int32_t) * ((size_t)G->B + 1));
  G->bkey = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nb > 0 ? nb : 1));
  G->bpm = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nb > 0 ? nb : 1));
  G->bcs = (int32_t*)malloc(sizeof(int32_t) * ((size_t)G->B + 1));
  int st = orc_bin(P, n, x, G->key, G->pm, G->cs);
  if (!st) st = orc_bin(P, nb, xb, G->bkey, G->bpm, G->bcs);
  if (st) orci_grid_free(G);
  return st;
}

/* ------------------------------------------------------------ neighbours --- */

/* Neighbour predicate: d^2 = ((dx dx + dy dy) + dz dz) < r^2, evaluated in double. */
int orci_is_nbr(const double* a, const double* b, double r2) {
  double dx = a[0] - b[0];
  double dy = a[1] - b[1];
  double dz = a[2] - b[2];
  double d2 = dx * dx;
  d2 = d2 + dy * dy;
  d2 = d2 + dz * dz;
  return d2 < r2;
}

/* N(i) searched over the (2 rings + 1)^3 blocks around block c (Section 3: neighbours
 * of particles in a block are found in the neighbouring blocks). */
int orci_nbr_list(const orc_params* P, const ogrid* G, int32_t n, const double* x,
                    const double* xb, int32_t i, const int c[3], int rings, double r2,
                    int32_t* out, int cap) {
  const double* xi = x + 3 * (int64_t)i;
  int cnt = 0;
  for (int dz = -rings; dz <= rings; ++dz) {
    int bz = c[2] + dz;
    if (bz < 0 || bz >= P->dim[2]) continue;
    for (int dy = -rings; dy <= rings; ++dy) {
      int by = c[1] + dy;
      if (by < 0 || by >= P->dim[1]) continue;
      for (int dx = -rings; dx <= rings; ++dx) {
        int bx = c[0] + dx;
        if (bx < 0 || bx >= P->dim[0]) continue;
        int32_t b = orci_block_lin(P, bx, by, bz);
        for (int32_t q = G->cs[b]; q < G->cs[b + 1]; ++q) {
          int32_t j = G->pm[q];
          if (j == i) continue;
          if (orci_is_nbr(xi, x + 3 * (int64_t)j, r2)) {
            if (cnt >= cap) return -1;
            out[cnt++] = j;
          }
        }
        for (int32_t q = G->bcs[b]; q < G->bcs[b + 1]; ++q) {
          int32_t j = G->bpm[q];
          if (orci_is_nbr(xi, xb + 3 * (int64_t)j, r2)) {
            if (cnt >= cap) return -1;
            out[cnt++] = n + j;
          }
        }
      }
    }
  }
  return cnt;
}

int64_t orc_neighbors_brute(int32_t n, const double* x, int32_t nb, const double* xb, double r,
                            int32_t* offsets, int32_t* idx) {
  double r2 = r * r;
  int64_t total = 0;
  for (int32_t i = 0; i < n; ++i) {
    offsets[i] = (int32_t)total;
    for (int32_t j = 0; j < n; ++j) {
      if (j == i || !orci_is_nbr(x + 3 * (int64_t)i, x + 3 * (int64_t)j, r2)) continue;
      if (idx) idx[total] = j;
      ++total;
    }
    for (int32_t j = 0; j < nb; ++j) {
      if (!orci_is_nbr(x + 3 * (int64_t)i, xb + 3 * (int64_t)j, r2)) continue;
      if (idx) idx[total] = n + j;
      ++total;
    }
  }
  offsets[n] = (int32_t)total;
  return total;
}

int64_t orc_neighbors_grid(const orc_params* P, int32_t n, const double* x, int32_t nb,
                           const double* xb, int32_t rings, int32_t* offsets, int32_t* idx) {
  ogrid G;
  if (orci_grid_build(P, n, x, nb, xb, &G)) return -ORC_ERR_DOMAIN;
  double r2 = P->r * P->r;
  int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * NBR_CAP);
  int64_t total = 0;
  for (int32_t i = 0; i < n; ++i) {
    int c[3];
    orci_block_coords(P, x + 3 * (int64_t)i, c);
    int cnt = orci_nbr_list(P, &G, n, x, xb, i, c, rings, r2, buf, NBR_CAP);
    if (cnt < 0) { total = -ORC_ERR_CAPACITY; break; }
    offsets[i] = (int32_t)total;
    if (idx) memcpy(idx + total, buf, sizeof(int32_t) * (size_t)cnt);
    total += cnt;
  }
  if (total >= 0) offsets[n] = (int32_t)total;
  free(buf);
  orci_grid_free(&G);
  return total;
}

/* ------------------------------------------------------------ WCSPH physics --- */

double orci_particle_mass(const orc_params* P) { return P->rho0 * P->s * P->s * P->s; }

/* Tait equation of state, p = B ((rho / rho0)^gamma - 1), B = c^2 rho0 / gamma,
 * clamped at zero. */
static double tait(const orc_params* P, double rho) {
  double B = P->tait_B > 0.0 ? P->tait_B : P->c_s * P->c_s * P->rho0 / P->gamma;
  double p = B * (pow(rho / P->rho0, P->gamma) - 1.0);
  return (p > 0.0 || P->tait_no_clamp) ? p : 0.0;
}

double orc_tait(const orc_params* P, double rho) { return tait(P, rho); }

/* rho_i = m W(0) + sum_{j in N(i)} m W(|x_i - x_j|), fluid and boundary j. */
static int density_one(const orc_params* P, const ogrid* G, int32_t n, const double* x,
                       const double* xb, int32_t i, int32_t* buf, double* rho, int32_t* nbr) {
  int c[3];
  if (orci_block_coords(P, x + 3 * (int64_t)i, c)) return ORC_ERR_DOMAIN;
  int cnt = orci_nbr_list(P, G, n, x, xb, i, c, 1, P->r * P->r, buf, NBR_CAP);
  if (cnt < 0) return ORC_ERR_CAPACITY;
  double h = 0.5 * P->r, m = orci_particle_mass(P);
  const double* xi = x + 3 * (int64_t)i;
  double sum = m * orc_kernel_W(0.0, h);
  for (int q = 0; q < cnt; ++q) {
    const double* xj = buf[q] < n ? x + 3 * (int64_t)buf[q] : xb + 3 * (int64_t)(buf[q] - n);
    double dx = xi[0] - xj[0], dy = xi[1] - xj[1], dz = xi[2] - xj[2];
    sum += m * orc_kernel_W(sqrt(dx * dx + dy * dy + dz * dz), h);
  }
  *rho = sum;
  if (nbr) *nbr = cnt;
  return ORC_OK;
}

/* a_i = g - sum_j m (p_i / rho_i^2 + p_j / rho_j^2) grad W_ij - sum_j m Pi_ij grad W_ij,
 * Pi_ij = -nu (v_ij . x_ij) / (|x_ij|^2 + 0.01 h^2) for v_ij . x_ij < 0,
 * nu = 2 alpha h c / (rho_i + rho_j).  Boundary j: p_j = 0, rho_j = rho_i, v_j = 0. */
static int accel_one(const orc_params* P, const ogrid* G, int32_t n, const double* x,
                     const double* v, const double* rho, const double* p, const double* xb,
                     int32_t i, int32_t* buf, double* out) {
  int c[3];
  if (orci_block_coords(P, x + 3 * (int64_t)i, c)) return ORC_ERR_DOMAIN;
  int cnt = orci_nbr_list(P, G, n, x, xb, i, c, 1, P->r * P->r, buf, NBR_CAP);
  if (cnt < 0) return ORC_ERR_CAPACITY;
  double h = 0.5 * P->r, m = orci_particle_mass(P);
  const double* xi = x + 3 * (int64_t)i;
  const double* vi = v + 3 * (int64_t)i;
  double ri = rho[i], pi = p[i];
  double a[3] = {P->g[0], P->g[1], P->g[2]};
  for (int q = 0; q < cnt; ++q) {
    int32_t j = buf[q];
    const double* xj;
    double vj[3], rj, pj;
    if (j < n) {
      xj = x + 3 * (int64_t)j;
      vj[0] = v[3 * (int64_t)j]; vj[1] = v[3 * (int64_t)j + 1]; vj[2] = v[3 * (int64_t)j + 2];
      rj = rho[j]; pj = p[j];
    } else {
      xj = xb + 3 * (int64_t)(j - n);
      vj[0] = vj[1] = vj[2] = 0.0;
      rj = ri; pj = 0.0;
    }
    double xij[3] = {xi[0] - xj[0], xi[1] - xj[1], xi[2] - xj[2]};
    double d2 = xij[0] * xij[0] + xij[1] * xij[1] + xij[2] * xij[2];
    double d = sqrt(d2);
    double gw[3] = {0.0, 0.0, 0.0};
    if (d > 0.0) {
      double f = orc_kernel_dW(d, h) / d;
      gw[0] = f * xij[0]; gw[1] = f * xij[1]; gw[2] = f * xij[2];
    }
    double pterm = pi / (ri * ri) + pj / (rj * rj);
    double vij[3] = {vi[0] - vj[0], vi[1] - vj[1], vi[2] - vj[2]};
    double vx = vij[0] * xij[0] + vij[1] * xij[1] + vij[2] * xij[2];
    double visc = 0.0;
    if (vx < 0.0) {
      double nu = 2.0 * P->visc_alpha * h * P->c_s / (ri + rj);
      visc = -nu * vx / (d2 + 0.01 * h * h);
    }
    for (int k = 0; k < 3; ++k) a[k] -= m * (pterm + visc) * gw[k];
  }
  out[0] = a[0]; out[1] = a[1]; out[2] = a[2];
  return ORC_OK;
}

static int density_masked(const orc_params* P, const ogrid* G, int32_t n, const double* x,
                          const double* xb, const uint8_t* mask, double* rho, double* p,
                          int32_t* nbr) {
  int err = ORC_OK;
#pragma omp parallel
  {
    int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * NBR_CAP);
#pragma omp for schedule(dynamic, 256)
    for (int32_t i = 0; i < n; ++i) {
      if (mask && !mask[i]) continue;
      int32_t cnt = 0;
      int st = density_one(P, G, n, x, xb, i, buf, &rho[i], &cnt);
      if (st) {
#pragma omp critical
        err = st;
        continue;
      }
      p[i] = tait(P, rho[i]);
      if (nbr) nbr[i] = cnt;
    }
    free(buf);
  }
  return err;
}

static int accel_masked(const orc_params* P, const ogrid* G, int32_t n, const double* x,
                        const double* v, const double* rho, const double* p, const double* xb,
                        const uint8_t* mask, double* a_out) {
  int err = ORC_OK;
#pragma omp parallel
  {
    int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * NBR_CAP);
#pragma omp for schedule(dynamic, 256)
    for (int32_t i = 0; i < n; ++i) {
      if (mask && !mask[i]) continue;
      int st = accel_one(P, G, n, x, v, rho, p, xb, i, buf, a_out + 3 * (int64_t)i);
      if (st) {
#pragma omp critical
        err = st;
      }
    }
    free(buf);
  }
  return err;
}

int orc_wcsph_density(const orc_params* P, int32_t n, const double* x, int32_t nb,
                      const double* xb, const uint8_t* mask, double* rho, double* p,
                      int32_t* nbr) {
  ogrid G;
  int st = orci_grid_build(P, n, x, nb, xb, &G);
  if (st) return st;
  st = density_masked(P, &G, n, x, xb, mask, rho, p, nbr);
  orci_grid_free(&G);
  return st;
}

int orc_wcsph_accel(const orc_params* P, int32_t n, const double* x, const double* v,
                    const double* rho, const double* p, int32_t nb, const double* xb,
                    const uint8_t* mask, double* a_out) {
  ogrid G;
  int st = orci_grid_build(P, n, x, nb, xb, &G);
  if (st) return st;
  st = accel_masked(P, &G, n, x, v, rho, p, xb, mask, a_out);
  orci_grid_free(&G);
  return st;
}

/* ----------------------------------------------------------- classification --- */

/* Eq. 1: dt_n <= lambda_v r / c_s (WCSPH only).  Eq. 2 squared twice with F = m |a|:
 * |a|^2 <= (lambda_f^2 r / dt_n^2)^2.  Eq. 3: |v|^2 <= (alpha beta_n r / dt_n)^2. */
void orc_level_thresholds(const orc_params* P, double* vthr2, double* athr2, int32_t* eq1) {
  for (int L = 0; L < P->n_levels; ++L) {
    double dt = (double)P->mult[L] * P->dt_b;
    double vt = P->alpha * P->beta[L] * P->r / dt;
    vthr2[L] = vt * vt;
    double at = P->lambda_f * P->lambda_f * P->r / (dt * dt);
    athr2[L] = at * at;
    eq1[L] = P->scheme == 0 ? (dt <= P->lambda_v * P->r / P->c_s) : 1;
  }
}

double orci_norm2(const double* u) {
  double s = u[0] * u[0];
  s = s + u[1] * u[1];
  s = s + u[2] * u[2];
  return s;
}

/* Section 3.1: a block takes the largest level whose criteria hold for the maximum
 * velocity and force of its particles; level 0 if none holds. */
int32_t orci_pick_level(const orc_params* P, const double* vthr2, const double* athr2,
                          const int32_t* eq1, double vmax2, double amax2) {
  int32_t L = 0;
  for (int l = 0; l < P->n_levels; ++l)
    if (eq1[l] && vmax2 <= vthr2[l] && amax2 <= athr2[l]) L = l;
  return L;
}

/* Raw block levels from the block maxima (Section 3.1 steps 1-2). */
int orci_raw_levels(const orc_params* P, int32_t n, const double* x, const double* v,
                      const double* a, int32_t* raw) {
  int32_t B = orci_n_blocks(P);
  double* vmax = (double*)malloc(sizeof(double) * (size_t)B);
  double* amax = (double*)malloc(sizeof(double) * (size_t)B);
  for (int32_t b = 0; b < B; ++b) { vmax[b] = -1.0; amax[b] = -1.0; }
  int st = ORC_OK;
  for (int32_t i = 0; i < n; ++i) {
    int32_t key;
    st = orc_block_key(P, x + 3 * (int64_t)i, &key);
    if (st) break;
    double v2 = orci_norm2(v + 3 * (int64_t)i), a2 = orci_norm2(a + 3 * (int64_t)i);
    if (v2 > vmax[key]) vmax[key] = v2;
    if (a2 > amax[key]) amax[key] = a2;
  }
  if (!st) {
    double vthr2[8], athr2[8];
    int32_t eq1[8];
    orc_level_thresholds(P, vthr2, athr2, eq1);
    for (int32_t b = 0; b < B; ++b)
      raw[b] = vmax[b] < 0.0 ? -1 : orci_pick_level(P, vthr2, athr2, eq1, vmax[b], amax[b]);
  }
  free(vmax);
  free(amax);
  return st;
}

/* Section 4.2 R_min: a filled block takes the smallest level among itself and its
 * filled 26 neighbours (one pass, reading the unsmoothed levels). */
void orci_rmin_smooth(const orc_params* P, const int32_t* raw, int32_t* out) {
  for (int bz = 0; bz < P->dim[2]; ++bz)
    for (int by = 0; by < P->dim[1]; ++by)
      for (int bx = 0; bx < P->dim[0]; ++bx) {
        int32_t b = orci_block_lin(P, bx, by, bz);
        int32_t L = raw[b];
        if (L >= 0) {
          for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
              for (int dx = -1; dx <= 1; ++dx) {
                int cx = bx + dx, cy = by + dy, cz = bz + dz;
                if (cx < 0 || cy < 0 || cz < 0 || cx >= P->dim[0] || cy >= P->dim[1] ||
                    cz >= P->dim[2])
                  continue;
                int32_t Lc = raw[orci_block_lin(P, cx, cy, cz)];
                if (Lc >= 0 && Lc < L) L = Lc;
              }
        }
        out[b] = L;
      }
}

int orc_classify_wcsph(const orc_params* P, int32_t n, const double* x, const double* v,
                       const double* a, int32_t* raw, int32_t* level) {
  int32_t B = orci_n_blocks(P);
  int32_t* r = raw ? raw : (int32_t*)malloc(sizeof(int32_t) * (size_t)B);
  int st = orci_raw_levels(P, n, x, v, a, r);
  if (!st) {
    if (P->force_level >= 0) {
      for (int32_t b = 0; b < B; ++b) level[b] = r[b] < 0 ? -1 : P->force_level;
    } else {
      orci_rmin_smooth(P, r, level);
    }
  }
  if (!raw) free(r);
  return st;
}

/* --------------------------------------------------- Algorithm 1 (WCSPH RTS) --- */

/* Density, pressure and acceleration of the particles with mask set, at the
 * current positions and velocities; every other particle keeps its held values. */
static int evaluate_masked(const orc_params* P, orc_wstate* S, const uint8_t* mask,
                           double* anew) {
  ogrid G;
  int st = orci_grid_build(P, S->n, S->x, S->nb, S->xb, &G);
  if (st) return st;
  st = density_masked(P, &G, S->n, S->x, S->xb, mask, S->rho, S->p, S->nbr);
  if (!st) st = accel_masked(P, &G, S->n, S->x, S->v, S->rho, S->p, S->xb, mask, anew);
  orci_grid_free(&G);
  return st;
}

/* Section 4.1 correction at the end of a particle's true step of length dt:
 * x += (a_new - a_old) dt^2 / 6, v += (a_new - a_old) dt / 2. */
static void serna_correct(const orc_params* P, double* x, double* v, double* a,
                          const double* anew, double dt) {
  for (int k = 0; k < 3; ++k) {
    double da = anew[k] - a[k];
    if (!P->serna_off) {
      x[k] = x[k] + da * dt * dt / 6.0;
      v[k] = v[k] + da * dt / 2.0;
    }
    a[k] = anew[k];
  }
}

/* Container walls.  The paper's static boundary particles come with no force law; the
 * particles exert -m p_i/rho_i^2 grad W, which a fast particle can overcome, so a
 * position update is followed by the non-penetration correction of particle-based
 * boundary handling: a coordinate beyond a face of the box is set to the face and the
 * velocity component into the face is dropped (tangential motion is kept). */
void orci_wall_project(const orc_params* P, double* x3, double* v3) {
  if (!P->wall_project) return;
  for (int k = 0; k < 3; ++k) {
    if (x3[k] < P->wall_lo[k]) {
      x3[k] = P->wall_lo[k];
      if (v3[k] < 0.0) v3[k] = 0.0;
    }
    if (x3[k] > P->wall_hi[k]) {
      x3[k] = P->wall_hi[k];
      if (v3[k] > 0.0) v3[k] = 0.0;
    }
  }
}

/* Section 4.1 predictor: x~ = x + v dt + a dt^2 / 2, v~ = v + a dt (all particles),
 * then the container correction. */
static void serna_predict(const orc_params* P, int32_t n, double* x, double* v, const double* a,
                          double dt) {
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < 3 * (int64_t)n; ++q) {
    x[q] = x[q] + v[q] * dt + a[q] * dt * dt / 2.0;
    v[q] = v[q] + a[q] * dt;
  }
  for (int32_t i = 0; i < n; ++i) orci_wall_project(P, x + 3 * (int64_t)i, v + 3 * (int64_t)i);
}

/* Validity of a particle that starts a true step of multiplier m at substep k:
 * Algorithm 1 counts m substeps; the level-aligned variant counts to the next multiple
 * of m, so the particles of a level compute together. */
static int32_t new_validity(const orc_params* P, int32_t m, int64_t k) {
  return P->level_clock ? (int32_t)(m - k % m) : m;
}

static int32_t particle_block_level(const orc_params* P, const orc_wstate* S, int32_t i) {
  int32_t key;
  if (orc_block_key(P, S->x + 3 * (int64_t)i, &key)) return -1;
  return S->block_level[key];
}

/* Priming evaluation at time k dt_b: every particle computes (validity 0) and takes
 * its block's level; no time passes, so the correction vanishes. */
int orc_wcsph_evaluate(const orc_params* P, orc_wstate* S) {
  int32_t n = S->n;
  int st = orc_classify_wcsph(P, n, S->x, S->v, S->a, NULL, S->block_level);
  if (st) return st;
  for (int32_t i = 0; i < n; ++i) {
    int32_t L = particle_block_level(P, S, i);
    S->level[i] = L;
    S->validity[i] = new_validity(P, P->mult[L], S->k);
    S->compute[i] = 1;
  }
  double* anew = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  st = evaluate_masked(P, S, NULL, anew);
  if (!st) {
    for (int32_t i = 0; i < n; ++i) {
      for (int k = 0; k < 3; ++k) S->a[3 * (int64_t)i + k] = anew[3 * (int64_t)i + k];
      S->klast[i] = (int32_t)S->k;
    }
    S->primed = 1;
  }
  free(anew);
  return st;
}

/* One base substep k -> k + 1 of Algorithm 1: predict everyone, rebuild the grid,
 * assign block levels, decrement validity and pre-empt on level change, evaluate the
 * computing particles against everyone's predicted state, correct them. */
int orc_wcsph_substep(const orc_params* P, orc_wstate* S) {
  int st;
  if (!S->primed && (st = orc_wcsph_evaluate(P, S))) return st;
  int32_t n = S->n;
  int64_t k1 = S->k + 1;
  serna_predict(P, n, S->x, S->v, S->a, P->dt_b);
  st = orc_classify_wcsph(P, n, S->x, S->v, S->a, NULL, S->block_level);
  if (st) return st;
  for (int32_t i = 0; i < n; ++i) {
    int32_t Lb = particle_block_level(P, S, i);
    S->validity[i] -= 1;
    if (S->validity[i] <= 0 || S->level[i] < 0 || P->mult[Lb] != P->mult[S->level[i]]) {
      S->compute[i] = 1;
      S->level[i] = Lb;
      S->validity[i] = new_validity(P, P->mult[Lb], k1);
    } else {
      S->compute[i] = 0;
    }
  }
  double* anew = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  st = evaluate_masked(P, S, S->compute, anew);
  if (!st) {
    for (int32_t i = 0; i < n; ++i) {
      if (!S->compute[i]) continue;
      double dt = (double)(k1 - S->klast[i]) * P->dt_b;
      serna_correct(P, S->x + 3 * (int64_t)i, S->v + 3 * (int64_t)i, S->a + 3 * (int64_t)i,
                    anew + 3 * (int64_t)i, dt);
      S->klast[i] = (int32_t)k1;
    }
    S->k = k1;
  }
  free(anew);
  return st;
}

/* Global comparator (Section 6 "standard" stepping with the Section 3.1 criteria
 * applied to the whole fluid): one step of mult * dt_b, every particle active. */
int orc_wcsph_global_step(const orc_params* P, orc_wstate* S, int32_t max_mult,
                          int32_t* mult_used) {
  int st;
  if (!S->primed && (st = orc_wcsph_evaluate(P, S))) return st;
  int32_t n = S->n;
  int32_t L = 0;
  if (P->mode != 2) {
    double vmax2 = 0.0, amax2 = 0.0;
    for (int32_t i = 0; i < n; ++i) {
      double v2 = orci_norm2(S->v + 3 * (int64_t)i), a2 = orci_norm2(S->a + 3 * (int64_t)i);
      if (v2 > vmax2) vmax2 = v2;
      if (a2 > amax2) amax2 = a2;
    }
    double vthr2[8], athr2[8];
    int32_t eq1[8];
    orc_level_thresholds(P, vthr2, athr2, eq1);
    L = orci_pick_level(P, vthr2, athr2, eq1, vmax2, amax2);
  }
  int32_t m = P->mult[L];
  if (m > max_mult) m = max_mult;
  if (m < 1) m = 1;
  int64_t k1 = S->k + m;
  serna_predict(P, n, S->x, S->v, S->a, (double)m * P->dt_b);
  for (int32_t i = 0; i < n; ++i) {
    S->compute[i] = 1;
    S->level[i] = L;
    S->validity[i] = m;
  }
  double* anew = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  st = evaluate_masked(P, S, NULL, anew);
  if (!st) {
    for (int32_t i = 0; i < n; ++i) {
      double dt = (double)(k1 - S->klast[i]) * P->dt_b;
      serna_correct(P, S->x + 3 * (int64_t)i, S->v + 3 * (int64_t)i, S->a + 3 * (int64_t)i,
                    anew + 3 * (int64_t)i, dt);
      S->klast[i] = (int32_t)k1;
    }
    S->k = k1;
    if (mult_used) *mult_used = m;
  }
  free(anew);
  return st;
}
