/* oracle_internal.h - helpers shared by the oracle's C files (test infrastructure). */
#ifndef ORACLE_INTERNAL_H
#define ORACLE_INTERNAL_H
#include "rts_oracle.h"

#define NBR_CAP 8192

typedef struct {
  int32_t B;
  int32_t *key, *cs, *pm;    /* fluid */
  int32_t *bkey, *bcs, *bpm; /* boundary */
} ogrid;

int orci_block_coords(const orc_params* P, const double* x, int c[3]);
int32_t orci_block_lin(const orc_params* P, int bx, int by, int bz);
int32_t orci_n_blocks(const orc_params* P);
int orci_is_nbr(const double* a, const double* b, double r2);
double orci_norm2(const double* u);
int32_t orci_pick_level(const orc_params* P, const double* vthr2, const double* athr2,
                        const int32_t* eq1, double vmax2, double amax2);
void orci_rmin_smooth(const orc_params* P, const int32_t* raw, int32_t* out);
int orci_raw_levels(const orc_params* P, int32_t n, const double* x, const double* v,
                    const double* a, int32_t* raw);
double orci_particle_mass(const orc_params* P);
int orci_grid_build(const orc_params* P, int32_t n, const double* x, int32_t nb,
                    const double* xb, ogrid* G);
void orci_grid_free(ogrid* G);
int orci_nbr_list(const orc_params* P, const ogrid* G, int32_t n, const double* x,
                  const double* xb, int32_t i, const int c[3], int rings, double r2,
                  int32_t* out, int cap);
void orci_wall_project(const orc_params* P, double* x3, double* v3);
#endif
