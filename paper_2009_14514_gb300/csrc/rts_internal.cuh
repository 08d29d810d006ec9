// rts_internal.cuh - device-side types shared by librts's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rts.h"

namespace rts {

constexpr int kMaxLevels = 8;

// Parameters as the kernels use them (FP32 physics, FP64 decision thresholds).
struct DevParams {
  // block grid (Section 3)
  float ox, oy, oz, edge, inv_edge;
  double oxd, oyd, ozd, edged;
  int nx, ny, nz;
  int nblocks;
  int max_per_block;
  // cubic spline kernel, h = r / 2, support r
  float r, r2, r2_lo, r2_hi, h, inv_h, sigma, sigma_h;  // sigma_h = sigma / h
  double r2d;
  // WCSPH physics
  float m, rho0, inv_rho0, tait_B, gamma;
  int gamma_is_7;
  float visc_coef;   // 2 alpha h c_s
  float eps_h2;      // 0.01 h^2
  float gx, gy, gz;
  int nbl_cap;       // neighbour list capacity per particle
  // levels (Section 3.1)
  int n_levels;
  int mult[kMaxLevels];
  double vthr2[kMaxLevels], athr2[kMaxLevels];
  int eq1[kMaxLevels];
  int force_level;
  float dt_b;
};

// Device control block: status and counters written by kernels.
struct Ctl {
  int status;                    // first device error (rts_status), 0 = none
  int n_act;                     // active blocks in the work list
  unsigned long long evals;      // evaluated particles
  unsigned long long pairs;      // neighbour pairs of evaluated particles
  unsigned long long act_blocks; // active blocks summed over steps
  unsigned long long cands;      // candidate pairs tested
  int n_filled;                  // blocks holding a fluid particle (filled list length)
  unsigned long long vmax2_bits; // global max |v|^2 (FP64 bits, non-negative)
  unsigned long long amax2_bits; // global max |a|^2
  unsigned long long level_count[kMaxLevels];
};

// Particle state in block-sorted order.  x.w = p / rho^2 and v.w = rho of the last
// evaluation, so a neighbour's force inputs arrive in two float4 loads.
struct PState {
  float4* x;
  float4* v;
  float4* a;        // held acceleration
  float* rho;
  float* prs;
  uint32_t* uid;    // caller's index
  int32_t* klast;   // substep of the last evaluation
  int32_t* valid;   // validity counter (base substeps)
  int32_t* level;   // particle level, -1 = none
  int32_t* nbr;     // neighbour count at the last evaluation
};

__device__ __forceinline__ void set_status(Ctl* ctl, int code) {
  atomicCAS(&ctl->status, 0, code);
}

// Activity kernel modes.
enum ActMode { kActRegional = 0, kActAll = 1, kActGlobal = 2 };

}  // namespace rts

// ------------------------------------------------------------------ context ---

struct rts_ctx {
  rts_params p;
  rts::DevParams dp;
  cudaStream_t stream;
  int n, nb;
  int64_t k;          // completed base substeps
  int primed;
  int sticky;         // pending device error
  int bins_valid;
  char err[512];

  // fluid state, double buffered for the block sort
  rts::PState s, s2;
  float4* anew;
  uint8_t* cflag;
  uint32_t* key;      // block of each sorted particle
  uint32_t* key_tmp;
  uint32_t* slot;
  uint32_t* tmp_uid;
  uint32_t* tmp_src;
  uint32_t* count;    // per block, kept zero between bins
  uint32_t* cstart;   // nblocks + 1
  uint32_t* tile_sums;
  int ntiles;
  // Per-block records stamped with the binning pass that wrote them, so nothing has to
  // be cleared between passes: a record is current iff its stamp equals c->stamp.
  uint32_t stamp;                 // binning pass counter (1 .. 2^24 - 1)
  unsigned long long* bmax_v;     // (stamp << 32) | FP32 bits of the block max |v|^2
  unsigned long long* bmax_a;     // (stamp << 32) | FP32 bits of the block max |a|^2
  uint32_t* raw;                  // (stamp << 8) | level from Eq. 1-3
  uint32_t* blevel;               // (stamp << 8) | level after smoothing
  uint32_t* filled;               // list of filled blocks of the current pass
  uint32_t* act;      // active block list
  rts::Ctl* ctl;
  rts::Ctl* h_ctl;    // pinned host mirror

  // boundary, binned once
  float4* xb;
  uint32_t* bcstart;

  // staging for caller-order I/O
  float* io;          // n * 4 floats
  int32_t* io_i;      // n ints

  int grid_persistent;  // CTAs of the persistent neighbour kernels
  uint32_t* nbl;        // neighbour lists of evaluated particles, nbl_cap per particle
  int nbl_cap;
  int last_global_level;

  // launch counting and optional per-phase event timing
  int cur_phase;
  int64_t kernels;
  int64_t launches[RTS_NUM_PHASES];
  int prof;
  double prof_ms[RTS_NUM_PHASES];
  cudaEvent_t* ev;    // 2 * kEvPairs events
  int* ev_phase;
  int nev;
};

namespace rts {
constexpr int kEvPairs = 1024;
inline void note_launch(rts_ctx* c, int k) {
  c->kernels += k;
  c->launches[c->cur_phase] += k;
}
}  // namespace rts

// Host helpers implemented in rts_api.cu / kernels implemented in the .cu files.
namespace rts {
rts_status launch_bin(rts_ctx* c, float dt_predict);
rts_status launch_bin_boundary(rts_ctx* c, const float4* xb_unsorted, int nb);
rts_status launch_classify(rts_ctx* c);
rts_status launch_activity(rts_ctx* c, int mode, int level_g, int mult_g);
rts_status launch_density(rts_ctx* c);
rts_status launch_force(rts_ctx* c);
rts_status launch_correct(rts_ctx* c, int64_t k1, int prime);
rts_status launch_global_max(rts_ctx* c);
rts_status launch_level_hist(rts_ctx* c);
const char* cuda_err(rts_ctx* c, cudaError_t e, const char* what);
}  // namespace rts
