// rts_internal.cuh - device-side types shared by librts's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rts.h"

namespace rts {

constexpr int kMaxLevels = 8;

// One scene of a batch: its own block grid (origin in its own coordinates, dims) placed
// in the stacked grid at z offset z0, and its container.
struct SceneGeo {
  float o[3];
  double od[3];
  int n[3];
  int z0;
  float band;        // FP32 block-coordinate band of this scene's grid (see block_coord)
  float wlo[3], whi[3];
};

// Parameters as the kernels use them (FP32 physics, FP64 decision thresholds).
struct DevParams {
  // block grid (Section 3)
  float ox, oy, oz, edge, inv_edge;
  double oxd, oyd, ozd, edged;
  int nx, ny, nz;
  int nblocks;
  // floor(u / nx) = (u * div_nx) >> 40 for every u < 2^24 (exact for divisors < 2^16:
  // div = floor(2^40 / d) + 1 overshoots 1/d by less than 2^-40, too little to reach the
  // next integer); the same for ny.
  unsigned long long div_nx, div_ny;
  int max_per_block;
  float key_band;    // FP32 block-coordinate band that defers to FP64 (see block_coord)
  // cubic spline kernel, h = r / 2, support r
  float r, r2, r2_lo, r2_hi, h, inv_h, sigma, sigma_h;  // sigma_h = sigma / h
  double r2d;
  float r2_dh, r2_dl, r2_win;  // r2d = r2_dh + r2_dl exactly; undecided window 2^-38 r2d
  // WCSPH physics
  float m, rho0, inv_rho0, tait_B, gamma;
  int gamma_is_7;
  float visc_coef;   // 2 alpha h c_s
  float eps_h2;      // 0.01 h^2
  float gx, gy, gz;
  int wall_project;        // non-penetration projection onto the container box
  float wlo[3], whi[3];
  int nbl_cap;       // neighbour list capacity per particle
  int n_fluid, n_bound;  // particle counts (bounds of the consistency checks)
  // PCISPH (Section 5)
  float eta, delta, visc_nu;   // tolerance, pressure scaling, alpha h c / rho0
  int r1_rings, expand_layers, n_minor;
  int sched[4][8];
  int refresh[8];
  // levels (Section 3.1)
  int n_levels;
  int mult[kMaxLevels];
  double vthr2[kMaxLevels], athr2[kMaxLevels];
  float vthr2f[kMaxLevels], athr2f[kMaxLevels];   // the same thresholds rounded to FP32
  float vthr2lo[kMaxLevels], athr2lo[kMaxLevels]; // and their FP32 residuals
  float vnear[kMaxLevels], anear[kMaxLevels];     // 2e-6 of each finite FP32 threshold, else -1
  int eq1[kMaxLevels];
  int levels_monotone;   // both thresholds non-increasing in the level (see k_block_levels)
  int force_level;
  int level_clock;   // 0: validity = multiplier (Algorithm 1); 1: aligned to multiples
  int no_clamp;      // 1: negative Tait pressure kept
  int serna_off;     // 1: the Section 4.1 correction is skipped (ablation)
  int r2_rings;      // PCISPH neighbour search rings of region 2
  float dt_b;
  // batched scenes (n_scenes = 0: one scene, the fields above describe its grid)
  int n_scenes;
  const SceneGeo* geo;       // per scene
  const uint32_t* fbase;     // n_scenes + 1: first fluid particle of each scene (caller
                             // order, and block order: scenes occupy disjoint z ranges)
  const uint32_t* bbase;     // n_scenes + 1: first boundary particle of each scene
  const int* zbase;          // n_scenes + 1: first z layer of each scene in the stacked grid
};

// Device control block: status and counters written by kernels.
struct Ctl {
  int status;                    // first device error (rts_status), 0 = none
  int n_act;                     // active blocks in the work list
  int n_plist;                   // evaluated particles in the particle work list
  int dens_next;                 // density pass: work items handed out after the first round
  unsigned long long evals;      // evaluated particles
  unsigned long long pairs;      // neighbour pairs of evaluated particles
  unsigned long long act_blocks; // active blocks summed over steps
  unsigned long long cands;      // candidates of the evaluated particles' 27-block stencils
  unsigned long long kept;       // candidate pairs tested after the per-group cull
  int n_filled;                  // blocks holding a fluid particle (filled list length)
  unsigned long long vmax2_bits; // global max |v|^2 (FP64 bits, non-negative)
  unsigned long long amax2_bits; // global max |a|^2
  unsigned int vmax2f_bits;      // the same maxima of the FP32 norms (FP32 bits)
  unsigned int amax2f_bits;
  unsigned long long level_count[kMaxLevels];
  unsigned int err_max_bits;      // PCISPH: max relative error (FP32 bits)
  unsigned long long err_sum_fx;  // PCISPH: sum of relative errors, fixed point 2^-32
  int chk_code;                   // first failed consistency check (CheckCode), 0 = none
  unsigned int chk_val;           // the offending value
  int bad_set;                    // a particle left the grid: its caller index and position
  unsigned int bad_uid;
  float bad_x, bad_y, bad_z;
  // Substeps that keep the previous sort: the largest per-axis distance (FP32 bits,
  // rounded up) by which a particle has left the block it was sorted into, in slot
  // stamp & 1 of the pass that computed it.
  unsigned int disp_bits[2];
  int n_filled_light[2];          // filled-list length of such a pass, slot stamp & 1
  int n_near[2];                  // its list of particles near a level threshold, slot stamp & 1
};

// Capacity of that list; beyond it the level fallback scans the sorted cells instead.
constexpr int kNearCap = 1 << 16;

// Device-side consistency checks: an index read from memory is tested before it is
// used; a failure records its code and value, sets RTS_ERR_INTERNAL and skips the access.
enum CheckCode {
  kChkNone = 0, kChkNeighbour = 1, kChkRun = 2, kChkGather = 3, kChkScatter = 4,
  kChkLevel = 5, kChkUid = 6, kChkActive = 7,
  kChkDisp = 8   // a particle moved half a block or more since the last sort
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
  float4* ap;       // PCISPH: pressure acceleration of the current minor step (else null)
  float* err;       // PCISPH: latest relative compression error (else null)
};

struct BatchState;  // batched scenes (rts_batch.cu)

__device__ __forceinline__ void set_status(Ctl* ctl, int code) {
  atomicCAS(&ctl->status, 0, code);
}

static __device__ __noinline__ void check_failed(Ctl* ctl, int code, unsigned int val) {
  if (atomicCAS(&ctl->chk_code, 0, code) == 0) ctl->chk_val = val;
  set_status(ctl, 9 /* RTS_ERR_INTERNAL */);
}

// Section 4.1 correction at the end of a particle's true step of length dt:
// x += (a_new - a_old) dt^2 / 6, v += (a_new - a_old) dt / 2 (w lanes untouched).
// Shared by the correction kernel and the key pass that applies a deferred correction,
// so both give the same bits.
__device__ __forceinline__ void serna_correct(float4& x, float4& v, const float4 ao,
                                              const float4 an, float dt) {
  const float c1 = dt * dt / 6.0f, c2 = 0.5f * dt;
  const float dax = an.x - ao.x, day = an.y - ao.y, daz = an.z - ao.z;
  x.x += dax * c1;
  x.y += day * c1;
  x.z += daz * c1;
  v.x += dax * c2;
  v.y += day * c2;
  v.z += daz * c2;
}

// A correction left pending by the last stepping call (applied by the next key pass,
// or by the correction kernel when the state is read).
enum PendMode { kPendNone = 0, kPendCorrect = 1, kPendPrime = 2 };

// Block coordinate floor((x - o) / edge).  The FP32 quotient t = (x - o) * (1 / edge)
// carries three roundings, so it is within 3 * 2^-24 * t of the exact one; within
// band (8 * 2^-24 * the largest coordinate of the grid, set on the host) of an integer
// the FP64 quotient decides, so the result is that of the double-precision definition.
// Outside the band the FP32 floor is the answer; its range test and conversion stay in
// FP32 (exact: n < 2^24), so FP64 (a small fraction of the FP32 rate here) runs only in
// the band.
__device__ __forceinline__ int block_coord(float x, float o, double od, float inv_e, double ed,
                                           int n, float band, int* bad) {
  float t = (x - o) * inv_e;
  float f = floorf(t);
  float fr = t - f;
  if (fr < band || fr > 1.0f - band) {
    const double fd = floor(__ddiv_rn(__dsub_rn((double)x, od), ed));
    if (!(fd >= 0.0 && fd < (double)n)) {
      *bad = 1;
      return 0;
    }
    return (int)fd;
  }
  if (!(f >= 0.0f && f < (float)n)) {
    *bad = 1;
    return 0;
  }
  return (int)f;
}

// ------------------------------------------------ exact neighbour predicate ---
//
// The neighbour test of the double-precision definition, |x_i - x_j|^2 < r^2 with the
// squared distance formed in FP64 from the FP32 positions, for pairs inside the FP32
// guard band.  FP64 runs at a small fraction of the FP32 rate on this GPU, and lattice
// states (resting pools, an undisturbed column) put many pairs at exactly r, so the
// squared distance S is first formed without rounding error in FP32 pieces: the
// coordinate differences by Knuth's TwoSum (d = dh + dl exactly), their squares by the
// FMA TwoProduct (dh^2 = p + e exactly), the three p summed by TwoSum; the small terms
// (e, 2 dh dl, the TwoSum errors; dl^2 <= 2^-48 dh^2 is dropped) are added in FP32.  S
// is then known within 2^-42 S, and FP64 forms it within 3 * 2^-53 S, so whenever the
// computed S - r^2 lies outside +-2^-38 r^2 both give the same answer; inside that
// window (a near or exact tie) the FP64 expression itself decides.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

static __device__ __noinline__ bool nbr_exact_fp64(float4 a, float4 b, double r2d) {
  const double dx = __dsub_rn((double)a.x, (double)b.x);
  const double dy = __dsub_rn((double)a.y, (double)b.y);
  const double dz = __dsub_rn((double)a.z, (double)b.z);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)) < r2d;
}

__device__ __forceinline__ bool nbr_exact(const DevParams& P, float4 a, float4 b) {
  float hx, lx, hy, ly, hz, lz;
  two_sum(a.x, -b.x, hx, lx);
  two_sum(a.y, -b.y, hy, ly);
  two_sum(a.z, -b.z, hz, lz);
  const float px = __fmul_rn(hx, hx), py = __fmul_rn(hy, hy), pz = __fmul_rn(hz, hz);
  const float ex = __fmaf_rn(hx, hx, -px), ey = __fmaf_rn(hy, hy, -py), ez = __fmaf_rn(hz, hz, -pz);
  float s1, t1, s2, t2;
  two_sum(px, py, s1, t1);
  two_sum(s1, pz, s2, t2);
  const float cross = __fmul_rn(2.0f, __fadd_rn(__fadd_rn(__fmul_rn(hx, lx), __fmul_rn(hy, ly)),
                                                  __fmul_rn(hz, lz)));
  const float small = __fadd_rn(__fadd_rn(__fadd_rn(ex, ey), __fadd_rn(ez, cross)), __fadd_rn(t1, t2));
  const float diff = __fadd_rn(__fsub_rn(s2, P.r2_dh), __fsub_rn(small, P.r2_dl));
  if (diff < -P.r2_win) return true;
  if (diff > P.r2_win) return false;
  return nbr_exact_fp64(a, b, P.r2d);
}

__device__ __forceinline__ uint32_t block_key(const DevParams& P, float4 p, int* bad) {
  int cx = block_coord(p.x, P.ox, P.oxd, P.inv_edge, P.edged, P.nx, P.key_band, bad);
  int cy = block_coord(p.y, P.oy, P.oyd, P.inv_edge, P.edged, P.ny, P.key_band, bad);
  int cz = block_coord(p.z, P.oz, P.ozd, P.inv_edge, P.edged, P.nz, P.key_band, bad);
  return ((uint32_t)cz * P.ny + cy) * P.nx + cx;
}

__device__ __forceinline__ uint32_t div_by(uint32_t u, unsigned long long m) {
  return (uint32_t)(((unsigned long long)u * m) >> 40);
}

// Non-penetration of the container box: a particle beyond a face is put back on it and
// the velocity component into that face is removed.
__device__ __forceinline__ void wall_project_box(const float* lo, const float* hi, float4& x,
                                                 float4& v) {
  if (x.x < lo[0]) { x.x = lo[0]; v.x = fmaxf(v.x, 0.f); }
  if (x.x > hi[0]) { x.x = hi[0]; v.x = fminf(v.x, 0.f); }
  if (x.y < lo[1]) { x.y = lo[1]; v.y = fmaxf(v.y, 0.f); }
  if (x.y > hi[1]) { x.y = hi[1]; v.y = fminf(v.y, 0.f); }
  if (x.z < lo[2]) { x.z = lo[2]; v.z = fmaxf(v.z, 0.f); }
  if (x.z > hi[2]) { x.z = hi[2]; v.z = fminf(v.z, 0.f); }
}

__device__ __forceinline__ void wall_project(const DevParams& P, float4& x, float4& v) {
  wall_project_box(P.wlo, P.whi, x, v);
}

// Scene of entry i of a base table (largest s with base[s] <= i; empty scenes share
// their successor's base and are skipped).
__device__ __forceinline__ int scene_of(const uint32_t* base, int ns, uint32_t i) {
  int lo = 0, hi = ns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(base + mid) <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int scene_of_z(const int* zbase, int ns, int z) {
  int lo = 0, hi = ns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(zbase + mid) <= z) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Block of a particle of scene sc in the stacked grid: the scene's own block coordinates
// (from its origin, in its own coordinates), shifted by the scene's z offset.
__device__ __forceinline__ uint32_t batch_key(const DevParams& P, float4 p, int sc, int* bad) {
  const SceneGeo& g = P.geo[sc];
  int cx = block_coord(p.x, g.o[0], g.od[0], P.inv_edge, P.edged, g.n[0], g.band, bad);
  int cy = block_coord(p.y, g.o[1], g.od[1], P.inv_edge, P.edged, g.n[1], g.band, bad);
  int cz = block_coord(p.z, g.o[2], g.od[2], P.inv_edge, P.edged, g.n[2], g.band, bad);
  return ((uint32_t)(cz + g.z0) * P.ny + cy) * P.nx + cx;
}

// Container of the particle at block-order index i (its scene's box in a batch).
__device__ __forceinline__ void wall_project_at(const DevParams& P, uint32_t i, float4& x,
                                                float4& v) {
  if (P.n_scenes) {
    const SceneGeo& g = P.geo[scene_of(P.fbase, P.n_scenes, i)];
    wall_project_box(g.wlo, g.whi, x, v);
  } else {
    wall_project(P, x, v);
  }
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
  uint32_t* key;      // block of each sorted particle (at the last sort)
  uint32_t* key_cur;  // current block of each particle on a substep that kept the sort
  int light_ok;       // a sort has ordered the arrays by key, so a substep may keep it
  int gmax_ok;        // ctl's FP32 maxima are those of the (corrected) state: the last
                      // force pass formed them and no key pass has cleared them since
  int64_t kept_sorts; // substeps that kept the last sort
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
  uint32_t* filled;               // list of filled blocks of the current pass (the sort's)
  uint32_t* filled_new;           // blocks filled since the sort (a pass that kept it)
  uint32_t* near_list;            // its particles with a norm near a level threshold
  uint32_t* act;      // active block list
  uint32_t* plist;    // evaluated particles (sorted-order indices), any order
  uint32_t* actflag;  // per block: stamp of the pass that listed it as active
  rts::Ctl* ctl;
  rts::Ctl* h_ctl;    // pinned host mirror

  // boundary, binned once
  float4* xb;
  uint32_t* bcstart;

  // staging for caller-order I/O
  float* io;          // n * 4 floats
  int32_t* io_i;      // n ints

  int grid_persistent;  // CTAs of the persistent neighbour kernels
  int pend_mode;        // PendMode of the deferred correction
  int64_t pend_k1;      // substep index the deferred correction completes
  uint32_t* nbl;        // neighbour lists of evaluated particles, nbl_cap per particle
  int nbl_cap;
  uint32_t* buid;       // boundary: caller index of each sorted boundary particle

  // PCISPH (Algorithms 2 and 3)
  float4* xs;           // predicted positions x*
  float* pbak;          // pressures before a run of local iterations
  uint8_t* in_se;       // particle in S_e
  uint8_t* in_re;       // block in R_e
  uint8_t* ob;          // block observed (R_ob)
  int32_t* preg;        // region of each block in the current major step (-1 = empty)
  int32_t* pnew;        // scratch region field (dilation, pre-emption)
  int minor, n_minor_cur, clean, shorten_now;
  int it_iters, it_global, it_local, it_reverts, it_notconv;
  double it_errmax, it_erravg;
  int64_t tot_iters, tot_local, tot_reverts, tot_steps;
  int last_global_level;

  // launch counting and optional per-phase event timing
  // batched scenes (null for a single scene)
  rts::BatchState* batch;

  int cur_phase;
  int64_t kernels;
  int64_t launches[RTS_NUM_PHASES];
  int prof;
  double prof_ms[RTS_NUM_PHASES];
  int64_t prof_timed[RTS_NUM_PHASES];
  int64_t prof_seen[RTS_NUM_PHASES];
  int64_t passes[RTS_NUM_PHASES];      // phase instances (always counted)
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

// Programmatic dependent launch.  A kernel launched with launch_pdl is scheduled as soon
// as every CTA of the kernel before it in the stream has exited, without waiting for that
// grid's completion to be signalled; its first statement is pdl_wait(), which returns
// once the previous kernel has completed and its writes are visible, so no memory access
// of the two overlaps.  Launched plainly, pdl_wait() is a no-op.  (Signalling dependents
// early, at the start of each CTA, was measured slower: the waiting CTAs of the next
// kernel crowd the tail of the current one.)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
template <typename... KArgs, typename... Args>
inline void launch_pdl(cudaStream_t st, void (*k)(KArgs...), int grid, int block, size_t smem,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, args...);   // a failure is left for cudaGetLastError
}
}  // namespace rts

// Host helpers implemented in rts_api.cu / kernels implemented in the .cu files.
namespace rts {
rts_status launch_bin(rts_ctx* c, float dt_predict);
rts_status launch_bin_light(rts_ctx* c, float dt_predict);
rts_status launch_bin_boundary(rts_ctx* c, const float4* xb_unsorted, int nb);
// stale: the substep kept the last sort (the light key pass's filled list, current blocks)
rts_status launch_classify(rts_ctx* c, bool stale);
rts_status launch_activity(rts_ctx* c, int mode, int level_g, int mult_g, int64_t k1,
                           bool stale);
void scan_block_counts(uint32_t* count, int nb, uint32_t* tile_sums, uint32_t* cstart,
                       cudaStream_t stream);
const char* validate_params(const rts_params* p, int32_t n, int32_t nb,
                            int max_dim = 4096);  // nullptr if valid
void make_dev_params(const rts_params& p, DevParams& d);
// Level of the global adaptive comparator from the FP32 maxima (as from the FP64 maxima);
// -1 when a maximum lies within 1e-5 of a threshold and the FP64 maxima must decide.
int pick_level_from_f32_max(const DevParams& d, float v2, float a2);
rts_status launch_density(rts_ctx* c, bool stale = false);
// gmode: 0; 1 the force pass also forms the maxima of the corrected state (global
// adaptive stepping, step ending at k1); 2 the same for a priming evaluation.
rts_status launch_force(rts_ctx* c, int gmode = 0, int64_t k1 = 0);
rts_status launch_correct(rts_ctx* c, int64_t k1, int prime);
rts_status finalize(rts_ctx* c);
rts_status launch_global_max(rts_ctx* c, int fp64);
rts_status launch_level_hist(rts_ctx* c);
const char* cuda_err(rts_ctx* c, cudaError_t e, const char* what);
rts_status pcisph_step(rts_ctx* c, int64_t max_mult);
// PCISPH minor step in three parts (shared by the single-scene and the batched step):
// major-step start when due, list refresh, non-pressure forces and the minor step's
// resets; then the density correction; then integration, validity and pre-emption.
void pcisph_minor_begin(rts_ctx* c);
rts_status pcisph_minor_end(rts_ctx* c, int j);
rts_status batch_step(rts_ctx* c);
void batch_free(rts_ctx* c);
void batch_delete(BatchState* b);   // a state not attached to a context
}  // namespace rts

// Batched scenes (rts_batch.cu): validation and layout, then the device tables.
const char* rts_batch_plan(const rts_params* params, int32_t n_scenes, const rts_scene* scenes,
                           rts_params* p2, int32_t* n_fluid, int32_t* n_boundary,
                           rts::BatchState** out);
rts_status rts_batch_attach(rts_ctx* c, rts::BatchState* b);
