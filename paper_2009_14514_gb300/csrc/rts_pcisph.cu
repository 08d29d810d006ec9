// rts_pcisph.cu - regional time stepping for PCISPH (Algorithms 2 and 3).
//
// A major step of n_minor minor steps of dt_b keeps the block grid (edge 2.2 s) built at
// its start (Section 5.6).  At the start: bin, regions from Eq. 2-3 (alpha = 1, no
// Eq. 1), R_min, expansion of R_1 and R_2 by expand_layers blocks (Section 5.5).  Each
// minor step refreshes the neighbour lists and non-pressure forces of the particles
// whose validity expired (1-ring search, 2 rings for R_1), then runs the density
// correction of Algorithm 3 with the per-region schedule, S_e and the observed blocks
// R_ob (Section 5.4), extra local / global iterations (Section 5.5), integrates every
// particle, and lowers the region of blocks around particles that need a smaller step.
//
// The correction loop is controlled from the host: after every iteration the maximum
// and the average relative error are read back (exact max, fixed-point sum) and the
// host decides the next iteration, as Algorithm 3 does.
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstring>

#include "rts_pcisph_dev.cuh"

namespace rts {

// ------------------------------------------------------------- regions ---

// Region of every block: a filled block's smoothed level (blevel carries this binning's
// stamp above the level for exactly the filled blocks), -1 for any other block.
__global__ void k_preg_from_blevel(DevParams P, const uint32_t* __restrict__ blevel,
                                   uint32_t stamp, int32_t* __restrict__ preg) {
  pdl_wait();
  const int64_t nb = (int64_t)P.nblocks;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb;
       b += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t v = blevel[b];
    preg[b] = (v >> 8) == stamp ? (int32_t)(v & 0xffu) : -1;
  }
}

// Section 5.5 expansion: a filled block within Chebyshev distance <= layers of a block
// of region <= target takes min(region, target) (Jacobi: reads in, writes out; filled
// blocks only).  The box is the product of three clipped intervals, so it is done as
// three separable passes: an x pass marks the blocks with a block of region <= target
// within `layers` along x (from the region field), a y pass widens the marks along y,
// and a pass over the filled blocks widens along z and applies the minimum; each block
// reads 2 layers + 1 values per pass instead of (2 layers + 1)^3.  The x pass also sets
// every block of the output field to -1 (the z pass writes the filled ones).
__global__ void k_dilate_x(DevParams P, const int32_t* __restrict__ in, int target, int layers,
                           uint8_t* __restrict__ mx, int32_t* __restrict__ out) {
  pdl_wait();
  const int64_t nb = (int64_t)P.nblocks;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int bx = (int)(b % P.nx);
    const int x0 = bx - layers < 0 ? 0 : bx - layers;
    const int x1 = bx + layers >= P.nx ? P.nx - 1 : bx + layers;
    const int32_t* row = in + (b - bx);
    uint8_t m = 0;
    for (int cx = x0; cx <= x1; ++cx) {
      const int Lc = row[cx];
      m |= (Lc >= 0 && Lc <= target) ? 1 : 0;
    }
    mx[b] = m;
    out[b] = -1;
  }
}

__global__ void k_dilate_y(DevParams P, const uint8_t* __restrict__ mx, int layers,
                           uint8_t* __restrict__ my) {
  pdl_wait();
  const int64_t nb = (int64_t)P.nblocks;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int by = (int)((b / P.nx) % P.ny);
    const int y0 = by - layers < 0 ? 0 : by - layers;
    const int y1 = by + layers >= P.ny ? P.ny - 1 : by + layers;
    const int64_t base = b - (int64_t)by * P.nx;
    uint8_t m = 0;
    for (int cy = y0; cy <= y1; ++cy) m |= mx[base + (int64_t)cy * P.nx];
    my[b] = m;
  }
}

__global__ void k_dilate_z(DevParams P, const uint32_t* __restrict__ filled, const Ctl* ctl,
                           const int32_t* __restrict__ in, const uint8_t* __restrict__ my,
                           int target, int layers, int32_t* __restrict__ out) {
  pdl_wait();
  const int nf = ctl->n_filled;
  const int64_t nxy = (int64_t)P.nx * P.ny;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nf; t += gridDim.x * blockDim.x) {
    const uint32_t b = filled[t];
    int L = in[b];
    if (L > target) {
      const int bz = (int)(b / nxy);
      const int z0 = bz - layers < 0 ? 0 : bz - layers;
      const int z1 = bz + layers >= P.nz ? P.nz - 1 : bz + layers;
      const int64_t base = (int64_t)b - (int64_t)bz * nxy;
      uint8_t m = 0;
      for (int cz = z0; cz <= z1; ++cz) m |= my[base + (int64_t)cz * nxy];
      if (m) L = target;
    }
    out[b] = L;
  }
}

// Every particle takes its block's region; neighbourhoods are refreshed at the start.
__global__ void k_assign_regions(DevParams P, int n, const uint32_t* __restrict__ key,
                                 const int32_t* __restrict__ preg, PState s,
                                 uint8_t* __restrict__ cflag) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int L = preg[key[i]];
  s.level[i] = L;
  s.valid[i] = P.refresh[L];
  cflag[i] = 1;
}

// R_ob (Section 5.4): filled blocks outside R_e bordering R_e or a smaller region.
__global__ void k_observed(DevParams P, const uint32_t* __restrict__ filled, const Ctl* ctl,
                           const int32_t* __restrict__ preg, const uint8_t* __restrict__ in_re,
                           uint8_t* __restrict__ ob) {
  pdl_wait();
  const int nf = ctl->n_filled;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nf; t += gridDim.x * blockDim.x) {
    uint32_t b = filled[t];
    ob[b] = observed_one(P, b, preg, in_re);
  }
}

// ---------------------------------------------------------- neighbours ---

// The neighbour predicate of the list refresh: FP32 outside the guard band, exact inside.
__device__ __forceinline__ bool list_test(const DevParams& P, float4 xi, float4 xj) {
  const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
  const float d2 = dx * dx + dy * dy + dz * dz;
  if (d2 < P.r2_lo) return true;
  return d2 < P.r2_hi && nbr_exact(P, xi, xj);
}

// Section 5.6: the neighbourhood of a refreshing particle is searched in the blocks
// around its block of the major-step start (2 rings for R_1; r2_rings for R_2, one
// unless the ablation asks for more) with current positions.
__global__ void k_lists(DevParams P, int n, const uint32_t* __restrict__ key,
                        const uint32_t* __restrict__ cstart, const uint32_t* __restrict__ bcstart,
                        PState s, const float4* __restrict__ xb, const uint8_t* __restrict__ cflag,
                        uint32_t* __restrict__ nbl, Ctl* ctl) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !cflag[i]) return;
  uint32_t b = key[i];
  int bx = b % P.nx, rr = b / P.nx, by = rr % P.ny, bz = rr / P.ny;
  int R = s.level[i] == 0 ? P.r1_rings : (s.level[i] == 1 ? P.r2_rings : 1);
  float4 xi = s.x[i];
  uint32_t* list = nbl + (size_t)i * P.nbl_cap;
  int cnt = 0;
  int x0 = bx - R < 0 ? 0 : bx - R;
  int x1 = bx + R >= P.nx ? P.nx - 1 : bx + R;
  for (int dz = -R; dz <= R; ++dz) {
    int cz = bz + dz;
    if (cz < 0 || cz >= P.nz) continue;
    for (int dy = -R; dy <= R; ++dy) {
      int cy = by + dy;
      if (cy < 0 || cy >= P.ny) continue;
      uint32_t rb = ((uint32_t)cz * P.ny + cy) * P.nx;
      for (int pass = 0; pass < 2; ++pass) {
        const uint32_t* cs = pass ? bcstart : cstart;
        const float4* src = pass ? xb : s.x;
        const uint32_t self = pass ? 0xffffffffu : (uint32_t)i;
        const uint32_t tag = pass ? kBnd : 0u;
        uint32_t j = cs[rb + x0];
        const uint32_t j1 = cs[rb + x1 + 1];
        // four candidate loads in flight, then the tests and appends in index order
        for (; j + 4 <= j1; j += 4) {
          float4 xq[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) xq[q] = __ldg(&src[j + q]);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (j + q != self && list_test(P, xi, xq[q])) {
              if (cnt < P.nbl_cap) list[cnt] = (j + q) | tag;
              ++cnt;
            }
          }
        }
        for (; j < j1; ++j) {
          if (j != self && list_test(P, xi, __ldg(&src[j]))) {
            if (cnt < P.nbl_cap) list[cnt] = j | tag;
            ++cnt;
          }
        }
      }
    }
  }
  if (cnt > P.nbl_cap) {
    set_status(ctl, RTS_ERR_CAPACITY);
    cnt = P.nbl_cap;
  }
  s.nbr[i] = cnt;
}

// Non-pressure acceleration of refreshing particles: gravity + artificial viscosity
// (nu = alpha h c / rho0) over the neighbourhood; boundary particles are at rest.  The
// minor step's resets ride along: pressure, pressure acceleration and S_e of every
// particle, and the R_e flags of the nbk blocks, are zeroed (none is read here).
template <int LANES>
__global__ void k_nonpressure(DevParams P, int n, PState s, const float4* __restrict__ xb,
                              const uint8_t* __restrict__ cflag, const uint32_t* __restrict__ nbl,
                              uint8_t* __restrict__ in_se, uint8_t* __restrict__ in_re,
                              size_t nbk) {
  pdl_wait();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;   // LANES lanes per particle
  const int i = t / LANES, sub = t % LANES;
  for (size_t b = (size_t)t; b < nbk; b += (size_t)gridDim.x * blockDim.x) in_re[b] = 0;
  if (i < n && sub == 0) {
    s.prs[i] = 0.f;
    s.ap[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    in_se[i] = 0;
  }
  const bool valid = i < n && cflag[i];
  float ax = 0.f, ay = 0.f, az = 0.f;
  if (valid) {
    const float4 xi = s.x[i], vi = s.v[i];
    const uint32_t* list = nbl + (size_t)i * P.nbl_cap;
    const int cnt = s.nbr[i];
    for (int e = sub; e < cnt; e += LANES) {
      const uint32_t j = list[e];
      float4 xj, vj = make_float4(0.f, 0.f, 0.f, 0.f);
      if (j & kBnd) {
        xj = xb[j & ~kBnd];
      } else {
        xj = s.x[j];
        vj = s.v[j];
      }
      const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
      const float d2 = dx * dx + dy * dy + dz * dz;
      if (!(d2 > 0.f)) continue;
      const float vx = (vi.x - vj.x) * dx + (vi.y - vj.y) * dy + (vi.z - vj.z) * dz;
      if (vx >= 0.f) continue;
      const float id = inv_len(d2);
      const float Pi = -P.visc_nu * __fdividef(vx, d2 + P.eps_h2);
      const float f = pdW(P, d2 * id * P.inv_h) * id;
      const float sc = -P.m * Pi * f;
      ax += sc * dx;
      ay += sc * dy;
      az += sc * dz;
    }
  }
  ax = group_sum<LANES>(ax);
  ay = group_sum<LANES>(ay);
  az = group_sum<LANES>(az);
  if (valid && sub == 0) s.a[i] = make_float4(P.gx + ax, P.gy + ay, P.gz + az, 0.f);
}

// ------------------------------------------------------- Algorithm 3 ---

// Predict v* = v + dt (a_np + a_p), x* = x + dt v*; the iteration's error reductions and
// R_e flags (nbk blocks) start from zero (the previous ones were read before).  With
// prev_mode < 0 every particle is predicted; otherwise only those whose pressure
// acceleration the previous iteration (prev_mode, prev_row of minor step j) updated —
// a turn or S_e — since x* of every other particle is unchanged (its w lane, p / rho^2,
// is refreshed by the density pass that changes its pressure).
__global__ void k_predict(DevParams P, int n, PState s, float4* __restrict__ xs, Ctl* ctl,
                          uint8_t* __restrict__ in_re, size_t nbk, int j, int prev_mode,
                          int prev_row, const uint8_t* __restrict__ in_se) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    ctl->err_max_bits = 0u;
    ctl->err_sum_fx = 0ull;
  }
  for (size_t b = (size_t)i; b < nbk; b += (size_t)gridDim.x * blockDim.x) in_re[b] = 0;
  if (i >= n) return;
  if (prev_mode >= 0 && !has_turn(P, prev_mode, prev_row, j, s.level[i]) && !in_se[i]) return;
  xs[i] = predict_one(P, s, i);
}

// Predicted density, relative error and pressure of the participants (turn, S_e, S_ob).
template <int LANES>
__global__ void k_pdensity(DevParams P, int n, int j_minor, int row, int mode,
                           const uint32_t* __restrict__ key, PState s,
                           const uint8_t* __restrict__ in_se, const uint8_t* __restrict__ ob,
                           float4* xs, const float4* __restrict__ xb,
                           const uint32_t* __restrict__ nbl) {
  pdl_wait();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;   // LANES lanes per particle
  const int i = t / LANES, sub = t % LANES;
  const bool valid =
      i < n && (has_turn(P, mode, row, j_minor, s.level[i]) || in_se[i] || ob[key[i]]);
  pdensity_group<LANES>(P, s, i, valid, sub, xs, xb, nbl);
}

// S_e = {err > eta / 2}; R_e = blocks holding an S_e particle; max and sum of the latest
// errors of all particles (exact max on FP32 bits, fixed-point sum).
__global__ void k_se_reduce(DevParams P, int n, const uint32_t* __restrict__ key, PState s,
                            uint8_t* __restrict__ in_se, uint8_t* __restrict__ in_re, Ctl* ctl) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  float e = 0.f;
  if (i < n) {
    e = s.err[i];
    bool se = e > 0.5f * P.eta;
    in_se[i] = se ? 1 : 0;
    if (se) in_re[key[i]] = 1;
  }
  unsigned mx = __float_as_uint(e);
  unsigned long long fx = err_fixed(e);
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    mx = max(mx, __shfl_down_sync(kFullMask, mx, o));
    fx += __shfl_down_sync(kFullMask, fx, o);
  }
  // one atomic per counter and CTA (256 threads): the counters are shared by every CTA
  __shared__ unsigned smx[8];
  __shared__ unsigned long long sfx[8];
  if ((threadIdx.x & 31) == 0) {
    smx[threadIdx.x >> 5] = mx;
    sfx[threadIdx.x >> 5] = fx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
      mx = max(mx, smx[k]);
      fx += sfx[k];
    }
    if (mx) atomicMax(&ctl->err_max_bits, mx);
    if (fx) atomicAdd(&ctl->err_sum_fx, fx);
  }
}

// Pressure acceleration of turn and S_e.
template <int LANES>
__global__ void k_ppressure(DevParams P, int n, int j_minor, int row, int mode, PState s,
                            const uint8_t* __restrict__ in_se, const float4* __restrict__ xs,
                            const float4* __restrict__ xb, const uint32_t* __restrict__ nbl) {
  pdl_wait();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;   // LANES lanes per particle
  const int i = t / LANES, sub = t % LANES;
  const bool valid = i < n && (has_turn(P, mode, row, j_minor, s.level[i]) || in_se[i]);
  ppressure_group<LANES>(P, s, i, valid, sub, xs, xb, nbl);
}

// ------------------------------------------------------- Algorithm 2 ---

__global__ void k_integrate(DevParams P, int n, PState s) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 x = s.x[i], v = s.v[i], a = s.a[i], pa = s.ap[i];
  float dt = P.dt_b;
  v.x += dt * (a.x + pa.x);
  v.y += dt * (a.y + pa.y);
  v.z += dt * (a.z + pa.z);
  x.x += dt * v.x;
  x.y += dt * v.y;
  x.z += dt * v.z;
  if (P.wall_project) wall_project_at(P, (uint32_t)i, x, v);
  s.x[i] = x;
  s.v[i] = v;
}

// Validity countdown (Algorithm 2); with rdst set, the nb block regions are copied from
// rsrc to rdst as well (the pre-emption pass that follows marks the copy).
__global__ void k_validity(DevParams P, int n, PState s, uint8_t* __restrict__ cflag,
                           const int32_t* __restrict__ rsrc, int32_t* __restrict__ rdst,
                           size_t nb) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (rdst)
    for (size_t b = (size_t)i; b < nb; b += (size_t)gridDim.x * blockDim.x) rdst[b] = rsrc[b];
  if (i >= n) return;
  int val = s.valid[i] - 1;
  if (val <= 0) {
    cflag[i] = 1;
    val = P.refresh[s.level[i]];
  } else {
    cflag[i] = 0;
  }
  s.valid[i] = val;
}

__device__ __forceinline__ int ppick(const DevParams& P, double v2, double a2) {
  int L = 0;
  for (int l = 0; l < P.n_levels; ++l)
    if (P.eq1[l] && v2 <= P.vthr2[l] && a2 <= P.athr2[l]) L = l;
  return L;
}

// The region Eq. 2-3 give a particle (as ppick on the FP64 norms): decided in FP32 where
// the FP32 squared norms are farther than 1e-5 relative from every finite threshold
// (their error is below 3e-7 relative), by the FP64 norms otherwise.
__device__ __forceinline__ int ppick_particle(const DevParams& P, float4 v, float4 a, float4 pa) {
  const float ax = a.x + pa.x, ay = a.y + pa.y, az = a.z + pa.z;
  const float v2 = __fadd_rn(__fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y)), __fmul_rn(v.z, v.z));
  const float a2 = __fadd_rn(__fadd_rn(__fmul_rn(ax, ax), __fmul_rn(ay, ay)), __fmul_rn(az, az));
  bool undecided = false;
  int L = 0;
  for (int l = 0; l < P.n_levels; ++l) {
    const float tv = P.vthr2f[l], ta = P.athr2f[l];
    if (isfinite(tv) && fabsf(v2 - tv) <= 1e-5f * tv) undecided = true;
    if (isfinite(ta) && fabsf(a2 - ta) <= 1e-5f * ta) undecided = true;
    if (P.eq1[l] && v2 <= tv && a2 <= ta) L = l;
  }
  if (undecided) L = ppick(P, pnorm2(v.x, v.y, v.z), pnorm2(ax, ay, az));
  return L;
}

// Section 5.6: a particle needing a smaller region lowers its block and the 26 around.
__global__ void k_preempt_mark(DevParams P, int n, const uint32_t* __restrict__ key, PState s,
                               int32_t* __restrict__ pnew) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int L = ppick_particle(P, s.v[i], s.a[i], s.ap[i]);
  if (P.force_level >= 0) L = P.force_level;
  if (L >= s.level[i]) return;
  uint32_t b = key[i];
  int bx = b % P.nx, r = b / P.nx, by = r % P.ny, bz = r / P.ny;
  for (int dz = -1; dz <= 1; ++dz) {
    int cz = bz + dz;
    if (cz < 0 || cz >= P.nz) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      int cy = by + dy;
      if (cy < 0 || cy >= P.ny) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        int cx = bx + dx;
        if (cx < 0 || cx >= P.nx) continue;
        size_t c = ((size_t)cz * P.ny + cy) * P.nx + cx;
        if (pnew[c] >= 0) atomicMin(&pnew[c], L);
      }
    }
  }
}

__global__ void k_preempt_apply(DevParams P, int n, const uint32_t* __restrict__ key,
                                const int32_t* __restrict__ pnew, PState s,
                                uint8_t* __restrict__ cflag) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int L = pnew[key[i]];
  if (L < s.level[i]) {
    s.level[i] = L;
    s.valid[i] = P.refresh[L];
    cflag[i] = 1;
  }
}

// ------------------------------------------------------------- host ---

static inline int grid_of(int n) { return (n + 255) / 256; }
// CTAs of 256 threads for `lanes` lanes per particle
static inline int grid_lanes(int n, int lanes) {
  return (int)(((int64_t)(n > 0 ? n : 1) * lanes + 255) / 256);
}

int filled_grid_size();

// Scope that counts launches against a phase (no event timing for PCISPH phases).
struct PPhase {
  rts_ctx* c;
  int prev;
  PPhase(rts_ctx* c_, int ph) : c(c_), prev(c_->cur_phase) { c->cur_phase = ph; }
  ~PPhase() { c->cur_phase = prev; }
};

static rts_status major_start(rts_ctx* c) {
  int n = c->n;
  size_t nbk = (size_t)c->dp.nblocks;
  {
    PPhase ph(c, RTS_PHASE_BIN);
    launch_bin(c, 0.0f);
  }
  PPhase ph(c, RTS_PHASE_CLASSIFY);
  launch_classify(c, false);      // Eq. 2-3 from the block maxima (thresholds for PCISPH)
  launch_activity(c, -1, 0, 0, 0, false);   // R_min (or the forced region)
  int fg = filled_grid_size();
  const int gg = (int)((nbk + 255) / 256 < (size_t)(fg * 4) ? (nbk + 255) / 256 : (size_t)(fg * 4));
  note_launch(c, 1);
  launch_pdl(c->stream, k_preg_from_blevel, gg, 256, 0, c->dp, c->blevel, c->stamp, c->preg);
  if (c->p.force_level < 0 && c->p.expand_layers > 0) {
    // R_e and R_ob are rebuilt at the next minor step: their bytes hold the marks here
    for (int target = 0; target <= 1; ++target) {
      note_launch(c, 3);
      launch_pdl(c->stream, k_dilate_x, gg, 256, 0, c->dp, c->preg, target, c->p.expand_layers,
                 c->in_re, c->pnew);
      launch_pdl(c->stream, k_dilate_y, gg, 256, 0, c->dp, c->in_re, c->p.expand_layers, c->ob);
      launch_pdl(c->stream, k_dilate_z, fg, 256, 0, c->dp, c->filled, c->ctl, c->preg, c->ob,
                 target, c->p.expand_layers, c->pnew);
      int32_t* t = c->preg;
      c->preg = c->pnew;
      c->pnew = t;
    }
  }
  if (n > 0) {
    note_launch(c, 1);
    launch_pdl(c->stream, k_assign_regions, grid_of(n), 256, 0, c->dp, n, c->key, c->preg, c->s,
               c->cflag);
  }
  c->shorten_now = 0;
  return RTS_OK;
}

// Algorithm 3 for minor step j with parameters Q.  plain: every particle in every
// iteration and only global extra iterations (the comparators' plain PCISPH).
static rts_status run_correction(rts_ctx* c, const DevParams& Q, int j, bool plain) {
  const int n = c->n;
  const int g = grid_of(n > 0 ? n : 1);
  const int fg = filled_grid_size();
  const size_t nbk = (size_t)c->dp.nblocks;
  int min_sched = 1 << 30;
  for (int r = 0; r < c->p.n_levels && r < 4; ++r)
    if (c->p.sched[r][j] < min_sched) min_sched = c->p.sched[r][j];
  int min_iter = 3, done = 0, row = 1, mode = kModeSched, local_run = 0, stay_global = 0;
  int prev_mode = -1, prev_row = 0;   // the last iteration's pressure participants (-1: all)
  rts_status status = RTS_OK;
  if (plain) {
    mode = kModeGlobal;
    stay_global = 1;
  }
  c->it_global = c->it_local = c->it_reverts = c->it_notconv = 0;
  for (;;) {
    const int all_turn = mode == kModeGlobal || (mode == kModeSched && row <= min_sched);
    {
      PPhase ph(c, RTS_PHASE_ITERATE);
      note_launch(c, all_turn ? 4 : 5);
      // one chain of programmatically dependent launches (see launch_pdl)
      cudaStream_t st = c->stream;
      // R_ob matters only to an iteration in which not every particle takes part: it is
      // formed here, before the predict pass clears R_e, from the R_e of the previous
      // iteration (cleared at the start of the minor step) and the regions
      if (!all_turn)
        launch_pdl(st, k_observed, fg, 256, 0, Q, c->filled, c->ctl, c->preg, c->in_re, c->ob);
      launch_pdl(st, k_predict, g, 256, 0, Q, n, c->s, c->xs, c->ctl, c->in_re, nbk, j, prev_mode,
                 prev_row, c->in_se);
      // every particle takes part (all_turn): kPLanes lanes each; else one
      if (all_turn)
        launch_pdl(st, k_pdensity<kPLanes>, grid_lanes(n, kPLanes), 256, 0, Q, n, j, row, mode,
                   c->key, c->s, c->in_se, c->ob, c->xs, c->xb, c->nbl);
      else
        launch_pdl(st, k_pdensity<1>, grid_lanes(n, 1), 256, 0, Q, n, j, row, mode, c->key, c->s,
                   c->in_se, c->ob, c->xs, c->xb, c->nbl);
      launch_pdl(st, k_se_reduce, g, 256, 0, Q, n, c->key, c->s, c->in_se, c->in_re, c->ctl);
      if (all_turn)
        launch_pdl(st, k_ppressure<kPLanes>, grid_lanes(n, kPLanes), 256, 0, Q, n, j, row, mode,
                   c->s, c->in_se, c->xs, c->xb, c->nbl);
      else
        launch_pdl(st, k_ppressure<1>, grid_lanes(n, 1), 256, 0, Q, n, j, row, mode, c->s,
                   c->in_se, c->xs, c->xb, c->nbl);
      prev_mode = mode;
      prev_row = row;
    }
    ++done;
    if (all_turn) ++c->it_global;
    if (mode == kModeLocal) ++c->it_local;
    // At least three iterations run, so the first two decide nothing: their reductions
    // are not read, and the next iteration is queued without a round trip to the host.
    if (done < 3 && done < c->p.max_iters) {
      ++row;
      continue;
    }
    // both reductions in one copy (err_max_bits and err_sum_fx are adjacent in Ctl)
    constexpr size_t kErrBytes =
        offsetof(Ctl, err_sum_fx) + sizeof(unsigned long long) - offsetof(Ctl, err_max_bits);
    cudaMemcpyAsync(&c->h_ctl->err_max_bits, &c->ctl->err_max_bits, kErrBytes,
                    cudaMemcpyDeviceToHost, c->stream);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      cuda_err(c, e, "PCISPH iteration");
      return RTS_ERR_CUDA;
    }
    float emax;
    unsigned bits = c->h_ctl->err_max_bits;
    memcpy(&emax, &bits, sizeof emax);
    c->it_errmax = emax;
    c->it_erravg = n > 0 ? (double)c->h_ctl->err_sum_fx / 4294967296.0 / n : 0.0;
    const bool converged = emax <= c->p.eta;
    if (done >= min_iter && converged) break;
    if (done >= c->p.max_iters) {
      status = RTS_ERR_NOT_CONVERGED;
      c->it_notconv = 1;
      break;
    }
    min_iter = done + 1;
    if (stay_global || c->it_erravg >= (double)c->p.eta_T) {
      mode = kModeGlobal;
      local_run = 0;
    } else {
      if (mode != kModeLocal) {
        cudaMemcpyAsync(c->pbak, c->s.prs, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice,
                        c->stream);
        local_run = 0;
      }
      mode = kModeLocal;
      if (++local_run > c->p.max_local_iters) {
        cudaMemcpyAsync(c->s.prs, c->pbak, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice,
                        c->stream);
        prev_mode = -1;   // every pressure changed: every x* (its w lane) is predicted anew
        ++c->it_reverts;
        mode = kModeGlobal;
        stay_global = 1;
        local_run = 0;
      }
    }
  }
  c->it_iters = done;
  c->tot_iters += done;
  c->tot_local += c->it_local;
  c->tot_reverts += c->it_reverts;
  c->tot_steps += 1;
  return status;
}

// Maxima of |v|^2 and |a_np + a_p|^2 over the fluid, order independent: of the FP32
// norms (fp64 = 0, maximum on FP32 bits) or of the FP64 norms (fp64 = 1, asked for only
// when the FP32 maxima lie at a threshold).
__global__ void k_pglobal_max(int n, PState s, Ctl* ctl, int fp64) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  __shared__ double svm[8], sam[8];   // one atomic per counter and CTA (256 threads)
  __shared__ unsigned svf[8], saf[8];
  if (!fp64) {
    unsigned vm = 0, am = 0;
    if (i < n) {
      const float4 v = s.v[i], a = s.a[i], pa = s.ap[i];
      const float ax = a.x + pa.x, ay = a.y + pa.y, az = a.z + pa.z;
      vm = __float_as_uint(__fadd_rn(__fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y)), __fmul_rn(v.z, v.z)));
      am = __float_as_uint(__fadd_rn(__fadd_rn(__fmul_rn(ax, ax), __fmul_rn(ay, ay)), __fmul_rn(az, az)));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      vm = max(vm, __shfl_down_sync(kFullMask, vm, o));
      am = max(am, __shfl_down_sync(kFullMask, am, o));
    }
    if ((threadIdx.x & 31) == 0) {
      svf[threadIdx.x >> 5] = vm;
      saf[threadIdx.x >> 5] = am;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
        vm = max(vm, svf[k]);
        am = max(am, saf[k]);
      }
      atomicMax(&ctl->vmax2f_bits, vm);
      atomicMax(&ctl->amax2f_bits, am);
    }
    return;
  }
  double vm = 0.0, am = 0.0;
  if (i < n) {
    float4 v = s.v[i], a = s.a[i], pa = s.ap[i];
    vm = pnorm2(v.x, v.y, v.z);
    am = pnorm2(a.x + pa.x, a.y + pa.y, a.z + pa.z);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    vm = fmax(vm, __shfl_down_sync(kFullMask, vm, o));
    am = fmax(am, __shfl_down_sync(kFullMask, am, o));
  }
  if ((threadIdx.x & 31) == 0) {
    svm[threadIdx.x >> 5] = vm;
    sam[threadIdx.x >> 5] = am;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
      vm = fmax(vm, svm[k]);
      am = fmax(am, sam[k]);
    }
    atomicMax(&ctl->vmax2_bits, (unsigned long long)__double_as_longlong(vm));
    atomicMax(&ctl->amax2_bits, (unsigned long long)__double_as_longlong(am));
  }
}

__global__ void k_all_region(int n, int L, PState s, uint8_t* __restrict__ cflag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  s.level[i] = L;
  s.valid[i] = 1;
  cflag[i] = 1;
}

// Global comparators (Section 6): plain PCISPH with one step of m dt_b for every particle,
// m from the finest region the criteria give for the whole fluid (global adaptive) or 1
// (constant); fresh grid and neighbourhoods every step, delta scaled by 1 / m^2.
static rts_status pcisph_global(rts_ctx* c, int64_t max_mult) {
  const int n = c->n;
  const int g = grid_of(n > 0 ? n : 1);
  int L = 0;
  if (c->p.mode == RTS_MODE_GLOBAL_ADAPTIVE && n > 0) {
    cudaMemsetAsync(&c->ctl->vmax2f_bits, 0, 2 * sizeof(unsigned int), c->stream);
    {
      PPhase ph(c, RTS_PHASE_CLASSIFY);
      note_launch(c, 1);
      k_pglobal_max<<<g, 256, 0, c->stream>>>(n, c->s, c->ctl, 0);
    }
    cudaMemcpyAsync(&c->h_ctl->vmax2f_bits, &c->ctl->vmax2f_bits, 2 * sizeof(unsigned int),
                    cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return RTS_ERR_CUDA;
    float v2f, a2f;
    memcpy(&v2f, &c->h_ctl->vmax2f_bits, sizeof v2f);
    memcpy(&a2f, &c->h_ctl->amax2f_bits, sizeof a2f);
    L = pick_level_from_f32_max(c->dp, v2f, a2f);
    if (L < 0) {   // a maximum at a threshold: the FP64 maxima decide
      L = 0;
      cudaMemsetAsync(&c->ctl->vmax2_bits, 0, 2 * sizeof(unsigned long long), c->stream);
      {
        PPhase ph(c, RTS_PHASE_CLASSIFY);
        note_launch(c, 1);
        k_pglobal_max<<<g, 256, 0, c->stream>>>(n, c->s, c->ctl, 1);
      }
      cudaMemcpyAsync(&c->h_ctl->vmax2_bits, &c->ctl->vmax2_bits, 2 * sizeof(unsigned long long),
                      cudaMemcpyDeviceToHost, c->stream);
      if (cudaStreamSynchronize(c->stream) != cudaSuccess) return RTS_ERR_CUDA;
      double v2, a2;
      memcpy(&v2, &c->h_ctl->vmax2_bits, sizeof v2);
      memcpy(&a2, &c->h_ctl->amax2_bits, sizeof a2);
      for (int l = 0; l < c->dp.n_levels; ++l)
        if (c->dp.eq1[l] && v2 <= c->dp.vthr2[l] && a2 <= c->dp.athr2[l]) L = l;
    }
  }
  int64_t m = c->p.level_mult[L];
  if (m > max_mult) m = max_mult;
  if (m < 1) m = 1;
  DevParams Q = c->dp;
  Q.dt_b = (float)((double)m * (double)c->p.dt_b);
  Q.delta = (float)((double)c->dp.delta / (double)(m * m));
  Q.r1_rings = 1;
  Q.r2_rings = 1;
  {
    PPhase ph(c, RTS_PHASE_BIN);
    launch_bin(c, 0.0f);
  }
  if (n > 0) {
    note_launch(c, 3);
    k_all_region<<<g, 256, 0, c->stream>>>(n, 0, c->s, c->cflag);
    {
      PPhase ph(c, RTS_PHASE_DENSITY);
      k_lists<<<g, 256, 0, c->stream>>>(Q, n, c->key, c->cstart, c->bcstart, c->s, c->xb, c->cflag,
                                        c->nbl, c->ctl);
    }
    {
      PPhase ph(c, RTS_PHASE_FORCE);
      k_nonpressure<kPLanes><<<grid_lanes(n, kPLanes), 256, 0, c->stream>>>(
          Q, n, c->s, c->xb, c->cflag, c->nbl, c->in_se, c->in_re, (size_t)0);
    }
  }
  const size_t n1 = (size_t)(n > 0 ? n : 1);
  cudaMemsetAsync(c->ob, 0, (size_t)c->dp.nblocks, c->stream);
  // the sort's spare buffers keep the step's start state for a rejected step
  if (c->p.mode == RTS_MODE_GLOBAL_ADAPTIVE && m > 1) {
    cudaMemcpyAsync(c->s2.x, c->s.x, sizeof(float4) * n1, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(c->s2.v, c->s.v, sizeof(float4) * n1, cudaMemcpyDeviceToDevice, c->stream);
  }
  rts_status status;
  for (;;) {
    cudaMemsetAsync(c->s.prs, 0, sizeof(float) * n1, c->stream);
    cudaMemsetAsync(c->s.ap, 0, sizeof(float4) * n1, c->stream);
    cudaMemsetAsync(c->in_se, 0, n1, c->stream);
    status = run_correction(c, Q, 0, true);
    if (status != RTS_OK && status != RTS_ERR_NOT_CONVERGED) return status;
    // density-error feedback: a step that does not converge is retried with m / 2
    if (status != RTS_ERR_NOT_CONVERGED || m == 1 || c->p.mode != RTS_MODE_GLOBAL_ADAPTIVE) break;
    m = m / 2 > 1 ? m / 2 : 1;
    Q.dt_b = (float)((double)m * (double)c->p.dt_b);
    Q.delta = (float)((double)c->dp.delta / (double)(m * m));
    cudaMemcpyAsync(c->s.x, c->s2.x, sizeof(float4) * n1, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(c->s.v, c->s2.v, sizeof(float4) * n1, cudaMemcpyDeviceToDevice, c->stream);
  }
  if (n > 0) {
    PPhase ph(c, RTS_PHASE_CORRECT);
    note_launch(c, 2);
    k_integrate<<<g, 256, 0, c->stream>>>(Q, n, c->s);
    k_all_region<<<g, 256, 0, c->stream>>>(n, L, c->s, c->cflag);
  }
  c->k += m;
  c->minor = 0;
  return status;
}

// Major-step start when due, neighbourhood refresh and non-pressure forces of the
// refreshing particles, and the resets of the minor step (pressures, S_e, R_e, R_ob).
void pcisph_minor_begin(rts_ctx* c) {
  const int n = c->n;
  const int g = grid_of(n > 0 ? n : 1);
  const size_t nbk = (size_t)c->dp.nblocks;
  if (c->n_minor_cur <= 0) c->n_minor_cur = c->p.n_minor;
  if (c->minor == 0) major_start(c);
  if (n > 0) {
    PPhase ph(c, RTS_PHASE_DENSITY);
    note_launch(c, 1);
    // At a major-step start the grid was just built from these positions: every particle
    // within r of another lies in the 27 blocks around its block (edge >= r), so one ring
    // gives the same list, in the same order, as the wider search of R_1 (and R_2).
    DevParams Q = c->dp;
    if (c->minor == 0) Q.r1_rings = Q.r2_rings = 1;
    launch_pdl(c->stream, k_lists, g, 256, 0, Q, n, c->key, c->cstart, c->bcstart, c->s, c->xb,
               c->cflag, c->nbl, c->ctl);
  }
  if (n > 0) {
    PPhase ph(c, RTS_PHASE_FORCE);
    note_launch(c, 1);
    // at a major-step start every particle refreshes: kPLanes lanes each; later few
    if (c->minor == 0)
      launch_pdl(c->stream, k_nonpressure<kPLanes>, grid_lanes(n, kPLanes), 256, 0, c->dp, n, c->s,
                 c->xb, c->cflag, c->nbl, c->in_se, c->in_re, nbk);
    else
      launch_pdl(c->stream, k_nonpressure<1>, grid_lanes(n, 1), 256, 0, c->dp, n, c->s, c->xb,
                 c->cflag, c->nbl, c->in_se, c->in_re, nbk);
  } else {
    cudaMemsetAsync(c->in_re, 0, nbk, c->stream);
  }
  // R_ob is formed in the density correction, before an iteration that reads it
}

// Integration, validity, pre-emption and the major-step bookkeeping after the density
// correction of minor step j (c->shorten_now set by the correction).
rts_status pcisph_minor_end(rts_ctx* c, int j) {
  const int n = c->n;
  const int g = grid_of(n > 0 ? n : 1);
  const size_t nbk = (size_t)c->dp.nblocks;
  PPhase ph(c, RTS_PHASE_CORRECT);
  note_launch(c, 2);
  k_integrate<<<g, 256, 0, c->stream>>>(c->dp, n, c->s);
  const int last = (j + 1 >= c->n_minor_cur) || c->shorten_now;
  // pre-emption follows unless the major step ends: the validity pass copies the regions
  const bool pre = !last && n > 0;
  launch_pdl(c->stream, k_validity, g, 256, 0, c->dp, n, c->s, c->cflag,
             pre ? c->preg : nullptr, pre ? c->pnew : nullptr, pre ? nbk : (size_t)0);
  if (pre) {
    note_launch(c, 2);
    launch_pdl(c->stream, k_preempt_mark, g, 256, 0, c->dp, n, c->key, c->s, c->pnew);
    launch_pdl(c->stream, k_preempt_apply, g, 256, 0, c->dp, n, c->key, c->pnew, c->s, c->cflag);
    int32_t* t = c->preg;
    c->preg = c->pnew;
    c->pnew = t;
  }
  c->k += 1;
  if (last) {
    if (c->shorten_now) {
      c->n_minor_cur = c->p.short_minor;
      c->clean = 0;
    } else if (c->n_minor_cur != c->p.n_minor) {
      if (++c->clean >= c->p.clean_majors) {
        c->n_minor_cur = c->p.n_minor;
        c->clean = 0;
      }
    }
    c->minor = 0;
  } else {
    c->minor = j + 1;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    cuda_err(c, e, "PCISPH step");
    return RTS_ERR_CUDA;
  }
  return RTS_OK;
}

rts_status pcisph_step(rts_ctx* c, int64_t max_mult) {
  if (c->p.mode != RTS_MODE_REGIONAL) return pcisph_global(c, max_mult);
  if (c->batch) return batch_step(c);
  pcisph_minor_begin(c);
  const int j = c->minor;
  rts_status status = run_correction(c, c->dp, j, false);
  if (status != RTS_OK && status != RTS_ERR_NOT_CONVERGED) return status;
  if (c->it_global > c->p.max_global_iters) c->shorten_now = 1;
  rts_status st = pcisph_minor_end(c, j);
  return st != RTS_OK ? st : status;
}

}  // namespace rts
