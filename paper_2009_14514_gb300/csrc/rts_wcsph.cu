// rts_wcsph.cu - region determination and the WCSPH neighbour passes.
//
// Classification (Section 3.1, Eq. 1-3; R_min of Section 4.2) runs one thread per
// block over the block-sorted particles.  The activity pass (Algorithm 1: validity,
// pre-emption on a level change) compacts the blocks holding an evaluated particle
// into a work list.  The neighbour passes are persistent: one warp per active block,
// its lanes split over the block's evaluated particles, every lane walking the 9
// contiguous candidate rows (x-neighbouring blocks are adjacent in block order) of
// the fluid and of the static boundary.  Inactive neighbours are read at their
// predicted state, which the key pass wrote (the "ghost at interpolated state").
#include <cuda_runtime.h>

#include "rts_internal.cuh"

namespace rts {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double norm2d(float x, float y, float z) {
  double dx = x, dy = y, dz = z;
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Section 3.1: the largest level whose criteria hold; level 0 if none does.
__device__ __forceinline__ int pick_level(const DevParams& P, double v2, double a2) {
  int L = 0;
  for (int l = 0; l < P.n_levels; ++l)
    if (P.eq1[l] && v2 <= P.vthr2[l] && a2 <= P.athr2[l]) L = l;
  return L;
}

// Raw block level from the block maxima of |v|^2 and |a|^2 (FP64, order independent).
__global__ void k_block_raw(DevParams P, const uint32_t* __restrict__ cstart,
                            const float4* __restrict__ v, const float4* __restrict__ a,
                            int8_t* __restrict__ raw) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= P.nblocks) return;
  uint32_t beg = cstart[b], end = cstart[b + 1];
  if (beg == end) {
    raw[b] = -1;
    return;
  }
  double vm = 0.0, am = 0.0;
  for (uint32_t i = beg; i < end; ++i) {
    float4 vi = v[i], ai = a[i];
    vm = fmax(vm, norm2d(vi.x, vi.y, vi.z));
    am = fmax(am, norm2d(ai.x, ai.y, ai.z));
  }
  raw[b] = (int8_t)pick_level(P, vm, am);
}

// R_min (Section 4.2): a filled block takes the smallest level among itself and its
// filled 26 neighbours (Jacobi: reads raw, writes lev), or the forced level.
__global__ void k_block_smooth(DevParams P, const int8_t* __restrict__ raw, int8_t* __restrict__ lev) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= P.nblocks) return;
  int L = raw[b];
  if (L < 0) {
    lev[b] = -1;
    return;
  }
  if (P.force_level >= 0) {
    lev[b] = (int8_t)P.force_level;
    return;
  }
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
        int Lc = raw[(cz * P.ny + cy) * P.nx + cx];
        if (Lc >= 0 && Lc < L) L = Lc;
      }
    }
  }
  lev[b] = (int8_t)L;
}

// Algorithm 1 region bookkeeping per particle; blocks with an evaluated particle are
// appended to the work list (warp-aggregated).
__global__ void k_activity(DevParams P, int mode, int level_g, int mult_g,
                           const uint32_t* __restrict__ cstart, const int8_t* __restrict__ lev,
                           PState s, uint8_t* __restrict__ cflag, uint32_t* __restrict__ act,
                           Ctl* ctl) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  int ncomp = 0;
  if (b < P.nblocks) {
    uint32_t beg = cstart[b], end = cstart[b + 1];
    if (beg != end) {
      int Lb = mode == kActGlobal ? level_g : (int)lev[b];
      int mb = mode == kActGlobal ? mult_g : P.mult[Lb];
      for (uint32_t i = beg; i < end; ++i) {
        int c;
        if (mode == kActRegional) {
          int val = s.valid[i] - 1;
          int li = s.level[i];
          if (val <= 0 || li < 0 || P.mult[li] != mb) {
            c = 1;
            s.level[i] = Lb;
            val = mb;
          } else {
            c = 0;
          }
          s.valid[i] = val;
        } else {
          c = 1;
          s.level[i] = Lb;
          s.valid[i] = mb;
        }
        cflag[i] = (uint8_t)c;
        ncomp += c;
      }
    }
  }
  unsigned m = __ballot_sync(kFull, ncomp > 0);
  int lane = threadIdx.x & 31;
  unsigned long long tot = ncomp;
#pragma unroll
  for (int o = 16; o; o >>= 1) tot += __shfl_down_sync(kFull, tot, o);
  int base = 0;
  if (lane == 0 && m) {
    base = atomicAdd(&ctl->n_act, __popc(m));
    atomicAdd(&ctl->evals, tot);
    atomicAdd(&ctl->act_blocks, (unsigned long long)__popc(m));
  }
  base = __shfl_sync(kFull, base, 0);
  if (ncomp > 0) act[base + __popc(m & ((1u << lane) - 1u))] = (uint32_t)b;
}

// ---------------------------------------------------------------- kernel W ---

__device__ __forceinline__ float spline_W(const DevParams& P, float q) {
  if (q < 1.0f) return P.sigma * (1.0f + q * q * (-1.5f + 0.75f * q));
  float t = 2.0f - q;
  return q < 2.0f ? 0.25f * P.sigma * t * t * t : 0.0f;
}

__device__ __forceinline__ float spline_dW(const DevParams& P, float q) {  // dW/dd
  if (q < 1.0f) return P.sigma_h * q * (-3.0f + 2.25f * q);
  float t = 2.0f - q;
  return q < 2.0f ? -0.75f * P.sigma_h * t * t : 0.0f;
}

// Exact neighbour predicate of the double-precision definition (used in the FP32
// guard band around r^2).
__device__ __forceinline__ bool exact_nbr(float4 a, float4 b, double r2d) {
  double dx = __dsub_rn((double)a.x, (double)b.x);
  double dy = __dsub_rn((double)a.y, (double)b.y);
  double dz = __dsub_rn((double)a.z, (double)b.z);
  double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  return d2 < r2d;
}

__device__ __forceinline__ float tait(const DevParams& P, float rho) {
  float r = rho * P.inv_rho0;
  float rg;
  if (P.gamma_is_7) {
    float r2 = r * r, r4 = r2 * r2;
    rg = r4 * r2 * r;
  } else {
    rg = powf(r, P.gamma);
  }
  return fmaxf(0.0f, P.tait_B * (rg - 1.0f));
}

// Candidate rows of block b: for each (dz, dy) the x range [bx - 1, bx + 1] is one
// contiguous run of the fluid (cstart) and of the boundary (bcstart) arrays.
template <class FluidFn, class BndFn>
__device__ __forceinline__ void for_candidates(const DevParams& P, int bx, int by, int bz,
                                               const uint32_t* __restrict__ cstart,
                                               const uint32_t* __restrict__ bcstart, int sub,
                                               int lpp, FluidFn&& ff, BndFn&& bf) {
  int xlo = bx > 0 ? bx - 1 : 0;
  int xhi = bx + 1 < P.nx ? bx + 1 : P.nx - 1;
  for (int dz = -1; dz <= 1; ++dz) {
    int cz = bz + dz;
    if (cz < 0 || cz >= P.nz) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      int cy = by + dy;
      if (cy < 0 || cy >= P.ny) continue;
      uint32_t rb = ((uint32_t)cz * P.ny + cy) * P.nx;
      uint32_t fs = __ldg(&cstart[rb + xlo]), fe = __ldg(&cstart[rb + xhi + 1]);
      for (uint32_t j = fs + sub; j < fe; j += lpp) ff(j);
      uint32_t bs = __ldg(&bcstart[rb + xlo]), be = __ldg(&bcstart[rb + xhi + 1]);
      for (uint32_t j = bs + sub; j < be; j += lpp) bf(j);
    }
  }
}

// MODE 0: density, Tait pressure, neighbour count.  MODE 1: acceleration.
template <int MODE>
__global__ void __launch_bounds__(256) k_neighbor(DevParams P, const uint32_t* __restrict__ act,
                                                  Ctl* ctl, const uint32_t* __restrict__ cstart,
                                                  const uint32_t* __restrict__ bcstart, PState s,
                                                  const float4* __restrict__ xb,
                                                  const uint8_t* __restrict__ cflag,
                                                  float4* __restrict__ anew) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int n_act = *(volatile int*)&ctl->n_act;
  unsigned long long pairs = 0, tests = 0;
  for (int t = warp; t < n_act; t += nwarps) {
    const uint32_t b = act[t];
    const int bx = b % P.nx, rr = b / P.nx, by = rr % P.ny, bz = rr / P.ny;
    const uint32_t beg = cstart[b], end = cstart[b + 1];
    for (uint32_t base = beg; base < end; base += 32) {
      const uint32_t ii = base + lane;
      const bool c = ii < end && cflag[ii];
      const unsigned m = __ballot_sync(kFull, c);
      if (!m) continue;
      const int nc = __popc(m);
      const int np2 = nc <= 1 ? 1 : 1 << (32 - __clz(nc - 1));
      const int lpp = 32 / np2;
      const int pid = lane / lpp, sub = lane - pid * lpp;
      int i = -1;
      if (pid < nc) {  // position of the pid-th set bit of m
        unsigned mm = m;
        for (int q = 0; q < pid; ++q) mm &= mm - 1u;
        i = (int)(base + (uint32_t)(__ffs(mm) - 1));
      }
      const float4 xi = i >= 0 ? s.x[i] : make_float4(0.f, 0.f, 0.f, 0.f);
      if (MODE == 0) {
        float wsum = 0.0f;
        int cnt = 0, ntest = 0;
        auto add = [&](float4 xj) {
          ++ntest;
          float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
          float d2 = dx * dx + dy * dy + dz * dz;
          if (d2 < P.r2_hi && (d2 < P.r2_lo || exact_nbr(xi, xj, P.r2d))) {
            ++cnt;
            wsum += spline_W(P, sqrtf(d2) * P.inv_h);
          }
        };
        for_candidates(P, bx, by, bz, cstart, bcstart, sub, lpp,
                       [&](uint32_t j) { add(s.x[j]); }, [&](uint32_t j) { add(xb[j]); });
        for (int o = lpp >> 1; o; o >>= 1) {
          wsum += __shfl_down_sync(kFull, wsum, o, lpp);
          cnt += __shfl_down_sync(kFull, cnt, o, lpp);
        }
        if (i >= 0) tests += (unsigned long long)ntest;
        if (sub == 0 && i >= 0) {
          float rho = P.m * wsum;
          float p = tait(P, rho);
          s.rho[i] = rho;
          s.prs[i] = p;
          s.nbr[i] = cnt - 1;  // the particle itself passed the predicate
          s.x[i].w = p / (rho * rho);
          s.v[i].w = rho;
          pairs += (unsigned long long)(cnt - 1);
        }
      } else {
        const float4 vi = i >= 0 ? s.v[i] : make_float4(0.f, 0.f, 0.f, 1.f);
        float ax = 0.f, ay = 0.f, az = 0.f;
        auto add = [&](float4 xj, float vjx, float vjy, float vjz, float pcj, float rhoj) {
          float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
          float d2 = dx * dx + dy * dy + dz * dz;
          if (d2 < P.r2 && d2 > 0.0f) {
            float d = sqrtf(d2);
            float f = spline_dW(P, d * P.inv_h) / d;
            float vx = (vi.x - vjx) * dx + (vi.y - vjy) * dy + (vi.z - vjz) * dz;
            float visc = vx < 0.0f ? -P.visc_coef * vx / ((vi.w + rhoj) * (d2 + P.eps_h2)) : 0.0f;
            float sc = -P.m * (xi.w + pcj + visc) * f;
            ax += sc * dx;
            ay += sc * dy;
            az += sc * dz;
          }
        };
        for_candidates(
            P, bx, by, bz, cstart, bcstart, sub, lpp,
            [&](uint32_t j) {
              float4 xj = s.x[j], vj = s.v[j];
              add(xj, vj.x, vj.y, vj.z, xj.w, vj.w);
            },
            [&](uint32_t j) { add(xb[j], 0.f, 0.f, 0.f, 0.f, vi.w); });
        for (int o = lpp >> 1; o; o >>= 1) {
          ax += __shfl_down_sync(kFull, ax, o, lpp);
          ay += __shfl_down_sync(kFull, ay, o, lpp);
          az += __shfl_down_sync(kFull, az, o, lpp);
        }
        if (sub == 0 && i >= 0) anew[i] = make_float4(P.gx + ax, P.gy + ay, P.gz + az, 0.f);
      }
    }
  }
  if (MODE == 0) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      pairs += __shfl_down_sync(kFull, pairs, o);
      tests += __shfl_down_sync(kFull, tests, o);
    }
    if (lane == 0 && pairs) atomicAdd(&ctl->pairs, pairs);
    if (lane == 0 && tests) atomicAdd(&ctl->cands, tests);
  }
}

// Section 4.1 correction of the evaluated particles: x += (a_new - a_old) dt^2 / 6,
// v += (a_new - a_old) dt / 2 with dt = (k1 - k_last) dt_b; a_old <- a_new.
// prime != 0: no time has passed; only a_old <- a_new, k_last <- k1.
__global__ void k_correct(DevParams P, const uint32_t* __restrict__ act, Ctl* ctl,
                          const uint32_t* __restrict__ cstart, PState s,
                          const uint8_t* __restrict__ cflag, const float4* __restrict__ anew,
                          int k1, int prime) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int n_act = *(volatile int*)&ctl->n_act;
  for (int t = warp; t < n_act; t += nwarps) {
    const uint32_t b = act[t];
    const uint32_t beg = cstart[b], end = cstart[b + 1];
    for (uint32_t i = beg + lane; i < end; i += 32) {
      if (!cflag[i]) continue;
      float4 an = anew[i];
      if (!prime) {
        float dt = (float)(k1 - s.klast[i]) * P.dt_b;
        float4 ao = s.a[i];
        float c1 = dt * dt / 6.0f, c2 = 0.5f * dt;
        float dax = an.x - ao.x, day = an.y - ao.y, daz = an.z - ao.z;
        float4 x = s.x[i], v = s.v[i];
        x.x += dax * c1;
        x.y += day * c1;
        x.z += daz * c1;
        v.x += dax * c2;
        v.y += day * c2;
        v.z += daz * c2;
        s.x[i] = x;
        s.v[i] = v;
      }
      s.a[i] = an;
      s.klast[i] = k1;
    }
  }
}

// Global maxima of |v|^2 and |a|^2 over the fluid (global adaptive comparator).
__global__ void k_global_max(int n, const float4* __restrict__ v, const float4* __restrict__ a,
                             Ctl* ctl) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double vm = 0.0, am = 0.0;
  if (i < n) {
    float4 vi = v[i], ai = a[i];
    vm = norm2d(vi.x, vi.y, vi.z);
    am = norm2d(ai.x, ai.y, ai.z);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    vm = fmax(vm, __shfl_down_sync(kFull, vm, o));
    am = fmax(am, __shfl_down_sync(kFull, am, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&ctl->vmax2_bits, (unsigned long long)__double_as_longlong(vm));
    atomicMax(&ctl->amax2_bits, (unsigned long long)__double_as_longlong(am));
  }
}

__global__ void k_level_hist(int n, const int32_t* __restrict__ level, Ctl* ctl) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    int L = level[i];
    if (L >= 0 && L < kMaxLevels) atomicAdd(&ctl->level_count[L], 1ull);
  }
}

// ------------------------------------------------------------------ launch ---

// CTAs of the persistent neighbour kernels: every resident slot of every SM.
int neighbor_grid_size() {
  int dev = 0, sms = 1, occ = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_neighbor<1>, 256, 0);
  if (occ < 1) occ = 1;
  return sms * occ;
}

rts_status launch_classify(rts_ctx* c) {
  int nb = c->dp.nblocks, tb = 256, g = (nb + tb - 1) / tb;
  note_launch(c, 2);
  k_block_raw<<<g, tb, 0, c->stream>>>(c->dp, c->cstart, c->s.v, c->s.a, c->raw);
  k_block_smooth<<<g, tb, 0, c->stream>>>(c->dp, c->raw, c->blevel);
  return RTS_OK;
}

rts_status launch_activity(rts_ctx* c, int mode, int level_g, int mult_g) {
  int nb = c->dp.nblocks, tb = 256, g = (nb + tb - 1) / tb;
  cudaMemsetAsync(&c->ctl->n_act, 0, sizeof(int), c->stream);
  note_launch(c, 1);
  k_activity<<<g, tb, 0, c->stream>>>(c->dp, mode, level_g, mult_g, c->cstart, c->blevel, c->s,
                                       c->cflag, c->act, c->ctl);
  return RTS_OK;
}

rts_status launch_density(rts_ctx* c) {
  note_launch(c, 1);
  k_neighbor<0><<<c->grid_persistent, 256, 0, c->stream>>>(c->dp, c->act, c->ctl, c->cstart,
                                                            c->bcstart, c->s, c->xb, c->cflag,
                                                            c->anew);
  return RTS_OK;
}

rts_status launch_force(rts_ctx* c) {
  note_launch(c, 1);
  k_neighbor<1><<<c->grid_persistent, 256, 0, c->stream>>>(c->dp, c->act, c->ctl, c->cstart,
                                                            c->bcstart, c->s, c->xb, c->cflag,
                                                            c->anew);
  return RTS_OK;
}

rts_status launch_correct(rts_ctx* c, int64_t k1, int prime) {
  note_launch(c, 1);
  k_correct<<<c->grid_persistent, 256, 0, c->stream>>>(c->dp, c->act, c->ctl, c->cstart, c->s,
                                                       c->cflag, c->anew, (int)k1, prime);
  return RTS_OK;
}

rts_status launch_global_max(rts_ctx* c) {
  cudaMemsetAsync(&c->ctl->vmax2_bits, 0, 2 * sizeof(unsigned long long), c->stream);
  int tb = 256, g = (c->n + tb - 1) / tb;
  if (c->n > 0) note_launch(c, 1);
  if (c->n > 0) k_global_max<<<g, tb, 0, c->stream>>>(c->n, c->s.v, c->s.a, c->ctl);
  return RTS_OK;
}

rts_status launch_level_hist(rts_ctx* c) {
  cudaMemsetAsync(&c->ctl->level_count[0], 0, sizeof(unsigned long long) * kMaxLevels, c->stream);
  int tb = 256, g = (c->n + tb - 1) / tb;
  if (c->n > 0) note_launch(c, 1);
  if (c->n > 0) k_level_hist<<<g, tb, 0, c->stream>>>(c->n, c->s.level, c->ctl);
  return RTS_OK;
}

}  // namespace rts
