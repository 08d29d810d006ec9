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

__device__ __forceinline__ uint32_t warp_incl_sum(uint32_t v, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t t = __shfl_up_sync(kFull, v, d);
    if (lane >= d) v += t;
  }
  return v;
}

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

// Section 3.1 in FP32: thresholds rounded to FP32; a maximum within 1e-6 of a finite
// threshold is undecided in FP32.  The FP32 square norm is within 3e-7 relative of the
// FP64 one of the same FP32 components (at most five roundings of half an ulp each, all
// terms non-negative) and the FP32 threshold within 6e-8 of the FP64 one, so outside the band
// both decide alike, with a margin of more than twice those errors.
__device__ __forceinline__ int pick_level_f(const DevParams& P, float v2, float a2, bool* undecided) {
  int L = 0;
  for (int l = 0; l < P.n_levels; ++l) {
    const float tv = P.vthr2f[l], ta = P.athr2f[l];
    if (isfinite(tv) && fabsf(v2 - tv) <= 1e-6f * tv) *undecided = true;
    if (isfinite(ta) && fabsf(a2 - ta) <= 1e-6f * ta) *undecided = true;
    if (P.eq1[l] && v2 <= tv && a2 <= ta) L = l;
  }
  return L;
}

// |u|^2 <= thr as the FP64 definition decides it, ((ux ux + uy uy) + uz uz) <= thr in
// double precision from FP32 components, without FP64 in the common case (FP64 runs at a
// small fraction of the FP32 rate here and a chain of dependent FP64 operations is slow):
// the squares are split exactly (FMA TwoProduct), summed with TwoSum, and compared with
// thr = th + tl (th = thr rounded to FP32, tl the FP32 residual, within 2^-48 thr).  The
// FP32 form is known within about 2^-42 of the larger side and the FP64 one within
// 2^-51 of the exact sum, so outside +-2^-38 thr both agree; inside, FP64 decides.
__device__ __forceinline__ bool norm2_le(float x, float y, float z, float th, float tl, double thd) {
  if (!isfinite(th)) return true;   // no bound (level 0 of Eq. 3)
  const float px = __fmul_rn(x, x), py = __fmul_rn(y, y), pz = __fmul_rn(z, z);
  if (!isfinite(px + py + pz)) return norm2d(x, y, z) <= thd;
  const float ex = __fmaf_rn(x, x, -px), ey = __fmaf_rn(y, y, -py), ez = __fmaf_rn(z, z, -pz);
  float s1, t1, s2, t2;
  two_sum(px, py, s1, t1);
  two_sum(s1, pz, s2, t2);
  const float small = __fadd_rn(__fadd_rn(__fadd_rn(ex, ey), ez), __fadd_rn(t1, t2));
  const float diff = __fadd_rn(__fsub_rn(s2, th), __fsub_rn(small, tl));
  const float win = 3.637978807091713e-12f * th;   // 2^-38 thr
  if (diff < -win) return true;
  if (diff > win) return false;
  return norm2d(x, y, z) <= thd;
}

// Level of a block from its particles when its FP32 maxima are undecided (Section 3.1,
// exact): a level passes iff every particle passes its tests; the block takes the
// largest passing level.  The block's particles are those whose current block (key_cur)
// is b: after a sort, block b's range; on a substep that kept the last sort, also in b's
// 26 sorted neighbours (particles move less than half a block between sorts).  The
// whole warp takes part (every lane calls it with the same b): the lanes share out the
// candidate particles, so the loads of one round are in flight together.
static __device__ __noinline__ int level_exact_warp(const DevParams& P, uint32_t b, int stale,
                                                    const uint32_t* __restrict__ cstart,
                                                    const uint32_t* __restrict__ key_cur,
                                                    const float4* __restrict__ v,
                                                    const float4* __restrict__ a,
                                                    const float4* __restrict__ ap, int lane) {
  const int bx = b % P.nx, rr = b / P.nx, by = rr % P.ny, bz = rr / P.ny;
  // lane c < ncells: cell c's range (the 27 cells around b, or b alone)
  const int ncells = stale ? 27 : 1;
  uint32_t st = 0, ln = 0;
  if (lane < ncells) {
    const int cx = bx + (stale ? lane % 3 - 1 : 0), cy = by + (stale ? (lane / 3) % 3 - 1 : 0),
              cz = bz + (stale ? lane / 9 - 1 : 0);
    if (cx >= 0 && cy >= 0 && cz >= 0 && cx < P.nx && cy < P.ny && cz < P.nz) {
      const uint32_t cb = ((uint32_t)cz * P.ny + cy) * P.nx + cx;
      st = cstart[cb];
      ln = cstart[cb + 1] - st;
    }
  }
  const uint32_t inc = warp_incl_sum(ln, lane);
  const uint32_t off = inc - ln;
  const uint32_t total = __shfl_sync(kFull, inc, 31);
  unsigned pass = (1u << P.n_levels) - 1u;
  for (uint32_t k0 = 0; k0 < total; k0 += 32) {
    const uint32_t k = k0 + lane;
    // the candidate's cell: the last with off <= k
    uint32_t i = 0xffffffffu;
    for (int c = 0; c < ncells; ++c) {
      const uint32_t oc = __shfl_sync(kFull, off, c), sc = __shfl_sync(kFull, st, c),
                     lc = __shfl_sync(kFull, ln, c);
      if (k < total && k >= oc && k < oc + lc) i = sc + (k - oc);
    }
    if (i == 0xffffffffu || (stale && key_cur[i] != b)) continue;
    const float4 vi = v[i];
    float4 ai = a[i];
    if (ap) {  // PCISPH: total acceleration
      const float4 pa = ap[i];
      ai.x += pa.x;
      ai.y += pa.y;
      ai.z += pa.z;
    }
    // outside 2e-6 of a threshold the FP32 norm decides (its error is below 3e-7)
    const float v2 = vi.x * vi.x + vi.y * vi.y + vi.z * vi.z;
    const float a2 = ai.x * ai.x + ai.y * ai.y + ai.z * ai.z;
    for (int l = 0; l < P.n_levels; ++l) {
      const float tv = P.vthr2f[l], ta = P.athr2f[l];
      bool ok_v = v2 <= tv, ok_a = a2 <= ta;
      if (isfinite(tv) && fabsf(v2 - tv) <= 2e-6f * tv)
        ok_v = norm2_le(vi.x, vi.y, vi.z, tv, P.vthr2lo[l], P.vthr2[l]);
      if (isfinite(ta) && fabsf(a2 - ta) <= 2e-6f * ta)
        ok_a = norm2_le(ai.x, ai.y, ai.z, ta, P.athr2lo[l], P.athr2[l]);
      if (!(ok_v && ok_a)) pass &= ~(1u << l);
    }
  }
  pass = __reduce_and_sync(kFull, pass);
  int L = 0;
  for (int l = 0; l < P.n_levels; ++l)
    if (P.eq1[l] && ((pass >> l) & 1u)) L = l;
  return L;
}

// The same decision on a substep that kept the sort, from the particles the key pass
// listed as near a threshold (within 2e-6 of one in FP32): a threshold that the block's
// FP32 maximum (vm, am) decides keeps that decision; an undecided one (the maximum within
// 1e-6 of it) can only be failed by listed particles, since every other particle of the
// block lies below it by more than the FP32 error, so the listed particles of block b
// decide it exactly.  The whole warp takes part (every lane calls it with the same b).
static __device__ __noinline__ int level_from_near(const DevParams& P, uint32_t b, float vm,
                                                   float am, const uint32_t* __restrict__ near,
                                                   int nn, const uint32_t* __restrict__ key_cur,
                                                   const float4* __restrict__ v,
                                                   const float4* __restrict__ a, int lane) {
  unsigned pv = (1u << P.n_levels) - 1u, pa = pv;
  for (int k0 = 0; k0 < nn; k0 += 32) {
    const int k = k0 + lane;
    if (k >= nn) continue;
    const uint32_t i = near[k];
    if (i >= (uint32_t)P.n_fluid || key_cur[i] != b) continue;
    const float4 vi = v[i], ai = a[i];
    const float v2 = vi.x * vi.x + vi.y * vi.y + vi.z * vi.z;
    const float a2 = ai.x * ai.x + ai.y * ai.y + ai.z * ai.z;
    for (int l = 0; l < P.n_levels; ++l) {
      const float tv = P.vthr2f[l], ta = P.athr2f[l];
      bool ok_v = v2 <= tv, ok_a = a2 <= ta;
      if (isfinite(tv) && fabsf(v2 - tv) <= 2e-6f * tv)
        ok_v = norm2_le(vi.x, vi.y, vi.z, tv, P.vthr2lo[l], P.vthr2[l]);
      if (isfinite(ta) && fabsf(a2 - ta) <= 2e-6f * ta)
        ok_a = norm2_le(ai.x, ai.y, ai.z, ta, P.athr2lo[l], P.athr2[l]);
      if (!ok_v) pv &= ~(1u << l);
      if (!ok_a) pa &= ~(1u << l);
    }
  }
  pv = __reduce_and_sync(kFull, pv);
  pa = __reduce_and_sync(kFull, pa);
  int L = 0;
  for (int l = 0; l < P.n_levels; ++l) {
    const float tv = P.vthr2f[l], ta = P.athr2f[l];
    const bool ok_v = (isfinite(tv) && fabsf(vm - tv) <= 1e-6f * tv) ? ((pv >> l) & 1u) : vm <= tv;
    const bool ok_a = (isfinite(ta) && fabsf(am - ta) <= 1e-6f * ta) ? ((pa >> l) & 1u) : am <= ta;
    if (P.eq1[l] && ok_v && ok_a) L = l;
  }
  return L;
}

// Raw levels (Section 3.1 steps 1-2) and R_min (Section 4.2) of every filled block in one
// pass, so that no pass over the grid has to finish between the raw levels and their
// minimum.  The thread of a filled block reads the stamped FP32 maxima of the block and
// its 26 neighbours (a neighbour whose maxima carry an older stamp holds no particle now
// and takes no part; an offset outside the grid stands for the block itself, which
// leaves the minimum unchanged).
//
// When both thresholds are non-increasing in the level (levels_monotone: a coarser level
// never admits a larger speed or acceleration), the levels a block passes on speed alone
// form a prefix 0..Lv of the levels, likewise on acceleration, and its raw level is the
// largest Eq. 1-admissible level up to min(Lv, La), a non-decreasing function of that
// minimum; the smallest raw level over the 27 blocks is therefore the raw level of the
// union of their particles, decided from the largest of their maxima.  Only when that
// decision is undecided (a maximum within 1e-6 of a threshold) does the thread decide
// each neighbour's raw level on its own and take the minimum, as it always does without
// the monotone thresholds.  An undecided raw level is taken from the block's particles
// with the exact decision of the double-precision definition (level_from_near /
// level_exact_warp) by the whole warp, one (lane, neighbour) at a time.
// The blocks: the sort's filled list, and with stale (a pass that kept the sort) also
// filled2, the blocks filled since; a block whose maxima carry an older stamp has emptied
// since the sort and gets no level.  Writes the raw level (raw) and R_min, or the forced
// level (blevel), both stamped.
// A lower bound of the exact level from FP32 maxima: every threshold within 1e-6 of them
// counts as failed (the exact decision can only pass it).
__device__ __forceinline__ int pick_level_lo(const DevParams& P, float v2, float a2) {
  int L = 0;
  for (int l = 0; l < P.n_levels; ++l) {
    const float tv = P.vthr2f[l], ta = P.athr2f[l];
    const bool ok_v = isfinite(tv) ? v2 < tv - 1e-6f * tv : true;
    const bool ok_a = isfinite(ta) ? a2 < ta - 1e-6f * ta : true;
    if (P.eq1[l] && ok_v && ok_a) L = l;
  }
  return L;
}

// Neighbour k (9 (dz + 1) + 3 (dy + 1) + dx + 1) of block (bx, by, bz); an axis that
// leaves the grid keeps the block's own coordinate.
__device__ __forceinline__ uint32_t nbr_block(const DevParams& P, int bx, int by, int bz, int k) {
  const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
  const int cx = (bx + dx >= 0 && bx + dx < P.nx) ? bx + dx : bx;
  const int cy = (by + dy >= 0 && by + dy < P.ny) ? by + dy : by;
  const int cz = (bz + dz >= 0 && bz + dz < P.nz) ? bz + dz : bz;
  return ((uint32_t)cz * P.ny + cy) * P.nx + cx;
}

__global__ void k_block_levels(DevParams P, const uint32_t* __restrict__ filled,
                               const int* __restrict__ nfilled, const uint32_t* __restrict__ filled2,
                               const int* __restrict__ nfilled2, const uint32_t* __restrict__ cstart,
                               const uint32_t* __restrict__ key_cur, int stale,
                               const uint32_t* __restrict__ near, const int* __restrict__ n_near,
                               const float4* __restrict__ v, const float4* __restrict__ a,
                               const float4* __restrict__ ap,
                               const unsigned long long* __restrict__ bmax_v,
                               const unsigned long long* __restrict__ bmax_a, uint32_t stamp,
                               uint32_t* __restrict__ raw, uint32_t* __restrict__ blevel) {
  pdl_wait();
  const int nf1 = *nfilled;
  const int nf = nf1 + (stale ? *nfilled2 : 0);
  const int nn = stale ? *n_near : 0;   // beyond kNearCap the sorted cells are scanned
  const int lane = threadIdx.x & 31;
  const int wstride = gridDim.x * blockDim.x;
  const int pl = P.nx * P.ny;
  // warp-uniform trip count (the exact decision needs every lane)
  for (int t0 = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; t0 < nf; t0 += wstride) {
    const int t = t0 + lane;
    uint32_t b = 0;
    bool live = false;
    int bx = 0, by = 0, bz = 0, own = 0, lmin = P.n_levels;
    uint32_t undec = 0;   // blocks (bit 9 (dz + 1) + 3 (dy + 1) + dx + 1) still to decide
    if (t < nf) {
      b = t < nf1 ? filled[t] : filled2[t - nf1];
      bx = (int)(b % (uint32_t)P.nx);
      const int rr = (int)(b / (uint32_t)P.nx);
      by = rr % P.ny;
      bz = rr / P.ny;
      const int ox[3] = {bx > 0 ? -1 : 0, 0, bx + 1 < P.nx ? 1 : 0};
      const int oy[3] = {by > 0 ? -P.nx : 0, 0, by + 1 < P.ny ? P.nx : 0};
      const int oz[3] = {bz > 0 ? -pl : 0, 0, bz + 1 < P.nz ? pl : 0};
      // the block's own maxima and those of the union (FP32 bits of non-negative values:
      // ordered as integers); the block's own stamp is checked after the loads
      uint32_t uv = 0, ua = 0, cv = 0, ca = 0;
#pragma unroll
      for (int zl = 0; zl < 3; ++zl) {
        unsigned long long rv[9], ra[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {   // one layer's 18 loads in flight together
          const int nb = (int)b + ox[q % 3] + oy[q / 3] + oz[zl];
          rv[q] = bmax_v[nb];
          ra[q] = bmax_a[nb];
        }
        if (zl == 1) {
          live = (uint32_t)(rv[4] >> 32) == stamp;
          cv = (uint32_t)rv[4];
          ca = (uint32_t)ra[4];
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          if ((uint32_t)(rv[q] >> 32) != stamp) continue;
          uv = (uint32_t)rv[q] > uv ? (uint32_t)rv[q] : uv;
          ua = (uint32_t)ra[q] > ua ? (uint32_t)ra[q] : ua;
        }
      }
      if (live) {
        bool u_own = false, u_all = !P.levels_monotone;
        own = pick_level_f(P, __uint_as_float(cv), __uint_as_float(ca), &u_own);
        if (u_own) undec |= 1u << 13;
        if (!u_all) lmin = pick_level_f(P, __uint_as_float(uv), __uint_as_float(ua), &u_all);
        if (u_all) {   // every block on its own: decided ones now, undecided ones below
          lmin = P.n_levels;
          for (int k = 0; k < 27; ++k) {
            const uint32_t nb = nbr_block(P, bx, by, bz, k);
            const unsigned long long rv = bmax_v[nb];
            if ((uint32_t)(rv >> 32) != stamp) continue;
            bool u = false;
            const int lk = pick_level_f(P, __uint_as_float((uint32_t)rv),
                                        __uint_as_float((uint32_t)bmax_a[nb]), &u);
            if (u) undec |= 1u << k;
            else lmin = lk < lmin ? lk : lmin;
          }
          // an undecided neighbour whose level cannot fall below the decided minimum
          // (every threshold near its maxima taken as failed) need not be decided
          for (uint32_t mm = undec & ~(1u << 13); mm; mm &= mm - 1u) {
            const int k = __ffs(mm) - 1;
            const uint32_t nb = nbr_block(P, bx, by, bz, k);
            if (pick_level_lo(P, __uint_as_float((uint32_t)bmax_v[nb]),
                              __uint_as_float((uint32_t)bmax_a[nb])) >= lmin)
              undec &= ~(1u << k);
          }
        }
      }
    }
    // undecided raw levels: the exact decision, warp-wide, one (lane, block) at a time
    for (;;) {
      const int k = undec ? __ffs(undec) - 1 : -1;
      const unsigned m = __ballot_sync(kFull, k >= 0);
      if (!m) break;
      const int src = __ffs(m) - 1;
      const uint32_t nbk = k >= 0 ? nbr_block(P, bx, by, bz, k) : 0u;
      const uint32_t bu = __shfl_sync(kFull, nbk, src);
      const float vmu = __uint_as_float((uint32_t)bmax_v[bu]);
      const float amu = __uint_as_float((uint32_t)bmax_a[bu]);
      const int lu = (stale && nn <= kNearCap)
                         ? level_from_near(P, bu, vmu, amu, near, nn, key_cur, v, a, lane)
                         : level_exact_warp(P, bu, stale, cstart, key_cur, v, a, ap, lane);
      // every lane takes it for each of its blocks that is bu (after the union's decision
      // a block's own level is never below it: the minimum keeps that decision)
      for (uint32_t mm = undec; mm; mm &= mm - 1u) {
        const int kk = __ffs(mm) - 1;
        if (nbr_block(P, bx, by, bz, kk) != bu) continue;
        if (kk == 13) own = lu;
        lmin = lu < lmin ? lu : lmin;
        undec &= ~(1u << kk);
      }
    }
    if (live) {
      raw[b] = (stamp << 8) | (uint32_t)own;
      blevel[b] = (stamp << 8) | (uint32_t)(P.force_level >= 0 ? P.force_level : lmin);
    }
  }
}

// Global adaptive stepping: every filled block takes the step's level.
__global__ void k_block_set_level(int level_g, const uint32_t* __restrict__ filled,
                                  const int* __restrict__ nfilled, uint32_t* __restrict__ blevel,
                                  uint32_t stamp) {
  pdl_wait();
  const int nf = *nfilled;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nf; t += gridDim.x * blockDim.x)
    blevel[filled[t]] = (stamp << 8) | (uint32_t)level_g;
}

// Algorithm 1's per-particle bookkeeping, in block order: validity -= 1; compute iff
// validity <= 0 or the block's level differs from the particle's (pre-emption); a
// computing particle takes the block's level and a new validity.  Work lists: the
// evaluated particles, and the blocks holding one (each run of equal blocks in a warp
// claims its block once through a stamped flag).  Each CTA takes kActItems chunks of 32
// particles per warp, gathers its list entries in shared memory (warp-aggregated shared
// atomics) and appends them with one global atomic per list: the lists' order is
// irrelevant to every consumer.
constexpr int kActThreads = 256;
constexpr int kActItems = 4;

// k1 mod mult[L] for every level (the level-aligned clock), computed once on the host.
struct LevelPhase {
  int v[kMaxLevels];
};

__global__ void __launch_bounds__(kActThreads, 8) k_particle_activity(
    DevParams P, int mode, int mult_g, LevelPhase kmod, int n, const uint32_t* __restrict__ key,
    const uint32_t* __restrict__ key_cur, const uint32_t* __restrict__ blevel, uint32_t stamp,
    PState s, uint8_t* __restrict__ cflag,
    uint32_t* __restrict__ actflag, uint32_t* __restrict__ act, uint32_t* __restrict__ plist,
    Ctl* ctl) {
  pdl_wait();
  __shared__ uint32_t sp[kActThreads * kActItems], sa[kActThreads * kActItems];
  __shared__ uint32_t scount[2], sbase[2];
  __shared__ int s_kmod[kMaxLevels];   // kmod in shared memory (a parameter array indexed
                                       // at run time would be copied to local memory)
  if (threadIdx.x < kMaxLevels) {
    int val = 0;
#pragma unroll
    for (int l = 0; l < kMaxLevels; ++l)
      if ((int)threadIdx.x == l) val = kmod.v[l];
    s_kmod[threadIdx.x] = val;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned below = (1u << lane) - 1u;
  // a grid of resident CTAs, each taking chunks of kActThreads x kActItems particles
  for (int chunk = blockIdx.x; chunk * (kActThreads * kActItems) < n; chunk += gridDim.x) {
    if (threadIdx.x < 2) scount[threadIdx.x] = 0u;
    __syncthreads();   // (also: the previous chunk's lists are written out)
    const int base0 = chunk * (kActThreads * kActItems) + w * (32 * kActItems) + lane;
    // loads of every item first (the block record depends on the key).  bk: the block the
    // particle is sorted in (its work-list entry); its level is that of its current block.
    uint32_t bk[kActItems], rec[kActItems], ck[kActItems];
    int vold[kActItems], lold[kActItems];
  #pragma unroll
    for (int it = 0; it < kActItems; ++it) {
      const int i = base0 + 32 * it;
      bk[it] = i < n ? key[i] : 0xffffffffu;
      ck[it] = i < n ? key_cur[i] : 0xffffffffu;
      vold[it] = (i < n && mode == kActRegional) ? s.valid[i] : 0;
      lold[it] = (i < n && mode == kActRegional) ? s.level[i] : 0;
    }
  #pragma unroll
    for (int it = 0; it < kActItems; ++it)
      rec[it] = ck[it] < (uint32_t)P.nblocks ? blevel[ck[it]] : 0u;
  #pragma unroll
    for (int it = 0; it < kActItems; ++it) {
      const int i = base0 + 32 * it;
      const bool valid = i < n;
      bool c = false;
      const uint32_t b = bk[it];
      if (valid) {
        int L = (int)(rec[it] & 0xffu);
        if ((rec[it] >> 8) != stamp || L >= P.n_levels) {
          check_failed(ctl, kChkLevel, rec[it]);
          L = 0;
        }
        const int mb = mode == kActGlobal ? mult_g : P.mult[L];
        // validity of a particle that starts a true step now (level-aligned variant: up
        // to the next multiple of the multiplier)
        const int vnew = (mode != kActGlobal && P.level_clock) ? mb - s_kmod[L] : mb;
        if (mode == kActRegional) {
          int val = vold[it] - 1;
          int li = lold[it];
          if (li >= P.n_levels) {
            check_failed(ctl, kChkLevel, (unsigned)li);
            li = -1;
          }
          if (val <= 0 || li < 0 || P.mult[li] != mb) {
            c = true;
            s.level[i] = L;
            val = vnew;
          }
          s.valid[i] = val;
        } else {
          c = true;
          s.level[i] = L;
          s.valid[i] = vnew;
        }
        cflag[i] = c ? 1 : 0;
      }
      const unsigned m = __ballot_sync(kFull, c);
      // runs of equal blocks in lane order; a run with an evaluated particle claims its block
      const uint32_t prevb = __shfl_up_sync(kFull, b, 1);
      const bool head = valid && (lane == 0 || prevb != b);
      const unsigned heads = __ballot_sync(kFull, head);
      const unsigned after = heads & ~(below | (1u << lane));
      const int next = after ? __ffs(after) - 1 : 32;
      const unsigned span = (next - lane >= 32) ? (kFull << lane) : (((1u << (next - lane)) - 1u) << lane);
      bool claim = false;
      if (head && (m & span)) claim = atomicExch(&actflag[b], stamp) != stamp;
      const unsigned cm = __ballot_sync(kFull, claim);
      uint32_t op = 0, oa = 0;
      if (lane == 0) {
        if (m) op = atomicAdd(&scount[0], (uint32_t)__popc(m));
        if (cm) oa = atomicAdd(&scount[1], (uint32_t)__popc(cm));
      }
      op = __shfl_sync(kFull, op, 0);
      oa = __shfl_sync(kFull, oa, 0);
      if (c) sp[op + __popc(m & below)] = (uint32_t)i;
      if (claim) sa[oa + __popc(cm & below)] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {   // one atomic per list and counter
      const uint32_t tp = scount[0], ta = scount[1];
      sbase[0] = tp ? (uint32_t)atomicAdd(&ctl->n_plist, (int)tp) : 0u;
      sbase[1] = ta ? (uint32_t)atomicAdd(&ctl->n_act, (int)ta) : 0u;
      if (tp) {
        atomicAdd(&ctl->evals, (unsigned long long)tp);
        atomicAdd(&ctl->act_blocks, (unsigned long long)ta);
      }
    }
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < scount[0]; k += blockDim.x) plist[sbase[0] + k] = sp[k];
    for (uint32_t k = threadIdx.x; k < scount[1]; k += blockDim.x) act[sbase[1] + k] = sa[k];
    __syncthreads();
  }
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

__device__ __forceinline__ float tait(const DevParams& P, float rho) {
  float r = rho * P.inv_rho0;
  float rg;
  if (P.gamma_is_7) {
    float r2 = r * r, r4 = r2 * r2;
    rg = r4 * r2 * r;
  } else {
    rg = powf(r, P.gamma);
  }
  const float p = P.tait_B * (rg - 1.0f);
  return P.no_clamp ? p : fmaxf(0.0f, p);
}

// ------------------------------------------------------ neighbour passes ---

constexpr int kNbThreads = 128;            // 4 warps per CTA, one active block per warp
constexpr int kCap = 320;                  // candidates staged per warp and chunk
constexpr uint32_t kBoundaryBit = 0x80000000u;  // neighbour index refers to a boundary particle

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}


// The candidates of block b are 18 contiguous runs: for each of the 9 (dz, dy) rows the
// x range [bx - 1, bx + 1] of the fluid array (runs 0-8) and of the boundary array
// (runs 9-17).  Lane r < 18 holds run r's start and length; off is the run's offset in
// the concatenation (fluid first).
struct Runs {
  uint32_t start, len, off, total, nfluid;
};

__device__ __forceinline__ Runs block_runs(const DevParams& P, int bx, int by, int bz,
                                           const uint32_t* __restrict__ cstart,
                                           const uint32_t* __restrict__ bcstart, int lane) {
  Runs R;
  R.start = 0;
  R.len = 0;
  if (lane < 18) {
    int row = lane < 9 ? lane : lane - 9;
    int cz = bz + row / 3 - 1, cy = by + row % 3 - 1;
    if (cz >= 0 && cz < P.nz && cy >= 0 && cy < P.ny) {
      int xlo = bx > 0 ? bx - 1 : 0;
      int xhi = bx + 1 < P.nx ? bx + 1 : P.nx - 1;
      uint32_t rb = ((uint32_t)cz * P.ny + cy) * P.nx;
      const uint32_t* cs = lane < 9 ? cstart : bcstart;
      R.start = __ldg(&cs[rb + xlo]);
      R.len = __ldg(&cs[rb + xhi + 1]) - R.start;
    }
  }
  uint32_t inc = warp_incl_sum(R.len, lane);
  R.off = inc - R.len;
  R.total = __shfl_sync(kFull, inc, 17);
  R.nfluid = __shfl_sync(kFull, inc, 8);
  return R;
}

// The evaluated particles of one active block, split over the warp's lanes: lpp lanes
// per particle (a power of two), particle pid of the group, lane sub within it.
struct Group {
  int i, lpp, pid, sub;
  unsigned gmask;
};

__device__ __forceinline__ bool next_group(uint32_t base, uint32_t end,
                                           const uint8_t* __restrict__ cflag, int lane, Group& G) {
  const uint32_t ii = base + lane;
  const bool c = ii < end && cflag[ii];
  const unsigned m = __ballot_sync(kFull, c);
  if (!m) return false;
  const int nc = __popc(m);
  const int np2 = nc <= 1 ? 1 : 1 << (32 - __clz(nc - 1));
  G.lpp = 32 / np2;
  G.pid = lane / G.lpp;
  G.sub = lane - G.pid * G.lpp;
  G.gmask = (G.lpp == 32 ? kFull : ((1u << G.lpp) - 1u)) << (G.pid * G.lpp);
  G.i = -1;
  if (G.pid < nc) {  // position of the pid-th set bit of m
    unsigned mm = m;
    for (int q = 0; q < G.pid; ++q) mm &= mm - 1u;
    G.i = (int)(base + (uint32_t)(__ffs(mm) - 1));
  }
  return true;
}

// Stage the candidates [c0, c0 + kCap) of the block's runs (tab: the 18 runs' start,
// length and offset in the concatenation) in shared memory with their indices (boundary:
// top bit); with cull, keep only those within the support radius of the box [lo, hi]
// bounding the group's evaluated particles (every neighbour of a particle in the box
// passes), compacted in place.  The copies are asynchronous, so all of a lane's loads are
// in flight at once; the cull reads shared memory.  Returns the number kept.
// nfr: fluid runs (runs 0 .. nfr - 1), nr: all runs; tab[3 nr ..] is a sentinel run.
__device__ __forceinline__ uint32_t stage_culled(const DevParams& P, const uint32_t* tab,
                                                 int nfr, int nr, uint32_t total, float3 lo,
                                                 float3 hi, uint32_t c0, bool cull,
                                                 const float4* __restrict__ xf,
                                                 const float4* __restrict__ xbnd, float4* sx,
                                                 uint32_t* sidx, int lane, Ctl* ctl) {
  const float cut2 = P.r2_hi * 1.0001f;
  const unsigned below = (1u << lane) - 1u;
  const uint32_t cnr = total - c0 < (uint32_t)kCap ? total - c0 : (uint32_t)kCap;
  int r = 0;
  for (uint32_t k = lane; k < cnr; k += 32) {
    const uint32_t kk = c0 + k;
    while (kk >= tab[3 * r + 2] + tab[3 * r + 1]) ++r;
    const uint32_t g = tab[3 * r] + (kk - tab[3 * r + 2]);
    if (r < nr && g < (uint32_t)(r < nfr ? P.n_fluid : P.n_bound)) {
      cp_async16(&sx[k], r < nfr ? &xf[g] : &xbnd[g]);
      sidx[k] = r < nfr ? g : (g | kBoundaryBit);
    } else {
      check_failed(ctl, kChkRun, g);
      sx[k] = make_float4(3e38f, 3e38f, 3e38f, 0.f);   // culled below
      sidx[k] = 0u;
    }
  }
  cp_async_wait_all();
  __syncwarp();
  if (!cull) return cnr;
  uint32_t kept = 0;
  for (uint32_t k0 = 0; k0 < cnr; k0 += 32) {
    const uint32_t k = k0 + lane;
    bool keep = false;
    float4 xj = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t tag = 0;
    if (k < cnr) {
      xj = sx[k];
      tag = sidx[k];
      const float ex = fmaxf(fmaxf(lo.x - xj.x, xj.x - hi.x), 0.f);
      const float ey = fmaxf(fmaxf(lo.y - xj.y, xj.y - hi.y), 0.f);
      const float ez = fmaxf(fmaxf(lo.z - xj.z, xj.z - hi.z), 0.f);
      keep = ex * ex + ey * ey + ez * ez <= cut2;
    }
    const unsigned m = __ballot_sync(kFull, keep);   // every read of the round precedes
    const uint32_t pos = kept + (uint32_t)__popc(m & below);   // the writes (pos <= k)
    if (keep) {
      sx[pos] = xj;
      sidx[pos] = tag;
    }
    kept += (uint32_t)__popc(m);
    __syncwarp();
  }
  return kept;
}

// Runs of the sorted blocks that can hold a neighbour of a group of evaluated particles
// on a substep that kept the last sort (stale bins): every particle is at most dlt (per
// axis) outside the block it was sorted into, so a neighbour of a particle in the box
// [lo, hi] was sorted into a block meeting [lo - r - dlt, hi + r + dlt] (rounded outward
// here).  Up to 7 x 7 rows of contiguous x runs (enough while particles stay within half
// a block of their sorted blocks), of the fluid (runs 0 .. nrow - 1) and of the static
// boundary (nrow .. 2 nrow - 1), written to tab with the sentinel; the candidates are a
// superset of the neighbours, which the exact predicate then selects, so the neighbour
// sets are those of a fresh sort.  Returns the candidate count.
constexpr int kStaleAxis = 7;
constexpr int kStaleRuns = 2 * kStaleAxis * kStaleAxis;   // 98
constexpr int kTabFresh = 64, kTabStale = 300;   // u32 per warp: 3 x (runs + sentinel)

__device__ __forceinline__ void axis_range(float l, float h, float ext, float o, float inv_e,
                                           int n, int* c0, int* c1, bool* clipped) {
  int a = (int)floorf((l - ext - o) * inv_e - 1e-3f);
  int b = (int)floorf((h + ext - o) * inv_e + 1e-3f);
  a = a < 0 ? 0 : a;
  b = b > n - 1 ? n - 1 : b;
  if (b - a + 1 > kStaleAxis) {
    *clipped = true;
    b = a + kStaleAxis - 1;
  }
  *c0 = a;
  *c1 = b;
}

__device__ __forceinline__ uint32_t stale_runs(const DevParams& P, float3 lo, float3 hi, float dlt,
                                               const uint32_t* __restrict__ cstart,
                                               const uint32_t* __restrict__ bcstart, uint32_t* tab,
                                               int lane, Ctl* ctl, int* nfr, int* nr) {
  const float ext = P.r + dlt;
  int x0, x1, y0, y1, z0, z1;
  bool clipped = false;
  axis_range(lo.x, hi.x, ext, P.ox, P.inv_edge, P.nx, &x0, &x1, &clipped);
  axis_range(lo.y, hi.y, ext, P.oy, P.inv_edge, P.ny, &y0, &y1, &clipped);
  axis_range(lo.z, hi.z, ext, P.oz, P.inv_edge, P.nz, &z0, &z1, &clipped);
  if (clipped && lane == 0) check_failed(ctl, kChkDisp, 0u);
  const int nyr = y1 - y0 + 1, nrow = nyr * (z1 - z0 + 1), nrun = 2 * nrow;
  constexpr int kH = (kStaleRuns + 31) / 32;
  uint32_t st[kH], ln[kH];
#pragma unroll
  for (int h = 0; h < kH; ++h) {
    const int e = lane + 32 * h;
    st[h] = 0;
    ln[h] = 0;
    if (e < nrun) {
      const bool fl = e < nrow;
      const int ri = fl ? e : e - nrow;
      const int cy = y0 + ri % nyr, cz = z0 + ri / nyr;
      const uint32_t rb = ((uint32_t)cz * P.ny + cy) * P.nx;
      const uint32_t* cs = fl ? cstart : bcstart;
      st[h] = __ldg(&cs[rb + x0]);
      ln[h] = __ldg(&cs[rb + x1 + 1]) - st[h];
    }
  }
  __syncwarp();   // the previous chunk's readers of tab are done
  uint32_t carry = 0;
#pragma unroll
  for (int h = 0; h < kH; ++h) {
    const uint32_t inc = warp_incl_sum(ln[h], lane) + carry;
    const int e = lane + 32 * h;
    if (e < nrun) {
      tab[3 * e] = st[h];
      tab[3 * e + 1] = ln[h];
      tab[3 * e + 2] = inc - ln[h];
    }
    carry = __shfl_sync(kFull, inc, 31);
  }
  const uint32_t total = carry;
  if (lane == 0) {  // sentinel run: never exhausted
    tab[3 * nrun] = 0;
    tab[3 * nrun + 1] = 0xffffffffu;
    tab[3 * nrun + 2] = 0;
  }
  __syncwarp();
  *nfr = nrow;
  *nr = nrun;
  return total;
}

// The density pass with one lane per particle, for a pass that sorted and evaluates at
// least half of the particles: each warp takes 32 consecutive sorted positions, and each
// lane whose particle is evaluated walks the 18 runs of its block's stencil (the fluid
// and boundary particles of the x range [bx - 1, bx + 1] of each of the 9 (dy, dz) rows)
// straight from the sorted arrays, which the warp's lanes share through L1 (they lie in a
// few neighbouring blocks).  Runs are taken 32 candidates at a time: distance tests only
// (a bit per candidate inside the guard band), then the exact predicate, kernel sum and
// list entry for those.  The neighbour list of a particle is in stencil order: fluid rows
// then boundary rows, each in sorted order.
// A sorted pass runs k_density_dense when it evaluates at least half of the particles and
// enough of them to fill the GPU with lanes (lanes_min); otherwise k_density.
__device__ __forceinline__ bool dense_pass(const DevParams& P, int np, int lanes_min) {
  return np > 0 && np >= lanes_min && 2 * (long long)np >= (long long)P.n_fluid;
}

// The next work item of a warp after its first: nwarps + a shared counter (every lane calls).
__device__ __forceinline__ int next_item(int* counter, int lane, int nwarps) {
  int v = 0;
  if (lane == 0) v = atomicAdd(counter, 1);
  return nwarps + __shfl_sync(kFull, v, 0);
}

constexpr int kDenseThreads = 256;

__global__ void __launch_bounds__(kDenseThreads) k_density_dense(
    DevParams P, const uint32_t* __restrict__ key, Ctl* ctl, const uint32_t* __restrict__ cstart,
    const uint32_t* __restrict__ bcstart, PState s, const float4* __restrict__ xb,
    const uint8_t* __restrict__ cflag, uint32_t* __restrict__ nbl, int lanes_min) {
  pdl_wait();
  if (!dense_pass(P, *(volatile int*)&ctl->n_plist, lanes_min)) return;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int n = P.n_fluid;
  const int pl = P.nx * P.ny;
  unsigned long long pairs = 0, tests = 0;
  // each warp's first 32 positions by its index, every further 32 from a shared counter
  for (int base = warp * 32; base < n; base = 32 * next_item(&ctl->dens_next, lane, nwarps)) {
    do {   // this lane's particle (break: nothing to do)
      const int i = base + lane;
      if (i >= n || !cflag[i]) break;
      const float4 xi = s.x[i];
      const uint32_t b = key[i];
      if (b >= (uint32_t)P.nblocks) {
        check_failed(ctl, kChkActive, b);
        break;
      }
      const int bx = (int)(b % (uint32_t)P.nx), rr = (int)(b / (uint32_t)P.nx);
      const int by = rr % P.ny, bz = rr / P.ny;
      const int xlo = bx > 0 ? bx - 1 : 0, xhi = bx + 1 < P.nx ? bx + 1 : P.nx - 1;
      uint32_t* list = nbl + (size_t)i * P.nbl_cap;
      float wsum = 0.f;
      int nn = 0;
      uint32_t ncand = 0;
      for (int r = 0; r < 18; ++r) {   // runs 0-8 fluid, 9-17 boundary
        const int row = r < 9 ? r : r - 9;
        const int cz = bz + row / 3 - 1, cy = by + row % 3 - 1;
        if (cz < 0 || cz >= P.nz || cy < 0 || cy >= P.ny) continue;
        const uint32_t rb = (uint32_t)cz * (uint32_t)pl + (uint32_t)cy * (uint32_t)P.nx;
        const uint32_t* cs = r < 9 ? cstart : bcstart;
        const float4* X = r < 9 ? s.x : xb;
        const uint32_t tag = r < 9 ? 0u : kBoundaryBit;
        const uint32_t lim = (uint32_t)(r < 9 ? P.n_fluid : P.n_bound);
        const uint32_t js = __ldg(&cs[rb + xlo]);
        uint32_t je = __ldg(&cs[rb + xhi + 1]);
        if (je > lim || js > je) {
          check_failed(ctl, kChkRun, je);
          je = js > lim ? js : lim;
          if (js >= je) continue;
        }
        ncand += je - js;
        for (uint32_t j0 = js; j0 < je; j0 += 32) {
          const uint32_t cnt = je - j0 < 32u ? je - j0 : 32u;
          // distance tests only, four candidates' loads in flight at a time
          uint32_t near = 0;
          uint32_t t0 = 0;
          for (; t0 + 4 <= cnt; t0 += 4) {   // whole groups of four, then the rest one by one
            float4 xj[4];
  #pragma unroll
            for (int u = 0; u < 4; ++u) xj[u] = X[j0 + t0 + u];
  #pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float dx = xi.x - xj[u].x, dy = xi.y - xj[u].y, dz = xi.z - xj[u].z;
              const float d2 = dx * dx + dy * dy + dz * dz;
              near |= d2 < P.r2_hi ? (1u << (t0 + u)) : 0u;
            }
          }
          for (; t0 < cnt; ++t0) {
            const float4 xj = X[j0 + t0];
            const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
            const float d2 = dx * dx + dy * dy + dz * dz;
            near |= d2 < P.r2_hi ? (1u << t0) : 0u;
          }
          // the exact predicate, kernel sum and list entry of the near ones
          for (uint32_t m = near; m; m &= m - 1u) {
            const uint32_t j = j0 + (uint32_t)(__ffs(m) - 1);
            const float4 xj = X[j];
            const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
            const float d2 = dx * dx + dy * dy + dz * dz;
            if (!(d2 < P.r2_lo || nbr_exact(P, xi, xj))) continue;
            bool put = true;
            if (d2 > 0.f) {
              wsum += spline_W(P, d2 * rsqrtf(d2) * P.inv_h);
            } else {
              wsum += P.sigma;   // the particle itself, or a coincident neighbour
              put = tag != 0u || j != (uint32_t)i;
            }
            if (put) {
              if (nn < P.nbl_cap) list[nn] = j | tag;
              ++nn;
            }
          }
        }
      }
      if (nn > P.nbl_cap) set_status(ctl, RTS_ERR_CAPACITY);
      const float rho = P.m * wsum;
      const float p = tait(P, rho);
      s.rho[i] = rho;
      s.prs[i] = p;
      s.nbr[i] = nn;
      s.x[i].w = p / (rho * rho);
      s.v[i].w = rho;
      pairs += (unsigned long long)nn;
      tests += ncand;
    } while (false);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    pairs += __shfl_down_sync(kFull, pairs, o);
    tests += __shfl_down_sync(kFull, tests, o);
  }
  // one atomic per counter and CTA (every candidate is tested: no cull)
  __shared__ unsigned long long red[2][kDenseThreads / 32];
  if (lane == 0) {
    red[0][wib] = pairs;
    red[1][wib] = tests;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long a = 0, t = 0;
    for (int k = 0; k < kDenseThreads / 32; ++k) {
      a += red[0][k];
      t += red[1][k];
    }
    if (a) atomicAdd(&ctl->pairs, a);
    if (t) {
      atomicAdd(&ctl->cands, t);
      atomicAdd(&ctl->kept, t);
    }
  }
}


// Density pass (Algorithm 1, "find neighborhoods" and "update rho, p"): every evaluated
// particle tests the candidates kept for its group with the exact predicate, sums m W
// over its neighbours (itself included), applies the Tait equation and records its
// neighbour list for the force pass.  Each round of up to 32 candidates per lane first
// tests distances only (a bit per candidate inside the guard band), then evaluates the
// kernel for those, then appends the neighbours in a fixed order.  kStale: a substep
// that kept the last sort; the candidates of each group come from stale_runs instead of
// the 27 blocks around the active block.
template <bool kStale>
__global__ void __launch_bounds__(kNbThreads, 6) k_density(DevParams P, const uint32_t* __restrict__ act,
                                                        const uint32_t* __restrict__ plist,
                                                        Ctl* ctl, const uint32_t* __restrict__ cstart,
                                                        const uint32_t* __restrict__ bcstart, PState s,
                                                        const float4* __restrict__ xb,
                                                        const uint8_t* __restrict__ cflag,
                                                        uint32_t* __restrict__ nbl, uint32_t stamp,
                                                        int lanes_min) {
  pdl_wait();
  constexpr int kTab = kStale ? kTabStale : kTabFresh;
  extern __shared__ float4 smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  float4* sx = smem + wib * kCap;
  uint32_t* sidx = reinterpret_cast<uint32_t*>(smem + (kNbThreads / 32) * kCap) + wib * kCap;
  uint32_t* tab = reinterpret_cast<uint32_t*>(smem + (kNbThreads / 32) * kCap) +
                  (kNbThreads / 32) * kCap + wib * kTab;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int n_act = *(volatile int*)&ctl->n_act;
  const float dlt = kStale ? __uint_as_float(*(volatile unsigned int*)&ctl->disp_bits[stamp & 1]) : 0.f;
  // kStale with at most one evaluated particle per warp of the grid (the substeps where
  // only the finest levels are due): one warp per particle (all 32 lanes on its
  // candidates) instead of one per active block, so that no warp walks a block with many
  // evaluated particles while the others idle
  const int np = *(volatile int*)&ctl->n_plist;
  if (!kStale && dense_pass(P, np, lanes_min)) return;   // k_density_dense runs this pass
  const bool by_particle = kStale && np <= nwarps;
  const int n_items = by_particle ? np : n_act;
  unsigned long long pairs = 0, tests = 0, kept_tests = 0;
  // each warp's first item by its index, every further one from a shared counter, so that
  // warps that drew cheap blocks take more of them (the blocks' costs differ widely)
  for (int t = warp; t < n_items; t = next_item(&ctl->dens_next, lane, nwarps)) {
    uint32_t beg = 0, end = 1;   // by_particle: one group, the particle plist[t]
    if (by_particle) {
      if (plist[t] >= (uint32_t)P.n_fluid) {
        if (lane == 0) check_failed(ctl, kChkActive, plist[t]);
        continue;
      }
    } else {
      const uint32_t b = act[t];
      if (b >= (uint32_t)P.nblocks) {
        if (lane == 0) check_failed(ctl, kChkActive, b);
        continue;
      }
      beg = cstart[b];
      end = cstart[b + 1];
    }
    uint32_t total = 0;
    int nfr = 9, nr = 18;
    if (!kStale) {
      const uint32_t b = act[t];
      const int bx = b % P.nx, rr = b / P.nx, by = rr % P.ny, bz = rr / P.ny;
      const Runs R = block_runs(P, bx, by, bz, cstart, bcstart, lane);
      total = R.total;
      __syncwarp();
      if (lane < 18) {
        tab[3 * lane] = R.start;
        tab[3 * lane + 1] = R.len;
        tab[3 * lane + 2] = R.off;
      }
      if (lane == 18) {  // sentinel run: never exhausted
        tab[3 * 18] = 0;
        tab[3 * 18 + 1] = 0xffffffffu;
        tab[3 * 18 + 2] = 0;
      }
      __syncwarp();
    }
    for (uint32_t base = beg; base < end; base += 32) {
      Group G;
      if (by_particle) {
        G.i = (int)plist[t];
        G.lpp = 32;
        G.pid = 0;
        G.sub = lane;
        G.gmask = kFull;
      } else if (!next_group(base, end, cflag, lane, G)) {
        continue;
      }
      const int i = G.i;
      const bool gvalid = i >= 0;
      const uint32_t lpp = (uint32_t)G.lpp, sub = (uint32_t)G.sub;
      const float4 xi = gvalid ? s.x[i] : make_float4(0.f, 0.f, 0.f, 0.f);
      // box of the group's evaluated particles; a group of one or two (16 or 32 lanes per
      // particle) tests every staged candidate instead: culling would cost it more than it
      // saves (the kept candidates, and so the neighbours, are the same either way)
      const bool cull = lpp < 16;
      float3 lo = gvalid ? make_float3(xi.x, xi.y, xi.z) : make_float3(3e38f, 3e38f, 3e38f);
      float3 hi = gvalid ? make_float3(xi.x, xi.y, xi.z) : make_float3(-3e38f, -3e38f, -3e38f);
      if (cull || kStale) {
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          lo.x = fminf(lo.x, __shfl_xor_sync(kFull, lo.x, o));
          lo.y = fminf(lo.y, __shfl_xor_sync(kFull, lo.y, o));
          lo.z = fminf(lo.z, __shfl_xor_sync(kFull, lo.z, o));
          hi.x = fmaxf(hi.x, __shfl_xor_sync(kFull, hi.x, o));
          hi.y = fmaxf(hi.y, __shfl_xor_sync(kFull, hi.y, o));
          hi.z = fmaxf(hi.z, __shfl_xor_sync(kFull, hi.z, o));
        }
      }
      if (kStale) total = stale_runs(P, lo, hi, dlt, cstart, bcstart, tab, lane, ctl, &nfr, &nr);
      uint32_t* list = nbl + (size_t)(gvalid ? i : 0) * P.nbl_cap;
      float wsum = 0.f;
      int nn = 0;
      for (uint32_t c0 = 0; c0 < total; c0 += kCap) {
        __syncwarp();
        const uint32_t cn = stage_culled(P, tab, nfr, nr, total, lo, hi, c0, cull, s.x, xb, sx,
                                         sidx, lane, ctl);
        if (cn == 0) continue;
        const uint32_t iters = (cn + lpp - 1) / lpp;  // uniform over the warp
        for (uint32_t r0 = 0; r0 < iters; r0 += 32) {
          const uint32_t rn = iters - r0 < 32u ? iters - r0 : 32u;
          // 1. distance test only: candidates below the upper edge of the guard band
          uint32_t near = 0;
          if (gvalid) {
#pragma unroll 4
            for (uint32_t j = 0; j < rn; ++j) {
              const uint32_t k = (r0 + j) * lpp + sub;
              const float4 xj = sx[k < cn ? k : 0u];
              const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
              const float d2 = dx * dx + dy * dy + dz * dz;
              near |= (k < cn && d2 < P.r2_hi) ? (1u << j) : 0u;
            }
          }
          // 2. exact predicate, kernel sum and neighbour bits for the near candidates
          uint32_t put = 0;
          for (uint32_t m = near; m; m &= m - 1u) {
            const uint32_t j = (uint32_t)(__ffs(m) - 1);
            const uint32_t k = (r0 + j) * lpp + sub;
            const float4 xj = sx[k];
            const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
            const float d2 = dx * dx + dy * dy + dz * dz;
            if (!(d2 < P.r2_lo || nbr_exact(P, xi, xj))) continue;
            if (d2 > 0.f) {
              wsum += spline_W(P, d2 * rsqrtf(d2) * P.inv_h);
              put |= 1u << j;
            } else {
              wsum += P.sigma;  // the particle itself, or a coincident neighbour
              if (sidx[k] != (uint32_t)i) put |= 1u << j;
            }
          }
          // 3. append: segmented exclusive prefix over the group's lanes
          const int c = __popc(put);
          int inc = c;
          for (uint32_t o = 1; o < lpp; o <<= 1) {
            int tv = __shfl_up_sync(kFull, inc, o, lpp);
            if (sub >= o) inc += tv;
          }
          const int tot = __shfl_sync(kFull, inc, lpp - 1, lpp);
          int pos = nn + inc - c;
          for (uint32_t m = put; m; m &= m - 1u) {
            const uint32_t j = (uint32_t)(__ffs(m) - 1);
            if (pos < P.nbl_cap) list[pos] = sidx[(r0 + j) * lpp + sub];
            ++pos;
          }
          nn += tot;
        }
        if (gvalid && sub == 0) kept_tests += cn;
      }
      if (gvalid && sub == 0) tests += total;
      for (uint32_t o = lpp >> 1; o; o >>= 1) wsum += __shfl_down_sync(kFull, wsum, o, lpp);
      if (sub == 0 && gvalid) {
        if (nn > P.nbl_cap) set_status(ctl, RTS_ERR_CAPACITY);
        float rho = P.m * wsum;
        float p = tait(P, rho);
        s.rho[i] = rho;
        s.prs[i] = p;
        s.nbr[i] = nn;
        s.x[i].w = p / (rho * rho);
        s.v[i].w = rho;
        pairs += (unsigned long long)nn;
      }
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    pairs += __shfl_down_sync(kFull, pairs, o);
    tests += __shfl_down_sync(kFull, tests, o);
    kept_tests += __shfl_down_sync(kFull, kept_tests, o);
  }
  // one atomic per counter and CTA (the counters are shared by every CTA)
  __shared__ unsigned long long red[3][kNbThreads / 32];
  if (lane == 0) {
    red[0][wib] = pairs;
    red[1][wib] = tests;
    red[2][wib] = kept_tests;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long a = 0, b = 0, c = 0;
    for (int k = 0; k < kNbThreads / 32; ++k) {
      a += red[0][k];
      b += red[1][k];
      c += red[2][k];
    }
    if (a) atomicAdd(&ctl->pairs, a);
    if (b) atomicAdd(&ctl->cands, b);
    if (c) atomicAdd(&ctl->kept, c);
  }
}

// Force pass (Algorithm 1, "update F^{p,v,g}"): every evaluated particle walks the
// neighbour list of the density pass.  Pressure: -m (p_i/rho_i^2 + p_j/rho_j^2) grad W;
// boundary neighbours: -m p_i/rho_i^2 grad W.  Artificial viscosity for approaching
// pairs with nu = 2 alpha h c / (rho_i + rho_j) (boundary: rho_j = rho_i, v_j = 0).
constexpr int kForceLanes = 4;

// FP32 squared norm without contraction (3 products, 2 sums, each rounded).
__device__ __forceinline__ float norm2f(float x, float y, float z) {
  return __fadd_rn(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)), __fmul_rn(z, z));
}

// One round of the force pass: slot's particle (t = r * nslots + slot) walked by LANES
// lanes.  Every lane of a warp runs the same rounds (the shuffles).
// gmode != 0 (global adaptive stepping): also the maxima over the evaluated particles of
// |v|^2 and |a_new|^2 of the state the Section 4.1 correction of this step (ending at
// substep k1) will give (gmode 1; gmode 2: a priming evaluation, no correction), the
// inputs of the next step size; *vm, *am collect this thread's (FP32 bits).
template <int LANES>
__device__ __forceinline__ void force_rounds(const DevParams& P, const uint32_t* __restrict__ plist,
                                             Ctl* ctl, const PState& s,
                                             const float4* __restrict__ xb,
                                             const uint32_t* __restrict__ nbl,
                                             float4* __restrict__ anew, int np, int gmode, int k1,
                                             unsigned* vm, unsigned* am) {
  const int lane = threadIdx.x & 31;
  const int sub = lane & (LANES - 1);
  const int slot = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 / LANES) + lane / LANES;
  const int nslots = ((gridDim.x * blockDim.x) >> 5) * (32 / LANES);
  const float4* __restrict__ xf = s.x;
  const float4* __restrict__ vf = s.v;
  const int rounds = (np + nslots - 1) / nslots;
  for (int r = 0; r < rounds; ++r) {
    const int t = r * nslots + slot;
    float ax = 0.f, ay = 0.f, az = 0.f;
    int i = -1;
    if (t < np) {
      i = (int)plist[t];
      if ((uint32_t)i >= (uint32_t)P.n_fluid) {
        if (sub == 0) check_failed(ctl, kChkActive, (unsigned)i);
        i = -1;
      }
    }
    if (i >= 0) {
      const float4 xi = xf[i], vi = vf[i];
      int nn = s.nbr[i];
      if (nn > P.nbl_cap) nn = P.nbl_cap;
      const uint32_t* list = nbl + (size_t)i * P.nbl_cap;
      for (int e = sub; e < nn; e += LANES) {
        const uint32_t jg = __ldg(&list[e]);
        float4 xj, vj;
        float pcj;
        const bool bnd = (jg & kBoundaryBit) != 0;
        if (bnd ? (jg & ~kBoundaryBit) >= (uint32_t)P.n_bound : jg >= (uint32_t)P.n_fluid) {
          check_failed(ctl, kChkNeighbour, jg);
          continue;
        }
        if (bnd) {
          xj = __ldg(&xb[jg & ~kBoundaryBit]);
          vj = make_float4(0.f, 0.f, 0.f, vi.w);
          pcj = 0.f;
        } else {
          xj = xf[jg];
          vj = vf[jg];
          pcj = xj.w;
        }
        const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
        const float d2 = dx * dx + dy * dy + dz * dz;
        if (d2 > 0.f) {
          const float inv_d = rsqrtf(d2);
          const float f = spline_dW(P, d2 * inv_d * P.inv_h) * inv_d;
          const float vx = (vi.x - vj.x) * dx + (vi.y - vj.y) * dy + (vi.z - vj.z) * dz;
          const float visc =
              vx < 0.0f ? -P.visc_coef * __fdividef(vx, (vi.w + vj.w) * (d2 + P.eps_h2)) : 0.0f;
          const float sc = -P.m * (xi.w + pcj + visc) * f;
          ax += sc * dx;
          ay += sc * dy;
          az += sc * dz;
        }
      }
    }
#pragma unroll
    for (int o = LANES >> 1; o; o >>= 1) {
      ax += __shfl_down_sync(kFull, ax, o, LANES);
      ay += __shfl_down_sync(kFull, ay, o, LANES);
      az += __shfl_down_sync(kFull, az, o, LANES);
    }
    if (sub == 0 && i >= 0) {
      const float4 an = make_float4(P.gx + ax, P.gy + ay, P.gz + az, 0.f);
      anew[i] = an;
      if (gmode) {   // the corrected velocity, with the correction's own arithmetic
        float4 xc = make_float4(0.f, 0.f, 0.f, 0.f), vc = vf[i];
        if (gmode == 1 && !P.serna_off)
          serna_correct(xc, vc, s.a[i], an, (float)(k1 - s.klast[i]) * P.dt_b);
        *vm = max(*vm, __float_as_uint(norm2f(vc.x, vc.y, vc.z)));
        *am = max(*am, __float_as_uint(norm2f(an.x, an.y, an.z)));
      }
    }
  }
}

// Particle-parallel over the evaluated-particle list: kForceLanes lanes per particle, so
// the cost per particle does not depend on how many particles of a block evaluate; when
// the list is short enough for one warp per particle (substeps where few particles are
// due), 32 lanes walk each list, which shortens the chain of dependent loads per
// particle.  The lane count only changes the summation order.
__global__ void __launch_bounds__(kNbThreads) k_force(DevParams P, const uint32_t* __restrict__ plist,
                                                      Ctl* ctl, PState s, const float4* __restrict__ xb,
                                                      const uint32_t* __restrict__ nbl,
                                                      float4* __restrict__ anew, int gmode, int k1) {
  pdl_wait();
  const int np = *(volatile int*)&ctl->n_plist;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  unsigned vm = 0u, am = 0u;
  if (np <= warps) force_rounds<32>(P, plist, ctl, s, xb, nbl, anew, np, gmode, k1, &vm, &am);
  else force_rounds<kForceLanes>(P, plist, ctl, s, xb, nbl, anew, np, gmode, k1, &vm, &am);
  if (gmode) {   // one atomic per CTA (the key pass of this step cleared the maxima)
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      vm = max(vm, __shfl_xor_sync(kFull, vm, o));
      am = max(am, __shfl_xor_sync(kFull, am, o));
    }
    __shared__ unsigned svm[kNbThreads / 32], sam[kNbThreads / 32];
    if ((threadIdx.x & 31) == 0) {
      svm[threadIdx.x >> 5] = vm;
      sam[threadIdx.x >> 5] = am;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int k = 1; k < kNbThreads / 32; ++k) {
        vm = max(vm, svm[k]);
        am = max(am, sam[k]);
      }
      if (vm) atomicMax(&ctl->vmax2f_bits, vm);
      if (am) atomicMax(&ctl->amax2f_bits, am);
    }
  }
}

// Section 4.1 correction of the evaluated particles: x += (a_new - a_old) dt^2 / 6,
// v += (a_new - a_old) dt / 2 with dt = (k1 - k_last) dt_b; a_old <- a_new.
// prime != 0: no time has passed; only a_old <- a_new, k_last <- k1.
__global__ void k_correct(DevParams P, const uint32_t* __restrict__ plist, Ctl* ctl, PState s,
                          const float4* __restrict__ anew, int k1, int prime) {
  pdl_wait();
  const int np = *(volatile int*)&ctl->n_plist;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < np; t += gridDim.x * blockDim.x) {
    const uint32_t i = plist[t];
    if (i >= (uint32_t)P.n_fluid) {
      check_failed(ctl, kChkActive, i);
      continue;
    }
    float4 an = anew[i];
    if (!prime && !P.serna_off) {
      float4 x = s.x[i], v = s.v[i];
      serna_correct(x, v, s.a[i], an, (float)(k1 - s.klast[i]) * P.dt_b);
      s.x[i] = x;
      s.v[i] = v;
    }
    s.a[i] = an;
    s.klast[i] = k1;
  }
}


// Global maxima of |v|^2 and |a|^2 over the fluid (global adaptive comparator): of the
// FP32 norms (fp64 = 0, exact maximum on FP32 bits), or of the FP64 norms (fp64 = 1),
// which the host asks for only when the FP32 maxima lie at a threshold.
__global__ void k_global_max(int n, const float4* __restrict__ v, const float4* __restrict__ a,
                             Ctl* ctl, int fp64) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  __shared__ double svm[8], sam[8];   // one atomic per counter and CTA (256 threads)
  __shared__ unsigned svf[8], saf[8];
  if (!fp64) {
    unsigned vm = 0, am = 0;
    if (i < n) {
      const float4 vi = v[i], ai = a[i];
      vm = __float_as_uint(norm2f(vi.x, vi.y, vi.z));
      am = __float_as_uint(norm2f(ai.x, ai.y, ai.z));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      vm = max(vm, __shfl_down_sync(kFull, vm, o));
      am = max(am, __shfl_down_sync(kFull, am, o));
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

__global__ void k_level_hist(int n, const int32_t* __restrict__ level, Ctl* ctl) {
  __shared__ unsigned int h[kMaxLevels];
  if (threadIdx.x < kMaxLevels) h[threadIdx.x] = 0;
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int L = level[i];
    if (L >= 0 && L < kMaxLevels) atomicAdd(&h[L], 1u);
  }
  __syncthreads();
  if (threadIdx.x < kMaxLevels && h[threadIdx.x])
    atomicAdd(&ctl->level_count[threadIdx.x], (unsigned long long)h[threadIdx.x]);
}

// ------------------------------------------------------------------ launch ---

// CTAs of the persistent neighbour kernels: every resident slot of every SM.
static int g_sms = 0;
static int sm_count() {
  if (!g_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms < 1) g_sms = 1;
  }
  return g_sms;
}

static size_t density_smem(bool stale) {
  return (size_t)(kNbThreads / 32) * (kCap * (sizeof(float4) + sizeof(uint32_t)) +
                                      (stale ? kTabStale : kTabFresh) * sizeof(uint32_t));
}

// Persistent grids: every resident slot of every SM, per kernel (the force and
// correction passes hold fewer registers and no shared memory, so more warps fit).
static int g_grid_force = 0, g_grid_stale = 0, g_grid_levels = 0, g_grid_act = 0, g_grid_dense = 0;
int neighbor_grid_size() {
  int occ0 = 1, occ1 = 1, occ2 = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ0, k_density<false>, kNbThreads, density_smem(false));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, k_force, kNbThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k_density<true>, kNbThreads, density_smem(true));
  if (occ0 < 1) occ0 = 1;
  if (occ1 < 1) occ1 = 1;
  if (occ2 < 1) occ2 = 1;
  int occ3 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ3, k_block_levels, 256, 0);
  if (occ3 < 1) occ3 = 1;
  g_grid_force = sm_count() * occ1;
  g_grid_stale = sm_count() * occ2;
  g_grid_levels = sm_count() * occ3;   // one resident wave; threads loop over the blocks
  int occ5 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ5, k_density_dense, kDenseThreads, 0);
  g_grid_dense = sm_count() * (occ5 < 1 ? 1 : occ5);
  int occ4 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ4, k_particle_activity, kActThreads, 0);
  g_grid_act = sm_count() * (occ4 < 1 ? 1 : occ4);
  return sm_count() * occ0;
}
static int force_grid(const rts_ctx* c) { return g_grid_force > 0 ? g_grid_force : c->grid_persistent; }

static int filled_grid() { return sm_count() * 8; }
int filled_grid_size() { return filled_grid(); }

// The blocks filled since the sort, and their count (a pass that kept the sort).
static const int* new_count(rts_ctx* c) { return &c->ctl->n_filled_light[c->stamp & 1]; }

rts_status launch_classify(rts_ctx* c, bool stale) {
  note_launch(c, 1);
  launch_pdl(c->stream, k_block_levels, g_grid_levels > 0 ? g_grid_levels : filled_grid(), 256, 0,
             c->dp, (const uint32_t*)c->filled,
             (const int*)&c->ctl->n_filled, (const uint32_t*)c->filled_new, new_count(c),
             (const uint32_t*)c->cstart, (const uint32_t*)(stale ? c->key_cur : c->key),
             stale ? 1 : 0, (const uint32_t*)c->near_list, (const int*)&c->ctl->n_near[c->stamp & 1],
             c->s.v, c->s.a, c->s.ap, c->bmax_v, c->bmax_a, c->stamp, c->raw, c->blevel);
  return RTS_OK;
}

// The block levels of this step: R_min from launch_classify, which every step of the
// regional modes launches first, or (global adaptive) the step's level.  mode < 0: the
// block levels only (public classification); otherwise also the activity pass.  The
// work-list counters n_act and n_plist were reset by the key pass of this step's binning
// (every step bins before its activity pass).
rts_status launch_activity(rts_ctx* c, int mode, int level_g, int mult_g, int64_t k1, bool stale) {
  if (mode == kActGlobal) {
    note_launch(c, 1);
    launch_pdl(c->stream, k_block_set_level, filled_grid(), 256, 0, level_g,
               (const uint32_t*)c->filled, (const int*)&c->ctl->n_filled, c->blevel, c->stamp);
  }
  if (mode >= 0 && c->n > 0) {
    note_launch(c, 1);
    int g = (c->n + kActThreads * kActItems - 1) / (kActThreads * kActItems);
    if (g_grid_act > 0 && g > g_grid_act) g = g_grid_act;
    LevelPhase kmod;
    for (int L = 0; L < kMaxLevels; ++L)
      kmod.v[L] = L < c->p.n_levels ? (int)(k1 % (int64_t)c->p.level_mult[L]) : 0;
    launch_pdl(c->stream, k_particle_activity, g, kActThreads, 0, c->dp, mode, mult_g, kmod, c->n,
               c->key, (const uint32_t*)(stale ? c->key_cur : c->key), c->blevel, c->stamp,
               c->s, c->cflag, c->actflag, c->act, c->plist, c->ctl);
  }
  return RTS_OK;
}

rts_status launch_density(rts_ctx* c, bool stale) {
  const int lanes_min = 8 * 32 * sm_count();   // eight warps of lanes per SM
  if (stale) {
    note_launch(c, 1);
    launch_pdl(c->stream, k_density<true>, g_grid_stale > 0 ? g_grid_stale : c->grid_persistent,
               kNbThreads, density_smem(true), c->dp, c->act, (const uint32_t*)c->plist, c->ctl,
               c->cstart, c->bcstart, c->s, c->xb, c->cflag, c->nbl, c->stamp, lanes_min);
  } else {
    // the two forms of a sorted pass: each finds from the evaluated-particle count
    // whether it is the one to run (dense_pass), and the other returns at once
    note_launch(c, 2);
    launch_pdl(c->stream, k_density_dense, g_grid_dense > 0 ? g_grid_dense : c->grid_persistent,
               kDenseThreads, 0, c->dp, (const uint32_t*)c->key, c->ctl, c->cstart, c->bcstart,
               c->s, c->xb, c->cflag, c->nbl, lanes_min);
    launch_pdl(c->stream, k_density<false>, c->grid_persistent, kNbThreads, density_smem(false),
               c->dp, c->act, (const uint32_t*)c->plist, c->ctl, c->cstart, c->bcstart, c->s, c->xb,
               c->cflag, c->nbl, c->stamp, lanes_min);
  }
  return RTS_OK;
}

rts_status launch_force(rts_ctx* c, int gmode, int64_t k1) {
  note_launch(c, 1);
  launch_pdl(c->stream, k_force, force_grid(c), kNbThreads, 0, c->dp, c->plist, c->ctl, c->s,
             c->xb, c->nbl, c->anew, gmode, (int)k1);
  return RTS_OK;
}

rts_status launch_correct(rts_ctx* c, int64_t k1, int prime) {
  note_launch(c, 1);
  launch_pdl(c->stream, k_correct, force_grid(c), kNbThreads, 0, c->dp, c->plist, c->ctl, c->s,
             c->anew, (int)k1, prime);
  return RTS_OK;
}

rts_status launch_global_max(rts_ctx* c, int fp64) {
  if (fp64)
    cudaMemsetAsync(&c->ctl->vmax2_bits, 0, 2 * sizeof(unsigned long long), c->stream);
  else
    cudaMemsetAsync(&c->ctl->vmax2f_bits, 0, 2 * sizeof(unsigned int), c->stream);
  int tb = 256, g = (c->n + tb - 1) / tb;
  if (c->n > 0) note_launch(c, 1);
  if (c->n > 0) k_global_max<<<g, tb, 0, c->stream>>>(c->n, c->s.v, c->s.a, c->ctl, fp64);
  return RTS_OK;
}

rts_status launch_level_hist(rts_ctx* c) {
  cudaMemsetAsync(&c->ctl->level_count[0], 0, sizeof(unsigned long long) * kMaxLevels, c->stream);
  if (c->n > 0) note_launch(c, 1);
  if (c->n > 0) k_level_hist<<<sm_count() * 4, 256, 0, c->stream>>>(c->n, c->s.level, c->ctl);
  return RTS_OK;
}

}  // namespace rts
