// rts_bin.cu - block grid binning (Section 3): every particle lies in exactly one block
// of a uniform grid; particles are kept sorted by block so that a block and its x
// neighbours are one contiguous range.
//
// Sort: counting sort on the block id.  An atomic per-block counter gives each
// particle a slot, an exclusive scan of the counts gives the block starts, and a
// rank pass orders each block's particles by the caller's index, so the sorted order
// is canonical (block, caller index) and independent of atomic arrival order.  The
// WCSPH predictor (Section 4.1) is fused into the key pass.
#include <cuda_runtime.h>

#include "rts_internal.cuh"

namespace rts {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Deferred correction of the last step's evaluated particles (pend), then predict
// (dt != 0: x~ = x + v dt + a dt^2 / 2, v~ = v + a dt) and the container correction, on
// loaded values: corr = the particle's correction is pending, an its new acceleration,
// dtc the length of its completed true step.  Returns whether x and v changed.  Both key
// passes use it, so they give the same bits.
__device__ __forceinline__ bool predict_math(const DevParams& P, float4& xi, float4& vi,
                                             float4& ai, bool corr, int pend, float4 an,
                                             float dtc, float dt) {
  bool moved = false;
  if (corr) {
    if (pend == kPendCorrect && !P.serna_off) {
      serna_correct(xi, vi, ai, an, dtc);
      moved = true;
    }
    ai = an;
  }
  if (dt != 0.0f) {
    const float hdt2 = 0.5f * dt * dt;
    xi.x = xi.x + vi.x * dt + ai.x * hdt2;
    xi.y = xi.y + vi.y * dt + ai.y * hdt2;
    xi.z = xi.z + vi.z * dt + ai.z * hdt2;
    vi.x = vi.x + ai.x * dt;
    vi.y = vi.y + ai.y * dt;
    vi.z = vi.z + ai.z * dt;
    if (P.wall_project) wall_project(P, xi, vi);
    moved = true;
  }
  return moved;
}

// predict_math on particle i, loads and stores included; returns its position.
__device__ __forceinline__ float4 predict_one(const DevParams& P, int i, float4* __restrict__ x,
                                              float4* __restrict__ v, float4* __restrict__ a,
                                              float dt, int pend, int pend_k1,
                                              const uint8_t* __restrict__ cflag,
                                              const float4* __restrict__ anew,
                                              int32_t* __restrict__ klast) {
  float4 xi = x[i];
  const bool corr = pend != kPendNone && cflag[i];
  if (corr || dt != 0.0f) {
    float4 vi = v[i], ai = a[i];
    float4 an = make_float4(0.f, 0.f, 0.f, 0.f);
    float dtc = 0.f;
    if (corr) {
      an = anew[i];
      dtc = (float)(pend_k1 - klast[i]) * P.dt_b;
      a[i] = an;
      klast[i] = pend_k1;
    }
    if (predict_math(P, xi, vi, ai, corr, pend, an, dtc, dt)) {
      x[i] = xi;
      v[i] = vi;
    }
  }
  return xi;
}

// Slots: particles arrive mostly in block order, so each run of equal keys in lane order
// takes one atomic on its block's counter.
__global__ void k_predict_key(DevParams P, int n, float4* __restrict__ x, float4* __restrict__ v,
                              float4* __restrict__ a, float dt, uint32_t* __restrict__ key,
                              uint32_t* __restrict__ slot, uint32_t* __restrict__ count, Ctl* ctl,
                              int pend, int pend_k1, const uint8_t* __restrict__ cflag,
                              const float4* __restrict__ anew, int32_t* __restrict__ klast,
                              const uint32_t* __restrict__ uid) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {   // the scan that follows appends the filled blocks, the activity pass
    ctl->n_filled = 0;   // the active blocks and the evaluated particles
    ctl->n_act = 0;
    ctl->n_plist = 0;
    ctl->dens_next = 0;
    // a following pass that keeps this sort counts into a clean slot
    ctl->n_filled_light[0] = ctl->n_filled_light[1] = 0;
    ctl->n_near[0] = ctl->n_near[1] = 0;
    ctl->disp_bits[0] = ctl->disp_bits[1] = 0u;
    ctl->vmax2f_bits = ctl->amax2f_bits = 0u;   // formed again by this step's force pass
  }
  if (i >= n) return;
  const float4 xi = predict_one(P, i, x, v, a, dt, pend, pend_k1, cflag, anew, klast);
  int bad = 0;
  // a batch: each particle is binned in its own scene's grid (the fluid pass has v, the
  // boundary pass not; the caller index gives the scene)
  uint32_t b = P.n_scenes ? batch_key(P, xi, scene_of(v ? P.fbase : P.bbase, P.n_scenes, uid[i]), &bad)
                          : block_key(P, xi, &bad);
  if (bad) {
    if (atomicCAS(&ctl->bad_set, 0, 1) == 0) {
      ctl->bad_uid = uid[i];
      ctl->bad_x = xi.x;
      ctl->bad_y = xi.y;
      ctl->bad_z = xi.z;
    }
    set_status(ctl, RTS_ERR_DOMAIN);
    b = 0;
  }
  key[i] = b;
  // the warp's lanes with i < n: a prefix of the warp (i = base + lane)
  const int lane = threadIdx.x & 31;
  const int wrem = n - (i - lane);
  const unsigned act = wrem >= 32 ? 0xffffffffu : ((1u << wrem) - 1u);
  __syncwarp(act);
  const uint32_t prevb = __shfl_up_sync(act, b, 1);
  const bool head = lane == 0 || prevb != b;
  const unsigned heads = __ballot_sync(act, head);
  const unsigned upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
  const int myhead = 31 - __clz(heads & upto);
  const unsigned after = heads & ~upto;
  const int next = after ? __ffs(after) - 1 : __popc(act);
  uint32_t base = 0;
  if (head) base = atomicAdd(&count[b], (uint32_t)(next - lane));
  base = __shfl_sync(act, base, myhead);
  slot[i] = base + (uint32_t)(lane - myhead);
}

// Key pass of a substep that keeps the previous sort (stale bins): the same correction,
// prediction and container as k_predict_key, then the particle's current block
// (key_cur; the arrays stay in the order of the last sort, whose blocks are skey), the
// block maxima of |v|^2 and |a|^2 merged by current block into the stamped records, and
// the largest distance, per axis, by which a particle has left the block it was sorted
// into (rounded up), which widens the density pass's search.  The blocks holding fluid
// are the sort's filled list (some may have emptied: their records keep an older stamp)
// plus the blocks the sort found empty that particles have moved into, listed here in
// filled_new by the first such particle to reach the block's record.  The maximum and the
// filled count live in slot stamp & 1, which the previous binning pass cleared (a sort
// clears both, a pass like this one the slot of the next stamp; the kernels in between
// never read it).  One atomic per CTA for the
// list (entries gathered in shared memory) and, only when it raises it, for the
// maximum, so neither counter is a point of contention.
constexpr int kLightThreads = 256;
constexpr int kLightItems = 1;

__global__ void __launch_bounds__(kLightThreads) k_predict_light(
    DevParams P, int n, float4* __restrict__ x, float4* __restrict__ v, float4* __restrict__ a,
    float dt, const uint32_t* __restrict__ skey, uint32_t* __restrict__ key_cur, Ctl* ctl,
    int pend, int pend_k1, const uint8_t* __restrict__ cflag, const float4* __restrict__ anew,
    int32_t* __restrict__ klast, const uint32_t* __restrict__ uid, uint32_t stamp,
    unsigned long long* __restrict__ bmax_v, unsigned long long* __restrict__ bmax_a,
    const uint32_t* __restrict__ cstart, uint32_t* __restrict__ filled,
    uint32_t* __restrict__ near_list) {
  pdl_wait();
  __shared__ float sdisp[kLightThreads / 32];
  __shared__ uint32_t sfill[kLightThreads * kLightItems];
  __shared__ uint32_t scount, sbase;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (blockIdx.x == 0 && threadIdx.x == 0) {   // the activity pass appends the work lists
    ctl->n_act = 0;
    ctl->n_plist = 0;
    ctl->dens_next = 0;
    ctl->disp_bits[(stamp + 1) & 1] = 0u;
    ctl->n_filled_light[(stamp + 1) & 1] = 0;
    ctl->n_near[(stamp + 1) & 1] = 0;
  }
  if (threadIdx.x == 0) scount = 0u;
  __syncthreads();
  float disp = 0.f;
  const int base0 = blockIdx.x * (kLightThreads * kLightItems) + w * (32 * kLightItems) + lane;
  // every item's loads first, so they are in flight together
  float4 xs[kLightItems], vs[kLightItems], as[kLightItems];
  uint32_t sk[kLightItems];
  bool cr[kLightItems];
#pragma unroll
  for (int it = 0; it < kLightItems; ++it) {
    const int i = base0 + 32 * it;
    const bool valid = i < n;
    xs[it] = valid ? x[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    vs[it] = valid ? v[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    as[it] = valid ? a[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    sk[it] = valid ? skey[i] : 0xffffffffu;
    cr[it] = valid && pend != kPendNone && cflag[i];
  }
#pragma unroll
  for (int it = 0; it < kLightItems; ++it) {
    const int i = base0 + 32 * it;
    const bool valid = i < n;
    uint32_t b = 0xffffffffu;
    float v2 = 0.f, a2 = 0.f;
    bool near = false;
    if (valid) {
      float4 xi = xs[it], vi = vs[it], ai = as[it];
      float4 an = make_float4(0.f, 0.f, 0.f, 0.f);
      float dtc = 0.f;
      if (cr[it]) {
        an = anew[i];
        dtc = (float)(pend_k1 - klast[i]) * P.dt_b;
        a[i] = an;
        klast[i] = pend_k1;
      }
      if (predict_math(P, xi, vi, ai, cr[it], pend, an, dtc, dt)) {
        x[i] = xi;
        v[i] = vi;
      }
      int bad = 0;
      b = block_key(P, xi, &bad);
      if (bad) {
        if (atomicCAS(&ctl->bad_set, 0, 1) == 0) {
          ctl->bad_uid = uid[i];
          ctl->bad_x = xi.x;
          ctl->bad_y = xi.y;
          ctl->bad_z = xi.z;
        }
        set_status(ctl, RTS_ERR_DOMAIN);
        b = 0;
      }
      key_cur[i] = b;
      v2 = vi.x * vi.x + vi.y * vi.y + vi.z * vi.z;
      a2 = ai.x * ai.x + ai.y * ai.y + ai.z * ai.z;
      for (int l = 0; l < P.n_levels; ++l)   // near a threshold: listed for the exact level
        near |= fabsf(v2 - P.vthr2f[l]) <= P.vnear[l] || fabsf(a2 - P.athr2f[l]) <= P.anear[l];
      const uint32_t sb = sk[it];
      if (sb != b && sb < (uint32_t)P.nblocks) {   // outside its sorted block: how far
        const uint32_t rr = div_by(sb, P.div_nx), rz = div_by(rr, P.div_ny);
        const int cx = (int)(sb - rr * (uint32_t)P.nx), cy = (int)(rr - rz * (uint32_t)P.ny);
        const int cz = (int)rz;
        const float lx = P.ox + (float)cx * P.edge, ly = P.oy + (float)cy * P.edge,
                    lz = P.oz + (float)cz * P.edge;
        const float dx = fmaxf(fmaxf(lx - xi.x, xi.x - (lx + P.edge)), 0.f);
        const float dy = fmaxf(fmaxf(ly - xi.y, xi.y - (ly + P.edge)), 0.f);
        const float dz = fmaxf(fmaxf(lz - xi.z, xi.z - (lz + P.edge)), 0.f);
        // rounded up by more than the FP32 errors of the box corners and differences
        disp = fmaxf(disp, fmaxf(fmaxf(dx, dy), dz) * 1.0001f + 1e-5f * P.edge);
      }
    }
    // segmented maxima over lanes of the same block on the FP32 bits (non-negative, so
    // ordered as integers), and whether the run holds a particle still in its sorted
    // block; every lane reaches the shuffles
    uint32_t mv = __float_as_uint(v2), ma = __float_as_uint(a2);
    uint32_t stay = (valid && sk[it] == b) ? 1u : 0u;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t ov = __shfl_down_sync(0xffffffffu, mv, d);
      const uint32_t oa = __shfl_down_sync(0xffffffffu, ma, d);
      const uint32_t os = __shfl_down_sync(0xffffffffu, stay, d);
      const uint32_t ob = __shfl_down_sync(0xffffffffu, b, d);
      if (lane + d < 32 && ob == b) {
        mv = ov > mv ? ov : mv;
        ma = oa > ma ? oa : ma;
        stay |= os;
      }
    }
    const uint32_t prevb = __shfl_up_sync(0xffffffffu, b, 1);
    bool claim = false;
    if (valid && (lane == 0 || prevb != b)) {
      const unsigned long long tag = (unsigned long long)stamp << 32;
      if (stay) {   // b held this particle at the sort: it is on the sort's filled list
        atomicMax(bmax_v + b, tag | mv);
        atomicMax(bmax_a + b, tag | ma);
      } else {      // only particles that moved in: list b if the sort found it empty
        const unsigned long long old = atomicMax(bmax_v + b, tag | mv);
        atomicMax(bmax_a + b, tag | ma);
        claim = (uint32_t)(old >> 32) != stamp && cstart[b + 1] == cstart[b];
      }
    }
    const unsigned nm = __ballot_sync(0xffffffffu, near);   // rare: one atomic per such warp
    if (nm) {
      uint32_t nb = 0;
      if (lane == 0) nb = (uint32_t)atomicAdd(&ctl->n_near[stamp & 1], __popc(nm));
      nb = __shfl_sync(0xffffffffu, nb, 0) + (uint32_t)__popc(nm & ((1u << lane) - 1u));
      if (near && nb < (uint32_t)kNearCap) near_list[nb] = (uint32_t)i;
    }
    const unsigned cm = __ballot_sync(0xffffffffu, claim);
    uint32_t off = 0;
    if (lane == 0 && cm) off = atomicAdd(&scount, (uint32_t)__popc(cm));
    off = __shfl_sync(0xffffffffu, off, 0);
    if (claim) sfill[off + __popc(cm & ((1u << lane) - 1u))] = b;
  }
#pragma unroll
  for (int d = 16; d; d >>= 1) disp = fmaxf(disp, __shfl_xor_sync(0xffffffffu, disp, d));
  if (lane == 0) sdisp[w] = disp;
  __syncthreads();
  if (threadIdx.x == 0)
    sbase = scount ? (uint32_t)atomicAdd(&ctl->n_filled_light[stamp & 1], (int)scount) : 0u;
  __syncthreads();
  if (sbase + scount > (uint32_t)P.nblocks) {   // a block listed twice: a broken invariant
    if (threadIdx.x == 0) check_failed(ctl, kChkGather, sbase + scount);
  } else {
    for (uint32_t k = threadIdx.x; k < scount; k += blockDim.x) filled[sbase + k] = sfill[k];
  }
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int k = 0; k < kLightThreads / 32; ++k) m = fmaxf(m, sdisp[k]);
    unsigned int* slot = &ctl->disp_bits[stamp & 1];
    if (m > 0.f && __float_as_uint(m) > *(volatile unsigned int*)slot) {
      atomicMax(slot, __float_as_uint(m));
      // the density pass searches at most 7 blocks per axis around a group, enough
      // while every particle stays within half a block of its sorted block
      if (m >= 0.5f * P.edge) check_failed(ctl, kChkDisp, __float_as_uint(m));
    }
  }
}

// ---- exclusive scan of the per-block counts (reduce, scan tile sums, apply) ----

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive scan of one value per thread across the CTA (up to 32 warps); returns the
// CTA total.  The warp offsets and the total live in separate slots: with 32 warps the
// last warp's offset and the total would otherwise share one.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_tot[33];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t inc = warp_incl_scan(v);
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < nw ? warp_tot[lane] : 0u;
    uint32_t ti = warp_incl_scan(t);
    if (lane < nw) warp_tot[lane] = ti - t;
    if (lane == nw - 1) warp_tot[32] = ti;
  }
  __syncthreads();
  uint32_t res = inc - v + warp_tot[w];
  *total = warp_tot[32];
  __syncthreads();
  return res;
}

// Eight consecutive counts of one thread (two 16-byte loads when the tile is full).
__device__ __forceinline__ void load8(const uint32_t* __restrict__ count, int nb, int base,
                                      uint32_t c[kScanItems]) {
  if (base + kScanItems <= nb) {
    uint4 a = *reinterpret_cast<const uint4*>(count + base);
    uint4 b = *reinterpret_cast<const uint4*>(count + base + 4);
    c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
    c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
  } else {
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) c[k] = base + k < nb ? count[base + k] : 0u;
  }
}

__global__ void k_scan_reduce(const uint32_t* __restrict__ count, int nb, uint32_t* tile_sums) {
  pdl_wait();
  int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  uint32_t c[kScanItems];
  load8(count, nb, base, c);
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) s += c[k];
  uint32_t tot;
  block_excl_scan(s, &tot);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// cstart[i] = exclusive prefix of count; count is reset to zero for the next binning.
// Filled blocks (count > 0) are appended to the filled list (warp-aggregated; the
// list's order is irrelevant to every consumer).
__global__ void k_scan_apply(uint32_t* __restrict__ count, int nb, const uint32_t* __restrict__ tile_sums,
                             uint32_t* __restrict__ cstart, uint32_t* __restrict__ filled,
                             Ctl* ctl) {
  pdl_wait();
  int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  uint32_t c[kScanItems];
  load8(count, nb, base, c);
  uint32_t s = 0;
  int nf = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    s += c[k];
    nf += c[k] ? 1 : 0;
  }
  // this tile's offset: the sum of the preceding tiles' totals (read by every CTA)
  uint32_t pre = 0;
  {
    uint32_t ps = 0;
    for (int k = threadIdx.x; k < (int)blockIdx.x; k += blockDim.x) ps += tile_sums[k];
    block_excl_scan(ps, &pre);
  }
  uint32_t tot;
  uint32_t ex = block_excl_scan(s, &tot) + pre;
  uint32_t o[kScanItems];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    o[k] = ex;
    ex += c[k];
  }
  if (base + kScanItems <= nb) {
    *reinterpret_cast<uint4*>(cstart + base) = make_uint4(o[0], o[1], o[2], o[3]);
    *reinterpret_cast<uint4*>(cstart + base + 4) = make_uint4(o[4], o[5], o[6], o[7]);
    *reinterpret_cast<uint4*>(count + base) = make_uint4(0u, 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(count + base + 4) = make_uint4(0u, 0u, 0u, 0u);
  } else {
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
      if (base + k < nb) {
        cstart[base + k] = o[k];
        count[base + k] = 0u;
      }
  }
  // the thread holding the last element writes the grand total
  if (base <= nb - 1 && nb - 1 < base + kScanItems) cstart[nb] = ex;
  if (filled) {   // one atomic per CTA on the list counter
    __shared__ uint32_t fbase;
    uint32_t ftot;
    const uint32_t fpre = block_excl_scan((uint32_t)nf, &ftot);
    if (threadIdx.x == 0) fbase = ftot ? (uint32_t)atomicAdd(&ctl->n_filled, (int)ftot) : 0u;
    __syncthreads();
    uint32_t pos = fbase + fpre;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
      if (c[k]) filled[pos++] = (uint32_t)(base + k);
  }
}

__global__ void k_scatter(int n, int nb, const uint32_t* __restrict__ key,
                          const uint32_t* __restrict__ slot, const uint32_t* __restrict__ uid,
                          const uint32_t* __restrict__ cstart, uint32_t* __restrict__ tkey,
                          uint32_t* __restrict__ tuid, uint32_t* __restrict__ tsrc, Ctl* ctl) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t b = key[i];
  if (b >= (uint32_t)nb) {
    check_failed(ctl, kChkScatter, b);
    return;
  }
  uint32_t q = cstart[b] + slot[i];
  if (q >= (uint32_t)n || q >= cstart[b + 1]) {
    check_failed(ctl, kChkScatter, q);
    return;
  }
  tkey[q] = b;
  tuid[q] = uid[i];
  tsrc[q] = (uint32_t)i;
}

// Warp-segmented maximum over lanes holding the same block (lanes of one block are
// consecutive); the first lane of each segment merges it into the block's stamped record.
__device__ __forceinline__ void block_max_merge(uint32_t b, bool valid, float val, uint32_t stamp,
                                                unsigned long long* rec) {
  const unsigned full = 0xffffffffu;
  int lane = threadIdx.x & 31;
  unsigned long long tagged = valid ? (((unsigned long long)stamp << 32) | __float_as_uint(val)) : 0ull;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    unsigned long long o = __shfl_down_sync(full, tagged, d);
    uint32_t ob = __shfl_down_sync(full, b, d);
    if (lane + d < 32 && ob == b && o > tagged) tagged = o;
  }
  uint32_t prev = __shfl_up_sync(full, b, 1);
  bool head = valid && (lane == 0 || prev != b);
  if (head) atomicMax(rec + b, tagged);
}

// Order each block's particles by caller index and move every field to its place; the
// fluid pass also merges |v|^2 and |a|^2 into the block maxima (Section 3.1 step 2).
__global__ void k_canon_gather(int n, int nb, int max_per_block, const uint32_t* __restrict__ cstart,
                               const uint32_t* __restrict__ tkey, const uint32_t* __restrict__ tuid,
                               const uint32_t* __restrict__ tsrc, PState src, PState dst,
                               uint32_t* __restrict__ key_out, Ctl* ctl, uint32_t stamp,
                               unsigned long long* bmax_v, unsigned long long* bmax_a) {
  pdl_wait();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t b = 0xffffffffu, s = 0, u = 0;
  bool ok = false;
  if (q < n) {
    b = tkey[q];
    s = tsrc[q];
    u = tuid[q];
    ok = b < (uint32_t)nb && s < (uint32_t)n;
    if (!ok) {
      check_failed(ctl, kChkGather, b < (uint32_t)nb ? s : b);
      b = 0xffffffffu;
    }
  }
  // the payload loads do not depend on the in-block rank: issue them first
  float4 px = make_float4(0.f, 0.f, 0.f, 0.f), pv = px, pa = px, pap = px;
  float prho = 0.f, pprs = 0.f, perr = 0.f;
  int32_t pkl = 0, pval = 0, plev = 0, pnbr = 0;
  if (ok) {
    px = src.x[s];
    if (src.v) {
      pv = src.v[s];
      pa = src.a[s];
      prho = src.rho[s];
      pprs = src.prs[s];
      pkl = src.klast[s];
      pval = src.valid[s];
      plev = src.level[s];
      pnbr = src.nbr[s];
      if (src.ap) {
        pap = src.ap[s];
        perr = src.err[s];
      }
    }
  }
  if (bmax_v) {  // every lane reaches the shuffles of block_max_merge
    float v2 = 0.f, a2 = 0.f;
    if (ok) {
      const float ax = pa.x + pap.x, ay = pa.y + pap.y, az = pa.z + pap.z;  // PCISPH: total
      v2 = pv.x * pv.x + pv.y * pv.y + pv.z * pv.z;
      a2 = src.ap ? ax * ax + ay * ay + az * az : pa.x * pa.x + pa.y * pa.y + pa.z * pa.z;
    }
    block_max_merge(b, ok, v2, stamp, bmax_v);
    block_max_merge(b, ok, a2, stamp, bmax_a);
  }
  if (!ok) return;
  const uint32_t beg = cstart[b], end = cstart[b + 1];
  if (q == (int)beg && (int)(end - beg) > max_per_block) set_status(ctl, RTS_ERR_CAPACITY);
  uint32_t rank = 0;
  for (uint32_t r = beg; r < end; ++r) rank += (tuid[r] < u) ? 1u : 0u;
  const uint32_t f = beg + rank;
  if (f >= end) {
    check_failed(ctl, kChkGather, f);
    return;
  }
  key_out[f] = b;
  dst.uid[f] = u;
  dst.x[f] = px;
  if (src.v) {
    dst.v[f] = pv;
    dst.a[f] = pa;
    dst.rho[f] = prho;
    dst.prs[f] = pprs;
    dst.klast[f] = pkl;
    dst.valid[f] = pval;
    dst.level[f] = plev;
    dst.nbr[f] = pnbr;
    if (src.ap) {
      dst.ap[f] = pap;
      dst.err[f] = perr;
    }
  }
}

// Exclusive scan of nb block counts into cstart (nb + 1 entries); the counts are reset
// to zero.  tile_sums holds ceil(nb / 2048) entries.
void scan_block_counts(uint32_t* count, int nb, uint32_t* tile_sums, uint32_t* cstart,
                       cudaStream_t stream) {
  int ntiles = (nb + kScanTile - 1) / kScanTile;
  launch_pdl(stream, k_scan_reduce, ntiles, kScanThreads, 0, count, nb, tile_sums);
  launch_pdl(stream, k_scan_apply, ntiles, kScanThreads, 0, count, nb, tile_sums, cstart,
             (uint32_t*)nullptr, (Ctl*)nullptr);
}

// Exclusive scan of the block counts into cstart (tile totals, then each tile adds the
// totals before it); the filled list is appended to (its counter was reset by the key pass).
static rts_status scan_counts(rts_ctx* c, uint32_t* filled) {
  int nb = c->dp.nblocks;
  int ntiles = (nb + kScanTile - 1) / kScanTile;
  launch_pdl(c->stream, k_scan_reduce, ntiles, kScanThreads, 0, c->count, nb, c->tile_sums);
  launch_pdl(c->stream, k_scan_apply, ntiles, kScanThreads, 0, c->count, nb, c->tile_sums,
             c->cstart, filled, c->ctl);
  return RTS_OK;
}

// Next stamp; on wrap-around every stamped record is cleared once.
static void next_stamp(rts_ctx* c) {
  if (++c->stamp >= (1u << 24)) {
    size_t nb = (size_t)c->dp.nblocks;
    cudaMemsetAsync(c->bmax_v, 0, sizeof(unsigned long long) * nb, c->stream);
    cudaMemsetAsync(c->bmax_a, 0, sizeof(unsigned long long) * nb, c->stream);
    cudaMemsetAsync(c->raw, 0, sizeof(uint32_t) * nb, c->stream);
    cudaMemsetAsync(c->blevel, 0, sizeof(uint32_t) * nb, c->stream);
    cudaMemsetAsync(c->actflag, 0, sizeof(uint32_t) * nb, c->stream);
    // two passes in a row now share a parity: clear the slots of the kept-sort passes
    cudaMemsetAsync(c->ctl->n_filled_light, 0, sizeof(c->ctl->n_filled_light), c->stream);
    cudaMemsetAsync(c->ctl->n_near, 0, sizeof(c->ctl->n_near), c->stream);
    cudaMemsetAsync(c->ctl->disp_bits, 0, sizeof(c->ctl->disp_bits), c->stream);
    c->stamp = 1;
  }
}

// A substep that keeps the previous sort (see k_predict_light).
rts_status launch_bin_light(rts_ctx* c, float dt) {
  int n = c->n;
  const int g = (n + kLightThreads * kLightItems - 1) / (kLightThreads * kLightItems);
  note_launch(c, 1);
  next_stamp(c);
  launch_pdl(c->stream, k_predict_light, g, kLightThreads, 0, c->dp, n, c->s.x, c->s.v, c->s.a,
             dt, c->key, c->key_cur, c->ctl, c->pend_mode, (int)c->pend_k1, c->cflag, c->anew,
             c->s.klast, c->s.uid, c->stamp, c->bmax_v, c->bmax_a, c->cstart, c->filled_new,
             c->near_list);
  c->pend_mode = kPendNone;
  return RTS_OK;
}

rts_status launch_bin(rts_ctx* c, float dt) {
  c->light_ok = 1;   // the arrays are block-sorted by c->key from here on
  c->gmax_ok = 0;    // the key pass clears the maxima of the global step size
  int n = c->n;
  if (n == 0) {
    next_stamp(c);
    cudaMemsetAsync(c->cstart, 0, sizeof(uint32_t) * ((size_t)c->dp.nblocks + 1), c->stream);
    cudaMemsetAsync(&c->ctl->n_filled, 0, sizeof(int), c->stream);
    return RTS_OK;
  }
  int tb = 256, g = (n + tb - 1) / tb;
  note_launch(c, 5);
  next_stamp(c);
  // the binning chain is launched with programmatic dependencies (each kernel waits for
  // the previous one before its first access; see launch_pdl)
  launch_pdl(c->stream, k_predict_key, g, tb, 0, c->dp, n, c->s.x, c->s.v, c->s.a, dt, c->key,
             c->slot, c->count, c->ctl, c->pend_mode, (int)c->pend_k1, c->cflag, c->anew,
             c->s.klast, c->s.uid);
  c->pend_mode = kPendNone;
  scan_counts(c, c->filled);
  launch_pdl(c->stream, k_scatter, g, tb, 0, n, c->dp.nblocks, c->key, c->slot, c->s.uid,
             c->cstart, c->key_tmp, c->tmp_uid, c->tmp_src, c->ctl);
  launch_pdl(c->stream, k_canon_gather, g, tb, 0, n, c->dp.nblocks, c->dp.max_per_block,
             c->cstart, c->key_tmp, c->tmp_uid, c->tmp_src, c->s, c->s2, c->key, c->ctl,
             c->stamp, c->bmax_v, c->bmax_a);
  PState t = c->s;
  c->s = c->s2;
  c->s2 = t;
  return RTS_OK;
}

// Boundary particles are static: sort them once by (block, index) into xb / bcstart.
__global__ void k_iota(int n, uint32_t* u) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) u[i] = (uint32_t)i;
}

rts_status launch_bin_boundary(rts_ctx* c, const float4* xb_unsorted, int nb) {
  if (nb == 0) {
    cudaMemsetAsync(c->bcstart, 0, sizeof(uint32_t) * ((size_t)c->dp.nblocks + 1), c->stream);
    return RTS_OK;
  }
  uint32_t *key, *slot, *tkey, *tuid, *tsrc, *uid, *uid2;
  size_t sz = sizeof(uint32_t) * (size_t)nb;
  cudaError_t e = cudaSuccess;
  uint32_t** bufs[] = {&key, &slot, &tkey, &tuid, &tsrc, &uid, &uid2};
  for (auto b : bufs)
    if (e == cudaSuccess) e = cudaMalloc((void**)b, sz);
  if (e != cudaSuccess) {
    cuda_err(c, e, "boundary binning buffers");
    return RTS_ERR_OOM;
  }
  int tb = 256, g = (nb + tb - 1) / tb;
  k_iota<<<g, tb, 0, c->stream>>>(nb, uid);
  k_predict_key<<<g, tb, 0, c->stream>>>(c->dp, nb, const_cast<float4*>(xb_unsorted), nullptr,
                                          nullptr, 0.0f, key, slot, c->count, c->ctl, kPendNone, 0,
                                          nullptr, nullptr, nullptr, uid);
  uint32_t* save = c->cstart;
  c->cstart = c->bcstart;
  scan_counts(c, nullptr);
  c->cstart = save;
  k_scatter<<<g, tb, 0, c->stream>>>(nb, c->dp.nblocks, key, slot, uid, c->bcstart, tkey, tuid,
                                      tsrc, c->ctl);
  PState src{}, dst{};
  src.x = const_cast<float4*>(xb_unsorted);
  src.uid = uid;
  dst.x = c->xb;
  dst.uid = uid2;
  k_canon_gather<<<g, tb, 0, c->stream>>>(nb, c->dp.nblocks, 1 << 30, c->bcstart, tkey, tuid, tsrc,
                                           src, dst, key, c->ctl, 0u, nullptr, nullptr);
  cudaMemcpyAsync(c->buid, uid2, sz, cudaMemcpyDeviceToDevice, c->stream);
  e = cudaStreamSynchronize(c->stream);
  for (auto b : bufs) cudaFree(*b);
  if (e != cudaSuccess) {
    cuda_err(c, e, "boundary binning");
    return RTS_ERR_CUDA;
  }
  return RTS_OK;
}

}  // namespace rts
