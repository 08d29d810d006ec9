// rts_pcisph_dev.cuh - per-particle device code of PCISPH (Algorithm 3), shared by the
// single-scene kernels (rts_pcisph.cu) and the batched work-queue kernels
// (rts_batch.cu), so both evaluate every particle with the same instructions and give
// the same bits.
#pragma once

#include "rts_internal.cuh"

namespace rts {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr uint32_t kBnd = 0x80000000u;
constexpr int kModeSched = 0, kModeGlobal = 1, kModeLocal = 2;

// cubic spline W(q) and dW/dr(q), q = r / h
__device__ __forceinline__ float pW(const DevParams& P, float q) {
  if (q < 1.0f) return P.sigma * (1.0f + q * q * (-1.5f + 0.75f * q));
  float t = 2.0f - q;
  return q < 2.0f ? 0.25f * P.sigma * t * t * t : 0.0f;
}

__device__ __forceinline__ float pdW(const DevParams& P, float q) {
  if (q < 1.0f) return P.sigma_h * q * (-3.0f + 2.25f * q);
  float t = 2.0f - q;
  return q < 2.0f ? -0.75f * P.sigma_h * t * t : 0.0f;
}

__device__ __forceinline__ double pnorm2(float x, float y, float z) {
  double dx = x, dy = y, dz = z;
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Does region L have a correction turn in iteration `row` of minor step j?
__device__ __forceinline__ bool has_turn(const DevParams& P, int mode, int row, int j, int L) {
  return mode == kModeGlobal || (mode == kModeSched && row <= P.sched[L][j]);
}

// x* = x + dt v*, v* = v + dt (a_np + a_p); the w lane carries p / rho^2 of the particle's
// current pressure and density (its pressure-force coefficient as a neighbour), which the
// density pass refreshes for the particles whose pressure it updates.
__device__ __forceinline__ float4 predict_one(const DevParams& P, const PState& s, int i) {
  float4 x = s.x[i], v = s.v[i], a = s.a[i], pa = s.ap[i];
  float dt = P.dt_b;
  float vx = v.x + dt * (a.x + pa.x), vy = v.y + dt * (a.y + pa.y), vz = v.z + dt * (a.z + pa.z);
  const float rho = s.rho[i];
  return make_float4(x.x + dt * vx, x.y + dt * vy, x.z + dt * vz, s.prs[i] / (rho * rho));
}

// |x| / h of a separation with squared length d2 > 0, and 1 / |x| (no divide, no IEEE sqrt)
__device__ __forceinline__ float inv_len(float d2) { return rsqrtf(d2); }

// The list-walking passes give each particle a group of LANES consecutive lanes: lane
// sub of the group takes list entries sub, sub + LANES, ...; the group's partial sums are
// combined by shuffles and lane 0 of the group writes.  Every lane of the warp calls
// these functions (lanes without a particle with valid = false), since the shuffles span
// the full warp.  Iterations in which every particle takes part use kPLanes lanes per
// particle (more loads in flight per particle); sparse ones (a few regions, S_e, R_ob)
// one lane, so that scanning the non-participants stays cheap.  The choice depends only
// on the iteration's mode and row, so a scene gives the same bits alone or in a batch.
constexpr int kPLanes = 4;

template <int LANES>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = 1; o < LANES; o <<= 1) v += __shfl_xor_sync(kFullMask, v, o);
  return v;
}

// rho* = m (W(0) + sum W(|x*_i - x*_j|)), err = max(0, rho* - rho0) / rho0,
// p += delta max(0, rho* - rho0)
template <int LANES>
__device__ __forceinline__ void pdensity_group(const DevParams& P, const PState& s, int i,
                                               bool valid, int sub, float4* xs,
                                               const float4* __restrict__ xb,
                                               const uint32_t* __restrict__ nbl) {
  float w = 0.f;
  if (valid) {
    const float4 xi = xs[i];
    const uint32_t* list = nbl + (size_t)i * P.nbl_cap;
    const int cnt = s.nbr[i];
    for (int e = sub; e < cnt; e += LANES) {
      const uint32_t j = list[e];
      const float4 xj = (j & kBnd) ? xb[j & ~kBnd] : xs[j];
      const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
      const float d2 = dx * dx + dy * dy + dz * dz;
      w += pW(P, d2 > 0.f ? d2 * inv_len(d2) * P.inv_h : 0.f);
    }
  }
  w = group_sum<LANES>(w);
  if (valid && sub == 0) {
    const float rho = P.m * (P.sigma + w);   // W(0): the particle itself
    const float comp = fmaxf(0.f, rho - P.rho0);
    const float p = s.prs[i] + P.delta * comp;
    s.rho[i] = rho;
    s.err[i] = comp * P.inv_rho0;
    s.prs[i] = p;
    xs[i].w = p / (rho * rho);
  }
}

// a_p = -m sum (p_i/rho_i*^2 + p_j/rho_j*^2) grad W(x*_ij) with the coefficients from the
// w lanes of x*; boundary neighbours contribute the p_i/rho_i*^2 term only.
template <int LANES>
__device__ __forceinline__ void ppressure_group(const DevParams& P, const PState& s, int i,
                                                bool valid, int sub,
                                                const float4* __restrict__ xs,
                                                const float4* __restrict__ xb,
                                                const uint32_t* __restrict__ nbl) {
  float ax = 0.f, ay = 0.f, az = 0.f;
  if (valid) {
    const float4 xi = xs[i];
    const float ci = xi.w;   // p_i / rho_i^2
    const uint32_t* list = nbl + (size_t)i * P.nbl_cap;
    const int cnt = s.nbr[i];
    for (int e = sub; e < cnt; e += LANES) {
      const uint32_t j = list[e];
      float4 xj;
      float cj;
      if (j & kBnd) {
        xj = xb[j & ~kBnd];
        cj = 0.f;
      } else {
        xj = xs[j];
        cj = xj.w;
      }
      const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
      const float d2 = dx * dx + dy * dy + dz * dz;
      if (!(d2 > 0.f)) continue;
      const float id = inv_len(d2);
      const float f = pdW(P, d2 * id * P.inv_h) * id;
      const float sc = -P.m * (ci + cj) * f;
      ax += sc * dx;
      ay += sc * dy;
      az += sc * dz;
    }
  }
  ax = group_sum<LANES>(ax);
  ay = group_sum<LANES>(ay);
  az = group_sum<LANES>(az);
  if (valid && sub == 0) s.ap[i] = make_float4(ax, ay, az, 0.f);
}

// R_ob (Section 5.4): is filled block b outside R_e and bordering R_e or a smaller region?
__device__ __forceinline__ uint8_t observed_one(const DevParams& P, uint32_t b,
                                                const int32_t* __restrict__ preg,
                                                const uint8_t* __restrict__ in_re) {
  uint8_t o = 0;
  if (!in_re[b]) {
    int L = preg[b];
    int bx = b % P.nx, r = b / P.nx, by = r % P.ny, bz = r / P.ny;
    for (int dz = -1; dz <= 1 && !o; ++dz) {
      int cz = bz + dz;
      if (cz < 0 || cz >= P.nz) continue;
      for (int dy = -1; dy <= 1 && !o; ++dy) {
        int cy = by + dy;
        if (cy < 0 || cy >= P.ny) continue;
        for (int dx = -1; dx <= 1 && !o; ++dx) {
          int cx = bx + dx;
          if (cx < 0 || cx >= P.nx || (!dx && !dy && !dz)) continue;
          size_t c = ((size_t)cz * P.ny + cy) * P.nx + cx;
          int Lc = preg[c];
          if (Lc < 0) continue;
          if (in_re[c] || Lc < L) o = 1;
        }
      }
    }
  }
  return o;
}

// Latest error as a fixed-point summand (2^-32 units): sums are exact and independent of
// the order in which threads add them.  floor(e 2^32 + 1/2) for e >= 0, formed in
// integers from e = m 2^(E - 150) (the value of (unsigned long long)((double)e * 2^32 +
// 0.5), without FP64; saturated for e >= 2^40).
__device__ __forceinline__ unsigned long long err_fixed(float e) {
  if (!(e > 0.f)) return 0ull;
  const unsigned u = __float_as_uint(e);
  int E = (int)(u >> 23);
  unsigned long long m = u & 0x7fffffu;
  if (E == 0) E = 1; else m |= 0x800000u;   // subnormal / normal
  const int sh = E - 118;                  // e 2^32 = m 2^sh
  if (sh > 40) return ~0ull;
  if (sh >= 0) return m << sh;
  if (sh < -25) return 0ull;               // e 2^32 < 1/2
  return (m + (1ull << (-sh - 1))) >> (-sh);
}

}  // namespace rts
