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

// x* = x + dt v*, v* = v + dt (a_np + a_p)
__device__ __forceinline__ float4 predict_one(const DevParams& P, const PState& s, int i) {
  float4 x = s.x[i], v = s.v[i], a = s.a[i], pa = s.ap[i];
  float dt = P.dt_b;
  float vx = v.x + dt * (a.x + pa.x), vy = v.y + dt * (a.y + pa.y), vz = v.z + dt * (a.z + pa.z);
  return make_float4(x.x + dt * vx, x.y + dt * vy, x.z + dt * vz, 0.f);
}

// rho* = m W(0) + sum m W(|x*_i - x*_j|), err = max(0, rho* - rho0) / rho0,
// p += delta max(0, rho* - rho0)
__device__ __forceinline__ void pdensity_one(const DevParams& P, const PState& s, int i,
                                             const float4* __restrict__ xs,
                                             const float4* __restrict__ xb,
                                             const uint32_t* __restrict__ nbl) {
  float4 xi = xs[i];
  float w = P.sigma;  // W(0): the particle itself
  const uint32_t* list = nbl + (size_t)i * P.nbl_cap;
  int cnt = s.nbr[i];
  for (int e = 0; e < cnt; ++e) {
    uint32_t j = list[e];
    float4 xj = (j & kBnd) ? xb[j & ~kBnd] : xs[j];
    float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
    float d2 = dx * dx + dy * dy + dz * dz;
    w += pW(P, sqrtf(d2) * P.inv_h);
  }
  float rho = P.m * w;
  float comp = fmaxf(0.f, rho - P.rho0);
  float p = s.prs[i] + P.delta * comp;
  s.rho[i] = rho;
  s.err[i] = comp * P.inv_rho0;
  s.prs[i] = p;
}

// a_p = -m sum (p_i/rho_i*^2 + p_j/rho_j*^2) grad W(x*_ij); boundary neighbours contribute
// the p_i/rho_i*^2 term only.
__device__ __forceinline__ void ppressure_one(const DevParams& P, const PState& s, int i,
                                              const float4* __restrict__ xs,
                                              const float4* __restrict__ xb,
                                              const uint32_t* __restrict__ nbl) {
  float4 xi = xs[i];
  const float ri = s.rho[i];
  float ci = s.prs[i] / (ri * ri);
  float ax = 0.f, ay = 0.f, az = 0.f;
  const uint32_t* list = nbl + (size_t)i * P.nbl_cap;
  int cnt = s.nbr[i];
  for (int e = 0; e < cnt; ++e) {
    uint32_t j = list[e];
    float4 xj;
    float cj;
    if (j & kBnd) {
      xj = xb[j & ~kBnd];
      cj = 0.f;
    } else {
      xj = xs[j];
      const float rj = s.rho[j];
      cj = s.prs[j] / (rj * rj);
    }
    float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
    float d2 = dx * dx + dy * dy + dz * dz;
    if (!(d2 > 0.f)) continue;
    float d = sqrtf(d2);
    float f = pdW(P, d * P.inv_h) / d;
    float sc = -P.m * (ci + cj) * f;
    ax += sc * dx;
    ay += sc * dy;
    az += sc * dz;
  }
  s.ap[i] = make_float4(ax, ay, az, 0.f);
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
// the order in which threads add them.
__device__ __forceinline__ unsigned long long err_fixed(float e) {
  return (unsigned long long)((double)e * 4294967296.0 + 0.5);
}

}  // namespace rts
