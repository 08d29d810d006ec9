// rts_diff.cu - differentiable WCSPH rollout and its hand-written adjoint.
//
// The rollout is global constant stepping at dt_b (every particle active every step)
// with the Serna predictor-corrector of Section 4.1 and the WCSPH physics of the regional
// path (summation density, Tait pressure clamped at 0, symmetric pressure force, artificial
// viscosity, gravity, static boundary particles, the container correction): priming
// evaluation a_0 = A(x_0, v_0); per step x~ = x + v dt + a dt^2 / 2, v~ = v + a dt, the
// container, a' = A(x~, v~), x <- x~ + (a' - a) dt^2 / 6, v <- v~ + (a' - a) dt / 2, a <- a'.
// After the last step rho_T = rho(x_T).  Particles stay in the caller's order; each
// evaluation builds a cell list (block grid of the parameters, cells ranked by particle
// index, so every pass is deterministic and a recomputed step repeats the forward bit for
// bit).
//
// Backward: reverse mode written out.  For an ordered pair (i, j) of i's list the scalar
// S = P_i + P_j + Pi_ij (P = p / rho^2) and G = W'(r)/r x_ij enter a_i with -m S G and a_j
// with +m S G; with w = abar_i - abar_j, Sbar = -m G . w and Gbar = -m S w.  Pass A
// gathers Pbar_i = sum Sbar, the viscosity's density terms and the stiffness and viscosity
// adjoints, giving rhobar_i; pass B gathers the position and velocity adjoints of every
// pair (kernel gradient, the density sums of both particles, viscosity).  Checkpoints of
// (x, v, a) every ckpt steps; a segment is recomputed forward with its evaluation points,
// neighbour lists and container masks recorded, then reversed.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "rts_internal.cuh"

void rts_set_global_error(const char* msg);  // rts_api.cu

struct rts_diff {
  rts_params p;
  rts::DevParams dp;
  int n, nb, steps, ckpt, nseg, cap;
  cudaStream_t stream;
  char err[512];
  int sticky;
  float B, alpha;          // parameters of the last forward
  bool have_forward;
  // static boundary, sorted by block once
  float4* xb;
  uint32_t* bcstart;
  // cell list of one evaluation
  uint32_t *key, *count, *cstart, *tile_sums, *perm_tmp, *perm;
  // state and checkpoints (caller order)
  float4 *x, *v, *a, *xt, *vt, *an;
  float4 *ck_x, *ck_v, *ck_a;   // (nseg + 1) x n
  float *rho, *prs;
  uint32_t* list;               // n x cap of the current evaluation
  int* nn;
  // records of a segment: ckpt evaluations
  float4 *rec_xt, *rec_vt;
  float *rec_rho, *rec_prs;
  uint32_t* rec_list;
  int* rec_nn;
  uint8_t* rec_mask;
  // adjoints
  float4 *xbar, *vbar, *abar, *anbar, *akbar;
  float* rhobar;
  double* red;                  // Bbar, alphabar
  double* h_red;
  rts::Ctl* ctl;
  rts::Ctl* h_ctl;
};

namespace rts {
namespace {

constexpr uint32_t kBnd = 0x80000000u;
constexpr int kT = 256;

inline int grid_of(int n) { return (n + kT - 1) / kT; }

__device__ __forceinline__ void spline3(const DevParams& P, float r, float& W, float& dW, float& d2W) {
  const float q = r * P.inv_h;
  const float sh2 = P.sigma_h * P.inv_h;
  if (q < 1.f) {
    W = P.sigma * (1.f + q * q * (-1.5f + 0.75f * q));
    dW = P.sigma_h * q * (-3.f + 2.25f * q);
    d2W = sh2 * (-3.f + 4.5f * q);
  } else if (q < 2.f) {
    const float t = 2.f - q;
    W = 0.25f * P.sigma * t * t * t;
    dW = -0.75f * P.sigma_h * t * t;
    d2W = 1.5f * sh2 * t;
  } else {
    W = dW = d2W = 0.f;
  }
}

__device__ __forceinline__ float tait_p(const DevParams& P, float B, float rho) {
  const float r = rho * P.inv_rho0;
  float rg;
  if (P.gamma_is_7) {
    const float r2 = r * r, r4 = r2 * r2;
    rg = r4 * r2 * r;
  } else {
    rg = powf(r, P.gamma);
  }
  const float p = B * (rg - 1.f);
  return P.no_clamp ? p : fmaxf(0.f, p);
}

// ------------------------------------------------------------------ cell list ---

__global__ void kd_key(DevParams P, int n, const float4* __restrict__ x, uint32_t* __restrict__ key,
                       uint32_t* __restrict__ count, Ctl* ctl) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int bad = 0;
  uint32_t b = block_key(P, x[i], &bad);
  if (bad) {
    if (atomicCAS(&ctl->bad_set, 0, 1) == 0) {
      ctl->bad_uid = (unsigned)i;
      ctl->bad_x = x[i].x;
      ctl->bad_y = x[i].y;
      ctl->bad_z = x[i].z;
    }
    set_status(ctl, RTS_ERR_DOMAIN);
    b = 0;
  }
  key[i] = b;
  atomicAdd(&count[b], 1u);
}

__global__ void kd_place(int n, const uint32_t* __restrict__ key, const uint32_t* __restrict__ cstart,
                         uint32_t* __restrict__ count, uint32_t* __restrict__ perm_tmp) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t b = key[i];
  perm_tmp[cstart[b] + atomicAdd(&count[b], 1u)] = (uint32_t)i;
}

// Rank within the cell by particle index (deterministic order); resets the counters.
__global__ void kd_rank(int n, const uint32_t* __restrict__ key, const uint32_t* __restrict__ cstart,
                        uint32_t* __restrict__ count, const uint32_t* __restrict__ perm_tmp,
                        uint32_t* __restrict__ perm) {
  pdl_wait();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const uint32_t i = perm_tmp[q];
  const uint32_t b = key[i];
  const uint32_t beg = cstart[b], end = cstart[b + 1];
  uint32_t rank = 0;
  for (uint32_t r = beg; r < end; ++r) rank += perm_tmp[r] < i ? 1u : 0u;
  perm[beg + rank] = i;
  if ((uint32_t)q == beg) count[b] = 0;
}

__global__ void kd_gather_sorted(int n, const uint32_t* __restrict__ perm, const float4* __restrict__ in,
                                 float4* __restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) out[q] = in[perm[q]];
}

// ---------------------------------------------------------------- evaluation ---

// Neighbour list, density and pressure of every particle (thread per particle; the 27
// cells of its block, fluid through the cell list, boundary from the sorted array).
__global__ void kd_density(DevParams P, int n, float B, const float4* __restrict__ x,
                           const uint32_t* __restrict__ key, const uint32_t* __restrict__ cstart,
                           const uint32_t* __restrict__ perm, const float4* __restrict__ xb,
                           const uint32_t* __restrict__ bcstart, int cap, float* __restrict__ rho,
                           float* __restrict__ prs, uint32_t* __restrict__ list,
                           int* __restrict__ nn, Ctl* ctl) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 xi = x[i];
  const uint32_t b = key[i];
  const int bx = b % P.nx, rr = b / P.nx, by = rr % P.ny, bz = rr / P.ny;
  const int xlo = bx > 0 ? bx - 1 : 0, xhi = bx + 1 < P.nx ? bx + 1 : P.nx - 1;
  float sum = P.sigma;   // the particle itself, W(0)
  int cnt = 0;
  uint32_t* li = list + (size_t)i * cap;
  for (int dz = -1; dz <= 1; ++dz) {
    const int cz = bz + dz;
    if (cz < 0 || cz >= P.nz) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int cy = by + dy;
      if (cy < 0 || cy >= P.ny) continue;
      const uint32_t row = ((uint32_t)cz * P.ny + cy) * P.nx;
      for (uint32_t q = cstart[row + xlo]; q < cstart[row + xhi + 1]; ++q) {
        const uint32_t j = perm[q];
        if (j == (uint32_t)i) continue;
        const float4 xj = x[j];
        const float dx = xi.x - xj.x, dy2 = xi.y - xj.y, dz2 = xi.z - xj.z;
        const float d2 = dx * dx + dy2 * dy2 + dz2 * dz2;
        if (d2 < P.r2) {
          float W, dW, d2W;
          spline3(P, sqrtf(d2), W, dW, d2W);
          sum += W;
          if (cnt < cap) li[cnt] = j;
          ++cnt;
        }
      }
      for (uint32_t q = bcstart[row + xlo]; q < bcstart[row + xhi + 1]; ++q) {
        const float4 xj = xb[q];
        const float dx = xi.x - xj.x, dy2 = xi.y - xj.y, dz2 = xi.z - xj.z;
        const float d2 = dx * dx + dy2 * dy2 + dz2 * dz2;
        if (d2 < P.r2) {
          float W, dW, d2W;
          spline3(P, sqrtf(d2), W, dW, d2W);
          sum += W;
          if (cnt < cap) li[cnt] = q | kBnd;
          ++cnt;
        }
      }
    }
  }
  if (cnt > cap) set_status(ctl, RTS_ERR_CAPACITY);
  const float r = P.m * sum;
  rho[i] = r;
  prs[i] = tait_p(P, B, r);
  nn[i] = cnt < cap ? cnt : cap;
}

// a = g - sum_j m (P_i + P_j + Pi_ij) W'(r)/r x_ij over the list (boundary: P_j = 0,
// rho_j = rho_i, v_j = 0).
__global__ void kd_force(DevParams P, int n, float K, const float4* __restrict__ x,
                         const float4* __restrict__ v, const float* __restrict__ rho,
                         const float* __restrict__ prs, const float4* __restrict__ xb,
                         const uint32_t* __restrict__ list, const int* __restrict__ nn, int cap,
                         float4* __restrict__ a) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 xi = x[i], vi = v[i];
  const float ri = rho[i], Pi = prs[i] / (ri * ri);
  float ax = P.gx, ay = P.gy, az = P.gz;
  const uint32_t* li = list + (size_t)i * cap;
  for (int e = 0; e < nn[i]; ++e) {
    const uint32_t jg = li[e];
    float4 xj, vj;
    float rj, Pj;
    if (jg & kBnd) {
      xj = xb[jg & ~kBnd];
      vj = make_float4(0.f, 0.f, 0.f, 0.f);
      rj = ri;
      Pj = 0.f;
    } else {
      xj = x[jg];
      vj = v[jg];
      rj = rho[jg];
      Pj = prs[jg] / (rj * rj);
    }
    const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
    const float d2 = dx * dx + dy * dy + dz * dz;
    if (d2 <= 0.f) continue;
    const float r = sqrtf(d2);
    float W, dW, d2W;
    spline3(P, r, W, dW, d2W);
    const float f = dW / r;
    const float u = (vi.x - vj.x) * dx + (vi.y - vj.y) * dy + (vi.z - vj.z) * dz;
    const float visc = u < 0.f ? -(K / (ri + rj)) * u / (d2 + P.eps_h2) : 0.f;
    const float s = -P.m * (Pi + Pj + visc) * f;
    ax += s * dx;
    ay += s * dy;
    az += s * dz;
  }
  a[i] = make_float4(ax, ay, az, 0.f);
}

// Predictor and the container; mask bits: 1 << k the coordinate k was clamped,
// 8 << k its velocity was zeroed.
__global__ void kd_predict(DevParams P, int n, float dt, const float4* __restrict__ x,
                           const float4* __restrict__ v, const float4* __restrict__ a,
                           float4* __restrict__ xt, float4* __restrict__ vt,
                           uint8_t* __restrict__ mask) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 xi = x[i], vi = v[i], ai = a[i];
  const float h = 0.5f * dt * dt;
  float px[3] = {xi.x + vi.x * dt + ai.x * h, xi.y + vi.y * dt + ai.y * h, xi.z + vi.z * dt + ai.z * h};
  float pv[3] = {vi.x + ai.x * dt, vi.y + ai.y * dt, vi.z + ai.z * dt};
  uint8_t m = 0;
  if (P.wall_project) {
    for (int k = 0; k < 3; ++k) {
      if (px[k] < P.wlo[k]) {
        px[k] = P.wlo[k];
        m |= (uint8_t)(1u << k);
        if (pv[k] < 0.f) {
          pv[k] = 0.f;
          m |= (uint8_t)(8u << k);
        }
      } else if (px[k] > P.whi[k]) {
        px[k] = P.whi[k];
        m |= (uint8_t)(1u << k);
        if (pv[k] > 0.f) {
          pv[k] = 0.f;
          m |= (uint8_t)(8u << k);
        }
      }
    }
  }
  xt[i] = make_float4(px[0], px[1], px[2], 0.f);
  vt[i] = make_float4(pv[0], pv[1], pv[2], 0.f);
  if (mask) mask[i] = m;
}

__global__ void kd_correct(int n, float dt, const float4* __restrict__ xt, const float4* __restrict__ vt,
                           const float4* __restrict__ an, float4* __restrict__ x, float4* __restrict__ v,
                           float4* __restrict__ a) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 p = xt[i], q = vt[i], n1 = an[i], o = a[i];
  const float c1 = dt * dt / 6.f, c2 = 0.5f * dt;
  x[i] = make_float4(p.x + (n1.x - o.x) * c1, p.y + (n1.y - o.y) * c1, p.z + (n1.z - o.z) * c1, 0.f);
  v[i] = make_float4(q.x + (n1.x - o.x) * c2, q.y + (n1.y - o.y) * c2, q.z + (n1.z - o.z) * c2, 0.f);
  a[i] = n1;
}

__global__ void kd_pack(int n, const float* __restrict__ in, float4* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in ? make_float4(in[3 * i], in[3 * i + 1], in[3 * i + 2], 0.f)
                         : make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void kd_unpack(int n, const float4* __restrict__ in, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 q = in[i];
  out[3 * i] = q.x;
  out[3 * i + 1] = q.y;
  out[3 * i + 2] = q.z;
}

// ------------------------------------------------------------------- adjoint ---

// One pair of i's list: positions, velocities, densities and the derived quantities.
struct PairQ {
  float dx, dy, dz, d2, f, d2W, u, D, nu, Pv, S, rs;   // rs = rho_i + rho_j
  float vx, vy, vz;
  bool fluid;
};

__device__ __forceinline__ bool pair_q(const DevParams& P, float K, const float4& xi, const float4& vi,
                                       float ri, float Pi, uint32_t jg, const float4* __restrict__ x,
                                       const float4* __restrict__ v, const float* __restrict__ rho,
                                       const float* __restrict__ prs, const float4* __restrict__ xb,
                                       PairQ& q) {
  float4 xj, vj;
  float rj, Pj;
  q.fluid = !(jg & kBnd);
  if (!q.fluid) {
    xj = xb[jg & ~kBnd];
    vj = make_float4(0.f, 0.f, 0.f, 0.f);
    rj = ri;
    Pj = 0.f;
  } else {
    xj = x[jg];
    vj = v[jg];
    rj = rho[jg];
    Pj = prs[jg] / (rj * rj);
  }
  q.dx = xi.x - xj.x;
  q.dy = xi.y - xj.y;
  q.dz = xi.z - xj.z;
  q.d2 = q.dx * q.dx + q.dy * q.dy + q.dz * q.dz;
  if (q.d2 <= 0.f) return false;
  const float r = sqrtf(q.d2);
  float W, dW;
  spline3(P, r, W, dW, q.d2W);
  q.f = dW / r;
  q.vx = vi.x - vj.x;
  q.vy = vi.y - vj.y;
  q.vz = vi.z - vj.z;
  q.u = q.vx * q.dx + q.vy * q.dy + q.vz * q.dz;
  q.D = q.d2 + P.eps_h2;
  q.rs = ri + rj;
  q.nu = K / q.rs;
  q.Pv = q.u < 0.f ? -q.nu * q.u / q.D : 0.f;
  q.S = Pi + Pj + q.Pv;
  return true;
}

__device__ __forceinline__ void cta_add2(double a, double b, double* red) {
  __shared__ double sa[kT / 32], sb[kT / 32];
  for (int o = 16; o; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sa[threadIdx.x >> 5] = a;
    sb[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      ta += sa[k];
      tb += sb[k];
    }
    if (ta != 0.0) atomicAdd(&red[0], ta);
    if (tb != 0.0) atomicAdd(&red[1], tb);
  }
}

// Pass A: rhobar_i from Pbar_i (= sum of Sbar over i's list) and the viscosity's density
// terms; the stiffness and viscosity adjoints into red[0], red[1].
__global__ void kd_adj_a(DevParams P, int n, float B, float K, float alpha, const float4* __restrict__ x,
                         const float4* __restrict__ v, const float* __restrict__ rho,
                         const float* __restrict__ prs, const float4* __restrict__ xb,
                         const uint32_t* __restrict__ list, const int* __restrict__ nn, int cap,
                         const float4* __restrict__ abar, float* __restrict__ rhobar,
                         double* __restrict__ red) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double bB = 0.0, bA = 0.0;
  if (i < n) {
    const float4 xi = x[i], vi = v[i], ai = abar[i];
    const float ri = rho[i], pi = prs[i], Pi = pi / (ri * ri);
    float Pbar = 0.f, rv = 0.f, al = 0.f;
    const uint32_t* li = list + (size_t)i * cap;
    for (int e = 0; e < nn[i]; ++e) {
      const uint32_t jg = li[e];
      PairQ q;
      if (!pair_q(P, K, xi, vi, ri, Pi, jg, x, v, rho, prs, xb, q)) continue;
      float wx = ai.x, wy = ai.y, wz = ai.z;
      if (q.fluid) {
        const float4 aj = abar[jg];
        wx -= aj.x;
        wy -= aj.y;
        wz -= aj.z;
      }
      const float Sbar = -P.m * q.f * (q.dx * wx + q.dy * wy + q.dz * wz);
      Pbar += Sbar;
      if (q.u < 0.f) {
        // d Pi / d rho_i = -Pi / (rho_i + rho_j); a boundary neighbour lends rho_i itself
        rv += Sbar * (q.fluid ? -q.Pv / q.rs : -q.Pv / ri);
        al += (q.fluid ? 0.5f : 1.f) * Sbar * q.Pv;
      }
    }
    float dPdr = 0.f, dPdB = 0.f;
    if (pi > 0.f || P.no_clamp) {
      const float rr = ri * P.inv_rho0;
      const float rg = P.gamma_is_7 ? rr * rr * rr * rr * rr * rr * rr : powf(rr, P.gamma);
      const float dp = P.gamma * B * rg / rr * P.inv_rho0;   // dp / drho
      dPdr = dp / (ri * ri) - 2.f * pi / (ri * ri * ri);
      dPdB = (rg - 1.f) / (ri * ri);
    }
    rhobar[i] = Pbar * dPdr + rv;
    bB = (double)Pbar * dPdB;
    bA = alpha > 0.f ? (double)al / alpha : 0.0;
  }
  cta_add2(bB, bA, red);
}

// Pass B: position and velocity adjoints of every pair of i's list, added to xbar, vbar.
__global__ void kd_adj_b(DevParams P, int n, float K, const float4* __restrict__ x,
                         const float4* __restrict__ v, const float* __restrict__ rho,
                         const float* __restrict__ prs, const float4* __restrict__ xb,
                         const uint32_t* __restrict__ list, const int* __restrict__ nn, int cap,
                         const float4* __restrict__ abar, const float* __restrict__ rhobar,
                         float4* __restrict__ xbar, float4* __restrict__ vbar) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 xi = x[i], vi = v[i], ai = abar[i];
  const float ri = rho[i], Pi = prs[i] / (ri * ri), rbi = rhobar[i];
  float gx = 0.f, gy = 0.f, gz = 0.f, hx = 0.f, hy = 0.f, hz = 0.f;
  const uint32_t* li = list + (size_t)i * cap;
  for (int e = 0; e < nn[i]; ++e) {
    const uint32_t jg = li[e];
    PairQ q;
    if (!pair_q(P, K, xi, vi, ri, Pi, jg, x, v, rho, prs, xb, q)) continue;
    float wx = ai.x, wy = ai.y, wz = ai.z, rb = rbi;
    if (q.fluid) {
      const float4 aj = abar[jg];
      wx -= aj.x;
      wy -= aj.y;
      wz -= aj.z;
      rb += rhobar[jg];
    }
    // kernel gradient: Gbar = -m S w
    const float Gx = -P.m * q.S * wx, Gy = -P.m * q.S * wy, Gz = -P.m * q.S * wz;
    const float xg = q.dx * Gx + q.dy * Gy + q.dz * Gz;
    const float coef = (q.d2W - q.f) / q.d2;
    float X0 = q.f * Gx + coef * xg * q.dx;
    float X1 = q.f * Gy + coef * xg * q.dy;
    float X2 = q.f * Gz + coef * xg * q.dz;
    // density sums of both particles
    const float dd = rb * P.m * q.f;
    X0 += dd * q.dx;
    X1 += dd * q.dy;
    X2 += dd * q.dz;
    // viscosity
    if (q.u < 0.f) {
      const float Sbar = -P.m * q.f * (q.dx * wx + q.dy * wy + q.dz * wz);
      const float ubar = Sbar * (-q.nu / q.D);
      const float r2bar = Sbar * q.nu * q.u / (q.D * q.D);
      X0 += ubar * q.vx + 2.f * r2bar * q.dx;
      X1 += ubar * q.vy + 2.f * r2bar * q.dy;
      X2 += ubar * q.vz + 2.f * r2bar * q.dz;
      hx += ubar * q.dx;
      hy += ubar * q.dy;
      hz += ubar * q.dz;
    }
    gx += X0;
    gy += X1;
    gz += X2;
  }
  float4 xo = xbar[i], vo = vbar[i];
  xbar[i] = make_float4(xo.x + gx, xo.y + gy, xo.z + gz, 0.f);
  vbar[i] = make_float4(vo.x + hx, vo.y + hy, vo.z + hz, 0.f);
}

// Adjoint of the summation density alone: xbar_i += sum (rhobar_i + rhobar_j) m f x_ij.
__global__ void kd_adj_density(DevParams P, int n, const float4* __restrict__ x,
                               const float4* __restrict__ xb, const uint32_t* __restrict__ list,
                               const int* __restrict__ nn, int cap, const float* __restrict__ rhobar,
                               float4* __restrict__ xbar) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 xi = x[i];
  float gx = 0.f, gy = 0.f, gz = 0.f;
  const uint32_t* li = list + (size_t)i * cap;
  for (int e = 0; e < nn[i]; ++e) {
    const uint32_t jg = li[e];
    const bool fluid = !(jg & kBnd);
    const float4 xj = fluid ? x[jg] : xb[jg & ~kBnd];
    const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
    const float d2 = dx * dx + dy * dy + dz * dz;
    if (d2 <= 0.f) continue;
    const float r = sqrtf(d2);
    float W, dW, d2W;
    spline3(P, r, W, dW, d2W);
    const float c = (rhobar[i] + (fluid ? rhobar[jg] : 0.f)) * P.m * dW / r;
    gx += c * dx;
    gy += c * dy;
    gz += c * dz;
  }
  const float4 o = xbar[i];
  xbar[i] = make_float4(o.x + gx, o.y + gy, o.z + gz, 0.f);
}

// Correction adjoint: anbar = abar + c1 xbar + c2 vbar; akbar = -c1 xbar - c2 vbar
// (xbar, vbar then stand for the adjoints of x~, v~).
__global__ void kd_adj_correct(int n, float dt, const float4* __restrict__ xbar,
                               const float4* __restrict__ vbar, const float4* __restrict__ abar,
                               float4* __restrict__ anbar, float4* __restrict__ akbar) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float c1 = dt * dt / 6.f, c2 = 0.5f * dt;
  const float4 xb = xbar[i], vb = vbar[i], ab = abar[i];
  anbar[i] = make_float4(ab.x + c1 * xb.x + c2 * vb.x, ab.y + c1 * xb.y + c2 * vb.y,
                         ab.z + c1 * xb.z + c2 * vb.z, 0.f);
  akbar[i] = make_float4(-c1 * xb.x - c2 * vb.x, -c1 * xb.y - c2 * vb.y, -c1 * xb.z - c2 * vb.z, 0.f);
}

// Container and predictor adjoint: clamped coordinates and zeroed velocities pass no
// adjoint; xbar <- x~bar, vbar <- x~bar dt + v~bar, abar <- akbar + x~bar dt^2/2 + v~bar dt.
__global__ void kd_adj_predict(int n, float dt, const uint8_t* __restrict__ mask,
                               float4* __restrict__ xbar, float4* __restrict__ vbar,
                               const float4* __restrict__ akbar, float4* __restrict__ abar) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 xt = xbar[i], vt = vbar[i];
  const uint8_t m = mask ? mask[i] : 0;
  if (m & 1) xt.x = 0.f;
  if (m & 2) xt.y = 0.f;
  if (m & 4) xt.z = 0.f;
  if (m & 8) vt.x = 0.f;
  if (m & 16) vt.y = 0.f;
  if (m & 32) vt.z = 0.f;
  const float4 ak = akbar[i];
  const float h = 0.5f * dt * dt;
  xbar[i] = make_float4(xt.x, xt.y, xt.z, 0.f);
  vbar[i] = make_float4(xt.x * dt + vt.x, xt.y * dt + vt.y, xt.z * dt + vt.z, 0.f);
  abar[i] = make_float4(ak.x + xt.x * h + vt.x * dt, ak.y + xt.y * h + vt.y * dt,
                        ak.z + xt.z * h + vt.z * dt, 0.f);
}

}  // namespace
}  // namespace rts

// ------------------------------------------------------------------- host ---

using namespace rts;

static rts_status dfail(rts_diff* d, rts_status st, const char* msg) {
  if (d) snprintf(d->err, sizeof d->err, "%s", msg);
  else rts_set_global_error(msg);
  return st;
}

#define DCK(expr)                                                             \
  do {                                                                        \
    cudaError_t _e = (expr);                                                  \
    if (_e != cudaSuccess) {                                                  \
      snprintf(d->err, sizeof d->err, "%s: %s", #expr, cudaGetErrorString(_e)); \
      d->sticky = RTS_ERR_CUDA;                                               \
      return _e == cudaErrorMemoryAllocation ? RTS_ERR_OOM : RTS_ERR_CUDA;    \
    }                                                                         \
  } while (0)

static rts_status dsync(rts_diff* d) {
  DCK(cudaMemcpyAsync(d->h_ctl, d->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, d->stream));
  DCK(cudaStreamSynchronize(d->stream));
  DCK(cudaGetLastError());
  const int st = d->h_ctl->status;
  if (st != 0) {
    d->sticky = st;
    if (st == RTS_ERR_DOMAIN && d->h_ctl->bad_set)
      snprintf(d->err, sizeof d->err, "device status %d: particle %u left the grid (at %g %g %g)", st,
               d->h_ctl->bad_uid, (double)d->h_ctl->bad_x, (double)d->h_ctl->bad_y,
               (double)d->h_ctl->bad_z);
    else
      snprintf(d->err, sizeof d->err, "device status %d (%s)", st,
               st == RTS_ERR_CAPACITY ? "a neighbour list exceeded max_neighbors" : "device error");
    return (rts_status)st;
  }
  return RTS_OK;
}

// Cell list of positions x (caller order).
static void build_cells(rts_diff* d, const float4* x) {
  const int n = d->n, g = grid_of(n);
  // the kernels of a step are chained with programmatic dependencies (see launch_pdl)
  launch_pdl(d->stream, kd_key, g, kT, 0, d->dp, n, x, d->key, d->count, d->ctl);
  scan_block_counts(d->count, d->dp.nblocks, d->tile_sums, d->cstart, d->stream);
  launch_pdl(d->stream, kd_place, g, kT, 0, n, d->key, d->cstart, d->count, d->perm_tmp);
  launch_pdl(d->stream, kd_rank, g, kT, 0, n, d->key, d->cstart, d->count, d->perm_tmp, d->perm);
}

// Density, lists and acceleration at (x, v) into rho/prs/list/nn and acc.
static void evaluate(rts_diff* d, const float4* x, const float4* v, float* rho, float* prs,
                     uint32_t* list, int* nn, float4* acc) {
  const int n = d->n, g = grid_of(n);
  const float K = (float)(2.0 * d->alpha * 0.5 * d->p.support_r * d->p.c_s);
  build_cells(d, x);
  launch_pdl(d->stream, kd_density, g, kT, 0, d->dp, n, d->B, x, d->key, d->cstart, d->perm, d->xb,
             d->bcstart, d->cap, rho, prs, list, nn, d->ctl);
  if (acc)
    launch_pdl(d->stream, kd_force, g, kT, 0, d->dp, n, K, x, v, rho, prs, d->xb, list, nn, d->cap,
               acc);
}

// One step from (x, v, a); with rec >= 0 the evaluation point is recorded in slot rec.
static void step(rts_diff* d, int rec) {
  const int n = d->n, g = grid_of(n);
  const float dt = d->p.dt_b;
  const size_t off = rec >= 0 ? (size_t)rec * n : 0;
  float4* xt = rec >= 0 ? d->rec_xt + off : d->xt;
  float4* vt = rec >= 0 ? d->rec_vt + off : d->vt;
  uint8_t* mk = rec >= 0 ? d->rec_mask + off : nullptr;
  launch_pdl(d->stream, kd_predict, g, kT, 0, d->dp, n, dt, d->x, d->v, d->a, xt, vt, mk);
  float* rho = rec >= 0 ? d->rec_rho + off : d->rho;
  float* prs = rec >= 0 ? d->rec_prs + off : d->prs;
  uint32_t* list = rec >= 0 ? d->rec_list + off * d->cap : d->list;
  int* nn = rec >= 0 ? d->rec_nn + off : d->nn;
  evaluate(d, xt, vt, rho, prs, list, nn, d->an);
  launch_pdl(d->stream, kd_correct, g, kT, 0, n, dt, xt, vt, d->an, d->x, d->v, d->a);
}

// Adjoint of A(x, v) at a recorded evaluation for the output adjoint abar_out; adds into
// xbar, vbar and the reductions.
static void eval_adjoint(rts_diff* d, const float4* x, const float4* v, const float* rho,
                         const float* prs, const uint32_t* list, const int* nn,
                         const float4* abar_out) {
  const int n = d->n, g = grid_of(n);
  const float K = (float)(2.0 * d->alpha * 0.5 * d->p.support_r * d->p.c_s);
  launch_pdl(d->stream, kd_adj_a, g, kT, 0, d->dp, n, d->B, K, d->alpha, x, v, rho, prs, d->xb,
             list, nn, d->cap, abar_out, d->rhobar, d->red);
  launch_pdl(d->stream, kd_adj_b, g, kT, 0, d->dp, n, K, x, v, rho, prs, d->xb, list, nn, d->cap,
             abar_out, d->rhobar, d->xbar, d->vbar);
}

extern "C" {

rts_status rts_diff_create(const rts_params* params, int32_t n_fluid, const float* x0,
                           int32_t n_boundary, const float* xb, int32_t n_steps, int32_t ckpt_every,
                           void* cuda_stream, rts_diff** out) {
  if (!out) return dfail(nullptr, RTS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!params || n_fluid < 1 || !x0 || n_boundary < 0 || (n_boundary > 0 && !xb))
    return dfail(nullptr, RTS_ERR_ARG, "bad sizes or pointers");
  if (params->scheme != RTS_WCSPH) return dfail(nullptr, RTS_ERR_ARG, "the differentiable rollout is WCSPH");
  if (n_steps < 1 || ckpt_every < 1 || ckpt_every > n_steps)
    return dfail(nullptr, RTS_ERR_ARG, "need n_steps >= 1 and 1 <= ckpt_every <= n_steps");
  if (const char* why = validate_params(params, n_fluid, n_boundary)) return dfail(nullptr, RTS_ERR_ARG, why);
  rts_diff* d = new (std::nothrow) rts_diff;
  if (!d) return dfail(nullptr, RTS_ERR_OOM, "host allocation failed");
  memset(d, 0, sizeof(*d));
  d->p = *params;
  make_dev_params(d->p, d->dp);
  d->dp.n_fluid = n_fluid;
  d->dp.n_bound = n_boundary;
  d->n = n_fluid;
  d->nb = n_boundary;
  d->steps = n_steps;
  d->ckpt = ckpt_every;
  d->nseg = (n_steps + ckpt_every - 1) / ckpt_every;
  d->cap = params->max_neighbors > 0 ? params->max_neighbors : 96;
  d->stream = (cudaStream_t)cuda_stream;
  const size_t n = (size_t)n_fluid, nbk = (size_t)d->dp.nblocks, f4 = sizeof(float4) * n;
  const size_t ntiles = (nbk + 2047) / 2048, R = (size_t)d->ckpt, cap = (size_t)d->cap;
  rts_status st = RTS_OK;
#define DALLOC(ptr, bytes)                                                       \
  do {                                                                           \
    cudaError_t _e = cudaMalloc((void**)&(ptr), (bytes));                        \
    if (_e != cudaSuccess) {                                                     \
      snprintf(d->err, sizeof d->err, "cudaMalloc %s: %s", #ptr, cudaGetErrorString(_e)); \
      st = RTS_ERR_OOM;                                                          \
      goto fail;                                                                 \
    }                                                                            \
  } while (0)
  DALLOC(d->xb, sizeof(float4) * (size_t)(n_boundary > 0 ? n_boundary : 1));
  DALLOC(d->bcstart, sizeof(uint32_t) * (nbk + 1));
  DALLOC(d->key, sizeof(uint32_t) * (n > (size_t)n_boundary ? n : (size_t)n_boundary));
  DALLOC(d->count, sizeof(uint32_t) * nbk);
  DALLOC(d->cstart, sizeof(uint32_t) * (nbk + 1));
  DALLOC(d->tile_sums, sizeof(uint32_t) * ntiles);
  DALLOC(d->perm_tmp, sizeof(uint32_t) * (n > (size_t)n_boundary ? n : (size_t)n_boundary));
  DALLOC(d->perm, sizeof(uint32_t) * (n > (size_t)n_boundary ? n : (size_t)n_boundary));
  DALLOC(d->x, f4);
  DALLOC(d->v, f4);
  DALLOC(d->a, f4);
  DALLOC(d->xt, f4);
  DALLOC(d->vt, f4);
  DALLOC(d->an, f4);
  DALLOC(d->ck_x, f4 * (d->nseg + 1));
  DALLOC(d->ck_v, f4 * (d->nseg + 1));
  DALLOC(d->ck_a, f4 * (d->nseg + 1));
  DALLOC(d->rho, sizeof(float) * n);
  DALLOC(d->prs, sizeof(float) * n);
  DALLOC(d->list, sizeof(uint32_t) * n * cap);
  DALLOC(d->nn, sizeof(int) * n);
  DALLOC(d->rec_xt, f4 * R);
  DALLOC(d->rec_vt, f4 * R);
  DALLOC(d->rec_rho, sizeof(float) * n * R);
  DALLOC(d->rec_prs, sizeof(float) * n * R);
  DALLOC(d->rec_list, sizeof(uint32_t) * n * cap * R);
  DALLOC(d->rec_nn, sizeof(int) * n * R);
  DALLOC(d->rec_mask, n * R);
  DALLOC(d->xbar, f4);
  DALLOC(d->vbar, f4);
  DALLOC(d->abar, f4);
  DALLOC(d->anbar, f4);
  DALLOC(d->akbar, f4);
  DALLOC(d->rhobar, sizeof(float) * n);
  DALLOC(d->red, 2 * sizeof(double));
  DALLOC(d->ctl, sizeof(Ctl));
#undef DALLOC
  if (cudaMallocHost((void**)&d->h_ctl, sizeof(Ctl)) != cudaSuccess ||
      cudaMallocHost((void**)&d->h_red, 2 * sizeof(double)) != cudaSuccess) {
    st = dfail(d, RTS_ERR_OOM, "pinned host allocation failed");
    goto fail;
  }
  {
    // initial positions; the boundary sorted by block, then index, into xb / bcstart
    const size_t nt = n > (size_t)n_boundary ? n : (size_t)n_boundary;
    float* tmp = nullptr;
    float4* bsrc = nullptr;
    cudaError_t e = cudaMemsetAsync(d->ctl, 0, sizeof(Ctl), d->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d->count, 0, sizeof(uint32_t) * nbk, d->stream);
    if (e == cudaSuccess) e = cudaMalloc((void**)&tmp, sizeof(float) * 3 * nt);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, x0, sizeof(float) * 3 * n, cudaMemcpyDefault, d->stream);
    if (e == cudaSuccess) {
      kd_pack<<<grid_of((int)n), kT, 0, d->stream>>>((int)n, tmp, d->ck_x);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess && n_boundary > 0) {
      const int gb = grid_of(n_boundary);
      e = cudaMalloc((void**)&bsrc, sizeof(float4) * (size_t)n_boundary);
      if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);   // tmp is reused
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(tmp, xb, sizeof(float) * 3 * (size_t)n_boundary, cudaMemcpyDefault, d->stream);
      if (e == cudaSuccess) {
        kd_pack<<<gb, kT, 0, d->stream>>>(n_boundary, tmp, bsrc);
        kd_key<<<gb, kT, 0, d->stream>>>(d->dp, n_boundary, bsrc, d->key, d->count, d->ctl);
        scan_block_counts(d->count, d->dp.nblocks, d->tile_sums, d->bcstart, d->stream);
        kd_place<<<gb, kT, 0, d->stream>>>(n_boundary, d->key, d->bcstart, d->count, d->perm_tmp);
        kd_rank<<<gb, kT, 0, d->stream>>>(n_boundary, d->key, d->bcstart, d->count, d->perm_tmp, d->perm);
        kd_gather_sorted<<<gb, kT, 0, d->stream>>>(n_boundary, d->perm, bsrc, d->xb);
        e = cudaGetLastError();
      }
    } else if (e == cudaSuccess) {
      e = cudaMemsetAsync(d->bcstart, 0, sizeof(uint32_t) * (nbk + 1), d->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    cudaFree(tmp);
    cudaFree(bsrc);
    if (e != cudaSuccess) {
      snprintf(d->err, sizeof d->err, "initial upload: %s", cudaGetErrorString(e));
      st = RTS_ERR_CUDA;
      goto fail;
    }
  }
  st = dsync(d);
  if (st != RTS_OK) goto fail;
  *out = d;
  return RTS_OK;
fail:
  rts_set_global_error(d->err);
  rts_diff_destroy(d);
  return st;
}

rts_status rts_diff_forward(rts_diff* d, const float* v0, float tait_B, float visc_alpha,
                            float* x_out, float* rho_out) {
  if (!d || !v0) return dfail(d, RTS_ERR_ARG, "ctx and v0 are required");
  if (d->sticky) return dfail(d, RTS_ERR_STATE, "a device error is pending; create a new context");
  if (!(tait_B > 0.f) || !(visc_alpha >= 0.f)) return dfail(d, RTS_ERR_ARG, "need tait_B > 0, visc_alpha >= 0");
  const int n = d->n, g = grid_of(n);
  d->B = tait_B;
  d->alpha = visc_alpha;
  float* tmp = nullptr;
  DCK(cudaMalloc((void**)&tmp, sizeof(float) * 3 * (size_t)n));
  DCK(cudaMemcpyAsync(tmp, v0, sizeof(float) * 3 * (size_t)n, cudaMemcpyDefault, d->stream));
  kd_pack<<<g, kT, 0, d->stream>>>(n, tmp, d->ck_v);
  DCK(cudaMemcpyAsync(d->x, d->ck_x, sizeof(float4) * n, cudaMemcpyDeviceToDevice, d->stream));
  DCK(cudaMemcpyAsync(d->v, d->ck_v, sizeof(float4) * n, cudaMemcpyDeviceToDevice, d->stream));
  evaluate(d, d->x, d->v, d->rho, d->prs, d->list, d->nn, d->a);   // priming a_0 = A(x_0, v_0)
  DCK(cudaMemcpyAsync(d->ck_a, d->a, sizeof(float4) * n, cudaMemcpyDeviceToDevice, d->stream));
  for (int k = 0; k < d->steps; ++k) {
    step(d, -1);
    if ((k + 1) % d->ckpt == 0 && (k + 1) / d->ckpt < d->nseg + 1) {
      const size_t c = (size_t)((k + 1) / d->ckpt) * n;
      DCK(cudaMemcpyAsync(d->ck_x + c, d->x, sizeof(float4) * n, cudaMemcpyDeviceToDevice, d->stream));
      DCK(cudaMemcpyAsync(d->ck_v + c, d->v, sizeof(float4) * n, cudaMemcpyDeviceToDevice, d->stream));
      DCK(cudaMemcpyAsync(d->ck_a + c, d->a, sizeof(float4) * n, cudaMemcpyDeviceToDevice, d->stream));
    }
  }
  evaluate(d, d->x, d->v, d->rho, d->prs, d->list, d->nn, nullptr);   // rho_T = rho(x_T)
  if (x_out) {
    kd_unpack<<<g, kT, 0, d->stream>>>(n, d->x, tmp);
    DCK(cudaMemcpyAsync(x_out, tmp, sizeof(float) * 3 * (size_t)n, cudaMemcpyDefault, d->stream));
  }
  if (rho_out) DCK(cudaMemcpyAsync(rho_out, d->rho, sizeof(float) * (size_t)n, cudaMemcpyDefault, d->stream));
  rts_status st = dsync(d);
  cudaFree(tmp);
  d->have_forward = st == RTS_OK;
  return st;
}

rts_status rts_diff_backward(rts_diff* d, const float* gx, const float* grho, float* gv0,
                             double* gB, double* galpha) {
  if (!d || !gv0) return dfail(d, RTS_ERR_ARG, "ctx and gv0 are required");
  if (d->sticky) return dfail(d, RTS_ERR_STATE, "a device error is pending; create a new context");
  if (!d->have_forward) return dfail(d, RTS_ERR_STATE, "call rts_diff_forward first");
  const int n = d->n, g = grid_of(n);
  const float dt = d->p.dt_b;
  float* tmp = nullptr;
  DCK(cudaMalloc((void**)&tmp, sizeof(float) * 3 * (size_t)n));
  DCK(cudaMemsetAsync(d->red, 0, 2 * sizeof(double), d->stream));
  DCK(cudaMemsetAsync(d->vbar, 0, sizeof(float4) * n, d->stream));
  DCK(cudaMemsetAsync(d->abar, 0, sizeof(float4) * n, d->stream));
  if (gx) {
    DCK(cudaMemcpyAsync(tmp, gx, sizeof(float) * 3 * (size_t)n, cudaMemcpyDefault, d->stream));
    kd_pack<<<g, kT, 0, d->stream>>>(n, tmp, d->xbar);
  } else {
    DCK(cudaMemsetAsync(d->xbar, 0, sizeof(float4) * n, d->stream));
  }
  if (grho) {
    // rho_T = rho(x_T): the lists of the final density pass are still in d->list
    DCK(cudaMemcpyAsync(d->rhobar, grho, sizeof(float) * (size_t)n, cudaMemcpyDefault, d->stream));
    kd_adj_density<<<g, kT, 0, d->stream>>>(d->dp, n, d->x, d->xb, d->list, d->nn, d->cap, d->rhobar,
                                            d->xbar);
  }
  for (int s = d->nseg - 1; s >= 0; --s) {
    const int k0 = s * d->ckpt, k1 = (k0 + d->ckpt < d->steps) ? k0 + d->ckpt : d->steps;
    const size_t c = (size_t)s * n;
    DCK(cudaMemcpyAsync(d->x, d->ck_x + c, sizeof(float4) * n, cudaMemcpyDeviceToDevice, d->stream));
    DCK(cudaMemcpyAsync(d->v, d->ck_v + c, sizeof(float4) * n, cudaMemcpyDeviceToDevice, d->stream));
    DCK(cudaMemcpyAsync(d->a, d->ck_a + c, sizeof(float4) * n, cudaMemcpyDeviceToDevice, d->stream));
    for (int k = k0; k < k1; ++k) step(d, k - k0);     // recompute with records
    for (int k = k1 - 1; k >= k0; --k) {
      const size_t off = (size_t)(k - k0) * n;
      launch_pdl(d->stream, kd_adj_correct, g, kT, 0, n, dt, d->xbar, d->vbar, d->abar, d->anbar,
                 d->akbar);
      eval_adjoint(d, d->rec_xt + off, d->rec_vt + off, d->rec_rho + off, d->rec_prs + off,
                   d->rec_list + off * d->cap, d->rec_nn + off, d->anbar);
      launch_pdl(d->stream, kd_adj_predict, g, kT, 0, n, dt, d->rec_mask + off, d->xbar, d->vbar,
                 d->akbar, d->abar);
    }
  }
  // priming evaluation a_0 = A(x_0, v_0): only its velocity (and parameter) adjoints matter
  DCK(cudaMemcpyAsync(d->x, d->ck_x, sizeof(float4) * n, cudaMemcpyDeviceToDevice, d->stream));
  DCK(cudaMemcpyAsync(d->v, d->ck_v, sizeof(float4) * n, cudaMemcpyDeviceToDevice, d->stream));
  evaluate(d, d->x, d->v, d->rho, d->prs, d->list, d->nn, nullptr);
  DCK(cudaMemsetAsync(d->xbar, 0, sizeof(float4) * n, d->stream));
  eval_adjoint(d, d->x, d->v, d->rho, d->prs, d->list, d->nn, d->abar);
  kd_unpack<<<g, kT, 0, d->stream>>>(n, d->vbar, tmp);
  DCK(cudaMemcpyAsync(gv0, tmp, sizeof(float) * 3 * (size_t)n, cudaMemcpyDefault, d->stream));
  DCK(cudaMemcpyAsync(d->h_red, d->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, d->stream));
  rts_status st = dsync(d);
  cudaFree(tmp);
  if (st != RTS_OK) return st;
  if (gB) *gB = d->h_red[0];
  if (galpha) *galpha = d->h_red[1];
  // the forward state (x_T) was overwritten by the recomputation
  d->have_forward = false;
  return RTS_OK;
}

const char* rts_diff_last_error(const rts_diff* d) { return d ? d->err : rts_last_error(nullptr); }

void rts_diff_destroy(rts_diff* d) {
  if (!d) return;
  cudaFree(d->xb); cudaFree(d->bcstart); cudaFree(d->key); cudaFree(d->count); cudaFree(d->cstart);
  cudaFree(d->tile_sums); cudaFree(d->perm_tmp); cudaFree(d->perm); cudaFree(d->x); cudaFree(d->v);
  cudaFree(d->a); cudaFree(d->xt); cudaFree(d->vt); cudaFree(d->an); cudaFree(d->ck_x);
  cudaFree(d->ck_v); cudaFree(d->ck_a); cudaFree(d->rho); cudaFree(d->prs); cudaFree(d->list);
  cudaFree(d->nn); cudaFree(d->rec_xt); cudaFree(d->rec_vt); cudaFree(d->rec_rho); cudaFree(d->rec_prs);
  cudaFree(d->rec_list); cudaFree(d->rec_nn); cudaFree(d->rec_mask); cudaFree(d->xbar); cudaFree(d->vbar);
  cudaFree(d->abar); cudaFree(d->anbar); cudaFree(d->akbar); cudaFree(d->rhobar); cudaFree(d->red);
  cudaFree(d->ctl);
  if (d->h_ctl) cudaFreeHost(d->h_ctl);
  if (d->h_red) cudaFreeHost(d->h_red);
  delete d;
}

}  // extern "C"
