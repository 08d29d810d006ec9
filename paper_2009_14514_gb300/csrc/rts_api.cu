// rts_api.cu - the C ABI of librts (declared in rts.h): context set-up, parameter
// validation, caller-order I/O and the step sequences of Algorithm 1 (WCSPH) and of
// the global comparators.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "rts_internal.cuh"

using namespace rts;

static char g_noctx_err[512] = "";

const char* rts::cuda_err(rts_ctx* c, cudaError_t e, const char* what) {
  char* dst = c ? c->err : g_noctx_err;
  snprintf(dst, 512, "%s: %s", what, cudaGetErrorString(e));
  return dst;
}

// Message for rts_last_error(NULL) from entry points that take no context.
void rts_set_global_error(const char* msg) { snprintf(g_noctx_err, sizeof g_noctx_err, "%s", msg); }

static rts_status fail(rts_ctx* c, rts_status st, const char* msg) {
  snprintf(c ? c->err : g_noctx_err, 512, "%s", msg);
  return st;
}

#define CK(expr)                                       \
  do {                                                 \
    cudaError_t _e = (expr);                           \
    if (_e != cudaSuccess) {                           \
      rts::cuda_err(c, _e, #expr);                     \
      return _e == cudaErrorMemoryAllocation ? RTS_ERR_OOM : RTS_ERR_CUDA; \
    }                                                  \
  } while (0)

namespace rts {
int neighbor_grid_size();
}

// ------------------------------------------------------------- parameters ---

static void level_thresholds(const rts_params& p, double* vthr2, double* athr2, int* eq1) {
  // Eq. 1: dt <= lambda_v r / c_s (WCSPH only).  Eq. 2 with F = m |a|, squared twice:
  // |a|^2 <= (lambda_f^2 r / dt^2)^2.  Eq. 3: |v|^2 <= (alpha beta r / dt)^2.
  for (int L = 0; L < p.n_levels; ++L) {
    double dt = (double)p.level_mult[L] * (double)p.dt_b;
    double vt = (double)p.alpha * (double)p.beta[L] * (double)p.support_r / dt;
    vthr2[L] = vt * vt;
    double at = (double)p.lambda_f * (double)p.lambda_f * (double)p.support_r / (dt * dt);
    athr2[L] = at * at;
    eq1[L] = p.scheme == RTS_WCSPH
                 ? (dt <= (double)p.lambda_v * (double)p.support_r / (double)p.c_s)
                 : 1;
  }
}

const char* rts::validate_params(const rts_params* p, int32_t n, int32_t nb, int max_dim) {
  if (!p) return "params is NULL";
  if (p->scheme != RTS_WCSPH && p->scheme != RTS_PCISPH) return "scheme must be RTS_WCSPH or RTS_PCISPH";
  if (p->mode < 0 || p->mode > 2) return "mode must be 0, 1 or 2";
  if (n < 0 || nb < 0) return "negative particle count";
  if (!(p->spacing > 0.f) || !(p->support_r > 0.f) || !(p->block_edge > 0.f))
    return "spacing, support_r and block_edge must be positive";
  if (p->block_edge < p->support_r) return "block_edge must be >= support_r";
  for (int d = 0; d < 3; ++d) {
    if (p->grid_dim[d] < 1 || p->grid_dim[d] > max_dim) return "grid_dim must be in [1, 4096]";
    if (!std::isfinite(p->domain_min[d]) || !std::isfinite(p->gravity[d])) return "non-finite domain_min or gravity";
  }
  if ((double)p->grid_dim[0] * p->grid_dim[1] * p->grid_dim[2] > 2.0e9) return "too many blocks";
  if (p->n_levels < 1 || p->n_levels > kMaxLevels) return "n_levels must be in [1, 8]";
  for (int L = 0; L < p->n_levels; ++L) {
    if (p->level_mult[L] < 1) return "level_mult must be >= 1";
    if (L > 0 && p->level_mult[L] <= p->level_mult[L - 1]) return "level_mult must increase";
    if (!(p->beta[L] > 0.f)) return "beta must be positive";
  }
  if (p->force_level >= p->n_levels) return "force_level must be < n_levels";
  if (!(p->dt_b > 0.f)) return "dt_b must be positive";
  if (p->max_per_block < 1 || p->max_per_block > 1024) return "max_per_block must be in [1, 1024]";
  if (p->max_neighbors < 8 || p->max_neighbors > 1024) return "max_neighbors must be in [8, 1024]";
  if (p->wall_project != 0 && p->wall_project != 1) return "wall_project must be 0 or 1";
  if (p->level_clock != 0 && p->level_clock != 1) return "level_clock must be 0 or 1";
  if (!(p->tait_B >= 0.f) || !(p->tait_B < 1e12f)) return "tait_B must be in [0, 1e12)";
  if (p->tait_no_clamp != 0 && p->tait_no_clamp != 1) return "tait_no_clamp must be 0 or 1";
  if (p->serna_off != 0 && p->serna_off != 1) return "serna_off must be 0 or 1";
  if (p->r2_search_rings < 0 || p->r2_search_rings > 3) return "r2_search_rings must be in [0, 3]";
  if (p->stale_bins < 0 || p->stale_bins > 64) return "stale_bins must be in [0, 64]";
  if (p->r1_search_rings < 0 || p->r1_search_rings > 3) return "r1_search_rings must be in [0, 3]";
  if (p->wall_project)
    for (int k = 0; k < 3; ++k)
      if (!(p->wall_lo[k] < p->wall_hi[k])) return "wall_lo must be below wall_hi on every axis";
  if (!(p->rho0 > 0.f) || !(p->c_s > 0.f) || !(p->gamma > 0.f) || !(p->visc_alpha >= 0.f))
    return "rho0, c_s, gamma must be positive and visc_alpha non-negative";
  if (!(p->lambda_f > 0.f) || !(p->alpha > 0.f) || !(p->lambda_v > 0.f)) return "lambda_v, lambda_f, alpha must be positive";
  if (p->scheme == RTS_PCISPH) {
    if (p->n_minor < 1 || p->n_minor > 8) return "n_minor must be in [1, 8]";
    if (p->n_levels > 4) return "PCISPH uses at most 4 regions";
    if (p->max_iters < 1 || p->max_neighbors < 8 || p->max_neighbors > 1024) return "bad PCISPH iteration or neighbour limits";
  }
  return nullptr;
}

void rts::make_dev_params(const rts_params& p, DevParams& d) {
  memset(&d, 0, sizeof(d));
  d.ox = p.domain_min[0];
  d.oy = p.domain_min[1];
  d.oz = p.domain_min[2];
  d.edge = p.block_edge;
  d.inv_edge = 1.0f / p.block_edge;
  d.oxd = d.ox;
  d.oyd = d.oy;
  d.ozd = d.oz;
  d.edged = d.edge;
  d.nx = p.grid_dim[0];
  d.ny = p.grid_dim[1];
  d.nz = p.grid_dim[2];
  d.nblocks = d.nx * d.ny * d.nz;
  d.div_nx = (1ull << 40) / (unsigned long long)d.nx + 1ull;
  d.div_ny = (1ull << 40) / (unsigned long long)d.ny + 1ull;
  {
    // the FP32 block coordinate of a point up to one block outside the grid carries at
    // most 3 * 2^-24 relative error; 8 * 2^-24 * (largest dim + 2) bounds it with margin
    int dmax = p.grid_dim[0];
    if (p.grid_dim[1] > dmax) dmax = p.grid_dim[1];
    if (p.grid_dim[2] > dmax) dmax = p.grid_dim[2];
    d.key_band = (float)(8.0 * ldexp(1.0, -24) * (dmax + 2));
  }
  d.max_per_block = p.max_per_block;
  d.r = p.support_r;
  d.r2 = p.support_r * p.support_r;
  d.r2d = (double)p.support_r * (double)p.support_r;
  d.r2_dh = (float)d.r2d;
  d.r2_dl = (float)(d.r2d - (double)d.r2_dh);
  d.r2_win = (float)ldexp(d.r2d, -38);
  d.r2_lo = (float)(d.r2d * (1.0 - 1e-5));
  d.r2_hi = (float)(d.r2d * (1.0 + 1e-5));
  double h = 0.5 * (double)p.support_r;
  double sigma = 1.0 / (M_PI * h * h * h);
  d.h = (float)h;
  d.inv_h = (float)(1.0 / h);
  d.sigma = (float)sigma;
  d.sigma_h = (float)(sigma / h);
  double s = p.spacing;
  d.m = (float)((double)p.rho0 * s * s * s);
  d.rho0 = p.rho0;
  d.inv_rho0 = (float)(1.0 / (double)p.rho0);
  d.tait_B = p.tait_B > 0.f ? p.tait_B : (float)((double)p.c_s * p.c_s * p.rho0 / p.gamma);
  d.gamma = p.gamma;
  d.gamma_is_7 = p.gamma == 7.0f;
  d.visc_coef = (float)(2.0 * p.visc_alpha * h * p.c_s);
  d.eps_h2 = (float)(0.01 * h * h);
  d.gx = p.gravity[0];
  d.gy = p.gravity[1];
  d.gz = p.gravity[2];
  d.wall_project = p.wall_project;
  d.level_clock = p.level_clock;
  d.no_clamp = p.tait_no_clamp;
  d.serna_off = p.serna_off;
  d.r2_rings = p.r2_search_rings > 1 ? p.r2_search_rings : 1;
  for (int k = 0; k < 3; ++k) {
    d.wlo[k] = p.wall_lo[k];
    d.whi[k] = p.wall_hi[k];
  }
  d.n_levels = p.n_levels;
  for (int L = 0; L < p.n_levels; ++L) d.mult[L] = p.level_mult[L];
  level_thresholds(p, d.vthr2, d.athr2, d.eq1);
  for (int L = 0; L < kMaxLevels; ++L) {
    d.vthr2f[L] = (float)d.vthr2[L];
    d.athr2f[L] = (float)d.athr2[L];
    // FP32 residuals: vthr2 = vthr2f + vthr2lo within 2^-48 (finite thresholds)
    d.vthr2lo[L] = std::isfinite(d.vthr2[L]) ? (float)(d.vthr2[L] - (double)d.vthr2f[L]) : 0.f;
    d.athr2lo[L] = std::isfinite(d.athr2[L]) ? (float)(d.athr2[L] - (double)d.athr2f[L]) : 0.f;
    // the key pass's near-threshold band, as the device forms it (one FP32 product)
    d.vnear[L] = std::isfinite(d.vthr2f[L]) ? 2e-6f * d.vthr2f[L] : -1.f;
    d.anear[L] = std::isfinite(d.athr2f[L]) ? 2e-6f * d.athr2f[L] : -1.f;
  }
  d.levels_monotone = 1;
  for (int L = 1; L < p.n_levels; ++L)
    if (!(d.vthr2[L] <= d.vthr2[L - 1]) || !(d.athr2[L] <= d.athr2[L - 1])) d.levels_monotone = 0;
  d.force_level = p.force_level;
  d.dt_b = p.dt_b;
  d.nbl_cap = p.max_neighbors > 0 ? p.max_neighbors : 96;
  // PCISPH (Section 5): Solenthaler-Pajarola scaling on a prototype particle with a full
  // cubic lattice of spacing s inside the support: delta = -1 / (beta (-|sum g|^2 -
  // sum |g|^2)), beta = 2 (dt_b m / rho0)^2, g = grad W.
  d.eta = p.eta;
  d.visc_nu = (float)((double)p.visc_alpha * h * p.c_s / p.rho0);
  d.r1_rings = p.r1_search_rings > 0 ? p.r1_search_rings : 1;
  d.expand_layers = p.expand_layers;
  d.n_minor = p.n_minor;
  for (int r = 0; r < 4; ++r)
    for (int j = 0; j < 8; ++j) d.sched[r][j] = p.sched[r][j];
  for (int L = 0; L < 8; ++L) d.refresh[L] = p.refresh[L] > 0 ? p.refresh[L] : 1;
  {
    double m = (double)p.rho0 * s * s * s, rr = (double)p.support_r;
    double g[3] = {0, 0, 0}, gg = 0.0;
    int R = (int)std::ceil(rr / s) + 1;
    for (int a = -R; a <= R; ++a)
      for (int b = -R; b <= R; ++b)
        for (int e = -R; e <= R; ++e) {
          if (!a && !b && !e) continue;
          double x[3] = {-a * s, -b * s, -e * s};
          double d2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
          if (!(d2 < rr * rr)) continue;
          double dd = std::sqrt(d2), q = dd / h;
          double dW = q < 1.0 ? sigma * (-3.0 * q + 2.25 * q * q) / h
                              : (q < 2.0 ? -0.75 * sigma * (2.0 - q) * (2.0 - q) / h : 0.0);
          for (int k = 0; k < 3; ++k) {
            double gk = dW / dd * x[k];
            g[k] += gk;
            gg += gk * gk;
          }
        }
    double beta = 2.0 * ((double)p.dt_b * m / p.rho0) * ((double)p.dt_b * m / p.rho0);
    double denom = -(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]) - gg;
    d.delta = (float)(-1.0 / (beta * denom));
  }
}

// ------------------------------------------------------------- profiling ---

// Accumulate the timed event pairs into prof_ms (synchronises the stream).
// Accumulate the first `upto` event pairs and move the rest to the front.  Only the
// last of those pairs is waited for; with upto = half the pool it is hundreds of phases
// old, so the stream keeps running.
static void prof_collect(rts_ctx* c, int upto) {
  if (!c->ev || upto <= 0) return;
  cudaEventSynchronize(c->ev[2 * (upto - 1) + 1]);
  for (int k = 0; k < upto; ++k) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[2 * k], c->ev[2 * k + 1]) == cudaSuccess)
      c->prof_ms[c->ev_phase[k]] += ms;
  }
  for (int k = upto; k < c->nev; ++k) {  // keep the newer pairs, recycle the handles
    cudaEvent_t a = c->ev[2 * (k - upto)], b = c->ev[2 * (k - upto) + 1];
    c->ev[2 * (k - upto)] = c->ev[2 * k];
    c->ev[2 * (k - upto) + 1] = c->ev[2 * k + 1];
    c->ev[2 * k] = a;
    c->ev[2 * k + 1] = b;
    c->ev_phase[k - upto] = c->ev_phase[k];
  }
  c->nev -= upto;
}

static void prof_flush(rts_ctx* c) {
  if (!c->ev || c->nev == 0) return;
  prof_collect(c, c->nev);
}

// Scope of one phase: sets the phase that launches are counted against and, when
// profiling is on, brackets the phase's launches with a pair of events.
struct Phase {
  rts_ctx* c;
  int prev, slot;
  Phase(rts_ctx* c_, int ph) : c(c_), prev(c_->cur_phase), slot(-1) {
    c->cur_phase = ph;
    c->passes[ph] += 1;
    bool timed = c->prof == 1;
    if (c->prof == 2 && (ph == RTS_PHASE_DENSITY || ph == RTS_PHASE_FORCE))
      timed = (c->prof_seen[ph]++ % 7) == 0;
    if (c->prof && c->ev && timed) {
      if (c->nev == kEvPairs) prof_collect(c, kEvPairs / 2);
      c->prof_timed[ph] += 1;
      slot = c->nev++;
      c->ev_phase[slot] = ph;
      cudaEventRecord(c->ev[2 * slot], c->stream);
    }
  }
  ~Phase() {
    if (slot >= 0) cudaEventRecord(c->ev[2 * slot + 1], c->stream);
    c->cur_phase = prev;
  }
};

// ------------------------------------------------------------ caller I/O ---

__global__ void k_pack3(int n, const float* __restrict__ in, float4* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_float4(in[3 * i], in[3 * i + 1], in[3 * i + 2], 0.f);
}

__global__ void k_in_vec(int n, const float* __restrict__ in, float4* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    float4 o = out[i];
    out[i] = in ? make_float4(in[3 * i], in[3 * i + 1], in[3 * i + 2], o.w)
                : make_float4(0.f, 0.f, 0.f, o.w);
  }
}

template <class T>
__global__ void k_in_scalar(int n, const T* __restrict__ in, T* __restrict__ out, T dflt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in ? in[i] : dflt;
}

// Identity order after an upload; x.w = p / rho^2, v.w = rho.
__global__ void k_finish_in(int n, PState s) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    float rho = s.rho[i];
    s.x[i].w = s.prs[i] / (rho * rho);
    s.v[i].w = rho;
    s.uid[i] = (uint32_t)i;
    s.nbr[i] = 0;
  }
}

__global__ void k_out_vec(int n, const uint32_t* __restrict__ uid, const float4* __restrict__ in,
                          float* __restrict__ out, Ctl* ctl) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    uint32_t u = uid[i];
    if (u >= (uint32_t)n) {
      check_failed(ctl, kChkUid, u);
      return;
    }
    float4 q = in[i];
    out[3 * u] = q.x;
    out[3 * u + 1] = q.y;
    out[3 * u + 2] = q.z;
  }
}

template <class T>
__global__ void k_out_scalar(int n, const uint32_t* __restrict__ uid, const T* __restrict__ in,
                             T* __restrict__ out, Ctl* ctl) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t u = uid[i];
  if (u >= (uint32_t)n) {
    check_failed(ctl, kChkUid, u);
    return;
  }
  out[u] = in[i];
}

static inline int nblk(int n) { return (n + 255) / 256; }

static rts_status upload_state(rts_ctx* c, const float* x, const float* v, const float* a,
                               const float* rho, const float* p, const int32_t* level,
                               const int32_t* validity, const int32_t* klast) {
  int n = c->n;
  if (n == 0) return RTS_OK;
  Phase ph(c, RTS_PHASE_OTHER);
  note_launch(c, 9);
  size_t v3 = sizeof(float) * 3 * (size_t)n, s1 = sizeof(float) * (size_t)n;
  float* io = c->io;
  int g = nblk(n);
  // scalars first: x.w and v.w are derived from rho and p
  if (rho) CK(cudaMemcpyAsync(io, rho, s1, cudaMemcpyDefault, c->stream));
  k_in_scalar<float><<<g, 256, 0, c->stream>>>(n, rho ? io : nullptr, c->s.rho, c->p.rho0);
  if (p) CK(cudaMemcpyAsync(io, p, s1, cudaMemcpyDefault, c->stream));
  k_in_scalar<float><<<g, 256, 0, c->stream>>>(n, p ? io : nullptr, c->s.prs, 0.0f);
  int32_t* ii = c->io_i;
  if (level) CK(cudaMemcpyAsync(ii, level, s1, cudaMemcpyDefault, c->stream));
  k_in_scalar<int32_t><<<g, 256, 0, c->stream>>>(n, level ? ii : nullptr, c->s.level, -1);
  if (validity) CK(cudaMemcpyAsync(ii, validity, s1, cudaMemcpyDefault, c->stream));
  k_in_scalar<int32_t><<<g, 256, 0, c->stream>>>(n, validity ? ii : nullptr, c->s.valid, 0);
  if (klast) CK(cudaMemcpyAsync(ii, klast, s1, cudaMemcpyDefault, c->stream));
  k_in_scalar<int32_t><<<g, 256, 0, c->stream>>>(n, klast ? ii : nullptr, c->s.klast, 0);
  CK(cudaMemcpyAsync(io, x, v3, cudaMemcpyDefault, c->stream));
  k_in_vec<<<g, 256, 0, c->stream>>>(n, io, c->s.x);
  CK(cudaMemcpyAsync(io, v, v3, cudaMemcpyDefault, c->stream));
  k_in_vec<<<g, 256, 0, c->stream>>>(n, io, c->s.v);
  if (a) CK(cudaMemcpyAsync(io, a, v3, cudaMemcpyDefault, c->stream));
  k_in_vec<<<g, 256, 0, c->stream>>>(n, a ? io : nullptr, c->s.a);
  k_finish_in<<<g, 256, 0, c->stream>>>(n, c->s);
  if (c->s.ap) {
    CK(cudaMemsetAsync(c->s.ap, 0, sizeof(float4) * (size_t)n, c->stream));
    CK(cudaMemsetAsync(c->s.err, 0, sizeof(float) * (size_t)n, c->stream));
    c->minor = 0;
    c->n_minor_cur = c->p.n_minor;
    c->clean = 0;
    c->shorten_now = 0;
  }
  CK(cudaGetLastError());
  // the staging buffers are reused by the next call: finish before returning
  CK(cudaStreamSynchronize(c->stream));
  return RTS_OK;
}

// --------------------------------------------------------------- status ---

static rts_status sync_status(rts_ctx* c) {
  CK(cudaMemcpyAsync(c->h_ctl, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaGetLastError());
  int st = c->h_ctl->status;
  if (st != 0 && st != RTS_ERR_NOT_CONVERGED) {
    c->sticky = st;
    const char* what = st == RTS_ERR_DOMAIN     ? "a particle left the block grid (or is NaN)"
                       : st == RTS_ERR_CAPACITY ? "a block or neighbour list exceeded its capacity"
                       : st == RTS_ERR_TIMEOUT  ? "a bounded device wait gave up"
                       : st == RTS_ERR_INTERNAL ? "a device-side consistency check failed"
                                                : "device error";
    const Ctl* h = c->h_ctl;
    if (st == RTS_ERR_DOMAIN && h->bad_set)
      snprintf(c->err, sizeof c->err, "device status %d: %s (particle %u at %g %g %g)", st, what,
               h->bad_uid, (double)h->bad_x, (double)h->bad_y, (double)h->bad_z);
    else if (st == RTS_ERR_INTERNAL)
      snprintf(c->err, sizeof c->err, "device status %d: %s (check %d, value %u)", st, what,
               h->chk_code, h->chk_val);
    else
      snprintf(c->err, sizeof c->err, "device status %d: %s", st, what);
    return (rts_status)st;
  }
  return (rts_status)st;
}

// --------------------------------------------------------- WCSPH stepping ---

// Density and forces of the evaluated particles; their Serna correction is deferred to
// the next key pass (which reads the same flags and accelerations) or to finalize().
static void run_physics(rts_ctx* c, int64_t k1, int prime, bool stale = false) {
  // global adaptive stepping: the force pass also forms the maxima that choose the next
  // step (of the state the deferred correction will give)
  const int gmode = c->p.mode == RTS_MODE_GLOBAL_ADAPTIVE ? (prime ? 2 : 1) : 0;
  { Phase ph(c, RTS_PHASE_DENSITY); launch_density(c, stale); }
  { Phase ph(c, RTS_PHASE_FORCE); launch_force(c, gmode, k1); }
  c->gmax_ok = gmode != 0;
  c->pend_mode = prime ? kPendPrime : kPendCorrect;
  c->pend_k1 = k1;
  // the force pass cleared the filled list; the next classification outside the
  // stepping loop bins the (corrected) positions afresh
  c->bins_valid = 0;
}

// Apply a deferred correction now (before the state is read or classified directly).
rts_status rts::finalize(rts_ctx* c) {
  if (c->pend_mode == kPendNone) return RTS_OK;
  Phase ph(c, RTS_PHASE_CORRECT);
  launch_correct(c, c->pend_k1, c->pend_mode == kPendPrime);
  c->pend_mode = kPendNone;
  return RTS_OK;
}

static rts_status wcsph_evaluate(rts_ctx* c) {
  { Phase ph(c, RTS_PHASE_BIN); launch_bin(c, 0.0f); }
  { Phase ph(c, RTS_PHASE_CLASSIFY); launch_classify(c, false); }
  { Phase ph(c, RTS_PHASE_ACTIVITY); launch_activity(c, kActAll, 0, 0, c->k, false); }
  run_physics(c, c->k, 1);
  c->primed = 1;
  CK(cudaGetLastError());
  return RTS_OK;
}

// Substeps that keep the last sort (stale_bins = S > 1, level-aligned clock): on a
// substep k1 that is not a multiple of S the particles are not re-sorted.  With
// S = level_mult[1] those are the substeps at which only the finest level is due, so
// their evaluations are few (the finest level and pre-emptions); the sort that the
// others need is done then.  Classification and activity use the current blocks; the
// density pass widens its search by how far particles have left their sorted blocks.
static bool keeps_sort(const rts_ctx* c, int64_t k1) {
  const rts_params& p = c->p;
  return c->light_ok && p.stale_bins > 1 && p.level_clock && p.mode == RTS_MODE_REGIONAL &&
         p.force_level < 0 && (k1 % p.stale_bins) != 0 && c->dp.nblocks < (1 << 24);
}

static rts_status wcsph_regional(rts_ctx* c) {
  int64_t k1 = c->k + 1;
  const bool keep = keeps_sort(c, k1);
  {
    Phase ph(c, RTS_PHASE_BIN);
    if (keep) launch_bin_light(c, c->p.dt_b);
    else launch_bin(c, c->p.dt_b);
  }
  { Phase ph(c, RTS_PHASE_CLASSIFY); launch_classify(c, keep); }
  { Phase ph(c, RTS_PHASE_ACTIVITY); launch_activity(c, kActRegional, 0, 0, k1, keep); }
  run_physics(c, k1, 0, keep);
  c->k = k1;
  if (keep) ++c->kept_sorts;
  CK(cudaGetLastError());
  return RTS_OK;
}

static int host_pick_level(const rts_ctx* c, double v2, double a2) {
  int L = 0;
  for (int l = 0; l < c->dp.n_levels; ++l)
    if (c->dp.eq1[l] && v2 <= c->dp.vthr2[l] && a2 <= c->dp.athr2[l]) L = l;
  return L;
}

int rts::pick_level_from_f32_max(const DevParams& d, float v2, float a2) {
  int L = 0;
  for (int l = 0; l < d.n_levels; ++l) {
    const float tv = d.vthr2f[l], ta = d.athr2f[l];
    if ((std::isfinite(tv) && std::fabs(v2 - tv) <= 1e-5f * tv) ||
        (std::isfinite(ta) && std::fabs(a2 - ta) <= 1e-5f * ta) || !std::isfinite(v2) ||
        !std::isfinite(a2))
      return -1;
    if (d.eq1[l] && v2 <= tv && a2 <= ta) L = l;
  }
  return L;
}

static rts_status wcsph_global(rts_ctx* c, int64_t max_mult) {
  int L = 0;
  if (c->p.mode == RTS_MODE_GLOBAL_ADAPTIVE) {
    // the step size is chosen from the corrected state: its FP32 maxima were formed by the
    // last force pass (the correction itself stays deferred to the next key pass), else
    // by a pass over the corrected state
    if (!c->gmax_ok) {
      finalize(c);
      Phase ph(c, RTS_PHASE_CLASSIFY);
      launch_global_max(c, 0);
    }
    CK(cudaMemcpyAsync(&c->h_ctl->vmax2f_bits, &c->ctl->vmax2f_bits, 2 * sizeof(unsigned int),
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    float v2f, a2f;
    memcpy(&v2f, &c->h_ctl->vmax2f_bits, sizeof v2f);
    memcpy(&a2f, &c->h_ctl->amax2f_bits, sizeof a2f);
    L = pick_level_from_f32_max(c->dp, v2f, a2f);
    if (L < 0) {   // a maximum at a threshold: the FP64 maxima decide
      finalize(c);
      {
        Phase ph(c, RTS_PHASE_CLASSIFY);
        launch_global_max(c, 1);
      }
      CK(cudaMemcpyAsync(&c->h_ctl->vmax2_bits, &c->ctl->vmax2_bits,
                         2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      double v2, a2;
      memcpy(&v2, &c->h_ctl->vmax2_bits, sizeof v2);
      memcpy(&a2, &c->h_ctl->amax2_bits, sizeof a2);
      L = host_pick_level(c, v2, a2);
    }
  }
  int64_t m = c->p.level_mult[L];
  if (m > max_mult) m = max_mult;
  if (m < 1) m = 1;
  int64_t k1 = c->k + m;
  { Phase ph(c, RTS_PHASE_BIN); launch_bin(c, (float)m * c->p.dt_b); }
  { Phase ph(c, RTS_PHASE_ACTIVITY); launch_activity(c, kActGlobal, L, (int)m, k1, false); }
  c->last_global_level = L;
  run_physics(c, k1, 0);
  c->k = k1;
  CK(cudaGetLastError());
  return RTS_OK;
}

static rts_status wcsph_step(rts_ctx* c, int64_t max_mult) {
  rts_status st;
  if (!c->primed && (st = wcsph_evaluate(c)) != RTS_OK) return st;
  if (c->p.mode == RTS_MODE_REGIONAL) return wcsph_regional(c);
  return wcsph_global(c, max_mult);
}

// ================================================================ C ABI ===

extern "C" {

}  // extern "C"

// Context constructor behind rts_init and rts_batch_init (batch: the stacked grid's
// parameters and the scene tables, owned by the context from here on).
static rts_status init_ctx(const rts_params* params, int32_t n_fluid, const float* x,
                           const float* v, int32_t n_boundary, const float* xb, void* cuda_stream,
                           rts_ctx** out, BatchState* batch) {
  if (!out) {
    rts::batch_delete(batch);
    return fail(nullptr, RTS_ERR_ARG, "out is NULL");
  }
  *out = nullptr;
  const char* why = validate_params(params, n_fluid, n_boundary, batch ? 65536 : 4096);
  if (!why && n_fluid > 0 && (!x || !v)) why = "x and v are required";
  if (!why && n_boundary > 0 && !xb) why = "xb is required";
  if (why) {
    rts::batch_delete(batch);
    return fail(nullptr, RTS_ERR_ARG, why);
  }
  rts_ctx* c = new (std::nothrow) rts_ctx;
  if (!c) {
    rts::batch_delete(batch);
    return fail(nullptr, RTS_ERR_OOM, "host allocation failed");
  }
  memset(c, 0, sizeof(*c));
  c->p = *params;
  make_dev_params(c->p, c->dp);
  c->dp.n_fluid = n_fluid;
  c->dp.n_bound = n_boundary;
  if (batch) {
    rts_status bst = rts_batch_attach(c, batch);
    if (bst != RTS_OK) {
      snprintf(g_noctx_err, sizeof g_noctx_err, "%s", c->err);
      rts_destroy(c);
      return bst;
    }
  }
  c->stream = (cudaStream_t)cuda_stream;
  c->n = n_fluid;
  c->nb = n_boundary;
  int n1 = n_fluid > 0 ? n_fluid : 1;
  size_t nbk = (size_t)c->dp.nblocks;
  c->ntiles = (int)((nbk + 2047) / 2048);
  rts_status st = RTS_OK;
#define ALLOC(ptr, bytes)                                                    \
  do {                                                                       \
    cudaError_t _e = cudaMalloc((void**)&(ptr), (bytes));                    \
    if (_e != cudaSuccess) {                                                 \
      rts::cuda_err(c, _e, "cudaMalloc " #ptr);                              \
      st = RTS_ERR_OOM;                                                      \
      goto fail_alloc;                                                       \
    }                                                                        \
  } while (0)
  {
    size_t f4 = sizeof(float4) * n1, f1 = sizeof(float) * n1, u1 = sizeof(uint32_t) * n1;
    PState* ss[2] = {&c->s, &c->s2};
    for (PState* s : ss) {
      ALLOC(s->x, f4);
      ALLOC(s->v, f4);
      ALLOC(s->a, f4);
      ALLOC(s->rho, f1);
      ALLOC(s->prs, f1);
      ALLOC(s->uid, u1);
      ALLOC(s->klast, u1);
      ALLOC(s->valid, u1);
      ALLOC(s->level, u1);
      ALLOC(s->nbr, u1);
    }
    ALLOC(c->anew, f4);
    ALLOC(c->cflag, (size_t)n1);
    ALLOC(c->key, u1);
    ALLOC(c->key_cur, u1);
    ALLOC(c->key_tmp, u1);
    ALLOC(c->slot, u1);
    ALLOC(c->tmp_uid, u1);
    ALLOC(c->tmp_src, u1);
    ALLOC(c->io, sizeof(float) * 4 * (size_t)n1);
    ALLOC(c->io_i, u1);
    ALLOC(c->count, sizeof(uint32_t) * nbk);
    ALLOC(c->cstart, sizeof(uint32_t) * (nbk + 1));
    ALLOC(c->bcstart, sizeof(uint32_t) * (nbk + 1));
    ALLOC(c->tile_sums, sizeof(uint32_t) * (size_t)c->ntiles);
    ALLOC(c->raw, sizeof(uint32_t) * nbk);
    ALLOC(c->blevel, sizeof(uint32_t) * nbk);
    ALLOC(c->bmax_v, sizeof(unsigned long long) * nbk);
    ALLOC(c->bmax_a, sizeof(unsigned long long) * nbk);
    ALLOC(c->filled, sizeof(uint32_t) * nbk);
    ALLOC(c->filled_new, sizeof(uint32_t) * nbk);
    ALLOC(c->near_list, sizeof(uint32_t) * kNearCap);
    c->nbl_cap = c->dp.nbl_cap;
    ALLOC(c->nbl, sizeof(uint32_t) * (size_t)n1 * (size_t)c->nbl_cap);
    ALLOC(c->buid, sizeof(uint32_t) * (size_t)(n_boundary > 0 ? n_boundary : 1));
    if (params->scheme == RTS_PCISPH) {
      for (PState* s : ss) {
        ALLOC(s->ap, f4);
        ALLOC(s->err, f1);
      }
      ALLOC(c->xs, f4);
      ALLOC(c->pbak, f1);
      ALLOC(c->in_se, (size_t)n1);
      ALLOC(c->in_re, nbk);
      ALLOC(c->ob, nbk);
      ALLOC(c->preg, sizeof(int32_t) * nbk);
      ALLOC(c->pnew, sizeof(int32_t) * nbk);
    }
    ALLOC(c->act, sizeof(uint32_t) * nbk);
    ALLOC(c->plist, u1);
    ALLOC(c->actflag, sizeof(uint32_t) * nbk);
    ALLOC(c->ctl, sizeof(Ctl));
    ALLOC(c->xb, sizeof(float4) * (size_t)(n_boundary > 0 ? n_boundary : 1));
    if (cudaMallocHost((void**)&c->h_ctl, sizeof(Ctl)) != cudaSuccess) {
      st = fail(c, RTS_ERR_OOM, "pinned host allocation failed");
      goto fail_alloc;
    }
  }
#undef ALLOC
  {
    cudaError_t e = cudaMemsetAsync(c->count, 0, sizeof(uint32_t) * nbk, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ctl, 0, sizeof(Ctl), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->raw, 0, sizeof(uint32_t) * nbk, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->blevel, 0, sizeof(uint32_t) * nbk, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->actflag, 0, sizeof(uint32_t) * nbk, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->bmax_v, 0, sizeof(unsigned long long) * nbk, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->bmax_a, 0, sizeof(unsigned long long) * nbk, c->stream);
    if (e == cudaSuccess && c->preg) e = cudaMemsetAsync(c->preg, 0xff, sizeof(int32_t) * nbk, c->stream);
    if (e == cudaSuccess && c->ob) e = cudaMemsetAsync(c->ob, 0, nbk, c->stream);
    c->stamp = 0;
    c->n_minor_cur = params->n_minor;
    if (e != cudaSuccess) {
      rts::cuda_err(c, e, "initial memset");
      st = RTS_ERR_CUDA;
      goto fail_alloc;
    }
  }
  c->grid_persistent = neighbor_grid_size();
  if (n_boundary > 0) {
    float *tmp3 = nullptr;
    float4* tmp4 = nullptr;
    size_t b3 = sizeof(float) * 3 * (size_t)n_boundary;
    cudaError_t e = cudaMalloc((void**)&tmp3, b3);
    if (e == cudaSuccess) e = cudaMalloc((void**)&tmp4, sizeof(float4) * (size_t)n_boundary);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp3, xb, b3, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) {
      k_pack3<<<nblk(n_boundary), 256, 0, c->stream>>>(n_boundary, tmp3, tmp4);
      st = launch_bin_boundary(c, tmp4, n_boundary);
    }
    cudaFree(tmp3);
    cudaFree(tmp4);
    if (e != cudaSuccess) {
      rts::cuda_err(c, e, "boundary upload");
      st = RTS_ERR_CUDA;
    }
    if (st != RTS_OK) goto fail_alloc;
    st = sync_status(c);
    if (st != RTS_OK) goto fail_alloc;
  } else {
    cudaMemsetAsync(c->bcstart, 0, sizeof(uint32_t) * (nbk + 1), c->stream);
  }
  if (n_fluid > 0) {
    st = upload_state(c, x, v, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    if (st != RTS_OK) goto fail_alloc;
  }
  c->k = 0;
  c->primed = 0;
  c->bins_valid = 0;
  *out = c;
  return RTS_OK;
fail_alloc:
  if (c->err[0]) snprintf(g_noctx_err, sizeof g_noctx_err, "%s", c->err);
  rts_destroy(c);
  return st;
}

extern "C" {

rts_status rts_init(const rts_params* params, int32_t n_fluid, const float* x, const float* v,
                    int32_t n_boundary, const float* xb, void* cuda_stream, rts_ctx** out) {
  return init_ctx(params, n_fluid, x, v, n_boundary, xb, cuda_stream, out, nullptr);
}

rts_status rts_batch_init(const rts_params* params, int32_t n_scenes, const rts_scene* scenes,
                          const float* x, const float* v, const float* xb, void* cuda_stream,
                          rts_ctx** out) {
  if (!out) return fail(nullptr, RTS_ERR_ARG, "out is NULL");
  *out = nullptr;
  rts_params p2;
  int32_t nf = 0, nbd = 0;
  BatchState* b = nullptr;
  if (const char* why = rts_batch_plan(params, n_scenes, scenes, &p2, &nf, &nbd, &b))
    return fail(nullptr, RTS_ERR_ARG, why);
  return init_ctx(&p2, nf, x, v, nbd, xb, cuda_stream, out, b);
}

rts_status rts_destroy(rts_ctx* c) {
  if (!c) return RTS_OK;
  cudaStreamSynchronize(c->stream);
  batch_free(c);
  PState* ss[2] = {&c->s, &c->s2};
  for (PState* s : ss) {
    cudaFree(s->x); cudaFree(s->v); cudaFree(s->a); cudaFree(s->rho); cudaFree(s->prs);
    cudaFree(s->uid); cudaFree(s->klast); cudaFree(s->valid); cudaFree(s->level); cudaFree(s->nbr);
  }
  cudaFree(c->anew); cudaFree(c->cflag); cudaFree(c->key); cudaFree(c->key_cur); cudaFree(c->key_tmp); cudaFree(c->slot);
  cudaFree(c->tmp_uid); cudaFree(c->tmp_src); cudaFree(c->io); cudaFree(c->io_i);
  cudaFree(c->count); cudaFree(c->cstart); cudaFree(c->bcstart); cudaFree(c->tile_sums);
  cudaFree(c->raw); cudaFree(c->blevel); cudaFree(c->act); cudaFree(c->plist); cudaFree(c->actflag); cudaFree(c->ctl); cudaFree(c->xb);
  cudaFree(c->bmax_v); cudaFree(c->bmax_a); cudaFree(c->filled); cudaFree(c->filled_new); cudaFree(c->near_list); cudaFree(c->nbl);
  cudaFree(c->buid); cudaFree(c->s.ap); cudaFree(c->s2.ap); cudaFree(c->s.err); cudaFree(c->s2.err);
  cudaFree(c->xs); cudaFree(c->pbak); cudaFree(c->in_se); cudaFree(c->in_re); cudaFree(c->ob);
  cudaFree(c->preg); cudaFree(c->pnew);
  if (c->h_ctl) cudaFreeHost(c->h_ctl);
  if (c->ev) {
    for (int k = 0; k < 2 * kEvPairs; ++k) cudaEventDestroy(c->ev[k]);
    delete[] c->ev;
    delete[] c->ev_phase;
  }
  delete c;
  return RTS_OK;
}

const char* rts_last_error(const rts_ctx* c) { return c ? c->err : g_noctx_err; }

int64_t rts_num_blocks(const rts_ctx* c) { return c ? (int64_t)c->dp.nblocks : 0; }

int64_t rts_substep_index(const rts_ctx* c) { return c ? c->k : 0; }

rts_status rts_sync(rts_ctx* c) {
  if (!c) return fail(nullptr, RTS_ERR_ARG, "ctx is NULL");
  return sync_status(c);
}

#define GUARD()                                                                  \
  do {                                                                           \
    if (!c) return fail(nullptr, RTS_ERR_ARG, "ctx is NULL");                    \
    if (c->sticky) return fail(c, RTS_ERR_STATE, "a device error is pending; call rts_set_state"); \
  } while (0)

rts_status rts_bin(rts_ctx* c) {
  GUARD();
  Phase ph(c, RTS_PHASE_BIN);
  launch_bin(c, 0.0f);
  c->bins_valid = 1;
  CK(cudaGetLastError());
  return RTS_OK;
}

rts_status rts_classify_blocks(rts_ctx* c) {
  GUARD();
  finalize(c);
  if (!c->bins_valid) {
    Phase ph(c, RTS_PHASE_BIN);
    launch_bin(c, 0.0f);
  }
  c->bins_valid = 1;
  {
    Phase ph(c, RTS_PHASE_CLASSIFY);
    launch_classify(c, false);
  }
  {
    Phase ph(c, RTS_PHASE_ACTIVITY);
    launch_activity(c, -1, 0, 0, c->k, false);
  }
  CK(cudaGetLastError());
  return RTS_OK;
}

rts_status rts_evaluate(rts_ctx* c) {
  GUARD();
  if (c->p.scheme != RTS_WCSPH) return fail(c, RTS_ERR_ARG, "rts_evaluate is the WCSPH evaluation");
  rts_status st = wcsph_evaluate(c);
  if (st == RTS_OK) finalize(c);
  return st;
}

rts_status rts_wcsph_substep(rts_ctx* c) {
  GUARD();
  if (c->p.scheme != RTS_WCSPH) return fail(c, RTS_ERR_ARG, "context was created for PCISPH");
  rts_status st = wcsph_step(c, (int64_t)1 << 40);
  finalize(c);
  return st;
}

rts_status rts_advance(rts_ctx* c, double t_sim, rts_stats* out) {
  GUARD();
  if (!std::isfinite(t_sim)) return fail(c, RTS_ERR_ARG, "t_sim must be finite");
  int64_t K = llround(t_sim / (double)c->p.dt_b);
  CK(cudaMemsetAsync(&c->ctl->evals, 0, 5 * sizeof(unsigned long long), c->stream));
  int64_t k0 = c->k, steps = 0;
  int64_t it0 = c->tot_iters, lo0 = c->tot_local, rv0 = c->tot_reverts;
  rts_status nconv = RTS_OK;
  rts_status st = RTS_OK;
  while (c->k < K) {
    if (c->p.scheme == RTS_WCSPH) {
      st = wcsph_step(c, K - c->k);
    } else {
      st = pcisph_step(c, K - c->k);
    }
    if (st != RTS_OK && st != RTS_ERR_NOT_CONVERGED) return st;
    if (st == RTS_ERR_NOT_CONVERGED) nconv = st;
    ++steps;
  }
  finalize(c);
  {
    Phase ph(c, RTS_PHASE_OTHER);
    launch_level_hist(c);
  }
  rts_status ds = sync_status(c);
  if (out) {
    memset(out, 0, sizeof(*out));
    out->substeps = c->k - k0;
    out->steps = steps;
    out->particle_evals = (int64_t)c->h_ctl->evals;
    out->pair_interactions = (int64_t)c->h_ctl->pairs;
    out->active_blocks = (int64_t)c->h_ctl->act_blocks;
    out->candidate_tests = (int64_t)c->h_ctl->cands;
    out->tests_performed = (int64_t)c->h_ctl->kept;
    out->pcisph_iterations = c->tot_iters - it0;
    out->pcisph_local_iterations = c->tot_local - lo0;
    out->pcisph_global_restarts = c->tot_reverts - rv0;
    for (int L = 0; L < kMaxLevels; ++L) out->level_count[L] = (int64_t)c->h_ctl->level_count[L];
    out->t_sim = (double)c->k * (double)c->p.dt_b;
  }
  return ds != RTS_OK ? ds : nconv;
}

rts_status rts_get_state(rts_ctx* c, float* x, float* v, float* a, float* rho, float* p,
                         int32_t* level, int32_t* validity, int32_t* klast, int32_t* nbr,
                         uint8_t* compute) {
  if (!c) return fail(nullptr, RTS_ERR_ARG, "ctx is NULL");
  finalize(c);
  int n = c->n;
  if (n == 0) return sync_status(c);
  int g = nblk(n);
  size_t v3 = sizeof(float) * 3 * (size_t)n, s1 = sizeof(float) * (size_t)n;
  Phase ph(c, RTS_PHASE_OTHER);
  note_launch(c, (x != nullptr) + (v != nullptr) + (a != nullptr) + (rho != nullptr) +
                     (p != nullptr) + (level != nullptr) + (validity != nullptr) +
                     (klast != nullptr) + (nbr != nullptr) + (compute != nullptr));
  const float4* vecs[3] = {c->s.x, c->s.v, c->s.a};
  float* vdst[3] = {x, v, a};
  for (int k = 0; k < 3; ++k) {
    if (!vdst[k]) continue;
    k_out_vec<<<g, 256, 0, c->stream>>>(n, c->s.uid, vecs[k], c->io, c->ctl);
    CK(cudaMemcpyAsync(vdst[k], c->io, v3, cudaMemcpyDefault, c->stream));
  }
  const float* fs[2] = {c->s.rho, c->s.prs};
  float* fdst[2] = {rho, p};
  for (int k = 0; k < 2; ++k) {
    if (!fdst[k]) continue;
    k_out_scalar<float><<<g, 256, 0, c->stream>>>(n, c->s.uid, fs[k], c->io, c->ctl);
    CK(cudaMemcpyAsync(fdst[k], c->io, s1, cudaMemcpyDefault, c->stream));
  }
  const int32_t* is[4] = {c->s.level, c->s.valid, c->s.klast, c->s.nbr};
  int32_t* idst[4] = {level, validity, klast, nbr};
  for (int k = 0; k < 4; ++k) {
    if (!idst[k]) continue;
    k_out_scalar<int32_t><<<g, 256, 0, c->stream>>>(n, c->s.uid, is[k], c->io_i, c->ctl);
    CK(cudaMemcpyAsync(idst[k], c->io_i, s1, cudaMemcpyDefault, c->stream));
  }
  if (compute) {
    k_out_scalar<uint8_t><<<g, 256, 0, c->stream>>>(n, c->s.uid, c->cflag, (uint8_t*)c->io_i, c->ctl);
    CK(cudaMemcpyAsync(compute, c->io_i, (size_t)n, cudaMemcpyDefault, c->stream));
  }
  CK(cudaGetLastError());
  return sync_status(c);
}

rts_status rts_set_state(rts_ctx* c, const float* x, const float* v, const float* a,
                         const float* rho, const float* p, const int32_t* level,
                         const int32_t* validity, const int32_t* klast, int64_t k,
                         int32_t primed) {
  if (!c) return fail(nullptr, RTS_ERR_ARG, "ctx is NULL");
  if (c->n > 0 && (!x || !v)) return fail(c, RTS_ERR_ARG, "x and v are required");
  if (k < 0) return fail(c, RTS_ERR_ARG, "k must be >= 0");
  c->pend_mode = kPendNone;  // the new state replaces any deferred correction
  rts_status st = upload_state(c, x, v, a, rho, p, level, validity, klast);
  if (st != RTS_OK) return st;
  CK(cudaMemsetAsync(c->ctl, 0, sizeof(Ctl), c->stream));
  CK(cudaMemsetAsync(c->cflag, 0, (size_t)(c->n > 0 ? c->n : 1), c->stream));
  c->sticky = 0;
  c->k = k;
  c->primed = primed ? 1 : 0;
  c->err[0] = 0;
  {
    Phase ph(c, RTS_PHASE_BIN);
    launch_bin(c, 0.0f);
  }
  c->bins_valid = 1;
  return sync_status(c);
}

rts_status rts_get_bins(rts_ctx* c, int32_t* key, int32_t* perm, int32_t* cstart) {
  if (!c) return fail(nullptr, RTS_ERR_ARG, "ctx is NULL");
  rts_status st = sync_status(c);
  if (st != RTS_OK) return st;
  int n = c->n;
  size_t nbk = (size_t)c->dp.nblocks;
  std::vector<uint32_t> hk(n), hu(n);
  if (n > 0) {
    CK(cudaMemcpy(hk.data(), c->key, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hu.data(), c->s.uid, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost));
  }
  if (key) {
    std::vector<int32_t> ku(n);
    for (int f = 0; f < n; ++f) ku[hu[f]] = (int32_t)hk[f];
    CK(cudaMemcpy(key, ku.data(), sizeof(int32_t) * n, cudaMemcpyDefault));
  }
  if (perm) CK(cudaMemcpy(perm, hu.data(), sizeof(int32_t) * n, cudaMemcpyDefault));
  if (cstart) CK(cudaMemcpy(cstart, c->cstart, sizeof(uint32_t) * (nbk + 1), cudaMemcpyDefault));
  return RTS_OK;
}

rts_status rts_get_blocks(rts_ctx* c, int32_t* raw, int32_t* level) {
  if (!c) return fail(nullptr, RTS_ERR_ARG, "ctx is NULL");
  rts_status st = sync_status(c);
  if (st != RTS_OK) return st;
  size_t nbk = (size_t)c->dp.nblocks;
  std::vector<uint32_t> h(nbk);
  std::vector<int32_t> w(nbk);
  const uint32_t* src[2] = {c->raw, c->blevel};
  int32_t* dst[2] = {raw, level};
  for (int k = 0; k < 2; ++k) {
    if (!dst[k]) continue;
    if (k == 1 && c->preg) {
      // PCISPH: the region field of the current major step (after expansion and
      // pre-emption), -1 for blocks without fluid
      CK(cudaMemcpy(dst[k], c->preg, sizeof(int32_t) * nbk, cudaMemcpyDefault));
      continue;
    }
    CK(cudaMemcpy(h.data(), src[k], sizeof(uint32_t) * nbk, cudaMemcpyDeviceToHost));
    // records of this binning pass hold a level; every other block has no fluid
    for (size_t b = 0; b < nbk; ++b) w[b] = (h[b] >> 8) == c->stamp ? (int32_t)(h[b] & 0xffu) : -1;
    CK(cudaMemcpy(dst[k], w.data(), sizeof(int32_t) * nbk, cudaMemcpyDefault));
  }
  return RTS_OK;
}

rts_status rts_profile_enable(rts_ctx* c, int32_t on) {
  if (!c) return fail(nullptr, RTS_ERR_ARG, "ctx is NULL");
  if (on && !c->ev) {
    c->ev = new (std::nothrow) cudaEvent_t[2 * kEvPairs];
    c->ev_phase = new (std::nothrow) int[kEvPairs];
    if (!c->ev || !c->ev_phase) return fail(c, RTS_ERR_OOM, "event pool allocation failed");
    for (int k = 0; k < 2 * kEvPairs; ++k) CK(cudaEventCreate(&c->ev[k]));
    c->nev = 0;
  }
  if (on < 0 || on > 2) return fail(c, RTS_ERR_ARG, "profile level must be 0, 1 or 2");
  if (!on) prof_flush(c);
  c->prof = on;
  return RTS_OK;
}

rts_status rts_profile_read(rts_ctx* c, rts_profile* out, int32_t reset) {
  if (!c || !out) return fail(c, RTS_ERR_ARG, "ctx or out is NULL");
  prof_flush(c);
  CK(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < RTS_NUM_PHASES; ++k) {
    out->ms[k] = c->prof_ms[k];
    out->launches[k] = c->launches[k];
    out->timed[k] = c->prof_timed[k];
    out->passes[k] = c->passes[k];
  }
  out->kernels = c->kernels;
  if (reset) {
    memset(c->prof_ms, 0, sizeof c->prof_ms);
    memset(c->launches, 0, sizeof c->launches);
    memset(c->prof_timed, 0, sizeof c->prof_timed);
    memset(c->prof_seen, 0, sizeof c->prof_seen);
    memset(c->passes, 0, sizeof c->passes);
    c->kernels = 0;
  }
  return RTS_OK;
}

rts_status rts_pcisph_step(rts_ctx* c) {
  GUARD();
  if (c->p.scheme != RTS_PCISPH) return fail(c, RTS_ERR_ARG, "context was created for WCSPH");
  return pcisph_step(c, (int64_t)1 << 40);
}

rts_status rts_pcisph_last(rts_ctx* c, rts_pcisph_info* out) {
  if (!c || !out) return fail(c, RTS_ERR_ARG, "ctx or out is NULL");
  out->iterations = c->it_iters;
  out->global_iterations = c->it_global;
  out->local_iterations = c->it_local;
  out->reverts = c->it_reverts;
  out->not_converged = c->it_notconv;
  out->minor = c->minor;
  out->n_minor_current = c->n_minor_cur;
  out->clean_majors = c->clean;
  out->err_max = c->it_errmax;
  out->err_avg = c->it_erravg;
  return RTS_OK;
}

rts_status rts_get_pcisph_state(rts_ctx* c, float* ap, float* err, uint8_t* in_se) {
  if (!c) return fail(nullptr, RTS_ERR_ARG, "ctx is NULL");
  if (c->p.scheme != RTS_PCISPH) return fail(c, RTS_ERR_ARG, "context was created for WCSPH");
  int n = c->n;
  if (n == 0) return sync_status(c);
  int g = nblk(n);
  Phase ph(c, RTS_PHASE_OTHER);
  if (ap) {
    note_launch(c, 1);
    k_out_vec<<<g, 256, 0, c->stream>>>(n, c->s.uid, c->s.ap, c->io, c->ctl);
    CK(cudaMemcpyAsync(ap, c->io, sizeof(float) * 3 * (size_t)n, cudaMemcpyDefault, c->stream));
  }
  if (err) {
    note_launch(c, 1);
    k_out_scalar<float><<<g, 256, 0, c->stream>>>(n, c->s.uid, c->s.err, c->io, c->ctl);
    CK(cudaMemcpyAsync(err, c->io, sizeof(float) * (size_t)n, cudaMemcpyDefault, c->stream));
  }
  if (in_se) {
    note_launch(c, 1);
    k_out_scalar<uint8_t><<<g, 256, 0, c->stream>>>(n, c->s.uid, c->in_se, (uint8_t*)c->io_i, c->ctl);
    CK(cudaMemcpyAsync(in_se, c->io_i, (size_t)n, cudaMemcpyDefault, c->stream));
  }
  CK(cudaGetLastError());
  return sync_status(c);
}

rts_status rts_get_neighbors(rts_ctx* c, int32_t* counts, int32_t* idx, int32_t cap) {
  if (!c || !counts || (idx && cap < 1)) return fail(c, RTS_ERR_ARG, "bad arguments");
  rts_status st = sync_status(c);
  if (st != RTS_OK && st != RTS_ERR_NOT_CONVERGED) return st;
  int n = c->n, nb = c->nb;
  if (n == 0) return RTS_OK;
  std::vector<uint32_t> uid(n), buid(nb > 0 ? nb : 1), lists((size_t)n * c->nbl_cap);
  std::vector<int32_t> cnt(n), ocnt(n);
  CK(cudaMemcpy(uid.data(), c->s.uid, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost));
  if (nb > 0) CK(cudaMemcpy(buid.data(), c->buid, sizeof(uint32_t) * nb, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(cnt.data(), c->s.nbr, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(lists.data(), c->nbl, sizeof(uint32_t) * lists.size(), cudaMemcpyDeviceToHost));
  std::vector<int32_t> out(idx ? (size_t)n * cap : 0, -1);
  for (int f = 0; f < n; ++f) {
    if (uid[f] >= (uint32_t)n) return fail(c, RTS_ERR_INTERNAL, "rts_get_neighbors: caller index out of range");
    int u = (int)uid[f];
    int k = cnt[f] < c->nbl_cap ? cnt[f] : c->nbl_cap;
    if (k < 0) k = 0;
    ocnt[u] = k;
    if (!idx) continue;
    if (k > cap) return fail(c, RTS_ERR_CAPACITY, "rts_get_neighbors: cap smaller than a list");
    for (int e = 0; e < k; ++e) {
      uint32_t j = lists[(size_t)f * c->nbl_cap + e];
      if ((j & 0x80000000u) ? (j & 0x7fffffffu) >= (uint32_t)nb : j >= (uint32_t)n)
        return fail(c, RTS_ERR_INTERNAL, "rts_get_neighbors: neighbour index out of range");
      out[(size_t)u * cap + e] = (j & 0x80000000u) ? n + (int32_t)buid[j & 0x7fffffffu]
                                                   : (int32_t)uid[j];
    }
  }
  CK(cudaMemcpy(counts, ocnt.data(), sizeof(int32_t) * n, cudaMemcpyDefault));
  if (idx) CK(cudaMemcpy(idx, out.data(), sizeof(int32_t) * out.size(), cudaMemcpyDefault));
  return RTS_OK;
}

}  // extern "C"
