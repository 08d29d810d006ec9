// rts_bin_static.cu - block binning that allocates no device memory.
//
// Some callers cannot call cudaMalloc: hosts that reserve the whole device up front
// (a later allocation would fail), loops with a latency budget that an allocation's
// implicit synchronisation would break, and plugin environments whose host owns all
// device memory.  rts_bin_noalloc gives them the binning of rts_bin with its working
// memory in a fixed array compiled into this library.  That array exists once per
// device that loads the library and stays allocated until the process exits.
//
// The array is shared by every call.  Calls whose work overlaps on the GPU (different
// streams, or host threads racing) corrupt each other's results; serialise them.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "rts.h"

void rts_set_global_error(const char* msg);  // rts_api.cu

namespace {

constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;
constexpr int kTiles = RTS_NOALLOC_MAX_BLOCKS / kTile + 1;

// Layout of the fixed working memory.
struct Scratch {
  uint32_t count[RTS_NOALLOC_MAX_BLOCKS];       // per block, zeroed at the start of a call
  uint32_t tile_sums[kTiles];
  uint32_t slot[RTS_NOALLOC_MAX_PARTICLES];
  uint32_t tkey[RTS_NOALLOC_MAX_PARTICLES];
  uint32_t tuid[RTS_NOALLOC_MAX_PARTICLES];
  int status;                                   // 0, or RTS_ERR_DOMAIN
};

static __device__ __align__(256) Scratch g_scratch;

std::mutex g_mutex;
Scratch* g_addr[kMaxDevices] = {};

struct Grid {
  float ox, oy, oz, inv_edge;
  double oxd, oyd, ozd, edged;
  int nx, ny, nz, nblocks;
};

// floor((x - o) / edge) as the double-precision definition gives it: FP32 first, the
// FP64 quotient within 2e-3 of an integer (the same rule as rts_bin).
__device__ __forceinline__ int coord(float x, float o, double od, float inv_e, double ed, int n,
                                     int* bad) {
  float t = (x - o) * inv_e;
  float f = floorf(t);
  float fr = t - f;
  double fd = (fr < 2e-3f || fr > 0.998f) ? floor(__ddiv_rn(__dsub_rn((double)x, od), ed)) : (double)f;
  if (!(fd >= 0.0 && fd < (double)n)) {
    *bad = 1;
    return 0;
  }
  return (int)fd;
}

__global__ void k_key(Grid G, int n, const float* __restrict__ x, int32_t* __restrict__ key,
                      Scratch* S) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int bad = 0;
  int cx = coord(x[3 * i], G.ox, G.oxd, G.inv_edge, G.edged, G.nx, &bad);
  int cy = coord(x[3 * i + 1], G.oy, G.oyd, G.inv_edge, G.edged, G.ny, &bad);
  int cz = coord(x[3 * i + 2], G.oz, G.ozd, G.inv_edge, G.edged, G.nz, &bad);
  uint32_t b = ((uint32_t)cz * G.ny + cy) * G.nx + cx;
  if (bad) {
    atomicCAS(&S->status, 0, (int)RTS_ERR_DOMAIN);
    b = 0;
  }
  key[i] = (int32_t)b;
  S->slot[i] = atomicAdd(&S->count[b], 1u);
}

__device__ __forceinline__ uint32_t warp_scan(uint32_t v) {
  int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// The total has its own slot: with 32 warps it would overwrite the last warp's offset.
__device__ __forceinline__ uint32_t cta_excl_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t wt[33];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t inc = warp_scan(v);
  if (lane == 31) wt[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < nw ? wt[lane] : 0u;
    uint32_t ti = warp_scan(t);
    if (lane < nw) wt[lane] = ti - t;
    if (lane == nw - 1) wt[32] = ti;
  }
  __syncthreads();
  uint32_t r = inc - v + wt[w];
  *total = wt[32];
  __syncthreads();
  return r;
}

__global__ void k_tile_sums(int nb, Scratch* S) {
  int base = blockIdx.x * kTile + threadIdx.x * kItems;
  uint32_t s = 0;
  for (int k = 0; k < kItems; ++k)
    if (base + k < nb) s += S->count[base + k];
  uint32_t tot;
  cta_excl_scan(s, &tot);
  if (threadIdx.x == 0) S->tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_tile_sums(int ntiles, Scratch* S) {
  uint32_t carry = 0;
  for (int base = 0; base < ntiles; base += blockDim.x) {
    int i = base + threadIdx.x;
    uint32_t v = i < ntiles ? S->tile_sums[i] : 0u;
    uint32_t tot;
    uint32_t ex = cta_excl_scan(v, &tot);
    if (i < ntiles) S->tile_sums[i] = ex + carry;
    carry += tot;
  }
}

__global__ void k_starts(int nb, int32_t* __restrict__ cstart, Scratch* S) {
  int base = blockIdx.x * kTile + threadIdx.x * kItems;
  uint32_t c[kItems];
  uint32_t s = 0;
  for (int k = 0; k < kItems; ++k) {
    c[k] = base + k < nb ? S->count[base + k] : 0u;
    s += c[k];
  }
  uint32_t tot;
  uint32_t ex = cta_excl_scan(s, &tot) + S->tile_sums[blockIdx.x];
  for (int k = 0; k < kItems; ++k) {
    if (base + k < nb) cstart[base + k] = (int32_t)ex;
    ex += c[k];
  }
  if (base <= nb - 1 && nb - 1 < base + kItems) cstart[nb] = (int32_t)ex;
}

__global__ void k_place(int n, const int32_t* __restrict__ key, const int32_t* __restrict__ cstart,
                        Scratch* S) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t b = (uint32_t)key[i];
  uint32_t q = (uint32_t)cstart[b] + S->slot[i];
  S->tkey[q] = b;
  S->tuid[q] = (uint32_t)i;
}

// Within each block, order by particle index: rank among the block's entries.  The rank
// scans the block, so a block's cost grows with the square of its occupancy; a block
// holding more than RTS_NOALLOC_MAX_PER_BLOCK particles is not ranked and the call
// returns RTS_ERR_CAPACITY (at most n x RTS_NOALLOC_MAX_PER_BLOCK comparisons a call).
__global__ void k_rank(int n, const int32_t* __restrict__ cstart, int32_t* __restrict__ perm,
                       Scratch* S) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  uint32_t b = S->tkey[q];
  uint32_t beg = (uint32_t)cstart[b], end = (uint32_t)cstart[b + 1];
  if (end - beg > (uint32_t)RTS_NOALLOC_MAX_PER_BLOCK) {
    if (q == (int)beg) atomicCAS(&S->status, 0, (int)RTS_ERR_CAPACITY);
    return;
  }
  uint32_t u = S->tuid[q];
  uint32_t rank = 0;
  for (uint32_t r = beg; r < end; ++r) rank += S->tuid[r] < u ? 1u : 0u;
  perm[beg + rank] = (int32_t)u;
}

// Address of the fixed working memory on the current device (looked up once per device).
rts_status scratch_on_current_device(Scratch** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RTS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return RTS_ERR_CUDA;
    g_addr[dev] = static_cast<Scratch*>(p);
  }
  *out = g_addr[dev];
  return RTS_OK;
}

}  // namespace

static rts_status reject(rts_status st, const char* msg) {
  rts_set_global_error(msg);
  return st;
}

// A launch error of this call (read and cleared), reported with the kernel's name.
static bool launch_failed(const char* kernel) {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return false;
  char msg[256];
  snprintf(msg, sizeof msg, "rts_bin_noalloc: launching %s failed: %s", kernel,
           cudaGetErrorString(e));
  rts_set_global_error(msg);
  return true;
}

extern "C" rts_status rts_bin_noalloc(const rts_params* p, int32_t n, const float* x,
                                      int32_t* key, int32_t* perm, int32_t* cstart,
                                      void* cuda_stream) {
  if (!p || n < 0 || (n > 0 && (!x || !key || !perm)) || !cstart)
    return reject(RTS_ERR_ARG, "rts_bin_noalloc: NULL pointer or negative count");
  if (!(p->block_edge > 0.f)) return reject(RTS_ERR_ARG, "rts_bin_noalloc: block_edge must be positive");
  for (int d = 0; d < 3; ++d)
    if (p->grid_dim[d] < 1 || p->grid_dim[d] > 4096 || !std::isfinite(p->domain_min[d]))
      return reject(RTS_ERR_ARG, "rts_bin_noalloc: grid_dim must be in [1, 4096], domain_min finite");
  double nbd = (double)p->grid_dim[0] * p->grid_dim[1] * p->grid_dim[2];
  if (n > RTS_NOALLOC_MAX_PARTICLES || nbd > RTS_NOALLOC_MAX_BLOCKS)
    return reject(RTS_ERR_ARG,
                  "rts_bin_noalloc: more than RTS_NOALLOC_MAX_PARTICLES (262144) particles or "
                  "RTS_NOALLOC_MAX_BLOCKS (524288) blocks; its fixed working memory holds no more");
  {  // an error left by earlier work on this thread is not this call's: report it as such
    cudaError_t pre = cudaGetLastError();
    if (pre != cudaSuccess) {
      char msg[256];
      snprintf(msg, sizeof msg,
               "rts_bin_noalloc: a CUDA error from earlier work was pending (now cleared): %s; "
               "nothing was launched", cudaGetErrorString(pre));
      return reject(RTS_ERR_CUDA, msg);
    }
  }
  Scratch* S = nullptr;
  rts_status st = scratch_on_current_device(&S);
  if (st != RTS_OK) return reject(st, "rts_bin_noalloc: cudaGetSymbolAddress of the working memory failed");
  Grid G;
  G.ox = p->domain_min[0];
  G.oy = p->domain_min[1];
  G.oz = p->domain_min[2];
  G.inv_edge = 1.0f / p->block_edge;
  G.oxd = G.ox;
  G.oyd = G.oy;
  G.ozd = G.oz;
  G.edged = p->block_edge;
  G.nx = p->grid_dim[0];
  G.ny = p->grid_dim[1];
  G.nz = p->grid_dim[2];
  G.nblocks = G.nx * G.ny * G.nz;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the array keeps the previous call's contents: clear the counters and the status
  if (cudaMemsetAsync(S->count, 0, sizeof(uint32_t) * (size_t)G.nblocks, s) != cudaSuccess ||
      cudaMemsetAsync(&S->status, 0, sizeof(int), s) != cudaSuccess)
    return reject(RTS_ERR_CUDA, "rts_bin_noalloc: clearing the working memory failed");
  int g = (n + kThreads - 1) / kThreads;
  int ntiles = (G.nblocks + kTile - 1) / kTile;
  // each launch is checked before the next one is queued
  if (n > 0) {
    k_key<<<g, kThreads, 0, s>>>(G, n, x, key, S);
    if (launch_failed("k_key")) return RTS_ERR_CUDA;
  }
  k_tile_sums<<<ntiles, kThreads, 0, s>>>(G.nblocks, S);
  if (launch_failed("k_tile_sums")) return RTS_ERR_CUDA;
  k_scan_tile_sums<<<1, 1024, 0, s>>>(ntiles, S);
  if (launch_failed("k_scan_tile_sums")) return RTS_ERR_CUDA;
  k_starts<<<ntiles, kThreads, 0, s>>>(G.nblocks, cstart, S);
  if (launch_failed("k_starts")) return RTS_ERR_CUDA;
  if (n > 0) {
    k_place<<<g, kThreads, 0, s>>>(n, key, cstart, S);
    if (launch_failed("k_place")) return RTS_ERR_CUDA;
    k_rank<<<g, kThreads, 0, s>>>(n, cstart, perm, S);
    if (launch_failed("k_rank")) return RTS_ERR_CUDA;
  }
  int status = 0;
  cudaError_t e = cudaMemcpyAsync(&status, &S->status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    char msg[256];
    snprintf(msg, sizeof msg, "rts_bin_noalloc: reading the status failed: %s", cudaGetErrorString(e));
    return reject(RTS_ERR_CUDA, msg);
  }
  if (status == RTS_ERR_DOMAIN)
    return reject(RTS_ERR_DOMAIN, "rts_bin_noalloc: a particle lies outside the grid");
  if (status == RTS_ERR_CAPACITY)
    return reject(RTS_ERR_CAPACITY,
                  "rts_bin_noalloc: a block holds more than RTS_NOALLOC_MAX_PER_BLOCK particles");
  if (status) return reject(RTS_ERR_INTERNAL, "rts_bin_noalloc: unexpected device status");
  return RTS_OK;
}
