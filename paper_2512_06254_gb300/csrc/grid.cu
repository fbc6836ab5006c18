// S2-S3: coordinates and convolutional gridding (Section 3.2; Section 4.1
// stage 3 "place visibilities on a grid").
//
// Layout.  Only Re of the inverse transform is kept (the dirty image is
// real), so the grid is stored as its Hermitian half-plane
//     H[k] = G[k] + conj(G[-k]),   rows k2' = k2 - G/2 in [0, G/2),
// i.e. every sample contributes c_q at +k_q and conj(c_q) at -k_q, each
// clipped to the upper half-plane.  A baseline's samples lie on a radial
// track g(k) = G/2 + a k (k = nu / c), so each baseline gives two tracks: the
// one in the upper half-plane and its mirror, which only reaches the stored
// rows near k2' = 0.
//
// Work distribution.  The stored grid is cut into kTile x kTile tiles owned
// by one CTA each.  A binning pass lists, for every tile, the (track,
// 32-channel chunk) pairs whose kernel footprints touch it; the tile's CTA
// accumulates those samples in shared memory and writes the tile once (no
// global atomics, every cell written exactly once, empty tiles as zeros).
#include <cuda_fp16.h>
#include <math.h>

#include "toi_internal.cuh"

namespace toi {
namespace {

constexpr int kGridThreads = 256;
constexpr int kW = 8;   // kernel support compiled in (validated in toi_plan)

struct TrackGeom {
  double s1, s2;   // signed coefficients: g1 = G/2 + s1 k, y = s2 k (row coordinate)
  bool conj;
};

__device__ __forceinline__ TrackGeom track_geom(const BaselineCoef& cf, int mirror) {
  const bool orig_upper = (cf.a2 > 0.0) || (cf.a2 == 0.0 && cf.a1 >= 0.0);
  const bool use_orig = (mirror == 0) == orig_upper;
  TrackGeom t;
  t.s1 = use_orig ? cf.a1 : -cf.a1;
  t.s2 = use_orig ? cf.a2 : -cf.a2;
  t.conj = !use_orig;
  return t;
}

// Tile rectangle touched by the footprints of one chunk of a track (false
// when none of the stored grid is touched).  Coordinates are clamped in
// float64 before any integer conversion, so footprints far outside the grid
// (an oversized cell, reported through the status word) stay harmless.
__device__ __forceinline__ bool chunk_tiles(const TrackGeom& t, double kA, double kB, int G,
                                            int W, int ntx, int nty, int& tx0, int& tx1,
                                            int& ty0, int& ty1) {
  const double kmin = fmin(kA, kB), kmax = fmax(kA, kB);
  const double g1a = 0.5 * G + t.s1 * kmin, g1b = 0.5 * G + t.s1 * kmax;
  const double ya = t.s2 * kmin, yb = t.s2 * kmax;
  const double hw = 0.5 * W;
  const double x0 = ceil(fmin(g1a, g1b) - hw);
  const double x1 = ceil(fmax(g1a, g1b) - hw) + (W - 1);
  const double y0 = ceil(fmin(ya, yb) - hw);
  const double y1 = ceil(fmax(ya, yb) - hw) + (W - 1);
  if (!(x1 >= 0.0 && x0 <= G - 1.0 && y1 >= 0.0 && y0 <= 0.5 * G - 1.0)) return false;
  tx0 = (int)fmax(x0, 0.0) / kTile;
  tx1 = (int)fmin(x1, G - 1.0) / kTile;
  ty0 = (int)fmax(y0, 0.0) / kTile;
  ty1 = (int)fmin(y1, 0.5 * G - 1.0) / kTile;
  return tx0 <= tx1 && ty0 <= ty1 && tx1 < ntx && ty1 < nty;
}

__global__ void bin_count_kernel(const BaselineCoef* __restrict__ coef,
                                 const double* __restrict__ kch, int nbl, int nch, int G, int W,
                                 int ntx, int nty, int* __restrict__ tile_count) {
  const int nchunk = (nch + kChunk - 1) / kChunk;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)2 * nbl * nchunk) return;
  const int track = (int)(id / nchunk), chunk = (int)(id % nchunk);
  const TrackGeom t = track_geom(coef[track >> 1], track & 1);
  const int c0 = chunk * kChunk, c1 = min(nch, c0 + kChunk) - 1;
  int tx0, tx1, ty0, ty1;
  if (!chunk_tiles(t, kch[c0], kch[c1], G, W, ntx, nty, tx0, tx1, ty0, ty1)) return;
  for (int ty = ty0; ty <= ty1; ++ty)
    for (int tx = tx0; tx <= tx1; ++tx) atomicAdd(&tile_count[ty * ntx + tx], 1);
}

// Exclusive scan of the tile counts (one block), capacity check.
__global__ void bin_scan_kernel(const int* __restrict__ count, int n, int* __restrict__ offset,
                                int* __restrict__ cursor, int capacity, int* status) {
  __shared__ int part[1024];
  const int per = (n + 1023) / 1024;
  const int lo = threadIdx.x * per, hi = min(n, lo + per);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += count[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int d = 1; d < 1024; d <<= 1) {
    const int v = (int)threadIdx.x >= d ? part[threadIdx.x - d] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - s;
  for (int i = lo; i < hi; ++i) {
    offset[i] = run;
    cursor[i] = 0;
    run += count[i];
  }
  if (threadIdx.x == 1023) {
    offset[n] = part[1023];
    if (part[1023] > capacity) set_status(status, TOI_DEV_RANGE);
  }
}

__global__ void bin_fill_kernel(const BaselineCoef* __restrict__ coef,
                                const double* __restrict__ kch, int nbl, int nch, int G, int W,
                                int ntx, int nty, const int* __restrict__ offset,
                                int* __restrict__ cursor, GridItem* __restrict__ items,
                                int capacity) {
  const int nchunk = (nch + kChunk - 1) / kChunk;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)2 * nbl * nchunk) return;
  const int track = (int)(id / nchunk), chunk = (int)(id % nchunk);
  const TrackGeom t = track_geom(coef[track >> 1], track & 1);
  const int c0 = chunk * kChunk, c1 = min(nch, c0 + kChunk) - 1;
  int tx0, tx1, ty0, ty1;
  if (!chunk_tiles(t, kch[c0], kch[c1], G, W, ntx, nty, tx0, tx1, ty0, ty1)) return;
  for (int ty = ty0; ty <= ty1; ++ty)
    for (int tx = tx0; tx <= tx1; ++tx) {
      const int tile = ty * ntx + tx;
      const int pos = offset[tile] + atomicAdd(&cursor[tile], 1);
      if (pos < capacity) items[pos] = GridItem{track, chunk};
    }
}

// Exponential of semicircle, psi(x) = exp(beta (sqrt(1 - (2x/W)^2) - 1)),
// written as exp(-beta z^2 / (1 + sqrt(1 - z^2))) to avoid cancellation.
__device__ __forceinline__ float es_kernel(float x, float inv_half_w, float beta) {
  const float z = x * inv_half_w;
  const float z2 = fminf(z * z, 1.0f);
  const float s = sqrtf(1.0f - z2);
  return expf(-beta * z2 / (1.0f + s));
}

__device__ __forceinline__ void parallel_hands(int npol, int& pa, int& pb) {
  if (npol == 4) { pa = 0; pb = 3; }
  else if (npol == 2) { pa = 0; pb = 1; }
  else { pa = 0; pb = 0; }
}

template <bool HALF>
__device__ __forceinline__ float2 load_vis(const void* vis, size_t idx, float scale) {
  if (HALF) {
    const float2 f = __half22float2(reinterpret_cast<const __half2*>(vis)[idx]);
    return make_float2(f.x * scale, f.y * scale);
  } else {
    return reinterpret_cast<const float2*>(vis)[idx];
  }
}

template <bool HALF>
__global__ void __launch_bounds__(kGridThreads)
grid_tiles_kernel(const BaselineCoef* __restrict__ coef, const double* __restrict__ kch,
                  const void* __restrict__ vis, const float* __restrict__ chan_scale,
                  const float* __restrict__ weight, const uint8_t* __restrict__ flag, int nch,
                  int npol, int G, float beta_es, const int* __restrict__ offset,
                  const GridItem* __restrict__ items, int capacity, int ntx,
                  float2* __restrict__ H) {
  __shared__ float2 acc[kTile * kTile];
  const int tile = blockIdx.x;
  const int tx = tile % ntx, ty = tile / ntx;
  const int x0 = tx * kTile, y0 = ty * kTile;
  for (int i = threadIdx.x; i < kTile * kTile; i += kGridThreads) acc[i] = make_float2(0.f, 0.f);
  __syncthreads();
  const int lo = offset[tile];
  const int hi = min(offset[tile + 1], capacity);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int pa, pb;
  parallel_hands(npol, pa, pb);
  const float inv_hw = 2.0f / kW;
  for (int it = lo + warp; it < hi; it += kGridThreads / 32) {
    const GridItem item = items[it];
    const int ch = item.chunk * kChunk + lane;
    if (ch >= nch) continue;
    const int bl = item.track >> 1;
    const size_t o = ((size_t)bl * nch + ch) * npol;
    const bool fa = flag ? flag[o + pa] != 0 : false;
    const bool fb = flag ? flag[o + pb] != 0 : false;
    float wa = fa ? 0.f : (weight ? weight[o + pa] : 1.f);
    float wb = fb ? 0.f : (weight ? weight[o + pb] : 1.f);
    if (pa == pb) wb = 0.f;
    if (!(wa + wb > 0.f)) continue;
    const float sc = HALF ? chan_scale[ch] : 1.f;
    const float2 va = load_vis<HALF>(vis, o + pa, sc);
    float2 c = make_float2(wa * va.x, wa * va.y);
    if (pa != pb) {
      const float2 vb = load_vis<HALF>(vis, o + pb, sc);
      c.x += wb * vb.x;
      c.y += wb * vb.y;
    }
    const TrackGeom t = track_geom(coef[bl], item.track & 1);
    if (t.conj) c.y = -c.y;
    const double k = kch[ch];
    const double g1 = 0.5 * G + t.s1 * k;
    const double y = t.s2 * k;
    const double kx0d = ceil(g1 - 0.5 * kW), ky0d = ceil(y - 0.5 * kW);
    // a footprint entirely outside this tile contributes nothing (this also
    // keeps the integer conversion below in range for far-away samples)
    if (kx0d + (kW - 1) < x0 || kx0d > x0 + (kTile - 1) || ky0d + (kW - 1) < y0 ||
        ky0d > y0 + (kTile - 1))
      continue;
    const float fx = (float)(kx0d - g1), fy = (float)(ky0d - y);
    const int kx0 = (int)kx0d - x0, ky0 = (int)ky0d - y0;
    float px[kW], py[kW];
#pragma unroll
    for (int i = 0; i < kW; ++i) {
      px[i] = es_kernel(fx + (float)i, inv_hw, beta_es);
      py[i] = es_kernel(fy + (float)i, inv_hw, beta_es);
    }
#pragma unroll
    for (int j = 0; j < kW; ++j) {
      const int r = ky0 + j;
      if (r < 0 || r >= kTile) continue;
      const float2 cy = make_float2(c.x * py[j], c.y * py[j]);
#pragma unroll
      for (int i = 0; i < kW; ++i) {
        const int col = kx0 + i;
        if (col < 0 || col >= kTile) continue;
        float2* cell = &acc[r * kTile + col];
        atomicAdd(&cell->x, cy.x * px[i]);
        atomicAdd(&cell->y, cy.y * px[i]);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kTile * kTile; i += kGridThreads) {
    const int r = i / kTile, col = i % kTile;
    H[(size_t)(y0 + r) * G + x0 + col] = acc[i];
  }
}

}  // namespace

cudaError_t launch_grid(toi_plan_s* p, Slot& s, const double* freq, const void* vis,
                        const float* chan_scale, const float* weight, const uint8_t* flag,
                        int nbl, int nch) {
  (void)freq;
  const int ntx = p->ntiles_x, nty = p->ntiles_y, nt = ntx * nty;
  const int tok = prof_begin(p, PROF_BIN, 3);
  cudaError_t e = cudaMemsetAsync(p->tile_count, 0, sizeof(int) * nt, p->stream);
  if (e != cudaSuccess) return e;
  const int nchunk = (nch + kChunk - 1) / kChunk;
  const long long nwork = (long long)2 * nbl * nchunk;
  const int blocks = (int)((nwork + 255) / 256);
  bin_count_kernel<<<blocks, 256, 0, p->stream>>>(s.coef, p->kch, nbl, nch, p->G, p->W, ntx, nty,
                                                  p->tile_count);
  bin_scan_kernel<<<1, 1024, 0, p->stream>>>(p->tile_count, nt, p->tile_offset, p->tile_cursor,
                                             p->max_items, p->d_status);
  bin_fill_kernel<<<blocks, 256, 0, p->stream>>>(s.coef, p->kch, nbl, nch, p->G, p->W, ntx, nty,
                                                 p->tile_offset, p->tile_cursor, p->items,
                                                 p->max_items);
  prof_end(p, tok);
  const int tok2 = prof_begin(p, PROF_GRID, 1);
  const bool half = p->cfg.vis_dtype == TOI_VIS_C16_CHANSCALE;
  if (half)
    grid_tiles_kernel<true><<<nt, kGridThreads, 0, p->stream>>>(
        s.coef, p->kch, vis, chan_scale, weight, flag, nch, p->cfg.n_pol, p->G,
        (float)p->beta_es, p->tile_offset, p->items, p->max_items, ntx, s.grid);
  else
    grid_tiles_kernel<false><<<nt, kGridThreads, 0, p->stream>>>(
        s.coef, p->kch, vis, chan_scale, weight, flag, nch, p->cfg.n_pol, p->G,
        (float)p->beta_es, p->tile_offset, p->items, p->max_items, ntx, s.grid);
  prof_end(p, tok2);
  return cudaGetLastError();
}

}  // namespace toi
