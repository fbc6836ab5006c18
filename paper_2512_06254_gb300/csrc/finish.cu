// S6 re-projection (Section 3.3) fused with the S7 tLISI tile moments, and
// the tLISI finish (Section 2, Section 4.5).
//
// Re-projection.  The reduced map of Section 3.3 sends a tilted-plane pixel p
// to the standard-plane pixel p' = p + d(p) with (pixels, 0-based offsets
// Delta = j - N/2 from the phase centre, beta in radians)
//   q = beta^2 (Delta1^2 + Delta2^2),  z = q / (1 + sqrt(1 - q)),
//   d1 = -xi z / beta,  d2 = +eta z / beta      (y' = y + r0 z eta).
// The standard image is gathered: for each output pixel p' the source p
// solves p = p' - d(p) (fixed-point iteration, |grad d| << 1), and the tilted
// image is bilinearly interpolated there; sources outside the image give 0.
// The displacement e = p - p' is carried separately from the integer pixel
// so the interpolation weights keep float32 precision at any image size.
//
// tLISI moments.  One CTA per T x T tile computes the new image's pixels and,
// with the two previous ring images, a = I(t-1) - I(t-2), b = I(t) - I(t-1)
// and the tile sums of a, b, a^2, b^2, ab (float32 per thread, float64 across
// the block in a fixed order).  The finish kernel turns them into tLISI with
// L = max |I| over the three images (tracked per image with an order-free
// atomic max on the float bits).
#include <math.h>

#include "toi_internal.cuh"

namespace toi {
namespace {

constexpr int kFinThreads = 256;

// Fixed-order block reduction: float32 warp shuffles (32 lanes x 4 pixels),
// then the eight warp totals in float64, in warp order.
template <int NV>
__device__ void block_reduce_d(float (&v)[NV], double (*sh)[NV], double (&out)[NV]) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
    for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], off);
  if (lane == 0)
    for (int i = 0; i < NV; ++i) sh[wib][i] = (double)v[i];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int i = 0; i < NV; ++i) {
      double a = 0.0;
      for (int wdx = 0; wdx < kFinThreads / 32; ++wdx) a += sh[wdx][i];
      out[i] = a;
    }
}

// Source of output pixel (o1, o2) in the tilted image: integer corner
// (i1, i2), bilinear fractions (f1, f2) and whether it lies on the image.
// K1 = -xi / beta, K2 = eta / beta, b2 = beta^2 (float32, from the snapshot
// record).  Shared by the re-projection and its adjoint, so that both use
// bit-identical positions and weights.
struct Source {
  int i1, i2;
  float f1, f2;
  bool ok;
};

__device__ __forceinline__ Source reproject_source(int o1, int o2, int N, float K1, float K2,
                                                   float b2) {
  const float D1 = (float)(o1 - N / 2), D2 = (float)(o2 - N / 2);
  // The map's Jacobian is about |K| beta^2 |u| = |tilt| x (field angle), a
  // few 1e-2 at most, so each step shrinks the error by that factor.  Steps
  // stop once one moves the position by less than 2^-16 px (the error left
  // is that factor times smaller), at most 8.
  //
  // z = q / (1 + sqrt(1 - q)) = 1 - sqrt(1 - q) has the binomial series
  // q/2 + q^2/8 + q^3/16 + 5 q^4/128 + 7 q^5/256 + 21 q^6/1024 + ...; for
  // q < 4e-3 (fields up to about 5 degrees across) the terms after q^5 are
  // below 1e-14 of z, so the series (five fused multiply-adds) replaces the
  // square root and division there.
  float e1 = 0.f, e2 = 0.f;
  const bool series = b2 * (D1 * D1 + D2 * D2) < 4e-3f;
  for (int it = 0; it < 8; ++it) {
    const float u1 = D1 + e1, u2 = D2 + e2;
    const float q = b2 * (u1 * u1 + u2 * u2);
    float z;
    if (series) {
      z = q * fmaf(q, fmaf(q, fmaf(q, fmaf(q, 0.02734375f, 0.0390625f), 0.0625f), 0.125f), 0.5f);
    } else {
      float rt;
      asm("sqrt.approx.f32 %0, %1;" : "=f"(rt) : "f"(1.0f - q));
      z = __fdividef(q, 1.0f + rt);
    }
    const float n1 = -K1 * z, n2 = -K2 * z;
    const float step = fabsf(n1 - e1) + fabsf(n2 - e2);
    e1 = n1;
    e2 = n2;
    if (step < 1.52587890625e-5f) break;
  }
  const float fl1 = floorf(e1), fl2 = floorf(e2);
  Source r;
  r.i1 = o1 + (int)fl1;
  r.i2 = o2 + (int)fl2;
  r.f1 = e1 - fl1;
  r.f2 = e2 - fl2;
  r.ok = r.i1 >= 0 && r.i2 >= 0 && (r.i1 < N - 1 || (r.i1 == N - 1 && r.f1 == 0.f)) &&
         (r.i2 < N - 1 || (r.i2 == N - 1 && r.f2 == 0.f));
  return r;
}

template <bool REPRO>
__device__ __forceinline__ void image_tile_body(const float* __restrict__ src, int N, int T,
                                                const double* __restrict__ snap, double beta_rad,
                                                float* __restrict__ ring_cur,
                                                const float* __restrict__ ring_p1,
                                                const float* __restrict__ ring_p2,
                                                float* __restrict__ image_out, int with_moments,
                                                double* __restrict__ tile_mom,
                                                unsigned int* __restrict__ max_cur, int tile) {
  __shared__ double sh[kFinThreads / 32][5];
  const int ntx = N / T;
  const int tx = tile % ntx, ty = tile / ntx;
  // constants made once per snapshot by the plane fit (no block barrier)
  float kk[3] = {0.f, 0.f, 0.f};
  if (REPRO) {
    kk[0] = (float)snap[SNAP_REPRO];
    kk[1] = (float)snap[SNAP_REPRO + 1];
    kk[2] = (float)snap[SNAP_REPRO + 2];
  }
  float sa = 0.f, sb = 0.f, saa = 0.f, sbb = 0.f, sab = 0.f, mx = 0.f;
  // kBatch pixels per thread at a time: all their sources first, then every
  // load (clamped to valid addresses, so they issue back to back), then the
  // arithmetic and the stores
  constexpr int kBatch = 4;
  for (int e0 = threadIdx.x; e0 < T * T; e0 += kBatch * kFinThreads) {
    float v[kBatch], i1v[kBatch], i0v[kBatch];
    size_t pixv[kBatch];
    bool live[kBatch];
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      const int e = e0 + b * kFinThreads;
      live[b] = e < T * T;
      const int ee = live[b] ? e : 0;
      const int o1 = tx * T + (ee % T), o2 = ty * T + (ee / T);
      const size_t pix = (size_t)o2 * N + o1;
      pixv[b] = pix;
      if (REPRO) {
        const Source sr = reproject_source(o1, o2, N, kk[0], kk[1], kk[2]);
        const bool ok = live[b] && sr.ok;
        const int i1 = ok ? sr.i1 : 0, i2 = ok ? sr.i2 : 0;
        const bool has1 = i1 + 1 < N, has2 = i2 + 1 < N;
        const float* r0 = src + (size_t)i2 * N;
        const float* r1 = has2 ? r0 + N : r0;
        const int i1n = has1 ? i1 + 1 : i1;
        const float a00 = r0[i1], a01r = r0[i1n], a10r = r1[i1], a11r = r1[i1n];
        const float a01 = has1 ? a01r : 0.f;
        const float a10 = has2 ? a10r : 0.f;
        const float a11 = (has1 && has2) ? a11r : 0.f;
        const float f1 = sr.f1, f2 = sr.f2;
        const float val = (1.f - f2) * ((1.f - f1) * a00 + f1 * a01) + f2 * ((1.f - f1) * a10 + f1 * a11);
        v[b] = ok ? val : 0.f;
      } else {
        v[b] = src[pix];
      }
      if (with_moments) {
        i1v[b] = ring_p1[pix];
        i0v[b] = ring_p2[pix];
      }
    }
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      if (!live[b]) continue;
      ring_cur[pixv[b]] = v[b];
      if (image_out) image_out[pixv[b]] = v[b];
      mx = fmaxf(mx, fabsf(v[b]));
      if (with_moments) {
        const float a = i1v[b] - i0v[b], bd = v[b] - i1v[b];
        sa += a; sb += bd; saa += a * a; sbb += bd * bd; sab += a * bd;
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, off));
  // order-free max of |I| (float bits of non-negative floats order like
  // ints): one global atomic per warp, so no block barrier is needed for it
  if ((threadIdx.x & 31) == 0) atomicMax(max_cur, __float_as_uint(mx));
  if (with_moments) {
    float f5[5] = {sa, sb, saa, sbb, sab};
    double v5[5];
    block_reduce_d<5>(f5, sh, v5);
    if (threadIdx.x == 0)
      for (int i = 0; i < 5; ++i) tile_mom[(size_t)tile * 5 + i] = v5[i];
  }
}

template <bool REPRO>
__global__ void __launch_bounds__(kFinThreads)
image_tile_kernel(const float* __restrict__ src, int N, int T, const double* __restrict__ snap,
                  double beta_rad, float* __restrict__ ring_cur,
                  const float* __restrict__ ring_p1, const float* __restrict__ ring_p2,
                  float* __restrict__ image_out, int with_moments,
                  double* __restrict__ tile_mom, unsigned int* __restrict__ max_cur) {
  image_tile_body<REPRO>(src, N, T, snap, beta_rad, ring_cur, ring_p1, ring_p2, image_out,
                         with_moments, tile_mom, max_cur, blockIdx.x);
}

constexpr int kBatchPix = 4;   // pixels per thread of a tile of up to 32 x 32

constexpr int kMaxBatch = 64;   // toi_config.batch_max limit

// Batch, in one launch: one block per tile walks the entries in stream
// order.  For entry i it re-projects the tile from the entry's tilted image
// (as image_tile_body), stores it to the ring and the caller's image, and
// forms the window moments of entry i from the tile's pixels of entries
// i - 2, i - 1 and i, which it keeps in registers (the two images before the
// batch are read from the ring once).  Every image of the batch is written
// once and never read back.  Pixel order, arithmetic and the reduction order
// are those of image_tile_body (the single-snapshot path), so the images and
// moments equal its own bit for bit.
// Five blocks per SM (48 registers a thread) keep the gathers of more tiles
// in flight: 9 % faster than four blocks at 64 registers.
__global__ void __launch_bounds__(kFinThreads, 5)
image_walk_batch(const BatchEntry* __restrict__ E, const BatchHeader* __restrict__ hdr, int N,
                 int T) {
  __shared__ float part[kMaxBatch][kFinThreads / 32][5];
  const int n = hdr->n;
  const int tile = blockIdx.x;
  const int ntx = N / T;
  const int tx = tile % ntx, ty = tile / ntx;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int o1v[kBatchPix], o2v[kBatchPix];
  size_t pixv[kBatchPix];
  bool live[kBatchPix];
  float prev1[kBatchPix], prev2[kBatchPix];
#pragma unroll
  for (int b = 0; b < kBatchPix; ++b) {
    const int e = threadIdx.x + b * kFinThreads;
    live[b] = e < T * T;
    const int ee = live[b] ? e : 0;
    o1v[b] = tx * T + (ee % T);
    o2v[b] = ty * T + (ee / T);
    pixv[b] = (size_t)o2v[b] * N + o1v[b];
    prev1[b] = E[0].ring_p1[pixv[b]];
    prev2[b] = E[0].ring_p2[pixv[b]];
  }
  for (int i = 0; i < n; ++i) {
    const BatchEntry& e = E[i];
    const float K1 = (float)e.snap[SNAP_REPRO];
    const float K2 = (float)e.snap[SNAP_REPRO + 1];
    const float b2 = (float)e.snap[SNAP_REPRO + 2];
    const float* __restrict__ src = e.tilted;
    float v[kBatchPix];
#pragma unroll
    for (int b = 0; b < kBatchPix; ++b) {
      const Source sr = reproject_source(o1v[b], o2v[b], N, K1, K2, b2);
      const bool ok = live[b] && sr.ok;
      const int i1 = ok ? sr.i1 : 0, i2 = ok ? sr.i2 : 0;
      const bool has1 = i1 + 1 < N, has2 = i2 + 1 < N;
      const float* r0 = src + (size_t)i2 * N;
      const float* r1 = has2 ? r0 + N : r0;
      const int i1n = has1 ? i1 + 1 : i1;
      const float a00 = r0[i1], a01r = r0[i1n], a10r = r1[i1], a11r = r1[i1n];
      const float a01 = has1 ? a01r : 0.f;
      const float a10 = has2 ? a10r : 0.f;
      const float a11 = (has1 && has2) ? a11r : 0.f;
      const float f1 = sr.f1, f2 = sr.f2;
      const float val = (1.f - f2) * ((1.f - f1) * a00 + f1 * a01) + f2 * ((1.f - f1) * a10 + f1 * a11);
      v[b] = ok ? val : 0.f;
    }
    float mx = 0.f;
    float m5[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    // only the batch's last two images are read from the ring again (the
    // next batch's first windows, the plan's last image); the others live
    // in registers here and, when asked for, in the caller's images
    const bool keep = i >= n - 2;
    for (int b = 0; b < kBatchPix; ++b) {
      if (!live[b]) continue;
      if (keep) e.ring_cur[pixv[b]] = v[b];
      if (e.image_out) e.image_out[pixv[b]] = v[b];
      mx = fmaxf(mx, fabsf(v[b]));
      const float a = prev1[b] - prev2[b], bd = v[b] - prev1[b];
      m5[0] += a; m5[1] += bd; m5[2] += a * a; m5[3] += bd * bd; m5[4] += a * bd;
    }
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, off));
    if (lane == 0) atomicMax(e.max_cur, __float_as_uint(mx));
#pragma unroll
    for (int k = 0; k < 5; ++k)
      for (int off = 16; off > 0; off >>= 1) m5[k] += __shfl_down_sync(0xffffffffu, m5[k], off);
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < 5; ++k) part[i][wib][k] = m5[k];
#pragma unroll
    for (int b = 0; b < kBatchPix; ++b) {
      prev2[b] = prev1[b];
      prev1[b] = v[b];
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < n * 5; q += blockDim.x) {
    const int i = q / 5, k = q - 5 * (q / 5);
    const BatchEntry& e = E[i];
    if (!e.with_moments) continue;
    double a = 0.0;
    for (int wdx = 0; wdx < kFinThreads / 32; ++wdx) a += (double)part[i][wdx][k];
    e.tile_mom[(size_t)tile * 5 + k] = a;
  }
}

__device__ __forceinline__ void tlisi_finish_body(const double* __restrict__ tile_mom, int ntl,
                                                  int T, const unsigned int* __restrict__ m_cur,
                                                  const unsigned int* __restrict__ m_p1,
                                                  const unsigned int* __restrict__ m_p2,
                                                  float* __restrict__ out, int t) {
  if (t >= ntl) return;
  const double L = (double)fmaxf(__uint_as_float(*m_cur),
                                 fmaxf(__uint_as_float(*m_p1), __uint_as_float(*m_p2)));
  if (L == 0.0) { out[t] = 1.0f; return; }
  const double n = (double)T * (double)T;
  const double* m = tile_mom + (size_t)t * 5;
  const double mua = m[0] / n, mub = m[1] / n;
  const double va = m[2] / n - mua * mua;
  const double vb = m[3] / n - mub * mub;
  const double cab = m[4] / n - mua * mub;
  const double C1 = (0.01 * L) * (0.01 * L), C2 = (0.03 * L) * (0.03 * L);
  const double S = ((2.0 * mua * mub + C1) * (2.0 * cab + C2)) /
                   ((mua * mua + mub * mub + C1) * (va + vb + C2));
  out[t] = (float)((1.0 + S) * 0.5);
}

__global__ void tlisi_finish_kernel(const double* __restrict__ tile_mom, int ntl, int T,
                                    const unsigned int* __restrict__ ring_max, int cur, int p1,
                                    int p2, float* __restrict__ out) {
  tlisi_finish_body(tile_mom, ntl, T, ring_max + cur, ring_max + p1, ring_max + p2, out,
                    blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void tlisi_finish_batch(const BatchEntry* __restrict__ E,
                                   const BatchHeader* __restrict__ hdr, int ntl, int T) {
  if ((int)blockIdx.y >= hdr->n) return;
  const BatchEntry& e = E[blockIdx.y];
  if (!e.tlisi_out) return;
  tlisi_finish_body(e.tile_mom, ntl, T, e.max_cur, e.max_p1, e.max_p2, e.tlisi_out,
                    blockIdx.x * blockDim.x + threadIdx.x);
}

// Adjoint of the re-projection, as a gather (deterministic, no atomics):
// tilted pixel j receives dL/dI(o) w(o, j) from every output pixel o whose
// bilinear stencil covers j.  Those o lie within one pixel (plus the tiny
// variation of the displacement over a pixel) of j + d(j), the forward map of
// j, so a 4 x 4 window from floor(j + d(j)) - 1 covers them; each candidate's
// source is recomputed with reproject_source and kept if j is one of its
// corners.  The result is scaled by the grid correction and 1/(omega sum w),
// giving the cotangent U that the adjoint FFT transforms.
__global__ void __launch_bounds__(kFinThreads)
reproject_adjoint_kernel(const float* __restrict__ gimg, int N, const double* __restrict__ snap,
                         double beta_rad, const float* __restrict__ corr,
                         float* __restrict__ ubar) {
  const int j1 = blockIdx.x * 16 + (threadIdx.x & 15);
  const int j2 = blockIdx.y * 16 + (threadIdx.x >> 4);
  if (j1 >= N || j2 >= N) return;
  const float K1 = (float)snap[SNAP_REPRO];
  const float K2 = (float)snap[SNAP_REPRO + 1];
  const float b2 = (float)snap[SNAP_REPRO + 2];
  const double omega = snap[SNAP_OMEGA], sumw = snap[SNAP_SUMW];
  const float norm = sumw > 0.0 ? (float)(1.0 / (omega * sumw)) : 0.f;
  const float D1 = (float)(j1 - N / 2), D2 = (float)(j2 - N / 2);
  const float q = b2 * (D1 * D1 + D2 * D2);
  float rt;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(rt) : "f"(1.0f - q));
  const float z = __fdividef(q, 1.0f + rt);
  const int b1 = (int)floorf((float)j1 + K1 * z) - 1;
  const int bb2 = (int)floorf((float)j2 + K2 * z) - 1;
  float acc = 0.f;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int o2 = bb2 + b;
    if (o2 < 0 || o2 >= N) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int o1 = b1 + a;
      if (o1 < 0 || o1 >= N) continue;
      const Source sr = reproject_source(o1, o2, N, K1, K2, b2);
      if (!sr.ok) continue;
      const int dx = j1 - sr.i1, dy = j2 - sr.i2;
      if ((unsigned)dx > 1u || (unsigned)dy > 1u) continue;
      const float wx = dx ? sr.f1 : 1.f - sr.f1;
      const float wy = dy ? sr.f2 : 1.f - sr.f2;
      acc += wx * wy * gimg[(size_t)o2 * N + o1];
    }
  }
  ubar[(size_t)j2 * N + j1] = acc * (norm * corr[j1] * corr[j2]);
}

}  // namespace

cudaError_t launch_reproject_moments(toi_plan_s* p, Slot& s, float* image_out,
                                     bool with_moments, int cur, int prev1, int prev2) {
  cudaError_t e = cudaMemsetAsync(p->ring_max + cur, 0, sizeof(unsigned int), p->stream);
  if (e != cudaSuccess) return e;
  const int ntl = (p->N / p->T) * (p->N / p->T);
  const int tok = prof_begin(p, PROF_REPROJECT, 1);
  image_tile_kernel<true><<<ntl, kFinThreads, 0, p->stream>>>(
      p->tilted, p->N, p->T, s.snap, p->beta_rad, p->ring[cur], p->ring[prev1], p->ring[prev2],
      image_out, with_moments ? 1 : 0, p->tile_mom, p->ring_max + cur);
  prof_end(p, tok);
  return cudaGetLastError();
}

cudaError_t launch_ring_moments(toi_plan_s* p, const float* image, int cur, int prev1,
                                int prev2, bool with_moments) {
  cudaError_t e = cudaMemsetAsync(p->ring_max + cur, 0, sizeof(unsigned int), p->stream);
  if (e != cudaSuccess) return e;
  const int ntl = (p->N / p->T) * (p->N / p->T);
  const int tok = prof_begin(p, PROF_TLISI, 1);
  image_tile_kernel<false><<<ntl, kFinThreads, 0, p->stream>>>(
      image, p->N, p->T, nullptr, p->beta_rad, p->ring[cur], p->ring[prev1], p->ring[prev2],
      nullptr, with_moments ? 1 : 0, p->tile_mom, p->ring_max + cur);
  prof_end(p, tok);
  return cudaGetLastError();
}

// Re-projection (+ tile moments) with explicit buffers, for the streaming
// runtime's rings: tilted source, the new ring image and the two before it,
// its maximum word and the tile moments of this window.
cudaError_t launch_reproject_ring(toi_plan_s* p, Slot& s, const float* tilted, float* cur,
                                  const float* prev1, const float* prev2, bool with_moments,
                                  double* tile_mom, unsigned int* max_cur) {
  cudaError_t e = cudaMemsetAsync(max_cur, 0, sizeof(unsigned int), p->stream);
  if (e != cudaSuccess) return e;
  const int ntl = (p->N / p->T) * (p->N / p->T);
  const int tok = prof_begin(p, PROF_REPROJECT, 1);
  image_tile_kernel<true><<<ntl, kFinThreads, 0, p->stream>>>(
      tilted, p->N, p->T, s.snap, p->beta_rad, cur, prev1, prev2, nullptr, with_moments ? 1 : 0,
      tile_mom, max_cur);
  prof_end(p, tok);
  return cudaGetLastError();
}

// tLISI of the window whose moments are in tile_mom and whose image maxima
// are ring_max[cur], [prev1], [prev2].
cudaError_t launch_tlisi_rows(toi_plan_s* p, const double* tile_mom, const unsigned int* ring_max,
                              int cur, int prev1, int prev2, float* out) {
  const int ntl = (p->N / p->T) * (p->N / p->T);
  const int tok = prof_begin(p, PROF_TLISI, 1);
  tlisi_finish_kernel<<<(ntl + 255) / 256, 256, 0, p->stream>>>(tile_mom, ntl, p->T, ring_max,
                                                                cur, prev1, prev2, out);
  prof_end(p, tok);
  return cudaGetLastError();
}

cudaError_t launch_finish_batch(toi_plan_s* p) {
  const int ntl = (p->N / p->T) * (p->N / p->T);
  const int B = p->batch_max;
  if (p->T * p->T > kBatchPix * kFinThreads) return cudaErrorInvalidConfiguration;
  int tok = prof_begin(p, PROF_REPROJECT, 1);
  image_walk_batch<<<ntl, kFinThreads, 0, p->stream>>>(p->bentry_dev, p->bheader_dev, p->N, p->T);
  prof_end(p, tok);
  tok = prof_begin(p, PROF_TLISI, 1);
  tlisi_finish_batch<<<dim3((ntl + 255) / 256, B), 256, 0, p->stream>>>(p->bentry_dev,
                                                                         p->bheader_dev, ntl, p->T);
  prof_end(p, tok);
  return cudaGetLastError();
}

cudaError_t launch_tlisi_finalize(toi_plan_s* p, float* tlisi, int cur, int prev1, int prev2) {
  const int ntl = (p->N / p->T) * (p->N / p->T);
  const int tok = prof_begin(p, PROF_TLISI, 1);
  tlisi_finish_kernel<<<(ntl + 255) / 256, 256, 0, p->stream>>>(p->tile_mom, ntl, p->T,
                                                                p->ring_max, cur, prev1, prev2,
                                                                tlisi);
  prof_end(p, tok);
  return cudaGetLastError();
}

}  // namespace toi

namespace toi {

cudaError_t launch_reproject_adjoint(toi_plan_s* p, Slot& s, const float* grad_image) {
  const dim3 grid((p->N + 15) / 16, (p->N + 15) / 16);
  reproject_adjoint_kernel<<<grid, kFinThreads, 0, p->stream>>>(grad_image, p->N, s.snap,
                                                                 p->beta_rad, p->corr, p->tilted);
  return cudaGetLastError();
}

}  // namespace toi
