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

template <bool REPRO>
__global__ void __launch_bounds__(kFinThreads)
image_tile_kernel(const float* __restrict__ src, int N, int T, const double* __restrict__ snap,
                  double beta_rad, float* __restrict__ ring_cur,
                  const float* __restrict__ ring_p1, const float* __restrict__ ring_p2,
                  float* __restrict__ image_out, int with_moments,
                  double* __restrict__ tile_mom, unsigned int* __restrict__ max_cur) {
  __shared__ double sh[kFinThreads / 32][5];
  __shared__ float kk[3];
  __shared__ unsigned int smax;
  const int ntx = N / T;
  const int tx = blockIdx.x % ntx, ty = blockIdx.x / ntx;
  if (threadIdx.x == 0) {
    smax = 0u;
    if (REPRO) {
      kk[0] = (float)(-snap[SNAP_XI] / beta_rad);
      kk[1] = (float)(snap[SNAP_ETA] / beta_rad);
      kk[2] = (float)(beta_rad * beta_rad);
    }
  }
  __syncthreads();
  float sa = 0.f, sb = 0.f, saa = 0.f, sbb = 0.f, sab = 0.f, mx = 0.f;
  for (int e = threadIdx.x; e < T * T; e += kFinThreads) {
    const int o1 = tx * T + (e % T), o2 = ty * T + (e / T);
    const size_t pix = (size_t)o2 * N + o1;
    float v;
    if (REPRO) {
      const float K1 = kk[0], K2 = kk[1], b2 = kk[2];
      const float D1 = (float)(o1 - N / 2), D2 = (float)(o2 - N / 2);
      float e1 = 0.f, e2 = 0.f;
#pragma unroll
      for (int it = 0; it < 3; ++it) {
        const float u1 = D1 + e1, u2 = D2 + e2;
        const float q = b2 * (u1 * u1 + u2 * u2);
        float rt;
        asm("sqrt.approx.f32 %0, %1;" : "=f"(rt) : "f"(1.0f - q));
        const float z = __fdividef(q, 1.0f + rt);
        e1 = -K1 * z;
        e2 = -K2 * z;
      }
      const float fl1 = floorf(e1), fl2 = floorf(e2);
      const int i1 = o1 + (int)fl1, i2 = o2 + (int)fl2;
      const float f1 = e1 - fl1, f2 = e2 - fl2;
      const bool ok = i1 >= 0 && i2 >= 0 && (i1 < N - 1 || (i1 == N - 1 && f1 == 0.f)) &&
                      (i2 < N - 1 || (i2 == N - 1 && f2 == 0.f));
      v = 0.f;
      if (ok) {
        const float* r0 = src + (size_t)i2 * N;
        const float a00 = r0[i1];
        const float a01 = (i1 + 1 < N) ? r0[i1 + 1] : 0.f;
        float a10 = 0.f, a11 = 0.f;
        if (i2 + 1 < N) {
          const float* r1 = r0 + N;
          a10 = r1[i1];
          a11 = (i1 + 1 < N) ? r1[i1 + 1] : 0.f;
        }
        v = (1.f - f2) * ((1.f - f1) * a00 + f1 * a01) + f2 * ((1.f - f1) * a10 + f1 * a11);
      }
    } else {
      v = src[pix];
    }
    ring_cur[pix] = v;
    if (image_out) image_out[pix] = v;
    mx = fmaxf(mx, fabsf(v));
    if (with_moments) {
      const float i1v = ring_p1[pix], i0v = ring_p2[pix];
      const float a = i1v - i0v, b = v - i1v;
      sa += a; sb += b; saa += a * a; sbb += b * b; sab += a * b;
    }
  }
  // order-free max of |I| (float bits of non-negative floats order like ints)
  atomicMax(&smax, __float_as_uint(mx));
  if (with_moments) {
    float f5[5] = {sa, sb, saa, sbb, sab};
    double v5[5];
    block_reduce_d<5>(f5, sh, v5);
    if (threadIdx.x == 0)
      for (int i = 0; i < 5; ++i) tile_mom[(size_t)blockIdx.x * 5 + i] = v5[i];
  } else {
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(max_cur, smax);
}

__global__ void tlisi_finish_kernel(const double* __restrict__ tile_mom, int ntl, int T,
                                    const unsigned int* __restrict__ ring_max, int cur, int p1,
                                    int p2, float* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntl) return;
  const double L = (double)fmaxf(__uint_as_float(ring_max[cur]),
                                 fmaxf(__uint_as_float(ring_max[p1]), __uint_as_float(ring_max[p2])));
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
