// Adjoint of the imaging map: toi_degrid_backward.
//
// Section 1 of the paper notes that the dirty image is the adjoint of the
// measurement operator applied to the visibilities; this file runs the
// reverse mode of the whole snapshot image (gridding, inverse FFT,
// correction, re-projection) for a loss L with a given dL/dI.  For every
// sample q the cotangent of its gridded value c_q = w_a V_a + w_b V_b is
//   g_q = sum_k psi(k1 - g1_q) psi(k2 - g2_q) Hbar[k]      (ES degridding)
// with Hbar the forward DFT of the scaled image cotangent (fft.cu), whose
// rows k2' < 0 are conj(Hbar[-k']).  Complex gradients follow the convention
// dL/dRe z + i dL/dIm z.  From g_q:
//   grad_vis[p]    = w_p g_q for the parallel hands p (0 for cross hands and
//                    unselected samples),
//   grad_weight[p] = Re(conj(g_q) V_p) - <dL/dI, I> / sum w for unflagged
//                    parallel hands of selected samples (c_q is linear in w_p
//                    and the image carries 1 / sum w), else 0.
// The plane fit (V, omega, the selection w_q > 0) is held fixed: it is
// piecewise constant in the weights.
#include <cuda_fp16.h>

#include "toi_internal.cuh"

namespace toi {
cudaError_t launch_reproject_adjoint(toi_plan_s* p, Slot& s, const float* grad_image);
cudaError_t launch_fft_adjoint(toi_plan_s* p, Slot& s);

namespace {

constexpr int kDotBlocks = 304;       // 2 per SM
constexpr int kDotThreads = 256;
constexpr int kDegridThreads = 128;
constexpr int kW = 8;

// <a, b> over n floats in float64: block i takes the contiguous slice
// [i n / B, (i + 1) n / B), threads stride it, then a fixed tree.
__global__ void __launch_bounds__(kDotThreads)
dot_partial_kernel(const float* __restrict__ a, const float* __restrict__ b, long long n,
                   double* __restrict__ part) {
  __shared__ double sh[kDotThreads];
  const long long lo = n * blockIdx.x / gridDim.x, hi = n * (blockIdx.x + 1) / gridDim.x;
  double acc = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += kDotThreads)
    acc += (double)a[i] * (double)b[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kDotThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void dot_final_kernel(const double* __restrict__ part, int nb, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += 32) acc += part[i];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if (threadIdx.x == 0) *out = acc;
}

// psi(x) = exp(beta (sqrt(1 - (2x/W)^2) - 1)) for |x| <= W/2, else 0
__device__ __forceinline__ float es_psi(float x, float beta) {
  const float z = x * (2.0f / kW);
  const float s = 1.0f - z * z;
  return s >= 0.f ? expf(beta * (sqrtf(s) - 1.0f)) : 0.f;
}

__device__ __forceinline__ float2 read_vis(const void* vis, const float* chan_scale, int half,
                                           size_t idx, int ch) {
  if (half) {
    const __half2 h = reinterpret_cast<const __half2*>(vis)[idx];
    const float2 f = __half22float2(h);
    const float sc = chan_scale[ch];
    return make_float2(f.x * sc, f.y * sc);
  }
  return reinterpret_cast<const float2*>(vis)[idx];
}

// One thread per sample; the threads of a block walk consecutive channels of
// one baseline, whose footprints overlap, so the grid reads hit in L1.
__global__ void __launch_bounds__(kDegridThreads)
degrid_backward_kernel(const float2* __restrict__ K, int G, const BaselineCoef* __restrict__ coef,
                       const double* __restrict__ freq, const void* __restrict__ vis,
                       const float* __restrict__ chan_scale, int half,
                       const float* __restrict__ weight, const uint8_t* __restrict__ flag,
                       int nbl, int nch, int npol, const double* __restrict__ snap,
                       const double* __restrict__ dot, float beta_es,
                       float2* __restrict__ grad_sample, float2* __restrict__ grad_vis,
                       float* __restrict__ grad_weight) {
  const int ch = blockIdx.x * kDegridThreads + threadIdx.x;
  const int bl = blockIdx.y;
  if (ch >= nch || bl >= nbl) return;
  int pa, pb;
  parallel_hands(npol, pa, pb);
  const size_t q = (size_t)bl * nch + ch;
  const size_t o = q * npol;
  const bool fa = flag ? flag[o + pa] != 0 : false;
  const bool fb = flag ? flag[o + pb] != 0 : false;
  const float wa = fa ? 0.f : (weight ? weight[o + pa] : 1.f);
  const float wb = fb ? 0.f : (weight ? weight[o + pb] : 1.f);
  const bool sel = ((pa == pb) ? wa : wa + wb) > 0.f;

  float2 g = make_float2(0.f, 0.f);
  if (sel) {
    const BaselineCoef cf = coef[bl];
    const double k = freq[ch] / kCLight;
    const double g1 = 0.5 * G + cf.a1 * k, g2 = 0.5 * G + cf.a2 * k;
    const double s1 = ceil(g1 - 0.5 * kW), s2 = ceil(g2 - 0.5 * kW);
    const int k1 = (int)s1, k2 = (int)s2;
    // rows k2' = k2 + b - G/2; a footprint off the stored rows or columns
    // (only possible when toi_grid reported TOI_ERR_RANGE) is skipped
    const int r0 = k2 - G / 2;
    const bool inside = k1 >= 0 && k1 + kW <= G && r0 > -G / 2 && r0 + kW <= G / 2;
    if (inside) {
      const float d1 = (float)(s1 - g1), d2 = (float)(s2 - g2);
      float wx[kW], wy[kW];
#pragma unroll
      for (int a = 0; a < kW; ++a) {
        wx[a] = es_psi(d1 + (float)a, beta_es);
        wy[a] = es_psi(d2 + (float)a, beta_es);
      }
      float2 up = make_float2(0.f, 0.f), lo = make_float2(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < kW; ++b) {
        const int r = r0 + b;
        float2 acc = make_float2(0.f, 0.f);
        if (r >= 0) {
          const float2* row = K + (size_t)r * G + k1;
#pragma unroll
          for (int a = 0; a < kW; ++a) {
            const float2 v = row[a];
            acc.x += wx[a] * v.x;
            acc.y += wx[a] * v.y;
          }
          up.x += wy[b] * acc.x;
          up.y += wy[b] * acc.y;
        } else {
          // Hbar[k'] = conj(Hbar[-k']) = K[-k2'][G - n]
          const float2* row = K + (size_t)(-r) * G;
#pragma unroll
          for (int a = 0; a < kW; ++a) {
            const int n = k1 + a;
            const float2 v = row[n == 0 ? 0 : G - n];
            acc.x += wx[a] * v.x;
            acc.y += wx[a] * v.y;
          }
          lo.x += wy[b] * acc.x;
          lo.y += wy[b] * acc.y;
        }
      }
      // Hbar = conj(K) on the stored rows
      g = make_float2(up.x + lo.x, lo.y - up.y);
    }
  }
  if (grad_sample) grad_sample[q] = g;
  if (grad_vis) {
    for (int p = 0; p < npol; ++p) {
      float w = 0.f;
      if (sel) w = (p == pa) ? wa : (p == pb ? wb : 0.f);
      grad_vis[o + p] = make_float2(w * g.x, w * g.y);
    }
  }
  if (grad_weight) {
    const double sumw = snap[SNAP_SUMW];
    const float nterm = sumw > 0.0 ? (float)(*dot / sumw) : 0.f;
    for (int p = 0; p < npol; ++p) {
      float gw = 0.f;
      const bool hand = (p == pa) || (p == pb);
      const bool flagged = (p == pa) ? fa : (p == pb ? fb : true);
      if (sel && hand && !flagged) {
        const float2 v = read_vis(vis, chan_scale, half, o + p, ch);
        gw = g.x * v.x + g.y * v.y - nterm;
      }
      grad_weight[o + p] = gw;
    }
  }
}

// Clear the rows the adjoint wrote so that the slot is zero for the next
// gridding.
__global__ void clear_rows_kernel(float2* __restrict__ grid, int G, const double* __restrict__ snap) {
  const int row = blockIdx.x;
  const int r = (int)ceil(snap[SNAP_ROWMAX]);
  const int rmax = r < G / 2 ? r : G / 2 - 1;
  if (row > rmax) return;
  float4* dst = reinterpret_cast<float4*>(grid + (size_t)row * G);
  for (int n = threadIdx.x; n < G / 2; n += blockDim.x) dst[n] = make_float4(0.f, 0.f, 0.f, 0.f);
}

}  // namespace

size_t degrid_scratch_doubles() { return kDotBlocks + 2; }

cudaError_t launch_degrid_backward(toi_plan_s* p, Slot& s, const float* grad_image,
                                   const float* image, float2* grad_sample, float2* grad_vis,
                                   float* grad_weight) {
  const int tok = prof_begin(p, PROF_BACKWARD, grad_weight ? 6 : 4);
  const long long NN = (long long)p->N * p->N;
  double* dot = p->adj_scratch + kDotBlocks;
  if (grad_weight) {
    dot_partial_kernel<<<kDotBlocks, kDotThreads, 0, p->stream>>>(grad_image, image, NN,
                                                                  p->adj_scratch);
    dot_final_kernel<<<1, 32, 0, p->stream>>>(p->adj_scratch, kDotBlocks, dot);
  }
  cudaError_t e = launch_reproject_adjoint(p, s, grad_image);
  if (e == cudaSuccess) e = launch_fft_adjoint(p, s);
  if (e != cudaSuccess) return e;
  const dim3 grid((s.nch + kDegridThreads - 1) / kDegridThreads, s.nbl);
  degrid_backward_kernel<<<grid, kDegridThreads, 0, p->stream>>>(
      s.grid, p->G, s.coef, s.freq, s.vis, s.chan_scale,
      p->cfg.vis_dtype == TOI_VIS_C16_CHANSCALE ? 1 : 0, s.weight, s.flag, s.nbl, s.nch,
      p->cfg.n_pol, s.snap, dot, (float)p->beta_es, grad_sample, grad_vis, grad_weight);
  clear_rows_kernel<<<p->G / 2, 256, 0, p->stream>>>(s.grid, p->G, s.snap);
  prof_end(p, tok);
  return cudaGetLastError();
}

// The weight-gradient part of the reverse pass for a tilted-plane cotangent
// already transformed into the slot's grid (launch_fft_adjoint): grad_weight
// = Re(conj(g_q) V_p) - *dot / sum w on the unflagged parallel hands of
// selected samples, 0 elsewhere; the grid rows are cleared afterwards.
cudaError_t launch_degrid_weights(toi_plan_s* p, Slot& s, const double* dot, float* grad_weight) {
  const dim3 grid((s.nch + kDegridThreads - 1) / kDegridThreads, s.nbl);
  degrid_backward_kernel<<<grid, kDegridThreads, 0, p->stream>>>(
      s.grid, p->G, s.coef, s.freq, s.vis, s.chan_scale,
      p->cfg.vis_dtype == TOI_VIS_C16_CHANSCALE ? 1 : 0, s.weight, s.flag, s.nbl, s.nch,
      p->cfg.n_pol, s.snap, dot, (float)p->beta_es, nullptr, nullptr, grad_weight);
  clear_rows_kernel<<<p->G / 2, 256, 0, p->stream>>>(s.grid, p->G, s.snap);
  return cudaGetLastError();
}

}  // namespace toi
