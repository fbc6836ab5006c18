// Windowed point-source localisation: toi_localise_seed and toi_localise.
//
// A candidate window is a WIN x WIN block of a snapshot's tilted-plane image
// (Section 3.2) with corner (row j2c, column j1c).  Its model is the 2-D
// dirty image of one point source (l, m, S), V = S exp(-2 pi i k (u l + v m
// + w (n - 1))) in the parallel hands (Section 1's measurement equation),
// with the data's flags and weights, on the window's pixels.  The loss of a
// window is sum (D - M)^2 over its pixels, D the snapshot's tilted image.
//
// Faceted gridding.  Window w gets its own grid of F = 2 WIN cells (the
// oversampling of the full image) over the full grid's uv extent.  Sample q
// is rotated to the window centre t_c,
//   c'_q = S W_q exp(2 pi i k P_bw),  P_bw = r.t_c - b.(l, m, n - 1)  (metres,
//   r = V b in the tilted frame, only r1, r2 as in the 2-D image),
// and gridded with the ES kernel at gf = F/2 + (F / G) a k, the full grid's
// coordinate scaled.  The facet's inverse DFT cropped to the central WIN x
// WIN, times 1/psi_hat (for WIN pixels on F cells) and 1/(omega sum w), is
// the model window.  Facet indices wrap modulo F: at integer pixel offsets
// the image is F-periodic in k, so the wrap is exact.
//
// Reverse mode (complex gradients as dL/dRe + i dL/dIm):
//   g^M = -2 (D - M) on the window, K_w = the forward DFT of
//   g^M corr corr / (omega sum w) (the facet image's adjoint),
//   dL/dc'_q = sum psi psi K_w (degridding), zz = conj(dL/dc'_q) e^{2 pi i k P};
//   dL/dS = sum_q W_q Re zz,
//   dL/dl = sum_q S W_q 2 pi k (u - w l / n) Im zz   (m alike with v),
//   dL/dw_p = sum_w S_w Re zz_w                       (the models)
//           + Re(conj(g^D_q) V_p) - 2 L / sum w       (data, normalisation)
// on the unflagged parallel hands of selected samples, where g^D is the
// full-image adjoint of the data cotangent +2 (D - M) on the windows (the
// degridding of toi_degrid_backward without the re-projection step).
#include <math.h>

#include "toi_internal.cuh"

namespace toi {
cudaError_t launch_fft_adjoint(toi_plan_s* p, Slot& s);
cudaError_t launch_degrid_weights(toi_plan_s* p, Slot& s, const double* dot, float* grad_weight);

namespace {

constexpr int kWin = TOI_LOC_WINDOW;   // window side (pixels)
constexpr int kF = 2 * kWin;           // facet grid side (cells)
constexpr int kW = 8;                  // ES kernel support
constexpr int kGridThreads = 256;
constexpr int kDegridThreads = 256;
constexpr int kDegridRun = 8;          // samples per thread in the reverse pass
constexpr int kFinThreads = 256;
constexpr int kSortKeys = 2048;        // keys per block of the window selection
constexpr int kMergeKeys = 4096;

__device__ __forceinline__ void hands(int npol, int& pa, int& pb) {
  if (npol == 4) { pa = 0; pb = 3; }
  else if (npol == 2) { pa = 0; pb = 1; }
  else { pa = 0; pb = 0; }
}

// psi(x) = exp(beta (sqrt(1 - (2x/W)^2) - 1)) on |x| <= W/2, else 0
__device__ __forceinline__ float psi(float x, float beta) {
  const float z = x * (2.0f / kW);
  const float s = 1.0f - z * z;
  return s >= 0.f ? expf(beta * (sqrtf(s) - 1.0f)) : 0.f;
}

// Sample weight W_q = w_a + w_b of the parallel hands (0: not selected).
__device__ __forceinline__ float sample_weight(const float* __restrict__ weight,
                                               const uint8_t* __restrict__ flag, size_t o,
                                               int pa, int pb) {
  const bool fa = flag ? flag[o + pa] != 0 : false;
  const bool fb = flag ? flag[o + pb] != 0 : false;
  const float wa = fa ? 0.f : (weight ? weight[o + pa] : 1.f);
  const float wb = fb ? 0.f : (weight ? weight[o + pb] : 1.f);
  return pa == pb ? wa : wa + wb;
}

// Fractional turns of k P with k = kh + kl and P = Ph + Pl (float pairs):
// the leading product is split exactly by an FMA and its integer part
// removed before the small terms are added.
__device__ __forceinline__ float frac_turns(float kh, float kl, float Ph, float Pl) {
  const float p0 = kh * Ph;
  const float e0 = fmaf(kh, Ph, -p0);
  const float t = fmaf(kh, Pl, fmaf(kl, Ph, e0));
  return (p0 - rintf(p0)) + t;
}

// ---------------------------------------------------------------- set-up --

// k = nu / c as float pairs (hi + lo).
__global__ void loc_k_kernel(const double* __restrict__ freq, int nch, float2* __restrict__ kp) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nch) return;
  const double k = freq[c] / kCLight;
  const float hi = (float)k;
  kp[c] = make_float2(hi, (float)(k - (double)hi));
}

// Per window: corner, flux and validity; per (window, baseline): P_bw as a
// float pair and the factors 2 pi (u - w l / n), 2 pi (v - w m / n) of dl,
// dm.  A source off the unit disc, a non-finite flux or a window off the
// image marks the window invalid (every later stage skips it; its loss and
// gradients are 0) and latches TOI_ERR_RANGE in the status word.
__global__ void loc_coef_kernel(const double* __restrict__ uvw, int nbl,
                                const double* __restrict__ snap, const int* __restrict__ win,
                                const double* __restrict__ src, int nwin, int N, double beta,
                                float4* __restrict__ coef, int4* __restrict__ winfo,
                                int* __restrict__ status) {
  const int w = blockIdx.y;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const double l = src[3 * w], m = src[3 * w + 1], S = src[3 * w + 2];
  const int j2c = win[2 * w], j1c = win[2 * w + 1];
  const double rr = l * l + m * m;
  const bool ok = rr < 1.0 && isfinite(S) && j2c >= 0 && j1c >= 0 && j2c + kWin <= N &&
                  j1c + kWin <= N;
  if (b == 0) {
    winfo[w] = make_int4(j2c, j1c, __float_as_int((float)S), ok ? 1 : 0);
    if (!ok) set_status(status, TOI_DEV_RANGE);
  }
  if (b >= nbl || !ok) return;
  const double n = sqrt(1.0 - rr);
  const double nm1 = -rr / (1.0 + n);
  const double u = uvw[3 * b], v = uvw[3 * b + 1], ww = uvw[3 * b + 2];
  const double* V = snap + SNAP_V;
  const double r1 = V[0] * u + V[1] * v + V[2] * ww;
  const double r2 = V[3] * u + V[4] * v + V[5] * ww;
  const double t1c = -beta * (double)(j1c + kWin / 2 - N / 2);
  const double t2c = beta * (double)(j2c + kWin / 2 - N / 2);
  const double P = r1 * t1c + r2 * t2c - (u * l + v * m + ww * nm1);
  const float Ph = (float)P;
  const double twopi = 6.283185307179586476925;
  coef[(size_t)w * nbl + b] = make_float4(Ph, (float)(P - (double)Ph),
                                          (float)(twopi * (u - ww * l / n)),
                                          (float)(twopi * (v - ww * m / n)));
}

// ------------------------------------------------------- faceted gridding --

// Block (window w, chunk): its threads walk runs of `run` channels of one
// baseline each, keep the 8 x 8 footprint in registers while it stays on the
// same cells (consecutive channels move by ~1e-3 facet cells) and add it to
// the block's shared facet grid when it moves and at the end of the run; the
// block's grid is then added to the window's facet grid in global memory.
__global__ void __launch_bounds__(kGridThreads)
loc_grid_kernel(const BaselineCoef* __restrict__ bcoef, double fscale, const float2* __restrict__ kp,
                const float* __restrict__ weight, const uint8_t* __restrict__ flag, int nbl,
                int nch, int npol, int run, int runs_per_chunk, const float4* __restrict__ coef,
                const int4* __restrict__ winfo, float beta_es, float2* __restrict__ facets) {
  __shared__ float2 F[kF * kF];
  const int w = blockIdx.x;
  for (int i = threadIdx.x; i < kF * kF; i += blockDim.x) F[i] = make_float2(0.f, 0.f);
  __syncthreads();
  const float S = __int_as_float(winfo[w].z);
  if (!winfo[w].w) return;            // uniform per block
  int pa, pb;
  hands(npol, pa, pb);
  const int nrun = (nch + run - 1) / run;
  const long long total = (long long)nbl * nrun;
  const long long r0 = (long long)blockIdx.y * runs_per_chunk;
  const long long r1 = min(total, r0 + runs_per_chunk);
  for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const int b = (int)(r / nrun);
    const int c0 = (int)(r - (long long)b * nrun) * run;
    const int c1 = min(nch, c0 + run);
    const float a1 = (float)(bcoef[b].a1 * fscale), a2 = (float)(bcoef[b].a2 * fscale);
    const float4 cf = coef[(size_t)w * nbl + b];
    float2 acc[kW][kW];
#pragma unroll
    for (int y = 0; y < kW; ++y)
#pragma unroll
      for (int x = 0; x < kW; ++x) acc[y][x] = make_float2(0.f, 0.f);
    int o1 = 0, o2 = 0;
    bool live = false;
    for (int c = c0; c < c1; ++c) {
      const size_t o = ((size_t)b * nch + c) * npol;
      const float Wq = sample_weight(weight, flag, o, pa, pb);
      if (!(Wq > 0.f)) continue;
      const float2 k = kp[c];
      const float g1 = fmaf(a1, k.x, fmaf(a1, k.y, 0.5f * kF));
      const float g2 = fmaf(a2, k.x, fmaf(a2, k.y, 0.5f * kF));
      const int n1 = (int)ceilf(g1 - 0.5f * kW), n2 = (int)ceilf(g2 - 0.5f * kW);
      if (!live || n1 != o1 || n2 != o2) {
        if (live) {
#pragma unroll
          for (int y = 0; y < kW; ++y)
#pragma unroll
            for (int x = 0; x < kW; ++x) {
              float2* dst = &F[((o2 + y) & (kF - 1)) * kF + ((o1 + x) & (kF - 1))];
              atomicAdd(&dst->x, acc[y][x].x);
              atomicAdd(&dst->y, acc[y][x].y);
              acc[y][x] = make_float2(0.f, 0.f);
            }
        }
        o1 = n1;
        o2 = n2;
        live = true;
      }
      float wx[kW], wy[kW];
#pragma unroll
      for (int a = 0; a < kW; ++a) {
        wx[a] = psi((float)(n1 + a) - g1, beta_es);
        wy[a] = psi((float)(n2 + a) - g2, beta_es);
      }
      float sn, cs;
      sincospif(2.0f * frac_turns(k.x, k.y, cf.x, cf.y), &sn, &cs);
      const float sw = S * Wq;
      const float cr = sw * cs, ci = sw * sn;
#pragma unroll
      for (int y = 0; y < kW; ++y) {
        const float yr = wy[y] * cr, yi = wy[y] * ci;
#pragma unroll
        for (int x = 0; x < kW; ++x) {
          acc[y][x].x = fmaf(wx[x], yr, acc[y][x].x);
          acc[y][x].y = fmaf(wx[x], yi, acc[y][x].y);
        }
      }
    }
    if (live) {
#pragma unroll
      for (int y = 0; y < kW; ++y)
#pragma unroll
        for (int x = 0; x < kW; ++x) {
          float2* dst = &F[((o2 + y) & (kF - 1)) * kF + ((o1 + x) & (kF - 1))];
          atomicAdd(&dst->x, acc[y][x].x);
          atomicAdd(&dst->y, acc[y][x].y);
        }
    }
  }
  __syncthreads();
  float2* G = facets + (size_t)w * kF * kF;
  for (int i = threadIdx.x; i < kF * kF; i += blockDim.x) {
    const float2 v = F[i];
    if (v.x != 0.f || v.y != 0.f) {
      atomicAdd(&G[i].x, v.x);
      atomicAdd(&G[i].y, v.y);
    }
  }
}

// ------------------------------------------------------------- finish ----

// e^{sign 2 pi i m / F}
__device__ __forceinline__ float2 tw64(const float2* tw, int m, bool neg) {
  const float2 t = tw[m & (kF - 1)];
  return neg ? make_float2(t.x, -t.y) : t;
}

// One block per window: inverse DFT of the facet (rows, then columns, only
// the central WIN outputs), correction and normalisation -> M; the residual
// against the tilted image D, the loss (float64, fixed order), the data
// cotangent 2 (D - M) and the facet adjoint K_w of g^M = -2 (D - M).
__global__ void __launch_bounds__(kFinThreads)
loc_finish_kernel(const float2* __restrict__ facets, const int4* __restrict__ winfo,
                  const float* __restrict__ tilted, int N, const float* __restrict__ corr,
                  const double* __restrict__ snap, float* __restrict__ model_out,
                  double* __restrict__ loss_out, float* __restrict__ gD,
                  float2* __restrict__ Kout, double* __restrict__ loss2) {
  __shared__ float2 T[kF * kWin];        // row-pass output / adjoint rows
  __shared__ float U[kWin * kWin];       // model, then scaled g^M
  __shared__ float2 tw[kF];
  __shared__ double red[kFinThreads / 32];
  const int w = blockIdx.x;
  const int4 wi = winfo[w];
  float2* K = Kout + (size_t)w * kF * kF;
  if (!wi.w) {                        // invalid window: zero loss, model, cotangents
    for (int e = threadIdx.x; e < kF * kF; e += blockDim.x) K[e] = make_float2(0.f, 0.f);
    for (int e = threadIdx.x; e < kWin * kWin; e += blockDim.x) {
      if (model_out) model_out[(size_t)w * kWin * kWin + e] = 0.f;
      gD[(size_t)w * kWin * kWin + e] = 0.f;
    }
    if (threadIdx.x == 0) {
      if (loss_out) loss_out[w] = 0.0;
      loss2[w] = 0.0;
    }
    return;
  }
  for (int i = threadIdx.x; i < kF; i += blockDim.x) {
    float s, c;
    sincospif((float)i / (0.5f * kF), &s, &c);
    tw[i] = make_float2(c, s);
  }
  const float2* Fw = facets + (size_t)w * kF * kF;
  __syncthreads();
  // rows: T[k2][i1] = sum_k1 F[k2][k1] e^{2 pi i (k1 - F/2)(i1 - WIN/2) / F}
  for (int e = threadIdx.x; e < kF * kWin; e += blockDim.x) {
    const int k2 = e / kWin, i1 = e - k2 * kWin;
    const int d1 = i1 - kWin / 2;
    float2 acc = make_float2(0.f, 0.f);
    for (int k1 = 0; k1 < kF; ++k1) {
      const float2 f = __ldg(Fw + k2 * kF + k1);
      const float2 t = tw64(tw, (k1 - kF / 2) * d1, false);
      acc.x = fmaf(f.x, t.x, fmaf(-f.y, t.y, acc.x));
      acc.y = fmaf(f.x, t.y, fmaf(f.y, t.x, acc.y));
    }
    T[e] = acc;
  }
  __syncthreads();
  const double omega = snap[SNAP_OMEGA], sumw = snap[SNAP_SUMW];
  const float inorm = sumw > 0.0 ? (float)(1.0 / (omega * sumw)) : 0.f;
  double lsum = 0.0;
  for (int e = threadIdx.x; e < kWin * kWin; e += blockDim.x) {
    const int i2 = e / kWin, i1 = e - i2 * kWin;
    const int d2 = i2 - kWin / 2;
    float re = 0.f;
    for (int k2 = 0; k2 < kF; ++k2) {
      const float2 t = T[k2 * kWin + i1];
      const float2 c = tw64(tw, (k2 - kF / 2) * d2, false);
      re = fmaf(t.x, c.x, fmaf(-t.y, c.y, re));
    }
    const float sc = corr[i1] * corr[i2] * inorm;
    const float M = re * sc;
    const float D = tilted[(size_t)(wi.x + i2) * N + wi.y + i1];
    const float R = D - M;
    if (model_out) model_out[(size_t)w * kWin * kWin + e] = M;
    gD[(size_t)w * kWin * kWin + e] = 2.0f * R;
    U[e] = -2.0f * R * sc;           // g^M scaled by the forward's factor
    lsum += (double)R * (double)R;
  }
  for (int off = 16; off > 0; off >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kFinThreads / 32; ++i) t += red[i];
    if (loss_out) loss_out[w] = t;
    loss2[w] = 2.0 * t;
  }
  // adjoint: K[k2][k1] = sum_{i2, i1} U[i2][i1] e^{-2 pi i ((k1 - F/2) d1 + (k2 - F/2) d2) / F}
  for (int e = threadIdx.x; e < kWin * kF; e += blockDim.x) {
    const int i2 = e / kF, k1 = e - i2 * kF;
    float2 acc = make_float2(0.f, 0.f);
    for (int i1 = 0; i1 < kWin; ++i1) {
      const float u = U[i2 * kWin + i1];
      const float2 t = tw64(tw, (k1 - kF / 2) * (i1 - kWin / 2), true);
      acc.x = fmaf(u, t.x, acc.x);
      acc.y = fmaf(u, t.y, acc.y);
    }
    T[e] = acc;                       // T[i2][k1]
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kF * kF; e += blockDim.x) {
    const int k2 = e / kF, k1 = e - k2 * kF;
    float2 acc = make_float2(0.f, 0.f);
    for (int i2 = 0; i2 < kWin; ++i2) {
      const float2 v = T[i2 * kF + k1];
      const float2 t = tw64(tw, (k2 - kF / 2) * (i2 - kWin / 2), true);
      acc.x = fmaf(v.x, t.x, fmaf(-v.y, t.y, acc.x));
      acc.y = fmaf(v.x, t.y, fmaf(v.y, t.x, acc.y));
    }
    K[e] = acc;
  }
}

// The data cotangents 2 (D - M) of all windows into a zeroed tilted-plane
// image (overlapping windows add), scaled as the adjoint FFT passes expect:
// by the full image's grid correction and 1/(omega sum w).
__global__ void loc_scatter_kernel(const float* __restrict__ gD, const int4* __restrict__ winfo,
                                   int N, const float* __restrict__ corr,
                                   const double* __restrict__ snap, float* __restrict__ tilted) {
  const int w = blockIdx.x;
  const int4 wi = winfo[w];
  if (!wi.w) return;
  const double omega = snap[SNAP_OMEGA], sumw = snap[SNAP_SUMW];
  const float norm = sumw > 0.0 ? (float)(1.0 / (omega * sumw)) : 0.f;
  for (int e = threadIdx.x; e < kWin * kWin; e += blockDim.x) {
    const int j2 = wi.x + e / kWin, j1 = wi.y + e % kWin;
    atomicAdd(&tilted[(size_t)j2 * N + j1],
              gD[(size_t)w * kWin * kWin + e] * (norm * corr[j1] * corr[j2]));
  }
}

// Sum of 2 L_w over the windows (fixed order): the <g, image> term.
__global__ void loc_dot_kernel(const double* __restrict__ loss2, int nwin, double* __restrict__ dot) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < nwin; ++i) t += loss2[i];
    *dot = t;
  }
}

// ------------------------------------------------------------- reverse ---

// Thread = (baseline, run of kDegridRun channels); for each window in turn
// it degrids K_w at its samples and accumulates the window's dS, dl, dm
// (block partials, fixed order) and, per sample over all windows, the model
// part of the weight gradient, added to grad_weight at the end.
__global__ void __launch_bounds__(kDegridThreads)
loc_degrid_kernel(const BaselineCoef* __restrict__ bcoef, double fscale,
                  const float2* __restrict__ kp, const float* __restrict__ weight,
                  const uint8_t* __restrict__ flag, int nbl, int nch, int npol,
                  const float4* __restrict__ coef, const int4* __restrict__ winfo, int nwin,
                  const float2* __restrict__ Kall, float beta_es, double* __restrict__ part,
                  float* __restrict__ grad_weight) {
  __shared__ float red[kDegridThreads / 32][3];
  int pa, pb;
  hands(npol, pa, pb);
  const int nrun = (nch + kDegridRun - 1) / kDegridRun;
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = r < (long long)nbl * nrun;
  const int b = active ? (int)(r / nrun) : 0;
  const int c0 = active ? (int)(r - (long long)b * nrun) * kDegridRun : 0;
  float Wq[kDegridRun], Aq[kDegridRun];
  float a1 = 0.f, a2 = 0.f;
  if (active) {
    a1 = (float)(bcoef[b].a1 * fscale);
    a2 = (float)(bcoef[b].a2 * fscale);
  }
#pragma unroll
  for (int j = 0; j < kDegridRun; ++j) {
    const int c = c0 + j;
    Wq[j] = (active && c < nch)
                ? sample_weight(weight, flag, ((size_t)b * nch + c) * npol, pa, pb) : 0.f;
    Aq[j] = 0.f;
  }
  for (int w = 0; w < nwin; ++w) {
    float dS = 0.f, dl = 0.f, dm = 0.f;
    if (active && winfo[w].w) {
      const float S = __int_as_float(winfo[w].z);
      const float4 cf = coef[(size_t)w * nbl + b];
      const float2* K = Kall + (size_t)w * kF * kF;
#pragma unroll 1
      for (int j = 0; j < kDegridRun; ++j) {
        if (!(Wq[j] > 0.f)) continue;
        const float2 k = kp[c0 + j];
        const float g1 = fmaf(a1, k.x, fmaf(a1, k.y, 0.5f * kF));
        const float g2 = fmaf(a2, k.x, fmaf(a2, k.y, 0.5f * kF));
        const int n1 = (int)ceilf(g1 - 0.5f * kW), n2 = (int)ceilf(g2 - 0.5f * kW);
        float wx[kW];
#pragma unroll
        for (int a = 0; a < kW; ++a) wx[a] = psi((float)(n1 + a) - g1, beta_es);
        float gr = 0.f, gi = 0.f;
#pragma unroll
        for (int y = 0; y < kW; ++y) {
          const float wy = psi((float)(n2 + y) - g2, beta_es);
          const float2* row = K + ((n2 + y) & (kF - 1)) * kF;
          float rr = 0.f, ri = 0.f;
#pragma unroll
          for (int x = 0; x < kW; ++x) {
            const float2 v = __ldg(row + ((n1 + x) & (kF - 1)));
            rr = fmaf(wx[x], v.x, rr);
            ri = fmaf(wx[x], v.y, ri);
          }
          gr = fmaf(wy, rr, gr);
          gi = fmaf(wy, ri, gi);
        }
        float sn, cs;
        sincospif(2.0f * frac_turns(k.x, k.y, cf.x, cf.y), &sn, &cs);
        // zz = conj(g) e^{2 pi i k P}
        const float zr = gr * cs + gi * sn, zi = gr * sn - gi * cs;
        dS = fmaf(Wq[j], zr, dS);
        const float swk = S * Wq[j] * k.x;
        dl = fmaf(swk * cf.z, zi, dl);
        dm = fmaf(swk * cf.w, zi, dm);
        Aq[j] = fmaf(S, zr, Aq[j]);
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      dS += __shfl_down_sync(0xffffffffu, dS, off);
      dl += __shfl_down_sync(0xffffffffu, dl, off);
      dm += __shfl_down_sync(0xffffffffu, dm, off);
    }
    if ((threadIdx.x & 31) == 0) {
      red[threadIdx.x >> 5][0] = dl;      // grad_src order: l, m, S
      red[threadIdx.x >> 5][1] = dm;
      red[threadIdx.x >> 5][2] = dS;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      double t = 0.0;
      for (int i = 0; i < kDegridThreads / 32; ++i) t += (double)red[i][threadIdx.x];
      part[((size_t)blockIdx.x * nwin + w) * 3 + threadIdx.x] = t;
    }
    __syncthreads();
  }
  if (grad_weight && active) {
    const bool fl = flag != nullptr;
#pragma unroll
    for (int j = 0; j < kDegridRun; ++j) {
      const int c = c0 + j;
      if (c >= nch || !(Wq[j] > 0.f)) continue;
      const size_t o = ((size_t)b * nch + c) * npol;
      if (!(fl && flag[o + pa])) grad_weight[o + pa] += Aq[j];
      if (pb != pa && !(fl && flag[o + pb])) grad_weight[o + pb] += Aq[j];
    }
  }
}

// grad_src[w][j] = sum over blocks of the partials (fixed order).
__global__ void loc_reduce_kernel(const double* __restrict__ part, int nblk, int nwin,
                                  double* __restrict__ grad_src) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nwin * 3) return;
  double t = 0.0;
  for (int k = 0; k < nblk; ++k) t += part[(size_t)k * nwin * 3 + i];
  grad_src[i] = t;
}

// ---------------------------------------------------------- window seeds --

// Orderable key of a float (ascending; NaN after +inf) with the tile index.
__device__ __forceinline__ unsigned long long tile_key(float v, int idx) {
  unsigned int u = __float_as_uint(v);
  if (v != v) u = 0xffffffffu;
  else u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return ((unsigned long long)u << 32) | (unsigned int)idx;
}

template <int NK>
__device__ void bitonic_sort(unsigned long long* k) {
  for (int size = 2; size <= NK; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      for (int i = threadIdx.x; i < NK / 2; i += blockDim.x) {
        const int lo = 2 * stride * (i / stride) + (i % stride);
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const unsigned long long a = k[lo], c = k[hi];
        if ((a > c) == up) { k[lo] = c; k[hi] = a; }
      }
    }
  __syncthreads();
}

// Stage 1: each block sorts kSortKeys tiles and keeps its nwin smallest.
__global__ void __launch_bounds__(1024)
seed_sort_kernel(const float* __restrict__ tlisi, int ntiles, int nwin,
                 unsigned long long* __restrict__ best) {
  __shared__ unsigned long long k[kSortKeys];
  for (int i = threadIdx.x; i < kSortKeys; i += blockDim.x) {
    const int t = blockIdx.x * kSortKeys + i;
    k[i] = t < ntiles ? tile_key(tlisi[t], t) : ~0ull;
  }
  bitonic_sort<kSortKeys>(k);
  for (int i = threadIdx.x; i < nwin; i += blockDim.x) best[(size_t)blockIdx.x * nwin + i] = k[i];
}

// Stage 2: one block merges the blocks' candidates and keeps the nwin
// smallest tLISI tiles (ties by tile index).
__global__ void __launch_bounds__(1024)
seed_merge_kernel(const unsigned long long* __restrict__ best, int n, int nwin,
                  int* __restrict__ tiles) {
  __shared__ unsigned long long k[kMergeKeys];
  for (int i = threadIdx.x; i < kMergeKeys; i += blockDim.x) k[i] = i < n ? best[i] : ~0ull;
  bitonic_sort<kMergeKeys>(k);
  for (int i = threadIdx.x; i < nwin; i += blockDim.x)
    tiles[i] = k[i] == ~0ull ? -1 : (int)(k[i] & 0xffffffffull);
}

// Per window: corner centred on the tile (clamped to the image), the
// tilted-image maximum inside it (ties: first in row-major order), and the
// source at that pixel: tau = (t1, t2) of the pixel, tau3 the root of
// |V^T tau + z| = 1 nearest 0, (l, m) = (V^T tau)_{1,2}, S = omega x peak.
__global__ void seed_window_kernel(const int* __restrict__ tiles, int ntx, int T, int N,
                                   const float* __restrict__ tilted,
                                   const double* __restrict__ snap, double beta,
                                   int* __restrict__ win, double* __restrict__ src) {
  __shared__ float bv[32];
  __shared__ int bi[32];
  const int w = blockIdx.x;
  const int tile = tiles[w];
  int j2c = 0, j1c = 0;
  if (tile >= 0) {
    const int ty = tile / ntx, tx = tile - ty * ntx;
    j2c = min(max(ty * T + T / 2 - kWin / 2, 0), N - kWin);
    j1c = min(max(tx * T + T / 2 - kWin / 2, 0), N - kWin);
  }
  float best = -INFINITY;
  int bidx = 0x7fffffff;
  for (int e = threadIdx.x; e < kWin * kWin; e += blockDim.x) {
    const float v = tilted[(size_t)(j2c + e / kWin) * N + j1c + e % kWin];
    if (v > best || (v == best && e < bidx)) { best = v; bidx = e; }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const float ov = __shfl_down_sync(0xffffffffu, best, off);
    const int oi = __shfl_down_sync(0xffffffffu, bidx, off);
    if (ov > best || (ov == best && oi < bidx)) { best = ov; bidx = oi; }
  }
  if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = best; bi[threadIdx.x >> 5] = bidx; }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int i = 1; i < (int)(blockDim.x >> 5); ++i)
    if (bv[i] > best || (bv[i] == best && bi[i] < bidx)) { best = bv[i]; bidx = bi[i]; }
  const int j2 = j2c + bidx / kWin, j1 = j1c + bidx % kWin;
  const double* V = snap + SNAP_V;
  const double t1 = -beta * (double)(j1 - N / 2), t2 = beta * (double)(j2 - N / 2);
  const double a = t1 * t1 + 2.0 * t1 * V[2] + t2 * t2 + 2.0 * t2 * V[5];
  const double v33 = V[8];
  const double disc = v33 * v33 - a;
  const double t3 = disc >= 0.0 ? -copysign(1.0, v33) * a / (sqrt(disc) + fabs(v33)) : 0.0;
  const double l = V[0] * t1 + V[3] * t2 + V[6] * t3;
  const double m = V[1] * t1 + V[4] * t2 + V[7] * t3;
  win[2 * w] = j2c;
  win[2 * w + 1] = j1c;
  src[3 * w] = l;
  src[3 * w + 1] = m;
  src[3 * w + 2] = snap[SNAP_OMEGA] * (double)best;
}

}  // namespace

size_t loc_part_doubles(int max_bl, int max_ch, int max_win) {
  const long long runs = (long long)max_bl * ((max_ch + kDegridRun - 1) / kDegridRun);
  const long long blocks = (runs + kDegridThreads - 1) / kDegridThreads;
  return (size_t)blocks * max_win * 3;
}

int loc_seed_max_tiles(int nwin) {
  // stage 2 holds (blocks of stage 1) x nwin keys
  return nwin > 0 ? (kMergeKeys / nwin) * kSortKeys : 0;
}

cudaError_t launch_localise_seed(toi_plan_s* p, Slot& s, const float* tlisi, int nwin, int* win,
                                 double* src) {
  const int ntx = p->N / p->T, ntiles = ntx * ntx;
  const int nblk = (ntiles + kSortKeys - 1) / kSortKeys;
  seed_sort_kernel<<<nblk, 1024, 0, p->stream>>>(tlisi, ntiles, nwin, p->loc_keys);
  seed_merge_kernel<<<1, 1024, 0, p->stream>>>(p->loc_keys, nblk * nwin, nwin, p->loc_tiles);
  seed_window_kernel<<<nwin, 256, 0, p->stream>>>(p->loc_tiles, ntx, p->T, p->N, p->tilted,
                                                  s.snap, p->beta_rad, win, src);
  return cudaGetLastError();
}

cudaError_t launch_localise(toi_plan_s* p, Slot& s, int nwin, const int* win, const double* src,
                            float* model, double* loss, double* grad_src, float* grad_weight) {
  const int nbl = s.nbl, nch = s.nch, npol = p->cfg.n_pol;
  const double fscale = (double)kF / (double)p->G;
  const float beta_es = (float)p->beta_es;
  cudaError_t e = cudaMemsetAsync(p->loc_facets, 0, sizeof(float2) * kF * kF * nwin, p->stream);
  if (e != cudaSuccess) return e;
  loc_k_kernel<<<(nch + 255) / 256, 256, 0, p->stream>>>(s.freq, nch, p->loc_k);
  loc_coef_kernel<<<dim3((nbl + 127) / 128, nwin), 128, 0, p->stream>>>(
      s.uvw, nbl, s.snap, win, src, nwin, p->N, p->beta_rad, p->loc_coef, p->loc_win, p->d_status);
  // faceted gridding: about 8 blocks per SM over all windows
  const int run = nch < 128 ? nch : 128;
  const long long total = (long long)nbl * ((nch + run - 1) / run);
  int chunks = (8 * 152 + nwin - 1) / nwin;
  const long long maxchunks = (total + kGridThreads - 1) / kGridThreads;
  if (chunks > maxchunks) chunks = (int)maxchunks;
  if (chunks < 1) chunks = 1;
  const int per_chunk = (int)((total + chunks - 1) / chunks);
  loc_grid_kernel<<<dim3(nwin, chunks), kGridThreads, 0, p->stream>>>(
      s.coef, fscale, p->loc_k, s.weight, s.flag, nbl, nch, npol, run, per_chunk, p->loc_coef,
      p->loc_win, beta_es, p->loc_facets);
  loc_finish_kernel<<<nwin, kFinThreads, 0, p->stream>>>(
      p->loc_facets, p->loc_win, p->tilted, p->N, p->loc_corr, s.snap, model, loss, p->loc_gD,
      p->loc_K, p->loc_loss2);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (grad_weight) {
    // data term and normalisation through the full-image adjoint
    e = cudaMemsetAsync(p->tilted, 0, sizeof(float) * (size_t)p->N * p->N, p->stream);
    if (e != cudaSuccess) return e;
    loc_scatter_kernel<<<nwin, 256, 0, p->stream>>>(p->loc_gD, p->loc_win, p->N, p->corr, s.snap,
                                                    p->tilted);
    loc_dot_kernel<<<1, 32, 0, p->stream>>>(p->loc_loss2, nwin, p->loc_dot);
    if ((e = launch_fft_adjoint(p, s)) != cudaSuccess) return e;
    if ((e = launch_degrid_weights(p, s, p->loc_dot, grad_weight)) != cudaSuccess) return e;
  }
  if (grad_src || grad_weight) {
    const long long runs = (long long)nbl * ((nch + kDegridRun - 1) / kDegridRun);
    const int nblk = (int)((runs + kDegridThreads - 1) / kDegridThreads);
    loc_degrid_kernel<<<nblk, kDegridThreads, 0, p->stream>>>(
        s.coef, fscale, p->loc_k, s.weight, s.flag, nbl, nch, npol, p->loc_coef, p->loc_win,
        nwin, p->loc_K, beta_es, p->loc_part, grad_weight);
    if (grad_src)
      loc_reduce_kernel<<<(3 * nwin + 127) / 128, 128, 0, p->stream>>>(p->loc_part, nblk, nwin,
                                                                        grad_src);
  }
  return cudaGetLastError();
}

}  // namespace toi
