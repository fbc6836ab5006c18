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
constexpr int kPassBlocksPerSM = 4;       // facet passes: blocks over the baselines
constexpr int kFinThreads = 256;
constexpr int kSortKeys = 2048;        // keys per block of the window selection
constexpr int kMergeKeys = 4096;

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
//
// Both facet passes treat a chunk of kChunk consecutive channels of one
// baseline as a small matrix product over all windows.  For the chunk's
// samples whose footprint starts at the same facet cell (o1, o2) (all of
// them unless the track crosses a cell inside the chunk; then the chunk
// takes one pass per origin)
//   T[q][tap] = W_q psi(o2 + y - g2_q) psi(o1 + x - g1_q),   tap = 8 y + x,
//   E[q][w]   = exp(2 pi i k_q P_bw),
// the forward adds sum_q T[q][tap] S_w E[q][w] to facet cell o + tap of
// window w (64 taps x 64 windows per block, accumulated in registers while
// the origin stays and added to the facet grids in global memory when it
// moves), and the reverse pass forms G[q][w] = sum_tap T[q][tap] K_w[o + tap]
// from the 64 x 64 footprint of the windows' adjoints staged in shared
// memory.  One warp evaluates each sample's 16 kernel values once for all
// windows.

constexpr int kChunk = 32;          // samples (channels) per chunk: one warp
constexpr int kWG = 64;             // windows per block (blockIdx.y: window group)
constexpr int kTaps = kW * kW;
constexpr int kPassThreads = 256;     // forward pass block
constexpr int kRevThreads = 128;      // reverse pass block
constexpr int kTRow = kTaps + 4;      // padded row of T [q][tap]: rows start 4 banks apart

struct PassCtl {
  int o1, o2, active, more, flush;
};

// Sample weight table W_q = w_a + w_b (0: not selected) for both passes.
__global__ void loc_wq_kernel(const float* __restrict__ weight, const uint8_t* __restrict__ flag,
                              int nbl, int nch, int npol, float* __restrict__ wq) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)nbl * nch) return;
  int pa, pb;
  parallel_hands(npol, pa, pb);
  wq[q] = sample_weight(weight, flag, (size_t)q * npol, pa, pb);
}

// psi(x) = exp(beta (sqrt(1 - (2x/W)^2) - 1)) on |x| <= W/2, else 0, with
// the hardware approximations of exp2 and sqrt (relative error ~1e-6, far
// below the ES kernel's own error); beta_log2e = beta log2(e)
__device__ __forceinline__ float psi_fast(float x, float beta_log2e) {
  const float s = fmaf(x * x, -4.0f / (kW * kW), 1.0f);   // 1 - (2x/W)^2
  if (!(s >= 0.f)) return 0.f;
  float r, e;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(s));
  asm("ex2.approx.f32 %0, %1;" : "=f"(e) : "f"(fmaf(beta_log2e, r, -beta_log2e)));
  return e;
}

// exp(2 pi i f) for |f| <= ~0.5 (hardware sin/cos: absolute error ~5e-7)
__device__ __forceinline__ float2 cis_turns(float f) {
  float sn, cs;
  __sincosf(6.283185307179586f * f, &sn, &cs);
  return make_float2(cs, sn);
}

// exp(2 pi i k_q P) for m consecutive samples q0 .. q0 + m - 1 of a chunk:
// the first exactly (compensated k P), the others by the ratio
// exp(2 pi i dk P) when the channels are equally spaced (to the float
// resolution of dk P), else each one exactly.
template <int M>
__device__ __forceinline__ void phases(const float2* kq, int q0, float2 P, float2* e) {
  const float2 k0 = kq[q0];
  e[0] = cis_turns(frac_turns(k0.x, k0.y, P.x, P.y));
  const float2 k1 = kq[q0 + 1];
  const float dk = (k1.x - k0.x) + (k1.y - k0.y);
  bool uniform = dk != 0.f;
#pragma unroll
  for (int i = 2; i < M; ++i) {
    const float2 a = kq[q0 + i], b = kq[q0 + i - 1];
    const float d = (a.x - b.x) + (a.y - b.y);
    uniform = uniform && fabsf(d - dk) * fabsf(P.x) < 1e-7f;
  }
  if (uniform) {
    const float2 z = cis_turns(frac_turns(dk, 0.f, P.x, P.y));
#pragma unroll
    for (int i = 1; i < M; ++i)
      e[i] = make_float2(e[i - 1].x * z.x - e[i - 1].y * z.y, e[i - 1].x * z.y + e[i - 1].y * z.x);
  } else {
#pragma unroll
    for (int i = 1; i < M; ++i) {
      const float2 k = kq[q0 + i];
      e[i] = cis_turns(frac_turns(k.x, k.y, P.x, P.y));
    }
  }
}

// Warp 0 (lane = sample of the chunk): choose the next origin among the
// pending samples (the block's current origin first, so that a chunk that
// continues it costs no flush), write the pass's T (0 for samples outside
// it) and clear them from `pending` (warp-uniform).  TQ: T is [q][tap],
// else [tap][q].
template <bool TQ>
__device__ __forceinline__ void build_pass(float* T, unsigned& pending, float g1, float g2,
                                           float Wq, int cur1, int cur2, bool have,
                                           float beta_log2e, PassCtl* ctl) {
  const int lane = threadIdx.x;
  const int n1 = (int)ceilf(g1 - 0.5f * kW), n2 = (int)ceilf(g2 - 0.5f * kW);
  const bool mine = (pending >> lane) & 1u;
  const unsigned cur = __ballot_sync(0xffffffffu, mine && n1 == cur1 && n2 == cur2);
  int o1 = cur1, o2 = cur2;
  unsigned in = 0;
  if (have && cur) {
    in = cur;
  } else if (pending) {
    const int first = __ffs(pending) - 1;
    o1 = __shfl_sync(0xffffffffu, n1, first);
    o2 = __shfl_sync(0xffffffffu, n2, first);
    in = __ballot_sync(0xffffffffu, mine && n1 == o1 && n2 == o2);
  }
  const bool use = (in >> lane) & 1u;
  float wx[kW], wy[kW];
#pragma unroll
  for (int a = 0; a < kW; ++a) {
    wx[a] = use ? psi_fast((float)(o1 + a) - g1, beta_log2e) : 0.f;
    wy[a] = use ? Wq * psi_fast((float)(o2 + a) - g2, beta_log2e) : 0.f;
  }
#pragma unroll
  for (int y = 0; y < kW; ++y) {
    if (TQ) {
      float4* row = reinterpret_cast<float4*>(T + lane * kTRow + y * kW);
      row[0] = make_float4(wy[y] * wx[0], wy[y] * wx[1], wy[y] * wx[2], wy[y] * wx[3]);
      row[1] = make_float4(wy[y] * wx[4], wy[y] * wx[5], wy[y] * wx[6], wy[y] * wx[7]);
    } else {
#pragma unroll
      for (int x = 0; x < kW; ++x) T[(y * kW + x) * kChunk + lane] = wy[y] * wx[x];
    }
  }
  pending &= ~in;
  if (lane == 0) {
    ctl->o1 = o1;
    ctl->o2 = o2;
    ctl->active = in != 0;
    ctl->more = pending != 0;
    ctl->flush = have && in != 0 && (o1 != cur1 || o2 != cur2);
  }
}

// Block (baselines blockIdx.x, blockIdx.x + gridDim.x, ...; window group
// blockIdx.y).  Thread t accumulates taps 4 (t / 16) .. + 3 for windows
// 4 (t % 16) .. + 3 of the group.
__global__ void __launch_bounds__(kPassThreads, 3)
loc_grid_kernel(const BaselineCoef* __restrict__ bcoef, double fscale,
                const float2* __restrict__ kp, const float* __restrict__ wq, int nbl, int nch,
                const float4* __restrict__ coef, const int4* __restrict__ winfo, int nwin,
                float beta_log2e, float2* __restrict__ facets) {
  __shared__ __align__(16) float T[kChunk * kTRow];     // [q][tap], padded rows
  // C[q] holds S_w E[q][w] for w = 4 b + j at [(j / 2) 32 + 2 b + j % 2]: the
  // two float4 loads of a thread's four windows each cover 256 contiguous bytes
  __shared__ __align__(16) float2 C[kChunk * kWG];
  __shared__ float2 Pw[kWG];
  __shared__ float Sw[kWG];
  __shared__ float2 kq[kChunk];
  __shared__ PassCtl ctl;
  const int t = threadIdx.x;
  const int wg0 = blockIdx.y * kWG;
  if (t < kWG) {
    const int w = wg0 + t;
    Sw[t] = (w < nwin && winfo[w].w) ? __int_as_float(winfo[w].z) : 0.f;
  }
  const int tb = t >> 4, wb = t & 15;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  int o1 = 0, o2 = 0;
  bool have = false;

  auto flush = [&]() {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int tap = tb * 4 + i, y = tap >> 3, x = tap & 7;
      const int cell = ((o2 + y) & (kF - 1)) * kF + ((o1 + x) & (kF - 1));
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int w = wg0 + wb * 4 + j;
        if (w < nwin && (acc[i][j].x != 0.f || acc[i][j].y != 0.f)) {
          float2* dst = facets + (size_t)w * kF * kF + cell;
          atomicAdd(&dst->x, acc[i][j].x);
          atomicAdd(&dst->y, acc[i][j].y);
        }
        acc[i][j] = make_float2(0.f, 0.f);
      }
    }
  };

  for (int b = blockIdx.x; b < nbl; b += gridDim.x) {
    __syncthreads();                  // the previous baseline's Pw readers are done
    if (t < kWG) {
      const int w = wg0 + t;
      const float4 cf = w < nwin ? coef[(size_t)w * nbl + b] : make_float4(0.f, 0.f, 0.f, 0.f);
      Pw[t] = make_float2(cf.x, cf.y);
    }
    float a1 = 0.f, a2 = 0.f;
    if (t < kChunk) {
      a1 = (float)(bcoef[b].a1 * fscale);
      a2 = (float)(bcoef[b].a2 * fscale);
    }
    for (int ch0 = 0; ch0 < nch; ch0 += kChunk) {
      float g1 = 0.f, g2 = 0.f, W = 0.f;
      unsigned pending = 0;
      if (t < kChunk) {
        const int c = ch0 + t;
        float2 k = make_float2(0.f, 0.f);
        if (c < nch) {
          W = wq[(size_t)b * nch + c];
          k = kp[c];
        }
        g1 = fmaf(a1, k.x, fmaf(a1, k.y, 0.5f * kF));
        g2 = fmaf(a2, k.x, fmaf(a2, k.y, 0.5f * kF));
        kq[t] = k;
        pending = __ballot_sync(0xffffffffu, W > 0.f);
      }
      __syncthreads();                // kq and Pw written; the last chunk's T, C are read
      {
        // thread t: window t % 64, samples 8 (t / 64) .. + 7
        const int w = t & (kWG - 1), q0 = (t >> 6) * 8;
        float2 ph[8];
        phases<8>(kq, q0, Pw[w], ph);
        const int j = w & 3, col = (j >> 1) * 32 + (w >> 2) * 2 + (j & 1);
#pragma unroll
        for (int i = 0; i < 8; ++i)
          C[(q0 + i) * kWG + col] = make_float2(Sw[w] * ph[i].x, Sw[w] * ph[i].y);
      }
      while (true) {
        if (t < kChunk) build_pass<true>(T, pending, g1, g2, W, o1, o2, have, beta_log2e, &ctl);
        __syncthreads();
        const PassCtl c = ctl;
        if (!c.active) break;
        if (c.flush) flush();
        o1 = c.o1;
        o2 = c.o2;
        have = true;
#pragma unroll 4
        for (int q = 0; q < kChunk; ++q) {
          const float4 tv = *reinterpret_cast<const float4*>(T + q * kTRow + tb * 4);
          const float4 ca = *reinterpret_cast<const float4*>(C + q * kWG + wb * 2);
          const float4 cb = *reinterpret_cast<const float4*>(C + q * kWG + 32 + wb * 2);
          const float tt[4] = {tv.x, tv.y, tv.z, tv.w};
          const float2 cc[4] = {make_float2(ca.x, ca.y), make_float2(ca.z, ca.w),
                                make_float2(cb.x, cb.y), make_float2(cb.z, cb.w)};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              acc[i][j].x = fmaf(tt[i], cc[j].x, acc[i][j].x);
              acc[i][j].y = fmaf(tt[i], cc[j].y, acc[i][j].y);
            }
        }
        __syncthreads();              // T read before the next pass rewrites it
        if (!c.more) break;
      }
    }
  }
  if (have) flush();
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

// Block as loc_grid_kernel (kRevThreads threads).  Per pass, thread t forms G
// for samples 4 (t / 16) .. + 3 and windows 4 (t % 16) .. + 3 of the group,
// then
//   zz = conj(G) E;  dS_w += W Re zz;  dl_w += S W k fl Im zz;  dm_w alike;
//   A_q += S_w Re zz (the models' weight gradient, summed over the windows
//   in shared memory and added to grad_weight per chunk).
// The window sums are float per chunk, float64 across chunks; the block's
// totals go to part[block][w][3] in a fixed order.  Kf holds the footprint of
// windows 4 b + j at [tap][(j / 2) 32 + 2 b + j % 2], so that a thread's two
// float4 loads each read 256 contiguous bytes.
__global__ void __launch_bounds__(kRevThreads, 4)
loc_degrid_kernel(const BaselineCoef* __restrict__ bcoef, double fscale,
                  const float2* __restrict__ kp, const float* __restrict__ wq,
                  const uint8_t* __restrict__ flag, int nbl, int nch, int npol,
                  const float4* __restrict__ coef, const int4* __restrict__ winfo, int nwin,
                  const float2* __restrict__ Kall, float beta_log2e, double* __restrict__ part,
                  int nwin_part, float* __restrict__ grad_weight) {
  __shared__ __align__(16) float T2[kTaps * kChunk];    // [tap][q]
  __shared__ __align__(16) float2 Kf[kTaps * kWG];      // see above; reused for the final sums
  __shared__ float4 Cf[kWG];
  __shared__ float Sw[kWG];
  __shared__ float2 kq[kChunk];
  __shared__ float Wsh[kChunk];
  __shared__ float Ared[kChunk][17];
  __shared__ PassCtl ctl;
  const int t = threadIdx.x;
  const int wg0 = blockIdx.y * kWG;
  if (t < kWG) {
    const int w = wg0 + t;
    Sw[t] = (w < nwin && winfo[w].w) ? __int_as_float(winfo[w].z) : 0.f;
  }
  int pa, pb;
  parallel_hands(npol, pa, pb);
  const int qb = t >> 4, wb = t & 15;
  double sums[4][3];
#pragma unroll
  for (int j = 0; j < 4; ++j) sums[j][0] = sums[j][1] = sums[j][2] = 0.0;
  int o1 = 0, o2 = 0, k1 = -1 << 30, k2 = 0;     // pass origin, origin of the staged footprint
  bool have = false;
  for (int b = blockIdx.x; b < nbl; b += gridDim.x) {
    __syncthreads();
    if (t < kWG) {
      const int w = wg0 + t;
      Cf[t] = w < nwin ? coef[(size_t)w * nbl + b] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float a1 = 0.f, a2 = 0.f;
    if (t < kChunk) {
      a1 = (float)(bcoef[b].a1 * fscale);
      a2 = (float)(bcoef[b].a2 * fscale);
    }
    for (int ch0 = 0; ch0 < nch; ch0 += kChunk) {
      float g1 = 0.f, g2 = 0.f, W = 0.f;
      unsigned pending = 0;
      if (t < kChunk) {
        const int c = ch0 + t;
        float2 k = make_float2(0.f, 0.f);
        if (c < nch) {
          W = wq[(size_t)b * nch + c];
          k = kp[c];
        }
        g1 = fmaf(a1, k.x, fmaf(a1, k.y, 0.5f * kF));
        g2 = fmaf(a2, k.x, fmaf(a2, k.y, 0.5f * kF));
        kq[t] = k;
        Wsh[t] = W;
        for (int j = 0; j < 17; ++j) Ared[t][j] = 0.f;
        pending = __ballot_sync(0xffffffffu, W > 0.f);
      }
      float cs[4][3];
#pragma unroll
      for (int j = 0; j < 4; ++j) cs[j][0] = cs[j][1] = cs[j][2] = 0.f;
      while (true) {
        // T without the sample weight: the epilogue applies W itself
        if (t < kChunk) build_pass<false>(T2, pending, g1, g2, 1.0f, o1, o2, have, beta_log2e, &ctl);
        __syncthreads();
        const PassCtl c = ctl;
        if (!c.active) break;
        o1 = c.o1;
        o2 = c.o2;
        have = true;
        if (o1 != k1 || o2 != k2) {     // stage the windows' footprints at this origin
          for (int e = t; e < kTaps * kWG; e += kRevThreads) {
            const int tap = e >> 6, wl = e & (kWG - 1), w = wg0 + wl;
            const int y = tap >> 3, x = tap & 7;
            const int j = wl & 3;
            Kf[tap * kWG + (j >> 1) * 32 + (wl >> 2) * 2 + (j & 1)] =
                w < nwin ? __ldg(Kall + (size_t)w * kF * kF + ((o2 + y) & (kF - 1)) * kF +
                                 ((o1 + x) & (kF - 1)))
                         : make_float2(0.f, 0.f);
          }
          k1 = o1;
          k2 = o2;
          __syncthreads();
        }
        float2 g[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) g[i][j] = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int tap = 0; tap < kTaps; ++tap) {
          const float4 tv = *reinterpret_cast<const float4*>(T2 + tap * kChunk + qb * 4);
          const float4 ka = *reinterpret_cast<const float4*>(Kf + tap * kWG + wb * 2);
          const float4 kb = *reinterpret_cast<const float4*>(Kf + tap * kWG + 32 + wb * 2);
          const float tt[4] = {tv.x, tv.y, tv.z, tv.w};
          const float2 kk[4] = {make_float2(ka.x, ka.y), make_float2(ka.z, ka.w),
                                make_float2(kb.x, kb.y), make_float2(kb.z, kb.w)};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              g[i][j].x = fmaf(tt[i], kk[j].x, g[i][j].x);
              g[i][j].y = fmaf(tt[i], kk[j].y, g[i][j].y);
            }
        }
        float2 eph[4][4];             // [window][sample]
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float4 cf = Cf[wb * 4 + j];
          phases<4>(kq, qb * 4, make_float2(cf.x, cf.y), eph[j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int q = qb * 4 + i;
          const float2 k = kq[q];
          const float Wq = Wsh[q];
          float ap = 0.f;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float4 cf = Cf[wb * 4 + j];
            const float S = Sw[wb * 4 + j];
            const float2 e = eph[j][i];
            // zz = conj(g) e
            const float zr = g[i][j].x * e.x + g[i][j].y * e.y;
            const float zi = g[i][j].x * e.y - g[i][j].y * e.x;
            cs[j][2] = fmaf(Wq, zr, cs[j][2]);
            const float swk = S * Wq * k.x;
            cs[j][0] = fmaf(swk * cf.z, zi, cs[j][0]);
            cs[j][1] = fmaf(swk * cf.w, zi, cs[j][1]);
            ap = fmaf(S, zr, ap);
          }
          Ared[q][wb] += ap;
        }
        __syncthreads();              // T2, Kf read before the next pass
        if (!c.more) break;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int m = 0; m < 3; ++m) sums[j][m] += (double)cs[j][m];
      __syncthreads();                // Ared complete
      if (t < kChunk && grad_weight) {
        const int c = ch0 + t;
        if (c < nch && W > 0.f) {
          float A = 0.f;
          for (int j = 0; j < 16; ++j) A += Ared[t][j];
          const size_t o = ((size_t)b * nch + c) * npol;
          // with several window groups, blocks of the same baseline add to the
          // same records: atomically then (one group: plain, deterministic)
          const bool shared = gridDim.y > 1;
          if (!(flag && flag[o + pa])) {
            if (shared) atomicAdd(grad_weight + o + pa, A);
            else grad_weight[o + pa] += A;
          }
          if (pb != pa && !(flag && flag[o + pb])) {
            if (shared) atomicAdd(grad_weight + o + pb, A);
            else grad_weight[o + pb] += A;
          }
        }
      }
    }
  }
  // block totals per window: sum over the 8 sample blocks in a fixed order
  __syncthreads();
  double* red = reinterpret_cast<double*>(Kf);        // [8][64][3]
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int m = 0; m < 3; ++m) red[(qb * kWG + wb * 4 + j) * 3 + m] = sums[j][m];
  __syncthreads();
  for (int e = t; e < kWG * 3; e += kRevThreads) {
    const int w = wg0 + e / 3;
    if (w >= nwin) continue;
    double acc = 0.0;
    for (int i = 0; i < kChunk / 4; ++i) acc += red[i * kWG * 3 + e];
    part[((size_t)blockIdx.x * nwin_part + w) * 3 + e % 3] = acc;
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

size_t loc_part_doubles(int max_bl, int max_win, int nsm) {
  const int cap = kPassBlocksPerSM * nsm;
  const int blocks = max_bl < cap ? max_bl : cap;
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
  cudaError_t e = cudaMemsetAsync(p->loc_facets, 0, sizeof(float2) * kF * kF * nwin, p->stream);
  if (e != cudaSuccess) return e;
  loc_k_kernel<<<(nch + 255) / 256, 256, 0, p->stream>>>(s.freq, nch, p->loc_k);
  const long long nq = (long long)nbl * nch;
  loc_wq_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, p->stream>>>(s.weight, s.flag, nbl, nch,
                                                                     npol, p->loc_wq);
  loc_coef_kernel<<<dim3((nbl + 127) / 128, nwin), 128, 0, p->stream>>>(
      s.uvw, nbl, s.snap, win, src, nwin, p->N, p->beta_rad, p->loc_coef, p->loc_win, p->d_status);
  const float beta_log2e = (float)(p->beta_es * 1.4426950408889634);
  const int cap = kPassBlocksPerSM * p->nsm;
  const int nblk = nbl < cap ? nbl : cap;
  const dim3 pgrid(nblk, (nwin + kWG - 1) / kWG);
  loc_grid_kernel<<<pgrid, kPassThreads, 0, p->stream>>>(
      s.coef, fscale, p->loc_k, p->loc_wq, nbl, nch, p->loc_coef, p->loc_win, nwin, beta_log2e,
      p->loc_facets);
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
    loc_degrid_kernel<<<pgrid, kRevThreads, 0, p->stream>>>(
        s.coef, fscale, p->loc_k, p->loc_wq, s.flag, nbl, nch, npol, p->loc_coef, p->loc_win,
        nwin, p->loc_K, beta_log2e, p->loc_part, nwin, grad_weight);
    if (grad_src)
      loc_reduce_kernel<<<(3 * nwin + 127) / 128, 128, 0, p->stream>>>(p->loc_part, nblk, nwin,
                                                                        grad_src);
  }
  return cudaGetLastError();
}

}  // namespace toi
