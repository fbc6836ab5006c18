// Near-coplanar (3-D) mode (Section 3.4, Appendix B, Table 2).
//
// The residual phase exp(i 2 pi r3 t3) is kept: t3 lies on the celestial
// sphere, t3 = -V33 + sgn(V33) sqrt(1 - (t1 + V13)^2 - (t2 + V23)^2) (App. B.1),
// evaluated here without cancellation as -sgn(V33) a / (sqrt(V33^2 - a) + |V33|)
// with a = t1^2 + 2 t1 V13 + t2^2 + 2 t2 V23.  r3 is cut into N_slab slabs of
// half-width dr3; inside slab p, exp(i alpha s) with s = (r3 - r3_p) / dr3 and
// alpha = 2 pi dr3 t3 is expanded as sum_k c_k(alpha) T_k(s) with c_0 = J_0,
// c_k = 2 i^k J_k (Jacobi-Anger, App. B.2).  Each Chebyshev moment
// M_pk = sum_q T_k(s_q) c_q exp(i 2 pi (r1 t1 + r2 t2)) is an ordinary 2-D
// gridding + inverse FFT; the image is Re sum_p exp(i 2 pi r3_p t3)
// sum_k c_k M_pk.
//
// Selection (Eqs. 26-27): Phi_max = 2 pi t3max (r3max - r3min) / 2 over the
// selected samples and the image's pixel centres, N_slab = max(1,
// ceil(Phi_max / 10)), alpha_slab = 2 pi t3max dr3, K the smallest of
// {8, 16, 24, 32} whose sampled error max |exp(i alpha s) - sum_k c_k T_k(s)|
// over 256 alphas in [0, alpha_slab] and 257 s in [-1, 1] is below 1e-2.
// All of it runs on the device in float64 (the choices are integers and
// must match a float64 evaluation); the host reads the plan back once.
//
// Moment images are complex; each is formed as two real-output transforms
// of Hermitian half-plane grids: the real part from T_k c, the imaginary
// part from -i T_k c (Re of the transform of -i G is Im of that of G).  One
// gridding pass fills both grids (see the gridder's Sink).
#include <math.h>
#include <string.h>

#include <vector>

#include "toi_internal.cuh"

namespace toi {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kNAlpha = 256, kNS = 257, kKMax = 32;
constexpr double kGamma = 1e-2, kAlphaTarget = 10.0;

// m3_dev layout (8-byte words)
enum {
  M3_R3MIN = 0,   // ordered int64 key of the smallest selected r3
  M3_R3MAX = 1,   // ordered int64 key of the largest
  M3_T3MAX = 2,   // bits of max |t3| (non-negative double)
  M3_PHI = 3, M3_NSLAB = 4, M3_DR3 = 5, M3_ALPHA = 6, M3_K = 7, M3_ERR = 8,
  M3_ERRK = 9,    // 4 words: bits of the sampled error of K = 8, 16, 24, 32
  M3_HOST = 16,   // words copied back
  M3_J = 16       // [kNAlpha][kKMax] Bessel table
};

// order-preserving int64 key of a double (signed comparison)
__device__ __forceinline__ long long dkey(double d) {
  const long long b = __double_as_longlong(d);
  return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double dkey_inv(long long k) {
  return __longlong_as_double(k >= 0 ? k : (k ^ 0x7fffffffffffffffLL));
}

__global__ void m3_init_kernel(double* m3) {
  long long* k = reinterpret_cast<long long*>(m3);
  k[M3_R3MIN] = dkey(INFINITY);
  k[M3_R3MAX] = dkey(-INFINITY);
  reinterpret_cast<unsigned long long*>(m3)[M3_T3MAX] = 0ull;
  for (int i = 0; i < 4; ++i) reinterpret_cast<unsigned long long*>(m3)[M3_ERRK + i] = 0ull;
}

// r3 (wavelengths) range over the selected samples (w_q > 0, as the plane fit)
__global__ void m3_r3_range_kernel(const BaselineCoef* __restrict__ coef,
                                   const double* __restrict__ kch, const uint8_t* __restrict__ flag,
                                   const float* __restrict__ weight, int nbl, int nch, int npol,
                                   double* m3) {
  int pa, pb;
  parallel_hands(npol, pa, pb);
  double lo = INFINITY, hi = -INFINITY;
  const long long n = (long long)nbl * nch;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const int bl = (int)(q / nch), ch = (int)(q - (long long)bl * nch);
    const size_t o = (size_t)q * npol;
    const bool fa = flag ? flag[o + pa] != 0 : false;
    const bool fb = flag ? flag[o + pb] != 0 : false;
    const float wa = fa ? 0.f : (weight ? weight[o + pa] : 1.f);
    const float wb = fb ? 0.f : (weight ? weight[o + pb] : 1.f);
    if (((pa == pb) ? wa : wa + wb) > 0.f) {
      const double r3 = coef[bl].r3 * kch[ch];
      lo = fmin(lo, r3);
      hi = fmax(hi, r3);
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, off));
    hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, off));
  }
  if ((threadIdx.x & 31) == 0 && lo <= hi) {
    long long* k = reinterpret_cast<long long*>(m3);
    atomicMin(k + M3_R3MIN, dkey(lo));
    atomicMax(k + M3_R3MAX, dkey(hi));
  }
}

// max |t3| over the pixel centres, float64
__global__ void m3_t3max_kernel(const double* __restrict__ snap, int N, double beta, double* m3) {
  const int j1 = blockIdx.x * 16 + (threadIdx.x & 15);
  const int j2 = blockIdx.y * 16 + (threadIdx.x >> 4);
  double v = 0.0;
  if (j1 < N && j2 < N) {
    const double t1 = -beta * (j1 - N / 2), t2 = beta * (j2 - N / 2);
    const double V13 = snap[SNAP_V + 2], V23 = snap[SNAP_V + 5], V33 = snap[SNAP_V + 8];
    const double a = t1 * t1 + 2.0 * t1 * V13 + t2 * t2 + 2.0 * t2 * V23;
    v = fabs(a / (sqrt(V33 * V33 - a) + fabs(V33)));
    if (!(v == v)) v = 0.0;   // off the visible sphere: not a valid pixel
  }
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
  if ((threadIdx.x & 31) == 0)
    atomicMax(reinterpret_cast<unsigned long long*>(m3) + M3_T3MAX,
              (unsigned long long)__double_as_longlong(v));
}

// Eqs. 26-27 (one thread)
__global__ void m3_plan_kernel(double* m3) {
  const long long* k = reinterpret_cast<const long long*>(m3);
  const double r3min = dkey_inv(k[M3_R3MIN]), r3max = dkey_inv(k[M3_R3MAX]);
  const double t3max = __longlong_as_double(k[M3_T3MAX]);
  const bool empty = !(r3min <= r3max);
  const double span = empty ? 0.0 : r3max - r3min;
  const double phi = 2.0 * kPi * t3max * span / 2.0;
  const double ns = fmax(1.0, ceil(phi / kAlphaTarget));
  const double dr3 = span / (2.0 * ns);
  m3[M3_PHI] = phi;
  m3[M3_NSLAB] = ns;
  m3[M3_DR3] = dr3;
  m3[M3_ALPHA] = 2.0 * kPi * t3max * dr3;
}

// J_k(alpha_j), k < 32, at the sampled alphas, from the power series
// J_k(x) = sum_m (-1)^m (x/2)^(2m+k) / (m! (m+k)!)  (x <= 10 here: alpha_slab
// = Phi_max / N_slab <= alpha_target; the largest term is below 1e3, so the
// alternating sum keeps about 13 digits, ample for a 1e-2 decision)
__global__ void m3_bessel_kernel(double* m3) {
  const int j = threadIdx.x;
  if (j >= kNAlpha) return;
  const double x = m3[M3_ALPHA] * (double)j / (double)(kNAlpha - 1);
  const double h = 0.5 * x, h2 = h * h;
  double lead = 1.0;   // (x/2)^k / k!
  for (int kk = 0; kk < kKMax; ++kk) {
    double term = lead, sum = lead;
    for (int m = 1; m < 60; ++m) {
      term *= -h2 / ((double)m * (double)(m + kk));
      sum += term;
      if (fabs(term) < 1e-18 * fabs(sum) && m > 2) break;
    }
    m3[M3_J + j * kKMax + kk] = sum;
    lead *= h / (double)(kk + 1);
  }
}

// sampled error of the truncated Jacobi-Anger series for K = 8, 16, 24, 32
__global__ void m3_error_kernel(double* m3) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  double e[4] = {0.0, 0.0, 0.0, 0.0};
  if (id < kNAlpha * kNS) {
    const int j = id / kNS, i = id - (id / kNS) * kNS;
    const double x = m3[M3_ALPHA] * (double)j / (double)(kNAlpha - 1);
    const double s = -1.0 + 2.0 * (double)i / (double)(kNS - 1);
    const double* J = m3 + M3_J + j * kKMax;
    double sn, cs;
    sincos(x * s, &sn, &cs);
    double re = 0.0, im = 0.0, tkm1 = 1.0, tk = 1.0;   // T_{k-1}, T_k
    for (int k = 0; k < kKMax; ++k) {
      if (k == 1) {
        tkm1 = 1.0;
        tk = s;
      } else if (k >= 2) {
        const double tn = 2.0 * s * tk - tkm1;
        tkm1 = tk;
        tk = tn;
      }
      if (k == 0) {
        re += J[0];
      } else {
        const double c = 2.0 * J[k] * tk;       // 2 i^k J_k T_k
        switch (k & 3) {
          case 0: re += c; break;
          case 1: im += c; break;
          case 2: re -= c; break;
          default: im -= c; break;
        }
      }
      if ((k + 1) % 8 == 0) e[(k + 1) / 8 - 1] = hypot(cs - re, sn - im);
    }
  }
  for (int c = 0; c < 4; ++c) {
    double v = e[c];
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
    if ((threadIdx.x & 31) == 0)
      atomicMax(reinterpret_cast<unsigned long long*>(m3) + M3_ERRK + c,
                (unsigned long long)__double_as_longlong(v));
  }
}

__global__ void m3_choose_kernel(double* m3) {
  int K = 32;
  double err = __longlong_as_double(reinterpret_cast<long long*>(m3)[M3_ERRK + 3]);
  for (int c = 0; c < 4; ++c) {
    const double ec = __longlong_as_double(reinterpret_cast<long long*>(m3)[M3_ERRK + c]);
    if (ec < kGamma) { K = 8 * (c + 1); err = ec; break; }
  }
  m3[M3_K] = (double)K;
  m3[M3_ERR] = err;
}

// J_k(+-x), k < K (x >= 0, the sign given by neg), folded on the fly into
// sum_k w_k J_k M_k with w_0 = 1, w_k = 2 i^k; returns that complex sum.  x >= 1e-3: Miller's
// backward recurrence (J.C.P. Miller, 1952; Abramowitz & Stegun 9.12):
// J_{k-1} = (2k / x) J_k - J_{k+1} from an arbitrary start well above
// max(K, x), normalised by J_0 + 2 sum_{k even >= 2} J_k = 1, rescaled
// whenever the unnormalised values grow large.  x < 1e-3: two terms of the
// power series.
__device__ __forceinline__ float2 bessel_fold(float x, bool neg, int K,
                                              const float* __restrict__ re_img,
                                              const float* __restrict__ im_img, size_t pix,
                                              size_t stride) {
  auto add = [&](float2& acc, int k, float jk) {
    if (neg && (k & 1)) jk = -jk;     // J_k(-x) = (-1)^k J_k(x)
    const float mr = re_img[(size_t)(2 * k) * stride + pix];
    const float mi = im_img[(size_t)(2 * k) * stride + pix];
    float wr, wi;                     // w_k J_k
    if (k == 0) { wr = jk; wi = 0.f; }
    else {
      const float c = 2.f * jk;
      switch (k & 3) {
        case 0: wr = c; wi = 0.f; break;
        case 1: wr = 0.f; wi = c; break;
        case 2: wr = -c; wi = 0.f; break;
        default: wr = 0.f; wi = -c; break;
      }
    }
    acc.x += wr * mr - wi * mi;
    acc.y += wr * mi + wi * mr;
  };
  float2 acc = make_float2(0.f, 0.f);
  if (x < 1e-3f) {
    const float h = 0.5f * x, h2 = h * h;
    float lead = 1.f;
    for (int k = 0; k < K; ++k) {
      add(acc, k, lead * (1.f - h2 / (float)(k + 1)));
      lead *= h / (float)(k + 1);
      if (lead < 1e-30f) break;
    }
    return acc;
  }
  const int m0 = ((K + (int)x + 16) | 1) + 1;   // even start
  float jp = 0.f, jc = 1e-20f, norm = 0.f;      // J_{k+1}, J_k (unnormalised)
  for (int k = m0; k >= 1; --k) {
    const float jm = (2.f * (float)k / x) * jc - jp;   // J_{k-1}
    jp = jc;
    jc = jm;
    const int idx = k - 1;
    if (idx < K) add(acc, idx, jc);
    norm += (idx == 0) ? jc : ((idx & 1) == 0 ? 2.f * jc : 0.f);
    if (fabsf(jc) > 1e25f) {
      jc *= 1e-25f; jp *= 1e-25f; norm *= 1e-25f; acc.x *= 1e-25f; acc.y *= 1e-25f;
    }
  }
  const float inv = 1.f / norm;
  return make_float2(acc.x * inv, acc.y * inv);
}

// tilted image = Re sum_p exp(i 2 pi r3_p t3) sum_k c_k(2 pi dr3 t3) M_pk;
// moment images are already corrected and normalised by the column pass
__global__ void combine3_kernel(const float* __restrict__ moments, const float* __restrict__ centres,
                                int n_slab, int K, float dr3, const double* __restrict__ snap, int N,
                                double beta, float* __restrict__ out) {
  const int j1 = blockIdx.x * 16 + (threadIdx.x & 15);
  const int j2 = blockIdx.y * 16 + (threadIdx.x >> 4);
  if (j1 >= N || j2 >= N) return;
  const float t1 = (float)(-beta * (j1 - N / 2)), t2 = (float)(beta * (j2 - N / 2));
  const float V13 = (float)snap[SNAP_V + 2], V23 = (float)snap[SNAP_V + 5];
  const float V33 = (float)snap[SNAP_V + 8];
  const float a = t1 * t1 + 2.f * t1 * V13 + t2 * t2 + 2.f * t2 * V23;
  if (!(V33 * V33 - a >= 0.f)) {   // off the visible sphere: not a valid pixel
    out[(size_t)j2 * N + j1] = 0.f;
    return;
  }
  const float t3 = -copysignf(1.f, V33) * a / (sqrtf(V33 * V33 - a) + fabsf(V33));
  const float x = 2.f * (float)kPi * dr3 * fabsf(t3);
  const bool neg = t3 < 0.f;
  const size_t pix = (size_t)j2 * N + j1, NN = (size_t)N * N;
  float v = 0.f;
  for (int p = 0; p < n_slab; ++p) {
    const float* re_img = moments + (size_t)(p * K) * 2 * NN;
    const float2 s = bessel_fold(x, neg, K, re_img, re_img + NN, pix, NN);
    float sp, cp;
    sincospif(2.f * centres[p] * t3, &sp, &cp);
    v += cp * s.x - sp * s.y;
  }
  out[pix] = v;
}

}  // namespace

cudaError_t mode3_select(toi_plan_s* p, Slot& s, const float* weight, const uint8_t* flag,
                         int nbl, int nch) {
  double* m3 = p->m3_dev;
  m3_init_kernel<<<1, 1, 0, p->stream>>>(m3);
  m3_r3_range_kernel<<<8 * p->nsm, 256, 0, p->stream>>>(s.coef, p->kch, flag, weight, nbl, nch,
                                                         p->cfg.n_pol, m3);
  const dim3 g((p->N + 15) / 16, (p->N + 15) / 16);
  m3_t3max_kernel<<<g, 256, 0, p->stream>>>(s.snap, p->N, p->beta_rad, m3);
  m3_plan_kernel<<<1, 1, 0, p->stream>>>(m3);
  m3_bessel_kernel<<<1, kNAlpha, 0, p->stream>>>(m3);
  m3_error_kernel<<<(kNAlpha * kNS + 255) / 256, 256, 0, p->stream>>>(m3);
  m3_choose_kernel<<<1, 1, 0, p->stream>>>(m3);
  cudaError_t e = cudaMemcpyAsync(p->m3_host, m3, sizeof(double) * M3_HOST,
                                  cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return e;
  const double* h = p->m3_host;
  const long long kmin = reinterpret_cast<const long long*>(h)[M3_R3MIN];
  const long long kmax = reinterpret_cast<const long long*>(h)[M3_R3MAX];
  auto inv = [](long long k) {
    const long long b = k >= 0 ? k : (k ^ 0x7fffffffffffffffLL);
    double d;
    memcpy(&d, &b, sizeof d);
    return d;
  };
  Mode3Plan& m = s.m3;
  m.r3min = inv(kmin);
  m.r3max = inv(kmax);
  double t3;
  memcpy(&t3, &h[M3_T3MAX], sizeof t3);
  m.t3max = t3;
  m.phi = h[M3_PHI];
  m.n_slab = (int)h[M3_NSLAB];
  m.dr3 = h[M3_DR3];
  m.alpha_slab = h[M3_ALPHA];
  m.K = (int)h[M3_K];
  m.err = h[M3_ERR];
  m.ready = m.r3min <= m.r3max;
  if (m.ready && m.n_slab * m.K > p->cfg.max_moments) return cudaErrorNotSupported;
  return cudaSuccess;
}

cudaError_t mode3_moments(toi_plan_s* p, Slot& s, const void* vis, const float* chan_scale,
                          const float* weight, const uint8_t* flag, int nbl, int nch) {
  const Mode3Plan& m = s.m3;
  if (!m.ready) return cudaSuccess;
  std::vector<float> centres(m.n_slab);
  for (int q = 0; q < m.n_slab; ++q) centres[q] = (float)(m.r3min + (2.0 * q + 1.0) * m.dr3);
  cudaError_t e = cudaMemcpyAsync(p->m3_slabs, centres.data(), sizeof(float) * m.n_slab,
                                  cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);   // centres is a host local
  const size_t NN = (size_t)p->N * p->N;
  Slot s_im = s;          // the same snapshot record with the second grid
  s_im.grid = p->grid2;
  for (int q = 0; q < m.n_slab && e == cudaSuccess; ++q)
    for (int k = 0; k < m.K && e == cudaSuccess; ++k) {
      MomentPass mp;
      mp.zero_width = m.dr3 > 0.0 ? 0 : 1;
      mp.r3min = (float)m.r3min;
      mp.inv2dr3 = m.dr3 > 0.0 ? (float)(1.0 / (2.0 * m.dr3)) : 0.f;
      mp.centre = centres[q];
      mp.inv_dr3 = m.dr3 > 0.0 ? (float)(1.0 / m.dr3) : 0.f;
      mp.slab = q;
      mp.nslab = m.n_slab;
      mp.order = k;
      mp.imag = 0;
      mp.grid2 = p->grid2;       // one pass grids both parts
      float* re_img = p->moments + ((size_t)(q * m.K + k) * 2) * NN;
      e = launch_grid_moment(p, s, vis, chan_scale, weight, flag, nbl, nch, mp);
      if (e == cudaSuccess) e = launch_fft_to(p, s, re_img);
      if (e == cudaSuccess) e = launch_fft_to(p, s_im, re_img + NN);
    }
  return e;
}

cudaError_t launch_combine3(toi_plan_s* p, Slot& s) {
  const Mode3Plan& m = s.m3;
  const size_t NN = (size_t)p->N * p->N;
  if (!m.ready) return cudaMemsetAsync(p->tilted, 0, sizeof(float) * NN, p->stream);
  const dim3 g((p->N + 15) / 16, (p->N + 15) / 16);
  combine3_kernel<<<g, 256, 0, p->stream>>>(p->moments, p->m3_slabs, m.n_slab, m.K, (float)m.dr3,
                                            s.snap, p->N, p->beta_rad, p->tilted);
  return cudaGetLastError();
}

}  // namespace toi
