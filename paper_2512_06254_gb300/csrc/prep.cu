// S1: sample selection, weights and the SVD basis of one snapshot
// (Sections 3, 3.1 and 3.5; Eq. 11; Section 3.3 for xi and eta).
//
// The plane fit needs, over the selected samples b_q = uvw_bl k_ch
// (k = nu / c), the count, the first moments and the second moments.  They
// factor per baseline: sum_ch sel * k and sum_ch sel * k^2.  Only channels
// whose both parallel hands are flagged are deselected, so each baseline's
// sums are the all-channel sums minus the (rare) deselected ones; with unit
// weights the sum of weights is an exact integer count.
#include <math.h>
#include <stdint.h>

#include "toi_internal.cuh"

namespace toi {
namespace {

// Fixed-order block reduction of `n` doubles per thread (tree over threads).
template <int NT, int NV>
__device__ void block_reduce(double (&v)[NV], double* sh) {
  for (int i = 0; i < NV; ++i) sh[i * NT + threadIdx.x] = v[i];
  __syncthreads();
  for (int s = NT / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int i = 0; i < NV; ++i)
        sh[i * NT + threadIdx.x] = __dadd_rn(sh[i * NT + threadIdx.x], sh[i * NT + threadIdx.x + s]);
    __syncthreads();
  }
  for (int i = 0; i < NV; ++i) v[i] = sh[i * NT];
  __syncthreads();
}

// k = nu / c per channel, per-block sums of k and k^2, monotonicity.
__device__ __forceinline__ void prep_channels_body(const double* __restrict__ freq, int nch,
                                                   double* __restrict__ kch, float2* __restrict__ kf,
                                                   double* __restrict__ kpart, int* status, int blk) {
  __shared__ double sh[2 * 256];
  const int c = blk * 256 + threadIdx.x;
  double v[2] = {0.0, 0.0};
  bool bad = false;
  if (c < nch) {
    const double dir = nch > 1 ? freq[nch - 1] - freq[0] : 1.0;
    const double f = freq[c];
    const double k = f / kCLight;
    kch[c] = k;
    const float hi = (float)k;
    kf[c] = make_float2(hi, (float)(k - (double)hi));
    v[0] = k;
    v[1] = __dmul_rn(k, k);
    if (!(f > 0.0)) bad = true;
    if (c + 1 < nch && !((freq[c + 1] - f) * dir > 0.0)) bad = true;
  }
  if (bad) set_status(status, TOI_DEV_RANGE);
  block_reduce<256, 2>(v, sh);
  if (threadIdx.x == 0) {
    kpart[2 * blk] = v[0];
    kpart[2 * blk + 1] = v[1];
  }
}

__global__ void prep_channels_kernel(const double* __restrict__ freq, int nch,
                                     double* __restrict__ kch, float2* __restrict__ kf,
                                     double* __restrict__ kpart, int* status) {
  prep_channels_body(freq, nch, kch, kf, kpart, status, blockIdx.x);
}

// Per baseline (one warp): deselected channels (both parallel hands flagged
// or zero weight) and the sum of weights; then each block folds its
// baselines' contributions to the 11 plane-fit sums (count, first and second
// moments, sum of weights) into one partial record, in a fixed order.
constexpr int kMomWarps = 8;

__device__ __forceinline__ void
prep_baselines_body(const uint8_t* __restrict__ flag, const float* __restrict__ weight,
                    const double* __restrict__ kch, const double* __restrict__ kpart, int nkblk,
                    const double* __restrict__ uvw, int nbl, int nch, int npol,
                    double* __restrict__ bpart, int blk) {
  __shared__ double sk_all[2];
  __shared__ double contrib[kMomWarps][11];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (wib == 0) {   // lanes take the channel-block partials in a fixed stride, then a tree
    double a = 0.0, b = 0.0;
    for (int i = lane; i < nkblk; i += 32) {
      a = __dadd_rn(a, kpart[2 * i]);
      b = __dadd_rn(b, kpart[2 * i + 1]);
    }
    for (int off = 16; off > 0; off >>= 1) {
      a = __dadd_rn(a, __shfl_down_sync(0xffffffffu, a, off));
      b = __dadd_rn(b, __shfl_down_sync(0xffffffffu, b, off));
    }
    if (lane == 0) {
      sk_all[0] = a;
      sk_all[1] = b;
    }
  }
  __syncthreads();
  const int bl = blk * kMomWarps + wib;
  double out[11];
  for (int i = 0; i < 11; ++i) out[i] = 0.0;
  if (bl < nbl) {
    int pa, pb;
    parallel_hands(npol, pa, pb);
    const size_t base = (size_t)bl * nch * npol;
    double sk = 0.0, sk2 = 0.0, sw = 0.0;
    long long nd = 0, cnt = 0;
    // Per channel only float32 and integer work: a deselected channel sets a
    // bit of `dmask` (its float64 k sums are added afterwards in a
    // data-dependent loop, so they are never issued for the ~all selected
    // channels: float64 issue is scarce on this GPU), and weights are summed
    // with an error-free float32 two-sum, folded into float64 once per
    // iteration.
    float swh = 0.f, swl = 0.f;
    auto add_w = [&](float x) {
      const float t = swh + x;
      const float bp = t - swh;
      swl += (swh - (t - bp)) + (x - bp);
      swh = t;
    };
    // returns whether channel c (flags fa, fb) is deselected
    auto account = [&](int c, bool fa, bool fb) -> bool {
      const size_t o = base + (size_t)c * npol;
      float wa, wb;
      if (weight) {
        wa = fa ? 0.f : weight[o + pa];
        wb = fb ? 0.f : weight[o + pb];
      } else {
        wa = fa ? 0.f : 1.f;
        wb = fb ? 0.f : 1.f;
      }
      const float wq = (pa == pb) ? wa : wa + wb;
      if (wq > 0.f) {
        if (weight) {
          add_w(wa);
          if (pa != pb) add_w(wb);
        } else {
          cnt += (pa == pb) ? 1 : (int)(!fa) + (int)(!fb);
        }
        return false;
      }
      return true;
    };
    auto fold = [&](unsigned int dmask, auto chan_of_bit) {
      if (weight) {
        sw += (double)swh + (double)swl;
        swh = 0.f;
        swl = 0.f;
      }
      while (dmask) {
        const int bit = __ffs(dmask) - 1;
        dmask &= dmask - 1;
        const double k = kch[chan_of_bit(bit)];
        sk += k;
        sk2 += k * k;
        nd += 1;
      }
    };
    constexpr int U = 8;   // independent loads in flight per lane
    if (npol == 4 && flag && !weight && (nch & 3) == 0 &&
        (reinterpret_cast<uintptr_t>(flag) & 15) == 0) {
      // Unit weights (the common case): per channel only integer work on
      // the flag words, four channels at a time.  The two parallel-hand
      // bytes (pols 0 and 3) of two channels are gathered into one word
      // (byte permute), each byte's "nonzero" becomes its high bit (adding
      // 0x7f to the low seven bits carries into bit 7 exactly when they are
      // not all zero), the population count is the number of flagged hands,
      // and a channel with both hands set is deselected.  Loads past the end
      // are zero words: no hand flagged, counted out below.
      const uint4* f16 = reinterpret_cast<const uint4*>(flag + base);
      const int ngrp = nch >> 2;
      int flagged = 0;
      auto nonzero_bytes = [](unsigned int v) {
        return (((v & 0x7f7f7f7fu) + 0x7f7f7f7fu) | v) & 0x80808080u;
      };
      for (int g0 = lane; g0 < ngrp; g0 += 32 * U) {
        uint4 fv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int g = g0 + 32 * u;
          fv[u] = g < ngrp ? __ldcs(f16 + g) : make_uint4(0u, 0u, 0u, 0u);
        }
        unsigned int dmask = 0u;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          // bytes [c0 pol 0, c0 pol 3, c1 pol 0, c1 pol 3], likewise c2, c3
          const unsigned int ta = nonzero_bytes(__byte_perm(fv[u].x, fv[u].y, 0x7430));
          const unsigned int tb = nonzero_bytes(__byte_perm(fv[u].z, fv[u].w, 0x7430));
          flagged += __popc(ta) + __popc(tb);
          const unsigned int da = ta & (ta >> 8), db = tb & (tb >> 8);   // both hands
          if ((da | db) & 0x00800080u)
            dmask |= (((da >> 7) & 1u) | ((da >> 22) & 2u) | ((db >> 5) & 4u) | ((db >> 20) & 8u))
                     << (4 * u);
        }
        fold(dmask, [&](int bit) { return 4 * (g0 + 32 * (bit >> 2)) + (bit & 3); });
      }
      // the lane's hands: 8 per group it owns (groups lane, lane + 32, ...)
      const int mine = lane < ngrp ? 8 * ((ngrp - 1 - lane) / 32 + 1) : 0;
      cnt = mine - flagged;
    } else if (npol == 4 && flag && (nch & 3) == 0 &&
        (reinterpret_cast<uintptr_t>(flag) & 15) == 0) {
      // 16 bytes = the 4 pols of 4 consecutive channels; 32 KB per warp in flight
      const uint4* f16 = reinterpret_cast<const uint4*>(flag + base);
      const int ngrp = nch >> 2;
      for (int g0 = lane; g0 < ngrp; g0 += 32 * U) {
        uint4 fv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int g = g0 + 32 * u;
          fv[u] = g < ngrp ? __ldcs(f16 + g) : make_uint4(0u, 0u, 0u, 0u);
        }
        unsigned int dmask = 0u;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int g = g0 + 32 * u;
          if (g >= ngrp) continue;
          const unsigned int w4[4] = {fv[u].x, fv[u].y, fv[u].z, fv[u].w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (account(4 * g + i, (w4[i] & 0xffu) != 0, (w4[i] >> 24) != 0))
              dmask |= 1u << (4 * u + i);
        }
        fold(dmask, [&](int bit) { return 4 * (g0 + 32 * (bit >> 2)) + (bit & 3); });
      }
    } else {
      for (int c0 = lane; c0 < nch; c0 += 32 * U) {
        unsigned int f4[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int c = c0 + 32 * u;
          f4[u] = 0u;
          if (c < nch && flag) {
            const size_t o = base + (size_t)c * npol;
            if (npol == 4)
              f4[u] = __ldcs(reinterpret_cast<const unsigned int*>(flag + o));
            else
              f4[u] = (unsigned int)(flag[o + pa] != 0) | ((unsigned int)(flag[o + pb] != 0) << 24);
          }
        }
        unsigned int dmask = 0u;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int c = c0 + 32 * u;
          if (c < nch && account(c, (f4[u] & 0xffu) != 0, (f4[u] >> 24) != 0)) dmask |= 1u << u;
        }
        fold(dmask, [&](int bit) { return c0 + 32 * bit; });
      }
    }
    // fixed-order warp reduction
    for (int off = 16; off > 0; off >>= 1) {
      sk += __shfl_down_sync(0xffffffffu, sk, off);
      sk2 += __shfl_down_sync(0xffffffffu, sk2, off);
      sw += __shfl_down_sync(0xffffffffu, sw, off);
      nd += __shfl_down_sync(0xffffffffu, nd, off);
      cnt += __shfl_down_sync(0xffffffffu, cnt, off);
    }
    if (lane == 0) {
      const double n = (double)(nch - nd);
      const double s1 = sk_all[0] - sk, s2 = sk_all[1] - sk2;
      const double x = uvw[3 * bl], y = uvw[3 * bl + 1], z = uvw[3 * bl + 2];
      out[0] = n;
      out[1] = x * s1; out[2] = y * s1; out[3] = z * s1;
      out[4] = x * x * s2; out[5] = x * y * s2; out[6] = x * z * s2;
      out[7] = y * y * s2; out[8] = y * z * s2; out[9] = z * z * s2;
      out[10] = weight ? sw : (double)cnt;
    }
  }
  if (lane == 0)
    for (int i = 0; i < 11; ++i) contrib[wib][i] = out[i];
  __syncthreads();
  if (threadIdx.x < 11) {
    double a = 0.0;
    for (int wdx = 0; wdx < kMomWarps; ++wdx) a += contrib[wdx][threadIdx.x];
    bpart[(size_t)blk * 11 + threadIdx.x] = a;
  }
}

__global__ void __launch_bounds__(kMomWarps * 32)
prep_baselines_kernel(const uint8_t* __restrict__ flag, const float* __restrict__ weight,
                      const double* __restrict__ kch, const double* __restrict__ kpart, int nkblk,
                      const double* __restrict__ uvw, int nbl, int nch, int npol,
                      double* __restrict__ bpart) {
  prep_baselines_body(flag, weight, kch, kpart, nkblk, uvw, nbl, nch, npol, bpart, blockIdx.x);
}

// 1/x and 1/sqrt(x) for normal x (x > 0 for the square root) to float64
// accuracy with few dependent float64 operations: x = m 2^e with m in
// [1, 2) is split off through the IEEE-754 bit fields (so the float32 seed
// cannot overflow whatever the magnitude of x), a float32 seed is refined by
// two Newton steps in float64 (each squares the relative error: 2^-24 ->
// 2^-48 -> below one ulp), and 2^-e (2^(-e/2)) is applied exactly.
__device__ __forceinline__ double pow2_exact(int e) {   // 2^e, -1022 <= e <= 1023
  return __longlong_as_double((long long)(1023 + e) << 52);
}
__device__ __forceinline__ double split_exp(double x, int& e) {
  const long long b = __double_as_longlong(x);
  e = (int)((b >> 52) & 0x7ff) - 1023;
  return __longlong_as_double((b & (long long)0x800fffffffffffffULL) | (1023LL << 52));
}
__device__ __forceinline__ double rcp64(double x) {
  int e;
  const double m = split_exp(x, e);
  double r = (double)(1.0f / (float)m);
  r = __fma_rn(r, __fma_rn(-m, r, 1.0), r);
  r = __fma_rn(r, __fma_rn(-m, r, 1.0), r);
  return r * pow2_exact(-e);
}
__device__ __forceinline__ double rsqrt64(double x) {
  int e;
  double m = split_exp(x, e);
  if (e & 1) { m *= 2.0; e -= 1; }        // m in [1, 4), e even
  double r = (double)rsqrtf((float)m);
  const double h = 0.5 * m;
  r = __fma_rn(r, __fma_rn(-h * r, r, 0.5), r);
  r = __fma_rn(r, __fma_rn(-h * r, r, 0.5), r);
  return r * pow2_exact(-e / 2);
}

// Eigenvector of the smallest eigenvalue of the symmetric 3x3 C (float64
// accuracy).  A float32 Jacobi solve gives an approximate vector u; the
// float64 Rayleigh quotient l = u.Cu / u.u is then accurate to the square of
// its error, and the null vector of C - l I is the largest cross product of
// two of its rows.  Returns false when C has rank <= 1 (second singular value
// <= 1e-6 of the first), where no plane is defined.
__device__ bool smallest_eigvec(const double Cd[3][3], double v3[3]) {
  double tr = fabs(Cd[0][0]) + fabs(Cd[1][1]) + fabs(Cd[2][2]);
  if (!(tr > 0.0)) return false;
  const double itr = rcp64(tr);
  float a[3][3], e[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      a[i][j] = (float)(Cd[i][j] * itr);
      e[i][j] = (i == j) ? 1.f : 0.f;
    }
  // every index below is a compile-time constant after unrolling, so a and e
  // stay in registers
  for (int sweep = 0; sweep < 12; ++sweep) {
    const float off = fabsf(a[0][1]) + fabsf(a[0][2]) + fabsf(a[1][2]);
    if (off < 1e-30f) break;
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = p + 1; q < 3; ++q) {
        const float apq = a[p][q];
        if (apq == 0.f) continue;
        const float theta = (a[q][q] - a[p][p]) / (2.f * apq);
        const float t = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
        const float c = rsqrtf(t * t + 1.f), s = t * c;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - s * akq;
          a[k][q] = s * akp + c * akq;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - s * aqk;
          a[q][k] = s * apk + c * aqk;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float ekp = e[k][p], ekq = e[k][q];
          e[k][p] = c * ekp - s * ekq;
          e[k][q] = s * ekp + c * ekq;
        }
      }
  }
  const float d[3] = {a[0][0], a[1][1], a[2][2]};
  int imin = 0, imax = 0;
  if (d[1] < d[0]) imin = 1;
  if (d[2] < (imin == 0 ? d[0] : d[1])) imin = 2;
  if (d[1] > d[0]) imax = 1;
  if (d[2] > (imax == 0 ? d[0] : d[1])) imax = 2;
  const int imid = (imin == imax) ? (imin + 1) % 3 : 3 - imin - imax;
  auto pick = [&](int i) { return i == 0 ? d[0] : (i == 1 ? d[1] : d[2]); };
  const double lmax = fmax((double)pick(imax), 0.0), lmid = fmax((double)pick(imid), 0.0);
  // rank <= 1: the float32 estimate is ample for this 1e-6 test
  if (!(sqrt(lmid) > 1e-6 * sqrt(lmax))) return false;
  double u[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) u[r] = imin == 0 ? e[r][0] : (imin == 1 ? e[r][1] : e[r][2]);
  double Cu[3];
  for (int i = 0; i < 3; ++i) Cu[i] = Cd[i][0] * u[0] + Cd[i][1] * u[1] + Cd[i][2] * u[2];
  const double l = (u[0] * Cu[0] + u[1] * Cu[1] + u[2] * Cu[2]) *
                   rcp64(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  double M[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M[i][j] = Cd[i][j] - (i == j ? l : 0.0);
  double best[3] = {0.0, 0.0, 0.0}, bn = -1.0;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const double* m1 = M[r];
    const double* m2 = M[(r + 1) % 3];
    const double cx = m1[1] * m2[2] - m1[2] * m2[1];
    const double cy = m1[2] * m2[0] - m1[0] * m2[2];
    const double cz = m1[0] * m2[1] - m1[1] * m2[0];
    const double nn = cx * cx + cy * cy + cz * cz;
    if (nn > bn) { bn = nn; best[0] = cx; best[1] = cy; best[2] = cz; }
  }
  if (!(bn > 0.0)) {   // exactly diagonalised: u is already exact
    for (int i = 0; i < 3; ++i) v3[i] = u[i];
  } else {
    for (int i = 0; i < 3; ++i) v3[i] = best[i];
  }
  const double inv = rsqrt64(v3[0] * v3[0] + v3[1] * v3[1] + v3[2] * v3[2]);
  for (int i = 0; i < 3; ++i) v3[i] *= inv;
  return true;
}

__device__ __forceinline__ void prep_finalize_body(const double* __restrict__ bpart, int nbpart,
                                                   const double* __restrict__ kch, int nch,
                                                   double* __restrict__ snap, int* status,
                                                   double beta_rad) {
  // one warp per sum: lanes take partials in a fixed stride, then a fixed tree
  __shared__ double v[11];
  __shared__ unsigned long long kdev_bits;
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the channel grid against its chord k0 + c dk: the largest |deviation|
  // (non-negative doubles order like their bit patterns)
  if (threadIdx.x == 0) kdev_bits = 0ull;
  __syncthreads();
  {
    const double k0 = kch[0];
    const double dk = nch > 1 ? (kch[nch - 1] - k0) / (double)(nch - 1) : 0.0;
    double dev = 0.0;
    for (int c = threadIdx.x; c < nch; c += blockDim.x) dev = fmax(dev, fabs(kch[c] - (k0 + c * dk)));
    atomicMax(&kdev_bits, (unsigned long long)__double_as_longlong(dev));
    if (threadIdx.x == 0) {
      snap[SNAP_K0] = k0;
      snap[SNAP_DK] = dk;
    }
  }
  for (int i = wib; i < 11; i += blockDim.x >> 5) {
    double a = 0.0;
    for (int b = lane; b < nbpart; b += 32) a += bpart[(size_t)b * 11 + i];
    for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
    if (lane == 0) v[i] = a;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double N = v[0];
  const int empty = (N <= 0.0 || v[10] <= 0.0) ? 1 : 0;
  double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  if (!empty) {
    const double m1[3] = {v[1], v[2], v[3]};
    const double iN = rcp64(N);
    double C[3][3];
    C[0][0] = v[4] - m1[0] * m1[0] * iN;
    C[0][1] = v[5] - m1[0] * m1[1] * iN;
    C[0][2] = v[6] - m1[0] * m1[2] * iN;
    C[1][1] = v[7] - m1[1] * m1[1] * iN;
    C[1][2] = v[8] - m1[1] * m1[2] * iN;
    C[2][2] = v[9] - m1[2] * m1[2] * iN;
    C[1][0] = C[0][1]; C[2][0] = C[0][2]; C[2][1] = C[1][2];
    double v3[3];
    if (smallest_eigvec(C, v3)) {
      if (v3[2] < 0.0)
        for (int i = 0; i < 3; ++i) v3[i] = -v3[i];
      double e[3] = {1.0, 0.0, 0.0};
      if (fabs(v3[0]) > 0.999) { e[0] = 0.0; e[1] = 1.0; }
      const double d = e[0] * v3[0] + e[1] * v3[1] + e[2] * v3[2];
      double v1[3] = {e[0] - d * v3[0], e[1] - d * v3[1], e[2] - d * v3[2]};
      const double nn = rsqrt64(v1[0] * v1[0] + v1[1] * v1[1] + v1[2] * v1[2]);
      for (int i = 0; i < 3; ++i) v1[i] *= nn;
      const double v2[3] = {v3[1] * v1[2] - v3[2] * v1[1], v3[2] * v1[0] - v3[0] * v1[2],
                            v3[0] * v1[1] - v3[1] * v1[0]};
      for (int i = 0; i < 3; ++i) { V[0][i] = v1[i]; V[1][i] = v2[i]; V[2][i] = v3[i]; }
    }
  } else {
    set_status(status, TOI_DEV_EMPTY);
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) snap[SNAP_V + 3 * i + j] = V[i][j];
  snap[SNAP_OMEGA] = fabs(V[0][0] * V[1][1] - V[1][0] * V[0][1]);
  snap[SNAP_XI] = V[2][0] / V[2][2];
  snap[SNAP_ETA] = V[2][1] / V[2][2];
  snap[SNAP_SUMW] = empty ? 0.0 : v[10];
  snap[SNAP_NVIS] = empty ? 0.0 : N;
  snap[14] = 0.0;   // largest stored grid row touched (written by the coefficient kernel)
  snap[SNAP_RADMAX] = 0.0;   // largest footprint radius (likewise)
  // re-projection constants, once per snapshot instead of per block
  snap[SNAP_REPRO] = (double)(float)(-snap[SNAP_XI] / beta_rad);
  snap[SNAP_REPRO + 1] = (double)(float)(snap[SNAP_ETA] / beta_rad);
  snap[SNAP_REPRO + 2] = (double)(float)(beta_rad * beta_rad);
  snap[15] = 0.0;
  snap[SNAP_KDEV] = __longlong_as_double((long long)kdev_bits);
}

__global__ void prep_finalize_kernel(const double* __restrict__ bpart, int nbpart,
                                     const double* __restrict__ kch, int nch,
                                     double* __restrict__ snap, int* status, double beta_rad) {
  prep_finalize_body(bpart, nbpart, kch, nch, snap, status, beta_rad);
}

// Per baseline: R = V uvw (float64), grid coefficients a1 = -r1 beta G,
// a2 = r2 beta G, and the check that every footprint stays on the grid.
__device__ __forceinline__ void prep_coef_body(const double* __restrict__ uvw, int nbl, int nch,
                                               const double* __restrict__ kch,
                                               double* __restrict__ snap, double beta_rad, int G,
                                               int W, BaselineCoef* __restrict__ coef, int* status,
                                               int b) {
  if (b >= nbl) return;
  double Vs[9];
  for (int i = 0; i < 9; ++i) Vs[i] = snap[SNAP_V + i];
  const bool empty = !(snap[SNAP_SUMW] > 0.0);
  const double kmax = fmax(kch[0], kch[nch - 1]);
  const double lim = 0.5 * G - 0.5 * W;
  const double scale = beta_rad * (double)G;
  const double x = uvw[3 * b], y = uvw[3 * b + 1], z = uvw[3 * b + 2];
  const double r1 = Vs[0] * x + Vs[1] * y + Vs[2] * z;
  const double r2 = Vs[3] * x + Vs[4] * y + Vs[5] * z;
  const double r3 = Vs[6] * x + Vs[7] * y + Vs[8] * z;
  BaselineCoef cf;
  cf.a1 = empty ? 0.0 : -r1 * scale;
  cf.a2 = empty ? 0.0 : r2 * scale;
  cf.r3 = r3;
  cf.pad = 0.0;
  coef[b] = cf;
  if (fabs(cf.a1) * kmax > lim || fabs(cf.a2) * kmax > lim) set_status(status, TOI_DEV_RANGE);
  // largest stored row any footprint of this baseline reaches
  const double rowmax = fmin(fabs(cf.a2) * kmax + 0.5 * W + 1.0, 0.5 * G);
  atomicMax(reinterpret_cast<unsigned long long*>(snap + 14),
            (unsigned long long)__double_as_longlong(rowmax));
  // and the largest distance from the grid centre of any cell it reaches:
  // a sample lies at radius |a| k <= |a| kmax, its taps within W/2 sqrt(2) <
  // W of it (plus a cell of margin for rounding)
  const double radmax = sqrt(cf.a1 * cf.a1 + cf.a2 * cf.a2) * kmax + (double)W + 1.0;
  atomicMax(reinterpret_cast<unsigned long long*>(snap + SNAP_RADMAX),
            (unsigned long long)__double_as_longlong(radmax));
}

__global__ void prep_coef_kernel(const double* __restrict__ uvw, int nbl, int nch,
                                 const double* __restrict__ kch, double* __restrict__ snap,
                                 double beta_rad, int G, int W, BaselineCoef* __restrict__ coef,
                                 int* status) {
  prep_coef_body(uvw, nbl, nch, kch, snap, beta_rad, G, W, coef, status,
                 blockIdx.x * blockDim.x + threadIdx.x);
}

// ---- batched wrappers: blockIdx.y selects the entry; blocks beyond an
// entry's extent (or entries beyond the batch) leave at once ----
__global__ void prep_channels_batch(const BatchEntry* __restrict__ E,
                                    const BatchHeader* __restrict__ hdr, int* status) {
  if ((int)blockIdx.y >= hdr->n) return;
  const BatchEntry& e = E[blockIdx.y];
  if ((int)blockIdx.x * 256 >= e.nch) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) *e.max_cur = 0u;   // this image's max |I| starts at 0
  prep_channels_body(e.freq, e.nch, e.kch, e.kf, e.kpart, status, blockIdx.x);
}

__global__ void __launch_bounds__(kMomWarps * 32, 4)
prep_baselines_batch(const BatchEntry* __restrict__ E, const BatchHeader* __restrict__ hdr,
                     int npol) {
  if ((int)blockIdx.y >= hdr->n) return;
  const BatchEntry& e = E[blockIdx.y];
  if ((int)blockIdx.x * kMomWarps >= e.nbl) return;
  prep_baselines_body(e.flag, e.weight, e.kch, e.kpart, (e.nch + 255) / 256, e.uvw, e.nbl, e.nch,
                      npol, e.bpart, blockIdx.x);
}

__global__ void prep_finalize_batch(const BatchEntry* __restrict__ E,
                                    const BatchHeader* __restrict__ hdr, int* status,
                                    double beta_rad) {
  if ((int)blockIdx.y >= hdr->n) return;
  const BatchEntry& e = E[blockIdx.y];
  prep_finalize_body(e.bpart, (e.nbl + kMomWarps - 1) / kMomWarps, e.kch, e.nch, e.snap, status,
                     beta_rad);
}

__global__ void prep_coef_batch(const BatchEntry* __restrict__ E, const BatchHeader* __restrict__ hdr,
                                double beta_rad, int G, int W, int* status) {
  if ((int)blockIdx.y >= hdr->n) return;
  const BatchEntry& e = E[blockIdx.y];
  prep_coef_body(e.uvw, e.nbl, e.nch, e.kch, e.snap, beta_rad, G, W, e.coef, status,
                 blockIdx.x * blockDim.x + threadIdx.x);
}

}  // namespace

cudaError_t launch_prep(toi_plan_s* p, Slot& s, const double* uvw, const double* freq,
                        const float* weight, const uint8_t* flag, int nbl, int nch) {
  const int tok = prof_begin(p, PROF_PREP, 4);
  const int nkblk = (nch + 255) / 256;
  const int nbblk = (nbl + kMomWarps - 1) / kMomWarps;
  prep_channels_kernel<<<nkblk, 256, 0, p->stream>>>(freq, nch, p->kch, p->kf, p->kch_sum,
                                                     p->d_status);
  prep_baselines_kernel<<<nbblk, kMomWarps * 32, 0, p->stream>>>(
      flag, weight, p->kch, p->kch_sum, nkblk, uvw, nbl, nch, p->cfg.n_pol, p->bpart);
  prep_finalize_kernel<<<1, 352, 0, p->stream>>>(p->bpart, nbblk, p->kch, nch, s.snap,
                                                 p->d_status, p->beta_rad);
  prep_coef_kernel<<<(nbl + 127) / 128, 128, 0, p->stream>>>(uvw, nbl, nch, p->kch, s.snap,
                                                             p->beta_rad, p->G, p->W, s.coef,
                                                             p->d_status);
  prof_end(p, tok);
  return cudaGetLastError();
}

cudaError_t launch_prep_batch(toi_plan_s* p) {
  const int B = p->batch_max;
  const int maxch = p->cfg.max_channels, maxbl = p->cfg.max_baselines;
  const int tok = prof_begin(p, PROF_PREP, 4);
  prep_channels_batch<<<dim3((maxch + 255) / 256, B), 256, 0, p->stream>>>(
      p->bentry_dev, p->bheader_dev, p->d_status);
  prep_baselines_batch<<<dim3((maxbl + kMomWarps - 1) / kMomWarps, B), kMomWarps * 32, 0,
                         p->stream>>>(p->bentry_dev, p->bheader_dev, p->cfg.n_pol);
  prep_finalize_batch<<<dim3(1, B), 352, 0, p->stream>>>(p->bentry_dev, p->bheader_dev,
                                                         p->d_status, p->beta_rad);
  prep_coef_batch<<<dim3((maxbl + 127) / 128, B), 128, 0, p->stream>>>(
      p->bentry_dev, p->bheader_dev, p->beta_rad, p->G, p->W, p->d_status);
  prof_end(p, tok);
  return cudaGetLastError();
}

}  // namespace toi
