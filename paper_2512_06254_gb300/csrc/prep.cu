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

#include "toi_internal.cuh"

namespace toi {
namespace {

constexpr int kPrepThreads = 128;

__device__ __forceinline__ void parallel_hands(int npol, int& pa, int& pb) {
  if (npol == 4) { pa = 0; pb = 3; }
  else if (npol == 2) { pa = 0; pb = 1; }
  else { pa = 0; pb = 0; }
}

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
__global__ void prep_channels_kernel(const double* __restrict__ freq, int nch,
                                     double* __restrict__ kch, float2* __restrict__ kf,
                                     double* __restrict__ kpart, int* status) {
  __shared__ double sh[2 * 256];
  const int c = blockIdx.x * 256 + threadIdx.x;
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
    kpart[2 * blockIdx.x] = v[0];
    kpart[2 * blockIdx.x + 1] = v[1];
  }
}

// Per-baseline: deselected channels (both parallel hands flagged or zero
// weight) and the sum of weights.
__global__ void prep_baselines_kernel(const uint8_t* __restrict__ flag,
                                      const float* __restrict__ weight,
                                      const double* __restrict__ kch, int nch, int npol,
                                      BaselineMoments* __restrict__ mom) {
  __shared__ double sh[4 * kPrepThreads];
  const int bl = blockIdx.x;
  int pa, pb;
  parallel_hands(npol, pa, pb);
  const size_t base = (size_t)bl * nch * npol;
  double sk = 0.0, sk2 = 0.0, sw = 0.0;
  long long nd = 0, cnt = 0;
  for (int c = threadIdx.x; c < nch; c += kPrepThreads) {
    const size_t o = base + (size_t)c * npol;
    const bool fa = flag ? flag[o + pa] != 0 : false;
    const bool fb = flag ? flag[o + pb] != 0 : false;
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
        sw = __dadd_rn(sw, (pa == pb) ? (double)wa : __dadd_rn((double)wa, (double)wb));
      } else {
        cnt += (pa == pb) ? 1 : (int)(!fa) + (int)(!fb);
      }
    } else {
      const double k = kch[c];
      sk = __dadd_rn(sk, k);
      sk2 = __dadd_rn(sk2, __dmul_rn(k, k));
      nd += 1;
    }
  }
  double v[4] = {sk, sk2, sw, (double)nd};
  // counts are exact in float64 below 2^53
  v[2] = weight ? v[2] : (double)cnt;
  block_reduce<kPrepThreads, 4>(v, sh);
  if (threadIdx.x == 0) {
    mom[bl].sk_desel = v[0];
    mom[bl].sk2_desel = v[1];
    mom[bl].sumw = v[2];
    mom[bl].ndesel = (long long)v[3];
  }
}

// Eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi rotations
// (float64).  On return a holds the eigenvalues on its diagonal and the
// columns of e the eigenvectors.
__device__ void jacobi3(double a[3][3], double e[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) e[i][j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    const double off = fabs(a[0][1]) + fabs(a[0][2]) + fabs(a[1][2]);
    const double dia = fabs(a[0][0]) + fabs(a[1][1]) + fabs(a[2][2]);
    if (off == 0.0 || off <= 1e-300 + 1e-18 * dia) break;
    for (int p = 0; p < 2; ++p) {
      for (int q = p + 1; q < 3; ++q) {
        const double apq = a[p][q];
        if (apq == 0.0) continue;
        const double theta = (a[q][q] - a[p][p]) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0);
        const double s = t * c;
        for (int k = 0; k < 3; ++k) {   // A <- A J (columns p, q)
          const double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - s * akq;
          a[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {   // A <- J^T A (rows p, q)
          const double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - s * aqk;
          a[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {   // E <- E J
          const double ekp = e[k][p], ekq = e[k][q];
          e[k][p] = c * ekp - s * ekq;
          e[k][q] = s * ekp + c * ekq;
        }
      }
    }
  }
}

__global__ void prep_finalize_kernel(const double* __restrict__ uvw, int nbl, int nch,
                                     const double* __restrict__ kpart, int nkblk,
                                     const BaselineMoments* __restrict__ mom,
                                     double* __restrict__ snap, int* status) {
  constexpr int NT = 256;
  __shared__ double sh[11 * NT];
  __shared__ double ks[2];
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nkblk; ++i) {
      a = __dadd_rn(a, kpart[2 * i]);
      b = __dadd_rn(b, kpart[2 * i + 1]);
    }
    ks[0] = a;
    ks[1] = b;
  }
  __syncthreads();
  const double skall = ks[0], sk2all = ks[1];
  double v[11];
  for (int i = 0; i < 11; ++i) v[i] = 0.0;
  for (int b = threadIdx.x; b < nbl; b += NT) {
    const BaselineMoments m = mom[b];
    const double n = (double)(nch - m.ndesel);
    const double s1 = skall - m.sk_desel;
    const double s2 = sk2all - m.sk2_desel;
    const double x = uvw[3 * b], y = uvw[3 * b + 1], z = uvw[3 * b + 2];
    v[0] += n;
    v[1] += x * s1; v[2] += y * s1; v[3] += z * s1;
    v[4] += x * x * s2; v[5] += x * y * s2; v[6] += x * z * s2;
    v[7] += y * y * s2; v[8] += y * z * s2; v[9] += z * z * s2;
    v[10] += m.sumw;
  }
  block_reduce<NT, 11>(v, sh);
  if (threadIdx.x == 0) {
    const double N = v[0];
    const int empty = (N <= 0.0 || v[10] <= 0.0) ? 1 : 0;
    double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    if (!empty) {
      const double m1[3] = {v[1], v[2], v[3]};
      double C[3][3];
      C[0][0] = v[4] - m1[0] * m1[0] / N;
      C[0][1] = v[5] - m1[0] * m1[1] / N;
      C[0][2] = v[6] - m1[0] * m1[2] / N;
      C[1][1] = v[7] - m1[1] * m1[1] / N;
      C[1][2] = v[8] - m1[1] * m1[2] / N;
      C[2][2] = v[9] - m1[2] * m1[2] / N;
      C[1][0] = C[0][1]; C[2][0] = C[0][2]; C[2][1] = C[1][2];
      double E[3][3];
      jacobi3(C, E);
      int imin = 0, imax = 0;
      for (int i = 1; i < 3; ++i) {
        if (C[i][i] < C[imin][imin]) imin = i;
        if (C[i][i] > C[imax][imax]) imax = i;
      }
      const int imid = (imin == imax) ? (imin + 1) % 3 : 3 - imin - imax;
      // rank <= 1 (second singular value <= 1e-6 of the first): no plane, V = I
      const double lmax = fmax(C[imax][imax], 0.0), lmid = fmax(C[imid][imid], 0.0);
      const bool degenerate = !(sqrt(lmid) > 1e-6 * sqrt(lmax));
      double v3[3] = {E[0][imin], E[1][imin], E[2][imin]};
      double nn = sqrt(v3[0] * v3[0] + v3[1] * v3[1] + v3[2] * v3[2]);
      for (int i = 0; i < 3; ++i) v3[i] /= nn;
      if (v3[2] < 0.0)
        for (int i = 0; i < 3; ++i) v3[i] = -v3[i];
      double e[3] = {1.0, 0.0, 0.0};
      if (fabs(v3[0]) > 0.999) { e[0] = 0.0; e[1] = 1.0; }
      const double d = e[0] * v3[0] + e[1] * v3[1] + e[2] * v3[2];
      double v1[3] = {e[0] - d * v3[0], e[1] - d * v3[1], e[2] - d * v3[2]};
      nn = sqrt(v1[0] * v1[0] + v1[1] * v1[1] + v1[2] * v1[2]);
      for (int i = 0; i < 3; ++i) v1[i] /= nn;
      const double v2[3] = {v3[1] * v1[2] - v3[2] * v1[1], v3[2] * v1[0] - v3[0] * v1[2],
                            v3[0] * v1[1] - v3[1] * v1[0]};
      if (!degenerate)
        for (int i = 0; i < 3; ++i) { V[0][i] = v1[i]; V[1][i] = v2[i]; V[2][i] = v3[i]; }
    } else {
      set_status(status, TOI_DEV_EMPTY);
    }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) snap[SNAP_V + 3 * i + j] = V[i][j];
    snap[SNAP_OMEGA] = fabs(V[0][0] * V[1][1] - V[1][0] * V[0][1]);
    snap[SNAP_XI] = V[2][0] / V[2][2];
    snap[SNAP_ETA] = V[2][1] / V[2][2];
    snap[SNAP_SUMW] = empty ? 0.0 : v[10];
    snap[SNAP_NVIS] = empty ? 0.0 : v[0];
    snap[14] = 0.0;
    snap[15] = 0.0;
  }
}

// Per baseline: R = V uvw (float64), grid coefficients a1 = -r1 beta G,
// a2 = r2 beta G, and the check that every footprint stays on the grid.
__global__ void prep_coef_kernel(const double* __restrict__ uvw, int nbl, int nch,
                                 const double* __restrict__ kch, const double* __restrict__ snap,
                                 double beta_rad, int G, int W, BaselineCoef* __restrict__ coef,
                                 int* status) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
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
}

}  // namespace

cudaError_t launch_prep(toi_plan_s* p, Slot& s, const double* uvw, const double* freq,
                        const float* weight, const uint8_t* flag, int nbl, int nch) {
  const int tok = prof_begin(p, PROF_PREP, 4);
  const int nkblk = (nch + 255) / 256;
  prep_channels_kernel<<<nkblk, 256, 0, p->stream>>>(freq, nch, p->kch, p->kf, p->kch_sum,
                                                     p->d_status);
  prep_baselines_kernel<<<nbl, kPrepThreads, 0, p->stream>>>(flag, weight, p->kch, nch,
                                                             p->cfg.n_pol, p->mom);
  prep_finalize_kernel<<<1, 256, 0, p->stream>>>(uvw, nbl, nch, p->kch_sum, nkblk, p->mom, s.snap,
                                                 p->d_status);
  prep_coef_kernel<<<(nbl + 127) / 128, 128, 0, p->stream>>>(uvw, nbl, nch, p->kch, s.snap,
                                                             p->beta_rad, p->G, p->W, s.coef,
                                                             p->d_status);
  prof_end(p, tok);
  return cudaGetLastError();
}

}  // namespace toi
