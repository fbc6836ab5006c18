// S8: candidate search on the tLISI cube (Section 2: Fourier transform along
// time, harmonic summing, significance map, 5 sigma, connected tiles to
// bounding boxes; Section 6.3: sum of (1 - tLISI), 4 sigma).
//
// Every floating-point step is binary64 with an explicit rounding intrinsic
// (__dadd_rn, __dmul_rn, __ddiv_rn, __dsqrt_rn), so nothing is contracted into
// a fused multiply-add and the evaluation order below is the whole
// specification of the result:
//   twiddles   cos, sin of 2 pi m / S: quadrant q = floor(4m / S),
//              a = 4m - qS, r = (pi/2 * a) / S, 13-term Taylor series in r^2
//              by Horner from the highest term, then the quadrant's swap/sign;
//   mean       sequential sum over t of (double) tLISI, divided by S;
//   P_f        A = sum_t x_t cos_{ft mod S}, B = sum_t x_t sin_{ft mod S}
//              (sequential in t, x_t = tLISI_t - mean), P_f = A*A + B*B;
//   score      max over f = 1..S/2, h in {1,2,4,8} of
//              (sum_{i=1..h, i f <= S/2} P_{i f}) / sqrt(h)   (periodic)
//              or sequential sum over t of (1 - tLISI_t)       (non-periodic);
//   threshold  pairwise-tree sums (split at lo + n/2) for the mean and the
//              population variance over tiles; thr = mean + k * sqrt(var).
#include <limits.h>

#include "toi_internal.cuh"

namespace toi {
namespace {

constexpr int kTaylorTerms = 13;
constexpr double kPi2 = 1.5707963267948966;   // binary64 nearest pi/2

__global__ void twiddle_kernel(int S, double* __restrict__ ct, double* __restrict__ st) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= S) return;
  double fact[2 * kTaylorTerms + 2];
  fact[0] = 1.0;
  for (int n = 1; n < 2 * kTaylorTerms + 2; ++n) fact[n] = __dmul_rn(fact[n - 1], (double)n);
  const long long m4 = 4LL * m;
  const int q = (int)(m4 / S);
  const long long a = m4 - (long long)q * S;
  const double r = __ddiv_rn(__dmul_rn(kPi2, (double)a), (double)S);
  const double r2 = __dmul_rn(r, r);
  const int K = kTaylorTerms - 1;
  double c = __ddiv_rn((K % 2 == 0) ? 1.0 : -1.0, fact[2 * K]);
  double s = __ddiv_rn((K % 2 == 0) ? 1.0 : -1.0, fact[2 * K + 1]);
  for (int k = K - 1; k >= 0; --k) {
    const double sg = (k % 2 == 0) ? 1.0 : -1.0;
    c = __dadd_rn(__dmul_rn(c, r2), __ddiv_rn(sg, fact[2 * k]));
    s = __dadd_rn(__dmul_rn(s, r2), __ddiv_rn(sg, fact[2 * k + 1]));
  }
  s = __dmul_rn(s, r);
  double cc, ss;
  if (q == 0) { cc = c; ss = s; }
  else if (q == 1) { cc = -s; ss = c; }
  else if (q == 2) { cc = -c; ss = -s; }
  else { cc = s; ss = -c; }
  ct[m] = cc;
  st[m] = ss;
}

__global__ void mean_kernel(const float* __restrict__ cube, int S, int nt, int mode,
                            double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nt) return;
  double acc = 0.0;
  if (mode == TOI_CAND_NONPERIODIC) {
    for (int t = 0; t < S; ++t) acc = __dadd_rn(acc, __dsub_rn(1.0, (double)cube[(size_t)t * nt + k]));
    out[k] = acc;
  } else {
    for (int t = 0; t < S; ++t) acc = __dadd_rn(acc, (double)cube[(size_t)t * nt + k]);
    out[k] = __ddiv_rn(acc, (double)S);
  }
}

// The series of every tile, mean removed (x_t = tLISI_t - mean), folded once
// for the transform (reading c10): slot 0 holds x_0, slots 1..Th the sums
// u_t = x_t + x_{S-t}, slots Th+1..2Th the differences v_t = x_t - x_{S-t}
// (Th = floor((S-1)/2)), and for an even S slot S-1 the middle x_{S/2}.
__device__ __forceinline__ double folded(const float* __restrict__ cube, int S, int nt, int k,
                                         double m, int slot) {
  const int Th = (S - 1) / 2;
  auto xt = [&](int t) { return __dsub_rn((double)cube[(size_t)t * nt + k], m); };
  if (slot == 0) return xt(0);
  if (slot <= Th) return __dadd_rn(xt(slot), xt(S - slot));
  if (slot <= 2 * Th) return __dsub_rn(xt(slot - Th), xt(S - slot + Th));
  return xt(S / 2);
}

__global__ void centre_kernel(const float* __restrict__ cube, int S, int nt,
                              const double* __restrict__ mu, double* __restrict__ x) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)S * nt) return;
  const int k = (int)(id % nt);
  x[id] = folded(cube, S, nt, k, mu[k], (int)(id / nt));
}

// Odd S (an even S runs power_pairs_kernel below).  One thread per
// (frequency pair, tile): the powers P_f and P_{f+H} (H = ceil(F/2)) of the
// mean-removed series, so that each folded value feeds four independent
// sums.  The series is real, so times t and S - t share
// their cosine and have opposite sines: A_f = x_0 cos 0 + sum_t u_t cos(2 pi
// f t / S) [+ x_{S/2} cos(pi f)], B_f = sum_t v_t sin(2 pi f t / S) [+
// x_{S/2} sin(pi f)], t = 1..Th in order, half the products of the plain
// sum over t = 0..S-1.  xs is the folded series from centre_kernel, or NULL
// to fold here (bit-identical: the same operations).
__global__ void power_kernel(const float* __restrict__ cube, const double* __restrict__ xs,
                             int S, int nt, int F, const double* __restrict__ mu,
                             const double* __restrict__ ct, const double* __restrict__ st,
                             double* __restrict__ P) {
  const int H = (F + 1) / 2;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)H * nt) return;
  const int k = (int)(id % nt);
  const int f1 = (int)(id / nt) + 1, f2 = f1 + H;
  const bool two = f2 <= F;
  const double m = mu[k];
  const int Th = (S - 1) / 2;
  auto x = [&](int slot) {
    return xs ? xs[(size_t)slot * nt + k] : folded(cube, S, nt, k, m, slot);
  };
  const double x0 = x(0);
  double A1 = __dmul_rn(x0, ct[0]), B1 = 0.0;
  double A2 = two ? __dmul_rn(x0, ct[0]) : 0.0, B2 = 0.0;
  int i1 = 0, i2 = 0;   // (f * t) mod S, advanced incrementally
  for (int t = 1; t <= Th; ++t) {
    i1 += f1;
    if (i1 >= S) i1 -= S;
    i2 += two ? f2 : 0;
    if (i2 >= S) i2 -= S;
    const double u = x(t), v = x(Th + t);
    A1 = __dadd_rn(A1, __dmul_rn(u, ct[i1]));
    B1 = __dadd_rn(B1, __dmul_rn(v, st[i1]));
    if (two) {
      A2 = __dadd_rn(A2, __dmul_rn(u, ct[i2]));
      B2 = __dadd_rn(B2, __dmul_rn(v, st[i2]));
    }
  }
  if ((S & 1) == 0) {
    const double xm = x(S - 1);
    const int m1 = (f1 & 1) ? S / 2 : 0, m2 = (f2 & 1) ? S / 2 : 0;   // (f S/2) mod S
    A1 = __dadd_rn(A1, __dmul_rn(xm, ct[m1]));
    B1 = __dadd_rn(B1, __dmul_rn(xm, st[m1]));
    if (two) {
      A2 = __dadd_rn(A2, __dmul_rn(xm, ct[m2]));
      B2 = __dadd_rn(B2, __dmul_rn(xm, st[m2]));
    }
  }
  P[(size_t)f1 * nt + k] = __dadd_rn(__dmul_rn(A1, A1), __dmul_rn(B1, B1));
  if (two) P[(size_t)f2 * nt + k] = __dadd_rn(__dmul_rn(A2, A2), __dmul_rn(B2, B2));
}

// Even S: frequencies f and g = S/2 - f share their twiddles (2 pi g t / S
// = pi t - 2 pi f t / S: cos(...g...) = (-1)^t cos(...f...), sin(...g...) =
// -(-1)^t sin(...f...)), so one thread sums the even and odd times of the
// folded series apart and forms both transforms from them:
//   A_f = (x_0 cos 0 + Ae) + Ao,  A_g = (x_0 cos 0 + Ae) - Ao,
//   B_f = Be + Bo,               B_g = Bo - Be,
// then each adds its own middle time S/2.  Thread groups 0..NP-1 are the
// pairs f = 1..NP (NP = floor((S/2 - 1) / 2)); the rest are the frequencies
// without a partner, S/4 (when S/2 is even) and S/2, summed as in
// power_kernel.  Half the products of power_kernel again.
__global__ void power_pairs_kernel(const float* __restrict__ cube,
                                   const double* __restrict__ xs, int S, int nt,
                                   const double* __restrict__ mu,
                                   const double* __restrict__ ct,
                                   const double* __restrict__ st, double* __restrict__ P) {
  const int half = S / 2, Th = half - 1;
  const int NP = (half - 1) / 2;
  const int NS = (half % 2 == 0) ? 2 : 1;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)(NP + NS) * nt) return;
  const int k = (int)(id % nt);
  const int grp = (int)(id / nt);
  const double m = mu[k];
  auto x = [&](int slot) {
    return xs ? xs[(size_t)slot * nt + k] : folded(cube, S, nt, k, m, slot);
  };
  const double x0c = __dmul_rn(x(0), ct[0]);
  const double xm = x(S - 1);
  if (grp < NP) {
    const int f = grp + 1, g = half - f;
    double Ae = 0.0, Ao = 0.0, Be = 0.0, Bo = 0.0;
    int i = 0;   // (f * t) mod S
    for (int t = 1; t <= Th; ++t) {
      i += f;
      if (i >= S) i -= S;
      const double u = x(t), v = x(Th + t);
      if (t & 1) {
        Ao = __dadd_rn(Ao, __dmul_rn(u, ct[i]));
        Bo = __dadd_rn(Bo, __dmul_rn(v, st[i]));
      } else {
        Ae = __dadd_rn(Ae, __dmul_rn(u, ct[i]));
        Be = __dadd_rn(Be, __dmul_rn(v, st[i]));
      }
    }
    const double base = __dadd_rn(x0c, Ae);
    double Af = __dadd_rn(base, Ao), Ag = __dsub_rn(base, Ao);
    double Bf = __dadd_rn(Be, Bo), Bg = __dsub_rn(Bo, Be);
    const int mf = (f & 1) ? half : 0, mg = (g & 1) ? half : 0;   // (f S/2) mod S
    Af = __dadd_rn(Af, __dmul_rn(xm, ct[mf]));
    Bf = __dadd_rn(Bf, __dmul_rn(xm, st[mf]));
    Ag = __dadd_rn(Ag, __dmul_rn(xm, ct[mg]));
    Bg = __dadd_rn(Bg, __dmul_rn(xm, st[mg]));
    P[(size_t)f * nt + k] = __dadd_rn(__dmul_rn(Af, Af), __dmul_rn(Bf, Bf));
    P[(size_t)g * nt + k] = __dadd_rn(__dmul_rn(Ag, Ag), __dmul_rn(Bg, Bg));
  } else {
    const int f = (grp == NP && NS == 2) ? half / 2 : half;
    double A = x0c, B = 0.0;
    int i = 0;
    for (int t = 1; t <= Th; ++t) {
      i += f;
      if (i >= S) i -= S;
      A = __dadd_rn(A, __dmul_rn(x(t), ct[i]));
      B = __dadd_rn(B, __dmul_rn(x(Th + t), st[i]));
    }
    const int mf = (f & 1) ? half : 0;
    A = __dadd_rn(A, __dmul_rn(xm, ct[mf]));
    B = __dadd_rn(B, __dmul_rn(xm, st[mf]));
    P[(size_t)f * nt + k] = __dadd_rn(__dmul_rn(A, A), __dmul_rn(B, B));
  }
}

__global__ void harmonic_kernel(const double* __restrict__ P, int nt, int F,
                                double* __restrict__ score) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nt) return;
  const int hs[4] = {1, 2, 4, 8};
  double roots[4];
  for (int i = 0; i < 4; ++i) roots[i] = __dsqrt_rn((double)hs[i]);
  double best = 0.0;
  for (int f = 1; f <= F; ++f) {
    for (int hi = 0; hi < 4; ++hi) {
      double H = 0.0;
      for (int i = 1; i <= hs[hi]; ++i) {
        if (i * f > F) break;
        H = __dadd_rn(H, P[(size_t)(i * f) * nt + k]);
      }
      // H / sqrt(h): exact for h = 1 (H itself) and h = 4 (H times 0.5, the
      // same correctly rounded value as the division), divided otherwise
      const double q = hi == 0 ? H : (hi == 2 ? __dmul_rn(H, 0.5) : __ddiv_rn(H, roots[hi]));
      best = fmax(best, q);
    }
  }
  score[k] = best;
}

__device__ double pairwise_sum(const double* a, int lo, int hi) {
  const int n = hi - lo;
  if (n <= 0) return 0.0;
  if (n == 1) return a[lo];
  const int mid = lo + n / 2;
  return __dadd_rn(pairwise_sum(a, lo, mid), pairwise_sum(a, mid, hi));
}

// The pairwise tree of pairwise_sum(a, 0, n), evaluated by a whole block.
// Cut the tree at the depth D with 2^D <= min(n, blockDim.x): while 2^D <= n
// every node above that depth has at least two elements and splits in two, so
// the top of the tree is a perfect binary tree over the 2^D depth-D subtrees.
// Thread j sums subtree j (its interval follows from the bits of j, high bit
// first: 0 takes the left half [lo, lo + m/2), 1 the right), then the 2^D
// partial sums are combined level by level (node i adds children 2i, 2i + 1).
// Additions and their order are exactly those of the recursion.  `sh` holds
// blockDim.x doubles; every thread of the block must call this.
__device__ double block_pairwise_sum(const double* a, int n, double* sh) {
  int D = 0;
  while ((2 << D) <= n && (2 << D) <= (int)blockDim.x) ++D;
  const int L = 1 << D;
  for (int j = threadIdx.x; j < L; j += blockDim.x) {
    int lo = 0, m = n;
    for (int b = D - 1; b >= 0; --b) {
      const int h = m / 2;
      if ((j >> b) & 1) { lo += h; m -= h; } else { m = h; }
    }
    sh[j] = pairwise_sum(a, lo, lo + m);
  }
  __syncthreads();
  for (int half = L >> 1; half >= 1; half >>= 1) {
    for (int i = threadIdx.x; i < half; i += blockDim.x) sh[i] = __dadd_rn(sh[2 * i], sh[2 * i + 1]);
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// One block: threshold, candidate mask, 8-connected labelling (label = first
// tile of the component in raster order), boxes sorted by (y0, x0, label).
__global__ void __launch_bounds__(1024)
label_kernel(const double* __restrict__ score, int nty, int ntx, int T, double ksig,
             double* __restrict__ work, int* __restrict__ lab, int* __restrict__ bb,
             double* __restrict__ thr_out, int* __restrict__ nbox_out, int* __restrict__ boxes,
             int max_boxes) {
  const int nt = nty * ntx;
  __shared__ double s_thr;
  __shared__ int s_nroot;
  __shared__ double s_sum[1024];
  const double mu = __ddiv_rn(block_pairwise_sum(score, nt, s_sum), (double)nt);
  for (int k = threadIdx.x; k < nt; k += blockDim.x) {
    const double d = __dsub_rn(score[k], mu);
    work[k] = __dmul_rn(d, d);
  }
  __syncthreads();
  const double var = __ddiv_rn(block_pairwise_sum(work, nt, s_sum), (double)nt);
  if (threadIdx.x == 0) {
    s_thr = __dadd_rn(mu, __dmul_rn(ksig, __dsqrt_rn(var)));
    *thr_out = s_thr;
    s_nroot = 0;
  }
  __syncthreads();
  const double thr = s_thr;
  for (int k = threadIdx.x; k < nt; k += blockDim.x) {
    lab[k] = score[k] > thr ? k : INT_MAX;
    bb[4 * k + 0] = INT_MAX; bb[4 * k + 1] = INT_MAX;
    bb[4 * k + 2] = -1; bb[4 * k + 3] = -1;
  }
  __syncthreads();
  for (int iter = 0; iter < nt + 1; ++iter) {
    int changed = 0;
    for (int k = threadIdx.x; k < nt; k += blockDim.x) {
      const int l = lab[k];
      if (l == INT_MAX) continue;
      const int y = k / ntx, x = k % ntx;
      int m = l;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int yy = y + dy, xx = x + dx;
          if (yy < 0 || yy >= nty || xx < 0 || xx >= ntx) continue;
          const int ln = lab[yy * ntx + xx];
          if (ln < m) m = ln;
        }
      if (m < l) { atomicMin(&lab[k], m); changed = 1; }
    }
    if (!__syncthreads_or(changed)) break;
  }
  for (int k = threadIdx.x; k < nt; k += blockDim.x) {
    const int l = lab[k];
    if (l == INT_MAX) continue;
    const int y = k / ntx, x = k % ntx;
    atomicMin(&bb[4 * l + 0], x);
    atomicMin(&bb[4 * l + 1], y);
    atomicMax(&bb[4 * l + 2], x);
    atomicMax(&bb[4 * l + 3], y);
    if (l == k) atomicAdd(&s_nroot, 1);
  }
  __syncthreads();
  // rank of each root by (y0, x0, label)
  for (int k = threadIdx.x; k < nt; k += blockDim.x) {
    if (lab[k] != k) continue;
    const int x0 = bb[4 * k], y0 = bb[4 * k + 1];
    int rank = 0;
    for (int j = 0; j < nt; ++j) {
      if (lab[j] != j || j == k) continue;
      const int xj = bb[4 * j], yj = bb[4 * j + 1];
      if (yj < y0 || (yj == y0 && (xj < x0 || (xj == x0 && j < k)))) ++rank;
    }
    if (rank < max_boxes) {
      boxes[4 * rank + 0] = x0 * T;
      boxes[4 * rank + 1] = y0 * T;
      boxes[4 * rank + 2] = (bb[4 * k + 2] + 1) * T;
      boxes[4 * rank + 3] = (bb[4 * k + 3] + 1) * T;
    }
  }
  if (threadIdx.x == 0) *nbox_out = s_nroot;
}

}  // namespace

// Scratch layout (bytes) for S slices of an nt-tile cube.
size_t candidates_scratch_bytes(int S, int nt) {
  const int F = S / 2;
  size_t b = 0;
  b += sizeof(double) * (size_t)S * 2;          // twiddles
  b += sizeof(double) * (size_t)nt;             // mean / score
  b += sizeof(double) * (size_t)(F + 1) * nt;   // P
  b += sizeof(double) * (size_t)nt;             // work
  b += sizeof(double) * 2;                      // threshold + pad
  b += sizeof(int) * (size_t)nt * 5;            // labels + boxes by root
  b += sizeof(int) * 4;                         // count
  return b + 256;
}

// Bytes of the optional folded-series buffer (periodic mode): with it the
// series is centred and folded once instead of once per frequency.
size_t candidates_centre_bytes(int S, int nt) { return sizeof(double) * (size_t)S * nt; }

cudaError_t candidates_run(const float* cube, int S, int nty, int ntx, int T, int mode,
                           cudaStream_t st, void* scratch, double* scores_out, int max_boxes,
                           int* boxes_dev, double** thr_dev, int** nbox_dev, double* xbuf) {
  const int nt = nty * ntx;
  const int F = S / 2;
  char* p = reinterpret_cast<char*>(scratch);
  auto take = [&](size_t bytes) {
    void* r = p;
    p += (bytes + 15) & ~(size_t)15;
    return r;
  };
  double* ct = (double*)take(sizeof(double) * S);
  double* stw = (double*)take(sizeof(double) * S);
  double* mean = (double*)take(sizeof(double) * nt);
  double* P = (double*)take(sizeof(double) * (size_t)(F + 1) * nt);
  double* work = (double*)take(sizeof(double) * nt);
  double* thr = (double*)take(sizeof(double) * 2);
  int* lab = (int*)take(sizeof(int) * nt);
  int* bb = (int*)take(sizeof(int) * 4 * nt);
  int* nbox = (int*)take(sizeof(int) * 4);
  double* score = scores_out ? scores_out : mean;
  mean_kernel<<<(nt + 255) / 256, 256, 0, st>>>(cube, S, nt, mode, mode == TOI_CAND_NONPERIODIC ? score : mean);
  if (mode == TOI_CAND_PERIODIC) {
    if (F > 0) {
      twiddle_kernel<<<(S + 255) / 256, 256, 0, st>>>(S, ct, stw);
      if (xbuf) {
        const long long nx = (long long)S * nt;
        centre_kernel<<<(unsigned)((nx + 255) / 256), 256, 0, st>>>(cube, S, nt, mean, xbuf);
      }
      if (S % 2 == 0) {
        const int half = S / 2;
        const long long n = (long long)((half - 1) / 2 + (half % 2 == 0 ? 2 : 1)) * nt;
        power_pairs_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cube, xbuf, S, nt, mean,
                                                                        ct, stw, P);
      } else {
        const long long n = (long long)((F + 1) / 2) * nt;
        power_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cube, xbuf, S, nt, F, mean, ct,
                                                                  stw, P);
      }
      harmonic_kernel<<<(nt + 255) / 256, 256, 0, st>>>(P, nt, F, score);
    } else {
      cudaMemsetAsync(score, 0, sizeof(double) * nt, st);
    }
  }
  const double k = mode == TOI_CAND_PERIODIC ? 5.0 : 4.0;
  label_kernel<<<1, 1024, 0, st>>>(score, nty, ntx, T, k, work, lab, bb, thr, nbox, boxes_dev,
                                   max_boxes);
  *thr_dev = thr;
  *nbox_dev = nbox;
  return cudaGetLastError();
}

}  // namespace toi
