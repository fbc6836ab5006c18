// S4-S5: centred inverse 2-D FFT of the Hermitian half-plane grid, output
// pruned to the central N x N, Re, grid correction and normalisation
// (Section 4.1 stage 4; Section 3.2 with Eq. 11).
//
// With k' = k - G/2 and j' = j - N/2 the image is
//   I[j2', j1'] = 1/2 sum_{k2'} sum_{k1'} H[k2', k1'] e^{2 pi i (k1' j1' + k2' j2') / G}
// where H holds rows k2' >= 0 and rows k2' < 0 are conj(H[-k']) (the grid is
// stored as H = G + conj(G(-k)), hence the 1/2).
//   Pass 1 (rows, along k1'): T[k2', j1'] = sum_{k1'} H[k2', k1'] e^{..}; only
//            the N central j1' are written, as (-1)^j1' Z[j1' mod G] of the
//            plain inverse DFT Z of the row.
//   Pass 2 (columns, along k2'): the column sequence is Hermitian in k2', so
//            the full length-G sequence is rebuilt in shared memory from the
//            stored half, transformed, and 1/2 Re of the N central outputs is
//            multiplied by 1/psi_hat(j1') 1/psi_hat(j2') / (omega sum w).
// Each transform is a Stockham autosort FFT in shared memory: radix-8 passes
// (then one radix-4 or radix-2 pass) whose butterflies run in registers, with
// float32 twiddles e^{+2 pi i m / G} tabulated in float64 at plan time.
#include "toi_internal.cuh"

namespace toi {
namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiply by +i
__device__ __forceinline__ float2 cmuli(float2 a) { return make_float2(-a.y, a.x); }

// In-register inverse DFTs V[k] = sum_j v[j] e^{+2 pi i j k / R}.
__device__ __forceinline__ void dft2(float2* v) {
  const float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

__device__ __forceinline__ void dft4(float2* v) {
  const float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
  const float2 b0 = cadd(v[1], v[3]), b1 = cmuli(csub(v[1], v[3]));
  v[0] = cadd(a0, b0);
  v[2] = csub(a0, b0);
  v[1] = cadd(a1, b1);
  v[3] = csub(a1, b1);
}

__device__ __forceinline__ void dft8(float2* v) {
  const float r = 0.70710678118654752f;
  // decimation in frequency: first stage span 4 with twiddles e^{+2 pi i j/8}
  float2 t[8];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    t[j] = cadd(v[j], v[j + 4]);
    t[j + 4] = csub(v[j], v[j + 4]);
  }
  t[5] = make_float2(r * (t[5].x - t[5].y), r * (t[5].x + t[5].y));    // * (1+i)/sqrt2
  t[6] = cmuli(t[6]);                                                  // * i
  t[7] = make_float2(-r * (t[7].x + t[7].y), r * (t[7].x - t[7].y));   // * (-1+i)/sqrt2
  // two 4-point transforms on the halves; results in bit-reversed order
  float2 a[4] = {t[0], t[1], t[2], t[3]};
  float2 b[4] = {t[4], t[5], t[6], t[7]};
  dft4(a);
  dft4(b);
  v[0] = a[0]; v[2] = a[1]; v[4] = a[2]; v[6] = a[3];
  v[1] = b[0]; v[3] = b[1]; v[5] = b[2]; v[7] = b[3];
}

template <int R>
__device__ __forceinline__ void dftR(float2* v) {
  if (R == 8) dft8(v);
  else if (R == 4) dft4(v);
  else dft2(v);
}

// One Stockham pass of radix R over `nseq` sequences of length G in shared
// memory (in place: all loads, barrier, all stores, barrier).  BPT =
// butterflies per thread = nseq * G / R / blockDim.x.
template <int G, int R, int BPT>
__device__ __forceinline__ void stockham_pass(float2* x, int nseq, int Ns, const float2* __restrict__ tw) {
  constexpr int NB = G / R;   // butterflies per sequence
  float2 v[BPT][R];
  int jj[BPT], ss[BPT];
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    const int id = threadIdx.x + b * blockDim.x;
    const int seq = id / NB, j = id - seq * NB;
    jj[b] = j;
    ss[b] = seq;
    if (seq < nseq) {
      const float2* xs = x + (size_t)seq * G;
      const int k = j & (Ns - 1);
      const int step = (G / (Ns * R)) * k;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float2 val = xs[j + r * NB];
        if (r > 0 && k > 0) val = cmul(val, __ldg(tw + step * r));
        v[b][r] = val;
      }
      dftR<R>(v[b]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    if (ss[b] < nseq) {
      float2* xs = x + (size_t)ss[b] * G;
      const int j = jj[b];
      const int k = j & (Ns - 1);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) xs[base + r * Ns] = v[b][r];
    }
  }
  __syncthreads();
}

template <int G, int NSEQ, int NT>
__device__ __forceinline__ void fft_smem(float2* x, const float2* __restrict__ tw) {
  constexpr int LOG = (G >= 8192) ? 13 : (G >= 4096) ? 12 : (G >= 2048) ? 11 : (G >= 1024) ? 10
                    : (G >= 512) ? 9 : (G >= 256) ? 8 : 7;
  constexpr int N8 = LOG / 3;
  constexpr int REM = LOG - 3 * N8;
  constexpr int BPT8 = (NSEQ * (G / 8) + NT - 1) / NT;
  int Ns = 1;
#pragma unroll
  for (int p = 0; p < N8; ++p) {
    stockham_pass<G, 8, BPT8>(x, NSEQ, Ns, tw);
    Ns *= 8;
  }
  if (REM == 2) {
    constexpr int BPT4 = (NSEQ * (G / 4) + NT - 1) / NT;
    stockham_pass<G, 4, BPT4>(x, NSEQ, Ns, tw);
  } else if (REM == 1) {
    constexpr int BPT2 = (NSEQ * (G / 2) + NT - 1) / NT;
    stockham_pass<G, 2, BPT2>(x, NSEQ, Ns, tw);
  }
}

template <int G>
struct RowCfg {
  static constexpr int NT = (G / 8 < 64) ? 64 : (G / 8 > 512 ? 512 : G / 8);
};

template <int G>
__global__ void __launch_bounds__(RowCfg<G>::NT)
fft_rows_kernel(const float2* __restrict__ H, int N, const float2* __restrict__ tw,
                float2* __restrict__ T) {
  extern __shared__ float2 x[];
  const int row = blockIdx.x;
  const float2* src = H + (size_t)row * G;
  for (int n = threadIdx.x; n < G; n += blockDim.x) x[n] = src[n];
  __syncthreads();
  fft_smem<G, 1, RowCfg<G>::NT>(x, tw);
  float2* dst = T + (size_t)row * N;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const int jp = j - N / 2;
    float2 v = x[jp < 0 ? jp + G : jp];
    if (jp & 1) { v.x = -v.x; v.y = -v.y; }
    dst[j] = v;
  }
}

template <int G>
struct ColCfg {
  static constexpr int CW = (G >= 8192) ? 2 : 4;
  static constexpr int NT = 512;
};

template <int G>
__global__ void __launch_bounds__(ColCfg<G>::NT)
fft_cols_kernel(const float2* __restrict__ T, int N, const float2* __restrict__ tw,
                const float* __restrict__ corr, const double* __restrict__ snap,
                float* __restrict__ out) {
  constexpr int CW = ColCfg<G>::CW;
  extern __shared__ float2 x[];
  const int col0 = blockIdx.x * CW;
  constexpr int half = G / 2;
  for (int e = threadIdx.x; e < half * CW; e += blockDim.x) {
    const int r = e / CW, c = e - r * CW;
    const float2 v = T[(size_t)r * N + col0 + c];
    float2* xs = x + (size_t)c * G;
    xs[r] = v;
    if (r > 0) xs[G - r] = make_float2(v.x, -v.y);
    else xs[half] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft_smem<G, CW, ColCfg<G>::NT>(x, tw);
  const double omega = snap[SNAP_OMEGA], sumw = snap[SNAP_SUMW];
  const float norm = sumw > 0.0 ? (float)(0.5 / (omega * sumw)) : 0.f;
  for (int e = threadIdx.x; e < N * CW; e += blockDim.x) {
    const int j2 = e / CW, c = e - j2 * CW;
    const int jp = j2 - N / 2;
    const float v = x[(size_t)c * G + (jp < 0 ? jp + G : jp)].x;
    out[(size_t)j2 * N + col0 + c] = v * (norm * corr[col0 + c] * corr[j2]);
  }
}

template <int G>
cudaError_t configure_g() {
  cudaError_t e = cudaFuncSetAttribute(fft_rows_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       G * (int)sizeof(float2));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fft_cols_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              ColCfg<G>::CW * G * (int)sizeof(float2));
}

template <int G>
void launch_g(toi_plan_s* p, Slot& s) {
  const int N = p->N;
  int tok = prof_begin(p, PROF_FFT_ROWS, 1);
  fft_rows_kernel<G><<<G / 2, RowCfg<G>::NT, G * sizeof(float2), p->stream>>>(s.grid, N, p->twiddle,
                                                                             p->fft_tmp);
  prof_end(p, tok);
  tok = prof_begin(p, PROF_FFT_COLS, 1);
  constexpr int CW = ColCfg<G>::CW;
  fft_cols_kernel<G><<<N / CW, ColCfg<G>::NT, CW * G * sizeof(float2), p->stream>>>(
      p->fft_tmp, N, p->twiddle, p->corr, s.snap, p->tilted);
  prof_end(p, tok);
}

}  // namespace

cudaError_t fft_configure() {
  cudaError_t e;
  if ((e = configure_g<128>()) != cudaSuccess) return e;
  if ((e = configure_g<256>()) != cudaSuccess) return e;
  if ((e = configure_g<512>()) != cudaSuccess) return e;
  if ((e = configure_g<1024>()) != cudaSuccess) return e;
  if ((e = configure_g<2048>()) != cudaSuccess) return e;
  if ((e = configure_g<4096>()) != cudaSuccess) return e;
  return configure_g<8192>();
}

cudaError_t launch_fft(toi_plan_s* p, Slot& s) {
  switch (p->G) {
    case 128: launch_g<128>(p, s); break;
    case 256: launch_g<256>(p, s); break;
    case 512: launch_g<512>(p, s); break;
    case 1024: launch_g<1024>(p, s); break;
    case 2048: launch_g<2048>(p, s); break;
    case 4096: launch_g<4096>(p, s); break;
    case 8192: launch_g<8192>(p, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace toi
