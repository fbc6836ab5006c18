// S4-S5: centred inverse 2-D FFT of the Hermitian half-plane grid, output
// pruned to the central N x N, Re, grid correction and normalisation
// (Section 4.1 stage 4; Section 3.2 with Eq. 11).
//
// With k' = k - G/2 and j' = j - N/2 the image is
//   I[j2', j1'] = 1/2 sum_{k2'} sum_{k1'} H[k2', k1'] e^{2 pi i (k1' j1' + k2' j2') / G}
// where H holds rows k2' >= 0 and rows k2' < 0 are conj(H[-k']) (the grid is
// stored as H = G + conj(G(-k)), hence the 1/2).
//   Pass 1 (rows, along k1'): T[k2', j1'] = sum_{k1'} H[k2', k1'] e^{..}, only
//            the N central j1' are written.
//   Pass 2 (columns, along k2'): the column sequence is Hermitian in k2', so
//            the full length-G sequence is rebuilt in shared memory from the
//            stored half, transformed, and 1/2 Re of the N central outputs is
//            multiplied by 1/psi_hat(j1') 1/psi_hat(j2') / (omega sum w).
// The transforms are radix-2 decimation-in-time in shared memory with a
// float32 twiddle table e^{+2 pi i k / G} computed in float64 at plan time.
#include "toi_internal.cuh"

namespace toi {
namespace {

constexpr int kFftThreads = 512;

__device__ __forceinline__ int bitrev(int x, int logn) { return __brev(x) >> (32 - logn); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-place radix-2 DIT on `nseq` sequences of length G stored back to back
// in shared memory (inputs already in bit-reversed order).
__device__ void fft_stages(float2* x, int G, int logG, int nseq, const float2* __restrict__ tw) {
  const int nb = nseq * (G >> 1);
  for (int s = 1; s <= logG; ++s) {
    const int half = 1 << (s - 1);
    const int stride = G >> s;   // twiddle index step
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      const int seq = b / (G >> 1);
      const int bb = b - seq * (G >> 1);
      const int grp = bb >> (s - 1);
      const int pos = bb & (half - 1);
      float2* base = x + (size_t)seq * G;
      const int i = (grp << s) + pos;
      const int j = i + half;
      const float2 w = tw[pos * stride];
      const float2 t = cmul(w, base[j]);
      const float2 u = base[i];
      base[i] = make_float2(u.x + t.x, u.y + t.y);
      base[j] = make_float2(u.x - t.x, u.y - t.y);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kFftThreads)
fft_rows_kernel(const float2* __restrict__ H, int G, int logG, int N,
                const float2* __restrict__ tw, float2* __restrict__ T) {
  extern __shared__ float2 x[];
  const int row = blockIdx.x;
  const float2* src = H + (size_t)row * G;
  for (int n = threadIdx.x; n < G; n += blockDim.x) x[bitrev(n, logG)] = src[n];
  __syncthreads();
  fft_stages(x, G, logG, 1, tw);
  float2* dst = T + (size_t)row * N;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const int jp = j - N / 2;
    const int m = jp < 0 ? jp + G : jp;
    float2 v = x[m];
    if (jp & 1) { v.x = -v.x; v.y = -v.y; }
    dst[j] = v;
  }
}

__global__ void __launch_bounds__(kFftThreads)
fft_cols_kernel(const float2* __restrict__ T, int G, int logG, int N, int CW,
                const float2* __restrict__ tw, const float* __restrict__ corr,
                const double* __restrict__ snap, float* __restrict__ out) {
  extern __shared__ float2 x[];
  const int col0 = blockIdx.x * CW;
  const int half = G >> 1;
  for (int e = threadIdx.x; e < half * CW; e += blockDim.x) {
    const int r = e / CW, c = e - r * CW;
    const float2 v = T[(size_t)r * N + col0 + c];
    float2* xs = x + (size_t)c * G;
    xs[bitrev(r, logG)] = v;
    if (r > 0) xs[bitrev(G - r, logG)] = make_float2(v.x, -v.y);
    else xs[bitrev(half, logG)] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft_stages(x, G, logG, CW, tw);
  const double omega = snap[SNAP_OMEGA], sumw = snap[SNAP_SUMW];
  const float norm = sumw > 0.0 ? (float)(0.5 / (omega * sumw)) : 0.f;
  for (int e = threadIdx.x; e < N * CW; e += blockDim.x) {
    const int j2 = e / CW, c = e - j2 * CW;
    const int jp = j2 - N / 2;
    const int m = jp < 0 ? jp + G : jp;
    const float v = x[(size_t)c * G + m].x;
    out[(size_t)j2 * N + col0 + c] = v * (norm * corr[col0 + c] * corr[j2]);
  }
}

}  // namespace

int fft_col_width(int G) { return G >= 8192 ? 2 : 4; }

cudaError_t fft_configure() {
  cudaError_t e = cudaFuncSetAttribute(fft_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       8192 * 8);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fft_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              4 * 4096 * 8);
}

cudaError_t launch_fft(toi_plan_s* p, Slot& s) {
  const int G = p->G, N = p->N;
  int logG = 0;
  while ((1 << logG) < G) ++logG;
  const int CW = fft_col_width(G);
  int tok = prof_begin(p, PROF_FFT_ROWS, 1);
  fft_rows_kernel<<<G / 2, kFftThreads, (size_t)G * sizeof(float2), p->stream>>>(
      s.grid, G, logG, N, p->twiddle, p->fft_tmp);
  prof_end(p, tok);
  tok = prof_begin(p, PROF_FFT_COLS, 1);
  fft_cols_kernel<<<N / CW, kFftThreads, (size_t)CW * G * sizeof(float2), p->stream>>>(
      p->fft_tmp, G, logG, N, CW, p->twiddle, p->corr, s.snap, p->tilted);
  prof_end(p, tok);
  return cudaGetLastError();
}

}  // namespace toi
