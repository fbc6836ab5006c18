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
//            plain inverse DFT Z of the row.  Rows beyond the last one any
//            footprint reached are zero and skipped (input pruning); each row
//            read is cleared in the grid, which leaves the slot zeroed for the
//            next gridding.
//   Pass 2 (columns, along k2'): each column sequence is Hermitian in k2', so
//            its transform is real; two columns a, b are transformed together
//            as Z = U_a + i U_b (Re -> column a, Im -> column b), rebuilt over
//            the full length G from the stored half.  1/2 of the N central
//            outputs is multiplied by 1/psi_hat(j1') 1/psi_hat(j2') /
//            (omega sum w).
// Each transform is a Stockham autosort FFT in shared memory: radix-8 passes
// (then one radix-4 or radix-2 pass, and for G = 3 2^a or 5 2^a one radix-3
// or radix-5 pass) whose butterflies run in registers,
// twiddles from a float32 table e^{+2 pi i m / G} made in float64 at plan time
// (three table reads per radix-8 butterfly, the other powers by products).
// Shared memory is padded by one slot per sixteen: a half warp's run of 16
// consecutive complex values then fills the 32 banks exactly, which keeps
// every pass's loads and all but one radix-8 span's stores conflict-free.
// The image passes read their first pass's operands straight from global
// memory and write their last pass's outputs straight to it (fft_io), so
// only the passes in between go through shared memory.
#pragma once
#include "toi_internal.cuh"

namespace toi {

enum FftOp { FFT_FORWARD, FFT_BATCH, FFT_ADJOINT };

namespace {

__device__ __forceinline__ int pad(int a) { return a + (a >> 4); }

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
  float2 a[4] = {t[0], t[1], t[2], t[3]};
  float2 b[4] = {t[4], t[5], t[6], t[7]};
  dft4(a);
  dft4(b);
  v[0] = a[0]; v[2] = a[1]; v[4] = a[2]; v[6] = a[3];
  v[1] = b[0]; v[3] = b[1]; v[5] = b[2]; v[7] = b[3];
}

// radix 3: with s = sin(2 pi / 3), V1,2 = v0 - (v1 + v2) / 2 +- i s (v1 - v2)
__device__ __forceinline__ void dft3(float2* v) {
  const float s = 0.86602540378443865f;
  const float2 t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
  const float2 m = make_float2(v[0].x - 0.5f * t1.x, v[0].y - 0.5f * t1.y);
  const float2 is = make_float2(-s * t2.y, s * t2.x);
  v[0] = cadd(v[0], t1);
  v[1] = cadd(m, is);
  v[2] = csub(m, is);
}

// radix 5 from the symmetric and antisymmetric pairs (v1, v4), (v2, v3):
// V1,4 = v0 + c1 t1 + c2 t2 +- i (s1 d1 + s2 d2),
// V2,3 = v0 + c2 t1 + c1 t2 +- i (s2 d1 - s1 d2),
// with t = v1 + v4, v2 + v3, d = v1 - v4, v2 - v3, c_k = cos(2 pi k / 5),
// s_k = sin(2 pi k / 5).
__device__ __forceinline__ void dft5(float2* v) {
  const float c1 = 0.30901699437494742f, c2 = -0.80901699437494742f;
  const float s1 = 0.95105651629515357f, s2 = 0.58778525229247313f;
  const float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
  const float2 d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
  const float2 a1 = make_float2(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
  const float2 a2 = make_float2(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
  const float2 b1 = make_float2(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y);
  const float2 b2 = make_float2(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y);
  v[0] = cadd(v[0], cadd(t1, t2));
  v[1] = cadd(a1, cmuli(b1));
  v[4] = csub(a1, cmuli(b1));
  v[2] = cadd(a2, cmuli(b2));
  v[3] = csub(a2, cmuli(b2));
}

// radix 16 as 4 x 4: j = 4 j1 + j2, k = k1 + 4 k2; 4-point DFTs over j1, the
// twiddles e^{+2 pi i j2 k1 / 16}, 4-point DFTs over j2
__device__ __forceinline__ void dft16(float2* v) {
  const float c1 = 0.92387953251128676f, s1 = 0.38268343236508977f;   // cos, sin pi/8
  const float r = 0.70710678118654752f;
  float2 a[4][4];
#pragma unroll
  for (int j2 = 0; j2 < 4; ++j2) {
    float2 t[4] = {v[j2], v[4 + j2], v[8 + j2], v[12 + j2]};
    dft4(t);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) a[j2][k1] = t[k1];
  }
  // w^m, w = e^{+2 pi i / 16}, for m = j2 k1
  a[1][1] = cmul(a[1][1], make_float2(c1, s1));                          // m = 1
  a[1][2] = make_float2(r * (a[1][2].x - a[1][2].y), r * (a[1][2].x + a[1][2].y));   // m = 2
  a[1][3] = cmul(a[1][3], make_float2(s1, c1));                          // m = 3
  a[2][1] = make_float2(r * (a[2][1].x - a[2][1].y), r * (a[2][1].x + a[2][1].y));   // m = 2
  a[2][2] = cmuli(a[2][2]);                                              // m = 4
  a[2][3] = make_float2(-r * (a[2][3].x + a[2][3].y), r * (a[2][3].x - a[2][3].y));  // m = 6
  a[3][1] = cmul(a[3][1], make_float2(s1, c1));                          // m = 3
  a[3][2] = make_float2(-r * (a[3][2].x + a[3][2].y), r * (a[3][2].x - a[3][2].y));  // m = 6
  a[3][3] = cmul(a[3][3], make_float2(-c1, -s1));                        // m = 9
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 t[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
    dft4(t);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2];
  }
}

template <int R>
__device__ __forceinline__ void dftR(float2* v) {
  if constexpr (R == 16) dft16(v);
  else if constexpr (R == 8) dft8(v);
  else if constexpr (R == 5) dft5(v);
  else if constexpr (R == 4) dft4(v);
  else if constexpr (R == 3) dft3(v);
  else dft2(v);
}

// twiddle powers w^r, r = 1..R-1, with w = e^{+2 pi i step / G}
template <int R>
__device__ __forceinline__ void twiddles(const float2* __restrict__ tw, int step, float2* w) {
  if constexpr (R == 16) {
    const float2 w1 = __ldg(tw + step), w2 = __ldg(tw + 2 * step), w4 = __ldg(tw + 4 * step),
                 w8 = __ldg(tw + 8 * step);
    w[1] = w1; w[2] = w2; w[4] = w4; w[8] = w8;
    w[3] = cmul(w2, w1);
    w[5] = cmul(w4, w1);
    w[6] = cmul(w4, w2);
    w[7] = cmul(w4, w[3]);
#pragma unroll
    for (int r = 1; r < 8; ++r) w[8 + r] = cmul(w8, w[r]);
  } else if constexpr (R == 8) {
    const float2 w1 = __ldg(tw + step), w2 = __ldg(tw + 2 * step), w4 = __ldg(tw + 4 * step);
    w[1] = w1; w[2] = w2; w[4] = w4;
    w[3] = cmul(w2, w1);
    w[5] = cmul(w4, w1);
    w[6] = cmul(w4, w2);
    w[7] = cmul(w4, w[3]);
  } else if constexpr (R == 5) {
    const float2 w1 = __ldg(tw + step), w2 = __ldg(tw + 2 * step);
    w[1] = w1; w[2] = w2;
    w[3] = cmul(w2, w1);
    w[4] = cmul(w2, w2);
  } else if constexpr (R == 4 || R == 3) {
    const float2 w1 = __ldg(tw + step), w2 = __ldg(tw + 2 * step);
    w[1] = w1; w[2] = w2;
    if constexpr (R == 4) w[3] = cmul(w2, w1);
  } else {
    w[1] = __ldg(tw + step);
  }
}

// One Stockham pass of radix R over `nseq` padded sequences of length G in
// shared memory (in place: all loads, barrier, all stores, barrier).
template <int G, int R, int BPT>
__device__ __forceinline__ void stockham_pass(float2* x, int nseq, int Ns, const float2* __restrict__ tw) {
  constexpr int NB = G / R;       // butterflies per sequence
  constexpr int LEN = G + G / 16;  // padded sequence length
  float2 v[BPT][R];
  int jj[BPT], ss[BPT];
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    const int id = threadIdx.x + b * blockDim.x;
    const int seq = id / NB, j = id - seq * NB;
    jj[b] = j;
    ss[b] = seq;
    if (seq < nseq) {
      const float2* xs = x + (size_t)seq * LEN;
      const int k = j & (Ns - 1);
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = xs[pad(j + r * NB)];
      if (k > 0) {
        float2 w[R];
        twiddles<R>(tw, (G / (Ns * R)) * k, w);
#pragma unroll
        for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], w[r]);
      }
      dftR<R>(v[b]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    if (ss[b] < nseq) {
      float2* xs = x + (size_t)ss[b] * LEN;
      const int j = jj[b];
      const int k = j & (Ns - 1);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) xs[pad(base + r * Ns)] = v[b][r];
    }
  }
  __syncthreads();
}

constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

// G = F 2^LOG with F in {1, 3, 5}: radix-8 passes, one radix-4 or radix-2
// pass for the rest of the power of two, then one radix-F pass (last, so
// that every pass before it has a power-of-two span Ns).
template <int G>
struct Factors {
  static constexpr int F = (G % 3 == 0) ? 3 : ((G % 5 == 0) ? 5 : 1);
  static constexpr int LOG = ilog2(G / F);
  static_assert(F * (1 << LOG) == G, "transform length must be 2^a, 3 2^a or 5 2^a");
  static_assert(G % 8 == 0, "transform length must be a multiple of 8");
};

template <int G, int NSEQ, int NT>
__device__ __forceinline__ void fft_smem(float2* x, const float2* __restrict__ tw) {
  constexpr int F = Factors<G>::F, LOG = Factors<G>::LOG;
  // radix-16 passes while four bits remain, then at most one radix-8 pass:
  // fewer passes through shared memory than all-radix-8 (3 instead of 4 at
  // 4096 points)
  constexpr int N16 = LOG / 4;
  constexpr int N8 = (LOG - 4 * N16) / 3;
  constexpr int REM = LOG - 4 * N16 - 3 * N8;
  constexpr int BPT16 = (NSEQ * (G / 16) + NT - 1) / NT;
  constexpr int BPT8 = (NSEQ * (G / 8) + NT - 1) / NT;
  int Ns = 1;
#pragma unroll
  for (int p = 0; p < N16; ++p) {
    stockham_pass<G, 16, BPT16>(x, NSEQ, Ns, tw);
    Ns *= 16;
  }
#pragma unroll
  for (int p = 0; p < N8; ++p) {
    stockham_pass<G, 8, BPT8>(x, NSEQ, Ns, tw);
    Ns *= 8;
  }
  if constexpr (REM == 2) {
    constexpr int BPT4 = (NSEQ * (G / 4) + NT - 1) / NT;
    stockham_pass<G, 4, BPT4>(x, NSEQ, Ns, tw);
    Ns *= 4;
  } else if constexpr (REM == 1) {
    constexpr int BPT2 = (NSEQ * (G / 2) + NT - 1) / NT;
    stockham_pass<G, 2, BPT2>(x, NSEQ, Ns, tw);
    Ns *= 2;
  }
  if constexpr (F > 1) {
    constexpr int BPTF = (NSEQ * (G / F) + NT - 1) / NT;
    stockham_pass<G, F, BPTF>(x, NSEQ, Ns, tw);
  }
}

// The same transform with its first pass reading the input straight from
// global memory, load(seq, n) = x[n] of sequence seq, and its last pass
// handing the outputs to store(seq, m, X[m]) instead of shared memory: two
// of the shared-memory round trips (the staging of the input and the read of
// the outputs) are saved.  A first pass has span Ns = 1 (no twiddles); a last
// pass has Ns = G / R, so its butterfly j holds the outputs m = j + r Ns.
//
// With two sequences, neighbouring threads take the same butterfly of the
// two (seq = id mod 2): their global loads and stores then touch neighbouring
// 16-byte halves of one 32-byte sector.  The sequences lie SSTRIDE apart in
// shared memory, SSTRIDE = 8 (mod 16) slots, so that the two halves of a
// half-warp fall in opposite halves of the banks.
template <int G, int R, int BPT, int NSEQ, int SSTRIDE, bool FROM, bool TO, class Load, class Store>
__device__ __forceinline__ void stockham_io(float2* x, int Ns, const float2* __restrict__ tw,
                                            Load& load, Store& store) {
  constexpr int NB = G / R;
  constexpr int LEN = SSTRIDE;
  float2 v[BPT][R];
  int jj[BPT], ss[BPT];
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    const int id = threadIdx.x + b * blockDim.x;
    const int seq = id % NSEQ, j = id / NSEQ;
    jj[b] = j;
    ss[b] = seq;
    if (j < NB) {
      const int k = j & (Ns - 1);
      if constexpr (FROM) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[b][r] = load(seq, j + r * NB);
      } else {
        const float2* xs = x + (size_t)seq * LEN;
#pragma unroll
        for (int r = 0; r < R; ++r) v[b][r] = xs[pad(j + r * NB)];
      }
      if (k > 0) {
        float2 w[R];
        twiddles<R>(tw, (G / (Ns * R)) * k, w);
#pragma unroll
        for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], w[r]);
      }
      dftR<R>(v[b]);
    }
  }
  // in place: every read of this pass before any write (a first pass reads
  // no shared memory, a last pass writes none)
  if constexpr (!FROM && !TO) __syncthreads();
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    if (jj[b] < NB) {
      const int j = jj[b];
      const int k = j & (Ns - 1);
      const int base = (j - k) * R + k;
      if constexpr (TO) {
#pragma unroll
        for (int r = 0; r < R; ++r) store(ss[b], base + r * Ns, v[b][r]);
      } else {
        float2* xs = x + (size_t)ss[b] * LEN;
#pragma unroll
        for (int r = 0; r < R; ++r) xs[pad(base + r * Ns)] = v[b][r];
      }
    }
  }
  if constexpr (!TO) __syncthreads();
}

// Pass P of fft_io and the ones after it (the radices of fft_smem, in order).
template <int G, int NSEQ, int SSTRIDE, int NT, int P, class Load, class Store>
__device__ __forceinline__ void fft_io_from(float2* x, int Ns, const float2* __restrict__ tw,
                                            Load& load, Store& store) {
  constexpr int F = Factors<G>::F, LOG = Factors<G>::LOG;
  constexpr int N16 = LOG / 4;
  constexpr int N8 = (LOG - 4 * N16) / 3;
  constexpr int REM = LOG - 4 * N16 - 3 * N8;
  constexpr int NREM = REM > 0 ? 1 : 0;
  constexpr int NP = N16 + N8 + NREM + (F > 1 ? 1 : 0);
  static_assert(NP >= 2, "fft_io needs a first and a last pass");
  if constexpr (P < NP) {
    constexpr int R = P < N16 ? 16
                    : (P < N16 + N8 ? 8 : (P < N16 + N8 + NREM ? (REM == 2 ? 4 : 2) : F));
    constexpr int BPT = (NSEQ * (G / R) + NT - 1) / NT;
    stockham_io<G, R, BPT, NSEQ, SSTRIDE, P == 0, P == NP - 1>(x, Ns, tw, load, store);
    fft_io_from<G, NSEQ, SSTRIDE, NT, P + 1>(x, Ns * R, tw, load, store);
  }
}

template <int G, int NSEQ, int SSTRIDE, int NT, class Load, class Store>
__device__ __forceinline__ void fft_io(float2* x, const float2* __restrict__ tw, Load& load,
                                       Store& store) {
  static_assert(NSEQ == 1 || SSTRIDE % 16 == 8, "two sequences need a stride of 8 mod 16 slots");
  fft_io_from<G, NSEQ, SSTRIDE, NT, 0>(x, 1, tw, load, store);
}

__device__ __forceinline__ int row_limit(const double* snap, int G) {
  const int r = (int)ceil(snap[SNAP_ROWMAX]);
  return r < G / 2 ? r : G / 2 - 1;
}

// The row pass's output T, [G/2 rows][N columns] complex, is stored in
// column groups of four: element (r, j) at ((j / 4) (G/2) + r) 4 + j mod 4.
// A column-pass block reads the columns of one group (two transforms) down
// every row, now one contiguous run per warp instead of one 32-byte piece
// per row 8 N bytes apart; the row pass still writes whole 32-byte pieces.
template <int G>
__device__ __forceinline__ size_t tcol(int r, int j) {
  return ((size_t)(j >> 2) * (G / 2) + r) * 4 + (j & 3);
}

template <int G>
struct RowCfg {
  // one thread per radix-16 butterfly of a row (64 to 512 threads)
  static constexpr int NT = (G / 16 < 64) ? 64 : (G / 16 > 512 ? 512 : G / 16);
  // blocks per SM the registers are sized for: 1024 threads (64 registers a
  // thread) while two rows fit in shared memory, so that loads of several
  // rows are in flight; beyond that the shared memory allows one block
  static constexpr int MINB = G <= 8192 ? 1024 / NT : 1;
};

template <int G>
__device__ __forceinline__ void fft_rows_body(float2* __restrict__ H, int N,
                                              const float2* __restrict__ tw,
                                              const double* __restrict__ snap,
                                              float2* __restrict__ T, int row) {
  extern __shared__ float2 x[];
  if (row > row_limit(snap, G)) return;
  float2* src = H + (size_t)row * G;
  // columns of this row inside the disc that holds every non-zero cell (in
  // float32: radius and row are below 2^14, and the cell of margin on each
  // side covers its rounding; float64 is slow on this GPU)
  const float rad = (float)snap[SNAP_RADMAX];
  const float h2 = rad * rad - (float)row * (float)row;
  const float hw = h2 > 0.f ? sqrtf(h2) : 0.f;
  const int n_lo = max(0, (int)floorf(0.5f * G - hw) - 1);
  const int n_hi = min(G - 1, (int)ceilf(0.5f * G + hw) + 1);
  // first pass from the grid row (zero outside the disc), last pass straight
  // to the N central outputs: (-1)^j1' Z[j1' mod G]
  auto load = [&](int, int n) -> float2 {
    return (n >= n_lo && n <= n_hi) ? src[n] : make_float2(0.f, 0.f);
  };
  auto store = [&](int, int m, float2 v) {
    const int jp = m < G / 2 ? m : m - G;
    if (jp >= -N / 2 && jp < N / 2) {
      if (jp & 1) { v.x = -v.x; v.y = -v.y; }
      T[tcol<G>(row, jp + N / 2)] = v;
    }
  };
  fft_io<G, 1, G + G / 16, RowCfg<G>::NT>(x, tw, load, store);
  // leave the grid slot cleared for the next gridding (outside the disc it is
  // zero already)
  for (int n = n_lo + (int)threadIdx.x; n <= n_hi; n += blockDim.x) src[n] = make_float2(0.f, 0.f);
}

template <int G>
__global__ void __launch_bounds__(RowCfg<G>::NT, RowCfg<G>::MINB)
fft_rows_kernel(float2* __restrict__ H, int N, const float2* __restrict__ tw,
                const double* __restrict__ snap, float2* __restrict__ T) {
  fft_rows_body<G>(H, N, tw, snap, T, blockIdx.x);
}

template <int G>
__global__ void __launch_bounds__(RowCfg<G>::NT, RowCfg<G>::MINB)
fft_rows_batch(const BatchEntry* __restrict__ E, const BatchHeader* __restrict__ hdr, int N,
               const float2* __restrict__ tw) {
  if ((int)blockIdx.y >= hdr->n) return;
  const BatchEntry& e = E[blockIdx.y];
  fft_rows_body<G>(e.grid, N, tw, e.snap, e.fft_tmp, blockIdx.x);
}

template <int G>
struct ColCfg {
  // two real columns per complex transform; two transforms per block while
  // both fit in shared memory (G <= 8192), one beyond
  static constexpr int NSEQ = G <= 8192 ? 2 : 1;
  static constexpr int CW = 2 * NSEQ;     // columns per block
  static constexpr int NT = 512;
  static constexpr int LEN = G + G / 16;
  // distance of the two sequences in shared memory (8 mod 16 slots)
  static constexpr int SSTRIDE = NSEQ == 2 ? LEN + ((24 - LEN % 16) % 16) : LEN;
  static constexpr int SMEM = NSEQ * SSTRIDE * (int)sizeof(float2);
  // two blocks per SM (64 registers a thread) up to G = 4096; above that
  // the butterflies of a thread need more registers than 64 without spills
  static constexpr int MINB = G <= 4096 ? 2 : 1;
};

template <int G>
__device__ __forceinline__ void fft_cols_body(const float2* __restrict__ T, int N,
                                              const float2* __restrict__ tw,
                                              const float* __restrict__ corr,
                                              const double* __restrict__ snap,
                                              float* __restrict__ out, int blk) {
  constexpr int CW = ColCfg<G>::CW, NSEQ = ColCfg<G>::NSEQ;
  extern __shared__ float2 x[];
  const int col0 = blk * CW;
  constexpr int half = G / 2;
  const int rmax = row_limit(snap, G);
  // Sequence s transforms columns a = col0 + 2s, b = a + 1 of the row pass as
  // Z = U_a + i U_b over the full length G, rebuilt from the stored rows:
  //   Z[r] = U_a[r] + i U_b[r],  Z[G - r] = conj(U_a[r]) + i conj(U_b[r]),
  // rows beyond the last non-zero one and Z[G/2] zero.
  auto load = [&](int sq, int n) -> float2 {
    const int r = n < half ? n : G - n;
    if (n == half || r > rmax) return make_float2(0.f, 0.f);
    const float4 t = __ldg(reinterpret_cast<const float4*>(T + tcol<G>(r, col0 + 2 * sq)));
    return n < half ? make_float2(t.x - t.w, t.y + t.z) : make_float2(t.x + t.w, t.z - t.y);
  };
  const double omega = snap[SNAP_OMEGA], sumw = snap[SNAP_SUMW];
  const float norm = sumw > 0.0 ? (float)(0.5 / (omega * sumw)) : 0.f;
  float ca[NSEQ], cb[NSEQ];
#pragma unroll
  for (int q = 0; q < NSEQ; ++q) {
    ca[q] = corr[col0 + 2 * q];
    cb[q] = corr[col0 + 2 * q + 1];
  }
  // Re -> column a, Im -> column b of output row j2' = m (mod G), times the
  // grid correction of both axes and 1/2 1/(omega sum w)
  auto store = [&](int sq, int m, float2 z) {
    const int jp = m < half ? m : m - G;
    if (jp >= -N / 2 && jp < N / 2) {
      const int j2 = jp + N / 2;
      const float sc = norm * corr[j2];
      float cq_a = ca[0], cq_b = cb[0];
      if (NSEQ == 2 && sq == 1) { cq_a = ca[NSEQ - 1]; cq_b = cb[NSEQ - 1]; }
      *reinterpret_cast<float2*>(out + (size_t)j2 * N + col0 + 2 * sq) =
          make_float2(z.x * (sc * cq_a), z.y * (sc * cq_b));
    }
  };
  fft_io<G, NSEQ, ColCfg<G>::SSTRIDE, ColCfg<G>::NT>(x, tw, load, store);
}

template <int G>
__global__ void __launch_bounds__(ColCfg<G>::NT, ColCfg<G>::MINB)
fft_cols_kernel(const float2* __restrict__ T, int N, const float2* __restrict__ tw,
                const float* __restrict__ corr, const double* __restrict__ snap,
                float* __restrict__ out) {
  fft_cols_body<G>(T, N, tw, corr, snap, out, blockIdx.x);
}

template <int G>
__global__ void __launch_bounds__(ColCfg<G>::NT, ColCfg<G>::MINB)
fft_cols_batch(const BatchEntry* __restrict__ E, const BatchHeader* __restrict__ hdr, int N,
               const float2* __restrict__ tw, const float* __restrict__ corr) {
  if ((int)blockIdx.y >= hdr->n) return;
  const BatchEntry& e = E[blockIdx.y];
  fft_cols_body<G>(e.fft_tmp, N, tw, corr, e.snap, e.tilted, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Adjoint passes (toi_degrid_backward).  The sample cotangents need
//   Hbar[k'] = sum_j' U[j'] e^{-2 pi i (k1' j1' + k2' j2') / G}
// for rows k2' = 0..R, U the real N x N cotangent (already scaled by the grid
// correction and 1/(omega sum w)); rows k2' < 0 are conj(Hbar[-k']).  Both
// passes run the same e^{+} transform core and use that U is real:
//   pass A (columns, along j2'): Y[k2', j1'] = sum_j2' U e^{+2 pi i k2' j2' / G},
//       two real columns per complex transform (Z = U_a + i U_b, then
//       Y_a[k] = (Z[k] + conj Z[-k]) / 2, Y_b[k] = (Z[k] - conj Z[-k]) / 2i);
//   pass B (rows, along j1'): K[k2', n] = sum_j1' (-1)^j1' Y[k2', j1'] e^{+2 pi i n j1' / G},
//       n = k1' + G/2, so that Hbar[k2', n] = conj(K[k2', n]).
// They are the adjoints of pass 2 and pass 1 of the image, with the same row
// pruning.

template <int G>
__global__ void __launch_bounds__(ColCfg<G>::NT)
fft_adj_cols_kernel(const float* __restrict__ U, int N, const float2* __restrict__ tw,
                    const double* __restrict__ snap, float2* __restrict__ Y) {
  constexpr int CW = ColCfg<G>::CW, LEN = ColCfg<G>::LEN, NSEQ = ColCfg<G>::NSEQ;
  extern __shared__ float2 x[];
  const int col0 = blockIdx.x * CW;
  const int rmax = row_limit(snap, G);
  for (int e = threadIdx.x; e < NSEQ * LEN; e += blockDim.x) x[e] = make_float2(0.f, 0.f);
  __syncthreads();
  for (int j2 = threadIdx.x; j2 < N; j2 += blockDim.x) {
    const int jp = j2 - N / 2;
    const int m = pad(jp < 0 ? jp + G : jp);
    if constexpr (NSEQ == 2) {
      const float4 u = *reinterpret_cast<const float4*>(U + (size_t)j2 * N + col0);
      x[m] = make_float2(u.x, u.y);          // columns col0, col0 + 1
      x[LEN + m] = make_float2(u.z, u.w);    // columns col0 + 2, col0 + 3
    } else {
      x[m] = *reinterpret_cast<const float2*>(U + (size_t)j2 * N + col0);
    }
  }
  __syncthreads();
  fft_smem<G, NSEQ, ColCfg<G>::NT>(x, tw);
  for (int e = threadIdx.x; e < (rmax + 1) * NSEQ; e += blockDim.x) {
    const int r = e / NSEQ, pr = e - (e / NSEQ) * NSEQ;
    const float2* xs = x + (size_t)pr * LEN;
    const float2 z = xs[pad(r)], zm = xs[pad(r == 0 ? 0 : G - r)];
    const float4 o = make_float4(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y),
                                 0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
    *reinterpret_cast<float4*>(Y + (size_t)r * N + col0 + 2 * pr) = o;
  }
}

template <int G>
__global__ void __launch_bounds__(RowCfg<G>::NT)
fft_adj_rows_kernel(const float2* __restrict__ Y, int N, const float2* __restrict__ tw,
                    const double* __restrict__ snap, float2* __restrict__ K) {
  extern __shared__ float2 x[];
  const int row = blockIdx.x;
  if (row > row_limit(snap, G)) return;
  for (int n = threadIdx.x; n < G; n += blockDim.x) x[pad(n)] = make_float2(0.f, 0.f);
  __syncthreads();
  const float2* src = Y + (size_t)row * N;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const int jp = j - N / 2;
    float2 v = src[j];
    if (jp & 1) { v.x = -v.x; v.y = -v.y; }
    x[pad(jp < 0 ? jp + G : jp)] = v;
  }
  __syncthreads();
  fft_smem<G, 1, RowCfg<G>::NT>(x, tw);
  float2* dst = K + (size_t)row * G;
  for (int n = threadIdx.x; n < G; n += blockDim.x) dst[n] = x[pad(n)];
}

template <int G>
cudaError_t configure_g() {
  const int row_smem = (G + G / 16) * (int)sizeof(float2);
  const int col_smem = ColCfg<G>::SMEM;   // also covers the adjoint's NSEQ * LEN
  cudaError_t e = cudaFuncSetAttribute(fft_rows_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       row_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fft_cols_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, col_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fft_adj_rows_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             row_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fft_adj_cols_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             col_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fft_rows_batch<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, row_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fft_cols_batch<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, col_smem);
  return e;
}

template <int G>
void launch_batch_g(toi_plan_s* p) {
  const int N = p->N, B = p->batch_max;
  constexpr int CW = ColCfg<G>::CW;
  int tok = prof_begin(p, PROF_FFT_ROWS, 1);
  fft_rows_batch<G><<<dim3(G / 2, B), RowCfg<G>::NT, (G + G / 16) * sizeof(float2), p->stream>>>(
      p->bentry_dev, p->bheader_dev, N, p->twiddle);
  prof_end(p, tok);
  tok = prof_begin(p, PROF_FFT_COLS, 1);
  fft_cols_batch<G><<<dim3(N / CW, B), ColCfg<G>::NT, ColCfg<G>::SMEM,
                      p->stream>>>(p->bentry_dev, p->bheader_dev, N, p->twiddle, p->corr);
  prof_end(p, tok);
}

template <int G>
void launch_adj_g(toi_plan_s* p, Slot& s) {
  const int N = p->N;
  constexpr int CW = ColCfg<G>::CW;
  fft_adj_cols_kernel<G><<<N / CW, ColCfg<G>::NT, ColCfg<G>::NSEQ * ColCfg<G>::LEN * sizeof(float2), p->stream>>>(
      p->tilted, N, p->twiddle, s.snap, p->fft_tmp);
  fft_adj_rows_kernel<G><<<G / 2, RowCfg<G>::NT, (G + G / 16) * sizeof(float2), p->stream>>>(
      p->fft_tmp, N, p->twiddle, s.snap, s.grid);
}

template <int G>
void launch_g(toi_plan_s* p, Slot& s, float* out) {
  const int N = p->N;
  int tok = prof_begin(p, PROF_FFT_ROWS, 1);
  fft_rows_kernel<G><<<G / 2, RowCfg<G>::NT, (G + G / 16) * sizeof(float2), p->stream>>>(
      s.grid, N, p->twiddle, s.snap, p->fft_tmp);
  prof_end(p, tok);
  tok = prof_begin(p, PROF_FFT_COLS, 1);
  constexpr int CW = ColCfg<G>::CW;
  fft_cols_kernel<G><<<N / CW, ColCfg<G>::NT, ColCfg<G>::SMEM, p->stream>>>(
      p->fft_tmp, N, p->twiddle, p->corr, s.snap, out);
  prof_end(p, tok);
}

template <int G>
cudaError_t run_g(toi_plan_s* p, FftOp op, Slot* s, float* out) {
  switch (op) {
    case FFT_FORWARD: launch_g<G>(p, *s, out); break;
    case FFT_BATCH: launch_batch_g<G>(p); break;
    case FFT_ADJOINT: launch_adj_g<G>(p, *s); break;
  }
  return cudaGetLastError();
}

}  // namespace

// One translation unit per transform-length family (2^a, 3 2^a, 5 2^a):
// each returns cudaErrorInvalidValue for a length outside its family.
cudaError_t fft_configure_pow2(int G);
cudaError_t fft_run_pow2(toi_plan_s* p, FftOp op, Slot* s, float* out);
cudaError_t fft_configure_r3(int G);
cudaError_t fft_run_r3(toi_plan_s* p, FftOp op, Slot* s, float* out);
cudaError_t fft_configure_r5(int G);
cudaError_t fft_run_r5(toi_plan_s* p, FftOp op, Slot* s, float* out);

}  // namespace toi
