// S2-S3: coordinates and convolutional gridding (Section 3.2; Section 4.1
// stage 3 "place visibilities on a grid").
//
// Layout.  Only Re of the inverse transform is kept (the dirty image is
// real), so the grid is stored as its Hermitian half-plane
//     H[k] = G[k] + conj(G[-k]),   rows k2' = k2 - G/2 in [0, G/2),
// i.e. every sample contributes c_q at +k_q and conj(c_q) at -k_q, each
// clipped to the stored rows.  A baseline's samples lie on a radial track
// g(k) = G/2 + a k (k = nu / c); each baseline gives the track in the upper
// half-plane and its mirror, which only reaches rows near k2' = 0.
//
// Work distribution.  One warp per (track, channel segment); lane l walks a
// contiguous run of channels.  Consecutive channels of a track move by a
// small fraction of a cell, so each lane keeps the W x W footprint of its
// current sample in registers and accumulates successive samples there with
// register FMAs only.  When the track moves on by a cell, the column (or
// row) it leaves behind is complete and is added to the grid with one vector
// reduction per non-zero cell, and the (circular) window slides by one cell.  Grid
// traffic is therefore about W cells per cell of track length instead of
// W^2 per sample; the 67 MB
// half-plane grid of a 2048^2 image stays resident in L2 for these
// reductions, while each lane stages its stream of visibilities, weights and
// flags through shared memory with cp.async, two chunks ahead.
// The grid starts from zero (the FFT row pass clears what it reads).  Cell
// sums are exact up to float32 rounding order (the reductions commute).
#include <cuda_fp16.h>
#include <math.h>

#include "toi_internal.cuh"

namespace toi {
namespace {

constexpr int kW = 8;             // kernel support compiled in (validated in toi_plan)
constexpr int kWin = kW;          // register window side (the footprint itself)
constexpr int kWarps = 2;         // warps per block

struct TrackGeom {
  double s1, s2;   // signed coefficients: g1 = G/2 + s1 k, y = s2 k (row coordinate)
  bool conj;
};

__device__ __forceinline__ TrackGeom track_geom(const BaselineCoef& cf, int mirror) {
  const bool orig_upper = (cf.a2 > 0.0) || (cf.a2 == 0.0 && cf.a1 >= 0.0);
  const bool use_orig = (mirror == 0) == orig_upper;
  TrackGeom t;
  t.s1 = use_orig ? cf.a1 : -cf.a1;
  t.s2 = use_orig ? cf.a2 : -cf.a2;
  t.conj = !use_orig;
  return t;
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Exponential of semicircle psi(x) = exp(beta (sqrt(1 - (2x/W)^2) - 1)) with
// bl2 = beta * log2(e).
__device__ __forceinline__ float es_kernel(float x, float bl2) {
  const float t = fmaxf(fmaf(x * x, -4.0f / (kW * kW), 1.0f), 0.0f);   // 1 - (2x/W)^2
  return ex2_approx(fmaf(bl2, sqrt_approx(t), -bl2));                  // bl2 (sqrt - 1)
}

__device__ __forceinline__ void red_add(float2* p, float2 v) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(v.x), "f"(v.y));
}

// A lane's register window, kept circular: logical column i (in the
// direction of travel sx) is physical column (i + rx) mod W and lies at
// absolute grid column ox + sx * i; rows likewise with (ry, oy, sy).  A
// slide flushes the physical column (row) that holds logical column (row) 0,
// clears it for the incoming cells and advances the phase; nothing is moved
// between registers.  RH = W: one lane holds the whole W x W footprint.
// RH = W/2: two neighbouring lanes share a channel run, and lane h of the
// pair holds the physical rows [h W/2, h W/2 + W/2) - physical rows never
// move, so a column slide flushes W/2 cells in each lane and a row slide is
// done by the one lane that owns the row.  Half the window per lane halves
// its registers, doubling the resident warps.
template <int RH>
struct Window {
  float2 a[RH][kWin];   // a[owned physical row - row base][physical column]
};

// Where a window's cells go: the grid H, and in a near-coplanar pass also
// H2, which receives the imaginary-part moment.  Along one track the
// imaginary pass's values are -i times the real pass's on an upper track and
// +i times them on a mirror track (whose values are conjugated), so one
// window serves both grids: H2 gets rs * (-i v), rs = +1 or -1.
struct Sink {
  float2* H;
  float2* H2;
  float rs;
};

__device__ __forceinline__ void flush_cell(const Sink& snk, int G, int x, int y, float2 v) {
  if ((v.x != 0.f || v.y != 0.f) && x >= 0 && x < G && y >= 0 && y < (G >> 1)) {
    const size_t idx = (size_t)y * G + x;
    red_add(snk.H + idx, v);
    if (snk.H2) red_add(snk.H2 + idx, make_float2(snk.rs * v.y, -snk.rs * v.x));
  }
}

// absolute coordinate of physical index p for phase r, origin o, direction s
__device__ __forceinline__ int phys_to_abs(int p, int r, int o, int s) {
  return o + s * ((p - r) & (kWin - 1));
}

template <int RH>
__device__ __forceinline__ void flush_all(Window<RH>& w, const Sink& H, int G, int ox, int oy,
                                          int sx, int sy, int rx, int ry, int rbase) {
#pragma unroll
  for (int j = 0; j < RH; ++j) {
    const int y = phys_to_abs(rbase + j, ry, oy, sy);
#pragma unroll
    for (int i = 0; i < kWin; ++i) {
      flush_cell(H, G, phys_to_abs(i, rx, ox, sx), y, w.a[j][i]);
      w.a[j][i] = make_float2(0.f, 0.f);
    }
  }
}

template <int P, int RH>
__device__ __forceinline__ void flush_col(Window<RH>& w, const Sink& H, int G, int x, int oy,
                                          int sy, int ry, int rbase) {
#pragma unroll
  for (int j = 0; j < RH; ++j) {
    flush_cell(H, G, x, phys_to_abs(rbase + j, ry, oy, sy), w.a[j][P]);
    w.a[j][P] = make_float2(0.f, 0.f);
  }
}

template <int P, int RH>
__device__ __forceinline__ void flush_row(Window<RH>& w, const Sink& H, int G, int y, int ox,
                                          int sx, int rx) {
#pragma unroll
  for (int i = 0; i < kWin; ++i) {
    flush_cell(H, G, phys_to_abs(i, rx, ox, sx), y, w.a[P][i]);
    w.a[P][i] = make_float2(0.f, 0.f);
  }
}

// slide one column forwards: physical column rx (logical column 0) is final
template <int RH>
__device__ __forceinline__ void slide_x(Window<RH>& w, const Sink& H, int G, int ox, int oy,
                                        int sy, int rx, int ry, int rbase) {
  switch (rx) {
    case 0: flush_col<0>(w, H, G, ox, oy, sy, ry, rbase); break;
    case 1: flush_col<1>(w, H, G, ox, oy, sy, ry, rbase); break;
    case 2: flush_col<2>(w, H, G, ox, oy, sy, ry, rbase); break;
    case 3: flush_col<3>(w, H, G, ox, oy, sy, ry, rbase); break;
    case 4: flush_col<4>(w, H, G, ox, oy, sy, ry, rbase); break;
    case 5: flush_col<5>(w, H, G, ox, oy, sy, ry, rbase); break;
    case 6: flush_col<6>(w, H, G, ox, oy, sy, ry, rbase); break;
    default: flush_col<7>(w, H, G, ox, oy, sy, ry, rbase); break;
  }
}

// slide one row forwards: physical row ry is final (flushed by its owner)
template <int RH>
__device__ __forceinline__ void slide_y(Window<RH>& w, const Sink& H, int G, int ox, int oy,
                                        int sx, int rx, int ry, int rbase) {
  const int r = ry - rbase;
  if (RH == kWin) {
    switch (r) {
      case 0: flush_row<0>(w, H, G, oy, ox, sx, rx); break;
      case 1: flush_row<1 % RH>(w, H, G, oy, ox, sx, rx); break;
      case 2: flush_row<2 % RH>(w, H, G, oy, ox, sx, rx); break;
      case 3: flush_row<3 % RH>(w, H, G, oy, ox, sx, rx); break;
      case 4: flush_row<4 % RH>(w, H, G, oy, ox, sx, rx); break;
      case 5: flush_row<5 % RH>(w, H, G, oy, ox, sx, rx); break;
      case 6: flush_row<6 % RH>(w, H, G, oy, ox, sx, rx); break;
      default: flush_row<7 % RH>(w, H, G, oy, ox, sx, rx); break;
    }
  } else {
    switch (r) {
      case 0: flush_row<0>(w, H, G, oy, ox, sx, rx); break;
      case 1: flush_row<1 % RH>(w, H, G, oy, ox, sx, rx); break;
      case 2: flush_row<2 % RH>(w, H, G, oy, ox, sx, rx); break;
      case 3: flush_row<3 % RH>(w, H, G, oy, ox, sx, rx); break;
      default: break;   // the other lane of the pair owns this row
    }
  }
}

struct Sample {
  float2 c;      // weighted visibility
  float2 k;      // k = nu / c of its channel (float pair)
  bool sel;      // w_q > 0
};

// Tap origin of one axis.  The coordinate is g = c0 + 4 + s k with s (per
// track) and k = nu / c (per channel) known in float64, each held here as an
// unevaluated float sum hi + lo.  The product and the sum are formed with
// error-free transformations (Dekker / Knuth two-product and two-sum), so
// the first tap index q = ceil(g - 4) and the offset f = q - (g - 4) in [0, 1)
// carry about 2^-44 relative accuracy: the float64 result, from float32
// arithmetic.  c0 is an exact integer (G/2 - 4 or -4).
__device__ __forceinline__ void tap_origin(float shi, float slo, float khi, float klo, float c0,
                                           int& q, float& f) {
  const float p = __fmul_rn(shi, khi);
  const float e = __fmaf_rn(shi, khi, -p);
  const float l = __fmaf_rn(shi, klo, __fmaf_rn(slo, khi, e));
  const float A = __fadd_rn(c0, p);
  const float bb = __fsub_rn(A, c0);
  const float err = __fadd_rn(__fsub_rn(c0, __fsub_rn(A, bb)), __fsub_rn(p, bb));
  const float L = __fadd_rn(l, err);
  float qf = ceilf(A);
  float fr = __fsub_rn(__fsub_rn(qf, A), L);
  if (fr < 0.f) { qf += 1.f; fr += 1.f; }
  else if (fr >= 1.f) { qf -= 1.f; fr -= 1.f; }
  q = (int)qf;
  f = fr;
}

// Coordinates and kernel-argument bases of one sample.
struct Prepared {
  float2 c;        // weighted visibility (conjugated for a mirror track)
  float fxs, fys;  // offset of the first tap (direction of travel) from the sample
  int kx0, ky0;    // first tap (absolute grid index) on each axis
};

__device__ __forceinline__ void prepare(const Sample& s, float s1hi, float s1lo, float s2hi,
                                        float s2lo, float cx, float cy, int sx, int sy, bool conj,
                                        Prepared& p) {
  float fx, fy;
  tap_origin(s1hi, s1lo, s.k.x, s.k.y, cx, p.kx0, fx);
  tap_origin(s2hi, s2lo, s.k.x, s.k.y, cy, p.ky0, fy);
  p.fxs = sx > 0 ? fx - 0.5f * kW : fx + 0.5f * kW - 1.0f;
  p.fys = sy > 0 ? fy - 0.5f * kW : fy + 0.5f * kW - 1.0f;
  p.c = s.sel ? s.c : make_float2(0.f, 0.f);
  if (conj) p.c.y = -p.c.y;
}

// Near-coplanar moments (Section 3.4): a pass grids T_order(s_q) c_q (or
// -i T_order(s_q) c_q for the imaginary part) of the samples of one r3 slab,
// with r3_q = r3(baseline) k and s_q = (r3_q - r3_slab) / dr3.  The factor is
// applied before the mirror conjugation, so mirror tracks store conj of it.
__device__ __forceinline__ float2 moment_value(float2 c, float r3, const MomentPass& m) {
  float s = 0.f;
  if (!m.zero_width) {
    int p = (int)floorf((r3 - m.r3min) * m.inv2dr3);
    p = p < 0 ? 0 : (p > m.nslab - 1 ? m.nslab - 1 : p);
    if (p != m.slab) return make_float2(0.f, 0.f);
    s = (r3 - m.centre) * m.inv_dr3;
  }
  float t = m.order == 0 ? 1.f : s;   // T_order(s) by T_{k+1} = 2 s T_k - T_{k-1}
  float tm = 1.f;
  for (int k = 2; k <= m.order; ++k) {
    const float tn = 2.f * s * t - tm;
    tm = t;
    t = tn;
  }
  c.x *= t;
  c.y *= t;
  return m.imag ? make_float2(c.y, -c.x) : c;
}

// Per-lane shared-memory staging of the visibility stream: each lane keeps
// two stages of kStage samples in flight with cp.async (completion tracked by
// async-copy groups, so no register waits on outstanding loads).
constexpr int kStage = 8;

// Stage layout (per warp, struct of arrays so lane l's 4- and 8-byte words
// fall in distinct banks): [stage][sample][lane].
struct StageBuf {
  float2 va[2][kStage][32];
  float2 vb[2][kStage][32];
  unsigned int f[2][kStage][32];
  float wa[2][kStage][32];
  float wb[2][kStage][32];
};

__device__ __forceinline__ void cp_async(void* sdst, const void* gsrc, int bytes_tag) {
  const unsigned int d = (unsigned int)__cvta_generic_to_shared(sdst);
  if (bytes_tag == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

template <bool HALF>
__device__ __forceinline__ Sample read_staged(const StageBuf& sb, int sidx, int u, int lane,
                                              const float* chan_scale, const float* weight,
                                              const uint8_t* flag, const float2* kf, size_t o,
                                              int ch, int npol, int pa, int pb) {
  Sample s;
  s.k = kf[ch];
  bool fa = false, fb = false;
  if (flag) {
    if (npol == 4) {
      const unsigned int f = sb.f[sidx][u][lane];
      fa = (f & 0xffu) != 0;
      fb = (f >> 24) != 0;
    } else {
      fa = flag[o + pa] != 0;
      fb = flag[o + pb] != 0;
    }
  }
  const float wa = fa ? 0.f : (weight ? sb.wa[sidx][u][lane] : 1.f);
  float wb = fb ? 0.f : (weight ? sb.wb[sidx][u][lane] : 1.f);
  if (pa == pb) wb = 0.f;
  s.sel = wa + wb > 0.f;
  float2 va = sb.va[sidx][u][lane], vbv = (pa != pb) ? sb.vb[sidx][u][lane] : make_float2(0.f, 0.f);
  if (HALF) {
    const float sc = chan_scale[ch];
    const unsigned int ra = __float_as_uint(va.x), rb = __float_as_uint(vbv.x);
    const float2 fa2 = __half22float2(*reinterpret_cast<const __half2*>(&ra));
    const float2 fb2 = __half22float2(*reinterpret_cast<const __half2*>(&rb));
    va = make_float2(fa2.x * sc, fa2.y * sc);
    vbv = make_float2(fb2.x * sc, fb2.y * sc);
  }
  s.c = make_float2(wa * va.x + wb * vbv.x, wa * va.y + wb * vbv.y);
  return s;
}

// One warp's work: segment `seg` of track `track` (tracks [0, nbl) are the
// upper-half tracks of the baselines, [nbl, 2 nbl) their mirrors).
template <bool HALF, bool MOM, int RH>
__device__ __forceinline__ void grid_track(const BaselineCoef* __restrict__ coef,
                                           const float2* __restrict__ kf,
                                           const void* __restrict__ vis,
                                           const float* __restrict__ chan_scale,
                                           const float* __restrict__ weight,
                                           const uint8_t* __restrict__ flag, int nbl, int nch,
                                           int npol, int G, float bl2, int run, int track,
                                           int seg, StageBuf& sb, float2* __restrict__ H,
                                           const MomentPass& mp) {
  const int lane = threadIdx.x & 31;
  constexpr int RPW = 32 * RH / kWin;                   // channel runs per warp
  const int run_idx = (RH == kWin) ? lane : (lane >> 1);
  const int rbase = (RH == kWin) ? 0 : RH * (lane & 1); // first owned physical row
  const int mirror = track >= nbl ? 1 : 0;
  const int bl = track - mirror * nbl;
  const TrackGeom t = track_geom(coef[bl], mirror);
  const float2 kfirst = kf[0], klast = kf[nch - 1];
  const double kf0 = (double)kfirst.x + (double)kfirst.y;
  const double kf1 = (double)klast.x + (double)klast.y;
  // the mirror track only reaches the stored rows when it passes within
  // W/2 + 1 cells of k2' = 0
  if (mirror && fabs(t.s2) * fmin(kf0, kf1) > 0.5 * kW + 1.0) return;
  // a track far outside the grid (an oversized cell, reported by the plane
  // fit) stores nothing
  const double reach = fmax(fabs(t.s1), fabs(t.s2)) * fmax(kf0, kf1);
  if (!(reach < 2.0 * G)) return;
  const Sink snk{H, MOM ? mp.grid2 : nullptr, t.conj ? -1.f : 1.f};
  float r3bl = 0.f;
  if (MOM) {
    r3bl = (float)coef[bl].r3;
    if (!mp.zero_width && mp.nslab > 1) {
      // skip a segment whose r3 range misses the slab (channels are monotonic)
      const int w0 = seg * RPW * run, w1 = min(nch, (seg + 1) * RPW * run) - 1;
      const float2 ka = kf[w0], kb = kf[w1 < w0 ? w0 : w1];
      const float ra = r3bl * (ka.x + ka.y), rb = r3bl * (kb.x + kb.y);
      const float lo = fminf(ra, rb), hi = fmaxf(ra, rb);
      const float slo = mp.r3min + (float)mp.slab / mp.inv2dr3;
      const float shi = mp.r3min + (float)(mp.slab + 1) / mp.inv2dr3;
      const float tol = 1e-3f * (shi - slo);
      if ((mp.slab > 0 && hi < slo - tol) || (mp.slab < mp.nslab - 1 && lo > shi + tol)) return;
    }
  }
  const int c_begin = (seg * RPW + run_idx) * run;
  const int c_end = min(nch, c_begin + run);
  if (c_begin >= nch) return;
  int pa, pb;
  parallel_hands(npol, pa, pb);
  const float s1hi = (float)t.s1, s1lo = (float)(t.s1 - (double)s1hi);
  const float s2hi = (float)t.s2, s2lo = (float)(t.s2 - (double)s2hi);
  const float cx = (float)(G / 2 - kW / 2), cy = (float)(-kW / 2);
  const double dk = kf1 - kf0;
  const int sx = (t.s1 * dk >= 0.0) ? 1 : -1;
  const int sy = (t.s2 * dk >= 0.0) ? 1 : -1;
  const size_t obase = (size_t)bl * nch * npol;

  // lane-private staging: lane l only ever touches st[stage][u][l]

  Window<RH> w;
#pragma unroll
  for (int j = 0; j < RH; ++j)
#pragma unroll
    for (int i = 0; i < kWin; ++i) w.a[j][i] = make_float2(0.f, 0.f);

  const int nchunk = (c_end - c_begin + kStage - 1) / kStage;
  // staging helper: chunk q lands in stage q & 1
  auto issue = [&](int q) {
    if (q < nchunk) {
      const int c0 = c_begin + q * kStage;
      const int sidx = q & 1;
#pragma unroll
      for (int u = 0; u < kStage; ++u) {
        const int ch = c0 + u;
        if (ch < c_end) {
          const size_t o = obase + (size_t)ch * npol;
          const char* vb = reinterpret_cast<const char*>(vis);
          const int vbytes = HALF ? 4 : 8;
          cp_async(&sb.va[sidx][u][lane], vb + (o + pa) * vbytes, vbytes);
          if (pa != pb) cp_async(&sb.vb[sidx][u][lane], vb + (o + pb) * vbytes, vbytes);
          if (flag && npol == 4) cp_async(&sb.f[sidx][u][lane], flag + o, 4);
          if (weight) {
            cp_async(&sb.wa[sidx][u][lane], weight + o + pa, 4);
            if (pa != pb) cp_async(&sb.wb[sidx][u][lane], weight + o + pb, 4);
          }
        }
      }
    }
    cp_async_commit();
  };
  issue(0);
  issue(1);
  cp_async_wait1();   // chunk 0 landed

  Prepared cur;
  {
    const Sample s0 = read_staged<HALF>(sb, 0, 0, lane, chan_scale, weight, flag, kf,
                                        obase + (size_t)c_begin * npol, c_begin, npol, pa, pb);
    Sample s0m = s0;
    if (MOM) s0m.c = moment_value(s0.c, r3bl * (s0.k.x + s0.k.y), mp);
    prepare(s0m, s1hi, s1lo, s2hi, s2lo, cx, cy, sx, sy, t.conj, cur);
  }
  int ox = sx > 0 ? cur.kx0 : cur.kx0 + kW - 1;
  int oy = sy > 0 ? cur.ky0 : cur.ky0 + kW - 1;
  int rx = 0, ry = 0;
  const float fsx = (float)sx, fsy = (float)sy;
  // offset of physical column p from the first tap, in the direction of
  // travel: sx * ((p - rx) mod W); refreshed whenever the phase changes
  float ofx[kWin], ofy[RH];   // ofy: the owned rows only
#pragma unroll
  for (int p = 0; p < kWin; ++p) ofx[p] = fsx * (float)p;
#pragma unroll
  for (int r = 0; r < RH; ++r) ofy[r] = fsy * (float)(rbase + r);
  const Sample none{make_float2(0.f, 0.f), make_float2(0.f, 0.f), false};
#pragma unroll 1
  for (int ch = c_begin; ch < c_end; ++ch) {
    const int rel = ch - c_begin;
    const int q = rel / kStage, u = rel - q * kStage;
    // the next sample (ch + 1) may start a new chunk: wait for it, and refill
    // the stage that chunk q has just vacated
    const int chn = ch + 1;
    Sample sn = none;
    if (chn < c_end) {
      const int qn = q + (u + 1 == kStage ? 1 : 0);
      const int un = (u + 1 == kStage) ? 0 : u + 1;
      if (un == 0) {
        // chunk q is fully read: refill its stage with chunk qn + 1, then wait
        // until everything but that newest group (so chunk qn) has landed
        issue(qn + 1);
        cp_async_wait1();
      }
      sn = read_staged<HALF>(sb, qn & 1, un, lane, chan_scale, weight, flag, kf,
                             obase + (size_t)chn * npol, chn, npol, pa, pb);
    }
    // footprint start of the current sample in window coordinates
    int dx = sx > 0 ? cur.kx0 - ox : ox - (cur.kx0 + kW - 1);
    int dy = sy > 0 ? cur.ky0 - oy : oy - (cur.ky0 + kW - 1);
    if (dx < 0 || dy < 0 || dx >= kWin || dy >= kWin) {
      flush_all(w, snk, G, ox, oy, sx, sy, rx, ry, rbase);
      ox = sx > 0 ? cur.kx0 : cur.kx0 + kW - 1;
      oy = sy > 0 ? cur.ky0 : cur.ky0 + kW - 1;
      rx = 0;
      ry = 0;
      dx = 0;
      dy = 0;
#pragma unroll
      for (int p = 0; p < kWin; ++p) ofx[p] = fsx * (float)p;
#pragma unroll
      for (int r = 0; r < RH; ++r) ofy[r] = fsy * (float)(rbase + r);
    }
    if (dx > 0) {
      do { slide_x(w, snk, G, ox, oy, sy, rx, ry, rbase); ox += sx; rx = (rx + 1) & (kWin - 1); } while (--dx > 0);
#pragma unroll
      for (int p = 0; p < kWin; ++p) ofx[p] = fsx * (float)((p - rx) & (kWin - 1));
    }
    if (dy > 0) {
      do { slide_y(w, snk, G, ox, oy, sx, rx, ry, rbase); oy += sy; ry = (ry + 1) & (kWin - 1); } while (--dy > 0);
#pragma unroll
      for (int r = 0; r < RH; ++r) ofy[r] = fsy * (float)((rbase + r - ry) & (kWin - 1));
    }
    Prepared nxt;
    if (MOM) sn.c = moment_value(sn.c, r3bl * (sn.k.x + sn.k.y), mp);
    prepare(sn, s1hi, s1lo, s2hi, s2lo, cx, cy, sx, sy, t.conj, nxt);
    // kernel values in physical order: physical index p holds tap (p - r) mod W
    float px[kWin];
    float2 b[RH];
#pragma unroll
    for (int p = 0; p < kWin; ++p) px[p] = es_kernel(cur.fxs + ofx[p], bl2);
#pragma unroll
    for (int r = 0; r < RH; ++r) {
      const float py = es_kernel(cur.fys + ofy[r], bl2);
      b[r] = make_float2(cur.c.x * py, cur.c.y * py);
    }
#pragma unroll
    for (int j = 0; j < RH; ++j)
#pragma unroll
      for (int i = 0; i < kWin; ++i) {
        w.a[j][i].x = fmaf(px[i], b[j].x, w.a[j][i].x);
        w.a[j][i].y = fmaf(px[i], b[j].y, w.a[j][i].y);
      }
    cur = nxt;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  flush_all(w, snk, G, ox, oy, sx, sy, rx, ry, rbase);
}

template <bool HALF, bool MOM, int RH>
__global__ void __launch_bounds__(kWarps * 32)
grid_tracks_kernel(const BaselineCoef* __restrict__ coef, const float2* __restrict__ kf,
                   const void* __restrict__ vis, const float* __restrict__ chan_scale,
                   const float* __restrict__ weight, const uint8_t* __restrict__ flag, int nbl,
                   int nch, int npol, int G, float bl2, int run, int nseg,
                   float2* __restrict__ H, MomentPass mp) {
  __shared__ StageBuf stage_all[kWarps];
  const int wib = threadIdx.x >> 5;
  const int warp = blockIdx.x * kWarps + wib;
  if (warp >= 2 * nbl * nseg) return;
  // warps [0, nbl * nseg) walk the upper-half tracks, the rest their mirrors
  // (most mirror warps exit at once, so they are kept out of the busy blocks)
  grid_track<HALF, MOM, RH>(coef, kf, vis, chan_scale, weight, flag, nbl, nch, npol, G, bl2, run,
                            warp / nseg, warp % nseg, stage_all[wib], H, mp);
}

// Persistent gridder over a batch: each warp takes work items from a
// counter until none is left.  Items are numbered upper tracks of every
// entry first (the heavy ones, entries in table order), then the mirror
// tracks, most of which store nothing and leave at once.  Uneven entries
// (different channel counts and flag fractions) thus share the GPU without
// a partial last wave per entry.
template <bool HALF, int RH>
__global__ void __launch_bounds__(kWarps * 32)
grid_batch_kernel(const BatchEntry* __restrict__ E, const BatchHeader* __restrict__ hdr,
                  int* __restrict__ queue, int npol, int G, float bl2) {
  __shared__ StageBuf stage_all[kWarps];
  const int wib = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int n = hdr->n;
  const long long total = hdr->total_items;
  for (;;) {
    __syncwarp();   // lanes past their track's last channel rejoin here
    long long item = 0;
    if (lane == 0) item = (long long)atomicAdd(queue, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= total) break;
    // find the entry: upper items first, then mirror items
    int ent = -1;
    bool mir = false;
    long long local = 0;
    for (int i = 0; i < n; ++i) {
      const long long cnt = (long long)E[i].nbl * E[i].nseg;
      if (item >= E[i].up_begin && item < E[i].up_begin + cnt) { ent = i; local = item - E[i].up_begin; break; }
      if (item >= E[i].mi_begin && item < E[i].mi_begin + cnt) { ent = i; mir = true; local = item - E[i].mi_begin; break; }
    }
    if (ent < 0) continue;
    const BatchEntry& e = E[ent];
    const int seg = (int)(local % e.nseg);
    const int track = (int)(local / e.nseg) + (mir ? e.nbl : 0);
    const MomentPass none{};
    grid_track<HALF, false, RH>(e.coef, e.kf, e.vis, e.chan_scale, e.weight, e.flag, e.nbl,
                                e.nch, npol, G, bl2, e.run, track, seg, stage_all[wib], e.grid,
                                none);
  }
}

}  // namespace

// Channels per lane: each track is split into segments of 32 lanes so that
// there are several warps per SM slot (runs of at least 16 channels);
// nch / 128 measured best at 4096 channels (finer runs pay more window
// flushes, coarser ones leave a partial last wave of warps).
// Defaults when not tuned.  Single-snapshot launches: the whole window in
// one lane and runs of nch / 128 channels (measured best at 4096 channels:
// finer runs pay more window flushes, coarser ones leave a partial last wave
// of warps).  Batched launches: two lanes per run (half the registers, more
// resident warps) and long runs - the work queue removes the partial wave,
// and every run ends with a flush of its whole window, so fewer runs mean
// fewer grid reductions (358 us per snapshot at 256 channels vs 436 us at
// 32, MeerKAT-shaped); powers of two keep the last segment's lanes busy.
int grid_default_rows(bool batched) { return batched ? 4 : 8; }

int grid_default_run(int nch, bool batched) {
  if (batched) {
    int run = 16;
    while (run < 512 && run * 16 < nch) run *= 2;
    return run;
  }
  const int run = (nch + 127) / 128;
  return run < 16 ? 16 : run;
}

int channel_bucket(int nch) {
  return nch <= 1024 ? 0 : (nch <= 2048 ? 1 : (nch <= 4096 ? 2 : 3));
}

int grid_resident_blocks() {
  int lo = 1 << 30;
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, grid_batch_kernel<false, 8>, kWarps * 32, 0) != cudaSuccess) return 0;
  lo = b < lo ? b : lo;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, grid_batch_kernel<true, 8>, kWarps * 32, 0) != cudaSuccess) return 0;
  lo = b < lo ? b : lo;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, grid_batch_kernel<false, 4>, kWarps * 32, 0) != cudaSuccess) return 0;
  const int hi4 = b;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, grid_batch_kernel<true, 4>, kWarps * 32, 0) != cudaSuccess) return 0;
  // the persistent grid is sized for the half-window kernel (more resident
  // blocks); the full-window kernel then runs in waves of its own residency
  return hi4 < b ? hi4 : b;
}

int grid_runs_per_warp(int rows) { return 32 * rows / kWin; }

cudaError_t launch_grid_batch(toi_plan_s* p, bool half) {
  const float bl2 = (float)(p->beta_es * 1.4426950408889634);
  cudaError_t e = cudaMemsetAsync(p->bqueue, 0, sizeof(int), p->stream);
  if (e != cudaSuccess) return e;
  const int tok = prof_begin(p, PROF_GRID, 1);
  const bool split = p->batch_rows == 4;
  if (half && split)
    grid_batch_kernel<true, 4><<<p->grid_blocks, kWarps * 32, 0, p->stream>>>(
        p->bentry_dev, p->bheader_dev, p->bqueue, p->cfg.n_pol, p->G, bl2);
  else if (half)
    grid_batch_kernel<true, 8><<<p->grid_blocks, kWarps * 32, 0, p->stream>>>(
        p->bentry_dev, p->bheader_dev, p->bqueue, p->cfg.n_pol, p->G, bl2);
  else if (split)
    grid_batch_kernel<false, 4><<<p->grid_blocks, kWarps * 32, 0, p->stream>>>(
        p->bentry_dev, p->bheader_dev, p->bqueue, p->cfg.n_pol, p->G, bl2);
  else
    grid_batch_kernel<false, 8><<<p->grid_blocks, kWarps * 32, 0, p->stream>>>(
        p->bentry_dev, p->bheader_dev, p->bqueue, p->cfg.n_pol, p->G, bl2);
  prof_end(p, tok);
  return cudaGetLastError();
}

template <bool HALF, bool MOM>
static void launch_tracks(toi_plan_s* p, Slot& s, int rows, int blocks, const void* vis,
                          const float* chan_scale, const float* weight, const uint8_t* flag,
                          int nbl, int nch, float bl2, int run, int nseg, const MomentPass& m) {
  if (rows == 4)
    grid_tracks_kernel<HALF, MOM, 4><<<blocks, kWarps * 32, 0, p->stream>>>(
        s.coef, p->kf, vis, chan_scale, weight, flag, nbl, nch, p->cfg.n_pol, p->G, bl2, run,
        nseg, s.grid, m);
  else
    grid_tracks_kernel<HALF, MOM, 8><<<blocks, kWarps * 32, 0, p->stream>>>(
        s.coef, p->kf, vis, chan_scale, weight, flag, nbl, nch, p->cfg.n_pol, p->G, bl2, run,
        nseg, s.grid, m);
}

static cudaError_t launch_grid_impl(toi_plan_s* p, Slot& s, const void* vis,
                                    const float* chan_scale, const float* weight,
                                    const uint8_t* flag, int nbl, int nch, const MomentPass* mp) {
  const int tok = prof_begin(p, PROF_GRID, 1);
  // the slot is zero: cleared at plan creation, by the row pass of the
  // previous toi_image, or by toi_grid when a gridded slot is re-gridded
  // single launches keep their own defaults (the autotuner tunes the batch)
  const int run = p->cfg.grid_run > 0 ? p->cfg.grid_run : grid_default_run(nch, false);
  const int rows = p->cfg.grid_rows ? p->cfg.grid_rows : grid_default_rows(false);
  const int rpw = grid_runs_per_warp(rows);
  const int nseg = (nch + rpw * run - 1) / (rpw * run);
  const long long nwarps = 2LL * nbl * nseg;
  const int blocks = (int)((nwarps + kWarps - 1) / kWarps);
  const float bl2 = (float)(p->beta_es * 1.4426950408889634);
  const bool half = p->cfg.vis_dtype == TOI_VIS_C16_CHANSCALE;
  const MomentPass none{};
  const MomentPass m = mp ? *mp : none;
  if (half && mp) launch_tracks<true, true>(p, s, rows, blocks, vis, chan_scale, weight, flag, nbl, nch, bl2, run, nseg, m);
  else if (half) launch_tracks<true, false>(p, s, rows, blocks, vis, chan_scale, weight, flag, nbl, nch, bl2, run, nseg, m);
  else if (mp) launch_tracks<false, true>(p, s, rows, blocks, vis, chan_scale, weight, flag, nbl, nch, bl2, run, nseg, m);
  else launch_tracks<false, false>(p, s, rows, blocks, vis, chan_scale, weight, flag, nbl, nch, bl2, run, nseg, m);
  prof_end(p, tok);
  return cudaGetLastError();
}

cudaError_t launch_grid(toi_plan_s* p, Slot& s, const double* freq, const void* vis,
                        const float* chan_scale, const float* weight, const uint8_t* flag,
                        int nbl, int nch) {
  (void)freq;
  return launch_grid_impl(p, s, vis, chan_scale, weight, flag, nbl, nch, nullptr);
}

cudaError_t launch_grid_moment(toi_plan_s* p, Slot& s, const void* vis, const float* chan_scale,
                               const float* weight, const uint8_t* flag, int nbl, int nch,
                               const MomentPass& mp) {
  return launch_grid_impl(p, s, vis, chan_scale, weight, flag, nbl, nch, &mp);
}

}  // namespace toi
