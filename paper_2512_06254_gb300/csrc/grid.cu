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
constexpr int kStage = 4;

// Stage layout (per warp, struct of arrays so lane l's 4- and 8-byte words
// fall in distinct banks): [stage][sample][lane].
struct StageBuf {
  float2 va[2][kStage][32];
  float2 vb[2][kStage][32];
  unsigned int f[2][kStage][32];
  float wa[2][kStage][32];
  float wb[2][kStage][32];
  float sc[2][kStage][32];   // FP16 storage: the channel's scale
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

// ---------------------------------------------------------------------------
// Two-dimensional gridding with packed single-precision pairs.
//
// Blackwell executes fma / mul / add on two float32 values held in one
// 64-bit register pair as a single instruction (f32x2).  The gridder is
// bound by instruction issue, and nearly every one of its float operations
// comes in pairs: a window cell is a complex (re, im) that receives
// px * (re, im) of the sample, and the kernel values are evaluated for
// neighbouring taps.  This path therefore keeps the register window as packed
// (re, im) cells and evaluates the kernel two taps at a time; only the
// square root and exp2 (one MUFU operation each per value) stay scalar.
//
// Coordinates.  On a channel grid that is linear in k = nu / c (every
// Measurement-Set spectral window this library has seen; checked per
// snapshot by the plane fit, which records the largest deviation of any
// channel from the chord k0 + ch dk), a track's first-tap coordinate
// h(ch) = c0 + s k(ch) is an arithmetic progression.  Each lane starts from
// h(c_begin) rounded to 32.32 fixed point (from float64) and adds the
// rounded step once per channel: one 64-bit integer add per axis, exact
// apart from the step's rounding, under 2^-33 cell per channel (6e-8 cell
// over a 512-channel run).  The tap index is the ceiling of h and the
// offset f = q - h in [0, 1) comes from the fraction bits (truncated to
// float32's 23).  A snapshot whose channels deviate from the chord by more
// than 1e-7 cell on a track takes the error-free float32 route of
// tap_origin instead.

typedef unsigned long long f2x;   // two float32 in one 64-bit register pair

__device__ __forceinline__ f2x pk(float a, float b) {
  f2x r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk(f2x v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c) {
  f2x d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2x mul2(f2x a, f2x b) {
  f2x d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x add2(f2x a, f2x b) {
  f2x d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// psi at two packed arguments x in [-4, 4] (W = 8).  1 - (2x/W)^2 is formed
// as (1 - x/4)(1 + x/4): each factor is >= 0 for such x after rounding, so
// no clamp is needed, and it keeps its relative accuracy near the support
// edge where 1 - x^2/16 cancels.
__device__ __forceinline__ void es_kernel2(f2x x, f2x bl2x2, f2x nbl2x2, float& p0, float& p1) {
  const f2x u = fma2(x, pk(-0.25f, -0.25f), pk(1.f, 1.f));
  const f2x v = fma2(x, pk(0.25f, 0.25f), pk(1.f, 1.f));
  float t0, t1;
  upk(mul2(u, v), t0, t1);
  float e0, e1;
  upk(fma2(pk(sqrt_approx(t0), sqrt_approx(t1)), bl2x2, nbl2x2), e0, e1);
  p0 = ex2_approx(e0);
  p1 = ex2_approx(e1);
}

// first tap q = ceil(h) and offset f = q - h of a 32.32 fixed-point h
__device__ __forceinline__ void fixed_tap(long long h, int& q, float& f) {
  const unsigned int lo = (unsigned int)h;
  q = (int)(h >> 32) + (lo != 0u ? 1 : 0);
  const unsigned int fb = 0u - lo;   // (q - h) 2^32 in [0, 2^32)
  f = __uint_as_float(0x3f800000u | (fb >> 9)) - 1.0f;
}

__device__ __forceinline__ void flush_cell2(float2* H, int G, int x, int y, f2x v) {
  float re, im;
  upk(v, re, im);
  if ((re != 0.f || im != 0.f) && (unsigned)x < (unsigned)G && (unsigned)y < (unsigned)(G >> 1))
    red_add(H + (size_t)y * G + x, make_float2(re, im));
}

template <int RH>
struct Win2 {
  f2x a[RH][kWin];   // a[owned physical row - row base][physical column], (re, im)
};

template <int RH>
__device__ __forceinline__ void flush_all2(Win2<RH>& w, float2* H, int G, int ox, int oy, int sx,
                                           int sy, int rx, int ry, int rbase) {
#pragma unroll
  for (int j = 0; j < RH; ++j) {
    const int y = phys_to_abs(rbase + j, ry, oy, sy);
#pragma unroll
    for (int i = 0; i < kWin; ++i) {
      flush_cell2(H, G, phys_to_abs(i, rx, ox, sx), y, w.a[j][i]);
      w.a[j][i] = 0ull;
    }
  }
}

// Column slide: physical column P (logical column 0) is final.  Every other
// column moves one step closer to the sample's first tap and column P
// becomes the last (offset 7 steps): the packed offsets ofx2 follow.
template <int P, int RH>
__device__ __forceinline__ void slide_col2(Win2<RH>& w, f2x (&ofx2)[kWin / 2], f2x nsx2,
                                           float fsx7, float2* H, int G, int x, int oy, int sy,
                                           int ry, int rbase) {
#pragma unroll
  for (int j = 0; j < RH; ++j) {
    flush_cell2(H, G, x, phys_to_abs(rbase + j, ry, oy, sy), w.a[j][P]);
    w.a[j][P] = 0ull;
  }
#pragma unroll
  for (int i = 0; i < kWin / 2; ++i) ofx2[i] = add2(ofx2[i], nsx2);
  float a, b;
  upk(ofx2[P / 2], a, b);
  ofx2[P / 2] = (P & 1) ? pk(a, fsx7) : pk(fsx7, b);
}

template <int RH>
__device__ __forceinline__ void slide_x2(Win2<RH>& w, f2x (&ofx2)[kWin / 2], f2x nsx2, float fsx7,
                                         float2* H, int G, int ox, int oy, int sy, int rx, int ry,
                                         int rbase) {
  switch (rx) {
    case 0: slide_col2<0>(w, ofx2, nsx2, fsx7, H, G, ox, oy, sy, ry, rbase); break;
    case 1: slide_col2<1>(w, ofx2, nsx2, fsx7, H, G, ox, oy, sy, ry, rbase); break;
    case 2: slide_col2<2>(w, ofx2, nsx2, fsx7, H, G, ox, oy, sy, ry, rbase); break;
    case 3: slide_col2<3>(w, ofx2, nsx2, fsx7, H, G, ox, oy, sy, ry, rbase); break;
    case 4: slide_col2<4>(w, ofx2, nsx2, fsx7, H, G, ox, oy, sy, ry, rbase); break;
    case 5: slide_col2<5>(w, ofx2, nsx2, fsx7, H, G, ox, oy, sy, ry, rbase); break;
    case 6: slide_col2<6>(w, ofx2, nsx2, fsx7, H, G, ox, oy, sy, ry, rbase); break;
    default: slide_col2<7>(w, ofx2, nsx2, fsx7, H, G, ox, oy, sy, ry, rbase); break;
  }
}

// Row slide: physical row R (logical row 0) is final; its owner flushes it.
// Every owned row's offset moves one step closer and row R becomes the last.
template <int R, int RH>
__device__ __forceinline__ void slide_row2(Win2<RH>& w, f2x (&ofy2)[RH / 2], f2x nsy2, float fsy7,
                                           float2* H, int G, int y, int ox, int sx, int rx) {
#pragma unroll
  for (int i = 0; i < kWin; ++i) {
    flush_cell2(H, G, phys_to_abs(i, rx, ox, sx), y, w.a[R][i]);
    w.a[R][i] = 0ull;
  }
  float a, b;
  upk(ofy2[R / 2], a, b);
  ofy2[R / 2] = (R & 1) ? pk(a, fsy7) : pk(fsy7, b);
}

template <int RH>
__device__ __forceinline__ void slide_y2(Win2<RH>& w, f2x (&ofy2)[RH / 2], f2x nsy2, float fsy7,
                                         float2* H, int G, int ox, int oy, int sx, int rx, int ry,
                                         int rbase) {
#pragma unroll
  for (int i = 0; i < RH / 2; ++i) ofy2[i] = add2(ofy2[i], nsy2);
  const int r = ry - rbase;   // owned row index, or outside [0, RH)
  switch (r) {
    case 0: slide_row2<0>(w, ofy2, nsy2, fsy7, H, G, oy, ox, sx, rx); break;
    case 1: slide_row2<1 % RH>(w, ofy2, nsy2, fsy7, H, G, oy, ox, sx, rx); break;
    case 2: slide_row2<2 % RH>(w, ofy2, nsy2, fsy7, H, G, oy, ox, sx, rx); break;
    case 3: slide_row2<3 % RH>(w, ofy2, nsy2, fsy7, H, G, oy, ox, sx, rx); break;
    case 4: if (RH == kWin) slide_row2<4 % RH>(w, ofy2, nsy2, fsy7, H, G, oy, ox, sx, rx); break;
    case 5: if (RH == kWin) slide_row2<5 % RH>(w, ofy2, nsy2, fsy7, H, G, oy, ox, sx, rx); break;
    case 6: if (RH == kWin) slide_row2<6 % RH>(w, ofy2, nsy2, fsy7, H, G, oy, ox, sx, rx); break;
    case 7: if (RH == kWin) slide_row2<7 % RH>(w, ofy2, nsy2, fsy7, H, G, oy, ox, sx, rx); break;
    default: break;   // the other lane of the pair owns this row
  }
}

// One sample ready for the window: packed weighted visibility, offsets of
// its first taps (in the direction of travel) and the first taps.
struct Prep2 {
  f2x c;
  float fxs, fys;
  int kx0, ky0;
};

// The weighted visibility of a staged sample (flags, weights, parallel-hand
// average; Section 3.5), packed, or 0 when it is not selected.
template <bool HALF>
__device__ __forceinline__ f2x staged_vis(const StageBuf& sb, int sidx, int u, int lane,
                                          const float* chan_scale, const float* weight,
                                          const uint8_t* flag, size_t o, int ch, int npol,
                                          int pa, int pb) {
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
  float2 va = sb.va[sidx][u][lane], vbv = (pa != pb) ? sb.vb[sidx][u][lane] : make_float2(0.f, 0.f);
  float sa = wa, sbw = wb;   // weights, times the channel scale for FP16 storage
  if (HALF) {
    const float sc = sb.sc[sidx][u][lane];
    const unsigned int ra = __float_as_uint(va.x), rb = __float_as_uint(vbv.x);
    va = __half22float2(*reinterpret_cast<const __half2*>(&ra));
    vbv = __half22float2(*reinterpret_cast<const __half2*>(&rb));
    sa *= sc;
    sbw *= sc;
  }
  const f2x c = fma2(pk(sbw, sbw), pk(vbv.x, vbv.y), mul2(pk(sa, sa), pk(va.x, va.y)));
  return (wa + wb > 0.f) ? c : 0ull;
}

template <bool HALF, int RH>
__device__ __forceinline__ void grid_track2(const BaselineCoef* __restrict__ coef,
                                            const float2* __restrict__ kf,
                                            const double* __restrict__ snap,
                                            const void* __restrict__ vis,
                                            const float* __restrict__ chan_scale,
                                            const float* __restrict__ weight,
                                            const uint8_t* __restrict__ flag, int nbl, int nch,
                                            int npol, int G, float bl2, int run, int track,
                                            int seg, StageBuf& sb, float2* __restrict__ H) {
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
  int c_begin = (seg * RPW + run_idx) * run;
  int c_end = min(nch, c_begin + run);
  if (c_begin >= nch) return;
  int pa, pb;
  parallel_hands(npol, pa, pb);
  // coordinates: fixed-point steps on a linear channel grid, else tap_origin
  const double cxd = (double)(G / 2 - kW / 2), cyd = (double)(-kW / 2);
  const double k0 = snap[SNAP_K0], dkl = snap[SNAP_DK];
  const bool lin = snap[SNAP_KDEV] * fmax(fabs(t.s1), fabs(t.s2)) <= 1e-7;   // warp-uniform
  // Run alignment.  The lanes of a warp walk consecutive runs of one track,
  // all at the same speed v cells per channel; with runs of equal length
  // their fractional positions differ, so each lane slides its window at
  // its own iteration and the warp executes ~16 separate slides per cell of
  // travel.  When the track moves fast enough on its major axis (at least
  // one cell per kAlignChannels channels), every run boundary is moved
  // forward by less than one crossing period so that each run starts at the
  // fractional position of the track's first channel: the major-axis
  // crossings of all lanes then fall in the same iteration (or the next),
  // and one slide execution serves the whole warp.  Boundaries stay shared
  // between neighbouring runs, so every channel is still gridded once.
  if (lin) {
    constexpr double kAlignChannels = 64.0;
    const double vx = t.s1 * dkl, vy = t.s2 * dkl;
    const bool xmaj = fabs(vx) >= fabs(vy);
    const double v = xmaj ? vx : vy, sm = xmaj ? t.s1 : t.s2, cm = xmaj ? cxd : cyd;
    if (fabs(v) * kAlignChannels >= 1.0 && fabs(v) * run >= 4.0) {
      const double h0 = cm + sm * k0;
      const double ph0 = h0 - floor(h0);
      // first channel of the track's run L
      auto aligned = [&](int L) -> int {
        const int cn = L * run;
        if (L <= 0) return 0;
        if (cn >= nch) return nch;
        const double hn = cm + sm * (k0 + (double)cn * dkl);
        const double d = ph0 - (hn - floor(hn));
        const double delta = v > 0.0 ? (d - floor(d)) / v : ((-d) - floor(-d)) / (-v);
        return min(nch, cn + (int)rint(delta));
      };
      const int L = seg * RPW + run_idx;
      c_begin = aligned(L);
      c_end = aligned(L + 1);
      if (c_begin >= c_end) return;
    }
  }
  long long hx = 0, hy = 0, vx = 0, vy = 0;
  if (lin) {
    const double kb = k0 + (double)c_begin * dkl;
    hx = __double2ll_rn((cxd + t.s1 * kb) * 4294967296.0);
    hy = __double2ll_rn((cyd + t.s2 * kb) * 4294967296.0);
    vx = __double2ll_rn(t.s1 * dkl * 4294967296.0);
    vy = __double2ll_rn(t.s2 * dkl * 4294967296.0);
  }
  const float s1hi = (float)t.s1, s1lo = (float)(t.s1 - (double)s1hi);
  const float s2hi = (float)t.s2, s2lo = (float)(t.s2 - (double)s2hi);
  const float cx = (float)cxd, cy = (float)cyd;
  const double dk = kf1 - kf0;
  const int sx = (t.s1 * dk >= 0.0) ? 1 : -1;
  const int sy = (t.s2 * dk >= 0.0) ? 1 : -1;
  const float fsx = (float)sx, fsy = (float)sy;
  const float xoff = sx > 0 ? -0.5f * kW : 0.5f * kW - 1.0f;   // first tap in the direction of travel
  const float yoff = sy > 0 ? -0.5f * kW : 0.5f * kW - 1.0f;
  const f2x cflip = t.conj ? 0x8000000000000000ull : 0ull;     // conjugate: flip the sign of im
  const size_t obase = (size_t)bl * nch * npol;
  const f2x bl2x2 = pk(bl2, bl2), nbl2x2 = pk(-bl2, -bl2);

  // the coordinates of channel ch (called once per channel, in order)
  auto coords = [&](int ch, int& kx0, int& ky0, float& fx, float& fy) {
    if (lin) {
      fixed_tap(hx, kx0, fx);
      fixed_tap(hy, ky0, fy);
      hx += vx;
      hy += vy;
    } else {
      const float2 k = kf[ch];
      tap_origin(s1hi, s1lo, k.x, k.y, cx, kx0, fx);
      tap_origin(s2hi, s2lo, k.x, k.y, cy, ky0, fy);
    }
  };

  Win2<RH> w;
#pragma unroll
  for (int j = 0; j < RH; ++j)
#pragma unroll
    for (int i = 0; i < kWin; ++i) w.a[j][i] = 0ull;

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
          if (HALF) cp_async(&sb.sc[sidx][u][lane], chan_scale + ch, 4);
        }
      }
    }
    cp_async_commit();
  };
  issue(0);
  issue(1);
  cp_async_wait1();   // chunk 0 landed

  Prep2 cur;
  {
    float fx, fy;
    coords(c_begin, cur.kx0, cur.ky0, fx, fy);
    cur.fxs = fx + xoff;
    cur.fys = fy + yoff;
    cur.c = staged_vis<HALF>(sb, 0, 0, lane, chan_scale, weight, flag,
                             obase + (size_t)c_begin * npol, c_begin, npol, pa, pb) ^ cflip;
  }
  int ox = sx > 0 ? cur.kx0 : cur.kx0 + kW - 1;
  int oy = sy > 0 ? cur.ky0 : cur.ky0 + kW - 1;
  int rx = 0, ry = 0;
  const f2x nsx2 = pk(-fsx, -fsx), nsy2 = pk(-fsy, -fsy);
  const float fsx7 = 7.f * fsx, fsy7 = 7.f * fsy;
  // offset of physical column p from the first tap, in the direction of
  // travel: sx ((p - rx) mod W), packed in pairs; rows likewise (owned rows)
  f2x ofx2[kWin / 2], ofy2[RH / 2];
#pragma unroll
  for (int p = 0; p < kWin / 2; ++p) ofx2[p] = pk(fsx * (float)(2 * p), fsx * (float)(2 * p + 1));
#pragma unroll
  for (int r = 0; r < RH / 2; ++r)
    ofy2[r] = pk(fsy * (float)(rbase + 2 * r), fsy * (float)(rbase + 2 * r + 1));
#pragma unroll 1
  for (int ch = c_begin; ch < c_end; ++ch) {
    const int rel = ch - c_begin;
    const int q = rel / kStage, u = rel - q * kStage;
    // the next sample (ch + 1) may start a new chunk: wait for it, and refill
    // the stage that chunk q has just vacated
    const int chn = ch + 1;
    Prep2 nxt;
    nxt.c = 0ull;
    if (chn < c_end) {
      const int qn = q + (u + 1 == kStage ? 1 : 0);
      const int un = (u + 1 == kStage) ? 0 : u + 1;
      if (un == 0) {
        issue(qn + 1);
        cp_async_wait1();
      }
      nxt.c = staged_vis<HALF>(sb, qn & 1, un, lane, chan_scale, weight, flag,
                               obase + (size_t)chn * npol, chn, npol, pa, pb) ^ cflip;
    }
    // footprint start of the current sample in window coordinates
    int dx = sx > 0 ? cur.kx0 - ox : ox - (cur.kx0 + kW - 1);
    int dy = sy > 0 ? cur.ky0 - oy : oy - (cur.ky0 + kW - 1);
    if (dx < 0 || dy < 0 || dx >= kWin || dy >= kWin) {
      flush_all2(w, H, G, ox, oy, sx, sy, rx, ry, rbase);
      ox = sx > 0 ? cur.kx0 : cur.kx0 + kW - 1;
      oy = sy > 0 ? cur.ky0 : cur.ky0 + kW - 1;
      rx = 0;
      ry = 0;
      dx = 0;
      dy = 0;
#pragma unroll
      for (int p = 0; p < kWin / 2; ++p) ofx2[p] = pk(fsx * (float)(2 * p), fsx * (float)(2 * p + 1));
#pragma unroll
      for (int r = 0; r < RH / 2; ++r)
        ofy2[r] = pk(fsy * (float)(rbase + 2 * r), fsy * (float)(rbase + 2 * r + 1));
    }
    while (dx > 0) {
      slide_x2(w, ofx2, nsx2, fsx7, H, G, ox, oy, sy, rx, ry, rbase);
      ox += sx;
      rx = (rx + 1) & (kWin - 1);
      --dx;
    }
    while (dy > 0) {
      slide_y2(w, ofy2, nsy2, fsy7, H, G, ox, oy, sx, rx, ry, rbase);
      oy += sy;
      ry = (ry + 1) & (kWin - 1);
      --dy;
    }
    if (chn < c_end) {
      float fx, fy;
      coords(chn, nxt.kx0, nxt.ky0, fx, fy);
      nxt.fxs = fx + xoff;
      nxt.fys = fy + yoff;
    } else {
      nxt.kx0 = cur.kx0;
      nxt.ky0 = cur.ky0;
      nxt.fxs = cur.fxs;
      nxt.fys = cur.fys;
    }
    // kernel values in physical order: physical index p holds tap (p - r) mod W
    const f2x fxs2 = pk(cur.fxs, cur.fxs), fys2 = pk(cur.fys, cur.fys);
    float px[kWin], py[RH];
#pragma unroll
    for (int p = 0; p < kWin / 2; ++p)
      es_kernel2(add2(fxs2, ofx2[p]), bl2x2, nbl2x2, px[2 * p], px[2 * p + 1]);
#pragma unroll
    for (int r = 0; r < RH / 2; ++r)
      es_kernel2(add2(fys2, ofy2[r]), bl2x2, nbl2x2, py[2 * r], py[2 * r + 1]);
#pragma unroll
    for (int j = 0; j < RH; ++j) {
      const f2x b = mul2(cur.c, pk(py[j], py[j]));
#pragma unroll
      for (int i = 0; i < kWin; ++i) w.a[j][i] = fma2(pk(px[i], px[i]), b, w.a[j][i]);
    }
    cur = nxt;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  flush_all2(w, H, G, ox, oy, sx, sy, rx, ry, rbase);
}

template <bool HALF, bool MOM, int RH>
__global__ void __launch_bounds__(kWarps * 32)
grid_tracks_kernel(const BaselineCoef* __restrict__ coef, const float2* __restrict__ kf,
                   const double* __restrict__ snap, const void* __restrict__ vis,
                   const float* __restrict__ chan_scale, const float* __restrict__ weight,
                   const uint8_t* __restrict__ flag, int nbl, int nch, int npol, int G, float bl2,
                   int run, int nseg, float2* __restrict__ H, MomentPass mp) {
  __shared__ StageBuf stage_all[kWarps];
  const int wib = threadIdx.x >> 5;
  const int warp = blockIdx.x * kWarps + wib;
  if (warp >= 2 * nbl * nseg) return;
  // warps [0, nbl * nseg) walk the upper-half tracks, the rest their mirrors
  // (most mirror warps exit at once, so they are kept out of the busy blocks)
  if (MOM)
    grid_track<HALF, MOM, RH>(coef, kf, vis, chan_scale, weight, flag, nbl, nch, npol, G, bl2, run,
                              warp / nseg, warp % nseg, stage_all[wib], H, mp);
  else
    grid_track2<HALF, RH>(coef, kf, snap, vis, chan_scale, weight, flag, nbl, nch, npol, G, bl2,
                          run, warp / nseg, warp % nseg, stage_all[wib], H);
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
    grid_track2<HALF, RH>(e.coef, e.kf, e.snap, e.vis, e.chan_scale, e.weight, e.flag, e.nbl,
                          e.nch, npol, G, bl2, e.run, track, seg, stage_all[wib], e.grid);
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
        s.coef, p->kf, s.snap, vis, chan_scale, weight, flag, nbl, nch, p->cfg.n_pol, p->G, bl2,
        run, nseg, s.grid, m);
  else
    grid_tracks_kernel<HALF, MOM, 8><<<blocks, kWarps * 32, 0, p->stream>>>(
        s.coef, p->kf, s.snap, vis, chan_scale, weight, flag, nbl, nch, p->cfg.n_pol, p->G, bl2,
        run, nseg, s.grid, m);
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
