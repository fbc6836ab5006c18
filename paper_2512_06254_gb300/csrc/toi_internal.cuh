// Internal declarations shared by the libtoi translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "toi.h"

namespace toi {

constexpr double kCLight = 299792458.0;

// Largest tile grid the candidate search accepts.  Its threshold, labelling
// and box ranking run in one block: labels spread one tile per sweep, so a
// component winding through every tile needs up to one sweep per tile, and
// each root is ranked against every tile; 2^17 tiles (362 x 362, e.g.
// 10240 px in tiles of 32) bound that worst case to seconds.
constexpr long long kMaxCandTiles = 1LL << 17;
constexpr double kArcsec = 3.14159265358979323846 / 648000.0;


// Layout of the per-slot snapshot record (float64).
enum SnapField {
  SNAP_V = 0,       // 9 values, row major
  SNAP_OMEGA = 9,
  SNAP_XI = 10,
  SNAP_ETA = 11,
  SNAP_SUMW = 12,
  SNAP_NVIS = 13,
  SNAP_ROWMAX = 14,  // largest stored grid row reached by a footprint (+1 margin)
  SNAP_LEN = 16,     // the part copied to snap_info
  SNAP_REPRO = 16,   // float32 re-projection constants -xi/beta, eta/beta, beta^2 (as doubles)
  // linear model of the channel grid, k(ch) ~ k0 + ch dk (k = nu / c), and the
  // largest deviation of any channel from it (the gridder steps coordinates
  // in fixed point along a track when that deviation is negligible)
  SNAP_K0 = 20,
  SNAP_DK = 21,
  SNAP_KDEV = 22,
  // largest distance (cells) of any grid cell a footprint reaches from the
  // grid centre (G/2, 0): the FFT row pass reads and clears only the columns
  // of each row inside this disc (every other cell of the grid is zero)
  SNAP_RADMAX = 23,
  SNAP_ALLOC = 24
};

// Per-baseline record written by the plane fit: coefficients of the grid
// coordinates, g1 = G/2 + a1 k, g2 = G/2 + a2 k, k = nu / c (float64), and r3.
struct BaselineCoef {
  double a1, a2, r3, pad;
};

// One gridding pass of the near-coplanar mode: Chebyshev order `order` of
// r3 slab `slab` (real part, or the imaginary part when imag != 0).
struct MomentPass {
  float r3min = 0.f, inv2dr3 = 0.f;   // slab index = floor((r3 - r3min) * inv2dr3), clamped
  float centre = 0.f, inv_dr3 = 0.f;  // s = (r3 - centre) * inv_dr3
  int slab = 0, nslab = 1, order = 0, imag = 0;
  int zero_width = 1;                 // r3 range of zero width: s = 0 for every sample
  float2* grid2 = nullptr;            // also flush -i (upper) / +i (mirror) times the
                                      // window here: the imaginary-part moment
};

// Host copy of a snapshot's near-coplanar plan (Section 3.4, Eqs. 26-27).
struct Mode3Plan {
  bool ready = false;
  int n_slab = 0, K = 0;
  double r3min = 0, r3max = 0, t3max = 0, phi = 0, dr3 = 0, alpha_slab = 0, err = 0;
};

struct Slot {
  float2* grid = nullptr;          // [G/2][G] Hermitian half-plane grid
  double* snap = nullptr;          // [SNAP_ALLOC]
  BaselineCoef* coef = nullptr;    // [max_bl]
  // pointers of the last toi_grid call (for the adjoint)
  const double* uvw = nullptr;
  const double* freq = nullptr;
  const void* vis = nullptr;
  const float* chan_scale = nullptr;
  const float* weight = nullptr;
  const uint8_t* flag = nullptr;
  int nbl = 0, nch = 0;
  bool valid = false;   // holds a grid from toi_grid that toi_image has not consumed
  Mode3Plan m3;         // near-coplanar mode: the moment plan of the gridded snapshot
};

// One snapshot of a batch as the batched kernels see it (device copy of a
// host-built table; see toi_batch_prepare).
struct BatchEntry {
  // inputs (caller-owned)
  const double* uvw;
  const double* freq;
  const void* vis;
  const float* chan_scale;
  const float* weight;
  const uint8_t* flag;
  int nbl, nch;
  // per-entry workspace (plan-owned)
  float2* grid;
  double* snap;
  BaselineCoef* coef;
  double* kch;
  float2* kf;
  double* kpart;
  double* bpart;
  float2* fft_tmp;
  float* tilted;
  double* tile_mom;
  // image ring and outputs
  float* ring_cur;
  const float* ring_p1;
  const float* ring_p2;
  unsigned int* max_cur;
  const unsigned int* max_p1;
  const unsigned int* max_p2;
  float* image_out;     // caller's image or NULL
  float* tlisi_out;     // caller's tLISI row or NULL (no three-image window yet)
  int with_moments;
  // gridder work split: lanes walk `run` channels, a track has nseg
  // segments; upper-track items [up_begin, up_begin + nbl * nseg), mirror
  // items [mi_begin, mi_begin + nbl * nseg)
  int run, nseg;
  long long up_begin, mi_begin;
};

struct BatchHeader {
  int n;                 // entries in this batch
  int pad;
  long long total_items; // gridder work items over all entries
};

// Per-stage device-time accounting with CUDA events on the plan's stream.
enum ProfStage {
  // PROF_BIN is reserved (the gridder needs no binning pass)
  PROF_PREP = 0, PROF_BIN, PROF_GRID, PROF_FFT_ROWS, PROF_FFT_COLS, PROF_REPROJECT,
  PROF_TLISI, PROF_BACKWARD, PROF_LOCALISE, PROF_NSTAGE
};

struct ProfState {
  bool on = false;
  std::vector<cudaEvent_t> ev;       // pre-created pool
  std::vector<int> stage_of_pair;    // stage of each recorded (start, stop) pair
  int used = 0;                      // events consumed
  double ms[PROF_NSTAGE] = {0};
  long long launches[PROF_NSTAGE] = {0};   // kernel launches per stage (always counted)
};

}  // namespace toi

struct toi_plan_s {
  toi_config cfg;
  int N = 0, G = 0, W = 0, T = 0, nslot = 0;
  double beta_rad = 0.0;       // cell size in radians
  double beta_es = 0.0;        // ES kernel shape
  cudaStream_t stream = nullptr;
  std::string err;

  toi::Slot* slots = nullptr;
  // shared scratch
  double* kch = nullptr;                 // [max_ch] k = nu / c
  float2* kf = nullptr;                  // [max_ch] k as an unevaluated float sum hi + lo
  double* kch_sum = nullptr;             // [2 * ceil(max_ch / 256)] per-block sums of k, k^2
  double* bpart = nullptr;               // [ceil(max_bl / 8)][11] plane-fit partial sums
  float2* twiddle = nullptr;             // [G] exp(+2 pi i k / G)
  float* corr = nullptr;                 // [N] 1 / psi_hat((j - N/2) / G)
  float2* fft_tmp = nullptr;             // (G/2) x N after pass 1, in column groups of four
  float* tilted = nullptr;               // [N][N]
  std::vector<float*> ring;              // [R][N][N] image ring, R = max(3, batch_max + 2)
  unsigned int* ring_max = nullptr;      // [R] float bits of max |I|
  double* tile_mom = nullptr;            // [ntl][6]
  int* d_status = nullptr;               // device status word
  double* adj_scratch = nullptr;         // partial sums and <dL/dI, I> of the adjoint
  // near-coplanar mode
  float* moments = nullptr;              // [2 max_moments][N][N] Re / Im moment images
  double* m3_dev = nullptr;              // selection scratch (keys, errors, plan)
  double* m3_host = nullptr;             // pinned copy of the selection results
  float* m3_slabs = nullptr;             // [max_moments] slab centres (float)
  float2* grid2 = nullptr;               // [G/2][G] second grid (imaginary-part moments)
  long long nimg = 0;                    // images in the ring since reset
  const float* last_image = nullptr;     // output pointer of the last toi_image
  bool fused_pending = false;
  toi::ProfState prof;

  // batched path (toi_batch_*): batch_max entries with their own workspace
  int batch_max = 0;
  toi::BatchEntry* bentry_host = nullptr;   // pinned [batch_max]
  toi::BatchHeader* bheader_host = nullptr; // pinned
  toi::BatchEntry* bentry_dev = nullptr;
  toi::BatchHeader* bheader_dev = nullptr;
  int* bqueue = nullptr;                    // gridder work counter
  int bn = 0;                               // entries of the prepared batch (0: none)
  cudaEvent_t bcopied = nullptr;            // the table of the last toi_batch_run was copied
  bool bcopied_pending = false;
  toi::Slot* bslots = nullptr;              // [batch_max] grid, snap, coef of each entry
  double* b_kch = nullptr;                  // [batch_max][max_ch]
  float2* b_kf = nullptr;
  double* b_kpart = nullptr;                // [batch_max][2 ceil(max_ch / 256) + 2]
  double* b_bpart = nullptr;                // [batch_max][11 ceil(max_bl / 8)]
  float2* b_fft_tmp = nullptr;              // [batch_max] x (G/2) x N, as fft_tmp
  float* b_tilted = nullptr;                // [batch_max][N][N]
  double* b_tile_mom = nullptr;             // [batch_max][ntl][5]
  int grid_blocks = 0;                      // persistent gridder: resident blocks
  int tuned_run[4] = {0, 0, 0, 0};          // autotuned lane runs per channel bucket
  int batch_rows = 4;                       // window rows per lane of the batch gridder
  int nsm = 0;                              // SMs of the plan's device

  // localisation (toi_localise*): max_windows windows
  int tilted_slot = -1;                     // slot whose image p->tilted holds (-1: none)
  float2* loc_k = nullptr;                  // [max_ch] k as float pairs
  float* loc_wq = nullptr;                  // [max_bl][max_ch] sample weights w_a + w_b
  float4* loc_coef = nullptr;               // [max_windows][max_bl] P_bw (hi, lo), dl, dm factors
  int4* loc_win = nullptr;                  // [max_windows] corner, flux bits, validity
  float2* loc_facets = nullptr;             // [max_windows][64][64] facet grids
  float2* loc_K = nullptr;                  // [max_windows][64][64] facet adjoints
  float* loc_gD = nullptr;                  // [max_windows][32][32] data cotangents
  float* loc_corr = nullptr;                // [32] 1 / psi_hat for 32 pixels on 64 cells
  double* loc_loss2 = nullptr;              // [max_windows] 2 L_w
  double* loc_dot = nullptr;                // [1] sum 2 L_w
  double* loc_part = nullptr;               // reverse-pass block partials
  unsigned long long* loc_keys = nullptr;   // [4096] window selection keys
  int* loc_tiles = nullptr;                 // [max_windows] selected tiles
};

namespace toi {

// ------------------------------------------------------------- launches --
// prep.cu
cudaError_t launch_prep(toi_plan_s* p, Slot& s, const double* uvw, const double* freq,
                        const float* weight, const uint8_t* flag, int nbl, int nch);
// grid.cu
cudaError_t launch_grid(toi_plan_s* p, Slot& s, const double* freq, const void* vis,
                        const float* chan_scale, const float* weight, const uint8_t* flag,
                        int nbl, int nch);
// fft.cu
cudaError_t launch_fft(toi_plan_s* p, Slot& s);
cudaError_t launch_fft_to(toi_plan_s* p, Slot& s, float* out);
cudaError_t launch_grid_moment(toi_plan_s* p, Slot& s, const void* vis, const float* chan_scale,
                               const float* weight, const uint8_t* flag, int nbl, int nch,
                               const MomentPass& mp);
// mode3.cu
cudaError_t mode3_select(toi_plan_s* p, Slot& s, const float* weight, const uint8_t* flag,
                         int nbl, int nch);
cudaError_t mode3_moments(toi_plan_s* p, Slot& s, const void* vis, const float* chan_scale,
                          const float* weight, const uint8_t* flag, int nbl, int nch);
cudaError_t launch_combine3(toi_plan_s* p, Slot& s);
// finish.cu
cudaError_t launch_reproject_moments(toi_plan_s* p, Slot& s, float* image_out,
                                     bool with_moments, int cur, int prev1, int prev2);
cudaError_t launch_ring_moments(toi_plan_s* p, const float* image, int cur, int prev1,
                                int prev2, bool with_moments);
cudaError_t launch_tlisi_finalize(toi_plan_s* p, float* tlisi, int cur, int prev1, int prev2);

// batched path (one launch per stage over all entries of a batch)
cudaError_t launch_prep_batch(toi_plan_s* p);
cudaError_t launch_grid_batch(toi_plan_s* p, bool half);
cudaError_t launch_fft_batch(toi_plan_s* p);
cudaError_t launch_finish_batch(toi_plan_s* p);
int grid_resident_blocks();                 // persistent gridder blocks per SM
int grid_default_run(int nch, bool batched);
int grid_default_rows(bool batched);
int grid_runs_per_warp(int rows);
int channel_bucket(int nch);

// degrid.cu
size_t degrid_scratch_doubles();
cudaError_t launch_degrid_backward(toi_plan_s* p, Slot& s, const float* grad_image,
                                   const float* image, float2* grad_sample, float2* grad_vis,
                                   float* grad_weight);

// localise.cu
size_t loc_part_doubles(int max_bl, int max_win, int nsm);
int loc_seed_max_tiles(int nwin);
cudaError_t launch_localise_seed(toi_plan_s* p, Slot& s, const float* tlisi, int nwin, int* win,
                                 double* src);
cudaError_t launch_localise(toi_plan_s* p, Slot& s, int nwin, const int* win, const double* src,
                            float* model, double* loss, double* grad_src, float* grad_weight);

// host-side constant tables (api.cu)
void es_fourier_table(int N, int G, int W, double beta_es, float* out);

// Profiling: prof_begin returns a token (-1 when off) for prof_end.
int prof_begin(toi_plan_s* p, int stage, int nlaunch);
void prof_end(toi_plan_s* p, int token);

// Device helpers -----------------------------------------------------------
__device__ __forceinline__ void set_status(int* st, int code) {
  atomicCAS(st, 0, code);
}

// Parallel-hand polarisations (reading c13): XX,XY,YX,YY -> 0 and 3; two pols
// -> 0 and 1; Stokes I -> 0 (pa == pb).
__device__ __forceinline__ void parallel_hands(int npol, int& pa, int& pb) {
  if (npol == 4) { pa = 0; pb = 3; }
  else if (npol == 2) { pa = 0; pb = 1; }
  else { pa = 0; pb = 0; }
}

}  // namespace toi

// Status codes written by kernels into the device status word.
#define TOI_DEV_EMPTY 4
#define TOI_DEV_RANGE 7
