// libtoi C ABI: argument validation, plan ownership and the call sequence of
// each entry point (declared and documented in include/toi.h).
#include <math.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "toi_internal.cuh"

namespace toi {
cudaError_t fft_configure(int G);
bool fft_length_supported(int G);
size_t candidates_scratch_bytes(int S, int nt);
size_t candidates_centre_bytes(int S, int nt);
cudaError_t candidates_run(const float* cube, int S, int nty, int ntx, int T, int mode,
                           cudaStream_t st, void* scratch, double* scores_out, int max_boxes,
                           int* boxes_dev, double** thr_dev, int** nbox_dev, double* xbuf);

// psi_hat(f) = integral over |x| <= W/2 of psi(x) cos(2 pi x f) dx for the
// exponential of semicircle psi(x) = exp(beta (sqrt(1 - (2x/W)^2) - 1)).
// With 2x/W = sin(theta) the integrand becomes
//   (W/2) exp(beta (cos(theta) - 1)) cos(pi W f sin(theta)) cos(theta),
// smooth on [-pi/2, pi/2], integrated by the midpoint rule.  Table entry j
// holds 1 / psi_hat((j - N/2) / G).
void es_fourier_table(int N, int G, int W, double beta_es, float* out) {
  const int M = 2048;
  const double pi = 3.14159265358979323846;
  const double h = pi / M;
  double* wt = new double[M];
  double* sn = new double[M];
  for (int i = 0; i < M; ++i) {
    const double th = -0.5 * pi + (i + 0.5) * h;
    wt[i] = 0.5 * W * exp(beta_es * (cos(th) - 1.0)) * cos(th) * h;
    sn[i] = sin(th);
  }
  for (int j = 0; j < N; ++j) {
    const double f = (double)(j - N / 2) / (double)G;
    double acc = 0.0;
    for (int i = 0; i < M; ++i) acc += wt[i] * cos(pi * W * f * sn[i]);
    out[j] = (float)(1.0 / acc);
  }
  delete[] wt;
  delete[] sn;
}

int prof_begin(toi_plan_s* p, int stage, int nlaunch) {
  p->prof.launches[stage] += nlaunch;
  if (!p->prof.on) return -1;
  ProfState& q = p->prof;
  if (q.used + 2 > (int)q.ev.size()) {   // pool exhausted: fold what is recorded
    cudaEventSynchronize(q.ev[q.used - 1]);
    for (size_t i = 0; i < q.stage_of_pair.size(); ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, q.ev[2 * i], q.ev[2 * i + 1]);
      q.ms[q.stage_of_pair[i]] += ms;
    }
    q.stage_of_pair.clear();
    q.used = 0;
  }
  const int tok = q.used;
  cudaEventRecord(q.ev[tok], p->stream);
  q.used += 2;
  q.stage_of_pair.push_back(stage);
  return tok;
}

void prof_end(toi_plan_s* p, int token) {
  if (token < 0) return;
  cudaEventRecord(p->prof.ev[token + 1], p->stream);
}

}  // namespace toi

using toi::Slot;

namespace {

thread_local std::string g_last_error;

toi_status fail(toi_plan_s* p, toi_status s, const std::string& msg) {
  if (p) p->err = msg; else g_last_error = msg;
  return s;
}

toi_status cuda_fail(toi_plan_s* p, cudaError_t e, const char* where) {
  return fail(p, TOI_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}


// lengths of the per-snapshot partial-sum buffers of the plane fit
size_t kpart_len(int max_ch) { return 2 * (((size_t)max_ch + 255) / 256) + 2; }
size_t bpart_len(int max_bl) { return 11 * (((size_t)max_bl + 7) / 8); }

// ring position of stream image t (t may be negative for the images before
// the first, which are never read)
int ring_idx(const toi_plan_s* p, long long t) {
  const long long R = (long long)p->ring.size();
  return (int)(((t % R) + R) % R);
}

template <typename T>
toi_status dev_alloc(toi_plan_s* p, T** ptr, size_t count, const char* what) {
  cudaError_t e = cudaMalloc((void**)ptr, sizeof(T) * (count ? count : 1));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return fail(p, e == cudaErrorMemoryAllocation ? TOI_ERR_OOM : TOI_ERR_CUDA,
                std::string("allocating ") + what + ": " + cudaGetErrorString(e));
  }
  return TOI_OK;
}

void free_plan(toi_plan_s* p) {
  if (!p) return;
  if (p->slots) {
    for (int i = 0; i < p->nslot; ++i) {
      cudaFree(p->slots[i].grid);
      cudaFree(p->slots[i].snap);
      cudaFree(p->slots[i].coef);
    }
    delete[] p->slots;
  }
  cudaFree(p->kch); cudaFree(p->kf); cudaFree(p->kch_sum); cudaFree(p->bpart);
  cudaFree(p->twiddle); cudaFree(p->corr); cudaFree(p->fft_tmp);
  cudaFree(p->tilted);
  for (float* r : p->ring) cudaFree(r);
  cudaFree(p->ring_max); cudaFree(p->tile_mom); cudaFree(p->d_status);
  cudaFree(p->adj_scratch);
  cudaFree(p->moments); cudaFree(p->m3_dev); cudaFree(p->m3_slabs); cudaFreeHost(p->m3_host);
  cudaFree(p->grid2);
  cudaFree(p->loc_k); cudaFree(p->loc_wq); cudaFree(p->loc_coef); cudaFree(p->loc_win); cudaFree(p->loc_facets);
  cudaFree(p->loc_K); cudaFree(p->loc_gD); cudaFree(p->loc_corr); cudaFree(p->loc_loss2);
  cudaFree(p->loc_dot); cudaFree(p->loc_part); cudaFree(p->loc_keys); cudaFree(p->loc_tiles);
  if (p->bslots) {
    for (int i = 0; i < p->batch_max; ++i) {
      cudaFree(p->bslots[i].grid);
      cudaFree(p->bslots[i].snap);
      cudaFree(p->bslots[i].coef);
    }
    delete[] p->bslots;
  }
  cudaFreeHost(p->bentry_host); cudaFreeHost(p->bheader_host);
  cudaFree(p->bentry_dev); cudaFree(p->bheader_dev); cudaFree(p->bqueue);
  cudaFree(p->b_kch); cudaFree(p->b_kf); cudaFree(p->b_kpart); cudaFree(p->b_bpart);
  cudaFree(p->b_fft_tmp); cudaFree(p->b_tilted); cudaFree(p->b_tile_mom);
  if (p->bcopied) cudaEventDestroy(p->bcopied);
  for (cudaEvent_t ev : p->prof.ev) cudaEventDestroy(ev);
  delete p;
}

}  // namespace

namespace toi {
void set_planless_error(const std::string& msg) { g_last_error = msg; }
}  // namespace toi

extern "C" {

const char* toi_status_string(toi_status s) {
  switch (s) {
    case TOI_OK: return "ok";
    case TOI_ERR_ARG: return "invalid argument";
    case TOI_ERR_CUDA: return "CUDA error";
    case TOI_ERR_OOM: return "out of device memory";
    case TOI_ERR_EMPTY: return "no selected sample (sum of weights is zero)";
    case TOI_ERR_TIMEOUT: return "bounded device wait timed out";
    case TOI_ERR_UNSUPPORTED: return "unsupported configuration";
    case TOI_ERR_RANGE: return "kernel footprint outside the grid or bad frequencies";
  }
  return "unknown status";
}

const char* toi_last_error(toi_plan_t plan) {
  return plan ? plan->err.c_str() : g_last_error.c_str();
}

toi_status toi_config_default(toi_config* cfg, int32_t image_size, double cell_arcsec,
                              int32_t max_baselines, int32_t max_channels, int32_t n_pol) {
  if (!cfg) return fail(nullptr, TOI_ERR_ARG, "cfg is NULL");
  memset(cfg, 0, sizeof(*cfg));
  cfg->image_size = image_size;
  cfg->cell_arcsec = cell_arcsec;
  cfg->max_baselines = max_baselines;
  cfg->max_channels = max_channels;
  cfg->n_pol = n_pol;
  cfg->vis_dtype = TOI_VIS_C64;
  cfg->kernel_support = 8;
  cfg->oversample = 2;
  cfg->tlisi_tile = 32;
  cfg->grid_slots = 1;
  return TOI_OK;
}

toi_status toi_plan(const toi_config* cfg, void* cuda_stream, toi_plan_t* out) {
  if (!cfg || !out) return fail(nullptr, TOI_ERR_ARG, "cfg and out must be non-NULL");
  *out = nullptr;
  const toi_config c = *cfg;
  if (c.image_size < 64)
    return fail(nullptr, TOI_ERR_ARG, "image_size must be at least 64");
  if (c.image_size > 10240 || !toi::fft_length_supported(2 * c.image_size))
    return fail(nullptr, TOI_ERR_UNSUPPORTED,
                "image_size must be 2^a (64 ... 8192), 3 2^a (96 ... 6144) or 5 2^a (160 ... 10240)");
  if (!(c.cell_arcsec > 0.0) || !isfinite(c.cell_arcsec))
    return fail(nullptr, TOI_ERR_ARG, "cell_arcsec must be positive and finite");
  if (c.max_baselines < 1 || c.max_channels < 1)
    return fail(nullptr, TOI_ERR_ARG, "max_baselines and max_channels must be >= 1");
  if (!(c.n_pol == 1 || c.n_pol == 2 || c.n_pol == 4))
    return fail(nullptr, TOI_ERR_ARG, "n_pol must be 1, 2 or 4");
  if (!(c.vis_dtype == TOI_VIS_C64 || c.vis_dtype == TOI_VIS_C16_CHANSCALE))
    return fail(nullptr, TOI_ERR_ARG, "unknown vis_dtype");
  if (c.kernel_support != 8)
    return fail(nullptr, TOI_ERR_UNSUPPORTED, "kernel_support must be 8");
  if (c.oversample != 2)
    return fail(nullptr, TOI_ERR_UNSUPPORTED, "oversample must be 2");
  if (c.tlisi_tile < 1 || c.tlisi_tile > c.image_size || c.image_size % c.tlisi_tile != 0)
    return fail(nullptr, TOI_ERR_ARG, "tlisi_tile must divide image_size");
  if (c.grid_slots < 1 || c.grid_slots > 16)
    return fail(nullptr, TOI_ERR_ARG, "grid_slots must be in [1, 16]");
  if (c.grid_run != 0 && (c.grid_run < 8 || c.grid_run > 1024))
    return fail(nullptr, TOI_ERR_ARG, "grid_run must be 0 (automatic) or in [8, 1024]");
  if (c.batch_max < 0 || c.batch_max > 64)
    return fail(nullptr, TOI_ERR_ARG, "batch_max must be in [0, 64]");
  if (!(c.mode == 0 || c.mode == 2 || c.mode == 3))
    return fail(nullptr, TOI_ERR_ARG, "mode must be 2 (or 0) or 3");
  if (c.max_moments < 0 || c.max_moments > 1024)
    return fail(nullptr, TOI_ERR_ARG, "max_moments must be in [0, 1024]");
  if (c.mode == 3 && c.batch_max > 0)
    return fail(nullptr, TOI_ERR_UNSUPPORTED, "the batched path is 2-D only (mode 3 with batch_max > 0)");
  if (!(c.grid_rows == 0 || c.grid_rows == 4 || c.grid_rows == 8))
    return fail(nullptr, TOI_ERR_ARG, "grid_rows must be 0, 4 or 8");
  if (c.max_windows < 0 || c.max_windows > 256)
    return fail(nullptr, TOI_ERR_ARG, "max_windows must be in [0, 256]");
  if (c.reserved[0] != 0) return fail(nullptr, TOI_ERR_ARG, "reserved fields must be zero");
  if ((long long)c.max_baselines * c.max_channels * c.n_pol > (1LL << 40))
    return fail(nullptr, TOI_ERR_ARG, "max_baselines x max_channels too large");

  toi_plan_s* p = new (std::nothrow) toi_plan_s();
  if (!p) return fail(nullptr, TOI_ERR_OOM, "host allocation failed");
  p->cfg = c;
  if (p->cfg.mode == 0) p->cfg.mode = 2;
  if (p->cfg.max_moments == 0) p->cfg.max_moments = 64;
  p->N = c.image_size;
  p->G = c.oversample * c.image_size;
  p->W = c.kernel_support;
  p->T = c.tlisi_tile;
  p->nslot = c.grid_slots;
  p->beta_rad = c.cell_arcsec * toi::kArcsec;
  p->beta_es = 2.30 * c.kernel_support;
  p->stream = (cudaStream_t)cuda_stream;
  const int N = p->N, G = p->G;
  const int ntl = (N / p->T) * (N / p->T);
  toi_status st = TOI_OK;
  cudaError_t e = toi::fft_configure(G);
  if (e != cudaSuccess) { toi_status r = cuda_fail(nullptr, e, "configuring FFT kernels"); free_plan(p); return r; }
  {
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || p->nsm < 1) {
      toi_status r = cuda_fail(nullptr, e == cudaSuccess ? cudaErrorInvalidDevice : e, "device query");
      free_plan(p);
      return r;
    }
  }
  p->slots = new (std::nothrow) Slot[p->nslot];
  if (!p->slots) { free_plan(p); return fail(nullptr, TOI_ERR_OOM, "host allocation failed"); }
#define TOI_ALLOC(ptr, n, what) \
  if ((st = dev_alloc(p, &(ptr), (n), what)) != TOI_OK) { g_last_error = p->err; free_plan(p); return st; }
  for (int i = 0; i < p->nslot; ++i) {
    TOI_ALLOC(p->slots[i].grid, (size_t)(G / 2) * G, "grid slot");
    TOI_ALLOC(p->slots[i].snap, toi::SNAP_ALLOC, "snapshot record");
    TOI_ALLOC(p->slots[i].coef, (size_t)c.max_baselines, "baseline coefficients");
  }
  TOI_ALLOC(p->kch, (size_t)c.max_channels, "channel table");
  TOI_ALLOC(p->kf, (size_t)c.max_channels, "channel table (float pairs)");
  TOI_ALLOC(p->kch_sum, kpart_len(c.max_channels), "channel sums");
  TOI_ALLOC(p->bpart, bpart_len(c.max_baselines), "plane-fit partial sums");
  TOI_ALLOC(p->twiddle, (size_t)G, "FFT twiddles");
  TOI_ALLOC(p->corr, (size_t)N, "grid correction");
  TOI_ALLOC(p->fft_tmp, (size_t)(G / 2) * N, "FFT intermediate");
  TOI_ALLOC(p->tilted, (size_t)N * N, "tilted image");
  const int R = c.batch_max + 2 > 3 ? c.batch_max + 2 : 3;
  p->ring.assign(R, nullptr);
  for (int i = 0; i < R; ++i) TOI_ALLOC(p->ring[i], (size_t)N * N, "image ring");
  TOI_ALLOC(p->ring_max, (size_t)R, "ring maxima");
  TOI_ALLOC(p->tile_mom, (size_t)ntl * 5, "tile moments");
  TOI_ALLOC(p->d_status, 1, "status word");
  TOI_ALLOC(p->adj_scratch, toi::degrid_scratch_doubles(), "adjoint scratch");
  if (p->cfg.mode == 3) {
    TOI_ALLOC(p->moments, (size_t)2 * p->cfg.max_moments * N * N, "moment images");
    TOI_ALLOC(p->m3_dev, (size_t)16 + 256 * 32, "near-coplanar selection");
    TOI_ALLOC(p->m3_slabs, (size_t)p->cfg.max_moments, "slab centres");
    TOI_ALLOC(p->grid2, (size_t)(G / 2) * G, "second grid");
    e = cudaMallocHost((void**)&p->m3_host, sizeof(double) * 16);
    if (e != cudaSuccess) { toi_status r = cuda_fail(nullptr, e, "near-coplanar host buffer"); free_plan(p); return r; }
  }
  if (c.max_windows > 0) {
    const size_t nw = (size_t)c.max_windows;
    TOI_ALLOC(p->loc_k, (size_t)c.max_channels, "localisation channel table");
    TOI_ALLOC(p->loc_wq, (size_t)c.max_baselines * c.max_channels, "localisation sample weights");
    TOI_ALLOC(p->loc_coef, nw * c.max_baselines, "localisation coefficients");
    TOI_ALLOC(p->loc_win, nw, "localisation windows");
    TOI_ALLOC(p->loc_facets, nw * 64 * 64, "facet grids");
    TOI_ALLOC(p->loc_K, nw * 64 * 64, "facet adjoints");
    TOI_ALLOC(p->loc_gD, nw * TOI_LOC_WINDOW * TOI_LOC_WINDOW, "window cotangents");
    TOI_ALLOC(p->loc_corr, (size_t)TOI_LOC_WINDOW, "facet correction");
    TOI_ALLOC(p->loc_loss2, nw, "window losses");
    TOI_ALLOC(p->loc_dot, 1, "localisation dot");
    TOI_ALLOC(p->loc_part, toi::loc_part_doubles(c.max_baselines, c.max_windows, p->nsm),
              "localisation partial sums");
    TOI_ALLOC(p->loc_keys, (size_t)4096, "window selection keys");
    TOI_ALLOC(p->loc_tiles, nw, "selected tiles");
  }
  p->batch_rows = c.grid_rows ? c.grid_rows : toi::grid_default_rows(true);
  p->batch_max = c.batch_max;
  if (p->batch_max > 0) {
    const int B = p->batch_max;
    p->bslots = new (std::nothrow) Slot[B];
    if (!p->bslots) { free_plan(p); return fail(nullptr, TOI_ERR_OOM, "host allocation failed"); }
    for (int i = 0; i < B; ++i) {
      TOI_ALLOC(p->bslots[i].grid, (size_t)(G / 2) * G, "batch grid");
      TOI_ALLOC(p->bslots[i].snap, toi::SNAP_ALLOC, "batch snapshot record");
      TOI_ALLOC(p->bslots[i].coef, (size_t)c.max_baselines, "batch baseline coefficients");
    }
    TOI_ALLOC(p->b_kch, (size_t)B * c.max_channels, "batch channel tables");
    TOI_ALLOC(p->b_kf, (size_t)B * c.max_channels, "batch channel tables (float pairs)");
    TOI_ALLOC(p->b_kpart, (size_t)B * kpart_len(c.max_channels), "batch channel sums");
    TOI_ALLOC(p->b_bpart, (size_t)B * bpart_len(c.max_baselines), "batch plane-fit sums");
    TOI_ALLOC(p->b_fft_tmp, (size_t)B * (G / 2) * N, "batch FFT intermediates");
    TOI_ALLOC(p->b_tilted, (size_t)B * N * N, "batch tilted images");
    TOI_ALLOC(p->b_tile_mom, (size_t)B * ntl * 5, "batch tile moments");
    TOI_ALLOC(p->bentry_dev, (size_t)B, "batch table");
    TOI_ALLOC(p->bheader_dev, 1, "batch header");
    TOI_ALLOC(p->bqueue, 1, "gridder work counter");
    e = cudaMallocHost((void**)&p->bentry_host, sizeof(toi::BatchEntry) * B);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&p->bheader_host, sizeof(toi::BatchHeader));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->bcopied, cudaEventDisableTiming);
    if (e != cudaSuccess) { toi_status r = cuda_fail(nullptr, e, "batch tables"); free_plan(p); return r; }
    int dev = 0, nsm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = toi::grid_resident_blocks();
    if (e != cudaSuccess || per_sm < 1) {
      toi_status r = cuda_fail(nullptr, e == cudaSuccess ? cudaErrorInvalidConfiguration : e,
                               "persistent gridder occupancy");
      free_plan(p);
      return r;
    }
    p->grid_blocks = nsm * per_sm;
  }
#undef TOI_ALLOC
  // constant tables, computed in float64 on the host
  float2* tw = new float2[G];
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < G; ++k) {
    const double a = 2.0 * pi * (double)k / (double)G;
    tw[k] = make_float2((float)cos(a), (float)sin(a));
  }
  float* corr = new float[N];
  toi::es_fourier_table(N, G, p->W, p->beta_es, corr);
  e = cudaMemcpy(p->twiddle, tw, sizeof(float2) * G, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->corr, corr, sizeof(float) * N, cudaMemcpyHostToDevice);
  delete[] tw;
  delete[] corr;
  if (e == cudaSuccess && p->loc_corr) {
    float fc[TOI_LOC_WINDOW];
    toi::es_fourier_table(TOI_LOC_WINDOW, 2 * TOI_LOC_WINDOW, p->W, p->beta_es, fc);
    e = cudaMemcpy(p->loc_corr, fc, sizeof(fc), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(p->ring_max, 0, p->ring.size() * sizeof(unsigned int));
  for (size_t i = 0; i < p->ring.size() && e == cudaSuccess; ++i)
    e = cudaMemset(p->ring[i], 0, sizeof(float) * N * N);
  for (int i = 0; i < p->nslot && e == cudaSuccess; ++i)
    e = cudaMemset(p->slots[i].grid, 0, sizeof(float2) * (size_t)(G / 2) * G);
  for (int i = 0; i < p->batch_max && e == cudaSuccess; ++i)
    e = cudaMemset(p->bslots[i].grid, 0, sizeof(float2) * (size_t)(G / 2) * G);
  if (p->grid2 && e == cudaSuccess) e = cudaMemset(p->grid2, 0, sizeof(float2) * (size_t)(G / 2) * G);
  if (e != cudaSuccess) { toi_status r = cuda_fail(nullptr, e, "initialising plan tables"); free_plan(p); return r; }
  *out = p;
  return TOI_OK;
}

toi_status toi_plan_destroy(toi_plan_t plan) {
  if (!plan) return fail(nullptr, TOI_ERR_ARG, "plan is NULL");
  cudaStreamSynchronize(plan->stream);
  free_plan(plan);
  return TOI_OK;
}

toi_status toi_set_stream(toi_plan_t plan, void* cuda_stream) {
  if (!plan) return fail(nullptr, TOI_ERR_ARG, "plan is NULL");
  plan->stream = (cudaStream_t)cuda_stream;
  return TOI_OK;
}

// Host checks of one snapshot's arguments (toi_grid and the batch).
static toi_status check_snapshot(toi_plan_t p, const double* uvw_m, const double* freq_hz,
                                 const void* vis, const float* chan_scale, const float* weight,
                                 const uint8_t* flag, int32_t n_bl, int32_t n_ch) {
  if (!uvw_m || !freq_hz || !vis) return fail(p, TOI_ERR_ARG, "uvw, freq and vis must be non-NULL");
  if (n_bl < 1 || n_bl > p->cfg.max_baselines)
    return fail(p, TOI_ERR_ARG, "n_bl outside [1, max_baselines]");
  if (n_ch < 1 || n_ch > p->cfg.max_channels)
    return fail(p, TOI_ERR_ARG, "n_ch outside [1, max_channels]");
  const bool half = p->cfg.vis_dtype == TOI_VIS_C16_CHANSCALE;
  if (half && !chan_scale) return fail(p, TOI_ERR_ARG, "chan_scale required for float16 visibilities");
  if (!half && chan_scale) return fail(p, TOI_ERR_ARG, "chan_scale given for float32 visibilities");
  if (((uintptr_t)uvw_m & 7) || ((uintptr_t)freq_hz & 7) || ((uintptr_t)vis & (half ? 3 : 7)) ||
      ((uintptr_t)weight & 3) || ((uintptr_t)chan_scale & 3) ||
      (p->cfg.n_pol == 4 && ((uintptr_t)flag & 3)))
    return fail(p, TOI_ERR_ARG, "misaligned input pointer (element alignment; flags of 4 pols: 4 bytes)");
  return TOI_OK;
}

}  // extern "C"

namespace toi {
toi_status validate_snapshot(toi_plan_s* p, const toi_snapshot& sn) {
  return check_snapshot(p, sn.uvw, sn.freq, sn.vis, sn.chan_scale, sn.weight, sn.flag, sn.n_bl,
                        sn.n_ch);
}
}  // namespace toi

extern "C" {

toi_status toi_grid(toi_plan_t p, const double* uvw_m, const double* freq_hz, const void* vis,
                    const float* chan_scale, const float* weight, const uint8_t* flag,
                    int32_t n_bl, int32_t n_ch, int32_t slot) {
  if (!p) return fail(nullptr, TOI_ERR_ARG, "plan is NULL");
  const toi_status st = check_snapshot(p, uvw_m, freq_hz, vis, chan_scale, weight, flag, n_bl, n_ch);
  if (st != TOI_OK) return st;
  if (slot < 0 || slot >= p->nslot) return fail(p, TOI_ERR_ARG, "slot outside [0, grid_slots)");
  Slot& s = p->slots[slot];
  cudaError_t e;
  if (s.valid) {   // re-gridded before being imaged: start from zero again
    e = cudaMemsetAsync(s.grid, 0, sizeof(float2) * (size_t)(p->G / 2) * p->G, p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "toi_grid/clear");
  }
  e = toi::launch_prep(p, s, uvw_m, freq_hz, weight, flag, n_bl, n_ch);
  if (e != cudaSuccess) return cuda_fail(p, e, "toi_grid/prep");
  if (p->cfg.mode == 3) {
    e = toi::mode3_select(p, s, weight, flag, n_bl, n_ch);
    if (e == cudaErrorNotSupported)
      return fail(p, TOI_ERR_UNSUPPORTED,
                  "the snapshot needs N_slab K = " + std::to_string(s.m3.n_slab * s.m3.K) +
                      " moments, more than max_moments = " + std::to_string(p->cfg.max_moments));
    if (e != cudaSuccess) return cuda_fail(p, e, "toi_grid/mode3 selection");
    e = toi::mode3_moments(p, s, vis, chan_scale, weight, flag, n_bl, n_ch);
    if (e != cudaSuccess) return cuda_fail(p, e, "toi_grid/mode3 moments");
  } else {
    e = toi::launch_grid(p, s, freq_hz, vis, chan_scale, weight, flag, n_bl, n_ch);
    if (e != cudaSuccess) return cuda_fail(p, e, "toi_grid/grid");
  }
  s.uvw = uvw_m; s.freq = freq_hz; s.vis = vis; s.chan_scale = chan_scale;
  s.weight = weight; s.flag = flag; s.nbl = n_bl; s.nch = n_ch; s.valid = true;
  if (p->tilted_slot == slot) p->tilted_slot = -1;   // the slot holds another snapshot now
  return TOI_OK;
}

toi_status toi_image(toi_plan_t p, int32_t slot, float* image, double* snap_info) {
  if (!p) return fail(nullptr, TOI_ERR_ARG, "plan is NULL");
  if (slot < 0 || slot >= p->nslot) return fail(p, TOI_ERR_ARG, "slot outside [0, grid_slots)");
  Slot& s = p->slots[slot];
  if (!s.valid) return fail(p, TOI_ERR_ARG, "slot has not been gridded since its last toi_image");
  cudaError_t e = p->cfg.mode == 3 ? toi::launch_combine3(p, s) : toi::launch_fft(p, s);
  if (e != cudaSuccess) return cuda_fail(p, e, "toi_image/fft");
  s.valid = false;   // the row pass consumed (and cleared) the grid
  const int cur = ring_idx(p, p->nimg);
  const int prev1 = ring_idx(p, p->nimg - 1), prev2 = ring_idx(p, p->nimg - 2);
  e = toi::launch_reproject_moments(p, s, image, p->nimg >= 2, cur, prev1, prev2);
  if (e != cudaSuccess) return cuda_fail(p, e, "toi_image/reproject");
  if (snap_info) {
    e = cudaMemcpyAsync(snap_info, s.snap, sizeof(double) * toi::SNAP_LEN,
                        cudaMemcpyDeviceToDevice, p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "toi_image/snap_info");
  }
  p->nimg += 1;
  p->last_image = image ? image : p->ring[cur];
  p->fused_pending = true;
  p->tilted_slot = p->cfg.mode == 3 ? -1 : slot;
  return TOI_OK;
}


// ---------------------------------------------------------------- batch --

// Fill the host table for n snapshots: workspace of entry i, ring positions
// of stream images nimg + i, outputs, and the gridder's work split (runs[i]
// channels per lane).  Does not touch the plan's stream counters.
static void fill_batch_table(toi_plan_t p, const toi_snapshot* snaps, int n, float* tlisi,
                             const int* runs) {
  const int N = p->N, G = p->G;
  const int ntl = (N / p->T) * (N / p->T);
  long long up = 0;
  for (int i = 0; i < n; ++i) {
    const toi_snapshot& sn = snaps[i];
    toi::BatchEntry& e = p->bentry_host[i];
    Slot& sl = p->bslots[i];
    e.uvw = sn.uvw; e.freq = sn.freq; e.vis = sn.vis; e.chan_scale = sn.chan_scale;
    e.weight = sn.weight; e.flag = sn.flag; e.nbl = sn.n_bl; e.nch = sn.n_ch;
    e.grid = sl.grid; e.snap = sl.snap; e.coef = sl.coef;
    e.kch = p->b_kch + (size_t)i * p->cfg.max_channels;
    e.kf = p->b_kf + (size_t)i * p->cfg.max_channels;
    e.kpart = p->b_kpart + (size_t)i * kpart_len(p->cfg.max_channels);
    e.bpart = p->b_bpart + (size_t)i * bpart_len(p->cfg.max_baselines);
    e.fft_tmp = p->b_fft_tmp + (size_t)i * (G / 2) * N;
    e.tilted = p->b_tilted + (size_t)i * N * N;
    e.tile_mom = p->b_tile_mom + (size_t)i * ntl * 5;
    const long long t = p->nimg + i;
    const int cur = ring_idx(p, t), p1 = ring_idx(p, t - 1), p2 = ring_idx(p, t - 2);
    e.ring_cur = p->ring[cur]; e.ring_p1 = p->ring[p1]; e.ring_p2 = p->ring[p2];
    e.max_cur = p->ring_max + cur; e.max_p1 = p->ring_max + p1; e.max_p2 = p->ring_max + p2;
    e.image_out = sn.image;
    e.with_moments = t >= 2 ? 1 : 0;
    e.tlisi_out = (tlisi && t >= 2) ? tlisi + (size_t)i * ntl : nullptr;
    e.run = runs[i];
    const int rpw = toi::grid_runs_per_warp(p->batch_rows);
    e.nseg = (sn.n_ch + rpw * e.run - 1) / (rpw * e.run);
    e.up_begin = up;
    up += (long long)sn.n_bl * e.nseg;
  }
  long long mi = up;
  for (int i = 0; i < n; ++i) {
    toi::BatchEntry& e = p->bentry_host[i];
    e.mi_begin = mi;
    mi += (long long)e.nbl * e.nseg;
  }
  p->bheader_host->n = n;
  p->bheader_host->pad = 0;
  p->bheader_host->total_items = mi;
}

static int lane_run(toi_plan_t p, int nch) {
  if (p->cfg.grid_run > 0) return p->cfg.grid_run;
  const int t = p->tuned_run[toi::channel_bucket(nch)];
  return t > 0 ? t : toi::grid_default_run(nch, true);
}

toi_status toi_grid_lane_run(toi_plan_t p, int32_t n_ch, int32_t batched, int32_t* run,
                             int32_t* rows) {
  if (!p) return fail(nullptr, TOI_ERR_ARG, "plan is NULL");
  if (!run || !rows || n_ch < 1) return fail(p, TOI_ERR_ARG, "need run, rows and n_ch >= 1");
  if (batched) {
    *run = lane_run(p, n_ch);
    *rows = p->batch_rows;
  } else {
    *run = p->cfg.grid_run > 0 ? p->cfg.grid_run : toi::grid_default_run(n_ch, false);
    *rows = p->cfg.grid_rows ? p->cfg.grid_rows : toi::grid_default_rows(false);
  }
  return TOI_OK;
}

static toi_status check_batch(toi_plan_t p, const toi_snapshot* snaps, int32_t n) {
  if (!p) return fail(nullptr, TOI_ERR_ARG, "plan is NULL");
  if (p->batch_max < 1) return fail(p, TOI_ERR_ARG, "the plan was made with batch_max = 0");
  if (!snaps || n < 1 || n > p->batch_max)
    return fail(p, TOI_ERR_ARG, "need 1 <= n <= batch_max snapshots");
  if (p->T > 32) return fail(p, TOI_ERR_UNSUPPORTED, "the batched path needs tlisi_tile <= 32");
  for (int i = 0; i < n; ++i) {
    const toi_snapshot& sn = snaps[i];
    const toi_status st = check_snapshot(p, sn.uvw, sn.freq, sn.vis, sn.chan_scale, sn.weight,
                                         sn.flag, sn.n_bl, sn.n_ch);
    if (st != TOI_OK) return fail(p, st, "snapshot " + std::to_string(i) + ": " + p->err);
    if ((uintptr_t)sn.image & 3) return fail(p, TOI_ERR_ARG, "misaligned image pointer");
  }
  return TOI_OK;
}

toi_status toi_batch_prepare(toi_plan_t p, const toi_snapshot* snaps, int32_t n, float* tlisi,
                             int32_t* first_valid) {
  const toi_status st = check_batch(p, snaps, n);
  if (st != TOI_OK) return st;
  if ((uintptr_t)tlisi & 3) return fail(p, TOI_ERR_ARG, "misaligned tlisi pointer");
  // the previous batch's table must have been copied before it is rewritten
  if (p->bcopied_pending) {
    cudaError_t e = cudaEventSynchronize(p->bcopied);
    if (e != cudaSuccess) return cuda_fail(p, e, "toi_batch_prepare");
    p->bcopied_pending = false;
  }
  std::vector<int> runs(n);
  for (int i = 0; i < n; ++i) runs[i] = lane_run(p, snaps[i].n_ch);
  fill_batch_table(p, snaps, n, tlisi, runs.data());
  const long long t0 = p->nimg;
  if (first_valid) {
    const long long fv = 2 - t0;
    *first_valid = (int32_t)(fv < 0 ? 0 : (fv > n ? n : fv));
  }
  p->nimg += n;
  p->last_image = snaps[n - 1].image ? snaps[n - 1].image : p->ring[ring_idx(p, p->nimg - 1)];
  p->fused_pending = false;
  p->bn = n;
  return TOI_OK;
}

toi_status toi_batch_run(toi_plan_t p) {
  if (!p) return fail(nullptr, TOI_ERR_ARG, "plan is NULL");
  if (p->batch_max < 1) return fail(p, TOI_ERR_ARG, "the plan was made with batch_max = 0");
  if (p->bn < 1) return fail(p, TOI_ERR_ARG, "no batch prepared since the last toi_batch_run");
  cudaError_t e = cudaMemcpyAsync(p->bentry_dev, p->bentry_host,
                                  sizeof(toi::BatchEntry) * p->batch_max, cudaMemcpyHostToDevice,
                                  p->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->bheader_dev, p->bheader_host, sizeof(toi::BatchHeader),
                        cudaMemcpyHostToDevice, p->stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (e == cudaSuccess) e = cudaStreamIsCapturing(p->stream, &cap);
  if (e == cudaSuccess && cap == cudaStreamCaptureStatusNone) {
    e = cudaEventRecord(p->bcopied, p->stream);
    p->bcopied_pending = e == cudaSuccess;
  }
  if (e == cudaSuccess) e = toi::launch_prep_batch(p);
  if (e == cudaSuccess) e = toi::launch_grid_batch(p, p->cfg.vis_dtype == TOI_VIS_C16_CHANSCALE);
  if (e == cudaSuccess) e = toi::launch_fft_batch(p);
  if (e == cudaSuccess) e = toi::launch_finish_batch(p);
  p->bn = 0;
  if (e != cudaSuccess) return cuda_fail(p, e, "toi_batch_run");
  return TOI_OK;
}

toi_status toi_batch(toi_plan_t p, const toi_snapshot* snaps, int32_t n, float* tlisi,
                     int32_t* first_valid) {
  const toi_status st = toi_batch_prepare(p, snaps, n, tlisi, first_valid);
  if (st != TOI_OK) return st;
  return toi_batch_run(p);
}

toi_status toi_autotune(toi_plan_t p, const toi_snapshot* snaps, int32_t n, int32_t* runs_out,
                        double* us_out) {
  const toi_status st = check_batch(p, snaps, n);
  if (st != TOI_OK) return st;
  static const int kCand[] = {16, 32, 64, 128, 256};
  constexpr int kNc = (int)(sizeof(kCand) / sizeof(kCand[0]));
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (p->bcopied_pending && e == cudaSuccess) e = cudaEventSynchronize(p->bcopied);
  p->bcopied_pending = false;
  const long long nimg0 = p->nimg;
  // for each window split (8 or 4 rows per lane) the best run per bucket;
  // keep the split with the smallest total
  static const int kRows[] = {8, 4};
  double best_total = 1e300;
  int best_rows = p->batch_rows;
  int best_runs[4] = {0, 0, 0, 0};
  double best_us[4] = {0, 0, 0, 0};
  for (int ri = 0; ri < 2 && e == cudaSuccess; ++ri) {
    if (p->cfg.grid_rows && kRows[ri] != p->cfg.grid_rows) continue;
    p->batch_rows = kRows[ri];
    double total = 0.0;
    int runs_r[4] = {0, 0, 0, 0};
    double us_r[4] = {0, 0, 0, 0};
    for (int bucket = 0; bucket < 4 && e == cudaSuccess; ++bucket) {
      std::vector<toi_snapshot> sub;
      for (int i = 0; i < n; ++i)
        if (toi::channel_bucket(snaps[i].n_ch) == bucket) sub.push_back(snaps[i]);
      if (sub.empty()) continue;
      for (auto& sn : sub) sn.image = nullptr;
      double best = 1e300;
      int best_run = 0;
      for (int c = 0; c < kNc && e == cudaSuccess; ++c) {
        std::vector<int> runs(sub.size(), kCand[c]);
        fill_batch_table(p, sub.data(), (int)sub.size(), nullptr, runs.data());
        e = cudaMemcpyAsync(p->bentry_dev, p->bentry_host, sizeof(toi::BatchEntry) * p->batch_max,
                            cudaMemcpyHostToDevice, p->stream);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(p->bheader_dev, p->bheader_host, sizeof(toi::BatchHeader),
                              cudaMemcpyHostToDevice, p->stream);
        if (e == cudaSuccess) e = toi::launch_prep_batch(p);
        double t_min = 1e300;
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
          for (size_t i = 0; i < sub.size() && e == cudaSuccess; ++i)
            e = cudaMemsetAsync(p->bslots[i].grid, 0, sizeof(float2) * (size_t)(p->G / 2) * p->G,
                                p->stream);
          if (e == cudaSuccess) e = cudaEventRecord(a, p->stream);
          if (e == cudaSuccess) e = toi::launch_grid_batch(p, p->cfg.vis_dtype == TOI_VIS_C16_CHANSCALE);
          if (e == cudaSuccess) e = cudaEventRecord(b, p->stream);
          if (e == cudaSuccess) e = cudaEventSynchronize(b);
          float ms = 0.f;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
          if (e == cudaSuccess && ms < t_min) t_min = ms;
        }
        if (e == cudaSuccess && t_min < best) { best = t_min; best_run = kCand[c]; }
      }
      runs_r[bucket] = best_run;
      us_r[bucket] = best * 1e3 / (double)sub.size();
      total += best;
    }
    if (e == cudaSuccess && total < best_total) {
      best_total = total;
      best_rows = kRows[ri];
      for (int k = 0; k < 4; ++k) { best_runs[k] = runs_r[k]; best_us[k] = us_r[k]; }
    }
  }
  p->batch_rows = best_rows;
  for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
    if (!best_runs[k]) continue;
    p->tuned_run[k] = best_runs[k];
    if (runs_out) runs_out[k] = best_runs[k];
    if (us_out) us_out[k] = best_us[k];
  }
  // leave the batch grids zero and the stream position untouched
  for (int i = 0; i < p->batch_max && e == cudaSuccess; ++i)
    e = cudaMemsetAsync(p->bslots[i].grid, 0, sizeof(float2) * (size_t)(p->G / 2) * p->G, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  p->nimg = nimg0;
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_fail(p, e, "toi_autotune");
  return TOI_OK;
}

toi_status tlisi_update(toi_plan_t p, const float* image, float* tlisi, int32_t* valid) {
  if (!p) return fail(nullptr, TOI_ERR_ARG, "plan is NULL");
  if (!valid) return fail(p, TOI_ERR_ARG, "valid must be non-NULL");
  const bool fused = p->fused_pending && (image == nullptr || image == p->last_image);
  if (!fused) {
    if (!image) return fail(p, TOI_ERR_ARG, "no image given and none pending from toi_image");
    const int cur = ring_idx(p, p->nimg);
    const int prev1 = ring_idx(p, p->nimg - 1), prev2 = ring_idx(p, p->nimg - 2);
    cudaError_t e = toi::launch_ring_moments(p, image, cur, prev1, prev2, p->nimg >= 2);
    if (e != cudaSuccess) return cuda_fail(p, e, "tlisi_update/moments");
    p->nimg += 1;
  }
  p->fused_pending = false;
  if (p->nimg < 3) { *valid = 0; return TOI_OK; }
  if (!tlisi) return fail(p, TOI_ERR_ARG, "tlisi must be non-NULL");
  const int cur = ring_idx(p, p->nimg - 1);
  const int prev1 = ring_idx(p, p->nimg - 2), prev2 = ring_idx(p, p->nimg - 3);
  cudaError_t e = toi::launch_tlisi_finalize(p, tlisi, cur, prev1, prev2);
  if (e != cudaSuccess) return cuda_fail(p, e, "tlisi_update/finish");
  *valid = 1;
  return TOI_OK;
}

toi_status tlisi_reset(toi_plan_t p) {
  if (!p) return fail(nullptr, TOI_ERR_ARG, "plan is NULL");
  p->nimg = 0;
  p->fused_pending = false;
  p->last_image = nullptr;
  return TOI_OK;
}

toi_status tlisi_candidates(const float* cube, int32_t S, int32_t nty, int32_t ntx, int32_t tile,
                            int32_t mode, void* stream, double* threshold, int32_t* boxes,
                            int32_t* nboxes, int32_t max_boxes, double* scores) {
  if (!cube || !threshold || !nboxes) return fail(nullptr, TOI_ERR_ARG, "cube, threshold and nboxes must be non-NULL");
  if (S < 1 || nty < 1 || ntx < 1 || tile < 1) return fail(nullptr, TOI_ERR_ARG, "S, nty, ntx, tile must be >= 1");
  if ((long long)nty * ntx > toi::kMaxCandTiles)
    return fail(nullptr, TOI_ERR_ARG, "more than 131072 tiles (the labelling runs in one block)");
  if (mode != TOI_CAND_PERIODIC && mode != TOI_CAND_NONPERIODIC) return fail(nullptr, TOI_ERR_ARG, "unknown mode");
  if (max_boxes < 0 || (max_boxes > 0 && !boxes)) return fail(nullptr, TOI_ERR_ARG, "boxes must hold max_boxes entries");
  cudaStream_t st = (cudaStream_t)stream;
  const int nt = nty * ntx;
  // work, boxes, and (periodic) the centred series, each 256-byte aligned
  const size_t work = toi::candidates_scratch_bytes(S, nt);
  const size_t box_bytes = (sizeof(int) * 4 * (size_t)(max_boxes + 1) + 255) & ~(size_t)255;
  const size_t xoff = ((work + 255) & ~(size_t)255) + box_bytes;
  const size_t bytes = xoff + (mode == TOI_CAND_PERIODIC ? toi::candidates_centre_bytes(S, nt) : 0);
  void* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, bytes, st);
  if (e != cudaSuccess) { cudaGetLastError(); return cuda_fail(nullptr, e, "tlisi_candidates/scratch"); }
  int* boxes_dev = (int*)((char*)scratch + ((work + 255) & ~(size_t)255));
  double* xbuf = mode == TOI_CAND_PERIODIC ? (double*)((char*)scratch + xoff) : nullptr;
  double* thr_dev = nullptr;
  int* nbox_dev = nullptr;
  e = toi::candidates_run(cube, S, nty, ntx, tile, mode, st, scratch, scores, max_boxes, boxes_dev,
                          &thr_dev, &nbox_dev, xbuf);
  int nb = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(threshold, thr_dev, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nb, nbox_dev, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && max_boxes > 0 && nb > 0) {
    const int ncopy = nb < max_boxes ? nb : max_boxes;
    e = cudaMemcpyAsync(boxes, boxes_dev, sizeof(int) * 4 * (size_t)ncopy, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFreeAsync(scratch, st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "tlisi_candidates");
  *nboxes = nb;
  return TOI_OK;
}

toi_status toi_mode3_info(toi_plan_t p, int32_t slot, double* info) {
  if (!p || !info) return fail(p, TOI_ERR_ARG, "plan and info must be non-NULL");
  if (p->cfg.mode != 3) return fail(p, TOI_ERR_ARG, "the plan is not in mode 3");
  if (slot < 0 || slot >= p->nslot) return fail(p, TOI_ERR_ARG, "slot outside [0, grid_slots)");
  const toi::Mode3Plan& m = p->slots[slot].m3;
  if (!p->slots[slot].uvw) return fail(p, TOI_ERR_ARG, "slot has not been gridded");
  info[0] = m.n_slab; info[1] = m.K; info[2] = m.phi; info[3] = m.alpha_slab;
  info[4] = m.dr3; info[5] = m.r3min; info[6] = m.r3max; info[7] = m.t3max;
  return TOI_OK;
}

// NULL counts as aligned
static bool aligned(const void* ptr, uintptr_t a) { return ((uintptr_t)ptr & (a - 1)) == 0; }

toi_status toi_degrid_backward(toi_plan_t p, int32_t slot, const float* grad_image,
                               const float* image, void* grad_sample, void* grad_vis,
                               float* grad_weight) {
  if (!p) return fail(nullptr, TOI_ERR_ARG, "plan is NULL");
  if (slot < 0 || slot >= p->nslot) return fail(p, TOI_ERR_ARG, "slot outside [0, grid_slots)");
  if (!grad_image) return fail(p, TOI_ERR_ARG, "grad_image must be non-NULL");
  if (!grad_sample && !grad_vis && !grad_weight)
    return fail(p, TOI_ERR_ARG, "at least one of grad_sample, grad_vis, grad_weight is needed");
  if (grad_weight && !image) return fail(p, TOI_ERR_ARG, "grad_weight needs the image of toi_image");
  Slot& s = p->slots[slot];
  if (!s.uvw) return fail(p, TOI_ERR_ARG, "slot has not been gridded");
  if (p->cfg.mode == 3) return fail(p, TOI_ERR_UNSUPPORTED, "toi_degrid_backward is 2-D only");
  if (!aligned(grad_image, 4) || !aligned(image, 4) || !aligned(grad_sample, 8) ||
      !aligned(grad_vis, 8) || !aligned(grad_weight, 4))
    return fail(p, TOI_ERR_ARG, "misaligned pointer (element alignment)");
  cudaError_t e = toi::launch_degrid_backward(p, s, grad_image, image,
                                              reinterpret_cast<float2*>(grad_sample),
                                              reinterpret_cast<float2*>(grad_vis), grad_weight);
  // the adjoint used the slot's grid memory (and left it cleared) and the
  // tilted image as workspace
  s.valid = false;
  p->tilted_slot = -1;
  if (e != cudaSuccess) return cuda_fail(p, e, "toi_degrid_backward");
  return TOI_OK;
}

static toi_status localise_checks(toi_plan_t p, int32_t slot, int32_t n_win) {
  if (!p) return fail(nullptr, TOI_ERR_ARG, "plan is NULL");
  if (slot < 0 || slot >= p->nslot) return fail(p, TOI_ERR_ARG, "slot outside [0, grid_slots)");
  if (p->cfg.mode == 3) return fail(p, TOI_ERR_UNSUPPORTED, "localisation is 2-D only");
  if (p->cfg.max_windows < 1) return fail(p, TOI_ERR_ARG, "the plan has max_windows = 0");
  if (n_win < 1 || n_win > p->cfg.max_windows)
    return fail(p, TOI_ERR_ARG, "n_win must be in [1, max_windows]");
  if (!p->slots[slot].uvw) return fail(p, TOI_ERR_ARG, "slot has not been gridded");
  if (p->tilted_slot != slot)
    return fail(p, TOI_ERR_ARG, "the tilted image is not this slot's (toi_image(slot) must be "
                                "the last image call)");
  return TOI_OK;
}

toi_status toi_localise_seed(toi_plan_t p, int32_t slot, const float* tlisi, int32_t n_win,
                             int32_t* win, double* src) {
  toi_status st = localise_checks(p, slot, n_win);
  if (st != TOI_OK) return st;
  if (!tlisi || !win || !src) return fail(p, TOI_ERR_ARG, "tlisi, win and src must be non-NULL");
  if (!aligned(tlisi, 4) || !aligned(win, 4) || !aligned(src, 8))
    return fail(p, TOI_ERR_ARG, "misaligned pointer (element alignment)");
  const int nt = p->N / p->T;
  if (nt * nt > toi::loc_seed_max_tiles(n_win))
    return fail(p, TOI_ERR_UNSUPPORTED, "too many tLISI tiles for this many windows");
  const int tok = toi::prof_begin(p, toi::PROF_LOCALISE, 3);
  cudaError_t e = toi::launch_localise_seed(p, p->slots[slot], tlisi, n_win, win, src);
  toi::prof_end(p, tok);
  if (e != cudaSuccess) return cuda_fail(p, e, "toi_localise_seed");
  return TOI_OK;
}

toi_status toi_localise(toi_plan_t p, int32_t slot, int32_t n_win, const int32_t* win,
                        const double* src, float* model, double* loss, double* grad_src,
                        float* grad_weight) {
  toi_status st = localise_checks(p, slot, n_win);
  if (st != TOI_OK) return st;
  if (!win || !src) return fail(p, TOI_ERR_ARG, "win and src must be non-NULL");
  if (!aligned(win, 4) || !aligned(src, 8) || !aligned(model, 4) || !aligned(loss, 8) ||
      !aligned(grad_src, 8) || !aligned(grad_weight, 4))
    return fail(p, TOI_ERR_ARG, "misaligned pointer (element alignment)");
  Slot& s = p->slots[slot];
  const int tok = toi::prof_begin(p, toi::PROF_LOCALISE, grad_weight ? 13 : 7);
  cudaError_t e = toi::launch_localise(p, s, n_win, win, src, model, loss, grad_src, grad_weight);
  toi::prof_end(p, tok);
  if (grad_weight) {
    s.valid = false;          // the grid memory held the adjoint (cleared again)
    p->tilted_slot = -1;      // the tilted image held the cotangent
  }
  if (e != cudaSuccess) return cuda_fail(p, e, "toi_localise");
  return TOI_OK;
}

toi_status toi_plan_buffer(toi_plan_t p, int32_t which, int32_t slot, void* dst,
                           int64_t dst_bytes, int64_t* nbytes) {
  if (!p || !nbytes) return fail(p, TOI_ERR_ARG, "plan and nbytes must be non-NULL");
  if (slot < 0 || slot >= p->nslot) return fail(p, TOI_ERR_ARG, "slot outside [0, grid_slots)");
  const int64_t NN = (int64_t)p->N * p->N;
  const void* src = nullptr;
  switch (which) {
    case 0: src = p->slots[slot].grid; *nbytes = (int64_t)(p->G / 2) * p->G * 8; break;
    case 1: src = p->tilted; *nbytes = NN * 4; break;
    case 2: src = p->slots[slot].snap; *nbytes = toi::SNAP_LEN * 8; break;
    case 3: src = p->ring[ring_idx(p, p->nimg - 1)]; *nbytes = NN * 4; break;
    default: return fail(p, TOI_ERR_ARG, "unknown buffer");
  }
  if (dst) {
    if (dst_bytes < 0) return fail(p, TOI_ERR_ARG, "dst_bytes must be >= 0");
    const size_t n = (size_t)(dst_bytes < *nbytes ? dst_bytes : *nbytes);
    cudaError_t e = cudaMemcpyAsync(dst, src, n, cudaMemcpyDefault, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "toi_plan_buffer");
  }
  return TOI_OK;
}

toi_status toi_profile_enable(toi_plan_t p, int32_t enable) {
  if (!p) return fail(nullptr, TOI_ERR_ARG, "plan is NULL");
  if (enable && p->prof.ev.empty()) {
    p->prof.ev.resize(4096);
    for (auto& ev : p->prof.ev) {
      cudaError_t e = cudaEventCreate(&ev);
      if (e != cudaSuccess) return cuda_fail(p, e, "toi_profile_enable");
    }
  }
  p->prof.on = enable != 0;
  return TOI_OK;
}

toi_status toi_profile_read(toi_plan_t p, double* ms, int64_t* launches, int32_t nstages) {
  if (!p || nstages < 0) return fail(p, TOI_ERR_ARG, "bad arguments");
  toi::ProfState& q = p->prof;
  if (q.used > 0) {
    cudaError_t e = cudaEventSynchronize(q.ev[q.used - 1]);
    if (e != cudaSuccess) return cuda_fail(p, e, "toi_profile_read");
    for (size_t i = 0; i < q.stage_of_pair.size(); ++i) {
      float t = 0.f;
      cudaEventElapsedTime(&t, q.ev[2 * i], q.ev[2 * i + 1]);
      q.ms[q.stage_of_pair[i]] += t;
    }
    q.stage_of_pair.clear();
    q.used = 0;
  }
  for (int i = 0; i < nstages && i < toi::PROF_NSTAGE; ++i) {
    if (ms) ms[i] = q.ms[i];
    if (launches) launches[i] = q.launches[i];
    q.ms[i] = 0.0;
    q.launches[i] = 0;
  }
  return TOI_OK;
}

toi_status toi_sync_status(toi_plan_t p) {
  if (!p) return fail(nullptr, TOI_ERR_ARG, "plan is NULL");
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(p, e, "toi_sync_status");
  int st = 0;
  e = cudaMemcpy(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(p, e, "toi_sync_status");
  if (st == TOI_DEV_EMPTY) return fail(p, TOI_ERR_EMPTY, "no sample with positive weight");
  if (st == TOI_DEV_RANGE)
    return fail(p, TOI_ERR_RANGE, "kernel footprint outside the grid, non-monotone frequencies or bin overflow");
  return TOI_OK;
}

}  // extern "C"
