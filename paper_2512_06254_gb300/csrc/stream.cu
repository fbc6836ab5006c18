// Streaming runtime (toi_stream_*): the per-snapshot pipeline of Sections
// 4.1-4.4 with one CUDA stream per device stage, interlocked by events:
//   data_read    the caller fills pinned host buffers (toi_stream_input_free
//                says when a snapshot's buffers may be refilled)
//   copy_gpu     host -> device into a depth-2 staging ring; the
//                visibilities are split by baseline over n_copy copy streams
//   gridding     S1-S3 into grid slot s mod 3          (depth-3 grid ring)
//   fft          S4-S5 into tilted image s mod 3 (the row pass clears the slot)
//   interpolate  S6 into image ring slot s mod 5 (depth-5 image ring), fused
//                with the S7 tile moments of the window (s - 2, s - 1, s)
//   tlisi        S7 finish into device row s mod 2
//   copy_cpu     device -> pinned host row ring (host_depth rows)
//   data_write   the caller (toi_stream_pop)
// A ring slot is reused only after an event of its last reader, enqueued as
// a stream wait, so the host never waits inside toi_stream_push:
//   staging s mod 2          <- gridding(s - 2)     (prep and gridding read it)
//   grid slot, tilted s mod 3 <- interpolate(s - 3) (the snapshot record and
//                                                    tilted image of s - 3)
//   image ring s mod 5, its maximum and tile moments
//                            <- tlisi(s - 3)        (the last window reading
//                                                    image s - 5 ends at s - 3)
//   device row s mod 2       <- copy_cpu(s - 2)
// The depths are the paper's: 3 grids because the FFT works in place, 5
// images because tLISI needs the last three.
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "toi_internal.cuh"

namespace toi {
toi_status validate_snapshot(toi_plan_s* p, const toi_snapshot& sn);
cudaError_t launch_reproject_ring(toi_plan_s* p, Slot& s, const float* tilted, float* cur,
                                  const float* prev1, const float* prev2, bool with_moments,
                                  double* tile_mom, unsigned int* max_cur);
cudaError_t launch_tlisi_rows(toi_plan_s* p, const double* tile_mom, const unsigned int* ring_max,
                              int cur, int prev1, int prev2, float* out);
}  // namespace toi

using toi::Slot;

namespace {

constexpr int kStage = 2;     // staging (and device tLISI row) ring depth
constexpr int kGrids = 3;     // grid / tilted ring depth
constexpr int kImages = 5;    // image ring depth

toi_status sfail(toi_plan_s* p, toi_status st, const std::string& msg) {
  p->err = msg;
  return st;
}

toi_status scuda(toi_plan_s* p, cudaError_t e, const char* where) {
  return sfail(p, TOI_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

struct Staging {
  double* uvw = nullptr;
  double* freq = nullptr;
  void* vis = nullptr;
  float* chan_scale = nullptr;
  float* weight = nullptr;
  uint8_t* flag = nullptr;
};

// Temporarily route the plan's launches to one stage's stream.
struct OnStream {
  toi_plan_s* p;
  cudaStream_t old;
  OnStream(toi_plan_s* p_, cudaStream_t s) : p(p_), old(p_->stream) { p->stream = s; }
  ~OnStream() { p->stream = old; }
};

}  // namespace

struct toi_stream_s {
  toi_plan_s* plan = nullptr;
  int host_depth = 0, n_copy = 1, ntl = 0;
  bool weights = false;
  // stage streams
  std::vector<cudaStream_t> copy;   // [n_copy]
  cudaStream_t grid = nullptr, fft = nullptr, interp = nullptr, tlisi = nullptr, out = nullptr;
  // rings
  Staging stage[kStage];
  float* tilted[kGrids] = {};
  float* image[kImages] = {};
  unsigned int* ring_max = nullptr;            // [kImages]
  double* tile_mom = nullptr;                  // [kImages][ntl][5]
  float* dev_row[kStage] = {};
  float* host_rows = nullptr;                  // pinned [host_depth][ntl]
  // events (one per ring position of the stage that records them)
  std::vector<cudaEvent_t> ev_copied;          // [kStage][n_copy]
  cudaEvent_t ev_gridded[kStage] = {};          // gridding of the staging slot's snapshot
  cudaEvent_t ev_ffted[kGrids] = {};
  cudaEvent_t ev_interp[kGrids] = {};           // interpolate of the grid slot's snapshot
  cudaEvent_t ev_tlisi[kImages] = {};           // indexed by snapshot mod 5
  cudaEvent_t ev_row_out[kStage] = {};          // copy_cpu of the device row
  std::vector<cudaEvent_t> ev_host_row;         // [host_depth]
  long long pushed = 0, rows = 0, popped = 0;
};

namespace {

void destroy(toi_stream_s* st) {
  if (!st) return;
  for (cudaStream_t c : st->copy) if (c) cudaStreamSynchronize(c);
  for (cudaStream_t c : {st->grid, st->fft, st->interp, st->tlisi, st->out})
    if (c) cudaStreamSynchronize(c);
  for (int i = 0; i < kStage; ++i) {
    Staging& g = st->stage[i];
    cudaFree(g.uvw); cudaFree(g.freq); cudaFree(g.vis); cudaFree(g.chan_scale);
    cudaFree(g.weight); cudaFree(g.flag);
    cudaFree(st->dev_row[i]);
    if (st->ev_gridded[i]) cudaEventDestroy(st->ev_gridded[i]);
    if (st->ev_row_out[i]) cudaEventDestroy(st->ev_row_out[i]);
  }
  for (int i = 0; i < kGrids; ++i) {
    cudaFree(st->tilted[i]);
    if (st->ev_ffted[i]) cudaEventDestroy(st->ev_ffted[i]);
    if (st->ev_interp[i]) cudaEventDestroy(st->ev_interp[i]);
  }
  for (int i = 0; i < kImages; ++i) {
    cudaFree(st->image[i]);
    if (st->ev_tlisi[i]) cudaEventDestroy(st->ev_tlisi[i]);
  }
  cudaFree(st->ring_max);
  cudaFree(st->tile_mom);
  cudaFreeHost(st->host_rows);
  for (cudaEvent_t e : st->ev_copied) if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : st->ev_host_row) if (e) cudaEventDestroy(e);
  for (cudaStream_t c : st->copy) if (c) cudaStreamDestroy(c);
  for (cudaStream_t c : {st->grid, st->fft, st->interp, st->tlisi, st->out})
    if (c) cudaStreamDestroy(c);
  delete st;
}

template <typename T>
cudaError_t dalloc(T** ptr, size_t n) {
  return cudaMalloc((void**)ptr, sizeof(T) * (n ? n : 1));
}

}  // namespace

extern "C" {

toi_status toi_stream_open(toi_plan_t p, int32_t host_depth, int32_t n_copy, int32_t with_weights,
                           toi_stream_t* out) {
  if (!p || !out) return TOI_ERR_ARG;
  *out = nullptr;
  if (p->cfg.mode == 3) return sfail(p, TOI_ERR_UNSUPPORTED, "the streaming runtime is 2-D only");
  if (p->nslot < kGrids) return sfail(p, TOI_ERR_ARG, "the streaming runtime needs grid_slots >= 3");
  if (host_depth < 1 || host_depth > 4096) return sfail(p, TOI_ERR_ARG, "host_depth outside [1, 4096]");
  if (n_copy < 1 || n_copy > 16) return sfail(p, TOI_ERR_ARG, "n_copy outside [1, 16]");
  toi_stream_s* st = new (std::nothrow) toi_stream_s();
  if (!st) return sfail(p, TOI_ERR_OOM, "host allocation failed");
  st->plan = p;
  st->host_depth = host_depth;
  st->n_copy = n_copy;
  st->weights = with_weights != 0;
  const int N = p->N;
  const int nt = N / p->T;
  st->ntl = nt * nt;
  const size_t nbl = p->cfg.max_baselines, nch = p->cfg.max_channels, npol = p->cfg.n_pol;
  const bool half = p->cfg.vis_dtype == TOI_VIS_C16_CHANSCALE;
  cudaError_t e = cudaSuccess;
  st->copy.assign(n_copy, nullptr);
  for (int i = 0; i < n_copy && e == cudaSuccess; ++i)
    e = cudaStreamCreateWithFlags(&st->copy[i], cudaStreamNonBlocking);
  for (cudaStream_t* c : {&st->grid, &st->fft, &st->interp, &st->tlisi, &st->out})
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(c, cudaStreamNonBlocking);
  for (int i = 0; i < kStage && e == cudaSuccess; ++i) {
    Staging& g = st->stage[i];
    e = dalloc(&g.uvw, nbl * 3);
    if (e == cudaSuccess) e = dalloc(&g.freq, nch);
    if (e == cudaSuccess) e = cudaMalloc(&g.vis, nbl * nch * npol * (half ? 4 : 8));
    if (e == cudaSuccess && half) e = dalloc(&g.chan_scale, nch);
    if (e == cudaSuccess && st->weights) e = dalloc(&g.weight, nbl * nch * npol);
    if (e == cudaSuccess) e = dalloc(&g.flag, nbl * nch * npol);
    if (e == cudaSuccess) e = dalloc(&st->dev_row[i], (size_t)st->ntl);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st->ev_gridded[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st->ev_row_out[i], cudaEventDisableTiming);
  }
  for (int i = 0; i < kGrids && e == cudaSuccess; ++i) {
    e = dalloc(&st->tilted[i], (size_t)N * N);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st->ev_ffted[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st->ev_interp[i], cudaEventDisableTiming);
  }
  for (int i = 0; i < kImages && e == cudaSuccess; ++i) {
    e = dalloc(&st->image[i], (size_t)N * N);
    if (e == cudaSuccess) e = cudaMemset(st->image[i], 0, sizeof(float) * N * N);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st->ev_tlisi[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = dalloc(&st->ring_max, (size_t)kImages);
  if (e == cudaSuccess) e = cudaMemset(st->ring_max, 0, sizeof(unsigned int) * kImages);
  if (e == cudaSuccess) e = dalloc(&st->tile_mom, (size_t)kImages * st->ntl * 5);
  if (e == cudaSuccess)
    e = cudaMallocHost((void**)&st->host_rows, sizeof(float) * (size_t)host_depth * st->ntl);
  st->ev_copied.assign((size_t)kStage * n_copy, nullptr);
  for (auto& ev : st->ev_copied)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  st->ev_host_row.assign(host_depth, nullptr);
  for (auto& ev : st->ev_host_row)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  // the grid ring must start cleared (a slot gridded but never imaged)
  for (int i = 0; i < kGrids && e == cudaSuccess; ++i) {
    Slot& sl = p->slots[i];
    if (sl.valid) {
      e = cudaMemset(sl.grid, 0, sizeof(float2) * (size_t)(p->G / 2) * p->G);
      sl.valid = false;
    }
  }
  if (e != cudaSuccess) {
    const toi_status r = scuda(p, e, "toi_stream_open");
    cudaGetLastError();
    destroy(st);
    return r;
  }
  *out = st;
  return TOI_OK;
}

toi_status toi_stream_push(toi_stream_t st, const toi_snapshot* snap, int64_t* index) {
  if (!st || !snap) return TOI_ERR_ARG;
  toi_plan_s* p = st->plan;
  const toi_snapshot& sn = *snap;
  toi_status vs = toi::validate_snapshot(p, sn);
  if (vs != TOI_OK) return vs;
  if (sn.weight && !st->weights) return sfail(p, TOI_ERR_ARG, "weights given to a stream opened without");
  const long long s = st->pushed;
  // the tLISI row this snapshot completes goes to host row (s - 2) mod host_depth
  if (s >= 2 && (s - 2) - st->popped >= st->host_depth)
    return sfail(p, TOI_ERR_ARG, "the host row ring is full: toi_stream_pop first");
  const bool half = p->cfg.vis_dtype == TOI_VIS_C16_CHANSCALE;
  const size_t npol = p->cfg.n_pol;
  const int is = (int)(s % kStage), ig = (int)(s % kGrids), ii = (int)(s % kImages);
  Staging& g = st->stage[is];
  cudaError_t e = cudaSuccess;

  // copy_gpu: staging slot free once gridding(s - 2) is done
  for (int c = 0; c < st->n_copy && e == cudaSuccess; ++c)
    if (s >= kStage) e = cudaStreamWaitEvent(st->copy[c], st->ev_gridded[is], 0);
  const size_t rec = npol * (half ? 4 : 8);
  const size_t nch = sn.n_ch;
  cudaStream_t c0 = st->copy[0];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g.uvw, sn.uvw, sizeof(double) * 3 * sn.n_bl, cudaMemcpyHostToDevice, c0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g.freq, sn.freq, sizeof(double) * nch, cudaMemcpyHostToDevice, c0);
  if (e == cudaSuccess && half)
    e = cudaMemcpyAsync(g.chan_scale, sn.chan_scale, sizeof(float) * nch, cudaMemcpyHostToDevice, c0);
  for (int c = 0; c < st->n_copy && e == cudaSuccess; ++c) {
    const size_t b0 = (size_t)sn.n_bl * c / st->n_copy, b1 = (size_t)sn.n_bl * (c + 1) / st->n_copy;
    if (b1 <= b0) continue;
    const size_t off = b0 * nch * npol, cnt = (b1 - b0) * nch * npol;
    e = cudaMemcpyAsync((char*)g.vis + off * (rec / npol), (const char*)sn.vis + off * (rec / npol),
                        cnt * (rec / npol), cudaMemcpyHostToDevice, st->copy[c]);
    if (e == cudaSuccess && sn.flag)
      e = cudaMemcpyAsync(g.flag + off, sn.flag + off, cnt, cudaMemcpyHostToDevice, st->copy[c]);
    if (e == cudaSuccess && sn.weight)
      e = cudaMemcpyAsync(g.weight + off, sn.weight + off, sizeof(float) * cnt,
                          cudaMemcpyHostToDevice, st->copy[c]);
  }
  for (int c = 0; c < st->n_copy && e == cudaSuccess; ++c)
    e = cudaEventRecord(st->ev_copied[(size_t)is * st->n_copy + c], st->copy[c]);
  if (e != cudaSuccess) return scuda(p, e, "toi_stream_push/copy_gpu");

  // gridding: the copies of s; grid slot free once interpolate(s - 3) is done
  for (int c = 0; c < st->n_copy && e == cudaSuccess; ++c)
    e = cudaStreamWaitEvent(st->grid, st->ev_copied[(size_t)is * st->n_copy + c], 0);
  if (e == cudaSuccess && s >= kGrids) e = cudaStreamWaitEvent(st->grid, st->ev_interp[ig], 0);
  Slot& slot = p->slots[ig];
  {
    OnStream on(p, st->grid);
    if (e == cudaSuccess)
      e = toi::launch_prep(p, slot, g.uvw, g.freq, sn.weight ? g.weight : nullptr,
                           sn.flag ? g.flag : nullptr, sn.n_bl, sn.n_ch);
    if (e == cudaSuccess)
      e = toi::launch_grid(p, slot, g.freq, g.vis, half ? g.chan_scale : nullptr,
                           sn.weight ? g.weight : nullptr, sn.flag ? g.flag : nullptr, sn.n_bl,
                           sn.n_ch);
  }
  if (e == cudaSuccess) e = cudaEventRecord(st->ev_gridded[is], st->grid);
  if (e != cudaSuccess) return scuda(p, e, "toi_stream_push/gridding");
  slot.uvw = nullptr;            // the staging buffers are not the caller's: no adjoint
  slot.valid = false;
  if (p->tilted_slot == ig) p->tilted_slot = -1;

  // fft: after gridding(s); tilted slot free once interpolate(s - 3) is done
  e = cudaStreamWaitEvent(st->fft, st->ev_gridded[is], 0);
  if (e == cudaSuccess && s >= kGrids) e = cudaStreamWaitEvent(st->fft, st->ev_interp[ig], 0);
  {
    OnStream on(p, st->fft);
    if (e == cudaSuccess) e = toi::launch_fft_to(p, slot, st->tilted[ig]);
  }
  if (e == cudaSuccess) e = cudaEventRecord(st->ev_ffted[ig], st->fft);
  if (e != cudaSuccess) return scuda(p, e, "toi_stream_push/fft");

  // interpolate (+ tile moments): after fft(s); image slot, its maximum and
  // moments free once tlisi(s - 3) is done
  e = cudaStreamWaitEvent(st->interp, st->ev_ffted[ig], 0);
  if (e == cudaSuccess && s >= 3) e = cudaStreamWaitEvent(st->interp, st->ev_tlisi[(s - 3) % kImages], 0);
  const int i1 = (int)((s + kImages - 1) % kImages), i2 = (int)((s + kImages - 2) % kImages);
  {
    OnStream on(p, st->interp);
    if (e == cudaSuccess)
      e = toi::launch_reproject_ring(p, slot, st->tilted[ig], st->image[ii], st->image[i1],
                                     st->image[i2], s >= 2, st->tile_mom + (size_t)ii * st->ntl * 5,
                                     st->ring_max + ii);
  }
  if (e == cudaSuccess) e = cudaEventRecord(st->ev_interp[ig], st->interp);
  if (e != cudaSuccess) return scuda(p, e, "toi_stream_push/interpolate");

  // tlisi and copy_cpu (from the third snapshot on)
  if (s >= 2) {
    const long long r = s - 2;
    const int ir = (int)(r % kStage), ih = (int)(r % st->host_depth);
    e = cudaStreamWaitEvent(st->tlisi, st->ev_interp[ig], 0);
    if (e == cudaSuccess && r >= kStage) e = cudaStreamWaitEvent(st->tlisi, st->ev_row_out[ir], 0);
    {
      OnStream on(p, st->tlisi);
      if (e == cudaSuccess)
        e = toi::launch_tlisi_rows(p, st->tile_mom + (size_t)ii * st->ntl * 5, st->ring_max, ii,
                                   i1, i2, st->dev_row[ir]);
    }
    if (e == cudaSuccess) e = cudaEventRecord(st->ev_tlisi[ii], st->tlisi);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st->out, st->ev_tlisi[ii], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(st->host_rows + (size_t)ih * st->ntl, st->dev_row[ir],
                          sizeof(float) * st->ntl, cudaMemcpyDeviceToHost, st->out);
    if (e == cudaSuccess) e = cudaEventRecord(st->ev_row_out[ir], st->out);
    if (e == cudaSuccess) e = cudaEventRecord(st->ev_host_row[ih], st->out);
    if (e != cudaSuccess) return scuda(p, e, "toi_stream_push/tlisi");
    st->rows = r + 1;
  } else {
    // no window yet: mark the image slot's tLISI event as passed on this stream
    e = cudaStreamWaitEvent(st->tlisi, st->ev_interp[ig], 0);
    if (e == cudaSuccess) e = cudaEventRecord(st->ev_tlisi[ii], st->tlisi);
    if (e != cudaSuccess) return scuda(p, e, "toi_stream_push/tlisi");
  }
  st->pushed = s + 1;
  if (index) *index = s;
  return TOI_OK;
}

toi_status toi_stream_input_free(toi_stream_t st, int64_t index, int32_t wait, int32_t* is_free) {
  if (!st || !is_free) return TOI_ERR_ARG;
  toi_plan_s* p = st->plan;
  *is_free = 0;
  if (index < 0 || index >= st->pushed) return sfail(p, TOI_ERR_ARG, "no such pushed snapshot");
  // the slot's events belong to the latest snapshot copied through it; the
  // copy streams run in order, so their completion covers `index` too
  const int is = (int)(index % kStage);
  for (int c = 0; c < st->n_copy; ++c) {
    cudaEvent_t ev = st->ev_copied[(size_t)is * st->n_copy + c];
    cudaError_t e = wait ? cudaEventSynchronize(ev) : cudaEventQuery(ev);
    if (e == cudaErrorNotReady) return TOI_OK;
    if (e != cudaSuccess) return scuda(p, e, "toi_stream_input_free");
  }
  *is_free = 1;
  return TOI_OK;
}

toi_status toi_stream_pop(toi_stream_t st, float* row_out, int64_t* row_index, int32_t wait,
                          int32_t* got) {
  if (!st || !row_out || !got) return TOI_ERR_ARG;
  toi_plan_s* p = st->plan;
  *got = 0;
  if (st->popped >= st->rows) return TOI_OK;
  const long long r = st->popped;
  const int ih = (int)(r % st->host_depth);
  cudaError_t e = wait ? cudaEventSynchronize(st->ev_host_row[ih]) : cudaEventQuery(st->ev_host_row[ih]);
  if (e == cudaErrorNotReady) return TOI_OK;
  if (e != cudaSuccess) return scuda(p, e, "toi_stream_pop");
  std::memcpy(row_out, st->host_rows + (size_t)ih * st->ntl, sizeof(float) * st->ntl);
  if (row_index) *row_index = r;
  st->popped = r + 1;
  *got = 1;
  return TOI_OK;
}

toi_status toi_stream_close(toi_stream_t st) {
  if (!st) return TOI_ERR_ARG;
  destroy(st);
  return TOI_OK;
}

}  // extern "C"
