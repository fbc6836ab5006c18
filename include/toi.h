/*
 * toi.h - C ABI of libtoi, a GB300 (sm_103a) implementation of the FIP-TOI
 * hot path: per-snapshot Transient-Oriented Imager (TOI, 2-D mode) imaging of
 * interferometer visibilities into dirty images, FITrig's per-tile tLISI
 * statistic over the snapshot stream, and the candidate search on the tLISI
 * cube.  (Li et al., "FIP-TOI: Fast Imaging Pipeline for Pulsar Localisation
 * with a Transient-Oriented Radio Astronomical Imager".)
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All data pointers are caller-owned.  "dev" pointers are CUDA device
 *    memory of the current device, "host" pointers are host memory.  The
 *    library never frees or retains a caller pointer beyond the call, except
 *    that the images passed to tlisi_update are copied into the plan.
 *  - A plan owns all of its device scratch; it allocates only in toi_plan()
 *    and frees only in toi_plan_destroy() (no allocation in the per-snapshot
 *    loop, Section 4.2).  tlisi_candidates() allocates its own scratch per
 *    call (it runs once per observation).
 *  - Every per-snapshot call is asynchronous on the plan's stream (the stream
 *    given to toi_plan / toi_set_stream); none synchronises the host.
 *  - Errors are status codes, never aborts.  Argument errors are detected on
 *    the host before anything is launched.  Data-dependent errors found on
 *    the device (a kernel footprint leaving the grid, no selected sample,
 *    non-monotone frequencies) are latched in a device status word that
 *    toi_sync_status() reads; the affected outputs are then zero.
 *  - Array layouts are C order (last index fastest).  Images are [N][N] with
 *    row index j2 and column index j1, 0-based; pixel (j1, j2) is the paper's
 *    1-based (p1, p2) = (j1 + 1, j2 + 1) with the phase centre at N/2
 *    (Section 3.3: x = -beta (p1 - (N/2 + 1)), y = beta (p2 - (N/2 + 1))).
 */
#ifndef TOI_H
#define TOI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TOI_OK = 0,
  TOI_ERR_ARG = 1,          /* invalid argument (sizes, null pointers, config) */
  TOI_ERR_CUDA = 2,         /* a CUDA runtime call failed                       */
  TOI_ERR_OOM = 3,          /* device allocation failed in toi_plan             */
  TOI_ERR_EMPTY = 4,        /* no sample with positive weight (sum w == 0)      */
  TOI_ERR_TIMEOUT = 5,      /* a bounded device wait gave up                    */
  TOI_ERR_UNSUPPORTED = 6,  /* valid but not implemented (e.g. N not 2^k)       */
  TOI_ERR_RANGE = 7         /* a kernel footprint leaves the grid: cell too big,
                               or channel frequencies not monotone              */
} toi_status;

/* Visibility storage (Section 3.5 DATA column; FP16 variant of the precision
 * study): C64 = interleaved float32 (re, im); C16_CHANSCALE = interleaved
 * float16 (re, im) times a per-channel float32 scale. */
typedef enum { TOI_VIS_C64 = 0, TOI_VIS_C16_CHANSCALE = 1 } toi_vis_dtype;

/* Candidate scoring (Section 2: temporal FFT + harmonic summing, 5 sigma;
 * Section 6.3: sum of (1 - tLISI), 4 sigma). */
typedef enum { TOI_CAND_PERIODIC = 0, TOI_CAND_NONPERIODIC = 1 } toi_cand_mode;

typedef struct {
  int32_t image_size;       /* N (Section 2: user-supplied image size): 2^a
                               (64 ... 8192), 3 2^a (96 ... 6144) or 5 2^a
                               (160 ... 10240), the paper's sweep 2048 ...
                               10240 included                                  */
  double  cell_arcsec;      /* beta, pixel size in arcseconds (> 0)             */
  int32_t max_baselines;    /* largest n_bl a call may pass                     */
  int32_t max_channels;     /* largest n_ch a call may pass                     */
  int32_t n_pol;            /* 1, 2 or 4 (parallel hands: 0; 0,1; 0,3)         */
  int32_t vis_dtype;        /* toi_vis_dtype                                    */
  int32_t kernel_support;   /* W, gridding-kernel width in cells: 8 (default)   */
  int32_t oversample;       /* sigma, grid = sigma N: 2 (default)               */
  int32_t tlisi_tile;       /* T, tLISI tile side: 32 (default); divides N      */
  int32_t grid_slots;       /* grid buffers held by the plan (>= 1; default 1)  */
  int32_t grid_run;         /* channels each gridder lane walks: 0 = automatic
                               (default), else 8..1024; a tuning knob that
                               does not change results beyond float32
                               summation order                                 */
  int32_t batch_max;        /* largest batch of toi_batch (0 = no batched path,
                               default); each entry gets its own grid, FFT and
                               tilted-image workspace, and the image ring
                               holds batch_max + 2 images                       */
  int32_t mode;             /* 2 (TOI 2-D, default; 0 means 2) or 3 (near-
                               coplanar, Section 3.4: residual r3 t3 phase by
                               slabs and Chebyshev moments)                    */
  int32_t max_moments;      /* mode 3: largest N_slab K a snapshot may need
                               (0 = 64); two N x N float32 images each          */
  int32_t grid_rows;        /* rows of the W x W gridding window per lane: 0 =
                               automatic (or as tuned), 8 (one lane per
                               channel run) or 4 (two lanes per run); a tuning
                               knob like grid_run                              */
  int32_t max_windows;      /* largest n_win of toi_localise (0 = none,
                               default; at most 256); 64 KiB of facet grids
                               and a table of 16 B per baseline per window     */
  int32_t reserved[1];      /* must be zero                                     */
} toi_config;

typedef struct toi_plan_s* toi_plan_t;

/* Fill *cfg with the defaults above for the given geometry and maxima. */
toi_status toi_config_default(toi_config* cfg, int32_t image_size,
                              double cell_arcsec, int32_t max_baselines,
                              int32_t max_channels, int32_t n_pol);

/* Validate *cfg and allocate every device buffer the plan will use: grid
 * slots, the image ring (three images, Section 4.3 ring buffering), tilted
 * image, per-baseline and per-channel tables, the grid-correction table and
 * FFT twiddles (Section 5.2: allocation and FFT set-up happen once).
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).  On success
 * *out receives the plan.  Errors: TOI_ERR_ARG, TOI_ERR_UNSUPPORTED,
 * TOI_ERR_OOM, TOI_ERR_CUDA. */
toi_status toi_plan(const toi_config* cfg, void* cuda_stream, toi_plan_t* out);

/* Synchronise the plan's stream and free everything it owns. */
toi_status toi_plan_destroy(toi_plan_t plan);

/* Make subsequent calls of this plan run on cuda_stream. */
toi_status toi_set_stream(toi_plan_t plan, void* cuda_stream);

/* S1-S3 of one snapshot into grid slot `slot` (Sections 3, 3.1, 3.2, 3.5 and
 * Section 4.1 stage 3):
 *   - per sample q = (baseline, channel): w_q = w_a + w_b over the parallel
 *     hands, w_p = 0 if flagged else weight (or 1), c_q = w_a V_a + w_b V_b;
 *     samples with w_q > 0 are selected;
 *   - b_q = uvw * nu / c; V from the 3x3 covariance of the centred selected
 *     b_q (rows: basis vectors; v3 with V33 > 0 spans the residual axis, v1 is
 *     the u axis projected into the plane, v2 = v3 x v1); R = B V^T;
 *   - omega = |V11 V22 - V21 V12| (Eq. 11), xi = V31/V33, eta = V32/V33;
 *   - convolutional gridding of c_q at (r1, r2) with the exponential of
 *     semicircle kernel (W taps, beta_ES = 2.3 W) on a sigma N grid, stored as
 *     the Hermitian half-plane grid H[k] = G[k] + conj(G[-k]), rows k2' >= 0.
 * uvw_m:   dev float64 [n_bl][3], metres (UVW column).
 * freq_hz: dev float64 [n_ch], strictly monotone (CHAN_FREQ).
 * vis:     dev [n_bl][n_ch][n_pol] complex (float32 pairs, or float16 pairs
 *          when the plan's vis_dtype is TOI_VIS_C16_CHANSCALE).
 * chan_scale: dev float32 [n_ch] for C16_CHANSCALE, else NULL.
 * weight:  dev float32 [n_bl][n_ch][n_pol] (WEIGHT_SPECTRUM, >= 0) or NULL
 *          for unit weights.
 * flag:    dev uint8 [n_bl][n_ch][n_pol], nonzero = flagged, or NULL.
 * Errors: TOI_ERR_ARG (host checks); device: TOI_ERR_EMPTY, TOI_ERR_RANGE. */
toi_status toi_grid(toi_plan_t plan, const double* uvw_m, const double* freq_hz,
                    const void* vis, const float* chan_scale,
                    const float* weight, const uint8_t* flag,
                    int32_t n_bl, int32_t n_ch, int32_t slot);

/* S4-S6 for grid slot `slot` (Section 4.1 stages 4-5; Sections 3.2-3.3):
 * centred inverse 2-D FFT of the sigma N grid, cropped to N x N, Re,
 * divided by psi_hat(j1) psi_hat(j2) omega sum_w; then the reduced SIN
 * re-projection (x' = x + r0 z xi, y' = y + r0 z eta) gathered onto the
 * standard plane by bilinear interpolation (pixels whose source is outside
 * the tilted image are 0).  The result becomes the newest image of the
 * plan's ring; it is also written to `image` (dev float32 [N][N]) unless
 * image is NULL.  The call consumes the slot's grid (it is cleared while
 * being transformed): imaging a slot again needs a new toi_grid, and
 * gridding a slot that has not been imaged starts it from zero.  snap_info (dev float64 [16] or NULL) receives V (9, row
 * major), omega, xi, eta, sum_w, n_vis, 0, 0.  Per-tile tLISI moments of the
 * three youngest ring images are computed in the same pass. */
toi_status toi_image(toi_plan_t plan, int32_t slot, float* image,
                     double* snap_info);

/* S7, one tLISI matrix from the three youngest images (Section 2, 4.5):
 * D_a = I(t-1) - I(t-2), D_b = I(t) - I(t-1), per T x T tile
 *   S = ((2 mu_a mu_b + C1)(2 s_ab + C2)) / ((mu_a^2 + mu_b^2 + C1)(s_a^2 + s_b^2 + C2)),
 *   C1 = (0.01 L)^2, C2 = (0.03 L)^2, L = max |I| over the three images,
 *   tLISI = (1 + S) / 2 in [0, 1] (1 = identical).
 * image: dev float32 [N][N], or NULL / the pointer last written by
 *        toi_image to use the image toi_image just produced (fused path).
 *        Any other pointer is copied into the ring as the newest image.
 * tlisi: dev float32 [N/T][N/T] output (written only when *valid = 1).
 * valid: host int32: 0 for the first two images of the stream (fewer than
 *        three images exist, Section 4.1), else 1. */
toi_status tlisi_update(toi_plan_t plan, const float* image, float* tlisi,
                        int32_t* valid);

/* Forget the image history (the next two tlisi_update calls give valid=0). */
toi_status tlisi_reset(toi_plan_t plan);

/* S8 on a tLISI cube (Sections 2, 6.2, 6.3), evaluated in a fixed binary64
 * order (no fused multiply-add) so that any implementation of the same order
 * gives identical bits:
 *   periodic:     per tile x_t = tLISI_t - mean; P_f = A_f^2 + B_f^2 with
 *                 A_f, B_f the cosine/sine sums at f = 1..floor(S/2), taken
 *                 over the folded series x_t +- x_{S-t} (t = 1..(S-1)/2,
 *                 after x_0 and before the middle time of an even S) and,
 *                 for an even S, for f and S/2 - f together from the sums
 *                 over even and odd t;
 *                 score = max over f and h in {1,2,4,8} of
 *                 sum_{i<=h, i f <= F} P_{i f} / sqrt(h); k = 5;
 *   nonperiodic:  score = sum_t (1 - tLISI_t); k = 4;
 *   threshold = mean + k * std over tiles (pairwise-tree sums, population
 *   std); candidate tiles: score > threshold; 8-connected tiles merged into
 *   boxes [x0, y0, x1, y1) in 0-based pixels (tile bounds times T), sorted
 *   by (y0, x0, first tile in raster order).
 * cube:      dev float32 [S][nty][ntx].
 * stream:    cudaStream_t to run on (NULL = default stream).
 * threshold: host float64 out.  boxes: host int32 [max_boxes][4] out.
 * nboxes:    host int32 out, the number of boxes found (may exceed
 *            max_boxes; only the first max_boxes are written).
 * scores:    dev float64 [nty][ntx] out, or NULL.
 * nty * ntx may be at most 131072 (TOI_ERR_ARG beyond): the labelling runs
 * in one block, whose worst case (one component winding through every tile)
 * grows with the square of the tile count.
 * Allocates and frees its device scratch; synchronises `stream`. */
toi_status tlisi_candidates(const float* cube, int32_t S, int32_t nty,
                            int32_t ntx, int32_t tile, int32_t mode,
                            void* stream, double* threshold, int32_t* boxes,
                            int32_t* nboxes, int32_t max_boxes,
                            double* scores);

/* tlisi_candidates without any device allocation.  The paper has no
 * counterpart; this serves callers that cannot allocate device memory when
 * they search for candidates: a real-time pipeline that must not stall
 * (cudaMalloc may synchronise the device), an application whose device
 * memory is wholly owned by its own allocator, or code running where
 * allocation is not permitted.
 *
 * Same arguments, outputs and results as tlisi_candidates.  The scratch is
 * one fixed 16 MiB device array compiled into the library (every GPU that
 * loads the library holds it until the process exits).  A cube whose search
 * needs more than that (scratch grows as about 8 (S/2 + 1) nty ntx bytes,
 * e.g. 64 x 64 tiles up to about 960 slices) is rejected with TOI_ERR_ARG
 * and a message giving the size; use tlisi_candidates for those.  Every call
 * looks up the array's address on the calling thread's current device
 * (cudaGetSymbolAddress), so the address is never stale.  All calls on a
 * device share the one array: calls whose GPU work overlaps (other streams,
 * other host threads) race and must be serialised by the caller.  The array
 * keeps the last call's contents; the search writes every scratch word
 * before reading it, so nothing needs clearing.  With scores NULL the scores
 * stay in the array.  The call synchronises `stream` to return the
 * threshold and boxes, so it cannot be recorded into a CUDA graph by stream
 * capture. */
toi_status tlisi_candidates_noalloc(const float* cube, int32_t S, int32_t nty,
                                    int32_t ntx, int32_t tile, int32_t mode,
                                    void* stream, double* threshold, int32_t* boxes,
                                    int32_t* nboxes, int32_t max_boxes,
                                    double* scores);

/* One snapshot of a batch: the arguments of toi_grid (device pointers with
 * the same layouts and rules) plus where toi_image would write its image
 * (dev float32 [N][N] or NULL: the image is then not written out; the plan
 * keeps only a batch's last two images, for the next windows, and
 * toi_plan_buffer reads the last one). */
typedef struct {
  const double* uvw;
  const double* freq;
  const void* vis;
  const float* chan_scale;
  const float* weight;
  const uint8_t* flag;
  float* image;
  int32_t n_bl;
  int32_t n_ch;
} toi_snapshot;

/* Batched S1-S7 over n <= batch_max snapshots of the stream, in stream
 * order, with one launch per stage for the whole batch (Section 4.3: the
 * pipelined, stream-parallel execution of many snapshots; the batch may mix
 * channel counts and flag fractions).  The gridder is persistent: its warps
 * take (snapshot, track, segment) work items from a counter, so uneven
 * snapshots share the GPU without a partial last wave per snapshot.
 * Results equal n calls of toi_grid + toi_image + tlisi_update up to the
 * float32 summation order of the gridder.
 *
 * toi_batch_prepare validates the snapshots on the host and fills the
 * plan's pinned batch table; toi_batch_run enqueues the batch on the plan's
 * stream (two table copies, a counter reset, then 9 kernels).  toi_batch_run makes no host
 * call that a CUDA graph capture forbids, and its launch shapes do not
 * depend on the batch, so one captured toi_batch_run can be replayed for
 * every later batch: call toi_batch_prepare before each replay, after the
 * previous replay's table copies have run (for instance after synchronising
 * the stream).  Without capture, toi_batch_prepare waits for the previous
 * batch's table copies itself.
 *   tlisi        dev float32 [n][N/T][N/T] or NULL: row i receives the tLISI
 *                of the three-image window ending with snapshot i.
 *   first_valid  host, may be NULL: rows [first_valid, n) are written (the
 *                first two images of a stream have no window).
 * The batch uses its own grid slots (not those of toi_grid) and advances
 * the same image stream as toi_image / tlisi_update.  Errors: TOI_ERR_ARG
 * (batch_max = 0, n outside [1, batch_max], a snapshot failing toi_grid's
 * checks, run without prepare), TOI_ERR_UNSUPPORTED (tlisi_tile > 32),
 * TOI_ERR_CUDA; data errors as for toi_grid, via toi_sync_status. */
toi_status toi_batch_prepare(toi_plan_t plan, const toi_snapshot* snaps, int32_t n,
                             float* tlisi, int32_t* first_valid);
toi_status toi_batch_run(toi_plan_t plan);
/* toi_batch_prepare followed by toi_batch_run. */
toi_status toi_batch(toi_plan_t plan, const toi_snapshot* snaps, int32_t n, float* tlisi,
                     int32_t* first_valid);

/* Choose the gridder's channels per lane for each channel-count bucket
 * (n_ch <= 1024, <= 2048, <= 4096, larger) present among the n sample
 * snapshots, and its window split (the W x W footprint in one lane, or half
 * of it in each of two lanes), by timing the batched gridder for 16, 32, 64,
 * 128 and 256 channels per lane under both splits (best of three launches
 * each, CUDA events); the split with the smaller total time is kept.  The
 * choice is cached in the plan and used by the batch (the run when
 * config.grid_run is 0, the split when config.grid_rows is 0); single
 * toi_grid launches keep their own defaults.  runs_out[4] and us_out[4] (host, may be NULL)
 * receive the chosen run and its gridding time per snapshot in
 * microseconds for the buckets that were tuned.  Synchronous; needs
 * batch_max >= n; leaves the stream position and the batch grids as they
 * were.  Errors as toi_batch_prepare. */
toi_status toi_autotune(toi_plan_t plan, const toi_snapshot* snaps, int32_t n, int32_t* runs_out,
                        double* us_out);

/* Gridder work split the plan uses for a snapshot of n_ch channels (host
 * int32 outputs): *run = channels walked by one lane (or lane pair), *rows =
 * window rows held per lane (8: the whole W x W footprint, 4: half of it in
 * each lane of a pair), for batched launches (batched != 0, toi_batch*) or
 * single toi_grid launches.  It reflects config.grid_run / grid_rows, then
 * what toi_autotune chose, then the built-in defaults (Section 4.1 stage 3
 * is the gridding step; the split itself is this library's design).  Host
 * only, no device work.  TOI_ERR_ARG for a NULL plan or output or n_ch < 1. */
toi_status toi_grid_lane_run(toi_plan_t plan, int32_t n_ch, int32_t batched, int32_t* run,
                             int32_t* rows);

/* Near-coplanar plan of the snapshot gridded into `slot` (mode 3; host
 * double[8]): N_slab, K, Phi_max, alpha_slab, dr3 (wavelengths), r3min,
 * r3max (over the selected samples) and t3max (over the pixel centres) as
 * chosen by Section 3.4 (Eqs. 26-27, K from {8, 16, 24, 32} by the sampled
 * truncation error, gamma = 1e-2).  In mode 3 toi_grid does S1 and the
 * moment gridding and transforms (2 N_slab K passes into the plan's moment
 * images; it synchronises the stream once to read the selection), and
 * toi_image combines the moments per pixel before S6-S7.  Errors:
 * TOI_ERR_ARG (not mode 3, slot never gridded). */
toi_status toi_mode3_info(toi_plan_t plan, int32_t slot, double* info);

/* Reverse mode of one snapshot's image (gridding, inverse FFT, correction,
 * re-projection of toi_image) for a loss L whose gradient with respect to the
 * standard-plane image is grad_image.  Section 1 of the paper notes that the
 * dirty image is the adjoint of the measurement operator; this is that
 * adjoint applied to dL/dI, followed by the chain rule to the inputs.  The
 * plane fit (V, omega and the sample selection w_q > 0) is held fixed: it is
 * piecewise constant in the weights.  Complex gradients are
 * dL/dRe z + i dL/dIm z.
 *   grad_image   dev float32 [N][N] (row = p2, col = p1, as toi_image's image).
 *   image        dev float32 [N][N]: the image toi_image produced for this slot;
 *                needed only for grad_weight (NULL otherwise).
 *   grad_sample  dev complex64 [n_bl][n_ch] or NULL: g_q = dL/dc_q for the
 *                gridded value c_q = w_a V_a + w_b V_b; 0 for unselected samples.
 *   grad_vis     dev complex64 [n_bl][n_ch][n_pol] or NULL: w_p g_q for the
 *                parallel hands p of selected samples, 0 elsewhere.
 *   grad_weight  dev float32 [n_bl][n_ch][n_pol] or NULL: for unflagged
 *                parallel hands of selected samples
 *                Re(conj(g_q) V_p) - <grad_image, image> / sum w, else 0.
 * At least one output must be non-NULL.  The inputs of the last toi_grid on
 * `slot` (uvw, freq, vis, chan_scale, weight, flag) are read again and must
 * still hold the same data; the slot's snapshot record (from toi_grid) gives
 * V, omega and sum w.  The plan's tilted-image and FFT scratch and the slot's
 * grid memory are used as workspace: a grid not yet imaged is discarded and
 * the slot is left cleared for the next toi_grid.  Asynchronous on the
 * plan's stream.  Errors: TOI_ERR_ARG (NULL or misaligned pointers, slot never
 * gridded, grad_weight without image), TOI_ERR_CUDA. */
toi_status toi_degrid_backward(toi_plan_t plan, int32_t slot, const float* grad_image,
                               const float* image, void* grad_sample, void* grad_vis,
                               float* grad_weight);

/* Streaming runtime: the snapshot pipeline of Sections 4.1-4.4 with one
 * CUDA stream per device stage (copy_gpu over n_copy copy streams, gridding,
 * fft, interpolate fused with the tLISI tile moments, tlisi, copy_cpu),
 * interlocked by events; the caller is data_read (filling pinned host
 * buffers) and data_write (toi_stream_pop).  Rings: a depth-2 device staging
 * ring, the depth-3 grid ring (grid slots 0-2 and three tilted images), the
 * depth-5 image ring, two device tLISI rows and host_depth pinned host rows.
 * A ring slot is reused after an event of its last reader (a stream wait):
 * toi_stream_push never waits on the host.  Row r of the output is the
 * tLISI of snapshots (r, r + 1, r + 2) (float32 [N/T][N/T]).
 * The plan needs grid_slots >= 3 and 2-D mode; while a stream is open the
 * plan's grid slots 0-2 belong to it (no toi_grid/toi_image/toi_batch on
 * this plan until toi_stream_close).  Errors: TOI_ERR_ARG,
 * TOI_ERR_UNSUPPORTED, TOI_ERR_OOM, TOI_ERR_CUDA (plan-reported). */
typedef struct toi_stream_s* toi_stream_t;

/* Allocate the rings and streams.  host_depth in [1, 4096] pinned host tLISI
 * rows; n_copy in [1, 16] copy streams for the visibilities (and flags and
 * weights), split by baseline; with_weights: whether snapshots may carry
 * WEIGHT_SPECTRUM (staging for it is allocated). */
toi_status toi_stream_open(toi_plan_t plan, int32_t host_depth, int32_t n_copy,
                           int32_t with_weights, toi_stream_t* out);

/* Enqueue one snapshot through every device stage.  snap holds HOST
 * pointers (pinned memory, else the copies are not asynchronous), layouts
 * as toi_grid; snap->image is ignored.  The buffers must stay unchanged until
 * toi_stream_input_free reports them free.  *index (may be NULL) receives the
 * snapshot's position in the stream.  Fails with TOI_ERR_ARG when the host
 * row ring is full (pop first). */
toi_status toi_stream_push(toi_stream_t stream, const toi_snapshot* snap, int64_t* index);

/* *is_free = 1 once the host->device copies of snapshot `index` are done
 * (its host buffers may be refilled); wait != 0 blocks until then. */
toi_status toi_stream_input_free(toi_stream_t stream, int64_t index, int32_t wait,
                                 int32_t* is_free);

/* The oldest tLISI row not yet popped: copied to row (host float32
 * [N/T][N/T]) with *got = 1 and *row_index = r, or *got = 0 when none is
 * ready (none pushed yet, or wait == 0 and its copy is still running). */
toi_status toi_stream_pop(toi_stream_t stream, float* row, int64_t* row_index, int32_t wait,
                          int32_t* got);

/* Wait for the stages and free the stream's buffers, streams and events. */
toi_status toi_stream_close(toi_stream_t stream);

/* Side of a localisation window (pixels of the tilted-plane image). */
#define TOI_LOC_WINDOW 32

/* Candidate windows of one snapshot from its tLISI matrix (the sub-pixel
 * localisation of candidates, Sections 2 and 6): the n_win tiles with the
 * smallest tLISI (ties by tile index; NaN last) each give a TOI_LOC_WINDOW^2
 * window of the tilted-plane image centred on the tile (clamped to the
 * image), and a starting source at the window's largest pixel: with
 * tau = (t1, t2) of that pixel (t1 = -beta (j1 - N/2), t2 = beta (j2 - N/2))
 * and tau3 the root of |V^T tau + z| = 1 nearest 0, (l, m) = the first two
 * components of V^T tau and S = omega x the pixel value (the peak of an
 * unresolved source in the 2-D image is S / omega).
 *   tlisi  dev float32 [N/T][N/T], e.g. the row tlisi_update wrote.
 *   win    dev int32 [n_win][2] out: window corners (row j2c, column j1c).
 *   src    dev float64 [n_win][3] out: (l, m, S).
 * The slot's plane fit and the plan's tilted image must be this snapshot's
 * (toi_image(slot) was the last image call).  1 <= n_win <= max_windows and
 * (N/T)^2 <= 2048 floor(4096 / n_win) (TOI_ERR_UNSUPPORTED otherwise).
 * Asynchronous.  Errors: TOI_ERR_ARG, TOI_ERR_UNSUPPORTED, TOI_ERR_CUDA. */
toi_status toi_localise_seed(toi_plan_t plan, int32_t slot, const float* tlisi, int32_t n_win,
                             int32_t* win, double* src);

/* Windowed point-source fit of one snapshot: loss and gradients (the
 * differentiable localisation that Section 1's adjoint route permits).
 * Window w is the TOI_LOC_WINDOW^2 block of the tilted-plane image with
 * corner win[w]; its model M_w is the 2-D dirty image (Section 3.2) of one
 * point source (l, m, S) = src[w], V_p = S exp(-2 pi i k (u l + v m +
 * w (n - 1))) in the parallel hands (Section 1), with the snapshot's flags
 * and weights.  The model is made by faceted gridding: the samples rotated
 * to the window centre and gridded on a 2 TOI_LOC_WINDOW grid over the full
 * uv extent, so it equals the full image of the model on the window to the
 * ES kernel's accuracy.  With D the tilted image on the window:
 *   loss[w]        = sum (D - M_w)^2           (dev float64 [n_win], or NULL)
 *   model          = M_w                        (dev float32 [n_win][32][32], or NULL)
 *   grad_src[w]    = dL/d(l, m, S), L = sum_w loss[w]  (dev float64 [n_win][3], or NULL)
 *   grad_weight[p] = dL/dw_p for the unflagged parallel hands of selected
 *                    samples (both D and every M_w depend on the weights,
 *                    through c_q and 1 / sum w), else 0
 *                                               (dev float32 [n_bl][n_ch][n_pol], or NULL)
 * The plane fit (V, omega, the selection) is held fixed, as in
 * toi_degrid_backward.  Reads the inputs of the last toi_grid on `slot`
 * again (they must still hold the same data) and the plan's tilted image,
 * which must be this snapshot's (toi_image(slot) was the last image call).
 * With grad_weight the tilted image, the FFT scratch and the slot's grid are
 * used as workspace (the tilted image is not this snapshot's afterwards).
 * 1 <= n_win <= max_windows.  2-D mode only.  Asynchronous; a window off the
 * image or a source with l^2 + m^2 >= 1 gets zero loss and gradients and
 * latches TOI_ERR_RANGE (toi_sync_status).  Errors: TOI_ERR_ARG,
 * TOI_ERR_UNSUPPORTED, TOI_ERR_CUDA. */
toi_status toi_localise(toi_plan_t plan, int32_t slot, int32_t n_win, const int32_t* win,
                        const double* src, float* model, double* loss, double* grad_src,
                        float* grad_weight);

/* Copy of a plan-owned buffer, for checking intermediate stages:
 * which = 0 grid slot `slot` (complex float32 [G/2][G], the Hermitian
 * half-plane grid, rows k2' = 0..G/2-1, columns k1 = 0..G-1), 1 tilted-plane
 * image of the last toi_image (float32 [N][N]), 2 snapshot record of slot
 * `slot` (float64 [16], as snap_info), 3 newest ring image (float32 [N][N]).
 * *nbytes receives the buffer size; when dst is not NULL, min(dst_bytes,
 * size) bytes are copied to dst (device or host memory) after the plan's
 * stream has finished its queued work. */
toi_status toi_plan_buffer(toi_plan_t plan, int32_t which, int32_t slot, void* dst,
                           int64_t dst_bytes, int64_t* nbytes);

/* Device-time accounting per stage of this plan, measured with CUDA events
 * recorded on the plan's stream around each stage's kernels.  Stages:
 * 0 plane fit (4 kernels), 1 reserved (always 0), 2 gridding, 3 FFT rows,
 * 4 FFT columns + correction, 5 re-projection + tLISI moments, 6 tLISI
 * finish / external-image moments, 7 toi_degrid_backward, 8 toi_localise and
 * toi_localise_seed.  toi_batch_run's
 * kernels count under the same stages (one launch per stage per batch).
 * Kernel launches are counted per stage whether or not timing is enabled. */
toi_status toi_profile_enable(toi_plan_t plan, int32_t enable);

/* Read and reset the accumulated milliseconds (ms[nstages], may be NULL) and
 * launch counts (launches[nstages], may be NULL); waits for the recorded
 * events. */
toi_status toi_profile_read(toi_plan_t plan, double* ms, int64_t* launches, int32_t nstages);

/* Synchronise the plan's stream and return (and clear) the device status
 * word: TOI_OK, TOI_ERR_EMPTY or TOI_ERR_RANGE. */
toi_status toi_sync_status(toi_plan_t plan);

/* Human-readable text of the last error of this plan ("" if none); with a
 * NULL plan, of the last error of a plan-less call on this thread. */
const char* toi_last_error(toi_plan_t plan);

/* Static text for a status code. */
const char* toi_status_string(toi_status s);

#ifdef __cplusplus
}
#endif

#endif /* TOI_H */
