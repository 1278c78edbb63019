/*
 * pd.h — C ABI of the GB300 pixel-detector correction and photon-finding
 * library (libpd.so).
 *
 * The library runs, per frame, the classical integrating-pixel-detector chain
 * that Blaj, Chang and Kenney, "Ultrafast Processing of Pixel Detector Data
 * with Machine Learning Frameworks" (AIP Conf. Proc. 2054, 060077, 2019)
 * recast as fixed-weight tensor models:
 *
 *   raw -> dark (pedestal) subtraction           (Fig. b, "Dark and Gain")
 *       -> common-mode removal per unit           (Fig. c, "Common Mode")
 *       -> gain correction                        (Fig. b)
 *       -> noise zeroing, local maximum,          (Fig. e, "Photon Charge
 *          3x3 charge sum, photon count              Summing")
 *       -> centre-of-mass subpixel offset         (Fig. f, "Photon Subpixel
 *                                                   Resolution")
 *       -> sparse hit list, photon-count map,     ("Summarization")
 *          pixel and hit energy histograms
 *
 * Every step runs in hand-written sm_103a CUDA kernels; there is no CPU
 * fallback.  The arithmetic is FP32 with every operation rounded to nearest
 * in a fixed order, so results are reproducible bit for bit.
 *
 * Conventions common to all entry points
 *   - Return value: PD_OK (0) or one of the PD_E* codes below.  No C++
 *     exception crosses this boundary.  pd_strerror() names a code and
 *     pd_last_error() returns a thread-local message for the last failure.
 *   - "device" pointers are CUDA global-memory addresses on the current
 *     device; "host" pointers are ordinary (optionally page-locked) memory.
 *   - stream arguments are a cudaStream_t passed as void* (NULL = legacy
 *     default stream).  Calls that take a stream are asynchronous unless
 *     their comment says otherwise.
 *   - One pd_ctx may be used from one host thread / stream at a time.
 *
 * Frame layout (paper: rank-4 minibatch N x H x W x 1, section "Dark and
 * Gain"): raw frames are uint16 [n_frames][n_modules][rows][cols], row-major
 * and contiguous.  A module is one contiguous sensor; the 3x3 stencil never
 * crosses a module edge.  A common-mode unit is a unit_rows x unit_cols
 * rectangle; units tile every module (row units: unit_rows = 1; banks:
 * unit_rows x unit_cols sub-arrays).
 */
#ifndef PD_H
#define PD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------ */
#define PD_OK 0
#define PD_EINVAL 1     /* invalid argument or inconsistent geometry        */
#define PD_EALIGN 2     /* pointer or size not aligned as required          */
#define PD_ENOMEM 3     /* a device or host allocation failed               */
#define PD_EOVERFLOW 4  /* more hits than hit_capacity (count still exact)  */
#define PD_ETIMEDOUT 5  /* a bounded device-side or host-side wait gave up  */
#define PD_ECUDA 6      /* a CUDA runtime call failed                       */
#define PD_ENOTSUP 7    /* valid request the library does not support       */
#define PD_EBUSY 8      /* admission refused: no slot or memory budget free */

/* ---- common-mode estimators (paper Fig. c and its text) --------------- */
#define PD_CM_MEDIAN 0 /* lower median of d = raw - pedestal over d < cut  */
#define PD_CM_NONE 1   /* no common-mode correction (cm = 0)               */
/* The paper's estimator (section "Common Mode", Fig. c): over a group of G
 * pixels, N0 values v with v < cut (and v > -inf) summing to S give
 * cm = S / max(N0, sqrt(G)).  S is exact and independent of order: with M
 * the largest selected |v| and E = max(floor(log2 M), -60), each v is
 * rounded (to nearest even) to the grid 2^(E-38), the integers are added
 * exactly and the total is rounded once to float32; values down to
 * M * 2^-15 lie on that grid.  cm_min_count is not used.  Units must hold
 * fewer than 2^24 pixels. */
#define PD_CM_MEAN 2         /* one stage over each unit (v = d)           */
/* Three stacked stages (section "Performance"): units (v = d), then each
 * module row (v = d - cm_u), then each module column
 * (v = (d - cm_u) - cm_r); c = ((d - cm_u) - cm_r) - cm_c. */
#define PD_CM_MEAN_STACKED 3

/* ---- hit flags -------------------------------------------------------- */
#define PD_HIT_EDGE 1u      /* seed pixel lies on its module's border       */
#define PD_HIT_SATURATED 2u /* rint(E / photon_kev) exceeded 255 and clipped */
#define PD_HIT_LEARNED 4u   /* count and dx, dy come from the learned network */
#define PD_HIT_LINEARISED 8u /* dx, dy linearised by pd_eta_apply            */

/* Detector geometry.  Requirements (PD_EINVAL otherwise): all sizes > 0,
 * rows, cols <= 65535, fewer than 2^31 pixels per frame, rows % unit_rows
 * == 0 and cols % unit_cols == 0. */
typedef struct {
    uint32_t n_modules;
    uint32_t rows, cols;           /* pixels of one module                  */
    uint32_t unit_rows, unit_cols; /* common-mode unit                      */
    uint32_t cm_mode;              /* PD_CM_MEDIAN, _NONE, _MEAN, _MEAN_STACKED */
    /* 0 (default): common mode on d = raw - pedestal in ADU, then gain.
     * 1: the paper's order (Fig. a lists gain first; Fig. c takes the
     * gain-corrected Frames1): e0 = d * inv_gain, the common-mode set is
     * {e0 < cm_cut_kev} over unmasked pixels, the estimators work on e0,
     * e = e0 - cm (stacked: ((e0 - cm_u) - cm_r) - cm_c), masked pixels read
     * 0.  Not with pd_create_multigain. */
    uint32_t cm_after_gain;
} pd_geometry;

/* Thresholds and summary binning.  The paper exposes two noise thresholds
 * (section "Accuracy", Figs. c and e); the common-mode cut here is in ADU
 * because the correction is taken before gain.  Requirements: 0 <=
 * zero_thr_kev <= seed_thr_kev, photon_kev > 0, hist_bin_kev > 0,
 * 1 <= hist_bins <= PD_MAX_HIST_BINS, all finite. */
typedef struct {
    float cm_cut_adu;       /* pixel enters the common-mode set iff d < cut  */
    float zero_thr_kev;     /* s = e > zero_thr ? e : 0      (Fig. e)        */
    float seed_thr_kev;     /* a seed needs e > seed_thr                     */
    float photon_kev;       /* count n = rint(E / photon_kev)                */
    uint32_t cm_min_count;  /* min pixels below cut; 0 = ceil(sqrt(unit px)) */
    float hist_lo_kev;      /* histogram bin b covers lo + [b, b+1) * width  */
    float hist_bin_kev;     /*   (computed as floor((v - lo) * (1/width)))   */
    uint32_t hist_bins;     /* end bins are clamped                          */
    float cm_cut_kev;       /* common-mode cut when cm_after_gain = 1 (keV)  */
} pd_thresholds;

#define PD_MAX_HIST_BINS 4096u

/* Matched-filter charge summing (section "Photon Charge Summing", Figs. d
 * and e; centroids: section "Photon Subpixel Resolution", Fig. f).  A bank
 * of n_features features, each with four 4 x 5 filters and a threshold.
 * Filter tap [i][j] applied at pixel (r, c) meets pixel (r + i - 1,
 * c + j - 2) of the same module (zero outside): TF's conv2d "SAME"
 * alignment of a 4 x 5 kernel.  With s the zeroed signal (Fig. e "Signal")
 * and T = (s > 0), at every pixel and for each feature f:
 *   Size = sum T * f1   Droplet = sum s * f1   Overflow = sum T * f0
 *   Mx = sum s * f1_dx  My = sum s * f1_dy     (taps row-major from 0.0f)
 *   Valid = Overflow == 0 && Size >= f1_nmin
 * and over the valid features in order E = sum Droplet (Frames3),
 * dx = sum Mx / Droplet, dy = sum My / Droplet (features whose Droplet is
 * 0 add nothing to dx, dy).  A pixel with a valid feature and E != 0 is a
 * seed (hist_hit[bin(E)]); n = rint(E / photon_kev) clamped to 255 as in
 * the default chain, a hit iff n >= 1, npix = signal pixels under the
 * nonzero f1 taps of the first valid feature, flags as in the default
 * chain.  The paper gives its bank's values only as a picture; the bank is
 * the caller's.  All values finite, f1_nmin not NaN. */
#define PD_MAX_FEATURES 8u
typedef struct {
    uint32_t n_features;  /* 1 .. PD_MAX_FEATURES */
    float f0[PD_MAX_FEATURES][4][5];    /* overflow ring: must see no signal */
    float f1[PD_MAX_FEATURES][4][5];    /* footprint: size and droplet      */
    float f1_dx[PD_MAX_FEATURES][4][5]; /* column offsets for the centroid  */
    float f1_dy[PD_MAX_FEATURES][4][5]; /* row offsets for the centroid     */
    float f1_nmin[PD_MAX_FEATURES];     /* minimum Size of a valid match    */
} pd_filter_bank;

/* One photon hit (24 bytes).  pixel = module*rows*cols + row*cols + col of
 * the seed; dx, dy are the charge centre of mass in pixel pitches relative
 * to the seed pixel centre (Fig. f), so the position is
 * (col + 0.5 + dx, row + 0.5 + dy) in the module. */
typedef struct {
    uint32_t frame;      /* frame_base + index of the frame in the call      */
    uint32_t pixel;
    float energy_kev;    /* E: 3x3 sum of the zeroed signal                  */
    float dx, dy;
    uint8_t count;       /* n = clamp(rint(E / photon_kev), 0, 255), >= 1    */
    uint8_t npix;        /* pixels of the 3x3 with signal > 0                */
    uint16_t flags;      /* PD_HIT_* bits                                    */
} pd_hit;

/* Per-call outputs of pd_process.  All pointers are device memory owned by
 * the caller.  hits / n_hits are required; the others may be NULL. */
typedef struct {
    pd_hit* hits;          /* hit_capacity records; order is unspecified     */
    uint32_t hit_capacity;
    uint32_t* n_hits;      /* 1 x u32: set to the call's true hit count      */
    float* corrected;      /* [n_frames][pixels] e (keV) or NULL; 16-B aligned */
    float* cm;             /* [n_frames][cm_values_per_frame] common mode
                              (ADU) or NULL: the units' values (module-major,
                              row-major units), then for PD_CM_MEAN_STACKED
                              n_modules x rows row terms and n_modules x cols
                              column terms                                   */
} pd_outputs;

typedef struct pd_ctx pd_ctx;

/* Sizes derived from a context. */
typedef struct {
    uint32_t pixels_per_frame;
    uint32_t units_per_frame;
    uint32_t unit_pixels;
    uint32_t cm_min_count;   /* resolved value (0 replaced by the default) */
    uint32_t hist_bins;
    uint32_t masked_pixels;  /* pixels whose gain was <= 0 or not finite   */
    uint32_t cm_values_per_frame; /* common-mode values per frame (pd_outputs.cm) */
} pd_info;

/* pd_create — validate the geometry and thresholds, copy the pedestal and
 * gain maps (host float32 [n_modules][rows][cols]; pedestal in ADU, gain in
 * ADU/keV) to the device, and compute inv_gain = 1.0f / gain there-from on
 * the host (round to nearest; gain <= 0 or non-finite -> inv_gain = 0, the
 * pixel is masked; a non-finite pedestal is PD_EINVAL).  Allocates the
 * context's device state: maps, photon
 * count map (u32 per pixel) and two u64 histograms, all zeroed.  The device
 * is the current CUDA device.  On failure *out is NULL. */
int pd_create(const pd_geometry* geometry, const float* pedestal_host,
              const float* gain_host, const pd_thresholds* thresholds,
              pd_ctx** out);

/* pd_create_multigain — a context for auto-ranging detectors (the caption
 * of Fig. b: several darks and gains per pixel).  Each raw word carries its
 * gain stage in bits gain_shift..15 and its ADC value below:
 * stage = raw >> gain_shift, value = raw & (2^gain_shift - 1).
 * pedestal_host and gain_host hold n_gains maps, [n_gains][n_modules][rows]
 * [cols].  Then d = value - pedestal[stage]; the common mode (median, or
 * none) is taken over stage-0 pixels only and subtracted from them only:
 * e = (d - cm) * inv_gain[0] for stage 0, e = d * inv_gain[stage] for the
 * others; a stage >= n_gains marks a bad pixel, e = 0.  Everything after
 * the energy (zeroing, charge summing or matched filters, summaries) is
 * unchanged.  1 <= n_gains <= PD_MAX_GAINS, 1 <= gain_shift <= 15, cm_mode
 * PD_CM_MEDIAN or PD_CM_NONE; such contexts use the generic kernels (no
 * one-kernel chain, no mixed batch launch).  masked_pixels counts stage 0. */
#define PD_MAX_GAINS 4u
int pd_create_multigain(const pd_geometry* geometry, uint32_t n_gains, uint32_t gain_shift,
                        const float* pedestal_host, const float* gain_host,
                        const pd_thresholds* thresholds, pd_ctx** out);

int pd_query(const pd_ctx* ctx, pd_info* info);

/* pd_process — run the whole chain on n_frames device-resident raw frames
 * (16-byte aligned) and enqueue it on `stream`.  Writes the hit list and
 * *n_hits (zeroed by the call itself), and adds the frames' contributions
 * to the context's count map and histograms.  When more than hit_capacity
 * hits occur, the surplus records are dropped and *n_hits still holds the
 * true count (the caller compares after synchronising).  n_frames == 0 only
 * zeroes *n_hits.  Asynchronous: errors of the launch itself are returned,
 * device results are valid once the stream reaches this point. */
int pd_process(pd_ctx* ctx, const uint16_t* frames_dev, uint32_t n_frames,
               uint32_t frame_base, const pd_outputs* out, void* stream);

/* pd_process_noalloc — the same chain as pd_process, for callers that must
 * not allocate device memory during processing: for example a real-time
 * acquisition thread whose latency budget forbids the device-wide
 * synchronisation an allocation can cause, or a process whose device memory
 * is entirely owned by another allocator, so cudaMalloc would fail.
 * pd_process may allocate (it grows its common-mode scratch on demand);
 * this entry point never calls cudaMalloc, cudaFree or any allocating
 * routine.  The paper has no counterpart; this is a deployment variant.
 *
 * Its common-mode scratch is one fixed device array inside the library,
 * PD_NOALLOC_MAX_CM floats (4 MiB), present on every GPU that loads the
 * library until the process exits.  Limit: when out->cm is NULL and the
 * context runs the common-mode + stencil kernel pair, n_frames *
 * cm_values_per_frame must not exceed PD_NOALLOC_MAX_CM, else the call
 * returns PD_EINVAL (split the call, or pass out->cm, which is then used
 * instead); the one-kernel chain (pd_tuning.two_pass = 0) uses no scratch
 * and has no limit.  The array's device address is looked up by pd_create
 * on the context's device; under CUDA's lazy module loading that lookup is
 * what loads the module holding the array, so this entry point itself loads
 * nothing on a context's device (should pd_create's lookup have failed, the
 * first call here looks it up again: make that first call before any stream
 * capture).  The context's device must be current (PD_EINVAL otherwise).
 * The array is shared by all calls and keeps the last call's values;
 * nothing in it needs clearing (every value is written before it is read),
 * but calls whose work overlaps on the GPU (different streams, no ordering
 * between them) race on it: order them.  Runs on `stream` alone.
 * Arguments, outputs and errors as pd_process. */
#define PD_NOALLOC_MAX_CM (1u << 20)
int pd_process_noalloc(pd_ctx* ctx, const uint16_t* frames_dev, uint32_t n_frames,
                       uint32_t frame_base, const pd_outputs* out, void* stream);

/* pd_set_filter_bank — replace the 3x3 local-maximum charge summing of
 * this context (steps of section "Photon Charge Summing" as the default
 * chain reads them) by the matched filters of `bank` (copied; host memory),
 * or restore the default with bank == NULL.  Synchronises the device; do
 * not call while work of this context is in flight.  The one-kernel chain
 * and the mixed batch launch are not used with a bank.  When every feature
 * is binary (F1 taps 1 or 0, F0 taps positive or 0), the valid features
 * depend on a pixel's 4 x 5 signal mask alone: the context then allocates
 * a 2^20-byte device table (once; freed by pd_destroy) and fills it on the
 * device before returning.  PD_EINVAL for a feature count out of range or a
 * non-finite value, PD_ENOMEM when the table cannot be allocated. */
int pd_set_filter_bank(pd_ctx* ctx, const pd_filter_bank* bank);

/* pd_process_host — the same chain on host-resident frames.  Copies the
 * frames to the device in chunks of about 64 MB (pipelined on internal
 * streams, so page-locked host memory gives full link speed), processes
 * them, and copies the hit list and its count back: the hits of a chunk are
 * downloaded two chunks later, while later chunks upload (a page-locked
 * hits_host lets that download run asynchronously).  Synchronous: returns
 * after all hits are in hits_host.  Returns PD_EOVERFLOW if more than hit_capacity
 * hits occurred (*n_hits_host is then the true count, hits_host holds the
 * first hit_capacity records in unspecified order). */
int pd_process_host(pd_ctx* ctx, const uint16_t* frames_host,
                    uint32_t n_frames, uint32_t frame_base, pd_hit* hits_host,
                    uint32_t hit_capacity, uint32_t* n_hits_host);

/* pd_get_summary — copy the accumulated summaries to host buffers (any may
 * be NULL): count_map u32 [pixels], hist_pix u64 [hist_bins] (every
 * corrected pixel e), hist_hit u64 [hist_bins] (the 3x3 energy E of every
 * seed).  Synchronous on `stream`. */
int pd_get_summary(pd_ctx* ctx, uint32_t* count_map_host,
                   uint64_t* hist_pix_host, uint64_t* hist_hit_host,
                   void* stream);

/* pd_reset_summary — zero the count map and histograms (async on stream),
 * and clear the context's record of a timed-out device wait. */
int pd_reset_summary(pd_ctx* ctx, void* stream);

/* Bounded device waits.  The kernels that wait on a staged copy (the bank
 * median, the staged stencil) or on another CTA's result (the work-queue
 * launch) poll a bounded number of times; when a wait gives up, the kernel
 * waits out its copies in flight with the default bound, stops, and the
 * context records it: pd_get_summary then returns PD_ETIMEDOUT (results of
 * that call are not valid) until pd_reset_summary.  polls sets the bound of
 * the first wait (0: the kernels' defaults, about 2^20 polls of a copy and
 * 2^22 of a dependency); a small bound makes the timeout path run, which is
 * what it is for (tests).  Launches already queued keep their bound. */
int pd_set_wait_limit(pd_ctx* ctx, uint32_t polls);

/* pd_destroy — free the context's device state (NULL is a no-op).  Waits
 * for the device to finish work that may use it. */
void pd_destroy(pd_ctx* ctx);

/* Launch tuning of a context (the autotuner's search space).  Zero fields
 * keep the current value.  chunk_frames: frames per common-mode/stencil
 * launch pair (a chunk's raw frames are re-read from L2 by the second
 * pass); band_rows: rows per stencil tile; overlap: 1 runs the common mode
 * of the next chunk on a second stream beside the stencil of the current
 * one; two_pass: 0 runs the whole chain as one kernel per (frame, module)
 * where the geometry allows it (common-mode units that are full-height
 * column banks, at most two per module, or common mode off, with the median
 * or no common mode; columns a multiple of 4), 1 uses the common-mode + stencil kernel pair (the
 * default; pd_get_tuning reports 1 when the one-kernel form is not
 * available).
 * kernels: 1 runs the lean pair where the context allows it (the default:
 * the integer-coded bank median for units of 4096+ pixels whose pedestals
 * keep d = raw - pedestal exact inside the common-mode window, and the lean
 * band stencil for columns a multiple of 4, single-gain words, the median,
 * no or the one-stage mean common mode, subtracted before gain); 2 runs the
 * earlier kernel pair (pd_get_tuning reports 2 when the lean pair is not
 * available); 3 runs the lean pair as one persistent launch per call over a
 * work queue (bank medians of a few frames, then the stencil tiles of the
 * frames before them, so raw is re-read from L2; column-bank units, no
 * corrected frames, no matched filters; pd_get_tuning reports 1 where it
 * does not apply).
 * Results never depend on tuning. */
typedef struct {
    uint32_t chunk_frames;
    uint32_t band_rows;
    uint32_t overlap;
    uint32_t two_pass;
    uint32_t kernels;
} pd_tuning;

int pd_get_tuning(const pd_ctx* ctx, pd_tuning* tuning);
int pd_set_tuning(pd_ctx* ctx, const pd_tuning* tuning);

/* pd_autotune — choose the tuning of a context by timing candidates on the
 * caller's device frames (n_frames, 16-byte aligned): chunk sizes of about
 * 24-192 MB, band heights around the default, overlap on and off; each
 * candidate (and the one-kernel chain where available) runs once to warm
 * up and twice timed (CUDA events).  The
 * fastest is applied to the context and returned in *best (may be NULL),
 * with its time per frame in microseconds.  Allocates and frees temporary
 * device buffers; the context's summaries are saved and restored, so they
 * are unchanged.  Synchronous.  The paper has no tuner; the tile shapes of
 * a launch are this implementation's choice. */
int pd_autotune(pd_ctx* ctx, const uint16_t* frames_dev, uint32_t n_frames,
                pd_tuning* best, float* best_us_per_frame);

/* Batched launches over contexts of different geometries.  By default each
 * item runs as pd_process runs it (its context's chunks, band height and
 * two-stream overlap), item after item on the batch's stream, its common
 * mode in the batch's scratch.  With pd_batch_set_mixed(batch, 1) the
 * frames of all items are split into chunks of about 96 MB of raw data (a
 * chunk may hold frames of several items) and each chunk is one
 * persistent common-mode launch over every (item, frame, unit) of the chunk
 * and one persistent stencil launch over all its band tiles (items must
 * then use the band stencil, every geometry with at most 2048 columns per
 * module, and the median or no common mode; PD_ENOTSUP otherwise).  Either way each item is processed exactly
 * as pd_process would (same results; summaries go to the item's context),
 * and a batch can be captured once as a CUDA graph and replayed. */
typedef struct {
    pd_ctx* ctx;
    const uint16_t* frames;  /* device, 16-byte aligned                     */
    uint32_t n_frames;
    uint32_t frame_base;
    pd_outputs out;          /* as pd_process; out.cm NULL uses the batch's
                                scratch                                     */
} pd_batch_item;

typedef struct pd_batch pd_batch;

/* Allocates the device item table (max_items) and a common-mode scratch of
 * max_cm_values floats for items that pass out.cm == NULL. */
int pd_batch_create(uint32_t max_items, uint64_t max_cm_values, pd_batch** out);
/* mixed != 0: the persistent mixed-geometry launches (see above). */
int pd_batch_set_mixed(pd_batch* batch, int mixed);
/* Enqueue a batch on `stream` (asynchronous). */
int pd_batch_process(pd_batch* batch, const pd_batch_item* items, uint32_t n_items,
                     void* stream);
/* Record the same work as a CUDA graph held by the batch (replacing any
 * earlier one); `stream` must not be the legacy default stream.  Nothing
 * runs until pd_batch_replay.  The graph keeps the items' pointers: each
 * replay processes whatever the same frame buffers hold at that time. */
int pd_batch_capture(pd_batch* batch, const pd_batch_item* items, uint32_t n_items,
                     void* stream);
int pd_batch_replay(pd_batch* batch, void* stream);
void pd_batch_destroy(pd_batch* batch);

/* ---- Learned count / subpixel refinement ---------------------------------
 * The paper reports that off-the-shelf deep models lost photon information
 * and offers its fixed filters as the start of future learned models
 * (abstract; sections "Methods", "Conclusions").  pd_net is such a model: it
 * reads the 5x5 neighbourhood of a hit's seed (e / photon_kev, zero outside
 * the module) and predicts the photon count (0-4) and (dx, dy):
 *   conv3x3x32 -> ReLU -> conv3x3x32 -> ReLU -> FC64 -> ReLU -> 7 outputs
 * (5 count logits, dx, dy), 'same' zero padding.  Contractions run on the
 * tensor cores with bfloat16 operands (rounded to nearest even) and float32
 * accumulation.  Parameters are one float32 vector in the order W1 [32][9],
 * b1 [32], W2 [32][288] (column k*32 + c_in, k = 3*(dy+1) + dx+1), b2,
 * W3 [64][800] (column p*32 + c), b3, W4 [7][64], b4.
 * Loss = mean softmax cross-entropy of the count + lambda * sum of squared
 * (dx, dy) errors over hits with mask = 1, divided by n_reg. */
typedef struct pd_net pd_net;

uint32_t pd_net_num_params(void);
/* Device state for batches of up to max_batch patches; weights and biases
 * uniform in +-1/sqrt(fan_in) from a generator seeded with `seed`, Adam
 * state zero. */
int pd_net_create(uint32_t max_batch, uint64_t seed, pd_net** out);
int pd_net_set_params(pd_net* net, const float* params_host, uint32_t n_params);
int pd_net_get_params(pd_net* net, float* params_host, uint32_t n_params);
/* 5x5 patches (float [n_hits][25], device) of the hits of one pd_process
 * call: frames_dev, frame_base and cm_dev (out->cm of that call) as given
 * to / returned by it. */
int pd_net_gather(pd_ctx* ctx, const uint16_t* frames_dev, uint32_t frame_base,
                  const float* cm_dev, const pd_hit* hits_dev, uint32_t n_hits,
                  float* patches_dev, void* stream);
/* Network outputs float [n][7] (5 logits, dx, dy) for n patches (device),
 * on the tcgen05 tensor cores (bf16 operands, f32 accumulation), in chunks
 * of max_batch.  Synchronises `stream` at the end to report a timed-out
 * tensor-core pipeline wait (PD_ETIMEDOUT). */
int pd_net_forward(pd_net* net, const float* patches_dev, uint32_t n,
                   float* out_dev, void* stream);
/* Loss (added to *loss_dev if not NULL) and the gradient of every
 * parameter (float [n_params] into grads_dev if not NULL) for one batch of
 * n <= max_batch patches: counts u8 [n] (0-4), targets float [n][2],
 * mask u8 [n]. */
int pd_net_gradients(pd_net* net, const float* patches_dev, const uint8_t* counts_dev,
                     const float* targets_dev, const uint8_t* mask_dev, uint32_t n,
                     float n_reg, float lambda, float* grads_dev, float* loss_dev,
                     void* stream);
/* Rows idx_dev[0..n) (device, each < the set's size) of a training set
 * (patches float [][25], counts u8, targets float [][2], mask u8, all
 * device) into the batch arrays *_out (device, n rows each), for
 * pd_net_train_step without host work between steps.  Asynchronous on
 * `stream`.  Training batches are this implementation's (the paper trains
 * nothing). */
int pd_net_take(const float* patches_dev, const uint8_t* counts_dev, const float* targets_dev,
                const uint8_t* mask_dev, const uint32_t* idx_dev, uint32_t n,
                float* patches_out, uint8_t* counts_out, float* targets_out,
                uint8_t* mask_out, void* stream);
/* pd_net_gradients followed by one Adam step (beta 0.9 / 0.999, eps 1e-8). */
int pd_net_train_step(pd_net* net, const float* patches_dev, const uint8_t* counts_dev,
                      const float* targets_dev, const uint8_t* mask_dev, uint32_t n,
                      float n_reg, float lambda, float lr, float* loss_dev, void* stream);
/* Copy hits, replacing (dx, dy) by the network's where its softmax
 * confidence is >= conf and its most likely count is >= 1 (flag
 * PD_HIT_LEARNED), and the count too where the confidence is also >=
 * count_conf; elsewhere the classical values stay (the fallback).
 * count_conf > 1 never changes a count. */
int pd_net_refine(const float* out_dev, const pd_hit* hits_in_dev, uint32_t n,
                  float conf, float count_conf, pd_hit* hits_out_dev, void* stream);
void pd_net_destroy(pd_net* net);

/* ---- Streaming server -----------------------------------------------------
 * The paper targets real-time reduction at LCLS-II rates (100 kHz; section
 * "Introduction") and sparse photon lists that compress by about two orders
 * of magnitude over raw frames (section "Performance").  This is the online
 * form of the chain.  Continuous batching of frames of several geometries (one context each)
 * from page-locked host rings.  A producer writes a frame into a ring slot
 * (pd_server_acquire, or pd_server_ring_frame to pre-fill) and commits it
 * with its id; the commit time is its arrival time.  A dispatcher thread
 * keeps up to n_slots batches in flight, each on its own stream: when a
 * slot frees it takes every committed frame (up to max_batch_frames per
 * geometry), uploads, runs one pd_batch launch over all geometries and
 * downloads the hit counts and then the hits.  A frame's ring slot is free
 * again as soon as its upload has completed.  Latency = arrival to hits on
 * the host.  Host encoder threads then group the hits per frame, sort them
 * by pixel and encode them (pd_compress_hits format); a frame is done when
 * encoded.  Summaries accumulate in each context (running count map).
 * The device budget (bytes) bounds the slots: admission waits for a free
 * slot, and pd_server_create fails with PD_EBUSY if not even one fits. */
typedef struct pd_server pd_server;

typedef struct {
    uint32_t n_slots;           /* batches in flight at most               */
    uint32_t max_batch_frames;  /* frames per geometry per batch           */
    uint32_t ring_frames;       /* host ring slots per geometry            */
    uint32_t hits_per_frame;    /* hit capacity per frame of a batch       */
    uint64_t device_budget;     /* bytes of slot buffers; 0 = free device  *
                                 * memory at creation less 1 GiB            */
    uint32_t keep_hits;         /* 1: keep each frame's hits and stream    */
    uint32_t encode_threads;    /* host encoder threads; 0 = min(8, cores/2);
                                 * they run at nice +5, below the dispatcher */
    uint32_t max_uploading;     /* batches still uploading frames at most;  *
                                 * 0 = 1 (admission holds frames in the    *
                                 * ring while the link is this busy)       */
    uint32_t cpu_pin;           /* 0: host threads unpinned; c > 0: the     *
                                 * dispatcher runs on the (c-1)-th CPU the   *
                                 * process may use, encoder i on the         *
                                 * (c+i)-th, and the thread inside           *
                                 * pd_server_replay on the (c+encoders)-th   *
                                 * (modulo their number; Linux affinity,     *
                                 * the replaying thread's own mask is put    *
                                 * back when it returns)                     */
} pd_serve_config;

typedef struct {
    uint64_t frames_committed, frames_done, frames_rejected;
    uint64_t batches, max_batch_frames;
    uint64_t raw_bytes, compressed_bytes, hits;
    double elapsed_s;            /* first arrival to last completion        */
    double p50_us, p99_us, max_us, mean_us;
    /* latency split per frame: queued in the ring (arrival to batch issue),
     * issue to hit counts on the host (upload, kernels, count copy), then
     * to hits on the host (hit copy) */
    double wait_mean_us, wait_p99_us, device_mean_us, device_p99_us, fetch_mean_us;
    double encode_mean_us;       /* per batch and geometry: hits on the host
                                  * to all its frames encoded               */
    uint64_t replay_late;        /* replayed arrivals reached > 20 us late  */
    double replay_late_max_us;
    /* per batch on the device clock: the frames' upload, then the kernels
     * and the hit-count copy */
    double upload_mean_us, run_mean_us;
} pd_serve_stats;

int pd_server_create(pd_ctx* const* ctxs, uint32_t n_geometries, const pd_serve_config* cfg,
                     pd_server** out);
int pd_server_slots(const pd_server* server, uint32_t* n_slots);
/* hold != 0: issue no new batches (frames keep queueing in the rings);
 * 0: resume.  Batches already in flight complete. */
int pd_server_hold(pd_server* server, int hold);
/* Pointer to ring slot `slot` of a geometry (to pre-fill frames). */
int pd_server_ring_frame(pd_server* server, uint32_t geometry, uint32_t slot,
                         uint16_t** frame_host);
/* Next free slot of the geometry's ring (PD_EBUSY when the ring is full:
 * back-pressure; the frame is counted as rejected). */
int pd_server_acquire(pd_server* server, uint32_t geometry, uint16_t** frame_host,
                      uint32_t* slot);
int pd_server_commit(pd_server* server, uint32_t geometry, uint32_t slot, uint64_t frame_id);
/* Built-in producer: Poisson arrivals at rate_hz for duration_s, geometry
 * drawn with weights mix[n_geometries] (NULL = equal), each arrival commits
 * the next ring slot of its geometry (its content as pre-filled) with the
 * scheduled arrival time; ids from first_id.  Synchronous. */
int pd_server_replay(pd_server* server, double rate_hz, double duration_s, const float* mix,
                     uint64_t seed, uint64_t first_id);
/* Wait until every committed frame is done (PD_ETIMEDOUT after timeout_s). */
int pd_server_drain(pd_server* server, double timeout_s);
int pd_server_stats(pd_server* server, pd_serve_stats* stats);
int pd_server_reset_stats(pd_server* server);
/* Hits of a finished frame (keep_hits = 1), sorted by pixel, with frame =
 * the frame id; up to cap are copied, *n_hits is the full count. */
int pd_server_frame_hits(pd_server* server, uint64_t frame_id, pd_hit* out, uint32_t cap,
                         uint32_t* n_hits, float* latency_us);
/* The frame's compact hit stream (format of pd_compress_hits); *len is its
 * size (PD_EOVERFLOW if cap is smaller; out = NULL to query). */
int pd_server_frame_stream(pd_server* server, uint64_t frame_id, uint8_t* out, size_t cap,
                           size_t* len);
void pd_server_destroy(pd_server* server);

/* Compact hit stream of one frame (the sparse photon list of sections
 * "Summarization" and "Performance"): varint count, then per hit (sorted by
 * pixel) the varint pixel delta, energy u16 in 1/256 keV, dx and dy i8 in
 * 1/128 pixel (clipped), count u8.  Lossless for pixel and count. */
int pd_compress_hits(const pd_hit* hits, uint32_t n, uint8_t* out, size_t cap, size_t* out_len);
int pd_decompress_hits(const uint8_t* in, size_t len, uint32_t frame, pd_hit* out, uint32_t cap,
                       uint32_t* n_out);

/* ---- Centroid linearisation ----------------------------------------------
 * The centre-of-mass offset depends nonlinearly on where a photon landed,
 * and centroids need linearising to give positions (section "Photon
 * Subpixel Resolution", Fig. f and its caption).  With photons landing
 * uniformly inside the seed pixel, the true offset is F(d) - 1/2 with F the
 * cumulative distribution of the centroid d.  pd_eta estimates F per axis
 * from single-photon hits (count == 1, finite dx and dy): a histogram of d
 * over `bins` bins spanning [-1, 1] (centroids outside clip to the end
 * bins).  `bins` is odd so that d = 0, an atom of the distribution (all
 * neighbours below the zero threshold), lies in the middle of a bin and maps
 * to the middle of its probability mass.  For a centroid d, in float32
 * round-to-nearest in this order:
 *   t = (d + 1) * (bins * 0.5);  k = clamp(floor(t), 0, bins - 1);
 *   phi = clamp(t - k, 0, 1);  u = (C[k] + phi * h[k]) / N - 1/2
 * with h the counts, C[k] the counts below bin k and N the total.  With no
 * counts (N = 0) centroids are unchanged. */
typedef struct pd_eta pd_eta;
#define PD_MAX_ETA_BINS 4095u

/* bins: odd, 1 <= bins <= PD_MAX_ETA_BINS.  Histograms start at zero. */
int pd_eta_create(uint32_t bins, pd_eta** out);
/* Add the single-photon hits among n device hits to the histograms
 * (asynchronous on `stream`). */
int pd_eta_accumulate(pd_eta* eta, const pd_hit* hits_dev, uint32_t n, void* stream);
/* Cumulative counts of the current histograms; call before pd_eta_apply and
 * again after more pd_eta_accumulate calls (asynchronous). */
int pd_eta_finalize(pd_eta* eta, void* stream);
/* hits_out[i] = hits_in[i] with dx, dy of single-photon hits replaced by
 * their linearised values and PD_HIT_LINEARISED set; other hits are copied
 * unchanged.  hits_out may equal hits_in (asynchronous). */
int pd_eta_apply(const pd_eta* eta, const pd_hit* hits_in_dev, uint32_t n,
                 pd_hit* hits_out_dev, void* stream);
/* uint32 [2][bins]: the dx histogram, then the dy histogram (synchronous). */
int pd_eta_get_histogram(const pd_eta* eta, uint32_t* hist_host);
int pd_eta_reset(pd_eta* eta, void* stream);
void pd_eta_destroy(pd_eta* eta);

/* Kernel timing.  When enabled on a context, every kernel the context
 * launches is bracketed by CUDA events recorded on the launching stream;
 * pd_read_profile synchronises the device, reports the summed device time
 * and launch count per kernel name since the last read, and clears them.
 * Disabled by default; when disabled no event is recorded. */
#define PD_PROFILE_MAX_KERNELS 8
typedef struct {
    uint32_t n_kernels;
    char name[PD_PROFILE_MAX_KERNELS][32];
    uint32_t launches[PD_PROFILE_MAX_KERNELS];
    double total_ms[PD_PROFILE_MAX_KERNELS];
} pd_profile;

int pd_set_profiling(pd_ctx* ctx, int enable);
int pd_read_profile(pd_ctx* ctx, pd_profile* out);

const char* pd_strerror(int code);
const char* pd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PD_H */
