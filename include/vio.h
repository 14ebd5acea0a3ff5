/*
 * vio.h -- C ABI of the GB300 (sm_103a) pyramidal FAST detector with fused
 * 3x3 non-maxima suppression and one-feature-per-cell selection.
 *
 * What is computed (Nagy, Foehn, Scaramuzza, "Faster than FAST:
 * GPU-Accelerated Frontend for High-Speed VIO", IROS 2020):
 *
 *   Algorithm 1 (Section II-B): for every pyramid level, every pixel is put
 *   through the FAST segment test and scored (CRF); non-maxima suppression
 *   runs per level (NMS); then one feature per grid cell is kept over all
 *   levels (NMS-C).
 *
 *   Pyramid (Section II-B, Section III-C "each subsequent layer halves the
 *   resolution"): level k+1 is (W_k >> 1) x (H_k >> 1), each pixel the 2x2
 *   mean of level k rounded half up: (a + b + c + d + 2) >> 2.
 *
 *   Segment test (Section II-D, Eq. 1): the 16 points of the radius-3
 *   Bresenham circle are darker (I_x < I_c - thresh), brighter
 *   (I_x > I_c + thresh) or similar; the pixel is a corner when a
 *   contiguous arc of at least arc_len points is all darker or all
 *   brighter.  Pixels closer than 3 to a level border are not tested.
 *
 *   Scores (Section II-D): SAD-B = sum |I_x - I_c| over the circle;
 *   SAD-A = the same sum over the contiguous arc; MT = the largest
 *   threshold at which the pixel is still a corner; 0 if not a corner.
 *
 *   NMS (Algorithm 1, n = 1 of Section I-B): a pixel survives when its score
 *   is > 0 and >= the scores of its 8 neighbours (outside the level: 0).
 *
 *   NMS-C (Section II-B grid cells, Section II-C single grid over all
 *   levels): the level-0 image is cut into ceil(W/C) x ceil(H/C) cells of
 *   C x C pixels; a survivor (x, y) of level k belongs to cell
 *   ((x << k) / C, (y << k) / C).  Each cell reports its best survivor:
 *   highest score, then lower level, then lower y, then lower x.  The
 *   record is {x << k, y << k, k, score}; an empty cell is {-1, -1, -1, 0}.
 *   The result is unique, so the library's output is bit-exact.
 *
 * Conventions
 *   - Every call returns a vio_status; nothing aborts or prints.  Argument
 *     checks run on the host before anything is enqueued.
 *   - Device calls are asynchronous on the given stream (a cudaStream_t
 *     passed as vio_stream; NULL = the legacy default stream).  A CUDA error
 *     met while enqueuing returns VIO_ERR_CUDA; a device-side wait that ran
 *     out of time is reported by vio_sync() as VIO_ERR_TIMEOUT.
 *   - Ownership: caller-owned buffers stay caller-owned and are only read
 *     (frames) or written (outputs) by work enqueued on the stream.  The
 *     context owns its resident pyramid, cell-key, descriptor and
 *     tensor-map buffers; they grow on demand up to mem_budget_bytes
 *     (VIO_ERR_OOM past it).
 *   - Threading: a context serves one host thread at a time.
 */
#ifndef VIO_H_
#define VIO_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VIO_ABI_VERSION 2
#define VIO_MAX_LEVELS 5

typedef struct vio_ctx vio_ctx;
/* A cudaStream_t, declared without pulling in the CUDA headers. */
typedef struct CUstream_st* vio_stream;

typedef enum {
    VIO_OK = 0,
    VIO_ERR_INVALID_ARG = 1, /* an argument is outside its documented range */
    VIO_ERR_OOM = 2,         /* device memory or the context budget ran out */
    VIO_ERR_CUDA = 3,        /* a CUDA runtime/driver call failed            */
    VIO_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up           */
    VIO_ERR_BUSY = 5,        /* serving queue full                           */
    VIO_ERR_UNSUPPORTED = 6, /* the device is not an sm_103 GPU              */
    VIO_ERR_NOT_FOUND = 7    /* unknown serving ticket                       */
} vio_status;

typedef enum { VIO_SCORE_SAD_B = 0, VIO_SCORE_SAD_A = 1, VIO_SCORE_MT = 2 } vio_score;

typedef struct {
    int device;              /* CUDA device ordinal                                  */
    size_t mem_budget_bytes; /* 0 = no limit beyond device memory                    */
    int max_frames;          /* most frames one vio_detect call may carry (1..1024)  */
    int score;               /* a vio_score                                          */
    int autotune;            /* 1 = time tile shapes on the first call of a shape    */
    int use_graphs;          /* 1 = replay each batch shape as a captured CUDA graph */
    int profile;             /* 1 = record CUDA events around each stage (vio_stage_ms) */
    int nms_radius;          /* 1..4: non-maximum suppression keeps a pixel whose score
                                is >= every score of its (2r+1) x (2r+1) neighbourhood
                                (Section I-B; Table III compares r = 1..4)           */
} vio_config;

/* One frame: width, height, row pitch in bytes (pitch >= w). */
typedef struct {
    int32_t w, h, pitch;
} vio_dims;

/* One cell of the output grid (16 bytes); empty cell = {-1, -1, -1, 0}. */
typedef struct {
    int32_t x, y, level, score;
} vio_feature;

/* Fills *cfg with the defaults: device 0, no budget, 64 frames, SAD-B,
 * autotune off, graphs on, profiling off, 3 x 3 NMS (radius 1). */
void vio_config_default(vio_config* cfg);

/* Copies the configuration the context was created with into *out.
 * Errors: VIO_ERR_INVALID_ARG for NULL pointers. */
vio_status vio_get_config(const vio_ctx* ctx, vio_config* out);

/* Creates a context on cfg->device.  *out receives the context or NULL.
 * Errors: VIO_ERR_INVALID_ARG (NULL pointers, ranges), VIO_ERR_UNSUPPORTED
 * (device is not compute capability 10.3), VIO_ERR_CUDA, VIO_ERR_OOM. */
vio_status vio_create(vio_ctx** out, const vio_config* cfg);

/* Waits for the context's work, frees all of its buffers.  NULL is a no-op. */
vio_status vio_destroy(vio_ctx* ctx);

/* Static English description of a status. */
const char* vio_status_str(vio_status s);

/* The last error message recorded by the context (static storage of the
 * context, valid until its next call). */
const char* vio_last_error(const vio_ctx* ctx);

/* Number of cells ceil(w/cell) * ceil(h/cell); 0 when an argument is < 1. */
size_t vio_num_cells(int w, int h, int cell_size);

/*
 * Detects features in n_frames frames with one batched launch.
 *
 *   frames     host array of n_frames DEVICE pointers to uint8 frames.  A
 *              frame whose address is not 16-byte aligned or whose pitch is
 *              not a multiple of 16 is first copied into a context slot.
 *   dims       host array of n_frames vio_dims.
 *   thresh     0..255 (>= 1 when the context scores with MT, whose score
 *              would otherwise be 0 for a corner).
 *   arc_len    9..16.
 *   cell_size  a positive multiple of 32 (Section II-C: cell widths are
 *              multiples of the 32-thread warp), or 0: the context picks 32
 *              or 64 (the autotuner times both when autotune is on, else
 *              32); out_cells must then hold vio_num_cells(w_i, h_i, 32)
 *              records per frame, and vio_get_tuning reports the size used.
 *   levels     1..VIO_MAX_LEVELS; the smallest level must be >= 7 x 7.
 *   out_cells  host array of n_frames DEVICE pointers, frame i receiving
 *              vio_num_cells(w_i, h_i, cell_size) vio_feature records in
 *              row-major cell order.
 *   out_counts DEVICE int32[n_frames] receiving the number of non-empty
 *              cells per frame, or NULL.
 *
 * Each frame must satisfy 7 <= w <= 65535, 7 <= h <= 65535 and
 * w * h < 2^28 (the kernels find a level pixel's cell with a multiply-high
 * that is exact for level coordinates below 2^16; larger frames return
 * VIO_ERR_INVALID_ARG).  Asynchronous on `stream`.  Errors:
 * VIO_ERR_INVALID_ARG, VIO_ERR_OOM, VIO_ERR_CUDA.
 */
vio_status vio_detect(vio_ctx* ctx, const uint8_t* const* frames, const vio_dims* dims, int n_frames,
                      int thresh, int arc_len, int cell_size, int levels,
                      vio_feature* const* out_cells, int32_t* out_counts, vio_stream stream);

/*
 * Parameter sweep over one set of frames: detection p (p < n_params) uses
 * thresholds[p] and arc_lens[p] and gives exactly what vio_detect would;
 * the pyramid is built once and read by every detection.
 *
 *   thresholds, arc_lens  host int[n_params], 1 <= n_params <= 64
 *   out_cells             host array of n_params * n_frames DEVICE pointers,
 *                         parameter-major: entry p * n_frames + i is frame i
 *                         of detection p
 *   out_counts            DEVICE int32[n_params * n_frames] (same order) or NULL
 *
 * Other arguments, checks and errors as vio_detect (7 <= w, h <= 65535,
 * w * h < 2^28).  Asynchronous on `stream`.
 */
vio_status vio_detect_sweep(vio_ctx* ctx, const uint8_t* const* frames, const vio_dims* dims, int n_frames,
                            const int* thresholds, const int* arc_lens, int n_params, int cell_size, int levels,
                            vio_feature* const* out_cells, int32_t* out_counts, vio_stream stream);

/*
 * Same as vio_detect for frames and results in HOST memory; the call returns
 * when host_cells (host, per frame) and host_counts (host int32[n_frames] or
 * NULL) are written.  Upload: frames that lie one after another in host
 * memory (address and pitch multiples of 16, rows padded by at most 256
 * bytes, at most 4096 bytes between a frame's last pixel and the next
 * frame) are copied as one span by one copy-engine copy (a copy costs about
 * 2 us on top of its bytes, so 64 frames in one buffer upload about 1.5x
 * faster than 64 separate ones); frames alone in pinned (page-locked)
 * memory with address and pitch multiples of 16, when a call with more than
 * one level holds at least 4 of them, are read by the pyramid kernel through
 * their device mapping, which also writes the device copy of level 0 (one
 * pass over the host link, overlapped with the pyramid, no copy each); other
 * frames are copied one by one.  Records for pinned, 16-byte aligned
 * host_cells are written in place by the decode kernel; others come back
 * through a staging copy.  Frame sizes and the other arguments are checked
 * as by vio_detect (7 <= w, h <= 65535, w * h < 2^28).
 */
vio_status vio_detect_host(vio_ctx* ctx, const uint8_t* const* host_frames, const vio_dims* dims,
                           int n_frames, int thresh, int arc_len, int cell_size, int levels,
                           vio_feature* const* host_cells, int32_t* host_counts, vio_stream stream);

/*
 * Asynchronous form of vio_detect_host for pipelining batches: it enqueues
 * the copy of the frames into one of three rotating device input slots (copy
 * engines; frames that lie one after another in host memory as one span, as
 * in vio_detect_host), the detection and the result writes on `stream` and
 * returns.
 * The results are valid after vio_sync(ctx, stream).  Calls on different
 * streams overlap their frame copies with the previous call's kernels (the
 * kernels of one context still run one call after another).
 *
 *   host_frames  HOST frames, pinned or pageable (pageable frames make the
 *                copy synchronous); they must stay unchanged until the call
 *                completes
 *   host_cells   PINNED host arrays, 16-byte aligned, written in place by the
 *                device; they must not be read or reused before completion
 *   host_counts  PINNED host int32[n_frames] or NULL
 *
 * Errors: VIO_ERR_INVALID_ARG (as vio_detect, including 7 <= w, h <= 65535
 * and w * h < 2^28, or host_cells / host_counts not pinned), VIO_ERR_OOM,
 * VIO_ERR_CUDA.
 */
vio_status vio_detect_host_async(vio_ctx* ctx, const uint8_t* const* host_frames, const vio_dims* dims,
                                 int n_frames, int thresh, int arc_len, int cell_size, int levels,
                                 vio_feature* const* host_cells, int32_t* host_counts, vio_stream stream);

/* Stage durations of the context's most recent vio_detect call, in ms:
 * ms[0] pyramid, ms[1] fused FAST + NMS + cell max, ms[2] decode.  Needs
 * profile = 1 in the config; waits for that call to finish.  The events are
 * recorded on the call's stream (inside the replayed graph when graphs are
 * on), so the figures are device time of each kernel. */
vio_status vio_stage_ms(vio_ctx* ctx, float* ms3);

/* Copies level `level` (0 .. levels-1) of frame `frame` of the context's
 * most recent detection call (vio_detect, vio_detect_host[_async],
 * vio_detect_sweep) into dst: (w >> level) x (h >> level) pixels, rows of
 * dst_pitch bytes, dst in device or host memory; asynchronous on `stream`
 * (order it after the detection, e.g. the same stream).  Level 0 is the frame
 * the detection read (the caller's, or its staged copy); levels >= 1 are the
 * context's resident pyramid (Section II-B), valid until the context's next
 * detection call.  A diagnostic of the pyramid stage.  Errors:
 * VIO_ERR_INVALID_ARG (no detection yet, frame or level out of range, NULL
 * dst, dst_pitch < the level's width), VIO_ERR_CUDA. */
vio_status vio_copy_level(vio_ctx* ctx, int frame, int level, uint8_t* dst, int dst_pitch, vio_stream stream);

/* Waits for all work the context enqueued on `stream` and reports any
 * device-side status: VIO_ERR_TIMEOUT when a bounded wait gave up,
 * VIO_ERR_CUDA when the decode found a cell key that does not lie in its
 * cell (corrupted keys).  The status word is cleared. */
vio_status vio_sync(vio_ctx* ctx, vio_stream stream);

/* Diagnostic of the failure path: runs one warp that waits, with the same
 * bounded mbarrier wait the detect kernels use, on a barrier nothing ever
 * completes, limited to limit_us microseconds (1..1000000).  The kernel
 * records the timeout in the context's status word and returns; the call
 * waits for it and returns VIO_ERR_TIMEOUT (the status word is cleared, the
 * context stays usable).  Any other status means the mechanism failed. */
vio_status vio_selftest_timeout(vio_ctx* ctx, uint32_t limit_us);

/*
 * Launch configuration of the fused kernel.  tile_w x tile_h level pixels per
 * work item (tile_h / 8 score rows per warp: the warp-to-row mapping),
 * cta_per_sm resident CTAs per SM of the persistent launch (0 = as many as
 * fit), nms_radius the NMS window the variant was built for, cell_size the
 * grid cell size of the detection.
 *
 * vio_get_tuning reports the configuration of the context's most recent
 * detection (cta_per_sm resolved to the count launched; cell_size the one
 * used, also when vio_detect was given cell_size 0).  vio_set_tuning pins a
 * variant and a CTA count for later calls (NULL unpins; VIO_ERR_INVALID_ARG
 * if the variant is not one of the built ones, was built for another NMS
 * radius than the context's, or cta_per_sm is outside 0..4); its tile_w,
 * tile_h, nms_radius and cell_size fields are ignored.  With autotune on and
 * nothing pinned, the first vio_detect of a batch shape times every
 * combination of the radius's variants, 2 to 4 CTAs per SM (as far as they
 * fit) and, when cell_size is 0, cells of 32 and 64, and keeps the fastest
 * for that shape; vio_autotune_log returns what that run timed.
 */
typedef struct {
    int tile_w, tile_h, cta_per_sm, variant, nms_radius, cell_size;
} vio_tuning;

vio_status vio_get_tuning(const vio_ctx* ctx, vio_tuning* out);
vio_status vio_set_tuning(vio_ctx* ctx, const vio_tuning* t);
/* The configurations the context's most recent tuning run timed and the
 * device time of each, in ms per detection call (CUDA events over 5 calls
 * after 2 untimed ones): copies up to cap entries, returns how many there
 * are (0 before any tuning run; -1 for a NULL context). */
int vio_autotune_log(const vio_ctx* ctx, vio_tuning* configs, float* ms, int cap);
/* Number of built variants and the shape of variant i. */
int vio_num_variants(void);
vio_status vio_variant(int i, vio_tuning* out);

/* CUDA device ordinal of the context, or -1 for NULL. */
int vio_device(const vio_ctx* ctx);

/*
 * Serving: frames of many camera streams and sizes are submitted one by one
 * from host memory; a scheduler thread owned by the context batches the
 * pending frames into the next free lane (a CUDA stream with its own
 * resident buffers), so frames that arrive while other batches are on the
 * GPU are admitted as soon as a lane and device memory free up, and batches
 * on different lanes overlap on the device.  Every frame's result is the
 * same as a vio_detect of that frame alone.
 */
typedef struct {
    int thresh, arc_len, cell_size, levels; /* detection parameters, as vio_detect          */
    int max_batch;          /* most frames per launch (1..1024)                             */
    int max_wait_us;        /* a partial batch waits until its oldest frame is this old      */
    int lanes;              /* launches in flight at once, one CUDA stream each (1..8)       */
    size_t mem_budget_bytes;/* device bytes for the frames in flight (inputs, pyramid, keys, */
                            /* cells); 0 = unbounded                                         */
    int queue_capacity;     /* pending frames before vio_submit returns VIO_ERR_BUSY         */
    int keep_results;       /* 1 = keep each result until vio_poll takes it; 0 = stats only  */
} vio_serve_config;

typedef struct {
    uint64_t submitted, completed, rejected, batches;
    double mean_batch;      /* frames per launch                                             */
    double p50_us, p99_us, max_us, mean_us; /* submit -> cells in host memory, per frame      */
    double frames_per_s;    /* completed frames / (last completion - first submit)           */
    /* evidence of batching and overlap: */
    uint64_t max_batch_frames;   /* most frames one launch carried                           */
    uint64_t max_lanes_in_flight;/* most lanes with a launched, not yet retired batch at once */
    uint64_t overlapped_batches; /* batches whose device-time interval (CUDA events around the
                                    lane's work: upload, kernels, result copy) overlapped the
                                    interval of a batch on another lane                       */
} vio_serve_stats_t;

/* Defaults: thresh 15, arc 9, cell 32, levels 3, batch 32, no wait, 3 lanes,
 * 4 GiB budget, 65536 queue slots, results kept. */
void vio_serve_config_default(vio_serve_config* cfg);

/* Starts the scheduler thread of ctx.  VIO_ERR_BUSY if already serving. */
vio_status vio_serve_start(vio_ctx* ctx, const vio_serve_config* cfg);

/* Queues one frame.  host_frame must stay valid and unchanged until the
 * frame completes (pinned memory lets its copy overlap other work).
 * *ticket identifies the frame for vio_poll.  Errors: VIO_ERR_INVALID_ARG
 * (not serving, or dims outside vio_detect's limits: 7 <= w, h <= 65535,
 * w * h < 2^28, pitch >= w), VIO_ERR_BUSY (queue full), VIO_ERR_OOM (frame
 * larger than the budget), or the scheduler's own error. */
vio_status vio_submit(vio_ctx* ctx, int stream_id, const uint8_t* host_frame, vio_dims dims, uint64_t* ticket);

/* *done = 1 and the frame's cells (vio_num_cells records) and non-empty
 * count copied out when the frame has completed (the result is then
 * released); *done = 0 otherwise.  host_out / count may be NULL.
 * VIO_ERR_NOT_FOUND for a ticket never issued or already taken. */
vio_status vio_poll(vio_ctx* ctx, uint64_t ticket, vio_feature* host_out, int32_t* count, int* done);

/* Waits until every submitted frame has completed (VIO_ERR_TIMEOUT after
 * timeout_ms). */
vio_status vio_serve_drain(vio_ctx* ctx, int timeout_ms);

/* Counters and latency percentiles of the frames completed so far. */
vio_status vio_serve_stats(vio_ctx* ctx, vio_serve_stats_t* out);

/* Finishes the queued frames, stops the scheduler, frees the lanes. */
vio_status vio_serve_stop(vio_ctx* ctx);

/*
 * Detection of one frame that allocates nothing.  The paper has no
 * counterpart; this entry point exists for callers that cannot allocate when
 * they need a detection: code running under a memory pool that accounts for
 * every byte, real-time loops that may not pay cudaMalloc's device-wide
 * synchronisation and unbounded latency, or plug-ins whose host process owns
 * all allocations.  No context is used.  The working memory besides the
 * caller's frame and outputs (call block, counters, cell keys, pyramid
 * levels) is one fixed array of VIO_NOALLOC_SCRATCH_BYTES that the library
 * keeps on every device that loads it, until the process exits.
 *
 *   frame      DEVICE pointer, 16-byte aligned, dims.pitch a multiple of 16
 *   dims       as vio_detect (7 <= w, h <= 65535); the frame must also fit
 *              the array:
 *              4096 + 8 * cells (rounded up to 256)
 *              + sum over k >= 1 of round_up(w >> k, 128) * (h >> k),
 *              each level rounded up to 256, must not exceed
 *              VIO_NOALLOC_SCRATCH_BYTES (frames up to 3840 x 2160 at 4
 *              levels fit); larger frames return VIO_ERR_INVALID_ARG
 *              before anything is enqueued
 *   thresh, arc_len, cell_size, levels   as vio_detect
 *   score      a vio_score
 *   out_cells  DEVICE, vio_num_cells(w, h, cell_size) records
 *   out_count  DEVICE int32 receiving the non-empty cell count, or NULL
 *
 * Asynchronous on `stream`; the results equal vio_detect's.  Every call
 * shares the one array and clears the parts that must start at zero, so
 * calls that overlap on the GPU (another stream, another host thread) race
 * and must be serialised by the caller.  The first call on each device sets
 * up that device (it looks up the array's device address, with the device
 * current); make that first call before any stream capture.  The device-side
 * checks are not reported here: a bounded wait that expires, or a decoded
 * cell key that lies outside its cell, is recorded in the array's status
 * word, which this entry point never reads back (use vio_detect and vio_sync
 * where that matters).  Errors: VIO_ERR_INVALID_ARG,
 * VIO_ERR_UNSUPPORTED (not an sm_103 device), VIO_ERR_CUDA.
 */
#define VIO_NOALLOC_SCRATCH_BYTES (4u << 20)
vio_status vio_detect_noalloc(const uint8_t* frame, vio_dims dims, int thresh, int arc_len, int cell_size,
                              int levels, int score, vio_feature* out_cells, int32_t* out_count, vio_stream stream);

/*
 * Feature tracker (Section II-E, Eqs. 2-6): the pyramidal approximated
 * simultaneous inverse compositional Lucas-Kanade tracker.  For each feature
 * at a level-0 position (x, y) of a previous frame it estimates the
 * translation t = (t_x, t_y) and the affine intensity change (alpha, beta)
 * such that  next(p + t) ~ (1 + alpha) prev(p) + beta  over a square patch
 * around the feature, coarse to fine over a pyramid built like the
 * detector's (Section II-B).  Per level: the template patch and its
 * central-difference gradients are sampled once (bilinear), the Hessian
 * H = sum U U^T with U = [(1+alpha) dT/dx, (1+alpha) dT/dy, T, 1] (Eq. 4) is
 * formed once with the appearance at the start of the level, and each
 * iteration solves dq = H^-1 sum U r, r = next(p + t) - (1+alpha) T - beta
 * (Eq. 6), then t -= dt, alpha += d_alpha, beta += d_beta.  One warp tracks
 * one feature (Section II-E) and sums over the patch with a butterfly of
 * warp shuffles.  Arithmetic is fp32.
 *
 * Readings: a level-0 position x is (x + 0.5) / 2^k - 0.5 on level k; the
 * patch is P x P samples at offsets i - (P - 1) / 2; bilinear samples need
 * 0 <= x <= W_k - 2 and 0 <= y <= H_k - 2, and a sample outside it, or a
 * Hessian that is not positive definite, loses the track; the translation
 * doubles from one level to the next finer one.
 */
enum { VIO_TRACK_GAIN = 1, VIO_TRACK_OFFSET = 2 };

typedef struct {
    int levels;        /* 1..VIO_MAX_LEVELS; the smallest level must be >= 7 x 7          */
    int patch_fine;    /* patch side on level 0: 8 or 16                                    */
    int patch_coarse;  /* patch side on levels >= 1: 8 or 16                                */
    int max_iters;     /* iterations per level, 1..100                                      */
    float min_update;  /* a level ends when |dt| < min_update (pixels of that level); >= 0  */
    int model;         /* VIO_TRACK_GAIN | VIO_TRACK_OFFSET bits: parameters estimated      */
} vio_track_params;

/* One tracked feature (32 bytes). */
typedef struct {
    float x, y;          /* level-0 position in the next frame                         */
    float gain, offset;  /* alpha, beta                                                 */
    int32_t status;      /* 1 = tracked, 0 = lost                                       */
    int32_t iters;       /* iterations over all levels                                  */
    float residual;      /* RMS of the residual in the last iteration on level 0        */
    int32_t reserved;
} vio_track_result;

/* Fills *p with the defaults: 3 levels, 16 x 16 on level 0, 8 x 8 above,
 * 30 iterations, min_update 0.01, gain and offset estimated. */
void vio_track_params_default(vio_track_params* p);

/*
 * Tracks n_pts[i] features from prev[i] to next[i] for i < n_pairs, one
 * launch for all pairs.
 *
 *   prev, next  host arrays of n_pairs DEVICE pointers to uint8 frames; pair
 *               i has both frames of size dims[i] (pitch dims[i].pitch).
 *               Frames whose address or pitch is not a multiple of 16 are
 *               first copied into a context slot.
 *   pts         host array of n_pairs DEVICE pointers to float[2 * n_pts[i]]
 *               level-0 positions (x, y) in prev[i]
 *   n_pts       host int[n_pairs], each >= 0
 *   params      NULL for the defaults
 *   out         host array of n_pairs DEVICE pointers, pair i receiving
 *               n_pts[i] records
 *
 * Asynchronous on `stream`.  Errors: VIO_ERR_INVALID_ARG (NULL pointers,
 * ranges, frames smaller than the pyramid allows), VIO_ERR_OOM, VIO_ERR_CUDA.
 */
vio_status vio_track(vio_ctx* ctx, const uint8_t* const* prev, const uint8_t* const* next, const vio_dims* dims,
                     int n_pairs, const float* const* pts, const int* n_pts, const vio_track_params* params,
                     vio_track_result* const* out, vio_stream stream);

/*
 * vio_track on the detector's output: the features are the records of a
 * vio_detect / vio_detect_host call on prev[i] (DEVICE arrays of n_cells[i]
 * vio_feature, one per grid cell), tracked from their (x, y).  out[i]
 * receives one record per cell; an empty cell (level < 0) gives
 * {x = -1, y = -1, gain 0, offset 0, status 0, iters 0, residual 0}.  This is
 * the frontend loop of the paper (detect on one frame, track into the next)
 * without any copy of the features in between.  Arguments and errors as
 * vio_track.
 */
vio_status vio_track_cells(vio_ctx* ctx, const uint8_t* const* prev, const uint8_t* const* next,
                           const vio_dims* dims, int n_pairs, const vio_feature* const* cells, const int* n_cells,
                           const vio_track_params* params, vio_track_result* const* out, vio_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* VIO_H_ */
