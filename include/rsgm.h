/*
 * rsgm.h -- C ABI of the reduced-space SGM + per-pixel Kalman library (librsgm).
 *
 * The library runs, on one CUDA device, the per-frame path of "Computationally
 * efficient dense moving object detection based on reduced space disparity
 * estimation" (Popovic, Hadviger, Markovic, Petrovic):
 *
 *   1. prediction of the previous disparity and variance through the known
 *      ego-motion (Section 2.4, Eqs. 2-4), zoom-hole filling and the
 *      discontinuity reset (Section 2.4);
 *   2. census transform and Hamming matching cost (Section 2.1) over a per-pixel
 *      disparity window centred on the prediction ("two values for each pixel
 *      that define the range for disparity search", Section 2);
 *   3. multi-path cost aggregation, Eq. 1 (Section 2.2), and winner-takes-all
 *      (Section 2.3);
 *   4. the per-pixel scalar Kalman correction, Eqs. 5-6 (Section 2.4);
 *   5. a per-pixel moving-object gate on the innovation (Section 4 detects
 *      moving objects where predicted and measured disparity differ).
 *
 * A handle ("stream" below) holds B >= 1 camera streams of identical geometry
 * (width, height, disparity range) that advance one frame per call, in
 * lockstep; each has its own state and its own ego-motion.  All work is
 * enqueued on the CUDA stream given at init; calls return before it finishes.
 *
 * Conventions.
 *   - Images are uint8, row-major, pitch = width, stream-major:
 *     element (b, y, x) at b*H*W + y*W + x.  Per-pixel outputs use the same
 *     layout.
 *   - Ego-motion of stream b: X_k = R_b X_{k-1} + t_b, metres, left-camera
 *     frame (x right, y down, z forward); R_b row-major 3x3.  This is the
 *     metric form of the paper's 4x4 H^k_{k-1} acting on (x, y, d, 1).
 *   - K is the row-major 3x3 pinhole matrix [fx 0 cx; 0 fy cy; 0 0 1] of the
 *     rectified left camera (zero skew); d = fx * baseline / Z; pixel centres
 *     sit at integer coordinates.
 *
 * Pointers.  Image inputs and state outputs may be device pointers or host
 * pointers (pinned or pageable); host data is copied through library-owned
 * device buffers on the handle's stream.  With host outputs, call rsgm_sync
 * before reading them.  Arrays passed by value (R, t, K) are copied during the
 * call.  Input buffers must stay valid and unchanged until the enqueued work
 * has completed.
 *
 * Errors.  Every function returns RSGM_OK (0) or a negative status.  Argument
 * errors are detected before any work is enqueued and leave the handle
 * unchanged.  Asynchronous device errors surface as RSGM_ERR_CUDA at a later
 * call or at rsgm_sync; rsgm_last_error() gives a text description of the
 * calling thread's most recent failure.
 */
#ifndef RSGM_H_
#define RSGM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RSGM_OK 0
#define RSGM_ERR_INVALID_ARG (-1) /* bad pointer, size or parameter */
#define RSGM_ERR_NO_STATE (-2)    /* reduced frame before any full frame / set_state */
#define RSGM_ERR_OOM (-3)         /* device allocation failed at init */
#define RSGM_ERR_CUDA (-4)        /* a CUDA runtime call or kernel failed */
#define RSGM_ERR_TIMEOUT (-5)     /* reserved: a bounded device wait expired */
#define RSGM_ERR_CHECK_FAILED (-6) /* a device-side consistency check failed */

/* Search-window rule for pixels with a valid prediction (Section 2.4). */
#define RSGM_RADIUS_FIXED 0     /* [c - radius, c + radius], c = round(d_pred) */
#define RSGM_RADIUS_VARIANCE 1  /* half-width ceil(p_pred) clamped to [1, D]: the paper's d +- p */
#define RSGM_RADIUS_FULL 2      /* whole range [0, D): plain SGM + Kalman ("plain form") */
#define RSGM_RADIUS_LEARNED 3   /* half-width and measurement variance per pixel from an attached
                                   network (rsgm_attach_cnn); r_meas is then unused */

#define RSGM_MAX_BATCH 256
#define RSGM_MAX_DISP 256

typedef struct rsgm_stream_s *rsgm_stream; /* opaque, owned by the library */

/*
 * Parameters.  Paper-fixed defaults (Table 1): 5x5 census, P1 = 6, P2 = 65,
 * 8 paths, 128 disparities.  The remaining defaults are readings of the
 * paper: q = 0.15 px^2 (more than 99 % of ego-motion errors within +-1 px,
 * Section 3.1), r_meas = 1 px^2, p_reset = D^2/12 (variance of a uniform
 * distribution over the whole range, Section 2.4), tau_disc = 2 px,
 * gate_gamma = 6.635 (chi-square, 1 degree of freedom, 99 %).
 */
typedef struct {
    int32_t width, height;   /* pixels, >= 1 */
    int32_t max_disp;        /* D: disparities 0 .. D-1, 1 <= D <= RSGM_MAX_DISP */
    int32_t batch;           /* B camera streams per handle, 1 <= B <= RSGM_MAX_BATCH */
    int32_t census_w, census_h; /* odd, <= 15, census_w * census_h - 1 <= 64 bits */
    uint32_t path_mask;      /* bit i enables direction i; 0x0F non-diagonal, 0xF0 diagonal, 0xFF all */
    int32_t radius_mode;     /* RSGM_RADIUS_* */
    int32_t radius;          /* half-width for RSGM_RADIUS_FIXED, >= 0 */
    int32_t P1, P2;          /* Eq. 1 penalties, 0 .. 4000 */
    float q;                 /* process noise (Eq. 4), >= 0 */
    float r_meas;            /* measurement noise (Eq. 6), > 0 */
    float p_reset;           /* variance after a discontinuity reset; <= 0 selects D^2/12 */
    float tau_disc;          /* discontinuity threshold, px, >= 0 */
    float gate_gamma;        /* moving-object gate: nu^2 > gamma (p_pred + r_meas), > 0 */
} rsgm_params;

/* Path directions r = (dx, dy) by path_mask bit: the predecessor of p is p - r.
 *   bit 0 (+1, 0)  bit 1 (-1, 0)  bit 2 (0, +1)  bit 3 (0, -1)
 *   bit 4 (+1,+1)  bit 5 (-1,-1)  bit 6 (-1,+1)  bit 7 (+1,-1)            */

/* Fills *p with the defaults above for a width x height, D = 128, B = 1
 * stream.  Returns RSGM_ERR_INVALID_ARG if p is NULL. */
int rsgm_default_params(rsgm_params *p, int32_t width, int32_t height);

/*
 * Creates a handle on the current CUDA device and allocates, once, every
 * device buffer the path needs at its worst case (every pixel searching the
 * whole range): about B*W*H*(3*D + 70) bytes.  cuda_stream is a cudaStream_t
 * (NULL = the legacy default stream); all later work of the handle is
 * enqueued on it.  Requires B*W*H*round4(D) < 2^32, round4(D) = D rounded up
 * to a multiple of 4 (each pixel's window is stored as a 4-aligned run of
 * cells).  On error *out is set to NULL.
 */
int rsgm_init_stream(rsgm_stream *out, const rsgm_params *p, void *cuda_stream);

/* Device bytes rsgm_init_stream allocates for these parameters (for
 * admission control by memory footprint). */
int rsgm_footprint(const rsgm_params *p, uint64_t *bytes);

/*
 * The initial frame (Section 2.4, last paragraph: limits initially cover the
 * whole search space, i.e. conventional SGM).  Every pixel searches [0, D);
 * the state becomes d = d_z (the measurement), p = r_meas; the mask is 0.
 * left, right: B*H*W uint8 each (device or host pointers).
 */
int rsgm_full_frame(rsgm_stream s, const uint8_t *left, const uint8_t *right);

/*
 * One frame of the method for all B streams: predict the previous state
 * through (R_b, t_b), search each pixel's window, aggregate (Eq. 1), take the
 * winner, correct (Eqs. 5-6) and gate.  R: B*9 floats, t: B*3 floats, K: 9
 * floats, all host memory, copied during the call; baseline in metres (> 0).
 * Returns RSGM_ERR_NO_STATE if some stream of the handle has no state yet.
 */
int rsgm_reduced_frame(rsgm_stream s, const uint8_t *left, const uint8_t *right,
                       const float *R, const float *t, const float *K, float baseline);

/*
 * One frame in which each of the handle's B streams ("slots") has its own
 * role, for serving many camera streams from one handle: a slot's stream
 * advances only when its next frame has arrived, and a slot freed by a
 * finished stream takes a new stream, which starts with a full-range frame.
 *   RSGM_SLOT_IDLE     the stream does not advance: no cells are searched
 *                      and its state and per-pixel outputs stay as they are
 *   RSGM_SLOT_REDUCED  a frame of the method, exactly as rsgm_reduced_frame
 *   RSGM_SLOT_FULL     an initial frame, exactly as rsgm_full_frame (the
 *                      paper's first frame: the whole range, Section 2.4)
 * roles: host array of B bytes.  left, right: B*H*W uint8 each (device or
 * host); every slot's images are read, but only those of advancing slots
 * matter.  R, t, K, baseline as in rsgm_reduced_frame (R and t of idle and
 * full slots are ignored).  A slot's results do not depend on the roles of
 * the others.  A reduced slot without a state: RSGM_ERR_NO_STATE; a role
 * other than the three: RSGM_ERR_INVALID_ARG.  All slots idle: nothing is
 * enqueued.
 */
#define RSGM_SLOT_IDLE 0
#define RSGM_SLOT_REDUCED 1
#define RSGM_SLOT_FULL 2
int rsgm_slot_frame(rsgm_stream s, const uint8_t *roles, const uint8_t *left, const uint8_t *right,
                    const float *R, const float *t, const float *K, float baseline);

/*
 * Copies the current state out: disparity d (float), variance p (float),
 * moving-object mask (uint8, 1 = gated), integer winner (int16).  Each
 * B*H*W elements; any pointer may be NULL to skip it; device or host memory.
 */
int rsgm_state(rsgm_stream s, float *disp, float *var, uint8_t *moving_mask, int16_t *disp_int);

/* Imports a state (B*H*W floats each, device or host), e.g. to resume a
 * checkpointed stream; the next rsgm_reduced_frame predicts from it. */
int rsgm_set_state(rsgm_stream s, const float *disp, const float *var);

/* Intermediate buffers of the most recent frame, for inspection and tests. */
#define RSGM_BUF_CENSUS_L 0   /* uint64 per pixel */
#define RSGM_BUF_CENSUS_R 1   /* uint64 per pixel */
#define RSGM_BUF_WINDOW 2     /* uint32 per pixel: lo | (width << 16) */
#define RSGM_BUF_OFFSET 3     /* uint32 per pixel: first cell of the pixel's window in the
                                 RSGM_BUF_COST / _AGGREGATED layout (prefix sum of the widths) */
#define RSGM_BUF_CLASS 4      /* uint8 per pixel: 0 predicted, 1 discontinuity reset, 2 no prediction,
                                 3 idle slot (rsgm_slot_frame) */
#define RSGM_BUF_D_PRED 5     /* float per pixel: predicted disparity (undefined where class 2) */
#define RSGM_BUF_P_PRED 6     /* float per pixel: predicted variance (undefined where class 2) */
#define RSGM_BUF_COST 7       /* uint8 per cell, N cells: ragged cost volume, pixels' windows
                                 back to back in raster order */
#define RSGM_BUF_AGGREGATED 8 /* uint16 per cell: S, the sum over enabled paths of Eq. 1 */
#define RSGM_BUF_D_MEAS 9     /* float per pixel: sub-pixel measurement d_z */
#define RSGM_BUF_INNOVATION 10 /* float per pixel: d_z - d_pred (0 where class 2) */
/* RSGM_RADIUS_LEARNED handles only (the latest reduced frame): */
#define RSGM_BUF_CNN_INPUT 11 /* bfloat16 x 16 per pixel: the network's 4 inputs, then 12 zeros */
#define RSGM_BUF_CNN_OUTPUT 12 /* float x 8 per pixel: 5 class logits, log r, 2 unused */
#define RSGM_BUF_RADIUS 13    /* uint8 per pixel: the decided half-width */
#define RSGM_BUF_R_MEAS 14    /* float per pixel: the decided measurement variance */

/* Copies buffer `which` into dst (device or host) if capacity >= its size;
 * *bytes receives the size (may be queried with dst = NULL).  Synchronises
 * the handle's stream. */
int rsgm_read_buffer(rsgm_stream s, int which, void *dst, size_t capacity, size_t *bytes);

/* Frames processed (summed over the B streams) and cost cells searched
 * (summed over frames) since init; cells of the last frame.  Synchronises. */
int rsgm_counters(rsgm_stream s, uint64_t *frames, uint64_t *cells, uint64_t *last_cells);

/*
 * Displayed disparity: the 3x3 median of the current state's d (Section 2.3:
 * a block median filter in postprocessing, outside the Kalman loop, so it
 * does not change the state).  Border pixels use clamped coordinates.  out:
 * B*H*W floats, device or host (host: call rsgm_sync before reading).
 */
int rsgm_median(rsgm_stream s, float *out);

/* Moving-object boxes (Section 4), half-open pixel rectangles. */
typedef struct {
    int32_t x0, y0, x1, y1;
} rsgm_box;

#define RSGM_MAX_WINDOW_SIZES 8

/*
 * Parameters of the box detection.  Defaults (rsgm_default_detect_params):
 * window sizes 20x20, 30x30, 40x40, 50x50, 50x75 (the paper's range is 20x20
 * to 50x75), stride 10 px, the upper third of the image skipped (1/3),
 * detection when the window's mean |d_pred - d_meas| exceeds 1 px, grouping
 * while any IoU > 0/1 (any overlap), boxes under 1500 px^2 dropped.  The
 * paper gives no numbers beyond the window range and the skipped third;
 * these are readings.
 */
typedef struct {
    int32_t nsizes;                              /* 1 .. RSGM_MAX_WINDOW_SIZES */
    int32_t sizes[RSGM_MAX_WINDOW_SIZES][2];     /* (width, height) >= 1 */
    int32_t stride;                              /* window grid step, >= 1 */
    int32_t skip_num, skip_den;                  /* rows y < H * skip_num / skip_den are not searched */
    float thresh_px;                             /* mean |nu| threshold, >= 0 */
    int32_t iou_num, iou_den;                    /* group while IoU > iou_num / iou_den */
    int32_t min_area;                            /* smaller final boxes are dropped */
} rsgm_detect_params;

int rsgm_default_detect_params(rsgm_detect_params *p);

/*
 * Boxes of the latest frame, for every stream: the |d_pred - d_meas| map
 * (quantised to 1/16 px; 0 where there was no prediction) is summed over
 * sliding windows with an integral image (inclusion-exclusion); windows whose
 * mean exceeds the threshold are grouped greedily (the pair of highest IoU is
 * replaced by its bounding box until no pair exceeds the IoU threshold) and
 * small boxes are dropped.  boxes: host array of B * capacity boxes (stream b
 * at b * capacity); counts: host array of B (the number found, which may
 * exceed capacity: only the first `capacity` are written).  Synchronises.
 */
int rsgm_detect(rsgm_stream s, const rsgm_detect_params *p, rsgm_box *boxes, int32_t capacity, int32_t *counts);

/*
 * The grouping step of the box detection (Section 4) on caller-supplied
 * boxes, on the CPU (no device work).  `in` holds n boxes in window order
 * (host).  While some pair has IoU > iou_num / iou_den, compared exactly on
 * integer areas, the pair of highest IoU is replaced by its bounding box in
 * the place of the first; ties go to the first pair (i, j).  Boxes smaller
 * than min_area are then dropped.
 * out: host, up to `capacity` boxes in order; *count: the number kept (may
 * exceed capacity).  rsgm_detect groups each stream's windows this way.
 * Every coordinate must lie in [-RSGM_BOX_COORD_LIMIT, RSGM_BOX_COORD_LIMIT]
 * (so that areas and the exact IoU comparisons cannot overflow); otherwise
 * RSGM_ERR_INVALID_ARG.
 */
#define RSGM_BOX_COORD_LIMIT 1048576 /* 2^20 */
int rsgm_group_boxes(const rsgm_box *in, int32_t n, int32_t iou_num, int32_t iou_den, int32_t min_area,
                     rsgm_box *out, int32_t capacity, int32_t *count);

/* Stage timing.  While enabled, every frame records CUDA events on the
 * handle's stream around its stages: RSGM_STAGE_PREDICT (splat, hole fill,
 * reset, window), _SCAN (cell offsets), _CENSUS, _COST, _AGGREGATE (all path
 * directions, Eq. 1) and _UPDATE (winner, Kalman, gate).  Up to 4096 frames
 * are kept; further frames are not timed. */
#define RSGM_STAGE_PREDICT 0
#define RSGM_STAGE_SCAN 1
#define RSGM_STAGE_CENSUS 2
#define RSGM_STAGE_COST 3
#define RSGM_STAGE_AGGREGATE 4
#define RSGM_STAGE_UPDATE 5
#define RSGM_NUM_STAGES 6
int rsgm_enable_stage_timing(rsgm_stream s, int enable);

/* Synchronises, writes the milliseconds spent in each stage summed over the
 * frames timed since the last call (ms: RSGM_NUM_STAGES doubles) and the
 * number of frames to *frames, then starts a new accumulation. */
int rsgm_stage_times(rsgm_stream s, double *ms, int32_t *frames);

/*
 * Offsets of a ragged cell volume without allocating device memory.  The
 * paper has no counterpart: this exists for callers that cannot call
 * cudaMalloc (for example a host application that allots all device memory
 * up front, or code running where a device allocation would synchronise the
 * device or be refused).
 *
 * windows: device, rows*width uint32 in the RSGM_BUF_WINDOW format
 * (lo | width << 16, raster order).  offsets: device, rows*width uint32,
 * receives the exclusive prefix sum of the widths in raster order (the
 * RSGM_BUF_OFFSET layout of a handle whose B*H rows are `rows`).  total:
 * device uint32 receiving the sum of all widths, or NULL.  The sum must stay
 * below 2^32.  Work is enqueued on cuda_stream (cudaStream_t, NULL = legacy
 * default stream); nothing is allocated.
 *
 * Scratch: a fixed 512 KiB array of device memory inside the library (row
 * totals and row bases for up to 65536 rows), held on every GPU where the
 * library's device code has been loaded, until the process exits.  rows >
 * 65536 is rejected with RSGM_ERR_INVALID_ARG.  The first call on a device
 * looks up the array's device address (with that device current).  Under
 * CUDA's lazy module loading (the default) that lookup is also what loads the
 * library's device code on that device and places the array, which takes
 * device memory: a caller that reserves all device memory up front must make
 * this first call before reserving it, and before any stream capture.  Every call shares the one array: calls that overlap
 * on the GPU (different streams, no ordering between them) race and give
 * wrong offsets.  Each call writes every scratch entry it reads, so no
 * clearing is needed between calls.
 */
int rsgm_window_offsets_noalloc(const uint32_t *windows, int32_t width, int32_t rows,
                                uint32_t *offsets, uint32_t *total, void *cuda_stream);

/*
 * Schedule autotuner.  The aggregation kernel walks one path line per lane;
 * a lane keeps windows of up to a "register capacity" of cells in registers
 * and leaves wider ones to its whole warp; a warp walks 32 vertical or
 * diagonal lines.  The rows go to a row sweep or to the line sweep (see
 * rsgm_set_rows_per_warp).  rsgm_autotune times the aggregation on the
 * handle's latest frame with each capacity (2, 6, 10, 18 cells) and each way
 * of sweeping the rows, each timed as a frame runs it (behind the cost
 * kernel, which it re-runs on the unchanged census and windows), and keeps
 * the fastest for later frames (the capacity is written to *cells if not
 * NULL; rsgm_get_schedule reads both choices).
 * Results do not depend on the choice; only speed does.  Requires a
 * processed frame; synchronises.
 */
int rsgm_autotune(rsgm_stream s, int32_t *cells);

/* Sets the register capacity by hand: 0 = the radius mode's default
 * (2 radius + 1 for fixed windows), else 1 .. 32 cells, rounded up to the
 * nearest of 2, 6, 10, 18; the rows return to their default sweep (the
 * row sweep, see rsgm_set_rows_per_warp).  Results do not depend on it. */
int rsgm_set_schedule(rsgm_stream s, int32_t cells);

/* How the horizontal directions are swept: 0 (the default) by the row
 * sweep, G lanes sharing each row, on a stream of the handle's own that runs
 * beside the other directions' sweep; 8, 16 or 32 by the line sweep with
 * that many rows per warp.  Results do not depend on it. */
int rsgm_set_rows_per_warp(rsgm_stream s, int32_t rows);

/* The schedule later frames use: *cells = the register capacity (2, 6, 10
 * or 18), *rows = the rows' sweep (0: the row sweep, else rows per warp of
 * the line sweep), as set by rsgm_autotune, rsgm_set_schedule and
 * rsgm_set_rows_per_warp.  Either pointer may be NULL. */
int rsgm_get_schedule(rsgm_stream s, int32_t *cells, int32_t *rows);

/* What the latest rsgm_autotune measured: *count = the candidates it timed
 * (0 before the first call, 16 with horizontal directions, else 4); the
 * first min(n, *count) of them are written as (cells[i], rows[i], ms[i]),
 * ms = its time per aggregation launch.  n = 0 reads the count alone;
 * otherwise the three arrays must hold n entries. */
int rsgm_autotune_times(rsgm_stream s, int32_t *cells, int32_t *rows, float *ms, int32_t n, int32_t *count);

/*
 * A group advances several handles of possibly different geometry by one
 * reduced frame each in a single CUDA graph launch: every member's launches
 * are captured on a stream of its own (forked from and joined back into one),
 * so members run concurrently, and the executable graph is updated in place
 * from tick to tick.  Members must share one device and one CUDA stream (the
 * graph is launched on it) and stay alive while the group exists; the group
 * does not own them.
 */
typedef struct rsgm_group_s *rsgm_group;
int rsgm_group_create(rsgm_group *out, rsgm_stream *members, int32_t n);

/* One reduced frame of every member k: left[k], right[k] are device images
 * (as in rsgm_reduced_frame), R[k], t[k], K[k] host arrays, baseline[k]. */
int rsgm_group_reduced_frame(rsgm_group g, const uint8_t *const *left, const uint8_t *const *right,
                             const float *const *R, const float *const *t, const float *const *K,
                             const float *baseline);

/* Waits for the group's work and frees it (not its members).  NULL is a no-op. */
int rsgm_group_destroy(rsgm_group g);

/*
 * The learned search window.  The paper sizes each pixel's search range from
 * its predicted variance (Section 2.4, d_pred +- p).  This variant lets a
 * per-pixel network choose the half-width from {1, 2, 4, 8, 16} and the
 * measurement variance r of the Kalman correction (Eqs. 5-6).  Its inputs
 * come from the hole-filled prediction before the discontinuity reset:
 * d / D, sqrt(p) / D, census Hamming distance at the rounded predicted
 * disparity / census bits, and Sobel magnitude / 2040.  A pixel without a
 * prediction takes 0, 1 and 1 for the first three.
 *
 * The network has 4 layers of 3x3 correlations with zero padding and ReLU
 * between them: 4 -> 32 -> 32 -> 32 -> 6 channels.  It runs in bfloat16 with
 * fp32 accumulation.  The output gives 5 class logits and log r.  The
 * half-width is the most probable class's radius when its softmax
 * probability is at least 0.9, else 8.  r = exp(log r), clamped to
 * [1/16, 64].  Discontinuity resets and pixels without a prediction keep
 * the full range.
 *
 * Parameters are RSGM_CNN_PARAMS floats, layer by layer: weights in
 * (out, in, ky, kx) order, then the bias.
 */
#define RSGM_CNN_PARAMS 21414
typedef struct rsgm_cnn_s *rsgm_cnn;

/* Creates a network on the current device from host parameters, trained on
 * `cuda_stream` (may be NULL). */
int rsgm_cnn_create(rsgm_cnn *out, const float *params, void *cuda_stream);

/* Copies the current parameters, or the gradient of the latest training
 * step, into host memory (RSGM_CNN_PARAMS floats).  Synchronises. */
int rsgm_cnn_params(rsgm_cnn c, float *params);
int rsgm_cnn_grad(rsgm_cnn c, float *grad);

/* Frees the network.  Detach it first: destroy, or never again run, every
 * handle it is attached to.  NULL is a no-op. */
int rsgm_cnn_destroy(rsgm_cnn c);

/* Attaches the network to a handle created with RSGM_RADIUS_LEARNED on the
 * same device.  Allocates the handle's per-pixel network buffers: 261 bytes
 * per pixel, plus 160 at the first training step.  Its reduced frames then
 * run the network after the prediction.  Frames only read the network, so
 * handles on different CUDA streams may share one network (a request loop
 * serving many streams); a training step changes it, on the network's own
 * stream, so frames of handles on other streams must not overlap a training
 * step.  A learned handle cannot join a group. */
int rsgm_attach_cnn(rsgm_stream s, rsgm_cnn c);

/*
 * One training step on the handle's latest reduced frame, against a target
 * disparity map (device, B*H*W floats).  The handle must use the network's
 * CUDA stream (RSGM_ERR_INVALID_ARG otherwise).  The step reruns the network on the
 * frame's stored inputs with the current parameters, so repeated steps on
 * one frame descend properly.  The target is typically the state
 * of a full-range (RSGM_RADIUS_FULL) handle on the same frames.
 *
 * Trained pixels are those predicted and not reset (class 0).  Label: the
 * smallest radius covering |round(target) - round(d_pred)|, with centres
 * clamped to [0, D - 1], else 16.  Loss: cross-entropy plus
 * 0.1 * 0.5 (e^2 exp(-s) + s), where e = target - d_pred and s = log r,
 * averaged over all pixels.  Update: one Adam step (0.9, 0.999, 1e-8) with
 * learning rate lr; lr = 0 computes the gradient only.
 *
 * *loss (host, may be NULL) receives the loss before the step, which
 * synchronises.  The gradient stays readable by rsgm_cnn_grad.
 */
int rsgm_cnn_train_step(rsgm_cnn c, rsgm_stream s, const float *d_target, float lr, float *loss);

/*
 * Integer throughput of the current device, measured: every SM runs 16
 * independent chains per thread of one integer instruction, timed with CUDA
 * events on cuda_stream (NULL = legacy default stream), best of three
 * launches of several milliseconds each.  *ops_per_s receives scalar
 * operations per second; a packed instruction on two 16-bit lanes counts as
 * two.  The aggregation of Eq. 1 (Section 2.2) is additions and minima on
 * small unsigned losses, so these rates are the ceiling of its integer work:
 *   RSGM_PEAK_I32_ADD    32-bit add
 *   RSGM_PEAK_I32_MIN    32-bit unsigned minimum
 *   RSGM_PEAK_U16X2_MIN  minimum of two packed 16-bit lanes
 *   RSGM_PEAK_U16X2_MIX  alternating packed minimum and 32-bit add (a
 *                        carry-free add of two 16-bit lanes), Eq. 1's mix
 * Allocates nothing; synchronises cuda_stream.  Unknown kind or NULL
 * ops_per_s: RSGM_ERR_INVALID_ARG.
 */
#define RSGM_PEAK_I32_ADD 0
#define RSGM_PEAK_I32_MIN 1
#define RSGM_PEAK_U16X2_MIN 2
#define RSGM_PEAK_U16X2_MIX 3
int rsgm_measure_int_peak(int kind, void *cuda_stream, double *ops_per_s);

/* Waits for the handle's enqueued work; reports deferred device errors. */
int rsgm_sync(rsgm_stream s);

/* Waits for the handle's work and releases every resource.  NULL is a no-op. */
int rsgm_destroy_stream(rsgm_stream s);

/* Static text for a status code. */
const char *rsgm_status_string(int code);

/* Description of the calling thread's most recent failure ("" if none). */
const char *rsgm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RSGM_H_ */
