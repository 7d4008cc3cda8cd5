// Internal declarations shared by the CUDA translation units of librsgm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rsgm.h"

namespace rsgm {

// Geometry of one handle: B streams of H x W pixels, D disparities.
struct Geometry {
    int B, W, H, D;
    long long HW;    // pixels per stream
    long long NPIX;  // B * HW
};

// Cell layout.  Each pixel's window of w cells starts on a multiple of 4
// cells and occupies round4(w) cells (the ragged volume is a raster-order
// prefix sum of the rounded widths), so that every 4 cells of a window are
// one aligned 32-bit word of an 8-bit volume.  Cells [w, round4(w)) are
// padding: the cost volume holds 0xFF there, the other volumes anything.
__host__ __device__ inline int round4(int w) { return (w + 3) & ~3; }
// Worst-case cells of a frame (every pixel searching the whole range).
inline long long max_cells(const Geometry &g) { return g.NPIX * (long long)round4(g.D); }
// Elements between consecutive direction planes: the worst-case cell count,
// rounded up so that every plane starts 16-element aligned.
inline long long plane_stride(const Geometry &g) { return (max_cells(g) + 15) / 16 * 16; }

// Ego-motion of one stream: X_k = R X_{k-1} + t.
struct Motion {
    float R[9];
    float t[3];
};

// Role of each stream ("slot") of a handle in a frame: RSGM_SLOT_IDLE,
// RSGM_SLOT_REDUCED or RSGM_SLOT_FULL (include/rsgm.h).
typedef uint8_t SlotRoles[RSGM_MAX_BATCH];

// Kernel argument block of the forward splat (passed by value; copied at launch).
struct SplatArgs {
    Geometry g;
    float fx, fy, cx, cy, fb, q;
    Motion m[RSGM_MAX_BATCH];
    SlotRoles role;  // only RSGM_SLOT_REDUCED streams are predicted
};

// Launch plan of the line sweep: the directions it runs in launch order,
// the first warp of each (a warp walks up to 32 path lines of one stream:
// rows spread across the image, or 8 groups of 4 adjacent vertical or
// diagonal lines), the plane each writes, and the per-lane band of shared
// memory.
constexpr int kLineWarps = 4;  // warps per block of the aggregation kernel
struct LinePlan {
    Geometry g;
    int P1, P2;
    int pad;         // +inf slots kept on both sides of a band's window
    int band_words;  // 32-bit words of shared memory per lane
    int hlines;      // rows a warp walks for the horizontal directions (8, 16 or 32)
    int ndir;
    int dir[8];
    int plane_of[8];
    long long warp_begin[9];
    long long plane_stride;  // elements between consecutive planes
};

// Sliding-window plan of the moving-object boxes (Section 4): windows of size
// s are numbered first[s] + row * nx[s] + column.
struct DetectPlan {
    int nsizes;
    int size[RSGM_MAX_WINDOW_SIZES][2];
    int nx[RSGM_MAX_WINDOW_SIZES], ny[RSGM_MAX_WINDOW_SIZES];
    int first[RSGM_MAX_WINDOW_SIZES + 1];
    int total;
    int stride, y_min;
    unsigned thresh_q;  // mean |nu| threshold in 1/16 px
};

// Per-frame parameters of the resolve / update kernels.
struct FrameParams {
    int radius_mode, radius;
    int P1, P2, nbits;
    float q, r_meas, p_reset, tau_disc, gamma;
    SlotRoles role;
};

// Device buffers owned by a handle (all sized at the worst case at init).
struct Buffers {
    uint8_t *img_l, *img_r;             // staging for host inputs, NPIX each
    unsigned long long *cen_l, *cen_r;  // census codes, NPIX each
    float *d, *p;                       // state, NPIX each
    unsigned long long *key;            // splat z-buffer, NPIX, zero between frames
    float *d_pred, *p_pred;             // prediction after hole fill / reset, NPIX each
    uint32_t *win;                      // lo | width << 16, NPIX
    uint8_t *cls;                       // 0 predicted, 1 reset, 2 no prediction, 3 idle slot
    uint32_t *inrow;                    // exclusive offset within the pixel's row, NPIX
    uint2 *meta;                        // (first cell, window) of the pixel, NPIX
    uint32_t *row_total, *row_base;     // B*H each: rounded cells of the row, first cell of the row
    uint32_t *row_cells;                // B*H: cells of the row (sum of the true widths)
    uint8_t *cost;                      // ragged cost volume, max_cells + 128
    void *planes;                       // one plane of L_r per enabled direction, plane_stride each
    uint16_t *S;                        // ragged aggregated cost, max_cells
    int16_t *d_int;
    uint8_t *mask;
    float *d_z, *nu;
    unsigned long long *counters;       // [0] frames, [1] cells, [2] cells of the last frame,
                                        // [3] rounded cells of the last frame
    float *median;                      // 3x3 median of d, NPIX
    unsigned long long *sat;            // integral image of |nu|, B * (H+1) * (W+1)
    uint8_t *flags;                     // detection flag per window, B * RSGM_MAX_WINDOW_SIZES * H * W
    const uint8_t *radius;              // learned window half-width per pixel (RSGM_RADIUS_LEARNED), else NULL
};

// ---- the learned window (RSGM_RADIUS_LEARNED) ----

constexpr int kCnnLayers = 4;
constexpr int kCnnClasses = 5;   // radius classes 1, 2, 4, 8, 16
constexpr int kCnnOutPad = 8;    // output channels per pixel: 5 logits, log r, 2 unused
constexpr int kCnnParams = RSGM_CNN_PARAMS;
extern const int kCnnIn[kCnnLayers];   // 4, 32, 32, 32
extern const int kCnnOut[kCnnLayers];  // 32, 32, 32, 6

// Parameters on the device: fp32 master copy (layer by layer, weights
// (out, in, 3, 3) then bias), Adam moments and the gradient; per layer the
// bfloat16 forward weights [9][out padded][in padded], the bfloat16
// input-gradient weights [9][in][gradient channels] (layers 1-3) and the
// bias padded to the output channels.
struct CnnWeights {
    float *theta, *m, *v, *grad;
    void *wf[kCnnLayers], *wb[kCnnLayers];
    float *bias[kCnnLayers];
};

// Per-pixel buffers of a handle running the learned window (bfloat16
// activations, channels innermost): inputs (16 channels), three hidden
// layers (32), the output (fp32, kCnnOutPad), the decided half-width and
// measurement variance; the training gradients (allocated at the first
// training step) and the loss accumulator.
struct LearnedBuffers {
    void *feats;
    void *act[3];
    float *out;
    uint8_t *radius;
    float *r_map;
    void *g16, *ga, *gb;
    float *loss;
};

// Records msg as the calling thread's last error (rsgm_last_error) and returns code.
int record_error(int code, const char *msg);

long long cnn_param_offset(int layer);
cudaError_t cnn_pack(const CnnWeights &w, cudaStream_t st);
// Inputs, the four layers and the decision of the latest prediction.
cudaError_t cnn_forward(const CnnWeights &w, const LearnedBuffers &lb, const Buffers &b, const Geometry &g,
                        const uint8_t *left, int nbits, cudaStream_t st);
// The four layers again from the stored inputs, the loss against d_target
// and the gradient of every parameter (into w.grad).
cudaError_t cnn_backward(const CnnWeights &w, const LearnedBuffers &lb, const Buffers &b, const Geometry &g,
                         const float *d_target, int sm_count, cudaStream_t st);
// One Adam step (step counted from 1) and the repacked device weights.
cudaError_t cnn_adam(const CnnWeights &w, int step, float lr, cudaStream_t st);

// ---- launchers (each returns the cudaError_t of its launch) ----

// Prediction (Section 2.4): forward splat, hole fill, discontinuity reset,
// window and in-row prefix sum; the row-total scan; the full-range window.
cudaError_t launch_splat(const Buffers &b, const SplatArgs &a, cudaStream_t st);
cudaError_t launch_gather_fill(const Buffers &b, const Geometry &g, float q, cudaStream_t st);
cudaError_t launch_window(const Buffers &b, const Geometry &g, const FrameParams &fp, cudaStream_t st);
cudaError_t launch_full_window(const Buffers &b, const Geometry &g, cudaStream_t st);
// nstreams: the streams that advance this frame (counted as frames).
cudaError_t launch_row_scan(const Buffers &b, const Geometry &g, int nstreams, cudaStream_t st);

// Matching (Section 2.1).
cudaError_t launch_census(const Buffers &b, const Geometry &g, const uint8_t *left,
                          const uint8_t *right, int cw, int ch, cudaStream_t st);
cudaError_t launch_cost(const Buffers &b, const Geometry &g, int nbits, cudaStream_t st);

// Aggregation, Eq. 1 (Section 2.2), the line sweep: the directions of
// run_mask in one launch, one lane per path line, planes of `plane_bytes`
// (1 or 2) per cell.  Windows of up to `capacity`
// cells (rounded up by sweep_capacity to 2, 6, 10 or 18) are walked in a
// lane's registers, wider ones by the whole warp.
// path_mask numbers the planes (one per enabled direction, in bit order);
// run_mask selects the directions this launch sweeps.  hlines: rows a warp
// walks for the horizontal directions (8, 16 or 32; 0 = 16).
int sweep_capacity(int cells);
cudaError_t launch_paths(const Buffers &b, const Geometry &g, unsigned path_mask, unsigned run_mask, int P1, int P2,
                         int nbits, int plane_bytes, int capacity, int hlines, cudaStream_t st);
// The two horizontal directions (run_mask bits 0 and 1) with G lanes per row
// (lanes_per_line of the common window width).
int lanes_per_line(int window);
cudaError_t launch_rows(const Buffers &b, const Geometry &g, unsigned path_mask, unsigned run_mask, int P1, int P2,
                        int lanes, int plane_bytes, int sm_count, cudaStream_t st);

// Sum of the planes, winner-takes-all, Kalman correction and gate
// (Sections 2.2-2.4).
cudaError_t launch_update(const Buffers &b, const Geometry &g, const FrameParams &fp, const float *r_map, int nplanes,
                          int plane_bytes, cudaStream_t st);

// Integer-throughput microbenchmark (the ALU roofline's denominator).
cudaError_t launch_peak(int kind, int blocks, int iters, cudaStream_t st);
double peak_ops(int kind, int blocks, int iters);
int peak_blocks_per_sm();

// After the path (Section 2.3 median output, Section 4 boxes).
cudaError_t launch_median3(const float *d, float *out, const Geometry &g, cudaStream_t st);
cudaError_t launch_detect_windows(const Buffers &b, const Geometry &g, const DetectPlan &dp, cudaStream_t st);
int group_boxes(const uint8_t *flags, const DetectPlan &dp, int iou_num, int iou_den, long long min_area,
                int32_t *out, int capacity);

}  // namespace rsgm
