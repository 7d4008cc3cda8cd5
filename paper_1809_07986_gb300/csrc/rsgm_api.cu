// C ABI of librsgm: handle life cycle, argument checks, buffer ownership and
// the per-frame launch sequence (declared and documented in include/rsgm.h).
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <math.h>

#include <algorithm>
#include <new>
#include <thread>
#include <vector>

#include "rsgm_internal.cuh"

using namespace rsgm;

constexpr int kMaxTimedFrames = 4096;

// CUDA events around the stages of each timed frame.
struct StageTimer {
    bool on = false;
    int n = 0;  // frames recorded since the last read
    cudaEvent_t *ev = nullptr;  // kMaxTimedFrames * (RSGM_NUM_STAGES + 1)
};

struct rsgm_stream_s {
    rsgm_params P;
    StageTimer timer;
    cudaStream_t st;
    int device;
    Geometry g;
    int nbits;
    int nplanes;      // enabled path directions
    int capacity;     // window cells a path-sweep lane keeps in registers (default for the radius mode)
    int lanes;        // lanes per row of the row sweep (the common window width)
    cudaStream_t side;            // the row sweep runs here, beside the other directions' sweep
    cudaEvent_t fork_ev, join_ev;
    int sm_count;     // multiprocessors of the handle's device
    int tuned_cap;    // register capacity picked by rsgm_autotune / rsgm_set_schedule (0: default)
    int tuned_hl;     // horizontal directions: 0 = the row sweep, 8/16/32 = rows per warp of the line sweep
    int ntimed;                        // candidates the latest rsgm_autotune timed
    int timed_cap[16], timed_hl[16];   // their schedules
    float timed_ms[16];                // and their times, ms per launch
    bool capturing;   // enqueueing into a group's graph: no stage-timing events
    int plane_bytes;  // 1 if every L_r fits in 8 bits (nbits + P2 <= 255), else 2
    float p_reset;
    bool has_state;                    // some stream of the handle has a state
    uint8_t slot_state[RSGM_MAX_BATCH];  // per stream: 1 once it has a state
    Buffers buf;
    rsgm_cnn cnn;         // attached network (RSGM_RADIUS_LEARNED), not owned
    LearnedBuffers lb;    // its per-pixel buffers, owned
    bool learned_frame;   // the latest frame ran the network
};

struct rsgm_cnn_s {
    int device;
    cudaStream_t st;
    CnnWeights w;
    int step;  // Adam steps taken
};

namespace {

thread_local char g_last_error[512] = "";

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(RSGM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define RSGM_CUDA(call)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// Makes the handle's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool is_device_pointer(const void *ptr)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free error of an unknown pointer
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int check_params(const rsgm_params *p)
{
    if (!p) return fail(RSGM_ERR_INVALID_ARG, "params is NULL");
    if (p->width < 1 || p->height < 1 || p->width > 65535 || p->height > 65535)
        return fail(RSGM_ERR_INVALID_ARG, "width/height must be in [1, 65535]");
    if (p->max_disp < 1 || p->max_disp > RSGM_MAX_DISP)
        return fail(RSGM_ERR_INVALID_ARG, "max_disp must be in [1, %d]", RSGM_MAX_DISP);
    if (p->batch < 1 || p->batch > RSGM_MAX_BATCH)
        return fail(RSGM_ERR_INVALID_ARG, "batch must be in [1, %d]", RSGM_MAX_BATCH);
    if (p->census_w < 1 || p->census_h < 1 || !(p->census_w & 1) || !(p->census_h & 1) ||
        p->census_w > 15 || p->census_h > 15 || p->census_w * p->census_h - 1 > 64)
        return fail(RSGM_ERR_INVALID_ARG, "census window must be odd, <= 15 and have <= 64 bits");
    if (p->path_mask == 0 || p->path_mask > 0xFFu)
        return fail(RSGM_ERR_INVALID_ARG, "path_mask must enable 1..8 of the 8 directions");
    if (p->radius_mode < RSGM_RADIUS_FIXED || p->radius_mode > RSGM_RADIUS_LEARNED)
        return fail(RSGM_ERR_INVALID_ARG, "unknown radius_mode %d", p->radius_mode);
    if (p->radius < 0) return fail(RSGM_ERR_INVALID_ARG, "radius must be >= 0");
    if (p->P1 < 0 || p->P2 < 0 || p->P1 > 4000 || p->P2 > 4000)
        return fail(RSGM_ERR_INVALID_ARG, "P1, P2 must be in [0, 4000]");
    if (!(p->q >= 0.0f) || !(p->r_meas > 0.0f) || !(p->tau_disc >= 0.0f) || !(p->gate_gamma > 0.0f) ||
        p->p_reset != p->p_reset)
        return fail(RSGM_ERR_INVALID_ARG, "noise / threshold parameters out of range");
    unsigned long long cells = (unsigned long long)p->batch * p->width * p->height * round4(p->max_disp);
    if (cells >= 0xFFFFFFFFull)
        return fail(RSGM_ERR_INVALID_ARG, "batch*width*height*round4(max_disp) must be < 2^32");
    return RSGM_OK;
}

template <typename T>
int alloc(T **ptr, size_t count, void **all, int &nall)
{
    void *p = nullptr;
    if (cudaMalloc(&p, count * sizeof(T) ? count * sizeof(T) : 1) != cudaSuccess) {
        cudaGetLastError();
        return fail(RSGM_ERR_OOM, "cudaMalloc of %zu bytes failed", count * sizeof(T));
    }
    all[nall++] = p;
    *ptr = (T *)p;
    return RSGM_OK;
}

void free_buffers(Buffers &b)
{
    void *ptrs[] = {b.img_l, b.img_r, b.cen_l, b.cen_r, b.d,    b.p,    b.key,       b.d_pred,
                    b.p_pred, b.win, b.cls,   b.inrow, b.meta, b.row_total, b.row_base, b.row_cells, b.cost,
                    b.planes, b.S,   b.d_int, b.mask,  b.d_z,  b.nu,   b.counters, b.median,
                    b.sat,    b.flags};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    memset(&b, 0, sizeof(b));
}

void free_learned(LearnedBuffers &lb)
{
    void *ptrs[] = {lb.feats, lb.act[0], lb.act[1], lb.act[2], lb.out, lb.radius, lb.r_map, lb.g16, lb.ga, lb.gb,
                    lb.loss};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    memset(&lb, 0, sizeof(lb));
}

void free_cnn(rsgm_cnn c)
{
    void *ptrs[] = {c->w.theta, c->w.m, c->w.v, c->w.grad};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (int l = 0; l < kCnnLayers; ++l) {
        if (c->w.wf[l]) cudaFree(c->w.wf[l]);
        if (c->w.wb[l]) cudaFree(c->w.wb[l]);
        if (c->w.bias[l]) cudaFree(c->w.bias[l]);
    }
}

// The row sweep's side stream and its fork / join events.
void release_side(rsgm_stream_s *s)
{
    if (s->fork_ev) cudaEventDestroy(s->fork_ev);
    if (s->join_ev) cudaEventDestroy(s->join_ev);
    if (s->side) cudaStreamDestroy(s->side);
    s->fork_ev = s->join_ev = nullptr;
    s->side = nullptr;
}

FrameParams frame_params(const rsgm_stream_s *s, const uint8_t *roles = nullptr, uint8_t all = RSGM_SLOT_REDUCED)
{
    FrameParams fp;
    for (int b = 0; b < RSGM_MAX_BATCH; ++b) fp.role[b] = b < s->g.B ? (roles ? roles[b] : all) : RSGM_SLOT_IDLE;
    fp.radius_mode = s->P.radius_mode;
    fp.radius = s->P.radius;
    fp.P1 = s->P.P1;
    fp.P2 = s->P.P2;
    fp.nbits = s->nbits;
    fp.q = s->P.q;
    fp.r_meas = s->P.r_meas;
    fp.p_reset = s->p_reset;
    fp.tau_disc = s->P.tau_disc;
    fp.gamma = s->P.gate_gamma;
    return fp;
}

// Copies a host image batch into the staging buffer; device pointers pass through.
int stage_images(rsgm_stream s, const uint8_t *left, const uint8_t *right, const uint8_t **dl,
                 const uint8_t **dr)
{
    size_t bytes = (size_t)s->g.NPIX;
    *dl = left;
    *dr = right;
    if (s->capturing) return RSGM_OK;  // group frames take device images (checked before the capture)
    if (!is_device_pointer(left)) {
        RSGM_CUDA(cudaMemcpyAsync(s->buf.img_l, left, bytes, cudaMemcpyHostToDevice, s->st));
        *dl = s->buf.img_l;
    }
    if (!is_device_pointer(right)) {
        RSGM_CUDA(cudaMemcpyAsync(s->buf.img_r, right, bytes, cudaMemcpyHostToDevice, s->st));
        *dr = s->buf.img_r;
    }
    return RSGM_OK;
}

// Records stage boundary `k` (0 = frame start) of the current timed frame.
int mark(rsgm_stream s, int k)
{
    StageTimer &t = s->timer;
    if (!t.on || t.n >= kMaxTimedFrames || s->capturing) return RSGM_OK;
    RSGM_CUDA(cudaEventRecord(t.ev[t.n * (RSGM_NUM_STAGES + 1) + k], s->st));
    if (k == RSGM_NUM_STAGES) t.n++;
    return RSGM_OK;
}

#define RSGM_MARK(s, k)              \
    do {                             \
        int rc_ = mark((s), (k));    \
        if (rc_) return rc_;         \
    } while (0)

// Census, cost, aggregation and the update: the part shared by both frame
// kinds.  A learned frame has run the census already (the network reads it)
// and corrects with its per-pixel measurement variance r_map.
// Eq. 1 over every enabled direction.  By default the horizontal directions
// run in the row sweep on the handle's side stream, forked from and joined
// back into `st`, while the line sweep does the others; with rows = 8, 16 or
// 32 the line sweep does all of them.
cudaError_t launch_aggregation(rsgm_stream s, int capacity, int rows, cudaStream_t st)
{
    const unsigned mask = s->P.path_mask, hmask = mask & 3u;
    const Geometry &g = s->g;
    if (rows != 0 || hmask == 0)
        return launch_paths(s->buf, g, mask, mask, s->P.P1, s->P.P2, s->nbits, s->plane_bytes, capacity, rows, st);
    if ((mask & ~3u) == 0)
        return launch_rows(s->buf, g, mask, hmask, s->P.P1, s->P.P2, s->lanes, s->plane_bytes, s->sm_count, st);
    cudaError_t e = cudaEventRecord(s->fork_ev, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->side, s->fork_ev, 0);
    if (e == cudaSuccess)
        e = launch_rows(s->buf, g, mask, hmask, s->P.P1, s->P.P2, s->lanes, s->plane_bytes, s->sm_count, s->side);
    const cudaError_t e2 = launch_paths(s->buf, g, mask, mask & ~3u, s->P.P1, s->P.P2, s->nbits, s->plane_bytes,
                                        capacity, 16, st);
    // join even after a failed launch, so that the side stream never runs ahead
    const cudaError_t e3 = cudaEventRecord(s->join_ev, s->side);
    const cudaError_t e4 = e3 == cudaSuccess ? cudaStreamWaitEvent(st, s->join_ev, 0) : e3;
    return e != cudaSuccess ? e : (e2 != cudaSuccess ? e2 : e4);
}

int match_and_update(rsgm_stream s, const uint8_t *dl, const uint8_t *dr, bool census_done, const float *r_map,
                     const FrameParams &fp)
{
    const Geometry &g = s->g;
    int active = 0;
    for (int b = 0; b < g.B; ++b) active += fp.role[b] != RSGM_SLOT_IDLE;
    RSGM_MARK(s, 1);
    RSGM_CUDA(launch_row_scan(s->buf, g, active, s->st));
    RSGM_MARK(s, 2);
    if (!census_done) RSGM_CUDA(launch_census(s->buf, g, dl, dr, s->P.census_w, s->P.census_h, s->st));
    RSGM_MARK(s, 3);
    RSGM_CUDA(launch_cost(s->buf, g, s->nbits, s->st));
    RSGM_MARK(s, 4);
    RSGM_CUDA(launch_aggregation(s, s->tuned_cap ? s->tuned_cap : s->capacity, s->tuned_hl, s->st));
    RSGM_MARK(s, 5);
    RSGM_CUDA(launch_update(s->buf, g, fp, r_map, s->nplanes, s->plane_bytes, s->st));
    RSGM_MARK(s, 6);
    return RSGM_OK;
}

int check_reduced_args(rsgm_stream s, const uint8_t *left, const uint8_t *right, const float *R, const float *t,
                       const float *K, float baseline)
{
    if (!s || !left || !right || !R || !t || !K)
        return fail(RSGM_ERR_INVALID_ARG, "NULL handle, image or motion array");
    if (!(baseline > 0.0f) || !(K[0] > 0.0f) || !(K[4] > 0.0f) || K[1] != 0.0f || K[3] != 0.0f ||
        K[6] != 0.0f || K[7] != 0.0f || K[8] != 1.0f)
        return fail(RSGM_ERR_INVALID_ARG, "K must be [fx 0 cx; 0 fy cy; 0 0 1] with fx, fy > 0; baseline > 0");
    for (int b = 0; b < s->g.B; ++b)
        if (!s->slot_state[b]) return fail(RSGM_ERR_NO_STATE, "reduced frame of stream %d before its first frame", b);
    if (s->P.radius_mode == RSGM_RADIUS_LEARNED && !s->cnn)
        return fail(RSGM_ERR_INVALID_ARG, "RSGM_RADIUS_LEARNED handle without an attached network");
    return RSGM_OK;
}

// Enqueues one reduced frame of all the handle's streams on s->st (arguments
// already checked, the handle's device current).
int enqueue_reduced(rsgm_stream s, const uint8_t *left, const uint8_t *right, const float *R, const float *t,
                    const float *K, float baseline, const uint8_t *roles = nullptr)
{
    const uint8_t *dl, *dr;
    int rc = stage_images(s, left, right, &dl, &dr);
    if (rc) return rc;
    // The argument block is large but copied at launch: no host buffer outlives the call.
    SplatArgs *a = (SplatArgs *)malloc(sizeof(SplatArgs));
    if (!a) return fail(RSGM_ERR_OOM, "host allocation failed");
    a->g = s->g;
    a->fx = K[0];
    a->cx = K[2];
    a->fy = K[4];
    a->cy = K[5];
    a->fb = K[0] * baseline;
    a->q = s->P.q;
    for (int b = 0; b < s->g.B; ++b) {
        memcpy(a->m[b].R, R + 9 * b, 9 * sizeof(float));
        memcpy(a->m[b].t, t + 3 * b, 3 * sizeof(float));
        a->role[b] = roles ? roles[b] : (uint8_t)RSGM_SLOT_REDUCED;
    }
    rc = mark(s, 0);
    if (rc) {
        free(a);
        return rc;
    }
    cudaError_t e = launch_splat(s->buf, *a, s->st);
    free(a);
    if (e != cudaSuccess) return cuda_fail(e, "splat launch");
    RSGM_CUDA(launch_gather_fill(s->buf, s->g, s->P.q, s->st));
    const bool learned = s->P.radius_mode == RSGM_RADIUS_LEARNED;
    if (learned) {
        // the network reads the census residual at the predicted disparity
        RSGM_CUDA(launch_census(s->buf, s->g, dl, dr, s->P.census_w, s->P.census_h, s->st));
        RSGM_CUDA(cnn_forward(s->cnn->w, s->lb, s->buf, s->g, dl, s->nbits, s->st));
    }
    FrameParams fp = frame_params(s, roles);
    RSGM_CUDA(launch_window(s->buf, s->g, fp, s->st));
    rc = match_and_update(s, dl, dr, learned, learned ? s->lb.r_map : nullptr, fp);
    if (rc) return rc;
    s->learned_frame = learned;
    return RSGM_OK;
}

void destroy_timer(StageTimer &t)
{
    if (t.ev) {
        for (int i = 0; i < kMaxTimedFrames * (RSGM_NUM_STAGES + 1); ++i)
            if (t.ev[i]) cudaEventDestroy(t.ev[i]);
        free(t.ev);
    }
    t.ev = nullptr;
    t.on = false;
    t.n = 0;
}


// The ragged volumes in their documented layout: each pixel's cells follow
// the previous pixel's, with no padding (the device keeps 4-aligned runs).
// Offsets are the prefix sum of the widths; costs and S are gathered run by
// run on the host.  Synchronises.
int read_ragged(rsgm_stream s, int which, void *dst, size_t capacity, size_t *bytes)
{
    const size_t n = (size_t)s->g.NPIX;
    unsigned long long cnt[4];
    RSGM_CUDA(cudaMemcpyAsync(cnt, s->buf.counters, sizeof(cnt), cudaMemcpyDeviceToHost, s->st));
    RSGM_CUDA(cudaStreamSynchronize(s->st));
    const size_t cells = (size_t)cnt[2], padded = (size_t)cnt[3];
    const size_t elem = which == RSGM_BUF_AGGREGATED ? 2 : (which == RSGM_BUF_COST ? 1 : 4);
    const size_t size = which == RSGM_BUF_OFFSET ? n * 4 : cells * elem;
    if (bytes) *bytes = size;
    if (!dst) return RSGM_OK;
    if (capacity < size) return fail(RSGM_ERR_INVALID_ARG, "capacity %zu < %zu bytes", capacity, size);
    uint2 *meta = (uint2 *)malloc(n * sizeof(uint2));
    uint8_t *vol = which == RSGM_BUF_OFFSET ? nullptr : (uint8_t *)malloc(padded * elem + 1);
    uint8_t *out = (uint8_t *)malloc(size + 1);
    int rc = RSGM_OK;
    if (!meta || !out || (which != RSGM_BUF_OFFSET && !vol)) {
        rc = fail(RSGM_ERR_OOM, "host allocation failed");
    } else {
        cudaError_t e = cudaMemcpyAsync(meta, s->buf.meta, n * sizeof(uint2), cudaMemcpyDeviceToHost, s->st);
        if (e == cudaSuccess && vol && padded)
            e = cudaMemcpyAsync(vol, which == RSGM_BUF_COST ? (const void *)s->buf.cost : (const void *)s->buf.S,
                                padded * elem, cudaMemcpyDeviceToHost, s->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
        if (e != cudaSuccess) rc = cuda_fail(e, "reading a ragged volume");
    }
    if (rc == RSGM_OK) {
        size_t at = 0;
        for (size_t i = 0; i < n; ++i) {
            const size_t w = meta[i].y >> 16;
            if (which == RSGM_BUF_OFFSET) {
                ((uint32_t *)out)[i] = (uint32_t)at;
            } else if (at + w <= cells && meta[i].x + w <= padded) {
                memcpy(out + at * elem, vol + (size_t)meta[i].x * elem, w * elem);
            }
            at += w;
        }
        cudaError_t e = cudaMemcpyAsync(dst, out, size, cudaMemcpyDefault, s->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
        if (e != cudaSuccess) rc = cuda_fail(e, "copying a ragged volume out");
    }
    free(meta);
    free(vol);
    free(out);
    return rc;
}
}  // namespace

namespace rsgm {
// Records `msg` as the calling thread's last error and returns `code`.
int record_error(int code, const char *msg) { return fail(code, "%s", msg); }
}  // namespace rsgm

extern "C" {

int rsgm_default_params(rsgm_params *p, int32_t width, int32_t height)
{
    if (!p) return fail(RSGM_ERR_INVALID_ARG, "params is NULL");
    memset(p, 0, sizeof(*p));
    p->width = width;
    p->height = height;
    p->max_disp = 128;
    p->batch = 1;
    p->census_w = 5;
    p->census_h = 5;
    p->path_mask = 0xFFu;
    p->radius_mode = RSGM_RADIUS_FIXED;
    p->radius = 4;
    p->P1 = 6;
    p->P2 = 65;
    p->q = 0.15f;
    p->r_meas = 1.0f;
    p->p_reset = 0.0f;  // -> D^2 / 12
    p->tau_disc = 2.0f;
    p->gate_gamma = 6.635f;
    return RSGM_OK;
}

int rsgm_footprint(const rsgm_params *p, uint64_t *bytes)
{
    if (!bytes) return fail(RSGM_ERR_INVALID_ARG, "bytes is NULL");
    int rc = check_params(p);
    if (rc) return rc;
    const uint64_t n = (uint64_t)p->batch * p->width * p->height;
    const uint64_t cells = n * (uint64_t)round4(p->max_disp);
    const int nbits = p->census_w * p->census_h - 1;
    const uint64_t plane_bytes = nbits + p->P2 <= 255 ? 1 : 2;
    const uint64_t stride = (cells + 15) / 16 * 16;
    const uint64_t per_pixel = 2 + 16 + 8 + 8 + 8 + 4 + 1 + 4 + 8 + 2 + 1 + 4 + 4 + 4 + RSGM_MAX_WINDOW_SIZES;
    *bytes = n * per_pixel + cells * (1 + 2) + 128 + 32 + (stride * __builtin_popcount(p->path_mask) + 16) * plane_bytes +
             (uint64_t)p->batch * p->height * 12 + (uint64_t)p->batch * (p->height + 1) * (p->width + 1) * 8 + 32 +
             (p->radius_mode == RSGM_RADIUS_LEARNED ? n * 261 : 0);
    return RSGM_OK;
}

int rsgm_init_stream(rsgm_stream *out, const rsgm_params *p, void *cuda_stream)
{
    if (!out) return fail(RSGM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int rc = check_params(p);
    if (rc) return rc;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    rsgm_stream s = new (std::nothrow) rsgm_stream_s();
    if (!s) return fail(RSGM_ERR_OOM, "host allocation failed");
    s->P = *p;
    s->st = (cudaStream_t)cuda_stream;
    s->device = dev;
    if (cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        s->sm_count = 0;
    }
    s->g.B = p->batch;
    s->g.W = p->width;
    s->g.H = p->height;
    s->g.D = p->max_disp;
    s->g.HW = (long long)p->width * p->height;
    s->g.NPIX = s->g.HW * p->batch;
    s->nbits = p->census_w * p->census_h - 1;
    s->nplanes = __builtin_popcount(p->path_mask);
    s->plane_bytes = s->nbits + p->P2 <= 255 ? 1 : 2;
    // Register capacity of a path-sweep lane: the common (predicted) window.
    // Learned windows: the fallback half-width 8; the paper's variance rule:
    // half-widths up to 4; full range: registers only if the whole range fits.
    s->capacity = p->radius_mode == RSGM_RADIUS_FIXED     ? 2 * p->radius + 1
                  : p->radius_mode == RSGM_RADIUS_LEARNED ? 17
                  : p->radius_mode == RSGM_RADIUS_VARIANCE ? 9
                  : (p->max_disp <= 18 ? p->max_disp : 2);
    s->lanes = lanes_per_line(p->radius_mode == RSGM_RADIUS_FIXED     ? 2 * p->radius + 1
                              : p->radius_mode == RSGM_RADIUS_LEARNED ? 17
                                                                      : p->max_disp);
    s->p_reset = p->p_reset > 0.0f ? p->p_reset : (float)p->max_disp * (float)p->max_disp / 12.0f;
    if ((e = cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking)) != cudaSuccess) {
        delete s;
        return cuda_fail(e, "cudaStreamCreateWithFlags");
    }
    if ((e = cudaEventCreateWithFlags(&s->fork_ev, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&s->join_ev, cudaEventDisableTiming)) != cudaSuccess) {
        if (s->fork_ev) cudaEventDestroy(s->fork_ev);
        cudaStreamDestroy(s->side);
        delete s;
        return cuda_fail(e, "cudaEventCreateWithFlags");
    }
    s->has_state = false;
    memset(s->slot_state, 0, sizeof(s->slot_state));
    memset(&s->buf, 0, sizeof(s->buf));
    Buffers &b = s->buf;
    const size_t n = (size_t)s->g.NPIX, rows = (size_t)p->batch * p->height;
    const size_t cells = (size_t)max_cells(s->g);
    void *all[40];
    int nall = 0;
    if ((rc = alloc(&b.img_l, n, all, nall)) || (rc = alloc(&b.img_r, n, all, nall)) ||
        (rc = alloc(&b.cen_l, n, all, nall)) || (rc = alloc(&b.cen_r, n, all, nall)) ||
        (rc = alloc(&b.d, n, all, nall)) || (rc = alloc(&b.p, n, all, nall)) ||
        (rc = alloc(&b.key, n, all, nall)) || (rc = alloc(&b.d_pred, n, all, nall)) ||
        (rc = alloc(&b.p_pred, n, all, nall)) || (rc = alloc(&b.win, n, all, nall)) ||
        (rc = alloc(&b.cls, n, all, nall)) || (rc = alloc(&b.inrow, n, all, nall)) ||
        (rc = alloc(&b.meta, n, all, nall)) || (rc = alloc(&b.row_total, rows, all, nall)) ||
        (rc = alloc(&b.row_base, rows, all, nall)) || (rc = alloc(&b.row_cells, rows, all, nall)) ||
        (rc = alloc(&b.cost, cells + 128, all, nall)) ||  // + the path sweep's prefetch past the last window (< 128 B)
        // + 16 cells: the update kernel reads and writes whole 16-cell chunks
        (rc = alloc((uint8_t **)&b.planes, ((size_t)plane_stride(s->g) * s->nplanes + 16) * s->plane_bytes, all, nall)) ||
        (rc = alloc(&b.S, cells + 16, all, nall)) || (rc = alloc(&b.d_int, n, all, nall)) ||
        (rc = alloc(&b.mask, n, all, nall)) || (rc = alloc(&b.d_z, n, all, nall)) ||
        (rc = alloc(&b.nu, n, all, nall)) || (rc = alloc(&b.counters, 4, all, nall)) ||
        (rc = alloc(&b.median, n, all, nall)) ||
        (rc = alloc(&b.sat, (size_t)p->batch * (p->height + 1) * (p->width + 1), all, nall)) ||
        (rc = alloc(&b.flags, n * RSGM_MAX_WINDOW_SIZES, all, nall))) {
        free_buffers(b);
        release_side(s);
        delete s;
        return rc;
    }
    // Zero what later frames rely on: the splat keys and the counters; the
    // remaining buffers are written before they are read.
    if ((e = cudaMemsetAsync(b.key, 0, n * sizeof(unsigned long long), s->st)) != cudaSuccess ||
        (e = cudaMemsetAsync(b.counters, 0, 4 * sizeof(unsigned long long), s->st)) != cudaSuccess ||
        (e = cudaMemsetAsync(b.mask, 0, n, s->st)) != cudaSuccess) {
        free_buffers(b);
        release_side(s);
        delete s;
        return cuda_fail(e, "cudaMemsetAsync");
    }
    *out = s;
    return RSGM_OK;
}

int rsgm_full_frame(rsgm_stream s, const uint8_t *left, const uint8_t *right)
{
    if (!s || !left || !right) return fail(RSGM_ERR_INVALID_ARG, "NULL handle or image");
    DeviceGuard dg(s->device);
    if (!dg.ok) return fail(RSGM_ERR_CUDA, "cannot select the handle's device");
    const uint8_t *dl, *dr;
    int rc = stage_images(s, left, right, &dl, &dr);
    if (rc) return rc;
    RSGM_MARK(s, 0);
    RSGM_CUDA(launch_full_window(s->buf, s->g, s->st));
    rc = match_and_update(s, dl, dr, false, nullptr, frame_params(s, nullptr, RSGM_SLOT_FULL));
    if (rc) return rc;
    s->has_state = true;
    memset(s->slot_state, 1, sizeof(s->slot_state));
    s->learned_frame = false;
    return RSGM_OK;
}

int rsgm_reduced_frame(rsgm_stream s, const uint8_t *left, const uint8_t *right, const float *R,
                       const float *t, const float *K, float baseline)
{
    int rc = check_reduced_args(s, left, right, R, t, K, baseline);
    if (rc) return rc;
    DeviceGuard dg(s->device);
    if (!dg.ok) return fail(RSGM_ERR_CUDA, "cannot select the handle's device");
    return enqueue_reduced(s, left, right, R, t, K, baseline);
}

int rsgm_slot_frame(rsgm_stream s, const uint8_t *roles, const uint8_t *left, const uint8_t *right, const float *R,
                    const float *t, const float *K, float baseline)
{
    if (!s || !roles) return fail(RSGM_ERR_INVALID_ARG, "NULL handle or roles");
    int nact = 0;
    for (int b = 0; b < s->g.B; ++b) {
        if (roles[b] > RSGM_SLOT_FULL) return fail(RSGM_ERR_INVALID_ARG, "role %d of stream %d", roles[b], b);
        nact += roles[b] != RSGM_SLOT_IDLE;
    }
    if (!left || !right || !R || !t || !K) return fail(RSGM_ERR_INVALID_ARG, "NULL image or motion array");
    if (!(baseline > 0.0f) || !(K[0] > 0.0f) || !(K[4] > 0.0f) || K[1] != 0.0f || K[3] != 0.0f ||
        K[6] != 0.0f || K[7] != 0.0f || K[8] != 1.0f)
        return fail(RSGM_ERR_INVALID_ARG, "K must be [fx 0 cx; 0 fy cy; 0 0 1] with fx, fy > 0; baseline > 0");
    for (int b = 0; b < s->g.B; ++b)
        if (roles[b] == RSGM_SLOT_REDUCED && !s->slot_state[b])
            return fail(RSGM_ERR_NO_STATE, "reduced frame of stream %d before its first frame", b);
    if (s->P.radius_mode == RSGM_RADIUS_LEARNED && !s->cnn)
        return fail(RSGM_ERR_INVALID_ARG, "RSGM_RADIUS_LEARNED handle without an attached network");
    if (nact == 0) return RSGM_OK;  // nothing advances
    DeviceGuard dg(s->device);
    if (!dg.ok) return fail(RSGM_ERR_CUDA, "cannot select the handle's device");
    int rc = enqueue_reduced(s, left, right, R, t, K, baseline, roles);
    if (rc) return rc;
    for (int b = 0; b < s->g.B; ++b)
        if (roles[b] == RSGM_SLOT_FULL) s->slot_state[b] = 1;
    s->has_state = true;
    return RSGM_OK;
}

int rsgm_state(rsgm_stream s, float *disp, float *var, uint8_t *moving_mask, int16_t *disp_int)
{
    if (!s) return fail(RSGM_ERR_INVALID_ARG, "NULL handle");
    if (!s->has_state) return fail(RSGM_ERR_NO_STATE, "no frame processed yet");
    DeviceGuard dg(s->device);
    if (!dg.ok) return fail(RSGM_ERR_CUDA, "cannot select the handle's device");
    size_t n = (size_t)s->g.NPIX;
    if (disp) RSGM_CUDA(cudaMemcpyAsync(disp, s->buf.d, n * sizeof(float), cudaMemcpyDefault, s->st));
    if (var) RSGM_CUDA(cudaMemcpyAsync(var, s->buf.p, n * sizeof(float), cudaMemcpyDefault, s->st));
    if (moving_mask) RSGM_CUDA(cudaMemcpyAsync(moving_mask, s->buf.mask, n, cudaMemcpyDefault, s->st));
    if (disp_int)
        RSGM_CUDA(cudaMemcpyAsync(disp_int, s->buf.d_int, n * sizeof(int16_t), cudaMemcpyDefault, s->st));
    return RSGM_OK;
}

int rsgm_set_state(rsgm_stream s, const float *disp, const float *var)
{
    if (!s || !disp || !var) return fail(RSGM_ERR_INVALID_ARG, "NULL handle or state");
    DeviceGuard dg(s->device);
    if (!dg.ok) return fail(RSGM_ERR_CUDA, "cannot select the handle's device");
    size_t n = (size_t)s->g.NPIX;
    RSGM_CUDA(cudaMemcpyAsync(s->buf.d, disp, n * sizeof(float), cudaMemcpyDefault, s->st));
    RSGM_CUDA(cudaMemcpyAsync(s->buf.p, var, n * sizeof(float), cudaMemcpyDefault, s->st));
    s->has_state = true;
    memset(s->slot_state, 1, sizeof(s->slot_state));
    return RSGM_OK;
}

int rsgm_read_buffer(rsgm_stream s, int which, void *dst, size_t capacity, size_t *bytes)
{
    if (!s) return fail(RSGM_ERR_INVALID_ARG, "NULL handle");
    DeviceGuard dg(s->device);
    if (!dg.ok) return fail(RSGM_ERR_CUDA, "cannot select the handle's device");
    size_t n = (size_t)s->g.NPIX;
    const void *src = nullptr;
    size_t size = 0;
    if (which == RSGM_BUF_COST || which == RSGM_BUF_AGGREGATED || which == RSGM_BUF_OFFSET)
        return read_ragged(s, which, dst, capacity, bytes);
    {
        switch (which) {
        case RSGM_BUF_CENSUS_L: src = s->buf.cen_l; size = n * 8; break;
        case RSGM_BUF_CENSUS_R: src = s->buf.cen_r; size = n * 8; break;
        case RSGM_BUF_WINDOW: src = s->buf.win; size = n * 4; break;
        case RSGM_BUF_CLASS: src = s->buf.cls; size = n; break;
        case RSGM_BUF_D_PRED: src = s->buf.d_pred; size = n * 4; break;
        case RSGM_BUF_P_PRED: src = s->buf.p_pred; size = n * 4; break;
        case RSGM_BUF_D_MEAS: src = s->buf.d_z; size = n * 4; break;
        case RSGM_BUF_INNOVATION: src = s->buf.nu; size = n * 4; break;
        case RSGM_BUF_CNN_INPUT: src = s->lb.feats; size = n * 32; break;
        case RSGM_BUF_CNN_OUTPUT: src = s->lb.out; size = n * kCnnOutPad * 4; break;
        case RSGM_BUF_RADIUS: src = s->lb.radius; size = n; break;
        case RSGM_BUF_R_MEAS: src = s->lb.r_map; size = n * 4; break;
        default: return fail(RSGM_ERR_INVALID_ARG, "unknown buffer %d", which);
        }
    }
    if (size && !src) return fail(RSGM_ERR_INVALID_ARG, "buffer %d does not exist: no network attached", which);
    if (bytes) *bytes = size;
    if (!dst) return RSGM_OK;
    if (capacity < size) return fail(RSGM_ERR_INVALID_ARG, "capacity %zu < %zu bytes", capacity, size);
    if (size) RSGM_CUDA(cudaMemcpyAsync(dst, src, size, cudaMemcpyDefault, s->st));
    RSGM_CUDA(cudaStreamSynchronize(s->st));
    return RSGM_OK;
}

int rsgm_counters(rsgm_stream s, uint64_t *frames, uint64_t *cells, uint64_t *last_cells)
{
    if (!s) return fail(RSGM_ERR_INVALID_ARG, "NULL handle");
    DeviceGuard dg(s->device);
    if (!dg.ok) return fail(RSGM_ERR_CUDA, "cannot select the handle's device");
    unsigned long long h[3];
    RSGM_CUDA(cudaMemcpyAsync(h, s->buf.counters, sizeof(h), cudaMemcpyDeviceToHost, s->st));
    RSGM_CUDA(cudaStreamSynchronize(s->st));
    if (frames) *frames = h[0];
    if (cells) *cells = h[1];
    if (last_cells) *last_cells = h[2];
    return RSGM_OK;
}

int rsgm_median(rsgm_stream s, float *out)
{
    if (!s || !out) return fail(RSGM_ERR_INVALID_ARG, "NULL handle or output");
    if (!s->has_state) return fail(RSGM_ERR_NO_STATE, "no frame processed yet");
    DeviceGuard dg(s->device);
    if (!dg.ok) return fail(RSGM_ERR_CUDA, "cannot select the handle's device");
    RSGM_CUDA(launch_median3(s->buf.d, s->buf.median, s->g, s->st));
    RSGM_CUDA(cudaMemcpyAsync(out, s->buf.median, (size_t)s->g.NPIX * sizeof(float), cudaMemcpyDefault, s->st));
    return RSGM_OK;
}

int rsgm_default_detect_params(rsgm_detect_params *p)
{
    if (!p) return fail(RSGM_ERR_INVALID_ARG, "params is NULL");
    memset(p, 0, sizeof(*p));
    const int sizes[5][2] = {{20, 20}, {30, 30}, {40, 40}, {50, 50}, {50, 75}};
    p->nsizes = 5;
    for (int i = 0; i < 5; ++i) {
        p->sizes[i][0] = sizes[i][0];
        p->sizes[i][1] = sizes[i][1];
    }
    p->stride = 10;
    p->skip_num = 1;
    p->skip_den = 3;
    p->thresh_px = 1.0f;
    p->iou_num = 0;
    p->iou_den = 1;
    p->min_area = 1500;
    return RSGM_OK;
}

int rsgm_detect(rsgm_stream s, const rsgm_detect_params *p, rsgm_box *boxes, int32_t capacity, int32_t *counts)
{
    if (!s || !p || !counts || capacity < 0 || (capacity > 0 && !boxes))
        return fail(RSGM_ERR_INVALID_ARG, "NULL handle, params, boxes or counts");
    if (p->nsizes < 1 || p->nsizes > RSGM_MAX_WINDOW_SIZES || p->stride < 1 || p->skip_den < 1 ||
        p->skip_num < 0 || p->skip_num > p->skip_den || p->iou_den < 1 || p->iou_num < 0 || p->min_area < 0 ||
        !(p->thresh_px >= 0.0f) || p->thresh_px > 4096.0f)
        return fail(RSGM_ERR_INVALID_ARG, "detection parameters out of range");
    for (int i = 0; i < p->nsizes; ++i)
        if (p->sizes[i][0] < 1 || p->sizes[i][1] < 1) return fail(RSGM_ERR_INVALID_ARG, "window size < 1");
    if (!s->has_state) return fail(RSGM_ERR_NO_STATE, "no frame processed yet");
    DeviceGuard dg(s->device);
    if (!dg.ok) return fail(RSGM_ERR_CUDA, "cannot select the handle's device");
    const Geometry &g = s->g;
    DetectPlan dp;
    memset(&dp, 0, sizeof(dp));
    dp.nsizes = p->nsizes;
    dp.stride = p->stride;
    dp.y_min = (int)((long long)g.H * p->skip_num / p->skip_den);
    dp.thresh_q = (unsigned)floorf(p->thresh_px * 16.0f + 0.5f);
    for (int i = 0; i < p->nsizes; ++i) {
        dp.size[i][0] = p->sizes[i][0];
        dp.size[i][1] = p->sizes[i][1];
        dp.nx[i] = p->sizes[i][0] <= g.W ? (g.W - p->sizes[i][0]) / p->stride + 1 : 0;
        dp.ny[i] = dp.y_min + p->sizes[i][1] <= g.H ? (g.H - p->sizes[i][1] - dp.y_min) / p->stride + 1 : 0;
        dp.first[i + 1] = dp.first[i] + dp.nx[i] * dp.ny[i];
    }
    dp.total = dp.first[p->nsizes];
    RSGM_CUDA(launch_detect_windows(s->buf, g, dp, s->st));
    const size_t nflags = (size_t)g.B * dp.total;
    uint8_t *flags = (uint8_t *)malloc(nflags ? nflags : 1);
    if (!flags) return fail(RSGM_ERR_OOM, "host allocation failed");
    cudaError_t e = nflags ? cudaMemcpyAsync(flags, s->buf.flags, nflags, cudaMemcpyDeviceToHost, s->st) : cudaSuccess;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) {
        free(flags);
        return cuda_fail(e, "detection flags");
    }
    // the streams' groupings are independent: spread them over host threads
    auto group = [&](int b) {
        counts[b] = group_boxes(flags + (size_t)b * dp.total, dp, p->iou_num, p->iou_den, p->min_area,
                                capacity > 0 ? (int32_t *)(boxes + (size_t)b * capacity) : nullptr, capacity);
    };
    const int nt = std::min(g.B, (int)std::max(1u, std::min(std::thread::hardware_concurrency(), 64u)));
    if (nt <= 1) {
        for (int b = 0; b < g.B; ++b) group(b);
    } else {
        std::vector<std::thread> pool;
        pool.reserve(nt);
        try {
            for (int t = 0; t < nt; ++t)
                pool.emplace_back([&, t] {
                    for (int b = t; b < g.B; b += nt) group(b);
                });
        } catch (...) {
            // a thread could not be started: its share runs here, below
        }
        for (std::thread &th : pool) th.join();
        for (int t = (int)pool.size(); t < nt; ++t)
            for (int b = t; b < g.B; b += nt) group(b);
    }
    free(flags);
    return RSGM_OK;
}

int rsgm_enable_stage_timing(rsgm_stream s, int enable)
{
    if (!s) return fail(RSGM_ERR_INVALID_ARG, "NULL handle");
    DeviceGuard dg(s->device);
    if (!dg.ok) return fail(RSGM_ERR_CUDA, "cannot select the handle's device");
    StageTimer &t = s->timer;
    if (enable && !t.ev) {
        int total = kMaxTimedFrames * (RSGM_NUM_STAGES + 1);
        t.ev = (cudaEvent_t *)calloc((size_t)total, sizeof(cudaEvent_t));
        if (!t.ev) return fail(RSGM_ERR_OOM, "host allocation failed");
        for (int i = 0; i < total; ++i) {
            cudaError_t e = cudaEventCreate(&t.ev[i]);
            if (e != cudaSuccess) {
                destroy_timer(t);
                return cuda_fail(e, "cudaEventCreate");
            }
        }
    }
    t.on = enable != 0;
    t.n = 0;
    return RSGM_OK;
}

int rsgm_stage_times(rsgm_stream s, double *ms, int32_t *frames)
{
    if (!s || !ms) return fail(RSGM_ERR_INVALID_ARG, "NULL handle or output");
    DeviceGuard dg(s->device);
    if (!dg.ok) return fail(RSGM_ERR_CUDA, "cannot select the handle's device");
    RSGM_CUDA(cudaStreamSynchronize(s->st));
    StageTimer &t = s->timer;
    for (int k = 0; k < RSGM_NUM_STAGES; ++k) ms[k] = 0.0;
    for (int f = 0; f < t.n; ++f) {
        cudaEvent_t *e = t.ev + f * (RSGM_NUM_STAGES + 1);
        for (int k = 0; k < RSGM_NUM_STAGES; ++k) {
            float dt = 0.0f;
            RSGM_CUDA(cudaEventElapsedTime(&dt, e[k], e[k + 1]));
            ms[k] += dt;
        }
    }
    if (frames) *frames = t.n;
    t.n = 0;
    return RSGM_OK;
}

int rsgm_measure_int_peak(int kind, void *cuda_stream, double *ops_per_s)
{
    if (!ops_per_s || kind < RSGM_PEAK_I32_ADD || kind > RSGM_PEAK_U16X2_MIX)
        return fail(RSGM_ERR_INVALID_ARG, "unknown peak kind %d or NULL output", kind);
    *ops_per_s = 0.0;
    int dev = 0, sms = 0;
    RSGM_CUDA(cudaGetDevice(&dev));
    RSGM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int blocks = sms * peak_blocks_per_sm();
    const int iters = 1 << 15;  // several milliseconds per launch at the expected rates
    cudaEvent_t e0, e1;
    RSGM_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(RSGM_ERR_CUDA, "cudaEventCreate failed");
    }
    float best = 0.0f;
    cudaError_t e = launch_peak(kind, blocks, iters, st);  // warm-up
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        float ms = 0.0f;
        if ((e = cudaEventRecord(e0, st)) != cudaSuccess || (e = launch_peak(kind, blocks, iters, st)) != cudaSuccess ||
            (e = cudaEventRecord(e1, st)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
            (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
            break;
        if (best == 0.0f || ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "integer peak launch");
    if (!(best > 0.0f)) return fail(RSGM_ERR_CUDA, "integer peak: no time measured");
    *ops_per_s = peak_ops(kind, blocks, iters) / (best * 1e-3);
    return RSGM_OK;
}

int rsgm_sync(rsgm_stream s)
{
    if (!s) return fail(RSGM_ERR_INVALID_ARG, "NULL handle");
    DeviceGuard dg(s->device);
    if (!dg.ok) return fail(RSGM_ERR_CUDA, "cannot select the handle's device");
    RSGM_CUDA(cudaStreamSynchronize(s->st));
    return RSGM_OK;
}

int rsgm_destroy_stream(rsgm_stream s)
{
    if (!s) return RSGM_OK;
    int rc = RSGM_OK;
    {
        DeviceGuard dg(s->device);
        cudaError_t e = cudaStreamSynchronize(s->st);
        if (e == cudaSuccess && s->side) e = cudaStreamSynchronize(s->side);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
        free_buffers(s->buf);
        free_learned(s->lb);
        destroy_timer(s->timer);
        release_side(s);
    }
    delete s;
    return rc;
}

const char *rsgm_status_string(int code)
{
    switch (code) {
    case RSGM_OK: return "ok";
    case RSGM_ERR_INVALID_ARG: return "invalid argument";
    case RSGM_ERR_NO_STATE: return "no state: run a full frame (or set_state) first";
    case RSGM_ERR_OOM: return "device allocation failed";
    case RSGM_ERR_CUDA: return "CUDA error";
    case RSGM_ERR_TIMEOUT: return "device wait timed out";
    case RSGM_ERR_CHECK_FAILED: return "device consistency check failed";
    default: return "unknown status";
    }
}

const char *rsgm_last_error(void) { return g_last_error; }

// ------------------------------------------------------------------ groups

// ------------------------------------------------------------------ the learned window

int rsgm_cnn_create(rsgm_cnn *out, const float *params, void *cuda_stream)
{
    if (!out || !params) return fail(RSGM_ERR_INVALID_ARG, "NULL output or parameters");
    *out = nullptr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    rsgm_cnn c = new (std::nothrow) rsgm_cnn_s();
    if (!c) return fail(RSGM_ERR_OOM, "host allocation failed");
    c->device = dev;
    c->st = (cudaStream_t)cuda_stream;
    CnnWeights &w = c->w;
    void *all[40];
    int nall = 0, rc = RSGM_OK;
    if ((rc = alloc(&w.theta, kCnnParams, all, nall)) || (rc = alloc(&w.m, kCnnParams, all, nall)) ||
        (rc = alloc(&w.v, kCnnParams, all, nall)) || (rc = alloc(&w.grad, kCnnParams, all, nall))) {
        free_cnn(c);
        delete c;
        return rc;
    }
    for (int l = 0; l < kCnnLayers && rc == RSGM_OK; ++l) {
        const size_t cinp = l == 0 ? 16 : 32, coutp = l == kCnnLayers - 1 ? kCnnOutPad : 32;
        const size_t kp = l == kCnnLayers - 1 ? 16 : 32;
        uint16_t *wf = nullptr, *wb = nullptr;
        rc = alloc(&wf, 9 * coutp * cinp, all, nall);
        w.wf[l] = wf;
        if (!rc && l > 0) {
            rc = alloc(&wb, 9 * 32 * kp, all, nall);
            w.wb[l] = wb;
        }
        if (!rc) rc = alloc(&w.bias[l], coutp, all, nall);
    }
    if (!rc) {
        if ((e = cudaMemcpyAsync(w.theta, params, kCnnParams * sizeof(float), cudaMemcpyDefault, c->st)) != cudaSuccess ||
            (e = cudaMemsetAsync(w.m, 0, kCnnParams * sizeof(float), c->st)) != cudaSuccess ||
            (e = cudaMemsetAsync(w.v, 0, kCnnParams * sizeof(float), c->st)) != cudaSuccess ||
            (e = cudaMemsetAsync(w.grad, 0, kCnnParams * sizeof(float), c->st)) != cudaSuccess ||
            (e = cnn_pack(w, c->st)) != cudaSuccess || (e = cudaStreamSynchronize(c->st)) != cudaSuccess)
            rc = cuda_fail(e, "network initialisation");
    }
    if (rc) {
        free_cnn(c);
        delete c;
        return rc;
    }
    *out = c;
    return RSGM_OK;
}

namespace {
int cnn_copy_out(rsgm_cnn c, float *host, const float *src)
{
    if (!c || !host) return fail(RSGM_ERR_INVALID_ARG, "NULL network or destination");
    DeviceGuard dg(c->device);
    if (!dg.ok) return fail(RSGM_ERR_CUDA, "cannot select the network's device");
    RSGM_CUDA(cudaMemcpyAsync(host, src, kCnnParams * sizeof(float), cudaMemcpyDefault, c->st));
    RSGM_CUDA(cudaStreamSynchronize(c->st));
    return RSGM_OK;
}
}  // namespace

int rsgm_cnn_params(rsgm_cnn c, float *params) { return cnn_copy_out(c, params, c ? c->w.theta : nullptr); }

int rsgm_cnn_grad(rsgm_cnn c, float *grad) { return cnn_copy_out(c, grad, c ? c->w.grad : nullptr); }

int rsgm_cnn_destroy(rsgm_cnn c)
{
    if (!c) return RSGM_OK;
    int rc = RSGM_OK;
    {
        DeviceGuard dg(c->device);
        cudaError_t e = cudaStreamSynchronize(c->st);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
        free_cnn(c);
    }
    delete c;
    return rc;
}

int rsgm_attach_cnn(rsgm_stream s, rsgm_cnn c)
{
    if (!s || !c) return fail(RSGM_ERR_INVALID_ARG, "NULL handle or network");
    if (s->P.radius_mode != RSGM_RADIUS_LEARNED)
        return fail(RSGM_ERR_INVALID_ARG, "the handle was not created with RSGM_RADIUS_LEARNED");
    if (s->device != c->device) return fail(RSGM_ERR_INVALID_ARG, "the network and the handle must share one device");
    DeviceGuard dg(s->device);
    if (!dg.ok) return fail(RSGM_ERR_CUDA, "cannot select the handle's device");
    if (!s->lb.feats) {
        LearnedBuffers &lb = s->lb;
        const size_t n = (size_t)s->g.NPIX;
        void *all[16];
        int nall = 0, rc;
        uint8_t *feats = nullptr, *a0 = nullptr, *a1 = nullptr, *a2 = nullptr;
        if ((rc = alloc(&feats, n * 32, all, nall)) || (rc = alloc(&a0, n * 64, all, nall)) ||
            (rc = alloc(&a1, n * 64, all, nall)) || (rc = alloc(&a2, n * 64, all, nall)) ||
            (rc = alloc(&lb.out, n * kCnnOutPad, all, nall)) || (rc = alloc(&lb.radius, n, all, nall)) ||
            (rc = alloc(&lb.r_map, n, all, nall))) {
            for (int i = 0; i < nall; ++i) cudaFree(all[i]);
            memset(&lb, 0, sizeof(lb));
            return rc;
        }
        lb.feats = feats;
        lb.act[0] = a0;
        lb.act[1] = a1;
        lb.act[2] = a2;
    }
    s->cnn = c;
    s->buf.radius = s->lb.radius;
    return RSGM_OK;
}

int rsgm_cnn_train_step(rsgm_cnn c, rsgm_stream s, const float *d_target, float lr, float *loss)
{
    if (!c || !s || !d_target) return fail(RSGM_ERR_INVALID_ARG, "NULL network, handle or target");
    if (s->cnn != c) return fail(RSGM_ERR_INVALID_ARG, "the network is not attached to this handle");
    if (s->st != c->st) return fail(RSGM_ERR_INVALID_ARG, "training runs on the network's own CUDA stream");
    if (!s->learned_frame) return fail(RSGM_ERR_NO_STATE, "no learned reduced frame to train on");
    if (!(lr >= 0.0f)) return fail(RSGM_ERR_INVALID_ARG, "lr must be >= 0");
    DeviceGuard dg(s->device);
    if (!dg.ok) return fail(RSGM_ERR_CUDA, "cannot select the handle's device");
    if (!is_device_pointer(d_target)) return fail(RSGM_ERR_INVALID_ARG, "d_target must be device memory");
    LearnedBuffers &lb = s->lb;
    if (!lb.g16) {
        const size_t n = (size_t)s->g.NPIX;
        void *all[8];
        int nall = 0, rc;
        uint8_t *g16 = nullptr, *ga = nullptr, *gb = nullptr;
        if ((rc = alloc(&g16, n * 32, all, nall)) || (rc = alloc(&ga, n * 64, all, nall)) ||
            (rc = alloc(&gb, n * 64, all, nall)) || (rc = alloc(&lb.loss, 1, all, nall))) {
            for (int i = 0; i < nall; ++i) cudaFree(all[i]);
            lb.loss = nullptr;
            return rc;
        }
        lb.g16 = g16;
        lb.ga = ga;
        lb.gb = gb;
    }
    RSGM_CUDA(cnn_backward(c->w, lb, s->buf, s->g, d_target, s->sm_count, s->st));
    if (lr > 0.0f) {
        c->step++;
        RSGM_CUDA(cnn_adam(c->w, c->step, lr, s->st));
    }
    if (loss) {
        RSGM_CUDA(cudaMemcpyAsync(loss, lb.loss, sizeof(float), cudaMemcpyDeviceToHost, s->st));
        RSGM_CUDA(cudaStreamSynchronize(s->st));
    }
    return RSGM_OK;
}

int rsgm_set_schedule(rsgm_stream s, int32_t cells)
{
    if (!s) return fail(RSGM_ERR_INVALID_ARG, "NULL handle");
    if (cells < 0 || cells > 32) return fail(RSGM_ERR_INVALID_ARG, "schedule (register capacity) in [0, 32]");
    s->tuned_cap = cells ? sweep_capacity(cells) : 0;
    s->tuned_hl = 0;
    return RSGM_OK;
}

int rsgm_set_rows_per_warp(rsgm_stream s, int32_t rows)
{
    if (!s) return fail(RSGM_ERR_INVALID_ARG, "NULL handle");
    if (rows != 0 && rows != 8 && rows != 16 && rows != 32)
        return fail(RSGM_ERR_INVALID_ARG, "rows per warp must be 0, 8, 16 or 32");
    s->tuned_hl = rows;
    return RSGM_OK;
}

int rsgm_get_schedule(rsgm_stream s, int32_t *cells, int32_t *rows)
{
    if (!s) return fail(RSGM_ERR_INVALID_ARG, "NULL handle");
    if (cells) *cells = s->tuned_cap ? s->tuned_cap : sweep_capacity(s->capacity);
    if (rows) *rows = s->tuned_hl;
    return RSGM_OK;
}

int rsgm_autotune_times(rsgm_stream s, int32_t *cells, int32_t *rows, float *ms, int32_t n, int32_t *count)
{
    if (!s || !count) return fail(RSGM_ERR_INVALID_ARG, "NULL handle or count");
    if (n < 0 || (n > 0 && (!cells || !rows || !ms))) return fail(RSGM_ERR_INVALID_ARG, "bad output arrays");
    *count = s->ntimed;
    for (int i = 0; i < s->ntimed && i < n; ++i) {
        cells[i] = s->timed_cap[i];
        rows[i] = s->timed_hl[i];
        ms[i] = s->timed_ms[i];
    }
    return RSGM_OK;
}

int rsgm_autotune(rsgm_stream s, int32_t *cells)
{
    if (!s) return fail(RSGM_ERR_INVALID_ARG, "NULL handle");
    if (!s->has_state) return fail(RSGM_ERR_NO_STATE, "autotuning needs a processed frame");
    DeviceGuard dg(s->device);
    if (!dg.ok) return fail(RSGM_ERR_CUDA, "cannot select the handle's device");
    s->ntimed = 0;
    // Each candidate is timed as a frame runs it: the cost kernel, then the
    // aggregation between two events (as the stage timer brackets it), kReps
    // times queued back to back behind one untimed round, so that the host's
    // cost of issuing the launches stays hidden behind GPU work.  Launches of
    // the aggregation alone, back to back, ran slower than inside frames and
    // misjudged the row sweep.  The cost kernel rewrites the same costs and
    // metadata from the unchanged census and windows, and every schedule
    // writes the same planes, so the handle's buffers end as they were.
    constexpr int kReps = 3;
    cudaEvent_t ev[2 * kReps] = {};
    int rc = RSGM_OK;
    for (int i = 0; i < 2 * kReps && rc == RSGM_OK; ++i)
        if (cudaEventCreate(&ev[i]) != cudaSuccess) rc = fail(RSGM_ERR_CUDA, "cudaEventCreate");
    // candidates: the instantiated register capacities, and the row sweep or
    // 8, 16 or 32 rows per warp of the line sweep for the horizontal directions
    const int caps[4] = {2, 6, 10, 18}, hls[4] = {0, 8, 16, 32};
    const int nh = (s->P.path_mask & 3u) ? 4 : 1, nc = 4 * nh;
    int best = 0, best_hl = 0;
    float best_ms = 0.0f;
    for (int ci = 0; ci < nc && rc == RSGM_OK; ++ci) {
        const int cand = caps[ci / nh], hl = hls[ci % nh];
        float ms = 1e30f;
        for (int trial = 0; trial < 2 && rc == RSGM_OK; ++trial) {
            cudaError_t e = launch_cost(s->buf, s->g, s->nbits, s->st);
            if (e == cudaSuccess) e = launch_aggregation(s, cand, hl, s->st);
            for (int rep = 0; rep < kReps && e == cudaSuccess; ++rep) {
                e = launch_cost(s->buf, s->g, s->nbits, s->st);
                if (e == cudaSuccess) e = cudaEventRecord(ev[2 * rep], s->st);
                if (e == cudaSuccess) e = launch_aggregation(s, cand, hl, s->st);
                if (e == cudaSuccess) e = cudaEventRecord(ev[2 * rep + 1], s->st);
            }
            if (e == cudaSuccess) e = cudaEventSynchronize(ev[2 * kReps - 1]);
            float total = 0.0f;
            for (int rep = 0; rep < kReps && e == cudaSuccess; ++rep) {
                float t = 0.0f;
                e = cudaEventElapsedTime(&t, ev[2 * rep], ev[2 * rep + 1]);
                total += t;
            }
            if (e != cudaSuccess) rc = cuda_fail(e, "autotune timing");
            if (total / kReps < ms) ms = total / kReps;
        }
        if (rc == RSGM_OK) {
            s->timed_cap[ci] = cand;
            s->timed_hl[ci] = hl;
            s->timed_ms[ci] = ms;
        }
        if (rc == RSGM_OK && (best == 0 || ms < best_ms)) {
            best = cand;
            best_hl = hl;
            best_ms = ms;
        }
    }
    for (int i = 0; i < 2 * kReps; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    if (rc) return rc;
    s->ntimed = nc;
    s->tuned_cap = best;
    s->tuned_hl = best_hl;
    if (cells) *cells = best;
    return RSGM_OK;
}

}  // extern "C"

struct rsgm_group_s {
    int n;
    rsgm_stream *members;   // not owned
    cudaStream_t launch;    // the members' stream: the graph is launched there
    cudaStream_t *cap;      // one capture stream per member
    cudaEvent_t fork;
    cudaEvent_t *join;
    cudaGraphExec_t exec;
    int device;
};

namespace {
void destroy_group(rsgm_group g)
{
    if (g->exec) cudaGraphExecDestroy(g->exec);
    for (int k = 0; k < g->n; ++k) {
        if (g->cap && g->cap[k]) cudaStreamDestroy(g->cap[k]);
        if (g->join && g->join[k]) cudaEventDestroy(g->join[k]);
    }
    if (g->fork) cudaEventDestroy(g->fork);
    free(g->cap);
    free(g->join);
    free(g->members);
    free(g);
}
}  // namespace

extern "C" {

int rsgm_group_create(rsgm_group *out, rsgm_stream *members, int32_t n)
{
    if (!out) return fail(RSGM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!members || n < 1 || n > 64) return fail(RSGM_ERR_INVALID_ARG, "a group has 1 to 64 members");
    for (int k = 0; k < n; ++k) {
        if (!members[k]) return fail(RSGM_ERR_INVALID_ARG, "NULL member");
        if (members[k]->P.radius_mode == RSGM_RADIUS_LEARNED)
            return fail(RSGM_ERR_INVALID_ARG, "a learned-window handle cannot join a group");
        if (members[k]->device != members[0]->device || members[k]->st != members[0]->st)
            return fail(RSGM_ERR_INVALID_ARG, "group members must share one device and one CUDA stream");
        for (int j = 0; j < k; ++j)
            if (members[j] == members[k]) return fail(RSGM_ERR_INVALID_ARG, "a handle appears twice in the group");
    }
    DeviceGuard dg(members[0]->device);
    if (!dg.ok) return fail(RSGM_ERR_CUDA, "cannot select the members' device");
    rsgm_group g = (rsgm_group)calloc(1, sizeof(rsgm_group_s));
    if (!g) return fail(RSGM_ERR_OOM, "host allocation failed");
    g->n = n;
    g->launch = members[0]->st;
    g->device = members[0]->device;
    g->members = (rsgm_stream *)calloc((size_t)n, sizeof(rsgm_stream));
    g->cap = (cudaStream_t *)calloc((size_t)n, sizeof(cudaStream_t));
    g->join = (cudaEvent_t *)calloc((size_t)n, sizeof(cudaEvent_t));
    if (!g->members || !g->cap || !g->join) {
        destroy_group(g);
        return fail(RSGM_ERR_OOM, "host allocation failed");
    }
    memcpy(g->members, members, (size_t)n * sizeof(rsgm_stream));
    cudaError_t e = cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming);
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&g->cap[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->join[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        destroy_group(g);
        return cuda_fail(e, "group streams");
    }
    *out = g;
    return RSGM_OK;
}

int rsgm_group_reduced_frame(rsgm_group g, const uint8_t *const *left, const uint8_t *const *right,
                             const float *const *R, const float *const *t, const float *const *K,
                             const float *baseline)
{
    if (!g || !left || !right || !R || !t || !K || !baseline)
        return fail(RSGM_ERR_INVALID_ARG, "NULL group or argument array");
    for (int k = 0; k < g->n; ++k) {
        int rc = check_reduced_args(g->members[k], left[k], right[k], R[k], t[k], K[k], baseline[k]);
        if (rc) return rc;
        if (!is_device_pointer(left[k]) || !is_device_pointer(right[k]))
            return fail(RSGM_ERR_INVALID_ARG, "group frames take device images");
    }
    DeviceGuard dg(g->device);
    if (!dg.ok) return fail(RSGM_ERR_CUDA, "cannot select the group's device");
    // Capture every member's frame on its own stream (forked from and joined
    // back into the first), so that the graph runs them concurrently.
    RSGM_CUDA(cudaStreamBeginCapture(g->cap[0], cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaEventRecord(g->fork, g->cap[0]);
    for (int k = 1; k < g->n && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(g->cap[k], g->fork, 0);
    int rc = e == cudaSuccess ? RSGM_OK : cuda_fail(e, "group fork");
    for (int k = 0; k < g->n && rc == RSGM_OK; ++k) {
        rsgm_stream m = g->members[k];
        cudaStream_t saved = m->st;
        m->st = g->cap[k];
        m->capturing = true;
        rc = enqueue_reduced(m, left[k], right[k], R[k], t[k], K[k], baseline[k]);
        m->capturing = false;
        m->st = saved;
    }
    for (int k = 1; k < g->n && rc == RSGM_OK; ++k) {
        e = cudaEventRecord(g->join[k], g->cap[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(g->cap[0], g->join[k], 0);
        if (e != cudaSuccess) rc = cuda_fail(e, "group join");
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(g->cap[0], &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    // Same launches every tick, new arguments: update the executable in place.
    if (g->exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(g->exec, graph, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(g->exec);
            g->exec = nullptr;
        }
    }
    if (!g->exec && (e = cudaGraphInstantiate(&g->exec, graph, 0)) != cudaSuccess) {
        cudaGraphDestroy(graph);
        g->exec = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    e = cudaGraphLaunch(g->exec, g->launch);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return RSGM_OK;
}

int rsgm_group_destroy(rsgm_group g)
{
    if (!g) return RSGM_OK;
    DeviceGuard dg(g->device);
    cudaError_t e = cudaStreamSynchronize(g->launch);
    destroy_group(g);
    return e == cudaSuccess ? RSGM_OK : cuda_fail(e, "cudaStreamSynchronize");
}

}  // extern "C"
