// The learned search window: a 4-layer 3x3 network per pixel picks the
// window half-width from {1, 2, 4, 8, 16} and a measurement variance r, in
// place of the fixed or variance-derived half-width of the search window
// (Section 2.4, d_pred +- p).  The ragged cell volume already admits any
// per-pixel width, so the rest of the path is unchanged.
//
// Inputs per pixel (from the hole-filled prediction, before the
// discontinuity reset): d / D, sqrt(p) / D, the census Hamming distance at the
// rounded predicted disparity / bits, and the Sobel magnitude / 2040 (1, 1 and
// 0 without a prediction).  Layers: 4 -> 32 -> 32 -> 32 -> 6 channels, 3x3,
// zero padding, ReLU between; outputs 5 class logits and log r.
//
// Activations are bfloat16, pixel-major with the channels innermost
// (NHWC); the convolutions are implicit GEMMs on the tensor cores
// (mma.sync m16n8k16, bfloat16 in, fp32 accumulate) over tiles staged in
// shared memory: a warp computes 16 consecutive pixels of one row against
// all output channels, the K dimension running over the 9 taps x 16-channel
// chunks.  The input gradient
// of a layer is the same correlation with the weights flipped and
// transposed, so the forward kernel serves it with a masked epilogue (the
// ReLU derivative).  Weight gradients are fp32 sums on the CUDA cores.
#include <cuda_bf16.h>

#include "rsgm_internal.cuh"

namespace rsgm {
namespace {

constexpr int kConvWarps = 4;
constexpr float kSobelScale = 2040.0f;
constexpr float kConfidence = 0.9f;
constexpr int kFallbackRadius = 8;
constexpr float kRMin = 1.0f / 16.0f, kRMax = 64.0f;
constexpr float kNllWeight = 0.1f;
__constant__ uint8_t kRadii[kCnnClasses] = {1, 2, 4, 8, 16};

enum ConvMode { kReluBf16 = 0, kLinearF32 = 1, kMaskBf16 = 2 };

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x (lower half) = lo
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xFFFF0000u); }

// D += A (16 x 16, row-major fragments) x B (16 x 8, column fragments).
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// The four inputs of each pixel, rounded to bfloat16, in 16 channels (the
// other 12 are zero).  Every quotient is one rounded single-precision
// division.
__global__ void __launch_bounds__(256) k_features(const uint8_t *__restrict__ left,
                                                  const unsigned long long *__restrict__ cen_l,
                                                  const unsigned long long *__restrict__ cen_r,
                                                  const float *__restrict__ d_pred,
                                                  const float *__restrict__ p_pred, Geometry g, int nbits,
                                                  uint4 *__restrict__ feats)
{
    const long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= g.NPIX) return;
    const int b = (int)(gi / g.HW);
    const int s = (int)(gi - (long long)b * g.HW);
    const int y = s / g.W, x = s - y * g.W;
    const uint8_t *img = left + (long long)b * g.HW;
    const int ym = max(y - 1, 0), yp = min(y + 1, g.H - 1), xm = max(x - 1, 0), xp = min(x + 1, g.W - 1);
    auto I = [&](int yy, int xx) { return (int)img[yy * g.W + xx]; };
    const int gx = (I(ym, xp) + 2 * I(y, xp) + I(yp, xp)) - (I(ym, xm) + 2 * I(y, xm) + I(yp, xm));
    const int gy = (I(yp, xm) + 2 * I(yp, x) + I(yp, xp)) - (I(ym, xm) + 2 * I(ym, x) + I(ym, xp));
    const float f3 = __fdiv_rn((float)(abs(gx) + abs(gy)), kSobelScale);
    const float d = d_pred[gi];
    float f0 = 0.0f, f1 = 1.0f, f2 = 1.0f;
    if (d >= 0.0f) {
        const float fD = (float)g.D;
        f0 = __fdiv_rn(d, fD);
        f1 = __fdiv_rn(__fsqrt_rn(p_pred[gi]), fD);
        const float cf = floorf(__fadd_rn(d, 0.5f));
        const int c = cf < 0.0f ? 0 : (cf > (float)(g.D - 1) ? g.D - 1 : (int)cf);
        if (x - c >= 0) f2 = __fdiv_rn((float)__popcll(cen_l[gi] ^ cen_r[gi - c]), (float)nbits);
    }
    feats[2 * gi] = make_uint4(pack_bf16x2(f0, f1), pack_bf16x2(f2, f3), 0u, 0u);
    feats[2 * gi + 1] = make_uint4(0u, 0u, 0u, 0u);
}

// One 3x3 layer as an implicit GEMM.  `in` has CINP channels per pixel, `wt`
// is [9 taps][COUTP][CINP] (B operand: n = output channel, k = input
// channel).  A block owns kConvPix consecutive pixels of one row and stages
// the three input rows they need (with a one-pixel halo, zero outside the
// image) and all the weights in shared memory, each pixel's and each weight
// row's channels padded by 8 so that a warp's fragment loads hit 32
// distinct banks.  Warp w computes pixels 16 w .. 16 w + 15 of the block:
// lane (group g, thread t) reads the A fragment rows g and g + 8 (pixels) at
// channels 2t, 2t + 1 and 2t + 8, 2t + 9 of each 16-channel chunk, and the
// B fragment column g (output channel) at the same channel offsets.
// Epilogue by mode: bias + ReLU to bfloat16, bias to fp32, or zeroed where
// mask <= 0 (the ReLU derivative) to bfloat16.
constexpr int kConvPix = kConvWarps * 16;

template <int CINP, int COUTP, int MODE>
__global__ void __launch_bounds__(kConvWarps * 32) k_conv(const uint32_t *__restrict__ in,
                                                          const uint32_t *__restrict__ wt,
                                                          const float *__restrict__ bias,
                                                          const __nv_bfloat16 *__restrict__ mask,
                                                          void *__restrict__ out, Geometry g, int blocks_x)
{
    static_assert(CINP % 16 == 0 && COUTP % 8 == 0, "channel padding");
    constexpr int NT = COUTP / 8;
    constexpr int XW = (CINP + 8) / 2;  // words per staged pixel
    constexpr int WW = (CINP + 8) / 2;  // words per staged weight row
    constexpr int NPX = kConvPix + 2;   // staged pixels per row
    constexpr int CH16 = CINP / 8;      // 16-byte chunks per pixel
    __shared__ __align__(16) uint32_t xs[3 * NPX * XW];
    __shared__ __align__(16) uint32_t ws[9 * COUTP * WW];
    const long long row = blockIdx.x / blocks_x;  // b * H + y
    const int xb = (int)(blockIdx.x - row * blocks_x) * kConvPix;
    const int y = (int)(row % g.H);
    const long long rbase = row * g.W;
    for (int i = threadIdx.x; i < 3 * NPX * CH16; i += blockDim.x) {
        const int r = i / (NPX * CH16), rem = i - r * NPX * CH16;
        const int px = rem / CH16, q = rem - px * CH16;
        const int yy = y + r - 1, xx = xb + px - 1;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (yy >= 0 && yy < g.H && xx >= 0 && xx < g.W)
            v = reinterpret_cast<const uint4 *>(in)[(rbase + (long long)(r - 1) * g.W + xx) * CH16 + q];
        uint32_t *d = xs + (r * NPX + px) * XW + q * 4;
        d[0] = v.x;
        d[1] = v.y;
        d[2] = v.z;
        d[3] = v.w;
    }
    for (int i = threadIdx.x; i < 9 * COUTP * (CINP / 2); i += blockDim.x) {
        const int wr = i / (CINP / 2);
        ws[wr * WW + (i - wr * (CINP / 2))] = wt[i];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x0 = xb + warp * 16;
    if (x0 >= g.W) return;  // after the only barrier
    const int grp = lane >> 2, tig = lane & 3;
    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
            const int tap = ky * 3 + kx;
            // staged pixel warp * 16 + m + kx holds image column x0 + m + kx - 1
            const uint32_t *xa = xs + (ky * NPX + warp * 16 + grp + kx) * XW;
            const uint32_t *xc = xa + 8 * XW;
#pragma unroll
            for (int c = 0; c < CINP / 16; ++c) {
                const int kw = c * 8 + tig;  // word of channels c * 16 + 2 t, + 1
                const uint32_t a0 = xa[kw], a1 = xc[kw], a2 = xa[kw + 4], a3 = xc[kw + 4];
#pragma unroll
                for (int j = 0; j < NT; ++j) {
                    const uint32_t *wrow = ws + (tap * COUTP + j * 8 + grp) * WW;
                    mma_bf16(acc[j], a0, a1, a2, a3, wrow[kw], wrow[kw + 4]);
                }
            }
        }
    }
    const long long rb = rbase;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int xm = x0 + grp + 8 * h;
        if (xm >= g.W) continue;
        const long long pix = rb + xm;
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const int ch = j * 8 + tig * 2;
            float v0 = acc[j][2 * h], v1 = acc[j][2 * h + 1];
            if (MODE == kReluBf16) {
                v0 = fmaxf(v0 + bias[ch], 0.0f);
                v1 = fmaxf(v1 + bias[ch + 1], 0.0f);
                reinterpret_cast<uint32_t *>(out)[(pix * COUTP + ch) >> 1] = pack_bf16x2(v0, v1);
            } else if (MODE == kLinearF32) {
                reinterpret_cast<float2 *>(out)[(pix * COUTP + ch) >> 1] = make_float2(v0 + bias[ch], v1 + bias[ch + 1]);
            } else {
                const uint32_t m = reinterpret_cast<const uint32_t *>(mask)[(pix * COUTP + ch) >> 1];
                v0 = bf16_lo(m) > 0.0f ? v0 : 0.0f;
                v1 = bf16_hi(m) > 0.0f ? v1 : 0.0f;
                reinterpret_cast<uint32_t *>(out)[(pix * COUTP + ch) >> 1] = pack_bf16x2(v0, v1);
            }
        }
    }
}

// Window half-width and measurement variance from the output: the most
// probable class's radius when its softmax probability is >= 0.9, else 8;
// r = exp(log r) clamped to [1/16, 64].
__global__ void __launch_bounds__(256) k_decide(const float *__restrict__ out, Geometry g,
                                                uint8_t *__restrict__ radius, float *__restrict__ r_map)
{
    const long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= g.NPIX) return;
    const float *o = out + gi * kCnnOutPad;
    int k = 0;
    float zmax = o[0];
#pragma unroll
    for (int i = 1; i < kCnnClasses; ++i)
        if (o[i] > zmax) {
            zmax = o[i];
            k = i;
        }
    float sum = 0.0f;
#pragma unroll
    for (int i = 0; i < kCnnClasses; ++i) sum = __fadd_rn(sum, expf(__fsub_rn(o[i], zmax)));
    const float conf = __fdiv_rn(1.0f, sum);
    radius[gi] = conf >= kConfidence ? kRadii[k] : (uint8_t)kFallbackRadius;
    r_map[gi] = fminf(fmaxf(expf(o[kCnnClasses]), kRMin), kRMax);
}

// Loss of the latest frame against a target disparity map and its gradient
// with respect to the output (bfloat16, 16 channels, zero where not
// trained).  Pixels of class 0 (predicted, not reset) are trained: the label
// is the smallest radius covering |round(target) - round(d_pred)| (centres
// clamped to [0, D - 1]), else the widest; the loss is cross-entropy plus
// 0.1 * 0.5 (e^2 exp(-s) + s), e = target - d_pred, s = log r, averaged over
// all pixels.
__global__ void __launch_bounds__(256) k_loss(const float *__restrict__ out, const float *__restrict__ d_pred,
                                              const uint8_t *__restrict__ cls, const float *__restrict__ d_target,
                                              Geometry g, float inv_npix, uint4 *__restrict__ grad,
                                              float *__restrict__ loss_sum)
{
    const long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float lv = 0.0f;
    if (gi < g.NPIX) {
        float gz[kCnnOutPad] = {0};
        if (cls[gi] == 0) {
            const float *o = out + gi * kCnnOutPad;
            const float dp = d_pred[gi], dt = d_target[gi];
            const float cf = fminf(fmaxf(floorf(__fadd_rn(dp, 0.5f)), 0.0f), (float)(g.D - 1));
            const float tf = fminf(fmaxf(floorf(__fadd_rn(dt, 0.5f)), 0.0f), (float)(g.D - 1));
            const float dist = fabsf(tf - cf);
            int lab = kCnnClasses - 1;
            for (int k = kCnnClasses - 1; k >= 0; --k)
                if (dist <= (float)kRadii[k]) lab = k;
            float zmax = o[0];
            for (int i = 1; i < kCnnClasses; ++i) zmax = fmaxf(zmax, o[i]);
            float e[kCnnClasses], sum = 0.0f;
            for (int i = 0; i < kCnnClasses; ++i) {
                e[i] = expf(o[i] - zmax);
                sum += e[i];
            }
            const float ce = zmax + logf(sum) - o[lab];
            const float err = dt - dp, s = o[kCnnClasses];
            const float es = err * err * expf(-s);
            lv = ce + kNllWeight * 0.5f * (es + s);
            for (int i = 0; i < kCnnClasses; ++i) gz[i] = (e[i] / sum - (i == lab ? 1.0f : 0.0f)) * inv_npix;
            gz[kCnnClasses] = kNllWeight * 0.5f * (1.0f - es) * inv_npix;
        }
        grad[2 * gi] = make_uint4(pack_bf16x2(gz[0], gz[1]), pack_bf16x2(gz[2], gz[3]), pack_bf16x2(gz[4], gz[5]),
                                  pack_bf16x2(gz[6], gz[7]));
        grad[2 * gi + 1] = make_uint4(0u, 0u, 0u, 0u);
    }
    for (int o = 16; o > 0; o >>= 1) lv += __shfl_down_sync(0xffffffffu, lv, o);
    if ((threadIdx.x & 31) == 0 && lv != 0.0f) atomicAdd(loss_sum, lv * inv_npix);
}

// Weight (and bias) gradient of one layer: dW[o][i][tap] = sum_p g[p][o]
// x[p + tap][i], db[o] = sum_p g[p][o], over 32-pixel row tiles staged in
// shared memory (fp32); a block accumulates its tiles in registers and adds
// its totals to the fp32 gradient once.  The gradient of a layer's weights
// is followed by that of its bias in the parameter vector, so output index
// o < cout * cin * 9 + cout addresses both.
constexpr int kWgTile = 32;
constexpr int kWgThreads = 256;
constexpr int kWgPer = (32 * 32 * 9 + 32 + kWgThreads - 1) / kWgThreads;

template <int CINP, int GP>
__global__ void __launch_bounds__(kWgThreads) k_wgrad(const __nv_bfloat16 *__restrict__ x,
                                                      const __nv_bfloat16 *__restrict__ gsrc, Geometry g,
                                                      int cin, int cout, int tiles_x, float *__restrict__ dW)
{
    __shared__ float xs[3][kWgTile + 2][CINP];
    __shared__ float gs[kWgTile][GP];
    const int no = cout * cin * 9;
    float acc[kWgPer];
#pragma unroll
    for (int i = 0; i < kWgPer; ++i) acc[i] = 0.0f;
    const long long ntiles = (long long)g.B * g.H * tiles_x;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long row = tile / tiles_x;
        const int x0 = (int)(tile - row * tiles_x) * kWgTile;
        const int y = (int)(row % g.H);
        const long long rbase = row * g.W;
        __syncthreads();
        for (int idx = threadIdx.x; idx < 3 * (kWgTile + 2) * CINP; idx += kWgThreads) {
            const int r = idx / ((kWgTile + 2) * CINP);
            const int rem = idx - r * (kWgTile + 2) * CINP;
            const int px = rem / CINP, ch = rem - px * CINP;
            const int yy = y + r - 1, xx = x0 + px - 1;
            float v = 0.0f;
            if (yy >= 0 && yy < g.H && xx >= 0 && xx < g.W)
                v = __bfloat162float(x[(rbase + (long long)(r - 1) * g.W + xx) * CINP + ch]);
            xs[r][px][ch] = v;
        }
        for (int idx = threadIdx.x; idx < kWgTile * GP; idx += kWgThreads) {
            const int px = idx / GP, ch = idx - px * GP;
            gs[px][ch] = x0 + px < g.W ? __bfloat162float(gsrc[(rbase + x0 + px) * GP + ch]) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kWgPer; ++i) {
            const int o = threadIdx.x + i * kWgThreads;
            float s = 0.0f;
            if (o < no) {
                const int co = o / (cin * 9), rem = o - co * cin * 9;
                const int ci = rem / 9, tap = rem - ci * 9;
                const int ky = tap / 3, kx = tap - ky * 3;
                for (int px = 0; px < kWgTile; ++px) s += gs[px][co] * xs[ky][px + kx][ci];
            } else if (o < no + cout) {
                const int co = o - no;
                for (int px = 0; px < kWgTile; ++px) s += gs[px][co];
            }
            acc[i] += s;
        }
    }
#pragma unroll
    for (int i = 0; i < kWgPer; ++i) {
        const int o = threadIdx.x + i * kWgThreads;
        if (o < no + cout && acc[i] != 0.0f) atomicAdd(dW + o, acc[i]);
    }
}

__global__ void __launch_bounds__(256) k_adam(float *__restrict__ theta, float *__restrict__ m, float *__restrict__ v,
                                              const float *__restrict__ grad, int n, float lr, float b1, float b2,
                                              float eps, float bc1, float bc2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gv = grad[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gv;
    const float vi = b2 * v[i] + (1.0f - b2) * gv * gv;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// Device layouts of one layer's parameters: the forward weights [9][COUTP][CINP]
// (bfloat16), the input-gradient weights [9][cin][KP] flipped and transposed
// (KP = the layer's gradient channels), and the bias padded to COUTP.
__global__ void __launch_bounds__(256) k_pack(const float *__restrict__ W, const float *__restrict__ b, int cin,
                                              int cout, int cinp, int coutp, int kp, __nv_bfloat16 *__restrict__ wf,
                                              __nv_bfloat16 *__restrict__ wb, float *__restrict__ bias_p)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int nf = 9 * coutp * cinp;
    if (idx < nf) {
        const int tap = idx / (coutp * cinp), n = (idx / cinp) % coutp, k = idx % cinp;
        wf[idx] = __float2bfloat16_rn(n < cout && k < cin ? W[(n * cin + k) * 9 + tap] : 0.0f);
    }
    if (wb && idx < 9 * cin * kp) {
        const int tap = idx / (cin * kp), n = (idx / kp) % cin, k = idx % kp;
        wb[idx] = __float2bfloat16_rn(k < cout ? W[(k * cin + n) * 9 + (8 - tap)] : 0.0f);
    }
    if (idx < coutp) bias_p[idx] = idx < cout ? b[idx] : 0.0f;
}

unsigned blocks_of(long long n, int per) { return (unsigned)((n + per - 1) / per); }

template <int CINP, int COUTP, int MODE>
cudaError_t conv(const void *in, const void *wt, const float *bias, const void *mask, void *out, const Geometry &g,
                 cudaStream_t st)
{
    const int blocks_x = (g.W + kConvPix - 1) / kConvPix;
    k_conv<CINP, COUTP, MODE><<<(unsigned)((long long)g.B * g.H * blocks_x), kConvWarps * 32, 0, st>>>(
        (const uint32_t *)in, (const uint32_t *)wt, bias, (const __nv_bfloat16 *)mask, out, g, blocks_x);
    return cudaGetLastError();
}

template <int CINP, int GP>
cudaError_t wgrad(const void *x, const void *gsrc, const Geometry &g, int cin, int cout, float *dW, int sm_count,
                  cudaStream_t st)
{
    const int tiles_x = (g.W + kWgTile - 1) / kWgTile;
    const long long ntiles = (long long)g.B * g.H * tiles_x;
    const long long cap = (long long)(sm_count > 0 ? sm_count : 152) * 4;
    k_wgrad<CINP, GP><<<(unsigned)(ntiles < cap ? ntiles : cap), kWgThreads, 0, st>>>(
        (const __nv_bfloat16 *)x, (const __nv_bfloat16 *)gsrc, g, cin, cout, tiles_x, dW);
    return cudaGetLastError();
}

#define RSGM_TRY(call)                       \
    do {                                     \
        cudaError_t e_ = (call);             \
        if (e_ != cudaSuccess) return e_;    \
    } while (0)

}  // namespace

const int kCnnIn[kCnnLayers] = {4, 32, 32, 32};
const int kCnnOut[kCnnLayers] = {32, 32, 32, kCnnClasses + 1};

long long cnn_param_offset(int layer)
{
    long long off = 0;
    for (int l = 0; l < layer; ++l) off += (long long)kCnnOut[l] * kCnnIn[l] * 9 + kCnnOut[l];
    return off;
}

cudaError_t cnn_pack(const CnnWeights &w, cudaStream_t st)
{
    for (int l = 0; l < kCnnLayers; ++l) {
        const float *W = w.theta + cnn_param_offset(l);
        const float *b = W + (long long)kCnnOut[l] * kCnnIn[l] * 9;
        const int cinp = l == 0 ? 16 : 32, coutp = l == kCnnLayers - 1 ? kCnnOutPad : 32;
        const int kp = l == kCnnLayers - 1 ? 16 : 32;  // channels of the gradient entering this layer
        const int n = 9 * 32 * 32;
        k_pack<<<blocks_of(n, 256), 256, 0, st>>>(W, b, kCnnIn[l], kCnnOut[l], cinp, coutp, kp,
                                                  (__nv_bfloat16 *)w.wf[l],
                                                  l > 0 ? (__nv_bfloat16 *)w.wb[l] : nullptr, w.bias[l]);
        RSGM_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}

namespace {
// The four layers from the stored inputs.
cudaError_t cnn_layers(const CnnWeights &w, const LearnedBuffers &lb, const Geometry &g, cudaStream_t st)
{
    RSGM_TRY((conv<16, 32, kReluBf16>(lb.feats, w.wf[0], w.bias[0], nullptr, lb.act[0], g, st)));
    RSGM_TRY((conv<32, 32, kReluBf16>(lb.act[0], w.wf[1], w.bias[1], nullptr, lb.act[1], g, st)));
    RSGM_TRY((conv<32, 32, kReluBf16>(lb.act[1], w.wf[2], w.bias[2], nullptr, lb.act[2], g, st)));
    RSGM_TRY((conv<32, kCnnOutPad, kLinearF32>(lb.act[2], w.wf[3], w.bias[3], nullptr, lb.out, g, st)));
    return cudaSuccess;
}
}  // namespace

cudaError_t cnn_forward(const CnnWeights &w, const LearnedBuffers &lb, const Buffers &b, const Geometry &g,
                        const uint8_t *left, int nbits, cudaStream_t st)
{
    k_features<<<blocks_of(g.NPIX, 256), 256, 0, st>>>(left, b.cen_l, b.cen_r, b.d_pred, b.p_pred, g, nbits,
                                                       (uint4 *)lb.feats);
    RSGM_TRY(cudaGetLastError());
    RSGM_TRY(cnn_layers(w, lb, g, st));
    k_decide<<<blocks_of(g.NPIX, 256), 256, 0, st>>>(lb.out, g, lb.radius, lb.r_map);
    return cudaGetLastError();
}

cudaError_t cnn_backward(const CnnWeights &w, const LearnedBuffers &lb, const Buffers &b, const Geometry &g,
                         const float *d_target, int sm_count, cudaStream_t st)
{
    // the layers again with the current parameters (earlier training steps
    // may have changed them since the frame ran)
    RSGM_TRY(cnn_layers(w, lb, g, st));
    RSGM_TRY(cudaMemsetAsync(w.grad, 0, (size_t)kCnnParams * sizeof(float), st));
    RSGM_TRY(cudaMemsetAsync(lb.loss, 0, sizeof(float), st));
    k_loss<<<blocks_of(g.NPIX, 256), 256, 0, st>>>(lb.out, b.d_pred, b.cls, d_target, g, 1.0f / (float)g.NPIX,
                                                   (uint4 *)lb.g16, lb.loss);
    RSGM_TRY(cudaGetLastError());
    float *dW = w.grad;
    // layer 3: input act[2] (32), gradient g16 (16 channels, 6 used)
    RSGM_TRY((wgrad<32, 16>(lb.act[2], lb.g16, g, kCnnIn[3], kCnnOut[3], dW + cnn_param_offset(3), sm_count, st)));
    RSGM_TRY((conv<16, 32, kMaskBf16>(lb.g16, w.wb[3], nullptr, lb.act[2], lb.ga, g, st)));
    // layer 2
    RSGM_TRY((wgrad<32, 32>(lb.act[1], lb.ga, g, kCnnIn[2], kCnnOut[2], dW + cnn_param_offset(2), sm_count, st)));
    RSGM_TRY((conv<32, 32, kMaskBf16>(lb.ga, w.wb[2], nullptr, lb.act[1], lb.gb, g, st)));
    // layer 1
    RSGM_TRY((wgrad<32, 32>(lb.act[0], lb.gb, g, kCnnIn[1], kCnnOut[1], dW + cnn_param_offset(1), sm_count, st)));
    RSGM_TRY((conv<32, 32, kMaskBf16>(lb.gb, w.wb[1], nullptr, lb.act[0], lb.ga, g, st)));
    // layer 0: input the features (16 channels, 4 used)
    RSGM_TRY((wgrad<16, 32>(lb.feats, lb.ga, g, kCnnIn[0], kCnnOut[0], dW + cnn_param_offset(0), sm_count, st)));
    return cudaSuccess;
}

cudaError_t cnn_adam(const CnnWeights &w, int step, float lr, cudaStream_t st)
{
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = (float)(1.0 - pow(0.9, step)), bc2 = (float)(1.0 - pow(0.999, step));
    k_adam<<<blocks_of(kCnnParams, 256), 256, 0, st>>>(w.theta, w.m, w.v, w.grad, kCnnParams, lr, b1, b2, 1e-8f,
                                                      bc1, bc2);
    RSGM_TRY(cudaGetLastError());
    return cnn_pack(w, st);
}

}  // namespace rsgm
