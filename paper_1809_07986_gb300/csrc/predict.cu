// Prediction step of the per-pixel Kalman filter (Section 2.4 of the paper):
// forward splat of the previous state through the ego-motion (Eqs. 2-4),
// zoom-hole filling, discontinuity reset, the per-pixel search window and the
// exclusive prefix sum that lays the windows out as a ragged cell volume.
//
// Floating-point values here decide integers (target pixel, window), so every
// operation is an explicit round-to-nearest intrinsic in a fixed order; the
// library is built with -fmad=false as a second guard against contraction.
#include "rsgm_internal.cuh"

namespace rsgm {
namespace {

constexpr unsigned kEmpty = 0u;  // key value of a pixel no point landed on

__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }

// K1: every pixel with d > 0.5 is back-projected (Z = fx b / d), moved with
// X' = R X + t and projected again (Eq. 2 in metric form).  The 64-bit key is
// (bits of d' << 32) | (~source index): d' > 0, so positive-float bit patterns
// order like the values and atomicMax keeps the nearest surface, breaking ties
// toward the smaller source index.
__global__ void __launch_bounds__(256) k_splat(const float *__restrict__ d,
                                               unsigned long long *__restrict__ key,
                                               const __grid_constant__ SplatArgs a)
{
    long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= a.g.NPIX) return;
    int b = (int)(gi / a.g.HW);
    int s = (int)(gi - (long long)b * a.g.HW);
    int y = s / a.g.W, x = s - y * a.g.W;
    if (a.role[b] != RSGM_SLOT_REDUCED) return;  // idle streams and new streams predict nothing
    float ds = d[gi];
    if (!(ds > 0.5f)) return;
    const Motion &m = a.m[b];
    float Z = fdiv(a.fb, ds);
    float X = fdiv(fmul(fsub((float)x, a.cx), Z), a.fx);
    float Y = fdiv(fmul(fsub((float)y, a.cy), Z), a.fy);
    float Xn = fadd(fadd(fadd(fmul(m.R[0], X), fmul(m.R[1], Y)), fmul(m.R[2], Z)), m.t[0]);
    float Yn = fadd(fadd(fadd(fmul(m.R[3], X), fmul(m.R[4], Y)), fmul(m.R[5], Z)), m.t[1]);
    float Zn = fadd(fadd(fadd(fmul(m.R[6], X), fmul(m.R[7], Y)), fmul(m.R[8], Z)), m.t[2]);
    if (!(Zn > 0.0f)) return;
    float xn = fadd(fdiv(fmul(a.fx, Xn), Zn), a.cx);
    float yn = fadd(fdiv(fmul(a.fy, Yn), Zn), a.cy);
    float dn = fdiv(a.fb, Zn);
    if (!isfinite(dn)) return;
    float xi = floorf(fadd(xn, 0.5f)), yi = floorf(fadd(yn, 0.5f));
    if (!(xi >= 0.0f && xi <= (float)(a.g.W - 1) && yi >= 0.0f && yi <= (float)(a.g.H - 1)))
        return;
    long long tgt = (long long)b * a.g.HW + (long long)((int)yi * a.g.W + (int)xi);
    unsigned long long k = ((unsigned long long)__float_as_uint(dn) << 32) |
                           (unsigned long long)(0xFFFFFFFFu - (unsigned)s);
    atomicMax(key + tgt, k);
}

// Eq. 3-4 for the splat encoded in key k (k != kEmpty) of a stream at `base`.
__device__ __forceinline__ void winner(unsigned long long k, const float *__restrict__ d,
                                       const float *__restrict__ p, long long base, float q, float &dd,
                                       float &pp)
{
    float dn = __uint_as_float((unsigned)(k >> 32));
    unsigned src = 0xFFFFFFFFu - (unsigned)(k & 0xFFFFFFFFull);
    float ds = d[base + src], ps = p[base + src];
    float phi = fdiv(dn, ds);                        // Eq. 3
    pp = fadd(fmul(fmul(phi, phi), ps), q);          // Eq. 4
    dd = dn;
}

// K1b: prediction per target pixel, with zoom holes (no point landed) filled
// from two known horizontal or two known vertical neighbours (both pairs:
// average of four).  Unknown pixels get d_pred = -1.  The pixel's and its
// four neighbours' keys are fetched together, then the sources they name, so
// that a hole costs two dependent fetches rather than up to ten.
__global__ void __launch_bounds__(256) k_gather_fill(const unsigned long long *__restrict__ key,
                                                     const float *__restrict__ d,
                                                     const float *__restrict__ p,
                                                     float *__restrict__ d_pred,
                                                     float *__restrict__ p_pred, Geometry g, float q)
{
    long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= g.NPIX) return;
    int b = (int)(gi / g.HW);
    long long base = (long long)b * g.HW;
    int s = (int)(gi - base);
    int y = s / g.W, x = s - y * g.W;
    const unsigned long long k0 = key[gi];
    const bool hx = x > 0 && x < g.W - 1, hy = y > 0 && y < g.H - 1;
    unsigned long long kl = kEmpty, kr = kEmpty, ku = kEmpty, kd = kEmpty;
    if (k0 == kEmpty) {
        if (hx) {
            kl = key[gi - 1];
            kr = key[gi + 1];
        }
        if (hy) {
            ku = key[gi - g.W];
            kd = key[gi + g.W];
        }
    }
    float dd, pp;
    if (k0 != kEmpty) {
        winner(k0, d, p, base, q, dd, pp);
        d_pred[gi] = dd;
        p_pred[gi] = pp;
        return;
    }
    float dl = 0, pl = 0, dr = 0, pr = 0, du = 0, pu = 0, dw = 0, pw = 0;
    const bool h = kl != kEmpty && kr != kEmpty;
    const bool v = ku != kEmpty && kd != kEmpty;
    if (h) {
        winner(kl, d, p, base, q, dl, pl);
        winner(kr, d, p, base, q, dr, pr);
    }
    if (v) {
        winner(ku, d, p, base, q, du, pu);
        winner(kd, d, p, base, q, dw, pw);
    }
    if (h && v) {
        d_pred[gi] = fmul(fadd(fadd(dl, dr), fadd(du, dw)), 0.25f);
        p_pred[gi] = fmul(fadd(fadd(pl, pr), fadd(pu, pw)), 0.25f);
    } else if (h) {
        d_pred[gi] = fmul(fadd(dl, dr), 0.5f);
        p_pred[gi] = fmul(fadd(pl, pr), 0.5f);
    } else if (v) {
        d_pred[gi] = fmul(fadd(du, dw), 0.5f);
        p_pred[gi] = fmul(fadd(pu, pw), 0.5f);
    } else {
        d_pred[gi] = -1.0f;
        p_pred[gi] = 0.0f;
    }
}

// Block-wide exclusive scan of one value per thread (blockDim.x = 256, 8 warps);
// the block total is written to `total` (shared).
__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned &total)
{
    __shared__ unsigned warp_pre[8];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned n = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += n;
    }
    if (lane == 31) warp_pre[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        unsigned w = lane < 8 ? warp_pre[lane] : 0u;
        unsigned wi = w;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            unsigned n = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += n;
        }
        unsigned tot = __shfl_sync(0xffffffffu, wi, 7);
        if (lane < 8) warp_pre[lane] = wi - w;
        if (lane == 0) total = tot;
    }
    __syncthreads();
    unsigned res = warp_pre[wid] + incl - v;
    __syncthreads();
    return res;
}

constexpr int kWinPer = 4;           // pixels per thread and tile for the in-row scan
constexpr int kWinTile = 256 * kWinPer;

// K1c: one block per image row, walking the row in tiles of kWinTile pixels.
// A tile's predicted disparities and those of the rows above and below
// (with a one-pixel halo; -1, "unknown", outside the image) are staged in
// shared memory with coalesced loads.  Then per pixel: discontinuity reset (a
// known pixel with a known 4-neighbour more than tau_disc away keeps d but
// takes p_reset and the full window), the search window, and the splat key
// cleared for the next frame; then the in-row exclusive prefix sum of the
// widths (carried across tiles) and the row total.
__global__ void __launch_bounds__(256) k_window(const float *__restrict__ d_pred, float *__restrict__ p_pred,
                                                uint32_t *__restrict__ win, uint8_t *__restrict__ cls,
                                                uint32_t *__restrict__ inrow,
                                                uint32_t *__restrict__ row_total,
                                                uint32_t *__restrict__ row_cells,
                                                unsigned long long *__restrict__ key,
                                                const uint8_t *__restrict__ radius_map, Geometry g,
                                                FrameParams fp)
{
    __shared__ float sd[3][kWinTile + 2];  // rows y-1, y, y+1; column x0 - 1 + i at index i
    __shared__ unsigned sw[kWinTile];
    __shared__ unsigned total;
    const int row = blockIdx.x;  // b * H + y
    const int y = row % g.H;
    const uint8_t role = fp.role[row / g.H];
    const long long rbase = (long long)row * g.W;
    unsigned carry = 0, cells = 0;
    for (int x0 = 0; x0 < g.W; x0 += kWinTile) {
        const int n = min(kWinTile, g.W - x0);
        for (int i = threadIdx.x; i < n + 2; i += blockDim.x) {
            const int x = x0 - 1 + i;
            const bool in = x >= 0 && x < g.W;
            sd[0][i] = in && y > 0 ? d_pred[rbase - g.W + x] : -1.0f;
            sd[1][i] = in ? d_pred[rbase + x] : -1.0f;
            sd[2][i] = in && y < g.H - 1 ? d_pred[rbase + g.W + x] : -1.0f;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const long long gi = rbase + x0 + i;
            const float dc = sd[1][i + 1];
            int lo = 0, w = g.D;
            uint8_t c = 2;
            if (role == RSGM_SLOT_IDLE) {
                // an idle stream searches nothing and keeps its state
                w = 0;
                c = 3;
            } else if (role == RSGM_SLOT_FULL) {
                // a new stream's first frame: the whole range, no prediction
            } else if (dc >= 0.0f) {
                const float nb[4] = {sd[1][i], sd[1][i + 2], sd[0][i + 1], sd[2][i + 1]};
                bool reset = false;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (nb[k] >= 0.0f && fabsf(fsub(nb[k], dc)) > fp.tau_disc) reset = true;
                if (reset) {
                    c = 1;
                    p_pred[gi] = fp.p_reset;
                } else {
                    c = 0;
                    if (fp.radius_mode != RSGM_RADIUS_FULL) {
                        int h;
                        if (fp.radius_mode == RSGM_RADIUS_VARIANCE) {
                            float cp = ceilf(p_pred[gi]);
                            h = cp < 1.0f ? 1 : (cp > (float)g.D ? g.D : (int)cp);
                        } else if (fp.radius_mode == RSGM_RADIUS_LEARNED) {
                            h = radius_map[gi];
                        } else {
                            h = fp.radius;
                        }
                        float cf = floorf(fadd(dc, 0.5f));
                        int cc = cf < 0.0f ? 0 : (cf > (float)(g.D - 1) ? g.D - 1 : (int)cf);
                        lo = max(0, cc - h);
                        int hi = min(g.D - 1, cc + h);
                        w = hi - lo + 1;
                    }
                }
            }
            win[gi] = (uint32_t)lo | ((uint32_t)w << 16);
            cls[gi] = c;
            key[gi] = 0ull;
            sw[i] = (unsigned)round4(w);  // cells are laid out in 4-aligned runs
            cells += (unsigned)w;
        }
        __syncthreads();
        const int j0 = threadIdx.x * kWinPer, j1 = min(j0 + kWinPer, n);
        unsigned local = 0;
        for (int j = j0; j < j1; ++j) local += sw[j];
        unsigned pre = block_exclusive_scan(local, total) + carry;
        for (int j = j0; j < j1; ++j) {
            const unsigned wv = sw[j];
            sw[j] = pre;
            pre += wv;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) inrow[rbase + x0 + i] = sw[i];
        carry += total;
        __syncthreads();  // the next tile reuses sd, sw and total
    }
    block_exclusive_scan(cells, total);
    if (threadIdx.x == 0) {
        row_total[row] = carry;
        row_cells[row] = total;
    }
}

// Initial frame: every pixel searches [0, D) and has no prediction.
__global__ void __launch_bounds__(256) k_full_window(uint32_t *__restrict__ win, uint8_t *__restrict__ cls,
                                                     uint32_t *__restrict__ inrow,
                                                     uint32_t *__restrict__ row_total,
                                                     uint32_t *__restrict__ row_cells, Geometry g)
{
    long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= g.NPIX) return;
    int x = (int)(gi % g.W);
    win[gi] = (uint32_t)g.D << 16;
    cls[gi] = 2;
    inrow[gi] = (uint32_t)x * (uint32_t)round4(g.D);
    if (x == 0) {
        row_total[gi / g.W] = (uint32_t)g.W * (uint32_t)round4(g.D);
        row_cells[gi / g.W] = (uint32_t)g.W * (uint32_t)g.D;
    }
}

// Exclusive scan of the B*H rounded row totals in one block (the first cell
// of every row); records the frame's cell count in the counters.
__global__ void __launch_bounds__(256) k_row_scan(const uint32_t *__restrict__ row_total,
                                                  const uint32_t *__restrict__ row_cells,
                                                  uint32_t *__restrict__ row_base, int nrows,
                                                  int nstreams,
                                                  unsigned long long *__restrict__ counters)
{
    __shared__ unsigned total;
    int chunk = (nrows + blockDim.x - 1) / blockDim.x;
    int r0 = threadIdx.x * chunk, r1 = min(nrows, r0 + chunk);
    unsigned local = 0, real = 0;
    for (int r = r0; r < r1; ++r) {
        local += row_total[r];
        real += row_cells[r];
    }
    unsigned pre = block_exclusive_scan(local, total);
    const unsigned rounded = total;
    for (int r = r0; r < r1; ++r) {
        row_base[r] = pre;
        pre += row_total[r];
    }
    block_exclusive_scan(real, total);
    if (threadIdx.x == 0) {
        counters[0] += (unsigned long long)nstreams;
        counters[1] += total;
        counters[2] = total;
        counters[3] = rounded;
    }
}

unsigned blocks_for(long long n, int per) { return (unsigned)((n + per - 1) / per); }

}  // namespace

cudaError_t launch_splat(const Buffers &b, const SplatArgs &a, cudaStream_t st)
{
    k_splat<<<blocks_for(a.g.NPIX, 256), 256, 0, st>>>(b.d, b.key, a);
    return cudaGetLastError();
}

cudaError_t launch_gather_fill(const Buffers &b, const Geometry &g, float q, cudaStream_t st)
{
    k_gather_fill<<<blocks_for(g.NPIX, 256), 256, 0, st>>>(b.key, b.d, b.p, b.d_pred, b.p_pred, g, q);
    return cudaGetLastError();
}

cudaError_t launch_window(const Buffers &b, const Geometry &g, const FrameParams &fp, cudaStream_t st)
{
    if (fp.radius_mode == RSGM_RADIUS_LEARNED && !b.radius) return cudaErrorInvalidValue;
    k_window<<<(unsigned)(g.B * g.H), 256, 0, st>>>(b.d_pred, b.p_pred, b.win, b.cls, b.inrow,
                                                     b.row_total, b.row_cells, b.key, b.radius, g, fp);
    return cudaGetLastError();
}

cudaError_t launch_full_window(const Buffers &b, const Geometry &g, cudaStream_t st)
{
    k_full_window<<<blocks_for(g.NPIX, 256), 256, 0, st>>>(b.win, b.cls, b.inrow, b.row_total, b.row_cells, g);
    return cudaGetLastError();
}

cudaError_t launch_row_scan(const Buffers &b, const Geometry &g, int nstreams, cudaStream_t st)
{
    k_row_scan<<<1, 256, 0, st>>>(b.row_total, b.row_cells, b.row_base, g.B * g.H, nstreams, b.counters);
    return cudaGetLastError();
}

}  // namespace rsgm
