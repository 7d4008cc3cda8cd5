// Matching cost (Section 2.1 of the paper): census transform over a cw x ch
// window (5 x 5 in Table 1) and the Hamming cost over each pixel's own
// disparity window, written into the ragged cell volume.
#include "rsgm_internal.cuh"

namespace rsgm {
namespace {

constexpr int kTileX = 32, kTileY = 8;
constexpr int kMaxHalf = 7;  // census_w, census_h <= 15

// K2: one 32 x 8 tile of one image per block, staged in shared memory with a
// clamped halo (pixels outside the image repeat the border).  Bit k of the
// code is set iff the k-th window pixel in row-major order (centre skipped)
// is darker than the centre.  blockIdx.z = 2 * stream + side.  HW, HH > 0 fix
// the half-window at compile time (the 5 x 5 of Table 1); 0 reads hw, hh.
template <int HW, int HH>
__global__ void __launch_bounds__(kTileX *kTileY) k_census(const uint8_t *__restrict__ left,
                                                           const uint8_t *__restrict__ right,
                                                           unsigned long long *__restrict__ cen_l,
                                                           unsigned long long *__restrict__ cen_r,
                                                           Geometry g, int hw_rt, int hh_rt)
{
    __shared__ uint8_t tile[kTileY + 2 * kMaxHalf][kTileX + 2 * kMaxHalf];
    const int hw = HW > 0 ? HW : hw_rt, hh = HH > 0 ? HH : hh_rt;
    const int b = blockIdx.z >> 1, side = blockIdx.z & 1;
    const uint8_t *img = (side ? right : left) + (long long)b * g.HW;
    unsigned long long *out = (side ? cen_r : cen_l) + (long long)b * g.HW;
    const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * kTileY;
    const int tw = kTileX + 2 * hw, th = kTileY + 2 * hh;
    for (int ty = threadIdx.y; ty < th; ty += kTileY) {
        const int gy = min(max(y0 - hh + ty, 0), g.H - 1);
        const uint8_t *row = img + (long long)gy * g.W;
        for (int tx = threadIdx.x; tx < tw; tx += kTileX) tile[ty][tx] = row[min(max(x0 - hw + tx, 0), g.W - 1)];
    }
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= g.W || y >= g.H) return;
    const int cx = threadIdx.x + hw, cy = threadIdx.y + hh;
    const uint8_t c = tile[cy][cx];
    unsigned long long code = 0;
    int bit = 0;
#pragma unroll
    for (int dy = -(HH > 0 ? HH : kMaxHalf); dy <= (HH > 0 ? HH : kMaxHalf); ++dy) {
        if (HH == 0 && (dy < -hh || dy > hh)) continue;
#pragma unroll
        for (int dx = -(HW > 0 ? HW : kMaxHalf); dx <= (HW > 0 ? HW : kMaxHalf); ++dx) {
            if (HW == 0 && (dx < -hw || dx > hw)) continue;
            if (dx == 0 && dy == 0) continue;
            if (tile[cy + dy][cx + dx] < c) code |= 1ull << bit;
            ++bit;
        }
    }
    out[(long long)y * g.W + x] = code;
}

constexpr int kCostWarps = 4;
constexpr int kLaneCells = 16;  // windows up to this width are filled by their own lane

// K3: one warp per 32 consecutive pixels.  Each lane finalises one pixel's
// metadata (first cell = row base + in-row prefix, window) and writes its
// window's costs C(p, d) = popcount(cL(x,y) ^ cR(x-d,y)), a match left of the
// image costing every census bit.  A window starts on a 4-cell boundary and
// is written as whole 32-bit words, the padding cells past its width holding
// 0xFF.  Narrow windows (up to kLaneCells cells) are filled by their own lane
// (neighbouring lanes read overlapping right census words, which the L1
// serves); wider ones by the whole warp, one pixel at a time, one word per
// lane per pass.
__device__ __forceinline__ unsigned cost_byte(unsigned long long cl, const unsigned long long *cr, int xr, int k,
                                              int w, int nbits)
{
    if (k >= w) return 0xFFu;
    return (unsigned)(xr >= 0 ? __popcll(cl ^ cr[xr]) : nbits);
}

__global__ void __launch_bounds__(kCostWarps * 32) k_cost(const unsigned long long *__restrict__ cen_l,
                                                         const unsigned long long *__restrict__ cen_r,
                                                         const uint32_t *__restrict__ win,
                                                         const uint32_t *__restrict__ inrow,
                                                         const uint32_t *__restrict__ row_base,
                                                         uint2 *__restrict__ meta, uint8_t *__restrict__ cost,
                                                         Geometry g, int nbits)
{
    const int lane = threadIdx.x & 31;
    const long long gi0 = ((long long)blockIdx.x * kCostWarps + (threadIdx.x >> 5)) * 32;
    if (gi0 >= g.NPIX) return;  // uniform per warp
    const long long gi = gi0 + lane;
    const bool valid = gi < g.NPIX;
    unsigned o = 0, wv = 0;
    int x = 0;
    long long row = 0;
    unsigned long long cl = 0;
    if (valid) {
        row = gi / g.W;
        x = (int)(gi - row * g.W);
        o = row_base[row] + inrow[gi];
        wv = win[gi];
        meta[gi] = make_uint2(o, wv);
        cl = cen_l[gi];
    }
    const int lo = (int)(wv & 0xFFFFu), w = (int)(wv >> 16);
    const unsigned long long *cr = cen_r + row * g.W;
    if (valid && w <= kLaneCells) {
        unsigned *dst = (unsigned *)(cost + o);
        for (int k0 = 0; k0 < w; k0 += 4) {
            const int xr = x - lo - k0;
            dst[k0 >> 2] = cost_byte(cl, cr, xr, k0, w, nbits) | (cost_byte(cl, cr, xr - 1, k0 + 1, w, nbits) << 8) |
                           (cost_byte(cl, cr, xr - 2, k0 + 2, w, nbits) << 16) |
                           (cost_byte(cl, cr, xr - 3, k0 + 3, w, nbits) << 24);
        }
    }
    unsigned wide = __ballot_sync(0xffffffffu, valid && w > kLaneCells);
    while (wide) {
        const int src = __ffs(wide) - 1;
        wide &= wide - 1;
        const unsigned o2 = __shfl_sync(0xffffffffu, o, src);
        const int w2 = __shfl_sync(0xffffffffu, w, src);
        const int xl = __shfl_sync(0xffffffffu, x - lo, src);  // right-image column of the window's first cell
        const long long r2 = __shfl_sync(0xffffffffu, row, src);
        const unsigned long long cl2 = __shfl_sync(0xffffffffu, cl, src);
        const unsigned long long *cr2 = cen_r + r2 * g.W;
        unsigned *dst = (unsigned *)(cost + o2);
        for (int k0 = 4 * lane; k0 < w2; k0 += 128) {
            const int xr = xl - k0;
            dst[k0 >> 2] = cost_byte(cl2, cr2, xr, k0, w2, nbits) | (cost_byte(cl2, cr2, xr - 1, k0 + 1, w2, nbits) << 8) |
                           (cost_byte(cl2, cr2, xr - 2, k0 + 2, w2, nbits) << 16) |
                           (cost_byte(cl2, cr2, xr - 3, k0 + 3, w2, nbits) << 24);
        }
    }
}

}  // namespace

cudaError_t launch_census(const Buffers &b, const Geometry &g, const uint8_t *left,
                          const uint8_t *right, int cw, int ch, cudaStream_t st)
{
    dim3 grid((g.W + kTileX - 1) / kTileX, (g.H + kTileY - 1) / kTileY, 2 * g.B);
    if (cw == 5 && ch == 5)
        k_census<2, 2><<<grid, dim3(kTileX, kTileY), 0, st>>>(left, right, b.cen_l, b.cen_r, g, 2, 2);
    else
        k_census<0, 0><<<grid, dim3(kTileX, kTileY), 0, st>>>(left, right, b.cen_l, b.cen_r, g, cw / 2, ch / 2);
    return cudaGetLastError();
}

cudaError_t launch_cost(const Buffers &b, const Geometry &g, int nbits, cudaStream_t st)
{
    const long long warps = (g.NPIX + 31) / 32;
    const unsigned blocks = (unsigned)((warps + kCostWarps - 1) / kCostWarps);
    k_cost<<<blocks, kCostWarps * 32, 0, st>>>(b.cen_l, b.cen_r, b.win, b.inrow, b.row_base, b.meta, b.cost, g, nbits);
    return cudaGetLastError();
}

}  // namespace rsgm
