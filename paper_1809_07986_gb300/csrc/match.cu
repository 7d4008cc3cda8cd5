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
// is darker than the centre.  blockIdx.z = 2 * stream + side.
__global__ void __launch_bounds__(kTileX *kTileY) k_census(const uint8_t *__restrict__ left,
                                                           const uint8_t *__restrict__ right,
                                                           unsigned long long *__restrict__ cen_l,
                                                           unsigned long long *__restrict__ cen_r,
                                                           Geometry g, int hw, int hh)
{
    __shared__ uint8_t tile[kTileY + 2 * kMaxHalf][kTileX + 2 * kMaxHalf];
    int b = blockIdx.z >> 1, side = blockIdx.z & 1;
    const uint8_t *img = (side ? right : left) + (long long)b * g.HW;
    unsigned long long *out = (side ? cen_r : cen_l) + (long long)b * g.HW;
    int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * kTileY;
    int tw = kTileX + 2 * hw, th = kTileY + 2 * hh;
    int tid = threadIdx.y * kTileX + threadIdx.x;
    for (int i = tid; i < tw * th; i += kTileX * kTileY) {
        int ty = i / tw, tx = i - ty * tw;
        int gx = min(max(x0 - hw + tx, 0), g.W - 1);
        int gy = min(max(y0 - hh + ty, 0), g.H - 1);
        tile[ty][tx] = img[(long long)gy * g.W + gx];
    }
    __syncthreads();
    int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= g.W || y >= g.H) return;
    int cx = threadIdx.x + hw, cy = threadIdx.y + hh;
    uint8_t c = tile[cy][cx];
    unsigned long long code = 0;
    int bit = 0;
    for (int dy = -hh; dy <= hh; ++dy) {
        for (int dx = -hw; dx <= hw; ++dx) {
            if (dx == 0 && dy == 0) continue;
            if (tile[cy + dy][cx + dx] < c) code |= 1ull << bit;
            ++bit;
        }
    }
    out[(long long)y * g.W + x] = code;
}

// K3: one thread per pixel.  Finalises the pixel's metadata (first cell =
// row base + in-row prefix, window) and writes C(p, d) = popcount(cL(x,y) ^ cR(x-d,y)) for its
// window; a match left of the image costs every census bit.
__global__ void __launch_bounds__(256) k_cost(const unsigned long long *__restrict__ cen_l,
                                              const unsigned long long *__restrict__ cen_r,
                                              const uint32_t *__restrict__ win,
                                              const uint32_t *__restrict__ inrow,
                                              const uint32_t *__restrict__ row_base,
                                              uint2 *__restrict__ meta, uint8_t *__restrict__ cost,
                                              Geometry g, int nbits)
{
    long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= g.NPIX) return;
    long long row = gi / g.W;
    int x = (int)(gi - row * g.W);
    uint32_t o = row_base[row] + inrow[gi];
    uint32_t wv = win[gi];
    meta[gi] = make_uint2(o, wv);
    int lo = (int)(wv & 0xFFFFu), w = (int)(wv >> 16);
    unsigned long long cl = cen_l[gi];
    const unsigned long long *rr = cen_r + row * g.W;
    for (int k = 0; k < w; ++k) {
        int xr = x - (lo + k);
        cost[o + k] = (uint8_t)(xr >= 0 ? __popcll(cl ^ rr[xr]) : nbits);
    }
}

}  // namespace

cudaError_t launch_census(const Buffers &b, const Geometry &g, const uint8_t *left,
                          const uint8_t *right, int cw, int ch, cudaStream_t st)
{
    dim3 grid((g.W + kTileX - 1) / kTileX, (g.H + kTileY - 1) / kTileY, 2 * g.B);
    k_census<<<grid, dim3(kTileX, kTileY), 0, st>>>(left, right, b.cen_l, b.cen_r, g, cw / 2, ch / 2);
    return cudaGetLastError();
}

cudaError_t launch_cost(const Buffers &b, const Geometry &g, int nbits, cudaStream_t st)
{
    unsigned blocks = (unsigned)((g.NPIX + 255) / 256);
    k_cost<<<blocks, 256, 0, st>>>(b.cen_l, b.cen_r, b.win, b.inrow, b.row_base, b.meta, b.cost, g, nbits);
    return cudaGetLastError();
}

}  // namespace rsgm
