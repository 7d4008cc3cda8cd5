// Cost aggregation, Eq. 1 (Section 2.2 of the paper), over the ragged cell
// volume: for path direction r the predecessor of p is p - r and
//   L_r(p,d) = C(p,d) + min(L_r(p-r,d), L_r(p-r,d+-1) + P1, m + P2) - m,
//   m = min_k L_r(p-r,k) over the predecessor's window,
// with L_r(p-r, .) = +inf outside that window and L_r = C at the first pixel
// of a path.  S(p,d) is the sum of L_r over the enabled directions.
//
// One warp walks one path line; the cells of the current pixel's window are
// spread over the lanes, the predecessor's losses sit in a per-warp shared
// buffer indexed by absolute disparity, and the minimum m comes from one warp
// reduction per pixel.  Directions run as consecutive launches: the first
// enabled one writes S, the others add to it.
#include "rsgm_internal.cuh"

namespace rsgm {
namespace {

constexpr int kWarpsPerBlock = 4;

// Start pixel (x, y) and length n of line j of direction (DX, DY).
template <int DX, int DY>
__device__ __forceinline__ void line_start(int j, int W, int H, int &x, int &y, int &n)
{
    if (DY == 0) {  // horizontal: one line per row
        y = j;
        x = DX > 0 ? 0 : W - 1;
        n = W;
    } else if (DX == 0) {  // vertical: one line per column
        x = j;
        y = DY > 0 ? 0 : H - 1;
        n = H;
    } else {
        // diagonal: lines start on the row the direction enters from (j < W),
        // then on the column it enters from.
        int yrow = DY > 0 ? 0 : H - 1;
        int xcol = DX > 0 ? 0 : W - 1;
        if (j < W) {
            x = j;
            y = yrow;
            int run_x = DX > 0 ? W - j : j + 1;
            n = min(run_x, H);
        } else {
            int k = j - W;                     // 0 .. H-2
            y = DY > 0 ? k + 1 : k;            // the row-start line covers the corner
            x = xcol;
            int run_y = DY > 0 ? H - y : y + 1;
            n = min(W, run_y);
        }
    }
}

template <int DX, int DY>
__device__ __forceinline__ int lines_per_stream(int W, int H)
{
    return DY == 0 ? H : (DX == 0 ? W : W + H - 1);
}

template <int DX, int DY>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_path(const uint8_t *__restrict__ cost, uint16_t *__restrict__ S, const uint32_t *__restrict__ win,
           const uint32_t *__restrict__ off, Geometry g, int P1, int P2, int first)
{
    extern __shared__ uint16_t smem[];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int nl = lines_per_stream<DX, DY>(g.W, g.H);
    long long line = (long long)blockIdx.x * kWarpsPerBlock + warp;
    if (line >= (long long)g.B * nl) return;  // uniform per warp
    int b = (int)(line / nl);
    int j = (int)(line - (long long)b * nl);
    int x, y, n;
    line_start<DX, DY>(j, g.W, g.H, x, y, n);
    uint16_t *buf0 = smem + warp * 2 * g.D;
    uint16_t *buf1 = buf0 + g.D;
    const long long base = (long long)b * g.HW;
    int plo = 0, pw = 0, pmin = 0;
    for (int i = 0; i < n; ++i, x += DX, y += DY) {
        long long gp = base + (long long)y * g.W + x;
        uint32_t wv = win[gp];
        int lo = (int)(wv & 0xFFFFu), w = (int)(wv >> 16);
        uint32_t o = off[gp];
        uint16_t *cur = (i & 1) ? buf1 : buf0;
        const uint16_t *prv = (i & 1) ? buf0 : buf1;
        unsigned lmin = 0xFFFFFFFFu;
        for (int k = lane; k < w; k += 32) {
            int d = lo + k;
            int c = cost[o + k];
            int L;
            if (i == 0) {
                L = c;
            } else {
                int best = pmin + P2;
                int r = d - plo;
                if (r >= 0 && r < pw) best = min(best, (int)prv[d]);
                if (r - 1 >= 0 && r - 1 < pw) best = min(best, (int)prv[d - 1] + P1);
                if (r + 1 >= 0 && r + 1 < pw) best = min(best, (int)prv[d + 1] + P1);
                L = c + best - pmin;
            }
            cur[d] = (uint16_t)L;
            if (first)
                S[o + k] = (uint16_t)L;
            else
                S[o + k] = (uint16_t)(S[o + k] + L);
            lmin = min(lmin, (unsigned)L);
        }
        pmin = (int)__reduce_min_sync(0xffffffffu, lmin);
        __syncwarp();
        plo = lo;
        pw = w;
    }
}

template <int DX, int DY>
cudaError_t launch_dir(const Buffers &b, const Geometry &g, int P1, int P2, int first, cudaStream_t st)
{
    long long lines = (long long)g.B * (DY == 0 ? g.H : (DX == 0 ? g.W : g.W + g.H - 1));
    unsigned blocks = (unsigned)((lines + kWarpsPerBlock - 1) / kWarpsPerBlock);
    size_t smem = (size_t)kWarpsPerBlock * 2 * g.D * sizeof(uint16_t);
    k_path<DX, DY><<<blocks, kWarpsPerBlock * 32, smem, st>>>(b.cost, b.S, b.win, b.off, g, P1, P2, first);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_paths(const Buffers &b, const Geometry &g, unsigned path_mask, int P1, int P2,
                         cudaStream_t st)
{
    typedef cudaError_t (*fn)(const Buffers &, const Geometry &, int, int, int, cudaStream_t);
    static const fn dirs[8] = {launch_dir<+1, 0>,  launch_dir<-1, 0>,  launch_dir<0, +1>,
                               launch_dir<0, -1>,  launch_dir<+1, +1>, launch_dir<-1, -1>,
                               launch_dir<-1, +1>, launch_dir<+1, -1>};
    int first = 1;
    for (int i = 0; i < 8; ++i) {
        if (!(path_mask & (1u << i))) continue;
        cudaError_t e = dirs[i](b, g, P1, P2, first, st);
        if (e != cudaSuccess) return e;
        first = 0;
    }
    return cudaSuccess;
}

}  // namespace rsgm
