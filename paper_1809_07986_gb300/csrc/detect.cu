// After the path: the displayed disparity map (a 3x3 median outside the Kalman
// loop, Section 2.3) and moving-object boxes from the innovation (Section 4):
// integral image of |d_pred - d_meas|, sliding windows over the lower part of
// the image, greedy grouping of overlapping windows, small-box discard.
#include <algorithm>
#include <numeric>
#include <vector>

#include "rsgm_internal.cuh"

namespace rsgm {
namespace {

__device__ __forceinline__ void cswap(float &a, float &b)
{
    const float lo = fminf(a, b), hi = fmaxf(a, b);
    a = lo;
    b = hi;
}

// Median of the 3x3 neighbourhood (clamped at the border) by a fixed
// compare-exchange network over the 9 values; selection only, so exact.
__global__ void __launch_bounds__(256) k_median3(const float *__restrict__ d, float *__restrict__ out, Geometry g)
{
    const long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= g.NPIX) return;
    const long long b = gi / g.HW;
    const int s = (int)(gi - b * g.HW);
    const int y = s / g.W, x = s - y * g.W;
    const float *img = d + b * g.HW;
    float v[9];
    int k = 0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
        const int yy = min(max(y + dy, 0), g.H - 1);
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) v[k++] = img[yy * g.W + min(max(x + dx, 0), g.W - 1)];
    }
    // full sort by odd-even transposition (9 rounds), then take the middle
#pragma unroll
    for (int r = 0; r < 9; ++r) {
#pragma unroll
        for (int i = r & 1; i + 1 < 9; i += 2) cswap(v[i], v[i + 1]);
    }
    out[gi] = v[4];
}

// Row pass of the integral image: a = floor(|nu| * 16 + 0.5) capped at 65535
// (0 without a prediction), prefix-summed along each row into row y + 1 of the
// (H+1) x (W+1) table; row 0 and column 0 are zero.  One block per image row.
__global__ void __launch_bounds__(256) k_sat_rows(const float *__restrict__ nu, const uint8_t *__restrict__ cls,
                                                  unsigned long long *__restrict__ sat, Geometry g)
{
    __shared__ unsigned long long warp_tot[8];
    const int row = blockIdx.x;  // b * H + y
    const long long b = row / g.H;
    const int y = row - (int)b * g.H;
    const long long src = (long long)row * g.W;
    unsigned long long *dst = sat + b * (long long)(g.H + 1) * (g.W + 1) + (long long)(y + 1) * (g.W + 1);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int chunk = (g.W + blockDim.x - 1) / blockDim.x;
    const int x0 = threadIdx.x * chunk, x1 = min(g.W, x0 + chunk);
    unsigned long long local = 0;
    for (int x = x0; x < x1; ++x) {
        const float q = floorf(fabsf(nu[src + x]) * 16.0f + 0.5f);
        local += cls[src + x] == 2 ? 0ull : (q > 65535.0f ? 65535ull : (unsigned long long)q);
    }
    unsigned long long incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    unsigned long long pre = incl - local;
    for (int w = 0; w < wid; ++w) pre += warp_tot[w];
    if (threadIdx.x == 0) dst[0] = 0;
    for (int x = x0; x < x1; ++x) {
        const float q = floorf(fabsf(nu[src + x]) * 16.0f + 0.5f);
        pre += cls[src + x] == 2 ? 0ull : (q > 65535.0f ? 65535ull : (unsigned long long)q);
        dst[x + 1] = pre;
    }
}

// Column pass: each thread accumulates one column of one stream downwards;
// row 0 is written as zeros.
__global__ void __launch_bounds__(256) k_sat_cols(unsigned long long *__restrict__ sat, Geometry g)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int cols = g.W + 1;
    if (t >= (long long)g.B * cols) return;
    const long long b = t / cols;
    const int x = (int)(t - b * cols);
    unsigned long long *s = sat + b * (long long)(g.H + 1) * cols;
    s[x] = 0;
    unsigned long long acc = 0;
    for (int y = 1; y <= g.H; ++y) {
        acc += s[(long long)y * cols + x];
        s[(long long)y * cols + x] = acc;
    }
}

// One thread per (stream, window): flag = the window's sum exceeds
// thresh_q * area.  Windows are numbered size-major, then row, then column.
__global__ void __launch_bounds__(256) k_windows(const unsigned long long *__restrict__ sat,
                                                 uint8_t *__restrict__ flags, Geometry g, DetectPlan dp)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)g.B * dp.total) return;
    const long long b = t / dp.total;
    int i = (int)(t - b * dp.total);
    int s = 0;
    while (s + 1 < dp.nsizes && i >= dp.first[s + 1]) ++s;
    i -= dp.first[s];
    const int ww = dp.size[s][0], wh = dp.size[s][1];
    const int ny = dp.ny[s], nx = dp.nx[s];
    (void)ny;
    const int iy = i / nx, ix = i - iy * nx;
    const int x0 = ix * dp.stride, y0 = dp.y_min + iy * dp.stride;
    const int x1 = x0 + ww, y1 = y0 + wh;
    const int cols = g.W + 1;
    const unsigned long long *S = sat + b * (long long)(g.H + 1) * cols;
    const unsigned long long sum = S[(long long)y1 * cols + x1] - S[(long long)y0 * cols + x1] -
                                   S[(long long)y1 * cols + x0] + S[(long long)y0 * cols + x0];
    flags[t] = sum > (unsigned long long)dp.thresh_q * (unsigned long long)(ww * wh) ? 1 : 0;
}

struct Box {
    int x0, y0, x1, y1;
};

long long area(const Box &a) { return (long long)(a.x1 - a.x0) * (a.y1 - a.y0); }

long long overlap(const Box &a, const Box &b)
{
    const int w = std::min(a.x1, b.x1) - std::max(a.x0, b.x0);
    const int h = std::min(a.y1, b.y1) - std::max(a.y0, b.y0);
    return (w > 0 && h > 0) ? (long long)w * h : 0;
}

// Groups of a partition by union-find.
struct Groups {
    std::vector<int> parent;
    explicit Groups(int n) : parent(n) { std::iota(parent.begin(), parent.end(), 0); }
    int find(int a)
    {
        while (parent[a] != a) a = parent[a] = parent[parent[a]];
        return a;
    }
    bool unite(int a, int b)
    {
        a = find(a);
        b = find(b);
        if (a == b) return false;
        parent[std::max(a, b)] = std::min(a, b);
        return true;
    }
};

// "Merge any overlap" (IoU threshold 0): merging overlapping boxes into their
// bounding box until none overlap ends in the same partition whatever the
// order of the merges (a merge that another order's final partition keeps
// apart would make two of its non-overlapping final boxes overlap), and each
// group ends at the position of its first window.  So the greedy result is
// this fixpoint, computed by rounds of overlap detection and union-find
// until a round merges nothing.
//
// Overlap detection: two half-open boxes share area exactly when they cover
// a common cell of the grid whose lines are every box's edges (coordinate
// compression); each round paints every box's cells, joining it with the
// cell's first owner.  A box without area covers no cell and never merges,
// as its IoU is 0.  Painting costs the cells the boxes cover, so when that
// total exceeds the pairs a sort-and-sweep over x could check (n^2 / 2), or
// the grid would be too large for the box count, the sweep finds the pairs
// instead.
// The sorted distinct x and y edges of the boxes with area.
void grid_lines(const std::vector<Box> &v, std::vector<int> &xs, std::vector<int> &ys)
{
    xs.clear();
    ys.clear();
    for (const Box &b : v) {
        if (b.x1 <= b.x0 || b.y1 <= b.y0) continue;
        xs.push_back(b.x0);
        xs.push_back(b.x1);
        ys.push_back(b.y0);
        ys.push_back(b.y1);
    }
    std::sort(xs.begin(), xs.end());
    xs.erase(std::unique(xs.begin(), xs.end()), xs.end());
    std::sort(ys.begin(), ys.end());
    ys.erase(std::unique(ys.begin(), ys.end()), ys.end());
}

bool unite_by_grid(const std::vector<Box> &v, const std::vector<int> &xs, const std::vector<int> &ys, Groups &gr)
{
    const int n = (int)v.size();
    const long long cw = (long long)xs.size() - 1, ch = (long long)ys.size() - 1;
    std::vector<int> owner((size_t)(cw * ch), -1);
    bool merged = false;
    auto at = [](const std::vector<int> &a, int c) { return (long long)(std::lower_bound(a.begin(), a.end(), c) - a.begin()); };
    for (int i = 0; i < n; ++i) {
        const Box &b = v[i];
        if (b.x1 <= b.x0 || b.y1 <= b.y0) continue;
        const long long cx0 = at(xs, b.x0), cx1 = at(xs, b.x1), cy0 = at(ys, b.y0), cy1 = at(ys, b.y1);
        for (long long cy = cy0; cy < cy1; ++cy)
            for (long long cx = cx0; cx < cx1; ++cx) {
                int &o = owner[(size_t)(cy * cw + cx)];
                if (o < 0)
                    o = i;
                else
                    merged |= gr.unite(o, i);
            }
    }
    return merged;
}

bool unite_by_sweep(const std::vector<Box> &v, Groups &gr)
{
    const int n = (int)v.size();
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return v[a].x0 < v[b].x0; });
    bool merged = false;
    for (int s = 0; s < n; ++s) {
        const Box &a = v[order[s]];
        if (a.x1 <= a.x0 || a.y1 <= a.y0) continue;
        for (int t = s + 1; t < n && v[order[t]].x0 < a.x1; ++t) {
            const Box &b = v[order[t]];
            if (b.x1 <= b.x0 || b.y1 <= b.y0) continue;
            if (b.y0 < a.y1 && a.y0 < b.y1) merged |= gr.unite(order[s], order[t]);
        }
    }
    return merged;
}

void merge_overlapping(std::vector<Box> &v)
{
    std::vector<int> xs, ys;
    for (;;) {
        const int n = (int)v.size();
        Groups gr(n);
        grid_lines(v, xs, ys);
        if (xs.size() < 2) return;  // no box has area: nothing overlaps
        const long long cells = ((long long)xs.size() - 1) * ((long long)ys.size() - 1);
        bool grid = cells <= std::max(1LL << 22, 256LL * n);
        if (grid) {
            const long long pairs = (long long)n * (n - 1) / 2;
            long long paint = 0;
            auto at = [](const std::vector<int> &a, int c) {
                return (long long)(std::lower_bound(a.begin(), a.end(), c) - a.begin());
            };
            for (const Box &b : v) {
                if (b.x1 <= b.x0 || b.y1 <= b.y0) continue;
                paint += (at(xs, b.x1) - at(xs, b.x0)) * (at(ys, b.y1) - at(ys, b.y0));
                if (paint > pairs) break;
            }
            grid = paint <= std::max(pairs, 4LL * n);
        }
        const bool merged = grid ? unite_by_grid(v, xs, ys, gr) : unite_by_sweep(v, gr);
        if (!merged) return;
        // groups in the order of their first window; each is its members' bounding box
        std::vector<Box> next;
        std::vector<int> slot(n, -1);
        for (int i = 0; i < n; ++i) {
            const int r = gr.find(i);
            if (slot[r] < 0) {
                slot[r] = (int)next.size();
                next.push_back(v[i]);
            } else {
                Box &g = next[slot[r]];
                g = Box{std::min(g.x0, v[i].x0), std::min(g.y0, v[i].y0), std::max(g.x1, v[i].x1),
                        std::max(g.y1, v[i].y1)};
            }
        }
        v.swap(next);
    }
}

// The paper's greedy grouping with an IoU threshold: while some pair overlaps
// with IoU above iou_num / iou_den, the pair of highest IoU (first pair in
// (i, j) order on ties) becomes its bounding box, in the place of the first.
// IoUs are compared exactly as fractions of integer areas.  Quadratic per
// merge.
void merge_greedy(std::vector<Box> &v, int iou_num, int iou_den)
{
    for (;;) {
        int bi = -1, bj = -1;
        long long best_in = 0, best_un = 1;
        for (size_t i = 0; i < v.size(); ++i) {
            for (size_t j = i + 1; j < v.size(); ++j) {
                const long long in = overlap(v[i], v[j]);
                if (!in) continue;
                const long long un = area(v[i]) + area(v[j]) - in;
                // areas reach 2^42 for coordinates within +-2^20: compare in 128 bits
                if ((__int128)in * iou_den <= (__int128)iou_num * un) continue;
                if (bi < 0 || (__int128)in * best_un > (__int128)best_in * un) {
                    bi = (int)i;
                    bj = (int)j;
                    best_in = in;
                    best_un = un;
                }
            }
        }
        if (bi < 0) return;
        Box &a = v[bi];
        const Box &c = v[bj];
        a = Box{std::min(a.x0, c.x0), std::min(a.y0, c.y0), std::max(a.x1, c.x1), std::max(a.y1, c.y1)};
        v.erase(v.begin() + bj);
    }
}

}  // namespace

cudaError_t launch_median3(const float *d, float *out, const Geometry &g, cudaStream_t st)
{
    k_median3<<<(unsigned)((g.NPIX + 255) / 256), 256, 0, st>>>(d, out, g);
    return cudaGetLastError();
}

cudaError_t launch_detect_windows(const Buffers &b, const Geometry &g, const DetectPlan &dp, cudaStream_t st)
{
    k_sat_rows<<<(unsigned)(g.B * g.H), 256, 0, st>>>(b.nu, b.cls, b.sat, g);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long cols = (long long)g.B * (g.W + 1);
    k_sat_cols<<<(unsigned)((cols + 255) / 256), 256, 0, st>>>(b.sat, g);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const long long n = (long long)g.B * dp.total;
    if (n > 0) k_windows<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(b.sat, b.flags, g, dp);
    return cudaGetLastError();
}

// Groups boxes given in window order (Section 4), then drops those under
// min_area; writes up to `capacity` boxes and returns the number kept.
int group_box_list(std::vector<Box> &v, int iou_num, int iou_den, long long min_area, int32_t *out, int capacity)
{
    if (iou_num == 0)
        merge_overlapping(v);
    else
        merge_greedy(v, iou_num, iou_den);
    int n = 0;
    for (const Box &a : v) {
        if (area(a) < min_area) continue;
        if (n < capacity) {
            out[4 * n] = a.x0;
            out[4 * n + 1] = a.y0;
            out[4 * n + 2] = a.x1;
            out[4 * n + 3] = a.y1;
        }
        ++n;
    }
    return n;
}

// Boxes of one stream (host): the flagged windows in window order, grouped.
int group_boxes(const uint8_t *flags, const DetectPlan &dp, int iou_num, int iou_den, long long min_area,
                int32_t *out, int capacity)
{
    std::vector<Box> v;
    for (int s = 0; s < dp.nsizes; ++s) {
        for (int i = 0; i < dp.ny[s] * dp.nx[s]; ++i) {
            if (!flags[dp.first[s] + i]) continue;
            const int iy = i / dp.nx[s], ix = i - iy * dp.nx[s];
            const int x0 = ix * dp.stride, y0 = dp.y_min + iy * dp.stride;
            v.push_back(Box{x0, y0, x0 + dp.size[s][0], y0 + dp.size[s][1]});
        }
    }
    return group_box_list(v, iou_num, iou_den, min_area, out, capacity);
}

}  // namespace rsgm

extern "C" int rsgm_group_boxes(const rsgm_box *in, int32_t n, int32_t iou_num, int32_t iou_den, int32_t min_area,
                                rsgm_box *out, int32_t capacity, int32_t *count)
{
    if (!count || n < 0 || capacity < 0 || (n > 0 && !in) || (capacity > 0 && !out))
        return rsgm::record_error(RSGM_ERR_INVALID_ARG, "NULL or negative box array argument");
    if (iou_den < 1 || iou_num < 0 || min_area < 0)
        return rsgm::record_error(RSGM_ERR_INVALID_ARG, "iou_den >= 1, iou_num >= 0 and min_area >= 0 required");
    const int32_t lim = RSGM_BOX_COORD_LIMIT;
    for (int32_t i = 0; i < n; ++i)
        if (in[i].x0 < -lim || in[i].x0 > lim || in[i].y0 < -lim || in[i].y0 > lim || in[i].x1 < -lim ||
            in[i].x1 > lim || in[i].y1 < -lim || in[i].y1 > lim)
            return rsgm::record_error(RSGM_ERR_INVALID_ARG, "box coordinates must lie in [-2^20, 2^20]");
    std::vector<rsgm::Box> v((size_t)n);
    for (int32_t i = 0; i < n; ++i) v[(size_t)i] = rsgm::Box{in[i].x0, in[i].y0, in[i].x1, in[i].y1};
    *count = rsgm::group_box_list(v, iou_num, iou_den, min_area, reinterpret_cast<int32_t *>(out), capacity);
    return RSGM_OK;
}
