// Cost aggregation along image rows, Eq. 1 (Section 2.2 of the paper), for
// the two horizontal directions: the predecessor of p is p - (dx, 0) and
//   L_r(p,d) = C(p,d) + min(L_r(p-r,d), L_r(p-r,d+-1) + P1, m + P2) - m,
//   m = min_k L_r(p-r,k) over the predecessor's window,
// with L_r(p-r, .) = +inf outside that window and L_r = C at the first pixel
// of a row.  Each direction writes its own plane of L_r.
//
// A row is W steps long, the longest dependency chain of the frame, so its
// steps are kept short: G lanes share a row's window (3 cells per lane), a
// warp walks 32/G rows, and the predecessor's losses sit in shared memory
// indexed by absolute disparity.  The other six directions run concurrently
// in the one-lane-per-line sweep of aggregate.cu.
#include "rsgm_internal.cuh"

namespace rsgm {
namespace {

// Launch plan: the row directions in launch order, the first warp of each,
// and the plane each writes.
struct RowPlan {
    Geometry g;
    int P1, P2;
    int lanes;           // lanes per row for narrow pixels (the common window width)
    int lines_per_warp;  // <= 32 / lanes
    int ndir;
    int dir[2];
    int plane_of[2];
    long long warp_begin[3];
    long long plane_stride;  // elements between consecutive planes
};

constexpr int kWarpsPerBlock = 4;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kInf = 0x7FFF;  // larger than any loss; + P1 still fits an int

// Start pixel (x, y) and length n of row j for direction dx.
__device__ __forceinline__ void line_start(int dx, int dy, int j, int W, int H, int &x, int &y, int &n)
{
    y = j;
    x = dx > 0 ? 0 : W - 1;
    n = W;
}

__host__ __device__ __forceinline__ int lines_per_stream(int dx, int dy, int W, int H) { return H; }

constexpr int kV = 3;   // cells per lane for narrow pixels
constexpr int kVW = 4;  // cells per lane for wide pixels
constexpr int kPad = 6; // uint16 padding between the lines' buffers: 3 banks apart

// uint16 elements of shared memory per line: two buffers of D losses + padding.
__host__ __device__ __forceinline__ int line_stride(int D) { return 2 * D + kPad; }

// Eq. 1 for kN consecutive cells d0 .. d0+kN-1 of one pixel (cells k0 + v of
// its window, up to w): the predecessor's losses at d0-1 .. d0+kN come from
// its buffer `prv` (+inf outside [plo, plo + pw)); cap = m + P2 (0 on the
// first pixel of a path), sub = m.  Writes the losses to `cur` and the plane,
// returns their minimum.
template <int kN, typename T>
__device__ __forceinline__ unsigned cells(const uint8_t *cst, T *pl, const uint16_t *prv, uint16_t *cur,
                                          int d0, int k0, int w, int plo, int pw, int cap, int sub, int P1)
{
    int pv[kN + 2];
#pragma unroll
    for (int t = 0; t < kN + 2; ++t) {
        const int dd = d0 - 1 + t;
        pv[t] = (unsigned)(dd - plo) < (unsigned)pw ? (int)prv[dd] : kInf;
    }
    unsigned m = kInf;
#pragma unroll
    for (int v = 0; v < kN; ++v) {
        // computed unconditionally; only the stores and the minimum are
        // predicated, so the body has no branches
        const int L = (int)cst[v] + min(min(pv[v + 1], cap), min(pv[v], pv[v + 2]) + P1) - sub;
        const bool in = k0 + v < w;
        if (in) {
            cur[d0 + v] = (uint16_t)L;
            pl[v] = (T)L;
        }
        m = in ? min(m, (unsigned)L) : m;
    }
    return m;
}

// Walks NS = 32 / G path lines of direction (dx, dy) with one warp.
//
// Narrow pixels (window width <= G * kV) are handled by the line's segment of
// G lanes, kV consecutive cells per lane.  Wide pixels (the full-range
// windows of discontinuity resets and pixels without a prediction) are
// handled afterwards by the whole warp, one pixel at a time, kVW cells per
// lane.  The predecessor's losses sit in a per-line shared buffer indexed by
// absolute disparity.  The direction is a run-time value so that one copy of
// this code serves all eight (a copy per direction overflows the instruction
// cache).  Metadata is fetched two pixels ahead, narrow pixels' costs one
// pixel ahead.  The lines' buffers are padded apart by three banks: adjacent
// lines read similar disparities at the same time.
//
// Loads and the first chunk of a wide pixel run without conditions (the
// cost volume is padded for the over-reads; cells outside a window are
// neither stored nor counted): guarded loads cost more issue slots than the
// loads themselves.  The segment minimum comes from shuffles: a masked
// reduction with a different mask per segment runs once per segment.
// GT > 0 fixes the lanes per line G at compile time; 0 takes G_rt.
template <typename T, int GT>
__device__ __forceinline__ void sweep(int dx, int dy, int G_rt, int NS, long long line0,
                                      const uint8_t *__restrict__ cost, T *__restrict__ plane,
                                      const uint2 *__restrict__ meta, const Geometry &g, int P1, int P2,
                                      uint16_t *wbuf)
{
    const int G = GT > 0 ? GT : G_rt;
    const int lane = threadIdx.x & 31;
    const int seg = lane / G;  // >= NS for the idle lanes above NS * G
    const int sl = lane - seg * G;
    const int kb = sl * kV;    // first window cell of this lane (narrow pixels)
    const int cap_n = G * kV;  // widest narrow window
    const int nl = lines_per_stream(dx, dy, g.W, g.H);
    // source lanes of the segment's other values (segments of at most 4 lanes)
    const int src1 = seg * G + (sl + 1) % G, src2 = seg * G + (sl + 2) % G, src3 = seg * G + (sl + 3) % G;
    const long long line = line0 + seg;
    int n = 0;
    const uint2 *mp = meta;
    if (seg < NS && line < (long long)g.B * nl) {
        const int b = (int)(line / nl);
        const int j = (int)(line - (long long)b * nl);
        int x, y;
        line_start(dx, dy, j, g.W, g.H, x, y, n);
        mp = meta + (long long)b * g.HW + (long long)y * g.W + x;
    }
    const int nmax = (int)__reduce_max_sync(kFull, (unsigned)n);
    const int step = dy * g.W + dx;
    uint16_t *bufA = wbuf + min(seg, NS - 1) * line_stride(g.D);
    uint16_t *bufB = bufA + g.D;

    uint2 mc = n > 0 ? mp[0] : make_uint2(0u, 0u);
    uint2 mn = n > 1 ? mp[step] : make_uint2(0u, 0u);
    uint8_t cc[kV];
#pragma unroll
    for (int v = 0; v < kV; ++v) cc[v] = cost[mc.x + kb + v];
    int plo = 0, pw = 0, pmin = 0;
    // unrolled by two so that the fetched-ahead registers swap roles instead
    // of being copied (a copy would wait for the fetch to land)
#pragma unroll 2
    for (int i = 0; i < nmax; ++i) {
        mp += step;
        const uint2 mnn = (i + 2 < n) ? mp[step] : make_uint2(0u, 0u);
        uint8_t cn[kV];
#pragma unroll
        for (int v = 0; v < kV; ++v) cn[v] = cost[mn.x + kb + v];
        const unsigned o = mc.x;
        const int lo = (int)(mc.y & 0xFFFFu);
        const int w = i < n ? (int)(mc.y >> 16) : 0;
        const int sel = i & 1;
        const int cap = i == 0 ? 0 : pmin + P2;

        unsigned lmin = kInf;
        if (w <= cap_n && kb < w)
            lmin = cells<kV, T>(cc, plane + o + kb, sel ? bufA : bufB, sel ? bufB : bufA, lo + kb, kb, w, plo, pw,
                                cap, pmin, P1);
        if (G == 32) {
            lmin = __reduce_min_sync(kFull, lmin);
        } else if (G <= 4) {
            // every lane gathers its segment's other G - 1 values
            const unsigned l0 = lmin;
            lmin = min(lmin, __shfl_sync(kFull, l0, src1));
            if (G > 2) lmin = min(lmin, __shfl_sync(kFull, l0, src2));
            if (G > 3) lmin = min(lmin, __shfl_sync(kFull, l0, src3));
        } else {
            for (int off = 1; off < G; off <<= 1) {
                const unsigned y = __shfl_down_sync(kFull, lmin, off);
                if (sl + off < G) lmin = min(lmin, y);
            }
            lmin = __shfl_sync(kFull, lmin, seg * G);
        }

        // wide pixels: the whole warp, one pixel at a time
        unsigned wide = __ballot_sync(kFull, seg < NS && sl == 0 && w > cap_n);
        while (wide) {
            const int src = __ffs(wide) - 1;
            wide &= wide - 1;
            const int s2 = src / G;
            const unsigned f1 = __shfl_sync(kFull, (unsigned)lo | ((unsigned)plo << 16), src);
            const unsigned f2 = __shfl_sync(kFull, (unsigned)w | ((unsigned)pw << 16), src);
            const int pmin2 = __shfl_sync(kFull, pmin, src);
            const unsigned o2 = __shfl_sync(kFull, o, src);
            const int lo2 = (int)(f1 & 0xFFFFu), plo2 = (int)(f1 >> 16);
            const int w2 = (int)(f2 & 0xFFFFu), pw2 = (int)(f2 >> 16);
            const int cap2 = i == 0 ? 0 : pmin2 + P2;
            uint16_t *b2 = wbuf + s2 * line_stride(g.D);
            unsigned m2 = kInf;
            int k0 = lane * kVW;
            do {
                uint8_t c4[kVW];
#pragma unroll
                for (int v = 0; v < kVW; ++v) c4[v] = cost[o2 + k0 + v];
                m2 = min(m2, cells<kVW, T>(c4, plane + o2 + k0, b2 + (sel ^ 1) * g.D, b2 + sel * g.D, lo2 + k0, k0,
                                           w2, plo2, pw2, cap2, pmin2, P1));
                k0 += 32 * kVW;
            } while (k0 < w2);
            m2 = __reduce_min_sync(kFull, m2);
            if (seg == s2) lmin = m2;
        }
        __syncwarp();
        pmin = (int)lmin;
        plo = lo;
        pw = w;
        mc = mn;
        mn = mnn;
#pragma unroll
        for (int v = 0; v < kV; ++v) cc[v] = cn[v];
    }
}

// Row directions by path_mask bit: the predecessor of p is p - (dx, 0).
__constant__ int kDX[2] = {+1, -1};
__constant__ int kDY[2] = {0, 0};

template <typename T, int GT>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 8)
    k_rows(const uint8_t *__restrict__ cost, T *__restrict__ planes, const uint2 *__restrict__ meta,
            const __grid_constant__ RowPlan plan)
{
    extern __shared__ uint16_t smem[];
    const int warp = threadIdx.x >> 5;
    const long long gw = (long long)blockIdx.x * kWarpsPerBlock + warp;
    if (gw >= plan.warp_begin[plan.ndir]) return;  // uniform per warp
    int s = 0;
    while (s + 1 < plan.ndir && gw >= plan.warp_begin[s + 1]) ++s;
    const long long line0 = (gw - plan.warp_begin[s]) * plan.lines_per_warp;
    uint16_t *wbuf = smem + warp * plan.lines_per_warp * line_stride(plan.g.D);
    T *plane = planes + (long long)plan.plane_of[s] * plan.plane_stride;
    const int dir = plan.dir[s];
    sweep<T, GT>(kDX[dir], kDY[dir], plan.lanes, plan.lines_per_warp, line0, cost, plane, meta, plan.g, plan.P1,
             plan.P2, wbuf);
}

template <typename T, int GT>
cudaError_t launch_g(const Buffers &b, const RowPlan &plan, cudaStream_t st)
{
    const long long warps = plan.warp_begin[plan.ndir];
    if (warps == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((warps + kWarpsPerBlock - 1) / kWarpsPerBlock);
    const size_t smem = (size_t)kWarpsPerBlock * plan.lines_per_warp * line_stride(plan.g.D) * sizeof(uint16_t);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_rows<T, GT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_rows<T, GT><<<blocks, kWarpsPerBlock * 32, smem, st>>>(b.cost, (T *)b.planes, b.meta, plan);
    return cudaGetLastError();
}

// The common lane counts (windows of 2r + 1 for r = 2 and 4; full range) are
// compile-time constants in their own instantiations: index arithmetic on
// G folds away, which shortens every step.
template <typename T>
cudaError_t launch_t(const Buffers &b, const RowPlan &plan, cudaStream_t st)
{
    switch (plan.lanes) {
    case 2: return launch_g<T, 2>(b, plan, st);
    case 3: return launch_g<T, 3>(b, plan, st);
    case 32: return launch_g<T, 32>(b, plan, st);
    default: return launch_g<T, 0>(b, plan, st);
    }
}

}  // namespace

int lanes_per_line(int window)
{
    // Enough lanes (3 cells each) for the common (predicted) window, at least
    // 2 (at most 16 rows per warp); wider windows go through the whole-warp
    // path.
    const int G = (window + kV - 1) / kV;
    return G < 2 ? 2 : (G > 32 ? 32 : G);
}

cudaError_t launch_rows(const Buffers &b, const Geometry &g, unsigned path_mask, unsigned run_mask, int P1, int P2,
                        int lanes, int plane_bytes, int sm_count, cudaStream_t st)
{
    RowPlan plan;
    plan.g = g;
    plan.P1 = P1;
    plan.P2 = P2;
    plan.plane_stride = plane_stride(g);
    // planes are numbered by direction bit order over every enabled direction
    int plane_index[8], np = 0;
    for (int i = 0; i < 8; ++i) plane_index[i] = (path_mask & (1u << i)) ? np++ : -1;
    plan.ndir = 0;
    plan.warp_begin[0] = 0;
    plan.lanes = lanes;
    // Rows per warp.  fill = lines per warp that would give every SM 32
    // warps, counting the lines of every enabled direction (the other
    // directions' sweep runs beside this one); about a quarter of it balances
    // a warp's sequential steps against the work its rows share per step
    // (measured on paper-shaped frames).  Capped by the lanes (32 / lanes) and
    // by the row buffers: those of 8 resident blocks stay within 168 KB of
    // shared memory.
    long long total_lines = 0;
    for (int dir = 0; dir < 8; ++dir)
        if (path_mask & (1u << dir))
            total_lines += (long long)g.B * (dir < 2 ? g.H : (dir < 4 ? g.W : g.W + g.H - 1));
    const long long fill = total_lines / ((long long)(sm_count > 0 ? sm_count : 152) * 32);
    const long long smem_cap = (168LL * 1024 / 8) / ((long long)kWarpsPerBlock * line_stride(g.D) * 2);
    long long most = 32 / lanes;
    if (smem_cap < most) most = smem_cap < 1 ? 1 : smem_cap;
    const long long pick = (fill + 2) / 4;
    plan.lines_per_warp = (int)(pick < 1 ? 1 : (pick > most ? most : pick));
    for (int dir = 0; dir < 2; ++dir) {
        if (!(run_mask & (1u << dir))) continue;
        const long long lines = (long long)g.B * g.H;
        plan.dir[plan.ndir] = dir;
        plan.plane_of[plan.ndir] = plane_index[dir];
        plan.warp_begin[plan.ndir + 1] =
            plan.warp_begin[plan.ndir] + (lines + plan.lines_per_warp - 1) / plan.lines_per_warp;
        plan.ndir++;
    }
    if (plan.ndir == 0) return cudaSuccess;
    return plane_bytes == 1 ? launch_t<uint8_t>(b, plan, st) : launch_t<uint16_t>(b, plan, st);
}

}  // namespace rsgm
