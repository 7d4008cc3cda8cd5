// Cost aggregation, Eq. 1 (Section 2.2 of the paper), over the ragged cell
// volume: for path direction r the predecessor of p is p - r and
//   L_r(p,d) = C(p,d) + min(L_r(p-r,d), L_r(p-r,d+-1) + P1, m + P2) - m,
//   m = min_k L_r(p-r,k) over the predecessor's window,
// with L_r(p-r, .) = +inf outside that window and L_r = C at the first pixel
// of a path.  Each enabled direction writes its own plane of L_r; the update
// kernel sums the planes into S.
//
// One lane walks one path line; a warp walks 32 parallel lines in lockstep
// (for vertical and diagonal directions, 8 groups of 4 adjacent lines, whose
// lanes visit 4 consecutive pixels of one image row at every step).  Losses are held as two 16-bit values per 32-bit
// register and combined with packed minima and carry-free 32-bit additions.
#include "rsgm_internal.cuh"

namespace rsgm {
namespace {

constexpr unsigned kFull = 0xffffffffu;
// +inf of a packed pair.  Every finite loss is at most census bits + P2
// (< 0x1000); a cell past the end of its window carries a cost of at least
// 0xFF, or 0x4000 with the general masking, so its loss exceeds every cap
// m + P2, and inf + P1 still fits 16 bits: no operation carries or borrows
// across the two halves.
constexpr unsigned kInf2 = 0x40004000u;

__device__ __forceinline__ unsigned vmin2(unsigned a, unsigned b)
{
    unsigned r;
    asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

__host__ __device__ __forceinline__ int lines_per_stream(int dx, int dy, int W, int H)
{
    return dy == 0 ? H : (dx == 0 ? W : W + H - 1);
}

// Eq. 1 for two cells (one packed pair): lft / rgt hold the predecessor's
// losses at d-1 and d+1 of each cell (two slots each, starting one slot apart
// from the pair), c the costs; cap2 = m + P2 and m2 = m in both halves.
__device__ __forceinline__ unsigned eq1(unsigned lft, unsigned rgt, unsigned c, unsigned P1x2, unsigned cap2,
                                        unsigned m2)
{
    const unsigned ctr = __byte_perm(lft, rgt, 0x5432);  // the predecessor at d
    unsigned t = vmin2(lft, rgt) + P1x2;
    t = vmin2(vmin2(t, ctr), cap2);
    return c + t - m2;  // t >= m in both halves: no borrow
}

// Cells at or past the window width w get a cost of at least 0x4000 (the
// general masking): per half, 0x8000 + slot - w has bit 15 set iff slot >= w.
__device__ __forceinline__ unsigned mask_pair(unsigned c, unsigned slots, unsigned w2)
{
    const unsigned x = (slots | 0x80008000u) - w2;
    return c | ((x >> 1) & 0x40004000u);
}

// Packs the low bytes of four 16-bit losses into one word of an 8-bit plane.
__device__ __forceinline__ unsigned pack4(unsigned a, unsigned b) { return __byte_perm(a, b, 0x6420); }

// n packed pairs of the band starting at slot t (any parity): slot s lives in
// half (s + pad) & 1 of word (s + pad) >> 1.
template <int N>
__device__ __forceinline__ void band_load(const unsigned *band, int t, int pad, unsigned (&u)[N])
{
    const int s = t + pad;
    const unsigned *p = band + (s >> 1);
    const unsigned sel = (s & 1) ? 0x5432u : 0x3210u;
    unsigned w0 = p[0];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const unsigned w1 = p[i + 1];
        u[i] = __byte_perm(w0, w1, sel);
        w0 = w1;
    }
}

// Byte bands (the cheap masking, where 0xFF acts as +inf): slot s is byte
// s + pad of the band.  n packed pairs starting at slot t (any alignment).
template <int N>
__device__ __forceinline__ void band_load8(const unsigned *band, int t, int pad, unsigned (&u)[N])
{
    const int s = t + pad;
    const unsigned *p = band + (s >> 2);
    const unsigned sh = 8u * (unsigned)(s & 3);
    constexpr int NWORDS = (2 * N + 3) / 4;  // aligned words of the 2N bytes
    unsigned w0 = p[0];
#pragma unroll
    for (int j = 0; j < NWORDS; ++j) {
        const unsigned w1 = p[j + 1];
        const unsigned a = __funnelshift_r(w0, w1, sh);
        if (2 * j < N) u[2 * j] = __byte_perm(a, 0u, 0x4140u);
        if (2 * j + 1 < N) u[2 * j + 1] = __byte_perm(a, 0u, 0x4342u);
        w0 = w1;
    }
}

// A pair saturated to 0xFF per half (a loss of at least 0xFF acts as +inf
// under the cheap masking, so saturating keeps every result).
__device__ __forceinline__ unsigned sat8(unsigned x) { return vmin2(x, 0x00FF00FFu); }

// Walks this lane's path line (the warp walks up to 32 lines of one
// direction and stream in lockstep, placed by the caller).
//
// Narrow pixels (window width <= 2 NR) are done by the line's own lane, the
// window in NR packed registers: slot k holds the loss at d = lo + k.  When
// the window moves by at most 2 against the predecessor's, the predecessor's
// losses are realigned in registers; otherwise they go through the lane's
// band in shared memory.  Wide pixels (the full-range windows of resets and
// pixels without a prediction) are done by the whole warp, with the
// predecessor's losses in the line's band.  A band holds a window at
// slots [0, w) with +inf on [-pad, 0) and on [round4(w), round4(w) + pad);
// reads that can see no slot of [0, w) take +inf without loading.
//
// Metadata is fetched two steps ahead; narrow costs, and the costs of the
// first two wide pixels of a step, one step ahead.  Wide pixels go two at a
// time, one per half-warp, 8 cells per lane: KW passes of 128 cells cover a
// window.
template <typename T, int NR, int KW, bool kCheap>
__device__ __forceinline__ void walk(int dx, int dy, int b, int k, bool line_ok, const uint8_t *__restrict__ cost,
                                     T *__restrict__ plane, const uint2 *__restrict__ meta, const LinePlan &plan,
                                     unsigned *band_all, unsigned *band)
{
    constexpr int NC = 2 * NR;        // narrow capacity in cells
    constexpr int NW = (NR + 1) / 2;  // cost words of a narrow window
    const Geometry &g = plan.g;
    const int lane = threadIdx.x & 31;
    const int W = g.W, H = g.H, pad = plan.pad;

    // this lane's active steps [s_first, s_last] and its pixel at step 0
    int s_first = 0, s_last = -1;
    long long gi0 = 0;
    if (line_ok) {
        if (dy == 0) {
            s_last = W - 1;
            gi0 = (long long)b * g.HW + (long long)k * W + (dx > 0 ? 0 : W - 1);
        } else {
            gi0 = (long long)b * g.HW + (long long)(dy > 0 ? 0 : H - 1) * W + k;
            if (dx == 0) {
                s_last = H - 1;
            } else if (dx > 0) {
                s_first = max(0, -k);
                s_last = min(H - 1, W - 1 - k);
            } else {
                s_first = max(0, k - (W - 1));
                s_last = min(H - 1, k);
            }
        }
    }
    const bool any = s_first <= s_last;
    const int s0 = (int)__reduce_min_sync(kFull, any ? (unsigned)s_first : 0x7FFFFFFFu);
    const int s1 = (int)__reduce_max_sync(kFull, any ? (unsigned)s_last : 0u);
    if (s0 > s1) return;  // no lane of this warp has a pixel (uniform)
    const long long step = (long long)dy * W + dx;
    auto active = [&](int s) { return s >= s_first && s <= s_last; };
    auto meta_at = [&](int s) { return active(s) ? meta[gi0 + s * step] : make_uint2(0u, 0u); };

    const unsigned P1x2 = (unsigned)plan.P1 * 0x10001u;
    unsigned P[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) P[i] = kInf2;
    int plo = 0, pw = 0, pm = 0;  // predecessor window and minimum; pw = 0: no predecessor
    bool inband = false;          // the predecessor's losses are in the band, not in P

    // the lane's narrow window into its band at slots [0, 2 NR), +inf after it
    auto spill = [&](const unsigned (&Pr)[NR]) {
        if (kCheap) {
            constexpr int NQ = (NR + 1) / 2;
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                band[(pad >> 2) + q] = pack4(sat8(Pr[2 * q]), 2 * q + 1 < NR ? sat8(Pr[2 * q + 1]) : 0x00FF00FFu);
            for (int q = 0; q < (pad >> 2); ++q) band[(pad >> 2) + NQ + q] = 0xFFFFFFFFu;
        } else {
#pragma unroll
            for (int i = 0; i < NR; ++i) band[(pad >> 1) + i] = Pr[i];
            for (int q = 0; q < (pad >> 1); ++q) band[(pad >> 1) + NR + q] = kInf2;
        }
    };

    // This lane's cost words of the first pass over the wide windows among
    // the pixels of `m`: the first two wide pixels, one per half-warp, 8
    // cells per lane and 128-cell pass.
    auto fetch_wide = [&](const uint2 &m, unsigned (&wp)[KW][2]) {
        unsigned wm = __ballot_sync(kFull, (int)(m.y >> 16) > NC);
#pragma unroll
        for (int it = 0; it < KW; ++it) wp[it][0] = wp[it][1] = 0u;
        if (!wm) return;  // uniform: no wide pixel among them
        const int sa = __ffs(wm) - 1;
        wm &= wm - 1;
        const int sb = wm ? __ffs(wm) - 1 : sa;
        const int src = (lane >> 4) ? sb : sa;
        const unsigned so = __shfl_sync(kFull, m.x, src), sw = __shfl_sync(kFull, m.y >> 16, src);
        const bool mine = !(lane >> 4) || sb != sa;
#pragma unroll
        for (int it = 0; it < KW; ++it) {
            const unsigned c0 = 8u * (lane & 15) + 128u * it;
            if (mine && c0 < sw) {
                const unsigned *p = (const unsigned *)(cost + so + c0);
                wp[it][0] = p[0];
                wp[it][1] = p[1];
            }
        }
    };
    auto fetch_narrow = [&](const uint2 &m, unsigned (&c)[NW]) {
        const int w = (int)(m.y >> 16);
        const unsigned *src = (const unsigned *)(cost + m.x);
#pragma unroll
        for (int q = 0; q < NW; ++q) c[q] = (w > 0 && w <= NC) ? src[q] : 0u;
    };

    uint2 mc = meta_at(s0), mn = meta_at(s0 + 1);
    unsigned cc[NW], wc[KW][2];
    fetch_narrow(mc, cc);
    fetch_wide(mc, wc);
#pragma unroll 2
    for (int s = s0; s <= s1; ++s) {
        const uint2 mnn = meta_at(s + 2);
        unsigned cn[NW], wn[KW][2];
        fetch_narrow(mn, cn);
        fetch_wide(mn, wn);
        const unsigned o = mc.x;
        const int lo = (int)(mc.y & 0xFFFFu), w = (int)(mc.y >> 16);

        if (w > 0 && w <= NC) {
            // ---- narrow: this lane alone
            unsigned U[NR + 1];
            unsigned cap2 = 0u, m2 = 0u;
            if (pw == 0) {
#pragma unroll
                for (int i = 0; i <= NR; ++i) U[i] = kInf2;
            } else {
                cap2 = (unsigned)(pm + plan.P2) * 0x10001u;
                m2 = (unsigned)pm * 0x10001u;
                const int e = lo - plo - 1;  // slot of the predecessor at d - 1 for the first cell
                if (inband || e < -3 || e > 1) {
                    if (!inband) {
                        // realign a large move through the band
                        spill(P);
                    }
                    if (e >= pw || e + NC + 1 < 0) {
#pragma unroll
                        for (int i = 0; i <= NR; ++i) U[i] = kInf2;
                    } else {
                        if (kCheap)
                            band_load8<NR + 1>(band, e, pad, U);
                        else
                            band_load<NR + 1>(band, e, pad, U);
                    }
                } else {
                    // e = 2 sh + odd with sh in {-2, -1, 0}: U[i] = Q[i + sh],
                    // Q[j] = predecessor slots (2j + odd, 2j + odd + 1)
                    const unsigned sel = (e & 1) ? 0x5432u : 0x3210u;
                    const int sh = e >> 1;
                    unsigned Q[NR + 3];  // Q[j + 2] for j = -2 .. NR
                    Q[0] = kInf2;
                    Q[1] = __byte_perm(kInf2, P[0], sel);
#pragma unroll
                    for (int j = 0; j < NR; ++j) Q[j + 2] = __byte_perm(P[j], j + 1 < NR ? P[j + 1] : kInf2, sel);
                    Q[NR + 2] = kInf2;
#pragma unroll
                    for (int i = 0; i <= NR; ++i) U[i] = sh == 0 ? Q[i + 2] : (sh == -1 ? Q[i + 1] : Q[i]);
                }
            }
            unsigned cw[NW];
#pragma unroll
            for (int q = 0; q < NW; ++q) cw[q] = (q == 0 || 4 * q < w) ? cc[q] : 0xFFFFFFFFu;
            const unsigned w2 = (unsigned)w * 0x10001u;
#pragma unroll
            for (int i = 0; i < NR; ++i) {
                unsigned c = __byte_perm(cw[i >> 1], 0u, (i & 1) ? 0x4342u : 0x4140u);
                if (!kCheap) c = mask_pair(c, (unsigned)(2 * i) | ((unsigned)(2 * i + 1) << 16), w2);
                P[i] = eq1(U[i], U[i + 1], c, P1x2, cap2, m2);
            }
            // the window's minimum as a tree: it feeds the next step's m + P2
            unsigned mt[NR];
#pragma unroll
            for (int i = 0; i < NR; ++i) mt[i] = P[i];
#pragma unroll
            for (int span = 1; span < NR; span *= 2)
#pragma unroll
                for (int i = 0; i + span < NR; i += 2 * span) mt[i] = vmin2(mt[i], mt[i + span]);
            const unsigned run = mt[0];
            // plane words of the pixel's cells [0, round4(w))
            if (sizeof(T) == 1) {
                unsigned *dst = (unsigned *)(plane + o);
#pragma unroll
                for (int q = 0; q < NW; ++q)
                    if (q == 0 || 4 * q < w) dst[q] = pack4(P[2 * q], 2 * q + 1 < NR ? P[2 * q + 1] : kInf2);
            } else {
                uint2 *dst = (uint2 *)(plane + o);
#pragma unroll
                for (int q = 0; q < NW; ++q)
                    if (q == 0 || 4 * q < w) dst[q] = make_uint2(P[2 * q], 2 * q + 1 < NR ? P[2 * q + 1] : kInf2);
            }
            plo = lo;
            pw = w;
            pm = (int)min(run & 0xFFFFu, run >> 16);
            inband = false;
        }

        // ---- wide: the whole warp, two pixels at a time (one per half-warp)
        unsigned wide = __ballot_sync(kFull, w > NC);
        if (wide) {
            if (w > NC && pw > 0 && !inband) {
                spill(P);
            }
            __syncwarp();
            const int half = lane >> 4, hl = lane & 15;
            for (int jp = 0; wide; ++jp) {
                const int sa = __ffs(wide) - 1;
                wide &= wide - 1;
                const int sb = wide ? __ffs(wide) - 1 : sa;
                if (sb != sa) wide &= wide - 1;
                const int src = half ? sb : sa;
                const bool mine = !half || sb != sa;  // this half-warp has a pixel
                const unsigned so = __shfl_sync(kFull, o, src);
                const unsigned f1 = __shfl_sync(kFull, (unsigned)lo | ((unsigned)w << 16), src);
                const unsigned f2 = __shfl_sync(kFull, (unsigned)plo | ((unsigned)pw << 16), src);
                const int spm = __shfl_sync(kFull, pm, src);
                const int slo = (int)(f1 & 0xFFFFu), sw = mine ? (int)(f1 >> 16) : 0;
                const int splo = (int)(f2 & 0xFFFFu), spw = (int)(f2 >> 16);
                unsigned *sbd = band_all + src * plan.band_words;
                const unsigned cap2 = spw ? (unsigned)(spm + plan.P2) * 0x10001u : 0u;
                const unsigned m2 = spw ? (unsigned)spm * 0x10001u : 0u;
                const unsigned w2 = (unsigned)sw * 0x10001u;
                unsigned Lr[KW][4];
                unsigned run = kInf2;
#pragma unroll
                for (int it = 0; it < KW; ++it) {
                    const int c0 = 8 * hl + 128 * it;
                    Lr[it][0] = Lr[it][1] = Lr[it][2] = Lr[it][3] = kInf2;
                    if (c0 < sw) {
                        unsigned U[5];
                        const int t0 = slo + c0 - 1 - splo;  // predecessor slot of d - 1 for cell c0
                        if (spw == 0 || t0 >= spw || t0 + 9 < 0) {
#pragma unroll
                            for (int i = 0; i < 5; ++i) U[i] = kInf2;
                        } else {
                            if (kCheap)
                                band_load8<5>(sbd, t0, pad, U);
                            else
                                band_load<5>(sbd, t0, pad, U);
                        }
                        unsigned cw0, cw1;  // the first pass's costs were fetched a step ahead
                        if (jp == 0) {
                            cw0 = wc[it][0];
                            cw1 = wc[it][1];
                        } else {
                            const unsigned *p = (const unsigned *)(cost + so + c0);
                            cw0 = p[0];
                            cw1 = p[1];
                        }
                        // the second word lies past the window's run when c0 + 4 >= w: it
                        // holds the next pixel's costs, which must not enter the minimum
                        if (kCheap && c0 + 4 >= sw) cw1 = 0xFFFFFFFFu;
                        unsigned c[4] = {__byte_perm(cw0, 0u, 0x4140u), __byte_perm(cw0, 0u, 0x4342u),
                                         __byte_perm(cw1, 0u, 0x4140u), __byte_perm(cw1, 0u, 0x4342u)};
                        if (!kCheap) {
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                c[i] = mask_pair(c[i], (unsigned)(c0 + 2 * i) | ((unsigned)(c0 + 2 * i + 1) << 16), w2);
                        }
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            Lr[it][i] = eq1(U[i], U[i + 1], c[i], P1x2, cap2, m2);
                            if (kCheap) Lr[it][i] = sat8(Lr[it][i]);  // byte bands: saturated
                            run = vmin2(run, Lr[it][i]);
                        }
                        if (sizeof(T) == 1) {
                            unsigned *dst = (unsigned *)(plane + so + c0);
                            dst[0] = pack4(Lr[it][0], Lr[it][1]);
                            if (c0 + 4 < sw) dst[1] = pack4(Lr[it][2], Lr[it][3]);
                        } else {
                            uint2 *dst = (uint2 *)(plane + so + c0);
                            dst[0] = make_uint2(Lr[it][0], Lr[it][1]);
                            if (c0 + 4 < sw) dst[1] = make_uint2(Lr[it][2], Lr[it][3]);
                        }
                    }
                }
                // minimum over each half-warp's cells
                unsigned r = min(run & 0xFFFFu, run >> 16);
#pragma unroll
                for (int off = 8; off >= 1; off >>= 1) r = min(r, __shfl_xor_sync(kFull, r, off));
                const unsigned ra = __shfl_sync(kFull, r, 0), rb = __shfl_sync(kFull, r, 16);
                __syncwarp();  // every read of the source bands is done
#pragma unroll
                for (int it = 0; it < KW; ++it) {
                    const int c0 = 8 * hl + 128 * it;
                    if (c0 < sw) {
                        // 32-bit stores: bands have an odd word stride, so a
                        // band word is not 8-byte aligned in general
                        if (kCheap) {
                            unsigned *q = sbd + ((c0 + pad) >> 2);
                            q[0] = pack4(Lr[it][0], Lr[it][1]);
                            if (c0 + 4 < sw) q[1] = pack4(Lr[it][2], Lr[it][3]);
                        } else {
                            unsigned *q = sbd + ((c0 + pad) >> 1);
                            q[0] = Lr[it][0];
                            q[1] = Lr[it][1];
                            if (c0 + 4 < sw) {
                                q[2] = Lr[it][2];
                                q[3] = Lr[it][3];
                            }
                        }
                    }
                }
                const int ext = (sw + 3) & ~3;
                if (kCheap) {
                    if (mine && hl < (pad >> 2)) sbd[((ext + pad) >> 2) + hl] = 0xFFFFFFFFu;
                } else {
                    if (mine && hl < (pad >> 1)) sbd[((ext + pad) >> 1) + hl] = kInf2;
                }
                __syncwarp();
                if (lane == sa || lane == sb) {  // the sources take their own window
                    plo = lo;
                    pw = w;
                    pm = (int)(lane == sa ? ra : rb);
                    inband = true;
                }
            }
        }
        if (w == 0) pw = 0;  // off the image: the next pixel starts the line

        mc = mn;
        mn = mnn;
#pragma unroll
        for (int q = 0; q < NW; ++q) cc[q] = cn[q];
#pragma unroll
        for (int it = 0; it < KW; ++it) {
            wc[it][0] = wn[it][0];
            wc[it][1] = wn[it][1];
        }
    }
}

// Path directions by path_mask bit: the predecessor of p is p - (dx, dy).
__constant__ int kDX[8] = {+1, -1, 0, 0, +1, -1, -1, +1};
__constant__ int kDY[8] = {0, 0, +1, -1, +1, -1, +1, -1};

template <typename T, int NR, int KW, bool kCheap>
__global__ void __launch_bounds__(kLineWarps * 32, (kCheap && KW == 1) ? 8 : 5)
    k_lines(const uint8_t *__restrict__ cost, T *__restrict__ planes, const uint2 *__restrict__ meta,
            const __grid_constant__ LinePlan plan)
{
    extern __shared__ unsigned smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long gw = (long long)blockIdx.x * kLineWarps + warp;
    if (gw >= plan.warp_begin[plan.ndir]) return;  // uniform per warp
    int si = 0;
    while (si + 1 < plan.ndir && gw >= plan.warp_begin[si + 1]) ++si;
    const int dir = plan.dir[si];
    const int dx = kDX[dir], dy = kDY[dir];
    const int nl = lines_per_stream(dx, dy, plan.g.W, plan.g.H);
    const int lpw = dy == 0 ? plan.hlines : 32;  // lines per warp
    const int wps = (nl + lpw - 1) / lpw;
    const long long wi = gw - plan.warp_begin[si];
    const int b = (int)(wi / wps), kw = (int)(wi - (long long)b * wps);
    const int kbase = (dx > 0 && dy != 0) ? -(plan.g.H - 1) : 0;
    // Lines are dealt to warps interleaved, so that every warp gets its share
    // of the image's full-range regions (the borders without a prediction,
    // rows of resets along depth edges): horizontal lines (rows, which no
    // warp reads coalesced) one by one, vertical and diagonal lines in groups
    // of 4 adjacent lines (32 bytes of metadata per group and step).  A
    // horizontal line is W steps long, the longest chain of the launch, so
    // horizontal warps may walk fewer than 32 rows to shorten their steps.
    const int li = dy == 0 ? kw + lane * wps : ((kw + (lane >> 2) * wps) << 2) + (lane & 3);
    const bool line_ok = li < nl && lane < lpw;
    unsigned *band_all = smem + warp * 32 * plan.band_words;
    unsigned *band = band_all + lane * plan.band_words;
    // slots [-pad, 0): always +inf
    if (kCheap)
        for (int q = 0; q < (plan.pad >> 2); ++q) band[q] = 0xFFFFFFFFu;
    else
        for (int q = 0; q < (plan.pad >> 1); ++q) band[q] = kInf2;
    __syncwarp();
    T *plane = planes + (long long)plan.plane_of[si] * plan.plane_stride;
    walk<T, NR, KW, kCheap>(dx, dy, b, kbase + li, line_ok, cost, plane, meta, plan, band_all, band);
}

template <typename T, int NR, int KW, bool kCheap>
cudaError_t launch_nr(const Buffers &b, const LinePlan &plan, cudaStream_t st)
{
    const long long warps = plan.warp_begin[plan.ndir];
    if (warps == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((warps + kLineWarps - 1) / kLineWarps);
    const size_t smem = (size_t)kLineWarps * 32 * plan.band_words * sizeof(unsigned);
    if (smem > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(k_lines<T, NR, KW, kCheap>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_lines<T, NR, KW, kCheap><<<blocks, kLineWarps * 32, smem, st>>>(b.cost, (T *)b.planes, b.meta, plan);
    return cudaGetLastError();
}

template <typename T, int KW, bool kCheap>
cudaError_t launch_kw(const Buffers &b, const LinePlan &plan, int nr, cudaStream_t st)
{
    switch (nr) {
    case 1: return launch_nr<T, 1, KW, kCheap>(b, plan, st);
    case 3: return launch_nr<T, 3, KW, kCheap>(b, plan, st);
    case 5: return launch_nr<T, 5, KW, kCheap>(b, plan, st);
    default: return launch_nr<T, 9, KW, kCheap>(b, plan, st);
    }
}

template <typename T, bool kCheap>
cudaError_t launch_t(const Buffers &b, const LinePlan &plan, int nr, cudaStream_t st)
{
    // one pass of 128 cells covers every window up to D = 128
    return plan.g.D <= 128 ? launch_kw<T, 1, kCheap>(b, plan, nr, st) : launch_kw<T, 2, kCheap>(b, plan, nr, st);
}

}  // namespace

const int kHostDX[8] = {+1, -1, 0, 0, +1, -1, -1, +1};
const int kHostDY[8] = {0, 0, +1, -1, +1, -1, +1, -1};

int sweep_capacity(int cells)
{
    // instantiated register capacities (2 NR cells): 2, 6, 10, 18
    return cells <= 2 ? 2 : (cells <= 6 ? 6 : (cells <= 10 ? 10 : 18));
}

cudaError_t launch_paths(const Buffers &b, const Geometry &g, unsigned path_mask, unsigned run_mask, int P1, int P2,
                         int nbits, int plane_bytes, int capacity, int hlines, cudaStream_t st)
{
    LinePlan plan;
    plan.g = g;
    plan.P1 = P1;
    plan.P2 = P2;
    plan.plane_stride = plane_stride(g);
    const int nr = sweep_capacity(capacity) / 2;
    // the cheap masking (cells past a window cost 0xFF) needs every cap
    // m + P2 <= nbits + 2 P2 below 0xFF; its losses then fit byte bands
    const bool cheap = plane_bytes == 1 && nbits + 2 * P2 < 255;
    // +inf padding around a band's window: at least the widest read past it
    // (a narrow read spans 2 NR + 2 slots, a wide one 10), a multiple of 4 so
    // that slot 0 is word aligned in byte and in 16-bit bands
    plan.pad = (max(10, 2 * nr + 2) + 3) & ~3;
    // slots [-pad, round4(max(D, 2 NR)) + pad) in 32-bit words, an odd count
    // so that the lanes' bands fall in different shared-memory banks
    const int cap = (max(g.D, 2 * nr) + 3) & ~3;
    int words = cheap ? (cap + 2 * plan.pad + 3) / 4 : (cap + 2 * plan.pad) / 2;
    if (!(words & 1)) ++words;
    plan.band_words = words;
    // rows per horizontal warp: 16 by default (fastest at 4 and 32
    // paper-shaped streams: 8 adds emptier warps, 32 lengthens the 1242-step
    // rows' critical path); the autotuner tries 8, 16 and 32
    plan.hlines = hlines == 8 || hlines == 32 ? hlines : 16;
    // Long lines first so that the tail of the launch is short: horizontal,
    // diagonal, vertical.  Planes are numbered by direction bit order.
    static const int order[8] = {0, 1, 4, 5, 6, 7, 2, 3};
    int plane_index[8], np = 0;
    for (int i = 0; i < 8; ++i) plane_index[i] = (path_mask & (1u << i)) ? np++ : -1;
    plan.ndir = 0;
    plan.warp_begin[0] = 0;
    for (int kk = 0; kk < 8; ++kk) {
        const int dir = order[kk];
        if (!(path_mask & run_mask & (1u << dir))) continue;
        const int lpw = kHostDY[dir] == 0 ? plan.hlines : 32;
        const long long warps =
            (long long)g.B * ((lines_per_stream(kHostDX[dir], kHostDY[dir], g.W, g.H) + lpw - 1) / lpw);
        plan.dir[plan.ndir] = dir;
        plan.plane_of[plan.ndir] = plane_index[dir];
        plan.warp_begin[plan.ndir + 1] = plan.warp_begin[plan.ndir] + warps;
        plan.ndir++;
    }
    if (plane_bytes == 1)
        return cheap ? launch_t<uint8_t, true>(b, plan, nr, st) : launch_t<uint8_t, false>(b, plan, nr, st);
    return launch_t<uint16_t, false>(b, plan, nr, st);
}

}  // namespace rsgm
