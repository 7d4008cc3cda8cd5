// Winner-takes-all (Section 2.3 of the paper), parabola sub-pixel step, the
// per-pixel Kalman correction (Eqs. 5-6, Section 2.4) and the moving-object
// gate on the innovation, fused in one pass over the aggregated costs.
#include "rsgm_internal.cuh"

namespace rsgm {
namespace {

__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }

constexpr int kUpdWarps = 4;
constexpr int kStageCells = 1024;  // per-warp staging of S; larger spans read S from global memory
constexpr int kLaneScan = 16;      // windows up to this width are scanned by their own lane
constexpr unsigned kFull = 0xffffffffu;

// S = sum of the direction planes over the cells [c0, c1), written to S and to
// the warp's staging buffer (indexed from a16 = c0 rounded down to 16 cells).
// 8-bit planes are read 16 cells per 128-bit load and summed as 16-bit pairs,
// which cannot carry: 8 planes x 255 < 2^16.  The whole chunks cover cells of
// the neighbouring warps' spans as well: S there is the same sum of the same
// planes, so writing it again changes nothing.  (Planes start 16-element
// aligned, and the planes and S have 16 cells of slack past the last one.)
__device__ __forceinline__ void sum_planes(const uint8_t *__restrict__ planes, long long stride, int nplanes,
                                           unsigned c0, unsigned c1, uint16_t *__restrict__ S,
                                           uint16_t *stage, int lane)
{
    const unsigned a16 = c0 & ~15u;
    const int nchunks = (int)((c1 - a16 + 15) >> 4);
    for (int ci = lane; ci < nchunks; ci += 32) {
        const unsigned cell = a16 + 16u * (unsigned)ci;
        uint4 ev = make_uint4(0u, 0u, 0u, 0u), od = ev;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (q < nplanes) {
                const uint4 v = *(const uint4 *)(planes + q * stride + cell);
                ev.x += v.x & 0x00FF00FFu;
                od.x += (v.x >> 8) & 0x00FF00FFu;
                ev.y += v.y & 0x00FF00FFu;
                od.y += (v.y >> 8) & 0x00FF00FFu;
                ev.z += v.z & 0x00FF00FFu;
                od.z += (v.z >> 8) & 0x00FF00FFu;
                ev.w += v.w & 0x00FF00FFu;
                od.w += (v.w >> 8) & 0x00FF00FFu;
            }
        }
        // word j of a chunk holds cells 4j .. 4j+3: (even lo, odd lo, even hi, odd hi)
        const uint4 sa = make_uint4(__byte_perm(ev.x, od.x, 0x5410u), __byte_perm(ev.x, od.x, 0x7632u),
                                    __byte_perm(ev.y, od.y, 0x5410u), __byte_perm(ev.y, od.y, 0x7632u));
        const uint4 sb = make_uint4(__byte_perm(ev.z, od.z, 0x5410u), __byte_perm(ev.z, od.z, 0x7632u),
                                    __byte_perm(ev.w, od.w, 0x5410u), __byte_perm(ev.w, od.w, 0x7632u));
        *(uint4 *)(S + cell) = sa;
        *(uint4 *)(S + cell + 8) = sb;
        if (stage) {
            *(uint4 *)(stage + (cell - a16)) = sa;
            *(uint4 *)(stage + (cell - a16) + 8) = sb;
        }
    }
}

__device__ __forceinline__ void sum_planes(const uint16_t *__restrict__ planes, long long stride, int nplanes,
                                           unsigned c0, unsigned c1, uint16_t *__restrict__ S,
                                           uint16_t *stage, int lane)
{
    for (unsigned c = c0 + lane; c < c1; c += 32) {
        unsigned v = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (q < nplanes) v += planes[q * stride + c];
        S[c] = (uint16_t)v;
        if (stage) stage[c - (c0 & ~15u)] = (uint16_t)v;
    }
}

// K5: one warp per 32 consecutive pixels.  Their cells are one contiguous
// span of the ragged volume (offsets are a raster-order prefix sum), so the
// warp first sums the direction planes cell by cell with coalesced loads,
// S(p,d) = sum_r L_r(p,d) (Section 2.2), writes S and, for spans of up to
// kStageCells cells, stages it in shared memory.  d_int = first minimum of S
// over the window: each lane scans its own pixel's window of up to kLaneScan
// cells; wider windows are scanned by the whole warp, one pixel at a time, as
// a minimum of (S << 16 | k) keys, from the staged copy or with coalesced
// loads.  With both neighbours inside the window and den = S- - 2 S0 + S+ > 0
// the measurement is d_int + (S- - S+) / (2 den).  Pixels without a
// prediction take the measurement (d = d_z, p = r).  Otherwise
// nu = d_z - d_pred; if nu^2 > gamma (p_pred + r) the pixel is flagged and
// reset to the measurement, else K = p_pred / (p_pred + r), d = d_pred + K nu,
// p = (1 - K)^2 p_pred + K^2 r.
template <typename T>
__global__ void __launch_bounds__(kUpdWarps * 32, 16) k_update(const T *__restrict__ planes, long long plane_stride,
                                                        int nplanes, uint16_t *__restrict__ S,
                                                        const uint2 *__restrict__ meta,
                                                        const uint8_t *__restrict__ cls,
                                                        const float *__restrict__ d_pred,
                                                        const float *__restrict__ p_pred,
                                                        float *__restrict__ d, float *__restrict__ p,
                                                        int16_t *__restrict__ d_int, uint8_t *__restrict__ mask,
                                                        float *__restrict__ d_z, float *__restrict__ nu_out,
                                                        const float *__restrict__ r_map, Geometry g,
                                                        FrameParams fp)
{
    extern __shared__ uint16_t sS[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long gi0 = ((long long)blockIdx.x * kUpdWarps + warp) * 32;
    if (gi0 >= g.NPIX) return;  // uniform per warp
    const long long gi = gi0 + lane;
    const bool valid = gi < g.NPIX;
    const uint2 m = valid ? meta[gi] : make_uint2(0u, 0u);
    const int lo = (int)(m.y & 0xFFFFu), w = valid ? (int)(m.y >> 16) : 0;
    const unsigned span0 = __shfl_sync(0xffffffffu, m.x, 0);
    const int nvalid = (int)min(32LL, g.NPIX - gi0);
    const unsigned last_end = __shfl_sync(0xffffffffu, m.x + (unsigned)w, nvalid - 1);
    const unsigned a16 = span0 & ~15u;  // the staging buffer starts at the span's 16-cell chunk
    const bool staged = last_end - a16 <= (unsigned)kStageCells;
    uint16_t *stage = staged ? sS + warp * kStageCells : nullptr;
    sum_planes(planes, plane_stride, nplanes, span0, last_end, S, stage, lane);
    __syncwarp();  // S (shared or global) complete for the warp
    const uint16_t *s = staged ? stage + (m.x - a16) : S + m.x;
    int best = 0;
    unsigned bs = 0;
    if (valid && w > 0 && w <= kLaneScan) {
        bs = s[0];
        for (int k = 1; k < w; ++k) {
            const unsigned v = s[k];
            if (v < bs) {
                bs = v;
                best = k;
            }
        }
    }
    {
        unsigned wide = __ballot_sync(kFull, valid && w > kLaneScan);
        while (wide) {
            const int src = __ffs(wide) - 1;
            wide &= wide - 1;
            const unsigned off = __shfl_sync(kFull, m.x, src);
            const int ww = __shfl_sync(kFull, w, src);
            const uint16_t *s2 = staged ? stage + (off - a16) : S + off;
            unsigned key = 0xFFFFFFFFu;  // S in the high half, k in the low: the first minimum wins
            for (int k = lane; k < ww; k += 32) key = min(key, ((unsigned)s2[k] << 16) | (unsigned)k);
            key = __reduce_min_sync(kFull, key);
            if (lane == src) {
                bs = key >> 16;
                best = (int)(key & 0xFFFFu);
            }
        }
    }
    if (!valid) return;
    const uint8_t role = fp.role[gi / g.HW];
    if (role == RSGM_SLOT_IDLE) return;  // the stream sits this frame out: state and outputs unchanged
    int di = lo + best;
    float dz = (float)di;
    if (best >= 1 && best + 1 < w) {
        int sm = s[best - 1], sp = s[best + 1];
        int den = sm - 2 * (int)bs + sp;
        if (den > 0) dz = fadd((float)di, fdiv((float)(sm - sp), (float)(2 * den)));
    }
    d_int[gi] = (int16_t)di;
    d_z[gi] = dz;
    // per pixel with the learned window; a new stream's first frame uses r_meas
    float r = (r_map && role != RSGM_SLOT_FULL) ? r_map[gi] : fp.r_meas;
    if (cls[gi] == 2) {
        d[gi] = dz;
        p[gi] = r;
        mask[gi] = 0;
        nu_out[gi] = 0.0f;
        return;
    }
    float dp = d_pred[gi], pv = p_pred[gi];
    float v = fsub(dz, dp);
    float sv = fadd(pv, r);
    nu_out[gi] = v;
    if (fmul(v, v) > fmul(fp.gamma, sv)) {
        d[gi] = dz;
        p[gi] = r;
        mask[gi] = 1;
        return;
    }
    float K = fdiv(pv, sv);
    d[gi] = fadd(dp, fmul(K, v));
    float omk = fsub(1.0f, K);
    p[gi] = fadd(fmul(fmul(omk, omk), pv), fmul(fmul(K, K), r));
    mask[gi] = 0;
}

}  // namespace

cudaError_t launch_update(const Buffers &b, const Geometry &g, const FrameParams &fp, const float *r_map,
                          int nplanes, int plane_bytes, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((g.NPIX + kUpdWarps * 32 - 1) / (kUpdWarps * 32));
    const long long stride = plane_stride(g);
    const size_t smem = (size_t)kUpdWarps * kStageCells * sizeof(uint16_t);
    if (plane_bytes == 1)
        k_update<uint8_t><<<blocks, kUpdWarps * 32, smem, st>>>((const uint8_t *)b.planes, stride, nplanes, b.S, b.meta,
                                                  b.cls, b.d_pred, b.p_pred, b.d, b.p, b.d_int, b.mask,
                                                  b.d_z, b.nu, r_map, g, fp);
    else
        k_update<uint16_t><<<blocks, kUpdWarps * 32, smem, st>>>((const uint16_t *)b.planes, stride, nplanes, b.S, b.meta,
                                                   b.cls, b.d_pred, b.p_pred, b.d, b.p, b.d_int, b.mask,
                                                   b.d_z, b.nu, r_map, g, fp);
    return cudaGetLastError();
}

}  // namespace rsgm
