/*
 * Oracle for the reduced-space SGM + per-pixel Kalman path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, single-threaded CPU
 * restatement of what the paper "Computationally efficient dense moving object
 * detection based on reduced space disparity estimation" (Popovic, Hadviger,
 * Markovic, Petrovic) defines, written as loops over pixels and disparities so
 * that each step can be checked against the paper by eye.  Only the test suite,
 * the package smoke check and the benchmark's CPU-baseline leg load it; the
 * product path never calls it and shares no code with it.
 *
 * Precision.  Integer stages (census, cost, aggregation, winner-takes-all) are
 * exact.  The stages whose floating-point values decide integers (the
 * ego-motion warp and its rounding to a target pixel, the search window) run in
 * IEEE single precision with one rounding per written operation, in the order
 * written below; build with -ffp-contract=off so that no multiply-add is fused.
 * The Kalman correction exists in a single-precision form (same order) and a
 * double-precision form (orc_kalman64) whose difference is reported.
 *
 * Readings of points the paper leaves open are marked "Reading:".
 *
 * Parity pins (tests/test_oracle_*.py) tie each function to something other
 * than itself: closed forms, exhaustive enumeration, hand-built fixtures.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_INF16 0xFFFFu

/* ------------------------------------------------------------------ */
/* Census transform (Section 2.1: census over an n x m window, Hamming  */
/* distance as matching cost; Table 1 fixes the window at 5 x 5).       */
/* ------------------------------------------------------------------ */

/* Number of census bits for a cw x ch window: every pixel but the centre. */
int orc_census_bits(int cw, int ch) { return cw * ch - 1; }

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/*
 * code[y*W+x]: bit k is set iff I(q_k) < I(centre), where q_0, q_1, ... are the
 * window pixels in row-major order with the centre skipped (bit 0 = top-left).
 * Reading: pixels outside the image take the value of the nearest border pixel
 * (clamped coordinates).
 */
void orc_census(const uint8_t *img, int W, int H, int cw, int ch, uint64_t *code)
{
    int hw = cw / 2, hh = ch / 2;
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            int centre = img[y * W + x];
            uint64_t c = 0;
            int bit = 0;
            for (int dy = -hh; dy <= hh; dy++) {
                for (int dx = -hw; dx <= hw; dx++) {
                    if (dx == 0 && dy == 0)
                        continue;
                    int qx = clampi(x + dx, 0, W - 1);
                    int qy = clampi(y + dy, 0, H - 1);
                    if (img[qy * W + qx] < centre)
                        c |= (uint64_t)1 << bit;
                    bit++;
                }
            }
            code[y * W + x] = c;
        }
    }
}

static int popcount64(uint64_t v)
{
    int n = 0;
    while (v) {
        n += (int)(v & 1u);
        v >>= 1;
    }
    return n;
}

/*
 * Matching cost over the ragged volume (Section 2.1): for every pixel p=(x,y)
 * and every d in its window [lo, lo+wd), C(p,d) = Hamming distance between the
 * left census at (x,y) and the right census at (x-d,y).  The cell of (p,d) is
 * cost[off[p] + d - lo[p]].
 * Reading: when x-d falls left of the image, C = number of census bits.
 */
void orc_cost(const uint64_t *cl, const uint64_t *cr, int W, int H, int nbits,
              const uint16_t *lo, const uint16_t *wd, const uint32_t *off, uint8_t *cost)
{
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            int p = y * W + x;
            for (int k = 0; k < wd[p]; k++) {
                int d = lo[p] + k;
                int c;
                if (x - d < 0)
                    c = nbits;
                else
                    c = popcount64(cl[p] ^ cr[y * W + (x - d)]);
                cost[off[p] + k] = (uint8_t)c;
            }
        }
    }
}

/* Exclusive prefix sum of the window widths in raster order; returns the total
 * number of cells.  (The ragged layout: "two values for each pixel that define
 * the range for disparity search", Section 2.) */
uint64_t orc_offsets(const uint16_t *wd, int64_t n, uint32_t *off)
{
    uint64_t acc = 0;
    for (int64_t i = 0; i < n; i++) {
        off[i] = (uint32_t)acc;
        acc += wd[i];
    }
    return acc;
}

/* ------------------------------------------------------------------ */
/* Cost aggregation, Eq. 1 (Section 2.2).                                */
/* ------------------------------------------------------------------ */

/*
 * One path direction r = (dx, dy): the predecessor of p is p - r.
 *
 *   L_r(p,d) = C(p,d) + min( L_r(p-r,d),
 *                            L_r(p-r,d-1) + P1, L_r(p-r,d+1) + P1,
 *                            min_k L_r(p-r,k) + P2 )  -  min_k L_r(p-r,k)
 *
 * Readings:
 *  - The trailing "- min_k L_r(p-r,k)" (Hirschmueller's normalisation) is added
 *    so that losses stay within 16 bits, as Section 2.2 states they do; it does
 *    not change the arg-min.
 *  - k ranges over the predecessor's own window; values of L_r(p-r, .) outside
 *    that window are +infinity.
 *  - The first pixel on a path (p-r outside the image) has L_r(p,d) = C(p,d).
 *
 * Pixels are visited in an order in which p-r always comes before p: rows
 * top-to-bottom when dy >= 0 (bottom-to-top otherwise), columns left-to-right
 * when dx >= 0 (right-to-left otherwise).
 */
void orc_aggregate_dir(const uint8_t *cost, int W, int H, const uint16_t *lo,
                       const uint16_t *wd, const uint32_t *off, int dx, int dy,
                       int P1, int P2, uint16_t *Lr)
{
    int y0 = dy >= 0 ? 0 : H - 1, ystep = dy >= 0 ? 1 : -1;
    int x0 = dx >= 0 ? 0 : W - 1, xstep = dx >= 0 ? 1 : -1;
    for (int iy = 0, y = y0; iy < H; iy++, y += ystep) {
        for (int ix = 0, x = x0; ix < W; ix++, x += xstep) {
            int p = y * W + x;
            int px = x - dx, py = y - dy;
            if (px < 0 || px >= W || py < 0 || py >= H) {
                for (int k = 0; k < wd[p]; k++)
                    Lr[off[p] + k] = cost[off[p] + k];
                continue;
            }
            int q = py * W + px;
            int plo = lo[q], pw = wd[q];
            int minprev = 1 << 30;
            for (int k = 0; k < pw; k++)
                if (Lr[off[q] + k] < minprev)
                    minprev = Lr[off[q] + k];
            for (int k = 0; k < wd[p]; k++) {
                int d = lo[p] + k;
                int best = minprev + P2;
                if (d >= plo && d < plo + pw && Lr[off[q] + (d - plo)] < best)
                    best = Lr[off[q] + (d - plo)];
                if (d - 1 >= plo && d - 1 < plo + pw && Lr[off[q] + (d - 1 - plo)] + P1 < best)
                    best = Lr[off[q] + (d - 1 - plo)] + P1;
                if (d + 1 >= plo && d + 1 < plo + pw && Lr[off[q] + (d + 1 - plo)] + P1 < best)
                    best = Lr[off[q] + (d + 1 - plo)] + P1;
                Lr[off[p] + k] = (uint16_t)(cost[off[p] + k] + best - minprev);
            }
        }
    }
}

/* The 8 path directions, in the bit order of path_mask. */
static const int DIR_DX[8] = {+1, -1, 0, 0, +1, -1, -1, +1};
static const int DIR_DY[8] = {0, 0, +1, -1, +1, -1, +1, -1};

void orc_direction(int i, int *dx, int *dy)
{
    *dx = DIR_DX[i];
    *dy = DIR_DY[i];
}

/* S(p,d) = sum over the enabled directions of L_r(p,d) (Section 2.2: "costs of
 * individual paths are aggregated into the final loss").  scratch must hold
 * ncells uint16 values. */
void orc_aggregate(const uint8_t *cost, int W, int H, const uint16_t *lo, const uint16_t *wd,
                   const uint32_t *off, uint64_t ncells, unsigned path_mask, int P1, int P2,
                   uint16_t *S, uint16_t *scratch)
{
    memset(S, 0, ncells * sizeof(uint16_t));
    for (int i = 0; i < 8; i++) {
        if (!(path_mask & (1u << i)))
            continue;
        orc_aggregate_dir(cost, W, H, lo, wd, off, DIR_DX[i], DIR_DY[i], P1, P2, scratch);
        for (uint64_t c = 0; c < ncells; c++)
            S[c] = (uint16_t)(S[c] + scratch[c]);
    }
}

/* ------------------------------------------------------------------ */
/* Winner-takes-all (Section 2.3) with a parabola sub-pixel step.        */
/* ------------------------------------------------------------------ */

/*
 * d_int = the d of minimum S within the window; the smallest d wins ties.
 * Reading (the paper stops at the integer winner): when both neighbours of the
 * winner lie in the window and den = S(d-1) - 2 S(d) + S(d+1) > 0, the
 * measurement is d_z = d_int + (S(d-1) - S(d+1)) / (2 den), in single
 * precision; otherwise d_z = d_int.
 */
void orc_wta(const uint16_t *S, int64_t n, const uint16_t *lo, const uint16_t *wd,
             const uint32_t *off, int16_t *d_int, float *d_z)
{
    for (int64_t p = 0; p < n; p++) {
        const uint16_t *s = S + off[p];
        int best = 0;
        for (int k = 1; k < wd[p]; k++)
            if (s[k] < s[best])
                best = k;
        int di = lo[p] + best;
        float dz = (float)di;
        if (best >= 1 && best + 1 < wd[p]) {
            int sm = s[best - 1], s0 = s[best], sp = s[best + 1];
            int den = sm - 2 * s0 + sp;
            if (den > 0) {
                float num = (float)(sm - sp);
                float twice = (float)(2 * den);
                float frac = num / twice;
                dz = (float)di + frac;
            }
        }
        d_int[p] = (int16_t)di;
        d_z[p] = dz;
    }
}

/* ------------------------------------------------------------------ */
/* Kalman prediction (Section 2.4, Eqs. 2-4).                            */
/* ------------------------------------------------------------------ */

/* Eq. 4: p^{k|k-1} = Phi^2 p^{k-1} + q, with Phi from Eq. 3. */
float orc_predict_variance(float phi, float p, float q)
{
    float phi2 = phi * phi;
    float a = phi2 * p;
    return a + q;
}

/*
 * Eq. 2 applied to every pixel of the previous state.  Reading: the 4x4
 * H^k_{k-1} acting on (x, y, d, 1) is taken as its metric factorisation:
 * back-project with the pinhole K and baseline b (Z = fx b / d), move the point
 * with X_k = R X_{k-1} + t, project again.  One rounding per operation, in this
 * order:
 *     fb = fx*b;  Z = fb/d;  X = ((x-cx)*Z)/fx;  Y = ((y-cy)*Z)/fy
 *     X' = ((R0 X + R1 Y) + R2 Z) + t0   (likewise Y', Z')
 *     x' = ((fx X')/Z') + cx;  y' = ((fy Y')/Z') + cy;  d' = fb/Z'
 *     target = (floor(x'+0.5), floor(y'+0.5));  Phi = d'/d  (Eq. 3)
 * Readings: only pixels with d > 0.5 are moved; a point is dropped when Z' <= 0,
 * d' is not finite, or the target lies outside the image.  When several
 * points land on one target the largest d' (the nearest surface) wins; on
 * equal d' the smallest source index wins.
 *
 * Outputs per target pixel: known0 (1 if some point landed), d0 = d' and
 * p0 = Eq. 4 of the winning point.  Optional per-source outputs (may be NULL):
 * target_of_src (-1 if dropped) and dn_of_src (d').
 */
void orc_warp(const float *d, const float *p, int W, int H, const float *R, const float *t,
              const float *K, float b, float q, float *d0, float *p0, uint8_t *known0,
              int32_t *target_of_src, float *dn_of_src)
{
    float fx = K[0], cx = K[2], fy = K[4], cy = K[5];
    int64_t n = (int64_t)W * H;
    int32_t *winner = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t i = 0; i < n; i++) {
        winner[i] = -1;
        known0[i] = 0;
        d0[i] = 0.0f;
        p0[i] = 0.0f;
    }
    float fb = fx * b;
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            int s = y * W + x;
            if (target_of_src) target_of_src[s] = -1;
            if (dn_of_src) dn_of_src[s] = 0.0f;
            float ds = d[s];
            if (!(ds > 0.5f))
                continue;
            float Z = fb / ds;
            float X = (((float)x - cx) * Z) / fx;
            float Y = (((float)y - cy) * Z) / fy;
            float Xn = ((R[0] * X + R[1] * Y) + R[2] * Z) + t[0];
            float Yn = ((R[3] * X + R[4] * Y) + R[5] * Z) + t[1];
            float Zn = ((R[6] * X + R[7] * Y) + R[8] * Z) + t[2];
            if (!(Zn > 0.0f))
                continue;
            float xn = ((fx * Xn) / Zn) + cx;
            float yn = ((fy * Yn) / Zn) + cy;
            float dn = fb / Zn;
            if (!isfinite(dn))
                continue;
            float xi = floorf(xn + 0.5f), yi = floorf(yn + 0.5f);
            if (!(xi >= 0.0f && xi <= (float)(W - 1) && yi >= 0.0f && yi <= (float)(H - 1)))
                continue;
            int tgt = (int)yi * W + (int)xi;
            if (target_of_src) target_of_src[s] = tgt;
            if (dn_of_src) dn_of_src[s] = dn;
            /* z-buffer: strictly larger d' replaces; raster order makes the
             * smallest source index win a tie. */
            if (winner[tgt] < 0 || dn > d0[tgt]) {
                float phi = dn / ds; /* Eq. 3 */
                winner[tgt] = s;
                d0[tgt] = dn;
                p0[tgt] = orc_predict_variance(phi, p[s], q);
                known0[tgt] = 1;
            }
        }
    }
    free(winner);
}

/*
 * Prediction clean-up and the search window (Section 2.4).
 *
 * Zoom holes: a pixel that received no point but has both horizontal, or both
 * vertical, neighbours known takes their average (d and p).  Reading: one pass
 * over the splatted map (not in place); with both pairs known the four are
 * averaged: ((l + r) + (u + dn)) * 0.25, a single pair as (a + b) * 0.5.
 *
 * Discontinuities: predictions "near disparity discontinuities" are rejected
 * and their variance reset to cover the whole disparity space.  Reading: a
 * known pixel with a known 4-neighbour whose d differs by more than tau_disc
 * (checked after hole filling) keeps d but gets p = p_reset and the full
 * window; cls = 1.
 *
 * Window: unknown pixels (cls = 2) and reset pixels search [0, D).  Otherwise
 * c = clamp(floor(d+0.5), 0, D-1) and the window is [max(0,c-h), min(D-1,c+h)]
 * with half-width h = radius (mode 0, fixed) or ceil(p) clamped to [1, D]
 * (mode 1, the paper's d +- p reading); mode 2 keeps the full range for every
 * pixel (the plain form: full-range SGM + Kalman).
 */
void orc_resolve_map(const float *d0, const float *p0, const uint8_t *known0, int W, int H, int D,
                     int radius_mode, int radius, const uint8_t *radius_map, float p_reset,
                     float tau_disc, float *d_pred, float *p_pred, uint8_t *cls, uint16_t *lo,
                     uint16_t *wd);

void orc_resolve(const float *d0, const float *p0, const uint8_t *known0, int W, int H, int D,
                 int radius_mode, int radius, float p_reset, float tau_disc, float *d_pred,
                 float *p_pred, uint8_t *cls, uint16_t *lo, uint16_t *wd)
{
    orc_resolve_map(d0, p0, known0, W, H, D, radius_mode, radius, NULL, p_reset, tau_disc, d_pred,
                    p_pred, cls, lo, wd);
}

/* The same with radius_mode 3: the half-width of a predicted pixel is
 * radius_map[i], one value per pixel (the learned window: a per-pixel radius
 * chosen before the search; the ragged volume accepts any width). */
void orc_resolve_map(const float *d0, const float *p0, const uint8_t *known0, int W, int H, int D,
                     int radius_mode, int radius, const uint8_t *radius_map, float p_reset,
                     float tau_disc, float *d_pred, float *p_pred, uint8_t *cls, uint16_t *lo,
                     uint16_t *wd)
{
    int64_t n = (int64_t)W * H;
    uint8_t *known1 = (uint8_t *)malloc((size_t)n);
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            int i = y * W + x;
            if (known0[i]) {
                d_pred[i] = d0[i];
                p_pred[i] = p0[i];
                known1[i] = 1;
                continue;
            }
            int h = x - 1 >= 0 && x + 1 < W && known0[i - 1] && known0[i + 1];
            int v = y - 1 >= 0 && y + 1 < H && known0[i - W] && known0[i + W];
            if (h && v) {
                d_pred[i] = ((d0[i - 1] + d0[i + 1]) + (d0[i - W] + d0[i + W])) * 0.25f;
                p_pred[i] = ((p0[i - 1] + p0[i + 1]) + (p0[i - W] + p0[i + W])) * 0.25f;
                known1[i] = 1;
            } else if (h) {
                d_pred[i] = (d0[i - 1] + d0[i + 1]) * 0.5f;
                p_pred[i] = (p0[i - 1] + p0[i + 1]) * 0.5f;
                known1[i] = 1;
            } else if (v) {
                d_pred[i] = (d0[i - W] + d0[i + W]) * 0.5f;
                p_pred[i] = (p0[i - W] + p0[i + W]) * 0.5f;
                known1[i] = 1;
            } else {
                d_pred[i] = 0.0f;
                p_pred[i] = 0.0f;
                known1[i] = 0;
            }
        }
    }
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            int i = y * W + x;
            if (!known1[i]) {
                cls[i] = 2;
                lo[i] = 0;
                wd[i] = (uint16_t)D;
                continue;
            }
            int reset = 0;
            const int nx[4] = {x - 1, x + 1, x, x};
            const int ny[4] = {y, y, y - 1, y + 1};
            for (int k = 0; k < 4; k++) {
                if (nx[k] < 0 || nx[k] >= W || ny[k] < 0 || ny[k] >= H)
                    continue;
                int j = ny[k] * W + nx[k];
                if (known1[j] && fabsf(d_pred[j] - d_pred[i]) > tau_disc)
                    reset = 1;
            }
            if (reset) {
                cls[i] = 1;
                p_pred[i] = p_reset;
                lo[i] = 0;
                wd[i] = (uint16_t)D;
                continue;
            }
            cls[i] = 0;
            if (radius_mode == 2) {
                lo[i] = 0;
                wd[i] = (uint16_t)D;
                continue;
            }
            int h;
            if (radius_mode == 1) {
                float cp = ceilf(p_pred[i]);
                h = cp < 1.0f ? 1 : (cp > (float)D ? D : (int)cp);
            } else if (radius_mode == 3) {
                h = radius_map[i];
            } else {
                h = radius;
            }
            float cf = floorf(d_pred[i] + 0.5f);
            int c = cf < 0.0f ? 0 : (cf > (float)(D - 1) ? D - 1 : (int)cf);
            int a = c - h < 0 ? 0 : c - h;
            int e = c + h > D - 1 ? D - 1 : c + h;
            lo[i] = (uint16_t)a;
            wd[i] = (uint16_t)(e - a + 1);
        }
    }
    free(known1);
}

/* ------------------------------------------------------------------ */
/* Kalman correction (Section 2.4, Eqs. 5-6) and the moving-object gate. */
/* ------------------------------------------------------------------ */

/*
 * Reading: the gain is the scalar Kalman gain K = p/(p + r); Eq. 5 gives the
 * mean and Eq. 6 (evaluated as written) the variance.  Gate: with innovation
 * nu = d_z - d^{k|k-1}, a pixel whose nu^2 > gamma (p + r) is flagged as moving
 * (mask = 1) and its state is reset to the measurement (d = d_z, p = r).  A
 * pixel without a prediction (cls = 2, also every pixel of the first frame,
 * Section 2.4 last paragraph) takes d = d_z, p = r, mask = 0, nu = 0.
 * Single precision, this order:
 *     nu = dz - dp;  s = dp_var + r;  gate: nu*nu > gamma*s
 *     K = pv/s;  d = dp + K*nu;  omk = 1 - K;  p = (omk*omk)*pv + (K*K)*r
 */
void orc_kalman_update32(float dp, float pv, int cls, float dz, float r, float gamma,
                         float *d, float *p, uint8_t *mask, float *nu)
{
    if (cls == 2) {
        *d = dz;
        *p = r;
        *mask = 0;
        *nu = 0.0f;
        return;
    }
    float v = dz - dp;
    float s = pv + r;
    *nu = v;
    if (v * v > gamma * s) {
        *d = dz;
        *p = r;
        *mask = 1;
        return;
    }
    float K = pv / s;
    float kv = K * v;
    *d = dp + kv;
    float omk = 1.0f - K;
    float a = (omk * omk) * pv;
    float c = (K * K) * r;
    *p = a + c;
    *mask = 0;
}

void orc_kalman32(const float *d_pred, const float *p_pred, const uint8_t *cls, const float *d_z,
                  int64_t n, float r, float gamma, float *d, float *p, uint8_t *mask, float *nu)
{
    for (int64_t i = 0; i < n; i++)
        orc_kalman_update32(d_pred[i], p_pred[i], cls[i], d_z[i], r, gamma, &d[i], &p[i],
                            &mask[i], &nu[i]);
}

/* The same with a measurement variance per pixel (r_map[i]). */
void orc_kalman32_rmap(const float *d_pred, const float *p_pred, const uint8_t *cls,
                       const float *d_z, int64_t n, const float *r_map, float gamma, float *d,
                       float *p, uint8_t *mask, float *nu)
{
    for (int64_t i = 0; i < n; i++)
        orc_kalman_update32(d_pred[i], p_pred[i], cls[i], d_z[i], r_map[i], gamma, &d[i], &p[i],
                            &mask[i], &nu[i]);
}

/* The same correction in double precision from the same single-precision
 * inputs; the gate decision is taken in single precision (as on the device)
 * so that both forms treat the same pixels as moving. */
void orc_kalman64_rmap(const float *d_pred, const float *p_pred, const uint8_t *cls,
                       const float *d_z, int64_t n, const float *r_map, float gamma, double *d,
                       double *p);

void orc_kalman64(const float *d_pred, const float *p_pred, const uint8_t *cls, const float *d_z,
                  int64_t n, float r, float gamma, double *d, double *p)
{
    for (int64_t i = 0; i < n; i++)
        orc_kalman64_rmap(d_pred + i, p_pred + i, cls + i, d_z + i, 1, &r, gamma, d + i, p + i);
}

/* Per-pixel measurement variance r_map[i]. */
void orc_kalman64_rmap(const float *d_pred, const float *p_pred, const uint8_t *cls,
                       const float *d_z, int64_t n, const float *r_map, float gamma, double *d,
                       double *p)
{
    for (int64_t i = 0; i < n; i++) {
        const float r = r_map[i];
        if (cls[i] == 2) {
            d[i] = d_z[i];
            p[i] = r;
            continue;
        }
        float v32 = d_z[i] - d_pred[i];
        float s32 = p_pred[i] + r;
        if (v32 * v32 > gamma * s32) {
            d[i] = d_z[i];
            p[i] = r;
            continue;
        }
        double pv = p_pred[i], rr = r;
        double K = pv / (pv + rr);
        d[i] = (double)d_pred[i] + K * ((double)d_z[i] - (double)d_pred[i]);
        p[i] = (1.0 - K) * (1.0 - K) * pv + K * K * rr;
    }
}

/* ------------------------------------------------------------------ */
/* After the path: the displayed map and moving-object boxes.            */
/* ------------------------------------------------------------------ */

/*
 * 3x3 median of the disparity map (Section 2.3: a block median filter of 3x3
 * pixels in postprocessing, outside the Kalman loop).  Reading: border pixels
 * use clamped coordinates; the median of 9 values is the 5th smallest.
 */
void orc_median3(const float *d, int W, int H, float *out)
{
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            float v[9];
            int n = 0;
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++)
                    v[n++] = d[clampi(y + dy, 0, H - 1) * W + clampi(x + dx, 0, W - 1)];
            for (int i = 1; i < 9; i++) { /* insertion sort */
                float t = v[i];
                int j = i - 1;
                while (j >= 0 && v[j] > t) {
                    v[j + 1] = v[j];
                    j--;
                }
                v[j + 1] = t;
            }
            out[y * W + x] = v[4];
        }
    }
}

/*
 * |d_pred - d_meas| per pixel (Section 4), quantised to 1/16 px so that the
 * sums below are exact integers: a = floor(|nu| * 16 + 0.5), capped at 65535;
 * pixels without a prediction (cls 2) contribute 0.  Single precision.
 */
void orc_abs_innovation_q(const float *nu, const uint8_t *cls, int64_t n, uint32_t *a)
{
    for (int64_t i = 0; i < n; i++) {
        if (cls[i] == 2) {
            a[i] = 0;
            continue;
        }
        float q = floorf(fabsf(nu[i]) * 16.0f + 0.5f);
        a[i] = q > 65535.0f ? 65535u : (uint32_t)q;
    }
}

/* Summed-area table with a zero first row and column: sat[(y+1)(W+1) + x+1] =
 * sum of a over [0, x] x [0, y] (Section 4: sub-matrix sums in constant time
 * by inclusion-exclusion). */
void orc_integral(const uint32_t *a, int W, int H, uint64_t *sat)
{
    for (int x = 0; x <= W; x++) sat[x] = 0;
    for (int y = 0; y < H; y++) {
        uint64_t row = 0;
        sat[(y + 1) * (W + 1)] = 0;
        for (int x = 0; x < W; x++) {
            row += a[y * W + x];
            sat[(y + 1) * (W + 1) + x + 1] = sat[y * (W + 1) + x + 1] + row;
        }
    }
}

/*
 * Sliding windows (Section 4): for every window size (ww, wh), top-left
 * corners on a `stride` grid with y0 >= y_min (the paper skips the upper third
 * of the image), windows inside the image; a window is a detection when its
 * sum exceeds thresh_q * area (mean |nu| above the threshold, in the same
 * 1/16 px units).  Writes the detections' boxes [x0, x1) x [y0, y1) in
 * size, then row, then column order; returns how many (at most cap).
 */
int orc_windows(const uint64_t *sat, int W, int H, const int *sizes, int nsizes, int stride, int y_min,
                uint32_t thresh_q, int32_t *boxes, int cap)
{
    int n = 0;
    for (int s = 0; s < nsizes; s++) {
        int ww = sizes[2 * s], wh = sizes[2 * s + 1];
        for (int y0 = y_min; y0 + wh <= H; y0 += stride) {
            for (int x0 = 0; x0 + ww <= W; x0 += stride) {
                int x1 = x0 + ww, y1 = y0 + wh;
                uint64_t sum = sat[y1 * (W + 1) + x1] - sat[y0 * (W + 1) + x1] - sat[y1 * (W + 1) + x0] +
                               sat[y0 * (W + 1) + x0];
                if (sum > (uint64_t)thresh_q * (uint64_t)(ww * wh)) {
                    if (n < cap) {
                        boxes[4 * n] = x0;
                        boxes[4 * n + 1] = y0;
                        boxes[4 * n + 2] = x1;
                        boxes[4 * n + 3] = y1;
                    }
                    n++;
                }
            }
        }
    }
    return n < cap ? n : cap;
}

static int64_t box_area(const int32_t *b) { return (int64_t)(b[2] - b[0]) * (b[3] - b[1]); }

static int64_t box_inter(const int32_t *a, const int32_t *b)
{
    int32_t x0 = a[0] > b[0] ? a[0] : b[0], y0 = a[1] > b[1] ? a[1] : b[1];
    int32_t x1 = a[2] < b[2] ? a[2] : b[2], y1 = a[3] < b[3] ? a[3] : b[3];
    if (x1 <= x0 || y1 <= y0) return 0;
    return (int64_t)(x1 - x0) * (y1 - y0);
}

/*
 * Greedy grouping (Section 4): as long as some pair of boxes overlaps with
 * intersection-over-union above iou_num / iou_den, the pair with the highest
 * IoU is replaced by the smallest box containing both; then boxes smaller
 * than min_area are discarded.  Readings: IoU compared exactly as fractions
 * of integer areas; ties go to the lexicographically smallest pair (i, j),
 * i < j; the union takes the place of box i and box j is removed, keeping
 * the order of the others.  Works in place; returns the number of boxes.
 */
int orc_merge_boxes(int32_t *boxes, int n, int64_t iou_num, int64_t iou_den, int64_t min_area)
{
    for (;;) {
        int bi = -1, bj = -1;
        int64_t bn = 0, bd = 1; /* best IoU as a fraction */
        for (int i = 0; i < n; i++) {
            for (int j = i + 1; j < n; j++) {
                int64_t in = box_inter(boxes + 4 * i, boxes + 4 * j);
                if (in == 0) continue;
                int64_t un = box_area(boxes + 4 * i) + box_area(boxes + 4 * j) - in;
                /* above the threshold: in / un > iou_num / iou_den */
                if (!(in * iou_den > iou_num * un)) continue;
                if (bi < 0 || in * bd > bn * un) {
                    bi = i;
                    bj = j;
                    bn = in;
                    bd = un;
                }
            }
        }
        if (bi < 0) break;
        int32_t *a = boxes + 4 * bi, *b = boxes + 4 * bj;
        if (b[0] < a[0]) a[0] = b[0];
        if (b[1] < a[1]) a[1] = b[1];
        if (b[2] > a[2]) a[2] = b[2];
        if (b[3] > a[3]) a[3] = b[3];
        for (int k = bj; k + 1 < n; k++)
            for (int c = 0; c < 4; c++) boxes[4 * k + c] = boxes[4 * (k + 1) + c];
        n--;
    }
    int m = 0;
    for (int i = 0; i < n; i++) {
        if (box_area(boxes + 4 * i) < min_area) continue;
        for (int c = 0; c < 4; c++) boxes[4 * m + c] = boxes[4 * i + c];
        m++;
    }
    return m;
}
