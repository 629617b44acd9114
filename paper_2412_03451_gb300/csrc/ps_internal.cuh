// ps_internal.cuh -- device helpers shared by the libps translation units.
// Every TU of the library is compiled with -fmad=false: multiply-adds are
// written as explicit fmaf() so that the forward and the backward kernels,
// which recompute the same per-pixel candidate list, evaluate bit-identical
// arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include "ps.h"

#define PS_CUDA_CHECK(expr)                                   \
    do {                                                      \
        cudaError_t e_ = (expr);                              \
        if (e_ != cudaSuccess) return PS_ERR_CUDA;            \
    } while (0)

#define PS_LAUNCH_CHECK()                                     \
    do {                                                      \
        cudaError_t e_ = cudaGetLastError();                  \
        if (e_ != cudaSuccess) return PS_ERR_CUDA;            \
    } while (0)

namespace ps {

constexpr int kRecFloats = 16;   // floats per record

__device__ __forceinline__ void set_status(int* st, ps_status code)
{
    if (st) atomicOr(st, 1 << (int)code);
}

// Global tile -> view by binary search over tile_off (views sorted by tile_off).
__device__ __forceinline__ int view_of_tile(const ps_view* views, int V, int tile)
{
    int lo = 0, hi = V - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(&views[mid].tile_off) <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One plane in camera coordinates, as stored in a record.
struct Rec {
    float4 n;    // n_c, s = n_c . p_c
    float4 vx;   // v^x_c, a_x = v^x_c . p_c
    float4 vy;   // v^y_c, a_y = v^y_c . p_c
    float4 r;    // r^x+, r^x-, r^y+, r^y-
};

// Evaluation of one (pixel ray, plane) pair: Eq. 4, 6-9 and the filter of
// Sec. 3.2.  d = (dx, dy, 1).  Returns true if the pair is a candidate.
struct PairEval {
    float t, w;        // depth, weight
    float m;           // margin of the active side
    float P;           // P_X or P_Y of the active side
    float den;         // d . n_c
    float dv;          // d . v_c of the active side
    bool sideX;        // active side is X (m_X < m_Y); ties go to Y
    bool pos;          // P > 0 on the active side (selects r^+)
    // both axes (used by the Gaussian weight of Eq. 5)
    float X, Y;        // P_X, P_Y
    float dvx, dvy;    // d . v^x_c, d . v^y_c
    float sX, sY;      // radius on the side of P_X, P_Y
};

struct SplatConst {
    float lam5;        // 5 lambda
    float w_min;
    float z_near, z_far;
    float reject;      // quick reject: margins below -reject cannot reach w_min
    int hard;          // PS_HARD
    int gauss;         // PS_GAUSSIAN: the Eq. 5 weight
    float kappa;       // Eq. 5: w >= w_min only within kappa radii of the centre on each axis
};

// Every operation is executed for every lane and the filter is applied at the
// end: lanes of a warp leave at different tests, so early returns would only
// serialise the warp.  The selected values are the same as with early exits.
__device__ __forceinline__ bool eval_pair(const float4& n, const float4& vx, const float4& vy,
                                          const float4& r, float dx, float dy,
                                          const SplatConst& c, PairEval& o)
{
    const float den = fmaf(dx, n.x, fmaf(dy, n.y, n.z));
    const float t = __fdividef(n.w, den);
    const float dvx = fmaf(dx, vx.x, fmaf(dy, vx.y, vx.z));
    const float dvy = fmaf(dx, vy.x, fmaf(dy, vy.y, vy.z));
    const float X = fmaf(t, dvx, -vx.w);
    const float Y = fmaf(t, dvy, -vy.w);
    const float sXr = X > 0.f ? r.x : r.y, sYr = Y > 0.f ? r.z : r.w;
    o.X = X; o.Y = Y; o.dvx = dvx; o.dvy = dvy; o.sX = sXr; o.sY = sYr;
    if (c.gauss) {
        // Eq. 5 in the plane's frame, the one-sided radii as the scales
        const float ux = __fdividef(X, sXr), uy = __fdividef(Y, sYr);
        const float w = __expf(-0.5f * (ux * ux + uy * uy));
        o.t = t; o.w = w; o.m = 0.f; o.den = den;
        o.sideX = false; o.P = Y; o.dv = dvy; o.pos = Y > 0.f;
        return (fabsf(den) > 1e-6f) && (t > c.z_near && t < c.z_far) && (w >= c.w_min);
    }
    const float mX = sXr - fabsf(X);
    const float mY = sYr - fabsf(Y);
    const bool sx = mX < mY;
    const float m = sx ? mX : mY;
    // w = min(1, 2 sigmoid(5 lambda m)); below the clamp 2 sigmoid(x) = 2 e^x / (1 + e^x)
    const float e = __expf(c.lam5 * m);
    const float w = (m >= 0.f) ? 1.f : __fdividef(2.f * e, 1.f + e);
    const bool ok = (fabsf(den) > 1e-6f) && (t > c.z_near && t < c.z_far) && !(m < -c.reject) &&
                    (m >= 0.f || !c.hard) && (w >= c.w_min);
    o.t = t; o.w = w; o.m = m; o.den = den;
    o.sideX = sx;
    o.P = sx ? X : Y;
    o.dv = sx ? dvx : dvy;
    o.pos = o.P > 0.f;
    return ok;
}

// Rays through the pixel centres at the corners of a warp's pixel rectangle.
struct WarpRegion {
    float dxa, dxb, dya, dyb;
};

// Conservative test whether a plane can pass the filter at any pixel of a
// warp's rectangle.  For a fixed plane, t = s / (d . n_c) and P = t (d . v_c) - a
// are linear-fractional in the ray d = (dx, dy, 1); if d . n_c keeps its sign
// over the rectangle they are monotone along every line, so their ranges over
// the rectangle are spanned by the four corner rays.  The corner values use
// the per-pixel formulas of eval_pair; the margins cover FP32 rounding.
__device__ __forceinline__ bool region_may_hit(const float4& n, const float4& vx, const float4& vy,
                                               const float4& r, const WarpRegion& g,
                                               const SplatConst& c)
{
    float tmin = INFINITY, tmax = -INFINITY, xmin = INFINITY, xmax = -INFINITY;
    float ymin = INFINITY, ymax = -INFINITY;
    int npos = 0, nneg = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float dx = (k & 1) ? g.dxb : g.dxa;
        const float dy = (k & 2) ? g.dyb : g.dya;
        const float den = fmaf(dx, n.x, fmaf(dy, n.y, n.z));
        npos += den > 2e-6f;
        nneg += den < -2e-6f;
        const float t = __fdividef(n.w, den);
        const float dvx = fmaf(dx, vx.x, fmaf(dy, vx.y, vx.z));
        const float dvy = fmaf(dx, vy.x, fmaf(dy, vy.y, vy.z));
        const float X = fmaf(t, dvx, -vx.w);
        const float Y = fmaf(t, dvy, -vy.w);
        tmin = fminf(tmin, t); tmax = fmaxf(tmax, t);
        xmin = fminf(xmin, X); xmax = fmaxf(xmax, X);
        ymin = fminf(ymin, Y); ymax = fmaxf(ymax, Y);
    }
    if (npos != 4 && nneg != 4) return true;       // d . n_c may vanish: no bound
    if (tmax < c.z_near * 0.99999f || tmin > c.z_far * 1.00001f) return false;
    // support: r + reject around the rectangle, or kappa r for the Eq. 5 weight
    const float sc = c.gauss ? c.kappa : 1.f;
    const float rej = c.gauss ? 0.f : c.reject;
    const float mx = rej + 1e-5f * (fabsf(xmin) + fabsf(xmax) + fabsf(tmax)) + 1e-6f;
    const float my = rej + 1e-5f * (fabsf(ymin) + fabsf(ymax) + fabsf(tmax)) + 1e-6f;
    if (xmax < -(sc * r.y + mx) || xmin > sc * r.x + mx) return false;
    if (ymax < -(sc * r.w + my) || ymin > sc * r.z + my) return false;
    return true;
}

// (t, id) lexicographic order of candidates.
__device__ __forceinline__ bool cand_less(float ta, int ia, float tb, int ib)
{
    return ta < tb || (ta == tb && ia < ib);
}

}  // namespace ps
