/*
 * ps_oracle.c -- plain, slow, FP64 CPU definition of PlanarSplatting's
 * differentiable planar-primitive rendering (arxiv 2412.03451, Sec. 3.2).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code, header, table or helper
 * with the CUDA library, and the CUDA library never calls it.
 *
 * Every function brute-forces the definition: every plane is tested at every
 * pixel, there is no tiling, no culling and no reordering beyond what the
 * paper states.  Build with -ffp-contract=off so that no multiply-add is
 * fused: the binning function below must give the same integers as any other
 * implementation of the same strict formula.
 *
 * Conventions (readings of the paper, listed with reasons in the design
 * notes of the repository):
 *   plane k: center p (3), quaternion q = (w,x,y,z) (4), radii
 *            r = (r^x+, r^x-, r^y+, r^y-) (4)                     [Eq. 1]
 *   v^x, v^y, n = columns 0,1,2 of R(q/|q|), Hamilton convention [Eq. 2-3]
 *   camera v: world->camera [R|t] row-major 3x4, intrinsics (fx,fy,cx,cy),
 *             OpenCV frame; pixel (i,j) ray d = ((i+.5-cx)/fx, (j+.5-cy)/fy, 1)
 *   intersection depth t = ((p_c - o).n_c)/(d.n_c) with o = 0; since d_z = 1
 *             t is the camera z-depth                              [Eq. 4]
 *   P_X = (t d - p_c).v^x_c, P_Y likewise                           [Eq. 6]
 *   w_X = min(1, 2 sigmoid(5 lambda (r_X - |P_X|))), r_X = r^x+ if P_X > 0
 *             else r^x-; w_Y likewise                               [Eq. 7-8]
 *   w = w_X if w_X < w_Y else w_Y                                   [Eq. 9]
 *   keep w >= w_min (1e-4) and z_near < t < z_far and |d.n_c| > 1e-6,
 *   sort by (t, plane id), keep the first M (30)          [Sec. 3.2, Blending]
 *   D = sum T_j w_j t_j, N = sum T_j w_j n_c,j, T_j = prod_{i<j} (1 - w_i)
 *                                                                  [Eq. 11-13]
 *   loss = a_cos sum |1 - N.N*| + a_l1n sum ||N - N*||_1 + a_depth sum |D - D*|
 *             over pixels with D* > 0                              [Eq. 14]
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Plane frame: Eq. 2-3.  Hamilton rotation matrix of the unit quaternion.   */
/* Returns 0 if |q| is zero or not finite.                                   */
static int plane_axes(const double* q, double* qn_out, double qhat[4],
                      double vx[3], double vy[3], double n[3])
{
    double s = sqrt(((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3]);
    if (!(s > 0.0) || !isfinite(s)) return 0;
    double is = 1.0 / s;
    double w = q[0] * is, x = q[1] * is, y = q[2] * is, z = q[3] * is;
    if (qn_out) *qn_out = s;
    if (qhat) { qhat[0] = w; qhat[1] = x; qhat[2] = y; qhat[3] = z; }
    /* R = [[1-2(y^2+z^2), 2(xy-wz), 2(xz+wy)],
            [2(xy+wz), 1-2(x^2+z^2), 2(yz-wx)],
            [2(xz-wy), 2(yz+wx), 1-2(x^2+y^2)]]                             */
    vx[0] = 1.0 - 2.0 * (y * y + z * z);
    vx[1] = 2.0 * (x * y + w * z);
    vx[2] = 2.0 * (x * z - w * y);
    vy[0] = 2.0 * (x * y - w * z);
    vy[1] = 1.0 - 2.0 * (x * x + z * z);
    vy[2] = 2.0 * (y * z + w * x);
    n[0] = 2.0 * (x * z + w * y);
    n[1] = 2.0 * (y * z - w * x);
    n[2] = 1.0 - 2.0 * (x * x + y * y);
    return 1;
}

static void rot_apply(const double* Rt /* 3x4 row major */, const double a[3], double out[3])
{
    for (int i = 0; i < 3; ++i)
        out[i] = (Rt[4 * i + 0] * a[0] + Rt[4 * i + 1] * a[1]) + Rt[4 * i + 2] * a[2];
}

static void rot_apply_T(const double* Rt, const double a[3], double out[3])
{
    for (int i = 0; i < 3; ++i)
        out[i] = (Rt[0 + i] * a[0] + Rt[4 + i] * a[1]) + Rt[8 + i] * a[2];
}

static double dot3(const double a[3], const double b[3])
{
    return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}

/* Camera-frame quantities of one plane in one view. */
typedef struct {
    int ok;
    double qs, qhat[4];
    double vx[3], vy[3], n[3];       /* world axes (Eq. 2-3)  */
    double pc[3], vxc[3], vyc[3], nc[3];
    double r[4];                     /* radii after the single-radii option */
    double pcn;                      /* |p_c|, scale of the FP32 noise model */
} plane_cam;

/* flags: bit 0 = single radii (Sec. 4.3), bit 2 = Gaussian weight (Eq. 5).   */
#define OR_SINGLE 1
#define OR_GAUSS 4

static void plane_to_cam(const double* p, const double* q, const double* r,
                         const double* Rt, int flags, plane_cam* o)
{
    const int single_radii = flags & OR_SINGLE;
    o->ok = plane_axes(q, &o->qs, o->qhat, o->vx, o->vy, o->n);
    if (!o->ok) return;
    double tmp[3];
    rot_apply(Rt, p, tmp);
    for (int i = 0; i < 3; ++i) o->pc[i] = tmp[i] + Rt[4 * i + 3];
    rot_apply(Rt, o->vx, o->vxc);
    rot_apply(Rt, o->vy, o->vyc);
    rot_apply(Rt, o->n, o->nc);
    o->pcn = sqrt(dot3(o->pc, o->pc));
    o->r[0] = r[0]; o->r[1] = single_radii ? r[0] : r[1];
    o->r[2] = r[2]; o->r[3] = single_radii ? r[2] : r[3];
}

/* ------------------------------------------------------------------------ */
/* Binning specification (screen bounds of the expanded rectangle).          */
/* The rectangle is widened by delta on every side; delta is the margin at   */
/* which 2 sigmoid(-5 lambda delta) = w_min, so every (pixel, plane) pair    */
/* that survives the w >= w_min filter of Sec. 3.2 lies inside it.  With the */
/* Gaussian weight of Eq. 5 (flag bit 2) every radius is multiplied by delta */
/* instead, delta = sqrt(2 ln(1 / w_min)): exp(-q/2) >= w_min needs          */
/* |P_X| <= delta sigma_X and |P_Y| <= delta sigma_Y.  The quad is clipped   */
/* to z >= z_near, projected, and its pixel bbox, padded by one pixel and    */
/* clamped to the image, is divided by the tile size.  The depth key is the  */
/* smallest z of the clipped polygon, a lower bound on the depth t of every  */
/* surviving intersection (up to the rounding of the formula).               */
/* The formula is evaluated in FP32 (every input rounded to float, delta    */
/* included) with plain + - * / sqrt, left to right as written, no FMA, so   */
/* that any IEEE implementation of it gives the same integers.  It is a      */
/* conservative bound, not part of the rendered value: the renderer below   */
/* stays in FP64.                                                           */
/* rect = (tx0, ty0, tx1, ty1) inclusive; culled planes get (0,0,-1,-1).     */

/* The plane's camera frame in FP32, the same formulas as plane_axes and     */
/* plane_to_cam in the same order.  Returns 0 for a zero or non-finite |q|.  */
typedef struct {
    float pc[3], vxc[3], vyc[3], nc[3], r[4];
} frame_f32;

static float rowf(const float* R, int i, const float a[3])
{
    return (R[4 * i + 0] * a[0] + R[4 * i + 1] * a[1]) + R[4 * i + 2] * a[2];
}

static int plane_frame_f32(const double* p, const double* q, const double* r,
                           const double* Rt, int flags, frame_f32* o)
{
    float R[12], pf[3], vx[3], vy[3], n[3];
    for (int i = 0; i < 12; ++i) R[i] = (float)Rt[i];
    for (int i = 0; i < 3; ++i) pf[i] = (float)p[i];
    float q0 = (float)q[0], q1 = (float)q[1], q2 = (float)q[2], q3 = (float)q[3];
    float s = sqrtf(((q0 * q0 + q1 * q1) + q2 * q2) + q3 * q3);
    if (!(s > 0.0f) || !isfinite(s)) return 0;
    float is = 1.0f / s;
    float w = q0 * is, x = q1 * is, y = q2 * is, z = q3 * is;
    vx[0] = 1.0f - 2.0f * (y * y + z * z);
    vx[1] = 2.0f * (x * y + w * z);
    vx[2] = 2.0f * (x * z - w * y);
    vy[0] = 2.0f * (x * y - w * z);
    vy[1] = 1.0f - 2.0f * (x * x + z * z);
    vy[2] = 2.0f * (y * z + w * x);
    n[0] = 2.0f * (x * z + w * y);
    n[1] = 2.0f * (y * z - w * x);
    n[2] = 1.0f - 2.0f * (x * x + y * y);
    for (int i = 0; i < 3; ++i) {
        o->pc[i] = rowf(R, i, pf) + R[4 * i + 3];
        o->vxc[i] = rowf(R, i, vx);
        o->vyc[i] = rowf(R, i, vy);
        o->nc[i] = rowf(R, i, n);
    }
    const int single_radii = flags & OR_SINGLE;
    o->r[0] = (float)r[0]; o->r[1] = (float)(single_radii ? r[0] : r[1]);
    o->r[2] = (float)r[2]; o->r[3] = (float)(single_radii ? r[2] : r[3]);
    return 1;
}

void or_bin_records(int K, int V,
                    const double* center, const double* quat, const double* radii,
                    const double* w2c, const double* intr, int H, int W,
                    int tile_w, int tile_h, double delta_d, double z_near_d, double z_far_d,
                    int flags, int* rect, double* key, float* key_f32)
{
    const int gauss = flags & OR_GAUSS;
    const float delta = (float)delta_d, z_near = (float)z_near_d, z_far = (float)z_far_d;
    for (int v = 0; v < V; ++v) {
        const double* Rt = w2c + 12 * v;
        float fx = (float)intr[4 * v + 0], fy = (float)intr[4 * v + 1];
        float cx = (float)intr[4 * v + 2], cy = (float)intr[4 * v + 3];
        for (int k = 0; k < K; ++k) {
            int* rc = rect + 4 * ((long)v * K + k);
            rc[0] = 0; rc[1] = 0; rc[2] = -1; rc[3] = -1;
            key[(long)v * K + k] = INFINITY;
            key_f32[(long)v * K + k] = INFINITY;
            frame_f32 f;
            if (!plane_frame_f32(center + 3 * k, quat + 4 * k, radii + 4 * k, Rt, flags, &f))
                continue;
            float exp_ = gauss ? f.r[0] * delta : f.r[0] + delta;
            float exm = gauss ? f.r[1] * delta : f.r[1] + delta;
            float eyp = gauss ? f.r[2] * delta : f.r[2] + delta;
            float eym = gauss ? f.r[3] * delta : f.r[3] + delta;
            /* corners in order (+x,+y), (-x,+y), (-x,-y), (+x,-y) */
            float ax[4] = {exp_, -exm, -exm, exp_};
            float ay[4] = {eyp, eyp, -eym, -eym};
            float C[4][3];
            for (int c = 0; c < 4; ++c)
                for (int i = 0; i < 3; ++i)
                    C[c][i] = (f.pc[i] + ax[c] * f.vxc[i]) + ay[c] * f.vyc[i];
            /* Sutherland-Hodgman against the half space z >= z_near */
            float P[8][3];
            int np = 0;
            for (int e = 0; e < 4; ++e) {
                const float* a = C[e];
                const float* b = C[(e + 1) & 3];
                int ina = a[2] >= z_near, inb = b[2] >= z_near;
                if (ina) { P[np][0] = a[0]; P[np][1] = a[1]; P[np][2] = a[2]; ++np; }
                if (ina != inb) {
                    float s = (z_near - a[2]) / (b[2] - a[2]);
                    P[np][0] = a[0] + s * (b[0] - a[0]);
                    P[np][1] = a[1] + s * (b[1] - a[1]);
                    P[np][2] = z_near;
                    ++np;
                }
            }
            if (np == 0) continue;
            float kmin = P[0][2];
            for (int i = 1; i < np; ++i) if (P[i][2] < kmin) kmin = P[i][2];
            if (!(kmin < z_far)) continue;
            float umin = 0, umax = 0, vmin = 0, vmax = 0;
            int bad = 0;
            for (int i = 0; i < np; ++i) {
                float iz = 1.0f / P[i][2];
                float u = fx * (P[i][0] * iz) + cx;
                float vv = fy * (P[i][1] * iz) + cy;
                if (isnan(u) || isnan(vv)) bad = 1;
                if (i == 0) { umin = umax = u; vmin = vmax = vv; }
                else {
                    if (u < umin) umin = u;
                    if (u > umax) umax = u;
                    if (vv < vmin) vmin = vv;
                    if (vv > vmax) vmax = vv;
                }
            }
            if (bad) continue;
            float px0 = floorf(umin) - 1.0f, px1 = floorf(umax) + 1.0f;
            float py0 = floorf(vmin) - 1.0f, py1 = floorf(vmax) + 1.0f;
            const float Wm = (float)(W - 1), Hm = (float)(H - 1);
            if (px1 < 0.0f || px0 > Wm || py1 < 0.0f || py0 > Hm) continue;
            if (px0 < 0.0f) px0 = 0.0f;
            if (py0 < 0.0f) py0 = 0.0f;
            if (px1 > Wm) px1 = Wm;
            if (py1 > Hm) py1 = Hm;
            rc[0] = (int)px0 / tile_w; rc[1] = (int)py0 / tile_h;
            rc[2] = (int)px1 / tile_w; rc[3] = (int)py1 / tile_h;
            key[(long)v * K + k] = (double)kmin;
            key_f32[(long)v * K + k] = kmin;
        }
    }
}

/* f32 camera-frame normal and offset of every (view, plane) record:         */
/* ns[4 (v K + k) + (0..2)] = n_c, ns[.. + 3] = n_c . p_c, from the FP32     */
/* frame of the binning specification above (zeros for a degenerate          */
/* quaternion).  The tile-list entry keys are computed from these.            */
void or_records_ns(int K, int V, const double* center, const double* quat, const double* radii,
                   const double* w2c, float* ns)
{
    for (int v = 0; v < V; ++v) {
        const double* Rt = w2c + 12 * v;
        for (int k = 0; k < K; ++k) {
            float* o = ns + 4 * ((long)v * K + k);
            frame_f32 f;
            if (!plane_frame_f32(center + 3 * k, quat + 4 * k, radii + 4 * k, Rt, 0, &f)) {
                o[0] = o[1] = o[2] = o[3] = 0.0f;
                continue;
            }
            o[0] = f.nc[0]; o[1] = f.nc[1]; o[2] = f.nc[2];
            o[3] = (f.nc[0] * f.pc[0] + f.nc[1] * f.pc[1]) + f.nc[2] * f.pc[2];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Per-(pixel, plane) evaluation of Eq. 4 and Eq. 6-9.                       */
typedef struct {
    int k;            /* plane index */
    double t, w;      /* depth and weight */
    double m, mX, mY; /* margins r - |P| */
    double PX, PY, den;
    double sX, sY;    /* radius on the side of P_X, P_Y (Eq. 7-8; Eq. 5 scales) */
    int branchX;      /* 1 if w came from the X side (w_X < w_Y) */
    /* FP32 rounding model (conditioning flags only; set by pixel_candidates):  */
    double kappa;     /* sum |d_i n_i| / |d . n|: condition number of Eq. 4's denominator */
    double eps_t;     /* size of an FP32 rounding effect on t                            */
    double eps_m;     /* size of an FP32 rounding effect on the active margin            */
} cand;

/* A composited pair whose Eq. 4 denominator is this ill-conditioned (the ray
   within about half a degree of the plane) carries an FP32 relative error of
   about eta * kappa into its gradient (t, and the chain through 1 / (d . n)):
   above 100 that passes a tenth of the 1e-3 gradient bar.                    */
#define OR_KAPPA_GRAD 100.0

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* w_X or w_Y of Eq. 7-8 with the clamp to 1 */
static double side_weight(double lambda, double m)
{
    double w = 2.0 * sigmoid(5.0 * lambda * m);
    return w < 1.0 ? w : 1.0;
}

/* Evaluates plane pc at ray d.  Returns 1 and fills c when t is in range and
   the ray is not grazing; the weight filter is applied by the caller.
   With gauss, w is the Gaussian of Eq. 5 in the plane's frame, its scales
   the one-sided radii: w = exp(-(P_X^2 / sigma_X^2 + P_Y^2 / sigma_Y^2) / 2)
   with sigma_X = r^x+ if P_X > 0 else r^x- (likewise Y).                    */
static int eval_pair(const plane_cam* pc, const double d[3], double lambda,
                     double z_near, double z_far, int gauss, cand* c)
{
    double den = dot3(d, pc->nc);
    if (!(fabs(den) > 1e-6)) return 0;
    double t = dot3(pc->pc, pc->nc) / den;
    if (!(t > z_near && t < z_far)) return 0;
    double x[3] = {t * d[0] - pc->pc[0], t * d[1] - pc->pc[1], t * d[2] - pc->pc[2]};
    double PX = dot3(x, pc->vxc), PY = dot3(x, pc->vyc);
    double rX = PX > 0.0 ? pc->r[0] : pc->r[1];
    double rY = PY > 0.0 ? pc->r[2] : pc->r[3];
    double mX = rX - fabs(PX), mY = rY - fabs(PY);
    c->t = t; c->den = den; c->PX = PX; c->PY = PY; c->mX = mX; c->mY = mY;
    c->sX = rX; c->sY = rY;
    if (gauss) {
        double qf = (PX / rX) * (PX / rX) + (PY / rY) * (PY / rY);
        c->w = exp(-0.5 * qf);
        c->branchX = 0;
        c->m = 0.0;
        return 1;
    }
    double wX = side_weight(lambda, mX), wY = side_weight(lambda, mY);
    if (wX < wY) { c->w = wX; c->branchX = 1; c->m = mX; }
    else { c->w = wY; c->branchX = 0; c->m = mY; }
    return 1;
}

static int cand_cmp(const void* a, const void* b)
{
    const cand* x = (const cand*)a;
    const cand* y = (const cand*)b;
    if (x->t < y->t) return -1;
    if (x->t > y->t) return 1;
    return (x->k > y->k) - (x->k < y->k);
}

typedef struct {
    double lambda, w_min, z_near, z_far;
    int M, flags;
} or_set;

/* Gathers, filters and sorts the candidates of one pixel.  Returns the
   number of candidates (before the top-M cut).  Also reports the smallest
   distance of any in-range plane's margin to the filter edge -delta, the
   closest pair of sorted depths, etc., for the conditioning flags.  out    
   has room for K candidates, so no plane is ever left out.                 */
static int pixel_candidates(const plane_cam* pcs, int K, const double d[3], const or_set* S,
                            double delta, double eta, cand* out, int* near_filter)
{
    int nc = 0;
    *near_filter = 0;
    for (int k = 0; k < K; ++k) {
        if (!pcs[k].ok) continue;
        cand c;
        if (!eval_pair(&pcs[k], d, S->lambda, S->z_near, S->z_far, S->flags & OR_GAUSS, &c)) continue;
        /* FP32 rounding of Eq. 4: the denominator d . n loses kappa ulps to cancellation
           at grazing incidence, so t carries a relative error of about eta kappa and the
           margin P = t (d . v) - a the same times t |d . v| */
        const double* n_ = pcs[k].nc;
        c.kappa = ((fabs(d[0] * n_[0]) + fabs(d[1] * n_[1])) + fabs(n_[2])) / fabs(c.den);
        double dv = (S->flags & OR_GAUSS)
                        ? fmax(fabs(dot3(d, pcs[k].vxc)), fabs(dot3(d, pcs[k].vyc)))
                        : fabs(dot3(d, c.branchX ? pcs[k].vxc : pcs[k].vyc));
        c.eps_t = eta * (1.0 + fabs(c.t)) * c.kappa;
        c.eps_m = eta * (1.0 + fabs(c.t) + pcs[k].pcn) + eta * fabs(c.t) * dv * (c.kappa - 1.0);
        double eps = c.eps_m;
        if (S->flags & OR_GAUSS) {
            /* w moves by about w (|P_X| / sigma_X^2 + |P_Y| / sigma_Y^2) eps */
            double dw = c.w * (fabs(c.PX) / (c.sX * c.sX) + fabs(c.PY) / (c.sY * c.sY)) * eps;
            if (fabs(c.w - S->w_min) < dw) *near_filter = 1;
        } else if (fabs(c.m + delta) < eps) *near_filter = 1;
        double et = fmax(eps, c.eps_t);
        if (fabs(c.t - S->z_near) < et || fabs(c.t - S->z_far) < et) *near_filter = 1;
        if (!(c.w >= S->w_min)) continue;
        c.k = k;
        out[nc++] = c;     /* out holds K entries: one per plane at most */
    }
    qsort(out, nc, sizeof(cand), cand_cmp);
    return nc;
}

/* ------------------------------------------------------------------------ */
/* Forward render (Eq. 11-13), brute force over all planes.                  */
/* Outputs per pixel: depth, normal (camera frame), alpha = sum T_j w_j,     */
/* n_sel = number composited (<= M), n_cand = number of (plane) candidates   */
/* with w >= w_min and t in range (the algorithmic pair count), and ill:     */
/*   bit 0: FP32 rounding could move D or N by more than tol_d/2 or        */
/*          tol_n/2, or flip the filter, the depth order or the z range.     */
/*          The rounding model: a margin error of eta (1 + t + |p_c|) +     */
/*          eta t |d . v| (kappa - 1) and a depth error of eta (1 + t) kappa, */
/*          kappa = sum |d_i n_i| / |d . n| (the denominator of Eq. 4 loses  */
/*          precision when the ray grazes the plane);                        */
/*   bit 1: bit 0, or the min / sign branch of a weighted, partly            */
/*          transparent entry is within its margin error of flipping, or a  */
/*          composited entry has kappa > OR_KAPPA_GRAD (gradients only);     */
/*   bit 2: of bit 0, the discontinuous part: the filter, the depth order or */
/*          the z range could flip;                                          */
/*   bit 3: of bit 1, the part that is not a smooth value error (a min /     */
/*          sign branch could flip, or a composited entry grazes).           */
/* sens (optional) [pixel][2]: the first-order size of those rounding        */
/* effects on D and on the largest component of N, sum over the composited  */
/* pairs of |dD/dm_j| times the margin error (likewise N), from the adjoint  */
/* of Eq. 11-13.                                                             */
/* Rows [row0, row1) of every view are rendered; others are left untouched.  */
void or_render(int K, int V, const double* center, const double* quat, const double* radii,
               const double* w2c, const double* intr, int H, int W,
               double lambda, double w_min, double z_near, double z_far, int M, int flags,
               double delta, double eta, double tol_d, double tol_n, int row0, int row1,
               double* depth, double* normal, double* alpha, int* n_sel, int* n_cand, int* ill,
               double* sens)
{
    or_set S = {lambda, w_min, z_near, z_far, M, flags};
    const int gauss = flags & OR_GAUSS;
    plane_cam* pcs = (plane_cam*)malloc(sizeof(plane_cam) * (size_t)(K > 0 ? K : 1));
    for (int v = 0; v < V; ++v) {
        const double* Rt = w2c + 12 * v;
        for (int k = 0; k < K; ++k)
            plane_to_cam(center + 3 * k, quat + 4 * k, radii + 4 * k, Rt, flags, &pcs[k]);
        double fx = intr[4 * v + 0], fy = intr[4 * v + 1];
        double cx = intr[4 * v + 2], cy = intr[4 * v + 3];
#pragma omp parallel
        {
            /* every plane can be a candidate of one pixel: room for all K */
            cand* cs = (cand*)malloc(sizeof(cand) * (size_t)(K > 0 ? K : 1));
            double* Tj = (double*)malloc(sizeof(double) * (size_t)(M + 1));
#pragma omp for schedule(dynamic, 1)
            for (int j = row0; j < row1; ++j) {
                for (int i = 0; i < W; ++i) {
                    long pix = ((long)v * H + j) * W + i;
                    double d[3] = {((double)i + 0.5 - cx) / fx, ((double)j + 0.5 - cy) / fy, 1.0};
                    int near_filter;
                    int nc = pixel_candidates(pcs, K, d, &S, delta, eta, cs, &near_filter);
                    int ns = nc < M ? nc : M;
                    double T = 1.0, D = 0.0, N[3] = {0, 0, 0}, A = 0.0;
                    for (int s = 0; s < ns; ++s) {
                        const plane_cam* p = &pcs[cs[s].k];
                        double tw = T * cs[s].w;
                        Tj[s] = T;
                        D += tw * cs[s].t;
                        N[0] += tw * p->nc[0]; N[1] += tw * p->nc[1]; N[2] += tw * p->nc[2];
                        A += tw;
                        T = T * (1.0 - cs[s].w);
                    }
                    /* conditioning */
                    int flip = near_filter, bad_grad = 0;
                    for (int s = 0; s + 1 < nc && s < M; ++s) {
                        double e = fmax(eta * (1.0 + fabs(cs[s + 1].t)), fmax(cs[s].eps_t, cs[s + 1].eps_t));
                        if (cs[s + 1].t - cs[s].t < e) flip = 1;
                    }
                    int bad_val = flip;
                    /* sensitivity of D, N to the margins: back-to-front sums */
                    double Ab = 0.0, Bb[3] = {0, 0, 0};
                    double sD = 0.0, sN[3] = {0, 0, 0};
                    for (int s = ns - 1; s >= 0; --s) {
                        const plane_cam* p = &pcs[cs[s].k];
                        double w = cs[s].w, t = cs[s].t, m = cs[s].m;
                        double e = cs[s].eps_m;
                        double slope;
                        if (gauss)                                  /* |dw/dP| summed over both axes */
                            slope = w * (fabs(cs[s].PX) / (cs[s].sX * cs[s].sX) +
                                         fabs(cs[s].PY) / (cs[s].sY * cs[s].sY));
                        else if (fabs(m) < e) slope = 2.5 * lambda; /* max of dw/dm near the kink */
                        else if (m < 0.0) {
                            double sg = sigmoid(5.0 * lambda * m);
                            slope = 10.0 * lambda * sg * (1.0 - sg);
                        } else slope = 0.0;
                        double gD = Tj[s] * (t - Ab);
                        sD += fabs(gD) * slope * e;
                        for (int c = 0; c < 3; ++c) sN[c] += fabs(Tj[s] * (p->nc[c] - Bb[c])) * slope * e;
                        if (Tj[s] > 0.0 && cs[s].kappa > OR_KAPPA_GRAD) bad_grad = 1;
                        if (gauss) {
                            /* the side (sigma) choice of P_X or P_Y flips near 0 */
                            if (Tj[s] > 0.0 && (fabs(cs[s].PX) < e || fabs(cs[s].PY) < e)) bad_grad = 1;
                        } else if (Tj[s] > 0.0 && m < e) {
                            if (fabs(cs[s].mX - cs[s].mY) < e) bad_grad = 1;
                            double Pa = cs[s].branchX ? cs[s].PX : cs[s].PY;
                            if (fabs(Pa) < e) bad_grad = 1;
                        }
                        Ab = w * t + (1.0 - w) * Ab;
                        for (int c = 0; c < 3; ++c) Bb[c] = w * p->nc[c] + (1.0 - w) * Bb[c];
                    }
                    if (sD > 0.5 * tol_d) bad_val = 1;
                    if (sN[0] > 0.5 * tol_n || sN[1] > 0.5 * tol_n || sN[2] > 0.5 * tol_n) bad_val = 1;
                    depth[pix] = D;
                    normal[3 * pix + 0] = N[0]; normal[3 * pix + 1] = N[1]; normal[3 * pix + 2] = N[2];
                    if (alpha) alpha[pix] = A;
                    if (n_sel) n_sel[pix] = ns;
                    if (n_cand) n_cand[pix] = nc;
                    if (ill) ill[pix] = (bad_val ? 3 : 0) | (bad_grad ? 10 : 0) | (flip ? 4 : 0);
                    if (sens) {
                        sens[2 * pix] = sD;
                        sens[2 * pix + 1] = fmax(sN[0], fmax(sN[1], sN[2]));
                    }
                }
            }
            free(cs);
            free(Tj);
        }
    }
    free(pcs);
}

/* ------------------------------------------------------------------------ */
/* Render loss, Eq. 14, with its gradient with respect to D and N.           */
/* Pixels with gt_depth <= 0 are not supervised.  view_sums[v] =             */
/* (sum |1 - N.N*|, sum ||N - N*||_1, sum |D - D*|, number of valid pixels). */
/* Returns the total loss.  sgn(0) = 0.                                       */
static double sgn(double x) { return (x > 0.0) - (x < 0.0); }

double or_loss(int V, int H, int W, const double* depth, const double* normal,
               const double* gt_depth, const double* gt_normal,
               double a_cos, double a_l1n, double a_depth,
               double* dLdD, double* dLdN, double* view_sums)
{
    double total = 0.0;
    long HW = (long)H * W;
    for (int v = 0; v < V; ++v) {
        double sc = 0, sl = 0, sd = 0, cnt = 0;
        for (long p = 0; p < HW; ++p) {
            long pix = (long)v * HW + p;
            const double* N = normal + 3 * pix;
            const double* Ns = gt_normal + 3 * pix;
            if (!(gt_depth[pix] > 0.0)) {
                dLdD[pix] = 0.0;
                dLdN[3 * pix] = dLdN[3 * pix + 1] = dLdN[3 * pix + 2] = 0.0;
                continue;
            }
            double cosv = 1.0 - dot3(N, Ns);
            double l1 = fabs(N[0] - Ns[0]) + fabs(N[1] - Ns[1]) + fabs(N[2] - Ns[2]);
            double dd = depth[pix] - gt_depth[pix];
            sc += fabs(cosv); sl += l1; sd += fabs(dd); cnt += 1.0;
            dLdD[pix] = a_depth * sgn(dd);
            for (int c = 0; c < 3; ++c)
                dLdN[3 * pix + c] = -a_cos * sgn(cosv) * Ns[c] + a_l1n * sgn(N[c] - Ns[c]);
        }
        if (view_sums) {
            view_sums[4 * v + 0] = sc; view_sums[4 * v + 1] = sl;
            view_sums[4 * v + 2] = sd; view_sums[4 * v + 3] = cnt;
        }
        total += a_cos * sc + a_l1n * sl + a_depth * sd;
    }
    return total;
}

/* ------------------------------------------------------------------------ */
/* Backward: gradient of sum_pixels (dLdD . D + dLdN . N) with respect to    */
/* every plane's center, quaternion and radii.  Per pixel the composited     */
/* list is rebuilt, the adjoint of Eq. 11-13 is taken back to front          */
/*   A_{n+1} = 0, A_j = w_j t_j + (1 - w_j) A_{j+1}                          */
/*   dD/dw_j = T_j (t_j - A_{j+1}),  dD/dt_j = T_j w_j,  dN/dn_j = T_j w_j   */
/* (no division by 1 - w), and chained through Eq. 9, 7-8, 6, 4 and 2-3 to   */
/* the world parameters.  The clamp min(1, .) has derivative 0 at m >= 0.   */
/* g_abs (optional, [K][11]): per plane and parameter, the sum over pixels of the   */
/* absolute per-pixel contributions; its ratio to |g| measures how much the sum    */
/* cancels, i.e. how far rounding of the parts can move the total.                 */
void or_backward(int K, int V, const double* center, const double* quat, const double* radii,
                 const double* w2c, const double* intr, int H, int W,
                 double lambda, double w_min, double z_near, double z_far, int M, int flags,
                 const double* dLdD, const double* dLdN,
                 double* g_center, double* g_quat, double* g_radii, double* g_abs)
{
    or_set S = {lambda, w_min, z_near, z_far, M, flags};
    const int single_radii = flags & OR_SINGLE, gauss = flags & OR_GAUSS;
    memset(g_center, 0, sizeof(double) * 3 * (size_t)K);
    memset(g_quat, 0, sizeof(double) * 4 * (size_t)K);
    memset(g_radii, 0, sizeof(double) * 4 * (size_t)K);
    plane_cam* pcs = (plane_cam*)malloc(sizeof(plane_cam) * (size_t)(K > 0 ? K : 1));
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    double* acc = (double*)calloc((size_t)nthreads * 11 * (size_t)K, sizeof(double));
    double* acc_abs = g_abs ? (double*)calloc((size_t)nthreads * 11 * (size_t)K, sizeof(double)) : NULL;
    /* per-view camera-frame gradient accumulators, chained to world per view */
    for (int v = 0; v < V; ++v) {
        const double* Rt = w2c + 12 * v;
        for (int k = 0; k < K; ++k)
            plane_to_cam(center + 3 * k, quat + 4 * k, radii + 4 * k, Rt, flags, &pcs[k]);
        double fx = intr[4 * v + 0], fy = intr[4 * v + 1];
        double cx = intr[4 * v + 2], cy = intr[4 * v + 3];
#pragma omp parallel
        {
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
            double* my = acc + (size_t)tid * 11 * K;
            /* every plane can be a candidate of one pixel: room for all K */
            cand* cs = (cand*)malloc(sizeof(cand) * (size_t)(K > 0 ? K : 1));
            double* Tj = (double*)malloc(sizeof(double) * (size_t)(M + 1));
#pragma omp for schedule(static)
            for (int j = 0; j < H; ++j) {
                for (int i = 0; i < W; ++i) {
                    long pix = ((long)v * H + j) * W + i;
                    double gD = dLdD[pix];
                    const double* gN = dLdN + 3 * pix;
                    if (gD == 0.0 && gN[0] == 0.0 && gN[1] == 0.0 && gN[2] == 0.0) continue;
                    double d[3] = {((double)i + 0.5 - cx) / fx, ((double)j + 0.5 - cy) / fy, 1.0};
                    int nf;
                    int nc = pixel_candidates(pcs, K, d, &S, 0.0, 0.0, cs, &nf);
                    int ns = nc < M ? nc : M;
                    double T = 1.0;
                    for (int s = 0; s < ns; ++s) { Tj[s] = T; T = T * (1.0 - cs[s].w); }
                    double A = 0.0, B[3] = {0, 0, 0};
                    for (int s = ns - 1; s >= 0; --s) {
                        const cand* c = &cs[s];
                        const plane_cam* p = &pcs[c->k];
                        double w = c->w, t = c->t;
                        double gw = Tj[s] * (gD * (t - A) + gN[0] * (p->nc[0] - B[0]) +
                                             gN[1] * (p->nc[1] - B[1]) + gN[2] * (p->nc[2] - B[2]));
                        double gt = Tj[s] * w * gD;
                        double gnc[3] = {Tj[s] * w * gN[0], Tj[s] * w * gN[1], Tj[s] * w * gN[2]};
                        A = w * t + (1.0 - w) * A;
                        for (int q = 0; q < 3; ++q) B[q] = w * p->nc[q] + (1.0 - w) * B[q];
                        /* Eq. 7-9: w = min(1, 2 sigmoid(5 lambda m)) on the active side */
                        double gm = 0.0;
                        if (c->m < 0.0) {
                            double sg = sigmoid(5.0 * lambda * c->m);
                            gm = gw * 10.0 * lambda * sg * (1.0 - sg);
                        }
                        double gr[4] = {0, 0, 0, 0};
                        double gPX = 0.0, gPY = 0.0;
                        if (gauss) {
                            /* Eq. 5: w = exp(-(P_X^2 / s_X^2 + P_Y^2 / s_Y^2) / 2) */
                            double sx2 = c->sX * c->sX, sy2 = c->sY * c->sY;
                            gPX = -gw * w * c->PX / sx2;
                            gPY = -gw * w * c->PY / sy2;
                            gr[c->PX > 0.0 ? 0 : 1] += gw * w * c->PX * c->PX / (sx2 * c->sX);
                            gr[c->PY > 0.0 ? 2 : 3] += gw * w * c->PY * c->PY / (sy2 * c->sY);
                        } else if (c->branchX) {
                            /* m_X = r_X - |P_X| */
                            if (c->PX > 0.0) gr[0] += gm; else gr[1] += gm;
                            gPX = -gm * sgn(c->PX);
                        } else {
                            if (c->PY > 0.0) gr[2] += gm; else gr[3] += gm;
                            gPY = -gm * sgn(c->PY);
                        }
                        if (single_radii) { gr[0] += gr[1]; gr[1] = 0.0; gr[2] += gr[3]; gr[3] = 0.0; }
                        /* Eq. 6: P = (t d - p_c) . v_c */
                        double x[3] = {t * d[0] - p->pc[0], t * d[1] - p->pc[1], t * d[2] - p->pc[2]};
                        double gpc[3], gvxc[3], gvyc[3];
                        gt += gPX * dot3(d, p->vxc) + gPY * dot3(d, p->vyc);
                        for (int q = 0; q < 3; ++q) {
                            gpc[q] = -gPX * p->vxc[q] - gPY * p->vyc[q];
                            gvxc[q] = gPX * x[q];
                            gvyc[q] = gPY * x[q];
                        }
                        /* Eq. 4: t = (p_c . n_c) / (d . n_c) */
                        double den = c->den;
                        for (int q = 0; q < 3; ++q) {
                            gpc[q] += gt * p->nc[q] / den;
                            gnc[q] += gt * (p->pc[q] - t * d[q]) / den;
                        }
                        /* camera frame -> world: p_c = R p + t, a_c = R a */
                        double gp[3], gvx[3], gvy[3], gn[3];
                        rot_apply_T(Rt, gpc, gp);
                        rot_apply_T(Rt, gvxc, gvx);
                        rot_apply_T(Rt, gvyc, gvy);
                        rot_apply_T(Rt, gnc, gn);
                        /* Eq. 2-3: columns of the Hamilton matrix of qhat */
                        double w_ = p->qhat[0], xq = p->qhat[1], yq = p->qhat[2], zq = p->qhat[3];
                        /* G[i][c]: gradient w.r.t. R_ic, column c = (vx, vy, n)[c] */
                        double G[3][3];
                        for (int q = 0; q < 3; ++q) { G[q][0] = gvx[q]; G[q][1] = gvy[q]; G[q][2] = gn[q]; }
                        double dRw[3][3] = {{0, -2 * zq, 2 * yq}, {2 * zq, 0, -2 * xq}, {-2 * yq, 2 * xq, 0}};
                        double dRx[3][3] = {{0, 2 * yq, 2 * zq}, {2 * yq, -4 * xq, -2 * w_}, {2 * zq, 2 * w_, -4 * xq}};
                        double dRy[3][3] = {{-4 * yq, 2 * xq, 2 * w_}, {2 * xq, 0, 2 * zq}, {-2 * w_, 2 * zq, -4 * yq}};
                        double dRz[3][3] = {{-4 * zq, -2 * w_, 2 * xq}, {2 * w_, -4 * zq, 2 * yq}, {2 * xq, 2 * yq, 0}};
                        double gqh[4] = {0, 0, 0, 0};
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b) {
                                gqh[0] += G[a][b] * dRw[a][b];
                                gqh[1] += G[a][b] * dRx[a][b];
                                gqh[2] += G[a][b] * dRy[a][b];
                                gqh[3] += G[a][b] * dRz[a][b];
                            }
                        /* qhat = q / |q| */
                        double proj = gqh[0] * w_ + gqh[1] * xq + gqh[2] * yq + gqh[3] * zq;
                        double gq[4] = {(gqh[0] - w_ * proj) / p->qs, (gqh[1] - xq * proj) / p->qs,
                                        (gqh[2] - yq * proj) / p->qs, (gqh[3] - zq * proj) / p->qs};
                        double* o = my + 11 * (size_t)c->k;
                        for (int q = 0; q < 3; ++q) o[q] += gp[q];
                        for (int q = 0; q < 4; ++q) o[3 + q] += gq[q];
                        for (int q = 0; q < 4; ++q) o[7 + q] += gr[q];
                        if (acc_abs) {
                            double* oa = acc_abs + (size_t)tid * 11 * K + 11 * (size_t)c->k;
                            for (int q = 0; q < 3; ++q) oa[q] += fabs(gp[q]);
                            for (int q = 0; q < 4; ++q) oa[3 + q] += fabs(gq[q]);
                            for (int q = 0; q < 4; ++q) oa[7 + q] += fabs(gr[q]);
                        }
                    }
                }
            }
            free(cs);
            free(Tj);
        }
    }
    for (int tid = 0; tid < nthreads; ++tid) {
        const double* my = acc + (size_t)tid * 11 * K;
        for (int k = 0; k < K; ++k) {
            for (int q = 0; q < 3; ++q) g_center[3 * k + q] += my[11 * k + q];
            for (int q = 0; q < 4; ++q) g_quat[4 * k + q] += my[11 * k + 3 + q];
            for (int q = 0; q < 4; ++q) g_radii[4 * k + q] += my[11 * k + 7 + q];
        }
    }
    if (acc_abs) {
        memset(g_abs, 0, sizeof(double) * 11 * (size_t)K);
        for (int tid = 0; tid < nthreads; ++tid)
            for (size_t e = 0; e < 11 * (size_t)K; ++e) g_abs[e] += acc_abs[(size_t)tid * 11 * K + e];
        free(acc_abs);
    }
    free(acc);
    free(pcs);
}

/* ------------------------------------------------------------------------ */
/* Exact ray caster of hard rectangles: nearest plane whose rectangle        */
/* (|P_X| <= r_X, |P_Y| <= r_Y, one-sided radii by sign) the pixel ray hits  */
/* with z_near < t < z_far.  Used to make ground-truth depth and normal      */
/* maps of synthetic rooms.  Pixels that hit nothing get depth 0, normal 0   */
/* and plane_id -1.  Rows [row0, row1) of every view are cast.              */
void or_raycast(int K, int V, const double* center, const double* quat, const double* radii,
                const double* w2c, const double* intr, int H, int W, double z_near, double z_far,
                int row0, int row1, double* depth, double* normal, int* plane_id)
{
    plane_cam* pcs = (plane_cam*)malloc(sizeof(plane_cam) * (size_t)(K > 0 ? K : 1));
    for (int v = 0; v < V; ++v) {
        const double* Rt = w2c + 12 * v;
        for (int k = 0; k < K; ++k)
            plane_to_cam(center + 3 * k, quat + 4 * k, radii + 4 * k, Rt, 0, &pcs[k]);
        double fx = intr[4 * v + 0], fy = intr[4 * v + 1];
        double cx = intr[4 * v + 2], cy = intr[4 * v + 3];
#pragma omp parallel for schedule(dynamic, 1)
        for (int j = row0; j < row1; ++j) {
            for (int i = 0; i < W; ++i) {
                long pix = ((long)v * H + j) * W + i;
                double d[3] = {((double)i + 0.5 - cx) / fx, ((double)j + 0.5 - cy) / fy, 1.0};
                double best = INFINITY;
                int bk = -1;
                for (int k = 0; k < K; ++k) {
                    const plane_cam* p = &pcs[k];
                    if (!p->ok) continue;
                    double den = dot3(d, p->nc);
                    if (!(fabs(den) > 1e-6)) continue;
                    double t = dot3(p->pc, p->nc) / den;
                    if (!(t > z_near && t < z_far)) continue;
                    double x[3] = {t * d[0] - p->pc[0], t * d[1] - p->pc[1], t * d[2] - p->pc[2]};
                    double PX = dot3(x, p->vxc), PY = dot3(x, p->vyc);
                    double rX = PX > 0.0 ? p->r[0] : p->r[1];
                    double rY = PY > 0.0 ? p->r[2] : p->r[3];
                    if (fabs(PX) > rX || fabs(PY) > rY) continue;
                    if (t < best || (t == best && k < bk)) { best = t; bk = k; }
                }
                if (bk < 0) {
                    depth[pix] = 0.0;
                    normal[3 * pix] = normal[3 * pix + 1] = normal[3 * pix + 2] = 0.0;
                } else {
                    depth[pix] = best;
                    for (int c = 0; c < 3; ++c) normal[3 * pix + c] = pcs[bk].nc[c];
                }
                if (plane_id) plane_id[pix] = bk;
            }
        }
    }
    free(pcs);
}

/* ------------------------------------------------------------------------ */
/* Adam (Kingma & Ba), bias-corrected, as used in Sec. 3.3 with lr = 1e-3.   */
/* After the update, values below clamp_min are raised to it (NaN: none).    */
void or_adam(long n, double* param, const double* grad, double* m, double* v,
             double lr, double b1, double b2, double eps, int step, double clamp_min)
{
    double bc1 = 1.0 - pow(b1, (double)step);
    double bc2 = 1.0 - pow(b2, (double)step);
    for (long i = 0; i < n; ++i) {
        double g = grad[i];
        m[i] = b1 * m[i] + (1.0 - b1) * g;
        v[i] = b2 * v[i] + (1.0 - b2) * g * g;
        double mh = m[i] / bc1, vh = v[i] / bc2;
        param[i] -= lr * mh / (sqrt(vh) + eps);
        if (!isnan(clamp_min) && param[i] < clamp_min) param[i] = clamp_min;
    }
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the parallel regions that follow (timing on one core). */
void or_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
