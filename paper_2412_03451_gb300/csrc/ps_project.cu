// ps_project.cu -- view planning (host), projection/culling, Adam.
//
// Projection follows Sec. 3.1 (Eq. 2-3: v^x, v^y, n are the columns of the
// rotation matrix of the normalised quaternion) and Sec. 3.2 (Eq. 4: rays from
// the camera centre, so planes are moved into the camera frame once per view).
// The record, the tile rectangle and the depth key are computed in FP32 with
// correctly rounded __fadd_rn/__fsub_rn/__fmul_rn/__fdiv_rn/__fsqrt_rn only, in
// a fixed order, so that they are reproducible bit for bit by any IEEE
// implementation of the same formula (divisions by |q| and by a corner's z are
// one reciprocal and products).  FP32 rather than FP64: this GPU's FP64 rate is
// a small fraction of its FP32 rate, and the rectangle is a conservative bound
// (widened by delta, padded by a pixel) whose exact value only has to agree
// between implementations.
#include <math.h>
#include <string.h>
#include "ps_internal.cuh"

using namespace ps;

extern "C" int ps_version(void) { return 1; }

extern "C" const char* ps_status_string(ps_status s)
{
    switch (s) {
    case PS_OK: return "ok";
    case PS_ERR_ARG: return "invalid argument";
    case PS_ERR_CUDA: return "CUDA error";
    case PS_ERR_CAPACITY: return "tile-list capacity exceeded";
    case PS_ERR_TIMEOUT: return "device wait timed out";
    case PS_ERR_NONFINITE: return "non-finite or zero-norm plane parameters";
    }
    return "unknown status";
}

extern "C" ps_status ps_plan_views(int n_views, const int* H, const int* W, const int* scene_of_view,
                                   int n_scenes, const int* plane_ptr, const float* w2c,
                                   const float* intr, int tile_w, int tile_h, ps_view* views_out,
                                   ps_frame* frame_out)
{
    if (n_views <= 0 || n_scenes <= 0 || !H || !W || !scene_of_view || !plane_ptr || !w2c ||
        !intr || !views_out || !frame_out)
        return PS_ERR_ARG;
    if (tile_w <= 0 || tile_h <= 0 || tile_w * tile_h > 1024) return PS_ERR_ARG;
    if (plane_ptr[0] != 0) return PS_ERR_ARG;
    for (int s = 0; s < n_scenes; ++s)
        if (plane_ptr[s + 1] < plane_ptr[s]) return PS_ERR_ARG;
    long long tiles = 0, recs = 0, pix = 0;
    int maxK = 0;
    for (int v = 0; v < n_views; ++v) {
        int s = scene_of_view[v];
        if (s < 0 || s >= n_scenes) return PS_ERR_ARG;
        if (v > 0 && s < scene_of_view[v - 1]) return PS_ERR_ARG;
        if (H[v] <= 0 || W[v] <= 0) return PS_ERR_ARG;
        ps_view& o = views_out[v];
        memset(&o, 0, sizeof(o));
        memcpy(o.w2c, w2c + 12 * (size_t)v, 12 * sizeof(float));
        o.fx = intr[4 * v + 0]; o.fy = intr[4 * v + 1];
        o.cx = intr[4 * v + 2]; o.cy = intr[4 * v + 3];
        if (!(o.fx != 0.f) || !(o.fy != 0.f)) return PS_ERR_ARG;
        o.H = H[v]; o.W = W[v];
        o.tiles_x = (W[v] + tile_w - 1) / tile_w;
        o.tiles_y = (H[v] + tile_h - 1) / tile_h;
        o.tile_off = (int)tiles;
        o.rec_off = (int)recs;
        o.plane_off = plane_ptr[s];
        o.K = plane_ptr[s + 1] - plane_ptr[s];
        o.pix_off = pix;
        o.gt_off = pix;
        o.scene = s;
        tiles += (long long)o.tiles_x * o.tiles_y;
        recs += o.K;
        pix += (long long)H[v] * W[v];
        if (o.K > maxK) maxK = o.K;
        if (tiles >= (1LL << 30) || recs >= (1LL << 30) || 3 * pix >= (1LL << 40))
            return PS_ERR_ARG;
    }
    frame_out->n_views = n_views;
    frame_out->n_records = (int)recs;
    frame_out->n_tiles = (int)tiles;
    frame_out->max_K = maxK;
    frame_out->n_pixels = pix;
    frame_out->views = nullptr;
    return PS_OK;
}

// ---------------------------------------------------------------------------
// Projection / culling.

namespace {

__device__ __forceinline__ float ad(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sb(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float ml(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float dv(float a, float b) { return __fdiv_rn(a, b); }

// rows of [R|t] applied to a (left-to-right sums)
__device__ __forceinline__ float row3(const float* R, int i, const float* a)
{
    return ad(ad(ml(R[4 * i + 0], a[0]), ml(R[4 * i + 1], a[1])), ml(R[4 * i + 2], a[2]));
}

struct ProjArgs {
    const float* center;
    const float* quat;
    const float* radii;
    const ps_view* views;
    float* rec;
    int4* rect;
    float* key;
    int* status;
    double delta;
    float z_near, z_far;
    const ps_step_state* d_state;
    int single_radii;
    int gauss;              // PS_GAUSSIAN: radii scaled by delta instead of widened
    int tile_w, tile_h;
};

__global__ void __launch_bounds__(128) k_project(ProjArgs a)
{
    const int v = blockIdx.y;
    const ps_view* vw = a.views + v;
    const int K = __ldg(&vw->K);
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int p = __ldg(&vw->plane_off) + k;
    const long long r = (long long)__ldg(&vw->rec_off) + k;

    float R[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) R[i] = __ldg(&vw->w2c[i]);
    const float fx = __ldg(&vw->fx), fy = __ldg(&vw->fy);
    const float cx = __ldg(&vw->cx), cy = __ldg(&vw->cy);
    const int H = __ldg(&vw->H), W = __ldg(&vw->W);

    float cf[3], qf[4], rf[4];
#pragma unroll
    for (int i = 0; i < 3; ++i) cf[i] = __ldg(&a.center[3 * (size_t)p + i]);
#pragma unroll
    for (int i = 0; i < 4; ++i) qf[i] = __ldg(&a.quat[4 * (size_t)p + i]);
#pragma unroll
    for (int i = 0; i < 4; ++i) rf[i] = __ldg(&a.radii[4 * (size_t)p + i]);
    bool finite = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) finite &= isfinite(cf[i]);
#pragma unroll
    for (int i = 0; i < 4; ++i) finite &= isfinite(qf[i]) && isfinite(rf[i]);

    int4 rc = make_int4(0, 0, -1, -1);
    float kf = INFINITY;
    float out[kRecFloats];
#pragma unroll
    for (int i = 0; i < kRecFloats; ++i) out[i] = 0.f;

    const float q0 = qf[0], q1 = qf[1], q2 = qf[2], q3 = qf[3];
    const float qs = __fsqrt_rn(ad(ad(ad(ml(q0, q0), ml(q1, q1)), ml(q2, q2)), ml(q3, q3)));
    bool ok = (qs > 0.f) && isfinite(qs);
    if (!finite || !ok) set_status(a.status, PS_ERR_NONFINITE);
    if (ok) {
        const float iq = dv(1.f, qs);
        const float w = ml(q0, iq), x = ml(q1, iq), y = ml(q2, iq), z = ml(q3, iq);
        float vxw[3], vyw[3], nw[3];
        vxw[0] = sb(1.f, ml(2.f, ad(ml(y, y), ml(z, z))));
        vxw[1] = ml(2.f, ad(ml(x, y), ml(w, z)));
        vxw[2] = ml(2.f, sb(ml(x, z), ml(w, y)));
        vyw[0] = ml(2.f, sb(ml(x, y), ml(w, z)));
        vyw[1] = sb(1.f, ml(2.f, ad(ml(x, x), ml(z, z))));
        vyw[2] = ml(2.f, ad(ml(y, z), ml(w, x)));
        nw[0] = ml(2.f, ad(ml(x, z), ml(w, y)));
        nw[1] = ml(2.f, sb(ml(y, z), ml(w, x)));
        nw[2] = sb(1.f, ml(2.f, ad(ml(x, x), ml(y, y))));
        float pc[3], vxc[3], vyc[3], nc[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            pc[i] = ad(row3(R, i, cf), R[4 * i + 3]);
            vxc[i] = row3(R, i, vxw);
            vyc[i] = row3(R, i, vyw);
            nc[i] = row3(R, i, nw);
        }
        // the Gaussian extent does not depend on lambda: the schedule's margin is not used
        const float delta = (float)((a.d_state && !a.gauss) ? __ldg(&a.d_state->delta) : a.delta);
        const float r0 = rf[0], r1 = a.single_radii ? rf[0] : rf[1];
        const float r2 = rf[2], r3 = a.single_radii ? rf[2] : rf[3];

        out[0] = nc[0]; out[1] = nc[1]; out[2] = nc[2];
        out[3] = ad(ad(ml(nc[0], pc[0]), ml(nc[1], pc[1])), ml(nc[2], pc[2]));
        out[4] = vxc[0]; out[5] = vxc[1]; out[6] = vxc[2];
        out[7] = ad(ad(ml(vxc[0], pc[0]), ml(vxc[1], pc[1])), ml(vxc[2], pc[2]));
        out[8] = vyc[0]; out[9] = vyc[1]; out[10] = vyc[2];
        out[11] = ad(ad(ml(vyc[0], pc[0]), ml(vyc[1], pc[1])), ml(vyc[2], pc[2]));
        out[12] = r0; out[13] = r1; out[14] = r2; out[15] = r3;

        // binning: widened quad (Eq. 5 weight: scaled quad), corners (+x,+y), (-x,+y),
        // (-x,-y), (+x,-y)
        const float exp_ = a.gauss ? ml(r0, delta) : ad(r0, delta);
        const float exm = a.gauss ? ml(r1, delta) : ad(r1, delta);
        const float eyp = a.gauss ? ml(r2, delta) : ad(r2, delta);
        const float eym = a.gauss ? ml(r3, delta) : ad(r3, delta);
        const float ax[4] = {exp_, -exm, -exm, exp_};
        const float ay[4] = {eyp, eyp, -eym, -eym};
        float C[4][3];
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int i = 0; i < 3; ++i)
                C[c][i] = ad(ad(pc[i], ml(ax[c], vxc[i])), ml(ay[c], vyc[i]));
        // clip against z >= z_near (Sutherland-Hodgman, one plane)
        float P[8][3];
        int np = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float* A = C[e];
            const float* B = C[(e + 1) & 3];
            const bool ina = A[2] >= a.z_near, inb = B[2] >= a.z_near;
            if (ina) { P[np][0] = A[0]; P[np][1] = A[1]; P[np][2] = A[2]; ++np; }
            if (ina != inb) {
                const float s = dv(sb(a.z_near, A[2]), sb(B[2], A[2]));
                P[np][0] = ad(A[0], ml(s, sb(B[0], A[0])));
                P[np][1] = ad(A[1], ml(s, sb(B[1], A[1])));
                P[np][2] = a.z_near;
                ++np;
            }
        }
        if (np > 0) {
            float kmin = P[0][2];
            for (int i = 1; i < np; ++i) if (P[i][2] < kmin) kmin = P[i][2];
            if (kmin < a.z_far) {
                float umin = 0.f, umax = 0.f, vmin = 0.f, vmax = 0.f;
                bool bad = false;
                for (int i = 0; i < np; ++i) {
                    const float iz = dv(1.f, P[i][2]);
                    const float u = ad(ml(fx, ml(P[i][0], iz)), cx);
                    const float vv = ad(ml(fy, ml(P[i][1], iz)), cy);
                    if (isnan(u) || isnan(vv)) bad = true;
                    if (i == 0) { umin = umax = u; vmin = vmax = vv; }
                    else {
                        if (u < umin) umin = u;
                        if (u > umax) umax = u;
                        if (vv < vmin) vmin = vv;
                        if (vv > vmax) vmax = vv;
                    }
                }
                if (!bad) {
                    float px0 = sb(floorf(umin), 1.f), px1 = ad(floorf(umax), 1.f);
                    float py0 = sb(floorf(vmin), 1.f), py1 = ad(floorf(vmax), 1.f);
                    const float Wm = (float)(W - 1), Hm = (float)(H - 1);
                    if (!(px1 < 0.f || px0 > Wm || py1 < 0.f || py0 > Hm)) {
                        if (px0 < 0.f) px0 = 0.f;
                        if (py0 < 0.f) py0 = 0.f;
                        if (px1 > Wm) px1 = Wm;
                        if (py1 > Hm) py1 = Hm;
                        rc.x = (int)px0 / a.tile_w; rc.y = (int)py0 / a.tile_h;
                        rc.z = (int)px1 / a.tile_w; rc.w = (int)py1 / a.tile_h;
                        kf = kmin;
                    }
                }
            }
        }
    }
    a.rect[r] = rc;
    a.key[r] = kf;
    float4* o4 = reinterpret_cast<float4*>(a.rec + (size_t)r * kRecFloats);
    o4[0] = make_float4(out[0], out[1], out[2], out[3]);
    o4[1] = make_float4(out[4], out[5], out[6], out[7]);
    o4[2] = make_float4(out[8], out[9], out[10], out[11]);
    o4[3] = make_float4(out[12], out[13], out[14], out[15]);
}

}  // namespace

extern "C" ps_status ps_project_cull(const ps_planes* planes, const ps_frame* frame,
                                     const ps_settings* s, float* rec, int* rect, float* key,
                                     int* d_status, ps_stream stream)
{
    if (!planes || !frame || !s || !rec || !rect || !key || !frame->views) return PS_ERR_ARG;
    if (!planes->center || !planes->quat || !planes->radii) return PS_ERR_ARG;
    if (frame->n_views <= 0 || frame->max_K < 0) return PS_ERR_ARG;
    if (s->tile_w <= 0 || s->tile_h <= 0) return PS_ERR_ARG;
    if (!(s->delta >= 0.0) && !s->d_state) return PS_ERR_ARG;
    if ((s->flags & PS_GAUSSIAN) && (!(s->delta > 0.0) || (s->flags & PS_HARD))) return PS_ERR_ARG;
    if (!(s->z_near > 0.f) || !(s->z_far > s->z_near)) return PS_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(rec) & 15) || (reinterpret_cast<uintptr_t>(rect) & 15))
        return PS_ERR_ARG;
    if (frame->max_K == 0 || frame->n_records == 0) return PS_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    ProjArgs a;
    a.center = planes->center; a.quat = planes->quat; a.radii = planes->radii;
    a.views = frame->views;
    a.rec = rec; a.rect = reinterpret_cast<int4*>(rect); a.key = key; a.status = d_status;
    a.delta = s->delta; a.z_near = s->z_near; a.z_far = s->z_far;
    a.d_state = s->d_state;
    a.single_radii = (s->flags & PS_SINGLE_RADII) ? 1 : 0;
    a.gauss = (s->flags & PS_GAUSSIAN) ? 1 : 0;
    a.tile_w = s->tile_w; a.tile_h = s->tile_h;
    dim3 grid((frame->max_K + 127) / 128, frame->n_views);
    k_project<<<grid, 128, 0, st>>>(a);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

// ---------------------------------------------------------------------------
// Adam.

namespace {
__global__ void k_step_advance(ps_step_state* st, const ps_step_state* sched, int n, int* iter)
{
    const int i = *iter;
    *st = sched[i < n ? i : n - 1];
    *iter = i + 1;
}

__global__ void k_adam_state(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                             float* __restrict__ v, long long n, float lr, float b1, float b2,
                             float eps, const ps_step_state* __restrict__ st, float clamp_min,
                             long long clamp_from)
{
    const float bc1 = __ldg(&st->bc1), bc2 = __ldg(&st->bc2);
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / bc1, vh = vi / bc2;
        float pi = p[i] - lr * mh / (sqrtf(vh) + eps);
        if (i >= clamp_from && pi < clamp_min) pi = clamp_min;
        p[i] = pi;
    }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps,
                       float bc1, float bc2, float clamp_min, int do_clamp)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / bc1, vh = vi / bc2;
        float pi = p[i] - lr * mh / (sqrtf(vh) + eps);
        if (do_clamp && pi < clamp_min) pi = clamp_min;
        p[i] = pi;
    }
}
}  // namespace

extern "C" ps_status ps_adam_step(float* param, const float* grad, float* m, float* v,
                                  long long n, float lr, float b1, float b2, float eps, int step,
                                  float clamp_min, ps_stream stream)
{
    if (n < 0 || step < 1) return PS_ERR_ARG;
    if (n == 0) return PS_OK;
    if (!param || !grad || !m || !v) return PS_ERR_ARG;
    const float bc1 = (float)(1.0 - pow((double)b1, (double)step));
    const float bc2 = (float)(1.0 - pow((double)b2, (double)step));
    const int do_clamp = isnan(clamp_min) ? 0 : 1;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_adam<<<(unsigned)blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        param, grad, m, v, n, lr, b1, b2, eps, bc1, bc2, clamp_min, do_clamp);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

// ---------------------------------------------------------------------------
// Host-side schedule of the optimisation (no device work).

extern "C" double ps_lambda_schedule(int ite)
{
    // Eq. 10: the sharpness of the rectangle weight grows with the iteration
    const double lam = 20.0 * exp(-(1.0 - 0.001 * (double)ite));
    return lam < 300.0 ? lam : 300.0;
}

extern "C" double ps_filter_margin(double lambda, double w_min)
{
    // Eq. 7-8 and the w >= w_min filter of Sec. 3.2: 2 sigmoid(-5 lambda delta) = w_min
    if (!(lambda > 0.0) || !(w_min > 0.0) || !(w_min < 1.0)) return NAN;
    const double h = 0.5 * w_min;
    return log((1.0 - h) / h) / (5.0 * lambda);
}

extern "C" double ps_gauss_extent(double w_min)
{
    // Eq. 5 on one axis: exp(-kappa^2 / 2) = w_min
    if (!(w_min > 0.0) || !(w_min < 1.0)) return NAN;
    return sqrt(2.0 * log(1.0 / w_min));
}

extern "C" ps_status ps_step_schedule(int first, int n, int lam_offset, float b1, float b2,
                                      double w_min, ps_step_state* out)
{
    if (first < 0 || n < 0 || (n > 0 && !out)) return PS_ERR_ARG;
    if (!(b1 >= 0.f && b1 < 1.f) || !(b2 >= 0.f && b2 < 1.f)) return PS_ERR_ARG;
    if (!(w_min > 0.0) || !(w_min < 1.0)) return PS_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        const int ite = first + i;
        const float lam = (float)ps_lambda_schedule(ite + lam_offset);
        out[i].lambda = lam;
        out[i].delta = ps_filter_margin((double)lam, w_min);
        out[i].step = ite + 1;
        // the same bias corrections as ps_adam_step computes for this step
        out[i].bc1 = (float)(1.0 - pow((double)b1, (double)(ite + 1)));
        out[i].bc2 = (float)(1.0 - pow((double)b2, (double)(ite + 1)));
    }
    return PS_OK;
}

extern "C" ps_status ps_step_advance(ps_step_state* d_state, const ps_step_state* d_sched,
                                     int n_sched, int* d_iter, ps_stream stream)
{
    if (!d_state || !d_sched || !d_iter || n_sched < 1) return PS_ERR_ARG;
    k_step_advance<<<1, 1, 0, reinterpret_cast<cudaStream_t>(stream)>>>(d_state, d_sched, n_sched,
                                                                        d_iter);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

extern "C" ps_status ps_adam_step_state(float* param, const float* grad, float* m, float* v,
                                        long long n, float lr, float b1, float b2, float eps,
                                        const ps_step_state* d_state, float clamp_min,
                                        long long clamp_from, ps_stream stream)
{
    if (n < 0 || !d_state || clamp_from < 0) return PS_ERR_ARG;
    if (n == 0) return PS_OK;
    if (!param || !grad || !m || !v) return PS_ERR_ARG;
    // no clamp: a start past every element
    if (isnan(clamp_min)) clamp_from = n;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_adam_state<<<(unsigned)blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        param, grad, m, v, n, lr, b1, b2, eps, d_state, clamp_min, clamp_from);
    PS_LAUNCH_CHECK();
    return PS_OK;
}
