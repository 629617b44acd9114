/*
 * ps.h -- C ABI of libps, a GB300 (sm_103a) CUDA implementation of the
 * differentiable planar-primitive rendering of PlanarSplatting
 * (arxiv 2412.03451, Sec. 3.2) and of the Adam step that fits it (Sec. 3.3).
 *
 * The calls follow the paper's statement of the problem: learnable planes
 * (Sec. 3.1) and posed views go in, depth and normal maps come out (Eq. 11-13),
 * the render loss of Eq. 14 gives per-pixel gradients, and the backward pass
 * turns them into gradients of every plane's center, quaternion and radii.
 *
 * Conventions shared by every call
 *   - All buffers are owned by the caller.  "device" pointers are CUDA device
 *     memory of the current device; "host" pointers are ordinary host memory.
 *     The library allocates nothing and keeps no state between calls.
 *   - Every call that launches work is asynchronous on the given stream, does
 *     not synchronise and does not allocate, so it may be captured in a CUDA
 *     graph.
 *   - Errors that the host can see (null pointers, bad sizes, bad settings)
 *     are returned before anything is launched.  A launch failure returns
 *     PS_ERR_CUDA.  Errors found on the device (capacity overflow, non-finite
 *     parameters) are OR-ed into the caller's device status word as
 *     (1 << code); the caller reads it after the stream is synchronised.
 *     No kernel traps or asserts.
 *
 * Plane parameters (Eq. 1-3), planes of all scenes concatenated, P planes:
 *   center [P][3] f32, quat [P][4] f32 (w,x,y,z; any nonzero norm; v^x, v^y, n
 *   are the columns of the Hamilton rotation matrix of quat/|quat|),
 *   radii [P][4] f32 (r^x+, r^x-, r^y+, r^y-).
 *
 * Views (OpenCV camera: x right, y down, z forward).  Pixel (i, j) of a view
 *   casts the ray d = ((i + 0.5 - cx)/fx, (j + 0.5 - cy)/fy, 1) from the
 *   camera centre, so the intersection parameter t of Eq. 4 is the z-depth.
 *   Views of one scene are consecutive; each view renders the planes of its
 *   own scene.  Per-pixel buffers of all views are concatenated (view v starts
 *   at pixel pix_off[v]); normals are 3 floats per pixel, in the camera frame.
 *
 * Records: one per (view, plane of the view's scene), view-major.  A record
 *   holds the plane in camera coordinates as 16 floats
 *   {n_c, n_c.p_c, v^x_c, v^x_c.p_c, v^y_c, v^y_c.p_c, r^x+, r^x-, r^y+, r^y-},
 *   its tile rectangle (4 ints, inclusive, empty = (0,0,-1,-1)) and its depth
 *   key (1 float: smallest camera z of the plane widened by the filter margin,
 *   evaluated in FP32, see ps_project_cull; a record whose key is >= z_far is
 *   culled).
 *
 * Tiles: each view is cut into tile_w x tile_h pixel tiles, numbered
 *   row-major within a view and concatenated over views.  A tile list holds the
 *   record ids whose tile rectangle covers the tile, each with an entry key (a
 *   lower bound of the plane's depth on every ray of the tile, see
 *   ps_bin_tiles), sorted by (entry key, record id).
 */
#ifndef PS_H_
#define PS_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ps_stream;   /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    PS_OK = 0,
    PS_ERR_ARG = 1,        /* bad argument, reported by the host before any launch */
    PS_ERR_CUDA = 2,       /* a CUDA launch or API call failed */
    PS_ERR_CAPACITY = 3,   /* tile-list capacity too small; required size written back */
    PS_ERR_TIMEOUT = 4,    /* a bounded device-side wait gave up */
    PS_ERR_NONFINITE = 5   /* NaN/Inf plane parameters (the plane is culled) */
} ps_status;

/* ps_settings.flags */
#define PS_SINGLE_RADII 1  /* use r^x+ for both X sides and r^y+ for both Y sides (the
                              "w/o Double Radii" ablation, Sec. 4.3) */
#define PS_HARD 2          /* hard rectangle: w = 1 inside (m >= 0), else filtered.
                              Used to ray-cast ground truth; no backward. */
#define PS_GAUSSIAN 4      /* the Gaussian splatting weight of Eq. 5 instead of Eq. 7-9
                              (the ablation of Sec. 3.2): w = exp(-(P_X^2 / s_X^2 +
                              P_Y^2 / s_Y^2) / 2), s_X = r^x+ if P_X > 0 else r^x-
                              (likewise Y); lambda is not used; delta must be
                              sqrt(2 ln(1 / w_min)) and multiplies the radii in the
                              binning (the margin of d_state is not used).  Not with
                              PS_HARD. */

#define PS_MAX_M 64        /* largest supported M (nearest intersections per ray) */

/* Per-iteration scalars kept in device memory, so that a captured CUDA graph of
   an optimisation step can be replayed for every iteration (see ps_step_advance). */
typedef struct ps_step_state {
    double delta;          /* binning margin of this iteration (see ps_settings.delta) */
    float lambda;          /* Eq. 10 value of this iteration */
    int step;              /* Adam step number, from 1 */
    float bc1, bc2;        /* Adam bias corrections 1 - b1^step, 1 - b2^step */
} ps_step_state;

/* Per-step settings.  Passed by host pointer; read on the host. */
typedef struct ps_settings {
    float lambda;          /* Eq. 10 value for this iteration */
    float w_min;           /* filter threshold, 1e-4 (Sec. 3.2) */
    float z_near, z_far;   /* valid intersection depth range (0.01, 100 m) */
    double delta;          /* binning margin: 2 sigmoid(-5 lambda delta) = w_min; 0 with PS_HARD;
                              the radius factor sqrt(2 ln(1 / w_min)) with PS_GAUSSIAN */
    int M;                 /* nearest intersections kept per ray, 30 (Sec. 3.2), <= PS_MAX_M */
    int tile_w, tile_h;    /* tile shape in pixels: 8x8, 16x16 or 32x8 */
    int flags;             /* PS_SINGLE_RADII | PS_HARD | PS_GAUSSIAN */
    float a_cos, a_l1n, a_depth;  /* Eq. 14 weights: alpha_1 = 5, alpha_1 = 5, alpha_2 = 1 */
    int cta_warps;         /* launch shape of the splat kernels: warps per CTA, 2, 4 or 8 (0: 4).
                              Each warp stages 32 plane records of its tile list per shared-memory
                              batch, so a CTA holds 32 x cta_warps records at a time.  Results
                              do not depend on it. */
    const ps_step_state* d_state; /* optional (device): if not NULL, lambda and delta are read
                                     from *d_state when the kernels run, not from the fields above */
} ps_settings;

/* Per-view descriptor, 128 bytes.  Filled on the host by ps_plan_views and
   copied to the device by the caller. */
typedef struct ps_view {
    float w2c[12];         /* world-to-camera [R|t], row-major 3x4 */
    float fx, fy, cx, cy;  /* intrinsics */
    int H, W;              /* image size */
    int tiles_x, tiles_y;  /* tile grid of this view */
    int tile_off;          /* first global tile of this view */
    int rec_off;           /* first record of this view */
    int plane_off;         /* first plane (row of center/quat/radii) of the view's scene */
    int K;                 /* planes in the view's scene */
    long long pix_off;     /* first pixel of this view in per-pixel buffers */
    int scene;             /* scene index */
    int reserved;
    long long gt_off;      /* first pixel of this view in the supervision buffers (gt_depth,
                              gt_normal); ps_plan_views sets it to pix_off, callers may point a
                              view at any image of a larger resident array */
    int reserved2[2];
} ps_view;

/* A batch of views: totals (host) and the descriptor array (device). */
typedef struct ps_frame {
    int n_views;           /* V */
    int n_records;         /* sum over views of K */
    int n_tiles;           /* sum over views of tiles_x * tiles_y */
    int max_K;             /* largest K of any view */
    long long n_pixels;    /* sum over views of H * W */
    const ps_view* views;  /* device [V] */
} ps_frame;

/* Plane parameters (device), P planes in total. */
typedef struct ps_planes {
    int n_planes;          /* P */
    int reserved;
    const float* center;   /* [P][3] */
    const float* quat;     /* [P][4] w,x,y,z */
    const float* radii;    /* [P][4] x+, x-, y+, y- */
} ps_planes;

/* Fills the host array views_out[V] and the totals of *frame_out (whose
   .views is left NULL for the caller to set to the device copy).
   scene_of_view[V] (host, non-decreasing) and plane_ptr[S+1] (host, CSR of
   the planes of each scene) describe the batch; w2c [V][12] and intr [V][4]
   are host arrays.  Returns PS_ERR_ARG on inconsistent input.  Host only. */
ps_status ps_plan_views(int n_views, const int* H, const int* W, const int* scene_of_view,
                        int n_scenes, const int* plane_ptr, const float* w2c, const float* intr,
                        int tile_w, int tile_h, ps_view* views_out, ps_frame* frame_out);

/* Projection and culling (Sec. 3.1 Eq. 2-3 and Sec. 3.2 Eq. 4, 6-9).
   For every (view, plane): normalise the quaternion, form v^x, v^y, n, move
   them and the center to the camera frame, and write the 16-float record.
   The tile rectangle and depth key come from the plane widened by
   settings->delta on every side (every pair that passes the w >= w_min filter
   lies inside), clipped to z >= z_near, projected, padded by one pixel and
   clamped to the image.  Record, rectangle and key are computed in FP32 with
   correctly rounded + - * / sqrt only, in a fixed order, from the float inputs
   (delta rounded to float), so they are reproducible bit for bit; the key
   bounds the plane's depths up to that rounding.
   rec [R][16] f32, rect [R][4] i32, key [R] f32 (device, written).
   Non-finite or zero-norm parameters cull the plane and set PS_ERR_NONFINITE. */
ps_status ps_project_cull(const ps_planes* planes, const ps_frame* frame,
                          const ps_settings* settings, float* rec, int* rect, float* key,
                          int* d_status, ps_stream stream);

/* Bytes of scratch that ps_bin_tiles needs for this frame and capacity. */
size_t ps_bin_workspace_bytes(const ps_frame* frame, long long capacity);

/* Binning and depth ordering (the near-to-far sort of Sec. 3.2, "Blending
   Composition", applied per tile to a conservative depth key).
   Inputs: rec [R][16], rect [R][4] and key [R] from ps_project_cull (device).
   Writes tile_ptr [n_tiles + 1] (device, CSR offsets), tile_ent [capacity]
   (device, record ids) and tile_key [capacity] (device, their entry keys),
   sorted by (entry key, record id) within each tile.  Entry key (computed
   bit-reproducibly in FP32 with correctly rounded + - * / only): for the rays
   d of the pixel centres at the tile's four corner pixels, den = (n_x d_x +
   n_y d_y) + n_z and t = s / den from the record's n_c and s; if den has one
   sign at all four and |den| > 0.01 (|n_x d_x| + |n_y d_y| + |n_z|) at each,
   c = max(min t, z_near), or +inf if max t <= z_near; otherwise c = z_near;
   the entry key is max(c, key[record]).
   The plane's depth on any ray of the tile is >= the key (up to FP32 rounding,
   which the splat kernels absorb with a relative margin of 1/4096).  The total
   number of entries goes to *d_required (device, 1 long long).  If it exceeds
   capacity, PS_ERR_CAPACITY is set in *d_status, tile_ptr is still complete,
   and the splat calls read only the first `capacity` entries.  ws (device,
   ws_bytes >= ps_bin_workspace_bytes) is scratch. */
ps_status ps_bin_tiles(const ps_frame* frame, const ps_settings* settings, const float* rec,
                       const int* rect, const float* key, int* tile_ptr, int* tile_ent,
                       float* tile_key, long long capacity, long long* d_required, void* ws,
                       size_t ws_bytes, int* d_status, ps_stream stream);

/* Bytes of scratch that ps_splat_fwd needs (its work counter). */
size_t ps_fwd_workspace_bytes(const ps_frame* frame);

/* Forward splatting (Sec. 3.2, Eq. 4, 6-9, 11-13).  For every pixel: intersect
   the ray with every plane of the pixel's tile list, weight it with
   w = min(1, 2 sigmoid(5 lambda min(m_X, m_Y))) (m = r - |P| on the side given
   by the sign of P), drop w < w_min and depths outside (z_near, z_far), keep
   the M nearest by (t, record id) and composite front to back:
   D = sum T_j w_j t_j, N = sum T_j w_j n_j, alpha = sum T_j w_j.
   depth [n_pixels], normal [n_pixels][3], alpha [n_pixels] (device, written;
   alpha may be NULL).  ws (device, 16-byte aligned, >= ps_fwd_workspace_bytes)
   is scratch (a work counter reset by the call). */
ps_status ps_splat_fwd(const ps_frame* frame, const ps_settings* settings, const float* rec,
                       const float* tile_key, const int* tile_ptr, const int* tile_ent,
                       long long capacity, float* depth, float* normal, float* alpha,
                       void* ws, size_t ws_bytes, int* d_status, ps_stream stream);

/* Plane-index map: for every pixel, the index (row of the plane arrays) of the
   nearest composited plane, -1 where none passes the filter.  With PS_HARD
   this is the plane a ray hits first.  Same walk as ps_splat_fwd; ids
   [n_pixels] (device, written), depth (device, optional) as in ps_splat_fwd;
   ws as in ps_splat_fwd.  Used to cut training patches into planes. */
ps_status ps_splat_ids(const ps_frame* frame, const ps_settings* settings, const float* rec,
                       const float* tile_key, const int* tile_ptr, const int* tile_ent,
                       long long capacity, int* ids, float* depth, void* ws, size_t ws_bytes,
                       int* d_status, ps_stream stream);

/* Render loss (Eq. 14) and its gradient with respect to the rendered maps.
   Pixels with gt_depth <= 0 are not supervised (zero gradient).
   dL_dD [n_pixels], dL_dN [n_pixels][3] (device, written);
   view_sums [V][4] f64 (device, overwritten): per view the sums of
   |1 - N.N*|, ||N - N*||_1, |D - D*| and the number of supervised pixels.
   Loss = a_cos*sum0 + a_l1n*sum1 + a_depth*sum2.  sgn(0) = 0. */
ps_status ps_loss(const ps_frame* frame, const ps_settings* settings, const float* depth,
                  const float* normal, const float* gt_depth, const float* gt_normal,
                  float* dL_dD, float* dL_dN, double* view_sums, ps_stream stream);

/* Bytes of scratch that ps_splat_bwd and ps_splat_fused need (per-record
   gradient accumulators, a work counter and, for ps_splat_fused, 32 partial
   loss sums per view). */
size_t ps_bwd_workspace_bytes(const ps_frame* frame);

/* Backward splatting: gradient of sum(dL_dD * D + dL_dN . N) with respect to
   every plane's center, quaternion and radii.  Recomputes each pixel's
   composited list from the tile lists (no per-pixel state is stored by the
   forward), takes the adjoint of Eq. 11-13 back to front
   (A_j = w_j t_j + (1 - w_j) A_{j+1}, dD/dw_j = T_j (t_j - A_{j+1}); no
   division by 1 - w), chains it through Eq. 9, 7-8, 6, 4 into per-record
   gradients and then through the camera transform and Eq. 2-3 (with the
   quaternion normalisation) into the world parameters.  The clamp
   min(1, .) has derivative 0 where m >= 0.  Ties of Eq. 9 go to the Y side.
   g_center [P][3], g_quat [P][4], g_radii [P][4] (device) are ACCUMULATED
   into (the caller zeroes them).  ws (device, >= ps_bwd_workspace_bytes) is
   scratch.  Float atomics make the summation order, and so the last bits,
   vary from run to run. */
ps_status ps_splat_bwd(const ps_planes* planes, const ps_frame* frame,
                       const ps_settings* settings, const float* rec, const float* tile_key,
                       const int* tile_ptr, const int* tile_ent, long long capacity,
                       const float* dL_dD, const float* dL_dN, float* g_center, float* g_quat,
                       float* g_radii, void* ws, size_t ws_bytes, int* d_status,
                       ps_stream stream);

/* ps_splat_bwd for callers that cannot allocate device memory (an engine whose
   device memory belongs to a fixed arena, a real-time loop that must never
   enter the CUDA allocator, a plug-in host without a device allocator).  The
   paper has no counterpart: this is a deployment variant of ps_splat_bwd.
   Same arguments, results and accumulate-into-gradients semantics as
   ps_splat_bwd, but without ws/ws_bytes: its scratch is a 4 MiB array
   compiled into the library, which every device that loads the library holds
   until the process exits.  Limit: frame->n_records <= 65536; larger frames
   return PS_ERR_ARG before anything is launched.  No cudaMalloc, cudaFree or
   other allocating call is made.  The first call on a device looks up the
   array's device address (cudaGetSymbolAddress) with that device current and
   caches it with the current CUDA context; a call under another context (after
   cudaDeviceReset, or with a context the caller made current) looks it up again.
   Make the first call in a context before any stream capture.  Every call
   clears the part of the array it uses, but all calls share the one array:
   calls that may overlap on the GPU (different streams, or different host
   threads on the same device) race and must be serialised by the caller. */
ps_status ps_splat_bwd_noalloc(const ps_planes* planes, const ps_frame* frame,
                               const ps_settings* settings, const float* rec, const float* tile_key,
                               const int* tile_ptr, const int* tile_ent, long long capacity,
                               const float* dL_dD, const float* dL_dN, float* g_center,
                               float* g_quat, float* g_radii, int* d_status, ps_stream stream);

/* Forward splatting, render loss and backward splatting fused (Sec. 3.2,
   Eq. 4, 6-14).  Because the loss of Eq. 14 is a sum of per-pixel terms, each
   pixel's composited list, built once, serves both the forward and the
   adjoint: the call renders D and N exactly as ps_splat_fwd, evaluates Eq. 14
   against gt_depth / gt_normal (pixels with gt_depth <= 0 unsupervised) as
   ps_loss, and accumulates the gradient of the loss into g_center, g_quat,
   g_radii exactly as ps_splat_bwd would with the loss's dL/dD and dL/dN.
   depth, normal, dL_dD, dL_dN (device, written) may each be NULL;
   view_sums [V][4] f64 (device) is overwritten as in ps_loss; gradients are
   accumulated (the caller zeroes them).  ws (device, 16-byte aligned,
   >= ps_bwd_workspace_bytes) is scratch. */
ps_status ps_splat_fused(const ps_planes* planes, const ps_frame* frame,
                         const ps_settings* settings, const float* rec, const float* tile_key,
                         const int* tile_ptr, const int* tile_ent, long long capacity,
                         const float* gt_depth, const float* gt_normal, float* depth,
                         float* normal, float* dL_dD, float* dL_dN, double* view_sums,
                         float* g_center, float* g_quat, float* g_radii, void* ws,
                         size_t ws_bytes, int* d_status, ps_stream stream);

/* Adam (Kingma & Ba; Sec. 3.3, lr = 1e-3 for every group, App. A.2),
   bias-corrected, on n floats in place: param, m, v (device, updated),
   grad (device, read).  step counts from 1.  After the update every value
   below clamp_min is raised to it; pass NaN for no clamp. */
ps_status ps_adam_step(float* param, const float* grad, float* m, float* v, long long n,
                       float lr, float b1, float b2, float eps, int step, float clamp_min,
                       ps_stream stream);

/* Work counts of one forward splat, for throughput and roofline reports:
   d_counts[0] = pairs tested (tile-list entries x pixels of the tile inside the
   image), d_counts[1] = candidate pairs (pairs that pass the w >= w_min and depth
   filters of Sec. 3.2: the algorithmic pair count, independent of tiling),
   d_counts[2] = composited pairs (per pixel, min(M, candidates up to and
   including the nearest one with w = 1)).  d_counts (device, 3 long long) is
   overwritten.  Walks every tile list completely; slower than ps_splat_fwd. */
ps_status ps_count_pairs(const ps_frame* frame, const ps_settings* settings, const float* rec,
                         const float* tile_key, const int* tile_ptr, const int* tile_ent,
                         long long capacity, long long* d_counts, ps_stream stream);

/* Graph replay support: copies d_sched[min(*d_iter, n_sched - 1)] into *d_state
   and increments *d_iter (one device thread; device pointers).  Launched at the
   start of a captured step, it makes every replay use the next iteration's
   lambda, delta and Adam bias corrections. */
ps_status ps_step_advance(ps_step_state* d_state, const ps_step_state* d_sched, int n_sched,
                          int* d_iter, ps_stream stream);

/* Scene initialisation (Sec. 3.1): every plane starts with its radii at half
   the distance from its centre to the nearest other centre.  For points (device
   f32 [n][3]): dist[i] (device f32 [n], or NULL) = the Euclidean distance from
   points[i] to the nearest other point, +inf if n == 1, exact up to FP32 rounding
   of the distances (the minimum over every other point); radii (device f32
   [n][4], 16-byte aligned, or NULL) = all four radii of plane i set to
   clamp(scale x dist[i], r_lo, r_hi) (scale 0.5 in the paper).  Points are
   counted into a hashed uniform grid (cell edge about the cube root of the
   bounding box's volume per point) and each query searches shells of cells around
   its own until the nearest point found lies within the searched radius.  ws
   (device, 16-byte aligned, >= ps_nn_workspace_bytes(n)) is scratch.  Asynchronous
   on the stream; five launches.  PS_ERR_ARG for n < 0, NULL points or ws, both
   outputs NULL, scale < 0, r_lo > r_hi or a small workspace. */
size_t ps_nn_workspace_bytes(int n);
ps_status ps_nn_distance(const float* points, int n, float scale, float r_lo, float r_hi,
                         float* dist, float* radii, void* ws, size_t ws_bytes, ps_stream stream);

/* ---- Host-side schedule of the optimisation.  Plain host functions: no device
   work, no CUDA call; usable without a GPU. ---- */

/* Eq. 10: lambda = min(20 exp(-(1 - 0.001 ite)), 300), evaluated in FP64; ite
   counts optimisation iterations from 0. */
double ps_lambda_schedule(int ite);

/* The binning margin delta of ps_settings: the distance outside a rectangle's
   edge at which the weight 2 sigmoid(5 lambda m) of Eq. 7-8 falls to the filter
   threshold of Sec. 3.2, 2 sigmoid(-5 lambda delta) = w_min, i.e.
   delta = ln((1 - w_min/2) / (w_min/2)) / (5 lambda), in FP64.  Returns NaN if
   lambda <= 0 or w_min is not in (0, 1). */
double ps_filter_margin(double lambda, double w_min);

/* With PS_GAUSSIAN the binning scales every radius by kappa, where the Eq. 5
   weight of one axis falls to w_min: exp(-kappa^2 / 2) = w_min, kappa =
   sqrt(2 ln(1 / w_min)).  NaN if w_min is not in (0, 1). */
double ps_gauss_extent(double w_min);

/* Fills out[0 .. n-1] (host memory, caller-owned) with the per-iteration scalars
   of iterations first .. first + n - 1 for ps_step_advance: lambda = Eq. 10 at
   iteration ite + lam_offset rounded to f32, delta = ps_filter_margin(that f32
   lambda, w_min), step = ite + 1 (Adam counts from 1), bc1 = 1 - b1^step and
   bc2 = 1 - b2^step rounded to f32 (the values ps_adam_step computes for that
   step).  A fit from a good initialisation may pass lam_offset > 0 to start the
   schedule later; Adam's step count is not shifted.  PS_ERR_ARG if first < 0,
   n < 0, out is NULL with n > 0, b1 or b2 is outside [0, 1) or w_min outside (0, 1). */
ps_status ps_step_schedule(int first, int n, int lam_offset, float b1, float b2, double w_min,
                           ps_step_state* out);

/* Plane splitting, part 1 (Sec. 3.3 "Plane Splitting", App. A.2): adds this
   step's radius gradients to a running sum.  g_radii [P][4] (device, the
   gradient of the loss with respect to r^x+, r^x-, r^y+, r^y-), acc [P][2]
   (device, updated): acc[p][0] += s_p (|g[p][0]| + |g[p][1]|) / 2 and
   acc[p][1] += s_p (|g[p][2]| + |g[p][3]|) / 2, with s_p = plane_scale[p]
   (device [P]) or, if plane_scale is NULL, the value scale.  The scale turns the
   summed loss of Eq. 14 into the per-pixel mean the split threshold refers to
   (1 / supervised pixels of the plane's scene in this step).  PS_ERR_ARG on bad
   sizes or NULL pointers. */
ps_status ps_radii_grad_accum(const float* g_radii, const float* plane_scale, float scale,
                              int n_planes, float* acc, ps_stream stream);

/* Plane splitting, part 2: every plane p whose mean radius gradient on an axis,
   acc[p][axis] / n_iter, exceeds tau is cut in two along the other axis (the
   larger axis if both exceed it): X -> a +X half and a -X half (centres
   p + r^x+/2 v^x and p - r^x-/2 v^x, X radii r^x+/2 and r^x-/2 on both sides,
   Y radii kept), Y likewise with v^y; the rotation is kept.  Planes whose
   quaternion is zero or non-finite are kept.
   params, m, v: device flat buffers of P planes, [center P x 3 | quat P x 4 |
   radii P x 4] (m, v: Adam moments in the same layout, may be NULL).
   plane_ptr [S+1] (device): CSR of the planes of each scene.  Output: the same
   layout for P' = P + splits planes in params_out (and m_out, v_out if not
   NULL; capacity planes of room each): scene s occupies plane_ptr_out[s] ..
   plane_ptr_out[s+1] - 1, its planes in their old order (a split plane's +half
   in its slot) followed by the -halves in the order of their parents.  Moments
   are copied for kept planes and zeroed for both halves.  split_rank [P+1]
   (device, written): split planes before each plane, [P] = their number;
   *d_count (device) = P'.  If P' > capacity only split_rank and *d_count are
   written.  One CTA; deterministic.  Host-side PS_ERR_ARG on bad sizes. */
ps_status ps_split_planes(const float* params, const float* m, const float* v, int n_scenes,
                          const int* plane_ptr, int n_planes, const float* acc, int n_iter,
                          float tau, float* params_out, float* m_out, float* v_out,
                          int* plane_ptr_out, int capacity, int* split_rank, int* d_count,
                          ps_stream stream);

/* Plane merging (Sec. 3.3 "Plane Merge"): groups fitted planes into plane
   instances.  Planes are taken by decreasing area (r^x+ + r^x-)(r^y+ + r^y-)
   (ties: lower index first); each joins the first existing group whose first
   plane has a normal within max_angle_deg of its own, up to sign (planes are
   two-sided), and an offset within max_offset, or starts a new group.  Offset
   = n . (p - scene_center) with n oriented like the group's normal.
   params: device flat [center P x 3 | quat P x 4 | radii P x 4], n_planes <= 8192;
   scene_center: host float[3].  Output (device): group_of[P] (group index, -1 for
   a zero or non-finite quaternion), rep_of_group[P] (first plane of each group),
   *d_groups = number of groups.  One CTA; deterministic. */
ps_status ps_merge_planes(const float* params, int n_planes, const float* scene_center,
                          float max_angle_deg, float max_offset, int* group_of, int* rep_of_group,
                          int* d_groups, ps_stream stream);

/* ps_adam_step with the step's bias corrections read from d_state (device).
   The clamp (unless clamp_min is NaN) applies to elements clamp_from .. n - 1
   only, so that one launch updates a whole parameter block whose tail (the
   radii) has a lower bound.  PS_ERR_ARG if clamp_from < 0 or n < 0. */
ps_status ps_adam_step_state(float* param, const float* grad, float* m, float* v, long long n,
                             float lr, float b1, float b2, float eps,
                             const ps_step_state* d_state, float clamp_min, long long clamp_from,
                             ps_stream stream);

/* BF16 GEMM on the tensor cores (tcgen05, FP32 accumulation in tensor memory)
   for the seed-proposal network (not part of the paper's renderer):
   C[M, N] = A[M, K] . B[N, K]^T (+ bias[N]) (then ReLU if relu).
   A, B: device bf16, row-major with K contiguous, 16-byte aligned; K must be a
   multiple of 64 (zero-pad).  C32: device fp32 [M, ldc] or NULL; C16: device
   bf16 [M, ldc] or NULL (at least one); with accumulate, C32 += result.
   bias: device fp32 [N] or NULL.  d_err: device status word (or NULL) into which
   (1 << PS_ERR_TIMEOUT) is OR-ed if a bounded wait for the copies or the tensor
   cores timed out (the tile is then not written; the copies and MMAs in flight
   get a bounded wait and the tensor memory is freed, so the context stays usable). */
ps_status ps_gemm_bf16(const void* A, const void* B, const float* bias, float* C32, void* C16,
                       int M, int N, int K, int ldc, int relu, int accumulate, int* d_err,
                       ps_stream stream);

/* Exercises the time-out path of the bounded device-side waits: one thread
   waits on an mbarrier that nothing arrives on (the wait routine of
   ps_gemm_bf16) for `polls` polls (1 .. 2^24), gives up and ORs
   (1 << PS_ERR_TIMEOUT) into *d_status (device).  Nothing else is issued, so the
   context stays usable.  For tests of the failure path; no fault is involved. */
ps_status ps_wait_selftest(int* d_status, long long polls, ps_stream stream);

/* ---- Seed-proposal network (not part of the paper: a learned initialiser of
   the planes of Sec. 3.1).  Four 3x3 stride-2 convolutions (64 channels, ReLU),
   global average pooling and a 64 -> 96 linear layer map a 64x64 patch of depth
   and camera-frame normals to 8 plane seeds.  Convolutions are im2col +
   ps_gemm_bf16.  Activations NHWC bf16; gradients fp32; the im2col column
   order is (ky, kx, c) zero-padded to Kp (a multiple of 64).  All pointers are
   device pointers; every call is asynchronous on the stream. ---- */

/* A[B*Ho*Wo, Kp] (bf16) = im2col of x[B, H, W, C] (bf16) for a 3x3 window,
   stride 2, padding 1; Ho = ceil(H/2), Wo = ceil(W/2). */
ps_status ps_seed_im2col(const void* x, int B, int H, int W, int C, int Kp, void* A,
                         ps_stream stream);
/* dx[B, H, W, C] (fp32) = adjoint of ps_seed_im2col applied to dA[B*Ho*Wo, Kp] (fp32). */
ps_status ps_seed_col2im(const float* dA, int B, int H, int W, int C, int Kp, float* dx,
                         ps_stream stream);
/* dz = scale * dy * (y > 0) over n elements (ReLU backward); dy fp32, y bf16;
   dz16 (bf16) and/or dz32 (fp32) written. */
ps_status ps_seed_relu_bwd(const float* dy, const void* y, long long n, float scale, void* dz16,
                           float* dz32, ps_stream stream);
/* out[c, r] = in[r, c] (bf16 out, leading dimension ldo >= R; columns R..ldo-1
   zero); in is bf16 if in_is_bf16 else fp32, leading dimension ldi. */
ps_status ps_seed_transpose(const void* in, int in_is_bf16, int R, int C, int ldi, void* out,
                            int ldo, ps_stream stream);
/* db[c] = sum over R rows of dz[r, c] (fp32, C <= 256). */
ps_status ps_seed_colsum(const float* dz, long long R, int C, float* db, ps_stream stream);
/* h[b, c] = mean over S positions of y[b, s, c] (y bf16; h32 fp32 and/or h16 bf16). */
ps_status ps_seed_pool(const void* y, int B, int S, int C, float* h32, void* h16,
                       ps_stream stream);
/* dy[b, s, c] = dh[b, c] / S (fp32). */
ps_status ps_seed_pool_bwd(const float* dh, int B, int S, int C, float* dy, ps_stream stream);
/* Set loss of the seed slots and its gradient.  out[B, slots * 12]: per slot
   centre (3), quaternion (4, unnormalised), log extents (4), confidence logit;
   tgt[B, slots, 12]: valid flag, centre, unit quaternion, log extents.  Per slot
   BCE(logit, valid) + valid (|c - c*|_1 + (1 - |q/|q| . q*|) + 0.5 |e - e*|_1),
   mean over the batch.  dout (fp32, same shape as out) written; sums[4] (or
   NULL) receives the four terms summed over the batch. */
ps_status ps_seed_loss(const float* out, const float* tgt, int B, int slots, float* dout,
                       float* sums, ps_stream stream);
/* out[R, Cp] (bf16) = in[R, Cin] (fp32) with zero columns Cin..Cp-1. */
ps_status ps_cast_bf16(const float* in, int R, int Cin, int Cp, void* out, ps_stream stream);

/* Human-readable name of a status code. */
const char* ps_status_string(ps_status status);

/* Library version, for the binding's sanity check. */
int ps_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PS_H_ */
