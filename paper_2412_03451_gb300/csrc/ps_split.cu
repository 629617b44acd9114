// ps_split.cu -- plane splitting (Sec. 3.3, "Plane Splitting"; App. A.2) and
// plane merging (Sec. 3.3, "Plane Merge").
//
// During the fit, every fixed number of iterations, a plane whose mean radius
// gradient on one axis exceeds a threshold is cut in two along the other axis:
// a large X-radius gradient (r^x+, r^x-) splits the plane along its Y axis into
// a +X half and a -X half, and vice versa.  Two kernels:
//   * k_radii_grad_accum adds, per plane and per step, the mean of |dL/dr^x+|
//     and |dL/dr^x-| and the mean of |dL/dr^y+| and |dL/dr^y-| (times a
//     per-plane scale that turns the summed loss of Eq. 14 into a per-pixel
//     mean) to a running sum;
//   * k_split_planes (one CTA) decides every plane, numbers the split planes
//     by an exclusive scan, and writes the new plane set scene by scene: the
//     +half of plane i takes i's slot (shifted by the splits of earlier
//     scenes), the -half is appended after the scene's planes in plane order,
//     so every scene's planes stay contiguous and the result is deterministic.
//     Adam moments are copied for unsplit planes and zeroed for both halves.
//   * k_merge_planes (one CTA) groups the fitted planes into plane instances:
//     planes are taken by decreasing area; each joins the first existing group
//     whose first (largest) plane has a normal within the angle threshold (up
//     to sign: planes are two-sided) and an offset -- the distance from the
//     scene centre to the plane along the normal oriented like the group's --
//     within the offset threshold, or starts a new group.
#include "ps_internal.cuh"

using namespace ps;

namespace {

constexpr int kSplitThreads = 1024;

__global__ void k_radii_grad_accum(const float* __restrict__ g_radii,
                                   const float* __restrict__ plane_scale, float scale, int P,
                                   float* __restrict__ acc)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const float s = plane_scale ? __ldg(&plane_scale[p]) : scale;
    const float* g = g_radii + 4 * (size_t)p;
    acc[2 * p] += s * 0.5f * (fabsf(__ldg(g)) + fabsf(__ldg(g + 1)));
    acc[2 * p + 1] += s * 0.5f * (fabsf(__ldg(g + 2)) + fabsf(__ldg(g + 3)));
}

// 0: keep; 1: large X-radius gradient -> halves along v^x; 2: halves along v^y.
__device__ __forceinline__ float4 load_quat(const float* __restrict__ quat, int i)
{
    const float* q = quat + 4 * (size_t)i;
    return make_float4(__ldg(q), __ldg(q + 1), __ldg(q + 2), __ldg(q + 3));
}

__device__ __forceinline__ int split_kind(const float* __restrict__ acc, const float* __restrict__ quat,
                                          int i, float inv_n, float tau)
{
    const float4 q = load_quat(quat, i);
    const float nq = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
    if (!(nq > 0.f) || !(nq < INFINITY)) return 0;
    const float gx = __ldg(&acc[2 * i]) * inv_n, gy = __ldg(&acc[2 * i + 1]) * inv_n;
    if (!(gx > tau) && !(gy > tau)) return 0;
    return gx >= gy ? 1 : 2;
}

__device__ __forceinline__ int block_excl_scan(int x, int* s_warp, int& total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int w = (lane < (int)(blockDim.x >> 5)) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    total = s_warp[(blockDim.x >> 5) - 1];
    const int r = incl - x + (wid > 0 ? s_warp[wid - 1] : 0);
    __syncthreads();
    return r;
}

struct SplitArgs {
    const float* params;      // [P*11] flat: center P x 3 | quat P x 4 | radii P x 4
    const float* m;           // same layout, or null
    const float* v;
    int n_scenes;
    const int* plane_ptr;     // [S+1]
    int P;
    const float* acc;         // [P][2]
    float inv_n, tau;
    float* params_out;        // [P'*11], P' = P + splits
    float* m_out;
    float* v_out;
    int* plane_ptr_out;       // [S+1]
    int P_cap;
    int* split_rank;          // [P+1]: splits before plane i; [P] = total
    int* d_count;             // P'
};

__global__ void __launch_bounds__(kSplitThreads) k_split_planes(SplitArgs a)
{
    __shared__ int s_warp[32];
    __shared__ int s_carry;
    const int P = a.P;
    const float* quat = a.params + 3 * (size_t)P;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    // pass 1: decisions and their exclusive scan
    for (int b0 = 0; b0 < P; b0 += kSplitThreads) {
        const int i = b0 + threadIdx.x;
        const int f = i < P ? (split_kind(a.acc, quat, i, a.inv_n, a.tau) != 0) : 0;
        int total;
        const int e = block_excl_scan(f, s_warp, total);
        if (i < P) a.split_rank[i] = s_carry + e;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += total;
        __syncthreads();
    }
    const int S = s_carry;
    const int Pn = P + S;
    if (threadIdx.x == 0) {
        a.split_rank[P] = S;
        *a.d_count = Pn;
    }
    __syncthreads();
    if (Pn > a.P_cap) return;
    for (int s = threadIdx.x; s <= a.n_scenes; s += kSplitThreads) {
        const int b = a.plane_ptr[s];
        a.plane_ptr_out[s] = b + a.split_rank[b];
    }
    // pass 2: write the new plane set
    const float* cin = a.params;
    const float* rin = a.params + 7 * (size_t)P;
    float* cout = a.params_out;
    float* qout = a.params_out + 3 * (size_t)Pn;
    float* rout = a.params_out + 7 * (size_t)Pn;
    for (int i = threadIdx.x; i < P; i += kSplitThreads) {
        // scene of plane i: last s with plane_ptr[s] <= i
        int lo = 0, hi = a.n_scenes - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.plane_ptr[mid] <= i) lo = mid; else hi = mid - 1;
        }
        const int base = a.plane_ptr[lo], K = a.plane_ptr[lo + 1] - base;
        const int shift = a.split_rank[base];
        const int pa = i + shift;
        const int kind = split_kind(a.acc, quat, i, a.inv_n, a.tau);
        const float4 q = load_quat(quat, i);
        float c[3] = {cin[3 * i], cin[3 * i + 1], cin[3 * i + 2]};
        float r[4] = {rin[4 * i], rin[4 * i + 1], rin[4 * i + 2], rin[4 * i + 3]};
        if (kind == 0) {
            for (int j = 0; j < 3; ++j) cout[3 * pa + j] = c[j];
            qout[4 * pa + 0] = q.x; qout[4 * pa + 1] = q.y; qout[4 * pa + 2] = q.z; qout[4 * pa + 3] = q.w;
            for (int j = 0; j < 4; ++j) rout[4 * pa + j] = r[j];
            for (int g = 0; g < 3; ++g) {
                const size_t oi = g == 0 ? 3 * (size_t)i : (g == 1 ? 3 * (size_t)P + 4 * i : 7 * (size_t)P + 4 * i);
                const size_t oo = g == 0 ? 3 * (size_t)pa : (g == 1 ? 3 * (size_t)Pn + 4 * pa : 7 * (size_t)Pn + 4 * pa);
                const int n = g == 0 ? 3 : 4;
                for (int j = 0; j < n; ++j) {
                    if (a.m_out) a.m_out[oo + j] = a.m ? a.m[oi + j] : 0.f;
                    if (a.v_out) a.v_out[oo + j] = a.v ? a.v[oi + j] : 0.f;
                }
            }
            continue;
        }
        const int pb = base + shift + K + (a.split_rank[i] - shift);
        // axes of the plane: columns 0 and 1 of R(q / |q|) (Eq. 2-3), (w, x, y, z) order
        const float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
        const float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
        const float ax[3] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y + w * z), 2.f * (x * z - w * y)};
        const float ay[3] = {2.f * (x * y - w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z + w * x)};
        const float* dir = kind == 1 ? ax : ay;
        const float rp = kind == 1 ? r[0] : r[2];     // extent on the + side of the cut axis
        const float rm = kind == 1 ? r[1] : r[3];     // extent on the - side
        float ra[4] = {r[0], r[1], r[2], r[3]}, rb[4] = {r[0], r[1], r[2], r[3]};
        const int o = kind == 1 ? 0 : 2;
        ra[o] = ra[o + 1] = 0.5f * rp;
        rb[o] = rb[o + 1] = 0.5f * rm;
        for (int j = 0; j < 3; ++j) {
            cout[3 * pa + j] = c[j] + 0.5f * rp * dir[j];
            cout[3 * pb + j] = c[j] - 0.5f * rm * dir[j];
        }
        qout[4 * pa + 0] = q.x; qout[4 * pa + 1] = q.y; qout[4 * pa + 2] = q.z; qout[4 * pa + 3] = q.w;
        qout[4 * pb + 0] = q.x; qout[4 * pb + 1] = q.y; qout[4 * pb + 2] = q.z; qout[4 * pb + 3] = q.w;
        for (int j = 0; j < 4; ++j) {
            rout[4 * pa + j] = ra[j];
            rout[4 * pb + j] = rb[j];
        }
        for (int pp = 0; pp < 2; ++pp) {
            const int t = pp == 0 ? pa : pb;
            for (int g = 0; g < 3; ++g) {
                const size_t oo = g == 0 ? 3 * (size_t)t : (g == 1 ? 3 * (size_t)Pn + 4 * t : 7 * (size_t)Pn + 4 * t);
                const int n = g == 0 ? 3 : 4;
                for (int j = 0; j < n; ++j) {
                    if (a.m_out) a.m_out[oo + j] = 0.f;
                    if (a.v_out) a.v_out[oo + j] = 0.f;
                }
            }
        }
    }
}

constexpr int kMergeThreads = 1024;
constexpr int kMergeMax = 8192;           // planes per call (one CTA, keys in shared memory)

// normal (column 2 of R(q / |q|)) and offset of plane i; false for a degenerate quaternion
__device__ __forceinline__ bool plane_normal_offset(const float* __restrict__ params, int P, int i,
                                                    float3 c0, float3& n, float& off)
{
    const float* c = params + 3 * (size_t)i;
    const float4 q = load_quat(params + 3 * (size_t)P, i);
    const float nq = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
    if (!(nq > 0.f) || !(nq < INFINITY)) return false;
    const float inv = rsqrtf(nq);
    const float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
    n = make_float3(2.f * (x * z + w * y), 2.f * (y * z - w * x), 1.f - 2.f * (x * x + y * y));
    off = n.x * (c[0] - c0.x) + n.y * (c[1] - c0.y) + n.z * (c[2] - c0.z);
    return true;
}

__global__ void __launch_bounds__(kMergeThreads) k_merge_planes(const float* __restrict__ params,
                                                               int P, float3 c0, float cos_max,
                                                               float off_max, int* __restrict__ group_of,
                                                               int* __restrict__ rep_of_group,
                                                               int* __restrict__ d_groups)
{
    // dynamic shared memory: keys [N] (area bits, ~index; larger area first),
    // per group its first plane's normal and offset [P], its first plane [P]
    extern __shared__ unsigned long long s_dyn[];
    __shared__ int s_groups, s_hit;
    const int tid = threadIdx.x;
    const float* radii = params + 7 * (size_t)P;
    int N = 2;                    // keeps the float4 block 16-byte aligned
    while (N < P) N <<= 1;
    unsigned long long* s_key = s_dyn;
    float4* s_n = reinterpret_cast<float4*>(s_dyn + N);
    int* s_rep = reinterpret_cast<int*>(s_n + P);
    for (int i = tid; i < N; i += kMergeThreads) {
        unsigned long long k = 0ull;                   // padding sorts last
        if (i < P) {
            const float* r = radii + 4 * (size_t)i;
            const float area = (r[0] + r[1]) * (r[2] + r[3]);
            const float a = area > 0.f ? area : 0.f;   // NaN and negative areas last among planes
            k = ((unsigned long long)__float_as_uint(a) << 32) | (unsigned)(0xffffffffu - (unsigned)i);
        }
        s_key[i] = k;
    }
    __syncthreads();
    // bitonic sort, descending
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < N; i += kMergeThreads) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long x = s_key[i], y = s_key[ixj];
                    const bool desc = (i & k) == 0;
                    if ((x < y) == desc) { s_key[i] = y; s_key[ixj] = x; }
                }
            }
            __syncthreads();
        }
    }
    if (tid == 0) s_groups = 0;
    __syncthreads();
    for (int o = 0; o < P; ++o) {
        const int i = (int)(0xffffffffu - (unsigned)(s_key[o] & 0xffffffffu));
        float3 n;
        float off;
        const bool ok = plane_normal_offset(params, P, i, c0, n, off);
        if (!ok) {                                     // degenerate: a group of its own
            if (tid == 0) { group_of[i] = -1; }
            __syncthreads();
            continue;
        }
        if (tid == 0) s_hit = 0x7fffffff;
        __syncthreads();
        const int G = s_groups;
        for (int g = tid; g < G; g += kMergeThreads) {
            const float4 m = s_n[g];
            const float d = n.x * m.x + n.y * m.y + n.z * m.z;
            const float sgn = d >= 0.f ? 1.f : -1.f;
            if (fabsf(d) >= cos_max && fabsf(sgn * off - m.w) < off_max) atomicMin(&s_hit, g);
        }
        __syncthreads();
        if (tid == 0) {
            int g = s_hit;
            if (g == 0x7fffffff) {
                g = s_groups;
                s_rep[g] = i;
                s_n[g] = make_float4(n.x, n.y, n.z, off);
                s_groups = g + 1;
            }
            group_of[i] = g;
        }
        __syncthreads();
    }
    const int G = s_groups;
    for (int g = tid; g < G; g += kMergeThreads) rep_of_group[g] = s_rep[g];
    if (tid == 0) *d_groups = G;
}

}  // namespace

extern "C" ps_status ps_merge_planes(const float* params, int n_planes, const float* scene_center,
                                     float max_angle_deg, float max_offset, int* group_of,
                                     int* rep_of_group, int* d_groups, ps_stream stream)
{
    if (n_planes < 0 || n_planes > kMergeMax || !scene_center || !d_groups) return PS_ERR_ARG;
    if (n_planes > 0 && (!params || !group_of || !rep_of_group)) return PS_ERR_ARG;
    if (!(max_angle_deg >= 0.f && max_angle_deg <= 90.f) || !(max_offset >= 0.f)) return PS_ERR_ARG;
    const float3 c0 = make_float3(scene_center[0], scene_center[1], scene_center[2]);
    const float cos_max = cosf(max_angle_deg * 3.14159265358979f / 180.f);
    int N = 2;
    while (N < n_planes) N <<= 1;
    const size_t dyn = sizeof(unsigned long long) * (size_t)N + (sizeof(float4) + sizeof(int)) * (size_t)n_planes;
    if (dyn > 48 * 1024)
        PS_CUDA_CHECK(cudaFuncSetAttribute(k_merge_planes, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)dyn));
    k_merge_planes<<<1, kMergeThreads, dyn, reinterpret_cast<cudaStream_t>(stream)>>>(
        params, n_planes, c0, cos_max, max_offset, group_of, rep_of_group, d_groups);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

extern "C" ps_status ps_radii_grad_accum(const float* g_radii, const float* plane_scale, float scale,
                                         int n_planes, float* acc, ps_stream stream)
{
    if (n_planes < 0 || (n_planes > 0 && (!g_radii || !acc))) return PS_ERR_ARG;
    if (n_planes == 0) return PS_OK;
    k_radii_grad_accum<<<(n_planes + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        g_radii, plane_scale, scale, n_planes, acc);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

extern "C" ps_status ps_split_planes(const float* params, const float* m, const float* v,
                                     int n_scenes, const int* plane_ptr, int n_planes,
                                     const float* acc, int n_iter, float tau, float* params_out,
                                     float* m_out, float* v_out, int* plane_ptr_out,
                                     int capacity, int* split_rank, int* d_count, ps_stream stream)
{
    if (n_scenes <= 0 || n_planes < 0 || n_iter <= 0 || !(tau >= 0.f)) return PS_ERR_ARG;
    if (!plane_ptr || !plane_ptr_out || !split_rank || !d_count || !params_out) return PS_ERR_ARG;
    if (n_planes > 0 && (!params || !acc)) return PS_ERR_ARG;
    if (capacity < n_planes || n_planes >= (1 << 29)) return PS_ERR_ARG;
    SplitArgs a;
    a.params = params; a.m = m; a.v = v;
    a.n_scenes = n_scenes; a.plane_ptr = plane_ptr; a.P = n_planes;
    a.acc = acc;
    a.inv_n = 1.f / (float)n_iter; a.tau = tau;
    a.params_out = params_out; a.m_out = m_out; a.v_out = v_out;
    a.plane_ptr_out = plane_ptr_out; a.P_cap = capacity;
    a.split_rank = split_rank; a.d_count = d_count;
    k_split_planes<<<1, kSplitThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(a);
    PS_LAUNCH_CHECK();
    return PS_OK;
}
