// ps_init.cu -- nearest-neighbour distances for the initial plane radii.
//
// Sec. 3.1 starts every plane with all four radii equal to half the distance
// from its centre to the nearest other centre.  ps_nn_distance computes that
// distance exactly (the minimum over every other point, in FP32) for all
// points at once:
//   1. one CTA finds the bounding box and picks the cell edge of a uniform grid
//      (about one point per cell of the box's volume, thin boxes padded);
//   2. points are counted per hashed cell, the counts scanned, the point ids
//      scattered into per-cell runs (a counting sort by hash);
//   3. each point searches the cells around its own in shells of growing
//      Chebyshev radius r; a point within distance r * cell of the query lies in a
//      cell at most r away on every axis, so once the nearest point found is
//      within r * cell no unsearched cell can hold a nearer one.  Hash collisions
//      only add real points to a run, which never breaks the minimum.
#include "ps_internal.cuh"

namespace {

constexpr int kScanThreads = 1024;

struct NnHeader {
    float lo[3];
    float cell;
    float inv_cell;
    int r_max;          // shells beyond this radius cover the whole box
    unsigned mask;      // hash table size - 1
    int pad;
};

__host__ __device__ inline unsigned table_size(int n)
{
    unsigned t = 1024;
    while (t < 2u * (unsigned)n) t <<= 1;
    return t;
}

__device__ __forceinline__ unsigned cell_hash(int ix, int iy, int iz, unsigned mask)
{
    const unsigned h = ((unsigned)ix * 73856093u) ^ ((unsigned)iy * 19349663u) ^ ((unsigned)iz * 83492791u);
    return h & mask;
}

__device__ __forceinline__ void cell_of(const NnHeader& hd, float x, float y, float z, int& ix, int& iy,
                                        int& iz)
{
    ix = (int)floorf((x - hd.lo[0]) * hd.inv_cell);
    iy = (int)floorf((y - hd.lo[1]) * hd.inv_cell);
    iz = (int)floorf((z - hd.lo[2]) * hd.inv_cell);
}

// One CTA: bounding box, cell edge, shell limit, table mask.
__global__ void __launch_bounds__(kScanThreads) k_nn_setup(const float* __restrict__ p, int n, NnHeader* hd)
{
    __shared__ float red[6][kScanThreads / 32];
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float v = p[3 * i + c];
            mn[c] = fminf(mn[c], v);
            mx[c] = fmaxf(mx[c], v);
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[c] = fminf(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], o));
            mx[c] = fmaxf(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], o));
        }
        if (lane == 0) { red[c][w] = mn[c]; red[3 + c][w] = mx[c]; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float lo[3], hi[3];
        for (int c = 0; c < 3; ++c) {
            lo[c] = red[c][0]; hi[c] = red[3 + c][0];
            for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
                lo[c] = fminf(lo[c], red[c][i]);
                hi[c] = fmaxf(hi[c], red[3 + c][i]);
            }
        }
        const float ex = hi[0] - lo[0], ey = hi[1] - lo[1], ez = hi[2] - lo[2];
        const float diag = sqrtf(ex * ex + ey * ey + ez * ez);
        // a flat or thin box (points on a plane or a line) is padded, so the cell
        // edge follows the spacing of the points rather than collapsing to zero
        const float pad = 1e-3f * diag + 1e-6f;
        const double vol = (double)fmaxf(ex, pad) * fmaxf(ey, pad) * fmaxf(ez, pad);
        float cell = (float)cbrt(vol / (double)(n > 0 ? n : 1));
        if (!(cell > 0.f)) cell = 1e-6f;
        for (int c = 0; c < 3; ++c) hd->lo[c] = lo[c];
        hd->cell = cell;
        hd->inv_cell = 1.f / cell;
        const float rm = ceilf(diag / cell) + 1.f;
        hd->r_max = rm < 1e6f ? (int)rm : 1000000;
        hd->mask = table_size(n) - 1;
        hd->pad = 0;
    }
}

__global__ void k_nn_count(const float* __restrict__ p, int n, const NnHeader* __restrict__ hd,
                           unsigned* __restrict__ count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const NnHeader h = *hd;
    int ix, iy, iz;
    cell_of(h, p[3 * i], p[3 * i + 1], p[3 * i + 2], ix, iy, iz);
    atomicAdd(&count[cell_hash(ix, iy, iz, h.mask)], 1u);
}

// One CTA: start[t] = exclusive prefix of count (T + 1 entries), cursor = start.
__global__ void __launch_bounds__(kScanThreads) k_nn_scan(const unsigned* __restrict__ count, unsigned T,
                                                          unsigned* __restrict__ start,
                                                          unsigned* __restrict__ cursor)
{
    __shared__ unsigned wsum[kScanThreads / 32];
    __shared__ unsigned carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (unsigned base = 0; base < T; base += kScanThreads) {
        const unsigned i = base + threadIdx.x;
        const unsigned v = i < T ? count[i] : 0u;
        unsigned x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            unsigned s = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        const unsigned excl = carry + (w > 0 ? wsum[w - 1] : 0u) + x - v;
        if (i < T) { start[i] = excl; cursor[i] = excl; }
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[T] = carry;
}

__global__ void k_nn_scatter(const float* __restrict__ p, int n, const NnHeader* __restrict__ hd,
                             unsigned* __restrict__ cursor, int* __restrict__ sorted)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const NnHeader h = *hd;
    int ix, iy, iz;
    cell_of(h, p[3 * i], p[3 * i + 1], p[3 * i + 2], ix, iy, iz);
    const unsigned slot = atomicAdd(&cursor[cell_hash(ix, iy, iz, h.mask)], 1u);
    sorted[slot] = i;
}

__global__ void k_nn_query(const float* __restrict__ p, int n, const NnHeader* __restrict__ hd,
                           const unsigned* __restrict__ start, const int* __restrict__ sorted,
                           float* __restrict__ dist, float* __restrict__ radii, float scale,
                           float r_lo, float r_hi)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const NnHeader h = *hd;
    const float x = p[3 * i], y = p[3 * i + 1], z = p[3 * i + 2];
    int cx, cy, cz;
    cell_of(h, x, y, z, cx, cy, cz);
    float best = INFINITY;       // squared distance
    for (int r = 1; r <= h.r_max; ++r) {
        for (int dz = -r; dz <= r; ++dz) {
            for (int dy = -r; dy <= r; ++dy) {
                const bool face = (dz == -r || dz == r || dy == -r || dy == r);
                // on the shell of radius r (the whole cube for r = 1)
                const int step = (face || r == 1) ? 1 : 2 * r;
                for (int dx = -r; dx <= r; dx += step) {
                    const unsigned t = cell_hash(cx + dx, cy + dy, cz + dz, h.mask);
                    const unsigned b = __ldg(&start[t]), e = __ldg(&start[t + 1]);
                    for (unsigned s = b; s < e; ++s) {
                        const int j = __ldg(&sorted[s]);
                        if (j == i) continue;
                        const float ax = __ldg(&p[3 * j]) - x, ay = __ldg(&p[3 * j + 1]) - y,
                                    az = __ldg(&p[3 * j + 2]) - z;
                        const float d2 = fmaf(ax, ax, fmaf(ay, ay, az * az));
                        best = fminf(best, d2);
                    }
                }
            }
        }
        // (0.999: the cell coordinates are rounded FP32 products, so keep a margin)
        const float reach = (float)r * h.cell * 0.999f;
        if (best <= reach * reach) break;
    }
    const float d = sqrtf(best);
    if (dist) dist[i] = d;
    if (radii) {
        // Sec. 3.1: all four radii start at scale x the nearest-centre distance
        const float r = fminf(fmaxf(scale * d, r_lo), r_hi);
        reinterpret_cast<float4*>(radii)[i] = make_float4(r, r, r, r);
    }
}

size_t nn_ws_bytes(int n)
{
    const size_t T = table_size(n);
    // header, counts [T], starts [T + 1], cursors [T], sorted ids [n]
    return 64 + sizeof(unsigned) * (3 * T + 1) + sizeof(int) * (size_t)n + 64;
}

}  // namespace

extern "C" size_t ps_nn_workspace_bytes(int n)
{
    if (n < 0) return 0;
    return nn_ws_bytes(n);
}

extern "C" ps_status ps_nn_distance(const float* points, int n, float scale, float r_lo, float r_hi,
                                    float* dist, float* radii, void* ws, size_t ws_bytes,
                                    ps_stream stream)
{
    if (n < 0) return PS_ERR_ARG;
    if (n == 0) return PS_OK;
    if (!points || (!dist && !radii) || !ws) return PS_ERR_ARG;
    if (radii && ((reinterpret_cast<uintptr_t>(radii) & 15) || !(scale >= 0.f) || !(r_lo <= r_hi)))
        return PS_ERR_ARG;
    if (ws_bytes < nn_ws_bytes(n) || (reinterpret_cast<uintptr_t>(ws) & 15)) return PS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const unsigned T = table_size(n);
    char* base = static_cast<char*>(ws);
    NnHeader* hd = reinterpret_cast<NnHeader*>(base);
    unsigned* count = reinterpret_cast<unsigned*>(base + 64);
    unsigned* start = count + T;
    unsigned* cursor = start + T + 1;
    int* sorted = reinterpret_cast<int*>(cursor + T);
    PS_CUDA_CHECK(cudaMemsetAsync(count, 0, sizeof(unsigned) * T, st));
    k_nn_setup<<<1, kScanThreads, 0, st>>>(points, n, hd);
    PS_LAUNCH_CHECK();
    const int blocks = (n + 255) / 256;
    k_nn_count<<<blocks, 256, 0, st>>>(points, n, hd, count);
    PS_LAUNCH_CHECK();
    k_nn_scan<<<1, kScanThreads, 0, st>>>(count, T, start, cursor);
    PS_LAUNCH_CHECK();
    k_nn_scatter<<<blocks, 256, 0, st>>>(points, n, hd, cursor, sorted);
    PS_LAUNCH_CHECK();
    k_nn_query<<<blocks, 256, 0, st>>>(points, n, hd, start, sorted, dist, radii, scale, r_lo, r_hi);
    PS_LAUNCH_CHECK();
    return PS_OK;
}
