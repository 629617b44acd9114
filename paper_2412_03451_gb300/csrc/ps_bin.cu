// ps_bin.cu -- per-tile lists of records, sorted near to far.
//
// Sec. 3.2 ("Blending Composition") sorts the intersections of a ray near to
// far.  The renderer gets there in two stages: here every tile receives the
// records whose screen rectangle covers it, sorted by the record's depth key (a
// lower bound of every depth the plane can produce in that tile); the splat
// kernels then merge per pixel by exact depth.  Keys are unique per list as
// (key bits, record id), so the output does not depend on the order in which
// the atomics below land.
//
//   1. count:   tile_cnt[t] += 1 for every tile of every record's rectangle
//   2. scan:    tile_ptr = exclusive prefix sum of tile_cnt, total -> d_required
//   3. scatter: record ids into their tiles' slots (unordered, via cursors)
//   4. sort:    each tile's slots by (key, record id): shared-memory bitonic
//               sort up to kSortCap entries, an O(n^2) rank sort beyond.
#include "ps_internal.cuh"

using namespace ps;

namespace {

constexpr int kSortCap = 4096;    // entries sorted in shared memory (32 KB of u64)
constexpr int kScanThreads = 1024;

struct BinWs {
    int* tile_cnt;      // [n_tiles]
    int* cursor;        // [n_tiles]
    int* ent_tmp;       // [capacity] unordered entries
};

__host__ __device__ inline size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

inline BinWs carve(void* ws, int n_tiles, long long capacity)
{
    char* p = static_cast<char*>(ws);
    BinWs w;
    w.tile_cnt = reinterpret_cast<int*>(p); p += align_up(sizeof(int) * (size_t)n_tiles);
    w.cursor = reinterpret_cast<int*>(p); p += align_up(sizeof(int) * (size_t)n_tiles);
    w.ent_tmp = reinterpret_cast<int*>(p);
    (void)capacity;
    return w;
}

inline size_t ws_bytes(int n_tiles, long long capacity)
{
    return 2 * align_up(sizeof(int) * (size_t)n_tiles) + align_up(sizeof(int) * (size_t)capacity);
}

// 1. count -------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_count(const int4* __restrict__ rect,
                                                const ps_view* __restrict__ views,
                                                int* __restrict__ tile_cnt)
{
    const int v = blockIdx.y;
    const ps_view* vw = views + v;
    const int K = __ldg(&vw->K);
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int4 rc = __ldg(&rect[(long long)__ldg(&vw->rec_off) + k]);
    if (rc.z < rc.x || rc.w < rc.y) return;
    const int tx = __ldg(&vw->tiles_x), off = __ldg(&vw->tile_off);
    for (int y = rc.y; y <= rc.w; ++y)
        for (int x = rc.x; x <= rc.z; ++x) atomicAdd(&tile_cnt[off + y * tx + x], 1);
}

// 2. scan (one CTA) -------------------------------------------------------------
__global__ void __launch_bounds__(kScanThreads) k_scan(const int* __restrict__ tile_cnt, int n,
                                                       int* __restrict__ tile_ptr,
                                                       int* __restrict__ cursor,
                                                       long long capacity,
                                                       long long* __restrict__ d_required,
                                                       int* status)
{
    __shared__ long long s_warp[kScanThreads / 32];
    const int tid = threadIdx.x;
    const int per = (n + kScanThreads - 1) / kScanThreads;
    const int b = min(n, tid * per), e = min(n, b + per);
    long long sum = 0;
    for (int i = b; i < e; ++i) sum += tile_cnt[i];
    // block exclusive scan of the per-thread sums
    long long x = sum;
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        long long w = (lane < kScanThreads / 32) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kScanThreads / 32) s_warp[lane] = w;
    }
    __syncthreads();
    long long excl = x - sum + (wid > 0 ? s_warp[wid - 1] : 0);
    long long run = excl;
    for (int i = b; i < e; ++i) {
        const int c = tile_cnt[i];
        const int vptr = (int)min(run, capacity);
        tile_ptr[i] = vptr;
        cursor[i] = vptr;
        run += c;
    }
    if (tid == kScanThreads - 1) {
        tile_ptr[n] = (int)min(run, capacity);
        *d_required = run;
        if (run > capacity) set_status(status, PS_ERR_CAPACITY);
    }
}

// 3. scatter -------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_scatter(const int4* __restrict__ rect,
                                                  const ps_view* __restrict__ views,
                                                  const int* __restrict__ tile_ptr,
                                                  int* __restrict__ cursor,
                                                  int* __restrict__ ent_tmp)
{
    const int v = blockIdx.y;
    const ps_view* vw = views + v;
    const int K = __ldg(&vw->K);
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int r = __ldg(&vw->rec_off) + k;
    const int4 rc = __ldg(&rect[r]);
    if (rc.z < rc.x || rc.w < rc.y) return;
    const int tx = __ldg(&vw->tiles_x), off = __ldg(&vw->tile_off);
    for (int y = rc.y; y <= rc.w; ++y)
        for (int x = rc.x; x <= rc.z; ++x) {
            const int t = off + y * tx + x;
            const int pos = atomicAdd(&cursor[t], 1);
            // tile_ptr is clamped to capacity, so positions past it belong to
            // lists that did not fit: drop them (status already set)
            if (pos < __ldg(&tile_ptr[t + 1])) ent_tmp[pos] = r;
        }
}

// 4. sort ----------------------------------------------------------------------
__device__ __forceinline__ unsigned long long sort_key(const float* __restrict__ key, int r)
{
    return ((unsigned long long)__float_as_uint(__ldg(&key[r])) << 32) | (unsigned)r;
}

__global__ void __launch_bounds__(256) k_sort(const int* __restrict__ tile_ptr,
                                               const int* __restrict__ ent_tmp,
                                               const float* __restrict__ key,
                                               int* __restrict__ tile_ent)
{
    __shared__ unsigned long long s[kSortCap];
    const int t = blockIdx.x;
    const int b = tile_ptr[t], e = tile_ptr[t + 1];
    const int n = e - b;
    if (n <= 0) return;
    const int tid = threadIdx.x, NT = blockDim.x;
    if (n == 1) {
        if (tid == 0) tile_ent[b] = ent_tmp[b];
        return;
    }
    if (n <= kSortCap) {
        int N = 2;
        while (N < n) N <<= 1;
        for (int i = tid; i < N; i += NT)
            s[i] = i < n ? sort_key(key, ent_tmp[b + i]) : ~0ull;
        __syncthreads();
        for (int k = 2; k <= N; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = tid; i < N; i += NT) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const unsigned long long x = s[i], y = s[ixj];
                        const bool up = (i & k) == 0;
                        if ((x > y) == up) { s[i] = y; s[ixj] = x; }
                    }
                }
                __syncthreads();
            }
        }
        for (int i = tid; i < n; i += NT) tile_ent[b + i] = (int)(unsigned)(s[i] & 0xffffffffu);
        return;
    }
    // long list: rank of each element = number of smaller keys (keys unique)
    for (int i0 = 0; i0 < n; i0 += NT) {
        const int i = i0 + tid;
        const unsigned long long ki = i < n ? sort_key(key, ent_tmp[b + i]) : 0ull;
        int rank = 0;
        for (int c0 = 0; c0 < n; c0 += kSortCap) {
            const int cn = min(kSortCap, n - c0);
            __syncthreads();
            for (int j = tid; j < cn; j += NT) s[j] = sort_key(key, ent_tmp[b + c0 + j]);
            __syncthreads();
            if (i < n)
                for (int j = 0; j < cn; ++j) rank += s[j] < ki;
        }
        if (i < n) tile_ent[b + rank] = (int)(unsigned)(ki & 0xffffffffu);
    }
}

}  // namespace

extern "C" size_t ps_bin_workspace_bytes(const ps_frame* frame, long long capacity)
{
    if (!frame || frame->n_tiles < 0 || capacity < 0) return 0;
    return ws_bytes(frame->n_tiles, capacity);
}

extern "C" ps_status ps_bin_tiles(const ps_frame* frame, const ps_settings* s, const int* rect,
                                  const float* key, int* tile_ptr, int* tile_ent,
                                  long long capacity, long long* d_required, void* ws,
                                  size_t ws_bytes_, int* d_status, ps_stream stream)
{
    if (!frame || !s || !rect || !key || !tile_ptr || !d_required || !ws || !frame->views)
        return PS_ERR_ARG;
    if (capacity < 0 || capacity >= (1LL << 31) - 1) return PS_ERR_ARG;
    if (capacity > 0 && !tile_ent) return PS_ERR_ARG;
    if (frame->n_tiles <= 0) return PS_ERR_ARG;
    if (ws_bytes_ < ws_bytes(frame->n_tiles, capacity)) return PS_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(ws) & 255) return PS_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(rect) & 15) return PS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    BinWs w = carve(ws, frame->n_tiles, capacity);
    PS_CUDA_CHECK(cudaMemsetAsync(w.tile_cnt, 0, sizeof(int) * (size_t)frame->n_tiles, st));
    const int4* rc = reinterpret_cast<const int4*>(rect);
    if (frame->max_K > 0) {
        dim3 grid((frame->max_K + 127) / 128, frame->n_views);
        k_count<<<grid, 128, 0, st>>>(rc, frame->views, w.tile_cnt);
        PS_LAUNCH_CHECK();
    }
    k_scan<<<1, kScanThreads, 0, st>>>(w.tile_cnt, frame->n_tiles, tile_ptr, w.cursor, capacity,
                                        d_required, d_status);
    PS_LAUNCH_CHECK();
    if (frame->max_K > 0 && capacity > 0) {
        dim3 grid((frame->max_K + 127) / 128, frame->n_views);
        k_scatter<<<grid, 128, 0, st>>>(rc, frame->views, tile_ptr, w.cursor, w.ent_tmp);
        PS_LAUNCH_CHECK();
        k_sort<<<frame->n_tiles, 256, 0, st>>>(tile_ptr, w.ent_tmp, key, tile_ent);
        PS_LAUNCH_CHECK();
    }
    return PS_OK;
}
