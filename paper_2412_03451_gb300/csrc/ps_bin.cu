// ps_bin.cu -- per-tile lists of records, sorted near to far.
//
// Sec. 3.2 ("Blending Composition") sorts the intersections of a ray near to
// far.  The renderer gets there in two stages: here every tile receives the
// records whose screen rectangle covers it, each with a depth key that bounds
// from below every depth the plane can produce in that tile, sorted by it;
// the splat kernels then merge per pixel by exact depth.  Keys are unique per
// list as (key bits, record id), so the output does not depend on the order in
// which the atomics below land.
//
// Entry key (bit-exact specification, FP32 with correctly rounded + - * /
// only, no contraction): the rays of the pixel centres at the tile's four
// corner pixels, d = ((x + 0.5 - cx) / fx, (y + 0.5 - cy) / fy, 1); per ray
// den = (n_x d_x + n_y d_y) + n_z and t = s / den with the record's f32 n_c and
// s = n_c . p_c.  Over the tile the depth s / (d . n_c) of the plane is
// linear-fractional in the ray, so if den has one sign at all four corners (and
// |den| > 0.01 (|n_x d_x| + |n_y d_y| + |n_z|) at each, which keeps FP32
// cancellation small) its range over the tile is spanned by the corners:
// c = max(min t, z_near), or +inf if max t <= z_near (no depth in range);
// otherwise c = z_near.  The entry key is max(c, the record's key), both lower
// bounds of every depth the plane produces in the tile.  Unlike the record key
// alone (the smallest z of the whole widened quad), this bound is as tight as
// the tile: entries of large or oblique planes no longer all sort to the front
// of every list.
//
//   1. record counts: tiles covered by each record's rectangle (+ the record's
//      first global tile and rectangle width), then an exclusive scan over
//      records numbers every (record, tile) pair.  The same thread marks its
//      rectangle in a difference array over the flat (view-major, row-major)
//      tile index: +1 where each row segment starts, -1 one past its end (the
//      whole rectangle is one segment when it spans the full width);
//   2. tile scan: the inclusive prefix of the difference array is the number
//      of records covering each tile, and tile_ptr is the exclusive prefix of
//      that, both in one pass; total -> d_required;
//   3. scatter: one thread per pair writes its record id and entry key into a
//      slot of its tile (unordered, via per-tile cursors);
//   4. sort: each tile's slots by (key, record id): one warp per tile sorts up
//      to kWarpSortCap entries in registers (a bitonic network over 1, 2, 4 or
//      8 keys per lane); persistent CTAs take the longer lists
//      (bitonic up to kSortCap entries, an O(n^2) rank sort beyond).
// Every pair gets its own thread, so a plane covering a thousand tiles costs
// no more latency than one covering a single tile.
#include "ps_internal.cuh"

#include <cooperative_groups.h>

using namespace ps;

namespace {

constexpr int kSortCap = 4096;     // entries sorted in shared memory by a CTA (32 KB of u64)
constexpr int kWarpSortCap = 256;  // entries sorted by one warp, in registers (8 per lane)
constexpr int kSortWarps = 8;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 9;      // elements per thread per scan tile (odd: a thread's run
                                   // starts 9 words after its neighbour's, no bank conflicts)
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kFlatBlocks = 152 * 8;
constexpr int kSortBlocks = 152 * 4;  // persistent blocks of the long-list sort
constexpr int kPairBlock = 256;       // pairs per scatter block = pairs per chunk of the chunk table

inline long long n_chunks(long long capacity) { return capacity / kPairBlock + 2; }

struct BinWs {
    int* rec_cnt;       // [R + 1] tiles per record -> exclusive prefix (pair numbering)
    int4* rec_info;     // [R] first global tile, rectangle width in tiles, tiles_x, view
    int* tile_cnt;      // [n_tiles] difference array of the tile counts
    int* cursor;        // [n_tiles]
    int* count;         // [n_tiles + 1] tile counts (arrays beyond one scan CTA)
    int* chunk_first;   // [n_chunks] record holding pair c * kPairBlock
    long long* part;    // [2 * max scan tiles] scan partial sums
    int* ent_tmp;       // [capacity] unordered entries
    float* key_tmp;     // [capacity] their keys
};

inline size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

inline int scan_tiles(long long n) { return (int)((n + kScanTile - 1) / kScanTile); }

inline size_t ws_bytes(int R, int n_tiles, long long capacity)
{
    const int parts = 2 * (scan_tiles(R + 1) > scan_tiles(n_tiles) ? scan_tiles(R + 1) : scan_tiles(n_tiles)) + 2;
    return align_up(sizeof(int) * (size_t)(R + 1)) + align_up(sizeof(int4) * (size_t)(R > 0 ? R : 1)) +
           2 * align_up(sizeof(int) * (size_t)n_tiles) + align_up(sizeof(int) * (size_t)(n_tiles + 1)) +
           align_up(sizeof(long long) * (size_t)parts) + align_up(sizeof(int) * (size_t)n_chunks(capacity)) +
           2 * align_up(sizeof(int) * (size_t)(capacity > 0 ? capacity : 1));
}

inline BinWs carve(void* ws, int R, int n_tiles, long long capacity)
{
    char* p = static_cast<char*>(ws);
    BinWs w;
    w.rec_cnt = reinterpret_cast<int*>(p); p += align_up(sizeof(int) * (size_t)(R + 1));
    w.rec_info = reinterpret_cast<int4*>(p); p += align_up(sizeof(int4) * (size_t)(R > 0 ? R : 1));
    w.tile_cnt = reinterpret_cast<int*>(p); p += align_up(sizeof(int) * (size_t)n_tiles);
    w.cursor = reinterpret_cast<int*>(p); p += align_up(sizeof(int) * (size_t)n_tiles);
    w.count = reinterpret_cast<int*>(p); p += align_up(sizeof(int) * (size_t)(n_tiles + 1));
    w.chunk_first = reinterpret_cast<int*>(p); p += align_up(sizeof(int) * (size_t)n_chunks(capacity));
    const int parts = 2 * (scan_tiles(R + 1) > scan_tiles(n_tiles) ? scan_tiles(R + 1) : scan_tiles(n_tiles)) + 2;
    w.part = reinterpret_cast<long long*>(p); p += align_up(sizeof(long long) * (size_t)parts);
    w.ent_tmp = reinterpret_cast<int*>(p);
    p += align_up(sizeof(int) * (size_t)(capacity > 0 ? capacity : 1));
    w.key_tmp = reinterpret_cast<float*>(p);
    return w;
}

// 1. record counts ---------------------------------------------------------------
__global__ void __launch_bounds__(128) k_rec_count(const int4* __restrict__ rect,
                                                    const ps_view* __restrict__ views,
                                                    int* __restrict__ rec_cnt,
                                                    int4* __restrict__ rec_info,
                                                    int* __restrict__ diff, int n_tiles)
{
    const int v = blockIdx.y;
    const ps_view* vw = views + v;
    const int K = __ldg(&vw->K);
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int r = __ldg(&vw->rec_off) + k;
    const int4 rc = __ldg(&rect[r]);
    const int tx = __ldg(&vw->tiles_x);
    int c = 0;
    int4 info = make_int4(0, 1, tx, v);
    if (rc.z >= rc.x && rc.w >= rc.y) {
        const int w = rc.z - rc.x + 1;
        c = w * (rc.w - rc.y + 1);
        const int first = __ldg(&vw->tile_off) + rc.y * tx + rc.x;
        info = make_int4(first, w, tx, v);
        if (w == tx) {
            // full rows: one contiguous run of c tiles
            atomicAdd(&diff[first], 1);
            if (first + c < n_tiles) atomicAdd(&diff[first + c], -1);
        } else {
            const int last = first + (rc.w - rc.y) * tx;   // first tile of the last row
            for (int a = first; a <= last; a += tx) {
                atomicAdd(&diff[a], 1);
                if (a + w < n_tiles) atomicAdd(&diff[a + w], -1);
            }
        }
    }
    rec_cnt[r] = c;
    rec_info[r] = info;
}

// Exclusive scan of int counts in three passes (tile sums, scan of the sums,
// tile scan + offset).  The last pass can clamp the offsets to a capacity and
// copy them to a cursor array (tile lists) and reports the total.
__device__ __forceinline__ long long block_scan_excl(long long x, long long* s_warp, long long& total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        long long w = (lane < (int)(blockDim.x >> 5)) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;   // inclusive warp totals
    }
    __syncthreads();
    total = s_warp[(blockDim.x >> 5) - 1];
    const long long r = incl - x + (wid > 0 ? s_warp[wid - 1] : 0);
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(const int* __restrict__ in, int n,
                                                            long long* __restrict__ part)
{
    __shared__ long long s_warp[32];
    const long long base = (long long)blockIdx.x * kScanTile;
    long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const long long j = base + (long long)i * kScanThreads + threadIdx.x;
        if (j < n) s += in[j];
    }
    long long total;
    block_scan_excl(s, s_warp, total);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_parts(long long* __restrict__ part, int nparts)
{
    // one block: exclusive scan of the tile sums in place (nparts <= 1024 * 8)
    __shared__ long long s_warp[32];
    __shared__ long long s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nparts; b0 += kScanThreads) {
        const int j = b0 + threadIdx.x;
        const long long x = j < nparts ? part[j] : 0;
        long long total;
        const long long e = block_scan_excl(x, s_warp, total);
        if (j < nparts) part[j] = e + s_carry;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) part[nparts] = s_carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int* __restrict__ in, int n,
                                                             const long long* __restrict__ part,
                                                             int nparts, int* __restrict__ out,
                                                             int* __restrict__ cursor,
                                                             long long capacity,
                                                             long long* __restrict__ d_total,
                                                             int* status)
{
    __shared__ long long s_warp[32];
    __shared__ int s_in[kScanTile];
    const long long base = (long long)blockIdx.x * kScanTile;
    // coalesced load of the tile
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const long long j = base + (long long)i * kScanThreads + threadIdx.x;
        s_in[i * kScanThreads + threadIdx.x] = j < n ? in[j] : 0;
    }
    __syncthreads();
    // each thread scans kScanItems consecutive elements
    long long loc[kScanItems];
    long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        loc[i] = s;
        s += s_in[threadIdx.x * kScanItems + i];
    }
    long long total;
    const long long e = block_scan_excl(s, s_warp, total) + part[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const long long j = base + (long long)threadIdx.x * kScanItems + i;
        if (j < n) {
            long long v = e + loc[i];
            if (v > capacity) v = capacity;
            out[j] = (int)v;
            if (cursor) cursor[j] = (int)v;
        }
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        const long long tot = part[nparts];
        out[n] = (int)(tot < capacity ? tot : capacity);
        if (d_total) *d_total = tot;
        if (status && tot > capacity) set_status(status, PS_ERR_CAPACITY);
    }
}

// Arrays of up to kScanOneMax elements: one launch, one thread-block cluster
// of kScanCtas CTAs per array.  Each CTA scans its own segment in shared memory
// (each thread a contiguous run, a block scan joining the runs), publishes the
// segment's aggregate in its shared memory, and after a cluster barrier reads
// the aggregates of the lower-ranked CTAs through distributed shared memory to
// get its carry.  With `twice`, the array is first replaced by its inclusive
// prefix (a difference array becomes the counts): a segment's aggregate is then
// (sum of its differences D, sum of its carry-free counts S, length L), and
// segments compose in order as (D1 + D2, S1 + S2 + L2 D1, L1 + L2).  With
// chunk_first, the store pass also writes the chunk table of the pair numbering
// (see k_chunk_first).  One launch runs one or two such jobs (one cluster each).
constexpr int kScanOneMax = 48 * 1024;
constexpr int kScanCtas = 8;             // CTAs per cluster (the portable maximum)

struct ScanJob {
    const int* in;
    int n;
    int* out;             // [n + 1] exclusive prefix clamped to capacity, out[n] = total
    int* cursor;          // optional copy of out[0 .. n)
    long long capacity;
    long long* d_total;   // optional
    int* status;          // optional: PS_ERR_CAPACITY when the total exceeds capacity
    int twice;
    int* chunk_first;     // optional chunk table [n_chunk]
    long long n_chunk;
};

__global__ void __cluster_dims__(kScanCtas, 1, 1) __launch_bounds__(kScanThreads)
k_scan_one(ScanJob j0, ScanJob j1)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ int s_seg[];
    __shared__ long long s_warp[32];
    __shared__ long long s_agg[3];
    const int rank = (int)cl.block_rank();
    const ScanJob& a = blockIdx.x < kScanCtas ? j0 : j1;
    const int n = a.n;
    // segments of a multiple of 4 elements: 16-byte accesses stay aligned
    const int seg = ((n + kScanCtas - 1) / kScanCtas + 3) & ~3;
    const int lo = min(rank * seg, n), m = min(lo + seg, n) - lo;
    const bool in_al = ((reinterpret_cast<uintptr_t>(a.in) | (size_t)lo * 4) & 15) == 0;
    const int m4 = in_al ? m >> 2 : 0;
    for (int j = threadIdx.x; j < m4; j += kScanThreads)
        reinterpret_cast<int4*>(s_seg)[j] = __ldg(reinterpret_cast<const int4*>(a.in + lo) + j);
    for (int j = 4 * m4 + threadIdx.x; j < m; j += kScanThreads) s_seg[j] = a.in[lo + j];
    __syncthreads();
    // contiguous runs of an odd length: the runs of a warp's threads start in 32
    // different banks, so the strided shared-memory passes below are conflict-free
    const int per = ((m + kScanThreads - 1) / kScanThreads) | 1;
    const int b = min((int)threadIdx.x * per, m), e = min(b + per, m);
    long long D = 0;
    if (a.twice) {
        int run = 0;
        for (int j = b; j < e; ++j) run += s_seg[j];
        long long c = block_scan_excl(run, s_warp, D);
        for (int j = b; j < e; ++j) {
            c += s_seg[j];
            s_seg[j] = (int)c;       // the count without the carry of the lower segments
        }
        __syncthreads();
    }
    long long sum = 0;
    for (int j = b; j < e; ++j) sum += s_seg[j];
    long long S;
    long long v = block_scan_excl(sum, s_warp, S);
    if (threadIdx.x == 0) { s_agg[0] = D; s_agg[1] = S; s_agg[2] = m; }
    cl.sync();
    long long cD = 0, cC = 0;    // carries: differences and counts of the lower segments
    for (int r = 0; r < rank; ++r) {
        const long long* g = cl.map_shared_rank(s_agg, r);
        cC += g[1] + g[2] * cD;
        cD += g[0];
    }
    cl.sync();                   // every rank has read the aggregates before any exits
    // offset of element j = cC + (j - lo) cD + (exclusive sum of the carry-free values)
    v += cC + (long long)b * cD;
    for (int j = b; j < e; ++j) {
        const long long x = s_seg[j] + cD;
        s_seg[j] = (int)(v < a.capacity ? v : a.capacity);
        v += x;
    }
    const long long seg_end = cC + (long long)m * cD + S;   // offset just past the segment
    __syncthreads();
    const long long cap_end = seg_end < a.capacity ? seg_end : a.capacity;
    const bool out_al = ((reinterpret_cast<uintptr_t>(a.out) | reinterpret_cast<uintptr_t>(a.cursor) |
                          (size_t)lo * 4) & 15) == 0;
    const int s4 = out_al ? m >> 2 : 0;
    for (int j = threadIdx.x; j < s4; j += kScanThreads) {
        const int4 x = reinterpret_cast<const int4*>(s_seg)[j];
        reinterpret_cast<int4*>(a.out + lo)[j] = x;
        if (a.cursor) reinterpret_cast<int4*>(a.cursor + lo)[j] = x;
    }
    for (int j = 4 * s4 + threadIdx.x; j < m; j += kScanThreads) {
        const int x = s_seg[j];
        a.out[lo + j] = x;
        if (a.cursor) a.cursor[lo + j] = x;
    }
    if (a.chunk_first) {
        for (int j = threadIdx.x; j < m; j += kScanThreads) {
            const int x = s_seg[j];
            const long long hi = j + 1 < m ? s_seg[j + 1] : cap_end;
            for (long long c = ((long long)x + kPairBlock - 1) / kPairBlock;
                 c < a.n_chunk && c * kPairBlock < hi; ++c)
                a.chunk_first[c] = lo + j;
        }
    }
    if (rank == kScanCtas - 1 && threadIdx.x == 0) {
        a.out[n] = (int)cap_end;
        if (a.d_total) *a.d_total = seg_end;
        if (a.status && seg_end > a.capacity) set_status(a.status, PS_ERR_CAPACITY);
    }
}

// One or two cluster scans in one launch (both arrays <= kScanOneMax).
cudaError_t scan_one(const ScanJob& j0, const ScanJob* j1, cudaStream_t st)
{
    int n = j0.n > 0 ? j0.n : 1;
    if (j1 && j1->n > n) n = j1->n;
    const size_t seg = (size_t)((n + kScanCtas - 1) / kScanCtas + 3) & ~(size_t)3;
    k_scan_one<<<(j1 ? 2 : 1) * kScanCtas, kScanThreads, sizeof(int) * seg, st>>>(j0, j1 ? *j1 : j0);
    return cudaGetLastError();
}

cudaError_t scan_exclusive(const int* in, int n, int* out, int* cursor, long long capacity,
                           long long* part, long long* d_total, int* status, cudaStream_t st,
                           int* twice_tmp = nullptr)
{
    if (n <= kScanOneMax) {
        const ScanJob j{in, n, out, cursor, capacity, d_total, status, twice_tmp ? 1 : 0, nullptr, 0};
        return scan_one(j, nullptr, st);
    }
    if (twice_tmp) {
        // inclusive prefix of in = the exclusive one shifted by one (twice_tmp [n + 1])
        cudaError_t e = scan_exclusive(in, n, twice_tmp, nullptr, (1LL << 31) - 1, part, nullptr,
                                       nullptr, st);
        if (e != cudaSuccess) return e;
        in = twice_tmp + 1;
    }
    const int nparts = scan_tiles(n > 0 ? n : 1);
    k_scan_sums<<<nparts, kScanThreads, 0, st>>>(in, n, part);
    k_scan_parts<<<1, kScanThreads, 0, st>>>(part, nparts);
    k_scan_apply<<<nparts, kScanThreads, 0, st>>>(in, n, part, nparts, out, cursor, capacity,
                                                  d_total, status);
    return cudaGetLastError();
}

// 3. one thread per (record, tile) pair ----------------------------------------
__device__ __forceinline__ int pair_record(const int* __restrict__ off, int lo, int hi, int i)
{
    // last r in [lo, hi] with off[r] <= i (off is non-decreasing, off[lo] <= i)
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&off[mid]) <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// chunk_first[c] = the record holding pair c * kPairBlock, for every chunk
// c < n_chunk that starts below the pair total (one thread per record).
__global__ void __launch_bounds__(256) k_chunk_first(const int* __restrict__ off, int R,
                                                      int* __restrict__ chunk_first, long long n_chunk)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const long long lo = __ldg(&off[r]), hi = __ldg(&off[r + 1]);
    for (long long c = (lo + kPairBlock - 1) / kPairBlock; c < n_chunk && c * kPairBlock < hi; ++c)
        chunk_first[c] = r;
}

// Pairs base .. base + kPairBlock - 1 of a block belong to records x .. y of the
// result: the chunk table gives the records holding this chunk's first pair and
// the next chunk's (an upper bound); beyond the table the whole record range is
// searched.  Every thread of the block computes the same two values (broadcast
// loads, no barrier) and then searches only that narrow range for its own pair.
__device__ __forceinline__ int2 chunk_record_range(const int* __restrict__ off, int R, int E, int base,
                                                   const int* __restrict__ chunk_first, long long n_chunk)
{
    const long long c = base / kPairBlock;
    const int lo = (c < n_chunk && c * kPairBlock < E) ? __ldg(&chunk_first[c])
                                                       : pair_record(off, 0, R - 1, base);
    const int hi = (c + 1 < n_chunk && (c + 1) * kPairBlock < E)
                       ? __ldg(&chunk_first[c + 1])
                       : pair_record(off, 0, R - 1, min(base + kPairBlock, E) - 1);
    return make_int2(lo, hi);
}

// The entry key of the specification above.
__device__ __forceinline__ float entry_key(float4 ns, const ps_view* __restrict__ vw, int tx, int ty,
                                           int tw, int th, float z_near)
{
    const float fx = __ldg(&vw->fx), fy = __ldg(&vw->fy), cx = __ldg(&vw->cx), cy = __ldg(&vw->cy);
    const float xs[2] = {(float)(tx * tw), (float)(tx * tw + tw - 1)};
    const float ys[2] = {(float)(ty * th), (float)(ty * th + th - 1)};
    int npos = 0, nneg = 0;
    bool weak = false;
    // the corners' den of largest and of smallest magnitude
    float dbig = 0.f, dsmall = INFINITY;
    const float dys[2] = {__fdiv_rn(__fsub_rn(__fadd_rn(ys[0], 0.5f), cy), fy),
                          __fdiv_rn(__fsub_rn(__fadd_rn(ys[1], 0.5f), cy), fy)};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float dx = __fdiv_rn(__fsub_rn(__fadd_rn(xs[a], 0.5f), cx), fx);
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const float dy = dys[b];
            const float p1 = __fmul_rn(ns.x, dx), p2 = __fmul_rn(ns.y, dy);
            const float den = __fadd_rn(__fadd_rn(p1, p2), ns.z);
            const float mag = __fadd_rn(__fadd_rn(fabsf(p1), fabsf(p2)), fabsf(ns.z));
            if (!(fabsf(den) > __fmul_rn(0.01f, mag))) weak = true;
            npos += den > 0.f;
            nneg += den < 0.f;
            if (fabsf(den) > fabsf(dbig)) dbig = den;
            if (fabsf(den) < fabsf(dsmall)) dsmall = den;
        }
    }
    if (weak || (npos != 4 && nneg != 4)) return z_near;
    // With one sign of den at the four corners, t = s / den has one sign and its
    // magnitude falls as |den| grows; correctly rounded division is monotone and
    // odd, so the extremes of the four rounded quotients are the quotients by the
    // extreme dens: the same bits as taking all four.
    const float ta = __fdiv_rn(ns.w, dbig), tb = __fdiv_rn(ns.w, dsmall);
    const float tmin = fminf(ta, tb), tmax = fmaxf(ta, tb);
    if (!(tmax > z_near)) return INFINITY;
    return fmaxf(tmin, z_near);
}

__global__ void __launch_bounds__(kPairBlock) k_pair_scatter(const int* __restrict__ rec_off, int R,
                                                       const int4* __restrict__ rec_info,
                                                       const int* __restrict__ tile_ptr,
                                                       int* __restrict__ cursor,
                                                       int* __restrict__ ent_tmp,
                                                       float* __restrict__ key_tmp,
                                                       const float4* __restrict__ rec,
                                                       const float* __restrict__ rec_key,
                                                       const ps_view* __restrict__ views,
                                                       int tw, int th, float z_near,
                                                       const int* __restrict__ chunk_first,
                                                       long long n_chunk)
{
    const int E = __ldg(&rec_off[R]);
    for (int base = blockIdx.x * kPairBlock; base < E; base += gridDim.x * kPairBlock) {
        const int2 rg = chunk_record_range(rec_off, R, E, base, chunk_first, n_chunk);
        const int i = base + threadIdx.x;
        if (i < E) {
            const int r = pair_record(rec_off, rg.x, rg.y, i);
            const int4 info = __ldg(&rec_info[r]);
            const int j = i - __ldg(&rec_off[r]);
            const int t = info.x + (j / info.y) * info.z + (j % info.y);
            // the key first, so that the slot atomic's latency overlaps nothing it waits on
            const ps_view* vw = views + info.w;
            const int lt = t - __ldg(&vw->tile_off);
            const float k = fmaxf(entry_key(__ldg(&rec[4 * (size_t)r]), vw, lt % info.z, lt / info.z,
                                            tw, th, z_near),
                                  __ldg(&rec_key[r]));
            const int lim = __ldg(&tile_ptr[t + 1]);
            const int pos = atomicAdd(&cursor[t], 1);
            // tile_ptr is clamped to the capacity: positions past it belong to lists
            // that did not fit and are dropped (the status word says so)
            if (pos < lim) {
                ent_tmp[pos] = r;
                key_tmp[pos] = k;
            }
        }
    }
}

// 4. sort -----------------------------------------------------------------------
// (key bits, record id) of slot j: keys are positive or +inf, so their bits sort like the values
__device__ __forceinline__ unsigned long long sort_key(const float* __restrict__ key_tmp,
                                                       const int* __restrict__ ent_tmp, int j)
{
    return ((unsigned long long)__float_as_uint(key_tmp[j]) << 32) | (unsigned)ent_tmp[j];
}

__device__ __forceinline__ void put(int* __restrict__ tile_ent, float* __restrict__ tile_key, int j,
                                    unsigned long long v)
{
    tile_ent[j] = (int)(unsigned)(v & 0xffffffffu);
    tile_key[j] = __uint_as_float((unsigned)(v >> 32));
}

// Bitonic network over 32 E keys held E per lane, key e * 32 + lane in v[e]:
// partners closer than 32 are in other lanes (shuffles), farther ones in the
// same lane (compare-exchange in registers).
template <int E>
__device__ __forceinline__ void warp_bitonic(unsigned long long (&v)[E], int lane)
{
#pragma unroll
    for (int k = 2; k <= 32 * E; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int je = j >> 5;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if ((e & je) == 0) {
                        const bool up = ((e * 32 + lane) & k) == 0;
                        const unsigned long long a = v[e], b = v[e + je];
                        const bool sw = (a > b) == up;
                        v[e] = sw ? b : a;
                        v[e + je] = sw ? a : b;
                    }
                }
            } else {
                const bool lower = (lane & j) == 0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const unsigned long long o = __shfl_xor_sync(0xffffffffu, v[e], j);
                    const bool up = ((e * 32 + lane) & k) == 0;
                    v[e] = (lower == up) ? (v[e] < o ? v[e] : o) : (v[e] < o ? o : v[e]);
                }
            }
        }
    }
}

template <int E>
__device__ __forceinline__ void warp_sort_list(const int* __restrict__ ent_tmp,
                                               const float* __restrict__ key_tmp,
                                               int* __restrict__ tile_ent, float* __restrict__ tile_key,
                                               int b, int n, int lane)
{
    unsigned long long v[E];
#pragma unroll
    for (int e = 0; e < E; ++e)
        v[e] = e * 32 + lane < n ? sort_key(key_tmp, ent_tmp, b + e * 32 + lane) : ~0ull;
    warp_bitonic<E>(v, lane);
#pragma unroll
    for (int e = 0; e < E; ++e)
        if (e * 32 + lane < n) put(tile_ent, tile_key, b + e * 32 + lane, v[e]);
}

// Short lists: one warp per tile.
__global__ void __launch_bounds__(kSortWarps * 32) k_sort_warp(const int* __restrict__ tile_ptr,
                                                               int n_tiles,
                                                               const int* __restrict__ ent_tmp,
                                                               const float* __restrict__ key_tmp,
                                                               int* __restrict__ tile_ent,
                                                               float* __restrict__ tile_key)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * kSortWarps + w;
    if (t >= n_tiles) return;
    const int b = tile_ptr[t], e = tile_ptr[t + 1];
    const int n = e - b;
    if (n <= 0 || n > kWarpSortCap) return;
    if (n == 1) {
        if (lane == 0) { tile_ent[b] = ent_tmp[b]; tile_key[b] = key_tmp[b]; }
        return;
    }
    if (n <= 32) { warp_sort_list<1>(ent_tmp, key_tmp, tile_ent, tile_key, b, n, lane); return; }
    if (n <= 64) { warp_sort_list<2>(ent_tmp, key_tmp, tile_ent, tile_key, b, n, lane); return; }
    if (n <= 128) { warp_sort_list<4>(ent_tmp, key_tmp, tile_ent, tile_key, b, n, lane); return; }
    warp_sort_list<8>(ent_tmp, key_tmp, tile_ent, tile_key, b, n, lane);
}

// Long lists: one CTA per tile (tiles with at most kWarpSortCap entries return at once).
__device__ void sort_long_list(const int* __restrict__ ent_tmp, const float* __restrict__ key_tmp,
                               int* __restrict__ tile_ent, float* __restrict__ tile_key, int b, int n,
                               unsigned long long* s);

// Blocks stride over the tiles 256 at a time: each thread checks one list
// length, the long lists found are sorted one after the other by the block.
__global__ void __launch_bounds__(256) k_sort(const int* __restrict__ tile_ptr, int n_tiles,
                                               const int* __restrict__ ent_tmp,
                                               const float* __restrict__ key_tmp,
                                               int* __restrict__ tile_ent,
                                               float* __restrict__ tile_key)
{
    __shared__ unsigned long long s[kSortCap];
    __shared__ int s_list[256];
    __shared__ int s_cnt;
    for (int t0 = blockIdx.x * 256; t0 < n_tiles; t0 += gridDim.x * 256) {
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        const int t = t0 + threadIdx.x;
        if (t < n_tiles && tile_ptr[t + 1] - tile_ptr[t] > kWarpSortCap)
            s_list[atomicAdd(&s_cnt, 1)] = t;
        __syncthreads();
        const int cnt = s_cnt;
        for (int q = 0; q < cnt; ++q) {
            const int tt = s_list[q];
            const int b = tile_ptr[tt];
            sort_long_list(ent_tmp, key_tmp, tile_ent, tile_key, b, tile_ptr[tt + 1] - b, s);
        }
        __syncthreads();
    }
}

__device__ void sort_long_list(const int* __restrict__ ent_tmp, const float* __restrict__ key_tmp,
                               int* __restrict__ tile_ent, float* __restrict__ tile_key, int b, int n,
                               unsigned long long* s)
{
    const int tid = threadIdx.x, NT = blockDim.x;
    if (n <= kSortCap) {
        int N = 2;
        while (N < n) N <<= 1;
        for (int i = tid; i < N; i += NT)
            s[i] = i < n ? sort_key(key_tmp, ent_tmp, b + i) : ~0ull;
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
        for (int i = tid; i < n; i += NT) put(tile_ent, tile_key, b + i, s[i]);
        __syncthreads();    // the block's next list reuses s
        return;
    }
    // rank of each element = number of smaller keys (keys are unique)
    for (int i0 = 0; i0 < n; i0 += NT) {
        const int i = i0 + tid;
        const unsigned long long ki = i < n ? sort_key(key_tmp, ent_tmp, b + i) : 0ull;
        int rank = 0;
        for (int c0 = 0; c0 < n; c0 += kSortCap) {
            const int cn = min(kSortCap, n - c0);
            __syncthreads();
            for (int j = tid; j < cn; j += NT) s[j] = sort_key(key_tmp, ent_tmp, b + c0 + j);
            __syncthreads();
            if (i < n)
                for (int j = 0; j < cn; ++j) rank += s[j] < ki;
        }
        if (i < n) put(tile_ent, tile_key, b + rank, ki);
    }
    __syncthreads();    // the block's next list reuses s
}

}  // namespace

extern "C" size_t ps_bin_workspace_bytes(const ps_frame* frame, long long capacity)
{
    if (!frame || frame->n_tiles < 0 || frame->n_records < 0 || capacity < 0) return 0;
    return ws_bytes(frame->n_records, frame->n_tiles, capacity);
}

extern "C" ps_status ps_bin_tiles(const ps_frame* frame, const ps_settings* s, const float* rec,
                                  const int* rect, const float* key, int* tile_ptr, int* tile_ent,
                                  float* tile_key, long long capacity, long long* d_required,
                                  void* ws, size_t ws_bytes_, int* d_status, ps_stream stream)
{
    if (!frame || !s || !rec || !rect || !key || !tile_ptr || !d_required || !ws || !frame->views)
        return PS_ERR_ARG;
    if (capacity < 0 || capacity >= (1LL << 31) - 1) return PS_ERR_ARG;
    if (capacity > 0 && (!tile_ent || !tile_key)) return PS_ERR_ARG;
    if (s->tile_w <= 0 || s->tile_h <= 0 || !(s->z_near > 0.f)) return PS_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(rec) & 15) return PS_ERR_ARG;
    if (frame->n_tiles <= 0 || frame->n_records < 0) return PS_ERR_ARG;
    const int R = frame->n_records;
    if (ws_bytes_ < ws_bytes(R, frame->n_tiles, capacity)) return PS_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(ws) & 255) return PS_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(rect) & 15) return PS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    BinWs w = carve(ws, R, frame->n_tiles, capacity);
    PS_CUDA_CHECK(cudaMemsetAsync(w.tile_cnt, 0, sizeof(int) * (size_t)frame->n_tiles, st));
    const int4* rc = reinterpret_cast<const int4*>(rect);
    const long long nch = n_chunks(capacity);
    if (R > 0) {
        dim3 grid((frame->max_K + 127) / 128, frame->n_views);
        k_rec_count<<<grid, 128, 0, st>>>(rc, frame->views, w.rec_cnt, w.rec_info, w.tile_cnt,
                                          frame->n_tiles);
        PS_LAUNCH_CHECK();
    }
    // Pair numbering: offsets clamp at the int range (still non-decreasing), so pairs
    // past it are never scattered, and the tile total then exceeds every capacity.
    if (R > 0 && R <= kScanOneMax && frame->n_tiles <= kScanOneMax) {
        // the pair numbering (and its chunk table) and the tile counts and offsets are
        // independent: one launch, one CTA each
        const ScanJob jr{w.rec_cnt, R, w.rec_cnt, nullptr, (1LL << 31) - 1, nullptr, nullptr, 0,
                         w.chunk_first, nch};
        const ScanJob jt{w.tile_cnt, frame->n_tiles, tile_ptr, w.cursor, capacity, d_required,
                         d_status, 1, nullptr, 0};
        if (scan_one(jr, &jt, st) != cudaSuccess) return PS_ERR_CUDA;
    } else {
        if (R > 0) {
            if (scan_exclusive(w.rec_cnt, R, w.rec_cnt, nullptr, (1LL << 31) - 1, w.part, nullptr,
                               nullptr, st) != cudaSuccess)
                return PS_ERR_CUDA;
            k_chunk_first<<<(R + 255) / 256, 256, 0, st>>>(w.rec_cnt, R, w.chunk_first, nch);
            PS_LAUNCH_CHECK();
        }
        if (scan_exclusive(w.tile_cnt, frame->n_tiles, tile_ptr, w.cursor, capacity, w.part,
                           d_required, d_status, st, w.count) != cudaSuccess)
            return PS_ERR_CUDA;
    }
    if (R > 0 && capacity > 0) {
        k_pair_scatter<<<kFlatBlocks, kPairBlock, 0, st>>>(w.rec_cnt, R, w.rec_info, tile_ptr, w.cursor,
                                                           w.ent_tmp, w.key_tmp,
                                                           reinterpret_cast<const float4*>(rec), key,
                                                           frame->views, s->tile_w, s->tile_h, s->z_near,
                                                           w.chunk_first, nch);
        PS_LAUNCH_CHECK();
        k_sort_warp<<<(frame->n_tiles + kSortWarps - 1) / kSortWarps, kSortWarps * 32, 0, st>>>(
            tile_ptr, frame->n_tiles, w.ent_tmp, w.key_tmp, tile_ent, tile_key);
        PS_LAUNCH_CHECK();
        const int sort_blocks = (frame->n_tiles + 255) / 256;
        k_sort<<<sort_blocks < kSortBlocks ? sort_blocks : kSortBlocks, 256, 0, st>>>(
            tile_ptr, frame->n_tiles, w.ent_tmp, w.key_tmp, tile_ent, tile_key);
        PS_LAUNCH_CHECK();
    }
    return PS_OK;
}
