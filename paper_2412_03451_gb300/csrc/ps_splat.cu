// ps_splat.cu -- forward and backward splatting, render loss.
//
// Forward (Sec. 3.2, Eq. 4, 6-9, 11-13).  Work is split into strips of 32
// pixels (a warp) of a tile; persistent warps take strips from a device
// counter, so heavy and light strips balance across the GPU and no warp ever
// waits for another.  A warp walks its tile's record list (sorted by depth key,
// ps_bin.cu) 32 entries at a time: each lane loads one entry and tests it
// against the warp's pixel rectangle (region_may_hit); a ballot leaves the
// entries that can matter, which are staged in the warp's slice of shared
// memory and evaluated by every lane for its own pixel in list order.
//
// Each pixel keeps the pairs that pass the w >= w_min filter and composites the
// M nearest by (t, record id) front to back in exact order, with a small sorted
// register buffer of pending pairs:
//   * a pending pair is composited once its depth is below the key of the next
//     list entry (keys bound every later depth from below);
//   * the nearest opaque (w = 1) pair, or the M-th pair, is a cut: pairs
//     behind it can never be composited (T = 0 behind an opaque pair) and are
//     dropped at once, and once the list keys pass the cut the pixel is done;
//   * if the buffer overflows, the largest pair is dropped and remembered;
//     compositing stops at the smallest dropped pair and the warp walks the
//     list again from the last composited pair (each pass composites at least
//     one pair, so there are at most M + 1 passes).
//
// Backward.  The same walk (bit-identical arithmetic) rebuilds each pixel's
// composited list and pushes (record, T_j) on a per-pixel stack in shared
// memory; the adjoint of Eq. 11-13 is then taken back to front:
//   A_j = w_j t_j + (1 - w_j) A_{j+1},  dD/dw_j = T_j (t_j - A_{j+1}),
//   dD/dt_j = T_j w_j,  dN/dn_j = T_j w_j,  and the same for N with n_j,
// so nothing is divided by 1 - w_j.  Each pair's gradient is chained through
// Eq. 9, 7-8, 6 and 4 into 16 record floats (the gradients of n_c, v^x_c, v^y_c
// at a fixed plane centre, of s, a_x, a_y and of the radii; the first three use
// the intersection relative to the centre, t d - p_c = P_X v^x + P_Y v^y, so no
// metre-sized terms are summed only to cancel), summed over the lanes of a warp
// that hold the same record and added to a per-record accumulator; a second
// kernel chains the records through the camera transform and Eq. 2-3 into the
// world parameters.
#include <mutex>

#include <cuda.h>

#include "ps_internal.cuh"

using namespace ps;

namespace {

// Pending-pair buffer per pixel: 4 deep for the rectangle weight (its opaque pairs cut
// the lists early; 4 was 1-2.4% faster than 5 and up to 3.7% faster than 3), 6 deep for
// the Eq. 5 weight, where every pair is partly transparent and more of them wait for the
// list keys to pass (6 was 13% faster than 4 there).
#ifndef PS_KPEND
#define PS_KPEND 4
#endif
constexpr int kPendRect = PS_KPEND;
constexpr int kPendGauss = 6;
constexpr unsigned kFull = 0xffffffffu;
// Warps per CTA of the splat kernels (ps_settings.cta_warps: 2, 4 or 8; 0 means 4).
// Each warp stages 32 plane records of its tile list per shared-memory batch, so a
// CTA holds 32 x warps records at a time; with the register budget below, 2 and 4
// warps give the same warps per SM and 8 fewer, larger CTAs.
constexpr int kDefaultWarps = 4;

// Resident CTAs per SM the register allocation is sized for: 24 warps per SM for
// the forward-only kernel (measured 8% faster than 20), 20 for the modes with the
// backward, where 24 would spill.
__host__ __device__ constexpr int min_blocks(int mode, int warps)
{
    return (mode == 0 ? 24 : 20) / warps;
}

// Kernel modes: forward only; backward from given dL/dD, dL/dN; or forward,
// Eq. 14 loss and backward fused in one walk per pixel.
constexpr int kFwd = 0, kBwd = 1, kFused = 2;

// Fused mode: per-view loss sums are added into kSlots partial sums per view
// (spread over L2 slices, so that strips of one view do not serialise on one
// address), which the chain kernel adds up into view_sums.
constexpr int kSlots = 32;

struct SplatArgs {
    const ps_view* views;
    int n_views;
    const float4* rec;        // [R][4]
    const float* key;         // [capacity] entry keys, parallel to tile_ent
    const int* tile_ptr;
    const int* tile_ent;
    long long capacity;
    SplatConst c;
    int M;
    int n_items;              // strips = n_tiles * (tile pixels / 32)
    int* counter;             // work counter (zeroed before the launch)
    const ps_step_state* d_state;   // if set, lambda and delta come from here
    // forward outputs
    float* depth;
    float* normal;
    float* alpha;
    int* ids;                 // optional: plane index of the nearest composited pair
    // backward inputs / outputs
    const float* dLdD;
    const float* dLdN;
    float4* g_rec;            // [R][4]
    int* status;
    // fused mode: supervision and loss outputs
    const float* gt_depth;
    const float* gt_normal;
    float* out_dLdD;          // optional
    float* out_dLdN;          // optional
    double* vs_slots;         // [V][kSlots][4] partial loss sums (zeroed before the launch)
    float a_cos, a_l1n, a_depth;
};

// A warp's staging area: one list chunk.
struct WarpStage {
    float4 rec[4][32];        // record float4 c of chunk entry e at rec[c][e] (no bank conflicts)
    int id[32];
    float key[33];            // entry keys x (1 - 1/4096); key[32]: the next chunk's first entry
};

__device__ __forceinline__ float sgnf(float x) { return (x > 0.f) ? 1.f : ((x < 0.f) ? -1.f : 0.f); }

// A candidate's place in the (t, id) order as one 64-bit key: t is positive
// (t > z_near > 0), so its bits order like its value, and the record id breaks
// ties.  kNoKey (all ones) is above every key.
typedef unsigned long long CKey;
constexpr CKey kNoKey = ~0ull;

__device__ __forceinline__ CKey ckey(float t, int id)
{
    return ((CKey)__float_as_uint(t) << 32) | (unsigned)id;
}
__device__ __forceinline__ float key_t(CKey k) { return __uint_as_float((unsigned)(k >> 32)); }
__device__ __forceinline__ int key_id(CKey k) { return (int)(unsigned)(k & 0xffffffffu); }

// Per-pixel walk state.
template <int KP>
struct Walk {
    float T;
    int cnt;
    bool done;
    int nb;
    CKey bk[KP];      // pending candidates, ascending
    float bw[KP];
    CKey floor_;      // last composited candidate (0: none yet)
    CKey ovf;         // smallest candidate dropped from a full buffer (kNoKey: none)
    CKey cut;         // nearest opaque (w = 1) candidate, or the M-th candidate (kNoKey: none)
};

template <int KP>
__device__ __forceinline__ void drop_note(Walk<KP>& s, CKey k)
{
    if (k < s.ovf) s.ovf = k;
}

template <int KP>
__device__ __forceinline__ void set_cut(Walk<KP>& s, CKey k)
{
    if (k < s.cut) s.cut = k;
    // pairs dropped from a full buffer that lie strictly behind the cut can never count
    if (s.cut < s.ovf) s.ovf = kNoKey;
}

// Adds a candidate.  Candidates behind the cut are dropped: nothing behind an
// opaque pair (T = 0 after it) or behind the M-th pair can be composited.  An
// opaque candidate becomes the cut and truncates the pending pairs behind it;
// when composited + pending exceeds M the largest pending pair is beyond the
// top M and goes, and the new M-th pair becomes the cut.
template <int KP>
__device__ __forceinline__ void pend_insert(Walk<KP>& s, CKey key, float w, int M)
{
    if (s.cut < key) return;     // strictly behind the cut
    if (s.nb == KP) {
        if (!(key < s.bk[KP - 1])) { drop_note(s, key); return; }
        drop_note(s, s.bk[KP - 1]);
        s.nb = KP - 1;
    }
    int pos = 0;
#pragma unroll
    for (int i = KP - 1; i >= 1; --i) {
        if (i <= s.nb) {
            if (key < s.bk[i - 1]) {
                s.bk[i] = s.bk[i - 1]; s.bw[i] = s.bw[i - 1];
            } else if (pos == 0) {
                s.bk[i] = key; s.bw[i] = w; pos = i;
            }
        }
    }
    if (pos == 0) { s.bk[0] = key; s.bw[0] = w; }
    ++s.nb;
    if (w == 1.f) {
        set_cut(s, key);
        s.nb = pos + 1;          // pending pairs behind an opaque one can never count
    }
    if (s.cnt + s.nb > M) {      // the largest pending pair is beyond the top M
        s.nb = M - s.cnt;
        CKey lk = s.bk[0];
#pragma unroll
        for (int i = 1; i < KP; ++i)
            if (i < s.nb) lk = s.bk[i];
        set_cut(s, lk);
    }
}

template <int KP>
__device__ __forceinline__ void pend_pop(Walk<KP>& s)
{
#pragma unroll
    for (int i = 0; i < KP - 1; ++i) {
        s.bk[i] = s.bk[i + 1]; s.bw[i] = s.bw[i + 1];
    }
    --s.nb;
}

// Forward accumulators.
struct Accum {
    float D, N0, N1, N2, A;
    int first;        // record id of the first composited pair, -1 if none
};

struct Sink {
    // forward: composite into Accum; backward: push (record, T) on the stack; fused: both
    Accum acc;
    int2* stk;        // this lane's column of the warp's stack [M][32]
};

template <int MODE, int KP>
__device__ __forceinline__ void composite(Walk<KP>& s, Sink& k, const float4& n, float t, float w, int id,
                                          int M)
{
    if constexpr (MODE != kFwd) k.stk[s.cnt * 32] = make_int2(id, __float_as_int(s.T));
    if constexpr (MODE != kBwd) {
        if (k.acc.first < 0) k.acc.first = id;
        const float tw = s.T * w;
        k.acc.D = fmaf(tw, t, k.acc.D);
        k.acc.N0 = fmaf(tw, n.x, k.acc.N0);
        k.acc.N1 = fmaf(tw, n.y, k.acc.N1);
        k.acc.N2 = fmaf(tw, n.z, k.acc.N2);
        k.acc.A = k.acc.A + tw;
    }
    s.T = s.T * (1.f - w);
    ++s.cnt;
    s.floor_ = ckey(t, id);
    if (s.cnt >= M || s.T == 0.f) s.done = true;
}

template <int MODE, int KP>
__device__ __forceinline__ void flush(Walk<KP>& s, Sink& k, const float4* __restrict__ rec,
                                      float bound, int M)
{
    // every later candidate lies behind the cut: nothing else can enter (no cut: NaN, false)
    const bool final_ = bound > key_t(s.cut);
    if (final_) bound = INFINITY;
    while (s.nb > 0 && !s.done) {
        const CKey k0 = s.bk[0];
        if (!(key_t(k0) < bound)) break;
        if (!(k0 < s.ovf)) break;
        const float w = s.bw[0];
        pend_pop(s);
        float4 n = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (MODE != kBwd) n = __ldg(&rec[(size_t)key_id(k0) * 4]);
        composite<MODE>(s, k, n, key_t(k0), w, key_id(k0), M);
    }
    if (final_ && s.nb == 0 && s.ovf == kNoKey) s.done = true;
}

// Walks one tile list for the warp's 32 pixels.
template <int MODE, int KP>
__device__ __forceinline__ void walk_strip(const SplatArgs& a, WarpStage& ws, Walk<KP>& s,
                                           Sink& k, float dx, float dy, const WarpRegion& g,
                                           int beg, int end)
{
    const int lane = threadIdx.x & 31;
    const float kMargin = 1.f - 1.f / 4096.f;
    for (int pass = 0; pass <= a.M + 1; ++pass) {
        for (int base = beg; base < end; base += 32) {
            if (__all_sync(kFull, s.done)) break;
            // stage: lane l loads entry base + l and tests it against the warp's pixels
            const int i = base + lane;
            bool ok = false;
            if (i < end) {
                const int id = __ldg(&a.tile_ent[i]);
                const float4* r = a.rec + (size_t)id * 4;
                const float4 n = __ldg(r + 0), vx = __ldg(r + 1), vy = __ldg(r + 2), rr = __ldg(r + 3);
                ok = region_may_hit(n, vx, vy, rr, g, a.c);
                ws.key[lane] = __ldg(&a.key[i]) * kMargin;
                if (ok) {
                    ws.id[lane] = id;
                    ws.rec[0][lane] = n; ws.rec[1][lane] = vx; ws.rec[2][lane] = vy; ws.rec[3][lane] = rr;
                }
            } else {
                ws.key[lane] = INFINITY;
            }
            if (lane == 0)
                ws.key[32] = (base + 32 < end) ? __ldg(&a.key[base + 32]) * kMargin : INFINITY;
            unsigned m = __ballot_sync(kFull, ok);
            __syncwarp();
            while (m) {
                // every pixel of the strip is finished: the rest of the chunk cannot matter
                // (forward only: measured slower in the modes with the backward)
                if constexpr (MODE == kFwd) {
                    if (__all_sync(kFull, s.done)) break;
                }
                const int e = __ffs(m) - 1;
                m &= m - 1;
                // keys are sorted and entries that fail the region test cannot reach any
                // pixel of the strip: the next surviving entry's key (or the next chunk's
                // first key) bounds every later depth
                const int en = m ? __ffs(m) - 1 : 32;
                if (!s.done) {
                    PairEval pe;
                    const int id = ws.id[e];
                    const float bound = ws.key[en];
                    const float4 n = ws.rec[0][e];
                    if (eval_pair(n, ws.rec[1][e], ws.rec[2][e], ws.rec[3][e], dx, dy, a.c, pe)) {
                        const CKey key = ckey(pe.t, id);
                        if (s.floor_ < key) {
                            // nothing pending and nothing later can come before it: composite
                            // at once (what inserting and flushing would do)
                            if (s.nb == 0 && pe.t < bound && key < s.ovf && !(s.cut < key))
                                composite<MODE>(s, k, n, pe.t, pe.w, id, a.M);
                            else
                                pend_insert(s, key, pe.w, a.M);
                        }
                    }
                    if (!s.done && (s.nb > 0 || s.cut != kNoKey)) flush<MODE>(s, k, a.rec, bound, a.M);
                }
            }
            // entries without a relevant successor in this chunk: bound by the next chunk
            if (!s.done && (s.nb > 0 || s.cut != kNoKey)) flush<MODE>(s, k, a.rec, ws.key[32], a.M);
            __syncwarp();
        }
        // end of list: everything pending below the smallest dropped pair is final
        flush<MODE>(s, k, a.rec, INFINITY, a.M);
        const bool again = !s.done && s.ovf != kNoKey;
        if (!again) s.done = true;
        if (!__any_sync(kFull, again)) break;
        if (again) { s.ovf = kNoKey; s.nb = 0; }
    }
}

// One strip: pixel setup, walk, then the forward output or the backward adjoint.
// Sums v[8] over the warp's 32 lanes as a transpose-reduction: after 3 exchange
// levels each lane carries one float (index bit2 + 2 bit3 + 4 bit4 of its lane),
// and two more levels leave lanes 4c .. 4c + 3 with the total of float c in v[0].
__device__ __forceinline__ void warp_transpose8(float (&v)[8])
{
    const int lane = threadIdx.x & 31;
    {
        const bool hi = lane & 16;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float send = hi ? v[c] : v[c + 4];
            const float keep = hi ? v[c + 4] : v[c];
            v[c] = keep + __shfl_xor_sync(kFull, send, 16);
        }
    }
    {
        const bool hi = lane & 8;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const float send = hi ? v[c] : v[c + 2];
            const float keep = hi ? v[c + 2] : v[c];
            v[c] = keep + __shfl_xor_sync(kFull, send, 8);
        }
    }
    {
        const bool hi = lane & 4;
        const float send = hi ? v[0] : v[1];
        const float keep = hi ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(kFull, send, 4);
    }
    v[0] += __shfl_xor_sync(kFull, v[0], 2);
    v[0] += __shfl_xor_sync(kFull, v[0], 1);
}

// The lane's Eq. 14 terms of a fused strip: |1 - N.N*|, ||N - N*||_1, |D - D*|,
// 1 (supervised pixels), and the strip's view.
struct StripLoss {
    int v;
    float sc, sl, sd, one;
};

template <int TW, int TH, int MODE, int KP>
__device__ __forceinline__ StripLoss run_strip(const SplatArgs& a, WarpStage& ws, int2* stk_warp,
                                               int item)
{
    constexpr int NS = TW * TH / 32;       // strips per tile
    const int lane = threadIdx.x & 31;
    const int tile = item / NS;
    const int strip = item - tile * NS;
    const int v = view_of_tile(a.views, a.n_views, tile);
    const ps_view* vw = a.views + v;
    const int W = __ldg(&vw->W), H = __ldg(&vw->H);
    const int tx_n = __ldg(&vw->tiles_x);
    const int lt = tile - __ldg(&vw->tile_off);
    const int tx0 = (lt % tx_n) * TW, ty0 = (lt / tx_n) * TH;
    const int q = strip * 32 + lane;        // pixel index within the tile, row-major
    const int px = tx0 + q % TW, py = ty0 + q / TW;
    const bool inside = px < W && py < H;
    const float fx = __ldg(&vw->fx), fy = __ldg(&vw->fy);
    const float cx = __ldg(&vw->cx), cy = __ldg(&vw->cy);
    const float dx = __fdiv_rn((float)px + 0.5f - cx, fx);
    const float dy = __fdiv_rn((float)py + 0.5f - cy, fy);
    const long long pix = __ldg(&vw->pix_off) + (long long)py * W + px;
    const long long gpix = __ldg(&vw->gt_off) + (long long)py * W + px;   // supervision pixel
    WarpRegion g;
    {
        constexpr int WX = TW < 32 ? TW : 32;
        constexpr int WY = TW < 32 ? 32 / TW : 1;
        const int q0 = strip * 32;
        const int gx0 = tx0 + q0 % TW, gy0 = ty0 + q0 / TW;
        g.dxa = __fdiv_rn((float)gx0 + 0.5f - cx, fx);
        g.dxb = __fdiv_rn((float)(gx0 + WX - 1) + 0.5f - cx, fx);
        g.dya = __fdiv_rn((float)gy0 + 0.5f - cy, fy);
        g.dyb = __fdiv_rn((float)(gy0 + WY - 1) + 0.5f - cy, fy);
    }
    const int beg = (int)min((long long)__ldg(&a.tile_ptr[tile]), a.capacity);
    const int end = (int)min((long long)__ldg(&a.tile_ptr[tile + 1]), a.capacity);

    Walk<KP> s;
    s.T = 1.f; s.cnt = 0; s.nb = 0;
    s.floor_ = 0ull; s.ovf = kNoKey; s.cut = kNoKey;
    s.done = !inside;
    Sink k;
    k.acc = Accum{0.f, 0.f, 0.f, 0.f, 0.f, -1};
    k.stk = stk_warp + lane;
    float gD = 0.f, gN0 = 0.f, gN1 = 0.f, gN2 = 0.f;
    // fused: the pixel's supervision is loaded before the walk so its latency is hidden
    float Dg = 0.f, G0 = 0.f, G1 = 0.f, G2 = 0.f;
    if constexpr (MODE == kFused) {
        if (inside) {
            Dg = __ldg(&a.gt_depth[gpix]);
            G0 = __ldg(&a.gt_normal[3 * gpix]);
            G1 = __ldg(&a.gt_normal[3 * gpix + 1]);
            G2 = __ldg(&a.gt_normal[3 * gpix + 2]);
        }
    }
    if constexpr (MODE == kBwd) {
        if (inside) {
            gD = __ldg(&a.dLdD[pix]);
            gN0 = __ldg(&a.dLdN[3 * pix + 0]);
            gN1 = __ldg(&a.dLdN[3 * pix + 1]);
            gN2 = __ldg(&a.dLdN[3 * pix + 2]);
            if (gD == 0.f && gN0 == 0.f && gN1 == 0.f && gN2 == 0.f) s.done = true;
        }
    }
    walk_strip<MODE>(a, ws, s, k, dx, dy, g, beg, end);

    if constexpr (MODE != kBwd) {
        if (inside) {
            if (a.depth) a.depth[pix] = k.acc.D;
            if (a.normal) {
                a.normal[3 * pix + 0] = k.acc.N0;
                a.normal[3 * pix + 1] = k.acc.N1;
                a.normal[3 * pix + 2] = k.acc.N2;
            }
            if (a.alpha) a.alpha[pix] = k.acc.A;
            if (a.ids)
                a.ids[pix] = k.acc.first < 0
                                 ? -1
                                 : k.acc.first - __ldg(&vw->rec_off) + __ldg(&vw->plane_off);
        }
    }
    bool supervised = inside;
    StripLoss out{v, 0.f, 0.f, 0.f, 0.f};
    if constexpr (MODE == kFused) {
        // Eq. 14 at this pixel and its gradient with respect to D and N
        float sc = 0.f, sl = 0.f, sd = 0.f, one = 0.f;
        if (inside) {
            supervised = Dg > 0.f;
            if (supervised) {
                const float N0 = k.acc.N0, N1 = k.acc.N1, N2 = k.acc.N2;
                const float c = 1.f - (N0 * G0 + N1 * G1 + N2 * G2);
                const float e0 = N0 - G0, e1 = N1 - G1, e2 = N2 - G2;
                const float dd = k.acc.D - Dg;
                sc = fabsf(c);
                sl = fabsf(e0) + fabsf(e1) + fabsf(e2);
                sd = fabsf(dd);
                one = 1.f;
                gD = a.a_depth * sgnf(dd);
                const float scc = -a.a_cos * sgnf(c);
                gN0 = scc * G0 + a.a_l1n * sgnf(e0);
                gN1 = scc * G1 + a.a_l1n * sgnf(e1);
                gN2 = scc * G2 + a.a_l1n * sgnf(e2);
            }
            if (a.out_dLdD) a.out_dLdD[pix] = gD;
            if (a.out_dLdN) {
                a.out_dLdN[3 * pix + 0] = gN0;
                a.out_dLdN[3 * pix + 1] = gN1;
                a.out_dLdN[3 * pix + 2] = gN2;
            }
        }
        out.sc = sc; out.sl = sl; out.sd = sd; out.one = one;
    }
    if constexpr (MODE != kFwd) {
        // back to front over the stack
        const int cnt = supervised ? s.cnt : 0;
        int wmax = cnt;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wmax = max(wmax, __shfl_xor_sync(kFull, wmax, o));
        float A = 0.f, B0 = 0.f, B1 = 0.f, B2 = 0.f;
        const float lam5 = a.c.lam5;
        // software pipeline: the record of stack entry j - 1 is loaded while j is processed
        int2 nxt = make_int2(-1, 0);
        float4 qn = make_float4(0.f, 0.f, 0.f, 0.f), qx = qn, qy = qn, qr = qn;
        if (wmax - 1 >= 0 && wmax - 1 < cnt) {
            nxt = k.stk[(wmax - 1) * 32];
            const float4* r = a.rec + (size_t)nxt.x * 4;
            qn = __ldg(r + 0); qx = __ldg(r + 1); qy = __ldg(r + 2); qr = __ldg(r + 3);
        }
        for (int j = wmax - 1; j >= 0; --j) {
            const bool act = j < cnt;
            float gr[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) gr[c] = 0.f;
            int id = -1;
            const int2 e = nxt;
            const float4 n = qn, vx = qx, vy = qy, rr = qr;
            if (j - 1 >= 0 && j - 1 < cnt) {
                nxt = k.stk[(j - 1) * 32];
                const float4* r = a.rec + (size_t)nxt.x * 4;
                qn = __ldg(r + 0); qx = __ldg(r + 1); qy = __ldg(r + 2); qr = __ldg(r + 3);
            }
            if (act) {
                id = e.x;
                const float Tj = __int_as_float(e.y);
                PairEval pe;
                eval_pair(n, vx, vy, rr, dx, dy, a.c, pe);   // same arithmetic as the walk
                const float t = pe.t, w = pe.w;
                const float gw = Tj * (gD * (t - A) + gN0 * (n.x - B0) + gN1 * (n.y - B1) +
                                       gN2 * (n.z - B2));
                const float Tw = Tj * w;
                float gt = Tw * gD;
                // the intersection relative to the plane centre, t d - p_c = P_X v^x + P_Y v^y
                // (Eq. 6 on the plane): radius-sized, so the gradients of n_c and v_c below
                // (at fixed p_c) are accumulated without the cancellation of t d against p_c
                const float ox = fmaf(pe.X, vx.x, pe.Y * vy.x);
                const float oy = fmaf(pe.X, vx.y, pe.Y * vy.y);
                const float oz = fmaf(pe.X, vx.z, pe.Y * vy.z);
                A = fmaf(w, t, (1.f - w) * A);
                B0 = fmaf(w, n.x, (1.f - w) * B0);
                B1 = fmaf(w, n.y, (1.f - w) * B1);
                B2 = fmaf(w, n.z, (1.f - w) * B2);
                if (a.c.gauss) {
                    // Eq. 5: w = exp(-(X^2 / sX^2 + Y^2 / sY^2) / 2):
                    // dw/dX = -w X / sX^2, dw/dsX = w X^2 / sX^3 (likewise Y)
                    const float ix = __fdividef(1.f, pe.sX), iy = __fdividef(1.f, pe.sY);
                    const float gX = -gw * w * pe.X * ix * ix;
                    const float gY = -gw * w * pe.Y * iy * iy;
                    const float grX = -gX * pe.X * ix, grY = -gY * pe.Y * iy;
                    // Eq. 6 on both axes: P = t (d . v_c) - a, dP/dv_c = t d - p_c at fixed p_c
                    gt = fmaf(gX, pe.dvx, gt);
                    gt = fmaf(gY, pe.dvy, gt);
                    // Eq. 4: t = s / (d . n_c); dt/dn_c = (p_c - t d) / (d . n_c) at fixed p_c
                    const float gs = __fdividef(gt, pe.den);
                    gr[0] = fmaf(-gs, ox, Tw * gN0); gr[1] = fmaf(-gs, oy, Tw * gN1);
                    gr[2] = fmaf(-gs, oz, Tw * gN2); gr[3] = gs;
                    gr[4] = gX * ox; gr[5] = gX * oy; gr[6] = gX * oz; gr[7] = -gX;
                    gr[8] = gY * ox; gr[9] = gY * oy; gr[10] = gY * oz; gr[11] = -gY;
                    const bool px = pe.X > 0.f, py = pe.Y > 0.f;
                    gr[12] = px ? grX : 0.f; gr[13] = px ? 0.f : grX;
                    gr[14] = py ? grY : 0.f; gr[15] = py ? 0.f : grY;
                } else {
                // Eq. 7-9: w = 2 sigmoid(5 lambda m) below the clamp, dw/dm = 5 lambda w (1 - w/2)
                const float gm = (pe.m < 0.f) ? gw * lam5 * w * (1.f - 0.5f * w) : 0.f;
                // m = r_side - |P|: the radius gets gm, P gets -gm sgn(P)
                const int ridx = (pe.sideX ? 0 : 2) + (pe.pos ? 0 : 1);
                const float gP = (pe.P > 0.f) ? -gm : ((pe.P < 0.f) ? gm : 0.f);
                // Eq. 6: P = t (d . v_c) - a, dP/dv_c = t d - p_c at fixed p_c
                gt = fmaf(gP, pe.dv, gt);
                // Eq. 4: t = s / (d . n_c); dt/dn_c = (p_c - t d) / (d . n_c) at fixed p_c
                const float gs = __fdividef(gt, pe.den);
                gr[0] = fmaf(-gs, ox, Tw * gN0); gr[1] = fmaf(-gs, oy, Tw * gN1);
                gr[2] = fmaf(-gs, oz, Tw * gN2); gr[3] = gs;
                const int vo = pe.sideX ? 4 : 8;
#pragma unroll
                for (int c = 4; c < 12; c += 4) {
                    if (c == vo) {
                        gr[c + 0] = gP * ox;
                        gr[c + 1] = gP * oy;
                        gr[c + 2] = gP * oz;
                        gr[c + 3] = -gP;
                    }
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) gr[12 + c] = (c == ridx) ? gm : 0.f;
                }
            }
            // warp aggregation: for each distinct record among the active lanes, the
            // 16 gradient floats are summed over its lanes by a transpose-reduction
            // and added with two 8-lane atomic instructions
            const unsigned actm = __ballot_sync(kFull, act);
            if (actm == 0) continue;
            const unsigned peers = __match_any_sync(kFull, id);
            unsigned rem = actm;
            while (rem) {
                const int leader = __ffs(rem) - 1;
                const unsigned gmask = __shfl_sync(kFull, peers, leader);
                const int gid = __shfl_sync(kFull, id, leader);
                rem &= ~gmask;
                const bool member = (gmask >> lane) & 1u;
                float* dst = reinterpret_cast<float*>(a.g_rec + (size_t)gid * 4);
                // two halves of 8 floats: lanes 4c..4c+3 end with the total of float c of the half
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float v[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c) v[c] = member ? gr[8 * h + c] : 0.f;
                    warp_transpose8(v);
                    if ((lane & 3) == 0) atomicAdd(dst + 8 * h + ((lane >> 2) & 7), v[0]);
                }
            }
        }
    }
    return out;
}

// Persistent warps: each takes strips from the work counter until none is left.
// lambda and the quick-reject margin from the device state (graph replay)
__device__ __forceinline__ void load_state(SplatArgs& a)
{
    if (a.d_state && !a.c.hard && !a.c.gauss) {
        a.c.lam5 = 5.f * __ldg(&a.d_state->lambda);
        a.c.reject = (float)(__ldg(&a.d_state->delta) * 1.02 + 1e-6);
    }
}

// G: the weight form of the instantiation (0: Eq. 7-9 rectangle weight, 1: Eq. 5 Gaussian),
// fixed at compile time so that the other form's branches fold away.
template <int TW, int TH, int MODE, int NW, int G>
__global__ void __launch_bounds__(NW * 32, min_blocks(MODE, NW)) k_splat(SplatArgs a_in)
{
    constexpr int KP = G ? kPendGauss : kPendRect;
    SplatArgs a = a_in;
    a.c.gauss = G;
    load_state(a);
    __shared__ WarpStage stage[NW];
    extern __shared__ int2 dyn_stk[];       // backward: [NW][M][32]
    const int w = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    int2* stk_warp = dyn_stk + (size_t)w * a.M * 32;
    // fused: the lane's loss terms over the warp's consecutive strips of one view (items
    // are handed out in increasing order, so a warp meets each view in one run)
    int vcur = -1;
    float l0 = 0.f, l1 = 0.f, l2 = 0.f, l3 = 0.f;
    const int slot = (blockIdx.x * NW + w) % kSlots;
    auto flush_loss = [&]() {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            l0 += __shfl_xor_sync(kFull, l0, o);
            l1 += __shfl_xor_sync(kFull, l1, o);
            l2 += __shfl_xor_sync(kFull, l2, o);
            l3 += __shfl_xor_sync(kFull, l3, o);
        }
        if (lane == 0 && l3 > 0.f) {
            double* d = a.vs_slots + ((size_t)vcur * kSlots + slot) * 4;
            atomicAdd(d + 0, (double)l0);
            atomicAdd(d + 1, (double)l1);
            atomicAdd(d + 2, (double)l2);
            atomicAdd(d + 3, (double)l3);
        }
        l0 = l1 = l2 = l3 = 0.f;
    };
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(a.counter, 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= a.n_items) break;
        const StripLoss sl = run_strip<TW, TH, MODE, KP>(a, stage[w], stk_warp, item);
        if constexpr (MODE == kFused) {
            if (sl.v != vcur) {
                if (vcur >= 0) flush_loss();
                vcur = sl.v;
            }
            l0 += sl.sc; l1 += sl.sl; l2 += sl.sd; l3 += sl.one;
        }
        __syncwarp();
    }
    if constexpr (MODE == kFused) {
        if (vcur >= 0) flush_loss();
    }
}

// Work counts (diagnostic): full walk of every tile list, no early exit.
template <int NT>
struct CountSmem {
    static constexpr int kBatch = NT < 128 ? NT : 128;
    float4 rec[kBatch][4];
    int id[kBatch];
    int view, beg, end;
};

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH) k_count_pairs(SplatArgs a_in, unsigned long long* counts)
{
    SplatArgs a = a_in;
    load_state(a);
    constexpr int NT = TW * TH;
    __shared__ CountSmem<NT> sm;
    __shared__ unsigned long long red[3];
    constexpr int B = CountSmem<NT>::kBatch;

    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    if (tid == 0) {
        sm.view = view_of_tile(a.views, a.n_views, tile);
        const long long b = __ldg(&a.tile_ptr[tile]), e = __ldg(&a.tile_ptr[tile + 1]);
        sm.beg = (int)min(b, a.capacity);
        sm.end = (int)min(e, a.capacity);
        red[0] = red[1] = red[2] = 0ull;
    }
    __syncthreads();
    const ps_view* vw = a.views + sm.view;
    const int W = __ldg(&vw->W), H = __ldg(&vw->H);
    const int tx_n = __ldg(&vw->tiles_x);
    const int lt = tile - __ldg(&vw->tile_off);
    const int px = (lt % tx_n) * TW + tid % TW;
    const int py = (lt / tx_n) * TH + tid / TW;
    const bool inside = px < W && py < H;
    const float dx = __fdiv_rn((float)px + 0.5f - __ldg(&vw->cx), __ldg(&vw->fx));
    const float dy = __fdiv_rn((float)py + 0.5f - __ldg(&vw->cy), __ldg(&vw->fy));
    unsigned long long n_cand = 0, n_front = 0;
    bool have_op = false;
    float op_t = 0.f;
    int op_id = 0;
    for (int pass = 0; pass < 2; ++pass) {
        for (int base = sm.beg; base < sm.end; base += B) {
            __syncthreads();
            if (tid < B && base + tid < sm.end) {
                const int id = __ldg(&a.tile_ent[base + tid]);
                sm.id[tid] = id;
                const float4* r = a.rec + (size_t)id * 4;
                sm.rec[tid][0] = __ldg(r + 0); sm.rec[tid][1] = __ldg(r + 1);
                sm.rec[tid][2] = __ldg(r + 2); sm.rec[tid][3] = __ldg(r + 3);
            }
            __syncthreads();
            const int nbat = min(B, sm.end - base);
            if (inside) {
                for (int e = 0; e < nbat; ++e) {
                    PairEval pe;
                    const int id = sm.id[e];
                    if (!eval_pair(sm.rec[e][0], sm.rec[e][1], sm.rec[e][2], sm.rec[e][3], dx, dy,
                                   a.c, pe))
                        continue;
                    if (pass == 0) {
                        ++n_cand;
                        if (pe.w == 1.f && (!have_op || cand_less(pe.t, id, op_t, op_id))) {
                            have_op = true; op_t = pe.t; op_id = id;
                        }
                    } else if (!have_op || !cand_less(op_t, op_id, pe.t, id)) {
                        ++n_front;
                    }
                }
            }
        }
    }
    const unsigned long long tested = inside ? (unsigned long long)(sm.end - sm.beg) : 0ull;
    const unsigned long long comp = n_front < (unsigned long long)a.M ? n_front : (unsigned long long)a.M;
    atomicAdd(&red[0], tested);
    atomicAdd(&red[1], n_cand);
    atomicAdd(&red[2], comp);
    __syncthreads();
    if (tid < 3) atomicAdd(&counts[tid], red[tid]);
}

// Per-record gradient -> world parameters (camera transform, Eq. 2-3 and the
// quaternion normalisation).
struct ChainArgs {
    const ps_view* views;
    const float* center;
    const float* quat;
    const float* radii;
    const float4* g_rec;
    float* g_center;
    float* g_quat;
    float* g_radii;
    int single_radii;
    const double* vs_slots;   // fused: [V][kSlots][4] partial loss sums, or NULL
    double* view_sums;        // fused: [V][4] written from vs_slots
};

__global__ void __launch_bounds__(128) k_chain(ChainArgs a)
{
    const int v = blockIdx.y;
    if (a.vs_slots && blockIdx.x == 0 && threadIdx.x < 4) {
        // the fused kernel's loss sums of view v, added up in a fixed order
        const double* sp = a.vs_slots + (size_t)v * kSlots * 4 + threadIdx.x;
        double t = 0.0;
        for (int i = 0; i < kSlots; ++i) t += sp[4 * i];
        a.view_sums[4 * v + threadIdx.x] = t;
    }
    if (!a.g_rec) return;
    const ps_view* vw = a.views + v;
    const int K = __ldg(&vw->K);
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const size_t r = (size_t)__ldg(&vw->rec_off) + k;
    const float4 g0 = a.g_rec[4 * r + 0], g1 = a.g_rec[4 * r + 1];
    const float4 g2 = a.g_rec[4 * r + 2], g3 = a.g_rec[4 * r + 3];
    if (g0.x == 0.f && g0.y == 0.f && g0.z == 0.f && g0.w == 0.f && g1.x == 0.f && g1.y == 0.f &&
        g1.z == 0.f && g1.w == 0.f && g2.x == 0.f && g2.y == 0.f && g2.z == 0.f && g2.w == 0.f &&
        g3.x == 0.f && g3.y == 0.f && g3.z == 0.f && g3.w == 0.f)
        return;
    const int p = __ldg(&vw->plane_off) + k;
    float R[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) R[i] = __ldg(&vw->w2c[i]);
    const float q0 = __ldg(&a.quat[4 * p + 0]), q1 = __ldg(&a.quat[4 * p + 1]);
    const float q2 = __ldg(&a.quat[4 * p + 2]), q3 = __ldg(&a.quat[4 * p + 3]);
    const float qs = sqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    if (!(qs > 0.f) || !isfinite(qs)) return;
    const float w = q0 / qs, x = q1 / qs, y = q2 / qs, z = q3 / qs;
    // world axes: columns of the Hamilton matrix (Eq. 2-3)
    const float vx[3] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y + w * z), 2.f * (x * z - w * y)};
    const float vy[3] = {2.f * (x * y - w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z + w * x)};
    const float nn[3] = {2.f * (x * z + w * y), 2.f * (y * z - w * x), 1.f - 2.f * (x * x + y * y)};
    float vxc[3], vyc[3], nc[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        vxc[i] = R[4 * i] * vx[0] + R[4 * i + 1] * vx[1] + R[4 * i + 2] * vx[2];
        vyc[i] = R[4 * i] * vy[0] + R[4 * i + 1] * vy[1] + R[4 * i + 2] * vy[2];
        nc[i] = R[4 * i] * nn[0] + R[4 * i + 1] * nn[1] + R[4 * i + 2] * nn[2];
    }
    // record = {n_c, s = n_c.p_c, v^x_c, a_x = v^x_c.p_c, v^y_c, a_y = v^y_c.p_c, r}; the splat
    // kernels accumulate the gradients of n_c, v^x_c, v^y_c at fixed p_c and those of s, a_x,
    // a_y, so the camera-frame gradient of p_c is gs n_c + gax v^x_c + gay v^y_c
    const float gs = g0.w, gax = g1.w, gay = g2.w;
    const float gnc[3] = {g0.x, g0.y, g0.z};
    const float gvxc[3] = {g1.x, g1.y, g1.z};
    const float gvyc[3] = {g2.x, g2.y, g2.z};
    float gpc[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) gpc[i] = gs * nc[i] + gax * vxc[i] + gay * vyc[i];
    // camera -> world: multiply by R^T
    float gp[3], gvx[3], gvy[3], gn[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        gp[i] = R[i] * gpc[0] + R[4 + i] * gpc[1] + R[8 + i] * gpc[2];
        gvx[i] = R[i] * gvxc[0] + R[4 + i] * gvxc[1] + R[8 + i] * gvxc[2];
        gvy[i] = R[i] * gvyc[0] + R[4 + i] * gvyc[1] + R[8 + i] * gvyc[2];
        gn[i] = R[i] * gnc[0] + R[4 + i] * gnc[1] + R[8 + i] * gnc[2];
    }
    // G[i][c] = dL/dR_ic with columns (v^x, v^y, n)
    const float G00 = gvx[0], G10 = gvx[1], G20 = gvx[2];
    const float G01 = gvy[0], G11 = gvy[1], G21 = gvy[2];
    const float G02 = gn[0], G12 = gn[1], G22 = gn[2];
    const float gw = 2.f * (-z * G01 + y * G02 + z * G10 - x * G12 - y * G20 + x * G21);
    const float gx = 2.f * (y * G01 + z * G02 + y * G10 - 2.f * x * G11 - w * G12 + z * G20 +
                            w * G21 - 2.f * x * G22);
    const float gy = 2.f * (-2.f * y * G00 + x * G01 + w * G02 + x * G10 + z * G12 - w * G20 +
                            z * G21 - 2.f * y * G22);
    const float gz = 2.f * (-2.f * z * G00 - w * G01 + x * G02 + w * G10 - 2.f * z * G11 +
                            y * G12 + x * G20 + y * G21);
    const float proj = gw * w + gx * x + gy * y + gz * z;
    atomicAdd(&a.g_center[3 * p + 0], gp[0]);
    atomicAdd(&a.g_center[3 * p + 1], gp[1]);
    atomicAdd(&a.g_center[3 * p + 2], gp[2]);
    atomicAdd(&a.g_quat[4 * p + 0], (gw - w * proj) / qs);
    atomicAdd(&a.g_quat[4 * p + 1], (gx - x * proj) / qs);
    atomicAdd(&a.g_quat[4 * p + 2], (gy - y * proj) / qs);
    atomicAdd(&a.g_quat[4 * p + 3], (gz - z * proj) / qs);
    float gr0 = g3.x, gr1 = g3.y, gr2 = g3.z, gr3 = g3.w;
    if (a.single_radii) { gr0 += gr1; gr1 = 0.f; gr2 += gr3; gr3 = 0.f; }
    atomicAdd(&a.g_radii[4 * p + 0], gr0);
    atomicAdd(&a.g_radii[4 * p + 1], gr1);
    atomicAdd(&a.g_radii[4 * p + 2], gr2);
    atomicAdd(&a.g_radii[4 * p + 3], gr3);
}

// Render loss, Eq. 14.
struct LossArgs {
    const ps_view* views;
    const float* depth;
    const float* normal;
    const float* gt_depth;
    const float* gt_normal;
    float* dLdD;
    float* dLdN;
    double* view_sums;
    float a_cos, a_l1n, a_depth;
};

__global__ void __launch_bounds__(256) k_loss(LossArgs a)
{
    const int v = blockIdx.y;
    const ps_view* vw = a.views + v;
    const long long HW = (long long)__ldg(&vw->H) * __ldg(&vw->W);
    const long long off = __ldg(&vw->pix_off);
    const long long goff = __ldg(&vw->gt_off);
    float sc = 0.f, sl = 0.f, sd = 0.f, cnt = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < HW;
         i += (long long)gridDim.x * blockDim.x) {
        const long long p = off + i;
        const long long q = goff + i;
        const float Dg = __ldg(&a.gt_depth[q]);
        if (!(Dg > 0.f)) {
            a.dLdD[p] = 0.f;
            a.dLdN[3 * p + 0] = 0.f; a.dLdN[3 * p + 1] = 0.f; a.dLdN[3 * p + 2] = 0.f;
            continue;
        }
        const float D = __ldg(&a.depth[p]);
        const float N0 = __ldg(&a.normal[3 * p]), N1 = __ldg(&a.normal[3 * p + 1]),
                    N2 = __ldg(&a.normal[3 * p + 2]);
        const float G0 = __ldg(&a.gt_normal[3 * q]), G1 = __ldg(&a.gt_normal[3 * q + 1]),
                    G2 = __ldg(&a.gt_normal[3 * q + 2]);
        const float c = 1.f - (N0 * G0 + N1 * G1 + N2 * G2);
        const float e0 = N0 - G0, e1 = N1 - G1, e2 = N2 - G2;
        const float dd = D - Dg;
        sc += fabsf(c);
        sl += fabsf(e0) + fabsf(e1) + fabsf(e2);
        sd += fabsf(dd);
        cnt += 1.f;
        a.dLdD[p] = a.a_depth * sgnf(dd);
        const float sc_ = -a.a_cos * sgnf(c);
        a.dLdN[3 * p + 0] = sc_ * G0 + a.a_l1n * sgnf(e0);
        a.dLdN[3 * p + 1] = sc_ * G1 + a.a_l1n * sgnf(e1);
        a.dLdN[3 * p + 2] = sc_ * G2 + a.a_l1n * sgnf(e2);
    }
    // block reduction in double
    __shared__ double red[4][8];
    double x[4] = {sc, sl, sd, cnt};
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x[q] += __shfl_xor_sync(kFull, x[q], o);
        if (lane == 0) red[q][wid] = x[q];
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[threadIdx.x][i];
        atomicAdd(&a.view_sums[4 * v + threadIdx.x], s);
    }
}

// ---------------------------------------------------------------------------
// Host side.

struct LaunchCache {
    int dev = -1;
    int blocks_per_sm = 0;
    size_t dyn = 0;
};

template <int TW, int TH, int MODE, int NW, int G>
cudaError_t launch_splat(SplatArgs a, int n_tiles, int M, cudaStream_t st, bool counter_zeroed)
{
    constexpr int NS = TW * TH / 32;
    a.n_items = n_tiles * NS;
    const size_t dyn = MODE != kFwd ? sizeof(int2) * (size_t)NW * M * 32 : 0;
    static LaunchCache cache[8];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    LaunchCache& c = cache[dev & 7];
    if (c.dev != dev || c.dyn != dyn) {
        if (dyn > 0) {
            // static + dynamic shared memory above 48 KB needs the opt-in
            e = cudaFuncSetAttribute(k_splat<TW, TH, MODE, NW, G>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
            if (e != cudaSuccess) return e;
        }
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_splat<TW, TH, MODE, NW, G>, NW * 32, dyn);
        if (e != cudaSuccess) return e;
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        c.dev = dev;
        c.dyn = dyn;
        c.blocks_per_sm = (nb > 0 ? nb : 1) * sms;
    }
    int blocks = c.blocks_per_sm;
    const int need = (a.n_items + NW - 1) / NW;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    if (!counter_zeroed) {
        e = cudaMemsetAsync(a.counter, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
    }
    k_splat<TW, TH, MODE, NW, G><<<blocks, NW * 32, dyn, st>>>(a);
    return cudaGetLastError();
}

ps_status check_common(const ps_frame* f, const ps_settings* s, const float* rec, const float* key,
                       const int* tile_ptr, const int* tile_ent, long long capacity)
{
    if (!f || !s || !rec || !key || !tile_ptr || !f->views) return PS_ERR_ARG;
    if (capacity < 0 || (capacity > 0 && !tile_ent)) return PS_ERR_ARG;
    if (f->n_tiles <= 0 || f->n_views <= 0) return PS_ERR_ARG;
    if (s->M < 1 || s->M > PS_MAX_M) return PS_ERR_ARG;
    if (!s->d_state && !(s->lambda > 0.f)) return PS_ERR_ARG;
    if (!(s->w_min > 0.f) || !(s->w_min < 1.f)) return PS_ERR_ARG;
    if (!(s->z_near > 0.f) || !(s->z_far > s->z_near)) return PS_ERR_ARG;
    if (!s->d_state && !(s->delta >= 0.0)) return PS_ERR_ARG;
    if ((s->flags & PS_GAUSSIAN) && (!(s->delta > 0.0) || (s->flags & PS_HARD))) return PS_ERR_ARG;
    const int tw = s->tile_w, th = s->tile_h;
    if (!((tw == 16 && th == 16) || (tw == 8 && th == 8) || (tw == 32 && th == 8))) return PS_ERR_ARG;
    const int nw = s->cta_warps;
    if (!(nw == 0 || nw == 2 || nw == 4 || nw == 8)) return PS_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(rec) & 15) return PS_ERR_ARG;
    return PS_OK;
}

SplatConst make_const(const ps_settings* s)
{
    SplatConst c;
    c.lam5 = 5.f * s->lambda;
    c.w_min = s->w_min;
    c.z_near = s->z_near;
    c.z_far = s->z_far;
    c.hard = (s->flags & PS_HARD) ? 1 : 0;
    c.gauss = (s->flags & PS_GAUSSIAN) ? 1 : 0;
    c.kappa = c.gauss ? (float)s->delta : 0.f;
    c.reject = (c.hard || c.gauss) ? 0.f : (float)(s->delta * 1.02 + 1e-6);
    return c;
}

template <int MODE, int NW, int G>
cudaError_t dispatch_tile(const SplatArgs& a, const ps_settings* s, int n_tiles, cudaStream_t st,
                          bool counter_zeroed)
{
    if (s->tile_w == 16) return launch_splat<16, 16, MODE, NW, G>(a, n_tiles, s->M, st, counter_zeroed);
    if (s->tile_w == 8) return launch_splat<8, 8, MODE, NW, G>(a, n_tiles, s->M, st, counter_zeroed);
    return launch_splat<32, 8, MODE, NW, G>(a, n_tiles, s->M, st, counter_zeroed);
}

template <int MODE, int G>
cudaError_t dispatch_warps(const SplatArgs& a, const ps_settings* s, int n_tiles, cudaStream_t st,
                           bool counter_zeroed)
{
    const int nw = s->cta_warps ? s->cta_warps : kDefaultWarps;
    if (nw == 2) return dispatch_tile<MODE, 2, G>(a, s, n_tiles, st, counter_zeroed);
    if (nw == 8) return dispatch_tile<MODE, 8, G>(a, s, n_tiles, st, counter_zeroed);
    return dispatch_tile<MODE, 4, G>(a, s, n_tiles, st, counter_zeroed);
}

template <int MODE>
cudaError_t dispatch(const SplatArgs& a, const ps_settings* s, int n_tiles, cudaStream_t st,
                     bool counter_zeroed = false)
{
    if (s->flags & PS_GAUSSIAN) return dispatch_warps<MODE, 1>(a, s, n_tiles, st, counter_zeroed);
    return dispatch_warps<MODE, 0>(a, s, n_tiles, st, counter_zeroed);
}

template <int TW, int TH>
cudaError_t launch_count(const SplatArgs& a, int n_tiles, unsigned long long* counts, cudaStream_t st)
{
    k_count_pairs<TW, TH><<<n_tiles, TW * TH, 0, st>>>(a, counts);
    return cudaGetLastError();
}

constexpr size_t kCounterBytes = 256;

// ps_splat_bwd: the record gradients, then the work counter
inline size_t bwd_ws(const ps_frame* f)
{
    return sizeof(float4) * 4 * (size_t)f->n_records + kCounterBytes;
}

// ps_splat_fused: as ps_splat_bwd, then the per-view partial loss sums
inline size_t fused_ws(const ps_frame* f)
{
    return bwd_ws(f) + sizeof(double) * 4 * kSlots * (size_t)f->n_views;
}

}  // namespace

extern "C" size_t ps_fwd_workspace_bytes(const ps_frame* f)
{
    (void)f;
    return kCounterBytes;
}

extern "C" ps_status ps_splat_fwd(const ps_frame* f, const ps_settings* s, const float* rec,
                                  const float* key, const int* tile_ptr, const int* tile_ent,
                                  long long capacity, float* depth, float* normal, float* alpha,
                                  void* ws, size_t ws_bytes, int* d_status, ps_stream stream)
{
    ps_status e = check_common(f, s, rec, key, tile_ptr, tile_ent, capacity);
    if (e != PS_OK) return e;
    if (!depth || !normal || !ws) return PS_ERR_ARG;
    if (ws_bytes < kCounterBytes || (reinterpret_cast<uintptr_t>(ws) & 15)) return PS_ERR_ARG;
    SplatArgs a{};
    a.views = f->views; a.n_views = f->n_views;
    a.rec = reinterpret_cast<const float4*>(rec); a.key = key;
    a.tile_ptr = tile_ptr; a.tile_ent = tile_ent; a.capacity = capacity;
    a.c = make_const(s); a.M = s->M; a.d_state = s->d_state;
    a.counter = static_cast<int*>(ws);
    a.depth = depth; a.normal = normal; a.alpha = alpha; a.status = d_status;
    if (dispatch<kFwd>(a, s, f->n_tiles, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
        return PS_ERR_CUDA;
    return PS_OK;
}

extern "C" ps_status ps_splat_ids(const ps_frame* f, const ps_settings* s, const float* rec,
                                  const float* key, const int* tile_ptr, const int* tile_ent,
                                  long long capacity, int* ids, float* depth, void* ws,
                                  size_t ws_bytes, int* d_status, ps_stream stream)
{
    ps_status e = check_common(f, s, rec, key, tile_ptr, tile_ent, capacity);
    if (e != PS_OK) return e;
    if (!ids || !ws) return PS_ERR_ARG;
    if (ws_bytes < kCounterBytes || (reinterpret_cast<uintptr_t>(ws) & 15)) return PS_ERR_ARG;
    SplatArgs a{};
    a.views = f->views; a.n_views = f->n_views;
    a.rec = reinterpret_cast<const float4*>(rec); a.key = key;
    a.tile_ptr = tile_ptr; a.tile_ent = tile_ent; a.capacity = capacity;
    a.c = make_const(s); a.M = s->M; a.d_state = s->d_state;
    a.counter = static_cast<int*>(ws);
    a.depth = depth; a.normal = nullptr; a.alpha = nullptr; a.ids = ids; a.status = d_status;
    if (dispatch<kFwd>(a, s, f->n_tiles, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
        return PS_ERR_CUDA;
    return PS_OK;
}

extern "C" size_t ps_bwd_workspace_bytes(const ps_frame* f)
{
    if (!f || f->n_records < 0 || f->n_views < 0) return 0;
    return fused_ws(f);
}

extern "C" ps_status ps_splat_bwd(const ps_planes* planes, const ps_frame* f, const ps_settings* s,
                                  const float* rec, const float* key, const int* tile_ptr,
                                  const int* tile_ent, long long capacity, const float* dLdD,
                                  const float* dLdN, float* g_center, float* g_quat, float* g_radii,
                                  void* ws, size_t ws_bytes, int* d_status, ps_stream stream)
{
    ps_status e = check_common(f, s, rec, key, tile_ptr, tile_ent, capacity);
    if (e != PS_OK) return e;
    if (!planes || !planes->center || !planes->quat || !planes->radii) return PS_ERR_ARG;
    if (!dLdD || !dLdN || !g_center || !g_quat || !g_radii || !ws) return PS_ERR_ARG;
    if (s->flags & PS_HARD) return PS_ERR_ARG;
    if (ws_bytes < bwd_ws(f) || (reinterpret_cast<uintptr_t>(ws) & 15)) return PS_ERR_ARG;
    if (f->n_records == 0) return PS_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t grec_bytes = sizeof(float4) * 4 * (size_t)f->n_records;
    // the record gradients and the work counter after them: one memset
    PS_CUDA_CHECK(cudaMemsetAsync(ws, 0, grec_bytes + sizeof(int), st));
    SplatArgs a{};
    a.views = f->views; a.n_views = f->n_views;
    a.rec = reinterpret_cast<const float4*>(rec); a.key = key;
    a.tile_ptr = tile_ptr; a.tile_ent = tile_ent; a.capacity = capacity;
    a.c = make_const(s); a.M = s->M; a.d_state = s->d_state;
    a.dLdD = dLdD; a.dLdN = dLdN; a.g_rec = reinterpret_cast<float4*>(ws); a.status = d_status;
    a.counter = reinterpret_cast<int*>(static_cast<char*>(ws) + grec_bytes);
    if (dispatch<kBwd>(a, s, f->n_tiles, st, true) != cudaSuccess) return PS_ERR_CUDA;
    ChainArgs c;
    c.views = f->views; c.center = planes->center; c.quat = planes->quat; c.radii = planes->radii;
    c.g_rec = a.g_rec; c.g_center = g_center; c.g_quat = g_quat; c.g_radii = g_radii;
    c.single_radii = (s->flags & PS_SINGLE_RADII) ? 1 : 0;
    c.vs_slots = nullptr; c.view_sums = nullptr;
    dim3 grid((f->max_K + 127) / 128, f->n_views);
    k_chain<<<grid, 128, 0, st>>>(c);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

extern "C" ps_status ps_splat_fused(const ps_planes* planes, const ps_frame* f,
                                    const ps_settings* s, const float* rec, const float* key,
                                    const int* tile_ptr, const int* tile_ent, long long capacity,
                                    const float* gt_depth, const float* gt_normal, float* depth,
                                    float* normal, float* dL_dD, float* dL_dN, double* view_sums,
                                    float* g_center, float* g_quat, float* g_radii, void* ws,
                                    size_t ws_bytes, int* d_status, ps_stream stream)
{
    ps_status e = check_common(f, s, rec, key, tile_ptr, tile_ent, capacity);
    if (e != PS_OK) return e;
    if (!planes || !planes->center || !planes->quat || !planes->radii) return PS_ERR_ARG;
    if (!gt_depth || !gt_normal || !view_sums || !g_center || !g_quat || !g_radii || !ws)
        return PS_ERR_ARG;
    if (s->flags & PS_HARD) return PS_ERR_ARG;
    if (ws_bytes < fused_ws(f) || (reinterpret_cast<uintptr_t>(ws) & 15)) return PS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t grec_bytes = sizeof(float4) * 4 * (size_t)f->n_records;
    // record gradients, work counter and partial loss sums: one memset
    PS_CUDA_CHECK(cudaMemsetAsync(ws, 0, fused_ws(f), st));
    double* slots = reinterpret_cast<double*>(static_cast<char*>(ws) + bwd_ws(f));
    SplatArgs a{};
    a.views = f->views; a.n_views = f->n_views;
    a.rec = reinterpret_cast<const float4*>(rec); a.key = key;
    a.tile_ptr = tile_ptr; a.tile_ent = tile_ent; a.capacity = capacity;
    a.c = make_const(s); a.M = s->M; a.d_state = s->d_state;
    a.depth = depth; a.normal = normal; a.alpha = nullptr;
    a.g_rec = reinterpret_cast<float4*>(ws); a.status = d_status;
    a.counter = reinterpret_cast<int*>(static_cast<char*>(ws) + grec_bytes);
    a.gt_depth = gt_depth; a.gt_normal = gt_normal;
    a.out_dLdD = dL_dD; a.out_dLdN = dL_dN; a.vs_slots = slots;
    a.a_cos = s->a_cos; a.a_l1n = s->a_l1n; a.a_depth = s->a_depth;
    if (dispatch<kFused>(a, s, f->n_tiles, st, true) != cudaSuccess) return PS_ERR_CUDA;
    ChainArgs c;
    c.views = f->views; c.center = planes->center; c.quat = planes->quat; c.radii = planes->radii;
    c.g_rec = f->n_records > 0 ? a.g_rec : nullptr;
    c.g_center = g_center; c.g_quat = g_quat; c.g_radii = g_radii;
    c.single_radii = (s->flags & PS_SINGLE_RADII) ? 1 : 0;
    c.vs_slots = slots; c.view_sums = view_sums;
    dim3 grid(f->max_K > 0 ? (f->max_K + 127) / 128 : 1, f->n_views);
    k_chain<<<grid, 128, 0, st>>>(c);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

extern "C" ps_status ps_loss(const ps_frame* f, const ps_settings* s, const float* depth,
                             const float* normal, const float* gt_depth, const float* gt_normal,
                             float* dLdD, float* dLdN, double* view_sums, ps_stream stream)
{
    if (!f || !s || !f->views || !depth || !normal || !gt_depth || !gt_normal || !dLdD || !dLdN ||
        !view_sums)
        return PS_ERR_ARG;
    if (f->n_views <= 0) return PS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    PS_CUDA_CHECK(cudaMemsetAsync(view_sums, 0, sizeof(double) * 4 * (size_t)f->n_views, st));
    LossArgs a;
    a.views = f->views; a.depth = depth; a.normal = normal; a.gt_depth = gt_depth;
    a.gt_normal = gt_normal; a.dLdD = dLdD; a.dLdN = dLdN; a.view_sums = view_sums;
    a.a_cos = s->a_cos; a.a_l1n = s->a_l1n; a.a_depth = s->a_depth;
    const long long per_view = (f->n_pixels + f->n_views - 1) / f->n_views;
    int bx = (int)((per_view + 256 * 8 - 1) / (256 * 8));
    if (bx < 1) bx = 1;
    if (bx > 1024) bx = 1024;
    k_loss<<<dim3(bx, f->n_views), 256, 0, st>>>(a);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

extern "C" ps_status ps_count_pairs(const ps_frame* f, const ps_settings* s, const float* rec,
                                    const float* key, const int* tile_ptr, const int* tile_ent,
                                    long long capacity, long long* d_counts, ps_stream stream)
{
    ps_status e = check_common(f, s, rec, key, tile_ptr, tile_ent, capacity);
    if (e != PS_OK) return e;
    if (!d_counts) return PS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    PS_CUDA_CHECK(cudaMemsetAsync(d_counts, 0, 3 * sizeof(long long), st));
    SplatArgs a{};
    a.views = f->views; a.n_views = f->n_views;
    a.rec = reinterpret_cast<const float4*>(rec); a.key = key;
    a.tile_ptr = tile_ptr; a.tile_ent = tile_ent; a.capacity = capacity;
    a.c = make_const(s); a.M = s->M; a.d_state = s->d_state;
    unsigned long long* c = reinterpret_cast<unsigned long long*>(d_counts);
    cudaError_t err;
    if (s->tile_w == 16) err = launch_count<16, 16>(a, f->n_tiles, c, st);
    else if (s->tile_w == 8) err = launch_count<8, 8>(a, f->n_tiles, c, st);
    else err = launch_count<32, 8>(a, f->n_tiles, c, st);
    return err == cudaSuccess ? PS_OK : PS_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Backward splatting for callers that cannot allocate device memory.
//
// Some callers have no way to hand the library a scratch buffer: an engine
// whose device memory is owned by a fixed arena that other code may not grow,
// a real-time loop that must never enter the CUDA allocator (cudaMalloc can
// synchronise the device and take unbounded time), or a host program that
// loads this library as a plug-in without a device allocator of its own.  For
// them ps_splat_bwd_noalloc uses a scratch array that is part of the library
// image itself: a file-scope __device__ array that every device holds from the
// moment the library's module is loaded on it until the process exits.
namespace {

constexpr long long kNoAllocMaxRecords = 65536;   // 64 bytes of gradient per record: 4 MiB
constexpr size_t kNoAllocBytes = sizeof(float4) * 4 * (size_t)kNoAllocMaxRecords + kCounterBytes;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch per device.  In host code the symbol's
// name is only a host-side stand-in, so the address is looked up with the
// device current and cached together with the CUDA context it belongs to: after
// cudaDeviceReset, or when the caller makes another context current, the
// library's module is loaded again and the address is looked up again.
std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {};
CUcontext g_noalloc_ctx[64] = {};

typedef CUresult (*CtxGetCurrent)(CUcontext*);

CtxGetCurrent ctx_get_current()
{
    static CtxGetCurrent fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrent>(p);
    }
    return fn;
}

}  // namespace

extern "C" ps_status ps_splat_bwd_noalloc(const ps_planes* planes, const ps_frame* f,
                                          const ps_settings* s, const float* rec,
                                          const float* key, const int* tile_ptr,
                                          const int* tile_ent, long long capacity,
                                          const float* dLdD, const float* dLdN, float* g_center,
                                          float* g_quat, float* g_radii, int* d_status,
                                          ps_stream stream)
{
    if (!f || f->n_records < 0) return PS_ERR_ARG;
    if ((long long)f->n_records > kNoAllocMaxRecords) return PS_ERR_ARG;   // too large for the static scratch
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return PS_ERR_CUDA;
    if (dev < 0 || dev >= 64) return PS_ERR_ARG;
    CtxGetCurrent get_ctx = ctx_get_current();
    CUcontext ctx = nullptr;
    if (!get_ctx || get_ctx(&ctx) != CUDA_SUCCESS) return PS_ERR_CUDA;
    void* ws = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!ctx || !g_noalloc_addr[dev] || g_noalloc_ctx[dev] != ctx) {
            // (this also makes the device's primary context current if none was)
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PS_ERR_CUDA;
            if (!ctx && (get_ctx(&ctx) != CUDA_SUCCESS || !ctx)) return PS_ERR_CUDA;
            g_noalloc_addr[dev] = p;
            g_noalloc_ctx[dev] = ctx;
        }
        ws = g_noalloc_addr[dev];
    }
    // ps_splat_bwd clears the accumulators and the work counter before use, so
    // whatever an earlier call left in the array does not leak into this one.
    return ps_splat_bwd(planes, f, s, rec, key, tile_ptr, tile_ent, capacity, dLdD, dLdN,
                        g_center, g_quat, g_radii, ws, kNoAllocBytes, d_status, stream);
}
