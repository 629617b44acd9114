// ps_seednet.cu -- the non-GEMM kernels of the seed-proposal network.
//
// The network (4 convolutions 3x3 stride 2 with 64 channels and ReLU, global
// average pooling, a 64 -> 96 linear layer) maps a 64x64 depth + normal patch
// to 8 plane seeds.  Convolutions run as im2col + tensor-core GEMM
// (ps_gemm.cu); this file holds the data movement around the GEMMs and the
// set loss.  Activations are NHWC bf16; gradients fp32 unless noted; the im2col
// column order is (ky, kx, c), zero-padded to a multiple of 64.
#include <cuda_bf16.h>

#include "ps_internal.cuh"

using namespace ps;

namespace {

constexpr int kT = 256;

inline int blocks_for(long long n)
{
    long long b = (n + kT - 1) / kT;
    if (b > 152 * 32) b = 152 * 32;
    return (int)(b < 1 ? 1 : b);
}

// A[p, k] = x[b, 2 oy - 1 + ky, 2 ox - 1 + kx, c] (0 outside), k = (ky 3 + kx) C + c
__global__ void k_im2col(const __nv_bfloat16* __restrict__ x, int B, int H, int W, int C, int Ho,
                         int Wo, int Kp, __nv_bfloat16* __restrict__ A)
{
    const long long n = (long long)B * Ho * Wo * Kp;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i % Kp);
        const long long p = i / Kp;
        __nv_bfloat16 v = __float2bfloat16(0.f);
        if (k < 9 * C) {
            const int tap = k / C, c = k - tap * C;
            const int ky = tap / 3, kx = tap - ky * 3;
            const int ox = (int)(p % Wo);
            const long long t = p / Wo;
            const int oy = (int)(t % Ho);
            const int b = (int)(t / Ho);
            const int y = 2 * oy - 1 + ky, xx = 2 * ox - 1 + kx;
            if (y >= 0 && y < H && xx >= 0 && xx < W) v = x[(((long long)b * H + y) * W + xx) * C + c];
        }
        A[i] = v;
    }
}

// dx[b, y, x, c] = sum over taps whose stride-2 window covers (y, x) of dA[p, k]
__global__ void k_col2im(const float* __restrict__ dA, int B, int H, int W, int C, int Ho, int Wo,
                         int Kp, float* __restrict__ dx)
{
    const long long n = (long long)B * H * W * C;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        long long t = i / C;
        const int x = (int)(t % W);
        t /= W;
        const int y = (int)(t % H);
        const int b = (int)(t / H);
        float s = 0.f;
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
            const int yy = y + 1 - ky;
            if (yy < 0 || (yy & 1) || (yy >> 1) >= Ho) continue;
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                const int xx = x + 1 - kx;
                if (xx < 0 || (xx & 1) || (xx >> 1) >= Wo) continue;
                const long long p = ((long long)b * Ho + (yy >> 1)) * Wo + (xx >> 1);
                s += dA[p * Kp + (ky * 3 + kx) * C + c];
            }
        }
        dx[i] = s;
    }
}

// dz = dy * (y > 0) (ReLU backward); bf16 copy and optional fp32 copy
__global__ void k_relu_bwd(const float* __restrict__ dy, const __nv_bfloat16* __restrict__ y,
                           long long n, float scale, __nv_bfloat16* __restrict__ dz16,
                           float* __restrict__ dz32)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float g = (__bfloat162float(y[i]) > 0.f) ? dy[i] * scale : 0.f;
        if (dz16) dz16[i] = __float2bfloat16(g);
        if (dz32) dz32[i] = g;
    }
}

// out[c, r] = in[r, c] for r < R, 0 for R <= r < ldo  (in fp32 or bf16, out bf16)
template <typename T>
__global__ void k_transpose(const T* __restrict__ in, int R, int Cc, int ldi, __nv_bfloat16* __restrict__ out,
                            int ldo)
{
    __shared__ float tile[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int r = r0 + j, c = c0 + threadIdx.x;
        float v = 0.f;
        if (r < R && c < Cc) v = (float)in[(long long)r * ldi + c];
        tile[j][threadIdx.x] = v;
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int c = c0 + j, r = r0 + threadIdx.x;
        if (c < Cc && r < ldo) out[(long long)c * ldo + r] = __float2bfloat16(tile[threadIdx.x][j]);
    }
}

// db[c] = sum_r dz[r, c]  (C <= 128 columns, fp32 input)
__global__ void k_colsum(const float* __restrict__ dz, long long R, int C, float* __restrict__ db)
{
    const int c = threadIdx.x % C;
    const int lanes = blockDim.x / C;
    const int sub = threadIdx.x / C;
    float s = 0.f;
    for (long long r = (long long)blockIdx.x * lanes + sub; r < R; r += (long long)gridDim.x * lanes)
        s += dz[r * C + c];
    if (sub < lanes) atomicAdd(&db[c], s);
}

// h[b, c] = mean over S positions of y[b, s, c]
__global__ void k_pool_fwd(const __nv_bfloat16* __restrict__ y, int B, int S, int C,
                           float* __restrict__ h32, __nv_bfloat16* __restrict__ h16)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * C) return;
    const int b = i / C, c = i - b * C;
    float s = 0.f;
    for (int k = 0; k < S; ++k) s += __bfloat162float(y[((long long)b * S + k) * C + c]);
    s /= (float)S;
    if (h32) h32[i] = s;
    if (h16) h16[i] = __float2bfloat16(s);
}

// dy[b, s, c] = dh[b, c] / S  (before the ReLU mask)
__global__ void k_pool_bwd(const float* __restrict__ dh, int B, int S, int C, float* __restrict__ dy)
{
    const long long n = (long long)B * S * C;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const int b = (int)(i / ((long long)S * C));
        dy[i] = dh[b * C + c] / (float)S;
    }
}

// Set loss of the seed slots.  out[b, 12 j + f]: f 0-2 centre, 3-6 quaternion
// (unnormalised), 7-10 log extents, 11 confidence logit.  tgt[b, j, f]: f 0
// valid, 1-3 centre, 4-7 unit quaternion, 8-11 log extents.  Per slot:
// BCE(logit, valid) + valid (|c - c*|_1 + (1 - |q^.q*|) + 0.5 |e - e*|_1),
// averaged over the batch; dout = d loss / d out; sums[0..3] += the four terms.
__global__ void k_seed_loss(const float* __restrict__ out, const float* __restrict__ tgt, int B,
                            int slots, float* __restrict__ dout, float* __restrict__ sums)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float lc = 0.f, lx = 0.f, lq = 0.f, le = 0.f;
    if (i < B * slots) {
        const float* o = out + (long long)i * 12;
        const float* t = tgt + (long long)i * 12;
        float* d = dout + (long long)i * 12;
        const float invB = 1.f / (float)B;
        const float z = o[11], yv = t[0];
        lc = fmaxf(z, 0.f) - z * yv + log1pf(__expf(-fabsf(z)));
        const float sig = 1.f / (1.f + __expf(-z));
        d[11] = (sig - yv) * invB;
        for (int f = 0; f < 11; ++f) d[f] = 0.f;
        if (yv > 0.5f) {
            for (int f = 0; f < 3; ++f) {
                const float e = o[f] - t[1 + f];
                lx += fabsf(e);
                d[f] = ((e > 0.f) - (e < 0.f)) * invB;
            }
            const float qn = sqrtf(o[3] * o[3] + o[4] * o[4] + o[5] * o[5] + o[6] * o[6]) + 1e-12f;
            float qh[4], dot = 0.f;
            for (int f = 0; f < 4; ++f) { qh[f] = o[3 + f] / qn; dot += qh[f] * t[4 + f]; }
            lq = 1.f - fabsf(dot);
            const float sg = (dot > 0.f) - (dot < 0.f);
            float gqh[4], proj = 0.f;
            for (int f = 0; f < 4; ++f) { gqh[f] = -sg * t[4 + f]; proj += gqh[f] * qh[f]; }
            for (int f = 0; f < 4; ++f) d[3 + f] = (gqh[f] - qh[f] * proj) / qn * invB;
            for (int f = 0; f < 4; ++f) {
                const float e = o[7 + f] - t[8 + f];
                le += 0.5f * fabsf(e);
                d[7 + f] = 0.5f * ((e > 0.f) - (e < 0.f)) * invB;
            }
        }
    }
    if (sums) {
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
            lc += __shfl_xor_sync(0xffffffffu, lc, o2);
            lx += __shfl_xor_sync(0xffffffffu, lx, o2);
            lq += __shfl_xor_sync(0xffffffffu, lq, o2);
            le += __shfl_xor_sync(0xffffffffu, le, o2);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&sums[0], lc); atomicAdd(&sums[1], lx);
            atomicAdd(&sums[2], lq); atomicAdd(&sums[3], le);
        }
    }
}

// out[r, c] = bf16(in[r, c]) for c < Cin, 0 for Cin <= c < Cp
__global__ void k_cast_pad(const float* __restrict__ in, int R, int Cin, int Cp,
                           __nv_bfloat16* __restrict__ out)
{
    const long long n = (long long)R * Cp;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % Cp);
        const long long r = i / Cp;
        out[i] = __float2bfloat16(c < Cin ? in[r * Cin + c] : 0.f);
    }
}

}  // namespace

#define ST(s) reinterpret_cast<cudaStream_t>(s)

extern "C" ps_status ps_seed_im2col(const void* x, int B, int H, int W, int C, int Kp, void* A,
                                    ps_stream stream)
{
    if (!x || !A || B <= 0 || H <= 1 || W <= 1 || C <= 0 || Kp < 9 * C || (Kp % 64)) return PS_ERR_ARG;
    const int Ho = (H + 1) / 2, Wo = (W + 1) / 2;
    const long long n = (long long)B * Ho * Wo * Kp;
    k_im2col<<<blocks_for(n), kT, 0, ST(stream)>>>(static_cast<const __nv_bfloat16*>(x), B, H, W, C,
                                                   Ho, Wo, Kp, static_cast<__nv_bfloat16*>(A));
    PS_LAUNCH_CHECK();
    return PS_OK;
}

extern "C" ps_status ps_seed_col2im(const float* dA, int B, int H, int W, int C, int Kp, float* dx,
                                    ps_stream stream)
{
    if (!dA || !dx || B <= 0 || H <= 1 || W <= 1 || C <= 0 || Kp < 9 * C) return PS_ERR_ARG;
    const int Ho = (H + 1) / 2, Wo = (W + 1) / 2;
    const long long n = (long long)B * H * W * C;
    k_col2im<<<blocks_for(n), kT, 0, ST(stream)>>>(dA, B, H, W, C, Ho, Wo, Kp, dx);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

extern "C" ps_status ps_seed_relu_bwd(const float* dy, const void* y, long long n, float scale,
                                      void* dz16, float* dz32, ps_stream stream)
{
    if (!dy || !y || n < 0 || (!dz16 && !dz32)) return PS_ERR_ARG;
    if (n == 0) return PS_OK;
    k_relu_bwd<<<blocks_for(n), kT, 0, ST(stream)>>>(dy, static_cast<const __nv_bfloat16*>(y), n,
                                                     scale, static_cast<__nv_bfloat16*>(dz16), dz32);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

extern "C" ps_status ps_seed_transpose(const void* in, int in_is_bf16, int R, int C, int ldi,
                                       void* out, int ldo, ps_stream stream)
{
    if (!in || !out || R <= 0 || C <= 0 || ldi < C || ldo < R) return PS_ERR_ARG;
    dim3 grid((ldo + 31) / 32, (C + 31) / 32), block(32, 8);
    if (in_is_bf16)
        k_transpose<__nv_bfloat16><<<grid, block, 0, ST(stream)>>>(
            static_cast<const __nv_bfloat16*>(in), R, C, ldi, static_cast<__nv_bfloat16*>(out), ldo);
    else
        k_transpose<float><<<grid, block, 0, ST(stream)>>>(static_cast<const float*>(in), R, C, ldi,
                                                           static_cast<__nv_bfloat16*>(out), ldo);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

extern "C" ps_status ps_seed_colsum(const float* dz, long long R, int C, float* db, ps_stream stream)
{
    if (!dz || !db || R < 0 || C <= 0 || C > 256) return PS_ERR_ARG;
    PS_CUDA_CHECK(cudaMemsetAsync(db, 0, sizeof(float) * C, ST(stream)));
    if (R == 0) return PS_OK;
    const int threads = (256 / C) * C;
    k_colsum<<<152, threads, 0, ST(stream)>>>(dz, R, C, db);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

extern "C" ps_status ps_seed_pool(const void* y, int B, int S, int C, float* h32, void* h16,
                                  ps_stream stream)
{
    if (!y || B <= 0 || S <= 0 || C <= 0 || (!h32 && !h16)) return PS_ERR_ARG;
    k_pool_fwd<<<(B * C + kT - 1) / kT, kT, 0, ST(stream)>>>(static_cast<const __nv_bfloat16*>(y), B,
                                                             S, C, h32,
                                                             static_cast<__nv_bfloat16*>(h16));
    PS_LAUNCH_CHECK();
    return PS_OK;
}

extern "C" ps_status ps_seed_pool_bwd(const float* dh, int B, int S, int C, float* dy, ps_stream stream)
{
    if (!dh || !dy || B <= 0 || S <= 0 || C <= 0) return PS_ERR_ARG;
    const long long n = (long long)B * S * C;
    k_pool_bwd<<<blocks_for(n), kT, 0, ST(stream)>>>(dh, B, S, C, dy);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

extern "C" ps_status ps_seed_loss(const float* out, const float* tgt, int B, int slots, float* dout,
                                  float* sums, ps_stream stream)
{
    if (!out || !tgt || !dout || B <= 0 || slots <= 0) return PS_ERR_ARG;
    if (sums) PS_CUDA_CHECK(cudaMemsetAsync(sums, 0, 4 * sizeof(float), ST(stream)));
    k_seed_loss<<<(B * slots + kT - 1) / kT, kT, 0, ST(stream)>>>(out, tgt, B, slots, dout, sums);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

extern "C" ps_status ps_cast_bf16(const float* in, int R, int Cin, int Cp, void* out, ps_stream stream)
{
    if (!in || !out || R <= 0 || Cin <= 0 || Cp < Cin) return PS_ERR_ARG;
    const long long n = (long long)R * Cp;
    k_cast_pad<<<blocks_for(n), kT, 0, ST(stream)>>>(in, R, Cin, Cp, static_cast<__nv_bfloat16*>(out));
    PS_LAUNCH_CHECK();
    return PS_OK;
}
