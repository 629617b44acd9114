// ps_gemm.cu -- BF16 GEMM on the 5th-generation tensor cores (tcgen05), FP32
// accumulation in tensor memory, for the seed-proposal network's convolutions
// (im2col form) and linear layer.
//
//   C[M, N] = A[M, K] . B[N, K]^T (+ bias[N]) (ReLU) , A and B bf16 row-major
//   (K contiguous), C fp32 or bf16 row-major with leading dimension ldc.
//
// One CTA computes a 128 x 64 tile of C.  Per 64-wide slice of K, the four
// warps copy the A (128 x 64) and B (64 x 64) slices into shared memory in the
// canonical K-major, non-swizzled core-matrix layout (8 rows x 16 bytes per
// core matrix, core matrices adjacent in K 128 bytes apart, adjacent in M/N
// 1,024 bytes apart), one thread issues four tcgen05.mma (M = 128, N = 64,
// K = 16 each) into a 64-column FP32 accumulator in tensor memory and commits
// them to an mbarrier; after the last slice every warp reads its 32 rows of the
// accumulator with tcgen05.ld and applies the epilogue.  Every mbarrier wait
// is bounded: on time-out the kernel sets an error flag, frees its tensor
// memory and returns.
#include <stdint.h>
#include <cuda_bf16.h>

#include "ps_internal.cuh"

using namespace ps;

namespace {

constexpr int BM = 128, BN = 64, BK = 64;
constexpr int kThreads = 128;
constexpr unsigned kTmemCols = 64;           // FP32 accumulator columns (= BN)
constexpr long long kWaitPolls = 1LL << 24;  // bounded mbarrier wait

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (K-major, no swizzle): start address, leading
// byte offset (between core matrices adjacent in K), stride byte offset
// (between core matrices adjacent in M/N), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: D f32, A and B bf16, both K-major, N, M.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase)
{
    for (long long i = 0; i < kWaitPolls; ++i) {
        uint32_t done = 0;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

struct GemmArgs {
    const __nv_bfloat16* A;   // [M, K]
    const __nv_bfloat16* B;   // [N, K]
    const float* bias;        // [N] or null
    float* C32;               // [M, ldc] fp32 output, or null
    __nv_bfloat16* C16;       // [M, ldc] bf16 output, or null
    int M, N, K, ldc;
    int relu;
    int accumulate;           // C32 += result
    int* err;                 // error flag (device), set on a wait time-out
};

__global__ void __launch_bounds__(kThreads, 1) k_gemm_tc(GemmArgs a)
{
    __shared__ __align__(1024) uint8_t sA[BM * BK * 2];
    __shared__ __align__(1024) uint8_t sB[BN * BK * 2];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ int failed;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = instr_desc(BM, BN);
    const int nk = a.K / BK;
    uint32_t phase = 0;

    for (int kt = 0; kt < nk; ++kt) {
        // A slice: 128 rows x 8 chunks of 16 bytes; B slice: 64 rows x 8 chunks
        for (int c = tid; c < BM * 8; c += kThreads) {
            const int r = c >> 3, k8 = c & 7;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (m0 + r < a.M)
                v = *reinterpret_cast<const uint4*>(a.A + (size_t)(m0 + r) * a.K + kt * BK + k8 * 8);
            *reinterpret_cast<uint4*>(sA + ((r >> 3) * 8 + k8) * 128 + (r & 7) * 16) = v;
        }
        for (int c = tid; c < BN * 8; c += kThreads) {
            const int r = c >> 3, k8 = c & 7;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (n0 + r < a.N)
                v = *reinterpret_cast<const uint4*>(a.B + (size_t)(n0 + r) * a.K + kt * BK + k8 * 8);
            *reinterpret_cast<uint4*>(sB + ((r >> 3) * 8 + k8) * 128 + (r & 7) * 16) = v;
        }
        // make the generic-proxy stores visible to the tensor cores
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                const uint64_t da = smem_desc(smem_u32(sA) + kk * 256, 128, 1024);
                const uint64_t db = smem_desc(smem_u32(sB) + kk * 256, 128, 1024);
                const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                    :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(&bar)) : "memory");
        }
        // every thread waits for the MMAs to finish reading shared memory
        if (!mbar_wait(smem_u32(&bar), phase)) {
            if (a.err) atomicExch(a.err, 1);
            failed = 1;
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();
        if (failed) break;
    }

    if (!failed && nk > 0) {
        // epilogue: warp w owns accumulator lanes (rows) 32w .. 32w + 31
        const int row = m0 + warp * 32 + lane;
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                  "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                  "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < a.M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = n0 + c0 + j;
                    if (col < a.N) {
                        float x = __uint_as_float(r[j]);
                        if (a.bias) x += a.bias[col];
                        if (a.relu) x = fmaxf(x, 0.f);
                        const size_t o = (size_t)row * a.ldc + col;
                        if (a.C32) a.C32[o] = a.accumulate ? a.C32[o] + x : x;
                        if (a.C16) a.C16[o] = __float2bfloat16(x);
                    }
                }
            }
        }
    }
    if (failed) {
        // give MMAs still in flight a bounded chance to finish before the
        // tensor memory they write is freed
        mbar_wait(smem_u32(&bar), phase);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace

extern "C" ps_status ps_gemm_bf16(const void* A, const void* B, const float* bias, float* C32,
                                  void* C16, int M, int N, int K, int ldc, int relu,
                                  int accumulate, int* d_err, ps_stream stream)
{
    if (!A || !B || (!C32 && !C16)) return PS_ERR_ARG;
    if (M <= 0 || N <= 0 || K <= 0 || (K % BK) != 0 || ldc < N) return PS_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15)) return PS_ERR_ARG;
    if (accumulate && !C32) return PS_ERR_ARG;
    GemmArgs a;
    a.A = static_cast<const __nv_bfloat16*>(A);
    a.B = static_cast<const __nv_bfloat16*>(B);
    a.bias = bias; a.C32 = C32; a.C16 = static_cast<__nv_bfloat16*>(C16);
    a.M = M; a.N = N; a.K = K; a.ldc = ldc; a.relu = relu; a.accumulate = accumulate;
    a.err = d_err;
    dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN);
    k_gemm_tc<<<grid, kThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(a);
    PS_LAUNCH_CHECK();
    return PS_OK;
}
