// ps_gemm.cu -- BF16 GEMM on the 5th-generation tensor cores (tcgen05), FP32
// accumulation in tensor memory, operands brought in by the Tensor Memory
// Accelerator, for the seed-proposal network's convolutions (im2col form) and
// linear layer.
//
//   C[M, N] = A[M, K] . B[N, K]^T (+ bias[N]) (ReLU) , A and B bf16 row-major
//   (K contiguous), C fp32 or bf16 row-major with leading dimension ldc.
//
// One CTA computes a 128 x 64 tile of C over 64-wide slices of K with
// kStages slices in flight: one thread issues, per slice, one TMA tile copy
// (cp.async.bulk.tensor.2d, 128-byte swizzle) of A (128 rows x 128 bytes) and
// one of B (64 rows) into a shared-memory stage -- rows of 128 bytes in
// 8-row, 1024-byte swizzle atoms, the canonical K-major SWIZZLE_128B layout --
// with an mbarrier counting the bytes; once a stage is full it issues four
// tcgen05.mma (M = 128, N = 64, K = 16; each K step starts 32 bytes further
// into the atom rows) into a 64-column FP32 accumulator in tensor memory and
// commits them to the stage's second mbarrier; the stage is refilled with the
// slice kStages ahead once those MMAs are done.  Rows past M or N and columns
// past K are zero-filled by the copies.  After the last slice every warp reads
// its 32 rows of the accumulator with tcgen05.ld and applies the epilogue.
// Every mbarrier wait is bounded: on time-out the kernel sets an error flag,
// waits (bounded) for the copies and MMAs it issued, frees its tensor memory
// and returns.
#include <stdint.h>
#include <cuda.h>
#include <cuda_bf16.h>

#include "ps_internal.cuh"

using namespace ps;

namespace {

constexpr int BM = 128, BN = 64, BK = 64;
constexpr int kThreads = 128;
constexpr unsigned kTmemCols = 64;           // FP32 accumulator columns (= BN)
constexpr long long kWaitPolls = 1LL << 24;  // bounded mbarrier wait
#ifndef PS_GEMM_STAGES
#define PS_GEMM_STAGES 2
#endif
constexpr int kStages = PS_GEMM_STAGES;
constexpr int kABytes = BM * BK * 2, kBBytes = BN * BK * 2;   // multiples of the 1024-byte atom
constexpr int kStageBytes = kABytes + kBBytes;
static_assert(kStages >= 2 && kStages * kStageBytes >= BM * (BN + 1) * 4, "epilogue tile fits the stages");

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor, K-major with 128-byte swizzle: start address,
// leading byte offset (unused by this layout when one MMA's K fits an atom row;
// 16 bytes), stride byte offset 1024 (between 8-row atoms along M/N), descriptor
// version 1, base offset 0 (atoms 1024-byte aligned), layout type 2 (SWIZZLE_128B).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::f16: D f32, A and B bf16, both K-major, N, M.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, long long polls = kWaitPolls)
{
    for (long long i = 0; i < polls; ++i) {
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
    const float* bias;        // [N] or null
    float* C32;               // [M, ldc] fp32 output, or null
    __nv_bfloat16* C16;       // [M, ldc] bf16 output, or null
    int M, N, K, ldc;
    int relu;
    int accumulate;           // C32 += result
    int* err;                 // status word (device): 1 << PS_ERR_TIMEOUT on a wait time-out
};

// k-slice j of A and B into the stage at sa / sb: one box each (x = j * 64 elements,
// 128 bytes: TMA-aligned), bytes counted on the stage's full barrier
__device__ __forceinline__ void issue_slice(const CUtensorMap* tmA, const CUtensorMap* tmB, uint32_t sa,
                                            uint32_t sb, uint32_t full, int j, int m0, int n0)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(full), "r"(kStageBytes) : "memory");
    const int x = j * BK;
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];"
        :: "r"(sa), "l"(reinterpret_cast<uint64_t>(tmA)), "r"(x), "r"(m0), "r"(full)
        : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];"
        :: "r"(sb), "l"(reinterpret_cast<uint64_t>(tmB)), "r"(x), "r"(n0), "r"(full)
        : "memory");
}

__global__ void __launch_bounds__(kThreads, 1) k_gemm_tc(const __grid_constant__ CUtensorMap tmA,
                                                        const __grid_constant__ CUtensorMap tmB,
                                                        GemmArgs a)
{
    extern __shared__ uint8_t s_dyn[];               // kStages x (A, B) stages, 1024-aligned below
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
    __shared__ uint32_t tmem_base;
    __shared__ int failed;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const uint32_t base = (smem_u32(s_dyn) + 1023u) & ~1023u;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&empty[s])) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        failed = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const int nk = a.K / BK;
    int issued = 0, consumed = 0, committed = 0;    // slices, per thread 0

    if (tid == 0 && nk > 0) {
        const uint32_t idesc = instr_desc(BM, BN);
        // the first kStages slices, one per stage
        for (int j = 0; j < nk && j < kStages; ++j) {
            const uint32_t st = base + (uint32_t)j * kStageBytes;
            issue_slice(&tmA, &tmB, st, st + kABytes, smem_u32(&full[j]), j, m0, n0);
            issued = j + 1;
        }
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % kStages;
            // the u-th use of a stage completes its barriers' phase u: parity (slice / kStages) & 1
            if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((kt / kStages) & 1))) {
                failed = 1;
                break;
            }
            consumed = kt + 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = base + (uint32_t)s * kStageBytes, sb = sa + kABytes;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                // K = 16 is 32 bytes of every 128-byte row of the swizzle atoms
                const uint64_t da = smem_desc_sw128(sa + kk * 32);
                const uint64_t db = smem_desc_sw128(sb + kk * 32);
                const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                    :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(&empty[s])) : "memory");
            committed = kt + 1;
            // refill the previous slice's stage (its MMAs were committed one slice ago)
            // with the slice kStages after it
            const int jn = kt - 1 + kStages;
            if (kt >= 1 && jn < nk) {
                const int sp = (kt - 1) % kStages;
                if (!mbar_wait(smem_u32(&empty[sp]), (uint32_t)(((kt - 1) / kStages) & 1))) {
                    failed = 1;
                    break;
                }
                const uint32_t st = base + (uint32_t)sp * kStageBytes;
                issue_slice(&tmA, &tmB, st, st + kABytes, smem_u32(&full[sp]), jn, m0, n0);
                issued = jn + 1;
            }
        }
        // the accumulator is complete once the last commit has arrived
        if (!failed && !mbar_wait(smem_u32(&empty[(nk - 1) % kStages]),
                                  (uint32_t)(((nk - 1) / kStages) & 1)))
            failed = 1;
        if (failed) {
            if (a.err) atomicOr(a.err, 1 << PS_ERR_TIMEOUT);
            // give copies and MMAs in flight a bounded chance to finish before the
            // shared and tensor memory they use is released
            for (int j = consumed; j < issued; ++j)
                mbar_wait(smem_u32(&full[j % kStages]), (uint32_t)((j / kStages) & 1));
            if (committed > 0)
                mbar_wait(smem_u32(&empty[(committed - 1) % kStages]),
                          (uint32_t)(((committed - 1) / kStages) & 1));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (!failed && nk > 0) {
        // epilogue: warp w reads accumulator lanes (rows) 32w .. 32w + 31 and parks them, with
        // bias and ReLU applied, in the (now free) stage memory, rows padded to 65 floats so
        // that neither the parking nor the row-wise read-back conflicts on banks; the tile
        // then leaves in coalesced row segments
        float* tile = reinterpret_cast<float*>(s_dyn + (base - smem_u32(s_dyn)));
        const int rl = warp * 32 + lane;
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
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int col = n0 + c0 + j;
                float x = __uint_as_float(r[j]);
                if (a.bias && col < a.N) x += a.bias[col];
                if (a.relu) x = fmaxf(x, 0.f);
                tile[rl * (BN + 1) + c0 + j] = x;
            }
        }
        __syncthreads();
        for (int i = tid; i < BM * BN; i += kThreads) {
            const int rr = i / BN, cc = i - rr * BN;
            const int row = m0 + rr, col = n0 + cc;
            if (row < a.M && col < a.N) {
                const float x = tile[rr * (BN + 1) + cc];
                const size_t o = (size_t)row * a.ldc + col;
                if (a.C32) a.C32[o] = a.accumulate ? a.C32[o] + x : x;
                if (a.C16) a.C16[o] = __float2bfloat16(x);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(tmem), "r"(kTmemCols) : "memory");
}

// The time-out path of mbar_wait on a barrier that nothing arrives on: one
// thread initialises an mbarrier expecting one arrival, waits `polls` polls for
// its first phase, gives up and reports PS_ERR_TIMEOUT; nothing else was issued,
// so nothing is left in flight.
__global__ void k_wait_selftest(int* status, long long polls)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    const uint32_t b = smem_u32(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(b, 0u, polls)) atomicOr(status, 1 << PS_ERR_TIMEOUT);
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" :: "r"(b) : "memory");
}

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                CUtensorMapFloatOOBfill);

EncodeTiled encoder()
{
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

// 2D map of a row-major bf16 matrix [rows][K], boxes of 64 columns (128 bytes) x
// box_rows rows, written to shared memory with the 128-byte swizzle
bool make_map(CUtensorMap* m, const void* ptr, int rows, int K, int box_rows)
{
    EncodeTiled enc = encoder();
    if (!enc) return false;
    const cuuint64_t dim[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t stride[1] = {(cuuint64_t)K * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dim, stride, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
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
    CUtensorMap tmA, tmB;
    if (!make_map(&tmA, A, M, K, BM) || !make_map(&tmB, B, N, K, BN)) return PS_ERR_CUDA;
    GemmArgs a;
    a.bias = bias; a.C32 = C32; a.C16 = static_cast<__nv_bfloat16*>(C16);
    a.M = M; a.N = N; a.K = K; a.ldc = ldc; a.relu = relu; a.accumulate = accumulate;
    a.err = d_err;
    const int dyn = kStages * kStageBytes + 1024;
    static int configured[64] = {0};   // dynamic shared memory attribute, per device
    int dev = 0;
    PS_CUDA_CHECK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        PS_CUDA_CHECK(cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
        if (dev >= 0 && dev < 64) configured[dev] = 1;
    }
    dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN);
    k_gemm_tc<<<grid, kThreads, dyn, reinterpret_cast<cudaStream_t>(stream)>>>(tmA, tmB, a);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

extern "C" ps_status ps_wait_selftest(int* d_status, long long polls, ps_stream stream)
{
    if (!d_status || polls < 1 || polls > (1LL << 24)) return PS_ERR_ARG;
    k_wait_selftest<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(d_status, polls);
    PS_LAUNCH_CHECK();
    return PS_OK;
}
