// BF16 tensor-core GEMM on the 5th-generation tensor cores (tcgen05), FP32
// accumulation in tensor memory, for the dense layers of the learned warm
// start (the message-passing network has no counterpart in the paper).
//
//   C[M x N] = epilogue(A[M x K] . B[K x N])
//
// A is row-major with K contiguous (bf16), B is given transposed, Bt[N x K]
// with K contiguous (bf16): both operands are "K-major".  One CTA of 128
// threads computes a 128-row tile with all N columns:
//   * the 4 warps copy the A tile (128 x K) and Bt (N x K) into shared memory
//     in the canonical no-swizzle layout: 8-row x 16-byte core matrices,
//     core (g, c) at g * SBO + c * LBO with LBO = 128 B (cores along K are
//     adjacent) and SBO = (K / 8) * 128 B (next group of 8 rows);
//   * warp 0 allocates N tensor-memory columns (fp32 accumulator: TMEM lane
//     = tile row, column = output column);
//   * one thread issues K / 16 tcgen05.mma (kind::f16, BF16 inputs, F32
//     accumulate, M = 128) and commits them to an mbarrier;
//   * every warp waits on the mbarrier (bounded: on timeout an error bit is
//     set and the kernel still frees its tensor memory), reads its 32 lanes
//     with tcgen05.ld and applies the epilogue.
// Shapes: K in {16, 32, 64, 128}, N in {16, 32, 64, 128}; M any (rows past M
// are zero-filled and not stored).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "pgcp_internal.h"

namespace pgcp {

namespace {

constexpr int TC_THREADS = 128;
constexpr int TC_M = 128;
constexpr unsigned long long TC_WAIT_LIMIT = 1ull << 24;   // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (tcgen05): start address, leading and stride
// byte offsets (all >> 4), fixed version bits 46-48 = 0b001, no swizzle.
__host__ __device__ constexpr uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: F32 accumulator (bits 4-5 = 1), BF16 A and
// B (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// Epilogues
enum : int { EPI_STORE_F32 = 0, EPI_BIAS_RELU_BF16 = 1, EPI_BIAS_F32 = 2 };

template <int N, int K, int EPI>
__global__ void __launch_bounds__(TC_THREADS) k_gemm_tc(const __nv_bfloat16* __restrict__ A, int64_t lda,
                                                        const __nv_bfloat16* __restrict__ Bt, int64_t M,
                                                        const float* __restrict__ bias, void* __restrict__ Cout,
                                                        int64_t ldc, float* __restrict__ Zout, int64_t ldz,
                                                        uint32_t* __restrict__ err) {
    static_assert(K % 16 == 0 && K >= 16 && K <= 128, "K");
    static_assert(N % 16 == 0 && N >= 16 && N <= 128, "N");
    constexpr uint32_t LBO = 128;
    constexpr uint32_t SBO_A = (K / 8) * 128;
    constexpr uint32_t A_BYTES = TC_M * K * 2;
    constexpr uint32_t NCOLS = N < 32 ? 32 : N;   // tensor-memory allocation: power of 2, >= 32
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;
    unsigned char* sB = smem + A_BYTES;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = (int64_t)blockIdx.x * TC_M;

    // tensor memory for the accumulator (warp 0 allocates and later frees it)
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(NCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    // operand tiles: 16-byte chunks (8 bf16) into the core-matrix layout.  A
    // warp takes RPG consecutive rows x CG consecutive chunks: each quarter
    // warp stores 8 rows of one chunk, 128 contiguous bytes (no bank
    // conflict), and the warp reads whole 32-byte sectors (CG * 16 bytes of
    // each of its rows).
    constexpr int KC = K / 8;               // chunks per row
    constexpr int CG = KC < 4 ? KC : 4;     // chunks per warp step
    constexpr int RPG = 32 / CG;            // rows per warp step
    auto chunk_of = [&](int t, int rows, int& m, int& c) {
        const int grp = t / 32, rg = grp % (rows / RPG), cg = grp / (rows / RPG);
        m = rg * RPG + t % RPG;
        c = cg * CG + (t / RPG) % CG;
    };
    for (int t = threadIdx.x; t < TC_M * KC; t += TC_THREADS) {
        int m, c;
        chunk_of(t, TC_M, m, c);
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (row0 + m < M) v = *reinterpret_cast<const uint4*>(A + (row0 + m) * lda + c * 8);
        *reinterpret_cast<uint4*>(sA + (m >> 3) * SBO_A + c * LBO + (m & 7) * 16) = v;
    }
    for (int t = threadIdx.x; t < N * KC; t += TC_THREADS) {
        int n, c;
        chunk_of(t, N, n, c);
        const uint4 v = *reinterpret_cast<const uint4*>(Bt + (int64_t)n * K + c * 8);
        *reinterpret_cast<uint4*>(sB + (n >> 3) * SBO_A + c * LBO + (n & 7) * 16) = v;
    }
    // make the generic-proxy stores visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;

    if (threadIdx.x == 0) {
        constexpr uint32_t idesc = umma_idesc_bf16(TC_M, N);
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
        for (int kk = 0; kk < K / 16; ++kk) {
            // one MMA consumes K = 16: two cores along K, i.e. 2 * LBO bytes further
            const uint64_t ad = umma_desc(a0 + kk * 2 * LBO, LBO, SBO_A);
            const uint64_t bd = umma_desc(b0 + kk * 2 * LBO, LBO, SBO_A);
            const uint32_t acc = kk > 0 ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&mbar)));
    }
    // wait for the accumulator (phase 0), bounded
    bool ok = false;
    for (unsigned long long it = 0; it < TC_WAIT_LIMIT; ++it) {
        uint32_t done = 0;
        asm volatile(
            "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, q;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(&mbar)), "r"(0u));
        if (done) {
            ok = true;
            break;
        }
    }
    ok = __all_sync(0xffffffffu, ok);   // tcgen05.ld is warp-collective: all lanes or none
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        // warp w reads tensor-memory lanes 32 w .. 32 w + 31 (= tile rows); each
        // thread writes its row's 16-column chunks with 16-byte stores when the
        // output rows are 16-byte aligned
        const int64_t row = row0 + warp * 32 + lane;
        constexpr int64_t CB = EPI == EPI_BIAS_RELU_BF16 ? 2 : 4;   // bytes per output value
        const bool vecc = (ldc * CB) % 16 == 0 && (reinterpret_cast<uintptr_t>(Cout) & 15) == 0;
        const bool vecz = (ldz * 4) % 16 == 0 && (reinterpret_cast<uintptr_t>(Zout) & 15) == 0;
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (row < M) {
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]) + (EPI == EPI_STORE_F32 ? 0.f : bias[c0 + j]);
                if (EPI == EPI_BIAS_RELU_BF16) {
                    if (Zout) {
                        float* zp = Zout + row * ldz + c0;
                        if (vecz) {
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                reinterpret_cast<float4*>(zp)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                        } else {
#pragma unroll
                            for (int j = 0; j < 16; ++j) zp[j] = v[j];
                        }
                    }
                    __nv_bfloat16* cp = reinterpret_cast<__nv_bfloat16*>(Cout) + row * ldc + c0;
                    if (vecc) {   // 16 values -> two 16-byte stores
                        uint32_t pk[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(v[2 * q], 0.f), fmaxf(v[2 * q + 1], 0.f));
                            pk[q] = *reinterpret_cast<const uint32_t*>(&h);
                        }
                        reinterpret_cast<uint4*>(cp)[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        reinterpret_cast<uint4*>(cp)[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j) cp[j] = __float2bfloat16_rn(fmaxf(v[j], 0.f));
                    }
                } else {
                    float* cp = reinterpret_cast<float*>(Cout) + row * ldc + c0;
                    if (vecc) {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            reinterpret_cast<float4*>(cp)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j) cp[j] = v[j];
                    }
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicOr(err, (uint32_t)DE_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS));
    }
}

template <int N, int K, int EPI>
void launch_tc(cudaStream_t s, const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* Bt, int64_t M,
               const float* bias, void* C, int64_t ldc, float* Z, int64_t ldz, uint32_t* err) {
    constexpr int smem = TC_M * K * 2 + N * K * 2;
    PGCP_CUDA(cudaFuncSetAttribute(k_gemm_tc<N, K, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const unsigned grid = (unsigned)ceil_div(M, (int64_t)TC_M);
    { k_gemm_tc<N, K, EPI><<<grid, TC_THREADS, smem, s>>>(A, lda, Bt, M, bias, C, ldc, Z, ldz, err); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
}

template <int EPI>
void dispatch_tc(cudaStream_t s, int N, int K, const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* Bt,
                 int64_t M, const float* bias, void* C, int64_t ldc, float* Z, int64_t ldz, uint32_t* err) {
#define PGCP_TC_CASE(NN, KK)                                                  \
    if (N == NN && K == KK) {                                                 \
        launch_tc<NN, KK, EPI>(s, A, lda, Bt, M, bias, C, ldc, Z, ldz, err); \
        return;                                                               \
    }
    PGCP_TC_CASE(16, 64)
    PGCP_TC_CASE(64, 16)
    PGCP_TC_CASE(64, 64)
    PGCP_TC_CASE(64, 128)
    PGCP_TC_CASE(128, 64)
    PGCP_TC_CASE(16, 16)
#undef PGCP_TC_CASE
    fail(PGCP_E_ARG, "tensor-core GEMM: unsupported shape N=" + std::to_string(N) + " K=" + std::to_string(K));
}

}  // namespace

void gemm_bf16_tc(cudaStream_t s, int epi, int N, int K, const void* A, int64_t lda, const void* Bt, int64_t M,
                  const float* bias, void* C, int64_t ldc, float* Z, int64_t ldz, uint32_t* err) {
    if (M <= 0) return;
    if (lda % 8 != 0 || (reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(Bt) & 15))
        fail(PGCP_E_ARG, "tensor-core GEMM: operands must be 16-byte aligned rows");
    const auto* a = static_cast<const __nv_bfloat16*>(A);
    const auto* b = static_cast<const __nv_bfloat16*>(Bt);
    switch (epi) {
        case EPI_STORE_F32: dispatch_tc<EPI_STORE_F32>(s, N, K, a, lda, b, M, bias, C, ldc, Z, ldz, err); break;
        case EPI_BIAS_RELU_BF16: dispatch_tc<EPI_BIAS_RELU_BF16>(s, N, K, a, lda, b, M, bias, C, ldc, Z, ldz, err); break;
        case EPI_BIAS_F32: dispatch_tc<EPI_BIAS_F32>(s, N, K, a, lda, b, M, bias, C, ldc, Z, ldz, err); break;
        default: fail(PGCP_E_ARG, "tensor-core GEMM: unknown epilogue");
    }
}

uint64_t umma_desc_host(uint32_t saddr, uint32_t lbo, uint32_t sbo) { return umma_desc(saddr, lbo, sbo); }
uint32_t umma_idesc_host(int m, int n) { return umma_idesc_bf16(m, n); }

}  // namespace pgcp
