// BF16 GEMM on the 5th-generation tensor cores (tcgen05) of sm_103a:
//   C[M x N] (fp32) = A[M x K] (bf16, row-major) * B[N x K]^T (bf16, row-major)
// Both operands are K-major.  One CTA of 128 threads computes a 128 x NT tile:
// it stages K-chunks of 64 of A and B in shared memory in the canonical
// no-swizzle layout (8-row x 16-byte core matrices; consecutive core matrices
// along K 128 bytes apart, along M/N 8 * 128 bytes apart), one elected thread
// issues tcgen05.mma (M = 128, N = NT, K = 16 per instruction) into a TMEM
// accumulator of NT fp32 columns, and tcgen05.commit signals an mbarrier when
// the MMAs have read the chunk.  The 4 warps then read their 32 TMEM lanes
// (rows) with tcgen05.ld and store the tile.  Every wait is bounded; on a
// timeout the kernel records it in the status word, frees its TMEM and leaves.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>

#include "mpm_internal.cuh"

namespace mpm {

constexpr int kUmmaM = 128;
constexpr int kUmmaKC = 64;                       // K per staged chunk
constexpr int kUmmaThreads = 128;

__device__ __forceinline__ uint32_t umma_smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading (K) and
// stride (M/N) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t umma_smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;                      // version
    return d;                                    // base offset 0, lbo mode 0, layout 0 (no swizzle)
}

// Instruction descriptor of tcgen05.mma kind::f16: fp32 accumulator, bf16 A and
// B, both K-major, shape M x N.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N)
{
    return (1u << 4)                  // D format: f32
           | (1u << 7)                // A format: bf16
           | (1u << 10)               // B format: bf16
           | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(umma_smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool umma_mbar_wait(uint64_t *bar, uint32_t phase)
{
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok)
                     : "r"(umma_smem_u32(bar)), "r"(phase)
                     : "memory");
        if (ok) return true;
    }
    return false;
}

template <int NT>
__global__ void __launch_bounds__(kUmmaThreads, 1)
    k_umma_gemm(int M, int N, int K, const __nv_bfloat16 *__restrict__ A, int lda, const __nv_bfloat16 *__restrict__ B,
                int ldb, float *__restrict__ Cout, int ldc, int32_t *__restrict__ status)
{
    static_assert(NT % 16 == 0 && NT >= 32 && NT <= 256, "tile width");
    constexpr int TMEM_COLS = NT <= 32 ? 32 : (NT <= 64 ? 64 : (NT <= 128 ? 128 : 256));
    constexpr uint32_t LBO = 128, SBO = (kUmmaKC / 8) * 128;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *sbase = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                             ~uintptr_t(1023));
    unsigned char *sA = sbase;                                    // 128 x 64 bf16 = 16 KB
    unsigned char *sB = sbase + kUmmaM * kUmmaKC * 2;             // NT x 64 bf16
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kUmmaM, n0 = blockIdx.y * NT;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         umma_smem_u32(&tmem_base)),
                     "r"((uint32_t)TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) umma_mbar_init(&mbar);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    uint32_t phase = 0;
    bool ok = true;
    const int nchunks = (K + kUmmaKC - 1) / kUmmaKC;
    for (int kc = 0; kc < nchunks && ok; ++kc) {
        const int k0 = kc * kUmmaKC;
        // stage A and B chunks: one 16-byte row of a core matrix per copy
        for (int q = tid; q < (kUmmaM + NT) * (kUmmaKC / 8); q += kUmmaThreads) {
            const bool isA = q < kUmmaM * (kUmmaKC / 8);
            const int qq = isA ? q : q - kUmmaM * (kUmmaKC / 8);
            const int r = qq / (kUmmaKC / 8), k8 = qq % (kUmmaKC / 8);
            const int grow = (isA ? m0 : n0) + r, gk = k0 + k8 * 8;
            const int rows = isA ? M : N;
            const __nv_bfloat16 *src = isA ? A + (int64_t)grow * lda + gk : B + (int64_t)grow * ldb + gk;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (grow < rows) {
                if (gk + 8 <= K) {
                    v = *reinterpret_cast<const uint4 *>(src);
                } else {
                    __nv_bfloat16 t[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) t[e] = gk + e < K ? src[e] : __float2bfloat16(0.f);
                    v = *reinterpret_cast<const uint4 *>(t);
                }
            }
            unsigned char *dst = (isA ? sA : sB) + ((r >> 3) * (kUmmaKC / 8) + k8) * 128 + (r & 7) * 16;
            *reinterpret_cast<uint4 *>(dst) = v;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t idesc = umma_idesc_bf16(kUmmaM, NT);
#pragma unroll
            for (int kk = 0; kk < kUmmaKC / 16; ++kk) {
                const uint64_t da = umma_smem_desc(umma_smem_u32(sA) + kk * 2 * 128, LBO, SBO);
                const uint64_t db = umma_smem_desc(umma_smem_u32(sB) + kk * 2 * 128, LBO, SBO);
                const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                             "l"(da), "l"(db), "r"(idesc), "r"(acc)
                             : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             umma_smem_u32(&mbar))
                         : "memory");
        }
        const bool done = umma_mbar_wait(&mbar, phase);
        phase ^= 1u;
        ok = __syncthreads_and(done);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (ok) {
        // epilogue: warp w holds TMEM lanes (rows) 32 w .. 32 w + 31
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < NT; c0 += 8) {
            uint32_t r[8];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7])
                         : "r"(taddr)
                         : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M) {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int col = n0 + c0 + e;
                    if (col < N) Cout[(int64_t)row * ldc + col] = __uint_as_float(r[e]);
                }
            }
        }
    } else if (tid == 0) {
        atomicOr(status, (int32_t)kStatusTimeout);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)TMEM_COLS)
                     : "memory");
}

template <int NT> constexpr size_t umma_smem_bytes() { return (size_t)(kUmmaM + NT) * kUmmaKC * 2 + 1024; }

// C = A B^T for bf16 row-major A (M x K) and B (N x K); fp32 C (M x N).
inline cudaError_t umma_gemm(int M, int N, int K, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb,
                             float *C, int ldc, int32_t *status, cudaStream_t stream)
{
    if (N <= 32) {
        static bool a = false;
        if (!a) { cudaFuncSetAttribute(k_umma_gemm<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)umma_smem_bytes<32>()); a = true; }
        dim3 g((M + kUmmaM - 1) / kUmmaM, (N + 31) / 32);
        k_umma_gemm<32><<<g, kUmmaThreads, umma_smem_bytes<32>(), stream>>>(M, N, K, A, lda, B, ldb, C, ldc, status);
    } else {
        static bool a = false;
        if (!a) { cudaFuncSetAttribute(k_umma_gemm<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)umma_smem_bytes<128>()); a = true; }
        dim3 g((M + kUmmaM - 1) / kUmmaM, (N + 127) / 128);
        k_umma_gemm<128><<<g, kUmmaThreads, umma_smem_bytes<128>(), stream>>>(M, N, K, A, lda, B, ldb, C, ldc, status);
    }
    return cudaGetLastError();
}

}  // namespace mpm
