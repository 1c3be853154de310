// BF16 GEMM on the 5th-generation tensor cores (tcgen05) of sm_103a:
//   C[M x N] (fp32) = A[M x K] (bf16, row-major) * B[N x K]^T (bf16, row-major)
// Both operands are K-major.  One CTA of 128 threads computes a 128 x NT tile
// with an fp32 accumulator of NT columns in TMEM (tcgen05.mma, M = 128, N = NT,
// K = 16 per instruction); the operand tiles arrive by TMA through a ring of
// shared-memory stages; the 4 warps read their 32 TMEM lanes (rows) with
// tcgen05.ld for the epilogue.  Every wait is bounded; on a timeout the kernel
// records it in the status word, frees its TMEM and leaves.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "mpm_internal.cuh"

namespace mpm {

constexpr int kUmmaM = 128;
constexpr int kUmmaKC = 64;                       // K per staged chunk
constexpr int kUmmaThreads = 128;

__device__ __forceinline__ uint32_t umma_smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
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


// Pipeline: the operand tiles are brought in by TMA (cp.async.bulk.tensor,
// 128-byte swizzle: a K-chunk of 64 bf16 is one 128-byte swizzle row per M/N
// row) through a ring of shared-memory stages.  Thread 0 produces
// (waits for a free stage, arms its mbarrier with the byte count, issues the
// two tile loads); thread 32 consumes (waits for a full stage, issues the four
// K = 16 MMAs, commits them to the stage's "empty" mbarrier so the producer can
// refill it).  A final commit signals the epilogue, which reads TMEM and either
// stores C or applies bias + GELU (bf16 copy for the next layer) or bias +
// scaled sigmoid.  All waits are bounded.
// Tile choice: 128 x 128 tiles through a ring of MPM_UMMA_STAGES stages; when N
// >= 256 and the 128 x 256 tiles alone fill every SM (MPM_UMMA_WIDE), 128 x 256
// tiles through MPM_UMMA_WIDE_STAGES stages (half the operand traffic per FLOP).
#ifndef MPM_UMMA_STAGES
#define MPM_UMMA_STAGES 4
#endif
#ifndef MPM_UMMA_WIDE
#define MPM_UMMA_WIDE 1
#endif
#ifndef MPM_UMMA_WIDE_STAGES
#define MPM_UMMA_WIDE_STAGES 4
#endif
// The 128 x 256 path as a persistent kernel with a double-buffered accumulator.
#ifndef MPM_UMMA_PERSIST
#define MPM_UMMA_PERSIST 1
#endif
enum UmmaEpilogue { kEpiStore = 0, kEpiBiasGelu = 1, kEpiBiasSigmoid = 2, kEpiBiasRelu = 3, kEpiBiasLinear = 4 };

struct UmmaEpi {
    int mode = kEpiStore;
    const float *bias = nullptr;      // N
    __nv_bfloat16 *xnext = nullptr;   // kEpiBiasGelu / kEpiBiasRelu: bf16 GELU(z) / max(z, 0), ld = ldc
    float *y = nullptr;               // kEpiBiasSigmoid: lo + (hi - lo) sigmoid(z); kEpiBiasLinear: z; ld = ldc
    float lo = 0.f, hi = 1.f;
};

// Shared-memory descriptor of a K-major tile written by TMA with 128-byte
// swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart (stride byte
// offset), layout type SWIZZLE_128B.
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                      // leading byte offset (unused within a swizzle row)
    d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset: 8 rows x 128 bytes
    d |= (uint64_t)1 << 46;                      // version
    d |= (uint64_t)2 << 61;                      // layout: 128-byte swizzle
    return d;
}

__device__ __forceinline__ bool umma_wait_parity(uint64_t *bar, uint32_t parity)
{
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok)
                     : "r"(umma_smem_u32(bar)), "r"(parity)
                     : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ float umma_gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

// The fused outputs of one accumulator value z (bias added) at offset o.
__device__ __forceinline__ void umma_epi_outputs(const UmmaEpi &epi, int64_t o, float z)
{
    if (epi.mode == kEpiBiasGelu) epi.xnext[o] = __float2bfloat16_rn(umma_gelu(z));
    else if (epi.mode == kEpiBiasRelu) epi.xnext[o] = __float2bfloat16_rn(fmaxf(z, 0.0f));
    else if (epi.mode == kEpiBiasSigmoid) epi.y[o] = epi.lo + (epi.hi - epi.lo) / (1.0f + expf(-z));
    else if (epi.mode == kEpiBiasLinear) epi.y[o] = z;
}

template <int NT, int STAGES>
__global__ void __launch_bounds__(kUmmaThreads, 1)
    k_umma_gemm_tma(int M, int N, int K, const __grid_constant__ CUtensorMap tmA,
                    const __grid_constant__ CUtensorMap tmB, float *__restrict__ Cout, int ldc, UmmaEpi epi,
                    int32_t *__restrict__ status)
{
    static_assert(NT % 16 == 0 && NT >= 32 && NT <= 256, "tile width");
    constexpr int TMEM_COLS = NT <= 32 ? 32 : (NT <= 64 ? 64 : (NT <= 128 ? 128 : 256));
    constexpr uint32_t A_BYTES = kUmmaM * kUmmaKC * 2, B_BYTES = NT * kUmmaKC * 2;
    constexpr uint32_t STAGE = A_BYTES + B_BYTES;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *sbase = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                             ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
    __shared__ uint32_t tmem_base;
    __shared__ int failed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kUmmaM, n0 = blockIdx.y * NT;
    const int nk = (K + kUmmaKC - 1) / kUmmaKC;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         umma_smem_u32(&tmem_base)),
                     "r"((uint32_t)TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(umma_smem_u32(&full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(umma_smem_u32(&empty[s])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(umma_smem_u32(&done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (tid == 0) {                                        // producer
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % STAGES;
            const uint32_t ph = (uint32_t)(kc / STAGES) & 1u;
            if (!umma_wait_parity(&empty[s], ph ^ 1u)) {
                failed = 1;
                break;
            }
            const uint32_t sa = umma_smem_u32(sbase + s * STAGE), sb = sa + A_BYTES;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(umma_smem_u32(&full[s])),
                         "r"(STAGE)
                         : "memory");
            asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                         " [%0], [%1, {%2, %3}], [%4];" ::"r"(sa),
                         "l"(reinterpret_cast<uint64_t>(&tmA)), "r"(kc * kUmmaKC), "r"(m0),
                         "r"(umma_smem_u32(&full[s]))
                         : "memory");
            asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                         " [%0], [%1, {%2, %3}], [%4];" ::"r"(sb),
                         "l"(reinterpret_cast<uint64_t>(&tmB)), "r"(kc * kUmmaKC), "r"(n0),
                         "r"(umma_smem_u32(&full[s]))
                         : "memory");
        }
    } else if (tid == 32) {                                // MMA issuer
        const uint32_t idesc = umma_idesc_bf16(kUmmaM, NT);
        bool ok = true;
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % STAGES;
            const uint32_t ph = (uint32_t)(kc / STAGES) & 1u;
            if (!umma_wait_parity(&full[s], ph)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = umma_smem_u32(sbase + s * STAGE), sb = sa + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < kUmmaKC / 16; ++kk) {
                const uint64_t da = umma_desc_sw128(sa + kk * 32), db = umma_desc_sw128(sb + kk * 32);
                const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                             "l"(da), "l"(db), "r"(idesc), "r"(acc)
                             : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             umma_smem_u32(&empty[s]))
                         : "memory");
        }
        if (!ok) failed = 1;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         umma_smem_u32(&done))
                     : "memory");
    }
    __syncwarp();
    const bool fin = umma_wait_parity(&done, 0u);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool ok = __syncthreads_and(fin) && !failed;
    if (ok) {
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
                    if (col >= N) continue;
                    float z = __uint_as_float(r[e]);
                    const int64_t o = (int64_t)row * ldc + col;
                    if (epi.mode != kEpiStore) z += epi.bias[col];
                    Cout[o] = z;
                    umma_epi_outputs(epi, o, z);
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

// Epilogue of one 8-column chunk of a row: C (and the fused GELU / sigmoid outputs).
__device__ __forceinline__ void umma_store8(const uint32_t r[8], int row, int col0, int N, float *Cout, int ldc,
                                            const UmmaEpi &epi)
{
    const int64_t o0 = (int64_t)row * ldc + col0;
    if (epi.mode == kEpiStore && col0 + 8 <= N && (ldc & 3) == 0) {     // two 16-byte stores
        float4 *d = reinterpret_cast<float4 *>(Cout + o0);
        d[0] = make_float4(__uint_as_float(r[0]), __uint_as_float(r[1]), __uint_as_float(r[2]), __uint_as_float(r[3]));
        d[1] = make_float4(__uint_as_float(r[4]), __uint_as_float(r[5]), __uint_as_float(r[6]), __uint_as_float(r[7]));
        return;
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int col = col0 + e;
        if (col >= N) continue;
        float z = __uint_as_float(r[e]);
        const int64_t o = o0 + e;
        if (epi.mode != kEpiStore) z += epi.bias[col];
        Cout[o] = z;
        umma_epi_outputs(epi, o, z);
    }
}

// Persistent, warp-specialised form for large problems: one CTA per SM walks the
// 128 x 256 tiles (M fastest within bands of 8 N-tiles, so that consecutive
// tiles of the SMs share their B tiles in L2).  Warp 0 produces (TMA into the
// ring of stages), warp 1 issues the MMAs, warps 2-5 run the epilogue; the fp32
// accumulator is double-buffered in TMEM (2 x 256 of the 512 columns), so the
// epilogue of one tile overlaps the main loop of the next.  Every wait is
// bounded; a timeout sets the status word and every role leaves.
constexpr int kUmmaPersistThreads = 192;
template <int STAGES>
__global__ void __launch_bounds__(kUmmaPersistThreads, 1)
    k_umma_gemm_persist(int M, int N, int K, const __grid_constant__ CUtensorMap tmA,
                        const __grid_constant__ CUtensorMap tmB, float *__restrict__ Cout, int ldc, UmmaEpi epi,
                        int32_t *__restrict__ status)
{
    constexpr int NT = 256;
    constexpr uint32_t A_BYTES = kUmmaM * kUmmaKC * 2, B_BYTES = NT * kUmmaKC * 2;
    constexpr uint32_t STAGE = A_BYTES + B_BYTES;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *sbase = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                             ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], acc_full[2], acc_empty[2], done;
    __shared__ uint32_t tmem_base;
    __shared__ int failed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nk = (K + kUmmaKC - 1) / kUmmaKC;
    const int tm = (M + kUmmaM - 1) / kUmmaM, tn = (N + NT - 1) / NT;
    const int n_tiles = tm * tn;
    constexpr int BAND = 8;                              // N-tiles per band
    auto tile_coords = [&](int t, int &m0, int &n0) {
        const int band = t / (BAND * tm);
        const int r = t - band * BAND * tm;
        const int bw = min(BAND, tn - band * BAND);
        m0 = (r / bw) * kUmmaM;
        n0 = (band * BAND + r % bw) * NT;
    };
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         umma_smem_u32(&tmem_base)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(umma_smem_u32(&full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(umma_smem_u32(&empty[s])) : "memory");
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(umma_smem_u32(&acc_full[b])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(umma_smem_u32(&acc_empty[b])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(umma_smem_u32(&done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp == 0) {                                     // producer
        if (lane == 0) {
            int it = 0;
            for (int t = blockIdx.x; t < n_tiles && !failed; t += gridDim.x) {
                int m0, n0;
                tile_coords(t, m0, n0);
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                    if (!umma_wait_parity(&empty[s], ph ^ 1u)) {
                        failed = 1;
                        break;
                    }
                    const uint32_t sa = umma_smem_u32(sbase + s * STAGE), sb = sa + A_BYTES;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                                     umma_smem_u32(&full[s])),
                                 "r"(STAGE)
                                 : "memory");
                    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                                 " [%0], [%1, {%2, %3}], [%4];" ::"r"(sa),
                                 "l"(reinterpret_cast<uint64_t>(&tmA)), "r"(kc * kUmmaKC), "r"(m0),
                                 "r"(umma_smem_u32(&full[s]))
                                 : "memory");
                    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                                 " [%0], [%1, {%2, %3}], [%4];" ::"r"(sb),
                                 "l"(reinterpret_cast<uint64_t>(&tmB)), "r"(kc * kUmmaKC), "r"(n0),
                                 "r"(umma_smem_u32(&full[s]))
                                 : "memory");
                }
            }
        }
    } else if (warp == 1) {                              // MMA issuer
        if (lane == 0) {
            const uint32_t idesc = umma_idesc_bf16(kUmmaM, NT);
            int it = 0, lt = 0;
            for (int t = blockIdx.x; t < n_tiles && !failed; t += gridDim.x, ++lt) {
                const int b = lt & 1;
                if (!umma_wait_parity(&acc_empty[b], ((uint32_t)(lt >> 1) & 1u) ^ 1u)) {
                    failed = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc_addr = tmem + (uint32_t)(b * NT);
                bool ok = true;
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                    if (!umma_wait_parity(&full[s], ph)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = umma_smem_u32(sbase + s * STAGE), sb = sa + A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < kUmmaKC / 16; ++kk) {
                        const uint64_t da = umma_desc_sw128(sa + kk * 32), db = umma_desc_sw128(sb + kk * 32);
                        const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
                        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc_addr),
                                     "l"(da), "l"(db), "r"(idesc), "r"(acc)
                                     : "memory");
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     umma_smem_u32(&empty[s]))
                                 : "memory");
                }
                if (!ok) {
                    failed = 1;
                    break;
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 umma_smem_u32(&acc_full[b]))
                             : "memory");
            }
            // every MMA this thread issued has completed before TMEM is released
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             umma_smem_u32(&done))
                         : "memory");
            if (!umma_wait_parity(&done, 0u)) failed = 1;
        }
    } else {                                             // epilogue: warps 2-5, TMEM lane quarter warp % 4
        const int q = warp & 3;
        int lt = 0;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++lt) {
            const int b = lt & 1;
            bool ok = false;
            if (lane == 0) ok = umma_wait_parity(&acc_full[b], (uint32_t)(lt >> 1) & 1u);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) {
                if (lane == 0) failed = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            int m0, n0;
            tile_coords(t, m0, n0);
            const int row = m0 + q * 32 + lane;
            for (int c0 = 0; c0 < NT; c0 += 8) {
                uint32_t r[8];
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * NT + c0);
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                               "=r"(r[6]), "=r"(r[7])
                             : "r"(taddr)
                             : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (row < M && n0 + c0 < N) umma_store8(r, row, n0 + c0, N, Cout, ldc, epi);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0)                               // this quarter of the accumulator is free again
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(umma_smem_u32(&acc_empty[b]))
                             : "memory");
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (failed && tid == 0) atomicOr(status, (int32_t)kStatusTimeout);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
}

template <int NT, int STAGES> constexpr size_t umma_tma_smem_bytes()
{
    return (size_t)STAGES * (kUmmaM + NT) * kUmmaKC * 2 + 1024;
}

// 2D tensor map of a row-major bf16 matrix (rows x cols, leading dimension ld
// elements) for boxes of box_rows x 64 with 128-byte swizzle.
inline bool umma_tensor_map(CUtensorMap *tm, const __nv_bfloat16 *ptr, int rows, int cols, int ld, int box_rows)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t gstride[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kUmmaKC, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(ptr), gdim, gstride, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int NT, int STAGES>
inline cudaError_t umma_launch(int M, int N, int K, const CUtensorMap &tmA, const CUtensorMap &tmB, float *C, int ldc,
                               const UmmaEpi &epi, int32_t *status, cudaStream_t stream)
{
    constexpr size_t smem = umma_tma_smem_bytes<NT, STAGES>();
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_umma_gemm_tma<NT, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    dim3 g((M + kUmmaM - 1) / kUmmaM, (N + NT - 1) / NT);
    k_umma_gemm_tma<NT, STAGES><<<g, kUmmaThreads, smem, stream>>>(M, N, K, tmA, tmB, C, ldc, epi, status);
    return cudaGetLastError();
}

// C = A B^T through the pipelined TMA kernel, with an optional fused epilogue.
inline cudaError_t umma_gemm_tma(int M, int N, int K, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B,
                                 int ldb, float *C, int ldc, const UmmaEpi &epi, int32_t *status, cudaStream_t stream)
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    }
    const int NT = N <= 32 ? 32
                   : (MPM_UMMA_WIDE && N >= 256 && (int64_t)((M + kUmmaM - 1) / kUmmaM) * ((N + 255) / 256) >= sms)
                       ? 256
                       : 128;
    CUtensorMap tmA, tmB;
    if (!umma_tensor_map(&tmA, A, M, K, lda, kUmmaM) || !umma_tensor_map(&tmB, B, N, K, ldb, NT))
        return cudaErrorInvalidValue;
    if (NT == 32) return umma_launch<32, 4>(M, N, K, tmA, tmB, C, ldc, epi, status, stream);
    if (NT == 256 && MPM_UMMA_PERSIST) {
        constexpr size_t smem = umma_tma_smem_bytes<256, MPM_UMMA_WIDE_STAGES>();
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_umma_gemm_persist<MPM_UMMA_WIDE_STAGES>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            attr = true;
        }
        const int tiles = ((M + kUmmaM - 1) / kUmmaM) * ((N + 255) / 256);
        k_umma_gemm_persist<MPM_UMMA_WIDE_STAGES><<<std::min(sms, tiles), kUmmaPersistThreads, smem, stream>>>(
            M, N, K, tmA, tmB, C, ldc, epi, status);
        return cudaGetLastError();
    }
    if (NT == 256) return umma_launch<256, MPM_UMMA_WIDE_STAGES>(M, N, K, tmA, tmB, C, ldc, epi, status, stream);
    return umma_launch<128, MPM_UMMA_STAGES>(M, N, K, tmA, tmB, C, ldc, epi, status, stream);
}


}  // namespace mpm
