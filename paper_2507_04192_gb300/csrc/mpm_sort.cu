// Sorting particles by (simulation, tile, cell) and building the tile work
// lists.  The paper scatters unsorted particles (Sec. 3.3.1, indexed
// scatter-add); sorting is what lets P2G reduce into shared memory.
//
// Keys are sorted with a stable least-significant-digit radix sort of 8-bit
// digits: a per-block digit histogram, one exclusive scan over
// [digit][block], and a stable scatter in which each warp ranks its elements
// with __match_any_sync.  The sorted order then yields, per tile, its particle
// range, which is cut into work chunks of at most `chunk` particles.
#include <cstdint>

#include "mpm_internal.cuh"

namespace mpm {

namespace {

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__global__ void __launch_bounds__(kSortThreads) k_rs_hist(const uint32_t *__restrict__ keys, int64_t n,
                                                          int shift, uint32_t *__restrict__ hist, int nblk)
{
    __shared__ uint32_t cnt[kRadixBins];
    for (int i = threadIdx.x; i < kRadixBins; i += blockDim.x) cnt[i] = 0u;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortChunk;
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & (kRadixBins - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x) hist[(int64_t)d * nblk + blockIdx.x] = cnt[d];
}

// Exclusive scan of len entries by one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan_exclusive(uint32_t *__restrict__ data, int64_t len)
{
    __shared__ uint32_t warp_sum[32];
    __shared__ uint32_t carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0u;
    __syncthreads();
    constexpr int kPer = 4;
    for (int64_t base = 0; base < len; base += 1024 * kPer) {
        uint32_t v[kPer];
        uint32_t sum = 0u;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t i = base + (int64_t)tid * kPer + k;
            v[k] = i < len ? data[i] : 0u;
            sum += v[k];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_sum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t ws = warp_sum[lane];
            uint32_t wi = ws;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            warp_sum[lane] = wi - ws;            // exclusive warp offsets
        }
        __syncthreads();
        uint32_t run = carry + warp_sum[warp] + (incl - sum);
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t i = base + (int64_t)tid * kPer + k;
            if (i < len) data[i] = run;
            run += v[k];
        }
        __syncthreads();
        if (tid == 1023) carry = run;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kSortThreads) k_rs_scatter(const uint32_t *__restrict__ kin,
                                                             const int32_t *__restrict__ vin,
                                                             uint32_t *__restrict__ kout,
                                                             int32_t *__restrict__ vout, int64_t n, int shift,
                                                             const uint32_t *__restrict__ hist, int nblk)
{
    constexpr int kWarps = kSortThreads / 32;
    __shared__ uint32_t run[kRadixBins];
    __shared__ uint32_t wcnt[kWarps][kRadixBins];
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int d = tid; d < kRadixBins; d += blockDim.x) {
        run[d] = hist[(int64_t)d * nblk + blockIdx.x];
        for (int w = 0; w < kWarps; ++w) wcnt[w][d] = 0u;
    }
    __syncthreads();
    const uint32_t lt = lanemask_lt();
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = (int64_t)blockIdx.x * kSortChunk + (int64_t)r * kSortThreads + tid;
        const bool valid = i < n;
        const uint32_t key = valid ? kin[i] : 0u;
        const uint32_t digit = (key >> shift) & (kRadixBins - 1);
        const uint32_t peers = __match_any_sync(0xffffffffu, valid ? digit : (uint32_t)kRadixBins);
        const uint32_t rank = __popc(peers & lt);
        if (valid && rank == 0u) wcnt[warp][digit] = __popc(peers);
        __syncthreads();
        if (tid < kRadixBins) {
            uint32_t acc = run[tid];
            for (int w = 0; w < kWarps; ++w) {
                const uint32_t c = wcnt[w][tid];
                wcnt[w][tid] = acc;
                acc += c;
            }
            run[tid] = acc;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = wcnt[warp][digit] + rank;
            kout[pos] = key;
            vout[pos] = vin[i];
        }
        __syncthreads();
        if (tid < kRadixBins)
            for (int w = 0; w < kWarps; ++w) wcnt[w][tid] = 0u;
        __syncthreads();
    }
}

__global__ void k_tile_bounds(const uint32_t *__restrict__ keys, int64_t n, int cell_bits,
                              int32_t *__restrict__ tstart, int32_t *__restrict__ tend)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = keys[i] >> cell_bits;
        if (i == 0 || (keys[i - 1] >> cell_bits) != t) tstart[t] = (int32_t)i;
        if (i == n - 1 || (keys[i + 1] >> cell_bits) != t) tend[t] = (int32_t)(i + 1);
    }
}

// Block-wide exclusive scan (1024 threads) of one value per thread.
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t *warp_sum, int32_t &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int32_t ws = warp_sum[lane];
        int32_t wi = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        warp_sum[lane] = wi - ws;
        if (lane == 31) warp_sum[32] = wi;
    }
    __syncthreads();
    const int32_t excl = warp_sum[warp] + incl - v;
    total = warp_sum[32];
    __syncthreads();
    return excl;
}

__global__ void __launch_bounds__(1024) k_build_chunks(const int32_t *__restrict__ tstart,
                                                       const int32_t *__restrict__ tend, int64_t ntiles,
                                                       int chunk, int4 *__restrict__ chunks, int64_t max_chunks,
                                                       int32_t *__restrict__ counters, int32_t *__restrict__ status)
{
    __shared__ int32_t warp_sum[33];
    int64_t carry_c = 0, carry_t = 0;
    bool overflow = false;
    for (int64_t base = 0; base < ntiles; base += 1024) {
        const int64_t t = base + threadIdx.x;
        const int32_t s = t < ntiles ? tstart[t] : -1;
        const int32_t cnt = s >= 0 ? tend[t] - s : 0;
        const int32_t nch = cnt > 0 ? (cnt + chunk - 1) / chunk : 0;
        int32_t tot_c, tot_t;
        const int32_t off = block_exclusive_scan(nch, warp_sum, tot_c);
        block_exclusive_scan(cnt > 0 ? 1 : 0, warp_sum, tot_t);
        for (int32_t j = 0; j < nch; ++j) {
            const int64_t idx = carry_c + off + j;
            if (idx < max_chunks) {
                const int32_t st = s + j * chunk;
                const int32_t c = min(chunk, cnt - j * chunk);
                chunks[idx] = make_int4((int32_t)t, st, c, 0);
            } else {
                overflow = true;
            }
        }
        carry_c += tot_c;
        carry_t += tot_t;
    }
    if (overflow) atomicOr(status, (int32_t)kStatusChunkOverflow);
    if (threadIdx.x == 0) {
        counters[0] = (int32_t)(carry_c < max_chunks ? carry_c : max_chunks);
        counters[1] = (int32_t)carry_t;
    }
}

}  // namespace

void radix_sort_pairs(const HostParams &hp, DevState &ds)
{
    const int64_t n = hp.n;
    const int nblk = (int)((n + kSortChunk - 1) / kSortChunk);
    int cur = 0;
    for (int shift = 0; shift < ds.key_bits; shift += kRadixBits) {
        k_rs_hist<<<nblk, kSortThreads, 0, ds.stream>>>(ds.keys[cur], n, shift, ds.hist, nblk);
        k_scan_exclusive<<<1, 1024, 0, ds.stream>>>(ds.hist, (int64_t)kRadixBins * nblk);
        k_rs_scatter<<<nblk, kSortThreads, 0, ds.stream>>>(ds.keys[cur], ds.vals[cur], ds.keys[cur ^ 1],
                                                           ds.vals[cur ^ 1], n, shift, ds.hist, nblk);
        cur ^= 1;
    }
    if (cur == 1) {
        uint32_t *tk = ds.keys[0]; ds.keys[0] = ds.keys[1]; ds.keys[1] = tk;
        int32_t *tv = ds.vals[0]; ds.vals[0] = ds.vals[1]; ds.vals[1] = tv;
    }
}

void build_tiles(const HostParams &hp, DevState &ds)
{
    const int64_t ntiles = (int64_t)hp.batch * hp.tiles_per_sim;
    const int cell_bits = hp.dim == 2 ? Geo<2>::CELL_BITS : Geo<3>::CELL_BITS;
    cudaMemsetAsync(ds.tile_start, 0xff, sizeof(int32_t) * ntiles, ds.stream);
    cudaMemsetAsync(ds.tile_end, 0, sizeof(int32_t) * ntiles, ds.stream);
    int64_t nb = (hp.n + 255) / 256;
    if (nb > (int64_t)ds.num_sms * 16) nb = (int64_t)ds.num_sms * 16;
    k_tile_bounds<<<(int)(nb < 1 ? 1 : nb), 256, 0, ds.stream>>>(ds.keys[0], hp.n, cell_bits, ds.tile_start,
                                                                 ds.tile_end);
    k_build_chunks<<<1, 1024, 0, ds.stream>>>(ds.tile_start, ds.tile_end, ntiles, hp.chunk, ds.chunks,
                                              ds.max_chunks, ds.counters, ds.status);
}

}  // namespace mpm
