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

// Compact list of the non-empty tiles: (tile key, first particle, count, 0).
__global__ void __launch_bounds__(1024) k_build_tiles(const int32_t *__restrict__ tstart,
                                                      const int32_t *__restrict__ tend, int64_t ntiles,
                                                      int4 *__restrict__ tiles, int64_t max_tiles,
                                                      int32_t *__restrict__ counters, int32_t *__restrict__ status)
{
    __shared__ int32_t warp_sum[33];
    int64_t carry = 0;
    bool overflow = false;
    for (int64_t base = 0; base < ntiles; base += 1024) {
        const int64_t t = base + threadIdx.x;
        const int32_t s = t < ntiles ? tstart[t] : -1;
        const int32_t cnt = s >= 0 ? tend[t] - s : 0;
        int32_t total;
        const int32_t off = block_exclusive_scan(cnt > 0 ? 1 : 0, warp_sum, total);
        if (cnt > 0) {
            const int64_t idx = carry + off;
            if (idx < max_tiles) tiles[idx] = make_int4((int32_t)t, s, cnt, 0);
            else overflow = true;
        }
        carry += total;
    }
    if (overflow) atomicOr(status, (int32_t)kStatusChunkOverflow);
    if (threadIdx.x == 0) counters[1] = (int32_t)(carry < max_tiles ? carry : max_tiles);
}

// Block-wide exclusive scan over TN cells held in shared memory (256 threads,
// TN / 256 consecutive cells per thread).  out[c] = sum of in[c'] for c' < c;
// returns the total.
template <int TN, class F>
__device__ __forceinline__ int32_t scan_cells(F value, int32_t *out, int32_t *warp_sum)
{
    constexpr int PER = TN / 256;
    const int tid = threadIdx.x;
    int32_t v[PER], local = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        v[j] = value(tid * PER + j);
        local += v[j];
    }
    const int lane = tid & 31, warp = tid >> 5;
    int32_t incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int32_t ws = lane < 8 ? warp_sum[lane] : 0;
        int32_t wi = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < 8) warp_sum[lane] = wi - ws;
        if (lane == 7) warp_sum[32] = wi;
    }
    __syncthreads();
    int32_t run = warp_sum[warp] + incl - local;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        out[tid * PER + j] = run;
        run += v[j];
    }
    const int32_t total = warp_sum[32];
    __syncthreads();
    return total;
}

// Reorder each tile from (cell, rank) to (rank, cell) order, where rank is a
// particle's position within its cell: consecutive slots then hold particles of
// distinct cells, so one thread per cell reads coalesced and one warp of
// particles writes distinct grid nodes.  Writes the gather permutation
// (perm[slot] = source slot), posmap (for the i-th particle in (cell, rank)
// order, its slot relative to the tile start) and the per-tile cell offsets
// into the (cell, rank) order.
constexpr int kRankCap = 32;

template <int TN>
__global__ void __launch_bounds__(256) k_tile_reorder(const int4 *__restrict__ tiles,
                                                      const int32_t *__restrict__ counters,
                                                      const uint32_t *__restrict__ keys,
                                                      const int32_t *__restrict__ vals, int32_t *__restrict__ perm,
                                                      int32_t *__restrict__ posmap, int32_t *__restrict__ cell_off)
{
    __shared__ int32_t cnt[TN];
    __shared__ int32_t cst[TN];
    __shared__ int32_t ovf[TN];
    __shared__ uint16_t Pr[kRankCap][TN];
    __shared__ int32_t Rr[kRankCap + 1];
    __shared__ int32_t warp_sum[33];
    __shared__ int32_t maxcnt;
    const int n_tiles = counters[1];
    for (int k = blockIdx.x; k < n_tiles; k += gridDim.x) {
        const int4 t = tiles[k];
        const int32_t start = t.y, count = t.z;
        for (int c = threadIdx.x; c < TN; c += blockDim.x) cnt[c] = 0;
        if (threadIdx.x == 0) maxcnt = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < count; i += blockDim.x) atomicAdd(&cnt[keys[start + i] & (TN - 1)], 1);
        __syncthreads();
        for (int c = threadIdx.x; c < TN; c += blockDim.x) atomicMax(&maxcnt, cnt[c]);
        scan_cells<TN>([&](int c) { return cnt[c]; }, cst, warp_sum);
        const int rmax = min(maxcnt, kRankCap);
        if (threadIdx.x == 0) Rr[0] = 0;
        for (int r = 0; r < rmax; ++r) {
            int32_t *row = ovf;                 // scratch row, copied to 16-bit storage below
            const int32_t tot = scan_cells<TN>([&](int c) { return cnt[c] > r ? 1 : 0; }, row, warp_sum);
            for (int c = threadIdx.x; c < TN; c += blockDim.x) Pr[r][c] = (uint16_t)row[c];
            if (threadIdx.x == 0) Rr[r + 1] = Rr[r] + tot;
            __syncthreads();
        }
        const bool has_ovf = maxcnt > kRankCap;
        if (has_ovf) scan_cells<TN>([&](int c) { return cnt[c] > kRankCap ? cnt[c] - kRankCap : 0; }, ovf, warp_sum);
        __syncthreads();
        for (int i = threadIdx.x; i < count; i += blockDim.x) {
            const int c = keys[start + i] & (TN - 1);
            const int r = i - cst[c];
            const int pos = r < kRankCap ? Rr[r] + Pr[r][c] : Rr[rmax] + ovf[c] + (r - kRankCap);
            perm[start + pos] = vals[start + i];
            posmap[start + i] = pos;
        }
        int32_t *co = cell_off + (int64_t)k * (TN + 1);
        for (int c = threadIdx.x; c < TN; c += blockDim.x) co[c] = cst[c];
        if (threadIdx.x == 0) co[TN] = count;
        __syncthreads();
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
    k_build_tiles<<<1, 1024, 0, ds.stream>>>(ds.tile_start, ds.tile_end, ntiles, ds.tiles, ds.max_tiles,
                                             ds.counters, ds.status);
    int64_t tb = ds.max_tiles < (int64_t)ds.num_sms * 4 ? ds.max_tiles : (int64_t)ds.num_sms * 4;
    if (tb < 1) tb = 1;
    if (hp.dim == 2)
        k_tile_reorder<Geo<2>::TN><<<(int)tb, 256, 0, ds.stream>>>(ds.tiles, ds.counters, ds.keys[0], ds.vals[0],
                                                                   ds.perm, ds.posmap, ds.cell_off);
    else
        k_tile_reorder<Geo<3>::TN><<<(int)tb, 256, 0, ds.stream>>>(ds.tiles, ds.counters, ds.keys[0], ds.vals[0],
                                                                   ds.perm, ds.posmap, ds.cell_off);
}

}  // namespace mpm
