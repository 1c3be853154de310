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

// Exclusive scan of data[begin, end) by one block of 1024 threads, starting
// from carry0.
__device__ void block_scan_exclusive(uint32_t *__restrict__ data, int64_t begin, int64_t end, uint32_t carry0)
{
    __shared__ uint32_t warp_sum[32];
    __shared__ uint32_t carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = carry0;
    __syncthreads();
    constexpr int kPer = 4;
    for (int64_t base = begin; base < end; base += 1024 * kPer) {
        uint32_t v[kPer];
        uint32_t sum = 0u;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t i = base + (int64_t)tid * kPer + k;
            v[k] = i < end ? data[i] : 0u;
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
            if (i < end) data[i] = run;
            run += v[k];
        }
        __syncthreads();
        if (tid == 1023) carry = run;
        __syncthreads();
    }
}

// Three-phase exclusive scan of the digit histogram: per-segment sums, a scan
// of the sums by one block, then each segment rescanned from its offset.
__global__ void __launch_bounds__(1024) k_scan_reduce(const uint32_t *__restrict__ data, int64_t len, int64_t seg,
                                                      uint32_t *__restrict__ partial)
{
    __shared__ uint32_t ws[32];
    const int64_t b0 = (int64_t)blockIdx.x * seg, b1 = b0 + seg < len ? b0 + seg : len;
    uint32_t s = 0u;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += 1024) s += data[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = ws[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) partial[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(1024) k_scan_top(uint32_t *__restrict__ partial, int nseg)
{
    block_scan_exclusive(partial, 0, nseg, 0u);
}

__global__ void __launch_bounds__(1024) k_scan_down(uint32_t *__restrict__ data, int64_t len, int64_t seg,
                                                    const uint32_t *__restrict__ partial)
{
    const int64_t b0 = (int64_t)blockIdx.x * seg, b1 = b0 + seg < len ? b0 + seg : len;
    block_scan_exclusive(data, b0, b1, partial[blockIdx.x]);
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

// Compact list of the non-empty tiles: (tile key, first particle, count, index in
// this list); the index stays with a tile in the largest-first copy below.
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
            if (idx < max_tiles) tiles[idx] = make_int4((int32_t)t, s, cnt, (int32_t)idx);
            else overflow = true;
        }
        carry += total;
    }
    if (overflow) atomicOr(status, (int32_t)kStatusChunkOverflow);
    if (threadIdx.x == 0) counters[1] = (int32_t)(carry < max_tiles ? carry : max_tiles);
}

// Copies the compact tile list, ordered by particle count with the largest
// first, to tiles + max_tiles: the persistent G2P blocks claim tiles from that
// copy in order and so finish together (longest-processing-time-first).  P2G
// keeps the spatial order of the original list, whose neighbouring tiles share
// the grid nodes of their windows.  Counting sort on buckets of 32 particles.
__global__ void __launch_bounds__(1024) k_order_tiles(int4 *__restrict__ tiles, const int32_t *__restrict__ counters,
                                                      int64_t max_tiles)
{
    constexpr int NB = 128;
    __shared__ int32_t hist[NB];
    const int n = counters[1];
    int4 *out = tiles + max_tiles;
    for (int b = threadIdx.x; b < NB; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    auto bucket = [](int cnt) { return NB - 1 - min(cnt >> 5, NB - 1); };
    for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&hist[bucket(tiles[i].z)], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int sum = 0;
        for (int b = 0; b < NB; ++b) {
            const int h = hist[b];
            hist[b] = sum;
            sum += h;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int4 t = tiles[i];
        out[atomicAdd(&hist[bucket(t.z)], 1)] = t;
    }
}

// Reorder each tile from (cell, rank) order to (group, rank, cell) order, where
// a group is NG consecutive cells (an 8 x 8 x 2 slab in 3D, the whole tile in
// 2D) and rank is a particle's position within its cell.  The particles of
// rank r of one group ("rank plane") are then contiguous and ordered by cell,
// so one thread per cell reads a plane coalesced and a warp of particles
// touches distinct grid nodes.  A particle of cell c (group g, local cell l)
// and rank r lands at
//     off[g NG] + sum_{r' < r} T_g(r') + #{l' < l : cnt[g NG + l'] > r}
// where off is the exclusive prefix of the cell counts and T_g(r') the number
// of cells of group g holding more than r' particles.  One block of NG threads per
// tile; writes the gather permutation, the position map (slot of each
// (cell, rank) particle) and the per-tile cell offsets.
template <int TN, int NG>
__global__ void __launch_bounds__(NG) k_tile_reorder(const int4 *__restrict__ tiles,
                                                     const int32_t *__restrict__ counters,
                                                     const uint32_t *__restrict__ keys,
                                                     const int32_t *__restrict__ vals, int32_t *__restrict__ perm,
                                                     int32_t *__restrict__ posmap, int32_t *__restrict__ cell_off)
{
    constexpr int NW = NG / 32;
    constexpr int PER = TN / NG;
    __shared__ int32_t cnt[TN];
    __shared__ int32_t cst[TN + 1];
    __shared__ int32_t wsum[NW + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n_tiles = counters[1];
    for (int k = blockIdx.x; k < n_tiles; k += gridDim.x) {
        const int4 t = tiles[k];
        const int32_t start = t.y, count = t.z;
        for (int c = tid; c < TN; c += NG) cnt[c] = 0;
        __syncthreads();
        for (int i = tid; i < count; i += NG) atomicAdd(&cnt[keys[start + i] & (TN - 1)], 1);
        __syncthreads();
        // exclusive prefix of the counts over the TN cells (PER consecutive cells per thread)
        {
            int32_t v[PER], local = 0;
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                v[j] = cnt[tid * PER + j];
                local += v[j];
            }
            int32_t incl = local;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t x = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += x;
            }
            if (lane == 31) wsum[warp] = incl;
            __syncthreads();
            if (tid == 0) {
                int32_t run = 0;
                for (int w = 0; w < NW; ++w) {
                    const int32_t x = wsum[w];
                    wsum[w] = run;
                    run += x;
                }
                wsum[NW] = run;
            }
            __syncthreads();
            int32_t run = wsum[warp] + incl - local;
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                cst[tid * PER + j] = run;
                run += v[j];
            }
            if (tid == 0) cst[TN] = wsum[NW];
            __syncthreads();
        }
        const uint32_t lt = (1u << lane) - 1u;
        for (int g = 0; g < TN / NG; ++g) {
            const int c = g * NG + tid;
            const int32_t my = cnt[c];
            const int32_t gbase = cst[g * NG];
            int32_t R = 0;
            for (int r = 0;; ++r) {
                const bool pred = my > r;
                const int32_t T = __syncthreads_count(pred);
                if (T == 0) break;
                const uint32_t ball = __ballot_sync(0xffffffffu, pred);
                if (lane == 0) wsum[warp] = __popc(ball);
                __syncthreads();
                int32_t before = 0;
                for (int w = 0; w < warp; ++w) before += wsum[w];
                if (pred) {
                    const int32_t pos = gbase + R + before + __popc(ball & lt);
                    perm[start + pos] = vals[start + cst[c] + r];
                    posmap[start + cst[c] + r] = pos;
                }
                R += T;
                __syncthreads();
            }
        }
        int32_t *co = cell_off + (int64_t)k * (TN + 1);
        for (int c = tid; c <= TN; c += NG) co[c] = cst[c];
        __syncthreads();
    }
}

}  // namespace

// Exclusive scan of len entries in place (partial: kScanSegments scratch words).
void scan_exclusive(uint32_t *data, int64_t len, uint32_t *partial, cudaStream_t stream)
{
    int64_t seg = (len + kScanSegments - 1) / kScanSegments;
    seg = (seg + 4095) / 4096 * 4096;
    if (seg < 4096) seg = 4096;
    const int nseg = (int)((len + seg - 1) / seg);
    if (nseg <= 1) {
        k_scan_top<<<1, 1024, 0, stream>>>(data, (int)len);
        return;
    }
    k_scan_reduce<<<nseg, 1024, 0, stream>>>(data, len, seg, partial);
    k_scan_top<<<1, 1024, 0, stream>>>(partial, nseg);
    k_scan_down<<<nseg, 1024, 0, stream>>>(data, len, seg, partial);
}

void radix_sort_pairs(const HostParams &hp, DevState &ds)
{
    const int64_t n = hp.n;
    const int nblk = (int)((n + kSortChunk - 1) / kSortChunk);
    int cur = 0;
    for (int shift = 0; shift < ds.key_bits; shift += kRadixBits) {
        k_rs_hist<<<nblk, kSortThreads, 0, ds.stream>>>(ds.keys[cur], n, shift, ds.hist, nblk);
        scan_exclusive(ds.hist, (int64_t)kRadixBins * nblk, ds.hist + (int64_t)kRadixBins * nblk, ds.stream);
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
    k_order_tiles<<<1, 1024, 0, ds.stream>>>(ds.tiles, ds.counters, ds.max_tiles);
    int64_t tb = ds.max_tiles < (int64_t)ds.num_sms * 8 ? ds.max_tiles : (int64_t)ds.num_sms * 8;
    if (tb < 1) tb = 1;
    if (hp.dim == 2)
        k_tile_reorder<Geo<2>::TN, Geo<2>::NG><<<(int)tb, Geo<2>::NG, 0, ds.stream>>>(
            ds.tiles, ds.counters, ds.keys[0], ds.vals[0], ds.perm, ds.posmap, ds.cell_off);
    else
        k_tile_reorder<Geo<3>::TN, Geo<3>::NG><<<(int)tb, Geo<3>::NG, 0, ds.stream>>>(
            ds.tiles, ds.counters, ds.keys[0], ds.vals[0], ds.perm, ds.posmap, ds.cell_off);
    cudaMemsetAsync(ds.counters + 2, 0, 2 * sizeof(int32_t), ds.stream);   // tile cursors
}

}  // namespace mpm
