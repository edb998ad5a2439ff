// (c) tile binning with a hand-written stable LSD radix sort.
//
// The per-tile lists are ordered by the composite key (tile, depth, primitive).
// An LSD radix sort of that key processes the depth digits first and the tile
// digits last.  Every pair of one primitive carries the same depth, so the depth
// passes run once over the N primitives (32-bit depth bits, 4 passes of 8 bits,
// values = primitive index, ties kept in index order by stability), the sorted
// primitives then emit their (tile, primitive) pairs in depth order, and the
// remaining passes sort the pairs stably by tile id (ceil(log2 tiles / 8)
// passes).  The result equals a stable sort of (tile << 32 | depth bits) keys
// emitted in primitive order, with depth ties broken by primitive index.
//
// One radix pass = histogram kernel (per-block digit counts) + column scan (one
// block per digit: its counts over the blocks, and the digit's total) + scatter
// kernel (the lower digits' totals added per block; stable in-block ranking
// with warp match/ballot, block-local reorder in shared memory, coalesced
// write-out).  Item counts may live on the device so the whole pipeline runs
// without a host round trip.
#include "gs_internal.h"

namespace gs {

namespace {

constexpr int kRT = 256;              // radix threads per block
constexpr int kRI = 16;               // items per thread
constexpr int kRTile = kRT * kRI;     // items per block
constexpr int kScanT = 1024;

__device__ __forceinline__ uint64_t item_count(const unsigned long long* dcount, uint64_t scount) {
    if (!dcount) return scount;
    uint64_t c = dcount[0];
    return c < scount ? c : scount;   // scount is the capacity
}

// zero_tail: blocks past the item count write zero counts (the whole-table
// scan reads them; the column scan stops at the last block that holds items)
__global__ __launch_bounds__(kRT) void k_radix_hist(const uint32_t* __restrict__ keys,
                                                   const unsigned long long* dcount, uint64_t scount, int shift,
                                                   uint32_t* __restrict__ hist, int nblocks, int zero_tail) {
    __shared__ uint32_t h[256];
    uint64_t count = item_count(dcount, scount);
    uint64_t base = (uint64_t)blockIdx.x * kRTile;
    if (!zero_tail && base >= count) return;   // uniform over the block
    h[threadIdx.x] = 0;
    __syncthreads();
    // all loads first (kRI in flight per thread), then the shared counts
    uint32_t kk[kRI];
#pragma unroll
    for (int r = 0; r < kRI; r++) {
        const uint64_t i = base + (uint64_t)r * kRT + threadIdx.x;
        kk[r] = i < count ? keys[i] : 0u;
    }
#pragma unroll
    for (int r = 0; r < kRI; r++) {
        const uint64_t i = base + (uint64_t)r * kRT + threadIdx.x;
        if (i < count) atomicAdd(&h[(kk[r] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(uint64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// block d: exclusive scan of digit d's counts over the blocks that hold items
// (in place; the others hold zeros and their scatter blocks return at once) and
// the digit's total; the scatter adds the totals of the lower digits itself
__global__ __launch_bounds__(kRT) void k_radix_colscan(uint32_t* __restrict__ hist, int nblocks,
                                                     const unsigned long long* dcount, uint64_t scount,
                                                     uint32_t* __restrict__ dtot) {
    __shared__ uint32_t wsum[kRT / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    uint32_t* col = hist + (uint64_t)blockIdx.x * nblocks;
    const int nb = (int)min((uint64_t)nblocks, (item_count(dcount, scount) + kRTile - 1) / kRTile);
    const int chunk = (nb + kRT - 1) / kRT;
    const int b = min(tid * chunk, nb), e = min(b + chunk, nb);
    uint32_t s = 0;
    for (int i = b; i < e; i++) s += col[i];
    uint32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    uint32_t run = x - s;
    for (int w = 0; w < wid; w++) run += wsum[w];
    for (int i = b; i < e; i++) {
        const uint32_t v = col[i];
        col[i] = run;
        run += v;
    }
    if (tid == kRT - 1) dtot[blockIdx.x] = run;
}

template <bool VALS>
__global__ __launch_bounds__(kRT) void k_radix_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                      uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                      const unsigned long long* dcount, uint64_t scount, int shift,
                                                      const uint32_t* __restrict__ hist, int nblocks,
                                                      const uint32_t* __restrict__ dtot) {
    // Stable block-local ranking with warp-private digit counters: warp w owns
    // the contiguous items [w * 32 kRI, (w + 1) * 32 kRI) of the block's tile, so
    // ordering by (digit, warp, rank inside the warp) keeps input order.
    __shared__ uint32_t sk[kRTile];
    __shared__ uint32_t sv[VALS ? kRTile : 1];
    __shared__ uint16_t wh[kRT / 32][256];   // per-warp digit counts, then per-warp digit offsets
    __shared__ uint32_t bexcl[256];
    __shared__ uint32_t gbase[256];
    __shared__ uint32_t wsum[kRT / 32];
    __shared__ uint32_t dsum[kRT / 32];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t count = item_count(dcount, scount);
    const uint64_t base = (uint64_t)blockIdx.x * kRTile;
    if (base >= count) return;
    const uint32_t nitems = (uint32_t)(count - base < (uint64_t)kRTile ? count - base : (uint64_t)kRTile);

#pragma unroll
    for (int w = 0; w < kRT / 32; w++) wh[w][tid] = 0;
    // all loads first (kRI in flight per thread)
    uint32_t kr[kRI], vr[kRI];
    const uint32_t wbase = (uint32_t)warp * 32u * kRI;
#pragma unroll
    for (int r = 0; r < kRI; r++) {
        const uint32_t i = wbase + (uint32_t)r * 32u + (uint32_t)lane;
        kr[r] = i < nitems ? kin[base + i] : 0u;
        vr[r] = (VALS && i < nitems) ? vin[base + i] : 0u;
    }
    __syncthreads();
    // rank inside the warp, round by round (the rounds are in item order)
    const unsigned lt_mask = (1u << lane) - 1u;
    uint32_t lrank[kRI];
#pragma unroll
    for (int r = 0; r < kRI; r++) {
        const bool valid = wbase + (uint32_t)r * 32u + (uint32_t)lane < nitems;
        const uint32_t d = valid ? ((kr[r] >> shift) & 255u) : 256u;
        // lanes holding the same digit (9 bits, so the invalid sentinel 256 stands apart)
        unsigned peers = 0xffffffffu;
#pragma unroll
        for (int bit = 0; bit < 9; bit++) {
            const unsigned m = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
            peers &= ((d >> bit) & 1u) ? m : ~m;
        }
        const uint32_t before = valid ? wh[warp][d] : 0u;
        __syncwarp();
        if (valid && (peers & lt_mask) == 0u) wh[warp][d] = (uint16_t)(before + __popc(peers));
        __syncwarp();
        lrank[r] = before + __popc(peers & lt_mask);
    }
    __syncthreads();
    // thread tid = digit: offsets of each warp inside the digit, digit totals,
    // block-exclusive scan of the totals
    {
        uint32_t tot = 0;
#pragma unroll
        for (int w = 0; w < kRT / 32; w++) {
            const uint32_t c = wh[w][tid];
            wh[w][tid] = (uint16_t)tot;
            tot += c;
        }
        uint32_t x = tot;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        // start of digit tid in the output: the lower digits' totals (none when the
        // histogram was scanned as one table over (digit, block))
        const uint32_t dt = dtot ? dtot[tid] : 0u;
        uint32_t dx = dt;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, dx, o);
            if (lane >= o) dx += y;
        }
        if (lane == 31) {
            wsum[warp] = x;
            dsum[warp] = dx;
        }
        __syncthreads();
        uint32_t add = 0, dadd = 0;
        for (int w = 0; w < warp; w++) {
            add += wsum[w];
            dadd += dsum[w];
        }
        bexcl[tid] = x - tot + add;
        gbase[tid] = hist[(uint64_t)tid * nblocks + blockIdx.x] + dx - dt + dadd;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRI; r++) {
        if (wbase + (uint32_t)r * 32u + (uint32_t)lane < nitems) {
            const uint32_t d = (kr[r] >> shift) & 255u;
            const uint32_t pos = bexcl[d] + wh[warp][d] + lrank[r];
            sk[pos] = kr[r];
            if (VALS) sv[pos] = vr[r];
        }
    }
    __syncthreads();
    for (uint32_t i = tid; i < nitems; i += kRT) {
        uint32_t key = sk[i];
        uint32_t d = (key >> shift) & 255u;
        uint64_t dst = (uint64_t)gbase[d] + (i - bexcl[d]);
        kout[dst] = key;
        if (VALS) vout[dst] = sv[i];
    }
}

// ---------------------------------------------------------------------------
// tiles per primitive (depth order), scan, pair emission, ranges
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t rect_tiles(uint2 r) {
    uint32_t x0 = r.x & 0xffff, y0 = r.x >> 16, x1 = r.y & 0xffff, y1 = r.y >> 16;
    return (x1 > x0 && y1 > y0) ? (x1 - x0) * (y1 - y0) : 0u;
}

__global__ void k_count_tiles(const uint32_t* __restrict__ sorted_ids, const uint2* __restrict__ rects, uint64_t n,
                              uint32_t* __restrict__ cnt) {
    uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) cnt[j] = rect_tiles(rects[sorted_ids[j]]);
}

constexpr int kScanItems = 16;
constexpr int kScanBlockT = 256;
constexpr int kScanTile = kScanItems * kScanBlockT;

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sh[w];
    __syncthreads();
    return s;
}

__global__ __launch_bounds__(kScanBlockT) void k_scan_partials(const uint32_t* __restrict__ in, uint64_t n,
                                                              unsigned long long* __restrict__ part) {
    __shared__ unsigned long long sh[kScanBlockT / 32];
    uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    unsigned long long s = 0;
    for (int r = 0; r < kScanItems; r++) {
        uint64_t i = base + (uint64_t)r * kScanBlockT + threadIdx.x;
        if (i < n) s += in[i];
    }
    s = block_sum_u64(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// exclusive scan of the block partials (single block) and the grand total
__global__ __launch_bounds__(kScanT) void k_scan_partials_top(unsigned long long* part, int nparts,
                                                             unsigned long long* total, uint64_t cap) {
    __shared__ unsigned long long wsum[kScanT / 32];
    int chunk = (nparts + kScanT - 1) / kScanT;
    int b = threadIdx.x * chunk, e = min(b + chunk, nparts);
    unsigned long long s = 0;
    for (int i = b; i < e; i++) s += part[i];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long x = s;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long t = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        wsum[lane] = t;
    }
    __syncthreads();
    unsigned long long run = x - s + (wid > 0 ? wsum[wid - 1] : 0ull);
    for (int i = b; i < e; i++) {
        unsigned long long v = part[i];
        part[i] = run;
        run += v;
    }
    if (threadIdx.x == kScanT - 1) {
        total[0] = run < cap ? run : cap;     // usable pair count
        total[1] = run > cap ? 1ull : 0ull;   // overflow flag
        total[2] = run;                       // true pair count
    }
}

// in and out may be the same array: every element is read and then written by
// the same thread, and by no other
__global__ __launch_bounds__(kScanBlockT) void k_scan_apply(const uint32_t* in, uint64_t n,
                                                           const unsigned long long* __restrict__ part,
                                                           uint32_t* out) {
    __shared__ uint32_t wsum[kScanBlockT / 32];
    __shared__ uint32_t carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    if (threadIdx.x == 0) carry = (uint32_t)part[blockIdx.x];
    // all loads first (kScanItems in flight per thread): the barriers of the
    // rounds below would otherwise expose one load latency per round
    uint32_t vv[kScanItems];
#pragma unroll
    for (int r = 0; r < kScanItems; r++) {
        const uint64_t i = base + (uint64_t)r * kScanBlockT + threadIdx.x;
        vv[r] = i < n ? in[i] : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kScanItems; r++) {
        uint64_t i = base + (uint64_t)r * kScanBlockT + threadIdx.x;
        uint32_t v = vv[r];
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        uint32_t add = carry;
        for (int w = 0; w < wid; w++) add += wsum[w];
        if (i < n) out[i] = add + x - v;
        __syncthreads();
        if (threadIdx.x == kScanBlockT - 1) carry = add + x;
        __syncthreads();
    }
}

constexpr uint32_t kBigPrim = 256;   // primitives with more tiles are emitted by a whole block

// thread per primitive (depth order): write its (tile, primitive) pairs, row-major over its rect
__global__ void k_emit(const uint32_t* __restrict__ sorted_ids, const uint2* __restrict__ rects,
                       const uint32_t* __restrict__ cnt, const uint32_t* __restrict__ off, uint64_t n, int tiles_x,
                       const unsigned long long* __restrict__ total, uint32_t* __restrict__ pkey,
                       uint32_t* __restrict__ pval, uint32_t* big_list, unsigned int* big_count) {
    // one warp per 32 consecutive primitives (depth order); their pairs are
    // written by consecutive lanes, so the stores coalesce
    const int lane = threadIdx.x & 31;
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (total[1]) return;   // nothing is emitted when the pairs overflow the capacity (uniform)
    uint32_t c = j < n ? cnt[j] : 0u;
    if (c > kBigPrim) {   // emitted by k_emit_big
        big_list[atomicAdd(big_count, 1u)] = (uint32_t)j;
        c = 0u;
    }
    uint32_t p = 0, o = 0, x0 = 0, y0 = 0, w = 1;
    if (c) {
        p = sorted_ids[j];
        const uint2 r = rects[p];
        x0 = r.x & 0xffff;
        y0 = r.x >> 16;
        w = (r.y & 0xffff) - x0;
        o = off[j];
    }
    uint32_t incl = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    const uint32_t excl = incl - c;
    const uint32_t wtotal = __shfl_sync(0xffffffffu, incl, 31);
    for (uint32_t b = 0; b < wtotal; b += 32) {
        const uint32_t q = b + (uint32_t)lane;
        // source lane: the last lane whose exclusive offset is <= q (lanes without
        // pairs share their neighbour's offset and are skipped by taking the last)
        int s = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int m = s + step;
            if (__shfl_sync(0xffffffffu, excl, m) <= q) s = m;
        }
        const uint32_t t = q - __shfl_sync(0xffffffffu, excl, s);
        const uint32_t so = __shfl_sync(0xffffffffu, o, s), sp = __shfl_sync(0xffffffffu, p, s);
        const uint32_t sx = __shfl_sync(0xffffffffu, x0, s), sy = __shfl_sync(0xffffffffu, y0, s);
        const uint32_t sw = __shfl_sync(0xffffffffu, w, s);
        if (q < wtotal) {
            pkey[so + t] = (sy + t / sw) * (uint32_t)tiles_x + sx + t % sw;
            pval[so + t] = sp;
        }
    }
}

__global__ void k_emit_big(const uint32_t* __restrict__ sorted_ids, const uint2* __restrict__ rects,
                           const uint32_t* __restrict__ off, int tiles_x, const unsigned long long* __restrict__ total,
                           uint32_t* __restrict__ pkey, uint32_t* __restrict__ pval, const uint32_t* big_list,
                           const unsigned int* big_count) {
    if (total[1]) return;
    unsigned int nb = *big_count;
    for (unsigned int b = blockIdx.x; b < nb; b += gridDim.x) {
        uint32_t j = big_list[b];
        uint32_t p = sorted_ids[j];
        uint2 r = rects[p];
        uint32_t x0 = r.x & 0xffff, y0 = r.x >> 16, x1 = r.y & 0xffff;
        uint32_t w = x1 - x0;
        uint32_t c = rect_tiles(r);
        uint32_t o = off[j];
        for (uint32_t m = threadIdx.x; m < c; m += blockDim.x) {
            uint32_t y = y0 + m / w, x = x0 + m % w;
            pkey[o + m] = y * (uint32_t)tiles_x + x;
            pval[o + m] = p;
        }
    }
}

__global__ void k_ranges(const uint32_t* __restrict__ keys, const unsigned long long* __restrict__ total,
                         uint64_t cap, uint2* __restrict__ ranges) {
    uint64_t cnt = total[0];
    if (total[1]) return;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t k = keys[i];
        if (i == 0 || keys[i - 1] != k) ranges[k].x = (uint32_t)i;
        if (i == cnt - 1 || keys[i + 1] != k) ranges[k].y = (uint32_t)(i + 1);
    }
}

__global__ void k_ranges_to_offsets(const uint2* ranges, int ntiles, uint32_t* offsets) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    // lists are contiguous in tile order: offset[t] = start of tile t's list or the running end
    if (t < ntiles) {
        uint2 r = ranges[t];
        offsets[t] = r.x;
        if (r.y == 0) offsets[t] = 0xffffffffu;   // empty: filled by the fix-up pass
    }
}

__global__ void k_offsets_fixup(uint32_t* offsets, int ntiles, const unsigned long long* total) {
    // single thread: empty tiles take the start of the next non-empty tile
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint32_t next = (uint32_t)total[0];
    offsets[ntiles] = next;
    for (int t = ntiles - 1; t >= 0; t--) {
        if (offsets[t] == 0xffffffffu)
            offsets[t] = next;
        else
            next = offsets[t];
    }
}

// rects clipped to the grid [0, tiles_x) x [0, tiles_y) here, so no list index
// can leave it whatever the caller passes
__global__ void k_rects_to_keys(const float* depth, const int32_t* rects, uint64_t n, int tiles_x, int tiles_y,
                                uint32_t* keys, uint32_t* vals, uint2* prect) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int x0 = min(max(rects[4 * i + 0], 0), tiles_x), y0 = min(max(rects[4 * i + 1], 0), tiles_y);
    const int x1 = min(max(rects[4 * i + 2], 0), tiles_x), y1 = min(max(rects[4 * i + 3], 0), tiles_y);
    bool vis = x1 > x0 && y1 > y0;
    keys[i] = vis ? __float_as_uint(depth[i]) : 0xffffffffu;
    vals[i] = (uint32_t)i;
    prect[i] = vis ? make_uint2((uint32_t)x0 | ((uint32_t)y0 << 16), (uint32_t)x1 | ((uint32_t)y1 << 16))
                   : make_uint2(0, 0);
}

int radix_blocks(uint64_t cap) { return (int)std::max<uint64_t>(1, div_up(cap, kRTile)); }

int hist_parts(uint64_t cap) { return (int)div_up((uint64_t)256 * radix_blocks(cap), kScanTile); }

// one stable LSD radix sort over `bits` key bits; `cur` returns the index
// (0/1) of the buffer holding the result.  The (digit, block) histogram is
// scanned by block partials -> single-block scan of the partials -> apply.
gs_status radix_sort(uint32_t* k[2], uint32_t* v[2], const unsigned long long* dcount, uint64_t cap, int bits,
                     uint32_t* hist, unsigned long long* hpart, int& cur, cudaStream_t st) {
    const int nblocks = radix_blocks(cap);
    // up to 16,384 blocks a column per digit is short enough for one block to scan
    // (only the blocks that hold items are scanned); beyond, the table is scanned
    // by all blocks (partials, their scan, apply)
    const bool by_column = nblocks <= 16384;
    uint32_t* dtot = by_column ? reinterpret_cast<uint32_t*>(hpart) : nullptr;   // 256 digit totals
    const uint64_t hlen = (uint64_t)256 * nblocks;
    const int nparts = hist_parts(cap);
    unsigned long long* htot = hpart + nparts + 1;   // scratch for the partial scan's totals
    for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<<<nblocks, kRT, 0, st>>>(k[cur], dcount, cap, shift, hist, nblocks, by_column ? 0 : 1);
        if (by_column) {
            k_radix_colscan<<<256, kRT, 0, st>>>(hist, nblocks, dcount, cap, dtot);
        } else {
            k_scan_partials<<<nparts, kScanBlockT, 0, st>>>(hist, hlen, hpart);
            k_scan_partials_top<<<1, kScanT, 0, st>>>(hpart, nparts, htot, ~0ull);
            k_scan_apply<<<nparts, kScanBlockT, 0, st>>>(hist, hlen, hpart, hist);
        }
        k_radix_scatter<true><<<nblocks, kRT, 0, st>>>(k[cur], v[cur], k[cur ^ 1], v[cur ^ 1], dcount, cap, shift,
                                                       hist, nblocks, dtot);
        cur ^= 1;
    }
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

}  // namespace

gs_status alloc_render_work(RenderWork& w, uint64_t n, uint64_t cap_pairs, int ntiles) {
    bool grow_n = n > w.n || !w.recs;
    bool grow_p = cap_pairs > w.cap_pairs || !w.pkey[0];
    bool grow_t = ntiles > w.ntiles_cap || !w.ranges;
    auto A = [](void** p, size_t bytes) -> gs_status {
        cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return set_error(GS_ERR_OOM, std::string("cudaMalloc failed for render scratch: ") + cudaGetErrorString(e));
        }
        return GS_OK;
    };
    uint64_t nn = std::max<uint64_t>(n, 1);
    if (grow_n) {
        cudaFree(w.recs);
        cudaFree(w.rects);
        for (int i = 0; i < 2; i++) {
            cudaFree(w.dkey[i]);
            cudaFree(w.dval[i]);
        }
        cudaFree(w.cnt);
        cudaFree(w.off);
        cudaFree(w.scan_tmp);
        GS_TRY(A((void**)&w.recs, sizeof(BlendRec) * nn));
        GS_TRY(A((void**)&w.rects, sizeof(uint2) * nn));
        for (int i = 0; i < 2; i++) {
            GS_TRY(A((void**)&w.dkey[i], 4 * nn));
            GS_TRY(A((void**)&w.dval[i], 4 * nn));
        }
        GS_TRY(A((void**)&w.cnt, 4 * nn));
        GS_TRY(A((void**)&w.off, 4 * nn));
        GS_TRY(A((void**)&w.scan_tmp, sizeof(unsigned long long) * (div_up(nn, kScanTile) + 1) + 4 * nn + 64));
        w.n = n;
    }
    if (grow_p || grow_n) {
        if (grow_p) {
            for (int i = 0; i < 2; i++) {
                cudaFree(w.pkey[i]);
                cudaFree(w.pval[i]);
            }
            uint64_t cp = std::max<uint64_t>(cap_pairs, 1);
            for (int i = 0; i < 2; i++) {
                GS_TRY(A((void**)&w.pkey[i], 4 * cp));
                GS_TRY(A((void**)&w.pval[i], 4 * cp));
            }
            w.cap_pairs = cap_pairs;
        }
        cudaFree(w.hist);
        cudaFree(w.hpart);
        const uint64_t big = std::max<uint64_t>(w.cap_pairs, w.n);
        uint64_t hb = std::max<uint64_t>(radix_blocks(big), 1);
        GS_TRY(A((void**)&w.hist, 4 * 256 * hb));
        GS_TRY(A((void**)&w.hpart, sizeof(unsigned long long) * std::max(hist_parts(big) + 8, 136)));
    }
    if (grow_t) {
        cudaFree(w.ranges);
        GS_TRY(A((void**)&w.ranges, sizeof(uint2) * std::max(ntiles, 1)));
        w.ntiles_cap = ntiles;
    }
    if (!w.total) {
        GS_TRY(A((void**)&w.total, sizeof(unsigned long long) * 8));
        if (cudaMallocHost((void**)&w.host_total, sizeof(unsigned long long) * 8) != cudaSuccess) {
            cudaGetLastError();
            return set_error(GS_ERR_OOM, "cudaMallocHost failed");
        }
    }
    return GS_OK;
}

void free_render_work(RenderWork& w) {
    cudaFree(w.recs);
    cudaFree(w.rects);
    for (int i = 0; i < 2; i++) {
        cudaFree(w.dkey[i]);
        cudaFree(w.dval[i]);
        cudaFree(w.pkey[i]);
        cudaFree(w.pval[i]);
    }
    cudaFree(w.cnt);
    cudaFree(w.off);
    cudaFree(w.hist);
    cudaFree(w.hpart);
    cudaFree(w.scan_tmp);
    cudaFree(w.ranges);
    cudaFree(w.total);
    if (w.host_total) cudaFreeHost(w.host_total);
    w = RenderWork();
}

// Sorts the preprocess output in w (dkey[0] = depth keys, dval[0] = primitive
// ids, rects) into per-tile lists: w.ranges[tile] and the id array returned in
// *ids_out.  total[0] = usable pair count, total[1] = overflow flag.
gs_status build_tile_lists(RenderWork& w, uint64_t n, int tiles_x, int tiles_y, uint32_t** ids_out, cudaStream_t st) {
    int ntiles = tiles_x * tiles_y;
    int cur = 0;
    // depth order of the primitives
    GS_TRY(radix_sort(w.dkey, w.dval, nullptr, n, 32, w.hist, w.hpart, cur, st));
    const uint32_t* sorted_ids = w.dval[cur];
    w.passes[0] = 4;   // 32-bit depth keys, 8 bits a pass
    // tiles per primitive in depth order, exclusive scan, pair count
    unsigned blocks = (unsigned)div_up(std::max<uint64_t>(n, 1), 256);
    k_count_tiles<<<blocks, 256, 0, st>>>(sorted_ids, w.rects, n, w.cnt);
    int nparts = (int)std::max<uint64_t>(div_up(n, kScanTile), 1);
    unsigned long long* part = (unsigned long long*)w.scan_tmp;
    uint32_t* big_list = (uint32_t*)(part + nparts + 1);
    unsigned int* big_count = big_list + std::max<uint64_t>(n, 1);
    k_scan_partials<<<nparts, kScanBlockT, 0, st>>>(w.cnt, n, part);
    k_scan_partials_top<<<1, kScanT, 0, st>>>(part, nparts, w.total, w.cap_pairs);
    k_scan_apply<<<nparts, kScanBlockT, 0, st>>>(w.cnt, n, part, w.off);
    GS_CUDA(cudaMemsetAsync(big_count, 0, sizeof(unsigned int), st));
    k_emit<<<blocks, 256, 0, st>>>(sorted_ids, w.rects, w.cnt, w.off, n, tiles_x, w.total, w.pkey[0], w.pval[0],
                                   big_list, big_count);
    k_emit_big<<<num_sms() * 2, 256, 0, st>>>(sorted_ids, w.rects, w.off, tiles_x, w.total, w.pkey[0], w.pval[0],
                                              big_list, big_count);
    // stable sort of the pairs by tile id
    int tbits = 1;
    while ((1 << tbits) < ntiles) tbits++;
    int pcur = 0;
    GS_TRY(radix_sort(w.pkey, w.pval, w.total, w.cap_pairs, tbits, w.hist, w.hpart, pcur, st));
    w.passes[1] = (tbits + 7) / 8;
    GS_CUDA(cudaMemsetAsync(w.ranges, 0, sizeof(uint2) * ntiles, st));
    k_ranges<<<num_sms() * 8, 256, 0, st>>>(w.pkey[pcur], w.total, w.cap_pairs, w.ranges);
    GS_CUDA(cudaGetLastError());
    *ids_out = w.pval[pcur];
    return GS_OK;
}

// exclusive scan of n u32 values into out (n entries); total[0..2] (device) gets
// the sum; scratch: div_up(n, kScanTile) + 1 u64
gs_status launch_exclusive_scan(const uint32_t* in, uint64_t n, uint32_t* out, unsigned long long* scratch,
                                unsigned long long* total, cudaStream_t st) {
    const int nparts = (int)std::max<uint64_t>(div_up(n, kScanTile), 1);
    k_scan_partials<<<nparts, kScanBlockT, 0, st>>>(in, n, scratch);
    k_scan_partials_top<<<1, kScanT, 0, st>>>(scratch, nparts, total, ~0ull);
    k_scan_apply<<<nparts, kScanBlockT, 0, st>>>(in, n, scratch, out);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}
uint64_t scan_scratch_len(uint64_t n) { return std::max<uint64_t>(div_up(n, kScanTile), 1) + 1; }

gs_status launch_ranges_to_offsets(const uint2* ranges, int ntiles, uint32_t* offsets,
                                   const unsigned long long* total, cudaStream_t st) {
    k_ranges_to_offsets<<<(ntiles + 255) / 256, 256, 0, st>>>(ranges, ntiles, offsets);
    k_offsets_fixup<<<1, 32, 0, st>>>(offsets, ntiles, total);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status launch_rects_to_keys(const float* depth, const int32_t* rects, uint64_t n, int tiles_x, int tiles_y,
                               uint32_t* keys, uint32_t* vals, uint2* prects, cudaStream_t st) {
    if (n == 0) return GS_OK;
    k_rects_to_keys<<<(unsigned)div_up(n, 256), 256, 0, st>>>(depth, rects, n, tiles_x, tiles_y, keys, vals, prects);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

}  // namespace gs
