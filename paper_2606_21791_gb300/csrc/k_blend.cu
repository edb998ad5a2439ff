// (d) front-to-back alpha blending and (e) comparison against the clean frame.
//
// Blend (3DGS forward pass, composited over white as in Sec. 3 "Metrics and
// severity"): one 256-thread block per 16x16 tile, one thread per pixel.  The
// tile's sorted list is staged through shared memory 256 records at a time.
// Each warp owns an 8x4 pixel block and skips, warp-uniformly, every staged
// primitive whose alpha >= 1/255 box (BlendRec::ex/ey, conservative) misses the
// block.  Per pixel: power = -(a dx^2 + c dy^2)/2 - b dx dy; skip power > 0;
// alpha = opacity exp(power); skip alpha < 1/255; alpha capped at 0.99; stop
// before the primitive that would take T below 1e-4; C += colour alpha T.
// The block leaves as soon as all of its pixels have stopped.
//
// Compare (Definitions 1-2): per tile, squared differences of [0,1]-clamped
// images (NaN counts as 0) are summed in a fixed reduction tree, turned into a
// fixed-point integer and added atomically, so a (variant, view) record does not
// depend on which tiles ran or in what order: a dirty-tile re-blend and a full
// re-render give identical records.
//
// Dirty-tile engine: a persistent kernel takes (variant, view, dirty tile) work
// items from an atomic queue.  A dirty tile is re-blended from the clean sorted
// list with the flipped primitive's clean entry removed and its corrupted record
// merged in at its (depth, index) position, and compared on the fly.
#include <mutex>

#include "gs_internal.h"

namespace gs {

namespace {

constexpr int kBT = 256;

// Shared staging of one batch of list entries.  box = conservative alpha box
// (x0, x1, y0, y1); q0 = (mean x, mean y, ca, cb), q1 = (cc, opacity, r, g), qb = b.
struct Stage {
    float4 box[kBT];
    float4 q0[kBT];
    float4 q1[kBT];
    float qb[kBT];
};

constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ void stage_put(Stage& s, int j, const BlendRec& q) {
    s.box[j] = make_float4(q.mx - q.ex, q.mx + q.ex, q.my - q.ey, q.my + q.ey);
    s.q0[j] = make_float4(q.mx, q.my, q.ca, q.cb);
    s.q1[j] = make_float4(q.cc, q.opac, q.r, q.g);
    s.qb[j] = q.b;
}

__device__ __forceinline__ BlendRec load_rec(const BlendRec* recs, uint32_t id) {
    const float4* p = reinterpret_cast<const float4*>(recs + id);
    float4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
    BlendRec q;
    q.mx = a.x;
    q.my = a.y;
    q.ca = a.z;
    q.cb = a.w;
    q.cc = b.x;
    q.opac = b.y;
    q.ex = b.z;
    q.ey = b.w;
    q.r = c.x;
    q.g = c.y;
    q.b = c.z;
    q.depth = c.w;
    return q;
}

struct Pix {
    float T, c0, c1, c2;
    bool done;
    uint32_t stop;   // list index of the entry that stopped the pixel (T would drop below 1e-4)
};

// Pixel geometry of thread `tid` in a tile: warp w covers an 8x4 block.
struct PixGeo {
    int px, py;
    float pxc, pyc;
    float wx0, wx1, wy0, wy1;   // pixel-centre bounds of the warp's block
    bool inside;
};

__device__ __forceinline__ PixGeo pix_geo(int tile_x, int tile_y, int W, int H) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    PixGeo g;
    int bx = tile_x * kTile + (warp & 1) * 8;
    int by = tile_y * kTile + (warp >> 1) * 4;
    g.px = bx + (lane & 7);
    g.py = by + (lane >> 3);
    g.pxc = (float)g.px + 0.5f;
    g.pyc = (float)g.py + 0.5f;
    g.wx0 = (float)bx + 0.5f;
    g.wx1 = (float)bx + 7.5f;
    g.wy0 = (float)by + 0.5f;
    g.wy1 = (float)by + 3.5f;
    g.inside = g.px < W && g.py < H;
    return g;
}

// Natural pixel of thread index u in a tile (the pix_geo mapping).
__device__ __forceinline__ void pix_of(int tile_x, int tile_y, int u, int& px, int& py) {
    const int w = u >> 5, l = u & 31;
    px = tile_x * kTile + (w & 1) * 8 + (l & 7);
    py = tile_y * kTile + (w >> 1) * 4 + (l >> 3);
}

// 2^x (hardware approximation, flushes subnormal results to zero)
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Exponent of the Gaussian at offset (dx, dy): -(ca dx^2 + cc dy^2)/2 - cb dx dy,
// every operation rounded on its own in this order (no contraction), so it is
// reproducible bit for bit by any fp32 evaluation in the same order -- which
// matters for near-degenerate conics, where cancellation makes the rounding
// error large compared with the value.
__device__ __forceinline__ float gauss_power(float ca, float cb, float cc, float dx, float dy) {
    const float t1 = __fmul_rn(__fmul_rn(ca, dx), dx);
    const float t2 = __fmul_rn(__fmul_rn(cc, dy), dy);
    const float h = __fmul_rn(-0.5f, __fadd_rn(t1, t2));
    const float t3 = __fmul_rn(__fmul_rn(cb, dx), dy);
    return __fsub_rn(h, t3);
}

// alpha of a record at a pixel centre as the blend computes it, before the cap;
// returns false where the blend skips the record (power > 0 or alpha < 1/255).
__device__ __forceinline__ bool blend_alpha(float mx, float my, float ca, float cb, float cc, float opac, float pxc,
                                            float pyc, float& alpha) {
    const float power = gauss_power(ca, cb, cc, __fsub_rn(mx, pxc), __fsub_rn(my, pyc));
    if (power > 0.0f) return false;
    alpha = opac * ex2_approx(__fmul_rn(power, kLog2e));
    return !(alpha < 1.0f / 255.0f);
}

// Work counters (measurement builds of the kernels only): [0] pixel-primitive
// evaluations, [1] tiles blended, [2] list entries staged.
//
// Each warp tests 32 staged entries at a time against its pixel block (one box
// load per lane, a ballot), then walks only the survivors in list order.  An
// entry culled here cannot reach alpha >= 1/255 at any of the warp's pixels, so
// skipping it changes no pixel; a NaN box never culls.
// Checkpoints of the clean blend: the state (T, C) of every pixel of a tile after
// each kCkStride list entries, kept for the first `count` positions of the tile.
constexpr int kCkStride = 64;
constexpr int kCkMaxPerTile = 64;
struct CkWrite {
    float4* ck;      // NULL: no checkpoints
    uint32_t off;    // first checkpoint of this tile
    uint32_t count;  // checkpoints of this tile
};

// One list entry at one pixel: the front-to-back step.  Every operation has
// explicit rounding, so the full-frame, clean and dirty-tile kernels compute the
// same bits wherever this is inlined.  Returns true when the pixel stops here.
__device__ __forceinline__ bool blend_entry(const float4 q0, const float4 q1, float qb, float pxc, float pyc, Pix& p) {
    float alpha;
    if (!blend_alpha(q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, pxc, pyc, alpha)) return false;
    alpha = alpha > 0.99f ? 0.99f : alpha;     // keeps NaN
    const float Tn = __fmul_rn(p.T, __fsub_rn(1.0f, alpha));
    if (Tn < 1e-4f) {
        p.done = true;
        return true;
    }
    const float w = __fmul_rn(alpha, p.T);
    p.c0 = __fmaf_rn(q1.z, w, p.c0);
    p.c1 = __fmaf_rn(q1.w, w, p.c1);
    p.c2 = __fmaf_rn(qb, w, p.c2);
    p.T = Tn;
    return false;
}

// Entries [c, c + 32) of a staged batch for one warp: cull 32 boxes against the
// warp's pixel block with one ballot, then walk the survivors in list order.  An
// entry culled here cannot reach alpha >= 1/255 at any of the warp's pixels, so
// skipping it changes no pixel; a NaN box never culls.
template <bool COUNT, bool TRACK>
__device__ __forceinline__ void blend_chunk(const float4* box, const float4* q0s, const float4* q1s, const float* qbs,
                                            int c, int cnt, uint32_t base, const PixGeo& g, Pix& p,
                                            unsigned int& nev) {
    const int lane = threadIdx.x & 31;
    const int j = c + lane;
    bool pass = false;
    if (j < cnt) {
        const float4 bx = box[j];
        pass = !(bx.y < g.wx0 || bx.x > g.wx1 || bx.w < g.wy0 || bx.z > g.wy1);
    }
    unsigned m = __ballot_sync(0xffffffffu, pass);
    while (m) {
        const int e = c + __ffs(m) - 1;
        m &= m - 1;
        if (p.done) continue;
        if (COUNT) nev++;
        if (blend_entry(q0s[e], q1s[e], qbs[e], g.pxc, g.pyc, p) && TRACK) p.stop = base + (uint32_t)e;
    }
}

template <bool COUNT, bool TRACK>
__device__ __forceinline__ void blend_batch(const Stage& s, int cnt, uint32_t base, const PixGeo& g, Pix& p,
                                            unsigned int& nev, const CkWrite& ckw = CkWrite{nullptr, 0u, 0u}) {
    for (int c = 0; c < cnt; c += 32) {
        if (__all_sync(0xffffffffu, p.done)) return;
        if (ckw.ck && base + (uint32_t)c > 0 && ((base + (uint32_t)c) % kCkStride) == 0) {
            // the state after entries [0, base + c) of the list
            const uint32_t j = (base + (uint32_t)c) / kCkStride;
            if (j <= ckw.count)
                ckw.ck[(size_t)(ckw.off + j - 1) * kBT + threadIdx.x] = make_float4(p.T, p.c0, p.c1, p.c2);
        }
        blend_chunk<COUNT, TRACK>(s.box, s.q0, s.q1, s.qb, c, cnt, base, g, p, nev);
    }
}

__device__ __forceinline__ float clamp01(float v) { return v > 0.0f ? (v < 1.0f ? v : 1.0f) : 0.0f; }

// One pixel's comparison terms: squared error of the [0,1]-clamped values in
// fixed point (integer sums do not depend on the order of accumulation), peak
// |difference|, footprint flag (> 1/255), non-finite flag of the new value.
struct PixCmp {
    unsigned long long fx;
    float m;
    bool foot, nonfin;
};

__device__ __forceinline__ PixCmp pixel_compare(float v0, float v1, float v2, const float* c) {
    PixCmp r;
    const float d0 = clamp01(v0) - clamp01(c[0]);
    const float d1 = clamp01(v1) - clamp01(c[1]);
    const float d2 = clamp01(v2) - clamp01(c[2]);
    const float sq = d0 * d0 + d1 * d1 + d2 * d2;
    r.fx = __float2ull_rn(sq * 549755813888.0f);   // 2^kSseFracBits
    r.m = fmaxf(fmaxf(fabsf(d0), fabsf(d1)), fabsf(d2));   // differences are finite
    r.foot = r.m > 1.0f / 255.0f;
    r.nonfin = !(isfinite(v0) && isfinite(v1) && isfinite(v2));
    return r;
}

// Compare this tile's pixels with the clean image and add to *acc (whole block).
__device__ __forceinline__ void compare_tile(const PixGeo& g, float v0, float v1, float v2, const float* clean, int W,
                                             CmpAcc* acc) {
    __shared__ unsigned long long wsse[kBT / 32];
    __shared__ float wmax[kBT / 32];
    PixCmp r{0ull, 0.0f, false, false};
    if (g.inside) r = pixel_compare(v0, v1, v2, clean + ((size_t)g.py * W + g.px) * 3);
    unsigned long long fx = r.fx;
    float m = r.m;
    for (int o = 16; o > 0; o >>= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        wsse[warp] = fx;
        wmax[warp] = m;
    }
    int nfoot = __syncthreads_count(r.foot);
    int nbad = __syncthreads_count(r.nonfin);
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        float mm = 0.0f;
#pragma unroll
        for (int w = 0; w < kBT / 32; w++) {
            t += wsse[w];
            mm = fmaxf(mm, wmax[w]);
        }
        if (t) atomicAdd(&acc->sse_fx, t);
        if (mm > 0.0f) atomicMax(&acc->maxabs_bits, __float_as_uint(mm));
        if (nfoot) atomicAdd(&acc->footprint, (unsigned)nfoot);
        if (nbad) atomicAdd(&acc->nonfinite, (unsigned)nbad);
    }
}

__device__ __forceinline__ void add_work(unsigned long long* work, unsigned int nev, unsigned int staged) {
    unsigned int w = __reduce_add_sync(0xffffffffu, nev);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(&work[0], (unsigned long long)w);
    if (threadIdx.x == 0) {
        atomicAdd(&work[1], 1ull);
        atomicAdd(&work[2], (unsigned long long)staged);
    }
}

// MODE 0: write the image; 1: compare with the clean image; 2: write the image
// and each pixel's stop index (0xffffffff if it never stopped), which the
// dirty-tile kernel uses to leave pixels that stopped before a change untouched.
template <int MODE, bool COUNT>
__global__ __launch_bounds__(kBT) void k_blend_full(const BlendRec* __restrict__ recs, const uint32_t* __restrict__ ids,
                                                   const uint2* __restrict__ ranges, int W, int H, int tiles_x,
                                                   float* __restrict__ img, const float* __restrict__ clean,
                                                   CmpAcc* acc, unsigned long long* work, uint32_t* __restrict__ stop,
                                                   uint32_t* __restrict__ tile_stop, float4* __restrict__ ck,
                                                   const uint32_t* __restrict__ ck_off,
                                                   const uint32_t* __restrict__ ck_cnt,
                                                   unsigned int* __restrict__ clean_nonfin) {
    __shared__ Stage s;
    const int tile = blockIdx.x;
    const CkWrite ckw{ck, ck ? ck_off[tile] : 0u, ck ? ck_cnt[tile] : 0u};
    const PixGeo g = pix_geo(tile % tiles_x, tile / tiles_x, W, H);
    Pix p{1.0f, 0.0f, 0.0f, 0.0f, !g.inside, 0xffffffffu};
    const uint2 rg = ranges[tile];
    unsigned int nev = 0, staged = 0;
    for (uint32_t base = rg.x; base < rg.y; base += kBT) {
        int cnt = (int)min((uint32_t)kBT, rg.y - base);
        if ((int)threadIdx.x < cnt) stage_put(s, threadIdx.x, load_rec(recs, ids[base + threadIdx.x]));
        __syncthreads();
        staged += cnt;
        blend_batch<COUNT, MODE == 2>(s, cnt, base - rg.x, g, p, nev, ckw);
        // also the barrier that lets the next batch overwrite the stage
        if (__syncthreads_count(p.done) == kBT) break;
    }
    if (COUNT) add_work(work, nev, staged);
    const float v0 = __fadd_rn(p.c0, p.T), v1 = __fadd_rn(p.c1, p.T), v2 = __fadd_rn(p.c2, p.T);   // over white
    if (MODE != 1) {
        if (g.inside) {
            const size_t px = (size_t)g.py * W + g.px;
            float* o = img + px * 3;
            o[0] = v0;
            o[1] = v1;
            o[2] = v2;
            if (MODE == 2) stop[px] = p.stop;
        }
        if (MODE == 2 && clean_nonfin) {
            const bool bad = g.inside && !(isfinite(v0) && isfinite(v1) && isfinite(v2));
            const int nbad = __syncthreads_count(bad);
            if (threadIdx.x == 0 && nbad) atomicAdd(clean_nonfin, (unsigned)nbad);
        }
        if (MODE == 2) {
            // the tile's largest stop index: a change at or after it leaves every pixel as it is
            __shared__ uint32_t wmax[kBT / 32];
            const uint32_t m = __reduce_max_sync(0xffffffffu, g.inside ? p.stop : 0u);
            if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t t = 0;
                for (int w = 0; w < kBT / 32; w++) t = max(t, wmax[w]);
                tile_stop[tile] = t;
            }
        }
    } else {
        compare_tile(g, v0, v1, v2, clean, W, acc);
    }
}

__global__ __launch_bounds__(kBT) void k_compare(const float* __restrict__ a, const float* __restrict__ b, int W, int H,
                                                int tiles_x, CmpAcc* acc) {
    const int tile = blockIdx.x;
    const PixGeo g = pix_geo(tile % tiles_x, tile / tiles_x, W, H);
    float v0 = 0.0f, v1 = 0.0f, v2 = 0.0f;
    if (g.inside) {
        const float* q = a + ((size_t)g.py * W + g.px) * 3;
        v0 = q[0];
        v1 = q[1];
        v2 = q[2];
    }
    compare_tile(g, v0, v1, v2, b, W, acc);
}

// clean_nonfin (dirty engine only): per view, the clean image's non-finite
// pixels, which count for every variant except where a pixel was re-blended.
__global__ void k_finalize(const CmpAcc* acc, int count, gs_result* out, const unsigned int* clean_nonfin, int K) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    CmpAcc a = acc[i];
    gs_result r;
    r.sse = (double)a.sse_fx * (1.0 / 549755813888.0);
    r.maxabs = __uint_as_float(a.maxabs_bits);
    r.footprint = a.footprint;
    r.nonfinite = a.nonfinite + (clean_nonfin ? clean_nonfin[i % K] - a.clean_nonfinite_replaced : 0u);
    r.clamps = a.clamps;
    out[i] = r;
}

__global__ void k_zero_acc(CmpAcc* acc, int count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) acc[i] = CmpAcc{0ull, 0u, 0u, 0u, 0u, 0u, 0u};
}

// ---------------------------------------------------------------------------
// dirty-tile persistent kernel
// ---------------------------------------------------------------------------
struct ViewPtrs {
    const BlendRec* recs;
    const uint32_t* ids;
    const uint32_t* dk;      // depth bits of ids[j] (list-aligned)
    const uint2* ranges;
    const float* clean;
    const uint32_t* stop;    // clean stop index of every pixel
    const uint32_t* tile_stop;   // largest stop index of each tile
    const float4* ck;            // clean-blend checkpoints (T, C) of every pixel
    const uint32_t* ck_off;      // first checkpoint of each tile
    const uint32_t* ck_cnt;      // checkpoints of each tile (after kCkStride, 2 kCkStride, ... entries)
    int W, H, tiles_x, pad;
};

// First index in [lo, hi) whose (depth bits, id) is not below (dkey, p); the
// lists are sorted by (depth, id).  Called by a whole warp: each round probes 31
// splitters and keeps the 1/32 of the interval that holds the answer.
__device__ __forceinline__ uint32_t warp_lower_bound(const uint32_t* __restrict__ dk, const uint32_t* __restrict__ ids,
                                                     uint32_t lo, uint32_t hi, uint32_t dkey, uint32_t p) {
    const int lane = threadIdx.x & 31;
    while (hi - lo > 32) {
        const uint32_t len = hi - lo;
        bool less = false;
        if (lane < 31) {
            const uint32_t pos = lo + (uint32_t)(((uint64_t)len * (uint32_t)(lane + 1)) >> 5);
            const uint32_t k = dk[pos], id = ids[pos];
            less = k < dkey || (k == dkey && id < p);
        }
        const int c = __popc(__ballot_sync(0xffffffffu, less));
        const uint32_t nlo = c == 0 ? lo : lo + (uint32_t)(((uint64_t)len * (uint32_t)c) >> 5) + 1;
        const uint32_t nhi = c == 31 ? hi : lo + (uint32_t)(((uint64_t)len * (uint32_t)(c + 1)) >> 5);
        lo = nlo;
        hi = nhi;
    }
    bool less = false;
    const uint32_t pos = lo + lane;
    if (pos < hi) {
        const uint32_t k = dk[pos], id = ids[pos];
        less = k < dkey || (k == dkey && id < p);
    }
    return lo + __popc(__ballot_sync(0xffffffffu, less));
}

// One dirty tile that needs re-blending (160 B).  ins is the insertion position
// in the clean list without the primitive's old entry; cut is the first changed
// position of the clean list; rec is the corrupted record (when flags bit 1);
// mask marks the tile's active pixels (natural order, 8 x 32 bits).
struct __align__(16) PlanItem {
    BlendRec rec;
    BlendRec orec;    // clean (old) record
    uint32_t mask[kBT / 32];
    uint32_t bk;      // (variant, view) = variant * K + view
    uint32_t tile;
    uint32_t s, e;    // clean list range
    uint32_t pp, ins, cut;
    uint32_t flags;   // bit 0: old entry in this tile, bit 1: corrupted entry in this tile
};

// A pixel of a dirty tile keeps its clean value, bit for bit, when its clean
// blend stopped before the first changed list position, or when its blend skips
// both the removed (clean) and the inserted (corrupted) record (power > 0 or
// alpha < 1/255, decided by the blend's own arithmetic): the state changes of
// its blend are then those of the clean blend.  Every other pixel is "active"
// and must be re-blended.
// Conservative tile test, all in fp32: false only if the blend cannot reach
// alpha >= 1/255 for record q at any pixel centre of the rectangle
// [x0, x1] x [y0, y1].  The blend's offsets d = mean - pixel are fp32
// differences, and rounding is monotone, so every pixel's d lies in the box
// spanned by the rounded corner offsets.  Its power is -q(d)/2 for
// q(d) = ca dx^2 + 2 cb dx dy + cc dy^2 up to a few ulps of
// M = ((|ca| + |cb|) max dx^2 + (|cc| + |cb|) max dy^2)/2 >= the sum of |terms|;
// g = 1e-5 covers that and the rounding of this test's own q (both about
// 1e-6 M).  alpha >= 1/255 needs -q/2 + g M >= -L with L = ln(255 opacity)
// + 1e-3 (the margin covers the fast log and exp2), so the rectangle is
// unreachable when the minimum of q over it exceeds 2 L + 2 g M.  With ca, cc > 0
// the minimum over each edge is that of a convex 1-D quadratic; it is 0 if the
// mean lies inside (then: reachable).  NaN opacity, or terms near overflow
// (where the blend's own power can be NaN, which it blends): reachable.
__device__ __forceinline__ bool tile_reachable(const BlendRec& q, float x0, float x1, float y0, float y1) {
    const float ca = q.ca, cb = q.cb, cc = q.cc;
    const float L = __logf(255.0f * q.opac) + 1e-3f;
    if (L < 0.0f) return false;   // alpha <= opacity < 1/255 everywhere (with margin); NaN falls through
    if (!(ca > 0.0f) || !(cc > 0.0f) || !(L < 3.0e38f)) return true;
    const float dx0 = q.mx - x1, dx1 = q.mx - x0;
    const float dy0 = q.my - y1, dy1 = q.my - y0;
    if (dx0 <= 0.0f && dx1 >= 0.0f && dy0 <= 0.0f && dy1 >= 0.0f) return true;
    const float mdx = fmaxf(dx0 * dx0, dx1 * dx1), mdy = fmaxf(dy0 * dy0, dy1 * dy1);
    const float M = 0.5f * ((ca + fabsf(cb)) * mdx + (cc + fabsf(cb)) * mdy);
    if (!(M < 1.0e37f)) return true;   // terms near overflow: the blend's power may be NaN
    auto qf = [&](float dx, float dy) { return ca * dx * dx + 2.0f * cb * dx * dy + cc * dy * dy; };
    const float rca = 1.0f / ca, rcc = 1.0f / cc;
    // the nearest point of each edge (dx fixed: dy = -cb dx / cc; dy fixed: dx = -cb dy / ca), clamped to it
    const float e0 = qf(dx0, fminf(fmaxf(-cb * dx0 * rcc, dy0), dy1));
    const float e1 = qf(dx1, fminf(fmaxf(-cb * dx1 * rcc, dy0), dy1));
    const float e2 = qf(fminf(fmaxf(-cb * dy0 * rca, dx0), dx1), dy0);
    const float e3 = qf(fminf(fmaxf(-cb * dy1 * rca, dx0), dx1), dy1);
    const float qmin = fminf(fminf(e0, e1), fminf(e2, e3));
    return !(qmin > 2.0f * L + 2.0e-5f * M);
}

__device__ __forceinline__ bool affects(const BlendRec& q, float x, float y) {
    float alpha;
    return blend_alpha(q.mx, q.my, q.ca, q.cb, q.cc, q.opac, x, y, alpha);
}

__device__ __forceinline__ bool pixel_active(int px, int py, int W, int H, uint32_t stop, uint32_t cut, bool has_old,
                                             const BlendRec& orec, bool has_new, const BlendRec& nrec) {
    if (px >= W || py >= H || stop < cut) return false;
    const float x = (float)px + 0.5f, y = (float)py + 0.5f;
    return (has_old && affects(orec, x, y)) || (has_new && affects(nrec, x, y));
}

// Plan: one warp per (variant, view, dirty tile) work item, grid-strided.
// Decodes the tile, finds the removal and insertion positions with warp
// searches, and drops the tile when none of its pixels is active (Delta = 0
// there); the rest are appended to the plan.
// counts[1]: plan items (tiles), zeroed by the injector.
template <bool COUNT>
__global__ __launch_bounds__(256) void k_plan(const ViewPtrs* __restrict__ views, const DirtyDesc* __restrict__ desc,
                                             const uint32_t* __restrict__ item_off, int BK, int K,
                                             PlanItem* __restrict__ plan, unsigned int* __restrict__ counts,
                                             unsigned long long* work) {
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t total = item_off[BK];
    unsigned int skipped = 0;
    for (uint32_t item = warp; item < total; item += nwarps) {
        // (variant, view) of this item: last bk with item_off[bk] <= item
        int lo = 0, hi = BK - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (item_off[mid] <= item) lo = mid; else hi = mid - 1;
        }
        const int bk = lo;
        const DirtyDesc& d = desc[bk];
        const uint32_t j = item - item_off[bk];
        int tx = 0, ty = 0;
        const uint32_t wn = (uint32_t)d.nx1 - d.nx0;
        const uint32_t an = d.new_vis ? wn * ((uint32_t)d.ny1 - d.ny0) : 0u;
        if (j < an) {
            tx = d.nx0 + (int)(j % wn);
            ty = d.ny0 + (int)(j / wn);
        } else {
            // tiles of the clean rect that are not in the corrupted rect, row-major
            uint32_t r = j - an;
            for (int y = d.oy0; y < d.oy1; y++) {
                int ex0 = d.ox0, ex1 = d.ox0;   // excluded x range of this row
                if (d.new_vis && y >= d.ny0 && y < d.ny1) {
                    ex0 = max((int)d.ox0, (int)d.nx0);
                    ex1 = min((int)d.ox1, (int)d.nx1);
                    if (ex1 < ex0) ex1 = ex0;
                }
                const uint32_t left = (uint32_t)(ex0 - d.ox0);
                const uint32_t row = (uint32_t)(d.ox1 - d.ox0) - (uint32_t)(ex1 - ex0);
                if (r < row) {
                    ty = y;
                    tx = r < left ? d.ox0 + (int)r : ex1 + (int)(r - left);
                    break;
                }
                r -= row;
            }
        }
        const ViewPtrs v = views[bk % K];
        const int tile = ty * v.tiles_x + tx;
        const bool has_old = d.old_vis && tx >= d.ox0 && tx < d.ox1 && ty >= d.oy0 && ty < d.oy1;
        const bool has_new = d.new_vis && tx >= d.nx0 && tx < d.nx1 && ty >= d.ny0 && ty < d.ny1;
        BlendRec orec = d.rec;
        if (has_old) orec = v.recs[d.prim];
        // first without the list positions: is any pixel reached by the old or the new record?
        unsigned reach[kBT / 32];
        bool any = false;
        {
            const float rx0 = (float)(tx * kTile) + 0.5f, ry0 = (float)(ty * kTile) + 0.5f;
            const float rx1 = fminf((float)(tx * kTile + kTile - 1), (float)(v.W - 1)) + 0.5f;
            const float ry1 = fminf((float)(ty * kTile + kTile - 1), (float)(v.H - 1)) + 0.5f;
            const bool near_old = has_old && tile_reachable(orec, rx0, rx1, ry0, ry1);
            const bool near_new = has_new && tile_reachable(d.rec, rx0, rx1, ry0, ry1);
            if (!near_old && !near_new) {
                skipped++;
                continue;
            }
        }
#pragma unroll
        for (int c = 0; c < kBT / 32; c++) {
            int px, py;
            pix_of(tx, ty, c * 32 + lane, px, py);
            const float x = (float)px + 0.5f, y = (float)py + 0.5f;
            const bool r = px < v.W && py < v.H &&
                           ((has_old && affects(orec, x, y)) || (has_new && affects(d.rec, x, y)));
            reach[c] = __ballot_sync(0xffffffffu, r);
            any |= reach[c] != 0u;
        }
        uint32_t pp = 0, ins = 0, cut = 0xffffffffu;
        uint2 rg = make_uint2(0u, 0u);
        if (any) {
            rg = v.ranges[tile];
            if (has_old) {
                pp = warp_lower_bound(v.dk, v.ids, rg.x, rg.y, __float_as_uint(orec.depth), d.prim) - rg.x;
                cut = pp;
            }
            if (has_new) {
                ins = warp_lower_bound(v.dk, v.ids, rg.x, rg.y, __float_as_uint(d.rec.depth), d.prim) - rg.x;
                cut = min(cut, ins);   // clean-list position of the insertion
                if (has_old && pp < ins) ins -= 1;
            }
            // then the reached pixels whose clean blend had not stopped before the change
            any = false;
            if (v.tile_stop[tile] >= cut) {
#pragma unroll
                for (int c = 0; c < kBT / 32; c++) {
                    int px, py;
                    pix_of(tx, ty, c * 32 + lane, px, py);
                    bool a = false;
                    if ((reach[c] >> lane) & 1u) a = v.stop[(size_t)py * v.W + px] >= cut;
                    reach[c] = __ballot_sync(0xffffffffu, a);   // now: active pixels
                    any |= reach[c] != 0u;
                }
            }
        }
        if (!any) {   // every pixel keeps its clean value
            skipped++;
            continue;
        }
        if (lane == 0) {
            PlanItem it;
            it.rec = d.rec;
            it.orec = orec;
#pragma unroll
            for (int c = 0; c < kBT / 32; c++) it.mask[c] = reach[c];
            it.bk = (uint32_t)bk;
            it.tile = (uint32_t)tile;
            it.s = rg.x;
            it.e = rg.y;
            it.pp = pp;
            it.ins = ins;
            it.cut = cut;
            it.flags = (has_old ? 1u : 0u) | (has_new ? 2u : 0u);
            plan[atomicAdd(&counts[1], 1u)] = it;
        }
    }
    if (COUNT && lane == 0 && skipped) atomicAdd(&work[3], (unsigned long long)skipped);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void fetch_plan_async(PlanItem* dst, const PlanItem* src) {
#pragma unroll
    for (int i = 0; i < (int)(sizeof(PlanItem) / 16); i++)
        cp_async16(reinterpret_cast<char*>(dst) + 16 * i, reinterpret_cast<const char*>(src) + 16 * i);
    cp_async_commit();
}

// Dirty-tile blend: persistent; each block takes plan items from a queue.  The
// next item is copied into the other half of a shared double buffer
// (cp.async) while the current one is blended.  A tile is re-blended from the
// clean list with the old entry removed and the corrupted record merged in,
// and compared on the fly with the clean tile.
template <bool COUNT>
__global__ __launch_bounds__(kBT, 5) void k_dirty(const ViewPtrs* __restrict__ views, int K,
                                                 const PlanItem* __restrict__ plan,
                                                 const unsigned int* __restrict__ counts,
                                                 CmpAcc* __restrict__ acc, unsigned int* __restrict__ queue,
                                                 unsigned long long* work) {
    __shared__ Stage s;
    __shared__ PlanItem pbuf[2];
    __shared__ int sh_ok;
    __shared__ uint32_t s_wcnt[kBT / 32];
    __shared__ uint16_t s_pix[kBT];
    __shared__ float3 s_out[kBT];
    const uint32_t total = counts[1];
    bool have = false;   // thread 0: pbuf[cur] holds (or is receiving) an item
    int cur = 0;
    if (threadIdx.x == 0) {
        const uint32_t i0 = atomicAdd(&queue[0], 1u);
        have = i0 < total;
        if (have) fetch_plan_async(&pbuf[0], &plan[i0]);
    }
    while (true) {
        if (threadIdx.x == 0) {
            cp_async_wait_all();
            sh_ok = have;
            if (have) {
                const uint32_t i1 = atomicAdd(&queue[0], 1u);
                have = i1 < total;
                if (have) fetch_plan_async(&pbuf[cur ^ 1], &plan[i1]);
            }
        }
        __syncthreads();
        if (!sh_ok) break;
        const PlanItem& it = pbuf[cur];
        const int bk = (int)it.bk;
        const ViewPtrs v = views[bk % K];
        const int tx = (int)(it.tile % (uint32_t)v.tiles_x), ty = (int)(it.tile / (uint32_t)v.tiles_x);
        const PixGeo g = pix_geo(tx, ty, v.W, v.H);   // this thread's natural pixel
        const uint32_t s0 = it.s, pp = it.pp, ins = it.ins, cut = it.cut;
        const bool has_old = it.flags & 1u, has_new = it.flags & 2u;
        const uint32_t L = (it.e - it.s) - (has_old ? 1u : 0u) + (has_new ? 1u : 0u);
        const size_t npx = g.inside ? (size_t)g.py * v.W + g.px : 0;
        const bool active = (it.mask[threadIdx.x >> 5] >> (threadIdx.x & 31)) & 1u;   // decided by the plan
        // compact the active pixels into the first threads (in natural order)
        const unsigned am = __ballot_sync(0xffffffffu, active);
        if ((threadIdx.x & 31) == 0) s_wcnt[threadIdx.x >> 5] = __popc(am);
        __syncthreads();
        uint32_t before = 0, n_active = 0;
#pragma unroll
        for (int w = 0; w < kBT / 32; w++) {
            const uint32_t c = s_wcnt[w];
            if (w < (int)(threadIdx.x >> 5)) before += c;
            n_active += c;
        }
        if (active) s_pix[before + __popc(am & ((1u << (threadIdx.x & 31)) - 1u))] = (uint16_t)threadIdx.x;
        __syncthreads();
        // thread t blends the t-th active pixel; its warp culls against the bounding
        // box of the warp's active pixels
        PixGeo ga;
        const bool mine = threadIdx.x < n_active;
        int ax = 0x7fffffff, ay = 0x7fffffff, bx = -1, by = -1;
        uint32_t u = 0;
        if (mine) {
            u = s_pix[threadIdx.x];
            pix_of(tx, ty, (int)u, ga.px, ga.py);
            ax = bx = ga.px;
            ay = by = ga.py;
        }
        ga.pxc = (float)ga.px + 0.5f;
        ga.pyc = (float)ga.py + 0.5f;
        ga.wx0 = (float)__reduce_min_sync(0xffffffffu, ax) + 0.5f;
        ga.wx1 = (float)__reduce_max_sync(0xffffffffu, bx) + 0.5f;
        ga.wy0 = (float)__reduce_min_sync(0xffffffffu, ay) + 0.5f;
        ga.wy1 = (float)__reduce_max_sync(0xffffffffu, by) + 0.5f;
        ga.inside = mine;
        Pix p{1.0f, 0.0f, 0.0f, 0.0f, !mine, 0u};
        // The merged list equals the clean list before `cut`, so an active pixel
        // (not stopped before `cut`) can resume from the clean blend's state at the
        // last checkpoint at or before `cut`.
        const uint32_t cstar = min(cut / (uint32_t)kCkStride, v.ck_cnt[it.tile]);
        const uint32_t start = cstar * (uint32_t)kCkStride;
        if (mine && cstar > 0) {
            const float4 st = v.ck[(size_t)(v.ck_off[it.tile] + cstar - 1) * kBT + u];
            p.T = st.x;
            p.c0 = st.y;
            p.c1 = st.z;
            p.c2 = st.w;
        }
        unsigned int nev = 0, staged = 0;
        for (uint32_t base = start; base < L && n_active > 0; base += kBT) {
            int cnt = (int)min((uint32_t)kBT, L - base);
            if ((int)threadIdx.x < cnt) {
                uint32_t m = base + threadIdx.x;
                if (has_new && m == ins) {
                    stage_put(s, threadIdx.x, it.rec);
                } else {
                    uint32_t j = (has_new && m > ins) ? m - 1 : m;
                    uint32_t ci = (has_old && j >= pp) ? j + 1 : j;
                    stage_put(s, threadIdx.x, load_rec(v.recs, v.ids[s0 + ci]));
                }
            }
            __syncthreads();
            staged += cnt;
            blend_batch<COUNT, false>(s, cnt, base, ga, p, nev);
            if (__syncthreads_count(p.done) == kBT) break;
        }
        if (COUNT) add_work(work, nev, staged);
        if (mine) s_out[u] = make_float3(__fadd_rn(p.c0, p.T), __fadd_rn(p.c1, p.T), __fadd_rn(p.c2, p.T));
        __syncthreads();
        // back in natural order: only the active pixels are compared; every other
        // pixel keeps its clean value (Delta = 0), and the clean image's non-finite
        // pixels are counted once per view at finalize
        float v0 = 0.0f, v1 = 0.0f, v2 = 0.0f;
        if (active) {
            const float3 o = s_out[threadIdx.x];
            v0 = o.x;
            v1 = o.y;
            v2 = o.z;
        }
        PixGeo gc = g;
        gc.inside = active;
        compare_tile(gc, v0, v1, v2, v.clean, v.W, &acc[bk]);
        // re-blended pixels whose clean value was non-finite (their clean count is withdrawn at finalize)
        const bool clean_bad = active && !(isfinite(v.clean[npx * 3]) && isfinite(v.clean[npx * 3 + 1]) &&
                                           isfinite(v.clean[npx * 3 + 2]));
        const int ncb = __syncthreads_count(clean_bad);
        if (threadIdx.x == 0 && ncb) atomicAdd(&acc[bk].clean_nonfinite_replaced, (unsigned)ncb);
        __syncthreads();
        cur ^= 1;
    }
}

__global__ void k_records_to_blend(const gs_record* in, uint64_t n, BlendRec* out) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    gs_record r = in[i];
    BlendRec q;
    q.mx = r.mx;
    q.my = r.my;
    q.ca = r.ca;
    q.cb = r.cb;
    q.cc = r.cc;
    q.opac = r.opac;
    q.r = r.r;
    q.g = r.g;
    q.b = r.b;
    q.depth = r.depth;
    // records from outside carry no alpha box: never cull
    q.ex = NAN;
    q.ey = NAN;
    out[i] = q;
}

__global__ void k_gather_depth(const BlendRec* recs, const uint32_t* ids, uint64_t n, uint32_t* dk) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dk[i] = __float_as_uint(recs[ids[i]].depth);
}

__global__ void k_offsets_to_ranges(const uint32_t* offsets, int ntiles, uint2* ranges) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ntiles) ranges[t] = make_uint2(offsets[t], offsets[t + 1]);
}

}  // namespace

gs_status launch_blend_image(const BlendRec* recs, const uint32_t* ids, const uint2* ranges, int W, int H, float* img,
                             cudaStream_t st) {
    int tx = (W + kTile - 1) / kTile, ty = (H + kTile - 1) / kTile;
    if (tx * ty == 0) return GS_OK;
    k_blend_full<0, false><<<tx * ty, kBT, 0, st>>>(recs, ids, ranges, W, H, tx, img, nullptr, nullptr, nullptr,
                                                     nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status launch_blend_compare(const BlendRec* recs, const uint32_t* ids, const uint2* ranges, int W, int H,
                               const float* clean, CmpAcc* acc, unsigned long long* work, cudaStream_t st) {
    int tx = (W + kTile - 1) / kTile, ty = (H + kTile - 1) / kTile;
    if (tx * ty == 0) return GS_OK;
    if (work)
        k_blend_full<1, true><<<tx * ty, kBT, 0, st>>>(recs, ids, ranges, W, H, tx, nullptr, clean, acc, work, nullptr,
                                                       nullptr, nullptr, nullptr, nullptr, nullptr);
    else
        k_blend_full<1, false><<<tx * ty, kBT, 0, st>>>(recs, ids, ranges, W, H, tx, nullptr, clean, acc, nullptr,
                                                        nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status launch_blend_image_stop(const BlendRec* recs, const uint32_t* ids, const uint2* ranges, int W, int H,
                                  float* img, uint32_t* stop, uint32_t* tile_stop, float4* ck, const uint32_t* ck_off,
                                  const uint32_t* ck_cnt, unsigned int* clean_nonfin, cudaStream_t st) {
    int tx = (W + kTile - 1) / kTile, ty = (H + kTile - 1) / kTile;
    if (tx * ty == 0) return GS_OK;
    k_blend_full<2, false><<<tx * ty, kBT, 0, st>>>(recs, ids, ranges, W, H, tx, img, nullptr, nullptr, nullptr, stop,
                                                     tile_stop, ck, ck_off, ck_cnt, clean_nonfin);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status launch_compare(const float* a, const float* b, int H, int W, CmpAcc* acc, cudaStream_t st) {
    int tx = (W + kTile - 1) / kTile, ty = (H + kTile - 1) / kTile;
    if (tx * ty == 0) return GS_OK;
    k_compare<<<tx * ty, kBT, 0, st>>>(a, b, W, H, tx, acc);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status launch_zero_acc(CmpAcc* acc, int count, cudaStream_t st) {
    if (count <= 0) return GS_OK;
    k_zero_acc<<<(count + 255) / 256, 256, 0, st>>>(acc, count);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status launch_finalize(const CmpAcc* acc, int count, gs_result* out, cudaStream_t st) {
    if (count <= 0) return GS_OK;
    k_finalize<<<(count + 255) / 256, 256, 0, st>>>(acc, count, out, nullptr, 1);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status launch_finalize_dirty(const CmpAcc* acc, int count, gs_result* out, const unsigned int* clean_nonfin, int K,
                                cudaStream_t st) {
    if (count <= 0) return GS_OK;
    k_finalize<<<(count + 255) / 256, 256, 0, st>>>(acc, count, out, clean_nonfin, K);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

int dirty_grid() {
    static int blocks = 0;
    if (!blocks) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dirty<false>, kBT, 0);
        if (per_sm < 1) per_sm = 1;
        blocks = per_sm * num_sms();
    }
    return blocks;
}

size_t plan_item_size() { return sizeof(PlanItem); }

// queue[0]: blend work queue, queue[1]: plan items (both zeroed by the injector)
gs_status launch_dirty_blend(const void* dev_views, const DirtyDesc* desc, const uint32_t* item_off, int BK, int K,
                             void* plan, CmpAcc* acc, unsigned int* queue, unsigned long long* work, cudaStream_t st) {
    const ViewPtrs* views = (const ViewPtrs*)dev_views;
    PlanItem* pl = (PlanItem*)plan;
    const int plan_blocks = num_sms() * 8;
    if (work) {
        k_plan<true><<<plan_blocks, 256, 0, st>>>(views, desc, item_off, BK, K, pl, queue, work);
        k_dirty<true><<<dirty_grid(), kBT, 0, st>>>(views, K, pl, queue, acc, queue, work);
    } else {
        k_plan<false><<<plan_blocks, 256, 0, st>>>(views, desc, item_off, BK, K, pl, queue, nullptr);
        k_dirty<false><<<dirty_grid(), kBT, 0, st>>>(views, K, pl, queue, acc, queue, nullptr);
    }
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

size_t view_ptrs_size() { return sizeof(ViewPtrs); }

gs_status launch_gather_depth(const BlendRec* recs, const uint32_t* ids, uint64_t n, uint32_t* dk, cudaStream_t st) {
    if (n == 0) return GS_OK;
    k_gather_depth<<<(unsigned)div_up(n, 256), 256, 0, st>>>(recs, ids, n, dk);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

int ck_stride_value() { return kCkStride; }
int ck_max_per_tile() { return kCkMaxPerTile; }

void fill_view_ptrs(void* host_dst, const BlendRec* recs, const uint32_t* ids, const uint32_t* dk, const uint2* ranges,
                    const float* clean, const uint32_t* stop, const uint32_t* tile_stop, const float4* ck,
                    const uint32_t* ck_off, const uint32_t* ck_cnt, int W, int H) {
    ViewPtrs v;
    v.recs = recs;
    v.ids = ids;
    v.dk = dk;
    v.ranges = ranges;
    v.clean = clean;
    v.stop = stop;
    v.tile_stop = tile_stop;
    v.ck = ck;
    v.ck_off = ck_off;
    v.ck_cnt = ck_cnt;
    v.W = W;
    v.H = H;
    v.tiles_x = (W + kTile - 1) / kTile;
    v.pad = 0;
    memcpy(host_dst, &v, sizeof(v));
}

gs_status launch_records_to_blend(const gs_record* in, uint64_t n, BlendRec* out, cudaStream_t st) {
    if (n == 0) return GS_OK;
    k_records_to_blend<<<(unsigned)div_up(n, 256), 256, 0, st>>>(in, n, out);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status launch_offsets_to_ranges(const uint32_t* offsets, int ntiles, uint2* ranges, cudaStream_t st) {
    if (ntiles <= 0) return GS_OK;
    k_offsets_to_ranges<<<(ntiles + 255) / 256, 256, 0, st>>>(offsets, ntiles, ranges);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free comparison.  The per-image accumulators live in one fixed
// device array instead of memory obtained at call time, for callers that may
// not allocate (see gs_compare_noalloc in gs.h).  Every GPU that loads this
// library holds the array until the process exits.
// ---------------------------------------------------------------------------
constexpr int kNoAllocMaxImages = 64;
constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) CmpAcc g_noalloc_acc[kNoAllocMaxImages];

namespace {
std::mutex g_noalloc_mu;
CmpAcc* g_noalloc_ptr[kNoAllocMaxDevices] = {};   // device address of the array, per device
}  // namespace

// Once per device, with that device current: the array's device address.  In
// host code the array's name is only a host-side stand-in, so kernels are given
// this address, never the name.
static gs_status noalloc_scratch(CmpAcc** out) {
    int dev = 0;
    GS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return set_error(GS_ERR_ARG, "device index out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_acc);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(no-alloc comparison scratch)");
        g_noalloc_ptr[dev] = (CmpAcc*)p;
    }
    *out = g_noalloc_ptr[dev];
    return GS_OK;
}

}  // namespace gs

extern "C" gs_status gs_compare_noalloc(const float* dev_a, const float* dev_b, int H, int W, int K,
                                        gs_result* dev_out, void* stream) {
    using namespace gs;
    if (!dev_a || !dev_b || !dev_out || H < 1 || W < 1 || K < 1)
        return set_error(GS_ERR_ARG, "bad gs_compare_noalloc arguments");
    if (K > kNoAllocMaxImages)
        return set_error(GS_ERR_ARG, "gs_compare_noalloc: at most 64 image pairs per call (fixed scratch size)");
    CmpAcc* acc = nullptr;
    GS_TRY(noalloc_scratch(&acc));
    cudaStream_t st = (cudaStream_t)stream;
    // the array keeps the previous call's sums: clear the K accumulators first
    GS_TRY(launch_zero_acc(acc, K, st));
    const size_t img = (size_t)H * W * 3;
    for (int k = 0; k < K; k++) GS_TRY(launch_compare(dev_a + k * img, dev_b + k * img, H, W, acc + k, st));
    return launch_finalize(acc, K, dev_out, st);
}
