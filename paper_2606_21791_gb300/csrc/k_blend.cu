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

// Pixel geometry of thread `tid` in a tw x th tile: warp w covers the 8x4 block w
// of the natural order.
struct PixGeo {
    int px, py;
    float pxc, pyc;
    float wx0, wx1, wy0, wy1;   // pixel-centre bounds of the warp's block
    bool inside;
};

__device__ __forceinline__ PixGeo pix_geo(int tile_x, int tile_y, int tw, int th, int W, int H) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lg = tile_lgx(tw);
    PixGeo g;
    int bx = tile_x * tw + (warp & ((1 << lg) - 1)) * 8;
    int by = tile_y * th + (warp >> lg) * 4;
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

// Natural pixel of index u in a tw x th tile (the pix_geo mapping).
__device__ __forceinline__ void pix_of(int tile_x, int tile_y, int tw, int th, int u, int& px, int& py) {
    const int w = u >> 5, l = u & 31, lg = tile_lgx(tw);
    px = tile_x * tw + (w & ((1 << lg) - 1)) * 8 + (l & 7);
    py = tile_y * th + (w >> lg) * 4 + (l >> 3);
}

// 8x8 block b of a tile with 8x4 blocks per row nbx = 1 << lg: its upper 8x4
// block in the natural order (the lower one is that + nbx) and its offset in the tile.
__host__ __device__ inline int block_upper(int b, int lg) { return (b & ((1 << lg) - 1)) + ((b >> lg) << (lg + 1)); }
__host__ __device__ inline int block_x0(int b, int lg) { return (b & ((1 << lg) - 1)) * 8; }
__host__ __device__ inline int block_y0(int b, int lg) { return (b >> lg) * 8; }

// 2^x (hardware approximation, flushes subnormal results to zero)
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Exponent of the Gaussian at offset (dx, dy): -(ca dx^2 + cc dy^2)/2 - cb dx dy,
// evaluated as s = fma(cc dy, dy, ca dx dx), power = fma(-cb dx, dy, -s/2): each
// product rounded on its own, each sum fused with its product (one rounding).
// Every evaluation here (and the oracle's) takes this order, so it is
// reproducible bit for bit -- which matters for near-degenerate conics, where
// cancellation makes the rounding error large compared with the value.  No
// product feeds a separate addition, so the packed two-pixel form in the walk
// (fp32x2 operations) computes the same bits as this scalar one.
__device__ __forceinline__ float gauss_power(float ca, float cb, float cc, float dx, float dy) {
    const float t1 = __fmul_rn(__fmul_rn(ca, dx), dx);
    const float s = __fmaf_rn(__fmul_rn(cc, dy), dy, t1);
    return __fmaf_rn(__fmul_rn(-cb, dx), dy, __fmul_rn(-0.5f, s));
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
    uint32_t pix;    // pixels of a tile (one checkpoint holds one state per pixel)
};

// Survivors a warp takes at a time: their alphas do not depend on the pixel
// state, so they are computed as independent chains, then applied in list order.
// The front-to-back step of one entry at one pixel (alpha capped at 0.99, NaN
// kept; stop when T would drop below 1e-4; C += colour * alpha * T) has explicit
// rounding in every operation, so the full-frame, clean and dirty-tile kernels
// compute the same bits wherever it is inlined.
constexpr int kAlphaGroup = 4;

// A staged entry as the walk needs it.
struct EntryQ {
    float4 q0;          // mx, my, ca, cb
    float cc, opac, r, g, b;
};

// One front-to-back step of an entry at one pixel, alpha already computed (ok:
// the blend takes the entry there; live: the pixel has not stopped): alpha
// capped at 0.99 (NaN kept), stop when T would drop below 1e-4, else
// C += colour * alpha * T.  Every operation is rounded on its own, so each
// kernel that inlines it computes the same bits.  Returns whether the pixel
// stopped at this entry.  (Packing the two pixels' steps into fp32x2
// operations computes the same bits but costs more than it saves: the state
// has to be packed and the updates selected per pixel.)
__device__ __forceinline__ bool apply_entry(Pix& p, bool live, bool ok, float a, float cr, float cg, float cb) {
    const bool act = live && ok;
    const float al = a > 0.99f ? 0.99f : a;   // keeps NaN
    const float Tn = __fmul_rn(p.T, __fsub_rn(1.0f, al));
    const bool stop_here = act && Tn < 1e-4f;
    const bool upd = act && !(Tn < 1e-4f);
    const float w = __fmul_rn(al, p.T);
    p.c0 = upd ? __fmaf_rn(cr, w, p.c0) : p.c0;
    p.c1 = upd ? __fmaf_rn(cg, w, p.c1) : p.c1;
    p.c2 = upd ? __fmaf_rn(cb, w, p.c2) : p.c2;
    p.T = upd ? Tn : p.T;
    p.done = p.done || stop_here;
    return stop_here;
}

// Walk the survivors m (bit i: entry c + i) in list order for this lane's two
// pixels, which share a column (centres (pxc, pyA) and (pxc, pyB)): the x
// offset and the exponent's terms that depend on it alone (ca dx dx, -cb dx) are
// computed once for both, the rest of gauss_power's order as packed fp32x2
// operations over the two pixels, so every pixel gets the bits of a one-pixel
// evaluation of the same entries.
// TRACK: record, per pixel, the list index (base + entry) where it stopped.
// steps (measurement builds only): [0] entries walked by the warp, [1] of them
// blended by at least one lane.
template <bool COUNT, bool TRACK, class Fetch>
__device__ __forceinline__ void walk_survivors2(unsigned m, int c, const Fetch& fetch, float pxc, float pyA,
                                                float pyB, Pix& pA, Pix& pB, unsigned int& nev, uint32_t base,
                                                unsigned* steps) {
    if (COUNT && steps) steps[0] += __popc(m);
    const float2 npy = make_float2(-pyA, -pyB);
    while (m) {
        int e[kAlphaGroup];
        bool v[kAlphaGroup], okA[kAlphaGroup], okB[kAlphaGroup];
        float aA[kAlphaGroup], aB[kAlphaGroup], cr[kAlphaGroup], cg[kAlphaGroup], cb[kAlphaGroup];
#pragma unroll
        for (int k = 0; k < kAlphaGroup; k++) {
            v[k] = m != 0u;
            e[k] = v[k] ? c + __ffs(m) - 1 : c;
            m &= m - 1u;
        }
#pragma unroll
        for (int k = 0; k < kAlphaGroup; k++) {
            const EntryQ q = fetch(e[k]);
            const float dx = __fsub_rn(q.q0.x, pxc);
            const float t1 = __fmul_rn(__fmul_rn(q.q0.z, dx), dx);
            const float bdxn = __fmul_rn(-q.q0.w, dx);
            const float2 dy = __fadd2_rn(make_float2(q.q0.y, q.q0.y), npy);   // my - py, one rounding each
            const float2 sq = __ffma2_rn(__fmul2_rn(make_float2(q.cc, q.cc), dy), dy, make_float2(t1, t1));
            const float2 pw = __ffma2_rn(make_float2(bdxn, bdxn), dy, __fmul2_rn(make_float2(-0.5f, -0.5f), sq));
            const float2 pl = __fmul2_rn(pw, make_float2(kLog2e, kLog2e));
            const float2 a = __fmul2_rn(make_float2(q.opac, q.opac), make_float2(ex2_approx(pl.x), ex2_approx(pl.y)));
            aA[k] = a.x;
            aB[k] = a.y;
            okA[k] = !(pw.x > 0.0f) && !(a.x < 1.0f / 255.0f);
            okB[k] = !(pw.y > 0.0f) && !(a.y < 1.0f / 255.0f);
            cr[k] = q.r;
            cg[k] = q.g;
            cb[k] = q.b;
        }
        // apply in list order with selects (no divergent branch per entry)
#pragma unroll
        for (int k = 0; k < kAlphaGroup; k++) {
            const bool liveA = v[k] && !pA.done, liveB = v[k] && !pB.done;
            if (COUNT) {
                nev += (liveA ? 1u : 0u) + (liveB ? 1u : 0u);
                if (steps) steps[1] += __any_sync(0xffffffffu, (liveA && okA[k]) || (liveB && okB[k])) ? 1u : 0u;
            }
            const bool sA = apply_entry(pA, liveA, okA[k], aA[k], cr[k], cg[k], cb[k]);
            const bool sB = apply_entry(pB, liveB, okB[k], aB[k], cr[k], cg[k], cb[k]);
            if (TRACK) {
                pA.stop = sA ? base + (uint32_t)e[k] : pA.stop;
                pB.stop = sB ? base + (uint32_t)e[k] : pB.stop;
            }
        }
    }
}

// The two pixels of a lane in a full-frame tile: 8x8 block b = warp of the
// tile, pixel A at (lane % 8, lane / 8) of the block, B four rows below; u0 and
// u1 are their indices in the tile's natural (8x4 block) order.
struct Pix2Geo {
    int px, pyA, pyB, u0, u1;
    float pxc, pycA, pycB;
    float wx0, wx1, wy0, wy1;   // pixel-centre box of the 8x8 block
    bool inA, inB;
};

__device__ __forceinline__ Pix2Geo pix2_geo(int tile_x, int tile_y, int tw, int th, int W, int H) {
    const int lane = threadIdx.x & 31, b = threadIdx.x >> 5, lg = tile_lgx(tw);
    Pix2Geo g;
    const int bx = tile_x * tw + block_x0(b, lg), by = tile_y * th + block_y0(b, lg);
    g.px = bx + (lane & 7);
    g.pyA = by + (lane >> 3);
    g.pyB = g.pyA + 4;
    g.u0 = block_upper(b, lg) * 32 + lane;
    g.u1 = g.u0 + (32 << lg);
    g.pxc = (float)g.px + 0.5f;
    g.pycA = (float)g.pyA + 0.5f;
    g.pycB = (float)g.pyB + 0.5f;
    g.wx0 = (float)bx + 0.5f;
    g.wx1 = (float)bx + 7.5f;
    g.wy0 = (float)by + 0.5f;
    g.wy1 = (float)by + 7.5f;
    g.inA = g.px < W && g.pyA < H;
    g.inB = g.px < W && g.pyB < H;
    return g;
}

// Entries [c, c + 32) of a staged batch for one warp: cull 32 boxes against the
// warp's 8x8 pixel block with one ballot, then walk the survivors in list order.
template <bool COUNT, bool TRACK>
__device__ __forceinline__ void blend_chunk2(const Stage& s, int c, int cnt, uint32_t base, const Pix2Geo& g, Pix& pA,
                                             Pix& pB, unsigned int& nev) {
    const int lane = threadIdx.x & 31;
    const int j = c + lane;
    bool pass = false;
    if (j < cnt) {
        const float4 bx = s.box[j];
        pass = !(bx.y < g.wx0 || bx.x > g.wx1 || bx.w < g.wy0 || bx.z > g.wy1);
    }
    const unsigned m = __ballot_sync(0xffffffffu, pass);
    auto fetch = [&](int e) {
        const float4 q1 = s.q1[e];
        return EntryQ{s.q0[e], q1.x, q1.y, q1.z, q1.w, s.qb[e]};
    };
    walk_survivors2<COUNT, TRACK>(m, c, fetch, g.pxc, g.pycA, g.pycB, pA, pB, nev, base, nullptr);
}

template <bool COUNT, bool TRACK>
__device__ __forceinline__ void blend_batch2(const Stage& s, int cnt, uint32_t base, const Pix2Geo& g, Pix& pA,
                                             Pix& pB, unsigned int& nev, const CkWrite& ckw) {
    for (int c = 0; c < cnt; c += 32) {
        if (__all_sync(0xffffffffu, pA.done && pB.done)) return;
        if (ckw.ck && base + (uint32_t)c > 0 && ((base + (uint32_t)c) % kCkStride) == 0) {
            // the state after entries [0, base + c) of the list
            const uint32_t j = (base + (uint32_t)c) / kCkStride;
            if (j <= ckw.count) {
                float4* row = ckw.ck + (size_t)(ckw.off + j - 1) * ckw.pix;
                row[g.u0] = make_float4(pA.T, pA.c0, pA.c1, pA.c2);
                row[g.u1] = make_float4(pB.T, pB.c0, pB.c1, pB.c2);
            }
        }
        blend_chunk2<COUNT, TRACK>(s, c, cnt, base, g, pA, pB, nev);
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
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
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

// Both pixels of a lane against the clean image, added to *acc for the block
// (fixed-point squared errors: the sum does not depend on the order).
__device__ __forceinline__ void compare_tile2(const Pix2Geo& g, float a0, float a1, float a2, float b0, float b1,
                                              float b2, const float* clean, int W, CmpAcc* acc) {
    __shared__ unsigned long long wsse[kBT / 32];
    __shared__ float wmax[kBT / 32];
    __shared__ unsigned wfoot[kBT / 32], wbad[kBT / 32];
    PixCmp rA{0ull, 0.0f, false, false}, rB{0ull, 0.0f, false, false};
    if (g.inA) rA = pixel_compare(a0, a1, a2, clean + ((size_t)g.pyA * W + g.px) * 3);
    if (g.inB) rB = pixel_compare(b0, b1, b2, clean + ((size_t)g.pyB * W + g.px) * 3);
    unsigned long long fx = rA.fx + rB.fx;
    float m = fmaxf(rA.m, rB.m);
    for (int o = 16; o > 0; o >>= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    const unsigned nf = __reduce_add_sync(0xffffffffu, (rA.foot ? 1u : 0u) + (rB.foot ? 1u : 0u));
    const unsigned nb = __reduce_add_sync(0xffffffffu, (rA.nonfin ? 1u : 0u) + (rB.nonfin ? 1u : 0u));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        wsse[warp] = fx;
        wmax[warp] = m;
        wfoot[warp] = nf;
        wbad[warp] = nb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        float mm = 0.0f;
        unsigned nfoot = 0, nbad = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            t += wsse[w];
            mm = fmaxf(mm, wmax[w]);
            nfoot += wfoot[w];
            nbad += wbad[w];
        }
        if (t) atomicAdd(&acc->sse_fx, t);
        if (mm > 0.0f) atomicMax(&acc->maxabs_bits, __float_as_uint(mm));
        if (nfoot) atomicAdd(&acc->footprint, nfoot);
        if (nbad) atomicAdd(&acc->nonfinite, nbad);
    }
}

// MODE 0: write the image; 1: compare with the clean image; 2: write the image
// and each pixel's stop index (0xffffffff if it never stopped), which the
// dirty-tile kernel uses to leave pixels that stopped before a change untouched.
// One block of tw * th / 2 threads per tw x th tile: warp b blends the tile's
// 8x8 block b, two pixels per lane (the dirty-tile kernel's walk).
template <int MODE, bool COUNT>
__global__ __launch_bounds__(kBT / 2) void k_blend_full(const BlendRec* __restrict__ recs,
                                                       const uint32_t* __restrict__ ids,
                                                       const uint2* __restrict__ ranges, int W, int H, int tiles_x,
                                                       int tw, int th, float* __restrict__ img,
                                                       const float* __restrict__ clean, CmpAcc* acc,
                                                       unsigned long long* work, uint32_t* __restrict__ stop,
                                                       uint32_t* __restrict__ tile_stop, float4* __restrict__ ck,
                                                       const uint32_t* __restrict__ ck_off,
                                                       const uint32_t* __restrict__ ck_cnt,
                                                       unsigned int* __restrict__ clean_nonfin) {
    __shared__ Stage s;
    const int tile = blockIdx.x;
    const uint32_t P = (uint32_t)(tw * th);   // pixels of a tile = records staged per batch
    const CkWrite ckw{ck, ck ? ck_off[tile] : 0u, ck ? ck_cnt[tile] : 0u, P};
    const Pix2Geo g = pix2_geo(tile % tiles_x, tile / tiles_x, tw, th, W, H);
    Pix pA{1.0f, 0.0f, 0.0f, 0.0f, !g.inA, 0xffffffffu}, pB{1.0f, 0.0f, 0.0f, 0.0f, !g.inB, 0xffffffffu};
    const uint2 rg = ranges[tile];
    unsigned int nev = 0, staged = 0;
    for (uint32_t base = rg.x; base < rg.y; base += P) {
        const int cnt = (int)min(P, rg.y - base);
        for (int j = threadIdx.x; j < cnt; j += blockDim.x) stage_put(s, j, load_rec(recs, ids[base + j]));
        __syncthreads();
        staged += cnt;
        blend_batch2<COUNT, MODE == 2>(s, cnt, base - rg.x, g, pA, pB, nev, ckw);
        // also the barrier that lets the next batch overwrite the stage
        if (__syncthreads_count(pA.done && pB.done) == (int)blockDim.x) break;
    }
    if (COUNT) add_work(work, nev, staged);
    const float a0 = __fadd_rn(pA.c0, pA.T), a1 = __fadd_rn(pA.c1, pA.T), a2 = __fadd_rn(pA.c2, pA.T);   // over white
    const float b0 = __fadd_rn(pB.c0, pB.T), b1 = __fadd_rn(pB.c1, pB.T), b2 = __fadd_rn(pB.c2, pB.T);
    if (MODE != 1) {
        if (g.inA) {
            const size_t px = (size_t)g.pyA * W + g.px;
            img[px * 3] = a0;
            img[px * 3 + 1] = a1;
            img[px * 3 + 2] = a2;
            if (MODE == 2) stop[px] = pA.stop;
        }
        if (g.inB) {
            const size_t px = (size_t)g.pyB * W + g.px;
            img[px * 3] = b0;
            img[px * 3 + 1] = b1;
            img[px * 3 + 2] = b2;
            if (MODE == 2) stop[px] = pB.stop;
        }
        if (MODE == 2 && clean_nonfin) {
            const int bad = (g.inA && !(isfinite(a0) && isfinite(a1) && isfinite(a2)) ? 1 : 0) +
                            (g.inB && !(isfinite(b0) && isfinite(b1) && isfinite(b2)) ? 1 : 0);
            const unsigned wb = __reduce_add_sync(0xffffffffu, (unsigned)bad);
            if ((threadIdx.x & 31) == 0 && wb) atomicAdd(clean_nonfin, wb);
        }
        if (MODE == 2) {
            // the tile's largest stop index: a change at or after it leaves every pixel as it is
            __shared__ uint32_t wmax[kBT / 32];
            const uint32_t m = __reduce_max_sync(0xffffffffu, max(g.inA ? pA.stop : 0u, g.inB ? pB.stop : 0u));
            if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t t = 0;
                for (int w = 0; w < (int)(blockDim.x >> 5); w++) t = max(t, wmax[w]);
                tile_stop[tile] = t;
            }
        }
    } else {
        compare_tile2(g, a0, a1, a2, b0, b1, b2, clean, W, acc);
    }
}

__global__ __launch_bounds__(kBT) void k_compare(const float* __restrict__ a, const float* __restrict__ b, int W, int H,
                                                int tiles_x, CmpAcc* acc) {
    const int tile = blockIdx.x;
    const PixGeo g = pix_geo(tile % tiles_x, tile / tiles_x, kTile, kTile, W, H);
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
    if (i < count) acc[i] = CmpAcc{0ull, 0u, 0u, 0u, 0u, 0u, 0u, 0ull, 0ull, 0ull};
}

// ---------------------------------------------------------------------------
// dirty-tile persistent kernel
// ---------------------------------------------------------------------------


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
__device__ __forceinline__ bool rect_reachable(float mx, float my, float ca, float cb, float cc, float opac, float x0,
                                               float x1, float y0, float y1) {
    const float L = __logf(255.0f * opac) + 1e-3f;
    if (L < 0.0f) return false;   // alpha <= opacity < 1/255 everywhere (with margin); NaN falls through
    if (!(ca > 1e-30f) || !(cc > 1e-30f) || !(L < 3.0e38f)) return true;
    const float dx0 = mx - x1, dx1 = mx - x0;
    const float dy0 = my - y1, dy1 = my - y0;
    if (dx0 <= 0.0f && dx1 >= 0.0f && dy0 <= 0.0f && dy1 >= 0.0f) return true;
    const float mdx = fmaxf(dx0 * dx0, dx1 * dx1), mdy = fmaxf(dy0 * dy0, dy1 * dy1);
    const float M = 0.5f * ((ca + fabsf(cb)) * mdx + (cc + fabsf(cb)) * mdy);
    if (!(M < 1.0e37f)) return true;   // terms near overflow: the blend's power may be NaN
    auto qf = [&](float dx, float dy) { return ca * dx * dx + 2.0f * cb * dx * dy + cc * dy * dy; };
    // approximate reciprocals: they only place the nearest point of an edge, and
    // a relative error e there raises q by about e^2 M, far inside the margin
    const float rca = __fdividef(1.0f, ca), rcc = __fdividef(1.0f, cc);
    // the nearest point of each edge (dx fixed: dy = -cb dx / cc; dy fixed: dx = -cb dy / ca), clamped to it
    const float e0 = qf(dx0, fminf(fmaxf(-cb * dx0 * rcc, dy0), dy1));
    const float e1 = qf(dx1, fminf(fmaxf(-cb * dx1 * rcc, dy0), dy1));
    const float e2 = qf(fminf(fmaxf(-cb * dy0 * rca, dx0), dx1), dy0);
    const float e3 = qf(fminf(fmaxf(-cb * dy1 * rca, dx0), dx1), dy1);
    const float qmin = fminf(fminf(e0, e1), fminf(e2, e3));
    return !(qmin > 2.0f * L + 2.0e-5f * M);
}

__device__ __forceinline__ bool tile_reachable(const BlendRec& q, float x0, float x1, float y0, float y1) {
    return rect_reachable(q.mx, q.my, q.ca, q.cb, q.cc, q.opac, x0, x1, y0, y1);
}

__device__ __forceinline__ bool affects(const BlendRec& q, float x, float y) {
    float alpha;
    return blend_alpha(q.mx, q.my, q.ca, q.cb, q.cc, q.opac, x, y, alpha);
}

// (variant, view) of a work item: the last bk with off[bk] <= item.
__device__ __forceinline__ int item_owner(const uint32_t* off, int BK, uint32_t item) {
    int lo = 0, hi = BK - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Tile of the j-th dirty tile of a (variant, view): the corrupted rect row-major,
// then the tiles of the clean rect outside it, row-major.  The clean rect minus
// the corrupted one is three bands: the rows above their overlap (full width),
// the overlapping rows (minus the overlap's columns) and the rows below.
__device__ __forceinline__ void item_tile(const DirtyDesc& d, uint32_t j, int& tx, int& ty) {
    const uint32_t wn = (uint32_t)d.nx1 - d.nx0;
    const uint32_t an = d.new_vis ? wn * ((uint32_t)d.ny1 - d.ny0) : 0u;
    if (j < an) {
        tx = d.nx0 + (int)(j % wn);
        ty = d.ny0 + (int)(j / wn);
        return;
    }
    uint32_t r = j - an;
    const uint32_t w0 = (uint32_t)d.ox1 - d.ox0;
    const int lx = max((int)d.ox0, (int)d.nx0), hx = min((int)d.ox1, (int)d.nx1);
    const int ly = max((int)d.oy0, (int)d.ny0), hy = min((int)d.oy1, (int)d.ny1);
    if (d.new_vis && hx > lx && hy > ly) {
        const uint32_t above = (uint32_t)(ly - d.oy0) * w0;
        if (r >= above) {
            r -= above;
            const uint32_t wb = w0 - (uint32_t)(hx - lx), left = (uint32_t)(lx - d.ox0);
            const uint32_t band = (uint32_t)(hy - ly) * wb;
            if (r < band) {
                const uint32_t q = r % wb;
                ty = ly + (int)(r / wb);
                tx = q < left ? d.ox0 + (int)q : hx + (int)(q - left);
                return;
            }
            r -= band;
            ty = hy + (int)(r / w0);
            tx = d.ox0 + (int)(r % w0);
            return;
        }
    }
    ty = d.oy0 + (int)(r / w0);
    tx = d.ox0 + (int)(r % w0);
}

// Plan, first pass: one (variant, view, dirty tile) work item per thread.
// Decodes the tile and drops it when every pixel's clean blend stopped before
// the first changed list position (stop-key test, exact) or when neither
// changed record can reach it (conservative tile test); the others are
// appended to cand as (bk, tx | ty << 16), counted in counts[2].
template <bool COUNT>
__global__ __launch_bounds__(256) void k_plan_filter(const ViewPtrs* __restrict__ views,
                                                    const DirtyDesc* __restrict__ desc,
                                                    const uint32_t* __restrict__ item_off, int BK, int K,
                                                    uint2* __restrict__ cand, unsigned int* __restrict__ counts,
                                                    unsigned long long* work) {
    const int lane = threadIdx.x & 31;
    __shared__ uint32_t s_off[kMaxPairs + 1];   // item_off[0, BK], BK <= kMaxPairs
    for (int i = threadIdx.x; i <= BK; i += blockDim.x) s_off[i] = item_off[i];
    __syncthreads();
    const uint32_t total = s_off[BK];
    const uint32_t stride = gridDim.x * blockDim.x;
    unsigned int drop_key = 0, drop_box = 0;
    // warp-uniform trip count (the ballot below needs the whole warp)
    for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < total; base += stride) {
        const uint32_t item = base + (uint32_t)lane;
        bool keep = false;
        int bk = 0, tx = 0, ty = 0;
        if (item < total) {
            bk = item_owner(s_off, BK, item);
            const DirtyDesc& d = desc[bk];
            item_tile(d, item - s_off[bk], tx, ty);
            const ViewPtrs& v = views[bk % K];
            const int tile = ty * v.tiles_x + tx;
            const bool has_old = d.old_vis && tx >= d.ox0 && tx < d.ox1 && ty >= d.oy0 && ty < d.oy1;
            const bool has_new = d.new_vis && tx >= d.nx0 && tx < d.nx1 && ty >= d.ny0 && ty < d.ny1;
            // every pixel of the tile stopped before the first changed list position
            // (tile_stop < cut) exactly when the entry at tile_stop sorts below the
            // keys of both changed entries
            unsigned long long kmin = ~0ull;
            if (has_old) kmin = ((unsigned long long)__float_as_uint(d.old_depth) << 32) | d.prim;
            if (has_new) kmin = min(kmin, ((unsigned long long)__float_as_uint(d.rec.depth) << 32) | d.prim);
            const bool stopped = v.stop_key[tile] < kmin;
            if (!stopped) {
                const float rx0 = (float)(tx * v.tile_w) + 0.5f, ry0 = (float)(ty * v.tile_h) + 0.5f;
                const float rx1 = fminf((float)(tx * v.tile_w + v.tile_w - 1), (float)(v.W - 1)) + 0.5f;
                const float ry1 = fminf((float)(ty * v.tile_h + v.tile_h - 1), (float)(v.H - 1)) + 0.5f;
                keep = (has_new && tile_reachable(d.rec, rx0, rx1, ry0, ry1)) ||
                       (has_old && tile_reachable(v.recs[d.prim], rx0, rx1, ry0, ry1));
            }
            if (COUNT && !keep) (stopped ? drop_key : drop_box)++;
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (m) {
            uint32_t b0 = 0;
            if (lane == 0) b0 = atomicAdd(&counts[2], (unsigned)__popc(m));
            b0 = __shfl_sync(0xffffffffu, b0, 0);
            if (keep)
                cand[b0 + __popc(m & ((1u << lane) - 1u))] =
                    make_uint2((uint32_t)bk, (uint32_t)tx | ((uint32_t)ty << 16));
        }
    }
    if (COUNT) {
        const unsigned k = __reduce_add_sync(0xffffffffu, drop_key), x = __reduce_add_sync(0xffffffffu, drop_box);
        if (lane == 0 && (k + x)) {
            atomicAdd(&work[3], (unsigned long long)(k + x));
            atomicAdd(&work[4], (unsigned long long)k);
            atomicAdd(&work[5], (unsigned long long)x);
        }
    }
}

// Plan, second pass: one warp per candidate tile (grid-strided, so the
// expensive tiles spread over all warps).  The exact per-pixel reach test, the
// removal and insertion positions (warp searches) and the per-pixel stop test;
// a tile with an active pixel is appended to the plan (counts[1]) with its
// groups (counts[3] heavy, counts[4] light), any other keeps its clean values
// (Delta = 0).
constexpr int kHeavyWalk = 1024;   // list entries
template <bool COUNT>
__global__ __launch_bounds__(256, 4) void k_plan_exact(const ViewPtrs* __restrict__ views,
                                                      const DirtyDesc* __restrict__ desc, int K,
                                                      const uint2* __restrict__ cand, PlanItem* __restrict__ plan,
                                                      uint32_t* __restrict__ groups, uint32_t gcap,
                                                      unsigned int* __restrict__ counts, unsigned long long* work,
                                                      SsimBufs sb) {
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t n = counts[2];
    unsigned int drop_reach = 0, drop_stop = 0;
    for (uint32_t i = warp; i < n; i += nwarps) {
        const uint2 c = cand[i];
        const int ibk = (int)c.x, itx = (int)(c.y & 0xffffu), ity = (int)(c.y >> 16);
        const DirtyDesc& d = desc[ibk];
        const ViewPtrs& v = views[ibk % K];
        const int tile = ity * v.tiles_x + itx;
        const bool has_old = d.old_vis && itx >= d.ox0 && itx < d.ox1 && ity >= d.oy0 && ity < d.oy1;
        const bool has_new = d.new_vis && itx >= d.nx0 && itx < d.nx1 && ity >= d.ny0 && ity < d.ny1;
        const BlendRec nrec = d.rec;
        const BlendRec orec = has_old ? v.recs[d.prim] : nrec;
        const uint32_t prim = d.prim;
        const int nw = (v.tile_w * v.tile_h) >> 5;   // 8x4 blocks of the tile
        unsigned reach[kBT / 32];
        bool any = false;
#pragma unroll
        for (int q = 0; q < kBT / 32; q++) {
            int px, py;
            pix_of(itx, ity, v.tile_w, v.tile_h, q * 32 + lane, px, py);
            const float x = (float)px + 0.5f, y = (float)py + 0.5f;
            const bool r = q < nw && px < v.W && py < v.H &&
                           ((has_old && affects(orec, x, y)) || (has_new && affects(nrec, x, y)));
            reach[q] = __ballot_sync(0xffffffffu, r);
            any |= reach[q] != 0u;
        }
        uint32_t pp = 0, ins = 0, cut = 0xffffffffu;
        uint2 rg = make_uint2(0u, 0u);
        if (any) {
            rg = v.ranges[tile];
            if (has_old) {
                pp = warp_lower_bound(v.dk, v.ids, rg.x, rg.y, __float_as_uint(orec.depth), prim) - rg.x;
                cut = pp;
            }
            if (has_new) {
                ins = warp_lower_bound(v.dk, v.ids, rg.x, rg.y, __float_as_uint(nrec.depth), prim) - rg.x;
                cut = min(cut, ins);   // clean-list position of the insertion
                if (has_old && pp < ins) ins -= 1;
            }
            // then the reached pixels whose clean blend had not stopped before the change
            any = false;
#pragma unroll
            for (int q = 0; q < kBT / 32; q++) {
                int px, py;
                pix_of(itx, ity, v.tile_w, v.tile_h, q * 32 + lane, px, py);
                bool a = false;
                if ((reach[q] >> lane) & 1u) a = v.stop[(size_t)py * v.W + px] >= cut;
                reach[q] = __ballot_sync(0xffffffffu, a);   // now: active pixels
                any |= reach[q] != 0u;
            }
        }
        if (!any) {   // every pixel keeps its clean value
            if (COUNT) (cut == 0xffffffffu ? drop_reach : drop_stop)++;
            continue;
        }
        // the item's 7 16-byte parts, one per lane; one group per 8x8 block with an
        // active pixel, (slot << 3) | block.  Groups of tiles with a long walk
        // ahead (from the checkpoint the blend resumes at) go to the front of the
        // group array and are blended first, the others to the back.
        const int lg = tile_lgx(v.tile_w), nb = nw >> 1;
        uint32_t word = 0;
#pragma unroll
        for (int b = 0; b < kDirtyBlocks; b++) {
            const int wa = block_upper(b, lg), wb = wa + (1 << lg);
            uint32_t bw = 0;
#pragma unroll
            for (int q = 0; q < kBT / 32; q++) bw |= (q == wa || q == wb) ? reach[q] : 0u;
            word = lane == b ? bw : word;
        }
        const unsigned gm = __ballot_sync(0xffffffffu, lane < nb && word != 0u);
        const uint32_t Lm = (rg.y - rg.x) - (has_old ? 1u : 0u) + (has_new ? 1u : 0u);
        const uint32_t walk = Lm - min(cut / (uint32_t)kCkStride, v.ck_cnt[tile]) * (uint32_t)kCkStride;
        const bool heavy = walk >= (uint32_t)kHeavyWalk;
        uint32_t slot = 0, gbase = 0;
        if (lane == 0) {
            slot = atomicAdd(&counts[1], 1u);
            gbase = atomicAdd(&counts[heavy ? 3 : 4], (unsigned)__popc(gm));
        }
        slot = __shfl_sync(0xffffffffu, slot, 0);
        gbase = __shfl_sync(0xffffffffu, gbase, 0);
        if ((gm >> lane) & 1u) {
            const uint32_t gi = gbase + __popc(gm & ((1u << lane) - 1u));
            groups[heavy ? gi : gcap - 1u - gi] = (slot << 3) | (uint32_t)lane;
        }
        if (sb.tile_map) {   // dirty-tile SSIM: tile -> slot of this batch, no block delta yet
            if (slot < sb.slot_cap) {
                if (lane < kTilePix / 32) sb.slot_group[(size_t)slot * 8 + lane] = 0xffffffffu;
                if (lane == 0) sb.slot_flags[slot] = 0u;
                if (lane == 0)
                    sb.tile_map[(size_t)ibk * sb.max_tiles + (size_t)tile] =
                        ((unsigned long long)counts[6] << 32) | slot;
            } else if (lane == 0) {
                atomicOr(sb.overflow, 1u);
            }
        }
        uint4* dst = reinterpret_cast<uint4*>(&plan[slot]);
        if (lane < 3) {
            dst[lane] = reinterpret_cast<const uint4*>(&d.rec)[lane];
        } else if (lane == 3) {
            dst[3] = make_uint4(reach[0], reach[1], reach[2], reach[3]);
        } else if (lane == 4) {
            dst[4] = make_uint4(reach[4], reach[5], reach[6], reach[7]);
        } else if (lane == 5) {
            dst[5] = make_uint4((uint32_t)ibk, (uint32_t)tile, rg.x, rg.y);
        } else if (lane == 6) {
            dst[6] = make_uint4(pp, ins, cut, (has_old ? 1u : 0u) | (has_new ? 2u : 0u));
        }
    }
    if (COUNT && lane == 0 && (drop_reach + drop_stop)) {   // warp-uniform counts
        atomicAdd(&work[3], (unsigned long long)(drop_reach + drop_stop));
        atomicAdd(&work[6], (unsigned long long)drop_reach);
        atomicAdd(&work[7], (unsigned long long)drop_stop);
    }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(gmem) : "memory");
}

// Dirty-tile blend, one warp per work unit: an 8x8 pixel block of a planned
// tile that holds an active pixel (the plan's groups, (item << 3) | block), two
// pixels per lane (one column, four rows apart, so the exponent's x terms are
// shared).
// The warp streams the tile's merged list -- the clean list with the old entry
// removed and the corrupted record inserted -- through a ring of kWarpRing
// chunks of 32 entries in shared memory, filled by cp.async gathers issued
// kWarpRing - 1 chunks ahead, so the gathers overlap the blend.  Each chunk is
// culled against the box of the block's pixels that are still blending (active
// and not stopped; recomputed per chunk) with one ballot and the survivors are
// walked in list order (the same arithmetic as the full-frame blend).  Active pixels resume from the clean blend's last checkpoint at or
// before the first changed position; the result is compared with the clean
// image on the fly.  Warps are independent: no block barrier.
constexpr int kWarpRing = 2;
constexpr int kDirtyWarps = 4;   // warps per block
struct WarpRing {
    float4 q[kWarpRing][3][32];   // [chunk slot][16-byte part of the record][entry]
};

// First index in [lo, hi) of the ascending array a whose value is not below key
// (whole warp: each round probes 31 splitters and keeps 1/32 of the interval).
__device__ __forceinline__ uint32_t warp_lower_bound_u32(const uint32_t* __restrict__ a, uint32_t lo, uint32_t hi,
                                                         uint32_t key) {
    const int lane = threadIdx.x & 31;
    while (hi - lo > 32) {
        const uint32_t len = hi - lo;
        bool less = false;
        if (lane < 31) less = a[lo + (uint32_t)(((uint64_t)len * (uint32_t)(lane + 1)) >> 5)] < key;
        const int c = __popc(__ballot_sync(0xffffffffu, less));
        const uint32_t nlo = c == 0 ? lo : lo + (uint32_t)(((uint64_t)len * (uint32_t)c) >> 5) + 1;
        const uint32_t nhi = c == 31 ? hi : lo + (uint32_t)(((uint64_t)len * (uint32_t)(c + 1)) >> 5);
        lo = nlo;
        hi = nhi;
    }
    const uint32_t pos = lo + (uint32_t)lane;
    const bool less = pos < hi && a[pos] < key;
    return lo + __popc(__ballot_sync(0xffffffffu, less));
}

// Entry m of the merged list: the inserted record (returns true) or the clean
// list entry ci (relative to the tile's range).
__device__ __forceinline__ bool merged_entry(uint32_t m, bool has_old, bool has_new, uint32_t pp, uint32_t ins,
                                             uint32_t& ci) {
    if (has_new && m == ins) return true;
    const uint32_t j = (has_new && m > ins) ? m - 1u : m;
    ci = (has_old && j >= pp) ? j + 1u : j;
    return false;
}

__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// One pixel's part of a block's comparison: fixed-point squared error, peak
// difference, footprint / non-finite / clean-non-finite flags and screen cell.
struct BlockCmp {
    unsigned long long fx = 0ull, cells = 0ull;
    float m = 0.0f;
    unsigned foot = 0u, bad = 0u, clean_bad = 0u;
};

__device__ __forceinline__ void block_cmp_add(BlockCmp& b, bool active, float v0, float v1, float v2, const float* c,
                                              int px, int py, int W, int H) {
    if (!active) return;
    const PixCmp r = pixel_compare(v0, v1, v2, c);
    b.fx += r.fx;
    b.m = fmaxf(b.m, r.m);
    b.foot += r.foot ? 1u : 0u;
    b.bad += r.nonfin ? 1u : 0u;
    b.clean_bad += !(isfinite(c[0]) && isfinite(c[1]) && isfinite(c[2])) ? 1u : 0u;
    if (r.foot) b.cells |= cell_bit(px, py, W, H);
}

template <bool COUNT>
__global__ __launch_bounds__(kDirtyWarps * 32, 6) void k_dirty(const ViewPtrs* __restrict__ views, int K,
                                                              const PlanItem* __restrict__ plan,
                                                              const uint32_t* __restrict__ groups, uint32_t gcap,
                                                              const unsigned int* __restrict__ counts,
                                                              CmpAcc* __restrict__ acc,
                                                              unsigned int* __restrict__ queue,
                                                              unsigned long long* work, SsimBufs sb) {
    __shared__ WarpRing rings[kDirtyWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpRing& R = rings[warp];
    const uint32_t nheavy = counts[3], ngroups = counts[3] + counts[4];
    // measurement builds: SM cycles each warp spends per phase (set-up of a group,
    // the walk, the comparison and reductions)
    long long t_pro = 0, t_walk = 0, t_epi = 0;
    while (true) {
        long long c0 = COUNT ? clock64() : 0;
        uint32_t gi = 0;
        if (lane == 0) gi = atomicAdd(&queue[0], 1u);
        gi = __shfl_sync(0xffffffffu, gi, 0);
        if (gi >= ngroups) break;
        // heavy groups first (front of the array), then the light ones (from the back)
        const uint32_t code = groups[gi < nheavy ? gi : gcap - 1u - (gi - nheavy)];
        const PlanItem* it = &plan[code >> 3];
        const int b = (int)(code & 7u);            // 8x8 block of the tile
        const uint4 f5 = reinterpret_cast<const uint4*>(it)[5];   // bk, tile, s, e
        const uint4 f6 = reinterpret_cast<const uint4*>(it)[6];   // pp, ins, cut, flags
        const int bk = (int)f5.x;
        const uint32_t tile = f5.y, pp = f6.x, ins = f6.y, cut = f6.z;
        const bool has_old = f6.w & 1u, has_new = f6.w & 2u;
        const ViewPtrs& v = views[bk % K];
        const int tw = v.tile_w, th = v.tile_h, lg = tile_lgx(tw), nb = (tw * th) >> 6;
        const int wA = block_upper(b, lg), wB = wA + (1 << lg);   // the block's upper and lower 8x4 halves
        const uint32_t amA = it->mask[wA], amB = it->mask[wB];
        const int tx = (int)(tile % (uint32_t)v.tiles_x), ty = (int)(tile / (uint32_t)v.tiles_x);
        // lane: pixel A of the upper half, pixel B four rows below it
        const int px = tx * tw + block_x0(b, lg) + (lane & 7);
        const int pyA = ty * th + block_y0(b, lg) + (lane >> 3);
        const int pyB = pyA + 4;
        const bool inA = (amA >> lane) & 1u, inB = (amB >> lane) & 1u;   // decided by the plan (inside the image)
        const bool act = inA || inB;
        PixGeo g;   // the box of the block's active pixel centres
        g.wx0 = (float)__reduce_min_sync(0xffffffffu, act ? px : 0x7fffffff) + 0.5f;
        g.wx1 = (float)__reduce_max_sync(0xffffffffu, act ? px : -1) + 0.5f;
        g.wy0 = (float)__reduce_min_sync(0xffffffffu, inA ? pyA : (inB ? pyB : 0x7fffffff)) + 0.5f;
        g.wy1 = (float)__reduce_max_sync(0xffffffffu, inB ? pyB : (inA ? pyA : -1)) + 0.5f;
        // this lane's pixels: A in the upper half, B four rows below it
        const int x0 = px, y0 = pyA, u0 = wA * 32 + lane, y1 = pyB, u1 = wB * 32 + lane;
        const bool actA = inA, actB = inB;
        const float pxc = (float)x0 + 0.5f, pycA = (float)y0 + 0.5f, pycB = (float)y1 + 0.5f;
        Pix pA{1.0f, 0.0f, 0.0f, 0.0f, !actA, 0u}, pB{1.0f, 0.0f, 0.0f, 0.0f, !actB, 0u};
        // The merged list equals the clean list before `cut`, so an active pixel
        // (not stopped before `cut`) can resume from the clean blend's state at the
        // last checkpoint at or before `cut`.
        const uint32_t cstar = min(cut / (uint32_t)kCkStride, v.ck_cnt[tile]);
        const uint32_t start = cstar * (uint32_t)kCkStride;
        if (cstar > 0) {
            const float4* ckt = v.ck + (size_t)(v.ck_off[tile] + cstar - 1) * (uint32_t)(tw * th);
            if (actA) {
                const float4 st = ckt[u0];
                pA.T = st.x;
                pA.c0 = st.y;
                pA.c1 = st.z;
                pA.c2 = st.w;
            }
            if (actB) {
                const float4 st = ckt[u1];
                pB.T = st.x;
                pB.c0 = st.y;
                pB.c1 = st.z;
                pB.c2 = st.w;
            }
        }
        // This block's sublist of the clean list (the entries whose box meets the
        // block, positions ascending) from `start`, without the old entry and with the
        // corrupted record at its place: every entry outside the sublist fails the
        // cull below anyway.
        const uint32_t boff = v.bl_off[(size_t)tile * nb + b];
        const uint32_t blen = v.bl_off[(size_t)tile * nb + b + 1] - boff;
        const uint32_t* B = v.bl_pos + boff;
        const uint32_t k0 = warp_lower_bound_u32(B, 0, blen, start);
        bool has_kpp = false;
        uint32_t kpp = 0, lins = 0;
        if (has_old) {
            kpp = warp_lower_bound_u32(B, 0, blen, pp);
            has_kpp = kpp < blen && B[kpp] == pp;
        }
        if (has_new) {
            // clean-list position before which the corrupted record goes (ins counts
            // the list without the old entry; at ins == pp both readings coincide)
            const uint32_t ins_c = (has_old && ins >= pp) ? ins + 1u : ins;
            const uint32_t tins = warp_lower_bound_u32(B, 0, blen, ins_c);
            lins = tins - k0 - ((has_kpp && kpp < tins) ? 1u : 0u);
        }
        const uint32_t Lb = (blen - k0) - (has_kpp ? 1u : 0u) + (has_new ? 1u : 0u);
        const uint32_t nch = (Lb + 31u) / 32u;
        // source of this lane's entry in chunk c (NULL past the end)
        auto src_of = [&](uint32_t c) -> const BlendRec* {
            const uint32_t m = c * 32u + (uint32_t)lane;
            if (c >= nch || m >= Lb) return nullptr;
            uint32_t ci = 0;
            if (merged_entry(m, has_kpp, has_new, kpp - k0, lins, ci)) return &it->rec;
            return v.bl_rec + boff + k0 + ci;   // the sublist's records are stored in order
        };
        auto issue = [&](uint32_t c, const BlendRec* src) {
            if (src) {
                const int slot = (int)(c % (uint32_t)kWarpRing);
#pragma unroll
                for (int part = 0; part < 3; part++)
                    cp_async16(&R.q[slot][part][lane], reinterpret_cast<const float4*>(src) + part);
            }
            cp_async_commit_group();
        };
        // the previous unit's copies may still be landing in the ring
        cp_async_wait_all();
        __syncwarp();
#pragma unroll
        for (int c = 0; c < kWarpRing - 1; c++) issue((uint32_t)c, src_of((uint32_t)c));
        const BlendRec* next_src = src_of(kWarpRing - 1);
        unsigned int nev = 0, staged = 0;
        unsigned steps[2] = {0u, 0u};
        long long c1 = COUNT ? clock64() : 0;
        for (uint32_t c = 0; c < nch; c++) {
            __syncwarp();   // every lane is done with the slot the next issue overwrites
            issue(c + kWarpRing - 1, next_src);
            next_src = src_of(c + kWarpRing);
            cp_async_wait_group<kWarpRing - 1>();   // this lane's copies of chunk c have landed
            __syncwarp();                            // and every other lane's
            const int slot = (int)(c % (uint32_t)kWarpRing);
            const uint32_t base = c * 32u;
            const int cnt = (int)min(32u, Lb - base);
            staged += (uint32_t)cnt;
            if (c > 0) {   // the box of the pixel centres still blending: a stopped pixel takes no entry
                const bool la = !pA.done, lb = !pB.done;
                g.wx0 = (float)__reduce_min_sync(0xffffffffu, (la || lb) ? px : 0x7fffffff) + 0.5f;
                g.wx1 = (float)__reduce_max_sync(0xffffffffu, (la || lb) ? px : -1) + 0.5f;
                g.wy0 = (float)__reduce_min_sync(0xffffffffu, la ? pyA : (lb ? pyB : 0x7fffffff)) + 0.5f;
                g.wy1 = (float)__reduce_max_sync(0xffffffffu, lb ? pyB : (la ? pyA : -1)) + 0.5f;
            }
            bool pass = false;
            if (lane < cnt) {
                const float4 a = R.q[slot][0][lane], bb = R.q[slot][1][lane];
                // the entry's box [mx - ex, mx + ex] x [my - ey, my + ey] against the block's,
                // then the conservative conic test over the block's pixel centres
                pass = !(a.x + bb.z < g.wx0 || a.x - bb.z > g.wx1 || a.y + bb.w < g.wy0 || a.y - bb.w > g.wy1) &&
                       rect_reachable(a.x, a.y, a.z, a.w, bb.x, bb.y, g.wx0, g.wx1, g.wy0, g.wy1);
            }
            const unsigned m = __ballot_sync(0xffffffffu, pass);
            auto fetch = [&](int e) {
                const float4 q1 = R.q[slot][1][e], q2 = R.q[slot][2][e];
                return EntryQ{R.q[slot][0][e], q1.x, q1.y, q2.x, q2.y, q2.z};
            };
            walk_survivors2<COUNT, false>(m, 0, fetch, pxc, pycA, pycB, pA, pB, nev, base, steps);
            if (__all_sync(0xffffffffu, pA.done && pB.done)) break;
        }
        long long c2 = COUNT ? clock64() : 0;
        // compare the active pixels with the clean image; every other pixel keeps
        // its clean value (Delta = 0), and the clean image's non-finite pixels are
        // counted once per view at finalize
        const float a0 = __fadd_rn(pA.c0, pA.T), a1 = __fadd_rn(pA.c1, pA.T), a2 = __fadd_rn(pA.c2, pA.T);
        const float b0 = __fadd_rn(pB.c0, pB.T), b1 = __fadd_rn(pB.c1, pB.T), b2 = __fadd_rn(pB.c2, pB.T);
        const float* cA = v.clean + ((size_t)y0 * v.W + x0) * 3;
        const float* cB = v.clean + ((size_t)y1 * v.W + px) * 3;
        if (sb.deltas) {   // dirty-tile SSIM: keep the block's new values, two 32-pixel delta units per group
            const uint32_t slot = code >> 3;
            if (2u * gi + 1u < sb.delta_cap && slot < sb.slot_cap) {
                // delta unit 2 gi: upper half, 2 gi + 1: lower half; one entry per pixel of the half
                if (actA) sb.deltas[(size_t)(2u * gi) * 32 + lane] = make_float4(a0, a1, a2, 0.0f);
                if (actB) sb.deltas[(size_t)(2u * gi + 1u) * 32 + lane] = make_float4(b0, b1, b2, 0.0f);
                if (lane == 0) {
                    sb.slot_group[(size_t)slot * 8 + wA] = 2u * gi;
                    sb.slot_group[(size_t)slot * 8 + wB] = 2u * gi + 1u;
                }
                // where the changed pixels are: which neighbouring tiles their SSIM windows reach
                auto edge = [&](bool a, int x, int y, float n0, float n1, float n2, const float* c) -> unsigned {
                    const bool ch = a && (__float_as_uint(n0) != __float_as_uint(c[0]) ||
                                          __float_as_uint(n1) != __float_as_uint(c[1]) ||
                                          __float_as_uint(n2) != __float_as_uint(c[2]));
                    const int lx = x - tx * tw, ly = y - ty * th;
                    return ch ? (16u | (lx < 5 ? 1u : 0u) | (lx > tw - 6 ? 2u : 0u) | (ly < 5 ? 4u : 0u) |
                                 (ly > th - 6 ? 8u : 0u))
                              : 0u;
                };
                const unsigned f = edge(actA, x0, y0, a0, a1, a2, cA) | edge(actB, px, y1, b0, b1, b2, cB);
                const unsigned fo = __reduce_or_sync(0xffffffffu, f);
                if (lane == 0 && fo) atomicOr(&sb.slot_flags[slot], fo);
            } else if (lane == 0) {
                atomicOr(sb.overflow, 1u);
            }
        }
        BlockCmp r;
        block_cmp_add(r, actA, a0, a1, a2, cA, x0, y0, v.W, v.H);
        block_cmp_add(r, actB, b0, b1, b2, cB, px, y1, v.W, v.H);
        unsigned long long fx = r.fx;
        float mx = r.m;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            fx += __shfl_xor_sync(0xffffffffu, fx, o);
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        const unsigned nfoot = __reduce_add_sync(0xffffffffu, r.foot);
        const unsigned nbad = __reduce_add_sync(0xffffffffu, r.bad);
        const unsigned ncb = __reduce_add_sync(0xffffffffu, r.clean_bad);
        // screen cells holding a footprint pixel (contamination of a sort-first partition)
        const unsigned long long cells =
            (unsigned long long)__reduce_or_sync(0xffffffffu, (unsigned)r.cells) |
            ((unsigned long long)__reduce_or_sync(0xffffffffu, (unsigned)(r.cells >> 32)) << 32);
        if (lane == 0) {
            CmpAcc* A = &acc[bk];
            if (cells) atomicOr(&A->reg_actual, cells);
            if (fx) atomicAdd(&A->sse_fx, fx);
            if (mx > 0.0f) atomicMax(&A->maxabs_bits, __float_as_uint(mx));
            if (nfoot) atomicAdd(&A->footprint, nfoot);
            if (nbad) atomicAdd(&A->nonfinite, nbad);
            if (ncb) atomicAdd(&A->clean_nonfinite_replaced, ncb);
        }
        if (COUNT) {
            const unsigned wn = __reduce_add_sync(0xffffffffu, nev);
            // a tile counts once, on its first group (lowest block with an active pixel)
            const bool first =
                __ballot_sync(0xffffffffu, lane < b && (it->mask[block_upper(lane & 3, lg)] |
                                                        it->mask[block_upper(lane & 3, lg) + (1 << lg)]) != 0u) == 0u;
            if (lane == 0) {
                if (wn) atomicAdd(&work[0], (unsigned long long)wn);
                if (first) atomicAdd(&work[1], 1ull);
                atomicAdd(&work[2], (unsigned long long)staged);
                atomicAdd(&work[8], (unsigned long long)steps[0]);
                atomicAdd(&work[9], (unsigned long long)steps[1]);
                atomicAdd(&work[10], 1ull);
                const unsigned npix = (unsigned)(__popc(amA) + __popc(amB));
                atomicAdd(&work[14], (unsigned long long)npix);
                atomicAdd(&work[15], (unsigned long long)npix * steps[0]);
            }
            t_pro += c1 - c0;
            t_walk += c2 - c1;
            t_epi += clock64() - c2;
        }
    }
    if (COUNT && lane == 0) {
        atomicAdd(&work[11], (unsigned long long)t_pro);
        atomicAdd(&work[12], (unsigned long long)t_walk);
        atomicAdd(&work[13], (unsigned long long)t_epi);
    }
    cp_async_wait_all();   // leave no copy in flight
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

gs_status launch_blend_image(const BlendRec* recs, const uint32_t* ids, const uint2* ranges, const DevCamera& cam,
                             float* img, cudaStream_t st) {
    const int tx = cam.tiles_x, ty = cam.tiles_y, P = cam.tile_w * cam.tile_h / 2;   // threads: two pixels each
    if (tx * ty == 0) return GS_OK;
    k_blend_full<0, false><<<tx * ty, P, 0, st>>>(recs, ids, ranges, cam.W, cam.H, tx, cam.tile_w, cam.tile_h, img,
                                                   nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                   nullptr, nullptr);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status launch_blend_compare(const BlendRec* recs, const uint32_t* ids, const uint2* ranges, const DevCamera& cam,
                               const float* clean, CmpAcc* acc, unsigned long long* work, cudaStream_t st) {
    const int tx = cam.tiles_x, ty = cam.tiles_y, P = cam.tile_w * cam.tile_h / 2;   // threads: two pixels each
    if (tx * ty == 0) return GS_OK;
    if (work)
        k_blend_full<1, true><<<tx * ty, P, 0, st>>>(recs, ids, ranges, cam.W, cam.H, tx, cam.tile_w, cam.tile_h,
                                                     nullptr, clean, acc, work, nullptr, nullptr, nullptr, nullptr,
                                                     nullptr, nullptr);
    else
        k_blend_full<1, false><<<tx * ty, P, 0, st>>>(recs, ids, ranges, cam.W, cam.H, tx, cam.tile_w, cam.tile_h,
                                                      nullptr, clean, acc, nullptr, nullptr, nullptr, nullptr,
                                                      nullptr, nullptr, nullptr);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status launch_blend_image_stop(const BlendRec* recs, const uint32_t* ids, const uint2* ranges, const DevCamera& cam,
                                  float* img, uint32_t* stop, uint32_t* tile_stop, float4* ck, const uint32_t* ck_off,
                                  const uint32_t* ck_cnt, unsigned int* clean_nonfin, cudaStream_t st) {
    const int tx = cam.tiles_x, ty = cam.tiles_y, P = cam.tile_w * cam.tile_h / 2;   // threads: two pixels each
    if (tx * ty == 0) return GS_OK;
    k_blend_full<2, false><<<tx * ty, P, 0, st>>>(recs, ids, ranges, cam.W, cam.H, tx, cam.tile_w, cam.tile_h, img,
                                                   nullptr, nullptr, nullptr, stop, tile_stop, ck, ck_off, ck_cnt,
                                                   clean_nonfin);
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

__global__ void k_regions_out(const CmpAcc* acc, int count, unsigned long long* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    out[2 * i] = acc[i].reg_actual;
    out[2 * i + 1] = acc[i].reg_pred;
}

gs_status launch_regions_out(const CmpAcc* acc, int count, unsigned long long* out, cudaStream_t st) {
    if (count > 0) k_regions_out<<<(count + 255) / 256, 256, 0, st>>>(acc, count, out);
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
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dirty<false>, kDirtyWarps * 32, 0);
        if (per_sm < 1) per_sm = 1;
        blocks = per_sm * num_sms();
    }
    return blocks;
}

size_t plan_item_size() { return sizeof(PlanItem); }

// ev_mid (optional): recorded between the plan kernels and the blend kernel.
// queue[0]: blend work queue, queue[1]: plan items, queue[2]: candidate tiles,
// queue[3] / queue[4]: heavy / light groups (all zeroed by the injector); cand
// holds as many entries as plan, groups gcap = 8 per plan entry.
gs_status launch_dirty_ssim(const void* dev_views, int K, const void* plan, const unsigned int* queue,
                            const SsimBufs& sb, CmpAcc* acc, cudaStream_t st);

gs_status launch_dirty_blend(const void* dev_views, const DirtyDesc* desc, const uint32_t* item_off, int BK, int K,
                             void* plan, uint2* cand, uint32_t* groups, uint32_t gcap, CmpAcc* acc,
                             unsigned int* queue, unsigned long long* work, cudaEvent_t ev_mid, const SsimBufs& sb,
                             cudaStream_t st) {
    const ViewPtrs* views = (const ViewPtrs*)dev_views;
    PlanItem* pl = (PlanItem*)plan;
    const int plan_blocks = num_sms() * 8;
    if (work) {
        k_plan_filter<true><<<plan_blocks, 256, 0, st>>>(views, desc, item_off, BK, K, cand, queue, work);
        k_plan_exact<true><<<plan_blocks, 256, 0, st>>>(views, desc, K, cand, pl, groups, gcap, queue, work, sb);
    } else {
        k_plan_filter<false><<<plan_blocks, 256, 0, st>>>(views, desc, item_off, BK, K, cand, queue, nullptr);
        k_plan_exact<false><<<plan_blocks, 256, 0, st>>>(views, desc, K, cand, pl, groups, gcap, queue, nullptr, sb);
    }
    if (ev_mid) {
        cudaError_t e = cudaEventRecordWithFlags(ev_mid, st, cudaEventRecordExternal);
        if (e != cudaSuccess) return set_error(GS_ERR_CUDA, cudaGetErrorString(e));
    }
    if (work)
        k_dirty<true><<<dirty_grid(), kDirtyWarps * 32, 0, st>>>(views, K, pl, groups, gcap, queue, acc, queue, work,
                                                                sb);
    else
        k_dirty<false><<<dirty_grid(), kDirtyWarps * 32, 0, st>>>(views, K, pl, groups, gcap, queue, acc, queue,
                                                                 nullptr, sb);
    if (sb.tile_map) GS_TRY(launch_dirty_ssim(dev_views, K, plan, queue, sb, acc, st));
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

// Per tile: the sort key (depth bits << 32 | id) of the list entry at which the
// last of its pixels stopped; ~0 when some pixel never stopped.  Every pixel of
// the tile stopped before a change whose key is above it.
__global__ void k_stop_keys(const uint2* __restrict__ ranges, const uint32_t* __restrict__ tile_stop,
                            const uint32_t* __restrict__ dk, const uint32_t* __restrict__ ids, int ntiles,
                            unsigned long long* __restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const uint2 rg = ranges[t];
    const uint32_t ts = tile_stop[t];
    unsigned long long key = ~0ull;
    if (ts != 0xffffffffu && ts < rg.y - rg.x)
        key = ((unsigned long long)dk[rg.x + ts] << 32) | (unsigned long long)ids[rg.x + ts];
    out[t] = key;
}

gs_status launch_stop_keys(const uint2* ranges, const uint32_t* tile_stop, const uint32_t* dk, const uint32_t* ids,
                           int ntiles, unsigned long long* out, cudaStream_t st) {
    if (ntiles > 0) k_stop_keys<<<(ntiles + 255) / 256, 256, 0, st>>>(ranges, tile_stop, dk, ids, ntiles, out);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

void fill_view_ptrs(void* host_dst, const ViewState& vs) {
    ViewPtrs v;
    v.recs = vs.recs;
    v.ids = vs.ids;
    v.dk = vs.dk;
    v.ranges = vs.ranges;
    v.clean = vs.clean;
    v.stop = vs.stop;
    v.tile_stop = vs.tile_stop;
    v.stop_key = vs.stop_key;
    v.bl_off = vs.bl_off;
    v.bl_pos = vs.bl_pos;
    v.bl_rec = vs.bl_rec;
    v.ck = vs.ck;
    v.ck_off = vs.ck_off;
    v.ck_cnt = vs.ck_cnt;
    v.W = vs.cam.W;
    v.H = vs.cam.H;
    v.tiles_x = vs.cam.tiles_x;
    v.tile_w = vs.cam.tile_w;
    v.tile_h = vs.cam.tile_h;
    v.pad[0] = v.pad[1] = v.pad[2] = 0;
    memcpy(host_dst, &v, sizeof(v));
}

// ---------------------------------------------------------------------------
// Per (tile, 8x8 block) sublists of the clean tile lists: the positions of the
// entries whose box [mx - ex, mx + ex] x [my - ey, my + ey] meets the block's
// pixel-centre box (the same comparisons as the dirty-tile cull, on a box that
// contains every active-pixel box of the block, so an entry left out would be
// culled there anyway).  One warp per tile; positions ascend in each sublist.
// ---------------------------------------------------------------------------
template <bool FILL>
__global__ void k_blists(const BlendRec* __restrict__ recs, const uint32_t* __restrict__ ids,
                         const uint2* __restrict__ ranges, int ntiles, int tiles_x, int tw, int th,
                         uint32_t* __restrict__ counts, const uint32_t* __restrict__ off, uint32_t* __restrict__ pos,
                         BlendRec* __restrict__ brec) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    const int lg = tile_lgx(tw), nb = (tw * th) >> 6;   // 8x8 blocks per tile
    for (int t = warp; t < ntiles; t += nwarps) {
        const uint2 rg = ranges[t];
        const int tx = t % tiles_x, ty = t / tiles_x;
        uint32_t base[kDirtyBlocks];
#pragma unroll
        for (int b = 0; b < kDirtyBlocks; b++) base[b] = (FILL && b < nb) ? off[(size_t)t * nb + b] : 0u;
        for (uint32_t j0 = 0; j0 < rg.y - rg.x; j0 += 32) {
            const uint32_t j = j0 + (uint32_t)lane;
            unsigned mb = 0u;
            uint32_t id = 0;
            if (j < rg.y - rg.x) {
                id = ids[rg.x + j];
                const float4* r = reinterpret_cast<const float4*>(recs + id);
                const float4 a = __ldg(r), b = __ldg(r + 1);   // (mx, my, ca, cb), (cc, opac, ex, ey)
#pragma unroll
                for (int k = 0; k < kDirtyBlocks; k++) {
                    const float wx0 = (float)(tx * tw + block_x0(k, lg)) + 0.5f, wx1 = wx0 + 7.0f;
                    const float wy0 = (float)(ty * th + block_y0(k, lg)) + 0.5f, wy1 = wy0 + 7.0f;
                    const bool pass =
                        k < nb && !(a.x + b.z < wx0 || a.x - b.z > wx1 || a.y + b.w < wy0 || a.y - b.w > wy1);
                    mb |= pass ? (1u << k) : 0u;
                }
            }
#pragma unroll
            for (int k = 0; k < kDirtyBlocks; k++) {
                const unsigned bw = __ballot_sync(0xffffffffu, (mb >> k) & 1u);
                if (FILL && ((mb >> k) & 1u)) {
                    const uint32_t q = base[k] + __popc(bw & ((1u << lane) - 1u));
                    pos[q] = j;
                    brec[q] = recs[id];
                }
                base[k] += (uint32_t)__popc(bw);
            }
        }
        if (!FILL && lane < nb) {
            uint32_t c = 0;
#pragma unroll
            for (int k = 0; k < kDirtyBlocks; k++) c = lane == k ? base[k] : c;
            counts[(size_t)t * nb + lane] = c;
        }
    }
}

gs_status launch_blists(const BlendRec* recs, const uint32_t* ids, const uint2* ranges, const DevCamera& cam,
                        uint32_t* counts, const uint32_t* off, uint32_t* pos, BlendRec* brec, cudaStream_t st) {
    const int ntiles = cam.tiles_x * cam.tiles_y;
    if (ntiles <= 0) return GS_OK;
    const int blocks = std::max(1, std::min((ntiles + 7) / 8, num_sms() * 16));
    if (pos)
        k_blists<true><<<blocks, 256, 0, st>>>(recs, ids, ranges, ntiles, cam.tiles_x, cam.tile_w, cam.tile_h, nullptr,
                                               off, pos, brec);
    else
        k_blists<false><<<blocks, 256, 0, st>>>(recs, ids, ranges, ntiles, cam.tiles_x, cam.tile_w, cam.tile_h, counts,
                                                nullptr, nullptr, nullptr);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
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
