// SSIM of a corrupted frame against the clean one (Sec. 3 "Metrics and
// severity", Wang et al. 2004): per channel, Gaussian-weighted local means,
// variances and covariance over an 11x11 window (sigma 1.5, weights normalised
// to sum 1), SSIM = (2 mx my + C1)(2 sxy + C2) / ((mx^2 + my^2 + C1)(sx^2 + sy^2
// + C2)), C1 = 0.01^2, C2 = 0.03^2, on [0,1]-clamped values; the frame's SSIM is
// the mean over the windows inside the frame (pixels at least 5 from every
// edge) and over the channels.
//
// One 16x16 tile per block: the tile and a 5-pixel halo (26x26) of both images
// are staged in shared memory, a horizontal pass of the 11-tap filter, then a
// vertical one.  Every operation is explicitly rounded, so the full-frame and
// the dirty-tile kernels compute the same bits per pixel.  The sum of
// (1 - SSIM) over the pixels is accumulated in fixed point (2^-32), so totals do
// not depend on the order tiles finish.  Where both images agree on a whole
// window the numerator and denominator are computed identically and SSIM is
// exactly 1 (a zero term), so the dirty-tile engine only visits tiles within
// one tile of a re-blended tile.
#include "gs_internal.h"

namespace gs {
namespace {

constexpr int kSR = 5;               // window radius
constexpr int kSS = kTile + 2 * kSR; // staged edge (26)
constexpr float kSsimFx = 4294967296.0f;   // 2^32

struct SsimW {
    float w[2 * kSR + 1];
};

struct SsimStage {
    float x[3][kSS][kSS];   // image under test (corrupted), clamped
    float y[3][kSS][kSS];   // clean image, clamped
    float h[5][3][kSS][kTile];   // horizontal sums of x, y, xx, yy, xy
};

__device__ __forceinline__ float clamp01(float v) { return v > 0.0f ? (v < 1.0f ? v : 1.0f) : 0.0f; }

// Horizontal then vertical filtering of the staged tile, then the SSIM of
// every channel of this thread's pixel; returns sum over channels of
// (1 - SSIM) in fixed point (0 outside the valid region or the frame).
__device__ __forceinline__ long long ssim_tile_pixel(SsimStage& s, const SsimW& W11, int tx, int ty, int W, int H) {
    for (int q = threadIdx.x; q < 3 * kSS * kTile; q += blockDim.x) {
        const int ch = q / (kSS * kTile), r = (q / kTile) % kSS, c = q % kTile;
        float sx = 0.0f, sy = 0.0f, sxx = 0.0f, syy = 0.0f, sxy = 0.0f;
#pragma unroll
        for (int j = 0; j < 2 * kSR + 1; j++) {
            const float u = s.x[ch][r][c + j], v = s.y[ch][r][c + j], w = W11.w[j];
            sx = __fmaf_rn(w, u, sx);
            sy = __fmaf_rn(w, v, sy);
            sxx = __fmaf_rn(w, __fmul_rn(u, u), sxx);
            syy = __fmaf_rn(w, __fmul_rn(v, v), syy);
            sxy = __fmaf_rn(w, __fmul_rn(u, v), sxy);
        }
        s.h[0][ch][r][c] = sx;
        s.h[1][ch][r][c] = sy;
        s.h[2][ch][r][c] = sxx;
        s.h[3][ch][r][c] = syy;
        s.h[4][ch][r][c] = sxy;
    }
    __syncthreads();
    const int li = threadIdx.x / kTile, lj = threadIdx.x % kTile;
    const int px = tx * kTile + lj, py = ty * kTile + li;
    long long fx = 0;
    if (px >= kSR && px < W - kSR && py >= kSR && py < H - kSR) {
        const float C1 = 1e-4f, C2 = 9e-4f;
#pragma unroll
        for (int ch = 0; ch < 3; ch++) {
            float mx = 0.0f, my = 0.0f, exx = 0.0f, eyy = 0.0f, exy = 0.0f;
#pragma unroll
            for (int k = 0; k < 2 * kSR + 1; k++) {
                const float w = W11.w[k];
                mx = __fmaf_rn(w, s.h[0][ch][li + k][lj], mx);
                my = __fmaf_rn(w, s.h[1][ch][li + k][lj], my);
                exx = __fmaf_rn(w, s.h[2][ch][li + k][lj], exx);
                eyy = __fmaf_rn(w, s.h[3][ch][li + k][lj], eyy);
                exy = __fmaf_rn(w, s.h[4][ch][li + k][lj], exy);
            }
            const float mxy = __fmul_rn(mx, my), mxx = __fmul_rn(mx, mx), myy = __fmul_rn(my, my);
            const float num = __fmul_rn(__fadd_rn(__fmul_rn(2.0f, mxy), C1),
                                        __fadd_rn(__fmul_rn(2.0f, __fsub_rn(exy, mxy)), C2));
            const float den = __fmul_rn(__fadd_rn(__fadd_rn(mxx, myy), C1),
                                        __fadd_rn(__fadd_rn(__fsub_rn(exx, mxx), __fsub_rn(eyy, myy)), C2));
            const float one_minus = __fsub_rn(1.0f, __fdiv_rn(num, den));
            fx += __float2ll_rn(__fmul_rn(one_minus, kSsimFx));
        }
    }
    return fx;
}

// block-wide sum of a 64-bit value, added to *dst by thread 0
__device__ __forceinline__ void block_add_ll(long long v, unsigned long long* dst) {
    __shared__ long long red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        if (t) atomicAdd(dst, (unsigned long long)t);
    }
    __syncthreads();
}

// stage the 26x26 neighbourhood of tile (tx, ty): x from `test` (or the clean
// image with dirty-tile deltas, see below), y from `clean`; outside the frame 0
__device__ __forceinline__ void stage_pair(SsimStage& s, const float* test, const float* clean, int tx, int ty, int W,
                                           int H) {
    for (int q = threadIdx.x; q < kSS * kSS; q += blockDim.x) {
        const int r = q / kSS, c = q % kSS;
        const int gx = tx * kTile - kSR + c, gy = ty * kTile - kSR + r;
        const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
        const size_t o = in ? ((size_t)gy * W + gx) * 3 : 0;
#pragma unroll
        for (int ch = 0; ch < 3; ch++) {
            s.x[ch][r][c] = in ? clamp01(test[o + ch]) : 0.0f;
            s.y[ch][r][c] = in ? clamp01(clean[o + ch]) : 0.0f;
        }
    }
    __syncthreads();
}

// full frame: one block per tile that holds a valid pixel
__global__ __launch_bounds__(kTilePix) void k_ssim_full(const float* __restrict__ test, const float* __restrict__ clean,
                                                       int W, int H, int tiles_x, SsimW w11,
                                                       unsigned long long* __restrict__ acc) {
    __shared__ SsimStage s;
    const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
    stage_pair(s, test, clean, tx, ty, W, H);
    block_add_ll(ssim_tile_pixel(s, w11, tx, ty, W, H), acc);
}

__global__ void k_ssim_finalize(const unsigned long long* acc, int count, int W, int H, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double nvalid = 3.0 * (double)max(W - 2 * kSR, 0) * (double)max(H - 2 * kSR, 0);
    out[i] = nvalid > 0 ? 1.0 - (double)(long long)acc[i] * (1.0 / 4294967296.0) / nvalid : 1.0;
}

}  // namespace

SsimW ssim_weights() {
    SsimW w;
    double v[2 * kSR + 1], t = 0.0;
    for (int i = -kSR; i <= kSR; i++) t += (v[i + kSR] = std::exp(-(double)(i * i) / (2.0 * 1.5 * 1.5)));
    for (int i = 0; i < 2 * kSR + 1; i++) w.w[i] = (float)(v[i] / t);
    return w;
}

// ---------------------------------------------------------------------------
// dirty-tile engine: the SSIM of every (variant, view) from the re-blended
// pixels.  Corrupted values: the clean image with each active pixel's new
// value (deltas written by the blend kernel, found through the per-(variant,
// view) tile -> plan slot map and the slot's block -> delta index table).
// Each tile within one tile of a planned tile is claimed once (atomicMax of a
// per-batch generation tag) and processed by one block.
// ---------------------------------------------------------------------------
__global__ __launch_bounds__(kTilePix) void k_dirty_ssim(const ViewPtrs* __restrict__ views, int K,
                                                        const PlanItem* __restrict__ plan,
                                                        const unsigned int* __restrict__ queue, SsimBufs sb,
                                                        SsimW w11, CmpAcc* __restrict__ acc) {
    __shared__ SsimStage s;
    __shared__ int claim;
    const uint32_t n_items = queue[1];
    const unsigned long long gen = (unsigned long long)queue[6] << 32;
    for (uint32_t pair = blockIdx.x; pair < n_items * 9u; pair += gridDim.x) {
        const uint32_t slot = pair / 9u, nb = pair % 9u;
        const PlanItem& it = plan[slot];
        const ViewPtrs& v = views[it.bk % (uint32_t)K];
        const int tiles_y = (v.H + kTile - 1) / kTile;
        const int tx = (int)(it.tile % (uint32_t)v.tiles_x) + (int)(nb % 3u) - 1;
        const int ty = (int)(it.tile / (uint32_t)v.tiles_x) + (int)(nb / 3u) - 1;
        if (threadIdx.x == 0) {
            claim = 0;
            // only where a changed pixel's window reaches: the tile itself if any pixel
            // changed, a neighbour if one changed within 5 pixels of the shared edge
            const unsigned f = slot < sb.slot_cap ? sb.slot_flags[slot] : 31u;
            const int dx = (int)(nb % 3u) - 1, dy = (int)(nb / 3u) - 1;
            const bool reach = (f & 16u) && (dx == 0 || (f & (dx < 0 ? 1u : 2u))) &&
                               (dy == 0 || (f & (dy < 0 ? 4u : 8u)));
            if (reach && tx >= 0 && ty >= 0 && tx < v.tiles_x && ty < tiles_y) {
                const unsigned long long old =
                    atomicMax(&sb.ssim_map[(size_t)it.bk * sb.max_tiles + (size_t)(ty * v.tiles_x + tx)], gen);
                claim = old < gen;
            }
        }
        __syncthreads();
        const int claimed = claim;
        __syncthreads();   // every thread has read the flag before thread 0 rewrites it
        if (!claimed) continue;   // block-uniform
        // the 3x3 tiles around (tx, ty): delta index and active mask of each 8x4 block
        // (0xffffffff / 0: no delta), resolved once for the staging below
        __shared__ uint32_t nb_gi[9][8], nb_mask[9][8];
        if (threadIdx.x < 72) {
            const int t = threadIdx.x / 8, w = threadIdx.x % 8;
            const int ntx = tx + t % 3 - 1, nty = ty + t / 3 - 1;
            uint32_t gi = 0xffffffffu, m = 0u;
            if (ntx >= 0 && nty >= 0 && ntx < v.tiles_x && nty < tiles_y) {
                const unsigned long long e = sb.tile_map[(size_t)it.bk * sb.max_tiles + (size_t)(nty * v.tiles_x + ntx)];
                if ((e & 0xffffffff00000000ull) == gen) {
                    const uint32_t slot2 = (uint32_t)e;
                    gi = sb.slot_group[(size_t)slot2 * 8 + w];
                    m = gi != 0xffffffffu ? plan[slot2].mask[w] : 0u;
                }
            }
            nb_gi[t][w] = gi;
            nb_mask[t][w] = m;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < kSS * kSS; q += blockDim.x) {
            const int r = q / kSS, c = q % kSS;
            const int gx = tx * kTile - kSR + c, gy = ty * kTile - kSR + r;
            const bool in = gx >= 0 && gx < v.W && gy >= 0 && gy < v.H;
            float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f;
            if (in) {
                const float* cl = v.clean + ((size_t)gy * v.W + gx) * 3;
                c0 = cl[0];
                c1 = cl[1];
                c2 = cl[2];
            }
            float t0 = c0, t1 = c1, t2 = c2;
            if (in) {
                const int t = (gy / kTile - ty + 1) * 3 + (gx / kTile - tx + 1);   // 0..8 (the halo is < 1 tile)
                const int lx = gx % kTile, ly = gy % kTile;
                const int w = (ly / 4) * 2 + lx / 8, lane = (ly % 4) * 8 + lx % 8;
                if ((nb_mask[t][w] >> lane) & 1u) {
                    const float4 d = sb.deltas[(size_t)nb_gi[t][w] * 32 + lane];
                    t0 = d.x;
                    t1 = d.y;
                    t2 = d.z;
                }
            }
            s.x[0][r][c] = clamp01(t0);
            s.x[1][r][c] = clamp01(t1);
            s.x[2][r][c] = clamp01(t2);
            s.y[0][r][c] = clamp01(c0);
            s.y[1][r][c] = clamp01(c1);
            s.y[2][r][c] = clamp01(c2);
        }
        __syncthreads();
        block_add_ll(ssim_tile_pixel(s, w11, tx, ty, v.W, v.H), &acc[it.bk].ssim_fx);
    }
}


gs_status launch_ssim_full(const float* test, const float* clean, int W, int H, unsigned long long* acc,
                           cudaStream_t st) {
    const int tx = (W + kTile - 1) / kTile, ty = (H + kTile - 1) / kTile;
    if (tx * ty > 0) k_ssim_full<<<tx * ty, kTilePix, 0, st>>>(test, clean, W, H, tx, ssim_weights(), acc);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status launch_ssim_finalize(const unsigned long long* acc, int count, int W, int H, double* out, cudaStream_t st) {
    if (count > 0) k_ssim_finalize<<<(count + 255) / 256, 256, 0, st>>>(acc, count, W, H, out);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status launch_dirty_ssim(const void* dev_views, int K, const void* plan, const unsigned int* queue,
                            const SsimBufs& sb, CmpAcc* acc, cudaStream_t st) {
    k_dirty_ssim<<<num_sms() * 4, kTilePix, 0, st>>>((const ViewPtrs*)dev_views, K, (const PlanItem*)plan, queue, sb,
                                                     ssim_weights(), acc);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

// per (variant, view): SSIM = 1 - sum (1 - SSIM) / (3 x valid pixels)
__global__ void k_ssim_out(const CmpAcc* acc, int count, const ViewPtrs* views, int K, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const ViewPtrs& v = views[i % K];
    const double nvalid = 3.0 * (double)max(v.W - 2 * kSR, 0) * (double)max(v.H - 2 * kSR, 0);
    out[i] = nvalid > 0 ? 1.0 - (double)(long long)acc[i].ssim_fx * (1.0 / 4294967296.0) / nvalid : 1.0;
}

gs_status launch_ssim_out(const CmpAcc* acc, int count, const void* dev_views, int K, double* out, cudaStream_t st) {
    if (count > 0) k_ssim_out<<<(count + 255) / 256, 256, 0, st>>>(acc, count, (const ViewPtrs*)dev_views, K, out);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

}  // namespace gs

// SSIM of K image pairs (see gs.h)
extern "C" gs_status gs_ssim(const float* dev_test, const float* dev_clean, int H, int W, int K, double* dev_out,
                             void* stream) {
    using namespace gs;
    if (!dev_test || !dev_clean || !dev_out || H < 1 || W < 1 || K < 1)
        return set_error(GS_ERR_ARG, "bad gs_ssim arguments");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long* acc = nullptr;
    GS_CUDA(cudaMallocAsync((void**)&acc, sizeof(unsigned long long) * K, st));
    gs_status rs = GS_OK;
    if (cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * K, st) != cudaSuccess) rs = set_error(GS_ERR_CUDA, "memset");
    const size_t img = (size_t)H * W * 3;
    for (int k = 0; k < K && rs == GS_OK; k++) rs = launch_ssim_full(dev_test + k * img, dev_clean + k * img, W, H, acc + k, st);
    if (rs == GS_OK) rs = launch_ssim_finalize(acc, K, W, H, dev_out, st);
    cudaFreeAsync(acc, st);
    return rs;
}
