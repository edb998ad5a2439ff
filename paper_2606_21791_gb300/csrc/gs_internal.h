// Internal declarations shared by the libgs translation units (GPU path only).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/gs.h"

namespace gs {

// Render tiles are tw x th pixels, tw and th in {8, 16, 32} with 64 <= tw * th
// <= 256 (a scene's shape is set by gs_set_tile; 16 x 16 by default).  A tile's
// pixels are numbered in 8x4 blocks ("natural order"): pixel u = 32 w + lane of
// block w sits at (8 (w % nbx) + lane % 8, 4 (w / nbx) + lane / 8), nbx = tw / 8.
// The dirty-tile blend works on 8x8 blocks (one warp, two pixels per lane):
// block b is the 8x4 blocks wA = b % nbx + 2 nbx (b / nbx) and wA + nbx.
constexpr int kTile = 16;                   // default tile edge; the full-frame SSIM's own tile edge
constexpr int kTilePix = 256;               // most pixels in a tile
constexpr int kDirtyBlocks = kTilePix / 64; // most 8x8 blocks in a tile
__host__ __device__ inline bool tile_shape_ok(int tw, int th) {
    const bool ew = tw == 8 || tw == 16 || tw == 32, eh = th == 8 || th == 16 || th == 32;
    return ew && eh && tw * th >= 64 && tw * th <= kTilePix;
}
// log2 of the 8x4 blocks per tile row (tw / 8 = 1, 2, 4)
__host__ __device__ inline int tile_lgx(int tw) { return tw == 8 ? 0 : (tw == 16 ? 1 : 2); }
constexpr int kMaxWords = 59;
constexpr int kMaxPairs = 8192;       // (variant, view) pairs per dirty-tile launch (one scan block)
constexpr int kMaxBatch = 2048;       // variants per dirty-tile launch (also <= kMaxPairs / views)
// first bit of the sign and exponent bits a sign+exponent code protects
__host__ __device__ inline int ecc_first_bit(int fmt) { return fmt == GS_FP32 ? 23 : (fmt == GS_FP16 ? 10 : 7); }
constexpr int kSseFracBits = 39;      // fixed-point scale of per-pixel squared errors (3 * 2^39 * 5.1e6 px < 2^64)

// ----------------------------------------------------------------------------
// error reporting
// ----------------------------------------------------------------------------
gs_status set_error(gs_status st, const std::string& msg);
gs_status cuda_error(cudaError_t e, const char* what);
#define GS_CUDA(call)                                          \
    do {                                                       \
        cudaError_t _e = (call);                               \
        if (_e != cudaSuccess) return gs::cuda_error(_e, #call); \
    } while (0)
#define GS_TRY(call)                          \
    do {                                      \
        gs_status _s = (call);                \
        if (_s != GS_OK) return _s;           \
    } while (0)

inline int words_for_degree(int d) { return 14 + ((d + 1) * (d + 1) - 1) * 3; }
inline int word_bytes(int fmt) { return fmt == GS_FP32 ? 4 : 2; }
inline uint64_t div_up(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

// ----------------------------------------------------------------------------
// device-side records
// ----------------------------------------------------------------------------
// Blend record of one primitive in one view (48 B, 16-B aligned).  ex, ey are
// the half extents (pixels) of a box that contains every pixel centre where the
// primitive's alpha can reach 1/255 (NaN if the opacity is NaN: never culled;
// negative if it can never reach 1/255).
struct __align__(16) BlendRec {
    float mx, my, ca, cb;
    float cc, opac, ex, ey;
    float r, g, b, depth;
};

// Camera with the per-view constants the preprocess needs.
struct DevCamera {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int W, H;
    float znear, zfar;
    int tiles_x, tiles_y;
    int tile_w, tile_h;   // render tile shape
};

// Per (variant, view) comparison accumulator (integer/ordered atomics only, so
// the result does not depend on the order in which tiles finish).
struct CmpAcc {
    unsigned long long sse_fx;  // sum of per-pixel squared errors, each rounded to fixed point 2^-kSseFracBits
    unsigned int maxabs_bits;   // float bits of the max |diff| (non-negative floats order as uints)
    unsigned int footprint;
    unsigned int nonfinite;
    unsigned int clamps;
    unsigned int clean_nonfinite_replaced;   // dirty engine: re-blended pixels whose clean value was non-finite
    unsigned int pad;
    unsigned long long reg_actual;   // dirty engine: 8x8 screen cells holding a footprint pixel
    unsigned long long reg_pred;     // dirty engine: cells met by the changed primitive's tile rects
    unsigned long long ssim_fx;      // sum over pixels and channels of (1 - SSIM), fixed point 2^-32 (signed)
};

// Screen cells of the contamination masks: an 8x8 grid, cell of pixel (x, y) =
// (8x / W, 8y / H), bit 8 cy + cx.
__host__ __device__ inline unsigned long long cell_bit(int x, int y, int W, int H) {
    // x < W <= 65535 * 16, so 8 x fits 32 bits
    const int cx = (int)((unsigned)x * 8u / (unsigned)W), cy = (int)((unsigned)y * 8u / (unsigned)H);
    return 1ull << (cy * 8 + cx);
}
// cells met by the pixels of a tile rect (packed x0 | y0 << 16, x1 | y1 << 16, half
// open in tiles of tw x th pixels)
__host__ __device__ inline unsigned long long rect_cells(uint2 rect, int W, int H, int tw, int th) {
    const int x0 = rect.x & 0xffff, y0 = rect.x >> 16, x1 = rect.y & 0xffff, y1 = rect.y >> 16;
    if (x1 <= x0 || y1 <= y0) return 0ull;
    const int px1 = min(x1 * tw, W) - 1, py1 = min(y1 * th, H) - 1;
    const int cx0 = (int)(((long long)x0 * tw * 8) / W), cx1 = (int)(((long long)px1 * 8) / W);
    const int cy0 = (int)(((long long)y0 * th * 8) / H), cy1 = (int)(((long long)py1 * 8) / H);
    unsigned long long m = 0ull;
    for (int cy = cy0; cy <= cy1; cy++)
        for (int cx = cx0; cx <= cx1; cx++) m |= 1ull << (cy * 8 + cx);
    return m;
}

struct ViewPtrs {
    const BlendRec* recs;
    const uint32_t* ids;
    const uint32_t* dk;      // depth bits of ids[j] (list-aligned)
    const uint2* ranges;
    const float* clean;
    const uint32_t* stop;    // clean stop index of every pixel
    const uint32_t* tile_stop;   // largest stop index of each tile
    const unsigned long long* stop_key;   // (depth bits, id) of the list entry at tile_stop; ~0 if none
    const uint32_t* bl_off;      // per (tile, 8x8 block): start of its sublist in bl_pos (ntiles * kDirtyBlocks + 1)
    const uint32_t* bl_pos;      // positions (in the tile's list) of the entries whose box meets the block
    const BlendRec* bl_rec;      // their records, same order
    const float4* ck;            // clean-blend checkpoints (T, C) of every pixel
    const uint32_t* ck_off;      // first checkpoint of each tile
    const uint32_t* ck_cnt;      // checkpoints of each tile (after kCkStride, 2 kCkStride, ... entries)
    int W, H, tiles_x, tile_w, tile_h, pad[3];
};

// One dirty tile that needs re-blending (112 B).  ins is the insertion position
// in the clean list without the primitive's old entry; cut is the first changed
// position of the clean list; rec is the corrupted record (when flags bit 1);
// mask marks the tile's active pixels (natural order, 8 x 32 bits).
struct __align__(16) PlanItem {
    BlendRec rec;
    uint32_t mask[kTilePix / 32];
    uint32_t bk;      // (variant, view) = variant * K + view
    uint32_t tile;
    uint32_t s, e;    // clean list range
    uint32_t pp, ins, cut;
    uint32_t flags;   // bit 0: old entry in this tile, bit 1: corrupted entry in this tile
};
static_assert(sizeof(PlanItem) == 112 && offsetof(PlanItem, mask) == 48 && offsetof(PlanItem, bk) == 80 &&
                  offsetof(PlanItem, pp) == 96,
              "k_plan writes PlanItem as 7 16-byte parts");

// Buffers of the dirty-tile SSIM (all NULL when it is off): per plan slot the
// delta index of each of its 8x4 blocks (0xffffffff: none), per delta index the
// new values of the block's 32 pixels, per (variant, view) and tile the plan
// slot (generation << 32 | slot) and the SSIM claim (generation << 32).
struct SsimBufs {
    uint32_t* slot_group;              // [slot_cap * 8]
    uint32_t* slot_flags;              // [slot_cap] changed pixels: bit 4 any, 0-3 within 5 of the left/right/top/bottom edge
    float4* deltas;                    // [delta_cap * 32]
    unsigned long long* tile_map;      // [B*K * max_tiles]
    unsigned long long* ssim_map;      // [B*K * max_tiles]
    unsigned int* overflow;            // set when a capacity is exceeded
    uint32_t slot_cap, delta_cap, max_tiles, pad;
};

// Dirty-tile work descriptor of one (variant, view).
struct DirtyDesc {
    BlendRec rec;          // corrupted primitive's record
    uint32_t prim;
    int32_t new_vis;       // corrupted primitive binned?
    int32_t old_vis;       // clean primitive binned?
    uint32_t n_items;      // dirty tiles
    uint16_t nx0, ny0, nx1, ny1;   // corrupted rect
    uint16_t ox0, oy0, ox1, oy1;   // clean rect
    float old_depth;       // clean primitive's depth (when old_vis)
    uint32_t pad[3];
};

// ----------------------------------------------------------------------------
// per-view clean state and scratch
// ----------------------------------------------------------------------------
struct ViewState {
    DevCamera cam{};
    BlendRec* recs = nullptr;        // [n]
    uint2* rects = nullptr;          // [n] (x0 | y0 << 16, x1 | y1 << 16)
    uint32_t* ids = nullptr;         // [npairs] sorted tile lists
    uint32_t* dk = nullptr;          // [npairs] depth bits of ids[j]
    uint2* ranges = nullptr;         // [ntiles] (start, end)
    float* clean = nullptr;          // [H*W*3]
    uint32_t* stop = nullptr;        // [H*W] list index that stopped each clean pixel
    uint32_t* tile_stop = nullptr;   // [ntiles] largest stop index in each tile
    unsigned long long* stop_key = nullptr;   // [ntiles] (depth bits << 32 | id) of the entry at tile_stop (~0: none)
    uint32_t* bl_off = nullptr;      // [ntiles * kDirtyBlocks + 1] start of each (tile, 8x8 block) sublist in bl_pos
    uint32_t* bl_pos = nullptr;      // list positions whose box meets the block, ascending per sublist
    BlendRec* bl_rec = nullptr;      // the records of those entries, in the same order (streamed by the blend)
    float4* ck = nullptr;            // clean-blend checkpoints [total][pixels of a tile]
    uint32_t* ck_off = nullptr;      // [ntiles]
    uint32_t* ck_cnt = nullptr;      // [ntiles]
    uint64_t ck_total = 0;
    uint64_t npairs = 0;
    uint64_t cap_pairs = 0;
};

// Scratch of the full render pipeline for one view.
struct RenderWork {
    uint64_t n = 0;
    uint64_t cap_pairs = 0;
    int ntiles_cap = 0;
    BlendRec* recs = nullptr;
    uint2* rects = nullptr;
    uint32_t* dkey[2] = {nullptr, nullptr};    // depth keys (ping-pong)
    uint32_t* dval[2] = {nullptr, nullptr};    // primitive ids (ping-pong)
    uint32_t* cnt = nullptr;                    // tiles per primitive, in depth order
    uint32_t* off = nullptr;                    // exclusive scan of cnt
    uint32_t* pkey[2] = {nullptr, nullptr};    // pair tile keys
    uint32_t* pval[2] = {nullptr, nullptr};    // pair primitive ids
    uint32_t* hist = nullptr;                   // radix histograms
    unsigned long long* hpart = nullptr;        // block partials of the histogram scan
    uint32_t* scan_tmp = nullptr;               // block sums for scans
    uint2* ranges = nullptr;
    unsigned long long* total = nullptr;        // [0] pair count, [1] overflow flag
    unsigned long long* host_total = nullptr;   // pinned mirror
    int passes[2] = {0, 0};                     // radix passes of the last build: depth keys, pair tile keys
};

struct GraphEntry {
    int B = 0;
    int guard = -2;
    uint64_t mask = 0;
    bool ssim = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

}  // namespace gs

struct gs_scene {
    uint64_t n = 0;
    int sh_degree = 0;
    int fmt = 0;
    int nwords = 0;
    void* planes = nullptr;                 // [nwords][n]
    uint32_t box_lo[gs::kMaxWords] = {};    // FIELD box (storage words)
    uint32_t box_hi[gs::kMaxWords] = {};
    void* pbox_lo = nullptr;                // PRIM box planes [nbox][n]
    void* pbox_hi = nullptr;
    int nbox_words = 0;
    uint32_t* dev_box = nullptr;            // FIELD box on device: lo[59], hi[59]
    unsigned int* dev_err = nullptr;        // sticky device error flags (bit 0: bad flip site)
    unsigned long long* dev_clamps = nullptr;

    // clean per-view state of the campaign
    int K = 0;
    std::vector<gs::ViewState> views;
    gs::DevCamera* dev_cams = nullptr;
    void* dev_views = nullptr;              // ViewPtrs[K]
    void* dev_clean_rects = nullptr;        // const uint2*[K]
    void* dev_clean_recs = nullptr;         // const BlendRec*[K]
    uint64_t full_cap_pairs = 0;
    int max_tiles = 0;
    gs::RenderWork work;                    // scratch of the full render pipeline
    int tile_w = gs::kTile, tile_h = gs::kTile;   // render tile shape (gs_set_tile)
    std::vector<gs_camera> host_cams;       // the cameras of gs_set_views (rebuilt on a tile change)

    // batch buffers (dirty engine and plain loop)
    int cap_B = 0;
    int cap_flips = 0;
    gs_flip* flip_stage = nullptr;
    gs_flip* host_io_flips = nullptr;       // device copies of gs_inject_and_render_host's inputs / outputs
    gs_result* host_io_out = nullptr;
    size_t host_io_flips_cap = 0, host_io_out_cap = 0;
    gs::DirtyDesc* desc = nullptr;
    uint32_t* item_off = nullptr;
    gs::CmpAcc* acc = nullptr;
    gs_result* res_stage = nullptr;
    unsigned int* queue = nullptr;
    void* plan = nullptr;                   // dirty tiles to re-blend (PlanItem[plan_cap])
    uint2* cand = nullptr;                  // candidate tiles of the plan's first pass [plan_cap]
    uint32_t* groups = nullptr;             // 8x8 pixel blocks to re-blend, (item << 3) | block [kDirtyBlocks * plan_cap]
    gs::SsimBufs ssim{};                    // dirty-tile SSIM buffers (allocated on first use, else NULL)
    uint64_t plan_cap = 0;
    unsigned int* clean_nonfin = nullptr;   // [K] non-finite pixels of each clean view
    uint32_t* saved = nullptr;
    bool use_graphs = true;
    int batch = 0;                          // variants per dirty-tile launch (0: default)
    unsigned long long* work_ctr = nullptr; // work counters, non-NULL while counting is on (no graphs then)
    cudaEvent_t ev_k0 = nullptr;            // timing on: before the plan kernel of the last batch,
    cudaEvent_t ev_kp = nullptr;            // between the plan and the blend kernel,
    cudaEvent_t ev_k1 = nullptr;            // after the blend kernel
    cudaEvent_t ev_r[4] = {};               // timing on, gs_render: before preprocess, after it, after the tile
                                            // lists, after the blend (last view of the last call)
    bool render_timed = false;              // ev_r holds a complete record
    uint64_t render_pairs = 0;              // tile pairs of that view
    std::vector<gs::GraphEntry> graphs;
};

namespace gs {

// k_guard.cu
int num_sms();
gs_status launch_field_box(const void* planes, int fmt, uint64_t n, int nwords, uint32_t* dev_keys, cudaStream_t st);
gs_status launch_guard(gs_scene* s, int mode, uint64_t mask, unsigned long long* dev_clamps, cudaStream_t st);
gs_status launch_guard_mark(gs_scene* s, int mode, uint64_t mask, uint32_t* bitmap, cudaStream_t st);
gs_status launch_save_sites(const void* planes, int fmt, uint64_t n, int nwords, const gs_flip* flips, int count,
                            uint32_t* saved, cudaStream_t st);
gs_status launch_restore_sites(void* planes, int fmt, uint64_t n, int nwords, const gs_flip* flips, int count,
                               const uint32_t* saved, cudaStream_t st);

// k_preprocess.cu
DevCamera make_dev_camera(const gs_camera& c, int tile_w, int tile_h);

// gs_api.cu: the camera sizes and focal lengths the kernels accept
bool valid_camera(const gs_camera& c);

// k_sort.cu
gs_status alloc_render_work(RenderWork& w, uint64_t n, uint64_t cap_pairs, int ntiles);
void free_render_work(RenderWork& w);
gs_status launch_rects_to_keys(const float* depth, const int32_t* rects, uint64_t n, int tiles_x, int tiles_y,
                               uint32_t* keys, uint32_t* vals, uint2* prects, cudaStream_t st);

// k_blend.cu (full-frame kernels take the view's camera for its size and tile shape)
gs_status launch_blend_image(const BlendRec* recs, const uint32_t* ids, const uint2* ranges, const DevCamera& cam,
                             float* img, cudaStream_t st);
gs_status launch_blend_compare(const BlendRec* recs, const uint32_t* ids, const uint2* ranges, const DevCamera& cam,
                               const float* clean, CmpAcc* acc, unsigned long long* work, cudaStream_t st);
gs_status launch_compare(const float* a, const float* b, int H, int W, CmpAcc* acc, cudaStream_t st);
gs_status launch_finalize(const CmpAcc* acc, int count, gs_result* out, cudaStream_t st);
gs_status launch_records_to_blend(const gs_record* in, uint64_t n, BlendRec* out, cudaStream_t st);

}  // namespace gs
