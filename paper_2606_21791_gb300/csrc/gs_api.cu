// C ABI of libgs: scene lifetime, the full render pipeline, the batched
// dirty-tile injection campaign (captured in CUDA graphs), the plain
// one-variant-at-a-time loop, and stage entry points.  All device work is done
// by the kernels in k_*.cu; this file only orchestrates.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "gs_internal.h"

namespace gs {

// implemented in the kernel translation units
gs_status launch_apply_flips(void* planes, int fmt, uint64_t n, int nwords, const gs_flip* flips, int64_t count,
                             unsigned int* err, uint64_t ecc_mask, cudaStream_t st);
gs_status launch_preprocess(const gs_scene* s, const DevCamera& cam, BlendRec* recs, uint2* rects, uint32_t* keys,
                            uint32_t* vals, gs_record* dbg, cudaStream_t st);
gs_status launch_inject_prep(const gs_scene* s, const DevCamera* dev_cams, int K, const gs_flip* flips, int B,
                             int guard_mode, uint64_t mask, const uint2* const* dev_clean_rects,
                             const BlendRec* const* dev_clean_recs, DirtyDesc* desc, uint32_t* item_off, CmpAcc* acc,
                             unsigned int* queue, cudaStream_t st);
gs_status build_tile_lists(RenderWork& w, uint64_t n, int tiles_x, int tiles_y, uint32_t** ids_out, cudaStream_t st);
gs_status launch_ranges_to_offsets(const uint2* ranges, int ntiles, uint32_t* offsets, const unsigned long long* total,
                                   cudaStream_t st);
gs_status launch_zero_acc(CmpAcc* acc, int count, cudaStream_t st);
gs_status launch_dirty_blend(const void* dev_views, const DirtyDesc* desc, const uint32_t* item_off, int BK, int K,
                             void* plan, uint2* cand, uint32_t* groups, uint32_t gcap, CmpAcc* acc,
                             unsigned int* queue, unsigned long long* work, cudaEvent_t ev_mid, const SsimBufs& sb,
                             cudaStream_t st);
gs_status launch_ssim_out(const CmpAcc* acc, int count, const void* dev_views, int K, double* out, cudaStream_t st);
gs_status launch_regions_out(const CmpAcc* acc, int count, unsigned long long* out, cudaStream_t st);
gs_status launch_finalize_dirty(const CmpAcc* acc, int count, gs_result* out, const unsigned int* clean_nonfin, int K,
                                cudaStream_t st);
size_t plan_item_size();
size_t view_ptrs_size();
gs_status launch_stop_keys(const uint2* ranges, const uint32_t* tile_stop, const uint32_t* dk, const uint32_t* ids,
                           int ntiles, unsigned long long* out, cudaStream_t st);
void fill_view_ptrs(void* host_dst, const ViewState& vs);
gs_status launch_blists(const BlendRec* recs, const uint32_t* ids, const uint2* ranges, const DevCamera& cam,
                        uint32_t* counts, const uint32_t* off, uint32_t* pos, BlendRec* brec, cudaStream_t st);
gs_status launch_exclusive_scan(const uint32_t* in, uint64_t n, uint32_t* out, unsigned long long* scratch,
                                unsigned long long* total, cudaStream_t st);
uint64_t scan_scratch_len(uint64_t n);
gs_status launch_blend_image_stop(const BlendRec* recs, const uint32_t* ids, const uint2* ranges, const DevCamera& cam,
                                  float* img, uint32_t* stop, uint32_t* tile_stop, float4* ck, const uint32_t* ck_off,
                                  const uint32_t* ck_cnt, unsigned int* clean_nonfin, cudaStream_t st);
int ck_stride_value();
int ck_max_per_tile();
gs_status launch_gather_depth(const BlendRec* recs, const uint32_t* ids, uint64_t n, uint32_t* dk, cudaStream_t st);
gs_status launch_offsets_to_ranges(const uint32_t* offsets, int ntiles, uint2* ranges, cudaStream_t st);
uint32_t key_to_bits(uint32_t key, int fmt);
int dirty_grid();

static thread_local std::string g_last_error;

gs_status set_error(gs_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

gs_status cuda_error(cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return set_error(GS_ERR_OOM, m);
    return set_error(GS_ERR_CUDA, m);
}

// the camera sizes and focal lengths the kernels accept (tile coordinates fit 16
// bits for the smallest tile edge, 8)
bool valid_camera(const gs_camera& c) {
    return c.width > 0 && c.height > 0 && c.width <= 65535 * 8 && c.height <= 65535 * 8 && c.fx > 0 &&
           c.fy > 0 && std::isfinite(c.fx) && std::isfinite(c.fy);
}

namespace {

__global__ void k_move_clamps(unsigned long long* ctr, CmpAcc* acc) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        acc->clamps = (unsigned int)(*ctr < 0xffffffffull ? *ctr : 0xffffffffull);
        *ctr = 0ull;
    }
}

gs_status dmalloc(void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(GS_ERR_OOM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
    return GS_OK;
}

// Full render pipeline of one view on scratch `w`: preprocess, depth sort,
// pair emission, tile sort, ranges.  Leaves records in w.recs, lists in *ids.
// ev (optional, 3 events): recorded before the preprocess, after it and after the tile lists.
gs_status render_lists(gs_scene* s, RenderWork& w, const DevCamera& cam, uint32_t** ids, cudaStream_t st,
                       cudaEvent_t* ev = nullptr) {
    if (ev) GS_CUDA(cudaEventRecord(ev[0], st));
    GS_TRY(launch_preprocess(s, cam, w.recs, w.rects, w.dkey[0], w.dval[0], nullptr, st));
    if (ev) GS_CUDA(cudaEventRecord(ev[1], st));
    GS_TRY(build_tile_lists(w, s->n, cam.tiles_x, cam.tiles_y, ids, st));
    if (ev) GS_CUDA(cudaEventRecord(ev[2], st));
    return GS_OK;
}

// Like render_lists but grows the pair capacity until the lists fit (host sync).
gs_status render_lists_sized(gs_scene* s, RenderWork& w, const DevCamera& cam, uint32_t** ids, uint64_t* npairs,
                             cudaStream_t st, cudaEvent_t* ev = nullptr) {
    int ntiles = cam.tiles_x * cam.tiles_y;
    uint64_t cap = std::max<uint64_t>(w.cap_pairs, std::max<uint64_t>(s->n * 2, 1024));
    for (int attempt = 0; attempt < 4; attempt++) {
        GS_TRY(alloc_render_work(w, s->n, cap, ntiles));
        GS_TRY(render_lists(s, w, cam, ids, st, ev));
        GS_CUDA(cudaMemcpyAsync(w.host_total, w.total, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        w.host_total[3] = 0ull;
        GS_CUDA(cudaMemcpyAsync(&w.host_total[3], s->dev_err, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
        GS_CUDA(cudaStreamSynchronize(st));
        if (w.host_total[3] & 2ull)
            return set_error(GS_ERR_TIMEOUT, "a bounded wait of the preprocess gave up (device error word bit 1)");
        if (!w.host_total[1]) {
            *npairs = w.host_total[0];
            return GS_OK;
        }
        uint64_t need = w.host_total[2];
        if (need >= 0xffffffffull) return set_error(GS_ERR_CAPACITY, "tile pair count exceeds 2^32");
        cap = need + need / 4 + 1024;
    }
    return set_error(GS_ERR_CAPACITY, "could not size the tile pair buffers");
}

void destroy_graphs(gs_scene* s) {
    for (auto& g : s->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
    }
    s->graphs.clear();
}

void free_ssim_buffers(gs_scene* s);

void free_views(gs_scene* s) {
    destroy_graphs(s);
    free_ssim_buffers(s);
    for (auto& v : s->views) {
        cudaFree(v.recs);
        cudaFree(v.rects);
        cudaFree(v.ids);
        cudaFree(v.dk);
        cudaFree(v.ranges);
        cudaFree(v.clean);
        cudaFree(v.stop);
        cudaFree(v.tile_stop);
        cudaFree(v.stop_key);
        cudaFree(v.bl_off);
        cudaFree(v.bl_pos);
        cudaFree(v.bl_rec);
        cudaFree(v.ck);
        cudaFree(v.ck_off);
        cudaFree(v.ck_cnt);
    }
    s->views.clear();
    s->K = 0;
    cudaFree(s->dev_cams);
    cudaFree(s->dev_views);
    cudaFree(s->dev_clean_rects);
    cudaFree(s->dev_clean_recs);
    cudaFree(s->clean_nonfin);
    s->clean_nonfin = nullptr;
    s->dev_cams = nullptr;
    s->dev_views = nullptr;
    s->dev_clean_rects = nullptr;
    s->dev_clean_recs = nullptr;
}

void free_ssim_buffers(gs_scene* s) {
    cudaFree(s->ssim.slot_group);
    cudaFree(s->ssim.slot_flags);
    cudaFree(s->ssim.deltas);
    cudaFree(s->ssim.tile_map);
    cudaFree(s->ssim.ssim_map);
    cudaFree(s->ssim.overflow);
    s->ssim = SsimBufs{};
}

// SSIM buffers sized for the current batch capacity (zeroed: generation 0 is never current)
static gs_status alloc_ssim_buffers(gs_scene* s) {
    const int K = std::max(s->K, 1);
    SsimBufs b{};
    b.slot_cap = (uint32_t)std::min<uint64_t>(s->plan_cap, 1ull << 18);
    b.delta_cap = (uint32_t)std::min<uint64_t>((kTilePix / 32) * s->plan_cap, 1ull << 19);
    b.max_tiles = (uint32_t)std::max(s->max_tiles, 1);
    const size_t maps = (size_t)s->cap_B * K * b.max_tiles;
    s->ssim = b;   // caps now; pointers below
    GS_TRY(dmalloc((void**)&s->ssim.slot_group, sizeof(uint32_t) * 8 * b.slot_cap));
    GS_TRY(dmalloc((void**)&s->ssim.slot_flags, sizeof(uint32_t) * b.slot_cap));
    GS_TRY(dmalloc((void**)&s->ssim.deltas, sizeof(float4) * 32 * (size_t)b.delta_cap));
    GS_TRY(dmalloc((void**)&s->ssim.tile_map, sizeof(unsigned long long) * maps));
    GS_TRY(dmalloc((void**)&s->ssim.ssim_map, sizeof(unsigned long long) * maps));
    GS_TRY(dmalloc((void**)&s->ssim.overflow, sizeof(unsigned int)));
    GS_CUDA(cudaMemset(s->ssim.tile_map, 0, sizeof(unsigned long long) * maps));
    GS_CUDA(cudaMemset(s->ssim.ssim_map, 0, sizeof(unsigned long long) * maps));
    GS_CUDA(cudaMemset(s->ssim.overflow, 0, sizeof(unsigned int)));
    return GS_OK;
}

// All or nothing: a set tile_map means every SSIM buffer is allocated and zeroed.
gs_status ensure_ssim_buffers(gs_scene* s) {
    if (s->ssim.tile_map) return GS_OK;
    const gs_status rs = alloc_ssim_buffers(s);
    if (rs != GS_OK) free_ssim_buffers(s);
    return rs;
}

gs_status ensure_batch_buffers(gs_scene* s, int B, int fpv) {
    int K = std::max(s->K, 1);
    if (B <= s->cap_B && fpv * B <= s->cap_flips) return GS_OK;
    destroy_graphs(s);
    free_ssim_buffers(s);
    cudaFree(s->flip_stage);
    cudaFree(s->desc);
    cudaFree(s->item_off);
    cudaFree(s->acc);
    cudaFree(s->res_stage);
    cudaFree(s->queue);
    cudaFree(s->saved);
    cudaFree(s->plan);
    cudaFree(s->cand);
    cudaFree(s->groups);
    s->flip_stage = nullptr;
    s->desc = nullptr;
    s->item_off = nullptr;
    s->acc = nullptr;
    s->res_stage = nullptr;
    s->queue = nullptr;
    s->saved = nullptr;
    s->plan = nullptr;
    s->cand = nullptr;
    s->groups = nullptr;
    const int cb = std::max(B, s->cap_B);
    const int cf = std::max(fpv * B, s->cap_flips);
    // no capacity until every buffer below is allocated: a failure part way (out
    // of memory) leaves nothing that a later call could take for usable
    s->cap_B = 0;
    s->cap_flips = 0;
    s->plan_cap = 0;
    GS_TRY(dmalloc((void**)&s->flip_stage, sizeof(gs_flip) * cf));
    GS_TRY(dmalloc((void**)&s->desc, sizeof(DirtyDesc) * cb * K));
    GS_TRY(dmalloc((void**)&s->item_off, sizeof(uint32_t) * (2 * cb * K + 1)));   // offsets + per-pair counts
    GS_TRY(dmalloc((void**)&s->acc, sizeof(CmpAcc) * cb * K));
    GS_TRY(dmalloc((void**)&s->res_stage, sizeof(gs_result) * cb * K));
    GS_TRY(dmalloc((void**)&s->queue, sizeof(unsigned int) * 8));
    GS_CUDA(cudaMemset(s->queue, 0, sizeof(unsigned int) * 8));   // queue[6]: batch generation
    GS_TRY(dmalloc((void**)&s->saved, sizeof(uint32_t) * cf));
    // every (variant, view) can dirty at most every tile of its view
    s->plan_cap = (uint64_t)cb * K * (uint64_t)std::max(s->max_tiles, 1);
    // groups are coded (plan slot << 3) | block in 32 bits
    if (s->plan_cap >= (1ull << 29)) return set_error(GS_ERR_CAPACITY, "too many dirty tiles per batch for this view size");
    GS_TRY(dmalloc(&s->plan, plan_item_size() * s->plan_cap));
    GS_TRY(dmalloc((void**)&s->cand, sizeof(uint2) * s->plan_cap));
    GS_TRY(dmalloc((void**)&s->groups, sizeof(uint32_t) * kDirtyBlocks * s->plan_cap));
    s->cap_B = cb;
    s->cap_flips = cf;
    return GS_OK;
}

// Variants per dirty-tile launch: the injector's scan covers at most 1024
// (variant, view) pairs in one block.
int max_batch(int K) { return std::max(1, std::min(kMaxBatch, kMaxPairs / K)); }

gs_status check_flip_args(gs_scene* s, const gs_flip* flips, int B, int fpv, int guard_mode, uint64_t mask) {
    if (!s || (!flips && B > 0) || B < 0 || fpv < 1) return set_error(GS_ERR_ARG, "bad campaign arguments");
    if (s->K == 0 || s->views.empty()) return set_error(GS_ERR_STATE, "gs_set_views was not called");
    if (guard_mode < -1 || guard_mode > 2) return set_error(GS_ERR_ARG, "guard_mode must be -1, 0, 1 or 2");
    if (guard_mode == GS_GUARD_PRIM) {
        if (!s->pbox_lo) return set_error(GS_ERR_STATE, "no per-primitive box set");
        uint64_t allowed = s->nbox_words >= 64 ? ~0ull : ((1ull << s->nbox_words) - 1ull);
        if (mask & ~allowed) return set_error(GS_ERR_ARG, "PRIM guard mask covers words without boxes");
    }
    return GS_OK;
}

// enqueue one dirty-tile batch (B <= cap_B, flips already in flip_stage)
gs_status enqueue_dirty(gs_scene* s, int B, int guard_mode, uint64_t mask, bool ssim, cudaStream_t st) {
    int K = s->K;
    GS_TRY(launch_inject_prep(s, s->dev_cams, K, s->flip_stage, B, guard_mode, mask,
                              (const uint2* const*)s->dev_clean_rects, (const BlendRec* const*)s->dev_clean_recs,
                              s->desc, s->item_off, s->acc, s->queue, st));
    // external records: inside a stream capture they become event-record nodes of the graph
    if (s->ev_k0) GS_CUDA(cudaEventRecordWithFlags(s->ev_k0, st, cudaEventRecordExternal));
    const SsimBufs sb = ssim ? s->ssim : SsimBufs{};
    GS_TRY(launch_dirty_blend(s->dev_views, s->desc, s->item_off, B * K, K, s->plan, s->cand, s->groups,
                              (uint32_t)(kDirtyBlocks * s->plan_cap), s->acc, s->queue, s->work_ctr, s->ev_kp, sb,
                              st));
    if (s->ev_k1) GS_CUDA(cudaEventRecordWithFlags(s->ev_k1, st, cudaEventRecordExternal));
    GS_TRY(launch_finalize_dirty(s->acc, B * K, s->res_stage, s->clean_nonfin, K, st));
    return GS_OK;
}

gs_status run_dirty_batch(gs_scene* s, int B, int guard_mode, uint64_t mask, bool ssim, cudaStream_t st) {
    if (!s->use_graphs || s->work_ctr) return enqueue_dirty(s, B, guard_mode, mask, ssim, st);
    GraphEntry* ge = nullptr;
    for (auto& g : s->graphs)
        if (g.B == B && g.guard == guard_mode && g.mask == mask && g.ssim == ssim) ge = &g;
    if (!ge) {
        dirty_grid();   // occupancy query outside the capture
        cudaStream_t cs;
        GS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        GraphEntry g;
        g.B = B;
        g.guard = guard_mode;
        g.mask = mask;
        g.ssim = ssim;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cs);
            return cuda_error(e, "cudaStreamBeginCapture");
        }
        gs_status qs = enqueue_dirty(s, B, guard_mode, mask, ssim, cs);
        e = cudaStreamEndCapture(cs, &g.graph);
        cudaStreamDestroy(cs);
        if (qs != GS_OK) {
            if (g.graph) cudaGraphDestroy(g.graph);
            return qs;
        }
        if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&g.exec, g.graph, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g.graph);
            return cuda_error(e, "cudaGraphInstantiate");
        }
        s->graphs.push_back(g);
        ge = &s->graphs.back();
    }
    GS_CUDA(cudaGraphLaunch(ge->exec, st));
    return GS_OK;
}

}  // namespace

gs_status render_lists_sized_ext(gs_scene* s, RenderWork& w, const DevCamera& cam, uint32_t** ids, uint64_t* npairs,
                                 cudaStream_t st) {
    return render_lists_sized(s, w, cam, ids, npairs, st);
}

}  // namespace gs

using namespace gs;

extern "C" {

const char* gs_last_error(void) { return g_last_error.c_str(); }

const char* gs_version(void) { return "libgs 0.1 (sm_103a)"; }

gs_status gs_load_scene(const void* planes, int src_on_device, uint64_t n, int sh_degree, gs_format fmt,
                        gs_scene** out) {
    if (!out) return set_error(GS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (sh_degree < 0 || sh_degree > 3) return set_error(GS_ERR_ARG, "sh_degree must be 0..3");
    if (fmt != GS_FP32 && fmt != GS_FP16 && fmt != GS_BF16) return set_error(GS_ERR_ARG, "unknown storage format");
    if (n > 0xffffffffull) return set_error(GS_ERR_ARG, "at most 2^32 - 1 primitives");
    if (n > 0 && !planes) return set_error(GS_ERR_ARG, "planes is NULL");
    gs_scene* s = new gs_scene();
    s->n = n;
    s->sh_degree = sh_degree;
    s->fmt = fmt;
    s->nwords = words_for_degree(sh_degree);
    size_t bytes = (size_t)n * s->nwords * word_bytes(fmt);
    // rounded up to 16 bytes: 16-bit words are flipped with 32-bit atomics on
    // the aligned word that contains them
    gs_status st = dmalloc(&s->planes, (bytes + 15) & ~(size_t)15);
    if (st == GS_OK) st = dmalloc((void**)&s->dev_box, sizeof(uint32_t) * 2 * kMaxWords);
    if (st == GS_OK) st = dmalloc((void**)&s->dev_err, sizeof(unsigned int) * 4);
    if (st == GS_OK) st = dmalloc((void**)&s->dev_clamps, sizeof(unsigned long long) * 2);
    if (st != GS_OK) {
        gs_free_scene(s);
        return st;
    }
    cudaError_t e = cudaMemcpy(s->planes, planes, bytes, src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(s->dev_err, 0, sizeof(unsigned int) * 4);
    if (e == cudaSuccess) e = cudaMemset(s->dev_clamps, 0, sizeof(unsigned long long) * 2);
    if (e != cudaSuccess) {
        gs_free_scene(s);
        return cuda_error(e, "gs_load_scene copy");
    }
    // Algorithm 1 precompute: per-word min/max box
    st = launch_field_box(s->planes, fmt, n, s->nwords, s->dev_box, 0);
    uint32_t keys[2 * kMaxWords];
    if (st == GS_OK) {
        e = cudaMemcpy(keys, s->dev_box, sizeof(keys), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_error(e, "field box readback");
    }
    if (st != GS_OK) {
        gs_free_scene(s);
        return st;
    }
    for (int w = 0; w < s->nwords; w++) {
        if (keys[w] == 0xffffffffu && keys[kMaxWords + w] == 0u) {   // no finite... no non-NaN value
            s->box_lo[w] = s->box_hi[w] = 0u;
        } else {
            s->box_lo[w] = key_to_bits(keys[w], fmt);
            s->box_hi[w] = key_to_bits(keys[kMaxWords + w], fmt);
        }
        keys[w] = s->box_lo[w];
        keys[kMaxWords + w] = s->box_hi[w];
    }
    e = cudaMemcpy(s->dev_box, keys, sizeof(keys), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        gs_free_scene(s);
        return cuda_error(e, "field box upload");
    }
    *out = s;
    return GS_OK;
}

gs_status gs_free_scene(gs_scene* s) {
    if (!s) return GS_OK;
    free_views(s);
    free_render_work(s->work);
    cudaFree(s->planes);
    cudaFree(s->pbox_lo);
    cudaFree(s->pbox_hi);
    cudaFree(s->dev_box);
    cudaFree(s->dev_err);
    cudaFree(s->dev_clamps);
    cudaFree(s->flip_stage);
    cudaFree(s->host_io_flips);
    cudaFree(s->host_io_out);
    cudaFree(s->desc);
    cudaFree(s->item_off);
    cudaFree(s->acc);
    cudaFree(s->res_stage);
    cudaFree(s->queue);
    cudaFree(s->saved);
    cudaFree(s->plan);
    cudaFree(s->cand);
    cudaFree(s->groups);
    free_ssim_buffers(s);
    cudaFree(s->clean_nonfin);
    cudaFree(s->work_ctr);
    if (s->ev_k0) cudaEventDestroy(s->ev_k0);
    if (s->ev_kp) cudaEventDestroy(s->ev_kp);
    if (s->ev_k1) cudaEventDestroy(s->ev_k1);
    for (auto& e : s->ev_r)
        if (e) cudaEventDestroy(e);
    delete s;
    return GS_OK;
}

gs_status gs_scene_info(const gs_scene* s, uint64_t* n, int* sh_degree, int* fmt, int* nwords) {
    if (!s) return set_error(GS_ERR_ARG, "scene is NULL");
    if (n) *n = s->n;
    if (sh_degree) *sh_degree = s->sh_degree;
    if (fmt) *fmt = s->fmt;
    if (nwords) *nwords = s->nwords;
    return GS_OK;
}

gs_status gs_scene_planes(gs_scene* s, void** dev_planes) {
    if (!s || !dev_planes) return set_error(GS_ERR_ARG, "NULL argument");
    *dev_planes = s->planes;
    return GS_OK;
}

gs_status gs_read_planes(gs_scene* s, void* dst, int dst_on_device, void* stream) {
    if (!s || !dst) return set_error(GS_ERR_ARG, "NULL argument");
    size_t bytes = (size_t)s->n * s->nwords * word_bytes(s->fmt);
    GS_CUDA(cudaMemcpyAsync(dst, s->planes, bytes, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            (cudaStream_t)stream));
    if (!dst_on_device) GS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return GS_OK;
}

gs_status gs_write_planes(gs_scene* s, const void* src, int src_on_device, void* stream) {
    if (!s || !src) return set_error(GS_ERR_ARG, "NULL argument");
    size_t bytes = (size_t)s->n * s->nwords * word_bytes(s->fmt);
    GS_CUDA(cudaMemcpyAsync(s->planes, src, bytes, src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            (cudaStream_t)stream));
    if (!src_on_device) GS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return GS_OK;
}

gs_status gs_scene_errors(gs_scene* s, uint32_t* host_flags) {
    if (!s || !host_flags) return set_error(GS_ERR_ARG, "NULL argument");
    GS_CUDA(cudaMemcpy(host_flags, s->dev_err, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    GS_CUDA(cudaMemset(s->dev_err, 0, sizeof(uint32_t)));
    return GS_OK;
}

gs_status gs_apply_flips(gs_scene* s, const gs_flip* dev_flips, int64_t count, void* stream) {
    if (!s || (count > 0 && !dev_flips) || count < 0) return set_error(GS_ERR_ARG, "bad gs_apply_flips arguments");
    return launch_apply_flips(s->planes, s->fmt, s->n, s->nwords, dev_flips, count, s->dev_err, 0ull,
                              (cudaStream_t)stream);
}

gs_status gs_field_box(gs_scene* s, uint32_t* host_lo, uint32_t* host_hi) {
    if (!s || !host_lo || !host_hi) return set_error(GS_ERR_ARG, "NULL argument");
    memcpy(host_lo, s->box_lo, sizeof(uint32_t) * s->nwords);
    memcpy(host_hi, s->box_hi, sizeof(uint32_t) * s->nwords);
    return GS_OK;
}

gs_status gs_set_prim_box(gs_scene* s, const void* lo, const void* hi, int src_on_device, int nbox_words) {
    if (!s || !lo || !hi || nbox_words < 1 || nbox_words > s->nwords)
        return set_error(GS_ERR_ARG, "bad gs_set_prim_box arguments");
    destroy_graphs(s);
    cudaFree(s->pbox_lo);
    cudaFree(s->pbox_hi);
    s->pbox_lo = s->pbox_hi = nullptr;
    size_t bytes = (size_t)s->n * nbox_words * word_bytes(s->fmt);
    GS_TRY(dmalloc(&s->pbox_lo, (bytes + 15) & ~(size_t)15));
    GS_TRY(dmalloc(&s->pbox_hi, (bytes + 15) & ~(size_t)15));
    cudaMemcpyKind kind = src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    GS_CUDA(cudaMemcpy(s->pbox_lo, lo, bytes, kind));
    GS_CUDA(cudaMemcpy(s->pbox_hi, hi, bytes, kind));
    s->nbox_words = nbox_words;
    return GS_OK;
}

gs_status gs_guard(gs_scene* s, int mode, uint64_t word_mask, uint64_t* dev_clamps, void* stream) {
    if (!s) return set_error(GS_ERR_ARG, "scene is NULL");
    if (mode != GS_GUARD_FIELD && mode != GS_GUARD_PRIM) return set_error(GS_ERR_ARG, "mode must be FIELD or PRIM");
    return launch_guard(s, mode, word_mask, (unsigned long long*)dev_clamps, (cudaStream_t)stream);
}

gs_status gs_guard_bitmap(gs_scene* s, int mode, uint64_t word_mask, uint64_t* dev_clamps, uint32_t* dev_bitmap,
                          void* stream) {
    if (!s) return set_error(GS_ERR_ARG, "scene is NULL");
    if (mode != GS_GUARD_FIELD && mode != GS_GUARD_PRIM) return set_error(GS_ERR_ARG, "mode must be FIELD or PRIM");
    if (!dev_bitmap && s->n > 0) return set_error(GS_ERR_ARG, "dev_bitmap is NULL");
    const cudaStream_t st = (cudaStream_t)stream;
    GS_TRY(launch_guard_mark(s, mode, word_mask, dev_bitmap, st));   // the decisions, on the words before the clamp
    return launch_guard(s, mode, word_mask, (unsigned long long*)dev_clamps, st);
}

gs_status gs_render(gs_scene* s, const gs_camera* host_cams, int K, float* dev_rgb, void* stream) {
    if (!s || !host_cams || !dev_rgb || K < 1) return set_error(GS_ERR_ARG, "bad gs_render arguments");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t* ev = s->ev_r[0] ? s->ev_r : nullptr;
    s->render_timed = false;
    size_t off = 0;
    for (int k = 0; k < K; k++) {
        if (!valid_camera(host_cams[k])) return set_error(GS_ERR_ARG, "invalid camera");
        DevCamera cam = make_dev_camera(host_cams[k], s->tile_w, s->tile_h);
        uint32_t* ids = nullptr;
        uint64_t np = 0;
        GS_TRY(render_lists_sized(s, s->work, cam, &ids, &np, st, ev));
        GS_TRY(launch_blend_image(s->work.recs, ids, s->work.ranges, cam, dev_rgb + off, st));
        if (ev) GS_CUDA(cudaEventRecord(ev[3], st));
        s->render_pairs = np;
        off += (size_t)cam.W * cam.H * 3;
    }
    s->render_timed = ev != nullptr;
    return GS_OK;
}

gs_status gs_compare(const float* dev_a, const float* dev_b, int H, int W, int K, gs_result* dev_out, void* stream) {
    if (!dev_a || !dev_b || !dev_out || H < 1 || W < 1 || K < 1) return set_error(GS_ERR_ARG, "bad gs_compare arguments");
    cudaStream_t st = (cudaStream_t)stream;
    CmpAcc* acc = nullptr;
    GS_CUDA(cudaMallocAsync((void**)&acc, sizeof(CmpAcc) * K, st));
    gs_status rs = launch_zero_acc(acc, K, st);
    size_t img = (size_t)H * W * 3;
    for (int k = 0; k < K && rs == GS_OK; k++) rs = launch_compare(dev_a + k * img, dev_b + k * img, H, W, acc + k, st);
    if (rs == GS_OK) rs = launch_finalize(acc, K, dev_out, st);
    cudaFreeAsync(acc, st);
    return rs;
}

// The clean per-view state of gs_set_views, for validated arguments.
static gs_status build_views(gs_scene* s, const gs_camera* host_cams, int K, cudaStream_t st) {
    free_views(s);
    s->views.resize(K);
    s->K = K;
    std::vector<DevCamera> dcams(K);
    std::vector<char> vptrs(view_ptrs_size() * K);
    std::vector<const uint2*> crects(K);
    std::vector<const BlendRec*> crecs(K);
    GS_TRY(dmalloc((void**)&s->clean_nonfin, sizeof(unsigned int) * K));
    GS_CUDA(cudaMemsetAsync(s->clean_nonfin, 0, sizeof(unsigned int) * K, st));
    uint64_t max_pairs = 0;
    int max_tiles = 0;
    for (int k = 0; k < K; k++) {
        ViewState& v = s->views[k];
        v.cam = make_dev_camera(host_cams[k], s->tile_w, s->tile_h);
        dcams[k] = v.cam;
        int ntiles = v.cam.tiles_x * v.cam.tiles_y;
        uint32_t* ids = nullptr;
        uint64_t np = 0;
        GS_TRY(render_lists_sized(s, s->work, v.cam, &ids, &np, st));
        GS_TRY(dmalloc((void**)&v.recs, sizeof(BlendRec) * std::max<uint64_t>(s->n, 1)));
        GS_TRY(dmalloc((void**)&v.rects, sizeof(uint2) * std::max<uint64_t>(s->n, 1)));
        GS_TRY(dmalloc((void**)&v.ids, sizeof(uint32_t) * std::max<uint64_t>(np, 1)));
        GS_TRY(dmalloc((void**)&v.dk, sizeof(uint32_t) * std::max<uint64_t>(np, 1)));
        GS_TRY(dmalloc((void**)&v.ranges, sizeof(uint2) * ntiles));
        GS_TRY(dmalloc((void**)&v.clean, sizeof(float) * (size_t)v.cam.W * v.cam.H * 3));
        GS_TRY(dmalloc((void**)&v.stop, sizeof(uint32_t) * (size_t)v.cam.W * v.cam.H));
        GS_TRY(dmalloc((void**)&v.tile_stop, sizeof(uint32_t) * ntiles));
        GS_TRY(dmalloc((void**)&v.stop_key, sizeof(unsigned long long) * ntiles));
        GS_CUDA(cudaMemcpyAsync(v.recs, s->work.recs, sizeof(BlendRec) * s->n, cudaMemcpyDeviceToDevice, st));
        GS_CUDA(cudaMemcpyAsync(v.rects, s->work.rects, sizeof(uint2) * s->n, cudaMemcpyDeviceToDevice, st));
        GS_CUDA(cudaMemcpyAsync(v.ids, ids, sizeof(uint32_t) * np, cudaMemcpyDeviceToDevice, st));
        GS_CUDA(cudaMemcpyAsync(v.ranges, s->work.ranges, sizeof(uint2) * ntiles, cudaMemcpyDeviceToDevice, st));
        GS_TRY(launch_blend_image_stop(v.recs, v.ids, v.ranges, v.cam, v.clean, v.stop, v.tile_stop, nullptr, nullptr,
                                       nullptr, s->clean_nonfin + k, st));
        GS_TRY(launch_gather_depth(v.recs, v.ids, np, v.dk, st));
        // checkpoints of the clean blend: per tile, every ck_stride list entries up to
        // (before) the tile's last stop index, at most ck_max_per_tile
        {
            std::vector<uint32_t> tstop(ntiles), cnt(ntiles), off(ntiles);
            std::vector<uint2> rg(ntiles);
            GS_CUDA(cudaMemcpyAsync(tstop.data(), v.tile_stop, 4 * ntiles, cudaMemcpyDeviceToHost, st));
            GS_CUDA(cudaMemcpyAsync(rg.data(), v.ranges, sizeof(uint2) * ntiles, cudaMemcpyDeviceToHost, st));
            GS_CUDA(cudaStreamSynchronize(st));
            uint64_t total = 0;
            const uint32_t G = (uint32_t)ck_stride_value();
            for (int t = 0; t < ntiles; t++) {
                const uint32_t L = rg[t].y - rg[t].x;
                const uint32_t last = L > 0 ? std::min(tstop[t], L - 1) : 0u;
                cnt[t] = std::min(last / G, (uint32_t)ck_max_per_tile());
                off[t] = (uint32_t)total;
                total += cnt[t];
            }
            if (total >= 0xffffffffull) return set_error(GS_ERR_CAPACITY, "too many blend checkpoints");
            v.ck_total = total;
            GS_TRY(dmalloc((void**)&v.ck, sizeof(float4) * (size_t)(v.cam.tile_w * v.cam.tile_h) *
                                              std::max<uint64_t>(total, 1)));
            GS_TRY(dmalloc((void**)&v.ck_off, 4 * ntiles));
            GS_TRY(dmalloc((void**)&v.ck_cnt, 4 * ntiles));
            GS_CUDA(cudaMemcpyAsync(v.ck_off, off.data(), 4 * ntiles, cudaMemcpyHostToDevice, st));
            GS_CUDA(cudaMemcpyAsync(v.ck_cnt, cnt.data(), 4 * ntiles, cudaMemcpyHostToDevice, st));
            GS_TRY(launch_blend_image_stop(v.recs, v.ids, v.ranges, v.cam, v.clean, v.stop, v.tile_stop, v.ck,
                                           v.ck_off, v.ck_cnt, nullptr, st));
            GS_CUDA(cudaStreamSynchronize(st));
        }
        GS_TRY(launch_stop_keys(v.ranges, v.tile_stop, v.dk, v.ids, ntiles, v.stop_key, st));
        v.npairs = np;
        // per (tile, 8x8 block) sublists of the clean lists
        {
            const uint64_t nb = (uint64_t)ntiles * (uint64_t)((v.cam.tile_w * v.cam.tile_h) / 64);
            uint32_t* counts = nullptr;
            unsigned long long* scratch = nullptr;
            GS_TRY(dmalloc((void**)&v.bl_off, sizeof(uint32_t) * (nb + 1)));
            GS_TRY(dmalloc((void**)&counts, sizeof(uint32_t) * nb));
            GS_TRY(dmalloc((void**)&scratch, sizeof(unsigned long long) * (scan_scratch_len(nb) + 3)));
            unsigned long long* total = scratch + scan_scratch_len(nb);
            gs_status bs =
                launch_blists(v.recs, v.ids, v.ranges, v.cam, counts, nullptr, nullptr, nullptr, st);
            if (bs == GS_OK) bs = launch_exclusive_scan(counts, nb, v.bl_off, scratch, total, st);
            unsigned long long tot = 0;
            if (bs == GS_OK && cudaMemcpyAsync(&tot, total, sizeof(tot), cudaMemcpyDeviceToHost, st) != cudaSuccess)
                bs = set_error(GS_ERR_CUDA, "sublist total");
            if (bs == GS_OK && cudaStreamSynchronize(st) != cudaSuccess) bs = set_error(GS_ERR_CUDA, "sublist sync");
            cudaFree(counts);
            cudaFree(scratch);
            GS_TRY(bs);
            if (tot >= 0xffffffffull) return set_error(GS_ERR_CAPACITY, "block sublists exceed 2^32 entries");
            const uint32_t tot32 = (uint32_t)tot;
            GS_CUDA(cudaMemcpyAsync(v.bl_off + nb, &tot32, sizeof(tot32), cudaMemcpyHostToDevice, st));
            GS_TRY(dmalloc((void**)&v.bl_pos, sizeof(uint32_t) * std::max<uint64_t>(tot, 1)));
            GS_TRY(dmalloc((void**)&v.bl_rec, sizeof(BlendRec) * std::max<uint64_t>(tot, 1)));
            GS_TRY(launch_blists(v.recs, v.ids, v.ranges, v.cam, nullptr, v.bl_off, v.bl_pos, v.bl_rec, st));
            GS_CUDA(cudaStreamSynchronize(st));
        }
        fill_view_ptrs(vptrs.data() + view_ptrs_size() * k, v);
        crects[k] = v.rects;
        crecs[k] = v.recs;
        max_pairs = std::max(max_pairs, np);
        max_tiles = std::max(max_tiles, ntiles);
    }
    GS_TRY(dmalloc((void**)&s->dev_cams, sizeof(DevCamera) * K));
    GS_TRY(dmalloc(&s->dev_views, vptrs.size()));
    GS_TRY(dmalloc((void**)&s->dev_clean_rects, sizeof(uint2*) * K));
    GS_TRY(dmalloc((void**)&s->dev_clean_recs, sizeof(BlendRec*) * K));
    GS_CUDA(cudaMemcpyAsync(s->dev_cams, dcams.data(), sizeof(DevCamera) * K, cudaMemcpyHostToDevice, st));
    GS_CUDA(cudaMemcpyAsync(s->dev_views, vptrs.data(), vptrs.size(), cudaMemcpyHostToDevice, st));
    GS_CUDA(cudaMemcpyAsync(s->dev_clean_rects, crects.data(), sizeof(uint2*) * K, cudaMemcpyHostToDevice, st));
    GS_CUDA(cudaMemcpyAsync(s->dev_clean_recs, crecs.data(), sizeof(BlendRec*) * K, cudaMemcpyHostToDevice, st));
    // the plain loop re-renders a single-flip variant: at most one primitive
    // changes, adding at most one grid's worth of pairs
    s->full_cap_pairs = max_pairs + (uint64_t)max_tiles + 1024;
    s->max_tiles = max_tiles;
    // buffers for the dirty engine
    s->cap_B = 0;
    s->cap_flips = 0;
    GS_TRY(ensure_batch_buffers(s, 64, 1));
    GS_CUDA(cudaStreamSynchronize(st));
    return GS_OK;
}

gs_status gs_set_views(gs_scene* s, const gs_camera* host_cams, int K, void* stream) {
    if (!s || !host_cams || K < 1 || K > 16) return set_error(GS_ERR_ARG, "bad gs_set_views arguments (1 <= K <= 16)");
    for (int k = 0; k < K; k++)
        if (!valid_camera(host_cams[k])) return set_error(GS_ERR_ARG, "invalid camera");
    const gs_status rs = build_views(s, host_cams, K, (cudaStream_t)stream);
    // a failure part way (out of memory, a capacity limit) leaves no half-built
    // views behind: campaign calls then report GS_ERR_STATE instead of reading them
    if (rs != GS_OK) {
        free_views(s);
        s->host_cams.clear();
        return rs;
    }
    s->host_cams.assign(host_cams, host_cams + K);
    return GS_OK;
}

gs_status gs_set_tile(gs_scene* s, int tile_w, int tile_h, void* stream) {
    if (!s || !tile_shape_ok(tile_w, tile_h))
        return set_error(GS_ERR_ARG, "tile shape must be tw x th with tw, th in {8, 16, 32} and 64 <= tw * th <= 256");
    if (tile_w == s->tile_w && tile_h == s->tile_h) return GS_OK;
    s->tile_w = tile_w;
    s->tile_h = tile_h;
    if (s->host_cams.empty()) return GS_OK;
    // rebuild the clean per-view state for the new tiles
    const std::vector<gs_camera> cams = s->host_cams;
    return gs_set_views(s, cams.data(), (int)cams.size(), stream);
}

gs_status gs_get_tile(gs_scene* s, int* tile_w, int* tile_h) {
    if (!s || !tile_w || !tile_h) return set_error(GS_ERR_ARG, "bad gs_get_tile arguments");
    *tile_w = s->tile_w;
    *tile_h = s->tile_h;
    return GS_OK;
}

gs_status gs_clean_image(gs_scene* s, int k, float* dev_rgb, void* stream) {
    if (!s || !dev_rgb || k < 0 || k >= s->K) return set_error(GS_ERR_ARG, "bad gs_clean_image arguments");
    const ViewState& v = s->views[k];
    GS_CUDA(cudaMemcpyAsync(dev_rgb, v.clean, sizeof(float) * (size_t)v.cam.W * v.cam.H * 3, cudaMemcpyDeviceToDevice,
                            (cudaStream_t)stream));
    return GS_OK;
}

namespace {
gs_status inject_and_render(gs_scene* s, const gs_flip* dev_flips, int B, int guard_mode, uint64_t word_mask,
                            gs_result* dev_out, uint64_t* dev_regions, double* dev_ssim, void* stream);
}

gs_status gs_inject_and_render(gs_scene* s, const gs_flip* dev_flips, int B, int flips_per_variant, int guard_mode,
                               uint64_t word_mask, gs_result* dev_out, void* stream) {
    GS_TRY(check_flip_args(s, dev_flips, B, flips_per_variant, guard_mode, word_mask));
    if (!dev_out && B > 0) return set_error(GS_ERR_ARG, "dev_out is NULL");
    if (flips_per_variant != 1)
        return gs_inject_and_render_full(s, dev_flips, B, flips_per_variant, guard_mode, word_mask, dev_out, stream);
    return inject_and_render(s, dev_flips, B, guard_mode, word_mask, dev_out, nullptr, nullptr, stream);
}

gs_status gs_inject_and_render_regions(gs_scene* s, const gs_flip* dev_flips, int B, int guard_mode,
                                       uint64_t word_mask, gs_result* dev_out, uint64_t* dev_regions, void* stream) {
    GS_TRY(check_flip_args(s, dev_flips, B, 1, guard_mode, word_mask));
    if ((!dev_out || !dev_regions) && B > 0) return set_error(GS_ERR_ARG, "dev_out or dev_regions is NULL");
    return inject_and_render(s, dev_flips, B, guard_mode, word_mask, dev_out, dev_regions, nullptr, stream);
}

gs_status gs_inject_and_render_ex(gs_scene* s, const gs_flip* dev_flips, int B, int guard_mode, uint64_t word_mask,
                                  gs_result* dev_out, uint64_t* dev_regions, double* dev_ssim, void* stream) {
    GS_TRY(check_flip_args(s, dev_flips, B, 1, guard_mode, word_mask));
    if (!dev_out && B > 0) return set_error(GS_ERR_ARG, "dev_out is NULL");
    return inject_and_render(s, dev_flips, B, guard_mode, word_mask, dev_out, dev_regions, dev_ssim, stream);
}

namespace {
gs_status inject_and_render(gs_scene* s, const gs_flip* dev_flips, int B, int guard_mode, uint64_t word_mask,
                            gs_result* dev_out, uint64_t* dev_regions, double* dev_ssim, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    const int K = s->K;
    const int max_chunk = max_batch(K);
    const int chunk = s->batch > 0 ? std::min(s->batch, max_chunk) : max_chunk;
    const bool ssim = dev_ssim != nullptr;
    if (ssim && (s->tile_w != kTile || s->tile_h != kTile))
        return set_error(GS_ERR_STATE, "the dirty-tile SSIM needs 16 x 16 render tiles (gs_set_tile)");
    GS_TRY(ensure_batch_buffers(s, chunk, 1));
    if (ssim) GS_TRY(ensure_ssim_buffers(s));
    for (int b0 = 0; b0 < B; b0 += chunk) {
        int nb = std::min(chunk, B - b0);
        GS_CUDA(cudaMemcpyAsync(s->flip_stage, dev_flips + b0, sizeof(gs_flip) * nb, cudaMemcpyDeviceToDevice, st));
        GS_TRY(run_dirty_batch(s, nb, guard_mode, word_mask, ssim, st));
        GS_CUDA(cudaMemcpyAsync(dev_out + (size_t)b0 * K, s->res_stage, sizeof(gs_result) * nb * K,
                                cudaMemcpyDeviceToDevice, st));
        if (dev_regions)
            GS_TRY(launch_regions_out(s->acc, nb * K, (unsigned long long*)dev_regions + (size_t)2 * b0 * K, st));
        if (ssim) GS_TRY(launch_ssim_out(s->acc, nb * K, s->dev_views, K, dev_ssim + (size_t)b0 * K, st));
    }
    if (ssim) {   // a capacity overflow leaves some SSIM values incomplete: report it
        unsigned int over = 0;
        GS_CUDA(cudaMemcpyAsync(&over, s->ssim.overflow, sizeof(over), cudaMemcpyDeviceToHost, st));
        GS_CUDA(cudaStreamSynchronize(st));
        if (over) {
            GS_CUDA(cudaMemset(s->ssim.overflow, 0, sizeof(unsigned int)));
            return set_error(GS_ERR_CAPACITY, "SSIM buffers too small for this batch: use a smaller batch");
        }
    }
    return GS_OK;
}
}  // namespace

gs_status gs_inject_and_render_host(gs_scene* s, const gs_flip* host_flips, int B, int flips_per_variant,
                                    int guard_mode, uint64_t word_mask, gs_result* host_out, void* stream) {
    GS_TRY(check_flip_args(s, host_flips, B, flips_per_variant, guard_mode, word_mask));
    if (!host_out && B > 0) return set_error(GS_ERR_ARG, "host_out is NULL");
    if (B == 0) return GS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nf = (size_t)B * flips_per_variant, nr = (size_t)B * s->K;
    if (nf > s->host_io_flips_cap) {
        cudaFree(s->host_io_flips);
        s->host_io_flips = nullptr;
        s->host_io_flips_cap = 0;
        GS_TRY(dmalloc((void**)&s->host_io_flips, sizeof(gs_flip) * nf));
        s->host_io_flips_cap = nf;
    }
    if (nr > s->host_io_out_cap) {
        cudaFree(s->host_io_out);
        s->host_io_out = nullptr;
        s->host_io_out_cap = 0;
        GS_TRY(dmalloc((void**)&s->host_io_out, sizeof(gs_result) * nr));
        s->host_io_out_cap = nr;
    }
    GS_CUDA(cudaMemcpyAsync(s->host_io_flips, host_flips, sizeof(gs_flip) * nf, cudaMemcpyHostToDevice, st));
    GS_TRY(gs_inject_and_render(s, s->host_io_flips, B, flips_per_variant, guard_mode, word_mask, s->host_io_out,
                                stream));
    GS_CUDA(cudaMemcpyAsync(host_out, s->host_io_out, sizeof(gs_result) * nr, cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    return GS_OK;
}

gs_status gs_inject_and_render_full(gs_scene* s, const gs_flip* dev_flips, int B, int flips_per_variant,
                                    int guard_mode, uint64_t word_mask, gs_result* dev_out, void* stream) {
    GS_TRY(check_flip_args(s, dev_flips, B, flips_per_variant, guard_mode, word_mask));
    if (!dev_out && B > 0) return set_error(GS_ERR_ARG, "dev_out is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const int K = s->K;
    const int fpv = flips_per_variant;
    GS_TRY(ensure_batch_buffers(s, 1, fpv));
    uint64_t cap = s->full_cap_pairs + (uint64_t)(fpv - 1) * s->max_tiles;
    GS_TRY(alloc_render_work(s->work, s->n, cap, s->max_tiles));
    for (int b = 0; b < B; b++) {
        const gs_flip* f = dev_flips + (size_t)b * fpv;
        GS_TRY(launch_zero_acc(s->acc, K, st));
        GS_TRY(launch_save_sites(s->planes, s->fmt, s->n, s->nwords, f, fpv, s->saved, st));
        GS_TRY(launch_apply_flips(s->planes, s->fmt, s->n, s->nwords, f, fpv, s->dev_err,
                                  guard_mode == GS_GUARD_ECC ? word_mask : 0ull, st));
        if (guard_mode == GS_GUARD_FIELD || guard_mode == GS_GUARD_PRIM) {
            GS_TRY(launch_guard(s, guard_mode, word_mask, s->dev_clamps, st));
            k_move_clamps<<<1, 32, 0, st>>>(s->dev_clamps, s->acc);
            GS_CUDA(cudaGetLastError());
        }
        for (int k = 0; k < K; k++) {
            const ViewState& v = s->views[k];
            uint32_t* ids = nullptr;
            GS_TRY(render_lists(s, s->work, v.cam, &ids, st));
            GS_TRY(launch_blend_compare(s->work.recs, ids, s->work.ranges, v.cam, v.clean, s->acc + k,
                                        s->work_ctr, st));
        }
        GS_TRY(launch_restore_sites(s->planes, s->fmt, s->n, s->nwords, f, fpv, s->saved, st));
        GS_TRY(launch_finalize(s->acc, K, dev_out + (size_t)b * K, st));
    }
    return GS_OK;
}

gs_status gs_preprocess(gs_scene* s, const gs_camera* host_cam, gs_record* dev_out, void* stream) {
    if (!s || !host_cam || !dev_out) return set_error(GS_ERR_ARG, "bad gs_preprocess arguments");
    if (!valid_camera(*host_cam)) return set_error(GS_ERR_ARG, "invalid camera");
    DevCamera cam = make_dev_camera(*host_cam, s->tile_w, s->tile_h);
    return launch_preprocess(s, cam, nullptr, nullptr, nullptr, nullptr, dev_out, (cudaStream_t)stream);
}

gs_status gs_bin_tiles(const float* dev_depth, const int32_t* dev_rects, uint64_t n, int tiles_x, int tiles_y,
                       uint32_t* dev_offsets, uint32_t* dev_ids, uint64_t ids_cap, uint64_t* host_total,
                       void* stream) {
    if ((!dev_depth || !dev_rects) && n > 0) return set_error(GS_ERR_ARG, "NULL input");
    if (!dev_offsets || !host_total || tiles_x < 1 || tiles_y < 1 || tiles_x > 65535 || tiles_y > 65535)
        return set_error(GS_ERR_ARG, "bad gs_bin_tiles arguments");
    cudaStream_t st = (cudaStream_t)stream;
    int ntiles = tiles_x * tiles_y;
    RenderWork w;
    gs_status rs = alloc_render_work(w, n, std::max<uint64_t>(ids_cap, 1), ntiles);
    if (rs == GS_OK) rs = launch_rects_to_keys(dev_depth, dev_rects, n, tiles_x, tiles_y, w.dkey[0], w.dval[0], w.rects, st);
    uint32_t* ids = nullptr;
    if (rs == GS_OK) rs = build_tile_lists(w, n, tiles_x, tiles_y, &ids, st);
    if (rs == GS_OK) rs = launch_ranges_to_offsets(w.ranges, ntiles, dev_offsets, w.total, st);
    if (rs == GS_OK) {
        cudaError_t e = cudaMemcpyAsync(w.host_total, w.total, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rs = cuda_error(e, "gs_bin_tiles readback");
    }
    if (rs == GS_OK) {
        *host_total = w.host_total[2];
        if (w.host_total[1]) {
            rs = set_error(GS_ERR_CAPACITY, "ids_cap too small");
        } else if (*host_total > 0) {
            if (!dev_ids) {
                rs = set_error(GS_ERR_ARG, "dev_ids is NULL");
            } else {
                cudaError_t e = cudaMemcpyAsync(dev_ids, ids, sizeof(uint32_t) * (*host_total), cudaMemcpyDeviceToDevice, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) rs = cuda_error(e, "gs_bin_tiles copy");
            }
        }
    }
    cudaStreamSynchronize(st);
    free_render_work(w);
    return rs;
}

gs_status gs_blend_lists(const gs_record* dev_recs, uint64_t n, const uint32_t* dev_offsets, const uint32_t* dev_ids,
                         int W, int H, float* dev_rgb, void* stream) {
    if (!dev_offsets || !dev_rgb || W < 1 || H < 1 || (n > 0 && !dev_recs)) return set_error(GS_ERR_ARG, "bad gs_blend_lists arguments");
    cudaStream_t st = (cudaStream_t)stream;
    gs_camera hc{};   // lists of 16 x 16 tiles
    hc.width = W;
    hc.height = H;
    const DevCamera cam = make_dev_camera(hc, kTile, kTile);
    const int ntiles = cam.tiles_x * cam.tiles_y;
    BlendRec* recs = nullptr;
    uint2* ranges = nullptr;
    GS_CUDA(cudaMallocAsync((void**)&recs, sizeof(BlendRec) * std::max<uint64_t>(n, 1), st));
    GS_CUDA(cudaMallocAsync((void**)&ranges, sizeof(uint2) * ntiles, st));
    gs_status rs = launch_records_to_blend(dev_recs, n, recs, st);
    if (rs == GS_OK) rs = launch_offsets_to_ranges(dev_offsets, ntiles, ranges, st);
    if (rs == GS_OK) rs = launch_blend_image(recs, dev_ids, ranges, cam, dev_rgb, st);
    cudaFreeAsync(recs, st);
    cudaFreeAsync(ranges, st);
    return rs;
}

gs_status gs_set_batch(gs_scene* s, int batch) {
    if (!s || batch < 0) return set_error(GS_ERR_ARG, "bad gs_set_batch arguments");
    s->batch = batch;
    return GS_OK;
}

gs_status gs_autotune(gs_scene* s, const gs_flip* dev_flips, int count, int guard_mode, uint64_t word_mask,
                      int* best_batch, float* best_us_per_variant, void* stream) {
    GS_TRY(check_flip_args(s, dev_flips, count, 1, guard_mode, word_mask));
    if (count < 1 || !best_batch) return set_error(GS_ERR_ARG, "bad gs_autotune arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const int K = s->K;
    const int max_chunk = max_batch(K);
    const int cands[9] = {8, 16, 32, 64, 128, 256, 512, 1024, 2048};
    gs_result* out = nullptr;
    GS_CUDA(cudaMallocAsync((void**)&out, sizeof(gs_result) * (size_t)count * K, st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        cudaFreeAsync(out, st);
        return set_error(GS_ERR_CUDA, "gs_autotune: event creation failed");
    }
    const int prev_batch = s->batch;
    int best = max_chunk;
    float best_t = 1e30f;
    gs_status rs = GS_OK;
    for (int c : cands) {
        if (c > max_chunk) break;
        s->batch = c;
        // warm (graph capture), then time the whole list at this batch size
        int warm = std::min(count, c);
        rs = gs_inject_and_render(s, dev_flips, warm, 1, guard_mode, word_mask, out, stream);
        if (rs != GS_OK) break;
        cudaEventRecord(e0, st);
        rs = gs_inject_and_render(s, dev_flips, count, 1, guard_mode, word_mask, out, stream);
        cudaEventRecord(e1, st);
        if (rs != GS_OK) break;
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        float per = ms * 1000.0f / count;
        if (per < best_t) {
            best_t = per;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(out, st);
    if (rs != GS_OK) {
        s->batch = prev_batch;   // a failed tuning run leaves the setting as it was
        return rs;
    }
    s->batch = best;
    *best_batch = best;
    if (best_us_per_variant) *best_us_per_variant = best_t;
    return GS_OK;
}

gs_status gs_autotune_tile(gs_scene* s, const gs_flip* dev_flips, int count, int guard_mode, uint64_t word_mask,
                           int* best_tile_w, int* best_tile_h, int* best_batch, float* best_us_per_variant,
                           void* stream) {
    GS_TRY(check_flip_args(s, dev_flips, count, 1, guard_mode, word_mask));
    if (count < 1 || !best_tile_w || !best_tile_h || !best_batch)
        return set_error(GS_ERR_ARG, "bad gs_autotune_tile arguments");
    const int shapes[3][2] = {{16, 16}, {8, 8}, {32, 8}};
    const int prev_w = s->tile_w, prev_h = s->tile_h, prev_batch = s->batch;
    int bw = prev_w, bh = prev_h, bb = 0;
    float bt = 1e30f;
    gs_status rs = GS_OK;
    for (const auto& sh : shapes) {
        rs = gs_set_tile(s, sh[0], sh[1], stream);
        if (rs != GS_OK) break;
        int b = 0;
        float us = 0.0f;
        rs = gs_autotune(s, dev_flips, count, guard_mode, word_mask, &b, &us, stream);
        if (rs != GS_OK) break;
        if (us < bt) {
            bt = us;
            bw = sh[0];
            bh = sh[1];
            bb = b;
        }
    }
    if (rs != GS_OK) {   // leave the scene as it was (views rebuilt for the previous tiles)
        const std::string msg = gs_last_error();
        gs_set_tile(s, prev_w, prev_h, stream);
        s->batch = prev_batch;
        return set_error(rs, msg);
    }
    GS_TRY(gs_set_tile(s, bw, bh, stream));
    s->batch = bb;
    *best_tile_w = bw;
    *best_tile_h = bh;
    *best_batch = bb;
    if (best_us_per_variant) *best_us_per_variant = bt;
    return GS_OK;
}

gs_status gs_count_work(gs_scene* s, int enable) {
    if (!s) return set_error(GS_ERR_ARG, "scene is NULL");
    if (enable && !s->work_ctr) {
        GS_TRY(dmalloc((void**)&s->work_ctr, sizeof(unsigned long long) * 16));
        GS_CUDA(cudaMemset(s->work_ctr, 0, sizeof(unsigned long long) * 16));
    }
    if (!enable && s->work_ctr) {
        cudaFree(s->work_ctr);
        s->work_ctr = nullptr;
    }
    return GS_OK;
}

gs_status gs_read_work(gs_scene* s, uint64_t* host_counts) {
    if (!s || !host_counts) return set_error(GS_ERR_ARG, "NULL argument");
    if (!s->work_ctr) return set_error(GS_ERR_STATE, "work counting is off");
    GS_CUDA(cudaMemcpy(host_counts, s->work_ctr, sizeof(unsigned long long) * 16, cudaMemcpyDeviceToHost));
    GS_CUDA(cudaMemset(s->work_ctr, 0, sizeof(unsigned long long) * 16));
    return GS_OK;
}

gs_status gs_time_kernels(gs_scene* s, int enable) {
    if (!s) return set_error(GS_ERR_ARG, "scene is NULL");
    destroy_graphs(s);   // the event records are part of the captured graph
    if (enable && !s->ev_k0) {
        GS_CUDA(cudaEventCreate(&s->ev_k0));
        GS_CUDA(cudaEventCreate(&s->ev_kp));
        GS_CUDA(cudaEventCreate(&s->ev_k1));
        for (auto& e : s->ev_r) GS_CUDA(cudaEventCreate(&e));
    }
    if (!enable && s->ev_k0) {
        cudaEventDestroy(s->ev_k0);
        cudaEventDestroy(s->ev_kp);
        cudaEventDestroy(s->ev_k1);
        s->ev_k0 = s->ev_kp = s->ev_k1 = nullptr;
        for (auto& e : s->ev_r) {
            cudaEventDestroy(e);
            e = nullptr;
        }
    }
    s->render_timed = false;
    return GS_OK;
}

gs_status gs_read_kernel_ms(gs_scene* s, float* ms) {
    if (!s || !ms) return set_error(GS_ERR_ARG, "NULL argument");
    if (!s->ev_k0) return set_error(GS_ERR_STATE, "kernel timing is off");
    GS_CUDA(cudaEventSynchronize(s->ev_k1));
    GS_CUDA(cudaEventElapsedTime(&ms[0], s->ev_k0, s->ev_kp));
    GS_CUDA(cudaEventElapsedTime(&ms[1], s->ev_kp, s->ev_k1));
    return GS_OK;
}

gs_status gs_read_render_ms(gs_scene* s, float* ms, uint64_t* counts) {
    if (!s || !ms || !counts) return set_error(GS_ERR_ARG, "NULL argument");
    if (!s->ev_r[0]) return set_error(GS_ERR_STATE, "kernel timing is off");
    if (!s->render_timed) return set_error(GS_ERR_STATE, "no gs_render since kernel timing was switched on");
    GS_CUDA(cudaEventSynchronize(s->ev_r[3]));
    for (int i = 0; i < 3; i++) GS_CUDA(cudaEventElapsedTime(&ms[i], s->ev_r[i], s->ev_r[i + 1]));
    counts[0] = s->n;
    counts[1] = s->render_pairs;
    counts[2] = (uint64_t)s->work.passes[0];
    counts[3] = (uint64_t)s->work.passes[1];
    return GS_OK;
}

gs_status gs_set_graphs(gs_scene* s, int enable) {
    if (!s) return set_error(GS_ERR_ARG, "scene is NULL");
    s->use_graphs = enable != 0;
    if (!enable) destroy_graphs(s);
    return GS_OK;
}

}  // extern "C"
