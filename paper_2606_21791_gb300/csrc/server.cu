// Serving loop: several resident scenes, render / injection-campaign / upset-
// storm requests admitted by an HBM budget, continuous batching over CUDA
// streams.
//
// Each worker slot owns a CUDA stream, a host thread and its own render
// scratch.  A free slot takes the first queued request that can start now:
// (1) its scene allows it -- renders without the guard only read the scene and
// run concurrently with each other and with campaigns; a campaign uses the
// scene's own batch buffers, so one campaign per scene at a time; a guarded
// render or a storm frame writes the resident parameters (flips, guard
// clamps) and runs alone on its scene; (2) the memory it would add (growth of
// the slot's render scratch) fits the budget next to the resident scenes and
// the scratch already held.  Requests that arrive while others run are admitted
// as soon as a slot and memory free up, so work from different requests
// overlaps on the device.  A request that can never fit is refused
// (GS_ERR_BUSY).  Latencies are taken on the host clock from submission (or the
// caller's arrival time) to completion of the request's stream work.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "gs_internal.h"

namespace gs {
gs_status render_lists_sized_ext(gs_scene* s, RenderWork& w, const DevCamera& cam, uint32_t** ids, uint64_t* npairs,
                                 cudaStream_t st);
gs_status launch_apply_flips(void* planes, int fmt, uint64_t n, int nwords, const gs_flip* flips, int64_t count,
                             unsigned int* err, uint64_t ecc_mask, cudaStream_t st);
}  // namespace gs

using namespace gs;

namespace {

struct Req {
    uint64_t ticket = 0;
    gs_request r{};
    double t_submit = 0.0, t_start = 0.0, t_done = 0.0;
    int status = -1;   // -1 queued, -2 running, >= 0 finished with this gs_status
    std::string err;
    int slot = -1;
    bool mem_waited = false;   // passed over at least once because its scratch did not fit the budget
};

struct SceneEntry {
    gs_scene* s = nullptr;
    uint64_t resident = 0;
    int readers = 0;
    bool campaign = false;
    bool writer = false;
};

struct Slot {
    cudaStream_t stream = nullptr;
    RenderWork work;
    uint64_t scratch = 0;
    unsigned long long* clamps = nullptr;
    std::thread th;
};

uint64_t render_scratch_bytes(uint64_t n, uint64_t pairs, int ntiles) {
    // records, rects, depth keys/values (x2), counts, offsets, scan space, pairs (x2 keys and values),
    // histograms, ranges
    return n * (sizeof(BlendRec) + 8 + 16 + 8 + 12) + pairs * 16 + ntiles * 8 + (pairs / 2048 + 1) * 1024 + (1 << 20);
}

uint64_t scene_resident_bytes(const gs_scene* s) {
    uint64_t b = s->n * (uint64_t)s->nwords * word_bytes(s->fmt);
    if (s->pbox_lo) b += 2ull * s->n * s->nbox_words * word_bytes(s->fmt);
    for (const auto& v : s->views)
        b += s->n * (sizeof(BlendRec) + 8) + v.npairs * 8 + (uint64_t)v.cam.tiles_x * v.cam.tiles_y * 8 +
             (uint64_t)v.cam.W * v.cam.H * 16 + v.ck_total * 16ull * (uint64_t)(v.cam.tile_w * v.cam.tile_h) +
             (uint64_t)v.cam.tiles_x * v.cam.tiles_y * 12;
    b += render_scratch_bytes(s->work.n, s->work.cap_pairs, s->work.ntiles_cap);
    return b;
}

double now_ms(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct gs_server {
    uint64_t budget = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req*> queue;
    std::map<uint64_t, Req*> all;
    std::deque<SceneEntry> scenes;   // stable references: a scene may be added while workers hold one
    std::vector<Slot> slots;
    uint64_t next_ticket = 1;
    uint64_t scratch_total = 0;
    bool stop = false;
    uint64_t completed = 0;
    uint64_t mem_delayed = 0;   // started requests that had waited for budget
};

namespace {

bool scene_allows(const SceneEntry& e, const gs_request& r) {
    if (e.writer) return false;
    const bool guards = r.guard_mode == GS_GUARD_FIELD || r.guard_mode == GS_GUARD_PRIM;
    bool writes = r.kind == GS_REQ_STORM || (r.kind == GS_REQ_RENDER && guards);
    if (writes) return e.readers == 0 && !e.campaign;
    if (r.kind == GS_REQ_CAMPAIGN) return !e.campaign;
    return true;
}

uint64_t request_need(gs_server* sv, const Req* q) {
    const gs_request& r = q->r;
    if (r.kind == GS_REQ_CAMPAIGN) return 0;   // runs in the scene's own (resident) buffers
    const gs_scene* s = sv->scenes[r.scene].s;
    DevCamera cam = make_dev_camera(r.cam, s->tile_w, s->tile_h);
    int ntiles = cam.tiles_x * cam.tiles_y;
    return render_scratch_bytes(s->n, std::max<uint64_t>(8 * s->n, 1024), ntiles);
}

uint64_t resident_total(gs_server* sv) {
    uint64_t r = 0;
    for (auto& e : sv->scenes) r += e.resident;
    return r;
}

// run one request on a slot's stream (scene s, taken under the server lock);
// returns its status
gs_status execute(gs_scene* s, Slot& sl, Req* q) {
    const gs_request& r = q->r;
    cudaStream_t st = sl.stream;
    if (r.kind == GS_REQ_CAMPAIGN) {
        GS_TRY(gs_inject_and_render(s, r.dev_flips, r.nflips, 1, r.guard_mode, r.word_mask, r.dev_results, st));
        GS_CUDA(cudaStreamSynchronize(st));
        return GS_OK;
    }
    if (r.kind == GS_REQ_STORM && r.nflips > 0)
        GS_TRY(launch_apply_flips(s->planes, s->fmt, s->n, s->nwords, r.dev_flips, r.nflips, s->dev_err,
                                  r.guard_mode == GS_GUARD_ECC ? r.word_mask : 0ull, st));
    if (r.guard_mode == GS_GUARD_FIELD || r.guard_mode == GS_GUARD_PRIM) {
        GS_CUDA(cudaMemsetAsync(sl.clamps, 0, sizeof(unsigned long long), st));
        GS_TRY(launch_guard(s, r.guard_mode, r.word_mask, sl.clamps, st));
        if (r.dev_clamps)
            GS_CUDA(cudaMemcpyAsync(r.dev_clamps, sl.clamps, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st));
    }
    DevCamera cam = make_dev_camera(r.cam, s->tile_w, s->tile_h);
    uint32_t* ids = nullptr;
    uint64_t np = 0;
    GS_TRY(render_lists_sized_ext(s, sl.work, cam, &ids, &np, st));
    if (r.dev_rgb) GS_TRY(launch_blend_image(sl.work.recs, ids, sl.work.ranges, cam, r.dev_rgb, st));
    GS_CUDA(cudaStreamSynchronize(st));
    return GS_OK;
}

void worker(gs_server* sv, int slot_id) {
    Slot& sl = sv->slots[slot_id];
    std::unique_lock<std::mutex> lk(sv->mu);
    while (true) {
        Req* pick = nullptr;
        uint64_t extra = 0;
        while (!pick) {
            if (sv->stop && sv->queue.empty()) return;
            uint64_t base = resident_total(sv) + sv->scratch_total;
            bool mem_blocked = false;
            for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it) {
                Req* q = *it;
                SceneEntry& e = sv->scenes[q->r.scene];
                if (!scene_allows(e, q->r)) continue;
                uint64_t need = request_need(sv, q);
                uint64_t add = need > sl.scratch ? need - sl.scratch : 0;
                if (base + add > sv->budget) {
                    mem_blocked = true;
                    q->mem_waited = true;
                    continue;
                }
                pick = q;
                extra = add;
                sv->queue.erase(it);
                break;
            }
            if (!pick) {
                if (sv->stop && sv->queue.empty()) return;
                if (mem_blocked && sl.scratch > 0) {
                    // memory blocks the queue: give this idle slot's scratch back
                    uint64_t give = sl.scratch;
                    sl.scratch = 0;
                    sv->scratch_total -= give;
                    lk.unlock();
                    free_render_work(sl.work);
                    lk.lock();
                    sv->cv_work.notify_all();
                    continue;
                }
                sv->cv_work.wait(lk);
            }
        }
        SceneEntry& e = sv->scenes[pick->r.scene];
        bool writes = pick->r.kind == GS_REQ_STORM ||
                      (pick->r.kind == GS_REQ_RENDER &&
                       (pick->r.guard_mode == GS_GUARD_FIELD || pick->r.guard_mode == GS_GUARD_PRIM));
        if (writes) e.writer = true;
        else if (pick->r.kind == GS_REQ_CAMPAIGN) e.campaign = true;
        else e.readers++;
        sl.scratch += extra;
        sv->scratch_total += extra;
        pick->status = -2;
        pick->slot = slot_id;
        if (pick->mem_waited) sv->mem_delayed++;
        pick->t_start = now_ms(sv->t0);
        gs_scene* scene = e.s;
        lk.unlock();

        gs_status rs = execute(scene, sl, pick);
        std::string msg = rs == GS_OK ? std::string() : std::string(gs_last_error());

        lk.lock();
        if (writes) e.writer = false;
        else if (pick->r.kind == GS_REQ_CAMPAIGN) e.campaign = false;
        else e.readers--;
        pick->t_done = now_ms(sv->t0);
        pick->err = msg;
        pick->status = rs;
        sv->completed++;
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
}

}  // namespace

extern "C" {

gs_status gs_server_create(uint64_t hbm_budget_bytes, int nslots, gs_server** out) {
    if (!out || nslots < 1 || nslots > 64) return set_error(GS_ERR_ARG, "bad gs_server_create arguments");
    gs_server* sv = new gs_server();
    sv->budget = hbm_budget_bytes;
    sv->t0 = std::chrono::steady_clock::now();
    sv->slots.resize(nslots);
    for (auto& sl : sv->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMalloc((void**)&sl.clamps, sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            for (auto& t : sv->slots) {
                if (t.stream) cudaStreamDestroy(t.stream);
                cudaFree(t.clamps);
            }
            delete sv;
            return set_error(GS_ERR_CUDA, "gs_server_create: stream or counter allocation failed");
        }
    }
    for (int i = 0; i < nslots; i++) sv->slots[i].th = std::thread(worker, sv, i);
    *out = sv;
    return GS_OK;
}

gs_status gs_server_add_scene(gs_server* sv, gs_scene* s, int* scene_id) {
    if (!sv || !s || !scene_id) return set_error(GS_ERR_ARG, "bad gs_server_add_scene arguments");
    std::lock_guard<std::mutex> lk(sv->mu);
    uint64_t res = scene_resident_bytes(s);
    if (resident_total(sv) + sv->scratch_total + res > sv->budget)
        return set_error(GS_ERR_BUSY, "scene does not fit the HBM budget");
    SceneEntry e;
    e.s = s;
    e.resident = res;
    sv->scenes.push_back(e);
    *scene_id = (int)sv->scenes.size() - 1;
    return GS_OK;
}

gs_status gs_server_submit(gs_server* sv, const gs_request* r, double arrival_ms, uint64_t* ticket) {
    if (!sv || !r || !ticket) return set_error(GS_ERR_ARG, "bad gs_server_submit arguments");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (r->scene < 0 || r->scene >= (int)sv->scenes.size()) return set_error(GS_ERR_ARG, "unknown scene id");
    if (r->kind < GS_REQ_RENDER || r->kind > GS_REQ_STORM) return set_error(GS_ERR_ARG, "unknown request kind");
    if (r->kind == GS_REQ_CAMPAIGN && (r->nflips < 0 || (r->nflips > 0 && (!r->dev_flips || !r->dev_results))))
        return set_error(GS_ERR_ARG, "campaign request needs flips and result buffers");
    if (r->kind != GS_REQ_CAMPAIGN) {
        const gs_camera& c = r->cam;
        if (!valid_camera(c)) return set_error(GS_ERR_ARG, "invalid camera");
        if (r->kind == GS_REQ_STORM && r->nflips > 0 && !r->dev_flips) return set_error(GS_ERR_ARG, "storm flips NULL");
    }
    Req* q = new Req();
    q->r = *r;
    q->ticket = sv->next_ticket++;
    q->t_submit = arrival_ms >= 0.0 ? arrival_ms : now_ms(sv->t0);
    // a request that cannot fit even on an idle server is refused now
    uint64_t need = request_need(sv, q);
    if (resident_total(sv) + need > sv->budget) {
        delete q;
        return set_error(GS_ERR_BUSY, "request exceeds the HBM budget");
    }
    sv->all[q->ticket] = q;
    sv->queue.push_back(q);
    *ticket = q->ticket;
    sv->cv_work.notify_all();
    return GS_OK;
}

static void fill_response(const Req* q, gs_response* out) {
    out->ticket = q->ticket;
    out->status = q->status;
    out->slot = q->slot;
    out->t_submit_ms = q->t_submit;
    out->t_start_ms = q->t_start;
    out->t_done_ms = q->t_done;
}

gs_status gs_server_wait(gs_server* sv, uint64_t ticket, int timeout_ms, gs_response* out) {
    if (!sv || !out) return set_error(GS_ERR_ARG, "bad gs_server_wait arguments");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return set_error(GS_ERR_STATE, "unknown ticket");
    Req* q = it->second;
    auto done = [&] { return q->status >= 0; };
    if (timeout_ms < 0)
        sv->cv_done.wait(lk, done);
    else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
        return set_error(GS_ERR_TIMEOUT, "request not finished");
    fill_response(q, out);
    gs_status rs = (gs_status)q->status;
    std::string err = q->err;
    sv->all.erase(it);
    delete q;
    if (rs != GS_OK) return set_error(rs, "request failed: " + err);
    return GS_OK;
}

gs_status gs_server_cancel(gs_server* sv, uint64_t ticket) {
    if (!sv) return set_error(GS_ERR_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return set_error(GS_ERR_STATE, "unknown ticket");
    Req* q = it->second;
    if (q->status != -1) return set_error(GS_ERR_BUSY, "request already started");
    sv->queue.erase(std::find(sv->queue.begin(), sv->queue.end(), q));
    sv->all.erase(it);
    delete q;
    return GS_OK;
}

gs_status gs_server_stats(gs_server* sv, uint64_t* host_stats) {
    if (!sv || !host_stats) return set_error(GS_ERR_ARG, "bad gs_server_stats arguments");
    std::lock_guard<std::mutex> lk(sv->mu);
    host_stats[0] = sv->budget;
    host_stats[1] = resident_total(sv);
    host_stats[2] = sv->scratch_total;
    host_stats[3] = sv->queue.size();
    host_stats[4] = sv->completed;
    host_stats[5] = sv->mem_delayed;
    return GS_OK;
}

gs_status gs_server_now(gs_server* sv, double* now_ms_out) {
    if (!sv || !now_ms_out) return set_error(GS_ERR_ARG, "bad gs_server_now arguments");
    *now_ms_out = now_ms(sv->t0);
    return GS_OK;
}

gs_status gs_server_destroy(gs_server* sv) {
    if (!sv) return GS_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->cv_work.notify_all();
    }
    for (auto& sl : sv->slots)
        if (sl.th.joinable()) sl.th.join();
    for (auto& sl : sv->slots) {
        cudaStreamSynchronize(sl.stream);
        free_render_work(sl.work);
        cudaFree(sl.clamps);
        cudaStreamDestroy(sl.stream);
    }
    for (auto& kv : sv->all) delete kv.second;
    delete sv;
    return GS_OK;
}

}  // extern "C"
