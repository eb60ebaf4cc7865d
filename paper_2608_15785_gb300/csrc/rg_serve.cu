// rg_serve.cu -- the request loop (rg_server_create, rg_submit, rg_poll,
// rg_server_stats): slots of stream + workspace + result buffer admitted by
// device memory, and a dispatcher thread with continuous batching.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "rg_host.h"

using namespace rg;

namespace {

// ---------------------------------------------------------------------------
// Request loop (serving): slots of stream + workspace + result buffer; a
// dispatcher thread admits queued requests into free slots as earlier ones
// complete, so requests overlap on the device (continuous batching).
// ---------------------------------------------------------------------------
using Clock = std::chrono::steady_clock;

struct ServeRequest {
    uint64_t ticket = 0;
    rg_camera cam;
    int scene = 0;
    Clock::time_point submitted;
};

struct ServeSlot {
    Workspace ws;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    float* out = nullptr;            // [3][max_h][max_w]
    Counters* pinned_ctr = nullptr;  // host copy of the frame counters of the request
    enum { FREE, RUNNING, DONE } state = FREE;
    ServeRequest req;
    FrameLayout F;
    rg_status result = RG_OK;
    int attempts = 0;
};

} // namespace

struct rg_server {
    int device = 0;
    std::vector<rg_scene*> scenes;
    int mode = RG_MODE_ROOFGS;
    uint32_t flags = 0;
    int max_w = 0, max_h = 0;
    int64_t budget = 0, slot_bytes = 0;
    std::vector<std::unique_ptr<ServeSlot>> slots;
    std::deque<ServeRequest> pending;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::vector<double> latencies_ms; // submit -> result ready
    std::vector<double> delivered_ms; // submit -> image in the caller's buffer (rg_poll)
    int max_in_flight = 0;
    int64_t completed = 0;
    std::string error;
};

namespace {

rg_status slot_launch(rg_server* sv, ServeSlot& sl)
{
    rg_scene* s = sv->scenes[sl.req.scene];
    RG_TRY(ensure_workspace(sl.ws, s->n, sv->mode, sl.F.tiles, sl.ws.cap > 0 ? sl.ws.cap : (int64_t)1 << 20));
    RG_TRY(render_once(s, sl.ws, sl.F, sv->mode, sv->flags & ~RG_FLAG_STAGE_EVENTS, sl.out, sl.stream));
    RG_CK(cudaMemcpyAsync(sl.pinned_ctr, sl.ws.ctrl.p, sizeof(Counters), cudaMemcpyDeviceToHost, sl.stream));
    RG_CK(cudaEventRecord(sl.done, sl.stream));
    return RG_OK;
}

// dispatcher: complete finished slots (re-render after growing on overflow), admit new requests
void server_loop(rg_server* sv)
{
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lock(sv->mu);
    while (true) {
        bool busy = false;
        for (auto& up : sv->slots) {
            ServeSlot& sl = *up;
            if (sl.state != ServeSlot::RUNNING) continue;
            busy = true;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                cudaGetLastError();
                sl.result = RG_ERR_CUDA;
                sl.state = ServeSlot::DONE;
                continue;
            }
            const Counters& c = *sl.pinned_ctr;
            if (c.error) {
                sl.result = RG_ERR_TIMEOUT;
            } else if (c.n_entries_total > (unsigned long long)sl.ws.cap && sl.attempts < 2) {
                // grow the slot and render the request again
                int64_t want = (int64_t)(c.n_entries_total + c.n_entries_total / 4 + 1024);
                sl.attempts++;
                rg_scene* s = sv->scenes[sl.req.scene];
                rg_status e = want > MAX_CAP ? RG_ERR_CAPACITY
                                             : ensure_workspace(sl.ws, s->n, sv->mode, sl.F.tiles, want);
                if (e == RG_OK) e = slot_launch(sv, sl);
                if (e == RG_OK) continue;
                sl.result = e;
            } else if (c.n_entries_total > (unsigned long long)sl.ws.cap) {
                sl.result = RG_ERR_CAPACITY;
            } else {
                sl.result = RG_OK;
            }
            sl.state = ServeSlot::DONE;
            sv->latencies_ms.push_back(
                std::chrono::duration<double, std::milli>(Clock::now() - sl.req.submitted).count());
            sv->completed++;
            sv->cv.notify_all();
        }
        // admit queued requests into free slots (first come, first served)
        for (auto& up : sv->slots) {
            if (sv->pending.empty()) break;
            ServeSlot& sl = *up;
            if (sl.state != ServeSlot::FREE) continue;
            sl.req = sv->pending.front();
            sv->pending.pop_front();
            sl.attempts = 0;
            make_layout(&sl.req.cam, sl.F); // validated at submit
            sl.state = ServeSlot::RUNNING;
            const rg_status e = slot_launch(sv, sl);
            if (e != RG_OK) {
                sl.result = e;
                sl.state = ServeSlot::DONE;
                sv->completed++;
                sv->cv.notify_all();
            }
            busy = true;
        }
        int running = 0;
        for (auto& up : sv->slots) running += up->state == ServeSlot::RUNNING;
        sv->max_in_flight = std::max(sv->max_in_flight, running);
        if (sv->stop && !busy && sv->pending.empty()) break;
        if (busy) {
            lock.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lock.lock();
        } else {
            sv->cv.wait_for(lock, std::chrono::milliseconds(5));
        }
    }
}

void server_free(rg_server* sv)
{
    for (auto& up : sv->slots) {
        ServeSlot& sl = *up;
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        sl.ws.release();
        if (sl.out) cudaFree(sl.out);
        if (sl.pinned_ctr) cudaFreeHost(sl.pinned_ctr);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    delete sv;
}

} // namespace

extern "C" {

rg_status rg_server_create(rg_scene* const* scenes, int32_t n_scenes, const rg_server_config* cfg, rg_server** out)
{
    if (!out) return fail(RG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!scenes || n_scenes <= 0 || !cfg) return fail(RG_ERR_INVALID_ARG, "bad arguments");
    if (cfg->mode != RG_MODE_EXACT && cfg->mode != RG_MODE_ROOFGS) return fail(RG_ERR_INVALID_ARG, "unknown mode");
    if (cfg->max_width <= 0 || cfg->max_height <= 0) return fail(RG_ERR_INVALID_ARG, "max resolution must be set");
    for (int k = 0; k < n_scenes; k++) {
        if (!scenes[k]) return fail(RG_ERR_INVALID_ARG, "NULL scene");
        if (cfg->mode == RG_MODE_EXACT && !(scenes[k]->storage & RG_STORE_FP32))
            return fail(RG_ERR_INVALID_ARG, "exact mode needs RG_STORE_FP32");
        if (cfg->mode == RG_MODE_ROOFGS && !(scenes[k]->storage & RG_STORE_COMPACT))
            return fail(RG_ERR_INVALID_ARG, "RoofGS mode needs RG_STORE_COMPACT");
    }
    std::unique_ptr<rg_server> sv(new rg_server());
    RG_CK(cudaGetDevice(&sv->device));
    sv->scenes.assign(scenes, scenes + n_scenes);
    sv->mode = cfg->mode;
    sv->flags = cfg->flags & ~(RG_FLAG_STAGE_EVENTS | RG_FLAG_BATCH_CHECKED);
    sv->max_w = cfg->max_width;
    sv->max_h = cfg->max_height;
    sv->budget = cfg->memory_budget > 0 ? cfg->memory_budget : (8ll << 30);
    // calibrate one slot: the largest scene at the largest resolution, pose of the first camera
    int big = 0;
    for (int k = 1; k < n_scenes; k++)
        if (scenes[k]->n > scenes[big]->n) big = k;
    std::unique_ptr<ServeSlot> probe(new ServeSlot());
    RG_CK(cudaStreamCreateWithFlags(&probe->stream, cudaStreamNonBlocking));
    RG_CK(cudaEventCreateWithFlags(&probe->done, cudaEventDisableTiming));
    const size_t out_bytes = (size_t)3 * sv->max_w * sv->max_h * 4;
    if (cudaMalloc(&probe->out, out_bytes) != cudaSuccess) return fail(RG_ERR_OOM, "slot output");
    if (cudaMallocHost(&probe->pinned_ctr, sizeof(Counters)) != cudaSuccess) return fail(RG_ERR_OOM, "pinned counters");
    int64_t entries = 0;
    if (cfg->calibration) {
        probe->req.cam = *cfg->calibration;
        probe->req.cam.width = sv->max_w;
        probe->req.cam.height = sv->max_h;
        probe->req.scene = big;
        RG_TRY(make_layout(&probe->req.cam, probe->F));
        RG_TRY(ensure_workspace(probe->ws, scenes[big]->n, sv->mode, probe->F.tiles, (int64_t)1 << 20));
        for (int attempt = 0; attempt < 2; attempt++) {
            RG_TRY(render_once(scenes[big], probe->ws, probe->F, sv->mode, sv->flags, probe->out, probe->stream));
            Counters c;
            RG_CK(cudaMemcpyAsync(&c, probe->ws.ctrl.p, sizeof(c), cudaMemcpyDeviceToHost, probe->stream));
            RG_CK(cudaStreamSynchronize(probe->stream));
            entries = (int64_t)c.n_entries_total;
            if (c.n_entries_total <= (unsigned long long)probe->ws.cap) break;
            RG_TRY(ensure_workspace(probe->ws, scenes[big]->n, sv->mode, probe->F.tiles,
                                    std::min<int64_t>(MAX_CAP, entries + entries / 4 + 1024)));
        }
        RG_CK(cudaMemsetAsync(scenes[big]->sticky.p, 0, sizeof(Sticky), probe->stream));
    }
    const int64_t cap = std::min<int64_t>(MAX_CAP, std::max<int64_t>(1 << 20, entries + entries / 2 + 1024));
    const int64_t ngauss = scenes[big]->n;
    const int64_t tiles = (int64_t)((sv->max_w + TILE - 1) / TILE) * ((sv->max_h + TILE - 1) / TILE);
    // bytes of one slot: 2 x (keys 8 B + values 4 B) per entry, sort status, per-Gaussian arrays (RoofGS:
    // records, depth order, row tests and row counts), ranges, image
    sv->slot_bytes = cap * 24 + (cap / 4096 + 1) * 2048 + ngauss * (sv->mode == RG_MODE_EXACT ? 72 : 112) +
                     tiles * 8 + (int64_t)out_bytes;
    int nslots = cfg->max_slots > 0 ? cfg->max_slots : 8;
    nslots = (int)std::max<int64_t>(1, std::min<int64_t>(nslots, sv->budget / std::max<int64_t>(sv->slot_bytes, 1)));
    for (int k = 0; k < nslots; k++) {
        std::unique_ptr<ServeSlot> sl;
        if (k == 0) {
            sl = std::move(probe);
        } else {
            sl.reset(new ServeSlot());
            RG_CK(cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking));
            RG_CK(cudaEventCreateWithFlags(&sl->done, cudaEventDisableTiming));
            if (cudaMalloc(&sl->out, out_bytes) != cudaSuccess) return fail(RG_ERR_OOM, "slot output");
            if (cudaMallocHost(&sl->pinned_ctr, sizeof(Counters)) != cudaSuccess)
                return fail(RG_ERR_OOM, "pinned counters");
        }
        for (int j = 0; j < n_scenes; j++)
            RG_TRY(ensure_workspace(sl->ws, scenes[j]->n, sv->mode, (int)tiles, std::max(cap, sl->ws.cap)));
        sv->slots.push_back(std::move(sl));
    }
    RG_CK(cudaDeviceSynchronize());
    rg_server* raw = sv.release();
    raw->worker = std::thread(server_loop, raw);
    *out = raw;
    return RG_OK;
}

rg_status rg_server_destroy(rg_server* server)
{
    if (!server) return RG_OK;
    {
        std::lock_guard<std::mutex> lock(server->mu);
        server->stop = true;
        server->cv.notify_all();
    }
    if (server->worker.joinable()) server->worker.join();
    server_free(server);
    return RG_OK;
}

rg_status rg_submit(rg_server* server, const rg_camera* cam, int32_t scene_slot, uint64_t* ticket)
{
    if (!server || !cam || !ticket) return fail(RG_ERR_INVALID_ARG, "NULL argument");
    if (scene_slot < 0 || scene_slot >= (int32_t)server->scenes.size()) return fail(RG_ERR_INVALID_ARG, "bad scene slot");
    FrameLayout F;
    RG_TRY(make_layout(cam, F));
    if (cam->width > server->max_w || cam->height > server->max_h)
        return fail(RG_ERR_INVALID_ARG, "request larger than the server's maximum resolution");
    ServeRequest r;
    r.cam = *cam;
    r.scene = scene_slot;
    r.submitted = Clock::now();
    std::lock_guard<std::mutex> lock(server->mu);
    if (server->stop) return fail(RG_ERR_BUSY, "server is stopping");
    r.ticket = server->next_ticket++;
    server->pending.push_back(r);
    *ticket = r.ticket;
    server->cv.notify_all();
    return RG_OK;
}

rg_status rg_poll(rg_server* server, uint64_t ticket, float* out_chw)
{
    if (!server || !out_chw) return fail(RG_ERR_INVALID_ARG, "NULL argument");
    ServeSlot* hit = nullptr;
    {
        std::lock_guard<std::mutex> lock(server->mu);
        for (auto& up : server->slots)
            if (up->state != ServeSlot::FREE && up->req.ticket == ticket) hit = up.get();
        if (!hit) {
            for (const ServeRequest& r : server->pending)
                if (r.ticket == ticket) return RG_ERR_NOT_READY;
            return fail(RG_ERR_INVALID_ARG, "unknown or already collected ticket");
        }
        if (hit->state != ServeSlot::DONE) return RG_ERR_NOT_READY;
    }
    rg_status res = hit->result;
    if (res == RG_OK) {
        const size_t bytes = (size_t)3 * hit->F.cam.W * hit->F.cam.H * 4;
        cudaError_t e = cudaMemcpyAsync(out_chw, hit->out, bytes, cudaMemcpyDefault, hit->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(hit->stream);
        if (e != cudaSuccess) res = fail(RG_ERR_CUDA, cudaGetErrorString(e));
    } else {
        fail(res, "request failed");
    }
    const double delivered = std::chrono::duration<double, std::milli>(Clock::now() - hit->req.submitted).count();
    std::lock_guard<std::mutex> lock(server->mu);
    if (res == RG_OK) server->delivered_ms.push_back(delivered);
    hit->state = ServeSlot::FREE;
    server->cv.notify_all();
    return res;
}

rg_status rg_server_stats(rg_server* server, rg_server_stats_t* st)
{
    if (!server || !st) return fail(RG_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lock(server->mu);
    std::vector<double> l = server->latencies_ms, d = server->delivered_ms;
    std::sort(l.begin(), l.end());
    std::sort(d.begin(), d.end());
    auto pct_of = [](const std::vector<double>& v, double p) {
        return v.empty() ? 0.0 : v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))];
    };
    auto pct = [&](double p) { return pct_of(l, p); };
    st->p50_delivered_ms = pct_of(d, 0.50);
    st->p99_delivered_ms = pct_of(d, 0.99);
    st->completed = server->completed;
    st->pending = (int64_t)server->pending.size();
    st->slots = (int32_t)server->slots.size();
    st->max_in_flight = server->max_in_flight;
    st->p50_ms = pct(0.50);
    st->p99_ms = pct(0.99);
    st->slot_bytes = server->slot_bytes;
    return RG_OK;
}

rg_status rg_server_reset_stats(rg_server* server)
{
    if (!server) return fail(RG_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lock(server->mu);
    server->latencies_ms.clear();
    server->delivered_ms.clear();
    server->completed = 0;
    server->max_in_flight = 0;
    return RG_OK;
}

} // extern "C"
