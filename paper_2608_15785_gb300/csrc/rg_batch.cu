// rg_batch.cu -- rg_render_batch / rg_batch_plan_info: batched multi-view
// rendering through captured CUDA graphs, with an autotuner over tile shape,
// lanes and pixels per thread.
#include <algorithm>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "rg_host.h"

using namespace rg;

namespace {

// ---------------------------------------------------------------------------
// Batched rendering: a plan per (scenes, resolutions, mode, flags) owns L lanes,
// each a stream and a workspace; a call captures every view's pipeline on the
// lanes (view v on lane v mod L) into one CUDA graph, updates the plan's
// instantiated graph in place and launches it once on the caller's stream.
// ---------------------------------------------------------------------------
constexpr int BATCH_MAX_LANES = 4;

struct BatchPlan {
    int device = 0;
    std::vector<rg_scene*> scenes;
    std::vector<int> widths, heights;
    int mode = 0;
    uint32_t flags = 0;
    int lanes = 1;
    uint32_t raster_flags = 0; // autotuned: 0 (two pixels per thread), RG_FLAG_SINGLE_PIXEL or RG_FLAG_QUAD_PIXEL
    int req_tw = 0, req_th = 0; // requested tile shape (0 x 0: autotuned)
    int tw = TILE, th = TILE;   // tile shape in use
    bool tuned = false;
    bool fused = false;         // autotuned: the fused path (RoofGS; see plan_capture_fused)
    std::unique_ptr<Workspace[]> ws{new Workspace[BATCH_MAX_LANES]};
    std::unique_ptr<Workspace[]> vws; // fused path: one workspace per view
    DevBuf claim;                     // fused path: work counters of the multi-view launches
    cudaStream_t streams[BATCH_MAX_LANES] = {nullptr};
    cudaEvent_t join[BATCH_MAX_LANES] = {nullptr};
    cudaEvent_t fork = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    int exec_lanes = 0;
    uint32_t exec_raster = 0;
    int exec_tw = 0;
    int exec_fused = -1;

    ~BatchPlan()
    {
        if (exec) cudaGraphExecDestroy(exec);
        for (int l = 0; l < BATCH_MAX_LANES; l++) {
            if (streams[l]) cudaStreamDestroy(streams[l]);
            if (join[l]) cudaEventDestroy(join[l]);
            ws[l].release();
        }
        if (vws)
            for (size_t v = 0; v < scenes.size(); v++) vws[v].release();
        claim.release();
        if (fork) cudaEventDestroy(fork);
        if (cap) cudaStreamDestroy(cap);
    }
};

std::mutex g_batch_mu;
std::vector<std::unique_ptr<BatchPlan>> g_plans;

rg_status plan_init(BatchPlan& P)
{
    for (int l = 0; l < BATCH_MAX_LANES; l++) {
        RG_CK(cudaStreamCreateWithFlags(&P.streams[l], cudaStreamNonBlocking));
        RG_CK(cudaEventCreateWithFlags(&P.join[l], cudaEventDisableTiming));
    }
    RG_CK(cudaEventCreateWithFlags(&P.fork, cudaEventDisableTiming));
    RG_CK(cudaStreamCreateWithFlags(&P.cap, cudaStreamNonBlocking));
    return RG_OK;
}

// The fused path: RoofGS, at most MAX_BATCH_VIEWS views, no test hook.
bool fused_possible(const BatchPlan& P)
{
    return P.mode == RG_MODE_ROOFGS && P.scenes.size() <= (size_t)MAX_BATCH_VIEWS &&
           !(P.flags & (RG_FLAG_TEST_STALL_SORT | RG_FLAG_BATCH_LANES | RG_FLAG_TILE_COUNTING_SORT));
}

// Size every lane for every view: render each view once on lane 0's workspace with
// the checked path, then give all lanes the largest capacity (+25 % headroom for
// other poses). Also runs each kernel once outside capture (first-use set-up).
rg_status plan_size(BatchPlan& P, const std::vector<FrameLayout>& F, float* const* outs, cudaStream_t st)
{
    int64_t cap = 0;
    int max_tiles = 1;
    int64_t max_n = 1;
    std::vector<int64_t> view_entries(F.size(), 0);
    for (size_t v = 0; v < F.size(); v++) {
        rg_scene* s = P.scenes[v];
        max_tiles = std::max(max_tiles, F[v].tiles);
        max_n = std::max<int64_t>(max_n, s->n);
        int64_t c = P.ws[0].cap > 0 ? P.ws[0].cap : std::max<int64_t>(1 << 20, 4 * s->n);
        if (c > MAX_CAP) c = MAX_CAP;
        RG_TRY(ensure_workspace(P.ws[0], s->n, P.mode, F[v].tiles, c));
        for (int attempt = 0; attempt < 2; attempt++) {
            RG_TRY(render_once(s, P.ws[0], F[v], P.mode, P.flags, outs[v], st));
            Counters c2;
            RG_CK(cudaMemcpyAsync(&c2, P.ws[0].ctrl.p, sizeof(c2), cudaMemcpyDeviceToHost, st));
            RG_CK(cudaStreamSynchronize(st));
            if (c2.error) return fail(RG_ERR_TIMEOUT, "a bounded device wait gave up");
            cap = std::max<int64_t>(cap, (int64_t)c2.n_entries_total);
            view_entries[v] = std::max<int64_t>(view_entries[v], (int64_t)c2.n_entries_total);
            if (c2.n_entries_total <= (unsigned long long)P.ws[0].cap) break;
            int64_t want = (int64_t)(c2.n_entries_total + c2.n_entries_total / 4 + 1024);
            if (want > MAX_CAP) return fail(RG_ERR_CAPACITY, "a view needs more than 2^30 - 1 entries");
            RG_TRY(ensure_workspace(P.ws[0], s->n, P.mode, F[v].tiles, want));
        }
    }
    cap = std::min<int64_t>(MAX_CAP, cap + cap / 4 + 1024);
    for (int l = 0; l < BATCH_MAX_LANES; l++) {
        for (size_t v = 0; v < F.size(); v++)
            RG_TRY(ensure_workspace(P.ws[l], P.scenes[v]->n, P.mode, max_tiles, std::max(cap, P.ws[l].cap)));
    }
    if (fused_possible(P)) { // the fused path keeps every view's frame at once: one workspace per view
        if (!P.vws) P.vws.reset(new Workspace[F.size()]);
        for (size_t v = 0; v < F.size(); v++) {
            const int64_t c = std::min<int64_t>(MAX_CAP, view_entries[v] + view_entries[v] / 4 + 1024);
            RG_TRY(ensure_workspace(P.vws[v], P.scenes[v]->n, P.mode, F[v].tiles, std::max(c, P.vws[v].cap)));
        }
        RG_TRY(ensure(P.claim, 256, "batch work counters"));
    }
    // the scenes' sticky flags of the sizing frames are not errors
    for (rg_scene* s : P.scenes) RG_CK(cudaMemsetAsync(s->sticky.p, 0, sizeof(Sticky), st));
    RG_CK(cudaStreamSynchronize(st));
    return RG_OK;
}

// The fused path's stages of every view, enqueued while P.cap is being captured: on the
// lanes, each view's counters are cleared and its Gaussians ordered by depth; then ONE
// front-end launch walks the Gaussians of every view (k_frontend_views); on the lanes,
// each view's entries are sorted; then ONE persistent rasterizer launch takes the
// (view, tile) items of every view from a work counter (k_raster_views).
rg_status enqueue_fused(BatchPlan& P, const std::vector<FrameLayout>& F, float* const* outs, int lanes, uint32_t fl)
{
    const int V = (int)F.size();
    std::unique_ptr<FrontendViews> fv(new FrontendViews());
    std::unique_ptr<RasterViews> rv(new RasterViews());
    std::vector<SortArgs> sorts((size_t)V);
    unsigned blocks = 0, items = 0;
    const int bt = frontend_block_threads();
    for (int v = 0; v < V; v++) {
        rg_scene* s = P.scenes[v];
        Workspace& w = P.vws[v];
        cudaStream_t ls = P.streams[v % lanes];
        RoofgsFrame f;
        RG_TRY(roofgs_build(s, w, F[v], fl, f));
        RG_CK(cudaMemsetAsync(w.ctrl.p, 0, CTRL_ALLOC, ls));
        RG_CK(cudaMemsetAsync(w.lb_status.p, 0, (size_t)((s->n + bt - 1) / bt + 1) * 8, ls));
        if (f.depth_order) roofgs_depth_order(f, w, ls);
        fv->views[v] = f.fa;
        fv->block_prefix[v] = blocks;
        blocks += (unsigned)((s->n + bt - 1) / bt);
        sorts[v] = f.sa;
    }
    fv->block_prefix[V] = blocks;
    fv->n_views = V;
    fv->claim = P.claim.as<unsigned>();
    RG_CK(cudaMemsetAsync(P.claim.p, 0, 2 * sizeof(unsigned), P.cap));
    for (int l = 0; l < lanes; l++) {
        RG_CK(cudaEventRecord(P.join[l], P.streams[l]));
        RG_CK(cudaStreamWaitEvent(P.cap, P.join[l], 0));
    }
    launch_frontend_views(*fv, P.cap);
    RG_CK(cudaEventRecord(P.fork, P.cap));
    for (int l = 0; l < lanes; l++) RG_CK(cudaStreamWaitEvent(P.streams[l], P.fork, 0));
    for (int v = 0; v < V; v++) launch_sort(sorts[v], P.streams[v % lanes], nullptr);
    for (int l = 0; l < lanes; l++) {
        RG_CK(cudaEventRecord(P.join[l], P.streams[l]));
        RG_CK(cudaStreamWaitEvent(P.cap, P.join[l], 0));
    }
    for (int v = 0; v < V; v++) {
        roofgs_raster_args(P.scenes[v], P.vws[v], F[v], fl, outs[v], rv->views[v]);
        rv->tile_prefix[v] = items;
        items += (unsigned)F[v].tiles;
    }
    rv->tile_prefix[V] = items;
    rv->n_views = V;
    rv->claim = P.claim.as<unsigned>() + 1;
    launch_raster_views(*rv, (fl & RG_FLAG_EXACT_EXP) ? 0 : 1, rv->views[0].ppt, P.cap);
    RG_CK(cudaGetLastError());
    return RG_OK;
}

// Capture all views on `lanes` lanes (the fused path if `fused`) and bring P.exec up to date.
rg_status plan_capture(BatchPlan& P, const std::vector<FrameLayout>& F, float* const* outs, int lanes,
                       uint32_t raster_flags, bool fused)
{
    RG_CK(cudaStreamBeginCapture(P.cap, cudaStreamCaptureModeThreadLocal));
    rg_status err = RG_OK;
    cudaError_t ce = cudaEventRecord(P.fork, P.cap);
    for (int l = 0; l < lanes && ce == cudaSuccess; l++) ce = cudaStreamWaitEvent(P.streams[l], P.fork, 0);
    const uint32_t fl = (P.flags & ~(RG_FLAG_STAGE_EVENTS | RG_FLAG_SINGLE_PIXEL | RG_FLAG_QUAD_PIXEL |
                                     RG_FLAG_BATCH_FUSED | RG_FLAG_BATCH_LANES)) | raster_flags;
    if (fused && ce == cudaSuccess) {
        err = enqueue_fused(P, F, outs, lanes, fl);
    } else {
        for (size_t v = 0; v < F.size() && ce == cudaSuccess && err == RG_OK; v++)
            err = render_once(P.scenes[v], P.ws[v % lanes], F[v], P.mode, fl, outs[v], P.streams[v % lanes]);
        for (int l = 0; l < lanes && ce == cudaSuccess; l++) {
            ce = cudaEventRecord(P.join[l], P.streams[l]);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(P.cap, P.join[l], 0);
        }
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(P.cap, &g);
    if (err != RG_OK) {
        if (g) cudaGraphDestroy(g);
        return err;
    }
    if (ce != cudaSuccess || ee != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(RG_ERR_CUDA, std::string("batch capture failed: ") +
                                     cudaGetErrorString(ce != cudaSuccess ? ce : ee));
    }
    bool fresh = !P.exec || P.exec_lanes != lanes || P.exec_raster != raster_flags ||
                 (!F.empty() && P.exec_tw != F[0].cam.tw) || P.exec_fused != (int)fused;
    if (!fresh) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(P.exec, g, &info) != cudaSuccess) {
            cudaGetLastError();
            fresh = true;
        }
    }
    if (fresh) {
        if (P.exec) cudaGraphExecDestroy(P.exec);
        P.exec = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&P.exec, g, 0);
        if (ie != cudaSuccess) {
            cudaGraphDestroy(g);
            P.exec = nullptr;
            return fail(RG_ERR_CUDA, std::string("graph instantiation failed: ") + cudaGetErrorString(ie));
        }
        P.exec_lanes = lanes;
        P.exec_raster = raster_flags;
        P.exec_tw = F.empty() ? 0 : F[0].cam.tw;
        P.exec_fused = (int)fused;
    }
    cudaGraphDestroy(g);
    return RG_OK;
}

// layouts of all views for one tile shape
rg_status layouts_for(const rg_camera* cams, int n, int tw, int th, std::vector<FrameLayout>& F)
{
    F.resize((size_t)n);
    for (int v = 0; v < n; v++) RG_TRY(make_layout(&cams[v], F[v], tw, th));
    return RG_OK;
}

// candidate tile shapes of a plan
std::vector<std::pair<int, int>> plan_shapes(const BatchPlan& P)
{
    if (P.req_tw) return {{P.req_tw, P.req_th}};
    return {{16, 16}, {32, 8}, {8, 32}};
}

// Pick the tile shape, the lane count and the pixels per thread by timing the captured batch.
rg_status plan_tune(BatchPlan& P, const rg_camera* cams, float* const* outs, cudaStream_t st)
{
    const int V = (int)P.scenes.size();
    float best = 1e30f;
    int best_l = 1, best_tw = TILE, best_th = TILE;
    uint32_t best_r = 0;
    bool best_fused = false;
    // paths: the lanes (1, 2 or 4), and the fused path on 4 lanes; RG_FLAG_BATCH_FUSED /
    // RG_FLAG_BATCH_LANES keep one of them
    std::vector<std::pair<int, bool>> paths;
    if (!(P.flags & RG_FLAG_BATCH_FUSED))
        for (int lanes : {1, 2, 4}) paths.push_back({lanes, false});
    if (fused_possible(P) && P.vws) paths.push_back({std::min(BATCH_MAX_LANES, std::max(1, V)), true});
    cudaEvent_t e0, e1;
    RG_CK(cudaEventCreate(&e0));
    RG_CK(cudaEventCreate(&e1));
    std::vector<FrameLayout> F;
    rg_status e = RG_OK;
    for (auto shape : plan_shapes(P)) {
        e = layouts_for(cams, V, shape.first, shape.second, F);
        for (auto path : paths) {
            const int lanes = path.first;
            if (e != RG_OK) break;
            if (lanes > V && lanes > 1) continue;
            for (uint32_t r : {0u, (uint32_t)RG_FLAG_SINGLE_PIXEL, (uint32_t)RG_FLAG_QUAD_PIXEL}) {
                if (P.mode != RG_MODE_ROOFGS && r) continue;
                e = plan_capture(P, F, outs, lanes, r, path.second);
                if (e != RG_OK) break;
                float ms = 0.f;
                if (cudaGraphLaunch(P.exec, st) != cudaSuccess || cudaEventRecord(e0, st) != cudaSuccess ||
                    cudaGraphLaunch(P.exec, st) != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
                    cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                    e = fail(RG_ERR_CUDA, "timing the captured batch failed");
                    break;
                }
                if (ms < best) {
                    best = ms;
                    best_fused = path.second;
                    best_l = lanes;
                    best_r = r;
                    best_tw = shape.first;
                    best_th = shape.second;
                }
            }
        }
        if (e != RG_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != RG_OK) return e;
    if (best >= 1e30f) return fail(RG_ERR_UNSUPPORTED, "no batch path applies to these views and flags");
    P.lanes = best_l;
    P.fused = best_fused;
    P.raster_flags = best_r;
    P.tw = best_tw;
    P.th = best_th;
    P.tuned = true;
    return RG_OK;
}


} // namespace

// drop every plan that renders from scene s (called when s is destroyed)
void rg::drop_plans_of(const rg_scene* s)
{
    std::lock_guard<std::mutex> lock(g_batch_mu);
    for (size_t k = 0; k < g_plans.size();) {
        bool uses = false;
        for (rg_scene* x : g_plans[k]->scenes) uses |= (x == s);
        if (uses) g_plans.erase(g_plans.begin() + k);
        else k++;
    }
}


extern "C" {

rg_status rg_render_batch(rg_scene* const* scenes, const int32_t* scene_idx, const rg_camera* cams, int32_t n,
                          const rg_render_opts* opts, float* const* outs, void* stream)
{
    if (n < 0) return fail(RG_ERR_INVALID_ARG, "negative view count");
    if (n == 0) return RG_OK;
    if (!scenes || !scene_idx || !cams || !opts || !outs) return fail(RG_ERR_INVALID_ARG, "NULL argument");
    const int mode = opts->mode;
    if (mode != RG_MODE_EXACT && mode != RG_MODE_ROOFGS) return fail(RG_ERR_INVALID_ARG, "unknown mode");
    // tile shape: 0 x 0 lets the autotuner choose among the built shapes
    const int req_tw = opts->tile_w, req_th = opts->tile_h;
    if ((req_tw || req_th) && !tile_shape_ok(req_tw, req_th))
        return fail(RG_ERR_UNSUPPORTED, "tile shapes built: 16x16, 32x8, 8x32 (or 0x0: autotuned)");
    std::vector<FrameLayout> F((size_t)n);
    std::vector<rg_scene*> vs((size_t)n);
    for (int v = 0; v < n; v++) {
        if (scene_idx[v] < 0) return fail(RG_ERR_INVALID_ARG, "negative scene index");
        rg_scene* s = scenes[scene_idx[v]];
        if (!s || !outs[v]) return fail(RG_ERR_INVALID_ARG, "NULL scene or output");
        if (mode == RG_MODE_EXACT && !(s->storage & RG_STORE_FP32))
            return fail(RG_ERR_INVALID_ARG, "exact mode needs RG_STORE_FP32");
        if (mode == RG_MODE_ROOFGS && !(s->storage & RG_STORE_COMPACT))
            return fail(RG_ERR_INVALID_ARG, "RoofGS mode needs RG_STORE_COMPACT");
        RG_TRY(make_layout(&cams[v], F[v], req_tw ? req_tw : TILE, req_th ? req_th : TILE));
        vs[v] = s;
    }
    int dev = 0;
    RG_CK(cudaGetDevice(&dev));
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(g_batch_mu);
    BatchPlan* P = nullptr;
    const uint32_t key_flags = opts->flags & ~(RG_FLAG_STAGE_EVENTS | RG_FLAG_SINGLE_PIXEL | RG_FLAG_QUAD_PIXEL | RG_FLAG_BATCH_CHECKED);
    if ((key_flags & RG_FLAG_BATCH_FUSED) && (mode != RG_MODE_ROOFGS || n > MAX_BATCH_VIEWS))
        return fail(RG_ERR_UNSUPPORTED, "the fused batch path renders RoofGS mode, at most 32 views");
    for (auto& p : g_plans) {
        if (p->device != dev || p->mode != mode || p->flags != key_flags || p->scenes != vs || p->req_tw != req_tw ||
            p->req_th != req_th)
            continue;
        bool same = true;
        for (int v = 0; v < n && same; v++) same = p->widths[v] == F[v].cam.W && p->heights[v] == F[v].cam.H;
        if (same) {
            P = p.get();
            break;
        }
    }
    const bool fresh = P == nullptr;
    if (fresh) {
        std::unique_ptr<BatchPlan> np(new BatchPlan());
        np->device = dev;
        np->scenes = vs;
        np->mode = mode;
        np->flags = key_flags;
        np->req_tw = req_tw;
        np->req_th = req_th;
        for (int v = 0; v < n; v++) {
            np->widths.push_back(F[v].cam.W);
            np->heights.push_back(F[v].cam.H);
        }
        RG_TRY(plan_init(*np));
        for (auto shape : plan_shapes(*np)) { // lanes sized for every candidate tile shape
            std::vector<FrameLayout> Fs;
            RG_TRY(layouts_for(cams, n, shape.first, shape.second, Fs));
            RG_TRY(plan_size(*np, Fs, outs, st));
        }
        RG_TRY(plan_tune(*np, cams, outs, st));
        if (g_plans.size() >= 8) g_plans.erase(g_plans.begin());
        g_plans.push_back(std::move(np));
        P = g_plans.back().get();
    }
    RG_TRY(layouts_for(cams, n, P->tw, P->th, F));
    RG_TRY(plan_capture(*P, F, outs, P->lanes, P->raster_flags, P->fused));
    RG_CK(cudaGraphLaunch(P->exec, st));
    if (opts->flags & RG_FLAG_BATCH_CHECKED) {
        // synchronous check: resize and render again if a view overflowed its lane
        bool over = false;
        for (rg_scene* s : P->scenes) {
            Sticky h;
            RG_CK(cudaMemcpyAsync(&h, s->sticky.p, sizeof(h), cudaMemcpyDeviceToHost, st));
            RG_CK(cudaStreamSynchronize(st));
            if (h.error) return fail(RG_ERR_TIMEOUT, "a bounded device wait gave up");
            over |= h.overflow != 0;
        }
        if (over) { // grow the lanes (never shrink) for these views and render again
            RG_TRY(plan_size(*P, F, outs, st));
            RG_TRY(plan_capture(*P, F, outs, P->lanes, P->raster_flags, P->fused));
            RG_CK(cudaGraphLaunch(P->exec, st));
            RG_CK(cudaStreamSynchronize(st));
        }
    }
    return RG_OK;
}

// Lane count and pixels per thread the autotuner chose for the plan of these views
// (0 lanes if no plan exists yet).
rg_status rg_batch_plan_info(rg_scene* const* scenes, const int32_t* scene_idx, const rg_camera* cams, int32_t n,
                             const rg_render_opts* opts, int32_t* lanes, int32_t* pixels_per_thread, int32_t* tile_w,
                             int32_t* tile_h, int32_t* fused)
{
    if (!scenes || !scene_idx || !cams || !opts || !lanes || !pixels_per_thread || n <= 0)
        return fail(RG_ERR_INVALID_ARG, "bad arguments");
    *lanes = 0;
    *pixels_per_thread = 0;
    int dev = 0;
    RG_CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_batch_mu);
    const uint32_t key_flags = opts->flags & ~(RG_FLAG_STAGE_EVENTS | RG_FLAG_SINGLE_PIXEL | RG_FLAG_QUAD_PIXEL | RG_FLAG_BATCH_CHECKED);
    for (auto& p : g_plans) {
        if (p->device != dev || p->mode != opts->mode || p->flags != key_flags || (int)p->scenes.size() != n ||
            p->req_tw != opts->tile_w || p->req_th != opts->tile_h)
            continue;
        bool same = true;
        for (int v = 0; v < n && same; v++)
            same = p->scenes[v] == scenes[scene_idx[v]] && p->widths[v] == cams[v].width && p->heights[v] == cams[v].height;
        if (same) {
            *lanes = p->lanes;
            *pixels_per_thread = (p->raster_flags & RG_FLAG_SINGLE_PIXEL) ? 1 : ((p->raster_flags & RG_FLAG_QUAD_PIXEL) ? 4 : 2);
            if (tile_w) *tile_w = p->tw;
            if (tile_h) *tile_h = p->th;
            if (fused) *fused = p->fused ? 1 : 0;
            return RG_OK;
        }
    }
    return RG_OK;
}

} // extern "C"
