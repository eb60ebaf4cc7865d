// rg_api.cu -- C ABI of the renderer: resident scenes, frame workspace and the
// per-frame launch sequence of both modes (see include/rg.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rg.h"
#include "rg_internal.cuh"

using namespace rg;

namespace {

thread_local std::string g_err;

rg_status fail(rg_status s, const std::string& msg)
{
    g_err = msg;
    return s;
}

#define RG_CK(call)                                                                                           \
    do {                                                                                                      \
        cudaError_t e_ = (call);                                                                              \
        if (e_ != cudaSuccess) return fail(RG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define RG_TRY(expr)                 \
    do {                             \
        rg_status s_ = (expr);       \
        if (s_ != RG_OK) return s_;  \
    } while (0)

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <typename T>
    T* as() const { return reinterpret_cast<T*>(p); }
};

// grow-only device allocation (contents are not preserved)
rg_status ensure(DevBuf& b, size_t bytes, const char* what)
{
    if (bytes == 0) bytes = 16;
    if (b.p && b.bytes >= bytes) return RG_OK;
    b.release();
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(RG_ERR_OOM, std::string("cudaMalloc failed for ") + what + " (" + std::to_string(bytes) + " bytes): " +
                                    cudaGetErrorString(e));
    }
    b.bytes = bytes;
    return RG_OK;
}

constexpr int EV_RING = 512;
constexpr int EV_PER_FRAME = 7; // start, depth order, front end, histogram, sort, ranges, raster
constexpr long long MAX_CAP = (1ll << 30) - 1;
constexpr size_t CTRL_BYTES = sizeof(Counters) + 8 * 256 * sizeof(unsigned);
constexpr size_t CTRL_ALLOC = 2 * CTRL_BYTES; // frame counters + the per-Gaussian depth sort's

} // namespace

void rg::set_last_error(const char* msg) { g_err = msg; }

struct rg_scene {
    int device = 0;
    int64_t n = 0;
    int sh_degree = 3;
    uint32_t storage = 0;
    int sh_scale_mode = 0;
    // exact-mode attributes (FP32)
    DevBuf means, scales, quats, opac, sh;
    // compact attributes (RoofGS mode)
    DevBuf geoA, geoB, shq;
    float band_scale[12] = {0};
    // frame workspace
    int64_t cap = 0;
    DevBuf keys[2], vals[2];
    DevBuf ranges;
    DevBuf ctrl;   // Counters followed by hist[8][256]
    DevBuf sticky; // Sticky
    DevBuf lb_status;
    DevBuf sort_status[2];
    DevBuf xy, depth, conic, rgb, rect, touched, offsets; // exact per-Gaussian
    DevBuf rec;                                           // RoofGS raster records
    DevBuf gkeys[2], gvals[2], gstatus[2];                // RoofGS per-Gaussian depth sort
    DevBuf gbuf;                                          // backward: image-space gradients [n][9]
    // last frame
    int last_mode = -1;
    int last_passes = 0;
    int last_tiles = 0;
    // stage events
    bool ev_init = false;
    cudaEvent_t ev[EV_RING][EV_PER_FRAME];
    int ev_next = 0;
    int ev_pending = 0;
};

namespace {

struct FrameLayout {
    Layout lay;
    CamDev cam;
    int tiles;
};

rg_status make_layout(const rg_camera* c, FrameLayout& f)
{
    if (!c) return fail(RG_ERR_INVALID_ARG, "camera is NULL");
    if (c->width <= 0 || c->height <= 0) return fail(RG_ERR_INVALID_ARG, "camera width/height must be positive");
    if (!(c->znear > 0.0f) || !(c->zfar > c->znear) || !std::isfinite(c->zfar))
        return fail(RG_ERR_INVALID_ARG, "camera needs 0 < znear < zfar < inf");
    for (int k = 0; k < 9; k++)
        if (!std::isfinite(c->R[k])) return fail(RG_ERR_INVALID_ARG, "camera rotation is not finite");
    for (int k = 0; k < 3; k++)
        if (!std::isfinite(c->t[k]) || !std::isfinite(c->bg[k]))
            return fail(RG_ERR_INVALID_ARG, "camera translation/background is not finite");
    if (!(c->fx > 0.0f) || !(c->fy > 0.0f) || !std::isfinite(c->fx) || !std::isfinite(c->fy) ||
        !std::isfinite(c->cx) || !std::isfinite(c->cy))
        return fail(RG_ERR_INVALID_ARG, "camera intrinsics must be finite with fx, fy > 0");
    Layout& L = f.lay;
    L.tiles_x = (c->width + TILE - 1) / TILE;
    L.tiles_y = (c->height + TILE - 1) / TILE;
    const long long nt = (long long)L.tiles_x * L.tiles_y;
    if (nt > (1ll << 26)) return fail(RG_ERR_INVALID_ARG, "image too large");
    int b = 0;
    while ((1ll << b) < nt) b++; // b_t = ceil(log2 N_t), Sec. IV-A.2
    L.b_t = b;
    L.b_d = 32 - b;
    L.qmax = (L.b_d >= 32) ? 0xffffffffu : (unsigned)((1ull << L.b_d) - 1ull);
    L.depth_scale = (float)((double)L.qmax / ((double)c->zfar - (double)c->znear));
    f.tiles = (int)nt;
    CamDev& d = f.cam;
    memcpy(d.R, c->R, sizeof(d.R));
    memcpy(d.t, c->t, sizeof(d.t));
    memcpy(d.bg, c->bg, sizeof(d.bg));
    d.fx = c->fx;
    d.fy = c->fy;
    d.cx = c->cx;
    d.cy = c->cy;
    d.W = c->width;
    d.H = c->height;
    d.zn = c->znear;
    d.zf = c->zfar;
    for (int j = 0; j < 3; j++)
        d.campos[j] = (float)-((double)c->R[j] * c->t[0] + (double)c->R[3 + j] * c->t[1] + (double)c->R[6 + j] * c->t[2]);
    // pinned FP32: 1.3 * ((0.5 * W) / f), one rounding per operation
    volatile float halfw = 0.5f * (float)c->width, halfh = 0.5f * (float)c->height;
    volatile float tx = halfw / c->fx, ty = halfh / c->fy;
    d.limx = 1.3f * tx;
    d.limy = 1.3f * ty;
    return RG_OK;
}

rg_status ensure_workspace(rg_scene* s, int mode, int tiles, int64_t cap)
{
    const int64_t n = s->n > 0 ? s->n : 1;
    if (cap > MAX_CAP) return fail(RG_ERR_CAPACITY, "entry capacity above 2^30 - 1");
    if (cap > s->cap || !s->keys[0].p) {
        for (int k = 0; k < 2; k++) {
            RG_TRY(ensure(s->keys[k], (size_t)cap * 8, "keys"));
            RG_TRY(ensure(s->vals[k], (size_t)cap * 4, "values"));
        }
        const int64_t max_tiles = (cap + sort_tile_items() - 1) / sort_tile_items();
        for (int k = 0; k < 2; k++) RG_TRY(ensure(s->sort_status[k], (size_t)max_tiles * 256 * 4, "sort status"));
        s->cap = cap;
    }
    RG_TRY(ensure(s->ranges, (size_t)tiles * sizeof(uint2), "ranges"));
    RG_TRY(ensure(s->ctrl, CTRL_ALLOC, "counters"));
    RG_TRY(ensure(s->lb_status, (size_t)((n + 255) / 256 + 1) * 8, "look-back status"));
    if (mode == RG_MODE_EXACT) {
        RG_TRY(ensure(s->xy, (size_t)n * 8, "xy"));
        RG_TRY(ensure(s->depth, (size_t)n * 4, "depth"));
        RG_TRY(ensure(s->conic, (size_t)n * 16, "conic"));
        RG_TRY(ensure(s->rgb, (size_t)n * 12, "rgb"));
        RG_TRY(ensure(s->rect, (size_t)n * 16, "rect"));
        RG_TRY(ensure(s->touched, (size_t)n * 4, "touched"));
        RG_TRY(ensure(s->offsets, (size_t)n * 4, "offsets"));
    } else {
        RG_TRY(ensure(s->rec, (size_t)n * 32, "records"));
        for (int k = 0; k < 2; k++) {
            RG_TRY(ensure(s->gkeys[k], (size_t)n * 4, "depth keys"));
            RG_TRY(ensure(s->gvals[k], (size_t)n * 4, "depth order"));
            RG_TRY(ensure(s->gstatus[k], (size_t)((n + sort_tile_items() - 1) / sort_tile_items()) * 256 * 4,
                          "depth sort status"));
        }
    }
    return RG_OK;
}

void init_events(rg_scene* s)
{
    if (s->ev_init) return;
    for (int f = 0; f < EV_RING; f++)
        for (int k = 0; k < EV_PER_FRAME; k++) cudaEventCreate(&s->ev[f][k]);
    s->ev_init = true;
}

// One frame on `st`; the caller has checked arguments and the workspace.
rg_status render_once(rg_scene* s, const FrameLayout& F, int mode, uint32_t flags, float* out, cudaStream_t st,
                      bool count = false)
{
    Counters* ctr = s->ctrl.as<Counters>();
    unsigned* hist = reinterpret_cast<unsigned*>(s->ctrl.as<unsigned char>() + sizeof(Counters));
    Sticky* sticky = s->sticky.as<Sticky>();
    const bool ev = (flags & RG_FLAG_STAGE_EVENTS) != 0;
    cudaEvent_t* E = nullptr;
    if (ev) {
        init_events(s);
        E = s->ev[s->ev_next];
        s->ev_next = (s->ev_next + 1) % EV_RING;
        if (s->ev_pending < EV_RING) s->ev_pending++;
        RG_CK(cudaEventRecord(E[0], st));
    }
    RG_CK(cudaMemsetAsync(s->ctrl.p, 0, CTRL_ALLOC, st));
    RG_CK(cudaMemsetAsync(s->ranges.p, 0, (size_t)F.tiles * sizeof(uint2), st));
    const long long n = s->n;
    SortArgs sa;
    memset(&sa, 0, sizeof(sa));
    for (int k = 0; k < 2; k++) {
        sa.keys[k] = s->keys[k].p;
        sa.vals[k] = s->vals[k].as<unsigned>();
        sa.status[k] = s->sort_status[k].as<unsigned>();
    }
    sa.cap = s->cap;
    sa.hist = hist;
    sa.max_tiles = (s->cap + sort_tile_items() - 1) / sort_tile_items();
    sa.ctr = ctr;
    sa.sticky = sticky;
    int tile_shift;
    if (mode == RG_MODE_EXACT) {
        ExactArgs a;
        memset(&a, 0, sizeof(a));
        a.means = s->means.as<float>();
        a.scales = s->scales.as<float>();
        a.quats = s->quats.as<float>();
        a.opac = s->opac.as<float>();
        a.sh = s->sh.as<float>();
        a.sh_degree = s->sh_degree;
        a.n = n;
        a.cam = F.cam;
        a.lay = F.lay;
        a.xy = s->xy.as<float2>();
        a.depth = s->depth.as<float>();
        a.conic_op = s->conic.as<float4>();
        a.rgb = s->rgb.as<float>();
        a.rect = s->rect.as<int4>();
        a.touched = s->touched.as<unsigned>();
        a.offsets = s->offsets.as<unsigned>();
        a.keys = s->keys[0].as<unsigned long long>();
        a.vals = s->vals[0].as<unsigned>();
        a.cap = s->cap;
        a.status = s->lb_status.as<unsigned long long>();
        a.ctr = ctr;
        a.sticky = sticky;
        RG_CK(cudaMemsetAsync(s->lb_status.p, 0, (size_t)((n + 2047) / 2048 + 1) * 8, st));
        if (ev) RG_CK(cudaEventRecord(E[1], st));
        launch_exact_preprocess(a, st);
        launch_exact_scan(a, st);
        launch_exact_duplicate(a, st);
        sa.key_bytes = 8;
        sa.passes = (32 + F.lay.b_t + 7) / 8; // only the bits that can be non-zero
        tile_shift = 32;
    } else {
        FrontendArgs a;
        memset(&a, 0, sizeof(a));
        a.geoA = s->geoA.as<float4>();
        a.geoB = s->geoB.as<uint4>();
        a.shq = s->shq.as<uint4>();
        for (int k = 0; k < 12; k++) a.band_scale[k] = (k / 3 <= s->sh_degree) ? s->band_scale[k] : 0.0f;
        a.per_gauss_scale = s->sh_scale_mode == RG_SH_SCALE_BAND_GAUSS;
        a.sh_degree = s->sh_degree;
        a.n = n;
        a.cam = F.cam;
        a.lay = F.lay;
        a.rec = s->rec.as<float4>();
        a.keys = s->keys[0].as<unsigned>();
        a.vals = s->vals[0].as<unsigned>();
        a.cap = s->cap;
        a.status = s->lb_status.as<unsigned long long>();
        a.ctr = ctr;
        a.sticky = sticky;
        RG_CK(cudaMemsetAsync(s->lb_status.p, 0, (size_t)((n + 255) / 256 + 1) * 8, st));
        sa.key_bytes = 4;
        if (flags & RG_FLAG_SORT_FULL_KEY) {
            // the paper's scheme: entries in Gaussian order, 4 passes over the 32-bit key
            sa.passes = 4;
            sa.bit0 = 0;
            if (ev) RG_CK(cudaEventRecord(E[1], st));
        } else {
            // Gaussians sorted by quantized depth first (stable, ties by index); the
            // entries then come out in (q_d, index) order and a stable sort of the
            // b_t tile bits alone yields the order of the full 32-bit key
            SortArgs ga;
            memset(&ga, 0, sizeof(ga));
            for (int k = 0; k < 2; k++) {
                ga.keys[k] = s->gkeys[k].p;
                ga.vals[k] = s->gvals[k].as<unsigned>();
                ga.status[k] = s->gstatus[k].as<unsigned>();
            }
            Counters* gctr = reinterpret_cast<Counters*>(s->ctrl.as<unsigned char>() + CTRL_BYTES);
            ga.cap = n;
            ga.key_bytes = 4;
            ga.passes = (F.lay.b_d + 7) / 8;
            ga.bit0 = 0;
            ga.hist = reinterpret_cast<unsigned*>(s->ctrl.as<unsigned char>() + CTRL_BYTES + sizeof(Counters));
            ga.max_tiles = (n + sort_tile_items() - 1) / sort_tile_items();
            ga.ctr = gctr;
            ga.sticky = sticky;
            launch_depth_keys(a, s->gkeys[0].as<unsigned>(), s->gvals[0].as<unsigned>(), gctr, st);
            launch_sort(ga, st, nullptr);
            a.order = s->gvals[ga.passes & 1].as<unsigned>();
            if (ev) RG_CK(cudaEventRecord(E[1], st));
            sa.passes = (F.lay.b_t + 7) / 8;
            sa.bit0 = F.lay.b_d;
            // depth-ordered entries of one Gaussian row carry consecutive tiles, so the warp
            // holds many distinct low tile digits: rank that pass with ballots
            sa.ballot_mask = 1;
        }
        launch_frontend_fused(a, st);
        tile_shift = F.lay.b_d;
    }
    if (ev) RG_CK(cudaEventRecord(E[2], st));
    if (ev && sa.passes <= 0) RG_CK(cudaEventRecord(E[3], st));
    launch_sort(sa, st, ev ? E[3] : nullptr);
    if (ev) RG_CK(cudaEventRecord(E[4], st));
    const int fin = sa.passes & 1;
    RangeArgs ra;
    ra.keys = s->keys[fin].p;
    ra.key_bytes = sa.key_bytes;
    ra.tile_shift = tile_shift;
    ra.ntiles = F.tiles;
    ra.ranges = s->ranges.as<uint2>();
    ra.ctr = ctr;
    launch_ranges(ra, st);
    if (ev) RG_CK(cudaEventRecord(E[5], st));
    s->last_mode = mode;
    s->last_passes = sa.passes;
    s->last_tiles = F.tiles;
    if (!out) { // front end, sort and ranges only (the backward replays the blend itself)
        if (ev) RG_CK(cudaEventRecord(E[6], st));
        RG_CK(cudaGetLastError());
        return RG_OK;
    }
    RasterArgs r;
    memset(&r, 0, sizeof(r));
    r.ranges = s->ranges.as<uint2>();
    r.vals = s->vals[fin].as<unsigned>();
    r.n = n;
    r.tiles_x = F.lay.tiles_x;
    r.tiles_y = F.lay.tiles_y;
    r.cam = F.cam;
    r.out = out;
    r.count = count ? ctr : nullptr;
    if (mode == RG_MODE_EXACT) {
        r.xy = s->xy.as<float2>();
        r.conic_op = s->conic.as<float4>();
        r.rgb = s->rgb.as<float>();
        launch_raster_exact(r, st);
    } else {
        r.rec = s->rec.as<float4>();
        r.fast_exp = (flags & RG_FLAG_EXACT_EXP) ? 0 : 1;
        r.dual_pixel = (flags & RG_FLAG_SINGLE_PIXEL) ? 0 : 1;
        launch_raster_roofgs(r, st);
    }
    if (ev) RG_CK(cudaEventRecord(E[6], st));
    RG_CK(cudaGetLastError());
    s->last_mode = mode;
    s->last_passes = sa.passes;
    s->last_tiles = F.tiles;
    return RG_OK;
}

rg_status upload(DevBuf& dst, const float* src, size_t count, int on_device, cudaStream_t st, const char* what)
{
    RG_TRY(ensure(dst, count * 4, what));
    if (count) RG_CK(cudaMemcpyAsync(dst.p, src, count * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    return RG_OK;
}

void destroy_scene(rg_scene* s)
{
    DevBuf* bufs[] = {&s->gbuf, &s->gkeys[0], &s->gkeys[1], &s->gvals[0], &s->gvals[1], &s->gstatus[0], &s->gstatus[1],
                      &s->means, &s->scales, &s->quats, &s->opac, &s->sh, &s->geoA, &s->geoB, &s->shq, &s->keys[0],
                      &s->keys[1], &s->vals[0], &s->vals[1], &s->ranges, &s->ctrl, &s->sticky, &s->lb_status,
                      &s->sort_status[0], &s->sort_status[1], &s->xy, &s->depth, &s->conic, &s->rgb, &s->rect,
                      &s->touched, &s->offsets, &s->rec};
    for (DevBuf* b : bufs) b->release();
    if (s->ev_init)
        for (int f = 0; f < EV_RING; f++)
            for (int k = 0; k < EV_PER_FRAME; k++) cudaEventDestroy(s->ev[f][k]);
    delete s;
}

} // namespace

extern "C" {

int32_t rg_version(void) { return 100; }

const char* rg_last_error(void) { return g_err.c_str(); }

rg_status rg_scene_create(const rg_scene_desc* desc, void* stream, rg_scene** out)
{
    if (!out) return fail(RG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!desc) return fail(RG_ERR_INVALID_ARG, "desc is NULL");
    if (desc->n < 0 || desc->n > (1ll << 31)) return fail(RG_ERR_INVALID_ARG, "n out of range");
    if (desc->sh_degree < 0 || desc->sh_degree > 3) return fail(RG_ERR_INVALID_ARG, "sh_degree must be 0..3");
    if (desc->sh_scale_mode != RG_SH_SCALE_BAND && desc->sh_scale_mode != RG_SH_SCALE_BAND_GAUSS)
        return fail(RG_ERR_INVALID_ARG, "unknown sh_scale_mode");
    const int64_t n = desc->n;
    if (n > 0 && (!desc->means || !desc->scales || !desc->quats || !desc->opacities || !desc->sh))
        return fail(RG_ERR_INVALID_ARG, "an attribute pointer is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    rg_scene* s = new rg_scene();
    cudaGetDevice(&s->device);
    s->n = n;
    s->sh_degree = desc->sh_degree;
    s->storage = desc->storage ? desc->storage : (RG_STORE_FP32 | RG_STORE_COMPACT);
    s->sh_scale_mode = desc->sh_scale_mode;
    auto bail = [&](rg_status e) {
        cudaStreamSynchronize(st);
        destroy_scene(s);
        return e;
    };
    // stage the FP32 inputs on the device
    DevBuf tm, ts, tq, to, tsh, flag, logo, maxbits;
    auto cleanup = [&]() {
        tm.release(); ts.release(); tq.release(); to.release(); tsh.release();
        flag.release(); logo.release(); maxbits.release();
    };
    rg_status e;
#define RG_STEP(expr)               \
    do {                            \
        e = (expr);                 \
        if (e != RG_OK) {           \
            cleanup();              \
            return bail(e);         \
        }                           \
    } while (0)
    const bool keep32 = (s->storage & RG_STORE_FP32) != 0;
    RG_STEP(upload(keep32 ? s->means : tm, desc->means, (size_t)n * 3, desc->on_device, st, "means"));
    RG_STEP(upload(keep32 ? s->scales : ts, desc->scales, (size_t)n * 3, desc->on_device, st, "scales"));
    RG_STEP(upload(keep32 ? s->quats : tq, desc->quats, (size_t)n * 4, desc->on_device, st, "quats"));
    RG_STEP(upload(keep32 ? s->opac : to, desc->opacities, (size_t)n, desc->on_device, st, "opacities"));
    RG_STEP(upload(keep32 ? s->sh : tsh, desc->sh, (size_t)n * 48, desc->on_device, st, "sh"));
    const float* dm = keep32 ? s->means.as<float>() : tm.as<float>();
    const float* ds = keep32 ? s->scales.as<float>() : ts.as<float>();
    const float* dq = keep32 ? s->quats.as<float>() : tq.as<float>();
    const float* dop = keep32 ? s->opac.as<float>() : to.as<float>();
    const float* dsh = keep32 ? s->sh.as<float>() : tsh.as<float>();
    RG_STEP(ensure(flag, 16, "flag"));
    RG_STEP(ensure(s->sticky, sizeof(Sticky), "sticky"));
    if (cudaMemsetAsync(s->sticky.p, 0, sizeof(Sticky), st) != cudaSuccess) RG_STEP(fail(RG_ERR_CUDA, "memset"));
    if (cudaMemsetAsync(flag.p, 0, 16, st) != cudaSuccess) RG_STEP(fail(RG_ERR_CUDA, "memset"));
    launch_check_finite(dm, n * 3, flag.as<unsigned>(), st);
    launch_check_finite(ds, n * 3, flag.as<unsigned>(), st);
    launch_check_finite(dq, n * 4, flag.as<unsigned>(), st);
    launch_check_finite(dop, n, flag.as<unsigned>(), st);
    launch_check_finite(dsh, n * 48, flag.as<unsigned>(), st);
    // opacities on the host: range check and log o (FP64 log, rounded to FP32)
    std::vector<float> o((size_t)n), lo((size_t)n);
    if (n && cudaMemcpyAsync(o.data(), dop, (size_t)n * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        RG_STEP(fail(RG_ERR_CUDA, "copy opacities"));
    unsigned hflag = 0;
    if (cudaMemcpyAsync(&hflag, flag.p, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) RG_STEP(fail(RG_ERR_CUDA, "copy flag"));
    if (cudaStreamSynchronize(st) != cudaSuccess) RG_STEP(fail(RG_ERR_CUDA, std::string("scene upload: ") + cudaGetErrorString(cudaGetLastError())));
    if (hflag) RG_STEP(fail(RG_ERR_INVALID_ARG, "scene attributes contain non-finite values"));
    for (int64_t i = 0; i < n; i++) {
        if (!(o[i] >= 0.0f && o[i] <= 1.0f)) RG_STEP(fail(RG_ERR_INVALID_ARG, "opacity outside [0, 1]"));
        lo[i] = (float)std::log((double)o[i]);
    }
    if (s->storage & RG_STORE_COMPACT) {
        RG_STEP(ensure(logo, (size_t)n * 4, "log o"));
        RG_STEP(ensure(maxbits, 12 * 4, "sh max"));
        if (n && cudaMemcpyAsync(logo.p, lo.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
            RG_STEP(fail(RG_ERR_CUDA, "copy log o"));
        if (cudaMemsetAsync(maxbits.p, 0, 48, st) != cudaSuccess) RG_STEP(fail(RG_ERR_CUDA, "memset"));
        launch_sh_absmax(dsh, n, maxbits.as<unsigned>(), st);
        unsigned mb[12];
        if (cudaMemcpyAsync(mb, maxbits.p, 48, cudaMemcpyDeviceToHost, st) != cudaSuccess) RG_STEP(fail(RG_ERR_CUDA, "copy"));
        if (cudaStreamSynchronize(st) != cudaSuccess) RG_STEP(fail(RG_ERR_CUDA, "sh max"));
        for (int k = 0; k < 12; k++) { // s_{d,c} = max |SH| / 127 in FP32, Eq. (8)
            float m;
            memcpy(&m, &mb[k], 4);
            volatile float q = m / 127.0f;
            s->band_scale[k] = q;
        }
        RG_STEP(ensure(s->geoA, (size_t)(n ? n : 1) * 16, "geoA"));
        RG_STEP(ensure(s->geoB, (size_t)(n ? n : 1) * 16, "geoB"));
        RG_STEP(ensure(s->shq, (size_t)(n ? n : 1) * 48, "sh codes"));
        launch_compact(dm, ds, dq, logo.as<float>(), dsh, n, s->band_scale, s->sh_scale_mode == RG_SH_SCALE_BAND_GAUSS,
                       s->geoA.as<float4>(), s->geoB.as<uint4>(), s->shq.as<uint4>(), st);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        RG_STEP(fail(RG_ERR_CUDA, "scene conversion failed"));
    cleanup();
#undef RG_STEP
    *out = s;
    return RG_OK;
}

rg_status rg_scene_destroy(rg_scene* scene)
{
    if (!scene) return RG_OK;
    cudaDeviceSynchronize();
    destroy_scene(scene);
    return RG_OK;
}

rg_status rg_scene_reserve(rg_scene* scene, int64_t n_entries)
{
    if (!scene || n_entries < 0) return fail(RG_ERR_INVALID_ARG, "bad scene or size");
    if (n_entries <= scene->cap) return RG_OK;
    RG_CK(cudaDeviceSynchronize());
    const int64_t cap = n_entries;
    for (int k = 0; k < 2; k++) {
        RG_TRY(ensure(scene->keys[k], (size_t)cap * 8, "keys"));
        RG_TRY(ensure(scene->vals[k], (size_t)cap * 4, "values"));
    }
    const int64_t max_tiles = (cap + sort_tile_items() - 1) / sort_tile_items();
    for (int k = 0; k < 2; k++) RG_TRY(ensure(scene->sort_status[k], (size_t)max_tiles * 256 * 4, "sort status"));
    scene->cap = cap;
    return RG_OK;
}

rg_status rg_render(rg_scene* s, const rg_camera* cam, const rg_render_opts* opts, float* out_chw, rg_stats* stats,
                    void* stream)
{
    if (!s) return fail(RG_ERR_INVALID_ARG, "scene is NULL");
    if (!opts) return fail(RG_ERR_INVALID_ARG, "opts is NULL");
    if (!out_chw) return fail(RG_ERR_INVALID_ARG, "out is NULL");
    const int mode = opts->mode;
    if (mode != RG_MODE_EXACT && mode != RG_MODE_ROOFGS) return fail(RG_ERR_INVALID_ARG, "unknown mode");
    const int tw = opts->tile_w ? opts->tile_w : TILE, th = opts->tile_h ? opts->tile_h : TILE;
    if (tw != TILE || th != TILE) return fail(RG_ERR_UNSUPPORTED, "only 16x16 tiles are built");
    if (mode == RG_MODE_EXACT && !(s->storage & RG_STORE_FP32))
        return fail(RG_ERR_INVALID_ARG, "exact mode needs RG_STORE_FP32");
    if (mode == RG_MODE_ROOFGS && !(s->storage & RG_STORE_COMPACT))
        return fail(RG_ERR_INVALID_ARG, "RoofGS mode needs RG_STORE_COMPACT");
    FrameLayout F;
    RG_TRY(make_layout(cam, F));
    cudaStream_t st = (cudaStream_t)stream;
    int64_t cap = s->cap > 0 ? s->cap : std::max<int64_t>(1 << 20, 4 * s->n);
    if (cap > MAX_CAP) cap = MAX_CAP;
    RG_TRY(ensure_workspace(s, mode, F.tiles, cap));
    RG_TRY(render_once(s, F, mode, opts->flags, out_chw, st, stats != nullptr));
    if (!stats) return RG_OK;
    Counters c;
    RG_CK(cudaMemcpyAsync(&c, s->ctrl.p, sizeof(c), cudaMemcpyDeviceToHost, st));
    RG_CK(cudaStreamSynchronize(st));
    int regrown = 0;
    if (c.error) return fail(RG_ERR_TIMEOUT, "a bounded device wait gave up");
    if (c.n_entries_total > (unsigned long long)s->cap) {
        int64_t want = (int64_t)(c.n_entries_total + c.n_entries_total / 4 + 1024);
        if ((unsigned long long)want > (unsigned long long)MAX_CAP) want = MAX_CAP;
        if ((unsigned long long)want < c.n_entries_total)
            return fail(RG_ERR_CAPACITY, "frame needs more than 2^30 - 1 entries");
        RG_TRY(rg_scene_reserve(s, want));
        RG_TRY(render_once(s, F, mode, opts->flags, out_chw, st, true));
        RG_CK(cudaMemcpyAsync(&c, s->ctrl.p, sizeof(c), cudaMemcpyDeviceToHost, st));
        RG_CK(cudaStreamSynchronize(st));
        if (c.error) return fail(RG_ERR_TIMEOUT, "a bounded device wait gave up");
        if (c.n_entries_total > (unsigned long long)s->cap) return fail(RG_ERR_CAPACITY, "workspace could not grow enough");
        regrown = 1;
    }
    // the overflow of the first attempt is not an error once re-rendered
    if (regrown) {
        Sticky z = {0u, 0u};
        RG_CK(cudaMemcpyAsync(s->sticky.p, &z, sizeof(z), cudaMemcpyHostToDevice, st));
        RG_CK(cudaStreamSynchronize(st));
    }
    stats->n_gaussians = s->n;
    stats->n_front = c.n_front;
    stats->n_pairs = (int64_t)c.n_pairs;
    stats->n_blends = (int64_t)c.n_blends;
    stats->n_visible = c.n_visible;
    stats->n_entries = (int64_t)c.n_entries_total;
    stats->capacity = s->cap;
    stats->regrown = regrown;
    stats->sort_passes = s->last_passes;
    stats->b_t = F.lay.b_t;
    stats->b_d = mode == RG_MODE_ROOFGS ? F.lay.b_d : 32;
    stats->tiles_x = F.lay.tiles_x;
    stats->tiles_y = F.lay.tiles_y;
    return RG_OK;
}

rg_status rg_scene_check(rg_scene* s, void* stream)
{
    if (!s) return fail(RG_ERR_INVALID_ARG, "scene is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    Sticky h = {0u, 0u}, z = {0u, 0u};
    RG_CK(cudaMemcpyAsync(&h, s->sticky.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    RG_CK(cudaMemcpyAsync(s->sticky.p, &z, sizeof(z), cudaMemcpyHostToDevice, st));
    RG_CK(cudaStreamSynchronize(st));
    if (h.error) return fail(RG_ERR_TIMEOUT, "a bounded device wait gave up since the last check");
    if (h.overflow) return fail(RG_ERR_CAPACITY, "a frame exceeded its entry capacity since the last check");
    return RG_OK;
}

rg_status rg_stage_times(rg_scene* s, float* ms7, int32_t* frames)
{
    if (!s || !ms7) return fail(RG_ERR_INVALID_ARG, "NULL argument");
    for (int k = 0; k < 7; k++) ms7[k] = 0.0f;
    const int cnt = s->ev_pending;
    if (frames) *frames = cnt;
    if (!s->ev_init || cnt == 0) return RG_OK;
    for (int f = 0; f < cnt; f++) {
        const int slot = ((s->ev_next - 1 - f) % EV_RING + EV_RING) % EV_RING;
        cudaEvent_t* E = s->ev[slot];
        RG_CK(cudaEventSynchronize(E[6]));
        float t;
        for (int k = 0; k < 6; k++) {
            RG_CK(cudaEventElapsedTime(&t, E[k], E[k + 1]));
            ms7[k] += t;
        }
        RG_CK(cudaEventElapsedTime(&t, E[0], E[6]));
        ms7[6] += t;
    }
    s->ev_pending = 0;
    return RG_OK;
}

rg_status rg_inspect(rg_scene* s, int32_t what, void* host_dst, int64_t cap_bytes, int64_t* out_bytes)
{
    if (!s) return fail(RG_ERR_INVALID_ARG, "scene is NULL");
    RG_CK(cudaDeviceSynchronize());
    const int64_t n = s->n;
    std::vector<unsigned char> tmp;
    const void* src = nullptr;
    int64_t bytes = 0;
    bool device_src = true;
    switch (what) {
    case RG_INSPECT_KEYS:
    case RG_INSPECT_VALUES:
    case RG_INSPECT_RANGES: {
        if (s->last_mode < 0) return fail(RG_ERR_INVALID_ARG, "no frame rendered yet");
        Counters c;
        RG_CK(cudaMemcpy(&c, s->ctrl.p, sizeof(c), cudaMemcpyDeviceToHost));
        const int fin = s->last_passes & 1;
        if (what == RG_INSPECT_KEYS) {
            src = s->keys[fin].p;
            bytes = (int64_t)c.n_entries * (s->last_mode == RG_MODE_EXACT ? 8 : 4);
        } else if (what == RG_INSPECT_VALUES) {
            src = s->vals[fin].p;
            bytes = (int64_t)c.n_entries * 4;
        } else {
            src = s->ranges.p;
            bytes = (int64_t)s->last_tiles * 8;
        }
        break;
    }
    case RG_INSPECT_SH_CODES:
    case RG_INSPECT_GAUSS_SCALE:
    case RG_INSPECT_GEOM16:
    case RG_INSPECT_LOG_OPACITY: {
        if (!(s->storage & RG_STORE_COMPACT)) return fail(RG_ERR_INVALID_ARG, "scene has no compact attributes");
        if (what == RG_INSPECT_SH_CODES) {
            std::vector<unsigned char> planes((size_t)n * 48);
            if (n) RG_CK(cudaMemcpy(planes.data(), s->shq.p, (size_t)n * 48, cudaMemcpyDeviceToHost));
            tmp.resize((size_t)n * 48);
            for (int64_t i = 0; i < n; i++)
                for (int p = 0; p < 3; p++) memcpy(&tmp[(size_t)i * 48 + 16 * p], &planes[((size_t)p * n + i) * 16], 16);
            bytes = n * 48;
        } else if (what == RG_INSPECT_LOG_OPACITY) {
            std::vector<float> ga((size_t)n * 4);
            if (n) RG_CK(cudaMemcpy(ga.data(), s->geoA.p, (size_t)n * 16, cudaMemcpyDeviceToHost));
            tmp.resize((size_t)n * 4);
            for (int64_t i = 0; i < n; i++) memcpy(&tmp[(size_t)i * 4], &ga[(size_t)i * 4 + 3], 4);
            bytes = n * 4;
        } else {
            std::vector<uint16_t> gb((size_t)n * 8);
            if (n) RG_CK(cudaMemcpy(gb.data(), s->geoB.p, (size_t)n * 16, cudaMemcpyDeviceToHost));
            if (what == RG_INSPECT_GEOM16) {
                tmp.resize((size_t)n * 16);
                if (n) memcpy(tmp.data(), gb.data(), (size_t)n * 16);
                bytes = n * 16;
            } else {
                tmp.resize((size_t)n * 2);
                for (int64_t i = 0; i < n; i++) memcpy(&tmp[(size_t)i * 2], &gb[(size_t)i * 8 + 7], 2);
                bytes = n * 2;
            }
        }
        src = tmp.data();
        device_src = false;
        break;
    }
    case RG_INSPECT_SH_SCALES:
        src = s->band_scale;
        bytes = 48;
        device_src = false;
        break;
    default:
        return fail(RG_ERR_INVALID_ARG, "unknown inspect selector");
    }
    if (out_bytes) *out_bytes = bytes;
    if (!host_dst) return RG_OK;
    if (cap_bytes < bytes) return fail(RG_ERR_INVALID_ARG, "destination too small");
    if (bytes == 0) return RG_OK;
    if (device_src) RG_CK(cudaMemcpy(host_dst, src, (size_t)bytes, cudaMemcpyDeviceToHost));
    else memcpy(host_dst, src, (size_t)bytes);
    return RG_OK;
}

// Diagnostic: evaluate the bit-level exponential of Eq. (24) on device arrays.
rg_status rg_eval_fast_exp(const float* P_dev, float* out_dev, int64_t n, void* stream)
{
    if (n < 0 || (n > 0 && (!P_dev || !out_dev))) return fail(RG_ERR_INVALID_ARG, "bad arguments");
    launch_fast_exp_eval(P_dev, out_dev, n, (cudaStream_t)stream);
    RG_CK(cudaGetLastError());
    return RG_OK;
}

rg_status rg_render_batch(rg_scene* const*, const int32_t*, const rg_camera*, int32_t, const rg_render_opts*,
                          float* const*, void*)
{
    return fail(RG_ERR_UNSUPPORTED, "rg_render_batch is not built yet");
}

rg_status rg_backward(rg_scene* s, const rg_camera* cam, const rg_render_opts* opts, const float* dL_dimg,
                      const rg_grads* grads, void* stream)
{
    if (!s || !opts || !dL_dimg || !grads) return fail(RG_ERR_INVALID_ARG, "NULL argument");
    if (opts->mode != RG_MODE_EXACT)
        return fail(RG_ERR_UNSUPPORTED, "rg_backward differentiates exact mode only (RoofGS storage is INT8/FP16)");
    if (!(s->storage & RG_STORE_FP32)) return fail(RG_ERR_INVALID_ARG, "rg_backward needs RG_STORE_FP32");
    const int tw = opts->tile_w ? opts->tile_w : TILE, th = opts->tile_h ? opts->tile_h : TILE;
    if (tw != TILE || th != TILE) return fail(RG_ERR_UNSUPPORTED, "only 16x16 tiles are built");
    if (s->n > 0 && (!grads->means || !grads->scales || !grads->quats || !grads->opacities || !grads->sh))
        return fail(RG_ERR_INVALID_ARG, "a gradient pointer is NULL");
    FrameLayout F;
    RG_TRY(make_layout(cam, F));
    cudaStream_t st = (cudaStream_t)stream;
    int64_t cap = s->cap > 0 ? s->cap : std::max<int64_t>(1 << 20, 4 * s->n);
    if (cap > MAX_CAP) cap = MAX_CAP;
    RG_TRY(ensure_workspace(s, RG_MODE_EXACT, F.tiles, cap));
    // forward front end, sort and ranges of this camera (checked: the gradient needs every entry)
    for (int attempt = 0; attempt < 2; attempt++) {
        RG_TRY(render_once(s, F, RG_MODE_EXACT, 0u, nullptr, st));
        Counters c;
        RG_CK(cudaMemcpyAsync(&c, s->ctrl.p, sizeof(c), cudaMemcpyDeviceToHost, st));
        RG_CK(cudaStreamSynchronize(st));
        if (c.error) return fail(RG_ERR_TIMEOUT, "a bounded device wait gave up");
        if (c.n_entries_total <= (unsigned long long)s->cap) break;
        if (attempt == 1) return fail(RG_ERR_CAPACITY, "workspace could not grow enough");
        int64_t want = (int64_t)(c.n_entries_total + c.n_entries_total / 4 + 1024);
        if (want > MAX_CAP) return fail(RG_ERR_CAPACITY, "frame needs more than 2^30 - 1 entries");
        RG_TRY(rg_scene_reserve(s, want));
    }
    RG_TRY(ensure(s->gbuf, (size_t)(s->n > 0 ? s->n : 1) * 9 * 4, "gradient buffer"));
    RG_CK(cudaMemsetAsync(s->gbuf.p, 0, (size_t)(s->n > 0 ? s->n : 1) * 9 * 4, st));
    BackwardArgs b;
    memset(&b, 0, sizeof(b));
    const int fin = s->last_passes & 1;
    b.ranges = s->ranges.as<uint2>();
    b.vals = s->vals[fin].as<unsigned>();
    b.n = s->n;
    b.tiles_x = F.lay.tiles_x;
    b.tiles_y = F.lay.tiles_y;
    b.cam = F.cam;
    b.xy = s->xy.as<float2>();
    b.conic_op = s->conic.as<float4>();
    b.rgb = s->rgb.as<float>();
    b.touched = s->touched.as<unsigned>();
    b.means = s->means.as<float>();
    b.scales = s->scales.as<float>();
    b.quats = s->quats.as<float>();
    b.sh = s->sh.as<float>();
    b.sh_degree = s->sh_degree;
    b.dL_dimg = dL_dimg;
    b.gbuf = s->gbuf.as<float>();
    b.dmeans = grads->means;
    b.dscales = grads->scales;
    b.dquats = grads->quats;
    b.dopac = grads->opacities;
    b.dsh = grads->sh;
    launch_raster_backward(b, st);
    launch_preprocess_backward(b, st);
    RG_CK(cudaGetLastError());
    return RG_OK;
}

rg_status rg_submit(rg_server*, const rg_camera*, int32_t, uint64_t*)
{
    return fail(RG_ERR_UNSUPPORTED, "rg_submit is not built yet");
}

rg_status rg_poll(rg_server*, uint64_t, float*)
{
    return fail(RG_ERR_UNSUPPORTED, "rg_poll is not built yet");
}

} // extern "C"
