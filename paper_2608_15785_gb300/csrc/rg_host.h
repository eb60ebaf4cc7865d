// rg_host.h -- host-side internals shared by the C ABI translation units
// (rg_api.cu: scenes, frames, scene files, backward; rg_batch.cu: batched
// rendering; rg_serve.cu: the request loop): error reporting, device buffers,
// the frame workspace, the scene object and the per-frame pipeline.
#pragma once

#include <cstdint>
#include <string>

#include "rg.h"
#include "rg_internal.cuh"

namespace rg {

// records the message rg_last_error() returns (thread-local) and returns s
rg_status fail(rg_status s, const std::string& msg);

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
rg_status ensure(DevBuf& b, size_t bytes, const char* what);

constexpr int EV_RING = 512;
constexpr int EV_PER_FRAME = 7; // start, depth order, front end, histogram, sort, ranges, raster
constexpr long long MAX_CAP = (1ll << 30) - 1;
constexpr size_t CTRL_BYTES = sizeof(Counters) + 8 * 256 * sizeof(unsigned);
// frame counters, the per-Gaussian depth sort's, then the producers' digit-count copies
// ([copy][2][256] from the fused front end, [copy][8][256] from the exact duplicate)
constexpr size_t FE_HIST_BYTES = (size_t)FE_HIST_COPIES * 8 * 256 * sizeof(unsigned);
constexpr size_t CTRL_ALLOC = 2 * CTRL_BYTES + FE_HIST_BYTES;

// Frame workspace: everything one frame in flight needs besides the scene.
// rg_render uses the scene's own workspace; a batch lane or a server slot owns one.
struct Workspace {
    int64_t cap = 0;
    DevBuf keys[2], vals[2];
    DevBuf ranges;
    DevBuf ctrl; // Counters followed by hist[8][256] (twice: frame, depth sort)
    DevBuf lb_status;
    DevBuf sort_status[2];
    DevBuf mean2, depth, quad, rgb, rect, touched, offsets; // exact per-Gaussian
    DevBuf rec;                                           // RoofGS raster records
    DevBuf gkeys[2], gvals[2], gstatus[2];                // RoofGS per-Gaussian depth sort
    DevBuf gbuf;                                          // backward: image-space gradients [n][9]
    DevBuf tsort;                                         // RoofGS per-tile counting sort: matrix + tile totals
    DevBuf rowbuf; // RoofGS row-bucketed front end: rows and row tests per slot, counts per tile row
    // last frame
    int last_mode = -1;
    int last_passes = 0;
    int last_tiles = 0;
    bool last_key16 = false; // entries carried 16-bit tile ids (the 32-bit keys are rebuilt on inspection)
    bool last_tilesort = false; // the entries were grouped by the per-tile counting sort (keys rebuilt from ranges)
    bool last_cols = false;  // the 16-bit keys were column-major (tx << 8 | ty): entries regrouped from the ranges
    int last_bd = 0;         // b_d of the last RoofGS frame
    int last_gfin = 0;       // buffer of the per-Gaussian depth sort's result
    // stage events
    bool ev_init = false;
    cudaEvent_t ev[EV_RING][EV_PER_FRAME];
    int ev_next = 0;
    int ev_pending = 0;

    void release()
    {
        DevBuf* bufs[] = {&keys[0], &keys[1], &vals[0], &vals[1], &ranges, &ctrl, &lb_status, &sort_status[0],
                          &sort_status[1], &mean2, &depth, &quad, &rgb, &rect, &touched, &offsets, &rec, &gkeys[0],
                          &gkeys[1], &gvals[0], &gvals[1], &gstatus[0], &gstatus[1], &gbuf, &tsort, &rowbuf};
        for (DevBuf* b : bufs) b->release();
        if (ev_init)
            for (int f = 0; f < EV_RING; f++)
                for (int k = 0; k < EV_PER_FRAME; k++) cudaEventDestroy(ev[f][k]);
        ev_init = false;
        cap = 0;
    }
};

} // namespace rg

struct rg_scene {
    int device = 0;
    int64_t n = 0;
    int sh_degree = 3;
    uint32_t storage = 0;
    int sh_scale_mode = 0;
    // exact-mode attributes (FP32)
    rg::DevBuf means, scales, quats, opac, sh;
    // compact attributes (RoofGS mode)
    rg::DevBuf geoA, geoB, shq;
    float band_scale[12] = {0};
    rg::DevBuf sticky; // Sticky flags of every frame rendered from this scene
    rg::Workspace ws;  // frame workspace of rg_render / rg_backward
};

namespace rg {

// camera, tile grid and key layout of one frame
struct FrameLayout {
    Layout lay;
    CamDev cam;
    int tiles;
};

// tile shapes with kernels: 16 x 16, 32 x 8, 8 x 32
bool tile_shape_ok(int tw, int th);
// tile shape of a render option block (0 = the default 16 x 16); RG_ERR_UNSUPPORTED otherwise
rg_status tile_shape(const rg_render_opts* o, int& tw, int& th);
// checks the camera and derives the frame layout (Sec. IV-A.2 key split) for a tile shape
rg_status make_layout(const rg_camera* c, FrameLayout& f, int tw = TILE, int th = TILE);
// grows a workspace for a frame of n_gauss Gaussians, `tiles` tiles and `cap` entries
rg_status ensure_workspace(Workspace& w, int64_t n_gauss, int mode, int tiles, int64_t cap);
// creates the stage events of a workspace on first use
void init_events(Workspace& w);
// enqueues one frame on `st` (arguments and workspace already checked); out == nullptr stops
// after the ranges; count selects the counting rasterizer
rg_status render_once(rg_scene* s, Workspace& w, const FrameLayout& F, int mode, uint32_t flags, float* out,
                      cudaStream_t st, bool count = false);
// RoofGS frame in stages (rg_render runs them back to back; a batch's fused path runs every
// view's front end in one launch and every view's rasterizer in one persistent launch)
struct RoofgsFrame {
    FrontendArgs fa;  // fused front end
    SortArgs ga;      // per-Gaussian depth sort (if depth_order)
    SortArgs sa;      // entry sort
    bool depth_order; // Gaussians pre-sorted by quantized depth (not with RG_FLAG_SORT_FULL_KEY)
    bool tile_sort;   // RG_FLAG_TILE_COUNTING_SORT: ts replaces the radix passes sa
    TileSortArgs ts;
    int tile_shift;   // sorted key >> tile_shift = tile id
};
// RG_ERR_UNSUPPORTED if the flags ask for what the frame cannot do
rg_status roofgs_build(rg_scene* s, Workspace& w, const FrameLayout& F, uint32_t flags, RoofgsFrame& f);
void roofgs_depth_order(const RoofgsFrame& f, Workspace& w, cudaStream_t st);
void roofgs_raster_args(rg_scene* s, Workspace& w, const FrameLayout& F, uint32_t flags, float* out, RasterArgs& r);
// frees a scene and its workspace
void destroy_scene(rg_scene* s);
// drops the batch plans that render from scene s (rg_batch.cu)
void drop_plans_of(const rg_scene* s);

} // namespace rg
