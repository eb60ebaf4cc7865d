// rg_api.cu -- C ABI of the renderer (declared in include/rg.h): resident
// scenes and scene files, the frame workspace and the per-frame launch sequence
// of both modes, inspection, and the backward. Batched rendering is in
// rg_batch.cu, the request loop in rg_serve.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "rg_host.h"

using namespace rg;

namespace {
thread_local std::string g_err;
} // namespace

rg_status rg::fail(rg_status s, const std::string& msg)
{
    g_err = msg;
    return s;
}

void rg::set_last_error(const char* msg) { g_err = msg; }

// grow-only device allocation (contents are not preserved)
rg_status rg::ensure(DevBuf& b, size_t bytes, const char* what)
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

namespace rg {

// Tile shapes with kernels: 256 pixels each, width a power of two.
bool tile_shape_ok(int tw, int th) { return (tw == 16 && th == 16) || (tw == 32 && th == 8) || (tw == 8 && th == 32); }

// tile shape of a render option block (0 = the default 16 x 16)
rg_status tile_shape(const rg_render_opts* o, int& tw, int& th)
{
    tw = o->tile_w ? o->tile_w : TILE;
    th = o->tile_h ? o->tile_h : TILE;
    if (!tile_shape_ok(tw, th)) return fail(RG_ERR_UNSUPPORTED, "tile shapes built: 16x16, 32x8, 8x32");
    return RG_OK;
}

rg_status make_layout(const rg_camera* c, FrameLayout& f, int tw, int th)
{
    if (!tile_shape_ok(tw, th)) return fail(RG_ERR_UNSUPPORTED, "tile shapes built: 16x16, 32x8, 8x32");
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
    L.tiles_x = (c->width + tw - 1) / tw;
    L.tiles_y = (c->height + th - 1) / th;
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
    d.tw = tw;
    d.th = th;
    d.tw_log2 = tw == 32 ? 5 : (tw == 16 ? 4 : 3);
    d.th_log2 = th == 32 ? 5 : (th == 16 ? 4 : 3);
    return RG_OK;
}

// one device word set from the stream (test hook of RG_FLAG_TEST_STALL_SORT)
__global__ void k_set_word(unsigned* p, unsigned v) { *p = v; }

// the row-bucketed front end's buffer for n slots: rows per slot (4 B, padded to 16 B), the
// row tests (3 x 16 B per slot), the per-block counts of up to 256 tile rows, the row totals
size_t row_buffer_bytes(int64_t n)
{
    const size_t nb = (size_t)((n + frontend_block_threads() - 1) / frontend_block_threads());
    return ((size_t)n * 4 + 15) / 16 * 16 + (size_t)n * 48 + (size_t)256 * nb * 4 + 256 * 8;
}

// points the row-bucketed front end's arrays of a into w.rowbuf (n = a.n slots)
void row_buffer_views(Workspace& w, FrontendArgs& a)
{
    const size_t n = (size_t)a.n;
    unsigned char* p = w.rowbuf.as<unsigned char>();
    a.row_n = reinterpret_cast<unsigned*>(p);
    p += (n * 4 + 15) / 16 * 16;
    a.row_rt = reinterpret_cast<float4*>(p);
    p += n * 48;
    const size_t nb = (n + frontend_block_threads() - 1) / frontend_block_threads();
    a.row_cnt = reinterpret_cast<unsigned*>(p);
    p += (size_t)256 * nb * 4;
    a.row_tot = reinterpret_cast<unsigned long long*>(p);
}

rg_status ensure_workspace(Workspace& w, int64_t n_gauss, int mode, int tiles, int64_t cap)
{
    const int64_t n = n_gauss > 0 ? n_gauss : 1;
    if (cap > MAX_CAP) return fail(RG_ERR_CAPACITY, "entry capacity above 2^30 - 1");
    if (cap > w.cap || !w.keys[0].p) {
        for (int k = 0; k < 2; k++) {
            RG_TRY(ensure(w.keys[k], (size_t)cap * 8, "keys"));
            RG_TRY(ensure(w.vals[k], (size_t)cap * 4, "values"));
        }
        const int64_t max_tiles = (cap + sort_tile_items() - 1) / sort_tile_items();
        for (int k = 0; k < 2; k++) RG_TRY(ensure(w.sort_status[k], (size_t)max_tiles * 256 * 4, "sort status"));
        w.cap = cap;
    }
    RG_TRY(ensure(w.ranges, (size_t)tiles * sizeof(uint2), "ranges"));
    RG_TRY(ensure(w.ctrl, CTRL_ALLOC, "counters"));
    const int64_t fe_blocks = (n + frontend_block_threads() - 1) / frontend_block_threads();
    RG_TRY(ensure(w.lb_status, (size_t)(std::max<int64_t>(fe_blocks, (n + 2047) / 2048) + 1) * 8, "look-back status"));
    if (mode == RG_MODE_EXACT) {
        RG_TRY(ensure(w.mean2, (size_t)n * 16, "projected means"));
        RG_TRY(ensure(w.depth, (size_t)n * 4, "depth"));
        RG_TRY(ensure(w.quad, (size_t)n * 16, "exponent coefficients"));
        RG_TRY(ensure(w.rgb, (size_t)n * 12, "rgb"));
        RG_TRY(ensure(w.rect, (size_t)n * 16, "rect"));
        RG_TRY(ensure(w.touched, (size_t)n * 4, "touched"));
        RG_TRY(ensure(w.offsets, (size_t)n * 4, "offsets"));
    } else {
        RG_TRY(ensure(w.rec, (size_t)n * 32, "records"));
        // the per-tile counting sort's count matrix (chunks x tiles, at most SMs x one block's shared
        // memory for any tile count) and tile totals: sized for any frame, so a workspace shared by
        // views of several resolutions never runs short
        RG_TRY(ensure(w.tsort, tilesort_matrix_bytes_max() + (size_t)tilesort_max_tiles() * 4, "tile counting sort"));
        RG_TRY(ensure(w.rowbuf, row_buffer_bytes(n), "row buckets"));
        for (int k = 0; k < 2; k++) {
            RG_TRY(ensure(w.gkeys[k], (size_t)n * 4, "depth keys"));
            RG_TRY(ensure(w.gvals[k], (size_t)n * 4, "depth order"));
            RG_TRY(ensure(w.gstatus[k], (size_t)((n + sort_tile_items() - 1) / sort_tile_items()) * 256 * 4,
                          "depth sort status"));
        }
    }
    return RG_OK;
}

void init_events(Workspace& w)
{
    if (w.ev_init) return;
    for (int f = 0; f < EV_RING; f++)
        for (int k = 0; k < EV_PER_FRAME; k++) cudaEventCreate(&w.ev[f][k]);
    w.ev_init = true;
}

// NVTX range around a stage's launches (host side; costs nothing without a tool attached),
// e.g. for `ncu --nvtx --nvtx-include "rg raster/"`
struct NvtxScope {
    explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope&) = delete;
    NvtxScope& operator=(const NvtxScope&) = delete;
};

// How the warps of each sort pass rank their digits (2 bits per pass, SORT_RANK_*): the
// depth order's passes, the tile-bit passes of the RoofGS entries, exact mode's passes.
#ifndef RG_DEPTH_RANK_MODES
#define RG_DEPTH_RANK_MODES sort_rank_modes(SORT_RANK_PEERS, SORT_RANK_PEERS, SORT_RANK_PEERS, SORT_RANK_PEERS)
#endif
#ifndef RG_TILE_RANK_MODES
#define RG_TILE_RANK_MODES sort_rank_modes(SORT_RANK_PEERS, SORT_RANK_PEERS)
#endif
#ifndef RG_EXACT_RANK_MODES
#define RG_EXACT_RANK_MODES sort_rank_modes(SORT_RANK_MATCH, SORT_RANK_MATCH, SORT_RANK_MATCH, SORT_RANK_MATCH) | \
                                (sort_rank_modes(SORT_RANK_PEERS, SORT_RANK_PEERS) << 8)
#endif

// Arguments of a RoofGS frame's front end and sorts on workspace w (nothing launched;
// records what rg_inspect needs about the frame in w).
rg_status roofgs_build(rg_scene* s, Workspace& w, const FrameLayout& F, uint32_t flags, RoofgsFrame& f)
{
    memset(&f, 0, sizeof(f));
    Counters* ctr = w.ctrl.as<Counters>();
    unsigned* hist = reinterpret_cast<unsigned*>(w.ctrl.as<unsigned char>() + sizeof(Counters));
    Sticky* sticky = s->sticky.as<Sticky>();
    const long long n = s->n;
    FrontendArgs& a = f.fa;
    a.geoA = s->geoA.as<float4>();
    a.geoB = s->geoB.as<uint4>();
    a.shq = s->shq.as<uint4>();
    for (int k = 0; k < 12; k++) a.band_scale[k] = (k / 3 <= s->sh_degree) ? s->band_scale[k] : 0.0f;
    a.per_gauss_scale = s->sh_scale_mode == RG_SH_SCALE_BAND_GAUSS;
    a.sh_degree = s->sh_degree;
    a.n = n;
    a.cam = F.cam;
    a.lay = F.lay;
    a.rec = w.rec.as<float4>();
    a.keys = w.keys[0].as<unsigned>();
    a.vals = w.vals[0].as<unsigned>();
    a.cap = w.cap;
    a.status = w.lb_status.as<unsigned long long>();
    a.ctr = ctr;
    a.sticky = sticky;
    SortArgs& sa = f.sa;
    for (int k = 0; k < 2; k++) {
        sa.keys[k] = w.keys[k].p;
        sa.vals[k] = w.vals[k].as<unsigned>();
        sa.status[k] = w.sort_status[k].as<unsigned>();
    }
    sa.cap = w.cap;
    sa.hist = hist;
    sa.max_tiles = (w.cap + sort_tile_items() - 1) / sort_tile_items();
    sa.ctr = ctr;
    sa.sticky = sticky;
    sa.key_bytes = 4;
    if (flags & RG_FLAG_SORT_FULL_KEY) {
        // the paper's scheme: entries in Gaussian order, 4 passes over the 32-bit key
        sa.passes = 4;
        sa.bit0 = 0;
    } else {
        // Gaussians sorted by quantized depth first (stable, ties by index); the
        // entries then come out in (q_d, index) order and a stable sort of the
        // b_t tile bits alone yields the order of the full 32-bit key
        f.depth_order = true;
        SortArgs& ga = f.ga;
        for (int k = 0; k < 2; k++) {
            ga.keys[k] = w.gkeys[k].p;
            ga.vals[k] = w.gvals[k].as<unsigned>();
            ga.status[k] = w.gstatus[k].as<unsigned>();
        }
        ga.cap = n;
        ga.key_bytes = 4;
        ga.passes = (F.lay.b_d + 7) / 8;
        ga.bit0 = 0;
        // Gaussians in index order carry scattered depth digits: every pass ranks with the
        // per-digit peer masks (measured 0.126 -> 0.124 ms at 4K, 0.086 -> 0.081 ms at 1080p
        // against ballots on the first pass and match_any on the others)
        ga.rank_modes = RG_DEPTH_RANK_MODES;
        ga.hist = reinterpret_cast<unsigned*>(w.ctrl.as<unsigned char>() + CTRL_BYTES + sizeof(Counters));
        ga.max_tiles = (n + sort_tile_items() - 1) / sort_tile_items();
        ga.ctr = reinterpret_cast<Counters*>(w.ctrl.as<unsigned char>() + CTRL_BYTES);
        ga.sticky = sticky;
        // the depth keys' digits are counted as they are written (ga.passes <= 4), and the
        // depth-key kernel clears the first pass's look-back status: no histogram kernel
        ga.hist_pre = ga.hist;
        ga.hist_done = 1;
        a.order = w.gvals[ga.passes & 1].as<unsigned>();
        sa.passes = (F.lay.b_t + 7) / 8;
        sa.bit0 = F.lay.b_d;
        // depth-ordered entries of one Gaussian row carry consecutive tiles, so the warp
        // holds many distinct low tile digits, and after that pass the high digits of
        // neighbouring entries are scattered too: both passes rank with the peer masks (4K
        // tile-bit passes 0.832 -> 0.778 ms against ballots on pass 0; with two ranking chains
        // per warp 0.682 -> 0.656 ms against match_any on pass 1)
        sa.rank_modes = RG_TILE_RANK_MODES;
        // up to 2 tile-bit passes (b_t <= 16): the front end counts the digits of its
        // entries per tile row, and the sort's histogram pass only runs on overflow;
        // the entries carry the 16-bit tile id alone (the depth code of a 32-bit key
        // follows from the value: entries stay in depth order within a tile)
        if (sa.passes <= 2) {
            a.hist = reinterpret_cast<unsigned*>(w.ctrl.as<unsigned char>() + 2 * CTRL_BYTES);
            a.hist_passes = sa.passes;
            sa.hist_copies = a.hist;
            sa.hist_copy_stride = 2;
            sa.hist_pre = hist + 4 * 256; // rows 4-5 of the frame's [8][256] histograms
            a.keys16 = w.keys[0].as<unsigned short>();
            sa.key_bytes = 2;
            sa.bit0 = 0;
        }
        w.last_gfin = ga.passes & 1;
    }
    if (flags & RG_FLAG_TILE_COUNTING_SORT) {
        // one stable counting sort by tile instead of the tile-bit radix passes: the front end
        // needs no digit counts; the values land in vals[1], the ranges come with them
        if (!f.depth_order || !a.keys16 || F.tiles > tilesort_max_tiles())
            return fail(RG_ERR_UNSUPPORTED, "RG_FLAG_TILE_COUNTING_SORT needs the depth pre-sort, 16-bit tile ids "
                                            "and at most 57,856 tiles");
        f.tile_sort = true;
        a.hist = nullptr;
        a.hist_passes = 0;
        TileSortArgs& t = f.ts;
        t.keys16 = w.keys[0].as<unsigned short>();
        t.vals = w.vals[0].as<unsigned>();
        t.vout = w.vals[1].as<unsigned>();
        t.T = F.tiles;
        t.chunks = tilesort_chunks(F.tiles);
        t.M = w.tsort.as<unsigned>();
        t.tot = t.M + (size_t)t.chunks * F.tiles;
        t.ranges = w.ranges.as<uint2>();
        t.ctr = ctr;
        sa.passes = 1; // the result's buffer: vals[1]
    }
    f.tile_shift = a.keys16 ? 0 : F.lay.b_d;
    w.last_key16 = a.keys16 != nullptr;
    w.last_cols = false;
    w.last_tilesort = f.tile_sort;
    w.last_bd = F.lay.b_d;
    w.last_mode = RG_MODE_ROOFGS;
    w.last_passes = sa.passes;
    w.last_tiles = F.tiles;
    return RG_OK;
}

// The per-Gaussian depth order of a RoofGS frame: quantized depth keys (with the sort's
// digit counts), then their stable sort.
void roofgs_depth_order(const RoofgsFrame& f, Workspace& w, cudaStream_t st)
{
    launch_depth_keys(f.fa, w.gkeys[0].as<unsigned>(), w.gvals[0].as<unsigned>(), f.ga.ctr, f.ga.hist, f.ga.passes,
                      f.ga.status[0], st);
    launch_sort(f.ga, st, nullptr);
}

// The RoofGS rasterizer's arguments for a frame built by roofgs_build (non-counting).
void roofgs_raster_args(rg_scene* s, Workspace& w, const FrameLayout& F, uint32_t flags, float* out, RasterArgs& r)
{
    memset(&r, 0, sizeof(r));
    const int fin = w.last_passes & 1;
    r.ranges = w.ranges.as<uint2>();
    r.vals = w.vals[fin].as<unsigned>();
    r.n = s->n;
    r.tiles_x = F.lay.tiles_x;
    r.tiles_y = F.lay.tiles_y;
    r.cam = F.cam;
    r.out = out;
    r.rec = w.rec.as<float4>();
    if (w.last_tilesort) { // the counting sort wrote the ranges: no search
    } else if (w.last_key16) {
        r.skeys16 = w.keys[fin].as<unsigned short>();
    } else {
        r.skeys = w.keys[fin].as<unsigned>();
    }
    r.key_cols = w.last_key16 && w.last_cols;
    r.tile_shift = w.last_key16 ? 0 : F.lay.b_d;
    r.ranges_out = w.ranges.as<uint2>();
    r.ctr = w.ctrl.as<Counters>();
    r.fast_exp = (flags & RG_FLAG_EXACT_EXP) ? 0 : 1;
    r.ppt = (flags & RG_FLAG_SINGLE_PIXEL) ? 1 : ((flags & RG_FLAG_QUAD_PIXEL) ? 4 : 2);
}

// One frame on `st`; the caller has checked arguments and the workspace.
rg_status render_once(rg_scene* s, Workspace& w, const FrameLayout& F, int mode, uint32_t flags, float* out,
                      cudaStream_t st, bool count)
{
    Counters* ctr = w.ctrl.as<Counters>();
    unsigned* hist = reinterpret_cast<unsigned*>(w.ctrl.as<unsigned char>() + sizeof(Counters));
    Sticky* sticky = s->sticky.as<Sticky>();
    const bool ev = (flags & RG_FLAG_STAGE_EVENTS) != 0;
    cudaEvent_t* E = nullptr;
    if (ev) {
        init_events(w);
        E = w.ev[w.ev_next];
        w.ev_next = (w.ev_next + 1) % EV_RING;
        if (w.ev_pending < EV_RING) w.ev_pending++;
        RG_CK(cudaEventRecord(E[0], st));
    }
    // RoofGS frames that rasterize find each tile's range inside the rasterizer (a search of
    // the sorted keys per tile block); the others run the ranges pass
    const bool tile_sort = mode == RG_MODE_ROOFGS && (flags & RG_FLAG_TILE_COUNTING_SORT);
    const bool search_ranges = mode == RG_MODE_ROOFGS && out != nullptr && !tile_sort;
    w.last_key16 = false;
    w.last_tilesort = false;
    w.last_cols = false;
    RG_CK(cudaMemsetAsync(w.ctrl.p, 0, CTRL_ALLOC, st));
    if (flags & RG_FLAG_TEST_STALL_SORT) { // tile 0 of the first entry-sort pass is never claimed
        k_set_word<<<1, 1, 0, st>>>(&ctr->sort_tile_ctr[0], 1u);
        RG_CK(cudaGetLastError());
    }
    if (!search_ranges) RG_CK(cudaMemsetAsync(w.ranges.p, 0, (size_t)F.tiles * sizeof(uint2), st));
    const long long n = s->n;
    SortArgs sa;
    memset(&sa, 0, sizeof(sa));
    for (int k = 0; k < 2; k++) {
        sa.keys[k] = w.keys[k].p;
        sa.vals[k] = w.vals[k].as<unsigned>();
        sa.status[k] = w.sort_status[k].as<unsigned>();
    }
    sa.cap = w.cap;
    sa.hist = hist;
    sa.max_tiles = (w.cap + sort_tile_items() - 1) / sort_tile_items();
    sa.ctr = ctr;
    sa.sticky = sticky;
    int tile_shift;
    TileSortArgs tsa;
    memset(&tsa, 0, sizeof(tsa));
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
        a.mean2 = w.mean2.as<float4>();
        a.depth = w.depth.as<float>();
        a.quad = w.quad.as<float4>();
        a.rgb = w.rgb.as<float>();
        a.rect = w.rect.as<int4>();
        a.touched = w.touched.as<unsigned>();
        a.offsets = w.offsets.as<unsigned>();
        a.keys = w.keys[0].as<unsigned long long>();
        a.vals = w.vals[0].as<unsigned>();
        a.cap = w.cap;
        a.status = w.lb_status.as<unsigned long long>();
        a.ctr = ctr;
        a.sticky = sticky;
        RG_CK(cudaMemsetAsync(w.lb_status.p, 0, (size_t)((n + 2047) / 2048 + 1) * 8, st));
        sa.key_bytes = 8;
        sa.passes = (32 + F.lay.b_t + 7) / 8; // only the bits that can be non-zero
        // passes 0-3 (depth bits: the entries of one Gaussian share them) rank with match_any,
        // the tile-bit passes 4-5 (consecutive tiles) with the peer masks: 4K sort 10.66 ->
        // 10.09 ms (every pass with the peer masks: 11.43 ms)
        sa.rank_modes = RG_EXACT_RANK_MODES;
        tile_shift = 32;
        if (sa.passes <= 6) { // up to 2 tile-bit passes: the duplicate kernel counts every digit
            a.hist = reinterpret_cast<unsigned*>(w.ctrl.as<unsigned char>() + 2 * CTRL_BYTES);
            a.tile_passes = sa.passes - 4;
            sa.hist_copies = a.hist;
            sa.hist_copy_stride = 8;
            sa.hist_pre = hist + 2 * 256; // rows 2-7 of the frame's [8][256] histograms
        }
        if (ev) RG_CK(cudaEventRecord(E[1], st));
        {
            NvtxScope r_("rg front end");
            launch_exact_preprocess(a, st);
            launch_exact_scan(a, st);
            launch_exact_duplicate(a, st);
        }
    } else {
        RoofgsFrame f;
        RG_TRY(roofgs_build(s, w, F, flags, f));
        // the row-bucketed front end: column-major 16-bit keys grouped by tile row, one 8-bit
        // pass over the column left to the sort (the rasterizer finds the ranges)
        const bool rows = !(flags & RG_FLAG_ORDERED_FRONT_END) && search_ranges && f.depth_order && f.fa.keys16 &&
                          !f.tile_sort && F.lay.tiles_x <= 256 && F.lay.tiles_y <= 256 && n > 0;
        if (rows) {
            f.fa.rows = F.lay.tiles_y;
            row_buffer_views(w, f.fa);
            f.fa.hist_passes = 1; // the column digits
            f.sa.passes = 1;
            f.sa.bit0 = 8;
            f.sa.rank_modes = sort_rank_modes(SORT_RANK_PEERS);
            w.last_cols = true;
        } else {
            RG_CK(cudaMemsetAsync(w.lb_status.p, 0,
                                  (size_t)((n + frontend_block_threads() - 1) / frontend_block_threads() + 1) * 8, st));
        }
        if (f.depth_order) {
            NvtxScope r_("rg depth order");
            roofgs_depth_order(f, w, st);
        }
        if (ev) RG_CK(cudaEventRecord(E[1], st));
        {
            NvtxScope r_("rg front end");
            if (rows) launch_frontend_rows(f.fa, st);
            else launch_frontend_fused(f.fa, st);
        }
        sa = f.sa;
        tile_shift = f.tile_shift;
        tsa = f.ts;
    }
    if (ev) RG_CK(cudaEventRecord(E[2], st));
    if (ev && (sa.passes <= 0 || tile_sort)) RG_CK(cudaEventRecord(E[3], st));
    if (tile_sort) {
        NvtxScope r_("rg sort");
        launch_tile_counting_sort(tsa, st);
    } else {
        NvtxScope r_("rg sort");
        launch_sort(sa, st, ev ? E[3] : nullptr);
    }
    if (ev) RG_CK(cudaEventRecord(E[4], st));
    const int fin = sa.passes & 1;
    if (!search_ranges && !tile_sort) {
        RangeArgs ra;
        ra.keys = w.keys[fin].p;
        ra.key_bytes = sa.key_bytes;
        ra.tile_shift = tile_shift;
        ra.ntiles = F.tiles;
        ra.ranges = w.ranges.as<uint2>();
        ra.ctr = ctr;
        NvtxScope r_("rg ranges");
        launch_ranges(ra, st);
    }
    if (ev) RG_CK(cudaEventRecord(E[5], st));
    w.last_mode = mode;
    w.last_passes = sa.passes;
    w.last_tiles = F.tiles;
    w.last_tilesort = tile_sort;
    if (!out) { // front end, sort and ranges only (the backward replays the blend itself)
        if (ev) RG_CK(cudaEventRecord(E[6], st));
        RG_CK(cudaGetLastError());
        return RG_OK;
    }
    RasterArgs r;
    memset(&r, 0, sizeof(r));
    r.ranges = w.ranges.as<uint2>();
    r.vals = w.vals[fin].as<unsigned>();
    r.n = n;
    r.tiles_x = F.lay.tiles_x;
    r.tiles_y = F.lay.tiles_y;
    r.cam = F.cam;
    r.out = out;
    r.count = count ? ctr : nullptr;
    if (mode == RG_MODE_EXACT) {
        r.mean2 = w.mean2.as<float4>();
        r.quad = w.quad.as<float4>();
        r.rgb = w.rgb.as<float>();
        NvtxScope r_("rg raster");
        launch_raster_exact(r, st);
    } else {
        roofgs_raster_args(s, w, F, flags, out, r);
        r.count = count ? ctr : nullptr;
        NvtxScope r_("rg raster");
        launch_raster_roofgs(r, st);
    }
    if (ev) RG_CK(cudaEventRecord(E[6], st));
    RG_CK(cudaGetLastError());
    w.last_mode = mode;
    w.last_passes = sa.passes;
    w.last_tiles = F.tiles;
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
    DevBuf* bufs[] = {&s->means, &s->scales, &s->quats, &s->opac, &s->sh, &s->geoA, &s->geoB, &s->shq, &s->sticky};
    for (DevBuf* b : bufs) b->release();
    s->ws.release();
    delete s;
}


} // namespace rg

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
    drop_plans_of(scene);
    destroy_scene(scene);
    return RG_OK;
}

rg_status rg_scene_reserve(rg_scene* scene, int64_t n_entries)
{
    if (!scene || n_entries < 0) return fail(RG_ERR_INVALID_ARG, "bad scene or size");
    if (n_entries <= scene->ws.cap) return RG_OK;
    RG_CK(cudaDeviceSynchronize());
    const int64_t cap = n_entries;
    for (int k = 0; k < 2; k++) {
        RG_TRY(ensure(scene->ws.keys[k], (size_t)cap * 8, "keys"));
        RG_TRY(ensure(scene->ws.vals[k], (size_t)cap * 4, "values"));
    }
    const int64_t max_tiles = (cap + sort_tile_items() - 1) / sort_tile_items();
    for (int k = 0; k < 2; k++) RG_TRY(ensure(scene->ws.sort_status[k], (size_t)max_tiles * 256 * 4, "sort status"));
    scene->ws.cap = cap;
    return RG_OK;
}

// ---------------------------------------------------------------------------
// Scene files: a fixed header, then the stored buffers in a fixed order (FP32 means,
// scales, quats, opacities, SH if RG_STORE_FP32; compact geoA, geoB, SH codes if
// RG_STORE_COMPACT), raw little-endian, so a load needs no re-encoding.
// ---------------------------------------------------------------------------
namespace {

struct SceneFileHeader {
    char magic[8];
    uint32_t version;
    uint32_t storage;
    int64_t n;
    int32_t sh_degree;
    int32_t sh_scale_mode;
    float band_scale[12];
    uint64_t reserved[4];
};
constexpr char SCENE_MAGIC[8] = {'R', 'G', 'S', 'C', 'E', 'N', 'E', '1'};
constexpr uint32_t SCENE_VERSION = 1;

// (buffer, bytes) of a scene in file order
std::vector<std::pair<DevBuf*, size_t>> scene_buffers(rg_scene* s)
{
    std::vector<std::pair<DevBuf*, size_t>> v;
    const size_t n = (size_t)s->n;
    if (s->storage & RG_STORE_FP32) {
        v.push_back({&s->means, n * 12});
        v.push_back({&s->scales, n * 12});
        v.push_back({&s->quats, n * 16});
        v.push_back({&s->opac, n * 4});
        v.push_back({&s->sh, n * 192});
    }
    if (s->storage & RG_STORE_COMPACT) {
        v.push_back({&s->geoA, n * 16});
        v.push_back({&s->geoB, n * 16});
        v.push_back({&s->shq, n * 48});
    }
    return v;
}

constexpr size_t IO_CHUNK = 64u << 20;

} // namespace

rg_status rg_scene_save(rg_scene* s, const char* path)
{
    if (!s || !path) return fail(RG_ERR_INVALID_ARG, "NULL argument");
    RG_CK(cudaDeviceSynchronize());
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(RG_ERR_INVALID_ARG, std::string("cannot open for writing: ") + path);
    SceneFileHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, SCENE_MAGIC, 8);
    h.version = SCENE_VERSION;
    h.storage = s->storage;
    h.n = s->n;
    h.sh_degree = s->sh_degree;
    h.sh_scale_mode = s->sh_scale_mode;
    memcpy(h.band_scale, s->band_scale, sizeof(h.band_scale));
    bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1;
    std::vector<unsigned char> buf;
    for (auto& b : scene_buffers(s)) {
        for (size_t off = 0; ok && off < b.second; off += IO_CHUNK) {
            const size_t len = std::min(IO_CHUNK, b.second - off);
            buf.resize(len);
            if (cudaMemcpy(buf.data(), b.first->as<unsigned char>() + off, len, cudaMemcpyDeviceToHost) != cudaSuccess) {
                std::fclose(f);
                return fail(RG_ERR_CUDA, "copy of scene buffer to host failed");
            }
            ok = std::fwrite(buf.data(), 1, len, f) == len;
        }
    }
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(RG_ERR_INVALID_ARG, std::string("write failed: ") + path);
    return RG_OK;
}

rg_status rg_scene_load(const char* path, void* stream, rg_scene** out)
{
    if (!out) return fail(RG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!path) return fail(RG_ERR_INVALID_ARG, "path is NULL");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(RG_ERR_INVALID_ARG, std::string("cannot open: ") + path);
    SceneFileHeader h;
    auto bad = [&](const char* why) {
        std::fclose(f);
        return fail(RG_ERR_INVALID_ARG, std::string("not a valid scene file (") + why + "): " + path);
    };
    if (std::fread(&h, sizeof(h), 1, f) != 1) return bad("short header");
    if (memcmp(h.magic, SCENE_MAGIC, 8) != 0) return bad("magic");
    if (h.version != SCENE_VERSION) return bad("version");
    if (h.n < 0 || h.n > (1ll << 31)) return bad("n");
    if (h.sh_degree < 0 || h.sh_degree > 3) return bad("sh_degree");
    if (h.sh_scale_mode != RG_SH_SCALE_BAND && h.sh_scale_mode != RG_SH_SCALE_BAND_GAUSS) return bad("sh_scale_mode");
    if (h.storage == 0 || (h.storage & ~(RG_STORE_FP32 | RG_STORE_COMPACT))) return bad("storage");
    for (int k = 0; k < 12; k++)
        if (!std::isfinite(h.band_scale[k])) return bad("band scales");
    {
        const size_t n = (size_t)h.n;
        size_t want = sizeof(h);
        if (h.storage & RG_STORE_FP32) want += n * (12 + 12 + 16 + 4 + 192);
        if (h.storage & RG_STORE_COMPACT) want += n * (16 + 16 + 48);
        if (std::fseek(f, 0, SEEK_END) != 0 || (size_t)std::ftell(f) != want) return bad("size");
        std::fseek(f, (long)sizeof(h), SEEK_SET);
    }
    rg_scene* s = new rg_scene();
    cudaGetDevice(&s->device);
    s->n = h.n;
    s->sh_degree = h.sh_degree;
    s->storage = h.storage;
    s->sh_scale_mode = h.sh_scale_mode;
    memcpy(s->band_scale, h.band_scale, sizeof(h.band_scale));
    auto bufs = scene_buffers(s);
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<unsigned char> buf;
    rg_status e = ensure(s->sticky, sizeof(Sticky), "sticky");
    if (e == RG_OK && cudaMemsetAsync(s->sticky.p, 0, sizeof(Sticky), st) != cudaSuccess) e = fail(RG_ERR_CUDA, "memset");
    for (auto& b : bufs) {
        if (e != RG_OK) break;
        e = ensure(*b.first, b.second ? b.second : 16, "scene buffer");
        for (size_t off = 0; e == RG_OK && off < b.second; off += IO_CHUNK) {
            const size_t len = std::min(IO_CHUNK, b.second - off);
            buf.resize(len);
            if (std::fread(buf.data(), 1, len, f) != len) {
                e = fail(RG_ERR_INVALID_ARG, std::string("short read: ") + path);
                break;
            }
            if (cudaMemcpyAsync(b.first->as<unsigned char>() + off, buf.data(), len, cudaMemcpyHostToDevice, st) !=
                    cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                e = fail(RG_ERR_CUDA, "copy of scene buffer to the device failed");
        }
    }
    std::fclose(f);
    if (e != RG_OK) {
        cudaStreamSynchronize(st);
        destroy_scene(s);
        return e;
    }
    *out = s;
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
    int tw, th;
    RG_TRY(tile_shape(opts, tw, th));
    if (mode == RG_MODE_EXACT && !(s->storage & RG_STORE_FP32))
        return fail(RG_ERR_INVALID_ARG, "exact mode needs RG_STORE_FP32");
    if (mode == RG_MODE_ROOFGS && !(s->storage & RG_STORE_COMPACT))
        return fail(RG_ERR_INVALID_ARG, "RoofGS mode needs RG_STORE_COMPACT");
    FrameLayout F;
    RG_TRY(make_layout(cam, F, tw, th));
    cudaStream_t st = (cudaStream_t)stream;
    int64_t cap = s->ws.cap > 0 ? s->ws.cap : std::max<int64_t>(1 << 20, 4 * s->n);
    if (cap > MAX_CAP) cap = MAX_CAP;
    RG_TRY(ensure_workspace(s->ws, s->n, mode, F.tiles, cap));
    RG_TRY(render_once(s, s->ws, F, mode, opts->flags, out_chw, st, stats != nullptr));
    if (!stats) return RG_OK;
    Counters c;
    RG_CK(cudaMemcpyAsync(&c, s->ws.ctrl.p, sizeof(c), cudaMemcpyDeviceToHost, st));
    RG_CK(cudaStreamSynchronize(st));
    int regrown = 0;
    if (c.error) return fail(RG_ERR_TIMEOUT, "a bounded device wait gave up");
    if (c.n_entries_total > (unsigned long long)s->ws.cap) {
        int64_t want = (int64_t)(c.n_entries_total + c.n_entries_total / 4 + 1024);
        if ((unsigned long long)want > (unsigned long long)MAX_CAP) want = MAX_CAP;
        if ((unsigned long long)want < c.n_entries_total)
            return fail(RG_ERR_CAPACITY, "frame needs more than 2^30 - 1 entries");
        RG_TRY(rg_scene_reserve(s, want));
        RG_TRY(render_once(s, s->ws, F, mode, opts->flags, out_chw, st, true));
        RG_CK(cudaMemcpyAsync(&c, s->ws.ctrl.p, sizeof(c), cudaMemcpyDeviceToHost, st));
        RG_CK(cudaStreamSynchronize(st));
        if (c.error) return fail(RG_ERR_TIMEOUT, "a bounded device wait gave up");
        if (c.n_entries_total > (unsigned long long)s->ws.cap) return fail(RG_ERR_CAPACITY, "workspace could not grow enough");
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
    stats->capacity = s->ws.cap;
    stats->regrown = regrown;
    stats->sort_passes = s->ws.last_passes;
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
    const int cnt = s->ws.ev_pending;
    if (frames) *frames = cnt;
    if (!s->ws.ev_init || cnt == 0) return RG_OK;
    for (int f = 0; f < cnt; f++) {
        const int slot = ((s->ws.ev_next - 1 - f) % EV_RING + EV_RING) % EV_RING;
        cudaEvent_t* E = s->ws.ev[slot];
        RG_CK(cudaEventSynchronize(E[6]));
        float t;
        for (int k = 0; k < 6; k++) {
            RG_CK(cudaEventElapsedTime(&t, E[k], E[k + 1]));
            ms7[k] += t;
        }
        RG_CK(cudaEventElapsedTime(&t, E[0], E[6]));
        ms7[6] += t;
    }
    s->ws.ev_pending = 0;
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
        if (s->ws.last_mode < 0) return fail(RG_ERR_INVALID_ARG, "no frame rendered yet");
        Counters c;
        RG_CK(cudaMemcpy(&c, s->ws.ctrl.p, sizeof(c), cudaMemcpyDeviceToHost));
        const int fin = s->ws.last_passes & 1;
        // column-major keys: the entries are regrouped tile by tile in tile-id order (each tile's
        // range, in its order), which is the order of the entries sorted by tile id
        std::vector<uint32_t> cval;
        std::vector<uint2> cr;
        if (s->ws.last_key16 && s->ws.last_cols) {
            const size_t ne = c.n_entries;
            std::vector<uint32_t> v(ne);
            cr.resize((size_t)s->ws.last_tiles);
            RG_CK(cudaMemcpy(cr.data(), s->ws.ranges.p, cr.size() * 8, cudaMemcpyDeviceToHost));
            if (ne) RG_CK(cudaMemcpy(v.data(), s->ws.vals[fin].p, ne * 4, cudaMemcpyDeviceToHost));
            cval.reserve(ne);
            uint32_t at = 0;
            for (size_t t = 0; t < cr.size(); t++) {
                const uint32_t b = cr[t].x, e = std::min<uint32_t>(cr[t].y, (uint32_t)ne);
                const uint32_t len = e > b ? e - b : 0u;
                for (uint32_t j = b; j < b + len; j++) cval.push_back(v[j]);
                cr[t] = len ? make_uint2(at, at + len) : make_uint2(0u, 0u);
                at += len;
            }
        }
        if (what == RG_INSPECT_KEYS && s->ws.last_key16) {
            // the entries carried 16-bit tile ids: each 32-bit key (tile << b_d | q_d) is rebuilt
            // from the tile and the depth code of its Gaussian (the per-Gaussian depth sort's result);
            // after the per-tile counting sort the tile of each slot follows from the ranges
            const size_t ne = c.n_entries, ng = (size_t)n;
            std::vector<uint16_t> t16(ne);
            std::vector<uint32_t> val(ne), gq(ng), gi(ng), q(ng, 0u);
            if (ne) {
                if (s->ws.last_cols) {
                    for (size_t t = 0; t < cr.size(); t++)
                        for (uint32_t j = cr[t].x; j < cr[t].y; j++) t16[j] = (uint16_t)t;
                    for (size_t j = 0; j < ne; j++) val[j] = j < cval.size() ? cval[j] : 0u;
                } else if (s->ws.last_tilesort) {
                    std::vector<uint2> rr((size_t)s->ws.last_tiles);
                    RG_CK(cudaMemcpy(rr.data(), s->ws.ranges.p, rr.size() * 8, cudaMemcpyDeviceToHost));
                    for (size_t t = 0; t < rr.size(); t++)
                        for (uint32_t j = rr[t].x; j < rr[t].y && j < ne; j++) t16[j] = (uint16_t)t;
                } else {
                    RG_CK(cudaMemcpy(t16.data(), s->ws.keys[fin].p, ne * 2, cudaMemcpyDeviceToHost));
                }
                if (!s->ws.last_cols) RG_CK(cudaMemcpy(val.data(), s->ws.vals[fin].p, ne * 4, cudaMemcpyDeviceToHost));
            }
            if (ng) {
                RG_CK(cudaMemcpy(gq.data(), s->ws.gkeys[s->ws.last_gfin].p, ng * 4, cudaMemcpyDeviceToHost));
                RG_CK(cudaMemcpy(gi.data(), s->ws.gvals[s->ws.last_gfin].p, ng * 4, cudaMemcpyDeviceToHost));
            }
            for (size_t k = 0; k < ng; k++)
                if (gi[k] < ng) q[gi[k]] = gq[k];
            const int bd = s->ws.last_bd;
            tmp.resize(ne * 4);
            for (size_t j = 0; j < ne; j++) {
                const uint32_t qd = val[j] < ng ? q[val[j]] : 0u;
                const uint32_t key = bd >= 32 ? qd : (((uint32_t)t16[j] << bd) | qd);
                memcpy(&tmp[j * 4], &key, 4);
            }
            src = tmp.data();
            device_src = false;
            bytes = (int64_t)ne * 4;
        } else if (what == RG_INSPECT_KEYS) {
            src = s->ws.keys[fin].p;
            bytes = (int64_t)c.n_entries * (s->ws.last_mode == RG_MODE_EXACT ? 8 : 4);
        } else if (what == RG_INSPECT_VALUES && s->ws.last_key16 && s->ws.last_cols) {
            cval.resize(c.n_entries, 0u);
            tmp.resize(cval.size() * 4);
            if (!cval.empty()) memcpy(tmp.data(), cval.data(), tmp.size());
            src = tmp.data();
            device_src = false;
            bytes = (int64_t)tmp.size();
        } else if (what == RG_INSPECT_VALUES) {
            src = s->ws.vals[fin].p;
            bytes = (int64_t)c.n_entries * 4;
        } else if (s->ws.last_key16 && s->ws.last_cols) {
            tmp.resize(cr.size() * 8);
            if (!cr.empty()) memcpy(tmp.data(), cr.data(), tmp.size());
            src = tmp.data();
            device_src = false;
            bytes = (int64_t)tmp.size();
        } else {
            src = s->ws.ranges.p;
            bytes = (int64_t)s->ws.last_tiles * 8;
        }
        break;
    }
    case RG_INSPECT_SH_CODES:
    case RG_INSPECT_GAUSS_SCALE:
    case RG_INSPECT_GEOM16:
    case RG_INSPECT_LOG_OPACITY: {
        if (!(s->storage & RG_STORE_COMPACT)) return fail(RG_ERR_INVALID_ARG, "scene has no compact attributes");
        if (what == RG_INSPECT_SH_CODES) {
            tmp.resize((size_t)n * 48);
            if (n) RG_CK(cudaMemcpy(tmp.data(), s->shq.p, (size_t)n * 48, cudaMemcpyDeviceToHost));
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

rg_status rg_backward(rg_scene* s, const rg_camera* cam, const rg_render_opts* opts, const float* dL_dimg,
                      const rg_grads* grads, void* stream)
{
    if (!s || !opts || !dL_dimg || !grads) return fail(RG_ERR_INVALID_ARG, "NULL argument");
    if (opts->mode != RG_MODE_EXACT)
        return fail(RG_ERR_UNSUPPORTED, "rg_backward differentiates exact mode only (RoofGS storage is INT8/FP16)");
    if (!(s->storage & RG_STORE_FP32)) return fail(RG_ERR_INVALID_ARG, "rg_backward needs RG_STORE_FP32");
    int tw, th;
    RG_TRY(tile_shape(opts, tw, th));
    if (s->n > 0 && (!grads->means || !grads->scales || !grads->quats || !grads->opacities || !grads->sh))
        return fail(RG_ERR_INVALID_ARG, "a gradient pointer is NULL");
    FrameLayout F;
    RG_TRY(make_layout(cam, F, tw, th));
    cudaStream_t st = (cudaStream_t)stream;
    int64_t cap = s->ws.cap > 0 ? s->ws.cap : std::max<int64_t>(1 << 20, 4 * s->n);
    if (cap > MAX_CAP) cap = MAX_CAP;
    RG_TRY(ensure_workspace(s->ws, s->n, RG_MODE_EXACT, F.tiles, cap));
    // forward front end, sort and ranges of this camera (checked: the gradient needs every entry)
    for (int attempt = 0; attempt < 2; attempt++) {
        RG_TRY(render_once(s, s->ws, F, RG_MODE_EXACT, 0u, nullptr, st));
        Counters c;
        RG_CK(cudaMemcpyAsync(&c, s->ws.ctrl.p, sizeof(c), cudaMemcpyDeviceToHost, st));
        RG_CK(cudaStreamSynchronize(st));
        if (c.error) return fail(RG_ERR_TIMEOUT, "a bounded device wait gave up");
        if (c.n_entries_total <= (unsigned long long)s->ws.cap) break;
        if (attempt == 1) return fail(RG_ERR_CAPACITY, "workspace could not grow enough");
        int64_t want = (int64_t)(c.n_entries_total + c.n_entries_total / 4 + 1024);
        if (want > MAX_CAP) return fail(RG_ERR_CAPACITY, "frame needs more than 2^30 - 1 entries");
        RG_TRY(rg_scene_reserve(s, want));
    }
    RG_TRY(ensure(s->ws.gbuf, (size_t)(s->n > 0 ? s->n : 1) * 9 * 4, "gradient buffer"));
    RG_CK(cudaMemsetAsync(s->ws.gbuf.p, 0, (size_t)(s->n > 0 ? s->n : 1) * 9 * 4, st));
    BackwardArgs b;
    memset(&b, 0, sizeof(b));
    const int fin = s->ws.last_passes & 1;
    b.ranges = s->ws.ranges.as<uint2>();
    b.vals = s->ws.vals[fin].as<unsigned>();
    b.n = s->n;
    b.tiles_x = F.lay.tiles_x;
    b.tiles_y = F.lay.tiles_y;
    b.cam = F.cam;
    b.mean2 = s->ws.mean2.as<float4>();
    b.quad = s->ws.quad.as<float4>();
    b.rgb = s->ws.rgb.as<float>();
    b.touched = s->ws.touched.as<unsigned>();
    b.means = s->means.as<float>();
    b.scales = s->scales.as<float>();
    b.quats = s->quats.as<float>();
    b.sh = s->sh.as<float>();
    b.sh_degree = s->sh_degree;
    b.dL_dimg = dL_dimg;
    b.gbuf = s->ws.gbuf.as<float>();
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

} // extern "C"
