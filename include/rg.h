/*
 * rg.h -- C ABI of the GB300 RoofGS renderer (librg.so).
 *
 * Forward render of 3D Gaussian Splatting in two modes:
 *   RG_MODE_EXACT   the plain 3DGS path: FP32 attributes (236 bytes per
 *                   Gaussian, paper Sec. III-A, Eq. (3)), separate
 *                   preprocess / scan / duplicate kernels, 64-bit
 *                   tile|float-depth keys (Sec. IV-A.2), IEEE expf in the
 *                   rasterizer (Eqs. (7), (10)-(12));
 *   RG_MODE_ROOFGS  the paper's method: compact attributes (FP32 mean, FP16
 *                   rotation and scale, INT8 spherical harmonics with one
 *                   scale per degree and channel, Sec. IV-A.1, Eq. (8)), one
 *                   fused preprocess+duplicate+key kernel (Sec. IV-A.3), the
 *                   resolution-adaptive 32-bit key (Sec. IV-A.2, Eq. (9)),
 *                   coefficient folding and dual-pixel evaluation
 *                   (Sec. IV-B.1, Eqs. (13)-(20)) and the range-aware bit-level
 *                   exponential (Sec. IV-B.2, Eqs. (23)-(25)).
 *
 * Conventions for every entry point:
 *   - Functions never abort or trap; they return an rg_status. On failure,
 *     rg_last_error() returns a thread-local message.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Work is stream-ordered; only rg_scene_create, rg_scene_destroy,
 *     rg_scene_reserve, rg_inspect and an rg_render call given a non-NULL
 *     `stats` synchronise the stream.
 *   - Device pointers must be CUDA device memory of the current device.
 *     Output buffers are owned by the caller. Input arrays may be freed after
 *     rg_scene_create returns.
 *   - One scene owns one frame workspace: rg_render calls on the same scene
 *     must be ordered on one stream (calls on different streams race).
 */
#ifndef RG_H
#define RG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RG_OK = 0,
    RG_ERR_INVALID_ARG = 1,  /* a NULL pointer, a bad size, a non-finite input, ... */
    RG_ERR_OOM = 2,          /* a device allocation failed */
    RG_ERR_CUDA = 3,         /* a CUDA call failed (message in rg_last_error) */
    RG_ERR_CAPACITY = 4,     /* entries exceeded the workspace and it could not grow */
    RG_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up (result invalid) */
    RG_ERR_BUSY = 6,
    RG_ERR_NOT_READY = 7,
    RG_ERR_UNSUPPORTED = 8   /* option not supported (e.g. rg_backward in RoofGS mode) */
} rg_status;

typedef struct rg_scene rg_scene;   /* opaque; owns every device buffer it allocates */
typedef struct rg_server rg_server; /* opaque; request loop (rg_server_create) */

/* storage flags of rg_scene_desc */
#define RG_STORE_FP32 1u     /* keep the FP32 attributes (needed by RG_MODE_EXACT) */
#define RG_STORE_COMPACT 2u  /* build the compact attributes (needed by RG_MODE_ROOFGS) */

/* sh_scale_mode of rg_scene_desc */
#define RG_SH_SCALE_BAND 0       /* Eq. (8): one INT8 scale per SH degree d and channel c */
#define RG_SH_SCALE_BAND_GAUSS 1 /* additionally one FP16 factor per Gaussian */

/*
 * Scene description (paper Table I notation: mean mu, rotation r, scale s,
 * opacity, plus degree-3 spherical harmonics).
 *   means     [n][3] FP32 world positions
 *   scales    [n][3] FP32 activated scales (standard deviations along the axes)
 *   quats     [n][4] FP32 rotations (w, x, y, z); normalised by the renderer
 *   opacities [n]    FP32 activated opacities in [0, 1]
 *   sh        [n][16][3] FP32 coefficients, index k = l^2 + l + m (real
 *             orthonormal harmonics without Condon-Shortley phase), then RGB
 *   on_device 1 if the five pointers are device memory, 0 if host memory
 * Every value must be finite; opacities outside [0, 1] are rejected.
 */
typedef struct {
    int64_t n;
    int32_t sh_degree; /* 0..3: coefficients beyond (deg+1)^2 are ignored */
    int32_t on_device;
    const float* means;
    const float* scales;
    const float* quats;
    const float* opacities;
    const float* sh;
    uint32_t storage;      /* RG_STORE_* bits; 0 means both */
    int32_t sh_scale_mode; /* RG_SH_SCALE_* */
} rg_scene_desc;

/*
 * Pinhole camera. world -> camera: p = R mu + t (R row-major); the camera looks
 * along +z with x right and y down. Pixel (i, j) is sampled at the continuous
 * point (i, j): u = fx p_x / p_z + cx, v = fy p_y / p_z + cy. Gaussians with
 * p_z outside (znear, zfar] are culled (Sec. IV-A.2: the quantization interval
 * [z_near, z_far] is fixed per camera). bg is added with the final
 * transmittance: out = C + T bg.
 */
typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
    float znear, zfar;
    float bg[3];
} rg_camera;

#define RG_MODE_EXACT 0
#define RG_MODE_ROOFGS 1

/* RoofGS-mode ingredient flags (ignored in exact mode) */
#define RG_FLAG_EXACT_EXP (1u << 0)    /* use expf instead of the bit-level exponential of Eq. (24) */
#define RG_FLAG_SINGLE_PIXEL (1u << 1) /* one pixel per thread instead of the dual-pixel scheme, Eq. (20) */
/* sort the entries in 4 radix passes over the full 32-bit key, in Gaussian order (the
 * paper's scheme, Sec. IV-A.2), instead of ordering the Gaussians by quantized depth
 * first and sorting only the b_t tile bits of the entries; both give the same order */
#define RG_FLAG_SORT_FULL_KEY (1u << 2)
/* four vertically adjacent pixels per thread (Eq. (20) applied three times) instead of
 * two; RG_FLAG_SINGLE_PIXEL takes precedence when both are given */
#define RG_FLAG_QUAD_PIXEL (1u << 3)
/* flags for both modes */
#define RG_FLAG_STAGE_EVENTS (1u << 8) /* record per-stage CUDA events (rg_stage_times) */
#define RG_FLAG_BATCH_CHECKED (1u << 9) /* rg_render_batch: synchronise, and re-size and render again on overflow */
/* rg_render_batch: keep only the fused path (RoofGS, at most 32 views) or only the lanes (the
 * autotuner chooses between them otherwise) */
#define RG_FLAG_BATCH_FUSED (1u << 11)
#define RG_FLAG_BATCH_LANES (1u << 12)
/* RoofGS: group the depth-ordered entries by tile with one stable counting sort (per-chunk
 * tile counts, their prefix, one in-order scatter that also writes the tile ranges) instead
 * of the radix passes over the tile bits; the same entries and images. Needs the depth
 * pre-sort (not RG_FLAG_SORT_FULL_KEY), tile ids of at most 16 bits and at most 57,856
 * tiles (one 4-byte offset per tile in a block's shared memory); RG_ERR_UNSUPPORTED
 * otherwise. Not for rg_render_batch's fused path (its plans take the lanes). */
#define RG_FLAG_TILE_COUNTING_SORT (1u << 13)
/* RoofGS: the fused front end with the ordered allocation (one contiguous run of entries
 * per block, 16-bit tile ids) and the two 8-bit radix passes over the tile id, instead of the
 * default row-bucketed front end. The row-bucketed front end (frames with an image, the
 * depth pre-sort and at most 256 x 256 tiles) runs a count kernel (the fused front end's
 * work without the emission), a per-tile-row scan of its block counts and a scatter kernel
 * that writes each Gaussian's tile-row runs straight into their tile row's part of the
 * entry array under the column-major key tx << 8 | ty; one 8-bit pass over the column then
 * groups the entries by tile. Both give the same entries per tile in the same order, hence
 * the same images; rg_inspect returns the entries in tile-id order either way. Other frames
 * always take the fused front end. */
#define RG_FLAG_ORDERED_FRONT_END (1u << 14)
/* test hook for the failure path: the first radix pass of the entry sort never processes its
 * first tile, so the next tile's bounded look-back wait runs out (about a second); the frame
 * is invalid, kernels finish with in-bounds writes only, and the next rg_scene_check (or this
 * call, given stats) returns RG_ERR_TIMEOUT. The scene renders normally afterwards. */
#define RG_FLAG_TEST_STALL_SORT (1u << 10)

typedef struct {
    int32_t mode;   /* RG_MODE_EXACT or RG_MODE_ROOFGS */
    uint32_t flags; /* RG_FLAG_* */
    int32_t tile_w; /* tile shape in pixels: 16 x 16 (0 x 0 = default), 32 x 8 or 8 x 32; others */
    int32_t tile_h; /* return RG_ERR_UNSUPPORTED. rg_render_batch: 0 x 0 = autotuned */
} rg_render_opts;

/* Frame statistics (filled only when rg_render is given a non-NULL stats pointer). */
typedef struct {
    int64_t n_gaussians;
    int64_t n_front;    /* Gaussians inside (znear, zfar] (RoofGS: also with o >= 1/255) */
    int64_t n_visible;  /* Gaussians that emitted at least one (tile, Gaussian) entry */
    int64_t n_entries;  /* N_dup: (tile, Gaussian) entries sorted this frame */
    int64_t capacity;   /* entry capacity of the workspace after the call */
    int64_t n_pairs;    /* (Gaussian, pixel) exponents the rasterizer evaluated for unfinished pixels */
    int64_t n_blends;   /* of those, pairs inside the alpha >= 1/255 range (blended, or ending the pixel) */
    int32_t regrown;    /* 1 if the call grew the workspace and rendered again */
    int32_t sort_passes;
    int32_t b_t, b_d;   /* key bit split (RoofGS) or tile bits used (exact) */
    int32_t tiles_x, tiles_y;
} rg_stats;

/*
 * Create a resident scene (Sec. IV-A.1 for the compact layout): copies the FP32
 * attributes (RG_STORE_FP32) and/or builds the compact attributes
 * (RG_STORE_COMPACT): FP16 rotation and scale, FP32 mean, log o in FP32, and the
 * INT8 SH codes of Eq. (8) with their 12 band scales. Synchronises `stream`.
 * Errors: RG_ERR_INVALID_ARG (NULL/negative sizes, non-finite values,
 * opacity outside [0, 1], sh_degree outside 0..3), RG_ERR_OOM, RG_ERR_CUDA.
 */
rg_status rg_scene_create(const rg_scene_desc* desc, void* stream, rg_scene** out);

/* Free every device buffer of the scene (synchronises the device). NULL is a no-op. */
rg_status rg_scene_destroy(rg_scene* scene);

/*
 * Scene files (checkpoint / resume of a resident scene; the paper has no counterpart):
 * rg_scene_save writes the scene's stored buffers (the FP32 attributes and/or the compact
 * attributes with their 12 band scales) to `path` after a fixed header, raw little-endian;
 * rg_scene_load creates a scene from such a file on the current device without re-encoding,
 * so it renders bit-identically to the saved one. Both synchronise (the device / `stream`).
 * Errors: RG_ERR_INVALID_ARG (NULL argument, a file that cannot be opened, written or read,
 * or whose magic, version, fields or size do not match), RG_ERR_OOM, RG_ERR_CUDA.
 */
rg_status rg_scene_save(rg_scene* scene, const char* path);
rg_status rg_scene_load(const char* path, void* stream, rg_scene** out);

/* Grow the frame workspace to hold at least n_entries (tile, Gaussian) entries. Synchronous. */
rg_status rg_scene_reserve(rg_scene* scene, int64_t n_entries);

/*
 * Render one view into out_chw, a caller-owned buffer of 3*H*W FP32 values laid
 * out [channel][row][column]: device memory, or pinned host memory that the
 * device addresses (the image is then written straight to the host).
 * Pipeline (exact): preprocess -> scan -> duplicate -> 64-bit radix sort ->
 * tile ranges -> rasterizer (Sec. II-A pipeline, Sec. III). The exponent of
 * Eq. (10) is evaluated from the projected mean carried at twice single
 * precision and the quadratic form completed in dx, so the image stays within
 * 2e-4 per channel of an FP64 evaluation except where a pair's alpha or T lies
 * within rounding of the 1/255 or 1e-4 thresholds.
 * Pipeline (RoofGS): Gaussians ordered by quantized depth -> front end (by
 * default row-bucketed: the entries leave it grouped by tile row, in depth order)
 * -> stable radix sort of the remaining tile bits (one pass over the tile column;
 * two tile-bit passes after the fused front end of RG_FLAG_ORDERED_FRONT_END;
 * either way the order of the full 32-bit key; RG_FLAG_SORT_FULL_KEY sorts all
 * 32 bits in 4 passes instead) -> fast-exp rasterizer with 2 (dual-pixel), 1 or
 * 4 pixels per thread, each tile block finding its own range of the sorted
 * entries (Sec. IV).
 * The number of entries stays on the device: with stats == NULL the call does
 * not synchronise; if the entries exceed the workspace the image is
 * incomplete and the overflow is recorded (see rg_scene_check). With stats
 * != NULL the call synchronises, grows the workspace and renders again if
 * needed, and fills *stats.
 * Errors: RG_ERR_INVALID_ARG (NULL, width/height <= 0, zfar <= znear, a mode
 * whose storage the scene lacks), RG_ERR_UNSUPPORTED (a tile shape other than
 * 16x16, 32x8, 8x32), RG_ERR_CAPACITY, RG_ERR_TIMEOUT, RG_ERR_CUDA, RG_ERR_OOM.
 */
rg_status rg_render(rg_scene* scene, const rg_camera* cam, const rg_render_opts* opts, float* out_chw,
                    rg_stats* stats, void* stream);

/*
 * Report and clear the sticky device flags of every render since the last
 * check: RG_ERR_CAPACITY if a frame overflowed its workspace,
 * RG_ERR_TIMEOUT if a bounded device wait gave up, else RG_OK. Synchronous.
 */
rg_status rg_scene_check(rg_scene* scene, void* stream);

/*
 * Per-stage device times (ms) of the frames rendered with RG_FLAG_STAGE_EVENTS
 * since the last call (at most the last 512 frames), summed: ms7[0] = depth order of
 * the Gaussians (RoofGS; 0 otherwise), ms7[1] = front end (RoofGS fused kernel; exact
 * preprocess + scan + duplicate), ms7[2] = sort histogram, ms7[3] = sort passes,
 * ms7[4] = tile ranges, ms7[5] = rasterizer, ms7[6] = whole frame. *frames receives
 * the number of frames summed. Synchronises the recorded events.
 */
rg_status rg_stage_times(rg_scene* scene, float* ms7, int32_t* frames);

/* rg_inspect selectors: copy internal buffers of the last frame to host memory */
#define RG_INSPECT_KEYS 1        /* sorted keys: uint32 (RoofGS) or uint64 (exact), n_entries of them;
                                    RoofGS frames with at most 16 tile bits sort 16-bit tile keys and
                                    the 32-bit keys (tile << b_d | q_d) are rebuilt on the host from
                                    the values and the per-Gaussian depth codes; the entries of a
                                    row-bucketed frame (column-major tile keys) are first regrouped in
                                    tile-id order from the tile ranges, so every frame reports the
                                    order of the 32-bit key */
#define RG_INSPECT_VALUES 2      /* sorted values: uint32 Gaussian indices (in the same order) */
#define RG_INSPECT_RANGES 3      /* uint32 [tiles][2] = [start, end) per tile (of the same order) */
#define RG_INSPECT_SH_CODES 4    /* int8 [n][16][3] compact SH codes */
#define RG_INSPECT_SH_SCALES 5   /* float [4][3] band scales s_{d,c} */
#define RG_INSPECT_GAUSS_SCALE 6 /* uint16 [n] FP16 per-Gaussian SH factors */
#define RG_INSPECT_GEOM16 7      /* uint16 [n][8] = q (4), s (3), g as FP16 bits */
#define RG_INSPECT_LOG_OPACITY 8 /* float [n] stored log o */

/*
 * Copy one internal buffer to host memory (synchronises the device).
 * *out_bytes receives the buffer size; if cap_bytes is smaller nothing is
 * copied and RG_ERR_INVALID_ARG is returned.
 */
rg_status rg_inspect(rg_scene* scene, int32_t what, void* host_dst, int64_t cap_bytes, int64_t* out_bytes);

/*
 * Diagnostic: out_dev[i] = exp^(P_dev[i]), the bit-level exponential of Eq. (24)
 * exactly as the RoofGS rasterizer evaluates it (FP32, valid on [-ln 255, 0]).
 * Device arrays of n floats; stream-ordered.
 */
rg_status rg_eval_fast_exp(const float* P_dev, float* out_dev, int64_t n, void* stream);

/*
 * Allocation-free sort (the paper has no counterpart: it is a service of this
 * library for callers that must not allocate device memory -- a real-time
 * render thread, where cudaMalloc may block on the device; a plugin whose
 * host application owns all device memory; work being recorded into a CUDA
 * graph). Sorts the n (key, value) pairs of the caller's device arrays in
 * place, stably, by the low key_bits bits of the key (8, 16, 24 or 32), with
 * the same radix-sort kernels as rg_render. All scratch memory (alternate
 * buffers, histograms, look-back status, counters) is one static device array
 * of about 4.3 MiB that every GPU loading the library keeps until the process
 * exits; nothing is allocated or freed.
 *   keys, vals  device arrays of n uint32 (input and output), each starting on a
 *               16-byte boundary (cudaMalloc gives 256); a misaligned pointer
 *               returns RG_ERR_INVALID_ARG before anything is launched
 *   n           0 .. 524288; larger n returns RG_ERR_INVALID_ARG
 *   error_dev   optional device uint32: receives 0, or non-zero error bits if a
 *               bounded device wait gave up (the output is then invalid)
 * Stream-ordered, no host synchronisation. The first call on a device looks up
 * that device's scratch address (once per device, with the device current);
 * make that first call before any stream capture. Every call shares the one
 * scratch array, which keeps the previous call's contents (the sort clears
 * what must start at zero): calls that overlap on the GPU -- on different
 * streams, or from different host threads -- race and must be ordered by the
 * caller. A CUDA error left pending by an earlier call is reported as
 * RG_ERR_CUDA and left pending (nothing is launched).
 */
rg_status rg_sort_pairs_noalloc(uint32_t* keys, uint32_t* vals, int64_t n, int32_t key_bits, uint32_t* error_dev,
                                void* stream);

/*
 * Gradients of an exact-mode render (not in the paper: the backward of the
 * forward of Sec. III-D, Eqs. (7), (10)-(12)). Output arrays are caller-owned
 * device buffers with the layout of rg_scene_desc; every value is written.
 */
typedef struct {
    float* means;     /* [n][3] dL/dmeans */
    float* scales;    /* [n][3] dL/dscales (activated scales) */
    float* quats;     /* [n][4] dL/dquats (raw quaternion, through the normalisation) */
    float* opacities; /* [n]    dL/dopacities (activated) */
    float* sh;        /* [n][16][3] dL/dSH */
} rg_grads;

/*
 * Given dL/dimage (device [3][H][W]) for the image rg_render produces for this
 * scene, camera and opts, write the gradients of L with respect to the scene's
 * FP32 attributes. Runs the front end, sort and ranges of the frame again,
 * then a rasterizer backward that replays each pixel's front-to-back blend to
 * recover its transmittance (nothing is stored between forward and backward),
 * walks the pairs back to front, and a per-Gaussian backward through the conic,
 * the EWA covariance, the quaternion rotation, the projected mean and the SH
 * colour. Synchronises the stream once (to check the entry capacity).
 * Errors: RG_ERR_UNSUPPORTED for RoofGS mode (INT8/FP16 storage and the
 * bit-level exponential are not differentiated), RG_ERR_INVALID_ARG, ...
 */
rg_status rg_backward(rg_scene* scene, const rg_camera* cam, const rg_render_opts* opts, const float* dL_dimg,
                      const rg_grads* grads, void* stream);

/*
 * Batched multi-view rendering (not in the paper; serving-oriented). View v is
 * rendered from scenes[scene_idx[v]] with cams[v] (any resolution) into outs[v]
 * (device [3][H][W], caller-owned), all in opts->mode. The first call for a set of
 * (scenes, resolutions, mode, flags) creates a plan: lanes of stream + workspace,
 * sized by rendering every view once per candidate tile shape (synchronous), then an
 * autotuner times the captured batch with every tile shape (16 x 16, 32 x 8, 8 x 32,
 * unless opts gives one), every path and 1, 2 and 4 pixels per thread (RoofGS) and
 * keeps the fastest. Paths: (a) lanes: each view's whole pipeline on its lane (view v
 * on lane v mod lanes; 1, 2 or 4 lanes, each a stream and a workspace); (b) fused
 * (RoofGS, at most 32 views; one workspace per view): each view's depth order on the
 * lanes, then ONE front-end launch over the Gaussians of every view, each view's
 * entry sort on the lanes, then ONE persistent rasterizer launch whose blocks take the
 * (view, tile) items of every view from a work counter. Every call captures the batch
 * into one CUDA graph, updates the plan's instantiated graph in place (cameras are
 * kernel parameters) and launches it once on `stream`: no host synchronisation
 * (unless RG_FLAG_BATCH_CHECKED). Images are identical to rg_render's. An entry
 * overflow is recorded in the scene's sticky flags (rg_scene_check), as for
 * rg_render without stats. Scenes may repeat across views freely. A plan keeps its
 * workspaces until one of its scenes is destroyed (at most 8 plans are kept).
 * RG_ERR_UNSUPPORTED: RG_FLAG_BATCH_FUSED with exact mode or more than 32 views.
 */
rg_status rg_render_batch(rg_scene* const* scenes, const int32_t* scene_idx, const rg_camera* cams, int32_t n,
                          const rg_render_opts* opts, float* const* outs, void* stream);

/* The autotuned lane count, pixels per thread, tile shape and path (fused 1, lanes 0) of
 * the plan for these views (lanes 0 if no plan exists yet); tile_w, tile_h and fused may
 * be NULL. */
rg_status rg_batch_plan_info(rg_scene* const* scenes, const int32_t* scene_idx, const rg_camera* cams, int32_t n,
                             const rg_render_opts* opts, int32_t* lanes, int32_t* pixels_per_thread, int32_t* tile_w,
                             int32_t* tile_h, int32_t* fused);

/*
 * Request loop (serving; not in the paper). A server keeps its scenes resident and
 * owns slots: one CUDA stream, one frame workspace and one result buffer of the
 * largest resolution each. The slot count is cfg->max_slots (0 = 8), cut down to
 * what cfg->memory_budget (0 = 8 GiB) holds at the calibrated slot size (the
 * largest scene rendered once at the largest resolution from cfg->calibration's
 * pose, +50 % headroom): admission by device memory. A dispatcher thread takes
 * queued requests in submission order into free slots as earlier ones complete,
 * so requests that arrive while others run are admitted and overlap on the
 * device (continuous batching); a request whose entries overflow its slot is
 * rendered again after the slot grows. Results are those of rg_render.
 */
typedef struct {
    int32_t max_slots;           /* concurrent requests (0 = 8) */
    int64_t memory_budget;       /* device bytes for slots (0 = 8 GiB) */
    int32_t max_width, max_height; /* largest request resolution */
    int32_t mode;                /* RG_MODE_* for every request */
    uint32_t flags;              /* RG_FLAG_* (ingredient flags) for every request */
    const rg_camera* calibration; /* pose used to size slots (NULL: start small, grow on demand) */
} rg_server_config;

typedef struct {
    int64_t completed;     /* requests finished since the last reset */
    int64_t pending;       /* requests waiting for a slot */
    int32_t slots;         /* slots admitted by the memory budget */
    int32_t max_in_flight; /* most requests rendering at once since the last reset */
    double p50_ms, p99_ms; /* submit -> result ready latency percentiles since the last reset */
    int64_t slot_bytes;    /* calibrated bytes per slot */
    double p50_delivered_ms, p99_delivered_ms; /* submit -> image copied into the caller's buffer by
                                                  rg_poll (includes the caller's polling delay) */
} rg_server_stats_t;

/* Create a server over n_scenes resident scenes (the scenes must outlive it). Synchronous. */
rg_status rg_server_create(rg_scene* const* scenes, int32_t n_scenes, const rg_server_config* cfg, rg_server** out);
/* Finish queued and running requests, stop the dispatcher, free the slots. */
rg_status rg_server_destroy(rg_server* server);
/* Queue one request (camera of at most the maximum resolution, scene index); non-blocking. */
rg_status rg_submit(rg_server* server, const rg_camera* cam, int32_t scene_slot, uint64_t* ticket);
/*
 * RG_ERR_NOT_READY while the request waits or renders. When it is done, copy its
 * image into out_chw ([3][H][W] of the request's camera, device or pinned host
 * memory; the copy is complete when rg_poll returns), free the slot and return
 * RG_OK (or the request's error: RG_ERR_TIMEOUT, RG_ERR_CAPACITY, ...). A ticket
 * can be collected once.
 */
rg_status rg_poll(rg_server* server, uint64_t ticket, float* out_chw);
rg_status rg_server_stats(rg_server* server, rg_server_stats_t* stats);
rg_status rg_server_reset_stats(rg_server* server);

/* Message of the last failed call on this thread ("" if none). */
const char* rg_last_error(void);

/* ABI version: 100 * major + minor. */
int32_t rg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RG_H */
