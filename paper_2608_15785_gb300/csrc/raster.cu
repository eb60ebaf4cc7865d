// raster.cu -- tile rasterizers (one thread block per tile of 256 pixels:
// 16x16, 32x8 or 8x32).
//
// Front-to-back alpha blending of Sec. III-D, Eq. (7): for each pixel, over
// the tile's depth-sorted Gaussians, alpha = min(0.99, o exp(p)) (Eqs. (10)-(12)),
// pairs with alpha < 1/255 are skipped, the loop stops (without adding) once
// the transmittance would fall below 1e-4, C += c alpha T, out = C + T bg.
//
// RoofGS mode (Sec. IV-B): the block first finds its tile's [start, end) in
// the sorted keys (warp-cooperative search). While a batch of records is
// staged in shared memory, each Gaussian's coefficients are folded (Eqs.
// (13)-(15)) -- -1/2 and log o absorbed, C1..C6 -- in TILE-LOCAL coordinates
// (pixel and mean shifted by the tile origin, so the FP32 terms stay small at
// 4K); every thread owns PPT vertically adjacent pixels (x, y) ... (x,
// y+PPT-1), two by default (the paper's dual-pixel scheme), one or four on
// request: the first exponent is the FMA chain of Eq. (16) on hoisted x^2, xy,
// y^2, x, y, each next one follows from Eq. (20) (two additions per extra
// row). Pairs with P < -ln 255 are skipped before any exponential (Eq. (23));
// alpha = min(0.99, exp^(P)) with the bit-level exponential of Eq. (24)
// (Eq. (25)). With 2 or 4 pixels per thread the timed kernel blends the thread's
// pixels in pairs with packed FP32x2 FMAs (the same roundings as one at a time). A
// warp whose pixels are all finished skips the batch (vote); the block leaves once
// every pixel is finished.
#include "rg_internal.cuh"

namespace rg {

// Eq. (24) evaluated in FP32: I = floor(P 2^23 log2 e + 2^23 (127 - sigma)).
// With w = fma(P, log2 e, 127 - sigma) in [64, 128) (P in [-ln 255, 0]),
// 2^23 * w is exactly the FP32 result of fma(P, 2^23 log2 e, 2^23 (127 - sigma))
// (scaling by 2^23 commutes with rounding) and is an integer multiple of 64, so
// I = 2^23 w = 2^29 + 64 * mantissa(w) = (bits(w) << 6) + 2^31 (mod 2^32):
// one FFMA and one integer shift-add instead of a float->int conversion.
__device__ __forceinline__ float fast_exp(float P)
{
    const float w = fmaf(P, 1.44269502f, 126.954323f);
    return __uint_as_float((__float_as_uint(w) << 6) + 0x80000000u);
}

__global__ void k_fast_exp_eval(const float* P, float* out, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = fast_exp(P[i]);
}

template <bool FAST, bool COUNT>
__device__ __forceinline__ void blend(float P, float r, float g, float b, float& T, float& c0, float& c1, float& c2,
                                      bool& done, unsigned& n_eval, unsigned& n_blend)
{
    if (COUNT && !done) {
        n_eval++;
        if (P >= -LN255F) n_blend++;
    }
    if (!done && P >= -LN255F) {
        const float e = FAST ? fast_exp(P) : expf(P);
        const float alpha = fminf(0.99f, e);
        const float Tn = fmaf(-T, alpha, T); // T (1 - alpha)
        if (Tn < 1e-4f) {
            done = true;
        } else {
            const float wgt = alpha * T;
            c0 = fmaf(r, wgt, c0);
            c1 = fmaf(g, wgt, c1);
            c2 = fmaf(b, wgt, c2);
            T = Tn;
        }
    }
}

// A thread's pixels blended in pairs with packed FP32x2 arithmetic (FFMA2 / FMUL2: one
// instruction for both pixels of a pair). Per pixel the operations and roundings of
// blend<true, false>, written with -alpha (the shift-add of Eq. (24) without its + 2^31
// is -exp^(P): that addition only sets the sign bit) and with the negated colours nr, ng,
// nb: T + T (-alpha) = T (1 - alpha) and c + (-r)(-alpha T) = c + r (alpha T) round to the
// same values. A pixel's state is its skip threshold thr: -ln 255 while it blends, +inf
// once finished; a pixel below its threshold takes -alpha = 0, which leaves its T and
// colour unchanged. One branch skips the Gaussian when no pixel of the thread needs it;
// the stop below 1e-4 (at most once in a pixel's life) is a branch around the common path
// (4K raster 0.558 -> 0.476 ms against selects on every pair and a finished flag beside
// the threshold test; 0.476 -> 0.453 ms with the branches taken once for all of the
// thread's pairs instead of once per pair).
template <int NH>
__device__ __forceinline__ void blend_pairs_fast(const float (&P)[2 * NH], float2 nr, float2 ng, float2 nb,
                                                 float2 (&T)[NH], float2 (&cr)[NH], float2 (&cg)[NH],
                                                 float2 (&cb)[NH], float (&thr)[2 * NH])
{
    bool u[2 * NH];
    bool any = false;
#pragma unroll
    for (int i = 0; i < 2 * NH; i++) {
        u[i] = P[i] >= thr[i];
        any = any || u[i];
    }
    if (!any) return;
    float2 Tn[NH], nw[NH];
    bool stop = false;
#pragma unroll
    for (int h = 0; h < NH; h++) {
        const float2 w = __ffma2_rn(make_float2(P[2 * h], P[2 * h + 1]), make_float2(1.44269502f, 1.44269502f),
                                    make_float2(126.954323f, 126.954323f));
        const float ea = __uint_as_float(__float_as_uint(w.x) << 6); // -exp^(P)
        const float eb = __uint_as_float(__float_as_uint(w.y) << 6);
        const float2 na = make_float2(u[2 * h] ? fmaxf(-0.99f, ea) : 0.0f, u[2 * h + 1] ? fmaxf(-0.99f, eb) : 0.0f);
        Tn[h] = __ffma2_rn(T[h], na, T[h]);
        nw[h] = __fmul2_rn(na, T[h]); // -alpha T
        stop = stop || Tn[h].x < 1e-4f || Tn[h].y < 1e-4f;
    }
    if (stop) { // a pixel that would fall below 1e-4 adds nothing (weight 0, T kept) and finishes
#pragma unroll
        for (int h = 0; h < NH; h++) {
            if (Tn[h].x < 1e-4f) {
                nw[h].x = 0.0f;
                Tn[h].x = T[h].x;
                thr[2 * h] = __int_as_float(0x7f800000); // +inf: finished
            }
            if (Tn[h].y < 1e-4f) {
                nw[h].y = 0.0f;
                Tn[h].y = T[h].y;
                thr[2 * h + 1] = __int_as_float(0x7f800000);
            }
        }
    }
#pragma unroll
    for (int h = 0; h < NH; h++) {
        cr[h] = __ffma2_rn(nr, nw[h], cr[h]);
        cg[h] = __ffma2_rn(ng, nw[h], cg[h]);
        cb[h] = __ffma2_rn(nb, nw[h], cb[h]);
        T[h] = Tn[h];
    }
}

// The same blend for a thread with one pixel: the skip threshold as its state, the stop
// below 1e-4 a branch around the common path (bit-identical to blend<true, false>).
__device__ __forceinline__ void blend_one_fast(float P, float nr, float ng, float nb, float& T, float& cr, float& cg,
                                               float& cb, float& thr)
{
    if (!(P >= thr)) return;
    const float w = fmaf(P, 1.44269502f, 126.954323f);
    const float na = fmaxf(-0.99f, __uint_as_float(__float_as_uint(w) << 6)); // -alpha
    float Tn = fmaf(T, na, T);
    float nw = na * T; // -alpha T
    if (Tn < 1e-4f) { // once in the pixel's life: adds nothing, T kept, finished
        nw = 0.0f;
        Tn = T;
        thr = __int_as_float(0x7f800000);
    }
    cr = fmaf(nr, nw, cr);
    cg = fmaf(ng, nw, cg);
    cb = fmaf(nb, nw, cb);
    T = Tn;
}

// sums the per-thread work counters of a counting launch into the frame counters
__device__ __forceinline__ void flush_counts(Counters* c, unsigned n_eval, unsigned n_blend)
{
    unsigned long long e = n_eval, b = n_blend;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&c->n_pairs, e);
        atomicAdd(&c->n_blends, b);
    }
}

// First index i in [0, n) with (keys[i] >> shift) >= t, n if none (keys sorted): a
// 33-ary search by one warp, each round 32 lanes probe and one ballot keeps the part
// that holds the boundary (six dependent loads for 68 M keys). Warp-uniform result.
// K: 32-bit keys or 16-bit tile ids.
template <typename K>
__device__ __forceinline__ unsigned warp_lower_bound(const K* __restrict__ keys, unsigned n, int shift, unsigned t)
{
    const int lane = threadIdx.x & 31;
    unsigned lo = 0, hi = n; // the answer lies in [lo, hi]
    while (hi - lo > 32) {
        const unsigned probe = lo + (unsigned)(((unsigned long long)(hi - lo) * (unsigned)(lane + 1)) / 33u);
        const bool less = (unsigned)((unsigned long long)__ldg(&keys[probe]) >> shift) < t;
        const int c = __popc(__ballot_sync(0xffffffffu, less)); // lanes 0..c-1 probe below the boundary
        const unsigned plo = __shfl_sync(0xffffffffu, probe, c > 0 ? c - 1 : 0);
        const unsigned phi = __shfl_sync(0xffffffffu, probe, c < 32 ? c : 31);
        if (c > 0) lo = plo + 1;
        if (c < 32) hi = phi;
    }
    const unsigned i = lo + (unsigned)lane;
    const bool less = i < hi && (unsigned)((unsigned long long)__ldg(&keys[i]) >> shift) < t;
    return lo + (unsigned)__popc(__ballot_sync(0xffffffffu, less));
}

// One tile of the RoofGS rasterizer (a block of 256 / PPT threads).
template <bool FAST, int PPT, bool COUNT>
__device__ __forceinline__ void raster_tile(const RasterArgs& a, const int tile)
{
    constexpr int NT = 256 / PPT; // threads per tile of 256 pixels (16 x 16, 32 x 8 or 8 x 32)
    constexpr int NH = (PPT + 1) / 2; // pixel pairs of a thread (one pixel of the last pair unused at PPT 1)
    __shared__ float4 s_c0[NT];       // C1, C2, C3, C4
    __shared__ float4 s_c1[NT];       // C5, C6, -b, -b (1 pixel per thread: C5, C6, -r, -g)
    // -r, -r, -g, -g (pairs for the packed blend; 1 pixel per thread: -b in .x)
    __shared__ float4 s_cn[PPT == 1 ? 1 : NT];
    __shared__ float s_cb[PPT == 1 ? NT : 1];
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int x0 = tx * a.cam.tw, y0 = ty * a.cam.th;
    const int t = threadIdx.x;
    // the thread's pixels: (x, y), (x, y+1), ..., (x, y+PPT-1)
    const int lx = t & (a.cam.tw - 1);
    const int ly = (t >> a.cam.tw_log2) * PPT;
    const int px = x0 + lx, py = y0 + ly;
    const int W = a.cam.W, H = a.cam.H;
    bool done[PPT];
    // the packed pair blend keeps a pixel's state as its skip threshold instead: -ln 255 while it
    // blends, +inf once finished (one compare per pixel and Gaussian instead of two tests)
    constexpr bool PAIRS = FAST && !COUNT && PPT >= 2;
    constexpr bool ONE = FAST && !COUNT && PPT == 1;
    float thr[PPT];
    // transmittance and colour of pixel i in component i & 1 of pair i / 2
    float2 T2[NH], R2[NH], G2[NH], B2[NH];
#pragma unroll
    for (int h = 0; h < NH; h++) {
        T2[h] = make_float2(1.0f, 1.0f);
        R2[h] = G2[h] = B2[h] = make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int i = 0; i < PPT; i++) {
        done[i] = !(px < W && py + i < H);
        thr[i] = done[i] ? __int_as_float(0x7f800000) : -LN255F;
    }
    // hoisted pixel terms (tile-local)
    const float x = (float)lx, y = (float)ly;
    const float xx = x * x, xy = x * y, yy = y * y, y2p1 = 2.0f * y + 1.0f;
    unsigned n_eval = 0, n_blend = 0;
    uint2 range;
    if (a.skeys || a.skeys16) { // warps 0 and 1 search the first entries of tiles `tile` and `tile + 1`
        __shared__ unsigned s_bound[2];
        const int warp = t >> 5;
        if (warp < 2) {
            const unsigned n = a.ctr->n_entries;
            // the tile's key: its id, or tx << 8 | ty for column-major keys (ty + 1 <= 256
            // carries into the next column, whose first entry also ends this tile)
            const unsigned key = a.key_cols ? (((unsigned)tx << 8) | (unsigned)ty) : (unsigned)tile;
            const unsigned b = a.skeys16 ? warp_lower_bound(a.skeys16, n, 0, key + (unsigned)warp)
                                         : warp_lower_bound(a.skeys, n, a.tile_shift, key + (unsigned)warp);
            if ((t & 31) == 0) s_bound[warp] = b;
        }
        __syncthreads();
        range = s_bound[1] > s_bound[0] ? make_uint2(s_bound[0], s_bound[1]) : make_uint2(0u, 0u);
        if (t == 0) a.ranges_out[tile] = range;
    } else {
        range = a.ranges[tile];
    }
    for (unsigned start = range.x; start < range.y; start += NT) {
        bool all_done = true;
#pragma unroll
        for (int i = 0; i < PPT; i++)
            all_done = all_done && ((PAIRS || ONE) ? thr[i] == __int_as_float(0x7f800000) : done[i]);
        if (__syncthreads_count(!all_done) == 0) break;
        const unsigned j = start + t;
        if (j < range.y) {
            unsigned id = a.vals[j];
            if (id >= (unsigned long long)a.n) id = 0; // only after a failed (timed-out) sort
            const float4 q0 = __ldg(&a.rec[2 * id]);
            const float4 q1 = __ldg(&a.rec[2 * id + 1]);
            const float u = q0.x - (float)x0, v = q0.y - (float)y0;
            const float ca = q0.z, cbq = q0.w, cc = q1.x, logo = q1.y;
            // Eq. (15): folded coefficients
            const float C1 = -0.5f * ca, C2 = -0.5f * cbq, C3 = -0.5f * cc;
            const float C4 = fmaf(ca, u, 0.5f * cbq * v);
            const float C5 = fmaf(cc, v, 0.5f * cbq * u);
            const float C0 = fmaf(ca * u, u, fmaf(cbq * u, v, cc * v * v)); // Eq. (14)
            const float C6 = fmaf(-0.5f, C0, logo);
            const unsigned rg = __float_as_uint(q1.z), bb = __float_as_uint(q1.w);
            const float fr = __half2float(__ushort_as_half((unsigned short)(rg & 0xffffu)));
            const float fg = __half2float(__ushort_as_half((unsigned short)(rg >> 16)));
            const float fb = __half2float(__ushort_as_half((unsigned short)(bb & 0xffffu)));
            s_c0[t] = make_float4(C1, C2, C3, C4);
            if constexpr (PPT == 1) {
                s_c1[t] = make_float4(C5, C6, -fr, -fg);
                s_cb[t] = -fb;
            } else {
                s_c1[t] = make_float4(C5, C6, -fb, -fb);
                s_cn[t] = make_float4(-fr, -fr, -fg, -fg);
            }
        }
        __syncthreads();
        const int cnt = min((unsigned)NT, range.y - start);
        if (!__all_sync(0xffffffffu, all_done)) {
#pragma unroll(PPT == 4 ? 2 : 4) // records per iteration, 4K raster: 4 pixels 0.564 -> 0.558 ms (2), 2 pixels 0.549 -> 0.540 ms and 1 pixel 1.059 -> 0.900 ms (4)
            for (int k = 0; k < cnt; k++) {
                const float4 c0 = s_c0[k];
                const float4 c1 = s_c1[k];
                // negated colours, from the pairs' layout or the one-pixel layout
                float nr, ng, nb;
                float4 cn = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if constexpr (PPT == 1) {
                    nr = c1.z;
                    ng = c1.w;
                    nb = s_cb[k];
                } else {
                    cn = s_cn[k];
                    nr = cn.x;
                    ng = cn.z;
                    nb = c1.z;
                }
                // Eq. (16): P(x, y) = C1 x^2 + C2 xy + C3 y^2 + C4 x + C5 y + C6
                float P[PPT];
                P[0] = fmaf(c0.x, xx, fmaf(c0.y, xy, fmaf(c0.z, yy, fmaf(c0.w, x, fmaf(c1.x, y, c1.y)))));
                if (PPT >= 2) {
                    // Eq. (20): P(x, y+1) = P(x, y) + C2 x + C3 (2y + 1) + C5; the step to the next
                    // row grows by 2 C3 per row
                    float d = fmaf(c0.y, x, fmaf(c0.z, y2p1, c1.x));
#pragma unroll
                    for (int i = 1; i < PPT; i++) {
                        if (i > 1) d = fmaf(2.0f, c0.z, d);
                        P[i] = P[i - 1] + d;
                    }
                }
                if constexpr (PAIRS) {
                    blend_pairs_fast<NH>(P, make_float2(cn.x, cn.y), make_float2(cn.z, cn.w), make_float2(c1.z, c1.w),
                                         T2, R2, G2, B2, thr);
                } else if constexpr (ONE) {
                    blend_one_fast(P[0], nr, ng, nb, T2[0].x, R2[0].x, G2[0].x, B2[0].x, thr[0]);
                } else {
#pragma unroll
                    for (int i = 0; i < PPT; i++) {
                        float& Ti = (i & 1) ? T2[i >> 1].y : T2[i >> 1].x;
                        float& Ri = (i & 1) ? R2[i >> 1].y : R2[i >> 1].x;
                        float& Gi = (i & 1) ? G2[i >> 1].y : G2[i >> 1].x;
                        float& Bi = (i & 1) ? B2[i >> 1].y : B2[i >> 1].x;
                        blend<FAST, COUNT>(P[i], -nr, -ng, -nb, Ti, Ri, Gi, Bi, done[i], n_eval, n_blend);
                    }
                }
            }
        }
    }
    if (COUNT) flush_counts(a.count, n_eval, n_blend);
    const size_t plane = (size_t)W * H;
#pragma unroll
    for (int i = 0; i < PPT; i++) {
        if (px < W && py + i < H) {
            const size_t o = (size_t)(py + i) * W + px;
            const float Ti = (i & 1) ? T2[i >> 1].y : T2[i >> 1].x;
            a.out[o] = ((i & 1) ? R2[i >> 1].y : R2[i >> 1].x) + Ti * a.cam.bg[0];
            a.out[plane + o] = ((i & 1) ? G2[i >> 1].y : G2[i >> 1].x) + Ti * a.cam.bg[1];
            a.out[2 * plane + o] = ((i & 1) ? B2[i >> 1].y : B2[i >> 1].x) + Ti * a.cam.bg[2];
        }
    }
}

template <bool FAST, int PPT, bool COUNT>
__global__ void __launch_bounds__(256 / PPT) k_raster_roofgs(RasterArgs a)
{
    grid_dependency_wait();
    raster_tile<FAST, PPT, COUNT>(a, blockIdx.x);
}

// Every view of a batch in one persistent launch: each block takes (view, tile) items
// from one work counter (views in order, tiles in order) until all are done, and
// rasterizes the tile with that view's arguments (kernel parameter space).
template <bool FAST, int PPT>
__global__ void __launch_bounds__(256 / PPT) k_raster_views(const __grid_constant__ RasterViews m)
{
    __shared__ unsigned s_g;
    grid_dependency_wait();
    const unsigned total = m.tile_prefix[m.n_views];
    while (true) {
        if (threadIdx.x == 0) s_g = atomicAdd(m.claim, 1u);
        __syncthreads();
        const unsigned g = s_g;
        if (g >= total) break;
        int v = 0;
        while (v + 1 < m.n_views && m.tile_prefix[v + 1] <= g) v++;
        raster_tile<FAST, PPT, false>(m.views[v], (int)(g - m.tile_prefix[v]));
        __syncthreads(); // every thread has read s_g before it is claimed again
    }
}

template <bool FAST, int PPT>
static void raster_views_launch(const RasterViews& m, cudaStream_t s)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_raster_views<FAST, PPT>, 256 / PPT, 0);
    const unsigned total = m.tile_prefix[m.n_views];
    unsigned grid = (unsigned)((per_sm > 0 ? per_sm : 1) * device_sm_count());
    if (grid > total) grid = total;
    if (grid) launch_dependent(k_raster_views<FAST, PPT>, dim3(grid), dim3(256 / PPT), 0, s, m);
}

void launch_raster_views(const RasterViews& m, int fast_exp, int ppt, cudaStream_t s)
{
    if (fast_exp) {
        if (ppt == 1) raster_views_launch<true, 1>(m, s);
        else if (ppt == 4) raster_views_launch<true, 4>(m, s);
        else raster_views_launch<true, 2>(m, s);
    } else {
        if (ppt == 1) raster_views_launch<false, 1>(m, s);
        else if (ppt == 4) raster_views_launch<false, 4>(m, s);
        else raster_views_launch<false, 2>(m, s);
    }
}

template <bool COUNT>
static void raster_roofgs_variant(const RasterArgs& a, cudaStream_t s)
{
    const unsigned tiles = (unsigned)(a.tiles_x * a.tiles_y);
    if (a.fast_exp) {
        if (a.ppt == 1) launch_dependent(k_raster_roofgs<true, 1, COUNT>, dim3(tiles), dim3(256), 0, s, a);
        else if (a.ppt == 4) launch_dependent(k_raster_roofgs<true, 4, COUNT>, dim3(tiles), dim3(64), 0, s, a);
        else launch_dependent(k_raster_roofgs<true, 2, COUNT>, dim3(tiles), dim3(128), 0, s, a);
    } else {
        if (a.ppt == 1) launch_dependent(k_raster_roofgs<false, 1, COUNT>, dim3(tiles), dim3(256), 0, s, a);
        else if (a.ppt == 4) launch_dependent(k_raster_roofgs<false, 4, COUNT>, dim3(tiles), dim3(64), 0, s, a);
        else launch_dependent(k_raster_roofgs<false, 2, COUNT>, dim3(tiles), dim3(128), 0, s, a);
    }
}

void launch_raster_roofgs(const RasterArgs& a, cudaStream_t s)
{
    if (a.count) raster_roofgs_variant<true>(a, s);
    else raster_roofgs_variant<false>(a, s);
}

// Plain 3DGS rasterizer: one pixel per thread, expf. The exponent of Eq. (10) is
// evaluated in the completed-square form of exact_power() from the double-float
// mean, shifted to the tile origin when a record is staged (u.hi - x0 is exact).
constexpr int E_THREADS = 256;

template <bool COUNT>
__global__ void __launch_bounds__(E_THREADS) k_raster_exact(RasterArgs a)
{
    __shared__ float4 s_m[E_THREADS];
    __shared__ float4 s_q[E_THREADS];
    __shared__ float4 s_rgb[E_THREADS];
    grid_dependency_wait();
    const int tile = blockIdx.x;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int x0 = tx * a.cam.tw, y0 = ty * a.cam.th;
    const int lxi = threadIdx.x & (a.cam.tw - 1), lyi = threadIdx.x >> a.cam.tw_log2;
    const int px = x0 + lxi, py = y0 + lyi;
    const int W = a.cam.W, H = a.cam.H;
    const bool inside = px < W && py < H;
    bool done = !inside;
    const float lx = (float)lxi, ly = (float)lyi;
    float T = 1.0f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
    unsigned n_eval = 0, n_blend = 0;
    const uint2 range = a.ranges[tile];
    for (unsigned start = range.x; start < range.y; start += E_THREADS) {
        if (__syncthreads_count(!done) == 0) break;
        const unsigned j = start + threadIdx.x;
        if (j < range.y) {
            unsigned id = a.vals[j];
            if (id >= (unsigned long long)a.n) id = 0; // only after a failed (timed-out) sort
            const float4 m = a.mean2[id];
            s_m[threadIdx.x] = make_float4(m.x - (float)x0, m.y, m.z - (float)y0, m.w);
            s_q[threadIdx.x] = a.quad[id];
            s_rgb[threadIdx.x] = make_float4(a.rgb[3 * id], a.rgb[3 * id + 1], a.rgb[3 * id + 2], 0.f);
        }
        __syncthreads();
        const int cnt = min((unsigned)E_THREADS, range.y - start);
        for (int k = 0; !done && k < cnt; k++) {
            const float4 q = s_q[k];
            const float power = exact_power(s_m[k], q, lx, ly); // Eq. (10), <= 0
            if (COUNT) n_eval++;
            const float alpha = fminf(0.99f, q.w * expf(power)); // Eqs. (11)-(12)
            if (alpha < 1.0f / 255.0f) continue;
            if (COUNT) n_blend++;
            const float Tn = T * (1.0f - alpha);
            if (Tn < 1e-4f) {
                done = true;
                continue;
            }
            const float4 c = s_rgb[k];
            const float wgt = alpha * T;
            c0 += c.x * wgt;
            c1 += c.y * wgt;
            c2 += c.z * wgt;
            T = Tn;
        }
    }
    if (COUNT) flush_counts(a.count, n_eval, n_blend);
    if (inside) {
        const size_t plane = (size_t)W * H, o = (size_t)py * W + px;
        a.out[o] = c0 + T * a.cam.bg[0];
        a.out[plane + o] = c1 + T * a.cam.bg[1];
        a.out[2 * plane + o] = c2 + T * a.cam.bg[2];
    }
}

void launch_raster_exact(const RasterArgs& a, cudaStream_t s)
{
    const unsigned tiles = (unsigned)(a.tiles_x * a.tiles_y);
    if (a.count) launch_dependent(k_raster_exact<true>, dim3(tiles), dim3(E_THREADS), 0, s, a);
    else launch_dependent(k_raster_exact<false>, dim3(tiles), dim3(E_THREADS), 0, s, a);
}

void launch_fast_exp_eval(const float* P, float* out, long long n, cudaStream_t s)
{
    if (n <= 0) return;
    k_fast_exp_eval<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P, out, n);
}

} // namespace rg
