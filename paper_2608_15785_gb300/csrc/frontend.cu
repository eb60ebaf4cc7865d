// frontend.cu -- front ends of the renderer and the scene conversion kernels.
//
//  * k_frontend_fused: the RoofGS fused preprocess + duplicate + key kernel
//    (Sec. IV-A.3): one thread per Gaussian (taken in quantized-depth order
//    when the Gaussians were sorted by depth first) projects, culls, decodes
//    INT8 SH (Eq. (8)) and FP16 geometry (Sec. IV-A.1), computes the snug box
//    and the 32-bit tile|quantized-depth key (Sec. IV-A.2, Eq. (9)); the warps
//    then walk the Gaussians' tile rows in parallel (lane k takes the k-th
//    row), keep per row only the tiles the ellipse reaches, and count entries;
//    the block allocates its entries with one shared-memory prefix sum and one
//    device-wide slot (decoupled look-back, ordered by block, so equal keys stay
//    in Gaussian order) and writes the (key or 16-bit tile id, value) array
//    cooperatively: consecutive lanes write consecutive entries (coalesced), whichever
//    Gaussian and row they belong to. Only the raster record and the key-value
//    array go to global memory, besides the digit counts of the entry sort
//    (each tile row is a run of consecutive tile ids; counted per block in
//    shared memory, added to one of a few global copies).
//  * k_frontend_count -> k_row_scan -> k_frontend_scatter: the row-bucketed front
//    end (the renderer's default where it applies): the fused kernel's work without
//    the allocation and emission, a per-tile-row prefix of the block counts, and a
//    scatter of each Gaussian's tile-row runs into their tile row's part of the entry
//    array under the column-major key tx << 8 | ty, so one 8-bit pass over the tile
//    column is left to the sort.
//  * k_depth_keys: quantized depth and index of every Gaussian, the input of
//    the per-Gaussian depth sort, and the digit counts of that sort.
//  * k_exact_*: the plain 3DGS front end (preprocess -> scan -> duplicate,
//    Sec. II-A), 64-bit keys of 32-bit tile id | 32-bit float depth.
//  * scene conversion: finite-value check, per-(degree, channel) max |SH|,
//    and the compact attribute encoder.
#include "rg_internal.cuh"

namespace rg {

__device__ __forceinline__ float h_lo(unsigned w) { return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu))); }
__device__ __forceinline__ float h_hi(unsigned w) { return __half2float(__ushort_as_half((unsigned short)(w >> 16))); }

// signed INT8 code j (0..47) of a 48-byte code block held in 12 words
__device__ __forceinline__ float sh_code(const unsigned (&w)[12], int j)
{
    return (float)(((int)(w[j >> 2] << (24 - 8 * (j & 3)))) >> 24);
}

__device__ __forceinline__ int sh_band(int k) { return k == 0 ? 0 : (k < 4 ? 1 : (k < 9 ? 2 : 3)); }

// two FP32 values rounded to FP16 (round to nearest even), packed low | high << 16
__device__ __forceinline__ unsigned pack_h2(float lo, float hi)
{
    return (unsigned)__half_as_ushort(__float2half_rn(lo)) | ((unsigned)__half_as_ushort(__float2half_rn(hi)) << 16);
}

// ---------------------------------------------------------------------------
// Fused front end (RoofGS)
// ---------------------------------------------------------------------------
#ifndef RG_FE_THREADS
#define RG_FE_THREADS 256
#endif
constexpr int FE_THREADS = RG_FE_THREADS;
constexpr int FE_WARPS = FE_THREADS / 32;
constexpr int RADIX_FE = 256;

// Adds the digits of the w consecutive tiles t0 .. t0 + w - 1 to the block's
// digit counts: pass 0 digit t & 255 (difference array: +1 where a run of digits
// starts, -1 after it ends, full cycles of 256 added to every digit via entry 0),
// pass 1 digit t >> 8 (t < 2^16).
__device__ __forceinline__ void count_tile_digits(unsigned* s_d0, unsigned* s_h1, int passes, unsigned t0, unsigned w)
{
    const unsigned full = w >> 8, r = w & 255u;
    if (full) atomicAdd(&s_d0[0], full);
    if (r) {
        const unsigned d = t0 & 255u, e = d + r;
        atomicAdd(&s_d0[d], 1u);
        if (e < 256u) {
            atomicSub(&s_d0[e], 1u);
        } else if (e > 256u) { // the run wraps past digit 255
            atomicAdd(&s_d0[0], 1u);
            atomicSub(&s_d0[e - 256u], 1u);
        }
    }
    if (passes > 1) {
        const unsigned t1 = t0 + w - 1u, h0 = t0 >> 8, h1 = t1 >> 8;
        if (h0 == h1) {
            atomicAdd(&s_h1[h0], w);
        } else {
            atomicAdd(&s_h1[h0], ((h0 + 1u) << 8) - t0);
            for (unsigned h = h0 + 1u; h < h1; h++) atomicAdd(&s_h1[h], 256u);
            atomicAdd(&s_h1[h1], t1 - (h1 << 8) + 1u);
        }
    }
}

__device__ __forceinline__ unsigned warp_inclusive_scan(unsigned x, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// One block of the fused front end: virtual block vb (blocks of a view are numbered in
// the order they claimed work, so every predecessor of the ordered allocation is
// running or done) of the view described by a.
// ROWS: the count kernel of the row-bucketed front end instead (launch_frontend_rows):
// the same per-Gaussian work and entry counts, but no allocation and no emission; the
// block stores each slot's row test, its entries per tile row and the column digits.
template <bool ROWS>
__device__ __forceinline__ void frontend_block(const FrontendArgs& a, const unsigned vb)
{
    __shared__ unsigned s_wsum[FE_WARPS];
    __shared__ RowTestS s_rt[FE_THREADS];   // per-row test of each thread's Gaussian
    __shared__ unsigned s_q[FE_THREADS];    // quantized depth, Eq. (9)
    __shared__ unsigned s_id[FE_THREADS];   // Gaussian index of each slot
    __shared__ unsigned s_cnt[FE_THREADS];  // entries of each slot's Gaussian
    __shared__ unsigned long long s_base;
    // digit counts of the block's entries for the entry sort (8-bit digits of the
    // tile id): pass 0 as a difference array over the digits (tile rows are runs of
    // consecutive tiles), pass 1 as plain counts. ROWS: s_d0 over the tile columns,
    // s_h1 the entries of each tile row.
    __shared__ unsigned s_d0[RADIX_FE + 1], s_h1[RADIX_FE];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (a.hist_passes)
        for (int j = tid; j < 2 * RADIX_FE + 1; j += FE_THREADS) (j <= RADIX_FE ? s_d0[j] : s_h1[j - RADIX_FE - 1]) = 0u;
    __syncthreads();
    const long long slot = (long long)vb * FE_THREADS + tid;
    // Gaussian of this slot: slots follow depth order when an order is given, so
    // the entries come out sorted by depth and only the tile bits remain to sort
    const long long i = slot < a.n ? (a.order ? (long long)a.order[slot] : slot) : a.n;

    bool front = false;
    RowTest rt;
    rt.ty0 = 0;
    rt.ty1 = -1; // no rows unless the box is non-empty
    unsigned qd = 0;
    if (i < a.n) {
        const float4 ga = __ldg(&a.geoA[i]); // mean, log o
        const float pz = view_z(a.cam, ga.x, ga.y, ga.z);
        // depth interval (Sec. IV-A.2) and opacity culling o >= 1/255
        front = pz > a.cam.zn && pz <= a.cam.zf && ga.w >= -LN255F;
        if (front) {
            const uint4 gb = __ldg(&a.geoB[i]);
            Binned b;
            if (project_bin(a.cam, ga.x, ga.y, ga.z, pz, h_lo(gb.x), h_hi(gb.x), h_lo(gb.y), h_hi(gb.y), h_lo(gb.z),
                            h_hi(gb.z), h_lo(gb.w), true, ga.w, b)) {
                rt = row_test(b);
                if constexpr (ROWS) { // the row test for the scatter kernel, stored before the SH work
                    s_rt[tid] = shared_row_test(rt);
                    if (rt.ty1 >= rt.ty0) { // three coalesced planes
                        a.row_rt[slot] = make_float4(rt.u, rt.v, rt.tt, rt.isc);
                        a.row_rt[a.n + slot] = make_float4(rt.ys, rt.cc, rt.kk, rt.xl);
                        a.row_rt[2 * a.n + slot] = make_float4(rt.xh, rt.yl, rt.yh, __int_as_float(rt.ty0));
                    }
                }
                qd = quantize_depth(pz, a.cam.zn, a.lay);
                // conic in the paper's (a, b, c) of Eq. (10): b multiplies dx*dy
                const float inv = 1.0f / b.det;
                const float ca = b.sc * inv, cb = -2.0f * b.sb * inv, cc = b.sa * inv;
                // INT8 SH (Eq. (8)) decoded in registers, evaluated per band
                unsigned w[12];
                {
                    const uint4 p0 = __ldg(&a.shq[3 * i]); // one 48-byte block per Gaussian
                    const uint4 p1 = __ldg(&a.shq[3 * i + 1]);
                    const uint4 p2 = __ldg(&a.shq[3 * i + 2]);
                    w[0] = p0.x; w[1] = p0.y; w[2] = p0.z; w[3] = p0.w;
                    w[4] = p1.x; w[5] = p1.y; w[6] = p1.z; w[7] = p1.w;
                    w[8] = p2.x; w[9] = p2.y; w[10] = p2.z; w[11] = p2.w;
                }
                float dx, dy, dz;
                view_dir(a.cam, ga.x, ga.y, ga.z, dx, dy, dz);
                float Y[16];
                sh_basis(dx, dy, dz, Y);
                float acc[4][3];
#pragma unroll
                for (int d = 0; d < 4; d++) acc[d][0] = acc[d][1] = acc[d][2] = 0.0f;
#pragma unroll
                for (int k = 0; k < 16; k++)
#pragma unroll
                    for (int ch = 0; ch < 3; ch++)
                        acc[sh_band(k)][ch] = fmaf(Y[k], sh_code(w, 3 * k + ch), acc[sh_band(k)][ch]);
                const float g = a.per_gauss_scale ? h_hi(gb.w) : 1.0f;
                float rgb[3];
#pragma unroll
                for (int ch = 0; ch < 3; ch++) {
                    float sum = a.band_scale[ch] * acc[0][ch];
                    sum = fmaf(a.band_scale[3 + ch], acc[1][ch], sum);
                    sum = fmaf(a.band_scale[6 + ch], acc[2][ch], sum);
                    sum = fmaf(a.band_scale[9 + ch], acc[3][ch], sum);
                    rgb[ch] = clamp01(fmaf(g, sum, 0.5f));
                }
                a.rec[2 * i] = make_float4(b.u, b.v, ca, cb);
                a.rec[2 * i + 1] = make_float4(cc, ga.w, __uint_as_float(pack_h2(rgb[0], rgb[1])),
                                               __uint_as_float(pack_h2(rgb[2], 0.0f)));
            }
        }
    }
    if constexpr (!ROWS) s_rt[tid] = shared_row_test(rt); // (ROWS: stored above; read only for rows > 0)
    s_q[tid] = qd;
    s_id[tid] = (unsigned)i;
    if (ROWS && slot < a.n) a.row_n[slot] = rt.ty1 >= rt.ty0 ? (unsigned)(rt.ty1 - rt.ty0 + 1) : 0u;
    __syncwarp();

    // Entries per Gaussian. The warp's Gaussians have rows_l tile rows each; the
    // warp walks all of its rows 32 at a time (lane k takes the k-th row of the
    // chunk, whichever Gaussian it belongs to) and adds each row's width to its
    // Gaussian's count with a shared-memory atomic (measured faster than a
    // segmented warp reduction: a chunk's rows belong to few Gaussians).
    const int rows_l = rt.ty1 - rt.ty0 + 1 > 0 ? rt.ty1 - rt.ty0 + 1 : 0;
    const unsigned rincl = warp_inclusive_scan((unsigned)rows_l, lane);
    const unsigned rexcl = rincl - (unsigned)rows_l;
    const unsigned wrows = __shfl_sync(0xffffffffu, rincl, 31);
    s_cnt[tid] = 0u;
    __syncwarp();
    for (unsigned r0 = 0; r0 < wrows; r0 += 32) {
        const unsigned k = r0 + (unsigned)lane;
        int owner = 0; // Gaussian (lane) of warp row k
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
            if (__shfl_sync(0xffffffffu, rincl, owner + step - 1) <= k) owner += step;
        const unsigned rl = k - __shfl_sync(0xffffffffu, rexcl, owner);
        unsigned w = 0;
        int txa, txb;
        const int ty = k < wrows ? s_rt[warp * 32 + owner].ty0 + (int)rl : 0;
        if (k < wrows && row_range(s_rt[warp * 32 + owner], ty, a.cam.tw_log2, a.cam.th, txa, txb))
            w = (unsigned)(txb - txa + 1);
        if (w) {
            atomicAdd(&s_cnt[warp * 32 + owner], w);
            if (ROWS) { // tile row ty (the scatter's digit) and columns txa .. txb (the sort's)
                atomicAdd(&s_h1[ty], w);
                count_tile_digits(s_d0, s_h1, 1, (unsigned)txa, w);
            } else if (a.hist_passes) {
                count_tile_digits(s_d0, s_h1, a.hist_passes, (unsigned)ty * (unsigned)a.lay.tiles_x + (unsigned)txa, w);
            }
        }
    }
    __syncwarp();
    const unsigned cnt = s_cnt[tid];
    if constexpr (ROWS) {
        const int nfront = __syncthreads_count(front);
        const int nvis = __syncthreads_count(cnt > 0); // the block's counts are complete after it
        const unsigned nbl = (unsigned)((a.n + FE_THREADS - 1) / FE_THREADS);
        if (tid < a.rows) a.row_cnt[(size_t)tid * nbl + vb] = s_h1[tid];
        if (tid == 0) {
            if (nvis) atomicAdd(&a.ctr->n_visible, (unsigned)nvis);
            if (nfront) atomicAdd(&a.ctr->n_front, (unsigned)nfront);
        }
    } else {
        // block-level prefix sum of the entry counts
        const unsigned x = warp_inclusive_scan(cnt, lane);
        if (lane == 31) s_wsum[warp] = x;
        const int nfront = __syncthreads_count(front);
        const int nvis = __syncthreads_count(cnt > 0);
        if (warp == 0) {
            unsigned ws = lane < FE_WARPS ? s_wsum[lane] : 0u;
            ws = warp_inclusive_scan(ws, lane);
            if (lane < FE_WARPS) s_wsum[lane] = ws; // inclusive warp totals
        }
        __syncthreads();
        const unsigned block_total = s_wsum[FE_WARPS - 1];

        // one device-wide allocation per block, ordered by block
        if (warp == 0) {
            const unsigned long long base =
                lookback_exclusive(a.status, vb, (unsigned long long)block_total, a.ctr, a.sticky, ERR_FE_LOOKBACK);
            if (lane == 0) {
                s_base = base;
                if (nvis) atomicAdd(&a.ctr->n_visible, (unsigned)nvis);
                if (nfront) atomicAdd(&a.ctr->n_front, (unsigned)nfront);
                const unsigned nblocks = (unsigned)((a.n + FE_THREADS - 1) / FE_THREADS);
                if (vb == nblocks - 1) {
                    const unsigned long long total = base + block_total;
                    a.ctr->n_entries_total = total;
                    a.ctr->n_entries = (unsigned)(total < (unsigned long long)a.cap ? total : (unsigned long long)a.cap);
                }
                if (base + block_total > (unsigned long long)a.cap) {
                    atomicOr(&a.ctr->overflow, 1u);
                    atomicOr(&a.sticky->overflow, 1u);
                }
            }
        }
        __syncthreads();
        const unsigned long long base = s_base;

        // Emission: the warp's entries are contiguous and in (Gaussian, row, tile)
        // order, so the warp walks its rows again 32 at a time, scans the row
        // widths, and writes 32 consecutive entries per store instruction (lane e
        // finds the row of its entry with a 5-step search over the scan and takes
        // the row's first tile, depth and Gaussian from that lane).
        const int b_d = a.lay.b_d;
        const unsigned tiles_x = (unsigned)a.lay.tiles_x;
        unsigned long long out = base + (warp ? s_wsum[warp - 1] : 0u); // the warp's first entry
        for (unsigned r0 = 0; r0 < wrows; r0 += 32) {
            const unsigned k = r0 + (unsigned)lane;
            int owner = 0;
    #pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (__shfl_sync(0xffffffffu, rincl, owner + step - 1) <= k) owner += step;
            const unsigned rl = k - __shfl_sync(0xffffffffu, rexcl, owner);
            unsigned w = 0, tb = 0, q = 0, id = 0;
            if (k < wrows) {
                const RowTestS& G = s_rt[warp * 32 + owner];
                const int ty = G.ty0 + (int)rl;
                int txa, txb;
                if (row_range(G, ty, a.cam.tw_log2, a.cam.th, txa, txb)) {
                    w = (unsigned)(txb - txa + 1);
                    tb = (unsigned)ty * tiles_x + (unsigned)txa; // tile of the row's first entry
                }
                q = s_q[warp * 32 + owner];
                id = s_id[warp * 32 + owner];
            }
            const unsigned incl = warp_inclusive_scan(w, lane);
            const unsigned chunk = __shfl_sync(0xffffffffu, incl, 31);
            tb -= incl - w; // entry e of the chunk, if in this row, has tile tb + e (mod 2^32)
            // entries at or past the capacity are counted but not written
            const bool fits = out < (unsigned long long)a.cap;
            const unsigned room = fits ? (unsigned)((unsigned long long)a.cap - out) : 0u;
            const unsigned long long o = fits ? out : 0ull;
            unsigned* const kp = a.keys + o;
            unsigned short* const kp16 = a.keys16 ? a.keys16 + o : nullptr;
            unsigned* const vp = a.vals + o;
            for (unsigned e0 = 0; e0 < chunk; e0 += 32) {
                const unsigned e = e0 + (unsigned)lane;
                int pos = 0; // row (lane) of entry e
    #pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                    if (__shfl_sync(0xffffffffu, incl, pos + step - 1) <= e) pos += step;
                const unsigned tile = __shfl_sync(0xffffffffu, tb, pos) + e;
                const unsigned qe = __shfl_sync(0xffffffffu, q, pos);
                const unsigned ide = __shfl_sync(0xffffffffu, id, pos);
                if (e < chunk && e < room) {
                    if (a.keys16) kp16[e] = (unsigned short)tile;
                    else kp[e] = (b_d >= 32) ? qe : ((tile << b_d) | qe);
                    vp[e] = ide;
                }
            }
            out += chunk;
        }
    }

    // The block's digit counts (complete since the barriers after the count
    // loop) go to one copy of the frame's histograms: the last warp turns the
    // difference array into counts, 8 digits per lane.
    if (a.hist_passes && warp == FE_WARPS - 1) {
        unsigned* const H = a.hist + (size_t)(vb % FE_HIST_COPIES) * (2 * RADIX_FE);
        unsigned c[8], run = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            run += s_d0[8 * lane + j];
            c[j] = run;
        }
        const unsigned incl = warp_inclusive_scan(run, lane);
        const unsigned before = incl - run;
#pragma unroll
        for (int j = 0; j < 8; j++)
            if (c[j] + before) atomicAdd(&H[8 * lane + j], c[j] + before);
        if (a.hist_passes > 1) {
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const unsigned v = s_h1[8 * lane + j];
                if (v) atomicAdd(&H[RADIX_FE + 8 * lane + j], v);
            }
        }
    }
}

// Full occupancy (64 warps per SM, 32 registers): the kernel is latency-bound on
// its depth-ordered gathers and shuffles, and 8 blocks of 256 threads per SM
// measured 0.41 ms at 4K against 0.52 ms at 4 blocks per SM (61 registers)
__global__ void __launch_bounds__(FE_THREADS, 2048 / FE_THREADS) k_frontend_fused(FrontendArgs a)
{
    __shared__ unsigned s_vb;
    grid_dependency_wait();
    if (threadIdx.x == 0) s_vb = atomicAdd(&a.ctr->fe_block_ctr, 1u);
    __syncthreads();
    frontend_block<false>(a, s_vb);
}

// Every view of a batch in one grid: a block claims the next of all views' blocks
// (views in order, each view's blocks in order) and runs it with that view's
// arguments, read from the kernel's parameter space.
__global__ void __launch_bounds__(FE_THREADS, 2048 / FE_THREADS)
    k_frontend_views(const __grid_constant__ FrontendViews m)
{
    __shared__ unsigned s_g;
    grid_dependency_wait();
    if (threadIdx.x == 0) s_g = atomicAdd(m.claim, 1u);
    __syncthreads();
    const unsigned g = s_g;
    int v = 0;
    while (v + 1 < m.n_views && m.block_prefix[v + 1] <= g) v++;
    frontend_block<false>(m.views[v], g - m.block_prefix[v]);
}

void launch_frontend_views(const FrontendViews& m, cudaStream_t s)
{
    const unsigned blocks = m.block_prefix[m.n_views];
    if (blocks == 0) return;
    launch_dependent(k_frontend_views, dim3(blocks), dim3(FE_THREADS), 0, s, m);
}

// Grid-stride over the Gaussians; each block also counts the 8-bit digits of its
// keys for the depth sort's passes in shared memory and adds them to `hist`
// ([passes][256], zeroed beforehand) once at the end.
__global__ void __launch_bounds__(256) k_depth_keys(FrontendArgs a, unsigned* keys, unsigned* vals, Counters* ctr,
                                                    unsigned* hist, int passes, unsigned* status0,
                                                    long long status_words)
{
    __shared__ unsigned s_h[4][256];
    grid_dependency_wait();
    for (int j = threadIdx.x; j < 4 * 256; j += 256) (&s_h[0][0])[j] = 0u;
    // the look-back status of the depth sort's first pass (no histogram kernel runs before it)
    for (long long j = (long long)blockIdx.x * 256 + threadIdx.x; j < status_words; j += (long long)gridDim.x * 256)
        status0[j] = 0u;
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr->n_entries = (unsigned)a.n;
    for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < a.n; i += (long long)gridDim.x * 256) {
        const float4 ga = __ldg(&a.geoA[i]);
        const float pz = view_z(a.cam, ga.x, ga.y, ga.z);
        const bool front = pz > a.cam.zn && pz <= a.cam.zf && ga.w >= -LN255F;
        const unsigned q = front ? quantize_depth(pz, a.cam.zn, a.lay) : a.lay.qmax;
        keys[i] = q;
        vals[i] = (unsigned)i;
        for (int p = 0; p < passes; p++) atomicAdd(&s_h[p][(q >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < passes * 256; j += 256) {
        const unsigned c = (&s_h[0][0])[j];
        if (c) atomicAdd(&hist[j], c);
    }
}

void launch_depth_keys(const FrontendArgs& a, unsigned* keys, unsigned* vals, Counters* ctr, unsigned* hist,
                       int passes, unsigned* status0, cudaStream_t s)
{
    const int grid_cap = 8 * device_sm_count();
    const long long need = (a.n + 255) / 256;
    const unsigned blocks = (unsigned)(need < 1 ? 1 : (need < grid_cap ? need : grid_cap));
    launch_dependent(k_depth_keys, dim3(blocks), dim3(256), 0, s, a, keys, vals, ctr, hist, passes, status0,
                     sort_status_words(4, a.n));
}

int frontend_block_threads() { return FE_THREADS; }

void launch_frontend_fused(const FrontendArgs& a, cudaStream_t s)
{
    if (a.n <= 0) return;
    const unsigned blocks = (unsigned)((a.n + FE_THREADS - 1) / FE_THREADS);
    launch_dependent(k_frontend_fused, dim3(blocks), dim3(FE_THREADS), 0, s, a);
}

// ---------------------------------------------------------------------------
// Row-bucketed front end (RoofGS, at most 256 x 256 tiles)
// ---------------------------------------------------------------------------
// The fused kernel hands each block one contiguous run of entries (the ordered
// allocation) and leaves two 8-bit passes over the tile id to the sort. Here the entries
// carry the column-major key tx << 8 | ty and the front end itself places them by tile
// row: one tile row of one Gaussian is a run of entries that share ty, so ranking a
// block's entries by tile row takes one count per run, not one per entry.
//  * k_frontend_count: the fused kernel's per-Gaussian work and entry counts (records,
//    row tests, entries per tile row per block, the column digits); no emission;
//  * k_row_scan: per tile row, the exclusive prefix of the block counts over the blocks
//    and the row's total;
//  * k_frontend_scatter: the block's runs in (slot, row) order, 256 at a time; a run's
//    first slot = its tile row's start + the earlier blocks' entries of that row + the
//    block's earlier runs of that row; the entries go out 32 per store as in the fused
//    kernel.
// The entries come out grouped by tile row, in slot (depth) order within a row, so one
// stable 8-bit pass over the column leaves each tile's entries contiguous and in the order
// of the 32-bit key of Sec. IV-A.2.
constexpr unsigned ROW_PREFIX_SAT = 0x7fffffffu; // above any entry capacity (below 2^30)

// resident count kernels per SM: 6 (40 registers, 24 bytes of spill) measured faster than the fused
// kernel's 8 (32 registers, 88 bytes of spill): 4K front end 0.671 -> 0.630 ms
#ifndef RG_FEC_MIN_BLOCKS
#define RG_FEC_MIN_BLOCKS 6
#endif

__global__ void __launch_bounds__(FE_THREADS, RG_FEC_MIN_BLOCKS) k_frontend_count(FrontendArgs a)
{
    grid_dependency_wait();
    frontend_block<true>(a, blockIdx.x);
}

// one block of 1024 threads per tile row: the exclusive prefix of the row's block counts
// over the blocks (in place) and the row's total
__global__ void __launch_bounds__(1024) k_row_scan(FrontendArgs a)
{
    __shared__ unsigned long long s_w[32];
    grid_dependency_wait();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned nbl = (unsigned)((a.n + FE_THREADS - 1) / FE_THREADS);
    unsigned* const col = a.row_cnt + (size_t)blockIdx.x * nbl;
    const unsigned per = (nbl + 1023u) / 1024u;
    const unsigned b0 = (unsigned)tid * per;
    unsigned long long sum = 0;
#pragma unroll 4
    for (unsigned k = 0; k < per; k++)
        if (b0 + k < nbl) sum += col[b0 + k];
    unsigned long long x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long v = s_w[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        s_w[lane] = v;
    }
    __syncthreads();
    unsigned long long run = x - sum + (warp ? s_w[warp - 1] : 0ull);
#pragma unroll 4
    for (unsigned k = 0; k < per; k++) {
        const unsigned b = b0 + k;
        if (b >= nbl) break;
        const unsigned c = col[b];
        col[b] = run < ROW_PREFIX_SAT ? (unsigned)run : ROW_PREFIX_SAT;
        run += c;
    }
    if (tid == 1023) a.row_tot[blockIdx.x] = s_w[31];
}

// inclusive scan of one value per thread over a block of FE_THREADS threads (every thread
// calls it); s_w holds FE_WARPS words; total = the block's sum
template <typename T>
__device__ __forceinline__ T fe_block_inclusive_scan(T v, T* s_w, T& total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    T before = 0, all = 0;
#pragma unroll
    for (int q = 0; q < FE_WARPS; q++) {
        const T t = s_w[q];
        if (q < warp) before += t;
        all += t;
    }
    total = all;
    __syncthreads(); // s_w may be written again after the call
    return x + before;
}

__global__ void __launch_bounds__(FE_THREADS, 6) k_frontend_scatter(FrontendArgs a)
{
    __shared__ RowTestS s_rt[FE_THREADS];         // row test of each slot's Gaussian
    __shared__ unsigned s_incl[FE_THREADS];       // inclusive prefix of the slots' tile rows
    __shared__ unsigned s_id[FE_THREADS];         // Gaussian of each slot
    __shared__ unsigned s_run[RADIX_FE];          // next entry slot of each tile row
    __shared__ unsigned s_wt[FE_WARPS][RADIX_FE]; // this round: each warp's entries per tile row
    __shared__ unsigned s_wp[FE_WARPS][RADIX_FE]; // this round: each warp's first slot per tile row
    __shared__ unsigned s_w[FE_WARPS][32];        // widths of a warp's runs
    __shared__ unsigned s_sc[FE_WARPS];
    __shared__ unsigned long long s_sc64[FE_WARPS];
    grid_dependency_wait();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned vb = blockIdx.x;
    const unsigned nbl = (unsigned)((a.n + FE_THREADS - 1) / FE_THREADS);
    const unsigned long long cap = (unsigned long long)a.cap;
    const long long slot = (long long)vb * FE_THREADS + tid;
    unsigned nr = 0;
    if (slot < a.n) {
        nr = a.row_n[slot];
        if (nr) {
            const float4 r0 = a.row_rt[slot], r1 = a.row_rt[a.n + slot], r2 = a.row_rt[2 * a.n + slot];
            s_rt[tid] = RowTestS{r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w, r2.x, r2.y, r2.z, __float_as_int(r2.w)};
            s_id[tid] = a.order ? a.order[slot] : (unsigned)slot;
        }
    }
    for (int j = tid; j < FE_WARPS * RADIX_FE; j += FE_THREADS) (&s_wt[0][0])[j] = 0u;
    unsigned R; // the block's tile rows (runs, some possibly empty)
    s_incl[tid] = fe_block_inclusive_scan(nr, s_sc, R);
    // first slot of each tile row's entries in this block: the earlier tile rows' entries
    // (clamped at the capacity: slots past it are not written), then the earlier blocks'
    // entries of the row; below 2^30 + 2^31 and raised by at most 2^16 per block
    const unsigned long long tot = tid < a.rows ? a.row_tot[tid] : 0ull;
    unsigned long long all;
    const unsigned long long tincl = fe_block_inclusive_scan(tot, s_sc64, all);
    if (tid < a.rows) {
        const unsigned long long start = tincl - tot;
        s_run[tid] = (unsigned)(start < cap ? start : cap) + a.row_cnt[(size_t)tid * nbl + vb];
    }
    if (vb == 0 && tid == 0) {
        a.ctr->n_entries_total = all;
        a.ctr->n_entries = (unsigned)(all < cap ? all : cap);
        if (all > cap) {
            atomicOr(&a.ctr->overflow, 1u);
            atomicOr(&a.sticky->overflow, 1u);
        }
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (unsigned r0 = 0; r0 < R; r0 += FE_THREADS) {
        // run k of the block: slot s (the first with s_incl[s] > k), tile row ty
        const unsigned k = r0 + (unsigned)tid;
        unsigned w = 0, d = 0, ta = 0, id = 0;
        if (k < R) {
            int s = 0;
#pragma unroll
            for (int step = FE_THREADS / 2; step > 0; step >>= 1)
                if (s_incl[s + step - 1] <= k) s += step;
            const RowTestS& G = s_rt[s];
            const int ty = G.ty0 + (int)(k - (s ? s_incl[s - 1] : 0u));
            int txa, txb;
            if (row_range(G, ty, a.cam.tw_log2, a.cam.th, txa, txb)) {
                w = (unsigned)(txb - txa + 1);
                d = (unsigned)ty;
                ta = (unsigned)txa;
                id = s_id[s];
            }
        }
        // entries before the run among the warp's runs of the same tile row (lane order)
        const unsigned peers = __match_any_sync(0xffffffffu, w ? d : 0x100u + (unsigned)lane);
        s_w[warp][lane] = w;
        __syncwarp();
        unsigned pre = 0;
        if (w)
            for (unsigned m = peers & lt; m; m &= m - 1u) pre += s_w[warp][__ffs(m) - 1];
        if (w && (peers >> lane) == 1u) s_wt[warp][d] = pre + w; // the group's last lane: its total
        __syncthreads();
        // per tile row: each warp's first slot this round, in warp order
        if (tid < a.rows) {
            unsigned run = s_run[tid];
#pragma unroll
            for (int q = 0; q < FE_WARPS; q++) {
                const unsigned c = s_wt[q][tid];
                s_wp[q][tid] = run;
                s_wt[q][tid] = 0u;
                run += c;
            }
            s_run[tid] = run;
        }
        __syncthreads();
        // the warp's entries, 32 per store: entry e of the warp's runs, in run r, goes to
        // slot dbase(r) + e with key kbase(r) + (e << 8) (low 16 bits)
        const unsigned incl = warp_inclusive_scan(w, lane);
        const unsigned chunk = __shfl_sync(0xffffffffu, incl, 31);
        const unsigned excl = incl - w;
        const unsigned dbase = (w ? s_wp[warp][d] + pre : 0u) - excl;
        const unsigned kbase = ((ta - excl) << 8) + d;
        for (unsigned e0 = 0; e0 < chunk; e0 += 32) {
            const unsigned e = e0 + (unsigned)lane;
            int pos = 0; // run (lane) of entry e
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (__shfl_sync(0xffffffffu, incl, pos + step - 1) <= e) pos += step;
            const unsigned dst = __shfl_sync(0xffffffffu, dbase, pos) + e;
            const unsigned key = __shfl_sync(0xffffffffu, kbase, pos) + (e << 8);
            const unsigned ide = __shfl_sync(0xffffffffu, id, pos);
            if (e < chunk && dst < cap) {
                a.keys16[dst] = (unsigned short)key;
                a.vals[dst] = ide;
            }
        }
    }
}

void launch_frontend_rows(const FrontendArgs& a, cudaStream_t s)
{
    if (a.n <= 0 || a.rows <= 0) return;
    const unsigned blocks = (unsigned)((a.n + FE_THREADS - 1) / FE_THREADS);
    launch_dependent(k_frontend_count, dim3(blocks), dim3(FE_THREADS), 0, s, a);
    launch_dependent(k_row_scan, dim3(a.rows), dim3(1024), 0, s, a);
    launch_dependent(k_frontend_scatter, dim3(blocks), dim3(FE_THREADS), 0, s, a);
}

// ---------------------------------------------------------------------------
// Plain 3DGS front end (exact mode)
// ---------------------------------------------------------------------------
constexpr int EX_THREADS = 256;

__global__ void __launch_bounds__(EX_THREADS) k_exact_preprocess(ExactArgs a)
{
    grid_dependency_wait();
    const long long i = (long long)blockIdx.x * EX_THREADS + threadIdx.x;
    if (i >= a.n) return;
    a.touched[i] = 0;
    const float mx = a.means[3 * i], my = a.means[3 * i + 1], mz = a.means[3 * i + 2];
    const float pz = view_z(a.cam, mx, my, mz);
    const bool front = pz > a.cam.zn && pz <= a.cam.zf;
    const unsigned fm = __ballot_sync(__activemask(), front);
    if (front && __popc(fm & ((1u << (threadIdx.x & 31)) - 1u)) == 0) atomicAdd(&a.ctr->n_front, (unsigned)__popc(fm));
    if (!front) return;
    const float4 q = *reinterpret_cast<const float4*>(&a.quats[4 * i]);
    Binned b;
    const bool vis = project_bin(a.cam, mx, my, mz, pz, q.x, q.y, q.z, q.w, a.scales[3 * i], a.scales[3 * i + 1],
                                 a.scales[3 * i + 2], false, 0.0f, b);
    const unsigned vm = __ballot_sync(__activemask(), vis);
    if (vis && __popc(vm & ((1u << (threadIdx.x & 31)) - 1u)) == 0) atomicAdd(&a.ctr->n_visible, (unsigned)__popc(vm));
    if (!vis) return;
    // the rasterizer's exponent (Eq. (10)) with the quadratic form completed in dx:
    // -1/2 ((Sigma'_yy / det) (dx - c dy)^2 + dy^2 / Sigma'_yy), c = Sigma'_xy / Sigma'_yy
    // (no cancellation for thin Gaussians); the mean as double-floats (the FP32 u, v
    // above only bin the Gaussian)
    a.quad[i] = make_float4(-0.5f * __fdiv_rn(b.sc, b.det), __fdiv_rn(b.sb, b.sc), __fdiv_rn(-0.5f, b.sc), a.opac[i]);
    a.mean2[i] = project_mean_df(a.cam, mx, my, mz);
    a.depth[i] = pz;
    a.rect[i] = make_int4(b.tx0, b.ty0, b.tx1, b.ty1);
    a.touched[i] = (unsigned)((b.tx1 - b.tx0 + 1) * (b.ty1 - b.ty0 + 1));
    // degree-3 SH colour from FP32 coefficients
    float dx, dy, dz;
    view_dir(a.cam, mx, my, mz, dx, dy, dz);
    float Y[16];
    sh_basis(dx, dy, dz, Y);
    const int nk = (a.sh_degree + 1) * (a.sh_degree + 1);
    const float4* shp = reinterpret_cast<const float4*>(a.sh + 48 * i);
    float c[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
    for (int v4 = 0; v4 < 12; v4++) {
        const float4 f = shp[v4];
        const float e[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int j = 4 * v4 + u;
            const int k = j / 3, ch = j % 3;
            if (k < nk) c[ch] = fmaf(Y[k], e[u], c[ch]);
        }
    }
    a.rgb[3 * i] = clamp01(c[0]);
    a.rgb[3 * i + 1] = clamp01(c[1]);
    a.rgb[3 * i + 2] = clamp01(c[2]);
}

constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = EX_THREADS * SCAN_ITEMS;

// Exclusive scan of the tile counts (single pass, decoupled look-back).
__global__ void __launch_bounds__(EX_THREADS) k_exact_scan(ExactArgs a)
{
    __shared__ unsigned s_vb;
    __shared__ unsigned long long s_wsum[EX_THREADS / 32];
    grid_dependency_wait();
    __shared__ unsigned long long s_base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_vb = atomicAdd(&a.ctr->fe_block_ctr, 1u);
    __syncthreads();
    const unsigned vb = s_vb;
    const long long start = (long long)vb * SCAN_TILE + (long long)tid * SCAN_ITEMS;
    unsigned v[SCAN_ITEMS];
    unsigned long long sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        v[k] = (start + k < a.n) ? a.touched[start + k] : 0u;
        sum += v[k];
    }
    unsigned long long x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long ws = lane < EX_THREADS / 32 ? s_wsum[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, ws, o);
            if (lane >= o) ws += y;
        }
        if (lane < EX_THREADS / 32) s_wsum[lane] = ws;
    }
    __syncthreads();
    const unsigned long long block_total = s_wsum[EX_THREADS / 32 - 1];
    if (warp == 0) {
        const unsigned long long base = lookback_exclusive(a.status, vb, block_total, a.ctr, a.sticky, ERR_SCAN_LOOKBACK);
        if (lane == 0) {
            s_base = base;
            const unsigned nblocks = (unsigned)((a.n + SCAN_TILE - 1) / SCAN_TILE);
            if (vb == nblocks - 1) {
                const unsigned long long total = base + block_total;
                a.ctr->n_entries_total = total;
                a.ctr->n_entries = (unsigned)(total < (unsigned long long)a.cap ? total : (unsigned long long)a.cap);
                if (total > (unsigned long long)a.cap) {
                    atomicOr(&a.ctr->overflow, 1u);
                    atomicOr(&a.sticky->overflow, 1u);
                }
            }
        }
    }
    __syncthreads();
    unsigned long long run = s_base + (x - sum) + (warp ? s_wsum[warp - 1] : 0ull);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        if (start + k < a.n) a.offsets[start + k] = (unsigned)(run > 0xffffffffull ? 0xffffffffull : run);
        run += v[k];
    }
}

// Duplicate (plain 3DGS, Sec. II-A): one (64-bit key, value) entry per tile of each
// Gaussian's rectangle, at the Gaussian's exclusive-scan offset. The entries of a
// warp's 32 consecutive Gaussians are contiguous and in (Gaussian, row, tile) order,
// so the warp walks their tile rows 32 at a time (lane k takes the k-th row) and
// writes 32 consecutive entries per store instruction, as the fused front end does.
// It also counts the sort's digits: the four depth digits are the same for every
// entry of a Gaussian (one shared atomic each per Gaussian), the tile digits of a
// row are a run of consecutive tile ids (count_tile_digits); the block's counts go
// to one of FE_HIST_COPIES copies once, at the end of its grid-stride loop.
constexpr int DUP_HIST_STRIDE = 8; // passes per copy of the digit counts ([copy][8][256])

__global__ void __launch_bounds__(EX_THREADS) k_exact_duplicate(ExactArgs a)
{
    __shared__ unsigned s_hd[4][RADIX_FE];             // depth digits (key bits 0..31)
    __shared__ unsigned s_d0[RADIX_FE + 1], s_h1[RADIX_FE]; // tile digits (key bits 32..47)
    grid_dependency_wait();
    const int tid = threadIdx.x, lane = tid & 31;
    const bool count = a.hist != nullptr;
    if (count) {
        for (int j = tid; j < 4 * RADIX_FE; j += EX_THREADS) (&s_hd[0][0])[j] = 0u;
        for (int j = tid; j < 2 * RADIX_FE + 1; j += EX_THREADS) (j <= RADIX_FE ? s_d0[j] : s_h1[j - RADIX_FE - 1]) = 0u;
        __syncthreads();
    }
    const unsigned tiles_x = (unsigned)a.lay.tiles_x;
    for (long long base = (long long)blockIdx.x * EX_THREADS; base < a.n; base += (long long)gridDim.x * EX_THREADS) {
        const long long i = base + tid;
        unsigned cnt = 0, zb = 0, off = 0;
        int4 r = make_int4(0, 0, -1, -1);
        if (i < a.n) {
            cnt = a.touched[i];
            off = a.offsets[i];
            if (cnt) {
                r = a.rect[i];
                zb = __float_as_uint(a.depth[i]);
                if (count)
#pragma unroll
                    for (int p = 0; p < 4; p++) atomicAdd(&s_hd[p][(zb >> (8 * p)) & 255u], cnt);
            }
        }
        const int rows_l = cnt ? r.w - r.y + 1 : 0;
        const unsigned width = cnt ? (unsigned)(r.z - r.x + 1) : 0u;
        const unsigned rincl = warp_inclusive_scan((unsigned)rows_l, lane);
        const unsigned rexcl = rincl - (unsigned)rows_l;
        const unsigned wrows = __shfl_sync(0xffffffffu, rincl, 31);
        // the warp's first entry: the offset of its first Gaussian (lanes past n hold the total)
        unsigned long long out = __shfl_sync(0xffffffffu, off, 0);
        for (unsigned r0 = 0; r0 < wrows; r0 += 32) {
            const unsigned k = r0 + (unsigned)lane;
            int owner = 0; // lane (Gaussian) of warp row k
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (__shfl_sync(0xffffffffu, rincl, owner + step - 1) <= k) owner += step;
            const unsigned rl = k - __shfl_sync(0xffffffffu, rexcl, owner);
            const unsigned ow = __shfl_sync(0xffffffffu, width, owner);
            const int oty = __shfl_sync(0xffffffffu, r.y, owner);
            const int otx = __shfl_sync(0xffffffffu, r.x, owner);
            const unsigned oz = __shfl_sync(0xffffffffu, zb, owner);
            unsigned w = 0, tb = 0;
            if (k < wrows) {
                w = ow;
                tb = (unsigned)(oty + (int)rl) * tiles_x + (unsigned)otx; // tile of the row's first entry
                if (count) count_tile_digits(s_d0, s_h1, a.tile_passes, tb, w);
            }
            const unsigned incl = warp_inclusive_scan(w, lane);
            const unsigned chunk = __shfl_sync(0xffffffffu, incl, 31);
            tb -= incl - w; // entry e of the chunk, if in this row, has tile tb + e
            for (unsigned e0 = 0; e0 < chunk; e0 += 32) {
                const unsigned e = e0 + (unsigned)lane;
                int pos = 0; // row (lane) of entry e
#pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                    if (__shfl_sync(0xffffffffu, incl, pos + step - 1) <= e) pos += step;
                const unsigned tile = __shfl_sync(0xffffffffu, tb, pos) + e;
                const unsigned z = __shfl_sync(0xffffffffu, oz, pos);
                const unsigned gl = (unsigned)__shfl_sync(0xffffffffu, owner, pos);
                const unsigned long long dst = out + e;
                if (e < chunk && dst < (unsigned long long)a.cap) {
                    a.keys[dst] = ((unsigned long long)tile << 32) | z;
                    a.vals[dst] = (unsigned)(base + (long long)(tid & ~31) + gl);
                }
            }
            out += chunk;
        }
    }
    if (count) {
        __syncthreads();
        unsigned* const H = a.hist + (size_t)(blockIdx.x % FE_HIST_COPIES) * (DUP_HIST_STRIDE * RADIX_FE);
        for (int j = tid; j < 4 * RADIX_FE; j += EX_THREADS) {
            const unsigned c = (&s_hd[0][0])[j];
            if (c) atomicAdd(&H[j], c);
        }
        if (tid < 32) { // the tile digits: difference array -> counts, 8 digits per lane
            unsigned c[8], run = 0;
#pragma unroll
            for (int j = 0; j < 8; j++) {
                run += s_d0[8 * lane + j];
                c[j] = run;
            }
            const unsigned incl = warp_inclusive_scan(run, lane);
            const unsigned before = incl - run;
#pragma unroll
            for (int j = 0; j < 8; j++)
                if (c[j] + before) atomicAdd(&H[4 * RADIX_FE + 8 * lane + j], c[j] + before);
        }
        if (a.tile_passes > 1)
            for (int j = tid; j < RADIX_FE; j += EX_THREADS)
                if (s_h1[j]) atomicAdd(&H[5 * RADIX_FE + j], s_h1[j]);
    }
}

void launch_exact_preprocess(const ExactArgs& a, cudaStream_t s)
{
    if (a.n <= 0) return;
    launch_dependent(k_exact_preprocess, dim3((unsigned)((a.n + EX_THREADS - 1) / EX_THREADS)), dim3(EX_THREADS), 0, s, a);
}
void launch_exact_scan(const ExactArgs& a, cudaStream_t s)
{
    if (a.n <= 0) return;
    launch_dependent(k_exact_scan, dim3((unsigned)((a.n + SCAN_TILE - 1) / SCAN_TILE)), dim3(EX_THREADS), 0, s, a);
}
void launch_exact_duplicate(const ExactArgs& a, cudaStream_t s)
{
    if (a.n <= 0) return;
    const long long need = (a.n + EX_THREADS - 1) / EX_THREADS;
    const long long cap = 8ll * device_sm_count(); // grid-stride: digit counts flushed once per block
    launch_dependent(k_exact_duplicate, dim3((unsigned)(need < cap ? need : cap)), dim3(EX_THREADS), 0, s, a);
}

// ---------------------------------------------------------------------------
// Scene conversion (one-off at scene creation)
// ---------------------------------------------------------------------------
__global__ void k_check_finite(const float* p, long long count, unsigned* flag)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    bool bad = false;
    for (; i < count; i += stride) bad |= !isfinite(p[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

void launch_check_finite(const float* p, long long count, unsigned* flag, cudaStream_t s)
{
    if (count <= 0) return;
    long long blocks = (count + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_check_finite<<<(unsigned)blocks, 256, 0, s>>>(p, count, flag);
}

// max |SH| per (degree, channel): float bits of non-negative values order like integers
__global__ void k_sh_absmax(const float* sh, long long n, unsigned* maxbits)
{
    __shared__ unsigned s_max[12];
    if (threadIdx.x < 12) s_max[threadIdx.x] = 0u;
    __syncthreads();
    unsigned local[12];
#pragma unroll
    for (int k = 0; k < 12; k++) local[k] = 0u;
    const long long total = n * 48;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < total; j += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(j % 48), k = e / 3, ch = e % 3;
        const unsigned bits = __float_as_uint(fabsf(sh[j]));
        const int slot = sh_band(k) * 3 + ch;
#pragma unroll
        for (int t = 0; t < 12; t++)
            if (t == slot) local[t] = max(local[t], bits);
    }
#pragma unroll
    for (int t = 0; t < 12; t++) atomicMax(&s_max[t], local[t]);
    __syncthreads();
    if (threadIdx.x < 12) atomicMax(&maxbits[threadIdx.x], s_max[threadIdx.x]);
}

void launch_sh_absmax(const float* sh, long long n, unsigned* maxbits, cudaStream_t s)
{
    if (n <= 0) return;
    long long blocks = (n * 48 + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_sh_absmax<<<(unsigned)blocks, 256, 0, s>>>(sh, n, maxbits);
}

struct CompactParams {
    float band_scale[12];
    int per_gauss;
};

__global__ void k_compact(const float* means, const float* scales, const float* quats, const float* logo,
                          const float* sh, long long n, CompactParams p, float4* geoA, uint4* geoB, uint4* shq)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* c = sh + 48 * i;
    float g = 1.0f;
    if (p.per_gauss) {
        float gm = 0.0f;
        for (int e = 0; e < 48; e++) {
            const float s = p.band_scale[sh_band(e / 3) * 3 + e % 3];
            const float den127 = __fmul_rn(127.0f, s);
            const float r = den127 > 0.0f ? __fdiv_rn(fabsf(c[e]), den127) : 0.0f;
            gm = fmaxf(gm, r);
        }
        g = __half2float(__float2half_rn(gm));
    }
    unsigned char codes[48];
    for (int e = 0; e < 48; e++) {
        const float s = p.band_scale[sh_band(e / 3) * 3 + e % 3];
        const float den = p.per_gauss ? __fmul_rn(g, s) : s;
        int q = 0;
        if (den > 0.0f) {
            q = __float2int_rn(__fdiv_rn(c[e], den));
            q = max(-127, min(127, q));
        }
        codes[e] = (unsigned char)(signed char)q;
    }
    for (int pl = 0; pl < 3; pl++) {
        unsigned w[4];
        for (int k = 0; k < 4; k++)
            w[k] = (unsigned)codes[16 * pl + 4 * k] | ((unsigned)codes[16 * pl + 4 * k + 1] << 8) |
                   ((unsigned)codes[16 * pl + 4 * k + 2] << 16) | ((unsigned)codes[16 * pl + 4 * k + 3] << 24);
        shq[3 * i + pl] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    geoA[i] = make_float4(means[3 * i], means[3 * i + 1], means[3 * i + 2], logo[i]);
    geoB[i] = make_uint4(pack_h2(quats[4 * i], quats[4 * i + 1]), pack_h2(quats[4 * i + 2], quats[4 * i + 3]),
                         pack_h2(scales[3 * i], scales[3 * i + 1]), pack_h2(scales[3 * i + 2], g));
}

void launch_compact(const float* means, const float* scales, const float* quats, const float* logo, const float* sh,
                    long long n, const float* band_scale, int per_gauss, float4* geoA, uint4* geoB, uint4* shq,
                    cudaStream_t s)
{
    if (n <= 0) return;
    CompactParams p;
    for (int k = 0; k < 12; k++) p.band_scale[k] = band_scale[k];
    p.per_gauss = per_gauss;
    k_compact<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(means, scales, quats, logo, sh, n, p, geoA, geoB, shq);
}

} // namespace rg
