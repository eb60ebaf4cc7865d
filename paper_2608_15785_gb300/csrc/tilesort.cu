// tilesort.cu -- the per-tile counting sort of RoofGS entries (RG_FLAG_TILE_COUNTING_SORT).
//
// The fused front end emits its (16-bit tile id, value) entries in (quantized depth,
// Gaussian index) order; the frame needs them grouped by tile with that order kept
// inside every tile (the order of the 32-bit key of Sec. IV-A.2, ties by index). A
// counting sort does it in one scatter instead of two 8-bit radix passes:
//
//  * k_tc_count: the entries are cut into C consecutive chunks; each chunk's block
//    counts its entries per tile in shared memory (one counter per tile of the image)
//    and stores the counts as row c of a C x T matrix;
//  * k_tc_colscan: per tile, the exclusive prefix of its counts over the chunks (the
//    entries of that tile in earlier chunks) and the tile's total;
//  * k_tc_tilescan: the exclusive prefix of the totals over the tiles: each tile's first
//    slot, written as the tile ranges the rasterizer reads ([0, 0) for empty tiles);
//  * k_tc_scatter: each chunk's block holds one running offset per tile in shared
//    memory and scatters its entries in order: 1024 entries at a time, every warp ranks
//    its 4 x 32 entries by tile (match_any), then the warps take the tiles' offsets in
//    warp order (one barrier per warp), so equal tiles keep the entries' order.
//
// The per-tile offsets make a block's shared memory 4 B x tiles (130 KB at 3840x2160),
// so 4K runs one such block per SM; stability forces the warps of a block to take their
// offsets in turn.
#include <algorithm>
#include <mutex>

#include "rg_internal.cuh"

namespace rg {

constexpr int TC_THREADS = 256;
constexpr int TC_WARPS = TC_THREADS / 32;
constexpr int TC_GROUPS = 4;                           // 32-entry groups per warp per round
constexpr int TC_BATCH = TC_THREADS * TC_GROUPS;       // entries per round of the scatter
constexpr unsigned TC_NONE = 0xFFFFu;                  // no entry (past the chunk's end)

__global__ void __launch_bounds__(TC_THREADS) k_tc_count(TileSortArgs a)
{
    extern __shared__ unsigned s_cnt[];
    grid_dependency_wait();
    for (int t = threadIdx.x; t < a.T; t += TC_THREADS) s_cnt[t] = 0u;
    __syncthreads();
    const unsigned n = a.ctr->n_entries;
    const unsigned S = ((n + a.chunks - 1) / a.chunks + TC_BATCH - 1) / TC_BATCH * TC_BATCH;
    const unsigned b = blockIdx.x * S;
    const unsigned e = b + S < n ? b + S : n;
    for (unsigned j = b + threadIdx.x; j < e; j += TC_THREADS) {
        const unsigned t = a.keys16[j];
        if (t < (unsigned)a.T) atomicAdd(&s_cnt[t], 1u);
    }
    __syncthreads();
    unsigned* const row = a.M + (size_t)blockIdx.x * a.T;
    for (int t = threadIdx.x; t < a.T; t += TC_THREADS) row[t] = s_cnt[t];
}

// one thread per tile: column prefix over the chunks (coalesced across threads)
__global__ void __launch_bounds__(256) k_tc_colscan(TileSortArgs a)
{
    grid_dependency_wait();
    const int t = blockIdx.x * 256 + threadIdx.x;
    if (t >= a.T) return;
    unsigned run = 0u;
    for (int c = 0; c < a.chunks; c++) {
        unsigned* const p = a.M + (size_t)c * a.T + t;
        const unsigned x = *p;
        *p = run;
        run += x;
    }
    a.tot[t] = run;
}

// one block: exclusive prefix of the tile totals -> first slot of every tile (in tot)
// and the ranges
__global__ void __launch_bounds__(1024) k_tc_tilescan(TileSortArgs a)
{
    __shared__ unsigned s_w[32];
    grid_dependency_wait();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (a.T + 1023) / 1024;
    const int t0 = tid * per;
    unsigned sum = 0u;
    for (int k = 0; k < per; k++)
        if (t0 + k < a.T) sum += a.tot[t0 + k];
    unsigned x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned w = s_w[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_w[lane] = w;
    }
    __syncthreads();
    unsigned run = x - sum + (warp ? s_w[warp - 1] : 0u);
    for (int k = 0; k < per; k++) {
        const int t = t0 + k;
        if (t >= a.T) break;
        const unsigned c = a.tot[t];
        a.tot[t] = run;
        a.ranges[t] = c ? make_uint2(run, run + c) : make_uint2(0u, 0u);
        run += c;
    }
}

__global__ void __launch_bounds__(TC_THREADS) k_tc_scatter(TileSortArgs a)
{
    extern __shared__ unsigned s_off[];
    grid_dependency_wait();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned* const row = a.M + (size_t)blockIdx.x * a.T;
    for (int t = tid; t < a.T; t += TC_THREADS) s_off[t] = row[t] + a.tot[t];
    __syncthreads();
    const unsigned n = a.ctr->n_entries;
    const unsigned S = ((n + a.chunks - 1) / a.chunks + TC_BATCH - 1) / TC_BATCH * TC_BATCH;
    const unsigned b = blockIdx.x * S;
    const unsigned e = b + S < n ? b + S : n;
    const unsigned lt = (1u << lane) - 1u;
    for (unsigned base = b; base < e; base += TC_BATCH) {
        unsigned tt[TC_GROUPS], vv[TC_GROUPS], pos[TC_GROUPS], cnt[TC_GROUPS];
        int ld[TC_GROUPS];
        // rank every entry among the entries of the same tile in its group of 32
#pragma unroll
        for (int g = 0; g < TC_GROUPS; g++) {
            const unsigned j = base + (unsigned)(warp * 32 * TC_GROUPS + g * 32 + lane);
            unsigned t = TC_NONE;
            vv[g] = 0u;
            if (j < e) {
                t = a.keys16[j];
                vv[g] = a.vals[j];
                if (t >= (unsigned)a.T) t = TC_NONE;
            }
            const unsigned peers = __match_any_sync(0xffffffffu, t);
            tt[g] = t;
            pos[g] = (unsigned)__popc(peers & lt);
            cnt[g] = (unsigned)__popc(peers);
            ld[g] = __ffs(peers) - 1;
        }
        // the warps take their tiles' offsets in turn (warp order is entry order)
        for (int w = 0; w < TC_WARPS; w++) {
            if (warp == w) {
#pragma unroll
                for (int g = 0; g < TC_GROUPS; g++) {
                    unsigned o = 0u;
                    if (lane == ld[g] && tt[g] != TC_NONE) {
                        o = s_off[tt[g]];
                        s_off[tt[g]] = o + cnt[g];
                    }
                    __syncwarp(); // the next group of this warp sees the update
                    pos[g] += __shfl_sync(0xffffffffu, o, ld[g]);
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int g = 0; g < TC_GROUPS; g++)
            if (tt[g] != TC_NONE && pos[g] < n) a.vout[pos[g]] = vv[g];
    }
}

namespace {
constexpr int MAX_DEVICES = 64;
std::mutex g_tc_mu;
int g_tc_attr[MAX_DEVICES] = {0}; // largest dynamic shared memory set for the two kernels
} // namespace

int tilesort_max_tiles() { return (227 * 1024 - 1024) / 4; }

int tilesort_chunks(int T)
{
    if (T <= 0 || T > tilesort_max_tiles()) return 0;
    const size_t smem = (size_t)T * 4;
    const int per_sm = (int)std::min<size_t>(8, (size_t)(228 * 1024) / (smem + 1024 + 64));
    return (per_sm > 0 ? per_sm : 1) * device_sm_count();
}

size_t tilesort_matrix_bytes(int T) { return (size_t)tilesort_chunks(T) * (size_t)(T > 0 ? T : 0) * 4; }

// per_sm x (4T + 1088 + 64) <= 228 KB bounds per_sm x 4T, whatever T: the largest matrix
size_t tilesort_matrix_bytes_max() { return (size_t)device_sm_count() * 228 * 1024; }

void launch_tile_counting_sort(const TileSortArgs& a, cudaStream_t s)
{
    const size_t smem = (size_t)a.T * 4;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 0 || dev >= MAX_DEVICES) dev = 0;
        std::lock_guard<std::mutex> lock(g_tc_mu);
        if ((size_t)g_tc_attr[dev] < smem) { // once per device and size, with the device current
            cudaFuncSetAttribute(k_tc_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cudaFuncSetAttribute(k_tc_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            g_tc_attr[dev] = (int)smem;
        }
    }
    launch_dependent(k_tc_count, dim3(a.chunks), dim3(TC_THREADS), smem, s, a);
    launch_dependent(k_tc_colscan, dim3((a.T + 255) / 256), dim3(256), 0, s, a);
    launch_dependent(k_tc_tilescan, dim3(1), dim3(1024), 0, s, a);
    launch_dependent(k_tc_scatter, dim3(a.chunks), dim3(TC_THREADS), smem, s, a);
}

} // namespace rg
