// sort.cu -- stable LSD radix sort of (key, value) entries and per-tile ranges.
//
// Depth sort of Sec. III-C / Sec. IV-A.2: traffic ~ S_kv * N_dup * N_pass
// (Eq. (6)). 8-bit digits; 4 passes for the 32-bit RoofGS key (or only the
// ceil(b_t / 8) tile-bit passes when the Gaussians were put in depth order
// first: then, with b_t <= 16, the entries carry the 16-bit tile id alone) and
// ceil((32 + b_t) / 8) passes for the 64-bit exact-mode key (only the bits
// that can be non-zero are sorted).
//
// One histogram kernel reads every key once and counts the digits of all
// passes, unless the producer of the keys counted them (the depth-key kernel
// counts its codes' digits; the RoofGS front end counts the tile digits of its
// entries per tile row; the kernel then only clears look-back state, and counts
// if entries overflowed). Each pass is then ONE kernel over tiles of 6144
// (16- and 32-bit keys) or 4096 (64-bit keys) entries (one-sweep scheme): a
// persistent grid takes tiles
// in order from an atomic counter (and prefetches the tile half a grid ahead into
// L2), ranks the tile's digits per warp (stable; per pass one of: match_any,
// where a warp holds few distinct digits; a bit mask per digit in shared memory
// that every lane ORs its bit into, where it holds many; where shared memory
// allows, each warp's elements as two interleaved chains), publishes its
// per-digit counts, obtains the counts of all earlier tiles by decoupled
// look-back (bounded waits), reorders the tile in shared memory by digit and
// writes each digit run to its global position (runs of consecutive addresses).
// Per pass every entry is read once and written once. The number of entries is
// read on the device: no host round trip. k_ranges finds the per-tile
// [start, end) of a sorted array (exact mode; RoofGS frames find their ranges
// inside the rasterizer).
#include <algorithm>
#include <mutex>

#include "rg_internal.cuh"

namespace rg {

// Tile shape per key width: (threads, keys per thread, resident blocks per SM).
// Larger tiles amortise the per-tile barriers and look-back; two resident blocks
// per SM keep one block's loads in flight while the other waits at a barrier.
// 32-bit keys: 384 x 16 = 6144 entries at 80 registers; 64-bit keys: 512 x 8 =
// 4096 entries at 64 registers (16 keys of 64 bits would spill); 16-bit tile
// ids: 256 x 24 = 6144 entries, three blocks per SM (below).
template <typename K>
struct SortCfg;
#ifndef RG_SORT_T32
#define RG_SORT_T32 384
#define RG_SORT_K32 16
#define RG_SORT_B32 2
#endif
template <>
struct SortCfg<unsigned> {
    static constexpr int THREADS = RG_SORT_T32, KPT = RG_SORT_K32, MIN_BLOCKS = RG_SORT_B32;
    static constexpr bool STAGE_VALS = false;
};
// 16-bit tile ids: 6-byte entries leave room in shared memory for three CTAs of
// 256 x 24 = 6144 entries per SM (80 registers, a few spilled): measured 0.852 ms
// for the two 4K passes against 0.876 ms at 384 x 16 with two CTAs
#ifndef RG_SORT_T16
#define RG_SORT_T16 256
#define RG_SORT_K16 24
#define RG_SORT_B16 3
#endif
template <> // 16-bit tile ids (a key still takes a register)
struct SortCfg<unsigned short> {
    static constexpr int THREADS = RG_SORT_T16, KPT = RG_SORT_K16, MIN_BLOCKS = RG_SORT_B16;
    // values staged in shared memory by cp.async instead of registers: no spills at 80
    // registers, 71.7 KB per CTA (3 per SM still fit); 4K tile-bit passes 0.855 -> 0.835 ms
    static constexpr bool STAGE_VALS = true;
};
template <>
struct SortCfg<unsigned long long> {
    static constexpr int THREADS = 512, KPT = 8, MIN_BLOCKS = 2;
    static constexpr bool STAGE_VALS = false; // staging measured slower for the exact-mode keys (9.14 vs 8.81 ms)
};
template <typename K>
constexpr int tile_of() { return SortCfg<K>::THREADS * SortCfg<K>::KPT; }

constexpr int RADIX = 256;
constexpr int LB_WINDOW = 4; // predecessors inspected per round trip of the look-back (4K tile-bit passes 0.656 ms at 8, 0.638 at 4, 0.642 at 3, 0.646 at 2, 0.710 at 16)
constexpr unsigned SF_AGG = 1u << 30, SF_PRE = 2u << 30, SF_VAL = (1u << 30) - 1u;
constexpr int H_THREADS = 256;

long long sort_status_words(int key_bytes, long long n)
{
    const long long t = key_bytes == 2 ? tile_of<unsigned short>() : (key_bytes == 4 ? tile_of<unsigned>() : tile_of<unsigned long long>());
    return (n + t - 1) / t * RADIX;
}

// smallest tile of any key width: sizes the per-tile look-back status arrays
int sort_tile_items()
{
    int t = tile_of<unsigned long long>();
    if (tile_of<unsigned>() < t) t = tile_of<unsigned>();
    if (tile_of<unsigned short>() < t) t = tile_of<unsigned short>();
    return t;
}

// Launch shapes that depend on the device (SM count, resident one-sweep CTAs, the
// one-sweep kernels' shared-memory attribute), looked up once per device with that
// device current (the first launch on a device should come before any stream
// capture) and kept in a small table guarded by a mutex.
namespace {
constexpr int MAX_DEVICES = 64;
struct DeviceShape {
    int sms = 0;
    int onesweep_grid[3] = {0, 0, 0}; // 16-, 32- and 64-bit keys
};
std::mutex g_shape_mu;
DeviceShape g_shape[MAX_DEVICES];

int current_device()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) dev = 0;
    return dev;
}
} // namespace

int device_sm_count()
{
    const int dev = current_device();
    std::lock_guard<std::mutex> lock(g_shape_mu);
    DeviceShape& d = g_shape[dev];
    if (d.sms == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        d.sms = v > 0 ? v : 1;
    }
    return d.sms;
}

static int sm_count() { return device_sm_count(); }

// The producer's digit counts cover every entry it made; they are not used when
// entries did not fit (overflow) or its allocation gave up waiting (the error bit
// of its look-back, or of the exact scan's): the histogram kernel then counts the
// stored keys. Both flags
// are final before the sort starts.
__device__ __forceinline__ bool recount_digits(const Counters* ctr)
{
    return ctr->overflow != 0u || (ctr->error & (ERR_FE_LOOKBACK | ERR_SCAN_LOOKBACK)) != 0u;
}

// Digit histograms of every pass in one read of the keys (vector loads; the
// counts of equal digits within a warp are combined before the shared atomic).
// When the producer of the keys counted the digits already (only_on_overflow),
// this kernel clears the first pass's look-back status and counts only when
// recount_digits() says so.
template <typename K>
__global__ void __launch_bounds__(H_THREADS) k_sort_hist(const K* __restrict__ keys, int passes, int bit0,
                                                         unsigned* hist, unsigned* status0,
                                                         const Counters* __restrict__ ctr, unsigned* hist_pre,
                                                         const unsigned* __restrict__ hist_copies, int copy_stride)
{
    __shared__ unsigned s_h[8][RADIX];
    grid_dependency_wait();
    for (int j = threadIdx.x; j < 8 * RADIX; j += H_THREADS) (&s_h[0][0])[j] = 0u;
    __syncthreads();
    const long long n = ctr->n_entries;
    constexpr int S_TILE = tile_of<K>();
    const long long ntiles = (n + S_TILE - 1) / S_TILE;
    const long long gsz = (long long)gridDim.x * H_THREADS;
    const long long gid = (long long)blockIdx.x * H_THREADS + threadIdx.x;
    // clear the look-back status words of the first pass
    for (long long j = gid; j < ntiles * RADIX; j += gsz) status0[j] = 0u;
    if (hist_pre && !recount_digits(ctr)) {
        // the producer's counts: complete, or sum its copies (one digit of one pass per thread)
        if (!hist_copies) return;
        for (long long c = gid; c < (long long)passes * RADIX; c += gsz) {
            unsigned sum = 0u;
            for (int j = 0; j < FE_HIST_COPIES; j++) sum += hist_copies[(size_t)j * copy_stride * RADIX + c];
            hist_pre[c] = sum;
        }
        return;
    }
    constexpr int V = 16 / sizeof(K); // keys per 16-byte load
    const long long nv = n / V;
    // consecutive keys often share digits (entries of one Gaussian): runs of equal
    // digits among a thread's V keys take one shared atomic. Two 16-byte loads per
    // iteration keep more of the stream in flight.
    auto count = [&](const uint4& q) {
        K k[V];
        memcpy(k, &q, 16);
        for (int p = 0; p < passes; p++) {
            unsigned d = (unsigned)(k[0] >> (bit0 + 8 * p)) & 0xffu, c = 1u;
#pragma unroll
            for (int u = 1; u < V; u++) {
                const unsigned e = (unsigned)(k[u] >> (bit0 + 8 * p)) & 0xffu;
                if (e == d) {
                    c++;
                } else {
                    atomicAdd(&s_h[p][d], c);
                    d = e;
                    c = 1u;
                }
            }
            atomicAdd(&s_h[p][d], c);
        }
    };
    for (long long j = gid; j < nv; j += 2 * gsz) {
        const uint4 q0 = __ldg(reinterpret_cast<const uint4*>(keys) + j);
        const bool two = j + gsz < nv;
        const uint4 q1 = two ? __ldg(reinterpret_cast<const uint4*>(keys) + j + gsz) : q0;
        count(q0);
        if (two) count(q1);
    }
    // tail (fewer than V keys)
    for (long long j = nv * V + gid; j < n; j += gsz) {
        const K kk = keys[j];
        for (int p = 0; p < passes; p++) atomicAdd(&s_h[p][(unsigned)(kk >> (bit0 + 8 * p)) & 0xffu], 1u);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < passes * RADIX; j += H_THREADS) {
        const unsigned c = (&s_h[0][0])[j];
        if (c) atomicAdd(&hist[j], c);
    }
}

// exclusive scan over the first 256 threads (one digit each) of the block;
// every thread of the block must call it
__device__ __forceinline__ unsigned digit_exclusive_scan(unsigned v, unsigned* s_w)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31 && warp < RADIX / 32) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned w = lane < RADIX / 32 ? s_w[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < RADIX / 32) s_w[lane] = w;
    }
    __syncthreads();
    return x - v + (warp ? s_w[warp - 1] : 0u);
}

// asynchronous global -> shared copies (cp.async): the tile's values travel to shared
// memory while the keys are ranked, without passing through registers
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename K>
struct SortSmem {
    static constexpr int TILE = tile_of<K>(), WARPS = SortCfg<K>::THREADS / 32;
    K keys[TILE];
    unsigned vals[TILE];
    unsigned vin[SortCfg<K>::STAGE_VALS ? TILE : 1]; // the tile's values as loaded (element order), by cp.async
    unsigned whist[WARPS][RADIX]; // per-warp digit counters, then each warp's first slot of the digit in the tile
    unsigned goff[RADIX];         // global exclusive digit offsets of this pass
    unsigned gbase[RADIX];        // global start of this tile's run of each digit minus its local start
    unsigned scan[WARPS];
    unsigned tile;
};

template <typename K, int RM>
__global__ void __launch_bounds__(SortCfg<K>::THREADS, SortCfg<K>::MIN_BLOCKS) k_onesweep(const K* __restrict__ kin, const unsigned* __restrict__ vin,
                                                        K* __restrict__ kout, unsigned* __restrict__ vout, int pass,
                                                        int bit0, const unsigned* __restrict__ hist,
                                                        const unsigned* __restrict__ hist_pre, unsigned* status,
                                                        unsigned* status_next, Counters* ctr, Sticky* sticky)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    grid_dependency_wait();
    constexpr int S_THREADS = SortCfg<K>::THREADS, S_KPT = SortCfg<K>::KPT, S_TILE = tile_of<K>();
    // threads 0..255 each own one digit (scan, offsets, look-back): at least RADIX threads
    static_assert(S_THREADS >= RADIX && S_THREADS % 32 == 0, "sort tile needs one thread per digit");
    constexpr int S_WARPS = S_THREADS / 32;
    SortSmem<K>& S = *reinterpret_cast<SortSmem<K>*>(smem_raw);
    static_assert(S_WARPS * RADIX <= S_TILE, "the peer masks live in the reorder buffer's values");
    // two ranking chains per warp where the reorder buffer's values hold two sets of peer masks
    // and the counts of a chain fit 16 bits (32 x KPT / 2 elements)
    constexpr bool TWO_CHAINS = 2 * S_WARPS * RADIX <= S_TILE && S_KPT % 4 == 0;
    constexpr int HALF = S_KPT / 2;
    constexpr int PM_WORDS = (TWO_CHAINS ? 2 : 1) * S_WARPS * RADIX; // peer-mask words in S.vals
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // SORT_RANK_PEERS: this warp's bit mask per digit, in the reorder buffer's values (free until
    // barrier B; all zero whenever a tile's ranking starts)
    unsigned* const pmask = S.vals + warp * RADIX;
    const int shift = bit0 + 8 * pass;
    // entry counts stay below 2^30 (workspace limit): 32-bit indices throughout
    const unsigned n = ctr->n_entries;
    const unsigned ntiles = (n + S_TILE - 1) / S_TILE;
    {
        const unsigned* H = (hist_pre && !recount_digits(ctr)) ? hist_pre : hist;
        const unsigned h = tid < RADIX ? H[pass * RADIX + tid] : 0u;
        const unsigned e = digit_exclusive_scan(h, S.scan);
        if (tid < RADIX) S.goff[tid] = e;
    }
    const unsigned lt_mask = (1u << lane) - 1u;
    // The first tile is claimed here; each later one is claimed, and the warp
    // counters cleared, during the write-out of the tile before it. Five
    // barriers per tile: after ranking (B), after the digit scan (C), after the
    // local offsets (D), after the reorder (E) and after the write-out (A).
    for (int j = tid; j < S_WARPS * RADIX; j += S_THREADS) (&S.whist[0][0])[j] = 0u;
    if (RM == SORT_RANK_PEERS)
        for (int j = tid; j < PM_WORDS; j += S_THREADS) S.vals[j] = 0u;
    if (tid == 0) S.tile = atomicAdd(&ctr->sort_tile_ctr[pass], 1u);
    __syncthreads();
    while (true) {
        const unsigned tile = S.tile;
        if (tile >= ntiles) break;
        if (tid == 0) {
            // tiles are claimed in order, one per block at a time: the tile half a grid ahead is
            // claimed by some block about half a tile's time from now. Its keys and values go to
            // L2 by one bulk prefetch each (16-byte multiples inside the tile), so that block's
            // key loads hit L2 (4K tile-bit passes 0.778 -> 0.742 ms; the keys alone 0.748 ms,
            // the values alone 0.785 ms; a quarter grid ahead as good, one grid ahead 0.744 ms)
            const unsigned nx = tile + gridDim.x / 2;
            if (nx < ntiles) {
                const unsigned b = nx * S_TILE;
                const unsigned c = n - b < (unsigned)S_TILE ? n - b : (unsigned)S_TILE;
                const unsigned kb = (c * (unsigned)sizeof(K)) & ~15u, vb = (c * 4u) & ~15u;
                if (kb) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(kin + b), "r"(kb) : "memory");
                if (vb) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(vin + b), "r"(vb) : "memory");
            }
        }

        constexpr bool STAGE = SortCfg<K>::STAGE_VALS;
        if constexpr (STAGE) {
            // the tile's values go to shared memory asynchronously (16 bytes at a time; the tile
            // starts on a 16-byte boundary of a 16-byte-aligned array); read back by the reorder
            const unsigned base = tile * S_TILE;
            const unsigned cnt = n - base < (unsigned)S_TILE ? n - base : (unsigned)S_TILE;
            const unsigned full = cnt & ~3u;
            for (unsigned c = tid; c < full / 4; c += S_THREADS) cp_async16(&S.vin[4 * c], vin + base + 4 * c);
            for (unsigned j = full + tid; j < cnt; j += S_THREADS) cp_async4(&S.vin[j], vin + base + j);
        }
        // load the tile warp-striped: element = tile*TILE + warp*32*KPT + i*32 + lane
        const unsigned e0 = tile * S_TILE + warp * 32 * S_KPT + lane;
        K k[S_KPT];
        unsigned v[STAGE ? 1 : S_KPT];
#pragma unroll
        for (int i = 0; i < S_KPT; i++) {
            const unsigned e = e0 + 32 * i;
            const bool ok = e < n;
            k[i] = ok ? kin[e] : (K)~(K)0; // padding sorts last (digit 255, after the valid ones)
            if constexpr (!STAGE) v[i] = ok ? vin[e] : 0u;
        }
        // stable rank of each element among the warp's elements of the same digit
        // (below 32 * KPT: two ranks share a register)
        unsigned rank2[(S_KPT + 1) / 2];
        auto set_rank = [&](int i, unsigned r) {
            if (i & 1) rank2[i >> 1] |= r << 16;
            else rank2[i >> 1] = r;
        };
        if constexpr (TWO_CHAINS) {
            // two independent chains: elements 0 .. HALF-1 count in the low 16 bits of the warp's
            // digit counters, elements HALF .. KPT-1 in the high 16 bits (each with its own peer
            // masks), so the shared-memory round trips of one element overlap the other's
            unsigned* const pmask_b = pmask + S_WARPS * RADIX;
#pragma unroll
            for (int i = 0; i < HALF; i++) {
                const unsigned da = (unsigned)(k[i] >> shift) & 0xffu, db = (unsigned)(k[i + HALF] >> shift) & 0xffu;
                unsigned pa, pb;
                if (RM == SORT_RANK_PEERS) {
                    atomicOr(&pmask[da], 1u << lane);
                    atomicOr(&pmask_b[db], 1u << lane);
                    __syncwarp();
                    pa = pmask[da];
                    pb = pmask_b[db];
                } else {
                    pa = __match_any_sync(0xffffffffu, da);
                    pb = __match_any_sync(0xffffffffu, db);
                }
                const int la = __ffs(pa) - 1, lb = __ffs(pb) - 1;
                unsigned ba = 0, bb = 0;
                if (lane == la) ba = atomicAdd(&S.whist[warp][da], (unsigned)__popc(pa));
                if (lane == lb) bb = atomicAdd(&S.whist[warp][db], (unsigned)__popc(pb) << 16);
                ba = __shfl_sync(0xffffffffu, ba, la) & 0xffffu;
                bb = __shfl_sync(0xffffffffu, bb, lb) >> 16;
                if (RM == SORT_RANK_PEERS) { // every lane has read the masks (the shuffles)
                    if (lane == la) pmask[da] = 0u;
                    if (lane == lb) pmask_b[db] = 0u;
                }
                set_rank(i, ba + __popc(pa & lt_mask));
                set_rank(i + HALF, bb + __popc(pb & lt_mask));
                __syncwarp();
            }
        } else {
#pragma unroll
            for (int i = 0; i < S_KPT; i++) {
                const unsigned d = (unsigned)(k[i] >> shift) & 0xffu;
                unsigned peers;
                if (RM == SORT_RANK_PEERS) { // every lane sets its bit in its digit's mask
                    atomicOr(&pmask[d], 1u << lane);
                    __syncwarp();
                    peers = pmask[d];
                } else { // hardware match: fast when the warp holds few distinct digits
                    peers = __match_any_sync(0xffffffffu, d);
                }
                const int leader = __ffs(peers) - 1;
                unsigned b = 0;
                if (RM == SORT_RANK_PEERS) {
                    // one lane per digit: read and advance the warp's count, clear the mask once every
                    // lane has read it (after the shuffle)
                    if (lane == leader) b = S.whist[warp][d];
                    b = __shfl_sync(0xffffffffu, b, leader);
                    if (lane == leader) {
                        S.whist[warp][d] = b + (unsigned)__popc(peers);
                        pmask[d] = 0u;
                    }
                } else {
                    if (lane == leader) b = atomicAdd(&S.whist[warp][d], (unsigned)__popc(peers)); // one lane per digit
                    b = __shfl_sync(0xffffffffu, b, leader);
                }
                set_rank(i, b + __popc(peers & lt_mask));
                __syncwarp();
            }
        }
        __syncthreads(); // B
        // digit tid: tile count, per-warp exclusive offsets, publish the count,
        // issue the first look-back window (consumed after barrier D), and
        // scan the counts within the warp
        unsigned count = 0, incl = 0;
        unsigned sv[LB_WINDOW];
        if (tid < RADIX) {
#pragma unroll
            for (int w = 0; w < S_WARPS; w++) {
                const unsigned c = S.whist[w][tid];
                if constexpr (TWO_CHAINS) { // the warp's offsets of both chains, low and high half
                    const unsigned ca = c & 0xffffu;
                    S.whist[w][tid] = count | ((count + ca) << 16);
                    count += ca + (c >> 16);
                } else {
                    S.whist[w][tid] = count;
                    count += c;
                }
            }
            *reinterpret_cast<volatile unsigned*>(status + (size_t)tile * RADIX + tid) = (tile == 0 ? SF_PRE : SF_AGG) | count;
#pragma unroll
            for (int w = 0; w < LB_WINDOW; w++)
                sv[w] = ((int)tile - 1 - w >= 0)
                            ? *reinterpret_cast<volatile unsigned*>(status + (size_t)(tile - 1 - w) * RADIX + tid)
                            : (2u << 30); // before tile 0: prefix 0
            incl = count;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) S.scan[warp] = incl;
        }
        if constexpr (SortCfg<K>::STAGE_VALS) cp_async_wait_all(); // this thread's value copies, visible after C
        __syncthreads(); // C
        unsigned lo = 0;
        if (tid < RADIX) {
            lo = incl - count;
            for (int w = 0; w < warp; w++) lo += S.scan[w];
            // the tile-local start of the digit goes into every warp's offset (both chains' halves),
            // so that the reorder reads one word per element
            const unsigned lo2 = TWO_CHAINS ? (lo | (lo << 16)) : lo;
#pragma unroll
            for (int w = 0; w < S_WARPS; w++) S.whist[w][tid] += lo2;
        }
        __syncthreads(); // D
        // reorder the tile by digit in shared memory. Where every thread owns a digit (256 threads) the
        // reorder comes first and the look-back's first window (loaded before barrier C) arrives
        // meanwhile (4K tile-bit passes 0.714 -> 0.685 ms); with more threads the other warps reorder
        // while the digit threads look back
        auto reorder = [&]() {
#pragma unroll
            for (int i = 0; i < S_KPT; i++) {
                const unsigned d = (unsigned)(k[i] >> shift) & 0xffu;
                const unsigned r = (i & 1) ? (rank2[i >> 1] >> 16) : (rank2[i >> 1] & 0xffffu);
                unsigned woff = S.whist[warp][d];
                if constexpr (TWO_CHAINS) woff = i < HALF ? (woff & 0xffffu) : (woff >> 16);
                const unsigned pos = woff + r;
                S.keys[pos] = k[i];
                if constexpr (SortCfg<K>::STAGE_VALS) S.vals[pos] = S.vin[warp * 32 * S_KPT + 32 * i + lane];
                else S.vals[pos] = v[i];
            }
        };
        if constexpr (S_THREADS == RADIX) reorder();
        if (tid < RADIX) {
            // windowed decoupled look-back: LB_WINDOW predecessors per round trip,
            // sv[w] holding the status of tile t - w
            unsigned excl = 0;
            if (tile > 0) {
                int t = (int)tile - 1;
                bool timed_out = false;
                unsigned spins = 0;
                while (true) {
                    // use the window up to the first missing entry or the first prefix
                    int used = 0;
                    bool found = false;
                    unsigned add = 0;
#pragma unroll
                    for (int w = 0; w < LB_WINDOW; w++) {
                        if (used == w && !found) {
                            const unsigned f = sv[w] >> 30;
                            if (f != 0u) {
                                add += sv[w] & SF_VAL;
                                used = w + 1;
                                if (f == 2u) found = true;
                            }
                        }
                    }
                    excl += add;
                    t -= used;
                    if (found || t < 0) break;
                    if (used == 0) { // nearest predecessor not published yet
                        if (++spins > SPIN_LIMIT) {
                            timed_out = true;
                            break;
                        }
                        __nanosleep(32);
                    }
#pragma unroll
                    for (int w = 0; w < LB_WINDOW; w++)
                        sv[w] = (t - w >= 0) ? *reinterpret_cast<volatile unsigned*>(status + (size_t)(t - w) * RADIX + tid)
                                             : (2u << 30);
                }
                if (timed_out) {
                    atomicOr(&ctr->error, ERR_SORT_LOOKBACK);
                    atomicOr(&sticky->error, ERR_SORT_LOOKBACK);
                }
                *reinterpret_cast<volatile unsigned*>(status + (size_t)tile * RADIX + tid) = SF_PRE | ((excl + count) & SF_VAL);
            }
            // output index of tile-sorted element j of this digit = gbase[d] + j (mod 2^32)
            S.gbase[tid] = S.goff[tid] + excl - lo;
            if (status_next) status_next[(size_t)tile * RADIX + tid] = 0u;
        }
        if constexpr (S_THREADS != RADIX) reorder();
        __syncthreads(); // E
        const unsigned rem = n - tile * S_TILE;
        if (rem >= (unsigned)S_TILE) {
#pragma unroll
            for (int u = 0; u < S_KPT; u++) {
                const int j = tid + u * S_THREADS;
                const K kk = S.keys[j];
                const unsigned dst = S.gbase[(unsigned)(kk >> shift) & 0xffu] + (unsigned)j;
                if (dst < n) { // always true unless a bounded wait gave up
                    kout[dst] = kk;
                    vout[dst] = S.vals[j];
                }
            }
        } else {
            for (int j = tid; j < (int)rem; j += S_THREADS) {
                const K kk = S.keys[j];
                const unsigned dst = S.gbase[(unsigned)(kk >> shift) & 0xffu] + (unsigned)j;
                if (dst < n) {
                    kout[dst] = kk;
                    vout[dst] = S.vals[j];
                }
            }
        }
        // slot j of the reorder buffer is read above by thread j mod THREADS only: that thread
        // clears the peer masks it aliases
        for (int j = tid; j < S_WARPS * RADIX; j += S_THREADS) (&S.whist[0][0])[j] = 0u;
        if (RM == SORT_RANK_PEERS)
            for (int j = tid; j < PM_WORDS; j += S_THREADS) S.vals[j] = 0u;
        if (tid == 0) S.tile = atomicAdd(&ctr->sort_tile_ctr[pass], 1u);
        __syncthreads(); // A
    }
}

template <typename K, int RM>
static int onesweep_blocks_per_sm(size_t smem)
{
    cudaFuncSetAttribute(k_onesweep<K, RM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_onesweep<K, RM>, SortCfg<K>::THREADS, smem);
    return per_sm;
}

template <typename K>
static void sort_impl(const SortArgs& a, cudaStream_t s, cudaEvent_t ev_after_hist)
{
    const size_t smem = sizeof(SortSmem<K>);
    const int kind = sizeof(K) == 2 ? 0 : (sizeof(K) == 4 ? 1 : 2);
    const int sms = sm_count();
    int grid;
    {
        const int dev = current_device();
        std::lock_guard<std::mutex> lock(g_shape_mu);
        int& g = g_shape[dev].onesweep_grid[kind];
        if (g == 0) { // once per device and key width, with the device current
            // the two rankings share the tile shape and the launch bounds: the smaller
            // residency of the two sizes the persistent grid
            const int per_sm = std::min(onesweep_blocks_per_sm<K, SORT_RANK_MATCH>(smem),
                                        onesweep_blocks_per_sm<K, SORT_RANK_PEERS>(smem));
            g = (per_sm > 0 ? per_sm : 1) * sms;
        }
        grid = g;
    }
    // at most one tile per SM (the depth order of 0.5 M Gaussians has 82 tiles of 6144): one
    // block per SM, so that no two of the few tiles share an SM while others idle (1080p depth
    // order 0.066 -> 0.057 ms; 4K, 488 tiles, keeps two blocks per SM: 0.110 against 0.119 ms)
    if (a.cap <= (long long)tile_of<K>() * sms) grid = sms;
    const int hist_grid = 8 * sms;
    const K* kin = (const K*)a.keys[0];
    if (a.passes <= 0) return;
    if (!a.hist_done)
        launch_dependent(k_sort_hist<K>, dim3(hist_grid), dim3(H_THREADS), 0, s, kin, a.passes, a.bit0, a.hist,
                         a.status[0], a.ctr, a.hist_pre, a.hist_copies,
                         a.hist_copy_stride > 0 ? a.hist_copy_stride : 2);
    if (ev_after_hist) cudaEventRecord(ev_after_hist, s);
    for (int p = 0; p < a.passes; p++) {
        const int src = p & 1, dst = src ^ 1;
        unsigned* nxt = (p + 1 < a.passes) ? a.status[(p + 1) & 1] : nullptr;
        const int rm = (int)((a.rank_modes >> (2 * p)) & 3u);
        auto kern = rm == SORT_RANK_PEERS ? k_onesweep<K, SORT_RANK_PEERS> : k_onesweep<K, SORT_RANK_MATCH>;
        launch_dependent(kern, dim3(grid), dim3(SortCfg<K>::THREADS), smem, s, (const K*)a.keys[src], a.vals[src],
                         (K*)a.keys[dst], a.vals[dst], p, a.bit0, (const unsigned*)a.hist, (const unsigned*)a.hist_pre,
                         a.status[p & 1], nxt, a.ctr, a.sticky);
    }
}

void launch_sort(const SortArgs& a, cudaStream_t s, cudaEvent_t ev_after_hist)
{
    if (a.key_bytes == 2) sort_impl<unsigned short>(a, s, ev_after_hist);
    else if (a.key_bytes == 4) sort_impl<unsigned>(a, s, ev_after_hist);
    else sort_impl<unsigned long long>(a, s, ev_after_hist);
}

// ---------------------------------------------------------------------------
// Per-tile [start, end) ranges of the sorted entries (ranges zeroed beforehand).
// ---------------------------------------------------------------------------
template <typename K>
__device__ __forceinline__ void range_mark(uint2* ranges, long long ntiles, long long i, unsigned long long t,
                                           unsigned long long tprev, unsigned long long tnext, long long n)
{
    if (t >= (unsigned long long)ntiles) return; // only after a failed (timed-out) sort
    if (i == 0 || tprev != t) ranges[t].x = (unsigned)i;
    if (i == n - 1 || tnext != t) ranges[t].y = (unsigned)(i + 1);
}

// Each thread takes 16 bytes of consecutive keys and the key after them.
template <typename K>
__global__ void k_ranges(const K* __restrict__ keys, int tile_shift, long long ntiles, uint2* ranges,
                         const Counters* __restrict__ ctr)
{
    grid_dependency_wait();
    constexpr int V = 16 / sizeof(K);
    const long long n = ctr->n_entries;
    const long long nv = (n + V - 1) / V;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += (long long)gridDim.x * blockDim.x) {
        const long long i0 = j * V;
        unsigned long long t[V + 2];
        if (i0 + V <= n) {
            const uint4 q = __ldg(reinterpret_cast<const uint4*>(keys) + j);
            K k[V];
            memcpy(k, &q, 16);
#pragma unroll
            for (int u = 0; u < V; u++) t[u + 1] = (unsigned long long)k[u] >> tile_shift;
        } else {
#pragma unroll
            for (int u = 0; u < V; u++) t[u + 1] = (i0 + u < n) ? ((unsigned long long)keys[i0 + u] >> tile_shift) : ~0ull;
        }
        t[0] = i0 > 0 ? ((unsigned long long)keys[i0 - 1] >> tile_shift) : ~0ull;
        t[V + 1] = (i0 + V < n) ? ((unsigned long long)keys[i0 + V] >> tile_shift) : ~0ull;
#pragma unroll
        for (int u = 0; u < V; u++)
            if (i0 + u < n) range_mark<K>(ranges, ntiles, i0 + u, t[u + 1], t[u], t[u + 2], n);
    }
}

void launch_ranges(const RangeArgs& a, cudaStream_t s)
{
    const int grid = 8 * sm_count();
    if (a.key_bytes == 2)
        launch_dependent(k_ranges<unsigned short>, dim3(grid), dim3(256), 0, s, (const unsigned short*)a.keys, a.tile_shift,
                         a.ntiles, a.ranges, (const Counters*)a.ctr);
    else if (a.key_bytes == 4)
        launch_dependent(k_ranges<unsigned>, dim3(grid), dim3(256), 0, s, (const unsigned*)a.keys, a.tile_shift, a.ntiles,
                         a.ranges, (const Counters*)a.ctr);
    else
        launch_dependent(k_ranges<unsigned long long>, dim3(grid), dim3(256), 0, s, (const unsigned long long*)a.keys,
                         a.tile_shift, a.ntiles, a.ranges, (const Counters*)a.ctr);
}

} // namespace rg
