// sort_noalloc.cu -- rg_sort_pairs_noalloc: the renderer's stable radix sort of
// (uint32 key, uint32 value) pairs on caller buffers, with every byte of scratch
// memory taken from one static device array instead of an allocation.
//
// Who needs this: code that must not call cudaMalloc -- a render loop on a
// real-time thread (cudaMalloc can block on, or synchronise with, the device),
// a plugin whose host application owns all device memory through its own
// allocator, or a caller that records work into CUDA graphs and wants no
// allocation inside the recorded region. They pass their own key and value
// arrays; the sort's alternate buffers, digit histograms, look-back status
// words and counters live in g_noalloc_scratch below.
#include <cstdint>
#include <mutex>

#include "rg.h"
#include "rg_internal.cuh"

using namespace rg;

namespace {

constexpr long long NA_MAX = 1ll << 19;     // at most 524,288 pairs per call
constexpr long long NA_TILE = 4096;         // smallest sort tile the status arrays are sized for
constexpr long long NA_TILES = NA_MAX / NA_TILE;
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t OFF_KEYS = 0;
constexpr size_t OFF_VALS = OFF_KEYS + align256(NA_MAX * 4);
constexpr size_t OFF_STATUS0 = OFF_VALS + align256(NA_MAX * 4);
constexpr size_t OFF_STATUS1 = OFF_STATUS0 + align256(NA_TILES * 256 * 4);
constexpr size_t OFF_CTRL = OFF_STATUS1 + align256(NA_TILES * 256 * 4);
constexpr size_t CTRL_BYTES = sizeof(Counters) + 8 * 256 * sizeof(unsigned);
constexpr size_t OFF_STICKY = OFF_CTRL + align256(CTRL_BYTES);
constexpr size_t SCRATCH_BYTES = OFF_STICKY + align256(sizeof(Sticky)); // about 4.3 MiB

constexpr int MAX_DEVICES = 64;

std::mutex g_mu;
unsigned char* g_scratch[MAX_DEVICES] = {nullptr};

rg_status na_fail(rg_status s, const char* msg)
{
    set_last_error(msg); // reported by rg_last_error()
    return s;
}

} // namespace

// The scratch array. Every GPU that loads the library holds it until the
// process exits; every call on a device uses the same bytes.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

// Clear the counters, histograms and sticky flags; store the pair count.
__global__ void k_noalloc_begin(unsigned n)
{
    unsigned* ctrl = reinterpret_cast<unsigned*>(g_noalloc_scratch + OFF_CTRL);
    for (unsigned j = threadIdx.x; j < CTRL_BYTES / 4; j += blockDim.x) ctrl[j] = 0u;
    unsigned* st = reinterpret_cast<unsigned*>(g_noalloc_scratch + OFF_STICKY);
    if (threadIdx.x < sizeof(Sticky) / 4) st[threadIdx.x] = 0u;
    __syncthreads();
    if (threadIdx.x == 0) reinterpret_cast<Counters*>(ctrl)->n_entries = n;
}

// Copy the error bits of the bounded look-back waits to the caller's flag.
__global__ void k_noalloc_end(unsigned* error_out)
{
    const Counters* c = reinterpret_cast<const Counters*>(g_noalloc_scratch + OFF_CTRL);
    const Sticky* s = reinterpret_cast<const Sticky*>(g_noalloc_scratch + OFF_STICKY);
    *error_out = c->error | s->error;
}

extern "C" rg_status rg_sort_pairs_noalloc(uint32_t* keys, uint32_t* vals, int64_t n, int32_t key_bits,
                                           uint32_t* error_dev, void* stream)
{
    if (n < 0 || n > NA_MAX) return na_fail(RG_ERR_INVALID_ARG, "rg_sort_pairs_noalloc: n must be in [0, 524288]");
    if (n > 0 && (!keys || !vals)) return na_fail(RG_ERR_INVALID_ARG, "rg_sort_pairs_noalloc: keys or vals is NULL");
    // the histogram kernel reads the keys 16 bytes at a time
    if (n > 0 && ((reinterpret_cast<uintptr_t>(keys) | reinterpret_cast<uintptr_t>(vals)) & 15u))
        return na_fail(RG_ERR_INVALID_ARG, "rg_sort_pairs_noalloc: keys and vals must be 16-byte aligned");
    if (key_bits != 8 && key_bits != 16 && key_bits != 24 && key_bits != 32)
        return na_fail(RG_ERR_INVALID_ARG, "rg_sort_pairs_noalloc: key_bits must be 8, 16, 24 or 32");
    if (sort_tile_items() < NA_TILE) return na_fail(RG_ERR_CUDA, "rg_sort_pairs_noalloc: sort tile below the sized minimum");
    // an error left by an earlier, unrelated launch is not this call's: report it and leave
    // it pending for its owner
    if (cudaPeekAtLastError() != cudaSuccess)
        return na_fail(RG_ERR_CUDA, "rg_sort_pairs_noalloc: a CUDA error from an earlier call is pending");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
        return na_fail(RG_ERR_CUDA, "rg_sort_pairs_noalloc: no usable current device");
    unsigned char* base;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch[dev]) { // once per device, with that device current
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return na_fail(RG_ERR_CUDA, "rg_sort_pairs_noalloc: cudaGetSymbolAddress failed");
            }
            g_scratch[dev] = reinterpret_cast<unsigned char*>(p);
        }
        base = g_scratch[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    k_noalloc_begin<<<1, 256, 0, st>>>((unsigned)n);
    SortArgs a;
    memset(&a, 0, sizeof(a));
    a.keys[0] = keys;
    a.keys[1] = base + OFF_KEYS;
    a.vals[0] = vals;
    a.vals[1] = reinterpret_cast<unsigned*>(base + OFF_VALS);
    a.cap = NA_MAX;
    a.key_bytes = 4;
    a.passes = key_bits / 8;
    // arbitrary keys hold many distinct digits per warp: every pass ranks with the peer masks
    a.rank_modes = sort_rank_modes(SORT_RANK_PEERS, SORT_RANK_PEERS, SORT_RANK_PEERS, SORT_RANK_PEERS);
    a.hist = reinterpret_cast<unsigned*>(base + OFF_CTRL + sizeof(Counters));
    a.status[0] = reinterpret_cast<unsigned*>(base + OFF_STATUS0);
    a.status[1] = reinterpret_cast<unsigned*>(base + OFF_STATUS1);
    a.max_tiles = NA_TILES;
    a.ctr = reinterpret_cast<Counters*>(base + OFF_CTRL);
    a.sticky = reinterpret_cast<Sticky*>(base + OFF_STICKY);
    launch_sort(a, st, nullptr);
    if ((a.passes & 1) && n > 0) { // an odd pass count leaves the result in the scratch copy
        if (cudaMemcpyAsync(keys, a.keys[1], (size_t)n * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(vals, a.vals[1], (size_t)n * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
            cudaGetLastError();
            return na_fail(RG_ERR_CUDA, "rg_sort_pairs_noalloc: copy back failed");
        }
    }
    if (error_dev) k_noalloc_end<<<1, 1, 0, st>>>(error_dev);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(RG_ERR_CUDA, cudaGetErrorString(e));
    return RG_OK;
}
