// sph_noalloc.cu -- grid order of a point set without any memory allocation.
//
// Some callers cannot let a library allocate device memory: code that enqueues work while
// another component is capturing a CUDA graph (cudaMalloc is not permitted inside such a
// capture), host applications such as rendering or game engines and plugins that own the
// GPU's memory budget and forbid libraries from allocating, and real-time loops in which
// an allocation's latency or a possible out-of-memory failure is not acceptable.  For them
// sph_grid_order_noalloc runs the same counting sort as the per-step neighbour search
// (cell keys, histogram, decoupled look-back prefix sum, scatter, rank by index, with the
// crowded cells sorted by one block each) with its scratch in one file-scope static device
// array of fixed size, which every GPU that loads the library holds until the process
// exits.
#include "sph.h"
#include "sph_blocksort.cuh"
#include "sph_internal.cuh"

#include <cmath>
#include <cstddef>
#include <mutex>

using namespace sph;

namespace {

constexpr int64_t kMaxPoints = SPH_NOALLOC_MAX_POINTS;
constexpr int64_t kMaxCells = SPH_NOALLOC_MAX_CELLS;
constexpr int64_t kMaxTiles = (kMaxCells + 2047) / 2048;

// Byte offsets of the scratch regions (each a multiple of 256).
constexpr size_t kOffCount = 0;                                          // u32 [kMaxCells]
constexpr size_t kOffStart = kOffCount + 4 * kMaxCells;                  // u32 [kMaxCells + 1]
constexpr size_t kOffKey = kOffStart + ((4 * (kMaxCells + 1) + 255) / 256) * 256;  // u32 [kMaxPoints]
constexpr size_t kOffSlot = kOffKey + 4 * kMaxPoints;                    // u32 [kMaxPoints]
constexpr size_t kOffSid = kOffSlot + 4 * kMaxPoints;                    // u32 [kMaxPoints]
constexpr size_t kOffCell = kOffSid + 4 * kMaxPoints;                    // u32 [kMaxPoints]
constexpr size_t kOffStatus = kOffCell + 4 * kMaxPoints;                 // u64 [kMaxTiles]
constexpr size_t kOffCtl = kOffStatus + ((8 * kMaxTiles + 255) / 256) * 256;  // Control
constexpr int64_t kMaxLarge = kMaxPoints / (kRankSmall + 1) + 1;
constexpr size_t kOffLarge = kOffCtl + ((sizeof(Control) + 255) / 256) * 256;  // u32 [kMaxLarge]
constexpr size_t kScratchBytes = kOffLarge + ((4 * kMaxLarge + 255) / 256) * 256;

static __device__ __align__(256) unsigned char g_grid_scratch[kScratchBytes];

struct View {
    uint32_t *count, *start, *key, *slot, *sid, *cell;
    uint64_t *status;
    Control *ctl;
    uint32_t *large;
};

View carve(unsigned char *base)
{
    View v;
    v.count = reinterpret_cast<uint32_t *>(base + kOffCount);
    v.start = reinterpret_cast<uint32_t *>(base + kOffStart);
    v.key = reinterpret_cast<uint32_t *>(base + kOffKey);
    v.slot = reinterpret_cast<uint32_t *>(base + kOffSlot);
    v.sid = reinterpret_cast<uint32_t *>(base + kOffSid);
    v.cell = reinterpret_cast<uint32_t *>(base + kOffCell);
    v.status = reinterpret_cast<uint64_t *>(base + kOffStatus);
    v.ctl = reinterpret_cast<Control *>(base + kOffCtl);
    v.large = reinterpret_cast<uint32_t *>(base + kOffLarge);
    return v;
}

struct Grid {
    float origin[3], cell;
    int32_t dims[3];
};

// Everything that must start at zero: the histogram, the look-back tile words and the
// scan's control counters (the array keeps whatever the previous call left there).
__global__ void k_na_clear(View v, int64_t ncell, int32_t tiles)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = k; c < ncell; c += stride) v.count[c] = 0u;
    for (int64_t t = k; t < tiles; t += stride) v.status[t] = 0ull;
    if (k == 0) {
        v.ctl->scan[0].tile_counter = 0;
        v.ctl->scan[0].done = 0;
        v.ctl->scan[0].epoch = 0;
        v.ctl->error = 0;
        v.ctl->nlarge[0] = 0;
    }
}

__global__ void k_na_key_hist(View v, Grid g, const float *x, int64_t n, uint32_t *keys_out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t ix = cell_coord(x[3 * i + 0], g.origin[0], g.cell, g.dims[0]);
    int32_t iy = cell_coord(x[3 * i + 1], g.origin[1], g.cell, g.dims[1]);
    int32_t iz = cell_coord(x[3 * i + 2], g.origin[2], g.cell, g.dims[2]);
    uint32_t key = (uint32_t)ix + (uint32_t)g.dims[0] * ((uint32_t)iy + (uint32_t)g.dims[1] * (uint32_t)iz);
    v.key[i] = key;
    v.slot[i] = atomicAdd(&v.count[key], 1u);
    if (keys_out) keys_out[i] = key;
}

__global__ void k_na_scatter(View v, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t key = v.key[i];
    uint32_t s = v.start[key] + v.slot[i];
    v.sid[s] = (uint32_t)i;
    v.cell[s] = key;
}

// Rank inside the cell by counting the cell's smaller indices; a cell of more than
// kRankSmall points is queued for k_na_rank_large instead.
__global__ void k_na_rank(View v, int64_t n, int32_t *order)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    uint32_t c = v.cell[s];
    uint32_t b = v.start[c], e = v.start[c + 1];
    if (e - b > kRankSmall) {
        if ((uint32_t)s == b) v.large[atomicAdd(&v.ctl->nlarge[0], 1)] = c;
        return;
    }
    uint32_t my = v.sid[s];
    uint32_t rank = 0;
    for (uint32_t t = b; t < e; ++t) rank += (v.sid[t] < my) ? 1u : 0u;
    order[b + rank] = (int32_t)my;
}

// The queued crowded cells: one block per cell at a time sorts the cell's indices stably
// (the key and slot regions, free once scattered, are its scratch) and writes them out.
__global__ void __launch_bounds__(kLargeThreads) k_na_rank_large(View v, int32_t *order)
{
    const int nq = *reinterpret_cast<volatile int32_t *>(&v.ctl->nlarge[0]);
    for (int q = blockIdx.x; q < nq; q += gridDim.x) {
        const uint32_t c = v.large[q];
        const uint32_t b = v.start[c], e = v.start[c + 1];
        block_sort_segment(v.sid, v.cell, v.key, v.slot, b, e);
        for (uint32_t d = b + threadIdx.x; d < e; d += kLargeThreads) order[d] = (int32_t)v.sid[d];
        __syncthreads();
    }
}

std::mutex g_mu;
unsigned char *g_base[256] = {};

}  // namespace

extern "C" sph_status sph_grid_order_noalloc(const float *x, int64_t n, const float *domain_min,
                                             const float *domain_max, float cell_size, int32_t *order,
                                             uint32_t *keys, void *stream)
{
    if (n < 0 || n > kMaxPoints) return SPH_EINVAL;
    if (n > 0 && (!x || !order)) return SPH_EINVAL;
    if (!domain_min || !domain_max || !(cell_size > 0.0f) || !std::isfinite(cell_size)) return SPH_EINVAL;
    Grid g;
    g.cell = cell_size;
    int64_t ncell = 1;
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(domain_min[a]) || !std::isfinite(domain_max[a]) || !(domain_max[a] > domain_min[a]))
            return SPH_EINVAL;
        g.origin[a] = domain_min[a] - cell_size;
        float ext = (domain_max[a] - domain_min[a]) / cell_size;
        if (!(ext < 1e7f)) return SPH_EINVAL;
        g.dims[a] = (int32_t)std::ceil(ext) + 2;
        ncell *= g.dims[a];
        if (ncell > kMaxCells) return SPH_EINVAL;
    }
    if (n == 0) return SPH_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return SPH_ECUDA;
    unsigned char *base;
    {
        // once per device, with that device current: the device address of the array
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_base[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_grid_scratch) != cudaSuccess || !p) return SPH_ECUDA;
            g_base[dev] = static_cast<unsigned char *>(p);
        }
        base = g_base[dev];
    }
    View v = carve(base);
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t tiles = scan_tiles_for(ncell);
    const int t = 256;
    const int bp = (int)((n + t - 1) / t);
    k_na_clear<<<(int)std::min<int64_t>((ncell + t - 1) / t, 1184), t, 0, s>>>(v, ncell, tiles);
    k_na_key_hist<<<bp, t, 0, s>>>(v, g, x, n, keys);
    launch_scan(v.count, v.start, ncell, v.status, tiles, &v.ctl->scan[0], v.ctl, s);
    k_na_scatter<<<bp, t, 0, s>>>(v, n);
    k_na_rank<<<bp, t, 0, s>>>(v, n, order);
    k_na_rank_large<<<(int)std::min<int64_t>(n / (kRankSmall + 1) + 1, 152), kLargeThreads, 0, s>>>(v, order);
    return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ECUDA;
}

extern "C" sph_status sph_grid_order_noalloc_status(void *stream)
{
    // the scan's bounded waits record a timeout in the scratch's control word, which each
    // call clears before its scan: read it back once the stream's work is done (a copy
    // from the symbol into a host integer, nothing allocated)
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return SPH_ECUDA;
    int32_t err = 0;
    const size_t off = kOffCtl + offsetof(Control, error);
    if (cudaMemcpyFromSymbol(&err, g_grid_scratch, sizeof(err), off, cudaMemcpyDeviceToHost) != cudaSuccess)
        return SPH_ECUDA;
    return err != 0 ? SPH_ETIMEOUT : SPH_OK;
}
