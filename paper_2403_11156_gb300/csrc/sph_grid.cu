// sph_grid.cu -- uniform-grid neighbour search: cell keys, counting sort with a
// single-pass decoupled look-back prefix sum (the "prefix sum" of Sec. 5.6), and the
// stable reorder of every per-particle field into (cell key, particle id) order so that
// the 27-cell neighbourhood of a particle is 9 contiguous index ranges.
#include <algorithm>

#include "sph_blocksort.cuh"
#include "sph_internal.cuh"

namespace sph {

namespace {

__device__ __forceinline__ uint32_t cell_of(const SceneDev &sc, float4 p)
{
    int32_t ix = cell_coord(p.x, sc.origin[0], sc.cell, sc.dims[0]);
    int32_t iy = cell_coord(p.y, sc.origin[1], sc.cell, sc.dims[1]);
    int32_t iz = cell_coord(p.z, sc.origin[2], sc.cell, sc.dims[2]);
    return (uint32_t)ix + (uint32_t)sc.dims[0] * ((uint32_t)iy + (uint32_t)sc.dims[1] * (uint32_t)iz);
}

// 1) key and histogram: one thread per particle of the source (canonical) order.
template <int WHAT>
__global__ void __launch_bounds__(kBlock) k_key_hist(Ptrs P)
{
    kernel_enter(P.ctl, (WHAT == SORT_FLUID ? KID_KEY_HIST_F : KID_KEY_HIST_B));
    const int32_t *tab = WHAT == SORT_FLUID ? P.fblk_scene : P.bblk_scene;
    const SceneDev &sc = P.scenes[tab[blockIdx.x]];
    const int32_t first = WHAT == SORT_FLUID ? sc.fblk_first : sc.bblk_first;
    const int64_t off = WHAT == SORT_FLUID ? sc.f_off : sc.b_off;
    const int64_t n = WHAT == SORT_FLUID ? sc.nf : sc.nb;
    if (blockIdx.x == 0 && threadIdx.x == 0) P.ctl->nlarge[WHAT] = 0;   // this sort's crowded cells
    const int64_t local = (int64_t)(blockIdx.x - first) * kBlock + threadIdx.x;
    if (local >= n) return;
    const int64_t i = off + local;
    float4 p = WHAT == SORT_FLUID ? P.pos_c[i] : P.bx_o[i];
    uint32_t cell = (uint32_t)sc.c_off + cell_of(sc, p);
    uint32_t *count = WHAT == SORT_FLUID ? P.cell_count : P.bcell_count;
    uint32_t slot = atomicAdd(&count[cell], 1u);
    (WHAT == SORT_FLUID ? P.key_tmp : P.bkey_tmp)[i] = cell;
    (WHAT == SORT_FLUID ? P.slot_tmp : P.bslot_tmp)[i] = slot;
}

// 3) scatter into the cell's range (order inside a cell not yet fixed).
template <int WHAT>
__global__ void __launch_bounds__(kBlock) k_scatter(Ptrs P)
{
    kernel_enter(P.ctl, (WHAT == SORT_FLUID ? KID_SCATTER_F : KID_SCATTER_B));
    const int32_t *tab = WHAT == SORT_FLUID ? P.fblk_scene : P.bblk_scene;
    const SceneDev &sc = P.scenes[tab[blockIdx.x]];
    const int32_t first = WHAT == SORT_FLUID ? sc.fblk_first : sc.bblk_first;
    const int64_t off = WHAT == SORT_FLUID ? sc.f_off : sc.b_off;
    const int64_t n = WHAT == SORT_FLUID ? sc.nf : sc.nb;
    const int64_t local = (int64_t)(blockIdx.x - first) * kBlock + threadIdx.x;
    if (local >= n) return;
    const int64_t i = off + local;
    uint32_t cell = (WHAT == SORT_FLUID ? P.key_tmp : P.bkey_tmp)[i];
    uint32_t slot = (WHAT == SORT_FLUID ? P.slot_tmp : P.bslot_tmp)[i];
    const uint32_t *start = WHAT == SORT_FLUID ? P.cell_start : P.bcell_start;
    uint32_t s = start[cell] + slot;
    uint32_t id = WHAT == SORT_FLUID ? (uint32_t)P.id_c[i] : (uint32_t)local;
    (WHAT == SORT_FLUID ? P.sid_tmp : P.bsid_tmp)[s] = id;
    (WHAT == SORT_FLUID ? P.src_tmp : P.bsrc_tmp)[s] = (uint32_t)i;
    (WHAT == SORT_FLUID ? P.cell_tmp : P.bcell_tmp)[s] = cell;
}

// Copy particle src of the canonical (or original boundary) arrays to sorted slot d.
template <int WHAT>
__device__ __forceinline__ void gather_one(const Ptrs &P, uint32_t d, uint32_t src, uint32_t id)
{
    if (WHAT == SORT_FLUID) {
        float4 p = P.pos_c[src];
        p.w = 0.0f;
        P.pos_s[d] = p;
        P.vel_s[d] = P.vel_c[src];
        P.kprev_s[d] = P.kprev_c[src];
        P.kvprev_s[d] = P.kvprev_c[src];
        P.id_s[d] = (int32_t)id;
    } else {
        float4 p = P.bx_o[src];
        p.w = 0.0f;
        P.bpos_s[d] = p;
        P.bvel_s[d] = P.bv_o[src];
        P.bid_s[d] = (int32_t)id;
        P.bbody_s[d] = P.bbody[src];
    }
}

// 4) rank inside the cell by original id (deterministic (key, id) order) and gather.  A
// cell of more than kRankSmall particles is queued for k_rank_large instead.
template <int WHAT>
__global__ void __launch_bounds__(kBlock) k_rank_gather(Ptrs P)
{
    kernel_enter(P.ctl, (WHAT == SORT_FLUID ? KID_RANK_F : KID_RANK_B));
    const int32_t *tab = WHAT == SORT_FLUID ? P.fblk_scene : P.bblk_scene;
    const SceneDev &sc = P.scenes[tab[blockIdx.x]];
    const int32_t first = WHAT == SORT_FLUID ? sc.fblk_first : sc.bblk_first;
    const int64_t off = WHAT == SORT_FLUID ? sc.f_off : sc.b_off;
    const int64_t n = WHAT == SORT_FLUID ? sc.nf : sc.nb;
    const int64_t local = (int64_t)(blockIdx.x - first) * kBlock + threadIdx.x;
    if (local >= n) return;
    const int64_t s = off + local;
    const uint32_t *sid = WHAT == SORT_FLUID ? P.sid_tmp : P.bsid_tmp;
    const uint32_t *start = WHAT == SORT_FLUID ? P.cell_start : P.bcell_start;
    uint32_t cell = (WHAT == SORT_FLUID ? P.cell_tmp : P.bcell_tmp)[s];
    uint32_t b = start[cell], e = start[cell + 1];
    if (e - b > kRankSmall) {
        if ((uint32_t)s == b) {
            const int q = atomicAdd(&P.ctl->nlarge[WHAT], 1);
            (WHAT == SORT_FLUID ? P.large_f : P.large_b)[q] = cell;
        }
        return;
    }
    uint32_t my = sid[s];
    uint32_t rank = 0;
    for (uint32_t t = b; t < e; ++t) rank += (sid[t] < my) ? 1u : 0u;
    gather_one<WHAT>(P, b + rank, (WHAT == SORT_FLUID ? P.src_tmp : P.bsrc_tmp)[s], my);
}

// 5) the queued crowded cells: each block takes cells of the queue in turn, sorts the
// cell's (id, source) pairs stably by id and gathers them (the key and slot arrays, free
// once scattered, are the sort's scratch).  Exits at once when no cell was queued.
template <int WHAT>
__global__ void __launch_bounds__(kLargeThreads) k_rank_large(Ptrs P)
{
    kernel_enter(P.ctl, (WHAT == SORT_FLUID ? KID_RANK_LARGE_F : KID_RANK_LARGE_B));
    const int nq = *reinterpret_cast<volatile int32_t *>(&P.ctl->nlarge[WHAT]);
    const uint32_t *large = WHAT == SORT_FLUID ? P.large_f : P.large_b;
    const uint32_t *start = WHAT == SORT_FLUID ? P.cell_start : P.bcell_start;
    uint32_t *sid = WHAT == SORT_FLUID ? P.sid_tmp : P.bsid_tmp;
    uint32_t *src = WHAT == SORT_FLUID ? P.src_tmp : P.bsrc_tmp;
    uint32_t *sid2 = WHAT == SORT_FLUID ? P.key_tmp : P.bkey_tmp;
    uint32_t *src2 = WHAT == SORT_FLUID ? P.slot_tmp : P.bslot_tmp;
    for (int q = blockIdx.x; q < nq; q += gridDim.x) {
        const uint32_t cell = large[q];
        const uint32_t b = start[cell], e = start[cell + 1];
        block_sort_segment(sid, src, sid2, src2, b, e);
        for (uint32_t d = b + threadIdx.x; d < e; d += kLargeThreads) gather_one<WHAT>(P, d, src[d], sid[d]);
        __syncthreads();
    }
}

// 2) exclusive prefix sum of the cell counts, single pass (decoupled look-back).
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr uint64_t kFlagAgg = 1, kFlagIncl = 2;
constexpr int kSpinLimit = 1 << 22;

__device__ __forceinline__ uint64_t ld_acquire(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint64_t *p, uint64_t v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__global__ void __launch_bounds__(kScanThreads) k_scan(uint32_t *count, uint32_t *start, int64_t n,
                                                       uint64_t *status, int32_t tiles, ScanCtl *sc, Control *ctl)
{
    __shared__ int32_t s_tile;
    __shared__ uint32_t s_epoch;
    __shared__ uint32_t s_warp[kScanThreads / 32];
    __shared__ uint32_t s_prefix;
    kernel_enter(ctl, KID_SCAN);
    if (threadIdx.x == 0) {
        s_tile = atomicAdd(&sc->tile_counter, 1);
        s_epoch = *reinterpret_cast<volatile uint32_t *>(&sc->epoch);
    }
    __syncthreads();
    const int32_t tile = s_tile;
    const uint64_t epoch = s_epoch & 0x3fffffffu;
    const int64_t base = (int64_t)tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t idx = base + k;
        v[k] = idx < n ? count[idx] : 0u;
    }
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t idx = base + k;
        if (idx < n) count[idx] = 0u;      // histogram is consumed: reset for the next sort
    }
    uint32_t tsum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) tsum += v[k];
    // block exclusive scan of the per-thread sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kScanThreads / 32 ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kScanThreads / 32) s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t warp_excl = warp > 0 ? s_warp[warp - 1] : 0u;
    const uint32_t agg = s_warp[kScanThreads / 32 - 1];
    uint32_t texcl = warp_excl + x - tsum;
    if (threadIdx.x == 0) {
        uint32_t prefix = 0;
        if (tile == 0) {
            st_release(&status[0], (epoch << 34) | (kFlagIncl << 32) | agg);
        } else {
            st_release(&status[tile], (epoch << 34) | (kFlagAgg << 32) | agg);
            int32_t t = tile - 1;
            int spins = 0;
            while (t >= 0) {
                uint64_t w = ld_acquire(&status[t]);
                uint64_t f = (w >> 32) & 3u;
                if ((w >> 34) != epoch || f == 0) {
                    if (++spins > kSpinLimit) {       // predecessor never published
                        atomicExch(&ctl->error, 1);
                        break;
                    }
                    __nanosleep(32);
                    continue;
                }
                prefix += (uint32_t)(w & 0xffffffffu);
                if (f == kFlagIncl) break;
                --t;
            }
            st_release(&status[tile], (epoch << 34) | (kFlagIncl << 32) | (uint32_t)(prefix + agg));
        }
        s_prefix = prefix;
    }
    __syncthreads();
    uint32_t run = s_prefix + texcl;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t idx = base + k;
        if (idx < n) start[idx] = run;
        run += v[k];
    }
    if (base <= n - 1 && n - 1 < base + kScanItems) start[n] = s_prefix + agg;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&sc->done, 1) == tiles - 1) {
            sc->tile_counter = 0;
            sc->done = 0;
            uint32_t e = (s_epoch + 1u) & 0x3fffffffu;
            sc->epoch = e == 0 ? 1u : e;
            __threadfence();
        }
    }
}

}  // namespace

int32_t scan_tiles_for(int64_t n) { return (int32_t)((n + kScanTile - 1) / kScanTile); }
int64_t large_capacity(int64_t n) { return n / (kRankSmall + 1) + 1; }

void launch_scan(uint32_t *count, uint32_t *start, int64_t n, uint64_t *status, int32_t tiles,
                 ScanCtl *sc, Control *ctl, cudaStream_t s)
{
    if (n <= 0 || tiles <= 0) return;
    k_scan<<<tiles, kScanThreads, 0, s>>>(count, start, n, status, tiles, sc, ctl);
}

void launch_key_hist(const Ptrs &P, SortWhat what, cudaStream_t s)
{
    if (what == SORT_FLUID) {
        if (P.nfblk) k_key_hist<SORT_FLUID><<<P.nfblk, kBlock, 0, s>>>(P);
    } else if (P.nbblk) {
        k_key_hist<SORT_BOUNDARY><<<P.nbblk, kBlock, 0, s>>>(P);
    }
}
void launch_scan_cells(const Ptrs &P, SortWhat what, cudaStream_t s)
{
    if (what == SORT_FLUID) {
        if (P.nfblk)
            launch_scan(P.cell_count, P.cell_start, P.NC, P.scan_status, scan_tiles_for(P.NC), &P.ctl->scan[0],
                        P.ctl, s);
    } else if (P.nbblk) {
        launch_scan(P.bcell_count, P.bcell_start, P.NC, P.bscan_status, scan_tiles_for(P.NC), &P.ctl->scan[1],
                    P.ctl, s);
    }
}
void launch_scatter(const Ptrs &P, SortWhat what, cudaStream_t s)
{
    if (what == SORT_FLUID) {
        if (P.nfblk) k_scatter<SORT_FLUID><<<P.nfblk, kBlock, 0, s>>>(P);
    } else if (P.nbblk) {
        k_scatter<SORT_BOUNDARY><<<P.nbblk, kBlock, 0, s>>>(P);
    }
}
void launch_rank_gather(const Ptrs &P, SortWhat what, cudaStream_t s)
{
    // the crowded-cell pass takes as many blocks as cells could be queued, up to one per SM
    if (what == SORT_FLUID) {
        if (P.nfblk) {
            k_rank_gather<SORT_FLUID><<<P.nfblk, kBlock, 0, s>>>(P);
            k_rank_large<SORT_FLUID><<<(int)std::min<int64_t>(large_capacity(P.NF), 152), kLargeThreads, 0, s>>>(P);
        }
    } else if (P.nbblk) {
        k_rank_gather<SORT_BOUNDARY><<<P.nbblk, kBlock, 0, s>>>(P);
        k_rank_large<SORT_BOUNDARY><<<(int)std::min<int64_t>(large_capacity(P.NB), 152), kLargeThreads, 0, s>>>(P);
    }
}

}  // namespace sph
