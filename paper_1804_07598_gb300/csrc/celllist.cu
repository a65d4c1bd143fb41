// celllist.cu -- cell-list build: wrap -> cell index -> stable counting sort
// -> exclusive scan -> reorder (cell lists, Sec. 2; cache-friendly re-sorting,
// Sec. 3.6; getCellListSym / updateCellListSym of Listing 4.1).
//
// Kernels (one launch each, all gated by d_gate):
//   k_zero       count[ncell] = 0
//   k_bin        wrap, cell id, warp-aggregated histogram; the atomic returns
//                each particle's arrival rank inside its cell
//   k_scan_part  per-tile sums of count (4096 cells per tile)
//   k_scan_final exclusive scan -> cell_start
//   k_scatter    tmp[cell_start[c] + rank] = i (arrival order inside a cell)
//   k_sort_gather one warp per cell sorts the cell's slice of tmp by input
//                index (this makes the sort stable and deterministic), writes
//                perm and gathers pos / vel / id into sorted order; on sparse
//                grids k_sort_gather_sparse gives small cells a lane each
#include <climits>

#include "fpm_common.cuh"

namespace fpm {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

struct CellWs {
    size_t off_pos, off_vel, off_id, off_cell, off_rank, off_tmp, off_count, off_tiles, total;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static CellWs cell_ws_layout(int64_t n, int64_t ncell, size_t v4bytes)
{
    CellWs w{};
    size_t o = 0;
    w.off_pos = o; o = align256(o + (size_t)n * v4bytes);
    w.off_vel = o; o = align256(o + (size_t)n * v4bytes);
    w.off_id = o; o = align256(o + (size_t)n * 4);
    w.off_cell = o; o = align256(o + (size_t)n * 4);
    w.off_rank = o; o = align256(o + (size_t)n * 4);
    w.off_tmp = o; o = align256(o + (size_t)n * 4);
    w.off_count = o; o = align256(o + (size_t)ncell * 4);
    w.off_tiles = o; o = align256(o + (size_t)((ncell + kScanTile - 1) / kScanTile + 1) * 4);
    w.total = o;
    return w;
}

__global__ void k_zero(uint32_t *p, int64_t m, const uint32_t *gate)
{
    if (gated_off(gate)) return;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        p[k] = 0u;
}

template <typename T>
__global__ void k_bin(BoxT<T> box, GridD grid, int n, const V4<T> *__restrict__ pos_in,
                      const V4<T> *__restrict__ vel_in, const uint32_t *__restrict__ id_in,
                      V4<T> *stage_pos, V4<T> *stage_vel, uint32_t *stage_id, uint32_t *__restrict__ cell,
                      uint32_t *__restrict__ rank, uint32_t *count, fpm_dev_status *st, const uint32_t *gate)
{
    if (gated_off(gate)) return;
    // grid-stride; the loop bound is uniform per block, so whole warps
    // iterate together (the aggregated atomic below needs that)
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(base + threadIdx.x);
        const bool live = i < n;
        uint32_t c = UINT_MAX;
        if (live) {
            V4<T> p = pos_in[i];
            if (box.per[0]) p.x = wrap1(p.x, box.L[0]);
            if (box.per[1]) p.y = wrap1(p.y, box.L[1]);
            if (box.per[2]) p.z = wrap1(p.z, box.L[2]);
            bool bad = false;
            int cc[3];
            cell_of(p, box, grid, cc, bad);
            if (bad) {
                latch_flag(st, FPM_FLAG_DOMAIN);
                if (st) atomicExch(&st->bad_index, (uint32_t)i);
            }
            c = linear_cell(cc[0], cc[1], cc[2], grid);
            cell[i] = c;
            if (stage_pos) stage_pos[i] = p;
            if (stage_vel) stage_vel[i] = vel_in[i];
            if (stage_id) stage_id[i] = id_in ? id_in[i] : (uint32_t)i;
        }
        // warp-aggregated histogram: one atomic per distinct cell in the warp
        const unsigned lane = threadIdx.x & 31;
        const unsigned act = __ballot_sync(kFull, live);
        if (live) {
            const unsigned peers = __match_any_sync(act, c);
            const int leader = __ffs(peers) - 1;
            const unsigned below = peers & ((1u << lane) - 1u);
            uint32_t b = 0;
            if ((int)lane == leader) b = atomicAdd(&count[c], (uint32_t)__popc(peers));
            b = __shfl_sync(peers, b, leader);
            rank[i] = b + (uint32_t)__popc(below);
        }
    }
}

// Inclusive scan of one value per thread across a 1024-thread block.
__device__ __forceinline__ uint32_t block_inclusive_scan(uint32_t v, uint32_t *sh32, uint32_t &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) sh32[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = sh32[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += t;
        }
        sh32[lane] = w;
    }
    __syncthreads();
    total = sh32[31];
    uint32_t r = v + (warp > 0 ? sh32[warp - 1] : 0u);
    __syncthreads();
    return r;
}

// count[base .. base + 4) (zero past ncell): one 16-byte load when all four
// exist (count is 256-byte aligned and base a multiple of 4).
__device__ __forceinline__ void load_counts(const uint32_t *count, int ncell, int64_t base, uint32_t (&v)[kScanItems])
{
    static_assert(kScanItems == 4, "one uint4 per thread");
    if (base + kScanItems <= ncell) {
        const uint4 q = *reinterpret_cast<const uint4 *>(count + base);
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) v[k] = (base + k < ncell) ? count[base + k] : 0u;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_part(const uint32_t *count, int ncell, uint32_t *tiles,
                                                            const uint32_t *gate)
{
    if (gated_off(gate)) return;
    __shared__ uint32_t sh[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    load_counts(count, ncell, base, v);
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) s += v[k];
    uint32_t total;
    block_inclusive_scan(s, sh, total);
    if (threadIdx.x == 0) tiles[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_final(const uint32_t *count, int ncell, const uint32_t *tiles,
                                                             uint32_t *cell_start, int n, const uint32_t *gate)
{
    if (gated_off(gate)) return;
    __shared__ uint32_t sh[32];
    __shared__ uint32_t tile_off;
    // offset of this tile = sum of the previous tiles' totals
    uint32_t part = 0;
    for (int t = threadIdx.x; t < (int)blockIdx.x; t += blockDim.x) part += tiles[t];
    uint32_t tot;
    block_inclusive_scan(part, sh, tot);
    if (threadIdx.x == 0) tile_off = tot;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    load_counts(count, ncell, base, v);
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) s += v[k];
    uint32_t total;
    uint32_t incl = block_inclusive_scan(s, sh, total);
    uint32_t run = tile_off + incl - s;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < ncell) cell_start[base + k] = run;
        run += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) cell_start[ncell] = (uint32_t)n;
}

__global__ void k_scatter(int n, const uint32_t *__restrict__ cell, const uint32_t *__restrict__ rank,
                          const uint32_t *__restrict__ cell_start, uint32_t *__restrict__ tmp, const uint32_t *gate)
{
    if (gated_off(gate)) return;
    // four particles per thread from 16-byte loads of cell and rank (both
    // 256-byte aligned), then the tail
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n4 = n >> 2;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += stride) {
        const uint4 c = reinterpret_cast<const uint4 *>(cell)[q];
        const uint4 r = reinterpret_cast<const uint4 *>(rank)[q];
        const uint32_t i = (uint32_t)(q << 2);
        tmp[cell_start[c.x] + r.x] = i;
        tmp[cell_start[c.y] + r.y] = i + 1u;
        tmp[cell_start[c.z] + r.z] = i + 2u;
        tmp[cell_start[c.w] + r.w] = i + 3u;
    }
    for (int64_t i = (n4 << 2) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        tmp[cell_start[cell[i]] + rank[i]] = (uint32_t)i;
}

// Ascending bitonic sort of one value per lane across a full warp.
__device__ __forceinline__ uint32_t warp_sort32(uint32_t v)
{
    const unsigned lane = threadIdx.x & 31;
#pragma unroll
    for (unsigned k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (unsigned j = k >> 1; j > 0; j >>= 1) {
            uint32_t o = __shfl_xor_sync(kFull, v, j);
            bool up = (lane & k) == 0;
            bool low = (lane & j) == 0;
            v = (low == up) ? min(v, o) : max(v, o);
        }
    }
    return v;
}

template <typename T>
__device__ __forceinline__ void emit(uint32_t slot, uint32_t src, const BoxT<T> &box, const V4<T> *pos_src,
                                     const V4<T> *vel_src, const uint32_t *id_src, V4<T> *pos_out, V4<T> *vel_out,
                                     uint32_t *id_out, uint32_t *perm)
{
    V4<T> p = pos_src[src];
    if (box.per[0]) p.x = wrap1(p.x, box.L[0]);
    if (box.per[1]) p.y = wrap1(p.y, box.L[1]);
    if (box.per[2]) p.z = wrap1(p.z, box.L[2]);
    pos_out[slot] = p;
    if (vel_out) vel_out[slot] = vel_src[src];
    if (id_out) id_out[slot] = id_src ? id_src[src] : src;
    perm[slot] = src;
}

// A cell of more than 32 particles, by one warp: the rank of each element is
// the number of smaller input indices in the cell.
template <typename T>
__device__ __forceinline__ void sort_gather_large(uint32_t s, uint32_t k, const uint32_t *__restrict__ tmp,
                                               const BoxT<T> &box, const V4<T> *pos_src, const V4<T> *vel_src,
                                               const uint32_t *id_src, V4<T> *pos_out, V4<T> *vel_out,
                                               uint32_t *id_out, uint32_t *__restrict__ perm)
{
    const unsigned lane = threadIdx.x & 31;
    for (uint32_t e0 = 0; e0 < k; e0 += 32) {
        const bool mine = e0 + lane < k;
        const uint32_t v = mine ? tmp[s + e0 + lane] : UINT_MAX;
        uint32_t r = 0;
        for (uint32_t m0 = 0; m0 < k; m0 += 32) {
            const uint32_t w = (m0 + lane < k) ? tmp[s + m0 + lane] : UINT_MAX;
#pragma unroll 8
            for (int t = 0; t < 32; ++t) r += (__shfl_sync(kFull, w, t) < v) ? 1u : 0u;
        }
        if (mine) emit<T>(s + r, v, box, pos_src, vel_src, id_src, pos_out, vel_out, id_out, perm);
    }
}

// One warp per cell, two cells at a time (cells c and c + nwarps): both cells'
// bounds, slot lists and gathered records are loaded before either is stored,
// so each warp keeps two cells' memory accesses in flight.
template <typename T>
__global__ void k_sort_gather(BoxT<T> box, int ncell, const uint32_t *__restrict__ cell_start,
                              const uint32_t *__restrict__ tmp, const V4<T> *pos_src, const V4<T> *vel_src,
                              const uint32_t *id_src, V4<T> *pos_out, V4<T> *vel_out, uint32_t *id_out,
                              uint32_t *__restrict__ perm, const uint32_t *gate)
{
    if (gated_off(gate)) return;
    const unsigned lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // the loop bound is uniform per warp
    for (int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; c < ncell; c += 2 * nwarps) {
        const int64_t c1 = c + nwarps;
        const bool two = c1 < ncell;
        const uint32_t s0 = cell_start[c], k0 = cell_start[c + 1] - s0;
        const uint32_t s1 = two ? cell_start[c1] : 0u, k1 = two ? cell_start[c1 + 1] - s1 : 0u;
        if (k0 > 32u || k1 > 32u) {  // rare: a crowded cell; each cell on its own
            if (k0 > 32u)
                sort_gather_large<T>(s0, k0, tmp, box, pos_src, vel_src, id_src, pos_out, vel_out, id_out, perm);
            else if (k0 > 0u) {
                uint32_t v = lane < k0 ? tmp[s0 + lane] : UINT_MAX;
                v = warp_sort32(v);
                if (lane < k0) emit<T>(s0 + lane, v, box, pos_src, vel_src, id_src, pos_out, vel_out, id_out, perm);
            }
            if (k1 > 32u)
                sort_gather_large<T>(s1, k1, tmp, box, pos_src, vel_src, id_src, pos_out, vel_out, id_out, perm);
            else if (k1 > 0u) {
                uint32_t v = lane < k1 ? tmp[s1 + lane] : UINT_MAX;
                v = warp_sort32(v);
                if (lane < k1) emit<T>(s1 + lane, v, box, pos_src, vel_src, id_src, pos_out, vel_out, id_out, perm);
            }
            continue;
        }
        const bool a0 = lane < k0, a1 = lane < k1;
        uint32_t v0 = a0 ? tmp[s0 + lane] : UINT_MAX;
        uint32_t v1 = a1 ? tmp[s1 + lane] : UINT_MAX;
        v0 = warp_sort32(v0);
        v1 = warp_sort32(v1);
        V4<T> p0{}, p1{}, q0{}, q1{};
        uint32_t i0 = v0, i1 = v1;
        if (a0) p0 = pos_src[v0];
        if (a1) p1 = pos_src[v1];
        if (vel_out) {
            if (a0) q0 = vel_src[v0];
            if (a1) q1 = vel_src[v1];
        }
        if (id_out && id_src) {
            if (a0) i0 = id_src[v0];
            if (a1) i1 = id_src[v1];
        }
        if (a0) {
            if (box.per[0]) p0.x = wrap1(p0.x, box.L[0]);
            if (box.per[1]) p0.y = wrap1(p0.y, box.L[1]);
            if (box.per[2]) p0.z = wrap1(p0.z, box.L[2]);
            pos_out[s0 + lane] = p0;
            if (vel_out) vel_out[s0 + lane] = q0;
            if (id_out) id_out[s0 + lane] = i0;
            perm[s0 + lane] = v0;
        }
        if (a1) {
            if (box.per[0]) p1.x = wrap1(p1.x, box.L[0]);
            if (box.per[1]) p1.y = wrap1(p1.y, box.L[1]);
            if (box.per[2]) p1.z = wrap1(p1.z, box.L[2]);
            pos_out[s1 + lane] = p1;
            if (vel_out) vel_out[s1 + lane] = q1;
            if (id_out) id_out[s1 + lane] = i1;
            perm[s1 + lane] = v1;
        }
    }
}

// Sparse grids (a few particles per cell on average): a lane per cell.  A
// cell of up to kLaneCell particles is sorted by input index in registers
// (Batcher's odd-even merge network for 8 inputs, 19 compare-exchanges,
// empty slots padded with UINT_MAX) and gathered by its lane; the warp then
// takes its larger cells one by one as the dense kernel does.
constexpr uint32_t kLaneCell = 8;

__device__ __forceinline__ void cmpx(uint32_t &a, uint32_t &b)
{
    const uint32_t lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

__device__ __forceinline__ void sort8(uint32_t (&v)[8])
{
    cmpx(v[0], v[1]); cmpx(v[2], v[3]); cmpx(v[4], v[5]); cmpx(v[6], v[7]);
    cmpx(v[0], v[2]); cmpx(v[1], v[3]); cmpx(v[4], v[6]); cmpx(v[5], v[7]);
    cmpx(v[1], v[2]); cmpx(v[5], v[6]);
    cmpx(v[0], v[4]); cmpx(v[1], v[5]); cmpx(v[2], v[6]); cmpx(v[3], v[7]);
    cmpx(v[2], v[4]); cmpx(v[3], v[5]);
    cmpx(v[1], v[2]); cmpx(v[3], v[4]); cmpx(v[5], v[6]);
}

template <typename T>
__global__ void k_sort_gather_sparse(BoxT<T> box, int ncell, const uint32_t *__restrict__ cell_start,
                                     const uint32_t *__restrict__ tmp, const V4<T> *pos_src, const V4<T> *vel_src,
                                     const uint32_t *id_src, V4<T> *pos_out, V4<T> *vel_out, uint32_t *id_out,
                                     uint32_t *__restrict__ perm, const uint32_t *gate)
{
    if (gated_off(gate)) return;
    const unsigned lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // the loop bound is uniform per warp (base is the warp's first cell)
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31u); base < ncell; base += stride) {
        const int64_t c = base + lane;
        uint32_t s = 0, k = 0;
        if (c < ncell) {
            s = cell_start[c];
            k = cell_start[c + 1] - s;
        }
        if (k <= kLaneCell) {
            uint32_t v[8];
#pragma unroll
            for (uint32_t i = 0; i < 8; ++i) v[i] = i < k ? tmp[s + i] : UINT_MAX;
            sort8(v);
#pragma unroll
            for (uint32_t i = 0; i < 8; ++i)
                if (i < k) emit<T>(s + i, v[i], box, pos_src, vel_src, id_src, pos_out, vel_out, id_out, perm);
        }
        unsigned big = __ballot_sync(kFull, k > kLaneCell);
        while (big) {
            const int l = __ffs(big) - 1;
            big &= big - 1u;
            const uint32_t sb = __shfl_sync(kFull, s, l), kb = __shfl_sync(kFull, k, l);
            if (kb > 32u) {
                sort_gather_large<T>(sb, kb, tmp, box, pos_src, vel_src, id_src, pos_out, vel_out, id_out, perm);
            } else {
                uint32_t v = lane < kb ? tmp[sb + lane] : UINT_MAX;
                v = warp_sort32(v);
                if (lane < kb) emit<T>(sb + lane, v, box, pos_src, vel_src, id_src, pos_out, vel_out, id_out, perm);
            }
        }
    }
}

template <typename T>
__global__ void k_reorder(int n, const uint32_t *__restrict__ perm, const T *__restrict__ src, T *__restrict__ dst,
                          const uint32_t *gate)
{
    if (gated_off(gate)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[perm[i]];
}

template <typename T>
static fpm_status celllist_launch(const fpm_box &b, const fpm_grid &g, int n, const void *pos_in,
                                  const void *vel_in, const uint32_t *id_in, void *pos_out, void *vel_out,
                                  uint32_t *id_out, uint32_t *cell_start, uint32_t *perm, void *ws, size_t ws_bytes,
                                  fpm_dev_status *st, const uint32_t *gate, cudaStream_t stream)
{
    const CellWs L = cell_ws_layout(n, g.ncell, sizeof(V4<T>));
    if (!ws || ws_bytes < L.total)
        return fpm_fail(FPM_ERR_WORKSPACE, "fpm_celllist_build: workspace %zu < %zu bytes", ws_bytes, L.total);
    if (((uintptr_t)ws & 15u) != 0) return fpm_fail(FPM_ERR_WORKSPACE, "fpm_celllist_build: workspace not aligned");
    char *w = (char *)ws;
    const BoxT<T> box = make_box<T>(b);
    const GridD grid = make_grid(g);
    const V4<T> *pin = (const V4<T> *)pos_in;
    const V4<T> *vin = (const V4<T> *)vel_in;
    // stage inputs that alias an output (in-place reorder); read the others directly
    V4<T> *spos = (pos_in == pos_out) ? (V4<T> *)(w + L.off_pos) : nullptr;
    V4<T> *svel = (vel_in && vel_in == vel_out) ? (V4<T> *)(w + L.off_vel) : nullptr;
    uint32_t *sid = (id_out && id_in && id_in == id_out) ? (uint32_t *)(w + L.off_id) : nullptr;
    uint32_t *cell = (uint32_t *)(w + L.off_cell);
    uint32_t *rank = (uint32_t *)(w + L.off_rank);
    uint32_t *tmp = (uint32_t *)(w + L.off_tmp);
    uint32_t *count = (uint32_t *)(w + L.off_count);
    uint32_t *tiles = (uint32_t *)(w + L.off_tiles);

    const int ncell = g.ncell;
    const int ntiles = (ncell + kScanTile - 1) / kScanTile;
    k_zero<<<(ncell + 255) / 256 < 1184 ? (ncell + 255) / 256 : 1184, 256, 0, stream>>>(count, ncell, gate);
    if (n > 0)
        k_bin<T><<<grid_cap((n + 255) / 256), 256, 0, stream>>>(box, grid, n, pin, vin, id_in, spos, svel, sid, cell, rank,
                                                      count, st, gate);
    k_scan_part<<<ntiles, kScanThreads, 0, stream>>>(count, ncell, tiles, gate);
    k_scan_final<<<ntiles, kScanThreads, 0, stream>>>(count, ncell, tiles, cell_start, n, gate);
    if (n > 0) {
        k_scatter<<<grid_cap((n / 4 + 255) / 256 + 1), 256, 0, stream>>>(n, cell, rank, cell_start, tmp, gate);
        const V4<T> *psrc = spos ? spos : pin;
        const V4<T> *vsrc = svel ? svel : vin;
        const uint32_t *isrc = sid ? sid : id_in;
        if ((double)n < 4.0 * (double)ncell) {  // sparse: a lane per cell
            k_sort_gather_sparse<T><<<grid_cap(((int64_t)ncell + 255) / 256), 256, 0, stream>>>(
                box, ncell, cell_start, tmp, psrc, vel_out ? vsrc : nullptr, isrc, (V4<T> *)pos_out,
                (V4<T> *)vel_out, id_out, perm, gate);
        } else {  // a warp per cell
            const int64_t threads = (int64_t)ncell * 32;
            k_sort_gather<T><<<grid_cap((threads + 255) / 256), 256, 0, stream>>>(
                box, ncell, cell_start, tmp, psrc, vel_out ? vsrc : nullptr, isrc, (V4<T> *)pos_out,
                (V4<T> *)vel_out, id_out, perm, gate);
        }
    }
    return fpm_check_launch("fpm_celllist_build");
}

}  // namespace fpm

using namespace fpm;

extern "C" fpm_status fpm_celllist_workspace(int32_t n, const fpm_grid *grid, fpm_prec prec, size_t *bytes)
{
    if (!grid || !bytes || n < 0 || grid->ncell <= 0 || (prec != FPM_F32 && prec != FPM_F64))
        return fpm_fail(FPM_ERR_INVALID, "fpm_celllist_workspace: bad argument");
    *bytes = cell_ws_layout(n, grid->ncell, prec == FPM_F32 ? 16 : 32).total;
    return FPM_OK;
}

extern "C" fpm_status fpm_celllist_build(const fpm_box *box, const fpm_grid *grid, int32_t n, fpm_prec prec,
                                         const void *pos_in, const void *vel_in, const uint32_t *id_in,
                                         void *pos_out, void *vel_out, uint32_t *id_out, uint32_t *cell_start,
                                         uint32_t *perm, void *workspace, size_t workspace_bytes,
                                         fpm_dev_status *d_status, const uint32_t *d_gate, fpm_stream stream)
{
    if (!box || !grid || n < 0 || grid->ncell <= 0 || !cell_start || (n > 0 && (!pos_in || !pos_out || !perm)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_celllist_build: null pointer or bad size");
    if ((vel_in == nullptr) != (vel_out == nullptr))
        return fpm_fail(FPM_ERR_INVALID, "fpm_celllist_build: vel_in and vel_out must both be set or both NULL");
    if (prec != FPM_F32 && prec != FPM_F64) return fpm_fail(FPM_ERR_INVALID, "fpm_celllist_build: bad precision");
    for (int d = 0; d < 3; ++d)
        if (grid->nc[d] < 1 || !(box->L[d] > 0.0))
            return fpm_fail(FPM_ERR_INVALID, "fpm_celllist_build: bad grid or box");
    if ((int64_t)grid->nc[0] * grid->nc[1] * grid->nc[2] != grid->ncell)
        return fpm_fail(FPM_ERR_INVALID, "fpm_celllist_build: grid->ncell inconsistent with nc");
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == FPM_F32)
        return celllist_launch<float>(*box, *grid, n, pos_in, vel_in, id_in, pos_out, vel_out, id_out, cell_start,
                                      perm, workspace, workspace_bytes, d_status, d_gate, st);
    return celllist_launch<double>(*box, *grid, n, pos_in, vel_in, id_in, pos_out, vel_out, id_out, cell_start,
                                   perm, workspace, workspace_bytes, d_status, d_gate, st);
}

extern "C" fpm_status fpm_reorder(int32_t n, int32_t elem_bytes, const uint32_t *perm, const void *src, void *dst,
                                  const uint32_t *d_gate, fpm_stream stream)
{
    if (n < 0 || (n > 0 && (!perm || !src || !dst)) || src == dst)
        return fpm_fail(FPM_ERR_INVALID, "fpm_reorder: bad argument");
    if (n == 0) return FPM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    switch (elem_bytes) {
    case 4: k_reorder<uint32_t><<<blocks, 256, 0, st>>>(n, perm, (const uint32_t *)src, (uint32_t *)dst, d_gate); break;
    case 8: k_reorder<uint2><<<blocks, 256, 0, st>>>(n, perm, (const uint2 *)src, (uint2 *)dst, d_gate); break;
    case 16: k_reorder<uint4><<<blocks, 256, 0, st>>>(n, perm, (const uint4 *)src, (uint4 *)dst, d_gate); break;
    case 32:
        k_reorder<double4_32a><<<blocks, 256, 0, st>>>(n, perm, (const double4_32a *)src, (double4_32a *)dst,
                                                       d_gate);
        break;
    default: return fpm_fail(FPM_ERR_INVALID, "fpm_reorder: elem_bytes must be 4, 8, 16 or 32");
    }
    return fpm_check_launch("fpm_reorder");
}
