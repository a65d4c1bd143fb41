// batch.cu -- R independent periodic Lennard-Jones replicas of uneven size
// advanced together: the MD system of Sec. 4.1 (cell lists and Verlet lists
// of Sec. 2, the pair force of Listing 4.1, velocity Verlet) run as an
// ensemble.  The paper runs one system per process; here every operation is
// one launch over the whole batch.
//
// Layout.  Replica r owns particles [p0, p0+n) of the concatenated arrays,
// cells [c0, c0+ncell) of one concatenated cell_start (whose values index the
// concatenated arrays), and tiles [t0, t0+ntiles) of one Verlet-list object.
// Tiles, staging and the pair code are those of the single-system path
// (tiles.cuh, lj_pair.cuh); a block looks up the replica of its tile by
// binary search over t0 and takes that replica's box and grid.
//
// Rebuilds are per replica: the drift kernel flags a replica when one of its
// particles moved more than skin/2, and only flagged replicas are re-binned
// (one block per replica: the counting sort runs in shared memory) and get
// new tile descriptors and lists (a persistent scan over their tiles).
#include <algorithm>
#include <cmath>

#include "lj_pair.cuh"
#include "reduce.cuh"

namespace fpm {

constexpr int kBatchCellThreads = 1024;
constexpr int kBatchMaxCells = 32768;   // cells of one replica (shared-memory counters)
constexpr int kBatchMaxReplicas = 65535;

__host__ __device__ inline int rep_ntiles(const fpm_grid &g) { return g.tiles_x * g.nc[1] * g.nc[2]; }

// The replica holding particle i: the last r whose p0 is <= i.  (Tiles look
// their replica up in a map the Verlet build writes.)
__device__ __forceinline__ int replica_of_particle(const fpm_replica *__restrict__ reps, int R, uint32_t i)
{
    int lo = 0, hi = R - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((uint32_t)__ldg(&reps[mid].p0) <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}


// ---- drift + per-replica rebuild test ---------------------------------------

// One particle (every lane of the warp calls it; i may be past n).  A
// replica's flag is set by the first lane that finds it over; nflag, when
// given, counts the replicas flagged, and flist receives them (in no
// particular order).
__device__ __forceinline__ void bdrift_one(int i, int n, int R, const fpm_replica *__restrict__ reps, float hdt,
                                           float dt, float4 *__restrict__ pos, float4 *__restrict__ vel,
                                           const float4 *__restrict__ force, const float4 *__restrict__ ref, float th,
                                           uint32_t *__restrict__ flag, uint32_t *nflag = nullptr,
                                           uint32_t *flist = nullptr)
{
    bool over = false;
    if (i < n) {
        float4 x = pos[i], v = vel[i];
        const float4 f = force[i];
        v.x += hdt * f.x;
        v.y += hdt * f.y;
        v.z += hdt * f.z;
        x.x += dt * v.x;
        x.y += dt * v.y;
        x.z += dt * v.z;
        pos[i] = x;
        vel[i] = v;
        const float4 r0 = ref[i];
        const float dx = x.x - r0.x, dy = x.y - r0.y, dz = x.z - r0.z;
        over = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))) > th;
    }
    const unsigned m = __ballot_sync(kFull, over);
    if (!over) return;
    const int r = replica_of_particle(reps, R, (uint32_t)i);
    const unsigned peers = __match_any_sync(m, r);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1 && atomicOr(&flag[r], 1u) == 0u && nflag) {
        const uint32_t q = atomicAdd(nflag, 1u);
        if (flist) flist[q] = (uint32_t)r;
    }
}

__global__ void __launch_bounds__(256)
    k_bdrift_check(int n, int R, const fpm_replica *__restrict__ reps, float hdt, float dt, float4 *__restrict__ pos,
                   float4 *__restrict__ vel, const float4 *__restrict__ force, const float4 *__restrict__ ref,
                   float th, uint32_t *__restrict__ flag)
{
    bdrift_one(blockIdx.x * blockDim.x + threadIdx.x, n, R, reps, hdt, dt, pos, vel, force, ref, th, flag);
}

// ---- cell lists, one block per flagged replica ------------------------------

// In-place exclusive scan of a[0..m) in shared memory by the whole block
// (blockDim a multiple of 32); a[m] receives the total.
__device__ void smem_exclusive_scan(uint32_t *a, int m, uint32_t *wsum)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t carry = 0;
    for (int base = 0; base < m; base += blockDim.x) {
        const int k = base + threadIdx.x;
        const uint32_t v = k < m ? a[k] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = lane < nw ? wsum[lane] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, w, o);
                if (lane >= o) w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        if (k < m) a[k] = carry + x - v + (warp > 0 ? wsum[warp - 1] : 0u);
        carry += wsum[nw - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) a[m] = carry;
    __syncthreads();
}

// Ascending bitonic sort of one value per lane across a full warp.
__device__ __forceinline__ uint32_t bwarp_sort32(uint32_t v)
{
    const unsigned lane = threadIdx.x & 31;
#pragma unroll
    for (unsigned k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (unsigned j = k >> 1; j > 0; j >>= 1) {
            const uint32_t o = __shfl_xor_sync(kFull, v, j);
            const bool up = (lane & k) == 0;
            const bool low = (lane & j) == 0;
            v = (low == up) ? min(v, o) : max(v, o);
        }
    }
    return v;
}

struct BCellWs {
    float4 *spos, *svel;
    uint32_t *sid, *cell, *rank, *tmp;
    uint32_t *prid, *crid;  // the replica of every particle / cell (written by every cell-list build)
};

// Particle i wrapped into its box and binned: the wrapped position, velocity
// and id copied to the workspace, its cell (within the replica) stored and
// returned.  A coordinate outside the box latches FPM_FLAG_DOMAIN.
__device__ __forceinline__ uint32_t bcell_bin(uint32_t i, const BoxT<float> &box, const GridD &g,
                                              const float4 *__restrict__ pos, const float4 *__restrict__ vel,
                                              const uint32_t *__restrict__ ids, const BCellWs &w,
                                              fpm_dev_status *st)
{
    float4 p = pos[i];
    p.x = wrap1(p.x, box.L[0]);
    p.y = wrap1(p.y, box.L[1]);
    p.z = wrap1(p.z, box.L[2]);
    bool bad = false;
    int cc[3];
    cell_of(p, box, g, cc, bad);
    if (bad) {
        latch_flag(st, FPM_FLAG_DOMAIN);
        if (st) atomicExch(&st->bad_index, i);
    }
    const uint32_t c = linear_cell(cc[0], cc[1], cc[2], g);
    w.spos[i] = p;
    if (vel) w.svel[i] = vel[i];
    w.sid[i] = ids ? ids[i] : i;
    w.cell[i] = c;
    return c;
}

// One cell's slice [s, e) of the scattered indices (w.tmp), by a whole warp:
// sorted by particle index (the stable order), then pos / vel / ids gathered
// into place from the binned copies and perm written.
__device__ __forceinline__ void bcell_gather(uint32_t s, uint32_t e, const BCellWs &w, float4 *__restrict__ pos,
                                             float4 *__restrict__ vel, uint32_t *__restrict__ ids,
                                             uint32_t *__restrict__ perm)
{
    const int lane = threadIdx.x & 31;
    const uint32_t m = e - s;
    if (m == 0) return;
    if (m <= 32) {
        uint32_t v = (uint32_t)lane < m ? w.tmp[s + lane] : 0xffffffffu;
        v = bwarp_sort32(v);
        if ((uint32_t)lane < m) {
            const uint32_t slot = s + lane;
            pos[slot] = w.spos[v];
            if (vel) vel[slot] = w.svel[v];
            if (ids) ids[slot] = w.sid[v];
            if (perm) perm[slot] = v;
        }
        return;
    }
    // larger cells: a slice already in ascending order (a replica of one
    // cell, ranked in index order) is gathered as it stands
    bool sorted = true;
    for (uint32_t e0 = 0; e0 < m && sorted; e0 += 32) {
        const uint32_t j = e0 + lane;
        const bool ok = j + 1 >= m || w.tmp[s + j] < w.tmp[s + j + 1];
        sorted = __all_sync(kFull, ok);
    }
    if (sorted) {
        for (uint32_t j = lane; j < m; j += 32) {
            const uint32_t slot = s + j, v = w.tmp[slot];
            pos[slot] = w.spos[v];
            if (vel) vel[slot] = w.svel[v];
            if (ids) ids[slot] = w.sid[v];
            if (perm) perm[slot] = v;
        }
        return;
    }
    // otherwise: rank of each element = number of smaller indices
    for (uint32_t e0 = 0; e0 < m; e0 += 32) {
        const bool mine = e0 + lane < m;
        const uint32_t v = mine ? w.tmp[s + e0 + lane] : 0xffffffffu;
        uint32_t rk = 0;
        for (uint32_t m0 = 0; m0 < m; m0 += 32) {
            const uint32_t u = (m0 + lane < m) ? w.tmp[s + m0 + lane] : 0xffffffffu;
#pragma unroll 8
            for (int t = 0; t < 32; ++t) rk += (__shfl_sync(kFull, u, t) < v) ? 1u : 0u;
        }
        if (mine) {
            const uint32_t slot = s + rk;
            pos[slot] = w.spos[v];
            if (vel) vel[slot] = w.svel[v];
            if (ids) ids[slot] = w.sid[v];
            if (perm) perm[slot] = v;
        }
    }
}

// Per replica: wrap and bin into shared-memory counters (the atomic gives an
// arrival rank), exclusive scan -> cell_start, scatter of indices by (cell,
// rank), then one warp per cell sorts its slice by particle index (the
// stable order) and gathers pos / vel / ids into place.  Also records the
// replica of each of its particles and cells.
__global__ void __launch_bounds__(kBatchCellThreads)
    k_bcell(int R, const fpm_replica *__restrict__ reps, float4 *__restrict__ pos, float4 *__restrict__ vel,
            uint32_t *__restrict__ ids, uint32_t *__restrict__ cell_start, uint32_t *__restrict__ perm, BCellWs w,
            const uint32_t *__restrict__ flag, fpm_dev_status *st)
{
    extern __shared__ uint32_t cnt[];  // [ncell + 1]
    __shared__ uint32_t wsum[32];
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = blockIdx.x; r < R; r += gridDim.x) {
        if (flag && flag[r] == 0u) continue;
        const fpm_replica rp = reps[r];
        const BoxT<float> box = make_box<float>(rp.box);
        const GridD g = make_grid(rp.grid);
        const int ncell = rp.grid.ncell;
        const uint32_t p0 = (uint32_t)rp.p0, n = (uint32_t)rp.n;
        for (int c = threadIdx.x; c <= ncell; c += blockDim.x) {
            cnt[c] = 0u;
            if (c < ncell) w.crid[rp.c0 + c] = (uint32_t)r;
        }
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) {
            const uint32_t i = p0 + k;
            const uint32_t rk = atomicAdd(&cnt[bcell_bin(i, box, g, pos, vel, ids, w, st)], 1u);
            w.rank[i] = ncell == 1 ? k : rk;  // one cell: the index order is the sorted order
            w.prid[i] = (uint32_t)r;
        }
        __syncthreads();
        smem_exclusive_scan(cnt, ncell, wsum);
        for (int c = threadIdx.x; c <= ncell; c += blockDim.x) cell_start[rp.c0 + c] = p0 + cnt[c];
        for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) {
            const uint32_t i = p0 + k;
            w.tmp[p0 + cnt[w.cell[i]] + w.rank[i]] = i;
        }
        __syncthreads();
        for (int c = warp; c < ncell; c += nw) bcell_gather(p0 + cnt[c], p0 + cnt[c + 1], w, pos, vel, ids, perm);
        __syncthreads();  // cnt is reused by the next replica of this block
    }
}

// ---- Verlet lists of the flagged replicas -----------------------------------

// Exclusive prefix sum of one value per thread over the block (blockDim a
// multiple of 32, wsum: 32 words); *total receives the block's sum.  All
// threads call it; it ends with a barrier, so wsum may be reused.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *wsum, uint32_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t u = lane < nw ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, u, o);
            if (lane >= o) u += y;
        }
        wsum[lane] = u;
    }
    __syncthreads();
    const uint32_t off = x - v + (warp > 0 ? wsum[warp - 1] : 0u);
    *total = wsum[nw - 1];
    __syncthreads();
    return off;
}

// One block: the tile -> replica map of every tile (unless map is null: it
// never changes), the work list of the build (every tile of every flagged
// replica, in replica order), the scan's scheduling counters and the rebuild
// count.
// (clear: the flags are cleared as they are read, and the one-launch step's
// grid barrier is reset.  unf, when given, receives the tiles of the
// replicas NOT flagged, in replica order, and rep_scan[r] is zeroed for
// every flagged r.)
__device__ void bwork_block(int R, const fpm_replica *__restrict__ reps, uint32_t *__restrict__ flag,
                            uint32_t *__restrict__ work, uint32_t *__restrict__ map, uint32_t *__restrict__ header,
                            fpm_dev_status *st, bool clear, uint32_t *wsum, uint32_t *__restrict__ unf = nullptr,
                            uint32_t *__restrict__ rep_scan = nullptr)
{
    uint32_t carry = 0, carry_u = 0, nflag = 0;
    for (int base = 0; base < R; base += blockDim.x) {
        const int r = base + threadIdx.x;
        bool f = false;
        uint32_t nt = 0, nu = 0, t0 = 0, nr = 0;
        if (r < R) {
            f = !flag || flag[r] != 0u;
            if (flag && clear) flag[r] = 0u;
            nr = (uint32_t)rep_ntiles(reps[r].grid);
            t0 = (uint32_t)reps[r].t0;
            if (map)
                for (uint32_t j = 0; j < nr; ++j) map[t0 + j] = (uint32_t)r;
            nt = f ? nr : 0u;
            nu = f ? 0u : nr;
            if (f && rep_scan) rep_scan[r] = 0u;
        }
        nflag += (uint32_t)__syncthreads_count(f);
        uint32_t tot;
        const uint32_t off = carry + block_exclusive_scan(nt, wsum, &tot);
        for (uint32_t j = 0; j < nt; ++j) work[off + j] = t0 + j;
        carry += tot;
        if (unf) {
            const uint32_t ou = carry_u + block_exclusive_scan(nu, wsum, &tot);
            for (uint32_t j = 0; j < nu; ++j) unf[ou + j] = t0 + j;
            carry_u += tot;
        }
    }
    if (threadIdx.x == 0) {
        header[0] = carry;
        header[4] = 0u;  // the scan's ticket and completion counters (list header bytes 16..23)
        header[5] = 0u;
        if (clear) header[8] = 0u;  // the one-launch step's grid-barrier arrivals (list header bytes 32..35)
        if (st) st->nrebuild += nflag;
    }
}

__global__ void __launch_bounds__(1024)
    k_bwork(int R, const fpm_replica *__restrict__ reps, uint32_t *__restrict__ flag, uint32_t *__restrict__ work,
            uint32_t *__restrict__ map, uint32_t *__restrict__ header, fpm_dev_status *st)
{
    __shared__ uint32_t wsum[32];
    bwork_block(R, reps, flag, work, map, header, st, true, wsum);
}

// Shared state of a batched scan block.
struct BScanShared {
    TileGeom g;
    TileDesc d;
    TileCfg cfg;
    BoxT<float> box;
    int tile, c0;
};

// Work-list entry k: its tile's geometry, staging and scan (verlet_tile), then
// the tile's descriptor written for the force sweep.  All threads call it.
__device__ __forceinline__ void bscan_tile(uint32_t k, BScanShared &sh, const fpm_replica *__restrict__ reps,
                                           const uint32_t *__restrict__ map, const float4 *__restrict__ pos,
                                           const uint32_t *__restrict__ cs, float rl2, int cap, int64_t ld,
                                           int stage_cap, const uint32_t *__restrict__ work,
                                           uint32_t *__restrict__ words, uint32_t *__restrict__ nn,
                                           float4 *__restrict__ pos_ref, TileDesc *__restrict__ descs,
                                           fpm_dev_status *st, float4 *sp, uint64_t *bar, uint32_t &phase,
                                           uint32_t &maxc)
{
    if (threadIdx.x == 0) {
        const uint32_t tile = work[k];
        const fpm_replica rp = reps[map[tile]];
        sh.cfg = make_tile_cfg(rp.box, rp.grid);
        sh.box = make_box<float>(rp.box);
        sh.tile = (int)tile - rp.t0;
        sh.c0 = rp.c0;
    }
    __syncthreads();
    const TileCfg cfg = sh.cfg;
    const BoxT<float> box = sh.box;
    const uint32_t c = verlet_tile<float>(cfg, box, sh.tile, cs + sh.c0, pos, rl2, cap, ld, stage_cap, sh.g, sh.d,
                                          sp, bar, phase, words, nn, pos_ref, st);
    maxc = c > maxc ? c : maxc;
    // the tile's descriptor, for the force sweep (the geometry the scan computed)
    const int nwd = (int)(sizeof(TileDesc) / 4);
    uint32_t *o = (uint32_t *)(descs + work[k]);
    const uint32_t *dsrc = (const uint32_t *)&sh.d;
    for (int q = threadIdx.x; q < nwd; q += blockDim.x) o[q] = dsrc[q];
    if (threadIdx.x == 0 && st && sh.d.h1 > sh.d.h0) atomicMax(&st->max_staged, (uint32_t)sh.d.M);
}

__global__ void __launch_bounds__(kTileThreads)
    k_bverlet_scan(const fpm_replica *__restrict__ reps, const uint32_t *__restrict__ map,
                   const float4 *__restrict__ pos, const uint32_t *__restrict__ cs, float rl2, int cap, int64_t ld,
                   int stage_cap, const uint32_t *__restrict__ work, const uint32_t *__restrict__ count, Sched sched,
                   uint32_t *__restrict__ words, uint32_t *__restrict__ nn, float4 *__restrict__ pos_ref,
                   TileDesc *__restrict__ descs, fpm_dev_status *st)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float4 *sp = (float4 *)smem_raw;
    __shared__ BScanShared sh;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_k;
    __shared__ bool s_last;
    stage_init(&bar);
    uint32_t phase = 0, maxc = 0, ahead = 0;
    const uint32_t ntodo = *count;
    for (uint32_t k = blockIdx.x; k < ntodo; k = ticket_next(ahead, &s_k)) {
        ahead = ticket_ahead(sched);
        bscan_tile(k, sh, reps, map, pos, cs, rl2, cap, ld, stage_cap, work, words, nn, pos_ref, descs, st, sp, &bar,
                   phase, maxc);
    }
    const uint32_t m = __reduce_max_sync(kFull, maxc);
    if ((threadIdx.x & 31) == 0 && st && m > 0) atomicMax(&st->max_nn, m);
    sched_finish(sched, &s_last);
}

// ---- LJ forces over every tile of the batch ---------------------------------

// Force tiles of at most this many home particles split each list in two
// (see blj_tile).
constexpr uint32_t kSplitTile = 128;

// Shared state of a batched force block.
struct BLjShared {
    TileDesc d;
    TileCfg cfg;
    BoxT<float> box;
    int r, t0, nt;
    bool rep_last;
};

// Tile k of the batch: forces (and the closing half-kick when vel is given),
// the tile's U, W and pair count, and the replica's sums when this is its
// last tile to finish.  All threads call it.  The descriptor is read at L2:
// in the one-launch step it was written earlier in the same launch.
__device__ __forceinline__ void blj_tile(uint32_t k, BLjShared &sh, const fpm_replica *__restrict__ reps,
                                         const uint32_t *__restrict__ map, const float4 *__restrict__ pos,
                                         const ListView &lv, const uint32_t *__restrict__ nn, int64_t ld,
                                         int stage_cap, const LJParams<float> &P, float4 *__restrict__ force,
                                         double *part, uint32_t *rep_done, double *out, fpm_dev_status *status,
                                         float4 *__restrict__ vel, float hdt, float4 *sp, uint64_t *bar,
                                         uint32_t &phase)
{
    const uint32_t *__restrict__ words = lv.words;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        const int r = (int)map[k];
        const fpm_replica rp = reps[r];
        sh.cfg = make_tile_cfg(rp.box, rp.grid);
        sh.box = make_box<float>(rp.box);
        sh.r = r;
        sh.t0 = rp.t0;
        sh.nt = rep_ntiles(rp.grid);
    }
    load_desc_cg(lv.descs + k, sh.d);  // ends with a barrier: the replica's fields are visible
    const TileDesc &d = sh.d;
    const TileCfg cfg = sh.cfg;
    const BoxT<float> box = sh.box;
    float usum = 0.0f, wsum = 0.0f;
    uint32_t npsum = 0;
    if (d.h1 > d.h0) {
        if (d.h0 + threadIdx.x < d.h1) prefetch_home(pos, nn, words, ld, d.h0 + threadIdx.x, (int)kLjChunk);
        const bool in_smem = d.M <= stage_cap;
        if (!in_smem) note_spill(status);
        const bool staged = in_smem ? stage_positions(d, box, pos, sp, bar, phase, status) : true;
        const bool all_mode = cfg.mode[0] == kModeAll || cfg.mode[1] == kModeAll || cfg.mode[2] == kModeAll;
        const uint32_t nh = d.h1 - d.h0;
        if (nh <= kSplitTile) {
            // A small tile (the small replicas' tiles leave most of a block
            // idle): each home particle's list in two halves, the even and
            // the odd words, whose sums are added half 0 + half 1.  With a
            // lane per half the lane pair 2q, 2q + 1 takes particle q; with
            // fewer threads one thread takes both halves in turn.  The same
            // sums either way, whatever the block size.
            const bool pair = 2u * nh <= blockDim.x;
            const uint32_t q = pair ? (threadIdx.x >> 1) : threadIdx.x;
            // half sums of particle i: forces, S12 - S6 and 2 S12 - S6 (u, w), pairs
            auto half_sums = [&](uint32_t i, uint32_t half, const float4 &pi, uint32_t m, float (&o)[5],
                                 uint32_t &np) {
                o[0] = o[1] = o[2] = o[3] = o[4] = 0.0f;
                np = 0;
                if (!in_smem)
                    lj_sweep<float, false, false, 2>(cfg, box, d, pos, sp, pi, m, words + i, ld, P, o[0], o[1], o[2],
                                                     o[3], o[4], np, half);
                else if (d.slow && all_mode)
                    lj_sweep<float, false, true, 2>(cfg, box, d, pos, sp, pi, m, words + i, ld, P, o[0], o[1], o[2],
                                                    o[3], o[4], np, half);
                else if (d.slow)
                    lj_sweep_wall<float, 2>(box, sp, pi, m, words + i, ld, P, o[0], o[1], o[2], o[3], o[4], np, half);
                else
                    lj_sweep<float, true, true, 2>(cfg, box, d, pos, sp, pi, m, words + i, ld, P, o[0], o[1], o[2],
                                                   o[3], o[4], np, half);
            };
            if (staged && q < nh) {
                const uint32_t i = d.h0 + q;
                const float4 pi = pos[i];
                const uint32_t m = nn[i];
                float o[5];
                uint32_t np;
                if (pair) {
                    half_sums(i, threadIdx.x & 1u, pi, m, o, np);
                    // the lanes of this warp in the branch: a prefix (threadIdx.x < 2 nh)
                    const uint32_t live = 2u * nh - (threadIdx.x & ~31u);
                    const unsigned act = live >= 32u ? kFull : ((1u << live) - 1u);
                    float po[5];
#pragma unroll
                    for (int c = 0; c < 5; ++c) po[c] = __shfl_xor_sync(act, o[c], 1);
                    const uint32_t pnp = __shfl_xor_sync(act, np, 1);
                    if (threadIdx.x & 1u) {  // the odd lane holds half 1: half 0 + half 1 as below
#pragma unroll
                        for (int c = 0; c < 5; ++c) o[c] = po[c] + o[c];
                    } else {
#pragma unroll
                        for (int c = 0; c < 5; ++c) o[c] = o[c] + po[c];
                    }
                    np += pnp;
                } else {
                    float o1[5];
                    uint32_t np1;
                    half_sums(i, 0u, pi, m, o, np);
                    half_sums(i, 1u, pi, m, o1, np1);
#pragma unroll
                    for (int c = 0; c < 5; ++c) o[c] = o[c] + o1[c];
                    np += np1;
                }
                if (!pair || (threadIdx.x & 1u) == 0u) {
                    float4 f;
                    f.x = P.eps24 * o[0];
                    f.y = P.eps24 * o[1];
                    f.z = P.eps24 * o[2];
                    f.w = 0.5f * P.eps4 * o[3];
                    force[i] = f;
                    if (vel) {  // the closing half-kick of velocity Verlet, v += dt/2 F
                        float4 v = vel[i];
                        v.x += hdt * f.x;
                        v.y += hdt * f.y;
                        v.z += hdt * f.z;
                        vel[i] = v;
                    }
                    usum += P.eps4 * o[3];
                    wsum += P.eps24 * o[4];
                    npsum += np;
                }
            }
        }
        for (uint32_t i = d.h0 + threadIdx.x; staged && nh > kSplitTile && i < d.h1; i += blockDim.x) {
            const float4 pi = pos[i];
            const uint32_t m = nn[i];
            float fx = 0.0f, fy = 0.0f, fz = 0.0f, u = 0.0f, w = 0.0f;
            uint32_t np = 0;
            if (in_smem) {
                if (d.slow && all_mode)
                    lj_sweep<float, false, true>(cfg, box, d, pos, sp, pi, m, words + i, ld, P, fx, fy, fz, u, w, np);
                else if (d.slow)
                    lj_sweep_wall<float>(box, sp, pi, m, words + i, ld, P, fx, fy, fz, u, w, np);
                else
                    lj_sweep<float, true, true>(cfg, box, d, pos, sp, pi, m, words + i, ld, P, fx, fy, fz, u, w, np);
            } else {
                lj_sweep<float, false, false>(cfg, box, d, pos, sp, pi, m, words + i, ld, P, fx, fy, fz, u, w, np);
            }
            float4 f;
            f.x = P.eps24 * fx;
            f.y = P.eps24 * fy;
            f.z = P.eps24 * fz;
            f.w = 0.5f * P.eps4 * u;
            force[i] = f;
            if (vel) {  // the closing half-kick of velocity Verlet, v += dt/2 F
                float4 v = vel[i];
                v.x += hdt * f.x;
                v.y += hdt * f.y;
                v.z += hdt * f.z;
                vel[i] = v;
            }
            usum += P.eps4 * u;
            wsum += P.eps24 * w;
            npsum += np;
        }
    }
    if (out) {
        // this tile's U, W, pairs (halved: every pair is seen from both sides)
        const float v[3] = {0.5f * usum, 0.5f * wsum, 0.5f * (float)npsum};
        block_sum_store<3>(v, part + (size_t)k * 3);
        if (threadIdx.x == 0) {
            __threadfence();
            const uint32_t t = atomicAdd(&rep_done[sh.r], 1u);
            sh.rep_last = (t == (uint32_t)sh.nt - 1u);
        }
        __syncthreads();
        if (sh.rep_last) {  // the replica's last tile: its sums, in tile order
            __threadfence();
            if (warp == 0) {
                double acc[3] = {0.0, 0.0, 0.0};
                for (int j = lane; j < sh.nt; j += 32)
#pragma unroll
                    for (int q = 0; q < 3; ++q) acc[q] += __ldcg(part + (size_t)(sh.t0 + j) * 3 + q);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const double s = warp_sum(acc[q]);
                    if (lane == 0) out[(size_t)sh.r * 3 + q] = s;
                }
                if (lane == 0) rep_done[sh.r] = 0u;
            }
        }
    }
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS)
    k_blj_tiles(int ntiles, const fpm_replica *__restrict__ reps, const uint32_t *__restrict__ map,
                const float4 *__restrict__ pos, ListView lv, const uint32_t *__restrict__ nn, int64_t ld, int stage_cap,
                LJParams<float> P, float4 *__restrict__ force, Sched sched, double *part, uint32_t *rep_done,
                double *out, fpm_dev_status *status, float4 *__restrict__ vel, float hdt)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float4 *sp = (float4 *)smem_raw;
    __shared__ BLjShared sh;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_k;
    __shared__ bool s_last;
    stage_init(&bar);
    uint32_t phase = 0, ahead = 0;
    for (uint32_t k = blockIdx.x; k < (uint32_t)ntiles; k = ticket_next(ahead, &s_k)) {
        ahead = ticket_ahead(sched);
        blj_tile(k, sh, reps, map, pos, lv, nn, ld, stage_cap, P, force, part, rep_done, out, status, vel, hdt, sp,
                 &bar, phase);
    }
    sched_finish(sched, &s_last);
}

// ---- one persistent launch per step ----------------------------------------
// The whole batched step as phases of one cooperative kernel (all blocks
// resident at once), separated by grid barriers:
//   A   drift and per-replica rebuild test (every particle), listing the
//       flagged replicas (when there are none, B is skipped; B1, B3 and B4
//       visit only the listed replicas' particles and cells, through prefix
//       tables each block builds in shared memory);
//   B1  the particles of flagged replicas binned, each with its rank in its
//       cell from a global counter (in index order for a replica of one
//       cell, whose index order is the sorted order);
//   B2  per flagged replica (a block each): the counters scanned into
//       cell_start (and zeroed for the next step);
//   B3  every binned particle's index scattered to its (cell, rank) slot;
//   B4  per cell of a flagged replica (a warp each): the slice sorted by
//       particle index and pos / vel / ids / perm gathered into place; the
//       last block first writes the work lists;
//   CD  one ticket queue: first the Verlet scans of the flagged replicas'
//       tiles (which also write their descriptors), then the force tiles
//       (forces, the closing half-kick and the energies) of the replicas not
//       rebuilt, then those of the rebuilt replicas, each of which waits
//       (bounded) until every tile of its replica has been scanned.  Blocks
//       that run out of scans take force tiles, which need no scan, so the
//       scan's tail overlaps the force sweep.
// Every phase computes what the separate launches compute (the same cell
// order, lists, descriptors, forces and per-tile sums in tile order), so the
// results are those of the separate calls bit for bit.  The cell build runs
// over the whole grid instead of one block per replica, so the largest
// flagged replica no longer sets its time.
// A block never waits on a ticket it holds itself: tickets are handed out in
// increasing order, every scan ticket is below every force ticket, and a
// block's prefetched ticket is above its current one, so a block that waits
// for a replica's scans holds none of them; the blocks that hold them wait
// for nothing but their own copies.

struct BStepArgs {
    int n, R, ntiles, ncell, cap, stage_cap;
    int64_t ld;
    const fpm_replica *reps;
    float hdt, dt, th, rl2;
    float4 *pos, *vel, *force, *pos_ref;
    uint32_t *ids, *cell_start, *perm, *flag;
    BCellWs cw;
    uint32_t *gcnt;  // [ncell_total] cell counters, zero between steps
    uint32_t *header, *work, *map, *words, *nn;
    TileDesc *descs;
    ListView lv;
    LJParams<float> P;
    Sched sched;  // the CD queue's tickets (workspace counters)
    double *part, *out;
    uint32_t *rep_done, *unf, *rep_scan;
    fpm_dev_status *status;
    unsigned *gbar;   // grid barrier: [0] arrivals, [1] generation (list header bytes 32..39)
    uint32_t *nflag;  // replicas flagged this step (workspace bytes 48..51; zero between steps)
    uint32_t *flist;  // [R]: the flagged replicas, in the order they were flagged
    int smem_bytes, cnt_bytes;  // the block's dynamic shared memory; B2's counters at its start
};

// A barrier over every block of the (cooperative) grid.  Thread 0 of each
// block arrives on the counter and waits for the generation to change, at
// most kWaitCycles; the last to arrive resets the counter and advances the
// generation.  Returns false in every thread, with FPM_FLAG_TIMEOUT latched,
// if the wait expired.  The fences order each phase's writes before the
// next phase's reads, for the generic and (bulk copies) the async proxy.
__device__ bool grid_sync(unsigned *gbar, fpm_dev_status *st)
{
    __shared__ int s_ok;
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g = atomicAdd(gbar + 1, 0u);
        __threadfence();
        int ok = 1;
        if (atomicAdd(gbar, 1u) == gridDim.x - 1u) {
            atomicExch(gbar, 0u);
            __threadfence();
            atomicAdd(gbar + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (atomicAdd(gbar + 1, 0u) == g) {
                if (clock64() - t0 > kWaitCycles) {
                    ok = 0;
                    latch_flag(st, FPM_FLAG_TIMEOUT);
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    asm volatile("fence.proxy.async.global;\n\tfence.proxy.async.shared::cta;" ::: "memory");
    return s_ok != 0;
}

// B1 and B3 take four particles per thread at a time (grid-strided), so the
// loads of the four start together.
__device__ __forceinline__ void bstep_bin(const BStepArgs &a)
{
    const int stride = (int)(gridDim.x * blockDim.x);
    for (int i0 = (int)(blockIdx.x * blockDim.x + threadIdx.x); i0 < a.n; i0 += 4 * stride) {
        uint32_t r[4];
        bool f[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * stride;
            r[u] = i < a.n ? __ldcg(a.cw.prid + i) : 0u;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) f[u] = i0 + u * stride < a.n && __ldcg(a.flag + r[u]) != 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (!f[u]) continue;
            const int i = i0 + u * stride;
            const fpm_replica &rp = a.reps[r[u]];
            const BoxT<float> box = make_box<float>(rp.box);
            const GridD g = make_grid(rp.grid);
            const uint32_t c = bcell_bin((uint32_t)i, box, g, a.pos, a.vel, a.ids, a.cw, a.status);
            // one cell: the index order is the sorted order, and the count is n
            a.cw.rank[i] = rp.grid.ncell == 1 ? (uint32_t)(i - rp.p0) : atomicAdd(&a.gcnt[rp.c0 + (int)c], 1u);
        }
    }
}

__device__ __forceinline__ void bstep_cell_scan(const BStepArgs &a, int r, uint32_t *cnt, uint32_t *wsum)
{
    const int ncell = a.reps[r].grid.ncell, c0 = a.reps[r].c0;
    const uint32_t p0 = (uint32_t)a.reps[r].p0;
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
        cnt[c] = ncell == 1 ? (uint32_t)a.reps[r].n : __ldcg(a.gcnt + c0 + c);
        a.gcnt[c0 + c] = 0u;
    }
    __syncthreads();
    smem_exclusive_scan(cnt, ncell, wsum);
    for (int c = threadIdx.x; c <= ncell; c += blockDim.x) a.cell_start[c0 + c] = p0 + cnt[c];
    __syncthreads();
}

__device__ __forceinline__ void bstep_scatter(const BStepArgs &a)
{
    const int stride = (int)(gridDim.x * blockDim.x);
    for (int i0 = (int)(blockIdx.x * blockDim.x + threadIdx.x); i0 < a.n; i0 += 4 * stride) {
        uint32_t r[4];
        bool f[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * stride;
            r[u] = i < a.n ? __ldcg(a.cw.prid + i) : 0u;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) f[u] = i0 + u * stride < a.n && __ldcg(a.flag + r[u]) != 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (!f[u]) continue;
            const int i = i0 + u * stride;
            const uint32_t c = __ldcg(a.cw.cell + i);
            a.cw.tmp[__ldcg(a.cell_start + a.reps[r[u]].c0 + c) + __ldcg(a.cw.rank + i)] = (uint32_t)i;
        }
    }
}

// Warp w takes the cells w, w + nw, w + 2 nw, ... (nw warps in the grid), so
// the cells of the flagged replicas, which lie in runs, spread over every
// warp; it tests 32 of them at once and gathers the flagged ones in turn.
__device__ __forceinline__ void bstep_gather(const BStepArgs &a)
{
    const int lane = threadIdx.x & 31;
    const int nw = (int)(gridDim.x * blockDim.x) >> 5;
    const int w = (int)(blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    for (long long j0 = 0; w + j0 * nw < a.ncell; j0 += 32) {
        const long long gl = w + (j0 + lane) * nw;
        const int gc = gl < a.ncell ? (int)gl : a.ncell;
        const bool f = gc < a.ncell && __ldcg(a.flag + __ldcg(a.cw.crid + gc)) != 0u;
        const uint32_t s = f ? __ldcg(a.cell_start + gc) : 0u, e = f ? __ldcg(a.cell_start + gc + 1) : 0u;
        unsigned m = __ballot_sync(kFull, f);
        while (m) {
            const int q = __ffs(m) - 1;
            m &= m - 1u;
            bcell_gather(__shfl_sync(kFull, s, q), __shfl_sync(kFull, e, q), a.cw, a.pos, a.vel, a.ids, a.perm);
        }
    }
}

// The flagged replicas as tables in shared memory (the end of the block's
// dynamic shared memory, clear of B2's counters): fr[q] the replica,
// pp[q] / cp[q] the particles / cells of fr[0..q) (pp[nf], cp[nf] the
// totals).  Binning, scatter and gather then visit only the flagged
// replicas' particles and cells.  All threads call it; returns false (no
// tables) when they do not fit.
struct BFlagTab {
    uint32_t *fr, *pp, *cp;
    uint32_t nf;
};

__device__ __forceinline__ bool bstep_tables(const BStepArgs &a, unsigned char *smem_raw, uint32_t nf, uint32_t *wsum,
                                             BFlagTab &t)
{
    const size_t need = (3 * (size_t)nf + 2) * sizeof(uint32_t);
    if ((size_t)a.cnt_bytes + need + 16 > (size_t)a.smem_bytes) return false;
    uint32_t *base = (uint32_t *)(smem_raw + (((size_t)a.smem_bytes - need) & ~(size_t)15));  // >= cnt_bytes
    t.fr = base;
    t.pp = base + nf;
    t.cp = base + 2 * nf + 1;
    t.nf = nf;
    uint32_t carry_p = 0, carry_c = 0;
    for (uint32_t b0 = 0; b0 < nf; b0 += blockDim.x) {
        const uint32_t q = b0 + threadIdx.x;
        uint32_t r = 0, np = 0, nc = 0;
        if (q < nf) {
            r = __ldcg(a.flist + q);
            np = (uint32_t)a.reps[r].n;
            nc = (uint32_t)a.reps[r].grid.ncell;
            t.fr[q] = r;
        }
        uint32_t tp, tc;
        const uint32_t op = block_exclusive_scan(np, wsum, &tp);
        const uint32_t oc = block_exclusive_scan(nc, wsum, &tc);
        if (q < nf) {
            t.pp[q] = carry_p + op;
            t.cp[q] = carry_c + oc;
        }
        carry_p += tp;
        carry_c += tc;
    }
    if (threadIdx.x == 0) {
        t.pp[nf] = carry_p;
        t.cp[nf] = carry_c;
    }
    __syncthreads();
    return true;
}

// The entry q of a prefix table with tab[q] <= j < tab[q + 1].
__device__ __forceinline__ uint32_t tab_find(const uint32_t *tab, uint32_t nf, uint32_t j)
{
    uint32_t lo = 0, hi = nf - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (tab[mid] <= j) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void bstep_bin_tab(const BStepArgs &a, const BFlagTab &t)
{
    const uint32_t P = t.pp[t.nf], stride = gridDim.x * blockDim.x;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < P; j += stride) {
        const uint32_t q = tab_find(t.pp, t.nf, j);
        const fpm_replica &rp = a.reps[t.fr[q]];
        const uint32_t k = j - t.pp[q], i = (uint32_t)rp.p0 + k;
        const BoxT<float> box = make_box<float>(rp.box);
        const GridD g = make_grid(rp.grid);
        const uint32_t c = bcell_bin(i, box, g, a.pos, a.vel, a.ids, a.cw, a.status);
        // one cell: the index order is the sorted order, and the count is n
        a.cw.rank[i] = rp.grid.ncell == 1 ? k : atomicAdd(&a.gcnt[rp.c0 + (int)c], 1u);
    }
}

__device__ __forceinline__ void bstep_scatter_tab(const BStepArgs &a, const BFlagTab &t)
{
    const uint32_t P = t.pp[t.nf], stride = gridDim.x * blockDim.x;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < P; j += stride) {
        const uint32_t q = tab_find(t.pp, t.nf, j);
        const fpm_replica &rp = a.reps[t.fr[q]];
        const uint32_t i = (uint32_t)rp.p0 + (j - t.pp[q]);
        if (rp.grid.ncell == 1) {
            // a replica of one cell keeps its index order: its particles go
            // straight into place here, by every thread, instead of through
            // one warp in the gather
            a.pos[i] = __ldcg(a.cw.spos + i);
            if (a.vel) a.vel[i] = __ldcg(a.cw.svel + i);
            if (a.ids) a.ids[i] = __ldcg(a.cw.sid + i);
            if (a.perm) a.perm[i] = i;
            continue;
        }
        const uint32_t c = __ldcg(a.cw.cell + i);
        a.cw.tmp[__ldcg(a.cell_start + rp.c0 + c) + __ldcg(a.cw.rank + i)] = i;
    }
}

// Warp w takes the flagged cells w, w + nw, ... (nw warps), 32 at a time.
__device__ __forceinline__ void bstep_gather_tab(const BStepArgs &a, const BFlagTab &t)
{
    const int lane = threadIdx.x & 31;
    const uint32_t C = t.cp[t.nf];
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    for (uint64_t j0 = 0; w + j0 * nw < C; j0 += 32) {
        const uint64_t jl = w + (j0 + lane) * nw;
        const bool f = jl < C;
        uint32_t s = 0, e = 0;
        if (f) {
            const uint32_t j = (uint32_t)jl, q = tab_find(t.cp, t.nf, j);
            const fpm_replica &rp = a.reps[t.fr[q]];
            if (rp.grid.ncell > 1) {  // (a replica of one cell was placed by the scatter)
                const int gc = rp.c0 + (int)(j - t.cp[q]);
                s = __ldcg(a.cell_start + gc);
                e = __ldcg(a.cell_start + gc + 1);
            }
        }
        unsigned m = __ballot_sync(kFull, f && e > s);
        while (m) {
            const int qq = __ffs(m) - 1;
            m &= m - 1u;
            bcell_gather(__shfl_sync(kFull, s, qq), __shfl_sync(kFull, e, qq), a.cw, a.pos, a.vel, a.ids, a.perm);
        }
    }
}

// MINB: blocks per SM the register allocation is bounded for (4: 64
// registers; 2: no bound in practice, half the warps).
template <int MINB>
__global__ void __launch_bounds__(kTileThreads, MINB) k_batch_step(BStepArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float4 *sp = (float4 *)smem_raw;        // CD: staged positions
    uint32_t *cnt = (uint32_t *)smem_raw;   // B2: cell counters
    __shared__ BScanShared ssh;
    __shared__ BLjShared lsh;
    __shared__ uint32_t wsum[32];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_k;
    __shared__ bool s_last;
    stage_init(&bar);
    uint32_t phase = 0;
    const int stride = (int)(gridDim.x * blockDim.x);
    // A
    for (int base = (int)(blockIdx.x * blockDim.x); base < a.n; base += stride)
        bdrift_one(base + (int)threadIdx.x, a.n, a.R, a.reps, a.hdt, a.dt, a.pos, a.vel, a.force, a.pos_ref, a.th,
                   a.flag, a.nflag, a.flist);
    if (!grid_sync(a.gbar, a.status)) return;
    const uint32_t nf = __ldcg(a.nflag);  // the same in every block
    const bool rebuild = nf != 0u;
    uint32_t ntodo = 0;
    if (rebuild) {
        BFlagTab t;
        const bool tab = bstep_tables(a, smem_raw, nf, wsum, t);  // the same in every block
        // B1
        if (tab) bstep_bin_tab(a, t);
        else bstep_bin(a);
        if (!grid_sync(a.gbar, a.status)) return;
        // B2
        for (uint32_t q = blockIdx.x; q < nf; q += gridDim.x) bstep_cell_scan(a, (int)__ldcg(a.flist + q), cnt, wsum);
        if (!grid_sync(a.gbar, a.status)) return;
        // B3
        if (tab) bstep_scatter_tab(a, t);
        else bstep_scatter(a);
        if (!grid_sync(a.gbar, a.status)) return;
        // B4 (the work lists, needed from CD on, by the last block: the
        // gather's cells are spread thinly enough to hide it)
        if (blockIdx.x == gridDim.x - 1)
            bwork_block(a.R, a.reps, a.flag, a.work, nullptr, a.header, a.status, false, wsum, a.unf, a.rep_scan);
        if (tab) bstep_gather_tab(a, t);
        else bstep_gather(a);
        if (!grid_sync(a.gbar, a.status)) return;
        for (int r = (int)(blockIdx.x * blockDim.x + threadIdx.x); r < a.R; r += stride) a.flag[r] = 0u;
        ntodo = __ldcg(a.header);
    } else if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.header[0] = 0u;  // an empty work list, as the separate build leaves it
    }
    // CD (with no replica flagged the queue is every force tile in tile order)
    const uint32_t nunf = (uint32_t)a.ntiles - ntodo;
    const uint32_t total = ntodo + (uint32_t)a.ntiles;
    // Tickets rise, so a block's scans all come before its force tiles: two
    // loops in turn over the one queue.
    uint32_t maxc = 0, ahead = 0;
    uint32_t k = blockIdx.x;
    for (; k < ntodo; k = ticket_next(ahead, &s_k)) {
        ahead = ticket_ahead(a.sched);
        bscan_tile(k, ssh, a.reps, a.map, a.pos, a.cell_start, a.rl2, a.cap, a.ld, a.stage_cap, a.work, a.words,
                   a.nn, a.pos_ref, a.descs, a.status, sp, &bar, phase, maxc);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(a.rep_scan + __ldcg(a.map + __ldcg(a.work + k)), 1u);
        }
    }
    for (; k < total; k = ticket_next(ahead, &s_k)) {
        ahead = ticket_ahead(a.sched);
        const uint32_t f = k - ntodo;
        const bool rebuilt = f >= nunf;
        const uint32_t t = !rebuild ? f : rebuilt ? __ldcg(a.work + (f - nunf)) : __ldcg(a.unf + f);
        if (rebuilt && threadIdx.x == 0) {  // wait until every tile of the replica is scanned
            const int r = (int)__ldcg(a.map + t);
            const uint32_t need = (uint32_t)rep_ntiles(a.reps[r].grid);
            const long long t0 = clock64();
            while (atomicAdd(a.rep_scan + r, 0u) < need) {
                if (clock64() - t0 > kWaitCycles) {
                    latch_flag(a.status, FPM_FLAG_TIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
            __threadfence();
        }
        __syncthreads();
        blj_tile(t, lsh, a.reps, a.map, a.pos, a.lv, a.nn, a.ld, a.stage_cap, a.P, a.force, a.part, a.rep_done,
                 a.out, a.status, a.vel, a.hdt, sp, &bar, phase);
    }
    const uint32_t m = __reduce_max_sync(kFull, maxc);
    if ((threadIdx.x & 31) == 0 && a.status && m > 0) atomicMax(&a.status->max_nn, m);
    // the last block to finish: every block has read nflag, so it is reset
    if (sched_finish(a.sched, &s_last) && threadIdx.x == 0) *a.nflag = 0u;
}

// ---- host side -------------------------------------------------------------

struct BatchWs {
    Sched sched;
    double *part;
    uint32_t *rep_done;
};

// Force workspace: counters (bytes 16, 32, 48), the per-tile sums, the
// per-replica completion counters, and for the one-launch step the tiles of
// the replicas not rebuilt, the per-replica scanned-tile counters and the
// list of the flagged replicas.
static size_t bws_layout(const fpm_batch &b, size_t *off_done, size_t *off_unf = nullptr,
                         size_t *off_scan = nullptr, size_t *off_flist = nullptr)
{
    size_t o = 256 + (size_t)b.ntiles_total * 3 * sizeof(double);
    o = (o + 255) & ~(size_t)255;
    if (off_done) *off_done = o;
    o = (o + (size_t)b.R * sizeof(uint32_t) + 255) & ~(size_t)255;
    if (off_unf) *off_unf = o;
    o = (o + (size_t)b.ntiles_total * sizeof(uint32_t) + 255) & ~(size_t)255;
    if (off_scan) *off_scan = o;
    o = (o + (size_t)b.R * sizeof(uint32_t) + 255) & ~(size_t)255;
    if (off_flist) *off_flist = o;
    return o + (size_t)b.R * sizeof(uint32_t);
}

// Cell workspace: the binned copies (pos, vel, id), cell, rank, scattered
// index and replica per particle, the replica per cell, and the one-launch
// step's cell counters.
constexpr int kBcellRegions = 9;
static size_t bcell_layout(const fpm_batch &b, size_t off[kBcellRegions])
{
    const size_t n = (size_t)b.n_total, nc = (size_t)b.ncell_total;
    size_t o = 0;
    const size_t sz[kBcellRegions] = {n * 16, n * 16, n * 4, n * 4, n * 4, n * 4, n * 4, nc * 4, nc * 4};
    for (int k = 0; k < kBcellRegions; ++k) {
        off[k] = o;
        o = (o + sz[k] + 255) & ~(size_t)255;
    }
    return o;
}

static fpm_status batch_ok(const fpm_batch *b, const fpm_replica *d_reps, const char *who)
{
    if (!b || !d_reps || b->R < 1 || b->R > kBatchMaxReplicas || b->n_total < 0 || b->ncell_total < b->R ||
        b->ntiles_total < b->R || b->max_ncell < 1 || b->max_ncell > kBatchMaxCells)
        return fpm_fail(FPM_ERR_INVALID, "%s: bad batch", who);
    if (b->sweep_threads != 0 && b->sweep_threads != 128 && b->sweep_threads != 256 && b->sweep_threads != 512)
        return fpm_fail(FPM_ERR_INVALID, "%s: sweep_threads must be 0, 128, 256 or 512", who);
    if (b->step_blocks_per_sm < 0 || b->step_blocks_per_sm == 1 || b->step_blocks_per_sm > 4)
        return fpm_fail(FPM_ERR_INVALID, "%s: step_blocks_per_sm must be 0, 2, 3 or 4", who);
    return FPM_OK;
}

static int batch_stage_cap(const fpm_batch &b)
{
    const int maxe = (int)((size_t)kSmemBudget / sizeof(float4)) / 32 * 32;
    int e = b.stage_cap > 0 ? (b.stage_cap + 31) / 32 * 32 : maxe;
    return e > maxe ? maxe : e;
}

}  // namespace fpm

using namespace fpm;

extern "C" fpm_status fpm_batch_plan(int32_t R, const fpm_box *boxes, const int32_t *counts, double r_cell,
                                     int32_t tile_target, fpm_replica *reps, fpm_batch *batch)
{
    if (R < 1 || R > kBatchMaxReplicas || !boxes || !counts || !reps || !batch || !(r_cell > 0.0) ||
        tile_target < 0)
        return fpm_fail(FPM_ERR_INVALID, "fpm_batch_plan: bad argument");
    const double target = tile_target > 0 ? (double)tile_target : (double)kTileTarget;
    int64_t p0 = 0, c0 = 0, t0 = 0;
    int max_n = 0, max_ncell = 0, stage = 0;
    for (int r = 0; r < R; ++r) {
        const fpm_box &b = boxes[r];
        if (!b.periodic[0] || !b.periodic[1] || !b.periodic[2])
            return fpm_fail(FPM_ERR_INVALID, "fpm_batch_plan: replica %d is not periodic in every dimension", r);
        if (counts[r] < 0) return fpm_fail(FPM_ERR_INVALID, "fpm_batch_plan: counts[%d] < 0", r);
        fpm_grid g{};
        const fpm_status s = fpm_grid_make(&b, r_cell, counts[r], &g);
        if (s != FPM_OK) return s;
        if (g.ncell > kBatchMaxCells)
            return fpm_fail(FPM_ERR_INVALID, "fpm_batch_plan: replica %d has %d cells (limit %d)", r, g.ncell,
                            kBatchMaxCells);
        // tile width along x: about `target` particles per tile, at most 14 cells
        const double per_cell = counts[r] > 0 ? (double)counts[r] / (double)g.ncell : 1.0;
        int w = (int)std::lround(target / per_cell);
        w = std::max(1, std::min(kMaxTileCells, w));
        g.tiles_x = std::max(1, (g.nc[0] + w - 1) / w);
        g.stage_cap = 0;
        g.sweep_blocks = 0;
        reps[r].box = b;
        reps[r].grid = g;
        reps[r].p0 = (int32_t)p0;
        reps[r].n = counts[r];
        reps[r].c0 = (int32_t)c0;
        reps[r].t0 = (int32_t)t0;
        p0 += counts[r];
        c0 += g.ncell;
        t0 += rep_ntiles(g);
        if (p0 > (int64_t)INT32_MAX / 2 || c0 >= (int64_t)INT32_MAX / 2 || t0 >= (int64_t)INT32_MAX / 2)
            return fpm_fail(FPM_ERR_INVALID, "fpm_batch_plan: batch too large");
        max_n = std::max(max_n, counts[r]);
        max_ncell = std::max(max_ncell, g.ncell);
        stage = std::max(stage, stage_capacity(counts[r], g, sizeof(float4)));
    }
    batch->R = R;
    batch->n_total = (int32_t)p0;
    batch->ncell_total = (int32_t)c0;
    batch->ntiles_total = (int32_t)t0;
    batch->max_n = max_n;
    batch->max_ncell = max_ncell;
    batch->stage_cap = stage;
    batch->sweep_blocks = 0;
    batch->sweep_threads = 0;
    batch->step_blocks_per_sm = 0;
    return FPM_OK;
}

extern "C" fpm_status fpm_batch_drift_check(const fpm_batch *batch, const fpm_replica *d_reps, double dt, void *pos,
                                            void *vel, const void *force, const void *pos_ref, double skin,
                                            uint32_t *d_rep_flag, fpm_stream stream)
{
    fpm_status s = batch_ok(batch, d_reps, "fpm_batch_drift_check");
    if (s != FPM_OK) return s;
    const int n = batch->n_total;
    if (!d_rep_flag || !(skin >= 0.0) || (n > 0 && (!pos || !vel || !force || !pos_ref)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_batch_drift_check: null pointer or bad argument");
    if (n == 0) return FPM_OK;
    k_bdrift_check<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        n, batch->R, d_reps, (float)(0.5 * dt), (float)dt, (float4 *)pos, (float4 *)vel, (const float4 *)force,
        (const float4 *)pos_ref, (float)(0.25 * skin * skin), d_rep_flag);
    return fpm_check_launch("fpm_batch_drift_check");
}

extern "C" fpm_status fpm_batch_celllist_workspace(const fpm_batch *batch, size_t *bytes)
{
    if (!batch || !bytes || batch->n_total < 0) return fpm_fail(FPM_ERR_INVALID, "fpm_batch_celllist_workspace");
    size_t off[kBcellRegions];
    *bytes = bcell_layout(*batch, off);
    return FPM_OK;
}

extern "C" fpm_status fpm_batch_celllist_build(const fpm_batch *batch, const fpm_replica *d_reps, void *pos,
                                               void *vel, uint32_t *ids, uint32_t *cell_start, uint32_t *perm,
                                               void *workspace, size_t workspace_bytes, const uint32_t *d_rep_flag,
                                               fpm_dev_status *d_status, fpm_stream stream)
{
    fpm_status s = batch_ok(batch, d_reps, "fpm_batch_celllist_build");
    if (s != FPM_OK) return s;
    if (!cell_start || (batch->n_total > 0 && !pos))
        return fpm_fail(FPM_ERR_INVALID, "fpm_batch_celllist_build: null pointer");
    size_t off[kBcellRegions];
    const size_t need = bcell_layout(*batch, off);
    if (!workspace || workspace_bytes < need)
        return fpm_fail(FPM_ERR_WORKSPACE, "fpm_batch_celllist_build: workspace %zu < %zu bytes", workspace_bytes,
                        need);
    if (((uintptr_t)workspace & 15u) != 0)
        return fpm_fail(FPM_ERR_WORKSPACE, "fpm_batch_celllist_build: workspace not 16-B aligned");
    char *w = (char *)workspace;
    BCellWs ws{(float4 *)(w + off[0]), (float4 *)(w + off[1]), (uint32_t *)(w + off[2]),
               (uint32_t *)(w + off[3]), (uint32_t *)(w + off[4]), (uint32_t *)(w + off[5]),
               (uint32_t *)(w + off[6]), (uint32_t *)(w + off[7])};
    const size_t smem = ((size_t)batch->max_ncell + 1) * sizeof(uint32_t);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute((const void *)k_bcell, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_bcell<<<batch->R, kBatchCellThreads, smem, (cudaStream_t)stream>>>(batch->R, d_reps, (float4 *)pos,
                                                                         (float4 *)vel, ids, cell_start, perm, ws,
                                                                         d_rep_flag, d_status);
    return fpm_check_launch("fpm_batch_celllist_build");
}

// The batch's Verlet-list object: the single-system layout (header, tile
// descriptors, work list, ELL words) with one more region after the work
// list: the tile -> replica map (ntiles_total uint32).
static ListLayout batch_list_layout(const fpm_batch &b, int cap, size_t *off_map = nullptr)
{
    ListLayout L{};
    const size_t nt = (size_t)b.ntiles_total;
    L.ld = fpm_nbr_ld(b.n_total);
    L.words_per_particle = (cap + 1) / 2;
    L.off_tiles = 256;
    size_t t = L.off_tiles + nt * sizeof(TileDesc);
    L.off_active = (t + 255) & ~(size_t)255;
    t = L.off_active + nt * 4;
    const size_t om = (t + 255) & ~(size_t)255;
    if (off_map) *off_map = om;
    t = om + nt * 4;
    L.off_words = (t + 255) & ~(size_t)255;
    L.total = L.off_words + (size_t)L.words_per_particle * (size_t)L.ld * 4;
    return L;
}

extern "C" fpm_status fpm_batch_list_bytes(const fpm_batch *batch, int32_t cap, size_t *bytes)
{
    if (!batch || !bytes || cap < 1 || batch->ntiles_total < 1)
        return fpm_fail(FPM_ERR_INVALID, "fpm_batch_list_bytes: bad argument");
    *bytes = batch_list_layout(*batch, cap).total;
    return FPM_OK;
}

extern "C" fpm_status fpm_batch_verlet_build(const fpm_batch *batch, const fpm_replica *d_reps, const void *pos,
                                             const uint32_t *cell_start, double r_list, int32_t cap, void *list,
                                             size_t list_bytes, uint32_t *nn, void *pos_ref, uint32_t *d_rep_flag,
                                             fpm_dev_status *d_status, fpm_stream stream)
{
    fpm_status s = batch_ok(batch, d_reps, "fpm_batch_verlet_build");
    if (s != FPM_OK) return s;
    if (cap < 1 || !(r_list > 0.0) || !cell_start || !list || (batch->n_total > 0 && (!pos || !nn)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_batch_verlet_build: null pointer or bad size");
    const ListLayout L = batch_list_layout(*batch, cap);
    if (list_bytes < L.total)
        return fpm_fail(FPM_ERR_WORKSPACE, "fpm_batch_verlet_build: list object %zu < %zu bytes", list_bytes,
                        L.total);
    if (((uintptr_t)list & 255u) != 0)
        return fpm_fail(FPM_ERR_INVALID, "fpm_batch_verlet_build: list not 256-B aligned");
    cudaStream_t st = (cudaStream_t)stream;
    size_t off_map = 0;
    batch_list_layout(*batch, cap, &off_map);
    char *lb = (char *)list;
    TileDesc *descs = (TileDesc *)(lb + L.off_tiles);
    uint32_t *work = (uint32_t *)(lb + L.off_active);
    uint32_t *map = (uint32_t *)(lb + off_map);
    uint32_t *header = (uint32_t *)lb;
    const int R = batch->R;
    const int nt = batch->ntiles_total;
    k_bwork<<<1, 1024, 0, st>>>(R, d_reps, d_rep_flag, work, map, header, d_status);
    const int sc = batch_stage_cap(*batch);
    const size_t smem = (size_t)sc * sizeof(float4);
    smem_opt_in((const void *)k_bverlet_scan);
    fpm_grid gg{};
    gg.sweep_blocks = batch->sweep_blocks;
    const int blocks = persistent_blocks((const void *)k_bverlet_scan, kTileThreads, smem, gg, nt);
    k_bverlet_scan<<<blocks, kTileThreads, smem, st>>>(d_reps, map, (const float4 *)pos, cell_start,
                                                       (float)(r_list * r_list), cap, L.ld, sc, work, header,
                                                       Sched{(unsigned *)(lb + 16), (unsigned *)(lb + 20)},
                                                       (uint32_t *)(lb + L.off_words), nn, (float4 *)pos_ref,
                                                       descs, d_status);
    return fpm_check_launch("fpm_batch_verlet_build");
}

extern "C" fpm_status fpm_batch_verlet_decode(const fpm_batch *batch, int32_t cap, const void *list,
                                              const uint32_t *nn, uint32_t *out, fpm_stream stream)
{
    if (!batch || cap < 1 || !list || !nn || !out || batch->ntiles_total < 1)
        return fpm_fail(FPM_ERR_INVALID, "fpm_batch_verlet_decode: bad argument");
    const ListLayout L = batch_list_layout(*batch, cap);
    return verlet_decode_launch((const TileDesc *)((const char *)list + L.off_tiles),
                                (const uint32_t *)((const char *)list + L.off_words), nn, L.ld, out,
                                batch->ntiles_total, (cudaStream_t)stream);
}

extern "C" fpm_status fpm_batch_workspace(const fpm_batch *batch, size_t *bytes)
{
    if (!batch || !bytes || batch->R < 1 || batch->ntiles_total < 1)
        return fpm_fail(FPM_ERR_INVALID, "fpm_batch_workspace: bad argument");
    *bytes = bws_layout(*batch, nullptr);
    return FPM_OK;
}

static fpm_status batch_lj(const fpm_batch *batch, const fpm_replica *d_reps, const void *pos, const void *list,
                           const uint32_t *nn, int32_t cap, double eps, double sigma, double rc, void *force,
                           double *d_energy, void *workspace, size_t workspace_bytes, fpm_dev_status *d_status,
                           void *vel, double dt, fpm_stream stream)
{
    fpm_status s = batch_ok(batch, d_reps, "fpm_batch_lj_forces");
    if (s != FPM_OK) return s;
    if (cap < 1 || !(rc > 0.0) || !(sigma > 0.0) || !list || (batch->n_total > 0 && (!pos || !nn || !force)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_batch_lj_forces: null pointer or bad size");
    if (((uintptr_t)list & 255u) != 0) return fpm_fail(FPM_ERR_INVALID, "fpm_batch_lj_forces: list not aligned");
    size_t off_done = 0;
    const size_t need = bws_layout(*batch, &off_done);
    if (!workspace || workspace_bytes < need)
        return fpm_fail(FPM_ERR_WORKSPACE, "fpm_batch_lj_forces: workspace %zu < %zu bytes", workspace_bytes, need);
    if (((uintptr_t)workspace & 15u) != 0)
        return fpm_fail(FPM_ERR_WORKSPACE, "fpm_batch_lj_forces: workspace not 16-B aligned");
    char *w = (char *)workspace;
    size_t off_map = 0;
    const ListLayout L = batch_list_layout(*batch, cap, &off_map);
    LJParams<float> P;
    P.eps24 = (float)(24.0 * eps);
    P.eps4 = (float)(4.0 * eps);
    P.sig2 = (float)(sigma * sigma);
    P.rc2 = (float)(rc * rc);
    const int sc = batch_stage_cap(*batch);
    const size_t smem = (size_t)sc * sizeof(float4);
    const int threads = batch->sweep_threads == 0 ? 256 : batch->sweep_threads;
    auto kern = threads == 128 ? k_blj_tiles<128> : threads == 512 ? k_blj_tiles<512> : k_blj_tiles<256>;
    smem_opt_in((const void *)kern);
    fpm_grid gg{};
    gg.sweep_blocks = batch->sweep_blocks;
    const int nt = batch->ntiles_total;
    const int blocks = persistent_blocks((const void *)kern, threads, smem, gg, nt);
    kern<<<blocks, threads, smem, (cudaStream_t)stream>>>(
        nt, d_reps, (const uint32_t *)((const char *)list + off_map), (const float4 *)pos, list_view(list, L), nn,
        L.ld, sc, P, (float4 *)force,
        Sched{(unsigned *)(w + 16), (unsigned *)(w + 32)}, (double *)(w + 256), (uint32_t *)(w + off_done),
        d_energy, d_status, (float4 *)vel, (float)(0.5 * dt));
    return fpm_check_launch("fpm_batch_lj_forces");
}

extern "C" fpm_status fpm_batch_lj_forces(const fpm_batch *batch, const fpm_replica *d_reps, const void *pos,
                                          const void *list, const uint32_t *nn, int32_t cap, double eps,
                                          double sigma, double rc, void *force, double *d_energy, void *workspace,
                                          size_t workspace_bytes, fpm_dev_status *d_status, fpm_stream stream)
{
    return batch_lj(batch, d_reps, pos, list, nn, cap, eps, sigma, rc, force, d_energy, workspace, workspace_bytes,
                    d_status, nullptr, 0.0, stream);
}

extern "C" fpm_status fpm_batch_lj_forces_kick(const fpm_batch *batch, const fpm_replica *d_reps, const void *pos,
                                               const void *list, const uint32_t *nn, int32_t cap, double eps,
                                               double sigma, double rc, void *force, double *d_energy,
                                               void *workspace, size_t workspace_bytes, fpm_dev_status *d_status,
                                               void *vel, double dt, fpm_stream stream)
{
    if (!batch || (batch->n_total > 0 && !vel) || (vel && (vel == pos || vel == force)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_batch_lj_forces_kick: null vel, or vel aliases pos or force");
    return batch_lj(batch, d_reps, pos, list, nn, cap, eps, sigma, rc, force, d_energy, workspace, workspace_bytes,
                    d_status, vel, dt, stream);
}

extern "C" fpm_status fpm_batch_step(const fpm_batch *batch, const fpm_replica *d_reps, double dt, double skin,
                                     double r_list, int32_t cap, double eps, double sigma, double rc, void *pos,
                                     void *vel, void *force, void *pos_ref, uint32_t *ids, uint32_t *cell_start,
                                     uint32_t *perm, void *list, size_t list_bytes, uint32_t *nn,
                                     uint32_t *d_rep_flag, void *cell_ws, size_t cell_ws_bytes, void *workspace,
                                     size_t workspace_bytes, double *d_energy, fpm_dev_status *d_status,
                                     fpm_stream stream)
{
    fpm_status s = batch_ok(batch, d_reps, "fpm_batch_step");
    if (s != FPM_OK) return s;
    const int n = batch->n_total;
    if (cap < 1 || !(r_list > 0.0) || !(rc > 0.0) || !(sigma > 0.0) || !(skin >= 0.0) || !list || !cell_start ||
        !d_rep_flag || (n > 0 && (!pos || !vel || !force || !pos_ref || !nn)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_batch_step: null pointer or bad argument");
    if (n > 0 && (vel == pos || vel == force || pos == force))
        return fpm_fail(FPM_ERR_INVALID, "fpm_batch_step: pos, vel and force must be distinct");
    const ListLayout L = batch_list_layout(*batch, cap);
    if (list_bytes < L.total)
        return fpm_fail(FPM_ERR_WORKSPACE, "fpm_batch_step: list object %zu < %zu bytes", list_bytes, L.total);
    if (((uintptr_t)list & 255u) != 0) return fpm_fail(FPM_ERR_INVALID, "fpm_batch_step: list not 256-B aligned");
    size_t coff[kBcellRegions];
    const size_t cneed = bcell_layout(*batch, coff);
    if (!cell_ws || cell_ws_bytes < cneed || ((uintptr_t)cell_ws & 15u) != 0)
        return fpm_fail(FPM_ERR_WORKSPACE, "fpm_batch_step: cell workspace %zu < %zu bytes or not 16-B aligned",
                        cell_ws_bytes, cneed);
    size_t off_done = 0, off_unf = 0, off_scan = 0, off_flist = 0;
    const size_t need = bws_layout(*batch, &off_done, &off_unf, &off_scan, &off_flist);
    if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 15u) != 0)
        return fpm_fail(FPM_ERR_WORKSPACE, "fpm_batch_step: workspace %zu < %zu bytes or not 16-B aligned",
                        workspace_bytes, need);
    if (n == 0) return FPM_OK;

    size_t off_map = 0;
    batch_list_layout(*batch, cap, &off_map);
    char *lb = (char *)list, *cw = (char *)cell_ws, *w = (char *)workspace;
    BStepArgs a{};
    a.n = n;
    a.R = batch->R;
    a.ntiles = batch->ntiles_total;
    a.ncell = batch->ncell_total;
    a.cap = cap;
    a.stage_cap = batch_stage_cap(*batch);
    a.ld = L.ld;
    a.reps = d_reps;
    a.hdt = (float)(0.5 * dt);
    a.dt = (float)dt;
    a.th = (float)(0.25 * skin * skin);
    a.rl2 = (float)(r_list * r_list);
    a.pos = (float4 *)pos;
    a.vel = (float4 *)vel;
    a.force = (float4 *)force;
    a.pos_ref = (float4 *)pos_ref;
    a.ids = ids;
    a.cell_start = cell_start;
    a.perm = perm;
    a.flag = d_rep_flag;
    a.cw = BCellWs{(float4 *)(cw + coff[0]), (float4 *)(cw + coff[1]), (uint32_t *)(cw + coff[2]),
                   (uint32_t *)(cw + coff[3]), (uint32_t *)(cw + coff[4]), (uint32_t *)(cw + coff[5]),
                   (uint32_t *)(cw + coff[6]), (uint32_t *)(cw + coff[7])};
    a.gcnt = (uint32_t *)(cw + coff[8]);
    a.header = (uint32_t *)lb;
    a.work = (uint32_t *)(lb + L.off_active);
    a.map = (uint32_t *)(lb + off_map);
    a.words = (uint32_t *)(lb + L.off_words);
    a.nn = nn;
    a.descs = (TileDesc *)(lb + L.off_tiles);
    a.lv = list_view(list, L);
    a.P.eps24 = (float)(24.0 * eps);
    a.P.eps4 = (float)(4.0 * eps);
    a.P.sig2 = (float)(sigma * sigma);
    a.P.rc2 = (float)(rc * rc);
    a.sched = Sched{(unsigned *)(w + 16), (unsigned *)(w + 32)};
    a.part = (double *)(w + 256);
    a.rep_done = (uint32_t *)(w + off_done);
    a.unf = (uint32_t *)(w + off_unf);
    a.rep_scan = (uint32_t *)(w + off_scan);
    a.out = d_energy;
    a.status = d_status;
    a.gbar = (unsigned *)(lb + 32);
    a.nflag = (uint32_t *)(w + 48);
    a.flist = (uint32_t *)(w + off_flist);

    // Every block must be resident at once (the grid barriers): the grid is
    // the occupancy limit, or sweep_blocks when that is smaller, and the
    // launch is cooperative, so an oversized grid is refused, never run.
    const size_t cnt_bytes = ((size_t)batch->max_ncell + 1) * sizeof(uint32_t);
    const size_t stage_bytes = (size_t)a.stage_cap * sizeof(float4);
    const size_t smem = cnt_bytes > stage_bytes ? cnt_bytes : stage_bytes;
    a.smem_bytes = (int)smem;
    a.cnt_bytes = (int)cnt_bytes;
    const int minb = batch->step_blocks_per_sm == 0 ? 4 : batch->step_blocks_per_sm;
    auto kern = minb == 2 ? k_batch_step<2> : minb == 3 ? k_batch_step<3> : k_batch_step<4>;
    smem_opt_in((const void *)kern);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTileThreads, smem);
    if (per_sm < 1 || sms < 1)
        return fpm_fail(FPM_ERR_CUDA, "fpm_batch_step: the step kernel does not fit one SM (%zu B shared)", smem);
    int blocks = sms * per_sm;
    if (batch->sweep_blocks > 0 && batch->sweep_blocks < blocks) blocks = batch->sweep_blocks;
    cudaLaunchConfig_t lc{};
    lc.gridDim = dim3((unsigned)blocks);
    lc.blockDim = dim3(kTileThreads);
    lc.dynamicSmemBytes = smem;
    lc.stream = (cudaStream_t)stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&lc, kern, a);
    if (e != cudaSuccess) return fpm_fail(FPM_ERR_CUDA, "fpm_batch_step: launch: %s", cudaGetErrorString(e));
    return fpm_check_launch("fpm_batch_step");
}
