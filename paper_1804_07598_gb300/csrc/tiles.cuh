// tiles.cuh -- cell tiles shared by the Verlet build and the pair sweeps.
//
// A tile is a run of consecutive cells [a, b) along x in one (cy, cz) row of
// the cell grid.  Its "neighbourhood" is every cell of the 27-cell stencils of
// its cells: for each of the (up to) 9 stencil rows (dz, dy), the x cells
// a-1 .. b.  Because particles are sorted by cell, each stencil row is one to
// three contiguous index ranges ("pieces": the cell below x = 0 seen through
// the periodic wall, the interior run, the cell above ncx-1 seen through the
// wall).  A block stages the neighbourhood's positions into shared memory in
// that fixed order, and the Verlet list stores 16-bit indices into it.
//
// Periodic images are resolved by the stencil geometry, never by comparing
// coordinates.  In every periodic dimension with nc >= 3 ("wrap" mode) a
// neighbour reached through the lower wall is staged as x_j - L, and one
// reached through the upper wall keeps x_j but carries a flag telling the
// pair code to use x_i - L for the home particle.  Both shifts are exact (the
// shifted coordinate lies within a factor 2 of L), so the separation is
//     x_i - (x_j - L)   or   (x_i - L) - x_j
// with one rounding: the minimum-image separation as the oracle defines it.
// A periodic dimension with nc == 1 ("all" mode) holds every particle in the
// one cell and the pair code chooses the image by comparing with L/2.
//
// Positions must not be wrapped between a Verlet build and the sweeps that
// use its list (the drift of fpm_vv_step does not wrap; the cell-list build
// does): the image choice is frozen at build time.
#pragma once

#include <climits>

#include "fpm_common.cuh"

namespace fpm {

enum : int { kModeOpen = 0, kModeWrap = 1, kModeAll = 2 };

constexpr int kTileThreads = 256;          // threads per tile block (one per home particle)
constexpr int kTileTarget = 200;           // particles per tile the grid's tile width aims at (a tile
                                           // stays below kTileThreads, so no thread takes two particles)
constexpr int kMaxTileCells = 14;          // home cells per tile along x
constexpr int kMaxSeq = kMaxTileCells + 2; // staged cells per stencil row
constexpr int kMaxRows = 9;
constexpr int kPiecesPerRow = 3;
constexpr int kMaxPieces = kMaxRows * kPiecesPerRow;
constexpr int kMaxStaged = 65535;          // 16-bit list entries
constexpr int kSmemBudget = 200 * 1024;    // dynamic shared memory per tile block

// flags of a staged particle / piece (stored in the staged w component)
constexpr int kUpX = 1, kUpY = 2, kUpZ = 4;        // home uses x_i - L in that dim
constexpr int kLoX = 8, kLoY = 16, kLoZ = 32;      // staged as x_j - L in that dim

struct TileCfg {
    int nc[3];
    int mode[3];
    int tiles_x;
    int ntiles;
};

__host__ __device__ inline TileCfg make_tile_cfg(const fpm_box &b, const fpm_grid &g)
{
    TileCfg c{};
    for (int d = 0; d < 3; ++d) {
        c.nc[d] = g.nc[d];
        c.mode[d] = !b.periodic[d] ? kModeOpen : (g.nc[d] == 1 ? kModeAll : kModeWrap);
    }
    c.tiles_x = g.tiles_x;
    c.ntiles = g.tiles_x * g.nc[1] * g.nc[2];
    return c;
}

// One piece of a tile's neighbourhood: staged slots [soff, soff+len) hold
// particles [gstart, gstart+len) of the sorted arrays.
struct Piece {
    int soff;
    int len;
    uint32_t gstart;
    int flags;
};

// Per-tile descriptor written by the Verlet build and read by the sweeps.
struct TileDesc {
    uint32_t h0, h1;  // home particles [h0, h1)
    int M;            // staged particles
    int slow;         // 1 if any piece has kUp* flags or a dimension is in "all" mode
    Piece piece[kMaxPieces];
};

// Layout of a Verlet-list object in caller memory:
//   [0, 4)                          number of non-empty tiles
//   [16, 24)                        scheduling counters of the Verlet scan
//   [256, 256 + ntiles*sizeof(TileDesc))  tile descriptors
//   then ntiles uint32: the non-empty tiles in increasing order
//   then the ELL words: entry k of particle i is the 16-bit half (k & 1) of
//   word (k >> 1) * ld + i.
struct ListLayout {
    size_t off_tiles, off_active, off_words, total;
    int64_t ld;
    int words_per_particle;
};

inline ListLayout list_layout(int n, const TileCfg &c, int cap)
{
    ListLayout L{};
    L.ld = fpm_nbr_ld(n);
    L.words_per_particle = (cap + 1) / 2;
    L.off_tiles = 256;
    size_t t = L.off_tiles + (size_t)c.ntiles * sizeof(TileDesc);
    L.off_active = (t + 255) & ~(size_t)255;
    t = L.off_active + (size_t)c.ntiles * 4;
    L.off_words = (t + 255) & ~(size_t)255;
    L.total = L.off_words + (size_t)L.words_per_particle * (size_t)L.ld * 4;
    return L;
}

// Pointers into a list object.
struct ListView {
    const uint32_t *count;
    const TileDesc *descs;
    const uint32_t *active;
    const uint32_t *words;
};

inline ListView list_view(const void *list, const ListLayout &L)
{
    const char *b = (const char *)list;
    return ListView{(const uint32_t *)b, (const TileDesc *)(b + L.off_tiles), (const uint32_t *)(b + L.off_active),
                    (const uint32_t *)(b + L.off_words)};
}

// Stencil offsets of one row dimension: cell index and wrap class (-1: seen
// through the lower wall, +1: through the upper wall, 0: direct).  Returns the
// count and the index of the zero offset in *mid.
__device__ __forceinline__ int stencil_rows(int c, int nc, int mode, int cell[3], int wrap[3], int *mid)
{
    if (mode == kModeAll) {
        cell[0] = 0;
        wrap[0] = 0;
        *mid = 0;
        return 1;
    }
    int k = 0;
    for (int o = -1; o <= 1; ++o) {
        int cc = c + o, w = 0;
        if (mode == kModeWrap) {
            if (cc < 0) { cc += nc; w = -1; }
            else if (cc >= nc) { cc -= nc; w = 1; }
        } else if (cc < 0 || cc >= nc) {
            continue;
        }
        if (o == 0) *mid = k;
        cell[k] = cc;
        wrap[k] = w;
        ++k;
    }
    return k;
}

// Full tile geometry, built in shared memory by the Verlet build.
struct TileGeom {
    int nrows, nseq, seq_start, a, b, mid_row, M;
    int row_cy[kMaxRows], row_cz[kMaxRows], row_wy[kMaxRows], row_wz[kMaxRows];
    uint32_t start[kMaxRows][kMaxSeq];  // first sorted index of each staged cell
    int cnt[kMaxRows][kMaxSeq];
    int off[kMaxRows][kMaxSeq + 1];     // staged offset of each staged cell
};

__device__ __forceinline__ int seq_cell_x(int x, int ncx, int mode, int *wrap)
{
    *wrap = 0;
    if (mode == kModeWrap) {
        if (x < 0) { *wrap = -1; return x + ncx; }
        if (x >= ncx) { *wrap = 1; return x - ncx; }
    }
    return x;
}

// The stencil rows of a half-list tile (each pair once): the offsets
// (dz, dy) = (0, 0), (0, +1), (+1, -1), (+1, 0), (+1, +1), lexicographically
// after or equal to (0, 0), each kept if it exists (open boundaries) and
// distinct (an "all"-mode dimension has the single offset 0).  Row 0 is the
// tile's own row.  Returns the count.
__device__ __forceinline__ int half_rows(int cy, int cz, const TileCfg &cfg, int *rcy, int *rcz, int *rwy, int *rwz)
{
    int k = 0;
    for (int oz = 0; oz <= 1; ++oz) {
        if (oz == 1 && cfg.mode[2] == kModeAll) continue;
        int z = cz + oz, wz = 0;
        if (z >= cfg.nc[2]) {
            if (cfg.mode[2] != kModeWrap) continue;
            z -= cfg.nc[2];
            wz = 1;
        }
        for (int oy = (oz == 0 ? 0 : -1); oy <= 1; ++oy) {
            if (oy != 0 && cfg.mode[1] == kModeAll) continue;
            int y = cy + oy, wy = 0;
            if (y < 0 || y >= cfg.nc[1]) {
                if (cfg.mode[1] != kModeWrap) continue;
                if (y < 0) {
                    y += cfg.nc[1];
                    wy = -1;
                } else {
                    y -= cfg.nc[1];
                    wy = 1;
                }
            }
            rcy[k] = y;
            rcz[k] = z;
            rwy[k] = wy;
            rwz[k] = wz;
            ++k;
        }
    }
    return k;
}

// Computes the geometry of `tile` and its descriptor (in shared memory).  All
// threads of the block must call it.  HALF: the rows of a half-list tile
// (half_rows), and every piece staged at an offset of the parity of its
// first particle index, with a free slot after a piece that ends on an odd
// index, so that a piece's slots cover the even-aligned index range
// [gstart & ~1, (gstart + len + 1) & ~1) of a per-particle array (the
// half-list sweep returns its reactions per piece in that form); the free
// slots belong to no piece.
template <bool HALF = false>
__device__ inline void tile_geometry(const TileCfg &cfg, int tile, const uint32_t *__restrict__ cs, TileGeom &g,
                              TileDesc &d)
{
    const int tid = threadIdx.x;
    if (tid == 0) {
        const int tx = tile % cfg.tiles_x, row = tile / cfg.tiles_x;
        const int cy = row % cfg.nc[1], cz = row / cfg.nc[1];
        const int ncx = cfg.nc[0];
        const int a = (int)((int64_t)tx * ncx / cfg.tiles_x), b = (int)((int64_t)(tx + 1) * ncx / cfg.tiles_x);
        g.a = a;
        g.b = b;
        if (cfg.mode[0] == kModeAll) {
            g.seq_start = 0;
            g.nseq = 1;
        } else if (cfg.mode[0] == kModeWrap) {
            g.seq_start = a - 1;
            g.nseq = b - a + 2;
        } else {
            const int s = a > 0 ? a - 1 : 0, e = b < ncx ? b + 1 : ncx;
            g.seq_start = s;
            g.nseq = e - s;
        }
        if (HALF) {
            g.nrows = half_rows(cy, cz, cfg, g.row_cy, g.row_cz, g.row_wy, g.row_wz);
            g.mid_row = 0;
        } else {
            int zc[3], zw[3], yc[3], yw[3], zmid = 0, ymid = 0;
            const int kz = stencil_rows(cz, cfg.nc[2], cfg.mode[2], zc, zw, &zmid);
            const int ky = stencil_rows(cy, cfg.nc[1], cfg.mode[1], yc, yw, &ymid);
            int r = 0;
            for (int i = 0; i < kz; ++i)
                for (int j = 0; j < ky; ++j) {
                    g.row_cy[r] = yc[j];
                    g.row_cz[r] = zc[i];
                    g.row_wy[r] = yw[j];
                    g.row_wz[r] = zw[i];
                    if (i == zmid && j == ymid) g.mid_row = r;
                    ++r;
                }
            g.nrows = r;
        }
    }
    __syncthreads();
    const int tot = g.nrows * g.nseq;
    for (int k = tid; k < tot; k += blockDim.x) {
        const int r = k / g.nseq, t = k - r * g.nseq;
        int w;
        const int x = seq_cell_x(g.seq_start + t, cfg.nc[0], cfg.mode[0], &w);
        const uint32_t c = (uint32_t)(((int64_t)g.row_cz[r] * cfg.nc[1] + g.row_cy[r]) * cfg.nc[0] + x);
        const uint32_t s0 = cs[c], s1 = cs[c + 1];
        g.start[r][t] = s0;
        g.cnt[r][t] = (int)(s1 - s0);
    }
    __syncthreads();
    if (tid == 0) {
        int o = 0;
        for (int r = 0; r < g.nrows; ++r) {
            int wprev = 2;
            for (int t = 0; t < g.nseq; ++t) {
                if (HALF) {
                    int w;
                    seq_cell_x(g.seq_start + t, cfg.nc[0], cfg.mode[0], &w);
                    if (w != wprev) {  // a piece starts here: the previous one ends
                        if (t > 0 && ((g.start[r][t - 1] + (uint32_t)g.cnt[r][t - 1]) & 1u)) ++o;
                        if (((uint32_t)o ^ g.start[r][t]) & 1u) ++o;
                        wprev = w;
                    }
                }
                g.off[r][t] = o;
                o += g.cnt[r][t];
            }
            if (HALF && ((g.start[r][g.nseq - 1] + (uint32_t)g.cnt[r][g.nseq - 1]) & 1u)) ++o;
            g.off[r][g.nseq] = o;
        }
        g.M = o;
        d.M = o;
        // home particles: cells a .. b-1 of the middle row
        const int ta = g.a - g.seq_start, tb = g.b - 1 - g.seq_start;
        d.h0 = g.start[g.mid_row][ta];
        d.h1 = g.start[g.mid_row][tb] + (uint32_t)g.cnt[g.mid_row][tb];
        int slow = (cfg.mode[0] == kModeAll || cfg.mode[1] == kModeAll || cfg.mode[2] == kModeAll) ? 1 : 0;
        for (int r = 0; r < kMaxRows; ++r)
            for (int p = 0; p < kPiecesPerRow; ++p) d.piece[r * kPiecesPerRow + p] = Piece{0, 0, 0u, 0};
        for (int r = 0; r < g.nrows; ++r) {
            int p = 0, t = 0;
            const int rowflags = (g.row_wy[r] > 0 ? kUpY : 0) | (g.row_wz[r] > 0 ? kUpZ : 0) |
                                 (g.row_wy[r] < 0 ? kLoY : 0) | (g.row_wz[r] < 0 ? kLoZ : 0);
            while (t < g.nseq) {
                int w0;
                seq_cell_x(g.seq_start + t, cfg.nc[0], cfg.mode[0], &w0);
                int t1 = t;
                while (t1 + 1 < g.nseq) {
                    int w1;
                    seq_cell_x(g.seq_start + t1 + 1, cfg.nc[0], cfg.mode[0], &w1);
                    if (w1 != w0) break;
                    ++t1;
                }
                const int f = rowflags | (w0 > 0 ? kUpX : 0) | (w0 < 0 ? kLoX : 0);
                if (f & (kUpX | kUpY | kUpZ)) slow = 1;
                int len = 0;
                for (int q = t; q <= t1; ++q) len += g.cnt[r][q];
                d.piece[r * kPiecesPerRow + p] = Piece{g.off[r][t], len, g.start[r][t], f};
                ++p;
                t = t1 + 1;
            }
        }
        d.slow = slow;
    }
    __syncthreads();
}

// Counts a tile whose neighbourhood does not fit the staging buffer.
__device__ __forceinline__ void note_spill(fpm_dev_status *st)
{
    if (st && threadIdx.x == 0) atomicAdd(&st->spilled, 1u);
}

// Loads a tile descriptor from global memory into shared memory.
__device__ __forceinline__ void load_desc(const TileDesc *__restrict__ src, TileDesc &dst)
{
    const int words = (int)(sizeof(TileDesc) / 4);
    const uint32_t *s = (const uint32_t *)src;
    uint32_t *o = (uint32_t *)&dst;
    for (int k = threadIdx.x; k < words; k += blockDim.x) o[k] = __ldg(s + k);
    __syncthreads();
}

// load_desc for a descriptor that may have been written earlier in the same
// launch (by another block, ordered by a barrier or a flag): read at L2,
// never through the read-only path.
__device__ __forceinline__ void load_desc_cg(const TileDesc *src, TileDesc &dst)
{
    const int words = (int)(sizeof(TileDesc) / 4);
    const uint32_t *s = (const uint32_t *)src;
    uint32_t *o = (uint32_t *)&dst;
    for (int k = threadIdx.x; k < words; k += blockDim.x) o[k] = __ldcg(s + k);
    __syncthreads();
}

// ---- TMA bulk staging -------------------------------------------------------
// Every piece is a contiguous run of 16-byte (float4) or 32-byte (double4)
// records in the sorted position array, so one cp.async.bulk per piece copies
// it into shared memory; all copies complete on one mbarrier.  Waits are
// bounded (kWaitCycles); on expiry FPM_FLAG_TIMEOUT is latched.

constexpr long long kWaitCycles = 4000000000LL;  // about 2 s of SM clock

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Each round tests the phase without blocking, then gives up once the budget
// is spent or waits in the hardware's own suspended wait; a budget shorter
// than one suspended wait therefore expires unless the phase is complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long budget)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > budget) return false;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
}

// One-time set-up of the staging barrier of a block.
__device__ __forceinline__ void stage_init(uint64_t *bar)
{
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
}

// Stages the neighbourhood positions of a tile into shared memory: slot s of
// piece p holds pos[gstart + (s - soff)] with the lower-wall shifts applied
// and (in tiles that need them) the piece flags in w.  When aux is given, the
// same slots of a second per-particle array are copied unchanged into aux_st
// on the same barrier.  `phase` is the barrier's parity, flipped per use.
// wait0 is the budget of the first wait for the copies (the wait that lets
// copies in flight land after an expiry always has the full budget).
// Every thread must have finished with the previous tile's staged data (a
// __syncthreads) before the call.  Returns false, the same in every thread,
// if the copies did not complete within the wait budget.
template <typename T>
__device__ bool stage_positions(const TileDesc &d, const BoxT<T> &box, const V4<T> *__restrict__ pos,
                                V4<T> *__restrict__ st, uint64_t *bar, uint32_t &phase, fpm_dev_status *status,
                                const V4<T> *__restrict__ aux = nullptr, V4<T> *__restrict__ aux_st = nullptr,
                                long long wait0 = kWaitCycles)
{
    const uint32_t b = smem_u32(bar);
    static_assert(kMaxPieces <= 32, "one lane of warp 0 per piece");
    const int lane = (int)(threadIdx.x & 31u);
    if (threadIdx.x < 32u) {
        // lane 0 arms the barrier with the byte count; then lane p issues the
        // copy (or copies) of piece p.  Each issuing lane first orders the
        // block's earlier generic accesses of the buffers (made visible to it by
        // the caller's barrier) before its async copies.
        // the bytes the copies bring: the pieces' lengths (a half-list tile's
        // free slots between pieces are not copied)
        const uint32_t len = lane < kMaxPieces ? (uint32_t)d.piece[lane].len : 0u;
        const uint32_t staged = __reduce_add_sync(kFull, len);
        if (lane == 0) {
            const uint32_t bytes = staged * (uint32_t)sizeof(V4<T>) * (aux ? 2u : 1u);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
        }
        __syncwarp();
        if (lane < kMaxPieces) {
            const Piece pc = d.piece[lane];
            if (pc.len != 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                const uint32_t nb = (uint32_t)pc.len * (uint32_t)sizeof(V4<T>);
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(st + pc.soff)),
                    "l"(pos + pc.gstart), "r"(nb), "r"(b)
                    : "memory");
                if (aux)
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            smem_u32(aux_st + pc.soff)),
                        "l"(aux + pc.gstart), "r"(nb), "r"(b)
                        : "memory");
            }
        }
    }
    // the pieces that need the shifts or the flags: one piece per lane, every warp
    bool fix = false;
    if (lane < kMaxPieces) {
        const Piece pc = d.piece[lane];
        fix = pc.len != 0 && (pc.flags != 0 || d.slow);
    }
    uint32_t todo = __ballot_sync(kFull, fix);
    bool ok = mbar_wait(b, phase, wait0);
    if (!ok) {
        latch_flag(status, FPM_FLAG_TIMEOUT);
        ok = mbar_wait(b, phase, kWaitCycles);  // let copies in flight land before leaving
    }
    phase ^= 1u;
    if (!__syncthreads_and(ok)) return false;
    if (todo == 0u) return true;  // nothing written: the copies' completion was observed by every thread
    while (todo) {
        const int p = __ffs(todo) - 1;
        todo &= todo - 1u;
        const Piece pc = d.piece[p];
        const T sx = (pc.flags & kLoX) ? box.L[0] : (T)0;
        const T sy = (pc.flags & kLoY) ? box.L[1] : (T)0;
        const T sz = (pc.flags & kLoZ) ? box.L[2] : (T)0;
        for (int e = threadIdx.x; e < pc.len; e += blockDim.x) {
            V4<T> q = st[pc.soff + e];
            q.x = rsub(q.x, sx);
            q.y = rsub(q.y, sy);
            q.z = rsub(q.z, sz);
            q.w = flags_as<T>(pc.flags);
            st[pc.soff + e] = q;
        }
    }
    __syncthreads();
    return true;
}

// Sorted particle index held by staged slot s.
__device__ __forceinline__ uint32_t staged_index(const TileDesc &d, int s)
{
    uint32_t j = 0;
    for (int k = 0; k < kMaxPieces; ++k) {
        const Piece pc = d.piece[k];
        if (pc.len > 0 && s >= pc.soff && s < pc.soff + pc.len) j = pc.gstart + (uint32_t)(s - pc.soff);
    }
    return j;
}

// Position of staged slot s read straight from global memory (used when the
// neighbourhood does not fit in shared memory).
template <typename T>
__device__ __forceinline__ V4<T> staged_global(const TileDesc &d, const BoxT<T> &box, const V4<T> *__restrict__ pos,
                                               int s)
{
    int p = -1;
    for (int k = 0; k < kMaxPieces; ++k) {
        const Piece pc = d.piece[k];
        if (pc.len > 0 && s >= pc.soff && s < pc.soff + pc.len) {
            p = k;
            break;
        }
    }
    if (p < 0) {  // a free slot of a half-list tile: no particle, never inside any radius
        V4<T> q;
        q.x = q.y = q.z = q.w = (T)NAN;
        return q;
    }
    const Piece pc = d.piece[p];
    V4<T> q = ldcg4(pos + pc.gstart + (s - pc.soff));  // at L2: pos may have been written earlier in the launch
    if (pc.flags & kLoX) q.x = rsub(q.x, box.L[0]);
    if (pc.flags & kLoY) q.y = rsub(q.y, box.L[1]);
    if (pc.flags & kLoZ) q.z = rsub(q.z, box.L[2]);
    q.w = flags_as<T>(pc.flags);
    return q;
}

// Separation x_i - x_j for a staged neighbour (see the file comment).  FAST:
// the tile has no kUp flags and no "all"-mode dimension.
template <bool FAST, typename T>
__device__ __forceinline__ T tile_sep(const V4<T> &pi, const V4<T> &pj, const BoxT<T> &box, const TileCfg &cfg, T &dx,
                                      T &dy, T &dz)
{
    if (FAST) {
        dx = rsub(pi.x, pj.x);
        dy = rsub(pi.y, pj.y);
        dz = rsub(pi.z, pj.z);
    } else {
        const int f = flags_of(pj.w);
        dx = cfg.mode[0] == kModeAll ? sep1(pi.x, pj.x, box.L[0], box.h[0])
                                     : rsub((f & kUpX) ? rsub(pi.x, box.L[0]) : pi.x, pj.x);
        dy = cfg.mode[1] == kModeAll ? sep1(pi.y, pj.y, box.L[1], box.h[1])
                                     : rsub((f & kUpY) ? rsub(pi.y, box.L[1]) : pi.y, pj.y);
        dz = cfg.mode[2] == kModeAll ? sep1(pi.z, pj.z, box.L[2], box.h[2])
                                     : rsub((f & kUpZ) ? rsub(pi.z, box.L[2]) : pi.z, pj.z);
    }
    return rfma(dz, dz, rfma(dy, dy, rmul(dx, dx)));
}

// Separation for a staged neighbour of a tile with periodic-wall flags and
// no "all"-mode dimension: the home coordinate x_i - L (pim, computed once
// per home particle) where the neighbour's flags say so.  The same roundings
// as tile_sep<false> in "wrap" mode.
template <typename T>
__device__ __forceinline__ T tile_sep_wall(const V4<T> &pi, const V4<T> &pim, const V4<T> &pj, T &dx, T &dy, T &dz)
{
    const int f = flags_of(pj.w);
    dx = rsub((f & kUpX) ? pim.x : pi.x, pj.x);
    dy = rsub((f & kUpY) ? pim.y : pi.y, pj.y);
    dz = rsub((f & kUpZ) ? pim.z : pi.z, pj.z);
    return rfma(dz, dz, rfma(dy, dy, rmul(dx, dx)));
}

// Fire-and-forget L2 prefetch of the first list words (k = 0 .. 2*nwords-1),
// the position and the entry count of home particle i, issued before a
// tile's staging wait so that the sweep's first loads hit in L2.
template <typename V>
__device__ __forceinline__ void prefetch_home(const V *pos, const uint32_t *nn, const uint32_t *words, int64_t ld,
                                              uint32_t i, int nwords)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(pos + i));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(nn + i));
    for (int q = 0; q < nwords; ++q) asm volatile("prefetch.global.L2 [%0];" ::"l"(words + (int64_t)q * ld + i));
}

// Calls f(s) for the 16-bit entries of one particle's list held in words
// w_first, w_first + kStride, w_first + 2 kStride, ... (the column `col` of
// the ELL words, leading dimension ld; word w holds entries 2w and 2w + 1,
// of which the first m exist).  With kStride = 1 and w_first = 0 that is the
// whole list; kStride = 2 splits it between two threads.  The words are
// loaded kChunk at a time, one chunk ahead of their use, so that the loads'
// latency overlaps the pair arithmetic of the previous chunk; whole chunks
// run without per-entry guards.
template <uint32_t kChunk, uint32_t kStride = 1, typename F>
__device__ __forceinline__ void for_each_entry(uint32_t m, const uint32_t *__restrict__ col, int64_t ld, F &&f,
                                               uint32_t w_first = 0)
{
    const uint32_t nw = (m + 1u) >> 1;  // words holding entries
    const uint32_t nfw = m >> 1;        // words whose both entries exist
    const uint32_t mine = nfw > w_first ? (nfw - w_first + kStride - 1u) / kStride : 0u;
    const uint32_t nfull = mine / kChunk * kChunk;  // this walker's full words, in whole chunks
    const int64_t step = (int64_t)kStride * ld;
    uint32_t cur[kChunk], nxt[kChunk];
    const uint32_t *p = col + (int64_t)w_first * ld;  // next word to load
#pragma unroll
    for (uint32_t q = 0; q < kChunk; ++q) {
        cur[q] = q < nfull ? __ldcs(p) : 0u;
        p += step;
    }
    for (uint32_t k0 = 0; k0 < nfull; k0 += kChunk) {
        const bool more = k0 + kChunk < nfull;
#pragma unroll
        for (uint32_t q = 0; q < kChunk; ++q) {
            nxt[q] = more ? __ldcs(p) : 0u;
            p += step;
        }
#pragma unroll
        for (uint32_t q = 0; q < kChunk; ++q) {
            f((int)(cur[q] & 0xffffu));
            f((int)(cur[q] >> 16));
        }
#pragma unroll
        for (uint32_t q = 0; q < kChunk; ++q) cur[q] = nxt[q];
    }
    for (uint32_t w = w_first + nfull * kStride; w < nw; w += kStride) {
        const uint32_t wv = __ldcs(col + (int64_t)w * ld);
        f((int)(wv & 0xffffu));
        if (2u * w + 1u < m) f((int)(wv >> 16));
    }
}

// Verlet-list scan of one home particle i (staged slot `self`) over the
// staged cells t0..t1 of every stencil row (its 27 cells): every candidate
// inside r_list is written as a 16-bit staged index, two per word (entry k
// in half k & 1 of word (k >> 1) * ld + i).  Returns the candidate count
// (entries beyond cap are counted, not stored).  Candidates are tested 32 at
// a time into a bit mask (one shift-in per test); then only the set bits are
// appended, in increasing slot order.
// HALF: a half-list tile, each pair listed once.  In its own row the
// candidates are the home cell's particles on one side of `self` and the next
// cell (th + 1); the home cell is split circularly so that every particle
// gets the same count: with c particles and self at rank q, the particles at
// ranks q + 1 .. q + (c - 1)/2 (mod c), and for even c also q + c/2 when
// q < c/2.  (Taking every later particle instead would give the cell's first
// particle c - 1 candidates and its last none: uneven lists, idle lanes.)
// SEP: 0 a tile without wall flags (tile_sep<true>), 1 a tile with wall flags
// and no "all"-mode dimension (tile_sep_wall), 2 any tile (tile_sep<false>).
template <int SEP, bool SMEM, typename T, bool HALF = false>
__device__ __forceinline__ uint32_t scan_candidates(const TileCfg &cfg, const BoxT<T> &box, const TileGeom &g,
                                                    const TileDesc &d, const V4<T> *__restrict__ pos,
                                                    const V4<T> *__restrict__ st, const V4<T> &pi, int self,
                                                    int th, int t0, int t1, T rl2, int cap, int64_t ld, uint32_t i,
                                                    uint32_t *__restrict__ words)
{
    uint32_t cnt = 0, pending = 0;
    const uint32_t ucap = (uint32_t)cap;
    V4<T> pim = pi;  // the home coordinates x_i - L of the wall path
    if (SEP == 1) {
        pim.x = rsub(pi.x, box.L[0]);
        pim.y = rsub(pi.y, box.L[1]);
        pim.z = rsub(pi.z, box.L[2]);
    }
    // tests the staged slots [s0, s1) 32 at a time into a bit mask, then
    // appends the hits in increasing slot order
    auto scan_range = [&](int s0, int s1) {
        for (int base = s0; base < s1; base += 32) {
            const int e = base + 32 < s1 ? base + 32 : s1;
            uint32_t mask = 0;
#pragma unroll 8
            for (int s = base; s < e; ++s) {
                const V4<T> pj = SMEM ? st[s] : staged_global(d, box, pos, s);
                T dx, dy, dz;
                const T r2 = SEP == 0   ? tile_sep<true>(pi, pj, box, cfg, dx, dy, dz)
                             : SEP == 1 ? tile_sep_wall(pi, pim, pj, dx, dy, dz)
                                        : tile_sep<false>(pi, pj, box, cfg, dx, dy, dz);
                mask = (mask << 1) | (r2 < rl2 ? 1u : 0u);
            }
            if (!HALF && self >= base && self < e) mask &= ~(1u << (e - 1 - self));
            while (mask) {
                const int bit = 31 - __clz(mask);
                mask &= ~(1u << bit);
                const uint32_t s = (uint32_t)(e - 1 - bit);
                const bool room = cnt < ucap;
                const bool odd = (cnt & 1u) != 0u;
                if (room & odd) words[(int64_t)(cnt >> 1) * ld + i] = pending | (s << 16);
                pending = (room & !odd) ? s : pending;
                ++cnt;
            }
        }
    };
    for (int r = 0; r < g.nrows; ++r) {
        if (HALF && r == g.mid_row) {
            const int c = g.cnt[r][th], c0 = g.off[r][th], q = self - c0;
            const int h = (c - 1) / 2 + (((c & 1) == 0 && q < c / 2) ? 1 : 0);
            const int end = self + 1 + h;
            scan_range(self + 1, end < c0 + c ? end : c0 + c);
            if (end > c0 + c) scan_range(c0, c0 + (end - (c0 + c)));
            if (t1 > th) scan_range(g.off[r][th + 1], g.off[r][th + 1] + g.cnt[r][th + 1]);
        } else {
            scan_range(g.off[r][t0], g.off[r][t1 + 1]);
        }
    }
    const uint32_t stored = cnt < ucap ? cnt : ucap;
    if (stored & 1u) words[(int64_t)(stored >> 1) * ld + i] = pending;
    return cnt;
}

// The free slots of a staged half-list tile (between its pieces) are set to
// NaN positions, never inside any radius (the copies do not write them).
// Lanes of warp 0, one per piece; the caller's next barrier publishes them.
template <typename T>
__device__ __forceinline__ void fill_free_slots(const TileDesc &d, V4<T> *__restrict__ st)
{
    if (threadIdx.x >= (unsigned)kMaxPieces) return;
    const Piece pc = d.piece[threadIdx.x];
    if (pc.len == 0) return;
    const int cand[2] = {pc.soff - 1, pc.soff + pc.len};
    for (int q = 0; q < 2; ++q) {
        const int s = cand[q];
        if (s < 0 || s >= d.M) continue;
        bool used = false;
        for (int k = 0; k < kMaxPieces; ++k) {
            const Piece o = d.piece[k];
            used = used || (o.len > 0 && s >= o.soff && s < o.soff + o.len);
        }
        if (!used) {
            V4<T> nanv;
            nanv.x = nanv.y = nanv.z = nanv.w = (T)NAN;
            st[s] = nanv;
        }
    }
}

// One tile of the Verlet build (all threads of the block call it): its
// geometry and descriptor, the staging of its neighbourhood, and the scan of
// every home particle (pos_ref[i] := pos[i] when pos_ref is given).  Returns
// the largest candidate count this thread saw.
template <typename T, bool HALF = false>
__device__ __forceinline__ uint32_t verlet_tile(const TileCfg &cfg, const BoxT<T> &box, int tile,
                                                const uint32_t *__restrict__ cs, const V4<T> *__restrict__ pos,
                                                T rl2, int cap, int64_t ld, int stage_cap, TileGeom &g, TileDesc &d,
                                                V4<T> *sp, uint64_t *bar, uint32_t &phase,
                                                uint32_t *__restrict__ words, uint32_t *__restrict__ nn,
                                                V4<T> *__restrict__ pos_ref, fpm_dev_status *st)
{
    tile_geometry<HALF>(cfg, tile, cs, g, d);
    if (d.M > kMaxStaged) {  // 16-bit entries cannot address this neighbourhood
        for (uint32_t i = d.h0 + threadIdx.x; i < d.h1; i += blockDim.x) nn[i] = 0u;
        if (threadIdx.x == 0) latch_flag(st, FPM_FLAG_CAPACITY);
        return 0u;
    }
    const bool in_smem = d.M <= stage_cap;
    if (!in_smem) note_spill(st);
    if (HALF && in_smem) fill_free_slots<T>(d, sp);
    if (in_smem && !stage_positions(d, box, pos, sp, bar, phase, st)) {
        for (uint32_t i = d.h0 + threadIdx.x; i < d.h1; i += blockDim.x) nn[i] = 0u;
        return 0u;
    }
    uint32_t maxc = 0;
    const bool all_mode = cfg.mode[0] == kModeAll || cfg.mode[1] == kModeAll || cfg.mode[2] == kModeAll;
    for (uint32_t i = d.h0 + threadIdx.x; i < d.h1; i += blockDim.x) {
        const V4<T> pi = pos[i];
        if (pos_ref) pos_ref[i] = pi;
        // the home cell: the staged cell of the middle row holding i
        int th = g.a - g.seq_start;
        for (int t = g.a - g.seq_start; t < g.b - g.seq_start; ++t)
            if (i >= g.start[g.mid_row][t] && i < g.start[g.mid_row][t] + (uint32_t)g.cnt[g.mid_row][t]) th = t;
        const int self = g.off[g.mid_row][th] + (int)(i - g.start[g.mid_row][th]);
        const int t0 = th > 0 ? th - 1 : 0;
        const int t1 = th + 1 < g.nseq ? th + 1 : g.nseq - 1;
        uint32_t c;
        if (in_smem && !d.slow) {
            c = scan_candidates<0, true, T, HALF>(cfg, box, g, d, pos, sp, pi, self, th, t0, t1, rl2, cap, ld, i, words);
        } else if (in_smem && !all_mode) {
            c = scan_candidates<1, true, T, HALF>(cfg, box, g, d, pos, sp, pi, self, th, t0, t1, rl2, cap, ld, i, words);
        } else if (in_smem) {
            c = scan_candidates<2, true, T, HALF>(cfg, box, g, d, pos, sp, pi, self, th, t0, t1, rl2, cap, ld, i, words);
        } else {
            c = scan_candidates<2, false, T, HALF>(cfg, box, g, d, pos, sp, pi, self, th, t0, t1, rl2, cap, ld, i,
                                                   words);
        }
        nn[i] = c < (uint32_t)cap ? c : (uint32_t)cap;
        if (c > (uint32_t)cap) latch_flag(st, FPM_FLAG_CAPACITY);
        maxc = c > maxc ? c : maxc;
    }
    return maxc;
}

// Launches the list decoder (verlet.cu) over ntiles tile descriptors.
fpm_status verlet_decode_launch(const TileDesc *descs, const uint32_t *words, const uint32_t *nn, int64_t ld,
                                uint32_t *out, int ntiles, cudaStream_t stream);

// Shared-memory budget for staged positions: 1.4x the mean neighbourhood of
// a tile plus slack, capped by what one block may use.
// The particles per cell assumed are the larger of the mean (n / ncell) and
// the occupancy the tile width was chosen for (kTileTarget particles per
// tile), so that a grid whose tiles were sized for the dense part of a
// non-uniform system (set by the caller through fpm_grid.tiles_x) stages its
// dense tiles in shared memory.
inline int stage_capacity(int n, const fpm_grid &g, size_t elem_bytes)
{
    const int maxe0 = (int)((size_t)kSmemBudget / elem_bytes) / 32 * 32;
    if (g.stage_cap > 0) {
        const int e = (g.stage_cap + 31) / 32 * 32;
        return e > maxe0 ? maxe0 : e;
    }
    const int wx = (g.nc[0] + g.tiles_x - 1) / g.tiles_x;
    const double mean = g.ncell > 0 ? (double)n / g.ncell : 0.0;
    const double sized = (double)kTileTarget / (double)(wx + 1);
    const double rho_c = mean > sized ? mean : sized;
    const int seq = g.nc[0] == 1 ? 1 : wx + 2;
    const int rows = (g.nc[1] >= 3 ? 3 : g.nc[1]) * (g.nc[2] >= 3 ? 3 : g.nc[2]);
    const double want = 1.2 * rows * seq * rho_c + 96.0;
    const int maxe = (int)((size_t)kSmemBudget / elem_bytes);
    int e = want > maxe ? maxe : (int)want;
    e = (e + 31) / 32 * 32;
    if (e > maxe) e = maxe / 32 * 32;
    return e < 256 ? 256 : e;
}

// Lets a kernel use the full dynamic shared-memory budget (a host call, not a
// stream operation; safe during graph capture).
inline void smem_opt_in(const void *kernel)
{
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget);
}

// ---- dynamic tile scheduling of the persistent sweeps -----------------------
// A sweep's blocks take tickets k = 0, 1, ... from a work counter; ticket k is
// the k-th non-empty tile.  The last block to finish resets the counters, so
// they are zero again for the next launch (the memory holding them must be
// zero before the first launch).

struct Sched {
    unsigned *work;  // next ticket
    unsigned *done;  // blocks finished
};

// Tile tickets.  A block's first ticket is its own index; each later one is
// requested from the shared counter by thread 0 at the start of a tile
// (ticket_ahead) and handed to the whole block at the tile's end
// (ticket_next), so the atomic's latency hides behind the tile's work.
// Tickets from gridDim.x on are handed out once each, in counter order.
__device__ __forceinline__ uint32_t ticket_ahead(const Sched &sc)
{
    return threadIdx.x == 0 ? gridDim.x + atomicAdd(sc.work, 1u) : 0u;
}

// The block's next ticket (all threads get the same value).  It begins with
// a barrier, so the tile's shared data may be reused after it.
__device__ __forceinline__ uint32_t ticket_next(uint32_t ahead, uint32_t *s_k)
{
    __syncthreads();
    if (threadIdx.x == 0) *s_k = ahead;
    __syncthreads();
    return *s_k;
}

// Called by every block after its last ticket; returns true in the last block
// to finish (in all its threads), after resetting the counters.
__device__ __forceinline__ bool sched_finish(const Sched &sc, bool *s_last)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(sc.done, 1u);
        *s_last = (t == gridDim.x - 1);
        if (*s_last) {
            *sc.work = 0u;
            *sc.done = 0u;
        }
    }
    __syncthreads();
    return *s_last;
}

// Sums NV per-thread values over the block (FP32 or FP64 within warps, FP64
// across warps) and stores them, from thread 0, to dst[0..NV).  All threads
// must call it.
template <int NV, typename TV>
__device__ __forceinline__ void block_sum_store(const TV (&v)[NV], double *dst)
{
    __shared__ double sh[32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const TV s = warp_sum(v[k]);
        if (lane == 0) sh[warp][k] = (double)s;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = lane < nw ? sh[lane][k] : 0.0;
            s = warp_sum(s);
            if (lane == 0) dst[k] = s;
        }
    }
    __syncthreads();
}

// In the last block: out[k] (+)= scale[k] * sum over tickets j < count of
// part[j*NV + k], in ticket order (bit-reproducible).
template <int NV>
__device__ __forceinline__ void sum_tile_partials(const double *part, uint32_t count, double *out, bool accumulate,
                                                  const double *scale)
{
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    for (uint32_t j = threadIdx.x; j < count; j += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += __ldcg(part + (size_t)j * NV + k);
    __shared__ double sh[32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const double s = warp_sum(acc[k]);
        if (lane == 0) sh[warp][k] = s;
    }
    __syncthreads();
    if (warp == 0 && out) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = lane < nw ? sh[lane][k] : 0.0;
            s = warp_sum(s);
            const double v = scale ? scale[k] * s : s;
            if (lane == 0) out[k] = accumulate ? out[k] + v : v;
        }
    }
}

// Grid of a tile sweep (tiles are taken by ticket, see ticket_ahead):
// g.sweep_blocks > 0 blocks, or one per tile (-1), or by default as many as
// fit on the GPU at once; never more than there are tiles.
inline int persistent_blocks(const void *kernel, int threads, size_t smem, const fpm_grid &g, int ntiles)
{
    long long b;
    if (g.sweep_blocks > 0) {
        b = g.sweep_blocks;
    } else if (g.sweep_blocks < 0) {
        b = ntiles;
    } else {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
        b = (long long)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    }
    if (b > ntiles) b = ntiles;
    return b < 1 ? 1 : (int)b;
}

}  // namespace fpm
