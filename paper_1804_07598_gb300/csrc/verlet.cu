// verlet.cu -- Verlet-list build over cell tiles, list decoding, and the
// displacement test that decides when to rebuild (Verlet lists [46] of
// Sec. 2, used for the MD benchmark of Sec. 4.1; rebuild when a particle has
// moved more than half the skin).
//
// Per tile (tiles.cuh; persistent blocks take tiles by ticket): the tile's
// neighbourhood is staged in shared memory, one thread per home particle
// scans the three staged cells around its own cell in each of the up-to-9
// stencil rows, and writes the staged index of every neighbour inside
// r_list as a 16-bit entry.
#include "tiles.cuh"

namespace fpm {

// Phase 1, every tile: geometry and descriptor (no staging, little shared
// memory, so the many empty tiles of a sparse box cost almost nothing).
template <bool HALF>
__global__ void __launch_bounds__(128)
    k_tile_desc(TileCfg cfg, const uint32_t *__restrict__ cs, TileDesc *__restrict__ descs, fpm_dev_status *st,
                const uint32_t *gate)
{
    if (gated_off(gate)) return;
    __shared__ TileGeom g;
    __shared__ TileDesc d;
    for (int tile = blockIdx.x; tile < cfg.ntiles; tile += gridDim.x) {
        tile_geometry<HALF>(cfg, tile, cs, g, d);
        const int nw = (int)(sizeof(TileDesc) / 4);
        uint32_t *o = (uint32_t *)(descs + tile);
        const uint32_t *s = (const uint32_t *)&d;
        for (int k = threadIdx.x; k < nw; k += blockDim.x) o[k] = s[k];
        if (threadIdx.x == 0 && st && d.h1 > d.h0) atomicMax(&st->max_staged, (uint32_t)d.M);
        __syncthreads();  // d and g are rewritten for the next tile
    }
}

// Phase 2, one block: the non-empty tiles in increasing order (a block-wide
// exclusive scan of the emptiness flags, 1024 x 4 tiles per pass).
__global__ void __launch_bounds__(1024)
    k_tile_compact(const TileDesc *__restrict__ descs, int ntiles, uint32_t *__restrict__ active,
                   uint32_t *__restrict__ count, const uint32_t *gate)
{
    if (gated_off(gate)) return;
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c0 = 0; c0 < ntiles; c0 += 4 * (int)blockDim.x) {
        uint32_t f[4], s = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int t = c0 + 4 * (int)threadIdx.x + q;
            f[q] = (t < ntiles && descs[t].h1 > descs[t].h0) ? 1u : 0u;
            s += f[q];
        }
        uint32_t incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, w, o);
                if (lane >= o) w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        uint32_t pos = base + incl - s + (warp > 0 ? wsum[warp - 1] : 0u);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (f[q]) active[pos++] = (uint32_t)(c0 + 4 * (int)threadIdx.x + q);
        __syncthreads();
        if (threadIdx.x == 0) base += wsum[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *count = base;
        count[4] = 0u;  // the scan's ticket and completion counters (list header bytes 16..23)
        count[5] = 0u;
    }
}

// Phase 3, persistent over the non-empty tiles: stage the neighbourhood and
// scan each home particle's candidates.
template <typename T, bool HALF>
__global__ void __launch_bounds__(kTileThreads)
    k_verlet_scan(TileCfg cfg, BoxT<T> box, const V4<T> *__restrict__ pos, const uint32_t *__restrict__ cs, T rl2,
                  int cap, int64_t ld, int stage_cap, const uint32_t *__restrict__ active,
                  const uint32_t *__restrict__ count, Sched sched, uint32_t *__restrict__ words,
                  uint32_t *__restrict__ nn, V4<T> *__restrict__ pos_ref, fpm_dev_status *st, const uint32_t *gate)
{
    if (gated_off(gate)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    V4<T> *sp = (V4<T> *)smem_raw;
    __shared__ TileGeom g;
    __shared__ TileDesc d;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_k;
    __shared__ bool s_last;
    stage_init(&bar);
    uint32_t phase = 0;
    uint32_t maxc = 0;
    const uint32_t ntodo = *count;
    uint32_t ahead = 0;
    for (uint32_t k = blockIdx.x; k < ntodo; k = ticket_next(ahead, &s_k)) {
        ahead = ticket_ahead(sched);
        const uint32_t c = verlet_tile<T, HALF>(cfg, box, (int)active[k], cs, pos, rl2, cap, ld, stage_cap, g, d, sp, &bar,
                                          phase, words, nn, pos_ref, st);
        maxc = c > maxc ? c : maxc;
    }
    const uint32_t m = __reduce_max_sync(kFull, maxc);
    if ((threadIdx.x & 31) == 0 && st && m > 0) atomicMax(&st->max_nn, m);
    sched_finish(sched, &s_last);
}

__global__ void __launch_bounds__(kTileThreads)
    k_verlet_decode(const TileDesc *__restrict__ descs, const uint32_t *__restrict__ words,
                    const uint32_t *__restrict__ nn, int64_t ld, uint32_t *__restrict__ out)
{
    __shared__ TileDesc d;
    load_desc(descs + blockIdx.x, d);
    for (uint32_t i = d.h0 + threadIdx.x; i < d.h1; i += blockDim.x) {
        const uint32_t m = nn[i];
        for (uint32_t k = 0; k < m; ++k) {
            const uint32_t w = words[(int64_t)(k >> 1) * ld + i];
            const int s = (int)((k & 1u) ? (w >> 16) : (w & 0xffffu));
            uint32_t j = 0xffffffffu;
            for (int p = 0; p < kMaxPieces; ++p) {
                const Piece pc = d.piece[p];
                if (pc.len > 0 && s >= pc.soff && s < pc.soff + pc.len) j = pc.gstart + (uint32_t)(s - pc.soff);
            }
            out[(int64_t)k * ld + i] = j;
        }
    }
}

fpm_status verlet_decode_launch(const TileDesc *descs, const uint32_t *words, const uint32_t *nn, int64_t ld,
                                uint32_t *out, int ntiles, cudaStream_t stream)
{
    if (ntiles > 0) k_verlet_decode<<<ntiles, kTileThreads, 0, stream>>>(descs, words, nn, ld, out);
    return fpm_check_launch("fpm_verlet_decode");
}

__global__ void k_gate_done(uint32_t *gate, fpm_dev_status *st)
{
    if (*gate) {
        *gate = 0u;
        if (st) st->nrebuild += 1u;
    }
}

template <typename T>
__global__ void k_verlet_check(BoxT<T> box, int n, const V4<T> *__restrict__ pos, const V4<T> *__restrict__ ref,
                               T th, fpm_dev_status *st)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float d2f = 0.0f;
    bool over = false;
    if (i < n) {
        T dx, dy, dz;
        const T d2 = separation(pos[i], ref[i], box, dx, dy, dz);
        over = d2 > th;
        d2f = (float)d2;
    }
    disp_report(over, d2f, st);
}

template <typename T, bool HALF>
static fpm_status verlet_launch(const fpm_box &b, const fpm_grid &g, int n, const void *pos, const uint32_t *cs,
                                double r_list, int cap, void *list, uint32_t *nn, void *pos_ref, fpm_dev_status *st,
                                uint32_t *gate, cudaStream_t stream)
{
    const TileCfg cfg = make_tile_cfg(b, g);
    const ListLayout L = list_layout(n, cfg, cap);
    const BoxT<T> box = make_box<T>(b);
    const T rl2 = (T)(r_list * r_list);
    const int sc = stage_capacity(n, g, sizeof(V4<T>));
    if (n > 0) {
        char *lb = (char *)list;
        TileDesc *descs = (TileDesc *)(lb + L.off_tiles);
        uint32_t *active = (uint32_t *)(lb + L.off_active);
        uint32_t *count = (uint32_t *)lb;
        k_tile_desc<HALF><<<grid_cap(cfg.ntiles), 128, 0, stream>>>(cfg, cs, descs, st, gate);
        k_tile_compact<<<1, 1024, 0, stream>>>(descs, cfg.ntiles, active, count, gate);
        const size_t smem = (size_t)sc * sizeof(V4<T>);
        smem_opt_in((const void *)k_verlet_scan<T, HALF>);
        const int blocks = persistent_blocks((const void *)k_verlet_scan<T, HALF>, kTileThreads, smem, g, cfg.ntiles);
        k_verlet_scan<T, HALF><<<blocks, kTileThreads, smem, stream>>>(cfg, box, (const V4<T> *)pos, cs, rl2, cap, L.ld, sc,
                                                                 active, count,
                                                                 Sched{(unsigned *)(lb + 16), (unsigned *)(lb + 20)},
                                                                 (uint32_t *)(lb + L.off_words), nn, (V4<T> *)pos_ref, st,
                                                                 gate);
    }
    if (gate) k_gate_done<<<1, 1, 0, stream>>>(gate, st);
    return fpm_check_launch("fpm_verlet_build");
}

template <typename T>
static fpm_status check_launch(const fpm_box &b, int n, const void *pos, const void *ref, double skin,
                               fpm_dev_status *st, cudaStream_t stream)
{
    const BoxT<T> box = make_box<T>(b);
    const T th = (T)(0.25 * skin * skin);
    if (n > 0)
        k_verlet_check<T><<<(n + 255) / 256, 256, 0, stream>>>(box, n, (const V4<T> *)pos, (const V4<T> *)ref, th,
                                                               st);
    return fpm_check_launch("fpm_verlet_check");
}

}  // namespace fpm

using namespace fpm;

static bool box_ok(const fpm_box *b)
{
    if (!b) return false;
    for (int d = 0; d < 3; ++d)
        if (!(b->L[d] > 0.0)) return false;
    return true;
}

// Checks shared by every call taking a grid and a list.
fpm_status fpm_check_grid(const fpm_box *box, const fpm_grid *grid, const char *who)
{
    if (!box_ok(box) || !grid) return fpm_fail(FPM_ERR_INVALID, "%s: null box or grid", who);
    for (int d = 0; d < 3; ++d)
        if (grid->nc[d] < 1) return fpm_fail(FPM_ERR_INVALID, "%s: bad grid", who);
    if ((int64_t)grid->nc[0] * grid->nc[1] * grid->nc[2] != grid->ncell)
        return fpm_fail(FPM_ERR_INVALID, "%s: grid->ncell inconsistent with nc", who);
    if (grid->tiles_x < 1 || grid->tiles_x > grid->nc[0] ||
        (grid->nc[0] + grid->tiles_x - 1) / grid->tiles_x > kMaxTileCells)
        return fpm_fail(FPM_ERR_INVALID, "%s: grid->tiles_x inconsistent with nc[0]", who);
    for (int d = 0; d < 3; ++d)
        if (box->periodic[d] && grid->nc[d] == 2)
            return fpm_fail(FPM_ERR_INVALID, "%s: a periodic dimension cannot have 2 cells", who);
    return FPM_OK;
}

extern "C" fpm_status fpm_verlet_list_bytes(int32_t n, const fpm_grid *grid, int32_t cap, size_t *bytes)
{
    if (!grid || !bytes || n < 0 || cap < 1 || grid->tiles_x < 1)
        return fpm_fail(FPM_ERR_INVALID, "fpm_verlet_list_bytes: bad argument");
    TileCfg c{};
    c.ntiles = grid->tiles_x * grid->nc[1] * grid->nc[2];
    *bytes = list_layout(n, c, cap).total;
    return FPM_OK;
}

static fpm_status verlet_build(const fpm_box *box, const fpm_grid *grid, int32_t n, fpm_prec prec, const void *pos,
                               const uint32_t *cell_start, double r_list, int32_t cap, void *list, size_t list_bytes,
                               uint32_t *nn, void *pos_ref, fpm_dev_status *d_status, uint32_t *d_gate,
                               fpm_stream stream, bool half)
{
    fpm_status s = fpm_check_grid(box, grid, "fpm_verlet_build");
    if (s != FPM_OK) return s;
    if (n < 0 || cap < 1 || !(r_list > 0.0) || !cell_start || (n > 0 && (!pos || !list || !nn)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_verlet_build: null pointer or bad size");
    if (prec != FPM_F32 && prec != FPM_F64) return fpm_fail(FPM_ERR_INVALID, "fpm_verlet_build: bad precision");
    for (int d = 0; d < 3; ++d) {
        if (grid->nc[d] > 1 && box->L[d] / grid->nc[d] < r_list)
            return fpm_fail(FPM_ERR_INVALID, "fpm_verlet_build: cells narrower than r_list in dim %d", d);
        if (box->periodic[d] && !(box->L[d] > 2.0 * r_list * (1.0 + 1.0 / 1024.0)))
            return fpm_fail(FPM_ERR_INVALID, "fpm_verlet_build: periodic L[%d] must exceed 2 r_list", d);
    }
    size_t need = 0;
    fpm_verlet_list_bytes(n, grid, cap, &need);
    if (n > 0 && list_bytes < need)
        return fpm_fail(FPM_ERR_WORKSPACE, "fpm_verlet_build: list object %zu < %zu bytes", list_bytes, need);
    if (((uintptr_t)list & 255u) != 0) return fpm_fail(FPM_ERR_INVALID, "fpm_verlet_build: list not 256-B aligned");
    cudaStream_t st = (cudaStream_t)stream;
    if (half) {
        if (prec == FPM_F32)
            return verlet_launch<float, true>(*box, *grid, n, pos, cell_start, r_list, cap, list, nn, pos_ref,
                                              d_status, d_gate, st);
        return verlet_launch<double, true>(*box, *grid, n, pos, cell_start, r_list, cap, list, nn, pos_ref, d_status,
                                           d_gate, st);
    }
    if (prec == FPM_F32)
        return verlet_launch<float, false>(*box, *grid, n, pos, cell_start, r_list, cap, list, nn, pos_ref, d_status,
                                           d_gate, st);
    return verlet_launch<double, false>(*box, *grid, n, pos, cell_start, r_list, cap, list, nn, pos_ref, d_status,
                                        d_gate, st);
}

extern "C" fpm_status fpm_verlet_build(const fpm_box *box, const fpm_grid *grid, int32_t n, fpm_prec prec,
                                       const void *pos, const uint32_t *cell_start, double r_list, int32_t cap,
                                       void *list, size_t list_bytes, uint32_t *nn, void *pos_ref,
                                       fpm_dev_status *d_status, uint32_t *d_gate, fpm_stream stream)
{
    return verlet_build(box, grid, n, prec, pos, cell_start, r_list, cap, list, list_bytes, nn, pos_ref, d_status,
                        d_gate, stream, false);
}

extern "C" fpm_status fpm_verlet_build_half(const fpm_box *box, const fpm_grid *grid, int32_t n, fpm_prec prec,
                                            const void *pos, const uint32_t *cell_start, double r_list, int32_t cap,
                                            void *list, size_t list_bytes, uint32_t *nn, void *pos_ref,
                                            fpm_dev_status *d_status, uint32_t *d_gate, fpm_stream stream)
{
    return verlet_build(box, grid, n, prec, pos, cell_start, r_list, cap, list, list_bytes, nn, pos_ref, d_status,
                        d_gate, stream, true);
}

extern "C" fpm_status fpm_verlet_decode(const fpm_grid *grid, int32_t n, int32_t cap, const void *list,
                                        const uint32_t *nn, uint32_t *out, fpm_stream stream)
{
    if (!grid || n < 0 || cap < 1 || (n > 0 && (!list || !nn || !out)) || grid->tiles_x < 1)
        return fpm_fail(FPM_ERR_INVALID, "fpm_verlet_decode: bad argument");
    if (n == 0) return FPM_OK;
    TileCfg c{};
    c.ntiles = grid->tiles_x * grid->nc[1] * grid->nc[2];
    const ListLayout L = list_layout(n, c, cap);
    return verlet_decode_launch((const TileDesc *)((const char *)list + L.off_tiles),
                                (const uint32_t *)((const char *)list + L.off_words), nn, L.ld, out, c.ntiles,
                                (cudaStream_t)stream);
}

extern "C" fpm_status fpm_verlet_check(const fpm_box *box, int32_t n, fpm_prec prec, const void *pos,
                                       const void *pos_ref, double skin, fpm_dev_status *d_status, fpm_stream stream)
{
    if (!box_ok(box) || n < 0 || !d_status || !(skin >= 0.0) || (n > 0 && (!pos || !pos_ref)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_verlet_check: null pointer or bad size");
    if (prec != FPM_F32 && prec != FPM_F64) return fpm_fail(FPM_ERR_INVALID, "fpm_verlet_check: bad precision");
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == FPM_F32) return check_launch<float>(*box, n, pos, pos_ref, skin, d_status, st);
    return check_launch<double>(*box, n, pos, pos_ref, skin, d_status, st);
}
