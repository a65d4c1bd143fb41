// dem.cu -- DEM with the Silbert grain model (Sec. 4.5): Hertzian normal and
// tangential contact forces with a per-contact tangential deformation
// (Eqs. 9-12), Coulomb's limit, the leapfrog with rotation (Eq. 13), and the
// contact history carried through the Verlet rebuild's reorder.
//
// The contact sweep walks the tiled Verlet list like the LJ sweep
// (persistent blocks take cell tiles by ticket, one thread per home
// particle), but a grain has only ~6 list entries against a staged
// neighbourhood of ~10 slots per home grain, so the neighbourhood is not
// copied: each tile builds a slot map in shared memory (4 bytes per staged
// slot: the sorted index and the piece's periodic flags), and every entry
// gathers its neighbour's position (and, for a contact, its velocity and spin)
// from L2, with the lower-wall shift applied exactly as staging would.  The
// history u_t of list entry k of particle i lives at hist[k * ld + i]
// (float4, w unused), read and rewritten for every entry: coalesced across the
// home particles of a warp, and 0 for an entry that is not in contact.
#include "reduce.cuh"
#include "tiles.cuh"

namespace fpm {

struct DemK {
    float R, twoR, c2;  // radius, 2R, (2R)^2
    float inv2R;        // 1 / (2R)
    float kn, kt, gn_meff, gt_meff, mu2, inv_kt, dt;
    float inv_m, inv_I, g[3];
};

static DemK make_dem(const fpm_dem_params &p)
{
    DemK K{};
    K.R = (float)p.R;
    K.twoR = (float)(2.0 * p.R);
    K.c2 = (float)(4.0 * p.R * p.R);
    K.inv2R = (float)(0.5 / p.R);
    K.kn = (float)p.kn;
    K.kt = (float)p.kt;
    K.gn_meff = (float)(p.gn * 0.5 * p.m);
    K.gt_meff = (float)(p.gt * 0.5 * p.m);
    K.mu2 = (float)(p.mu * p.mu);
    K.inv_kt = p.kt > 0.0 ? (float)(1.0 / p.kt) : 0.0f;
    K.dt = (float)p.dt;
    K.inv_m = (float)(1.0 / p.m);
    K.inv_I = (float)(1.0 / p.I);
    for (int d = 0; d < 3; ++d) K.g[d] = (float)p.g[d];
    return K;
}

// Slot map entry: sorted index in the low 26 bits, the piece's flags above.
constexpr int kMapShift = 26;
constexpr uint32_t kMapIndex = (1u << kMapShift) - 1u;

// One list entry of home particle i (slot map entry e): the contact of
// Eqs. 9-12 when r < 2R, adding to the force and torque sums and updating
// the entry's u_t; u_t = 0 otherwise.
template <bool FAST>
__device__ __forceinline__ void dem_pair(const TileCfg &cfg, const BoxT<float> &box, const float4 *__restrict__ pos,
                                         const float4 *__restrict__ vel, const float4 *__restrict__ om, uint32_t e,
                                         const float4 &pi, const float4 &vi, const float4 &wi, const DemK &K,
                                         float4 &u, float3 &F, float3 &T, uint32_t &nc)
{
    const uint32_t j = e & kMapIndex;
    const int fl = (int)(e >> kMapShift);
    float4 pj = __ldg(pos + j);
    // the staged form of the neighbour: lower-wall images shifted by -L (exact)
    pj.x = rsub(pj.x, (fl & kLoX) ? box.L[0] : 0.0f);
    pj.y = rsub(pj.y, (fl & kLoY) ? box.L[1] : 0.0f);
    pj.z = rsub(pj.z, (fl & kLoZ) ? box.L[2] : 0.0f);
    pj.w = flags_as<float>(fl);
    float dx, dy, dz;
    const float r2 = tile_sep<FAST>(pi, pj, box, cfg, dx, dy, dz);
    if (!(r2 < K.c2 && r2 > 0.0f)) {
        u = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        return;
    }
    const float4 vj = __ldg(vel + j), wj = __ldg(om + j);
    const float r = sqrtf(r2);
    const float ir = 1.0f / r;
    const float delta = K.twoR - r;  // Eq. 9
    const float nx = dx * ir, ny = dy * ir, nz = dz * ir;
    const float vx = vi.x - vj.x, vy = vi.y - vj.y, vz = vi.z - vj.z;
    const float vn = vx * nx + vy * ny + vz * nz;
    const float wx = wi.x + wj.x, wy = wi.y + wj.y, wz = wi.z + wj.z;
    // v_t = v_pq - (v_pq.n) n - R (w_p + w_q) x n
    const float tx = vx - vn * nx - K.R * (wy * nz - wz * ny);
    const float ty = vy - vn * ny - K.R * (wz * nx - wx * nz);
    const float tz = vz - vn * nz - K.R * (wx * ny - wy * nx);
    float ux = u.x + tx * K.dt, uy = u.y + ty * K.dt, uz = u.z + tz * K.dt;  // Eq. 10
    const float f = sqrtf(delta * K.inv2R);
    const float an = f * (K.kn * delta - K.gn_meff * vn);  // Eq. 11: F_n = an n
    float ftx = -f * (K.kt * ux + K.gt_meff * tx);         // Eq. 12
    float fty = -f * (K.kt * uy + K.gt_meff * ty);
    float ftz = -f * (K.kt * uz + K.gt_meff * tz);
    const float ft2 = ftx * ftx + fty * fty + ftz * ftz;
    const float fn2 = an * an;
    if (ft2 > K.mu2 * fn2) {  // Coulomb: |F_t| cut to mu |F_n|, u_t made consistent with Eq. 12
        const float sc = sqrtf(K.mu2 * fn2 / ft2);
        ftx *= sc;
        fty *= sc;
        ftz *= sc;
        const float inf = 1.0f / f;
        ux = -(ftx * inf + K.gt_meff * tx) * K.inv_kt;
        uy = -(fty * inf + K.gt_meff * ty) * K.inv_kt;
        uz = -(ftz * inf + K.gt_meff * tz) * K.inv_kt;
    }
    F.x += an * nx + ftx;
    F.y += an * ny + fty;
    F.z += an * nz + ftz;
    // torque -1/2 (x_p - x_q) x F_t
    T.x -= 0.5f * (dy * ftz - dz * fty);
    T.y -= 0.5f * (dz * ftx - dx * ftz);
    T.z -= 0.5f * (dx * fty - dy * ftx);
    u = make_float4(ux, uy, uz, 0.0f);
    ++nc;
}

// The contacts of home particle i over its m list entries (entry k in half
// k & 1 of word (k >> 1) * ld of col), with their histories.  MAP: the slot
// map is in shared memory (else each slot is resolved from the pieces).
template <bool FAST, bool MAP>
__device__ __forceinline__ void dem_sweep(const TileCfg &cfg, const BoxT<float> &box, const TileDesc &d,
                                          const float4 *__restrict__ pos, const float4 *__restrict__ vel,
                                          const float4 *__restrict__ om, const uint32_t *__restrict__ smap,
                                          const float4 &pi, const float4 &vi, const float4 &wi, uint32_t m,
                                          const uint32_t *__restrict__ col, float4 *__restrict__ hcol, int64_t ld,
                                          const DemK &K, float3 &F, float3 &T, uint32_t &nc)
{
    auto entry = [&](int s) -> uint32_t {
        if (MAP) return smap[s];
        uint32_t e = 0u;
        for (int p = 0; p < kMaxPieces; ++p) {
            const Piece pc = d.piece[p];
            if (pc.len > 0 && s >= pc.soff && s < pc.soff + pc.len)
                e = (pc.gstart + (uint32_t)(s - pc.soff)) | ((uint32_t)pc.flags << kMapShift);
        }
        return e;
    };
    for (uint32_t k = 0; k < m; k += 2) {
        const uint32_t w = __ldcs(col + (int64_t)(k >> 1) * ld);
        float4 u0 = __ldcs(hcol + (int64_t)k * ld);
        dem_pair<FAST>(cfg, box, pos, vel, om, entry((int)(w & 0xffffu)), pi, vi, wi, K, u0, F, T, nc);
        __stcs(hcol + (int64_t)k * ld, u0);
        if (k + 1 < m) {
            float4 u1 = __ldcs(hcol + (int64_t)(k + 1) * ld);
            dem_pair<FAST>(cfg, box, pos, vel, om, entry((int)(w >> 16)), pi, vi, wi, K, u1, F, T, nc);
            __stcs(hcol + (int64_t)(k + 1) * ld, u1);
        }
    }
}

__global__ void __launch_bounds__(kTileThreads)
    k_dem_tiles(TileCfg cfg, BoxT<float> box, const float4 *__restrict__ pos, const float4 *__restrict__ vel,
                const float4 *__restrict__ om, ListView lv, const uint32_t *__restrict__ nn, int64_t ld,
                int map_cap, DemK K, float4 *__restrict__ hist, float4 *__restrict__ force,
                float4 *__restrict__ torque, uint32_t *ncontact, Sched sched)
{
    extern __shared__ __align__(16) uint32_t smap[];
    __shared__ TileDesc d;
    __shared__ uint32_t s_k;
    __shared__ bool s_last;
    const uint32_t *__restrict__ words = lv.words;
    const uint32_t ntodo = *lv.count;
    const int lane = (int)(threadIdx.x & 31u), warp = (int)(threadIdx.x >> 5), nwarp = (int)(blockDim.x >> 5);
    uint32_t ahead = 0, nc = 0;
    for (uint32_t k = blockIdx.x; k < ntodo; k = ticket_next(ahead, &s_k)) {
        ahead = ticket_ahead(sched);
        load_desc(lv.descs + lv.active[k], d);
        const bool map = d.M <= map_cap;
        if (map) {  // one warp per piece
            for (int p = warp; p < kMaxPieces; p += nwarp) {
                const Piece pc = d.piece[p];
                const uint32_t fl = (uint32_t)pc.flags << kMapShift;
                for (int e = lane; e < pc.len; e += 32) smap[pc.soff + e] = (pc.gstart + (uint32_t)e) | fl;
            }
            __syncthreads();
        }
        for (uint32_t i = d.h0 + threadIdx.x; i < d.h1; i += blockDim.x) {
            const float4 pi = pos[i], vi = vel[i], wi = om[i];
            const uint32_t m = nn[i];
            float3 F = make_float3(0.0f, 0.0f, 0.0f), T = make_float3(0.0f, 0.0f, 0.0f);
            if (map) {
                if (d.slow)
                    dem_sweep<false, true>(cfg, box, d, pos, vel, om, smap, pi, vi, wi, m, words + i, hist + i, ld, K,
                                           F, T, nc);
                else
                    dem_sweep<true, true>(cfg, box, d, pos, vel, om, smap, pi, vi, wi, m, words + i, hist + i, ld, K,
                                          F, T, nc);
            } else {
                dem_sweep<false, false>(cfg, box, d, pos, vel, om, smap, pi, vi, wi, m, words + i, hist + i, ld, K,
                                        F, T, nc);
            }
            force[i] = make_float4(F.x, F.y, F.z, 0.0f);
            torque[i] = make_float4(T.x, T.y, T.z, 0.0f);
        }
    }
    if (ncontact) {
        const unsigned t = __reduce_add_sync(kFull, nc);
        if (lane == 0 && t) atomicAdd(ncontact, t);
    }
    sched_finish(sched, &s_last);
}

// Eq. 13 for grains of type 0, then the rebuild test on the new positions.
__global__ void k_dem_leapfrog(int n, BoxT<float> box, DemK K, float4 *__restrict__ pos, float4 *__restrict__ vel,
                               float4 *__restrict__ om, const float4 *__restrict__ force,
                               const float4 *__restrict__ torque, const float4 *__restrict__ ref, float th,
                               fpm_dev_status *st)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool over = false;
    float d2 = 0.0f;
    if (i < n) {
        float4 p = pos[i];
        if (p.w == 0.0f) {
            float4 v = vel[i], w = om[i];
            const float4 f = force[i], t = torque[i];
            v.x += K.dt * (f.x * K.inv_m + K.g[0]);
            v.y += K.dt * (f.y * K.inv_m + K.g[1]);
            v.z += K.dt * (f.z * K.inv_m + K.g[2]);
            p.x += K.dt * v.x;
            p.y += K.dt * v.y;
            p.z += K.dt * v.z;
            w.x += K.dt * t.x * K.inv_I;
            w.y += K.dt * t.y * K.inv_I;
            w.z += K.dt * t.z * K.inv_I;
            pos[i] = p;
            vel[i] = v;
            om[i] = w;
        }
        if (ref) {
            float ex, ey, ez;
            d2 = separation(p, ref[i], box, ex, ey, ez);
            over = d2 > th;
        }
    }
    if (ref) disp_report(over, d2, st);
}

// ---- the state across a rebuild ---------------------------------------------
constexpr int kDemMaxSaved = 16;  // contacts saved per particle

// Layout of the packed buffer: [kDemMaxSaved * ld] float4 records
// (u_x, u_y, u_z, partner index as bits), [ld] float4 saved omega, [ld] uint32
// record counts.
struct DemPacked {
    float4 *rec;
    float4 *omega;
    uint32_t *count;
};

static DemPacked dem_packed(void *p, int n)
{
    const int64_t ld = fpm_nbr_ld(n);
    DemPacked q;
    q.rec = (float4 *)p;
    q.omega = q.rec + (size_t)kDemMaxSaved * ld;
    q.count = (uint32_t *)(q.omega + ld);
    return q;
}

// The sorted index of staged slot s of a tile (pieces in shared memory).
__device__ __forceinline__ uint32_t dem_slot_index(const TileDesc &d, int s)
{
    uint32_t j = 0xffffffffu;
    for (int p = 0; p < kMaxPieces; ++p) {
        const Piece pc = d.piece[p];
        if (pc.len > 0 && s >= pc.soff && s < pc.soff + pc.len) j = pc.gstart + (uint32_t)(s - pc.soff);
    }
    return j;
}

// Every particle: omega saved, no records yet; and the rebuild marked pending.
__global__ void k_dem_save_omega(int n, const float4 *__restrict__ om, DemPacked q, const uint32_t *gate,
                                 uint32_t *pending)
{
    if (gated_off(gate)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *pending = 1u;
    if (i < n) {
        q.omega[i] = om[i];
        q.count[i] = 0u;
    }
}

// One block per tile of the current list: the entries with nonzero u_t.
__global__ void k_dem_save(const TileDesc *__restrict__ descs, const uint32_t *__restrict__ words,
                           const uint32_t *__restrict__ nn, int64_t ld, const float4 *__restrict__ hist,
                           DemPacked q, const uint32_t *gate, fpm_dev_status *st)
{
    if (gated_off(gate)) return;
    __shared__ TileDesc d;
    load_desc(descs + blockIdx.x, d);
    for (uint32_t i = d.h0 + threadIdx.x; i < d.h1; i += blockDim.x) {
        const uint32_t m = nn[i];
        uint32_t c = 0;
        for (uint32_t k = 0; k < m; ++k) {
            const float4 u = hist[(int64_t)k * ld + i];
            if (u.x == 0.0f && u.y == 0.0f && u.z == 0.0f) continue;
            const uint32_t w = words[(int64_t)(k >> 1) * ld + i];
            const int s = (int)((k & 1u) ? (w >> 16) : (w & 0xffffu));
            if (c < (uint32_t)kDemMaxSaved)
                q.rec[(int64_t)c * ld + i] = make_float4(u.x, u.y, u.z, __uint_as_float(dem_slot_index(d, s)));
            ++c;
        }
        if (c > (uint32_t)kDemMaxSaved) latch_flag(st, FPM_FLAG_CAPACITY);
        q.count[i] = c < (uint32_t)kDemMaxSaved ? c : (uint32_t)kDemMaxSaved;
    }
}

// One block per tile of the new list.
__global__ void k_dem_restore(int n, const TileDesc *__restrict__ descs, const uint32_t *__restrict__ words,
                              const uint32_t *__restrict__ nn, int64_t ld, const uint32_t *__restrict__ perm,
                              DemPacked q, float4 *__restrict__ hist, float4 *__restrict__ om,
                              const uint32_t *pending)
{
    if (gated_off(pending)) return;
    __shared__ TileDesc d;
    load_desc(descs + blockIdx.x, d);
    for (uint32_t i = d.h0 + threadIdx.x; i < d.h1; i += blockDim.x) {
        const uint32_t io = perm[i];
        om[i] = q.omega[io];
        const uint32_t c = q.count[io];
        const uint32_t m = nn[i];
        for (uint32_t k = 0; k < m; ++k) {
            const uint32_t w = words[(int64_t)(k >> 1) * ld + i];
            const int s = (int)((k & 1u) ? (w >> 16) : (w & 0xffffu));
            const uint32_t j = dem_slot_index(d, s);
            const uint32_t target = j < (uint32_t)n ? perm[j] : 0xffffffffu;
            float4 u = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            for (uint32_t t = 0; t < c; ++t) {
                const float4 r = q.rec[(int64_t)t * ld + io];
                if (__float_as_uint(r.w) == target) u = make_float4(r.x, r.y, r.z, 0.0f);
            }
            hist[(int64_t)k * ld + i] = u;
        }
    }
}

__global__ void k_dem_clear(uint32_t *pending) { *pending = 0u; }

static fpm_status dem_params_ok(const fpm_dem_params *p, const char *who)
{
    if (!p || !(p->R > 0.0) || !(p->m > 0.0) || !(p->I > 0.0) || !(p->kn >= 0.0) || !(p->kt >= 0.0) ||
        !(p->gn >= 0.0) || !(p->gt >= 0.0) || !(p->mu >= 0.0) || !(p->dt > 0.0))
        return fpm_fail(FPM_ERR_INVALID, "%s: bad DEM parameters", who);
    return FPM_OK;
}

static ListLayout dem_list_layout(const fpm_grid &g, int n, int cap)
{
    TileCfg c{};
    c.ntiles = g.tiles_x * g.nc[1] * g.nc[2];
    return list_layout(n, c, cap);
}

}  // namespace fpm

using namespace fpm;

extern "C" fpm_status fpm_dem_forces(const fpm_box *box, const fpm_grid *grid, int32_t n, const void *pos,
                                     const void *vel, const void *omega, const void *list, const uint32_t *nn,
                                     int32_t cap, const fpm_dem_params *params, void *hist, void *force,
                                     void *torque, uint32_t *d_ncontact, void *workspace, size_t workspace_bytes,
                                     fpm_dev_status *d_status, fpm_stream stream)
{
    fpm_status s = fpm_check_grid(box, grid, "fpm_dem_forces");
    if (s != FPM_OK) return s;
    s = dem_params_ok(params, "fpm_dem_forces");
    if (s != FPM_OK) return s;
    if (n < 0 || n > (int32_t)kMapIndex || cap < 1 ||
        (n > 0 && (!pos || !vel || !omega || !list || !nn || !hist || !force || !torque)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_dem_forces: null pointer or bad size");
    if (((uintptr_t)list & 255u) != 0) return fpm_fail(FPM_ERR_INVALID, "fpm_dem_forces: list not 256-B aligned");
    if (((uintptr_t)hist & 15u) != 0) return fpm_fail(FPM_ERR_INVALID, "fpm_dem_forces: hist not 16-B aligned");
    if (n == 0) return FPM_OK;
    RedWs r{};
    s = red_ws(n, grid, workspace, workspace_bytes, "fpm_dem_forces", r);
    if (s != FPM_OK) return s;
    const TileCfg cfg = make_tile_cfg(*box, *grid);
    const ListLayout L = list_layout(n, cfg, cap);
    const int mc = stage_capacity(n, *grid, sizeof(uint32_t));  // slot-map entries per tile
    const size_t smem = (size_t)mc * sizeof(uint32_t);
    smem_opt_in((const void *)k_dem_tiles);
    const int blocks = persistent_blocks((const void *)k_dem_tiles, kTileThreads, smem, *grid, cfg.ntiles);
    k_dem_tiles<<<blocks, kTileThreads, smem, (cudaStream_t)stream>>>(
        cfg, make_box<float>(*box), (const float4 *)pos, (const float4 *)vel, (const float4 *)omega,
        list_view(list, L), nn, L.ld, mc, make_dem(*params), (float4 *)hist, (float4 *)force, (float4 *)torque,
        d_ncontact, Sched{r.work, r.done});
    return fpm_check_launch("fpm_dem_forces");
}

extern "C" fpm_status fpm_dem_leapfrog(const fpm_box *box, int32_t n, const fpm_dem_params *params, void *pos,
                                       void *vel, void *omega, const void *force, const void *torque,
                                       const void *pos_ref, double skin, fpm_dev_status *d_status, fpm_stream stream)
{
    fpm_status s = dem_params_ok(params, "fpm_dem_leapfrog");
    if (s != FPM_OK) return s;
    if (!box || n < 0 || (pos_ref && !d_status) || !(skin >= 0.0) ||
        (n > 0 && (!pos || !vel || !omega || !force || !torque)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_dem_leapfrog: null pointer or bad size");
    if (n == 0) return FPM_OK;
    k_dem_leapfrog<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        n, make_box<float>(*box), make_dem(*params), (float4 *)pos, (float4 *)vel, (float4 *)omega,
        (const float4 *)force, (const float4 *)torque, (const float4 *)pos_ref, (float)(0.25 * skin * skin),
        d_status);
    return fpm_check_launch("fpm_dem_leapfrog");
}

extern "C" size_t fpm_dem_packed_bytes(int32_t n)
{
    const int64_t ld = fpm_nbr_ld(n > 0 ? n : 1);
    return (size_t)(kDemMaxSaved + 1) * (size_t)ld * sizeof(float4) + (size_t)ld * sizeof(uint32_t);
}

extern "C" fpm_status fpm_dem_rebuild_begin(const fpm_grid *grid, int32_t n, int32_t cap, const void *list,
                                            const uint32_t *nn, const void *hist, const void *omega, void *packed,
                                            const uint32_t *d_gate, uint32_t *d_pending, fpm_dev_status *d_status,
                                            fpm_stream stream)
{
    if (!grid || n < 0 || cap < 1 || !d_pending || grid->tiles_x < 1 ||
        (n > 0 && (!list || !nn || !hist || !omega || !packed)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_dem_rebuild_begin: bad argument");
    if (n == 0) return FPM_OK;
    const ListLayout L = dem_list_layout(*grid, n, cap);
    const int ntiles = grid->tiles_x * grid->nc[1] * grid->nc[2];
    cudaStream_t st = (cudaStream_t)stream;
    const DemPacked q = dem_packed(packed, n);
    k_dem_save_omega<<<(n + 255) / 256, 256, 0, st>>>(n, (const float4 *)omega, q, d_gate, d_pending);
    k_dem_save<<<ntiles, kTileThreads, 0, st>>>((const TileDesc *)((const char *)list + L.off_tiles),
                                                (const uint32_t *)((const char *)list + L.off_words), nn, L.ld,
                                                (const float4 *)hist, q, d_gate, d_status);
    return fpm_check_launch("fpm_dem_rebuild_begin");
}

extern "C" fpm_status fpm_dem_rebuild_end(const fpm_grid *grid, int32_t n, int32_t cap, const void *list,
                                          const uint32_t *nn, const uint32_t *perm, const void *packed, void *hist,
                                          void *omega, uint32_t *d_pending, fpm_stream stream)
{
    if (!grid || n < 0 || cap < 1 || !d_pending || grid->tiles_x < 1 ||
        (n > 0 && (!list || !nn || !perm || !packed || !hist || !omega)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_dem_rebuild_end: bad argument");
    if (n == 0) return FPM_OK;
    const ListLayout L = dem_list_layout(*grid, n, cap);
    const int ntiles = grid->tiles_x * grid->nc[1] * grid->nc[2];
    cudaStream_t st = (cudaStream_t)stream;
    k_dem_restore<<<ntiles, kTileThreads, 0, st>>>(
        n, (const TileDesc *)((const char *)list + L.off_tiles), (const uint32_t *)((const char *)list + L.off_words),
        nn, L.ld, perm, dem_packed(const_cast<void *>(packed), n), (float4 *)hist, (float4 *)omega, d_pending);
    k_dem_clear<<<1, 1, 0, st>>>(d_pending);
    return fpm_check_launch("fpm_dem_rebuild_end");
}
