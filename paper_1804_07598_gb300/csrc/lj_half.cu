// lj_half.cu -- the symmetric Lennard-Jones sweep over a half Verlet list:
// each interacting pair is evaluated once and its force is applied to both
// particles (Newton's third law; the symmetric interactions of Sec. 4.1, whose
// cell list lists each pair once, with the reactions summed back as the
// paper's ghost_put with a sum does, Sec. 3.4).
//
// Per cell tile (persistent blocks take tiles by ticket): the half-list tile's
// neighbourhood (fpm_verlet_build_half: the tile's own row and the four rows
// after it) is staged in shared memory next to a reaction array of three
// 64-bit integers per staged slot.  One thread per home particle walks its
// list; the particle's own force accumulates in registers in single
// precision, and every pair's reaction -F_ij on the neighbour is added to the
// neighbour's reaction slot as a fixed-point integer (units of 2^-32), held in
// shared memory as two 32-bit sums per component (the multiples of 2^23 units
// and the rest: native 32-bit shared atomics, where a 64-bit shared atomic
// add is a compare-and-swap loop).  At the end of the tile each particle's own
// force joins its own slot, the two sums of every component become one 64-bit
// integer in place, and every piece of the neighbourhood is returned to the
// global fixed-point force array with one bulk reduce-add from shared to
// global memory (cp.reduce.async.bulk ... .add.u64): no per-element global
// atomics.  Integer addition is exact and order-free, so the forces are
// bit-reproducible whatever the order in which tiles and atomics land.  A
// second launch converts the fixed-point sums to forces (and applies the
// closing half-kick of velocity Verlet), clearing the array for the next
// sweep.  Energy, virial and pair count are reduced per tile in FP64 and then
// over the tiles in a fixed order, as in the full-list sweep.
#include "lj_pair.cuh"
#include "reduce.cuh"

namespace fpm {

constexpr float kFixUnscale = 2.3283064365386963e-10f;  // 2^-32: force per fixed-point unit

// Force component x as the fixed-point value x 2^32 split into hi 2^23 + lo:
// hi = floor(x 2^9) and lo = the rest, rounded to an integer in [0, 2^23]
// (the rest times 2^23 plus 2^23 lies in [2^23, 2^24], where the float
// spacing is 1, so the fused multiply-add rounds it to an integer and its
// bits minus those of 2^23 are that integer).
__device__ __forceinline__ void fix_split(float x, int &hi, unsigned &lo)
{
    const float t = x * 512.0f;
    const float hf = floorf(t);
    hi = __float2int_rz(hf);
    lo = __float_as_uint(__fmaf_rn(t - hf, 8388608.0f, 8388608.0f)) - 0x4B000000u;
}

__device__ __forceinline__ long long fix_join(int hi, unsigned lo) { return ((long long)hi << 23) + (long long)lo; }

// Adds (x, y, z) to reaction slot s: three (lo, hi) pairs of 32-bit sums in
// shared memory, or 64-bit integers in global memory.
template <bool SMEM>
__device__ __forceinline__ void fix_add(unsigned *R, unsigned long long *g, float x, float y, float z)
{
    int h0, h1, h2;
    unsigned l0, l1, l2;
    fix_split(x, h0, l0);
    fix_split(y, h1, l1);
    fix_split(z, h2, l2);
    if (SMEM) {
        atomicAdd(R, l0);
        atomicAdd((int *)R + 1, h0);
        atomicAdd(R + 2, l1);
        atomicAdd((int *)R + 3, h1);
        atomicAdd(R + 4, l2);
        atomicAdd((int *)R + 5, h2);
    } else {
        atomicAdd(g, (unsigned long long)fix_join(h0, l0));
        atomicAdd(g + 1, (unsigned long long)fix_join(h1, l1));
        atomicAdd(g + 2, (unsigned long long)fix_join(h2, l2));
    }
}

// The pair term of lj_pair for one half-list entry; returns the force factor
// g = a / r2 (zero beyond the cutoff) with the separation in dx, dy, dz.
// SEP: 0 a tile without wall flags, 1 a tile with wall flags and no "all"-mode
// dimension (tile_sep_wall), 2 any tile (tile_sep<false>).
template <int SEP>
__device__ __forceinline__ float half_pair(const TileCfg &cfg, const BoxT<float> &box, const float4 &pi,
                                           const float4 &pim, const float4 &pj, const LJParams<float> &P, float &dx,
                                           float &dy, float &dz, float &S12, float &S6, uint32_t &np, bool &in)
{
    float r2;
    if (SEP == 0)
        r2 = tile_sep<true>(pi, pj, box, cfg, dx, dy, dz);
    else if (SEP == 1)
        r2 = tile_sep_wall(pi, pim, pj, dx, dy, dz);
    else
        r2 = tile_sep<false>(pi, pj, box, cfg, dx, dy, dz);
    in = r2 < P.rc2;
    const float ir2 = recip(r2);
    const float s2 = P.sig2 * ir2;
    const float s6 = in ? s2 * s2 * s2 : 0.0f;
    const float s12 = s6 * s6;
    S12 += s12;
    S6 += s6;
    np += in ? 1u : 0u;
    return (2.0f * s12 - s6) * ir2;
}

// The half list of home particle i: own force sums in registers, reactions
// into the shared reaction array R (SMEM) or, for a tile whose neighbourhood
// did not fit, straight into the global array acc.
template <int SEP, bool SMEM>
__device__ __forceinline__ void half_sweep(const TileCfg &cfg, const BoxT<float> &box, const TileDesc &d,
                                           const float4 *__restrict__ pos, const float4 *__restrict__ st, unsigned *R,
                                           unsigned long long *acc, const float4 &pi, uint32_t m,
                                           const uint32_t *__restrict__ col, int64_t ld, const LJParams<float> &P,
                                           float &fx, float &fy, float &fz, float &S12, float &S6, uint32_t &np)
{
    float4 pim = pi;
    if (SEP == 1) {
        pim.x = rsub(pi.x, box.L[0]);
        pim.y = rsub(pi.y, box.L[1]);
        pim.z = rsub(pi.z, box.L[2]);
    }
    for_each_entry<kLjChunk>(m, col, ld, [&](int s) {
        const float4 pj = SMEM ? st[s] : staged_global(d, box, pos, s);
        float dx, dy, dz;
        bool in;
        const float g = half_pair<SEP>(cfg, box, pi, pim, pj, P, dx, dy, dz, S12, S6, np, in);
        fx += g * dx;
        fy += g * dy;
        fz += g * dz;
        if (in) {  // the reaction -24 eps g d on the neighbour
            const float gq = -P.eps24 * g;
            fix_add<SMEM>(R + 6 * s, SMEM ? nullptr : acc + 3 * (size_t)staged_index(d, s), gq * dx, gq * dy,
                          gq * dz);
        }
    });
}

__global__ void __launch_bounds__(kTileThreads)
    k_lj_half_tiles(TileCfg cfg, BoxT<float> box, const float4 *__restrict__ pos, ListView lv,
                    const uint32_t *__restrict__ nn, int64_t ld, int stage_cap, LJParams<float> P,
                    unsigned long long *__restrict__ acc, Sched sched, double *part, double *out,
                    fpm_dev_status *status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float4 *sp = (float4 *)smem_raw;
    unsigned *R = (unsigned *)(smem_raw + (size_t)stage_cap * sizeof(float4));  // [slot][3][lo, hi]
    __shared__ TileDesc d;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_k;
    __shared__ int s_home;
    __shared__ bool s_last;
    stage_init(&bar);
    uint32_t phase = 0;
    bool issued = false;  // this thread has bulk reductions in flight
    const uint32_t *__restrict__ words = lv.words;
    const uint32_t ntodo = *lv.count;
    const bool all_mode = cfg.mode[0] == kModeAll || cfg.mode[1] == kModeAll || cfg.mode[2] == kModeAll;
    uint32_t ahead = 0;
    for (uint32_t k = blockIdx.x; k < ntodo; k = ticket_next(ahead, &s_k)) {
        ahead = ticket_ahead(sched);
        load_desc(lv.descs + lv.active[k], d);
        if (d.h0 + threadIdx.x < d.h1) prefetch_home(pos, nn, words, ld, d.h0 + threadIdx.x, (int)kLjChunk);
        const bool in_smem = d.M <= stage_cap;
        if (!in_smem) note_spill(status);
        if (in_smem) {
            // clear the reaction slots (24 bytes per staged slot, free slots included)
            uint4 *r4 = (uint4 *)R;
            const int nz = (3 * d.M + 1) / 2;
            for (int q = threadIdx.x; q < nz; q += blockDim.x) r4[q] = make_uint4(0u, 0u, 0u, 0u);
        }
        if (threadIdx.x == 0) {  // the home cells: the piece of the tile's own row (row 0) seen directly,
                                 // not through a periodic wall (a wall piece may hold a copy of cell a)
            int h = 0;
            for (int p = 0; p < kPiecesPerRow; ++p) {
                const Piece pc = d.piece[p];
                if (pc.len > 0 && (pc.flags & (kLoX | kUpX)) == 0 && d.h0 >= pc.gstart &&
                    d.h0 < pc.gstart + (uint32_t)pc.len)
                    h = pc.soff + (int)(d.h0 - pc.gstart);
            }
            s_home = h;
        }
        const bool staged = in_smem ? stage_positions(d, box, pos, sp, &bar, phase, status) : true;
        float usum = 0.0f, wsum = 0.0f;
        uint32_t npsum = 0;
        for (uint32_t i = d.h0 + threadIdx.x; staged && i < d.h1; i += blockDim.x) {
            const float4 pi = pos[i];
            const uint32_t m = nn[i];
            float fx = 0.0f, fy = 0.0f, fz = 0.0f, S12 = 0.0f, S6 = 0.0f;
            uint32_t np = 0;
            if (in_smem) {
                if (!d.slow)
                    half_sweep<0, true>(cfg, box, d, pos, sp, R, acc, pi, m, words + i, ld, P, fx, fy, fz, S12, S6,
                                        np);
                else if (!all_mode)
                    half_sweep<1, true>(cfg, box, d, pos, sp, R, acc, pi, m, words + i, ld, P, fx, fy, fz, S12, S6,
                                        np);
                else
                    half_sweep<2, true>(cfg, box, d, pos, sp, R, acc, pi, m, words + i, ld, P, fx, fy, fz, S12, S6,
                                        np);
            } else {
                half_sweep<2, false>(cfg, box, d, pos, sp, R, acc, pi, m, words + i, ld, P, fx, fy, fz, S12, S6, np);
            }
            // the particle's own force joins its slot (or its global row)
            if (in_smem)
                fix_add<true>(R + 6 * (s_home + (int)(i - d.h0)), nullptr, P.eps24 * fx, P.eps24 * fy, P.eps24 * fz);
            else
                fix_add<false>(nullptr, acc + 3 * (size_t)i, P.eps24 * fx, P.eps24 * fy, P.eps24 * fz);
            usum += P.eps4 * (S12 - S6);
            wsum += P.eps24 * (2.0f * S12 - S6);
            npsum += np;
        }
        __syncthreads();  // every reaction of the tile is in R
        if (in_smem && staged) {  // each component's two 32-bit sums become one 64-bit integer, in place
            uint2 *cell = (uint2 *)R;
            for (int q = threadIdx.x; q < 3 * d.M; q += blockDim.x) {
                const uint2 v = cell[q];
                ((unsigned long long *)cell)[q] = (unsigned long long)fix_join((int)v.y, v.x);
            }
        }
        __syncthreads();
        if (in_smem && staged && threadIdx.x < (unsigned)kMaxPieces) {
            // piece p's slots cover the even-aligned index range of its particles
            // (tile_geometry<true>): one bulk reduce-add of 24-byte rows per piece
            const Piece pc = d.piece[threadIdx.x];
            if (pc.len > 0) {
                const uint32_t g0 = pc.gstart & ~1u, g1 = (pc.gstart + (uint32_t)pc.len + 1u) & ~1u;
                const int s0 = pc.soff - (int)(pc.gstart & 1u);
                const uint32_t bytes = (g1 - g0) * 24u;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.u64 [%0], [%1], %2;" ::"l"(
                                 acc + 3 * (size_t)g0),
                             "r"(smem_u32(R + 6 * s0)), "r"(bytes)
                             : "memory");
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                issued = true;
            }
        }
        if (out) {
            const float v[3] = {usum, wsum, (float)npsum};
            block_sum_store<3>(v, part + (size_t)k * 3);
        }
        // the reductions have read R before the next tile clears it
        if (issued) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
    if (issued) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    if (sched_finish(sched, &s_last) && out) {
        __threadfence();
        sum_tile_partials<3>(part, ntodo, out, false, nullptr);
    }
}

// Forces from the fixed-point sums (w = 0), the array cleared for the next
// sweep, and optionally the closing half-kick v += dt/2 F.
__global__ void k_lj_half_finish(int n, unsigned long long *__restrict__ acc, float4 *__restrict__ force,
                                 float4 *__restrict__ vel, float hdt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long *a = acc + 3 * (size_t)i;
    float4 f;
    f.x = __ll2float_rn((long long)a[0]) * kFixUnscale;
    f.y = __ll2float_rn((long long)a[1]) * kFixUnscale;
    f.z = __ll2float_rn((long long)a[2]) * kFixUnscale;
    f.w = 0.0f;
    a[0] = 0ull;
    a[1] = 0ull;
    a[2] = 0ull;
    force[i] = f;
    if (vel) {
        float4 v = vel[i];
        v.x += hdt * f.x;
        v.y += hdt * f.y;
        v.z += hdt * f.z;
        vel[i] = v;
    }
}

}  // namespace fpm

using namespace fpm;

extern "C" fpm_status fpm_lj_half_acc_bytes(int32_t n, size_t *bytes)
{
    if (n < 0 || !bytes) return fpm_fail(FPM_ERR_INVALID, "fpm_lj_half_acc_bytes: bad argument");
    *bytes = (size_t)((n + 1) & ~1) * 3 * sizeof(unsigned long long);
    return FPM_OK;
}

extern "C" fpm_status fpm_lj_forces_half(const fpm_box *box, const fpm_grid *grid, int32_t n, const void *pos,
                                         const void *list, const uint32_t *nn, int32_t cap, double eps, double sigma,
                                         double rc, void *force, double *d_energy, void *acc, size_t acc_bytes,
                                         void *workspace, size_t workspace_bytes, fpm_dev_status *d_status, void *vel,
                                         double dt, fpm_stream stream)
{
    fpm_status s = fpm_check_grid(box, grid, "fpm_lj_forces_half");
    if (s != FPM_OK) return s;
    if (n < 0 || cap < 1 || !(rc > 0.0) || !(sigma > 0.0) || (n > 0 && (!pos || !list || !nn || !force || !acc)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_lj_forces_half: null pointer or bad size");
    if (((uintptr_t)list & 255u) != 0) return fpm_fail(FPM_ERR_INVALID, "fpm_lj_forces_half: list not 256-B aligned");
    if (vel && (vel == pos || vel == force))
        return fpm_fail(FPM_ERR_INVALID, "fpm_lj_forces_half: vel aliases pos or force");
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) {
        if (d_energy && cudaMemsetAsync(d_energy, 0, 3 * sizeof(double), st) != cudaSuccess)
            return fpm_fail(FPM_ERR_CUDA, "fpm_lj_forces_half: cudaMemsetAsync failed");
        return FPM_OK;
    }
    size_t need = 0;
    fpm_lj_half_acc_bytes(n, &need);
    if (acc_bytes < need || ((uintptr_t)acc & 15u) != 0)
        return fpm_fail(FPM_ERR_WORKSPACE, "fpm_lj_forces_half: acc %zu < %zu bytes or not 16-B aligned", acc_bytes,
                        need);
    RedWs r{};
    s = red_ws(n, grid, workspace, workspace_bytes, "fpm_lj_forces_half", r);
    if (s != FPM_OK) return s;
    const TileCfg cfg = make_tile_cfg(*box, *grid);
    const ListLayout L = list_layout(n, cfg, cap);
    LJParams<float> P;
    P.eps24 = (float)(24.0 * eps);
    P.eps4 = (float)(4.0 * eps);
    P.sig2 = (float)(sigma * sigma);
    P.rc2 = (float)(rc * rc);
    // staged positions and the reaction slots: 16 + 24 bytes per staged slot
    const int sc = stage_capacity(n, *grid, sizeof(float4) + 3 * sizeof(unsigned long long));
    const size_t smem = (size_t)sc * (sizeof(float4) + 3 * sizeof(unsigned long long));
    smem_opt_in((const void *)k_lj_half_tiles);
    const int blocks = persistent_blocks((const void *)k_lj_half_tiles, kTileThreads, smem, *grid, cfg.ntiles);
    k_lj_half_tiles<<<blocks, kTileThreads, smem, st>>>(cfg, make_box<float>(*box), (const float4 *)pos,
                                                        list_view(list, L), nn, L.ld, sc, P,
                                                        (unsigned long long *)acc, Sched{r.work, r.done}, r.part,
                                                        d_energy, d_status);
    k_lj_half_finish<<<(n + 255) / 256, 256, 0, st>>>(n, (unsigned long long *)acc, (float4 *)force, (float4 *)vel,
                                                      (float)(0.5 * dt));
    return fpm_check_launch("fpm_lj_forces_half");
}
