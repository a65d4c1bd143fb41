// lj.cu -- Lennard-Jones pair sweep over the tiled Verlet list (Sec. 4.1:
// V(r) = 4 eps [(s/r)^12 - (s/r)^6] and the pair force
// 24 eps (2 s^12/r^14 - s^6/r^8)(x_p - x_q) of Listing 4.1, truncated at
// r_cut).
//
// Per cell tile (persistent blocks take tiles by ticket): the tile's
// neighbourhood positions are staged in shared memory (tiles.cuh), then one
// thread per home particle walks its 16-bit list entries, two per 32-bit
// word, reading neighbours from shared memory.  The sweep covers the FULL
// list (each pair from both sides): no atomics, bit-reproducible forces.
// Energy, virial and the pair count are reduced per tile in FP64 and then
// over the tiles in a fixed order.
#include <atomic>
#include <mutex>

#include "lj_pair.cuh"
#include "reduce.cuh"

namespace fpm {

template <typename T>
__global__ void __launch_bounds__(kTileThreads)
    k_lj_tiles(TileCfg cfg, BoxT<T> box, const V4<T> *__restrict__ pos, ListView lv, const uint32_t *__restrict__ nn,
               int64_t ld, int stage_cap, LJParams<T> P, V4<T> *__restrict__ force, Sched sched, double *part,
               double *out, fpm_dev_status *status, V4<T> *__restrict__ vel, T hdt, long long wait0)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    V4<T> *sp = (V4<T> *)smem_raw;
    __shared__ TileDesc d;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_k;
    __shared__ bool s_last;
    stage_init(&bar);
    uint32_t phase = 0;
    const uint32_t *__restrict__ words = lv.words;
    const uint32_t ntodo = *lv.count;
    uint32_t ahead = 0;
    for (uint32_t k = blockIdx.x; k < ntodo; k = ticket_next(ahead, &s_k)) {
        ahead = ticket_ahead(sched);
        load_desc(lv.descs + lv.active[k], d);
        if (d.h0 + threadIdx.x < d.h1) prefetch_home(pos, nn, words, ld, d.h0 + threadIdx.x, (int)kLjChunk);
        const bool in_smem = d.M <= stage_cap;
        if (!in_smem) note_spill(status);
        const bool staged =
            in_smem ? stage_positions(d, box, pos, sp, &bar, phase, status, nullptr, nullptr, wait0) : true;
        const bool all_mode = cfg.mode[0] == kModeAll || cfg.mode[1] == kModeAll || cfg.mode[2] == kModeAll;
        T usum = 0, wsum = 0;
        uint32_t npsum = 0;
        for (uint32_t i = d.h0 + threadIdx.x; staged && i < d.h1; i += blockDim.x) {
            const V4<T> pi = pos[i];
            const uint32_t m = nn[i];
            T fx = 0, fy = 0, fz = 0, u = 0, w = 0;
            uint32_t np = 0;
            if (in_smem) {
                if (d.slow && all_mode)
                    lj_sweep<T, false, true>(cfg, box, d, pos, sp, pi, m, words + i, ld, P, fx, fy, fz, u, w, np);
                else if (d.slow)
                    lj_sweep_wall<T>(box, sp, pi, m, words + i, ld, P, fx, fy, fz, u, w, np);
                else
                    lj_sweep<T, true, true>(cfg, box, d, pos, sp, pi, m, words + i, ld, P, fx, fy, fz, u, w, np);
            } else {
                lj_sweep<T, false, false>(cfg, box, d, pos, sp, pi, m, words + i, ld, P, fx, fy, fz, u, w, np);
            }
            V4<T> f;
            f.x = P.eps24 * fx;
            f.y = P.eps24 * fy;
            f.z = P.eps24 * fz;
            f.w = (T)0.5 * P.eps4 * u;
            force[i] = f;
            if (vel) {  // the closing half-kick of velocity Verlet, v += dt/2 F
                V4<T> v = vel[i];
                v.x += hdt * f.x;
                v.y += hdt * f.y;
                v.z += hdt * f.z;
                vel[i] = v;
            }
            usum += P.eps4 * u;
            wsum += P.eps24 * w;
            npsum += np;
        }
        if (out) {  // this tile's U, W, pairs (halved: every pair is seen from both sides)
            const T v[3] = {(T)0.5 * usum, (T)0.5 * wsum, (T)0.5 * (T)npsum};
            block_sum_store<3>(v, part + (size_t)k * 3);
        }
    }
    if (sched_finish(sched, &s_last) && out) {
        __threadfence();
        sum_tile_partials<3>(part, ntodo, out, false, nullptr);
    }
}

// The sweep for small systems, whose few tiles leave most of the GPU idle:
// KS threads per home particle (aligned lane groups), thread `part` walking
// the list words part, part + KS, ...; the KS partial sums are added by a
// fixed xor-shuffle tree (bit-reproducible; the grouping differs from the
// one-thread sweep's, so the forces agree with it to rounding).
template <typename T, uint32_t KS>
__global__ void __launch_bounds__(kTileThreads)
    k_lj_tiles_split(TileCfg cfg, BoxT<T> box, const V4<T> *__restrict__ pos, ListView lv,
                     const uint32_t *__restrict__ nn, int64_t ld, int stage_cap, LJParams<T> P,
                     V4<T> *__restrict__ force, Sched sched, double *part_sums, double *out, fpm_dev_status *status,
                     V4<T> *__restrict__ vel, T hdt, long long wait0)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    V4<T> *sp = (V4<T> *)smem_raw;
    __shared__ TileDesc d;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_k;
    __shared__ bool s_last;
    stage_init(&bar);
    uint32_t phase = 0;
    const uint32_t *__restrict__ words = lv.words;
    const uint32_t ntodo = *lv.count;
    const uint32_t part = threadIdx.x % KS, per_pass = blockDim.x / KS;
    uint32_t ahead = 0;
    for (uint32_t k = blockIdx.x; k < ntodo; k = ticket_next(ahead, &s_k)) {
        ahead = ticket_ahead(sched);
        load_desc(lv.descs + lv.active[k], d);
        if (d.h0 + threadIdx.x < d.h1) prefetch_home(pos, nn, words, ld, d.h0 + threadIdx.x, 1);
        const bool in_smem = d.M <= stage_cap;
        if (!in_smem) note_spill(status);
        const bool staged =
            in_smem ? stage_positions(d, box, pos, sp, &bar, phase, status, nullptr, nullptr, wait0) : true;
        const bool all_mode = cfg.mode[0] == kModeAll || cfg.mode[1] == kModeAll || cfg.mode[2] == kModeAll;
        T usum = 0, wsum = 0;
        uint32_t npsum = 0;
        const uint32_t nh = d.h1 - d.h0;
        for (uint32_t q0 = 0; staged && q0 < nh; q0 += per_pass) {  // the same trip count in every thread
            const uint32_t q = q0 + threadIdx.x / KS;
            const bool act = q < nh;
            const uint32_t i = d.h0 + (act ? q : 0u);
            T o[5] = {0, 0, 0, 0, 0};
            uint32_t np = 0;
            if (act) {
                const V4<T> pi = pos[i];
                const uint32_t m = nn[i];
                if (!in_smem)
                    lj_sweep<T, false, false, KS>(cfg, box, d, pos, sp, pi, m, words + i, ld, P, o[0], o[1], o[2],
                                                  o[3], o[4], np, part);
                else if (d.slow && all_mode)
                    lj_sweep<T, false, true, KS>(cfg, box, d, pos, sp, pi, m, words + i, ld, P, o[0], o[1], o[2],
                                                 o[3], o[4], np, part);
                else if (d.slow)
                    lj_sweep_wall<T, KS>(box, sp, pi, m, words + i, ld, P, o[0], o[1], o[2], o[3], o[4], np, part);
                else
                    lj_sweep<T, true, true, KS>(cfg, box, d, pos, sp, pi, m, words + i, ld, P, o[0], o[1], o[2], o[3],
                                                o[4], np, part);
            }
#pragma unroll
            for (uint32_t off = KS / 2; off >= 1; off >>= 1) {
#pragma unroll
                for (int c = 0; c < 5; ++c) o[c] += __shfl_xor_sync(kFull, o[c], off);
                np += __shfl_xor_sync(kFull, np, off);
            }
            if (act && part == 0) {
                V4<T> f;
                f.x = P.eps24 * o[0];
                f.y = P.eps24 * o[1];
                f.z = P.eps24 * o[2];
                f.w = (T)0.5 * P.eps4 * o[3];
                force[i] = f;
                if (vel) {  // the closing half-kick of velocity Verlet, v += dt/2 F
                    V4<T> v = vel[i];
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
        if (out) {  // this tile's U, W, pairs (halved: every pair is seen from both sides)
            const T v[3] = {(T)0.5 * usum, (T)0.5 * wsum, (T)0.5 * (T)npsum};
            block_sum_store<3>(v, part_sums + (size_t)k * 3);
        }
    }
    if (sched_finish(sched, &s_last) && out) {
        __threadfence();
        sum_tile_partials<3>(part_sums, ntodo, out, false, nullptr);
    }
}

// Systems of at most this many particles take k_lj_tiles_split.
constexpr int kSplitMaxN = 65536;

// Budget of the sweep's first wait on a tile's copies (fpm_test_wait_budget).
static std::atomic<long long> g_first_wait{0};

template <typename T>
static fpm_status lj_launch(const fpm_box &b, const fpm_grid &g, int n, const void *pos, const void *list,
                            const uint32_t *nn, int cap, double eps, double sigma, double rc, void *force,
                            double *d_energy, const RedWs &r, fpm_dev_status *status, cudaStream_t stream,
                            void *vel = nullptr, double dt = 0.0)
{
    const TileCfg cfg = make_tile_cfg(b, g);
    const ListLayout L = list_layout(n, cfg, cap);
    const BoxT<T> box = make_box<T>(b);
    LJParams<T> P;
    P.eps24 = (T)(24.0 * eps);
    P.eps4 = (T)(4.0 * eps);
    P.sig2 = (T)(sigma * sigma);
    P.rc2 = (T)(rc * rc);
    const int sc = stage_capacity(n, g, sizeof(V4<T>));
    const size_t smem = (size_t)sc * sizeof(V4<T>);
    const long long w0 = g_first_wait.load();
    if (n <= kSplitMaxN) {
        // threads per home particle: as many as a block holds for a tile of
        // 1.5x the mean occupancy (the kernel loops over larger tiles)
        const double per_tile = 1.5 * (double)n / (double)(cfg.ntiles > 0 ? cfg.ntiles : 1);
        const int ks = per_tile <= 32.0 ? 8 : per_tile <= 64.0 ? 4 : per_tile <= 128.0 ? 2 : 1;
        if (ks > 1) {
            auto kern = ks == 8 ? k_lj_tiles_split<T, 8> : ks == 4 ? k_lj_tiles_split<T, 4> : k_lj_tiles_split<T, 2>;
            smem_opt_in((const void *)kern);
            const int blocks = persistent_blocks((const void *)kern, kTileThreads, smem, g, cfg.ntiles);
            kern<<<blocks, kTileThreads, smem, stream>>>(cfg, box, (const V4<T> *)pos, list_view(list, L), nn, L.ld,
                                                          sc, P, (V4<T> *)force, Sched{r.work, r.done}, r.part,
                                                          d_energy, status, (V4<T> *)vel, (T)(0.5 * dt),
                                                          w0 > 0 ? w0 : kWaitCycles);
            return fpm_check_launch("fpm_lj_forces");
        }
    }
    smem_opt_in((const void *)k_lj_tiles<T>);
    const int blocks = persistent_blocks((const void *)k_lj_tiles<T>, kTileThreads, smem, g, cfg.ntiles);
    k_lj_tiles<T><<<blocks, kTileThreads, smem, stream>>>(cfg, box, (const V4<T> *)pos, list_view(list, L), nn, L.ld,
                                                          sc, P, (V4<T> *)force, Sched{r.work, r.done}, r.part,
                                                          d_energy, status, (V4<T> *)vel, (T)(0.5 * dt),
                                                          w0 > 0 ? w0 : kWaitCycles);
    return fpm_check_launch("fpm_lj_forces");
}

static fpm_status lj_args(const fpm_box *box, const fpm_grid *grid, int32_t n, fpm_prec prec, const void *pos,
                          const void *list, const uint32_t *nn, int32_t cap, double sigma, double rc, void *force,
                          const char *who)
{
    fpm_status s = fpm_check_grid(box, grid, who);
    if (s != FPM_OK) return s;
    if (n < 0 || cap < 1 || !(rc > 0.0) || !(sigma > 0.0) || (n > 0 && (!pos || !list || !nn || !force)))
        return fpm_fail(FPM_ERR_INVALID, "%s: null pointer or bad size", who);
    if (prec != FPM_F32 && prec != FPM_F64) return fpm_fail(FPM_ERR_INVALID, "%s: bad precision", who);
    if (((uintptr_t)list & 255u) != 0) return fpm_fail(FPM_ERR_INVALID, "%s: list not 256-B aligned", who);
    return FPM_OK;
}

// U, W and the pair count of an empty system: zeros, written on the stream.
static fpm_status zero_energy(double *d_energy, cudaStream_t st, const char *who)
{
    if (d_energy && cudaMemsetAsync(d_energy, 0, 3 * sizeof(double), st) != cudaSuccess)
        return fpm_fail(FPM_ERR_CUDA, "%s: cudaMemsetAsync failed", who);
    return FPM_OK;
}

}  // namespace fpm

using namespace fpm;

extern "C" fpm_status fpm_lj_forces(const fpm_box *box, const fpm_grid *grid, int32_t n, fpm_prec prec,
                                    const void *pos, const void *list, const uint32_t *nn, int32_t cap, double eps,
                                    double sigma, double rc, void *force, double *d_energy, void *workspace,
                                    size_t workspace_bytes, fpm_dev_status *d_status, fpm_stream stream)
{
    fpm_status s = lj_args(box, grid, n, prec, pos, list, nn, cap, sigma, rc, force, "fpm_lj_forces");
    if (s != FPM_OK) return s;
    if (n == 0) return zero_energy(d_energy, (cudaStream_t)stream, "fpm_lj_forces");
    RedWs r{};
    s = red_ws(n, grid, workspace, workspace_bytes, "fpm_lj_forces", r);
    if (s != FPM_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == FPM_F32)
        return lj_launch<float>(*box, *grid, n, pos, list, nn, cap, eps, sigma, rc, force, d_energy, r, d_status, st);
    return lj_launch<double>(*box, *grid, n, pos, list, nn, cap, eps, sigma, rc, force, d_energy, r, d_status, st);
}

extern "C" fpm_status fpm_lj_forces_kick(const fpm_box *box, const fpm_grid *grid, int32_t n, fpm_prec prec,
                                         const void *pos, const void *list, const uint32_t *nn, int32_t cap,
                                         double eps, double sigma, double rc, void *force, double *d_energy,
                                         void *workspace, size_t workspace_bytes, fpm_dev_status *d_status,
                                         void *vel, double dt, fpm_stream stream)
{
    fpm_status s = lj_args(box, grid, n, prec, pos, list, nn, cap, sigma, rc, force, "fpm_lj_forces_kick");
    if (s != FPM_OK) return s;
    if (n > 0 && !vel) return fpm_fail(FPM_ERR_INVALID, "fpm_lj_forces_kick: null vel");
    if (vel == pos || vel == force) return fpm_fail(FPM_ERR_INVALID, "fpm_lj_forces_kick: vel aliases pos or force");
    if (n == 0) return zero_energy(d_energy, (cudaStream_t)stream, "fpm_lj_forces_kick");
    RedWs r{};
    s = red_ws(n, grid, workspace, workspace_bytes, "fpm_lj_forces_kick", r);
    if (s != FPM_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == FPM_F32)
        return lj_launch<float>(*box, *grid, n, pos, list, nn, cap, eps, sigma, rc, force, d_energy, r, d_status, st,
                                vel, dt);
    return lj_launch<double>(*box, *grid, n, pos, list, nn, cap, eps, sigma, rc, force, d_energy, r, d_status, st,
                             vel, dt);
}

// ---------------------------------------------------------------------------
// fpm_lj_forces_noalloc: the same force sweep and energy reduction for callers
// that cannot allocate device memory (no cudaMalloc, no caching allocator).
// Its scratch (the per-block partial sums and the completion counter) is a
// file-scope device array, present on every GPU that loads this library.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocMaxN = 1 << 24;       // particles per call
constexpr int kNoAllocMaxBlocks = 1 << 16;  // tiles (blocks) per call
constexpr size_t kNoAllocBytes = 256 + (size_t)kNoAllocMaxBlocks * 8 * sizeof(double);  // 4 MiB + 256 B

static __device__ __align__(256) unsigned char g_lj_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_lj_scratch on the current device (looked up once per
// device; the host-side symbol itself is not a device address).
fpm_status scratch_for_current_device(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fpm_fail(FPM_ERR_CUDA, "fpm_lj_forces_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fpm_fail(FPM_ERR_INVALID, "fpm_lj_forces_noalloc: device %d", dev);
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_lj_scratch);
        if (e != cudaSuccess || !p)
            return fpm_fail(FPM_ERR_CUDA, "fpm_lj_forces_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return FPM_OK;
}

}  // namespace

extern "C" fpm_status fpm_lj_forces_noalloc(const fpm_box *box, const fpm_grid *grid, int32_t n, fpm_prec prec,
                                            const void *pos, const void *list, const uint32_t *nn, int32_t cap,
                                            double eps, double sigma, double rc, void *force, double *d_energy,
                                            fpm_dev_status *d_status, fpm_stream stream)
{
    if (n > kNoAllocMaxN)
        return fpm_fail(FPM_ERR_INVALID, "fpm_lj_forces_noalloc: n=%d exceeds the built-in scratch limit of %d particles",
                        n, kNoAllocMaxN);
    fpm_status s = lj_args(box, grid, n, prec, pos, list, nn, cap, sigma, rc, force, "fpm_lj_forces_noalloc");
    if (s != FPM_OK) return s;
    if ((int64_t)grid->tiles_x * grid->nc[1] * grid->nc[2] > kNoAllocMaxBlocks)
        return fpm_fail(FPM_ERR_INVALID, "fpm_lj_forces_noalloc: more than %d tiles exceed the built-in scratch limit",
                        kNoAllocMaxBlocks);
    if (n == 0) return zero_energy(d_energy, (cudaStream_t)stream, "fpm_lj_forces_noalloc");
    RedWs r{};
    cudaStream_t st = (cudaStream_t)stream;
    {
        void *scratch = nullptr;
        s = scratch_for_current_device(&scratch);
        if (s != FPM_OK) return s;
        // the scheduling counters must start at zero; the array keeps whatever
        // the previous call left there
        cudaError_t e = cudaMemsetAsync(scratch, 0, 64, st);
        if (e != cudaSuccess)
            return fpm_fail(FPM_ERR_CUDA, "fpm_lj_forces_noalloc: clearing the counters: %s", cudaGetErrorString(e));
        r.counter = (unsigned *)scratch;
        r.work = (unsigned *)((char *)scratch + 16);
        r.done = (unsigned *)((char *)scratch + 32);
        r.part = (double *)((char *)scratch + 256);
    }
    if (prec == FPM_F32)
        return lj_launch<float>(*box, *grid, n, pos, list, nn, cap, eps, sigma, rc, force, d_energy, r, d_status, st);
    return lj_launch<double>(*box, *grid, n, pos, list, nn, cap, eps, sigma, rc, force, d_energy, r, d_status, st);
}

extern "C" fpm_status fpm_test_wait_budget(int64_t cycles)
{
    g_first_wait.store(cycles > 0 ? (long long)cycles : 0);
    return FPM_OK;
}
