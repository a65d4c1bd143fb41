// verlet.cu -- Verlet-list build over the sorted cell list and the
// displacement test that decides when to rebuild it (Verlet lists [46] of
// Sec. 2, used for the MD benchmark of Sec. 4.1; skin and rebuild rule: half
// the skin, the textbook criterion).
//
// Thread per particle i (sorted order).  For each of the 9 (dz,dy) rows of
// the 27-cell stencil the three x-cells cx-1..cx+1 are consecutive in the
// sorted arrays, so a row is one index range (two when it wraps around the
// periodic x boundary); candidates are streamed from those ranges.
#include "fpm_common.cuh"

namespace fpm {

// Offsets of one dimension of the stencil: {c-1,c,c+1} (wrapped or clipped),
// or {c} when the dimension has one cell.  Returns how many.
__device__ __forceinline__ int stencil_dim(int c, int nc, int per, int out[3])
{
    if (nc == 1) {
        out[0] = 0;
        return 1;
    }
    int k = 0;
#pragma unroll
    for (int o = -1; o <= 1; ++o) {
        int cc = c + o;
        if (per) cc = cc < 0 ? cc + nc : (cc >= nc ? cc - nc : cc);
        else if (cc < 0 || cc >= nc) continue;
        out[k++] = cc;
    }
    return k;
}

template <typename T>
__global__ void __launch_bounds__(256) k_verlet_build(BoxT<T> box, GridD grid, int n, const V4<T> *__restrict__ pos,
                                                      const uint32_t *__restrict__ cs, T rl2, int cap, int64_t ld,
                                                      uint32_t *__restrict__ nbr, uint32_t *__restrict__ nn,
                                                      V4<T> *__restrict__ pos_ref, fpm_dev_status *st,
                                                      const uint32_t *gate)
{
    if (gated_off(gate)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t cnt = 0;
    if (i < n) {
        const V4<T> pi = pos[i];
        if (pos_ref) pos_ref[i] = pi;
        bool bad = false;
        int c[3];
        cell_of(pi, box, grid, c, bad);
        int oz[3], oy[3];
        const int kz = stencil_dim(c[2], grid.nc[2], box.per[2], oz);
        const int ky = stencil_dim(c[1], grid.nc[1], box.per[1], oy);
        const int ncx = grid.nc[0];
        // x range(s) of the row, as cell offsets [x0, x1] (inclusive) pieces
        int xa0, xa1, xb0 = 1, xb1 = 0;  // second piece empty unless wrapping
        if (ncx == 1) {
            xa0 = 0;
            xa1 = 0;
        } else if (box.per[0]) {
            if (c[0] == 0) {
                xa0 = 0; xa1 = 1; xb0 = ncx - 1; xb1 = ncx - 1;
            } else if (c[0] == ncx - 1) {
                xa0 = ncx - 2; xa1 = ncx - 1; xb0 = 0; xb1 = 0;
            } else {
                xa0 = c[0] - 1; xa1 = c[0] + 1;
            }
        } else {
            xa0 = c[0] > 0 ? c[0] - 1 : 0;
            xa1 = c[0] < ncx - 1 ? c[0] + 1 : ncx - 1;
        }
        for (int a = 0; a < kz; ++a) {
            for (int b = 0; b < ky; ++b) {
                const uint32_t row = linear_cell(0, oy[b], oz[a], grid);
#pragma unroll 1
                for (int piece = 0; piece < 2; ++piece) {
                    const int x0 = piece ? xb0 : xa0, x1 = piece ? xb1 : xa1;
                    if (x0 > x1) continue;
                    const uint32_t j0 = cs[row + x0], j1 = cs[row + x1 + 1];
                    for (uint32_t j = j0; j < j1; ++j) {
                        if (j == (uint32_t)i) continue;
                        const V4<T> pj = pos[j];
                        T dx, dy, dz;
                        const T r2 = separation(pi, pj, box, dx, dy, dz);
                        if (r2 < rl2) {
                            if (cnt < (uint32_t)cap) nbr[(int64_t)cnt * ld + i] = j;
                            ++cnt;
                        }
                    }
                }
            }
        }
        nn[i] = cnt < (uint32_t)cap ? cnt : (uint32_t)cap;
        if (cnt > (uint32_t)cap) latch_flag(st, FPM_FLAG_CAPACITY);
    }
    // one atomic max per warp
    uint32_t m = __reduce_max_sync(kFull, cnt);
    if ((threadIdx.x & 31) == 0 && st && m > 0) atomicMax(&st->max_nn, m);
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
    const unsigned any = __ballot_sync(kFull, over);
    const uint32_t m = __reduce_max_sync(kFull, __float_as_uint(d2f));
    if ((threadIdx.x & 31) == 0) {
        if (any) st->rebuild = 1u;
        if (m) atomicMax(&st->max_disp2, m);
    }
}

template <typename T>
static fpm_status verlet_launch(const fpm_box &b, const fpm_grid &g, int n, const void *pos, const uint32_t *cs,
                                double r_list, int cap, uint32_t *nbr, uint32_t *nn, void *pos_ref,
                                fpm_dev_status *st, uint32_t *gate, cudaStream_t stream)
{
    const BoxT<T> box = make_box<T>(b);
    const GridD grid = make_grid(g);
    const T rl2 = (T)(r_list * r_list);
    if (n > 0)
        k_verlet_build<T><<<(n + 255) / 256, 256, 0, stream>>>(box, grid, n, (const V4<T> *)pos, cs, rl2, cap,
                                                               fpm_nbr_ld(n), nbr, nn, (V4<T> *)pos_ref, st, gate);
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

extern "C" fpm_status fpm_verlet_build(const fpm_box *box, const fpm_grid *grid, int32_t n, fpm_prec prec,
                                       const void *pos, const uint32_t *cell_start, double r_list, int32_t cap,
                                       uint32_t *nbr, uint32_t *nn, void *pos_ref, fpm_dev_status *d_status,
                                       uint32_t *d_gate, fpm_stream stream)
{
    if (!box_ok(box) || !grid || n < 0 || cap < 1 || !(r_list > 0.0) || !cell_start ||
        (n > 0 && (!pos || !nbr || !nn)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_verlet_build: null pointer or bad size");
    if (prec != FPM_F32 && prec != FPM_F64) return fpm_fail(FPM_ERR_INVALID, "fpm_verlet_build: bad precision");
    for (int d = 0; d < 3; ++d) {
        if (grid->nc[d] < 1) return fpm_fail(FPM_ERR_INVALID, "fpm_verlet_build: bad grid");
        // every cell must be at least r_list wide, and a periodic box must hold the sphere
        if (grid->nc[d] > 1 && box->L[d] / grid->nc[d] < r_list)
            return fpm_fail(FPM_ERR_INVALID, "fpm_verlet_build: cells narrower than r_list in dim %d", d);
        if (box->periodic[d] && !(box->L[d] > 2.0 * r_list * (1.0 + 1.0 / 1024.0)))
            return fpm_fail(FPM_ERR_INVALID, "fpm_verlet_build: periodic L[%d] must exceed 2 r_list", d);
        if (box->periodic[d] && grid->nc[d] == 2)
            return fpm_fail(FPM_ERR_INVALID, "fpm_verlet_build: a periodic dim cannot have 2 cells");
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == FPM_F32)
        return verlet_launch<float>(*box, *grid, n, pos, cell_start, r_list, cap, nbr, nn, pos_ref, d_status, d_gate,
                                    st);
    return verlet_launch<double>(*box, *grid, n, pos, cell_start, r_list, cap, nbr, nn, pos_ref, d_status, d_gate, st);
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
