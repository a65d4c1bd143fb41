// fpm_common.cuh -- device helpers shared by the libfpm kernels (not by the
// oracle).  Geometry conventions are those stated in include/fpm.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fpm.h"

namespace fpm {

constexpr unsigned kFull = 0xffffffffu;

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4_32a; };
template <typename T> using V4 = typename Vec4<T>::type;

// The box as the kernels see it, in the path's precision.  h = L/2 exactly.
template <typename T> struct BoxT {
    T L[3];
    T h[3];
    int per[3];
};

template <typename T> __host__ __device__ inline BoxT<T> make_box(const fpm_box &b)
{
    BoxT<T> o;
    for (int d = 0; d < 3; ++d) {
        o.L[d] = (T)b.L[d];
        o.h[d] = (T)0.5 * o.L[d];
        o.per[d] = b.periodic[d] ? 1 : 0;
    }
    return o;
}

struct GridD {
    int nc[3];
    float inv[3];
};

__host__ __device__ inline GridD make_grid(const fpm_grid &g)
{
    GridD o;
    for (int d = 0; d < 3; ++d) {
        o.nc[d] = g.nc[d];
        o.inv[d] = g.inv[d];
    }
    return o;
}

// Read-only cached loads of a 4-vector.
__device__ __forceinline__ float4 ldg4(const float4 *p) { return __ldg(p); }
__device__ __forceinline__ double4_32a ldg4(const double4_32a *p)
{
    const double2 a = __ldg((const double2 *)p), b = __ldg((const double2 *)p + 1);
    double4_32a r;
    r.x = a.x;
    r.y = a.y;
    r.z = b.x;
    r.w = b.y;
    return r;
}

// Loads of a 4-vector cached at L2 only (coherent with writes made earlier in
// the same launch by other blocks, once ordered by a barrier or a flag).
__device__ __forceinline__ float4 ldcg4(const float4 *p) { return __ldcg(p); }
__device__ __forceinline__ double4_32a ldcg4(const double4_32a *p)
{
    const double2 a = __ldcg((const double2 *)p), b = __ldcg((const double2 *)p + 1);
    double4_32a r;
    r.x = a.x;
    r.y = a.y;
    r.z = b.x;
    r.w = b.y;
    return r;
}

// Small integer flags carried in the unused w component of a staged 4-vector.
template <typename T> __device__ __forceinline__ T flags_as(int f);
template <> __device__ __forceinline__ float flags_as<float>(int f) { return __int_as_float(f); }
template <> __device__ __forceinline__ double flags_as<double>(int f) { return __longlong_as_double((long long)f); }
__device__ __forceinline__ int flags_of(float w) { return __float_as_int(w); }
__device__ __forceinline__ int flags_of(double w) { return (int)__double_as_longlong(w); }

// Explicitly rounded arithmetic so that no contraction changes a decision the
// oracle takes with the same operations.
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }

// One-step periodic wrap into [0, L).
template <typename T> __device__ __forceinline__ T wrap1(T x, T L)
{
    if (x < (T)0) x = radd(x, L);
    if (x >= L) x = rsub(x, L);
    return x;
}

// Minimum-image separation of one periodic coordinate, x_i - x_j: past L/2
// the image shift is applied to the coordinate above L/2 first (exact), so the
// separation carries a single rounding, as for a pair inside the box.
template <typename T> __device__ __forceinline__ T sep1(T xi, T xj, T L, T h)
{
    const T d = rsub(xi, xj);
    if (d > h) return rsub(rsub(xi, L), xj);
    if (d < -h) return rsub(xi, rsub(xj, L));
    return d;
}

// Separation x_i - x_j under the box and its squared length
// r2 = fma(dz,dz, fma(dy,dy, dx*dx)).
template <typename T, typename P>
__device__ __forceinline__ T separation(const P &pi, const P &pj, const BoxT<T> &b, T &dx, T &dy, T &dz)
{
    dx = b.per[0] ? sep1(pi.x, pj.x, b.L[0], b.h[0]) : rsub(pi.x, pj.x);
    dy = b.per[1] ? sep1(pi.y, pj.y, b.L[1], b.h[1]) : rsub(pi.y, pj.y);
    dz = b.per[2] ? sep1(pi.z, pj.z, b.L[2], b.h[2]) : rsub(pi.z, pj.z);
    return rfma(dz, dz, rfma(dy, dy, rmul(dx, dx)));
}

// Cell coordinate of one wrapped coordinate; bad |= out of [0, L).
// The decision is taken in single precision for both position precisions.
__device__ __forceinline__ int cell_coord(float xf, float inv, int nc, bool &bad)
{
    if (!(xf >= 0.0f)) {
        bad = true;
        return 0;
    }
    float s = __fmul_rn(xf, inv);
    int c = (s >= (float)nc) ? nc : (int)s;
    return c > nc - 1 ? nc - 1 : c;
}

template <typename T, typename P>
__device__ __forceinline__ void cell_of(const P &p, const BoxT<T> &b, const GridD &g, int c[3], bool &bad)
{
    const T x[3] = {p.x, p.y, p.z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (x[d] >= b.L[d] || x[d] < (T)0) bad = true;
        c[d] = cell_coord((float)x[d], g.inv[d], g.nc[d], bad);
    }
}

__device__ __forceinline__ uint32_t linear_cell(int cx, int cy, int cz, const GridD &g)
{
    return (uint32_t)(((int64_t)cz * g.nc[1] + cy) * g.nc[0] + cx);
}

__device__ __forceinline__ bool gated_off(const uint32_t *gate)
{
    return gate != nullptr && *(volatile const uint32_t *)gate == 0u;
}

__device__ __forceinline__ void latch_flag(fpm_dev_status *st, uint32_t flag)
{
    if (st) atomicOr(&st->flags, flag);
}

// Reports a block's rebuild decision: the flag word is set if any thread saw
// a displacement above the threshold, and max_disp2 raised to the block's
// largest squared displacement (float bits; one atomic per block, skipped
// when it cannot raise the value).  All threads of the block must call it.
__device__ __forceinline__ void disp_report(bool over, float d2, fpm_dev_status *st)
{
    __shared__ unsigned s_any, s_max;
    if (threadIdx.x == 0) {
        s_any = 0u;
        s_max = 0u;
    }
    __syncthreads();
    const unsigned any = __ballot_sync(kFull, over);
    const unsigned m = __reduce_max_sync(kFull, __float_as_uint(d2));
    if ((threadIdx.x & 31) == 0) {
        if (any) atomicOr(&s_any, 1u);
        if (m) atomicMax(&s_max, m);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_any) st->rebuild = 1u;
        if (s_max > *(volatile unsigned *)&st->max_disp2) atomicMax(&st->max_disp2, s_max);
    }
}

// Warp-level sum with a fixed shuffle tree (deterministic: lane 0's result
// depends only on the 32 inputs).
template <typename TV> __device__ __forceinline__ TV warp_sum(TV v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Deterministic reduction of NV values per thread across the grid: within a
// warp in TV (the caller's accumulation type), from there on in FP64.  Every
// block writes its partial sums to part[blockIdx][NV]; the last block to
// finish (completion counter) sums the partials in index order and writes
// out[0..NV); it then resets the counter.  blockDim must be a multiple of 32
// and <= 1024.  All threads of the block must call it.  (FP64 arithmetic
// runs at a small fraction of the FP32 rate on this GPU, so the per-thread
// values are not widened before the warp stage.)
template <int NV, typename TV>
__device__ void grid_reduce(TV (&v)[NV], double *part, unsigned *counter, double *out, bool accumulate = false,
                            const double *scale = nullptr)
{
    __shared__ double sh[32][NV];
    __shared__ bool last;
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
            if (lane == 0) part[(size_t)blockIdx.x * NV + k] = s;
        }
        if (lane == 0) {
            __threadfence();
            unsigned t = atomicAdd(counter, 1u);
            last = (t == gridDim.x - 1);
        }
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += __ldcg(part + (size_t)b * NV + k);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s = warp_sum(acc[k]);
        if (lane == 0) sh[warp][k] = s;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = lane < nw ? sh[lane][k] : 0.0;
            s = warp_sum(s);
            const double val = scale ? scale[k] * s : s;
            if (lane == 0 && out) out[k] = accumulate ? out[k] + val : val;
        }
        if (lane == 0) *counter = 0u;
    }
}

}  // namespace fpm

// Host-side error plumbing (api.cu).
fpm_status fpm_fail(fpm_status s, const char *fmt, ...);
fpm_status fpm_check_launch(const char *what);

// Grid of a grid-stride kernel: `want` blocks, capped at 8 per SM.  The
// gated rebuild kernels use it, so that a launch whose gate is off retires
// in one short wave instead of one block per particle, cell or tile.
int grid_cap(long long want);
fpm_status fpm_check_grid(const fpm_box *box, const fpm_grid *grid, const char *who);
