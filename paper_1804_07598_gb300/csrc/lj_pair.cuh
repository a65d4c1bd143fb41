// lj_pair.cuh -- the Lennard-Jones pair term and the walk over one
// particle's 16-bit Verlet-list entries, shared by the single-system sweep
// (lj.cu) and the batched sweep (batch.cu).  Pair law of Sec. 4.1:
// V(r) = 4 eps [(s/r)^12 - (s/r)^6], force 24 eps (2 s^12/r^14 - s^6/r^8) r_ij.
#pragma once

#include "tiles.cuh"

namespace fpm {

// 1/x for the pair sweep.  Single precision: the hardware approximation
// refined by one Newton-Raphson step, y <- y + y (1 - x y) (the classical
// iteration for the reciprocal); inputs are squared distances (positive,
// normal).  Double precision: the correctly rounded reciprocal.
__device__ __forceinline__ float recip(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    const float e = __fmaf_rn(-x, y, 1.0f);
    return __fmaf_rn(y, e, y);
}
__device__ __forceinline__ double recip(double x) { return __drcp_rn(x); }

template <typename T> struct LJParams {
    T eps24, eps4, sig2, rc2;
};

// One list entry, masked (not branched) by the cutoff test.  With
// s6 = (sigma^2/r^2)^3 (zero beyond the cutoff) and a = 2 s6^2 - s6, the
// pair force is 24 eps a / r^2 (x_i - x_j), its virial 24 eps a and its
// energy 4 eps (s6^2 - s6).  The entry adds a / r^2 * d to the force sums
// and s6^2, s6 to S12, S6, from which the caller forms the energy sum
// S12 - S6 and the virial sum 2 S12 - S6; the constant factors 24 eps and
// 4 eps are applied once per particle.
template <typename T, bool FAST, bool SMEM>
__device__ __forceinline__ void lj_pair(const TileCfg &cfg, const BoxT<T> &box, const TileDesc &d,
                                        const V4<T> *__restrict__ pos, const V4<T> *__restrict__ st, const V4<T> &pi,
                                        int s, const LJParams<T> &P, T &fx, T &fy, T &fz, T &S12, T &S6, uint32_t &np)
{
    const V4<T> pj = SMEM ? st[s] : staged_global(d, box, pos, s);
    T dx, dy, dz;
    const T r2 = tile_sep<FAST>(pi, pj, box, cfg, dx, dy, dz);
    const bool in = r2 < P.rc2;
    const T ir2 = recip(r2);
    const T s2 = P.sig2 * ir2;
    const T s6 = in ? s2 * s2 * s2 : (T)0;
    const T s12 = s6 * s6;
    const T a = (T)2 * s12 - s6;
    const T g = a * ir2;
    fx += g * dx;
    fy += g * dy;
    fz += g * dz;
    S12 += s12;
    S6 += s6;
    np += in ? 1u : 0u;
}

// lj_pair for a tile with periodic-wall flags and no "all"-mode dimension,
// staged in shared memory (tile_sep_wall).
template <typename T>
__device__ __forceinline__ void lj_pair_wall(const V4<T> *__restrict__ st, const V4<T> &pi, const V4<T> &pim, int s,
                                             const LJParams<T> &P, T &fx, T &fy, T &fz, T &S12, T &S6, uint32_t &np)
{
    const V4<T> pj = st[s];
    T dx, dy, dz;
    const T r2 = tile_sep_wall(pi, pim, pj, dx, dy, dz);
    const bool in = r2 < P.rc2;
    const T ir2 = recip(r2);
    const T s2 = P.sig2 * ir2;
    const T s6 = in ? s2 * s2 * s2 : (T)0;
    const T s12 = s6 * s6;
    const T a = (T)2 * s12 - s6;
    const T g = a * ir2;
    fx += g * dx;
    fy += g * dy;
    fz += g * dz;
    S12 += s12;
    S6 += s6;
    np += in ? 1u : 0u;
}

// The LJ sums of one home particle over its list (list words prefetched
// kLjChunk at a time, see for_each_entry); with kStride = 2 over the words
// w_first, w_first + 2, ... only (half of the list).
constexpr uint32_t kLjChunk = 3;

template <typename T, bool FAST, bool SMEM, uint32_t kStride = 1>
__device__ __forceinline__ void lj_sweep(const TileCfg &cfg, const BoxT<T> &box, const TileDesc &d,
                                         const V4<T> *__restrict__ pos, const V4<T> *__restrict__ st,
                                         const V4<T> &pi, uint32_t m, const uint32_t *__restrict__ col, int64_t ld,
                                         const LJParams<T> &P, T &fx, T &fy, T &fz, T &u, T &w, uint32_t &np,
                                         uint32_t w_first = 0)
{
    T S12 = 0, S6 = 0;
    for_each_entry<kLjChunk, kStride>(
        m, col, ld, [&](int s) { lj_pair<T, FAST, SMEM>(cfg, box, d, pos, st, pi, s, P, fx, fy, fz, S12, S6, np); },
        w_first);
    u += S12 - S6;
    w += (T)2 * S12 - S6;
}

template <typename T, uint32_t kStride = 1>
__device__ __forceinline__ void lj_sweep_wall(const BoxT<T> &box, const V4<T> *__restrict__ st, const V4<T> &pi,
                                              uint32_t m, const uint32_t *__restrict__ col, int64_t ld,
                                              const LJParams<T> &P, T &fx, T &fy, T &fz, T &u, T &w, uint32_t &np,
                                              uint32_t w_first = 0)
{
    V4<T> pim = pi;
    pim.x = rsub(pi.x, box.L[0]);
    pim.y = rsub(pi.y, box.L[1]);
    pim.z = rsub(pi.z, box.L[2]);
    T S12 = 0, S6 = 0;
    for_each_entry<kLjChunk, kStride>(
        m, col, ld, [&](int s) { lj_pair_wall<T>(st, pi, pim, s, P, fx, fy, fz, S12, S6, np); }, w_first);
    u += S12 - S6;
    w += (T)2 * S12 - S6;
}

}  // namespace fpm
