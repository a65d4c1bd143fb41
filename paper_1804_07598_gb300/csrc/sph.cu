// sph.cu -- weakly compressible SPH rates (Sec. 4.2, Eqs. 1-5) over the tiled
// Verlet list, and the symplectic predictor / corrector.
//
// State per particle (sorted order): pos = (x, y, z, type) with type 0 for
// fluid and 1 for a fixed boundary particle; vr = (vx, vy, vz, drho) where
// drho = rho - rho0 (carrying the density deviation keeps the Tait pressure,
// a difference of nearly equal numbers, accurate in single precision).
// Rates: acc = (ax, ay, az, Drho/Dt).
//
// For each pair inside the kernel support 2h (the list is built with
// r_list = 2h + skin):
//   grad_p W = F (x_p - x_q),  F = (dW/dr)/r,
//   Drho_p  += m (v_p - v_q) . grad_p W                               (Eq. 2)
//   a_p     += -m [(P_p + P_q)/(rho_p rho_q) + Pi_pq] grad_p W         (Eq. 1)
//   Pi_pq    = -alpha c0 mu / rhobar when (v_p - v_q).(x_p - x_q) < 0, else 0,
//   mu       = h (v_p - v_q).(x_p - x_q) / (r^2 + eta^2)               (Eq. 5)
//   P        = b [(rho/rho0)^gamma - 1],  b = c0^2 rho0 / gamma       (Eqs. 3-4)
// with a_p += g for fluid and a_p = 0 for boundary particles.  The pressure is
// evaluated as b * sum_{k=1..gamma} C(gamma,k) x^k, x = drho/rho0 (the
// binomial expansion, no cancellation), which needs an integer gamma (<= 8).
#include "reduce.cuh"
#include "tiles.cuh"

namespace fpm {

struct SphK {
    float h, m, rho0, inv_rho0, c0, alpha, eta2, b, g[3];
    float two_h2;    // (2h)^2, the support test
    float wcoef;     // m times (Wendland: F = wcoef (1 - q/2)^3;  cubic: s/h^2)
    float visc2;     // -2 alpha c0 (Pi_pq = visc2 mu / (rho_p + rho_q))
    float inv_h;
    float wnorm;     // m W(0): m a (Wendland) or m s (cubic), the kernel's normalisation times m
    float binom[8];  // C(gamma, k), k = 1..gamma (0 beyond)
    int gamma;
    int kernel;      // 0 Wendland C2, 1 cubic spline
};

// 1/x by the hardware approximation alone (within 1 ulp, as the PTX ISA
// states for rcp.approx.f32): the SPH rates are held to 1e-4 of their RMS,
// four orders above that rounding.  (The LJ sweep refines its 1/r^2 with a
// Newton step: its forces are held to 1e-5 and carry r^-14.)
__device__ __forceinline__ float sph_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// b * ((1 + x)^gamma - 1) by Horner on the binomial coefficients.
__device__ __forceinline__ float tait(const SphK &K, float drho)
{
    const float x = drho * K.inv_rho0;
    float s = 0.0f;
#pragma unroll
    for (int k = 7; k >= 0; --k) s = __fmaf_rn(s, x, K.binom[k]);
    return K.b * (s * x);
}

// m (dW/dr)/r for r2 inside the support; KK = 0 Wendland C2, 1 cubic spline.
template <int KK>
__device__ __forceinline__ float grad_factor(const SphK &K, float r2)
{
    const float ir = rsqrtf(r2);
    const float q = r2 * ir * K.inv_h;
    if (KK == 0) {
        const float t = 1.0f - 0.5f * q;
        return K.wcoef * t * t * t;
    }
    // cubic spline: s/h^2 (-3 + 2.25 q) for q < 1; -0.75 s/h^2 (2-q)^2 / q for q >= 1
    const float t = 2.0f - q;
    return q < 1.0f ? K.wcoef * (-3.0f + 2.25f * q) : -0.75f * K.wcoef * t * t * sph_rcp(q);
}

// PRE: the staged slots already hold P_q in the position's w and rho_q in the
// velocity's w (written once per tile by k_sph_tiles for tiles without
// periodic-wall flags, whose position w is otherwise unused).
template <bool FAST, bool SMEM, int KK, bool PRE = false>
__device__ __forceinline__ void sph_pair(const TileCfg &cfg, const BoxT<float> &box, const TileDesc &d,
                                         const float4 *__restrict__ pos, const float4 *__restrict__ vr,
                                         const float4 *__restrict__ st, const float4 *__restrict__ sv,
                                         const float4 &pi, const float4 &vi, float rho_i, float P_i, int s,
                                         const SphK &K, float &ax, float &ay, float &az, float &dr, float &mumax)
{
    float4 pj, vj;
    if (SMEM) {
        pj = st[s];
        vj = sv[s];
    } else {
        pj = staged_global(d, box, pos, s);
        vj = ldg4(vr + staged_index(d, s));
    }
    float dx, dy, dz;
    const float r2 = tile_sep<FAST>(pi, pj, box, cfg, dx, dy, dz);
    const bool in = r2 < K.two_h2 && r2 > 0.0f;
    const float Fm = in ? grad_factor<KK>(K, r2) : 0.0f;  // m F
    const float vx = vi.x - vj.x, vy = vi.y - vj.y, vz = vi.z - vj.z;
    const float vdr = vx * dx + vy * dy + vz * dz;
    dr = fmaf(Fm, vdr, dr);
    const float rho_j = PRE ? vj.w : K.rho0 + vj.w;
    const float Pj = PRE ? pj.w : tait(K, vj.w);
    const float inv_rr = sph_rcp(rho_i * rho_j);
    const float mu = K.h * vdr * sph_rcp(r2 + K.eta2);
    const float visc = vdr < 0.0f ? K.visc2 * mu * sph_rcp(rho_i + rho_j) : 0.0f;
    const float c = ((P_i + Pj) * inv_rr + visc) * Fm;
    ax = fmaf(-c, dx, ax);
    ay = fmaf(-c, dy, ay);
    az = fmaf(-c, dz, az);
    if (in) mumax = fmaxf(mumax, fabsf(mu));
}

// One half of a home particle's list: words half, half + 2, ... (two threads
// share each particle and add their sums).
template <bool FAST, bool SMEM, int KK, bool PRE = false>
__device__ __forceinline__ void sph_sweep(const TileCfg &cfg, const BoxT<float> &box, const TileDesc &d,
                                          const float4 *__restrict__ pos, const float4 *__restrict__ vr,
                                          const float4 *__restrict__ st, const float4 *__restrict__ sv,
                                          const float4 &pi, const float4 &vi, float rho_i, float Pi, uint32_t m,
                                          uint32_t half, const uint32_t *__restrict__ col, int64_t ld,
                                          const SphK &K, float &ax, float &ay, float &az, float &dr, float &mumax)
{
    for_each_entry<2, 2>(
        m, col, ld,
        [&](int s) {
            sph_pair<FAST, SMEM, KK, PRE>(cfg, box, d, pos, vr, st, sv, pi, vi, rho_i, Pi, s, K, ax, ay, az, dr,
                                          mumax);
        },
        half);
}

// The sweep of a tile whose neighbourhood did not fit in shared memory (rare;
// out of line so that it does not add to the registers of the common path).
template <int KK>
__device__ __noinline__ void sph_sweep_spilled(const TileCfg &cfg, const BoxT<float> &box, const TileDesc &d,
                                               const float4 *__restrict__ pos, const float4 *__restrict__ vr,
                                               const float4 &pi, const float4 &vi, float rho_i, float P_i,
                                               uint32_t m, uint32_t half, const uint32_t *__restrict__ col,
                                               int64_t ld, const SphK &K, float *out5)
{
    float ax = 0.0f, ay = 0.0f, az = 0.0f, dr = 0.0f, mumax = 0.0f;
    sph_sweep<false, false, KK>(cfg, box, d, pos, vr, nullptr, nullptr, pi, vi, rho_i, P_i, m, half, col, ld, K, ax,
                                ay, az, dr, mumax);
    out5[0] = ax;
    out5[1] = ay;
    out5[2] = az;
    out5[3] = dr;
    out5[4] = mumax;
}

// Two threads per home particle (tiles of about 170 particles): 384-thread
// blocks, two per SM at 80 registers.
constexpr int kSphThreads = 384;

template <int KK>
__global__ void __launch_bounds__(kSphThreads, 2)
    k_sph_tiles(TileCfg cfg, BoxT<float> box, const float4 *__restrict__ pos, const float4 *__restrict__ vr,
                ListView lv, const uint32_t *__restrict__ nn, int64_t ld, int stage_cap, SphK K,
                float4 *__restrict__ acc, float *dtcons, Sched sched, fpm_dev_status *status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float4 *sp = (float4 *)smem_raw;
    float4 *sv = sp + stage_cap;
    __shared__ TileDesc d;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_k;
    __shared__ bool s_last;
    stage_init(&bar);
    uint32_t phase = 0;
    const uint32_t *__restrict__ words = lv.words;
    float amax = 0.0f, mumax = 0.0f;
    const uint32_t ntodo = *lv.count;
    uint32_t ahead = 0;
    for (uint32_t k = blockIdx.x; k < ntodo; k = ticket_next(ahead, &s_k)) {
        ahead = ticket_ahead(sched);
    load_desc(lv.descs + lv.active[k], d);
    if (d.h0 + threadIdx.x < d.h1) {
        prefetch_home(pos, nn, words, ld, d.h0 + threadIdx.x, 4);
        asm volatile("prefetch.global.L2 [%0];" ::"l"(vr + d.h0 + threadIdx.x));
    }
    const bool in_smem = d.M <= stage_cap;
    if (!in_smem) note_spill(status);
    const bool staged = in_smem ? stage_positions(d, box, pos, sp, &bar, phase, status, vr, sv) : true;
    // once per staged neighbour instead of once per pair: P_q and rho_q
    if (in_smem && staged && !d.slow) {
        for (int s = threadIdx.x; s < d.M; s += blockDim.x) {
            const float drho = sv[s].w;
            sp[s].w = tait(K, drho);
            sv[s].w = K.rho0 + drho;
        }
        __syncthreads();
    }
    // lanes 2t and 2t + 1 share home particle h0 + t, each walking half its list
    for (uint32_t t = threadIdx.x; staged && d.h0 + (t >> 1) < d.h1; t += blockDim.x) {
        const uint32_t i = d.h0 + (t >> 1), half = t & 1u;
        const float4 pi = pos[i];
        const float4 vi = vr[i];
        const uint32_t m = nn[i];
        const float rho_i = K.rho0 + vi.w;
        const float P_i = tait(K, vi.w);
        float ax = 0.0f, ay = 0.0f, az = 0.0f, dr = 0.0f;
        if (in_smem) {
            if (d.slow)
                sph_sweep<false, true, KK>(cfg, box, d, pos, vr, sp, sv, pi, vi, rho_i, P_i, m, half, words + i, ld,
                                           K, ax, ay, az, dr, mumax);
            else
                sph_sweep<true, true, KK, true>(cfg, box, d, pos, vr, sp, sv, pi, vi, rho_i, P_i, m, half, words + i,
                                                ld, K, ax, ay, az, dr, mumax);
        } else {
            float o5[5];
            sph_sweep_spilled<KK>(cfg, box, d, pos, vr, pi, vi, rho_i, P_i, m, half, words + i, ld, K, o5);
            ax = o5[0];
            ay = o5[1];
            az = o5[2];
            dr = o5[3];
            mumax = fmaxf(mumax, o5[4]);
        }
        // the lanes of this warp still in the loop: a prefix (t < 2 (h1 - h0)),
        // which holds both lanes of every pair
        const uint32_t tw = t - (threadIdx.x & 31u);
        const uint32_t live = 2u * (d.h1 - d.h0) - tw;
        const unsigned act = live >= 32u ? kFull : ((1u << live) - 1u);
        ax += __shfl_xor_sync(act, ax, 1);
        ay += __shfl_xor_sync(act, ay, 1);
        az += __shfl_xor_sync(act, az, 1);
        dr += __shfl_xor_sync(act, dr, 1);
        if (half == 0u) {
            float4 a;
            if (pi.w == 0.0f) {
                a.x = ax + K.g[0];
                a.y = ay + K.g[1];
                a.z = az + K.g[2];
                amax = fmaxf(amax, sqrtf(a.x * a.x + a.y * a.y + a.z * a.z));
            } else {
                a.x = a.y = a.z = 0.0f;
            }
            a.w = dr;
            acc[i] = a;
        }
    }
    }
    // one atomic max per warp on the (non-negative) float bits
    const unsigned ma = __reduce_max_sync(kFull, __float_as_uint(amax));
    const unsigned mm = __reduce_max_sync(kFull, __float_as_uint(mumax));
    if ((threadIdx.x & 31) == 0 && dtcons) {
        if (ma) atomicMax((unsigned *)dtcons, ma);
        if (mm) atomicMax((unsigned *)dtcons + 1, mm);
    }
    sched_finish(sched, &s_last);
}

// ---- density by summation ---------------------------------------------------
// rho_i = m W(0) + sum over the list entries inside the support of m W(r_ij),
// with W the kernel of Sec. 4.2 (Wendland C2: a (1 - q/2)^4 (2q + 1);
// cubic spline: s [1 - 1.5 q^2 + 0.75 q^3] for q < 1, s (2 - q)^3 / 4 for
// q < 2), q = r/h.  One thread per home particle, the tile's neighbourhood
// staged as in the other sweeps.

// m W(r) / (m W(0)) for r2 inside the support.
template <int KK>
__device__ __forceinline__ float kernel_shape(const SphK &K, float r2)
{
    const float q = sqrtf(r2) * K.inv_h;
    if (KK == 0) {
        const float t = 1.0f - 0.5f * q;
        const float t2 = t * t;
        return t2 * t2 * (2.0f * q + 1.0f);
    }
    if (q < 1.0f) return 1.0f - q * q * (1.5f - 0.75f * q);
    const float t = 2.0f - q;
    return 0.25f * t * t * t;
}

template <bool FAST, bool SMEM, int KK>
__device__ __forceinline__ float density_sweep(const TileCfg &cfg, const BoxT<float> &box, const TileDesc &d,
                                               const float4 *__restrict__ pos, const float4 *__restrict__ st,
                                               const float4 &pi, uint32_t m, const uint32_t *__restrict__ col,
                                               int64_t ld, const SphK &K)
{
    float sum = 1.0f;  // the particle itself, W(0)
    for_each_entry<3>(m, col, ld, [&](int s) {
        const float4 pj = SMEM ? st[s] : staged_global(d, box, pos, s);
        float dx, dy, dz;
        const float r2 = tile_sep<FAST>(pi, pj, box, cfg, dx, dy, dz);
        sum += r2 < K.two_h2 ? kernel_shape<KK>(K, r2) : 0.0f;
    });
    return K.wnorm * sum;
}

template <int KK>
__global__ void __launch_bounds__(kTileThreads)
    k_sph_density_tiles(TileCfg cfg, BoxT<float> box, const float4 *__restrict__ pos, ListView lv,
                        const uint32_t *__restrict__ nn, int64_t ld, int stage_cap, SphK K, float *__restrict__ rho,
                        Sched sched, fpm_dev_status *status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float4 *sp = (float4 *)smem_raw;
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
        if (d.h0 + threadIdx.x < d.h1) prefetch_home(pos, nn, words, ld, d.h0 + threadIdx.x, 3);
        const bool in_smem = d.M <= stage_cap;
        if (!in_smem) note_spill(status);
        const bool staged = in_smem ? stage_positions(d, box, pos, sp, &bar, phase, status) : true;
        for (uint32_t i = d.h0 + threadIdx.x; staged && i < d.h1; i += blockDim.x) {
            const float4 pi = pos[i];
            const uint32_t m = nn[i];
            float r;
            if (!in_smem)
                r = density_sweep<false, false, KK>(cfg, box, d, pos, sp, pi, m, words + i, ld, K);
            else if (d.slow)
                r = density_sweep<false, true, KK>(cfg, box, d, pos, sp, pi, m, words + i, ld, K);
            else
                r = density_sweep<true, true, KK>(cfg, box, d, pos, sp, pi, m, words + i, ld, K);
            rho[i] = r;
        }
    }
    sched_finish(sched, &s_last);
}

__device__ __forceinline__ float sph_dt(const float *dtcons, float h, float c0, float cfl)
{
    const float amax = dtcons[0], mumax = dtcons[1];
    const float dtf = amax > 0.0f ? sqrtf(h / amax) : 3.0e38f;
    const float dtv = h / (c0 + mumax);
    return cfl * fminf(dtf, dtv);
}

// Symplectic predictor: dt from the constraints of the rates at t^n; half
// step x += dt/2 v, v += dt/2 a (fluid), drho += dt/2 Drho (all).  Also runs
// the Verlet rebuild test on the half-step positions.
__global__ void k_sph_predict(int n, BoxT<float> box, const float4 *__restrict__ pos, const float4 *__restrict__ vr,
                              const float4 *__restrict__ acc, const float *__restrict__ dtcons, float h, float c0,
                              float cfl, float4 *__restrict__ pos_h, float4 *__restrict__ vr_h, float *d_dt,
                              float *dtcons_h, const float4 *__restrict__ ref, float th, fpm_dev_status *st)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const float dt = sph_dt(dtcons, h, c0, cfl);
    if (i == 0) {
        *d_dt = dt;
        dtcons_h[0] = 0.0f;
        dtcons_h[1] = 0.0f;
    }
    bool over = false;
    float d2 = 0.0f;
    if (i < n) {
        float4 p = pos[i], v = vr[i];
        const float4 a = acc[i];
        if (p.w == 0.0f) {
            p.x += 0.5f * dt * v.x;
            p.y += 0.5f * dt * v.y;
            p.z += 0.5f * dt * v.z;
            v.x += 0.5f * dt * a.x;
            v.y += 0.5f * dt * a.y;
            v.z += 0.5f * dt * a.z;
        }
        v.w += 0.5f * dt * a.w;
        pos_h[i] = p;
        vr_h[i] = v;
        if (ref) {
            float dx, dy, dz;
            d2 = separation(p, ref[i], box, dx, dy, dz);
            over = d2 > th;
        }
    }
    if (ref) disp_report(over, d2, st);
}

// Symplectic corrector with the rates at the half step:
//   v1 = v0 + dt a;  x1 = x0 + dt (v0 + v1)/2 (fluid only);
//   rho1 = rho0 (2 - e)/(2 + e), e = -(Drho/rho_half) dt, written as
//   drho1 = (drho0 (2 - e) - 2 rho0 e) / (2 + e).
// Then the rebuild test on x1 with a margin for the next half step:
// |x1 - x_ref| + dt |v1| > skin/2.  Clears the constraint buffer of t^n.
__global__ void k_sph_correct(int n, BoxT<float> box, float4 *__restrict__ pos, float4 *__restrict__ vr,
                              const float4 *__restrict__ vr_h, const float4 *__restrict__ acc_h,
                              const float *__restrict__ d_dt, float rho0, float *dtcons,
                              const float4 *__restrict__ ref, float half_skin, fpm_dev_status *st, double *time)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const float dt = *d_dt;
    bool over = false;
    float d2 = 0.0f;
    if (i < n) {
        float4 p = pos[i], v = vr[i];
        const float4 a = acc_h[i];
        const float4 vh = vr_h[i];
        const float rho_h = rho0 + vh.w;
        const float e = -(a.w / rho_h) * dt;
        v.w = (v.w * (2.0f - e) - 2.0f * rho0 * e) / (2.0f + e);
        if (p.w == 0.0f) {
            const float v0x = v.x, v0y = v.y, v0z = v.z;
            v.x = v0x + dt * a.x;
            v.y = v0y + dt * a.y;
            v.z = v0z + dt * a.z;
            p.x += dt * 0.5f * (v0x + v.x);
            p.y += dt * 0.5f * (v0y + v.y);
            p.z += dt * 0.5f * (v0z + v.z);
        }
        pos[i] = p;
        vr[i] = v;
        if (ref) {
            float dx, dy, dz;
            d2 = separation(p, ref[i], box, dx, dy, dz);
            const float reach = sqrtf(d2) + dt * sqrtf(v.x * v.x + v.y * v.y + v.z * v.z);
            over = reach > half_skin;
        }
    }
    if (i == 0) {
        dtcons[0] = 0.0f;
        dtcons[1] = 0.0f;
        if (time) *time += (double)dt;
    }
    if (ref) disp_report(over, d2, st);
}

static SphK make_sph(const fpm_sph_params &p)
{
    SphK K{};
    const double pi = 3.14159265358979323846;
    K.h = (float)p.h;
    K.m = (float)p.mass;
    K.rho0 = (float)p.rho0;
    K.inv_rho0 = (float)(1.0 / p.rho0);
    K.c0 = (float)p.c0;
    K.alpha = (float)p.alpha;
    K.eta2 = (float)p.eta2;
    K.gamma = (int)p.gamma;
    K.b = (float)(p.c0 * p.c0 * p.rho0 / p.gamma);
    for (int d = 0; d < 3; ++d) K.g[d] = (float)p.g[d];
    K.two_h2 = (float)(4.0 * p.h * p.h);
    K.inv_h = (float)(1.0 / p.h);
    K.kernel = p.kernel;
    if (p.kernel == 0) {
        const double a = 21.0 / (16.0 * pi * p.h * p.h * p.h);
        K.wcoef = (float)(p.mass * -5.0 * a / (p.h * p.h));
    } else {
        K.wcoef = (float)(p.mass / (pi * p.h * p.h * p.h) / (p.h * p.h));
    }
    K.visc2 = (float)(-2.0 * p.alpha * p.c0);
    K.wnorm = p.kernel == 0 ? (float)(p.mass * 21.0 / (16.0 * pi * p.h * p.h * p.h))
                            : (float)(p.mass / (pi * p.h * p.h * p.h));
    // C(gamma, k) for k = 1..gamma in binom[k-1], Horner from the highest
    double c = 1.0;
    for (int k = 1; k <= 8; ++k) {
        c = c * (double)(K.gamma - k + 1) / (double)k;
        K.binom[k - 1] = k <= K.gamma ? (float)c : 0.0f;
    }
    return K;
}

}  // namespace fpm

using namespace fpm;

static fpm_status sph_params_ok(const fpm_sph_params *p, const char *who)
{
    if (!p || !(p->h > 0.0) || !(p->mass > 0.0) || !(p->rho0 > 0.0) || !(p->c0 > 0.0) || !(p->eta2 >= 0.0))
        return fpm_fail(FPM_ERR_INVALID, "%s: bad SPH parameters", who);
    if (p->gamma != (double)(int)p->gamma || p->gamma < 1.0 || p->gamma > 8.0)
        return fpm_fail(FPM_ERR_INVALID, "%s: gamma must be an integer in [1, 8]", who);
    if (p->kernel != 0 && p->kernel != 1) return fpm_fail(FPM_ERR_INVALID, "%s: kernel must be 0 or 1", who);
    return FPM_OK;
}

extern "C" fpm_status fpm_sph_forces(const fpm_box *box, const fpm_grid *grid, int32_t n, const void *pos,
                                     const void *vr, const void *list, const uint32_t *nn, int32_t cap,
                                     const fpm_sph_params *params, void *acc, float *d_dtcons, void *workspace,
                                     size_t workspace_bytes, fpm_dev_status *d_status, fpm_stream stream)
{
    fpm_status s = fpm_check_grid(box, grid, "fpm_sph_forces");
    if (s != FPM_OK) return s;
    s = sph_params_ok(params, "fpm_sph_forces");
    if (s != FPM_OK) return s;
    if (n < 0 || cap < 1 || (n > 0 && (!pos || !vr || !list || !nn || !acc)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_sph_forces: null pointer or bad size");
    if (((uintptr_t)list & 255u) != 0) return fpm_fail(FPM_ERR_INVALID, "fpm_sph_forces: list not 256-B aligned");
    if (n == 0) return FPM_OK;
    RedWs r{};
    s = red_ws(n, grid, workspace, workspace_bytes, "fpm_sph_forces", r);
    if (s != FPM_OK) return s;
    const TileCfg cfg = make_tile_cfg(*box, *grid);
    const ListLayout L = list_layout(n, cfg, cap);
    // staged per neighbour: position, velocity + drho
    const size_t per = 2 * sizeof(float4);
    const int sc = stage_capacity(n, *grid, per);
    const size_t smem = (size_t)sc * per;
    const SphK K = make_sph(*params);
    const void *kern = K.kernel == 0 ? (const void *)k_sph_tiles<0> : (const void *)k_sph_tiles<1>;
    smem_opt_in(kern);
    const int blocks = persistent_blocks(kern, kSphThreads, smem, *grid, cfg.ntiles);
    auto launch = K.kernel == 0 ? k_sph_tiles<0> : k_sph_tiles<1>;
    launch<<<blocks, kSphThreads, smem, (cudaStream_t)stream>>>(
        cfg, make_box<float>(*box), (const float4 *)pos, (const float4 *)vr, list_view(list, L), nn, L.ld, sc,
        K, (float4 *)acc, d_dtcons, Sched{r.work, r.done}, d_status);
    return fpm_check_launch("fpm_sph_forces");
}

extern "C" fpm_status fpm_sph_density(const fpm_box *box, const fpm_grid *grid, int32_t n, const void *pos,
                                      const void *list, const uint32_t *nn, int32_t cap, const fpm_sph_params *params,
                                      float *rho, void *workspace, size_t workspace_bytes, fpm_dev_status *d_status,
                                      fpm_stream stream)
{
    fpm_status s = fpm_check_grid(box, grid, "fpm_sph_density");
    if (s != FPM_OK) return s;
    s = sph_params_ok(params, "fpm_sph_density");
    if (s != FPM_OK) return s;
    if (n < 0 || cap < 1 || (n > 0 && (!pos || !list || !nn || !rho)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_sph_density: null pointer or bad size");
    if (((uintptr_t)list & 255u) != 0) return fpm_fail(FPM_ERR_INVALID, "fpm_sph_density: list not 256-B aligned");
    if (n == 0) return FPM_OK;
    RedWs r{};
    s = red_ws(n, grid, workspace, workspace_bytes, "fpm_sph_density", r);
    if (s != FPM_OK) return s;
    const TileCfg cfg = make_tile_cfg(*box, *grid);
    const ListLayout L = list_layout(n, cfg, cap);
    const int sc = stage_capacity(n, *grid, sizeof(float4));
    const size_t smem = (size_t)sc * sizeof(float4);
    const SphK K = make_sph(*params);
    const void *kern = K.kernel == 0 ? (const void *)k_sph_density_tiles<0> : (const void *)k_sph_density_tiles<1>;
    smem_opt_in(kern);
    const int blocks = persistent_blocks(kern, kTileThreads, smem, *grid, cfg.ntiles);
    auto launch = K.kernel == 0 ? k_sph_density_tiles<0> : k_sph_density_tiles<1>;
    launch<<<blocks, kTileThreads, smem, (cudaStream_t)stream>>>(cfg, make_box<float>(*box), (const float4 *)pos,
                                                               list_view(list, L), nn, L.ld, sc, K, rho,
                                                               Sched{r.work, r.done}, d_status);
    return fpm_check_launch("fpm_sph_density");
}

extern "C" fpm_status fpm_sph_predict(const fpm_box *box, int32_t n, const fpm_sph_params *params, double cfl,
                                      const void *pos, const void *vr, const void *acc, const float *d_dtcons,
                                      void *pos_h, void *vr_h, float *d_dt, float *d_dtcons_h, const void *pos_ref,
                                      double skin, fpm_dev_status *d_status, fpm_stream stream)
{
    fpm_status s = sph_params_ok(params, "fpm_sph_predict");
    if (s != FPM_OK) return s;
    if (!box || n < 0 || !d_dtcons || !d_dt || !d_dtcons_h || (pos_ref && !d_status) ||
        (n > 0 && (!pos || !vr || !acc || !pos_h || !vr_h)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_sph_predict: null pointer or bad size");
    const int blocks = n > 0 ? (n + 255) / 256 : 1;
    k_sph_predict<<<blocks, 256, 0, (cudaStream_t)stream>>>(
        n, make_box<float>(*box), (const float4 *)pos, (const float4 *)vr, (const float4 *)acc, d_dtcons,
        (float)params->h, (float)params->c0, (float)cfl, (float4 *)pos_h, (float4 *)vr_h, d_dt, d_dtcons_h,
        (const float4 *)pos_ref, (float)(0.25 * skin * skin), d_status);
    return fpm_check_launch("fpm_sph_predict");
}

extern "C" fpm_status fpm_sph_correct(const fpm_box *box, int32_t n, const fpm_sph_params *params, void *pos,
                                      void *vr, const void *vr_h, const void *acc_h, const float *d_dt,
                                      float *d_dtcons, const void *pos_ref, double skin, fpm_dev_status *d_status,
                                      double *d_time, fpm_stream stream)
{
    fpm_status s = sph_params_ok(params, "fpm_sph_correct");
    if (s != FPM_OK) return s;
    if (!box || n < 0 || !d_dt || !d_dtcons || (pos_ref && !d_status) ||
        (n > 0 && (!pos || !vr || !vr_h || !acc_h)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_sph_correct: null pointer or bad size");
    const int blocks = n > 0 ? (n + 255) / 256 : 1;
    k_sph_correct<<<blocks, 256, 0, (cudaStream_t)stream>>>(
        n, make_box<float>(*box), (float4 *)pos, (float4 *)vr, (const float4 *)vr_h, (const float4 *)acc_h, d_dt,
        (float)params->rho0, d_dtcons, (const float4 *)pos_ref, (float)(0.5 * skin), d_status, d_time);
    return fpm_check_launch("fpm_sph_correct");
}
