// adjoint.cu -- hand-written adjoint of the LJ force sweep and of velocity
// Verlet (the differentiable workload; the paper has no adjoint: this is the
// chain rule applied to the LJ force of Sec. 4.1 and the integrator of
// Listing 4.1).
//
// With s = r^2, s6 = (sigma^2/s)^3 and the pair force factor
//   phi = 24 eps (2 s6^2 - s6) / s            (F_i = sum_j phi (x_i - x_j)),
// the Jacobian J = dF/dx is symmetric and
//   (J a)_i = sum_j [ phi (a_i - a_j) + 2 phi'(s) ((x_i - x_j).(a_i - a_j)) (x_i - x_j) ],
//   2 phi'(s) = 48 eps (4 s6 - 14 s6^2) / s^2,
//   dphi/dsigma = 24 eps (24 s6^2 - 6 s6) / (sigma s),
//   dU/deps = sum_pairs 4 (s6^2 - s6),  dU/dsigma = sum_pairs 24 eps (2 s6^2 - s6) / sigma.
// The sweep runs over the same tiled Verlet list as the force: the tile's
// positions and the vector a are staged together in shared memory.
#include "reduce.cuh"
#include "tiles.cuh"

namespace fpm {

__device__ __forceinline__ float arecip(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    const float e = __fmaf_rn(-x, y, 1.0f);
    return __fmaf_rn(y, e, y);
}
__device__ __forceinline__ double arecip(double x) { return __drcp_rn(x); }

template <typename T> struct HvpParams {
    T sig2, rc2;
};

// Per-particle accumulators of the backward sweep (in units that the caller
// scales once: 24 eps for forces and the HVP, 24 eps / sigma for sigma terms).
template <typename T> struct HvpAcc {
    T hx, hy, hz;     // sum [g da + 2 q (r.da) r]
    T fx, fy, fz;     // sum g r           (force / (24 eps))
    T sx, sy, sz;     // sum gs r          (dF/dsigma / (24 eps / sigma))
    T ue, us;         // sum (s12 - s6), sum (2 s12 - s6)
};

template <typename T, bool FAST, bool SMEM>
__device__ __forceinline__ void hvp_pair(const TileCfg &cfg, const BoxT<T> &box, const TileDesc &d,
                                         const V4<T> *__restrict__ pos, const V4<T> *__restrict__ avec,
                                         const V4<T> *__restrict__ st, const V4<T> *__restrict__ sa,
                                         const V4<T> &pi, const V4<T> &ai, int s, const HvpParams<T> &P,
                                         HvpAcc<T> &A)
{
    V4<T> pj, aj;
    if (SMEM) {
        pj = st[s];
        aj = sa[s];
    } else {
        pj = staged_global(d, box, pos, s);
        aj = ldg4(avec + staged_index(d, s));
    }
    T dx, dy, dz;
    const T r2 = tile_sep<FAST>(pi, pj, box, cfg, dx, dy, dz);
    const bool in = r2 < P.rc2;
    const T ir2 = arecip(r2);
    const T s2 = P.sig2 * ir2;
    const T s6 = s2 * s2 * s2;
    const T s12 = s6 * s6;
    const T g = in ? ir2 * ((T)2 * s12 - s6) : (T)0;
    const T q = in ? (T)2 * ir2 * ir2 * ((T)4 * s6 - (T)14 * s12) : (T)0;
    const T gs = in ? ir2 * ((T)24 * s12 - (T)6 * s6) : (T)0;
    const T ax = ai.x - aj.x, ay = ai.y - aj.y, az = ai.z - aj.z;
    const T rda = dx * ax + dy * ay + dz * az;
    const T c = q * rda;
    A.hx += g * ax + c * dx;
    A.hy += g * ay + c * dy;
    A.hz += g * az + c * dz;
    A.fx += g * dx;
    A.fy += g * dy;
    A.fz += g * dz;
    A.sx += gs * dx;
    A.sy += gs * dy;
    A.sz += gs * dz;
    A.ue += in ? s12 - s6 : (T)0;
    A.us += in ? (T)2 * s12 - s6 : (T)0;
}

template <typename T, bool FAST, bool SMEM>
__device__ __forceinline__ void hvp_sweep(const TileCfg &cfg, const BoxT<T> &box, const TileDesc &d,
                                          const V4<T> *__restrict__ pos, const V4<T> *__restrict__ avec,
                                          const V4<T> *__restrict__ st, const V4<T> *__restrict__ sa,
                                          const V4<T> &pi, const V4<T> &ai, uint32_t m,
                                          const uint32_t *__restrict__ col, int64_t ld, const HvpParams<T> &P,
                                          HvpAcc<T> &A)
{
    for_each_entry<4>(m, col, ld,
                      [&](int s) { hvp_pair<T, FAST, SMEM>(cfg, box, d, pos, avec, st, sa, pi, ai, s, P, A); });
}

// The sweep of a tile whose neighbourhood did not fit in shared memory (rare;
// out of line so that it does not add to the registers of the common path).
template <typename T>
__device__ __noinline__ void hvp_sweep_spilled(const TileCfg &cfg, const BoxT<T> &box, const TileDesc &d,
                                               const V4<T> *__restrict__ pos, const V4<T> *__restrict__ avec,
                                               const V4<T> &pi, const V4<T> &ai, uint32_t m,
                                               const uint32_t *__restrict__ col, int64_t ld, const HvpParams<T> &P,
                                               HvpAcc<T> *A)
{
    HvpAcc<T> a{};
    hvp_sweep<T, false, false>(cfg, box, d, pos, avec, nullptr, nullptr, pi, ai, m, col, ld, P, a);
    *A = a;
}

template <typename T>
__global__ void __launch_bounds__(kTileThreads, 3)
    k_lj_hvp_tiles(TileCfg cfg, BoxT<T> box, const V4<T> *__restrict__ pos, const V4<T> *__restrict__ avec,
                   ListView lv, const uint32_t *__restrict__ nn, int64_t ld, int stage_cap, HvpParams<T> P,
                   double hscale, double e24, double e24s, double eps4, double *__restrict__ adj_pos, Sched sched,
                   double *part, double *out, fpm_dev_status *status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    V4<T> *sp = (V4<T> *)smem_raw;
    V4<T> *sa = sp + stage_cap;
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
    T de = 0, ds = 0, ue = 0, us = 0;
    load_desc(lv.descs + lv.active[k], d);
    const bool in_smem = d.M <= stage_cap;
    if (!in_smem) note_spill(status);
    const bool staged = in_smem ? stage_positions(d, box, pos, sp, &bar, phase, status, avec, sa) : true;
    for (uint32_t i = d.h0 + threadIdx.x; staged && i < d.h1; i += blockDim.x) {
        const V4<T> pi = pos[i];
        const V4<T> ai = avec[i];
        const uint32_t m = nn[i];
        HvpAcc<T> A{};
        if (in_smem) {
            if (d.slow) hvp_sweep<T, false, true>(cfg, box, d, pos, avec, sp, sa, pi, ai, m, words + i, ld, P, A);
            else hvp_sweep<T, true, true>(cfg, box, d, pos, avec, sp, sa, pi, ai, m, words + i, ld, P, A);
        } else {
            hvp_sweep_spilled<T>(cfg, box, d, pos, avec, pi, ai, m, words + i, ld, P, &A);
        }
        // adj_pos += hscale * 24 eps * sum[...]  (FP64 accumulation of the adjoint state)
        double *o = adj_pos + 4 * (size_t)i;
        const double k = hscale * e24;
        o[0] += k * (double)A.hx;
        o[1] += k * (double)A.hy;
        o[2] += k * (double)A.hz;
        de += ai.x * A.fx + ai.y * A.fy + ai.z * A.fz;
        ds += ai.x * A.sx + ai.y * A.sy + ai.z * A.sz;
        ue += A.ue;
        us += A.us;
    }
    if (out) {
        const T v[4] = {de, ds, ue, us};
        block_sum_store<4>(v, part + (size_t)k * 4);
    }
    }
    if (sched_finish(sched, &s_last) && out) {
        // a.dF/deps = 24 sum a.(g r); a.dF/dsigma = (24 eps/sigma) sum a.(gs r);
        // dU/deps = 4 * 1/2 sum (s12 - s6); dU/dsigma = (24 eps/sigma) * 1/2 sum (2 s12 - s6)
        const double scale4[4] = {hscale * 24.0, hscale * e24s, 0.5 * 4.0, 0.5 * e24s};
        __threadfence();
        sum_tile_partials<4>(part, ntodo, out, true, scale4);
    }
    (void)eps4;
}

// One reverse velocity-Verlet update of the FP64 adjoint state, with the
// reorder of a cell-list rebuild undone first when perm is given:
//   j = perm[k] (or k);  xo[j] = xi[k];  vo[j] = vi[k] + dt xi[k];
//   a[j] = (T)(c vo[j])  (the vector for the next backward sweep).
template <typename T>
__global__ void k_vv_adjoint(int n, const uint32_t *__restrict__ perm, const uint32_t *__restrict__ gate, double dt,
                             double c, const double4_32a *__restrict__ xi, const double4_32a *__restrict__ vi,
                             double4_32a *__restrict__ xo, double4_32a *__restrict__ vo, V4<T> *__restrict__ a)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const bool use = perm != nullptr && (gate == nullptr || *gate != 0u);
    const int j = use ? (int)perm[k] : k;
    const double4_32a x = xi[k];
    double4_32a v = vi[k];
    v.x += dt * x.x;
    v.y += dt * x.y;
    v.z += dt * x.z;
    v.w = 0.0;
    xo[j] = x;
    vo[j] = v;
    V4<T> av;
    av.x = (T)(c * v.x);
    av.y = (T)(c * v.y);
    av.z = (T)(c * v.z);
    av.w = (T)0;
    a[j] = av;
}

// Seed of the loss U(x_T) + sum |F_i(x_T)|^2: xbar = -F, vbar = 0, a = F.
template <typename T>
__global__ void k_adjoint_seed(int n, const V4<T> *__restrict__ force, double4_32a *__restrict__ xbar,
                               double4_32a *__restrict__ vbar, V4<T> *__restrict__ a)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const V4<T> f = force[k];
    double4_32a x;
    x.x = -(double)f.x;
    x.y = -(double)f.y;
    x.z = -(double)f.z;
    x.w = 0.0;
    xbar[k] = x;
    double4_32a z;
    z.x = z.y = z.z = z.w = 0.0;
    vbar[k] = z;
    V4<T> av = f;
    av.w = (T)0;
    a[k] = av;
}

// L = U + 2 (1/2 sum |F|^2), one thread.
__global__ void k_adjoint_loss(const double *__restrict__ energy, const double *__restrict__ half_sumf2,
                               double *__restrict__ loss)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) loss[0] = energy[0] + 2.0 * half_sumf2[0];
}

// Rows of the adjoint state back to the caller's particle order, and the
// parameter gradient assembled from its partial sums (thread 0 of block 0).
__global__ void k_adjoint_finish(int n, const uint32_t *__restrict__ ids, const double4_32a *__restrict__ xbar,
                                 const double4_32a *__restrict__ vbar, const double *__restrict__ th_seed,
                                 const double *__restrict__ th_steps, double *__restrict__ gx,
                                 double *__restrict__ gv, double *__restrict__ gtheta)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) {
        gtheta[0] = th_seed[0] + th_seed[2] + th_steps[0];
        gtheta[1] = th_seed[1] + th_seed[3] + th_steps[1];
    }
    if (k >= n) return;
    const size_t o = 3 * (size_t)ids[k];
    const double4_32a x = xbar[k], v = vbar[k];
    gx[o] = x.x;
    gx[o + 1] = x.y;
    gx[o + 2] = x.z;
    gv[o] = v.x;
    gv[o + 1] = v.y;
    gv[o + 2] = v.z;
}

template <typename T>
static fpm_status hvp_launch(const fpm_box &b, const fpm_grid &g, int n, const void *pos, const void *list,
                             const uint32_t *nn, int cap, double eps, double sigma, double rc, const void *a,
                             double scale, double *adj_pos, double *d_params, const RedWs &r, fpm_dev_status *st,
                             cudaStream_t stream)
{
    const TileCfg cfg = make_tile_cfg(b, g);
    const ListLayout L = list_layout(n, cfg, cap);
    const BoxT<T> box = make_box<T>(b);
    HvpParams<T> P;
    P.sig2 = (T)(sigma * sigma);
    P.rc2 = (T)(rc * rc);
    // two staged arrays share the shared-memory budget
    int sc = stage_capacity(n, g, 2 * sizeof(V4<T>));
    const size_t smem = 2 * (size_t)sc * sizeof(V4<T>);
    smem_opt_in((const void *)k_lj_hvp_tiles<T>);
    const int blocks = persistent_blocks((const void *)k_lj_hvp_tiles<T>, kTileThreads, smem, g, cfg.ntiles);
    k_lj_hvp_tiles<T><<<blocks, kTileThreads, smem, stream>>>(cfg, box, (const V4<T> *)pos, (const V4<T> *)a,
                                                              list_view(list, L), nn, L.ld, sc, P, scale, 24.0 * eps,
                                                              24.0 * eps / sigma, 4.0 * eps, adj_pos,
                                                              Sched{r.work, r.done}, r.part, d_params, st);
    return fpm_check_launch("fpm_lj_backward");
}

}  // namespace fpm

using namespace fpm;

extern "C" fpm_status fpm_lj_backward(const fpm_box *box, const fpm_grid *grid, int32_t n, fpm_prec prec,
                                      const void *pos, const void *list, const uint32_t *nn, int32_t cap, double eps,
                                      double sigma, double rc, const void *a, double scale, double *adj_pos,
                                      double *d_params, void *workspace, size_t workspace_bytes,
                                      fpm_dev_status *d_status, fpm_stream stream)
{
    fpm_status s = fpm_check_grid(box, grid, "fpm_lj_backward");
    if (s != FPM_OK) return s;
    if (n < 0 || cap < 1 || !(rc > 0.0) || !(sigma > 0.0) || !(eps != 0.0) ||
        (n > 0 && (!pos || !list || !nn || !a || !adj_pos)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_lj_backward: null pointer or bad size");
    if (prec != FPM_F32 && prec != FPM_F64) return fpm_fail(FPM_ERR_INVALID, "fpm_lj_backward: bad precision");
    if (((uintptr_t)list & 255u) != 0 || ((uintptr_t)adj_pos & 31u) != 0)
        return fpm_fail(FPM_ERR_INVALID, "fpm_lj_backward: list must be 256-B and adj_pos 32-B aligned");
    if (n == 0) return FPM_OK;
    RedWs r{};
    s = red_ws(n, grid, workspace, workspace_bytes, "fpm_lj_backward", r);
    if (s != FPM_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == FPM_F32)
        return hvp_launch<float>(*box, *grid, n, pos, list, nn, cap, eps, sigma, rc, a, scale, adj_pos, d_params, r,
                                 d_status, st);
    return hvp_launch<double>(*box, *grid, n, pos, list, nn, cap, eps, sigma, rc, a, scale, adj_pos, d_params, r,
                              d_status, st);
}

extern "C" fpm_status fpm_vv_adjoint(int32_t n, fpm_prec prec, const uint32_t *perm, const uint32_t *d_gate,
                                     double dt, double c, const double *xbar_in, const double *vbar_in,
                                     double *xbar_out, double *vbar_out, void *a_out, fpm_stream stream)
{
    if (n < 0 || (n > 0 && (!xbar_in || !vbar_in || !xbar_out || !vbar_out || !a_out)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_vv_adjoint: null pointer or bad size");
    if (perm && (xbar_in == xbar_out || vbar_in == vbar_out))
        return fpm_fail(FPM_ERR_INVALID, "fpm_vv_adjoint: with perm, inputs and outputs must not alias");
    if (prec != FPM_F32 && prec != FPM_F64) return fpm_fail(FPM_ERR_INVALID, "fpm_vv_adjoint: bad precision");
    if (n == 0) return FPM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (prec == FPM_F32)
        k_vv_adjoint<float><<<blocks, 256, 0, st>>>(n, perm, d_gate, dt, c, (const double4_32a *)xbar_in,
                                                    (const double4_32a *)vbar_in, (double4_32a *)xbar_out,
                                                    (double4_32a *)vbar_out, (float4 *)a_out);
    else
        k_vv_adjoint<double><<<blocks, 256, 0, st>>>(n, perm, d_gate, dt, c, (const double4_32a *)xbar_in,
                                                     (const double4_32a *)vbar_in, (double4_32a *)xbar_out,
                                                     (double4_32a *)vbar_out, (double4_32a *)a_out);
    return fpm_check_launch("fpm_vv_adjoint");
}

extern "C" fpm_status fpm_adjoint_seed(int32_t n, fpm_prec prec, const void *force, double *xbar, double *vbar,
                                       void *a_out, fpm_stream stream)
{
    if (n < 0 || (n > 0 && (!force || !xbar || !vbar || !a_out)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_adjoint_seed: null pointer or bad size");
    if (prec != FPM_F32 && prec != FPM_F64) return fpm_fail(FPM_ERR_INVALID, "fpm_adjoint_seed: bad precision");
    if (n == 0) return FPM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (prec == FPM_F32)
        k_adjoint_seed<float><<<blocks, 256, 0, st>>>(n, (const float4 *)force, (double4_32a *)xbar,
                                                      (double4_32a *)vbar, (float4 *)a_out);
    else
        k_adjoint_seed<double><<<blocks, 256, 0, st>>>(n, (const double4_32a *)force, (double4_32a *)xbar,
                                                       (double4_32a *)vbar, (double4_32a *)a_out);
    return fpm_check_launch("fpm_adjoint_seed");
}

extern "C" fpm_status fpm_adjoint_loss(const double *d_energy, const double *d_half_sumf2, double *d_loss,
                                       fpm_stream stream)
{
    if (!d_energy || !d_half_sumf2 || !d_loss) return fpm_fail(FPM_ERR_INVALID, "fpm_adjoint_loss: null pointer");
    k_adjoint_loss<<<1, 32, 0, (cudaStream_t)stream>>>(d_energy, d_half_sumf2, d_loss);
    return fpm_check_launch("fpm_adjoint_loss");
}

extern "C" fpm_status fpm_adjoint_finish(int32_t n, const uint32_t *ids, const double *xbar, const double *vbar,
                                         const double *d_theta_seed, const double *d_theta_steps, double *grad_x,
                                         double *grad_v, double *d_grad_theta, fpm_stream stream)
{
    if (n < 0 || !d_theta_seed || !d_theta_steps || !d_grad_theta ||
        (n > 0 && (!ids || !xbar || !vbar || !grad_x || !grad_v)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_adjoint_finish: null pointer or bad size");
    if (grad_x == grad_v) return fpm_fail(FPM_ERR_INVALID, "fpm_adjoint_finish: grad_x aliases grad_v");
    const unsigned blocks = (unsigned)((n + 255) / 256 > 0 ? (n + 255) / 256 : 1);
    k_adjoint_finish<<<blocks, 256, 0, (cudaStream_t)stream>>>(n, ids, (const double4_32a *)xbar,
                                                             (const double4_32a *)vbar, d_theta_seed, d_theta_steps,
                                                             grad_x, grad_v, d_grad_theta);
    return fpm_check_launch("fpm_adjoint_finish");
}
