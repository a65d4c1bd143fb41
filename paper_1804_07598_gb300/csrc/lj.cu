// lj.cu -- Lennard-Jones pair sweep over the Verlet list (Sec. 4.1: the LJ
// potential V(r) = 4 eps [(s/r)^12 - (s/r)^6] and the pair force
// 24 eps (2 s^12/r^14 - s^6/r^8)(x_p - x_q) of Listing 4.1, truncated at
// r_cut), the two halves of velocity Verlet (Listing 4.1 time loop) and the
// FP64 kinetic-energy / momentum reduction.
//
// The force sweep walks the FULL list (every pair twice, once from each
// side): no atomics, so forces are bit-reproducible run to run and the sum
// of forces is the only place Newton's third law is checked.
#include "fpm_common.cuh"

namespace fpm {

__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return __drcp_rn(x); }

template <typename T>
__global__ void __launch_bounds__(256) k_lj_forces(BoxT<T> box, int n, const V4<T> *__restrict__ pos,
                                                   const uint32_t *__restrict__ nbr, const uint32_t *__restrict__ nn,
                                                   int64_t ld, T eps24, T eps4, T sig2, T rc2,
                                                   V4<T> *__restrict__ force, double *part, unsigned *counter,
                                                   double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    T fx = 0, fy = 0, fz = 0, u = 0, w = 0;
    uint32_t np = 0;
    if (i < n) {
        const V4<T> pi = pos[i];
        const uint32_t m = nn[i];
        const uint32_t *col = nbr + i;
        for (uint32_t k = 0; k < m; ++k) {
            const uint32_t j = __ldcs(col + (int64_t)k * ld);
            const V4<T> pj = ldg4(pos + j);
            T dx, dy, dz;
            const T r2 = separation(pi, pj, box, dx, dy, dz);
            if (r2 < rc2) {
                const T ir2 = recip(r2);
                const T s2 = sig2 * ir2;
                const T s6 = s2 * s2 * s2;
                const T fr = eps24 * ir2 * s6 * ((T)2 * s6 - (T)1);
                fx += fr * dx;
                fy += fr * dy;
                fz += fr * dz;
                u += eps4 * s6 * (s6 - (T)1);
                w += fr * r2;
                ++np;
            }
        }
        V4<T> f;
        f.x = fx;
        f.y = fy;
        f.z = fz;
        f.w = (T)0.5 * u;
        force[i] = f;
    }
    if (out) {
        double v[3] = {0.5 * (double)u, 0.5 * (double)w, 0.5 * (double)np};
        grid_reduce<3>(v, part, counter, out);
    }
}

template <typename T>
__global__ void k_vv_kick_drift(BoxT<T> box, int n, T hdt, T dt, V4<T> *__restrict__ pos, V4<T> *__restrict__ vel,
                                const V4<T> *__restrict__ force)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    V4<T> x = pos[i], v = vel[i];
    const V4<T> f = force[i];
    v.x += hdt * f.x;
    v.y += hdt * f.y;
    v.z += hdt * f.z;
    x.x += dt * v.x;
    x.y += dt * v.y;
    x.z += dt * v.z;
    if (box.per[0]) x.x = wrap1(x.x, box.L[0]);
    if (box.per[1]) x.y = wrap1(x.y, box.L[1]);
    if (box.per[2]) x.z = wrap1(x.z, box.L[2]);
    pos[i] = x;
    vel[i] = v;
}

template <typename T>
__global__ void k_vv_kick(int n, T hdt, V4<T> *__restrict__ vel, const V4<T> *__restrict__ force)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    V4<T> v = vel[i];
    const V4<T> f = force[i];
    v.x += hdt * f.x;
    v.y += hdt * f.y;
    v.z += hdt * f.z;
    vel[i] = v;
}

template <typename T>
__global__ void __launch_bounds__(256) k_kinetic(int n, const V4<T> *__restrict__ vel, double *part,
                                                 unsigned *counter, double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (i < n) {
        const V4<T> u = vel[i];
        const double x = u.x, y = u.y, z = u.z;
        v[0] = 0.5 * (x * x + y * y + z * z);
        v[1] = x;
        v[2] = y;
        v[3] = z;
    }
    grid_reduce<4>(v, part, counter, out);
}

// Reduction workspace: counter at offset 0, partials from byte 256.
struct RedWs {
    unsigned *counter;
    double *part;
};

static fpm_status red_ws(int n, void *ws, size_t bytes, const char *who, RedWs &r)
{
    size_t need = 0;
    fpm_reduce_workspace(n, &need);
    if (!ws || bytes < need) return fpm_fail(FPM_ERR_WORKSPACE, "%s: workspace %zu < %zu bytes", who, bytes, need);
    if (((uintptr_t)ws & 15u) != 0) return fpm_fail(FPM_ERR_WORKSPACE, "%s: workspace not 16-B aligned", who);
    r.counter = (unsigned *)ws;
    r.part = (double *)((char *)ws + 256);
    return FPM_OK;
}

template <typename T>
static fpm_status lj_launch(const fpm_box &b, int n, const void *pos, const uint32_t *nbr, const uint32_t *nn,
                            double eps, double sigma, double rc, void *force, double *d_energy, const RedWs &r,
                            cudaStream_t stream)
{
    const BoxT<T> box = make_box<T>(b);
    const T rc2 = (T)(rc * rc);
    const T sig2 = (T)(sigma * sigma);
    const int blocks = n > 0 ? (n + 255) / 256 : 1;
    k_lj_forces<T><<<blocks, 256, 0, stream>>>(box, n, (const V4<T> *)pos, nbr, nn, fpm_nbr_ld(n), (T)(24.0 * eps),
                                               (T)(4.0 * eps), sig2, rc2, (V4<T> *)force, r.part, r.counter,
                                               d_energy);
    return fpm_check_launch("fpm_lj_forces");
}

}  // namespace fpm

using namespace fpm;

extern "C" fpm_status fpm_lj_forces(const fpm_box *box, int32_t n, fpm_prec prec, const void *pos,
                                    const uint32_t *nbr, const uint32_t *nn, int32_t cap, double eps, double sigma,
                                    double rc, void *force, double *d_energy, void *workspace,
                                    size_t workspace_bytes, fpm_stream stream)
{
    if (!box || n < 0 || cap < 1 || !(rc > 0.0) || !(sigma > 0.0) || (n > 0 && (!pos || !nbr || !nn || !force)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_lj_forces: null pointer or bad size");
    if (prec != FPM_F32 && prec != FPM_F64) return fpm_fail(FPM_ERR_INVALID, "fpm_lj_forces: bad precision");
    if (n == 0 && !d_energy) return FPM_OK;
    RedWs r{nullptr, nullptr};
    if (d_energy) {
        fpm_status s = red_ws(n, workspace, workspace_bytes, "fpm_lj_forces", r);
        if (s != FPM_OK) return s;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == FPM_F32) return lj_launch<float>(*box, n, pos, nbr, nn, eps, sigma, rc, force, d_energy, r, st);
    return lj_launch<double>(*box, n, pos, nbr, nn, eps, sigma, rc, force, d_energy, r, st);
}

extern "C" fpm_status fpm_vv_step(const fpm_box *box, int32_t n, fpm_prec prec, int32_t half, double dt, void *pos,
                                  void *vel, const void *force, fpm_stream stream)
{
    if (!box || n < 0 || (half != 0 && half != 1) || (n > 0 && (!vel || !force || (half == 0 && !pos))))
        return fpm_fail(FPM_ERR_INVALID, "fpm_vv_step: null pointer or bad argument");
    if (prec != FPM_F32 && prec != FPM_F64) return fpm_fail(FPM_ERR_INVALID, "fpm_vv_step: bad precision");
    if (n == 0) return FPM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (prec == FPM_F32) {
        const BoxT<float> b = make_box<float>(*box);
        if (half == 0)
            k_vv_kick_drift<float><<<blocks, 256, 0, st>>>(b, n, (float)(0.5 * dt), (float)dt, (float4 *)pos,
                                                           (float4 *)vel, (const float4 *)force);
        else
            k_vv_kick<float><<<blocks, 256, 0, st>>>(n, (float)(0.5 * dt), (float4 *)vel, (const float4 *)force);
    } else {
        const BoxT<double> b = make_box<double>(*box);
        if (half == 0)
            k_vv_kick_drift<double><<<blocks, 256, 0, st>>>(b, n, 0.5 * dt, dt, (double4_32a *)pos,
                                                            (double4_32a *)vel, (const double4_32a *)force);
        else
            k_vv_kick<double><<<blocks, 256, 0, st>>>(n, 0.5 * dt, (double4_32a *)vel, (const double4_32a *)force);
    }
    return fpm_check_launch("fpm_vv_step");
}

extern "C" fpm_status fpm_kinetic(int32_t n, fpm_prec prec, const void *vel, double *d_out, void *workspace,
                                  size_t workspace_bytes, fpm_stream stream)
{
    if (n < 0 || !d_out || (n > 0 && !vel)) return fpm_fail(FPM_ERR_INVALID, "fpm_kinetic: bad argument");
    if (prec != FPM_F32 && prec != FPM_F64) return fpm_fail(FPM_ERR_INVALID, "fpm_kinetic: bad precision");
    RedWs r;
    fpm_status s = red_ws(n, workspace, workspace_bytes, "fpm_kinetic", r);
    if (s != FPM_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = n > 0 ? (n + 255) / 256 : 1;
    if (prec == FPM_F32)
        k_kinetic<float><<<blocks, 256, 0, st>>>(n, (const float4 *)vel, r.part, r.counter, d_out);
    else
        k_kinetic<double><<<blocks, 256, 0, st>>>(n, (const double4_32a *)vel, r.part, r.counter, d_out);
    return fpm_check_launch("fpm_kinetic");
}

// ---------------------------------------------------------------------------
// fpm_lj_forces_noalloc: the same force sweep and energy reduction for callers
// that cannot allocate device memory (no cudaMalloc, no caching allocator).
// Its scratch (the per-block partial sums and the completion counter) is a
// file-scope device array, present on every GPU that loads this library.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr int kNoAllocMaxN = 1 << 24;  // particles per call
constexpr size_t kNoAllocBytes = 256 + (size_t)((kNoAllocMaxN + 255) / 256) * 8 * sizeof(double);  // 4 MiB + 256 B

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

extern "C" fpm_status fpm_lj_forces_noalloc(const fpm_box *box, int32_t n, fpm_prec prec, const void *pos,
                                            const uint32_t *nbr, const uint32_t *nn, int32_t cap, double eps,
                                            double sigma, double rc, void *force, double *d_energy,
                                            fpm_stream stream)
{
    if (n > kNoAllocMaxN)
        return fpm_fail(FPM_ERR_INVALID, "fpm_lj_forces_noalloc: n=%d exceeds the built-in scratch limit of %d particles",
                        n, kNoAllocMaxN);
    if (!box || n < 0 || cap < 1 || !(rc > 0.0) || !(sigma > 0.0) || (n > 0 && (!pos || !nbr || !nn || !force)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_lj_forces_noalloc: null pointer or bad size");
    if (prec != FPM_F32 && prec != FPM_F64) return fpm_fail(FPM_ERR_INVALID, "fpm_lj_forces_noalloc: bad precision");
    if (n == 0 && !d_energy) return FPM_OK;
    RedWs r{nullptr, nullptr};
    cudaStream_t st = (cudaStream_t)stream;
    if (d_energy) {
        void *scratch = nullptr;
        fpm_status s = scratch_for_current_device(&scratch);
        if (s != FPM_OK) return s;
        // the completion counter must start at zero; the array keeps whatever
        // the previous call left there
        cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned), st);
        if (e != cudaSuccess)
            return fpm_fail(FPM_ERR_CUDA, "fpm_lj_forces_noalloc: clearing the counter: %s", cudaGetErrorString(e));
        r.counter = (unsigned *)scratch;
        r.part = (double *)((char *)scratch + 256);
    }
    if (prec == FPM_F32) return lj_launch<float>(*box, n, pos, nbr, nn, eps, sigma, rc, force, d_energy, r, st);
    return lj_launch<double>(*box, n, pos, nbr, nn, eps, sigma, rc, force, d_energy, r, st);
}
