// integrate.cu -- the two halves of velocity Verlet (the time loop of
// Listing 4.1, Sec. 4.1: v += dt/2 F; x += dt v; ...; v += dt/2 F; unit mass)
// and the FP64 kinetic-energy / momentum reduction.
#include "reduce.cuh"

namespace fpm {

// v += dt/2 F; x += dt v.  No wrap: a Verlet list fixes the image of each
// pair until the next build, which wraps.
template <typename T>
__global__ void k_vv_kick_drift(int n, T hdt, T dt, V4<T> *__restrict__ pos, V4<T> *__restrict__ vel,
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
    pos[i] = x;
    vel[i] = v;
}

// The same step fused with the Verlet rebuild test on the new positions
// (fpm_verlet_check), saving a second pass over positions.
template <typename T>
__global__ void k_vv_drift_check(BoxT<T> box, int n, T hdt, T dt, V4<T> *__restrict__ pos, V4<T> *__restrict__ vel,
                                 const V4<T> *__restrict__ force, const V4<T> *__restrict__ ref, T th,
                                 fpm_dev_status *st)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool over = false;
    float d2f = 0.0f;
    if (i < n) {
        V4<T> x = pos[i], v = vel[i];
        const V4<T> f = force[i];
        v.x += hdt * f.x;
        v.y += hdt * f.y;
        v.z += hdt * f.z;
        x.x += dt * v.x;
        x.y += dt * v.y;
        x.z += dt * v.z;
        pos[i] = x;
        vel[i] = v;
        T dx, dy, dz;
        const T d2 = separation(x, ref[i], box, dx, dy, dz);
        over = d2 > th;
        d2f = (float)d2;
    }
    disp_report(over, d2f, st);
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

}  // namespace fpm

using namespace fpm;

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
        if (half == 0)
            k_vv_kick_drift<float><<<blocks, 256, 0, st>>>(n, (float)(0.5 * dt), (float)dt, (float4 *)pos,
                                                           (float4 *)vel, (const float4 *)force);
        else
            k_vv_kick<float><<<blocks, 256, 0, st>>>(n, (float)(0.5 * dt), (float4 *)vel, (const float4 *)force);
    } else {
        if (half == 0)
            k_vv_kick_drift<double><<<blocks, 256, 0, st>>>(n, 0.5 * dt, dt, (double4_32a *)pos, (double4_32a *)vel,
                                                            (const double4_32a *)force);
        else
            k_vv_kick<double><<<blocks, 256, 0, st>>>(n, 0.5 * dt, (double4_32a *)vel, (const double4_32a *)force);
    }
    return fpm_check_launch("fpm_vv_step");
}

extern "C" fpm_status fpm_vv_drift_check(const fpm_box *box, int32_t n, fpm_prec prec, double dt, void *pos,
                                         void *vel, const void *force, const void *pos_ref, double skin,
                                         fpm_dev_status *d_status, fpm_stream stream)
{
    if (!box || n < 0 || !d_status || !(skin >= 0.0) || (n > 0 && (!pos || !vel || !force || !pos_ref)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_vv_drift_check: null pointer or bad argument");
    if (prec != FPM_F32 && prec != FPM_F64) return fpm_fail(FPM_ERR_INVALID, "fpm_vv_drift_check: bad precision");
    if (n == 0) return FPM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (prec == FPM_F32)
        k_vv_drift_check<float><<<blocks, 256, 0, st>>>(make_box<float>(*box), n, (float)(0.5 * dt), (float)dt,
                                                        (float4 *)pos, (float4 *)vel, (const float4 *)force,
                                                        (const float4 *)pos_ref, (float)(0.25 * skin * skin),
                                                        d_status);
    else
        k_vv_drift_check<double><<<blocks, 256, 0, st>>>(make_box<double>(*box), n, 0.5 * dt, dt, (double4_32a *)pos,
                                                         (double4_32a *)vel, (const double4_32a *)force,
                                                         (const double4_32a *)pos_ref, 0.25 * skin * skin, d_status);
    return fpm_check_launch("fpm_vv_drift_check");
}

extern "C" fpm_status fpm_kinetic(int32_t n, fpm_prec prec, const void *vel, double *d_out, void *workspace,
                                  size_t workspace_bytes, fpm_stream stream)
{
    if (n < 0 || !d_out || (n > 0 && !vel)) return fpm_fail(FPM_ERR_INVALID, "fpm_kinetic: bad argument");
    if (prec != FPM_F32 && prec != FPM_F64) return fpm_fail(FPM_ERR_INVALID, "fpm_kinetic: bad precision");
    RedWs r;
    fpm_status s = red_ws(n, nullptr, workspace, workspace_bytes, "fpm_kinetic", r);
    if (s != FPM_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = n > 0 ? (n + 255) / 256 : 1;
    if (prec == FPM_F32)
        k_kinetic<float><<<blocks, 256, 0, st>>>(n, (const float4 *)vel, r.part, r.counter, d_out);
    else
        k_kinetic<double><<<blocks, 256, 0, st>>>(n, (const double4_32a *)vel, r.part, r.counter, d_out);
    return fpm_check_launch("fpm_kinetic");
}

// ---- host-layout transfers: packed (x, y, z) <-> the 4-vector state ---------

namespace fpm {

template <typename T>
__global__ void k_unpack_xyz(int n, const T *__restrict__ src, V4<T> *__restrict__ dst)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    V4<T> v = dst[i];
    v.x = src[3 * (size_t)i];
    v.y = src[3 * (size_t)i + 1];
    v.z = src[3 * (size_t)i + 2];
    dst[i] = v;
}

template <typename T>
__global__ void k_pack_xyz(int n, const V4<T> *__restrict__ src, T *__restrict__ dst)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const V4<T> v = src[i];
    dst[3 * (size_t)i] = v.x;
    dst[3 * (size_t)i + 1] = v.y;
    dst[3 * (size_t)i + 2] = v.z;
}

// Single precision with 16-byte aligned packed arrays: thread t moves
// particles 4t .. 4t+3, reading or writing their twelve packed values as three
// 16-byte words, so a warp touches 1536 contiguous bytes of the packed array
// per instruction triple (full-width transactions, which matters most when
// the packed array is pinned host memory read or written across the host
// link).  The last n % 4 particles go through the scalar kernels.
__global__ void k_unpack_xyz4(int nq, const float4 *__restrict__ src, float4 *__restrict__ dst)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nq) return;
    const float4 a = src[3 * (size_t)t], b = src[3 * (size_t)t + 1], c = src[3 * (size_t)t + 2];
    float4 *d = dst + 4 * (size_t)t;
    float4 p0 = d[0], p1 = d[1], p2 = d[2], p3 = d[3];
    p0.x = a.x; p0.y = a.y; p0.z = a.z;
    p1.x = a.w; p1.y = b.x; p1.z = b.y;
    p2.x = b.z; p2.y = b.w; p2.z = c.x;
    p3.x = c.y; p3.y = c.z; p3.z = c.w;
    d[0] = p0;
    d[1] = p1;
    d[2] = p2;
    d[3] = p3;
}

__global__ void k_pack_xyz4(int nq, const float4 *__restrict__ src, float4 *__restrict__ dst)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nq) return;
    const float4 *s = src + 4 * (size_t)t;
    const float4 p0 = s[0], p1 = s[1], p2 = s[2], p3 = s[3];
    dst[3 * (size_t)t] = make_float4(p0.x, p0.y, p0.z, p1.x);
    dst[3 * (size_t)t + 1] = make_float4(p1.y, p1.z, p2.x, p2.y);
    dst[3 * (size_t)t + 2] = make_float4(p2.z, p3.x, p3.y, p3.z);
}

}  // namespace fpm

extern "C" fpm_status fpm_unpack_xyz(int32_t n, fpm_prec prec, const void *src_xyz, void *dst4, fpm_stream stream)
{
    if (n < 0 || (n > 0 && (!src_xyz || !dst4))) return fpm_fail(FPM_ERR_INVALID, "fpm_unpack_xyz: bad argument");
    if (prec != FPM_F32 && prec != FPM_F64) return fpm_fail(FPM_ERR_INVALID, "fpm_unpack_xyz: bad precision");
    if (n == 0) return FPM_OK;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == FPM_F32 && ((uintptr_t)src_xyz & 15u) == 0) {
        const int nq = n / 4, r = n - 4 * nq;
        if (nq > 0)
            k_unpack_xyz4<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(nq, (const float4 *)src_xyz, (float4 *)dst4);
        if (r > 0)
            k_unpack_xyz<float><<<1, 32, 0, st>>>(r, (const float *)src_xyz + 12 * (size_t)nq,
                                                 (float4 *)dst4 + 4 * (size_t)nq);
    } else if (prec == FPM_F32) {
        k_unpack_xyz<float><<<blocks, 256, 0, st>>>(n, (const float *)src_xyz, (float4 *)dst4);
    } else {
        k_unpack_xyz<double><<<blocks, 256, 0, st>>>(n, (const double *)src_xyz, (double4_32a *)dst4);
    }
    return fpm_check_launch("fpm_unpack_xyz");
}

extern "C" fpm_status fpm_pack_xyz(int32_t n, fpm_prec prec, const void *src4, void *dst_xyz, fpm_stream stream)
{
    if (n < 0 || (n > 0 && (!src4 || !dst_xyz))) return fpm_fail(FPM_ERR_INVALID, "fpm_pack_xyz: bad argument");
    if (prec != FPM_F32 && prec != FPM_F64) return fpm_fail(FPM_ERR_INVALID, "fpm_pack_xyz: bad precision");
    if (n == 0) return FPM_OK;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == FPM_F32 && ((uintptr_t)dst_xyz & 15u) == 0) {
        const int nq = n / 4, r = n - 4 * nq;
        if (nq > 0)
            k_pack_xyz4<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(nq, (const float4 *)src4, (float4 *)dst_xyz);
        if (r > 0)
            k_pack_xyz<float><<<1, 32, 0, st>>>(r, (const float4 *)src4 + 4 * (size_t)nq,
                                               (float *)dst_xyz + 12 * (size_t)nq);
    } else if (prec == FPM_F32) {
        k_pack_xyz<float><<<blocks, 256, 0, st>>>(n, (const float4 *)src4, (float *)dst_xyz);
    } else {
        k_pack_xyz<double><<<blocks, 256, 0, st>>>(n, (const double4_32a *)src4, (double *)dst_xyz);
    }
    return fpm_check_launch("fpm_pack_xyz");
}
