// p2m.cu -- particle-to-mesh and mesh-to-particle interpolation with the
// moment-conserving M'4 kernel (Sec. 4.4, the vortex method's interpolations).
//
// Mesh: N[d] nodes per dimension at x = i h_d, h_d = L_d / N_d, periodic.  A
// particle with s = x inv (inv = N / L, FP32) in cell c = floor(s) touches the
// nodes c - 1 .. c + 2 (mod N) with weight prod_d M'4(s_d - node_d).
//
// P2M is a gather, so it needs no atomics and is bit-reproducible: the
// particles are binned by mesh cell (fpm_celllist_build with a grid from
// fpm_mesh_grid, the values reordered as its `vel`), and node m sums over the
// particles of cells m - 2 .. m + 1 in each dimension.  One block per tile of
// kTX x kTY x kTZ nodes stages the particles of the tile's
// (kTX + 3) x (kTY + 3) x (kTZ + 3) cells in shared memory, each with its 12
// weights (4 per dimension, computed once) and its value; a node then needs
// per particle three weight lookups and four FMAs.
#include "fpm_common.cuh"

namespace fpm {

constexpr int kTX = 8, kTY = 8, kTZ = 4;  // nodes per tile (one thread each)
constexpr int kCX = kTX + 3, kCY = kTY + 3, kCZ = kTZ + 3;
constexpr int kTileCells = kCX * kCY * kCZ;
constexpr int kP2mThreads = kTX * kTY * kTZ;
static_assert(kP2mThreads == 256, "one thread per node of a tile");
constexpr int kP2mSmem = 96 * 1024;

// M'4: 1 - 5/2 x^2 + 3/2 |x|^3 (|x| < 1), (2 - |x|)^2 (1 - |x|) / 2 (|x| < 2).
__device__ __forceinline__ float m4p(float x)
{
    const float a = fabsf(x);
    if (a < 1.0f) return 1.0f + a * a * (1.5f * a - 2.5f);
    if (a < 2.0f) {
        const float b = 2.0f - a;
        return 0.5f * b * b * (1.0f - a);
    }
    return 0.0f;
}

// The four weights of one dimension for s in cell c: nodes c-1, c, c+1, c+2.
__device__ __forceinline__ void m4p4(float s, int c, float w[4])
{
    const float t = s - (float)c;  // in [0, 1]
    w[0] = m4p(t + 1.0f);
    w[1] = m4p(t);
    w[2] = m4p(t - 1.0f);
    w[3] = m4p(t - 2.0f);
}

struct MeshD {
    int N[3];
    float inv[3];
    float L[3];
};

// Scaled coordinate and cell of one dimension, exactly as the cell-list build
// wraps and bins (so that a staged particle's weights belong to its cell).
__device__ __forceinline__ void cell_s(float x, float L, float inv, int N, float &s, int &c)
{
    x = wrap1(x, L);
    s = __fmul_rn(x, inv);
    c = x >= 0.0f ? ((s >= (float)N) ? N : (int)s) : 0;
    if (c > N - 1) c = N - 1;
}

// i mod N for i in [-2, N + kCX): one add, then subtractions (a tile wraps a
// mesh of fewer nodes than its cells more than once).
__device__ __forceinline__ int wrapi(int i, int N)
{
    if (i < 0) i += N;
    while (i >= N) i -= N;
    return i;
}

// Staged particles, component-major (so that the threads of a warp, each
// reading another particle, spread over the banks): 12 weight rows of `cap`
// floats, then `cap` float4 values.
__global__ void __launch_bounds__(kP2mThreads)
    k_p2m(MeshD m, const float4 *__restrict__ pos, const float4 *__restrict__ val,
          const uint32_t *__restrict__ cs, int cap, float4 *__restrict__ mesh, fpm_dev_status *st)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *sv = (float4 *)smem_raw;
    float *sw = (float *)(sv + cap);  // sw[j * cap + e], j = 0..11
    __shared__ uint32_t coff[kTileCells + 1];  // staged offset of each tile cell
    __shared__ uint32_t cstart[kTileCells];    // its first particle (sorted index)
    __shared__ uint32_t wsum[kP2mThreads / 32];
    const int tilesx = (m.N[0] + kTX - 1) / kTX, tilesy = (m.N[1] + kTY - 1) / kTY;
    const int tx = blockIdx.x % tilesx, ty = (blockIdx.x / tilesx) % tilesy, tz = blockIdx.x / (tilesx * tilesy);
    const int x0 = tx * kTX, y0 = ty * kTY, z0 = tz * kTZ;
    const int t = threadIdx.x;
    // 1. particle counts of the tile's cells (local cell q = (cz*kCY + cy)*kCX + cx is
    //    global cell (x0-2+cx, y0-2+cy, z0-2+cz) mod N), exclusive scan into coff
    uint32_t cnt[4];
    uint32_t mine = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int q = t * 4 + r;
        cnt[r] = 0;
        if (q < kTileCells) {
            const int cx = q % kCX, cy = (q / kCX) % kCY, cz = q / (kCX * kCY);
            const uint32_t g = ((uint32_t)wrapi(z0 - 2 + cz, m.N[2]) * (uint32_t)m.N[1] +
                                (uint32_t)wrapi(y0 - 2 + cy, m.N[1])) * (uint32_t)m.N[0] +
                               (uint32_t)wrapi(x0 - 2 + cx, m.N[0]);
            const uint32_t a = cs[g];
            cstart[q] = a;
            cnt[r] = cs[g + 1] - a;
        }
        mine += cnt[r];
    }
    const int lane = t & 31, warp = t >> 5;
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t base = 0, total = 0;
    for (int w = 0; w < kP2mThreads / 32; ++w) {
        if (w < warp) base += wsum[w];
        total += wsum[w];
    }
    uint32_t run = base + incl - mine;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int q = t * 4 + r;
        if (q < kTileCells) coff[q] = run;
        run += cnt[r];
    }
    if (t == 0) coff[kTileCells] = total;
    __syncthreads();
    const bool staged = total <= (uint32_t)cap;
    if (!staged && t == 0 && st) atomicAdd(&st->spilled, 1u);
    // 2. stage the particles of every tile cell with their 12 weights (a
    //    thread per cell: cells hold about one particle)
    if (staged) {
        for (int q = t; q < kTileCells; q += kP2mThreads) {
            const uint32_t p0 = cstart[q], o = coff[q], k = coff[q + 1] - o;
            for (uint32_t e = 0; e < k; ++e) {
                const float4 p = pos[p0 + e];
                float w[12], s;
                int c;
                cell_s(p.x, m.L[0], m.inv[0], m.N[0], s, c);
                m4p4(s, c, w);
                cell_s(p.y, m.L[1], m.inv[1], m.N[1], s, c);
                m4p4(s, c, w + 4);
                cell_s(p.z, m.L[2], m.inv[2], m.N[2], s, c);
                m4p4(s, c, w + 8);
#pragma unroll
                for (int j = 0; j < 12; ++j) sw[j * cap + o + e] = w[j];
                sv[o + e] = val[p0 + e];
            }
        }
    }
    __syncthreads();
    // 3. node (x0 + a, y0 + b, z0 + c): in each of its 16 cell rows the cells
    //    a .. a+3 (local x) are consecutive in the staging; a particle of local
    //    cell node + k (per dimension) has weight index 3 - k.  The node walks
    //    the particles of its 16 rows as one sequence (row by row, in staging
    //    order), so that the lanes of a warp diverge only on their totals.
    const int a = t % kTX, b = (t / kTX) % kTY, c = t / (kTX * kTY);
    const int gx = x0 + a, gy = y0 + b, gz = z0 + c;
    if (gx >= m.N[0] || gy >= m.N[1] || gz >= m.N[2]) return;
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    int row = -1;  // ky + 4 kz of the current row
    int q0 = 0;
    uint32_t e = 0, b1 = 0, b2 = 0, b3 = 0, rend = 0;
    for (;;) {
        while (e == rend) {  // next non-empty row
            if (++row == 16) break;
            q0 = ((c + (row >> 2)) * kCY + (b + (row & 3))) * kCX + a;
            e = coff[q0];
            b1 = coff[q0 + 1];
            b2 = coff[q0 + 2];
            b3 = coff[q0 + 3];
            rend = coff[q0 + 4];
        }
        if (row == 16) break;
        const int kx = (e >= b1) + (e >= b2) + (e >= b3);
        const int ky = row & 3, kz = row >> 2;
        float wx, wy, wz;
        float4 v;
        if (staged) {
            wx = sw[(3 - kx) * cap + e];
            wy = sw[(7 - ky) * cap + e];
            wz = sw[(11 - kz) * cap + e];
            v = sv[e];
        } else {  // the particle from global memory
            const uint32_t i = cstart[q0 + kx] + (e - coff[q0 + kx]);
            const float4 p = pos[i];
            float w4[4], s;
            int cc;
            cell_s(p.x, m.L[0], m.inv[0], m.N[0], s, cc);
            m4p4(s, cc, w4);
            wx = w4[3 - kx];
            cell_s(p.y, m.L[1], m.inv[1], m.N[1], s, cc);
            m4p4(s, cc, w4);
            wy = w4[3 - ky];
            cell_s(p.z, m.L[2], m.inv[2], m.N[2], s, cc);
            m4p4(s, cc, w4);
            wz = w4[3 - kz];
            v = val[i];
        }
        const float w = wx * wy * wz;
        acc.x = fmaf(w, v.x, acc.x);
        acc.y = fmaf(w, v.y, acc.y);
        acc.z = fmaf(w, v.z, acc.z);
        acc.w = fmaf(w, v.w, acc.w);
        ++e;
    }
    mesh[((size_t)gz * (size_t)m.N[1] + (size_t)gy) * (size_t)m.N[0] + (size_t)gx] = acc;
}

// Mesh-to-particle: one thread per particle gathers its 64 nodes; thread t
// takes particle order[t] (neighbouring threads on neighbouring particles when
// order is a binning's permutation, so that their nodes are shared in L1).
__global__ void k_m2p(MeshD m, int n, const float4 *__restrict__ pos, const float4 *__restrict__ mesh,
                      const uint32_t *__restrict__ order, float4 *__restrict__ out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int i = order ? (int)order[t] : t;
    const float4 p = pos[i];
    float wx[4], wy[4], wz[4], s;
    int cx, cy, cz;
    cell_s(p.x, m.L[0], m.inv[0], m.N[0], s, cx);
    m4p4(s, cx, wx);
    cell_s(p.y, m.L[1], m.inv[1], m.N[1], s, cy);
    m4p4(s, cy, wy);
    cell_s(p.z, m.L[2], m.inv[2], m.N[2], s, cz);
    m4p4(s, cz, wz);
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int kz = 0; kz < 4; ++kz) {
        const int gz = (cz - 1 + kz + m.N[2]) % m.N[2];
        for (int ky = 0; ky < 4; ++ky) {
            const int gy = (cy - 1 + ky + m.N[1]) % m.N[1];
            const float wyz = wy[ky] * wz[kz];
            const float4 *row = mesh + ((size_t)gz * (size_t)m.N[1] + (size_t)gy) * (size_t)m.N[0];
#pragma unroll
            for (int kx = 0; kx < 4; ++kx) {
                const int gx = (cx - 1 + kx + m.N[0]) % m.N[0];
                const float w = wx[kx] * wyz;
                const float4 v = __ldg(row + gx);
                acc.x = fmaf(w, v.x, acc.x);
                acc.y = fmaf(w, v.y, acc.y);
                acc.z = fmaf(w, v.z, acc.z);
                acc.w = fmaf(w, v.w, acc.w);
            }
        }
    }
    out[i] = acc;
}

static fpm_status mesh_ok(const fpm_box *box, const fpm_grid *g, const char *who, MeshD &m)
{
    if (!box || !g) return fpm_fail(FPM_ERR_INVALID, "%s: null box or grid", who);
    for (int d = 0; d < 3; ++d) {
        if (!box->periodic[d]) return fpm_fail(FPM_ERR_INVALID, "%s: the mesh must be periodic in every dimension", who);
        if (g->nc[d] < 3 || !(box->L[d] > 0.0)) return fpm_fail(FPM_ERR_INVALID, "%s: bad mesh", who);
        m.N[d] = g->nc[d];
        m.inv[d] = g->inv[d];
        m.L[d] = (float)box->L[d];
    }
    if ((int64_t)g->nc[0] * g->nc[1] * g->nc[2] != g->ncell)
        return fpm_fail(FPM_ERR_INVALID, "%s: grid ncell inconsistent with nc", who);
    return FPM_OK;
}

}  // namespace fpm

using namespace fpm;

extern "C" fpm_status fpm_mesh_grid(const fpm_box *box, const int32_t N[3], fpm_grid *out)
{
    if (!box || !N || !out) return fpm_fail(FPM_ERR_INVALID, "fpm_mesh_grid: null pointer");
    int64_t total = 1;
    fpm_grid g{};
    for (int d = 0; d < 3; ++d) {
        if (N[d] < 3 || !(box->L[d] > 0.0) || !box->periodic[d])
            return fpm_fail(FPM_ERR_INVALID, "fpm_mesh_grid: need N >= 3 and a periodic box in every dimension");
        g.nc[d] = N[d];
        g.inv[d] = (float)((double)N[d] / box->L[d]);
        total *= N[d];
    }
    if (total > (int64_t)(1u << 24)) return fpm_fail(FPM_ERR_INVALID, "fpm_mesh_grid: more than 2^24 nodes");
    g.ncell = (int32_t)total;
    g.tiles_x = 1;
    *out = g;
    return FPM_OK;
}

extern "C" fpm_status fpm_p2m(const fpm_box *box, const fpm_grid *mesh_grid, int32_t n, const void *pos,
                              const void *val, const uint32_t *cell_start, void *mesh, fpm_dev_status *d_status,
                              fpm_stream stream)
{
    MeshD m{};
    fpm_status s = mesh_ok(box, mesh_grid, "fpm_p2m", m);
    if (s != FPM_OK) return s;
    if (n < 0 || !cell_start || !mesh || (n > 0 && (!pos || !val)))
        return fpm_fail(FPM_ERR_INVALID, "fpm_p2m: null pointer or bad size");
    const int tiles = ((m.N[0] + kTX - 1) / kTX) * ((m.N[1] + kTY - 1) / kTY) * ((m.N[2] + kTZ - 1) / kTZ);
    // staging room: 1.15x the tile cells' mean load + 96 (a uniform load stays
    // far below it: ~800 +- 30 particles at the paper's density), 64 B per
    // particle, within the budget; three blocks per SM at that size
    const double mean = (double)n / (double)mesh_grid->ncell * kTileCells;
    int cap = (int)(1.15 * mean) + 96;
    cap = (cap + 3) / 4 * 4;
    const int per = 12 * (int)sizeof(float) + (int)sizeof(float4);
    const int maxcap = kP2mSmem / per / 4 * 4;
    if (cap > maxcap) cap = maxcap;
    const size_t smem = (size_t)cap * per;
    cudaFuncSetAttribute((const void *)k_p2m, cudaFuncAttributeMaxDynamicSharedMemorySize, kP2mSmem);
    k_p2m<<<tiles, kP2mThreads, smem, (cudaStream_t)stream>>>(m, (const float4 *)pos, (const float4 *)val,
                                                                cell_start, cap, (float4 *)mesh, d_status);
    return fpm_check_launch("fpm_p2m");
}

extern "C" fpm_status fpm_m2p(const fpm_box *box, const fpm_grid *mesh_grid, int32_t n, const void *pos,
                              const void *mesh, const uint32_t *order, void *val, fpm_stream stream)
{
    MeshD m{};
    fpm_status s = mesh_ok(box, mesh_grid, "fpm_m2p", m);
    if (s != FPM_OK) return s;
    if (n < 0 || !mesh || (n > 0 && (!pos || !val))) return fpm_fail(FPM_ERR_INVALID, "fpm_m2p: null pointer");
    if (n == 0) return FPM_OK;
    k_m2p<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(m, n, (const float4 *)pos, (const float4 *)mesh,
                                                           order, (float4 *)val);
    return fpm_check_launch("fpm_m2p");
}
