// api.cu -- host-side part of the libfpm C ABI: error text, status decoding,
// the cell-grid rule and workspace sizes.  See include/fpm.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>

#include "tiles.cuh"

static thread_local char g_last_error[512] = "";

fpm_status fpm_fail(fpm_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return s;
}

fpm_status fpm_check_launch(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fpm_fail(FPM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return FPM_OK;
}

extern "C" const char *fpm_status_string(fpm_status s)
{
    switch (s) {
    case FPM_OK: return "ok";
    case FPM_ERR_INVALID: return "invalid argument";
    case FPM_ERR_CAPACITY: return "neighbour list capacity exceeded";
    case FPM_ERR_DOMAIN: return "particle outside a non-periodic box dimension";
    case FPM_ERR_CUDA: return "CUDA error";
    case FPM_ERR_TIMEOUT: return "device wait timed out";
    case FPM_ERR_WORKSPACE: return "workspace missing or too small";
    }
    return "unknown status";
}

extern "C" const char *fpm_last_error(void) { return g_last_error; }

extern "C" fpm_status fpm_status_from_device(const fpm_dev_status *h)
{
    if (!h) return fpm_fail(FPM_ERR_INVALID, "fpm_status_from_device: null pointer");
    if (h->flags & FPM_FLAG_CAPACITY) return FPM_ERR_CAPACITY;
    if (h->flags & FPM_FLAG_DOMAIN) return FPM_ERR_DOMAIN;
    if (h->flags & FPM_FLAG_TIMEOUT) return FPM_ERR_TIMEOUT;
    return FPM_OK;
}

extern "C" int64_t fpm_nbr_ld(int32_t n)
{
    if (n < 0) return 0;
    return ((int64_t)n + 31) / 32 * 32;
}

extern "C" fpm_status fpm_grid_make(const fpm_box *box, double r_cell, int32_t n_hint, fpm_grid *out)
{
    if (!box || !out) return fpm_fail(FPM_ERR_INVALID, "fpm_grid_make: null pointer");
    if (!(r_cell > 0.0) || !std::isfinite(r_cell))
        return fpm_fail(FPM_ERR_INVALID, "fpm_grid_make: r_cell must be positive");
    int64_t total = 1;
    fpm_grid g{};
    for (int d = 0; d < 3; ++d) {
        double L = box->L[d];
        if (!(L > 0.0) || !std::isfinite(L)) return fpm_fail(FPM_ERR_INVALID, "fpm_grid_make: L[%d] <= 0", d);
        if (box->periodic[d] && !(L > 2.0 * r_cell * (1.0 + 1.0 / 1024.0)))
            return fpm_fail(FPM_ERR_INVALID,
                            "fpm_grid_make: periodic L[%d]=%g must exceed 2*r_cell*(1+2^-10) (r_cell=%g)", d, L,
                            r_cell);
        double q = std::floor(L / (r_cell * (1.0 + 1.0 / 4096.0)));
        int64_t nc = q > 1048576.0 ? 1048576 : (int64_t)q;
        if (nc < 1) nc = 1;
        if (box->periodic[d] && nc < 3) nc = 1;
        g.nc[d] = (int32_t)nc;
        g.inv[d] = (float)((double)nc / L);
        total *= nc;
    }
    if (total > (int64_t)(1u << 24))
        return fpm_fail(FPM_ERR_INVALID, "fpm_grid_make: %lld cells exceed the 2^24 limit", (long long)total);
    g.ncell = (int32_t)total;
    // tile width along x: about kTileTarget particles per tile, at most 14 cells
    const double per_cell = n_hint > 0 ? (double)n_hint / (double)total : 16.0;
    int w = (int)std::lround((double)fpm::kTileTarget / (per_cell > 1e-9 ? per_cell : 1e-9));
    if (w < 1) w = 1;
    if (w > 14) w = 14;
    int tiles = (g.nc[0] + w - 1) / w;
    if (tiles < 1) tiles = 1;
    g.tiles_x = tiles;
    *out = g;
    return FPM_OK;
}

int grid_cap(long long want)
{
    static int cap = 0;
    if (cap == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cap = 8 * (sms > 0 ? sms : 1);
    }
    if (want < 1) return 1;
    return want < cap ? (int)want : cap;
}

extern "C" fpm_status fpm_reduce_workspace(int32_t n, const fpm_grid *grid, size_t *bytes)
{
    if (!bytes || n < 0) return fpm_fail(FPM_ERR_INVALID, "fpm_reduce_workspace: bad argument");
    // counter (256 B) + 8 doubles per block: blocks of 256 particles, or one
    // block per cell tile for the pair sweeps
    size_t blocks = ((size_t)n + 255) / 256;
    if (grid) {
        const size_t tiles = (size_t)(grid->tiles_x > 0 ? grid->tiles_x : 1) * (size_t)grid->nc[1] * (size_t)grid->nc[2];
        if (tiles > blocks) blocks = tiles;
    }
    if (blocks < 1) blocks = 1;
    *bytes = 256 + blocks * 8 * sizeof(double);
    return FPM_OK;
}
