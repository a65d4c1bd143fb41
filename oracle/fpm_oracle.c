/*
 * fpm_oracle.c -- plain, slow, obviously-correct CPU reference of the particle
 * hot path of OpenFPM (arXiv 1804.07598).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header, table or helper with the CUDA library; it is compiled by gcc
 * with -ffp-contract=off so that every floating-point operation written here
 * is the operation executed.
 *
 * Conventions (readings of the paper, which is silent on them):
 *   - The domain is the box [0,L0)x[0,L1)x[0,L2) with a per-dimension
 *     periodic flag (the paper's Box + bc, Listing 4.1 of Sec. 4.1).
 *   - Positions and velocities are stored as 4-vectors (x,y,z,w); w is unused.
 *   - Cell grid: nc = floor(L / (r_cell*(1+2^-12))); a periodic dimension with
 *     nc < 3 uses nc = 1 (all particles of that dimension are candidates);
 *     a periodic dimension needs L > 2*r_cell*(1+2^-10) so that the minimum
 *     image is unique inside r_cell.
 *   - Cell coordinate: ci = min((int)((float)x * inv), nc-1) with
 *     inv = (float)(nc/L), in single precision for both position precisions.
 *   - Minimum image per periodic dimension, d = x_i - x_j: if d > L/2 the
 *     separation is (x_i - L) - x_j, if d < -L/2 it is x_i - (x_j - L)
 *     (the exact image shift first, then one rounded subtraction).
 *   - Squared distance: r2 = fma(dz,dz, fma(dy,dy, dx*dx)) in the precision
 *     of the positions; a pair is inside a radius r iff r2 < (T)(r*r).
 *
 * Each function names the passage of the paper it follows.  Functions whose
 * parity is pinned by an independent test say so in the test-suite; none of
 * the functions here is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MARGIN_CELL (1.0 + 1.0 / 4096.0)
#define ORC_MARGIN_HALF (1.0 + 1.0 / 1024.0)

/* ------------------------------------------------------------------------ */
/* Cell grid (cell lists, Sec. 2; getCellListSym in Listing 4.1)             */
/* ------------------------------------------------------------------------ */

/* Returns 0 on success, 1 if the box cannot hold the cutoff sphere. */
int orc_cell_grid(const double L[3], const int periodic[3], double r_cell,
                  int nc[3], float inv[3])
{
    if (!(r_cell > 0.0)) return 1;
    for (int d = 0; d < 3; ++d) {
        if (!(L[d] > 0.0)) return 1;
        if (periodic[d] && !(L[d] > 2.0 * r_cell * ORC_MARGIN_HALF)) return 1;
        double q = floor(L[d] / (r_cell * ORC_MARGIN_CELL));
        int n = (q > 1048576.0) ? 1048576 : (int)q;
        if (n < 1) n = 1;
        if (periodic[d] && n < 3) n = 1;
        nc[d] = n;
        inv[d] = (float)((double)n / L[d]);
    }
    return 0;
}

/* Wrap one coordinate into [0,L): one correction step each way. */
static float wrap_f32(float x, float L)
{
    if (x < 0.0f) x = x + L;
    if (x >= L) x = x - L;
    return x;
}

static double wrap_f64(double x, double L)
{
    if (x < 0.0) x = x + L;
    if (x >= L) x = x - L;
    return x;
}

void orc_wrap_f32(int n, float *pos4, const double L[3], const int periodic[3])
{
    for (int i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d)
            if (periodic[d]) pos4[4 * i + d] = wrap_f32(pos4[4 * i + d], (float)L[d]);
}

void orc_wrap_f64(int n, double *pos4, const double L[3], const int periodic[3])
{
    for (int i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d)
            if (periodic[d]) pos4[4 * i + d] = wrap_f64(pos4[4 * i + d], L[d]);
}

/* Cell coordinate of one (already wrapped) coordinate.  *bad is set when the
 * coordinate lies outside [0,L) (only possible in a non-periodic dimension). */
static int cell_coord(float xf, float inv, int nc, int *bad)
{
    if (!(xf >= 0.0f)) { *bad = 1; return 0; }
    float s = xf * inv;
    int c = (s >= (float)nc) ? nc : (int)s;
    if (c > nc - 1) c = nc - 1;
    return c;
}

static uint32_t linear_cell(const int c[3], const int nc[3])
{
    return (uint32_t)(((int64_t)c[2] * nc[1] + c[1]) * nc[0] + c[0]);
}

/* Cell id of every particle; positions must already be wrapped.  Returns the
 * number of particles found outside a non-periodic dimension's [0,L). */
int orc_cell_index_f32(int n, const float *pos4, const int nc[3], const float inv[3],
                       const double L[3], uint32_t *cell)
{
    int nbad = 0;
    for (int i = 0; i < n; ++i) {
        int c[3], bad = 0;
        for (int d = 0; d < 3; ++d) {
            float x = pos4[4 * i + d];
            if (x >= (float)L[d]) bad = 1;
            c[d] = cell_coord(x, inv[d], nc[d], &bad);
        }
        nbad += bad;
        cell[i] = linear_cell(c, nc);
    }
    return nbad;
}

int orc_cell_index_f64(int n, const double *pos4, const int nc[3], const float inv[3],
                       const double L[3], uint32_t *cell)
{
    int nbad = 0;
    for (int i = 0; i < n; ++i) {
        int c[3], bad = 0;
        for (int d = 0; d < 3; ++d) {
            double x = pos4[4 * i + d];
            if (x >= L[d] || x < 0.0) bad = 1;
            c[d] = cell_coord((float)x, inv[d], nc[d], &bad);
        }
        nbad += bad;
        cell[i] = linear_cell(c, nc);
    }
    return nbad;
}

/* Stable counting sort by cell (the re-sorting of Sec. 3.6): perm lists the
 * particles cell by cell, ties in ascending input index; cell_start[c] is the
 * exclusive prefix sum of the cell counts, cell_start[ncell] = n. */
void orc_counting_sort(int n, int ncell, const uint32_t *cell,
                       uint32_t *cell_start, uint32_t *perm)
{
    uint32_t *fill = (uint32_t *)calloc((size_t)ncell + 1, sizeof(uint32_t));
    for (int c = 0; c <= ncell; ++c) cell_start[c] = 0;
    for (int i = 0; i < n; ++i) cell_start[cell[i] + 1] += 1;
    for (int c = 0; c < ncell; ++c) cell_start[c + 1] += cell_start[c];
    for (int i = 0; i < n; ++i) {
        uint32_t c = cell[i];
        perm[cell_start[c] + fill[c]] = (uint32_t)i;
        fill[c] += 1;
    }
    free(fill);
}

/* ------------------------------------------------------------------------ */
/* Pair geometry                                                             */
/* ------------------------------------------------------------------------ */

/* Minimum-image separation of one periodic coordinate, x_i - x_j.  When the
 * plain difference exceeds L/2 the image shift is applied to the coordinate
 * lying above L/2 before subtracting: (x_i - L) - x_j or x_i - (x_j - L).
 * That shift is exact (both operands within a factor 2), so the separation
 * carries one rounding, like a pair inside the box; shifting after the
 * subtraction would round twice and lose the low bits of the small
 * coordinate. */
static float sep1_f32(float xi, float xj, float L)
{
    float h = 0.5f * L;
    float d = xi - xj;
    if (d > h) d = (xi - L) - xj;
    else if (d < -h) d = xi - (xj - L);
    return d;
}

static double sep1_f64(double xi, double xj, double L)
{
    double h = 0.5 * L;
    double d = xi - xj;
    if (d > h) d = (xi - L) - xj;
    else if (d < -h) d = xi - (xj - L);
    return d;
}

/* Separation x_i - x_j (minimum image) and its squared length, float. */
static float sep_f32(const float *xi, const float *xj, const double L[3],
                     const int periodic[3], float dv[3])
{
    for (int d = 0; d < 3; ++d)
        dv[d] = periodic[d] ? sep1_f32(xi[d], xj[d], (float)L[d]) : xi[d] - xj[d];
    return fmaf(dv[2], dv[2], fmaf(dv[1], dv[1], dv[0] * dv[0]));
}

static double sep_f64(const double *xi, const double *xj, const double L[3],
                      const int periodic[3], double dv[3])
{
    for (int d = 0; d < 3; ++d)
        dv[d] = periodic[d] ? sep1_f64(xi[d], xj[d], L[d]) : xi[d] - xj[d];
    return fma(dv[2], dv[2], fma(dv[1], dv[1], dv[0] * dv[0]));
}

/* An oracle-private cell list over arbitrary-order positions. */
typedef struct {
    int nc[3];
    float inv[3];
    int ncell;
    uint32_t *cell;        /* [n] */
    uint32_t *cell_start;  /* [ncell+1] */
    uint32_t *perm;        /* [n] */
} orc_cells;

static int cells_build(orc_cells *cl, int n, const float *pf, const double *pd,
                       const double L[3], const int periodic[3], double r_cell)
{
    memset(cl, 0, sizeof(*cl));
    if (orc_cell_grid(L, periodic, r_cell, cl->nc, cl->inv)) return 1;
    cl->ncell = cl->nc[0] * cl->nc[1] * cl->nc[2];
    cl->cell = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    cl->perm = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    cl->cell_start = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)cl->ncell + 1));
    /* bin wrapped copies, so callers may pass positions one box length out */
    size_t m = 4 * (size_t)(n > 0 ? n : 1);
    if (pf) {
        float *w = (float *)malloc(sizeof(float) * m);
        memcpy(w, pf, sizeof(float) * 4 * (size_t)n);
        orc_wrap_f32(n, w, L, periodic);
        orc_cell_index_f32(n, w, cl->nc, cl->inv, L, cl->cell);
        free(w);
    } else {
        double *w = (double *)malloc(sizeof(double) * m);
        memcpy(w, pd, sizeof(double) * 4 * (size_t)n);
        orc_wrap_f64(n, w, L, periodic);
        orc_cell_index_f64(n, w, cl->nc, cl->inv, L, cl->cell);
        free(w);
    }
    orc_counting_sort(n, cl->ncell, cl->cell, cl->cell_start, cl->perm);
    return 0;
}

static void cells_free(orc_cells *cl)
{
    free(cl->cell);
    free(cl->perm);
    free(cl->cell_start);
}

/* The stencil offsets of one dimension: {-1,0,1}, or {0} when nc == 1. */
static int stencil_dim(int nc, int periodic, int c, int out[3])
{
    int k = 0;
    if (nc == 1) { out[k++] = 0; return k; }
    for (int o = -1; o <= 1; ++o) {
        int cc = c + o;
        if (periodic) cc = (cc + nc) % nc;
        else if (cc < 0 || cc >= nc) continue;
        out[k++] = cc;
    }
    return k;
}

/* Candidates of particle i: every particle of the 27 (or fewer) cells around
 * cell `ci`, in stencil order (z, then y, then x, each from -1 to 1), then in
 * ascending input index inside each cell.  Writes them to out (room for n
 * entries: a cell stencil never repeats a cell) and returns how many. */
static int stencil_candidates(const orc_cells *cl, const int periodic[3], uint32_t ci,
                              uint32_t *out)
{
    int c3[3], cz[3], cy[3], cx[3];
    c3[0] = (int)(ci % (uint32_t)cl->nc[0]);
    c3[1] = (int)((ci / (uint32_t)cl->nc[0]) % (uint32_t)cl->nc[1]);
    c3[2] = (int)(ci / ((uint32_t)cl->nc[0] * (uint32_t)cl->nc[1]));
    int kz = stencil_dim(cl->nc[2], periodic[2], c3[2], cz);
    int ky = stencil_dim(cl->nc[1], periodic[1], c3[1], cy);
    int kx = stencil_dim(cl->nc[0], periodic[0], c3[0], cx);
    int k = 0;
    for (int a = 0; a < kz; ++a)
        for (int b = 0; b < ky; ++b)
            for (int e = 0; e < kx; ++e) {
                int cc[3] = {cx[e], cy[b], cz[a]};
                uint32_t c = linear_cell(cc, cl->nc);
                for (uint32_t s = cl->cell_start[c]; s < cl->cell_start[c + 1]; ++s)
                    out[k++] = cl->perm[s];
            }
    return k;
}

/* ------------------------------------------------------------------------ */
/* Verlet lists (Sec. 2 "Verlet Lists [46]"; Sec. 4.1)                       */
/* ------------------------------------------------------------------------ */

/* Full neighbour lists: for every particle i, every j != i with
 * r2(i,j) < (T)(r_list^2), listed in stencil order.  CSR output: offsets[n+1],
 * nbr[offsets[i] .. offsets[i+1]).  Returns the total count, or -1 if it
 * exceeds cap_total (offsets are then still complete, nbr truncated), or -2
 * on an invalid box. */
static int64_t neighbors_impl(int n, const float *pf, const double *pd,
                              const double L[3], const int periodic[3],
                              double r_list, int64_t cap_total,
                              int64_t *offsets, uint32_t *nbr)
{
    orc_cells cl;
    if (cells_build(&cl, n, pf, pd, L, periodic, r_list)) return -2;
    float rl2f = (float)(r_list * r_list);
    double rl2d = r_list * r_list;
    int64_t total = 0;
    uint32_t *cand = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        offsets[i] = total;
        int m = stencil_candidates(&cl, periodic, cl.cell[i], cand);
        for (int t = 0; t < m; ++t) {
            uint32_t j = cand[t];
            if (j != (uint32_t)i) {
                int inside;
                if (pf) {
                    float dv[3];
                    inside = sep_f32(pf + 4 * (size_t)i, pf + 4 * (size_t)j, L, periodic, dv) < rl2f;
                } else {
                    double dv[3];
                    inside = sep_f64(pd + 4 * (size_t)i, pd + 4 * (size_t)j, L, periodic, dv) < rl2d;
                }
                if (inside) {
                    if (total < cap_total) nbr[total] = j;
                    total += 1;
                }
            }
        }
    }
    offsets[n] = total;
    free(cand);
    cells_free(&cl);
    return total > cap_total ? -1 : total;
}

int64_t orc_neighbors_f32(int n, const float *pos4, const double L[3], const int periodic[3],
                          double r_list, int64_t cap_total, int64_t *offsets, uint32_t *nbr)
{
    return neighbors_impl(n, pos4, NULL, L, periodic, r_list, cap_total, offsets, nbr);
}

int64_t orc_neighbors_f64(int n, const double *pos4, const double L[3], const int periodic[3],
                          double r_list, int64_t cap_total, int64_t *offsets, uint32_t *nbr)
{
    return neighbors_impl(n, NULL, pos4, L, periodic, r_list, cap_total, offsets, nbr);
}

/* Neighbour set of a single particle i by scanning all n particles (used for
 * sampled checks on large systems).  Returns the count written (up to cap). */
int orc_neighbors_one_f32(int n, const float *pos4, const double L[3], const int periodic[3],
                          double r_list, int i, int cap, uint32_t *out)
{
    float rl2f = (float)(r_list * r_list);
    int k = 0;
    for (int j = 0; j < n; ++j) {
        float dv[3];
        if (j != i && sep_f32(pos4 + 4 * (size_t)i, pos4 + 4 * (size_t)j, L, periodic, dv) < rl2f) {
            if (k < cap) out[k] = (uint32_t)j;
            k++;
        }
    }
    return k;
}

int orc_neighbors_one_f64(int n, const double *pos4, const double L[3], const int periodic[3],
                          double r_list, int i, int cap, uint32_t *out)
{
    double rl2d = r_list * r_list;
    int k = 0;
    for (int j = 0; j < n; ++j) {
        double dv[3];
        if (j != i && sep_f64(pos4 + 4 * (size_t)i, pos4 + 4 * (size_t)j, L, periodic, dv) < rl2d) {
            if (k < cap) out[k] = (uint32_t)j;
            k++;
        }
    }
    return k;
}

/* Verlet rebuild test: 1 iff some particle moved (minimum image) by more than
 * skin/2 since the reference positions, judged as d2 > (T)((skin/2)^2).  The
 * largest squared displacement is returned through max_d2. */
int orc_max_disp_f32(int n, const float *pos4, const float *ref4, const double L[3],
                     const int periodic[3], double skin, double *max_d2)
{
    float th = (float)(0.25 * skin * skin);
    float m = 0.0f;
    int flag = 0;
    for (int i = 0; i < n; ++i) {
        float dv[3];
        float d2 = sep_f32(pos4 + 4 * (size_t)i, ref4 + 4 * (size_t)i, L, periodic, dv);
        if (d2 > m) m = d2;
        if (d2 > th) flag = 1;
    }
    *max_d2 = m;
    return flag;
}

int orc_max_disp_f64(int n, const double *pos4, const double *ref4, const double L[3],
                     const int periodic[3], double skin, double *max_d2)
{
    double th = 0.25 * skin * skin;
    double m = 0.0;
    int flag = 0;
    for (int i = 0; i < n; ++i) {
        double dv[3];
        double d2 = sep_f64(pos4 + 4 * (size_t)i, ref4 + 4 * (size_t)i, L, periodic, dv);
        if (d2 > m) m = d2;
        if (d2 > th) flag = 1;
    }
    *max_d2 = m;
    return flag;
}

/* ------------------------------------------------------------------------ */
/* Lennard-Jones interaction (Sec. 4.1: V(r) = 4 eps [(s/r)^12 - (s/r)^6];    */
/* pair force 24 eps (2 s^12/r^14 - s^6/r^8) (x_p - x_q), truncated at r_cut) */
/* ------------------------------------------------------------------------ */

/* Pair inclusion test.  With mask_f32 != 0 the decision r2 < rc^2 is taken in
 * single precision on the single-precision positions (which the FP64 input
 * holds exactly), as a single-precision caller decides it; otherwise in FP64. */
static int pair_inside(const double *xi, const double *xj, const double L[3],
                       const int periodic[3], double rc, int mask_f32, double dv[3])
{
    double r2 = sep_f64(xi, xj, L, periodic, dv);
    if (mask_f32) {
        float a[3] = {(float)xi[0], (float)xi[1], (float)xi[2]};
        float b[3] = {(float)xj[0], (float)xj[1], (float)xj[2]};
        float df[3];
        return sep_f32(a, b, L, periodic, df) < (float)(rc * rc);
    }
    return r2 < rc * rc;
}

/* Forces, potential energy U = sum_{i<j} V(r_ij), virial
 * W = sum_{i<j} r_ij . F_ij and the number of interacting pairs.  Each pair
 * is visited once and applied to both particles (Newton's third law, the
 * symmetric interaction of Sec. 4.1).  force4 is [n][4] (w = per-particle
 * half pair energy).  out[0]=U, out[1]=W, out[2]=pairs. Returns 0 or 1. */
int orc_lj_forces(int n, const double *pos4, const double L[3], const int periodic[3],
                  double eps, double sigma, double rc, int mask_f32,
                  double *force4, double out[3])
{
    orc_cells cl;
    double r_cell = mask_f32 ? rc * (1.0 + 1.0 / 65536.0) : rc;
    if (cells_build(&cl, n, NULL, pos4, L, periodic, r_cell)) return 1;
    memset(force4, 0, sizeof(double) * 4 * (size_t)n);
    double U = 0.0, W = 0.0, pairs = 0.0;
    double s2 = sigma * sigma, s6 = s2 * s2 * s2, s12 = s6 * s6;
    uint32_t *cand = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        const double *xi = pos4 + 4 * (size_t)i;
        int m = stencil_candidates(&cl, periodic, cl.cell[i], cand);
        for (int t = 0; t < m; ++t) {
            uint32_t j = cand[t];
            if (j > (uint32_t)i) {
                double dv[3];
                const double *xj = pos4 + 4 * (size_t)j;
                if (pair_inside(xi, xj, L, periodic, rc, mask_f32, dv)) {
                    double r2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
                    double r6 = r2 * r2 * r2;
                    double r8 = r6 * r2, r14 = r6 * r6 * r2;
                    double f = 24.0 * eps * (2.0 * s12 / r14 - s6 / r8);
                    double v = 4.0 * eps * (s12 / (r6 * r6) - s6 / r6);
                    for (int d = 0; d < 3; ++d) {
                        force4[4 * (size_t)i + d] += f * dv[d];
                        force4[4 * (size_t)j + d] -= f * dv[d];
                    }
                    force4[4 * (size_t)i + 3] += 0.5 * v;
                    force4[4 * (size_t)j + 3] += 0.5 * v;
                    U += v;
                    W += f * r2;
                    pairs += 1.0;
                }
            }
        }
    }
    free(cand);
    cells_free(&cl);
    out[0] = U;
    out[1] = W;
    out[2] = pairs;
    return 0;
}

/* Forces on one particle i by scanning all n particles (sampled checks). */
void orc_lj_force_one(int n, const double *pos4, const double L[3], const int periodic[3],
                      double eps, double sigma, double rc, int mask_f32, int i, double f_out[4])
{
    double s2 = sigma * sigma, s6 = s2 * s2 * s2, s12 = s6 * s6;
    f_out[0] = f_out[1] = f_out[2] = f_out[3] = 0.0;
    for (int j = 0; j < n; ++j) {
        double dv[3];
        if (j == i) continue;
        if (!pair_inside(pos4 + 4 * (size_t)i, pos4 + 4 * (size_t)j, L, periodic, rc, mask_f32, dv))
            continue;
        double r2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
        double r6 = r2 * r2 * r2;
        double f = 24.0 * eps * (2.0 * s12 / (r6 * r6 * r2) - s6 / (r6 * r2));
        for (int d = 0; d < 3; ++d) f_out[d] += f * dv[d];
        f_out[3] += 0.5 * 4.0 * eps * (s12 / (r6 * r6) - s6 / r6);
    }
}

/* ------------------------------------------------------------------------ */
/* Velocity Verlet (Listing 4.1 time loop; unit mass)                        */
/* ------------------------------------------------------------------------ */

/* First half: v += dt/2 F; x += dt v; wrap into the periodic box. */
void orc_vv_kick_drift(int n, double dt, double *pos4, double *vel4, const double *force4,
                       const double L[3], const int periodic[3])
{
    for (int i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            size_t k = 4 * (size_t)i + d;
            vel4[k] = vel4[k] + 0.5 * dt * force4[k];
            pos4[k] = pos4[k] + dt * vel4[k];
            if (periodic[d]) pos4[k] = wrap_f64(pos4[k], L[d]);
        }
}

/* Second half: v += dt/2 F. */
void orc_vv_kick(int n, double dt, double *vel4, const double *force4)
{
    for (int i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            size_t k = 4 * (size_t)i + d;
            vel4[k] = vel4[k] + 0.5 * dt * force4[k];
        }
}

/* nsteps of NVE velocity Verlet from (pos4, vel4), in place.  Forces are
 * recomputed from the positions every step (no Verlet list: the force is the
 * sum over all pairs inside rc, which a correct Verlet list reproduces).
 * energies (optional, [nsteps+1][4]) receives KE, U, W, pairs after each
 * force evaluation, starting with the initial state. */
int orc_lj_nve(int n, double *pos4, double *vel4, const double L[3], const int periodic[3],
               double eps, double sigma, double rc, double dt, int nsteps, double *energies)
{
    double *f = (double *)malloc(sizeof(double) * 4 * (size_t)(n > 0 ? n : 1));
    double out[3];
    if (orc_lj_forces(n, pos4, L, periodic, eps, sigma, rc, 0, f, out)) { free(f); return 1; }
    for (int s = 0; s <= nsteps; ++s) {
        if (s > 0) {
            orc_vv_kick_drift(n, dt, pos4, vel4, f, L, periodic);
            orc_lj_forces(n, pos4, L, periodic, eps, sigma, rc, 0, f, out);
            orc_vv_kick(n, dt, vel4, f);
        }
        if (energies) {
            double ke = 0.0;
            for (int i = 0; i < n; ++i)
                for (int d = 0; d < 3; ++d) ke += 0.5 * vel4[4 * (size_t)i + d] * vel4[4 * (size_t)i + d];
            energies[4 * (size_t)s + 0] = ke;
            energies[4 * (size_t)s + 1] = out[0];
            energies[4 * (size_t)s + 2] = out[1];
            energies[4 * (size_t)s + 3] = out[2];
        }
    }
    free(f);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The NVE run on all host cores (OpenMP), used only to time the oracle as a */
/* multi-core CPU baseline; compiled without OpenMP it runs on one thread.   */
/* ------------------------------------------------------------------------ */

/* Threads an OpenMP loop of this library uses (1 without OpenMP). */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* The forces of orc_lj_forces (Sec. 4.1, unshifted LJ truncated at rc) with
 * every particle's sum taken from its own side, F_i = sum_{j != i, r < rc}
 * f r_ij, so that threads write disjoint rows (each pair is evaluated once
 * per side: the same sums up to the order of rounding).  out = (U, W, pairs)
 * from the halved two-sided sums. */
int orc_lj_forces_omp(int n, const double *pos4, const double L[3], const int periodic[3],
                      double eps, double sigma, double rc, double *force4, double out[3])
{
    orc_cells cl;
    if (cells_build(&cl, n, NULL, pos4, L, periodic, rc)) return 1;
    uint32_t maxc = 0;
    for (int c = 0; c < cl.ncell; ++c) {
        uint32_t k = cl.cell_start[c + 1] - cl.cell_start[c];
        if (k > maxc) maxc = k;
    }
    const size_t room = 27 * (size_t)maxc + 1;
    const double s2 = sigma * sigma, s6 = s2 * s2 * s2, s12 = s6 * s6;
    double U = 0.0, W = 0.0, pairs = 0.0;
#pragma omp parallel reduction(+ : U, W, pairs)
    {
        uint32_t *cand = (uint32_t *)malloc(sizeof(uint32_t) * room);
#pragma omp for schedule(static)
        for (int i = 0; i < n; ++i) {
            const double *xi = pos4 + 4 * (size_t)i;
            double F[4] = {0.0, 0.0, 0.0, 0.0};
            int m = stencil_candidates(&cl, periodic, cl.cell[i], cand);
            for (int t = 0; t < m; ++t) {
                uint32_t j = cand[t];
                double dv[3];
                if (j == (uint32_t)i || !pair_inside(xi, pos4 + 4 * (size_t)j, L, periodic, rc, 0, dv)) continue;
                double r2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
                double r6 = r2 * r2 * r2;
                double f = 24.0 * eps * (2.0 * s12 / (r6 * r6 * r2) - s6 / (r6 * r2));
                double v = 4.0 * eps * (s12 / (r6 * r6) - s6 / r6);
                for (int d = 0; d < 3; ++d) F[d] += f * dv[d];
                F[3] += 0.5 * v;
                U += 0.5 * v;
                W += 0.5 * f * r2;
                pairs += 0.5;
            }
            memcpy(force4 + 4 * (size_t)i, F, sizeof(F));
        }
        free(cand);
    }
    cells_free(&cl);
    out[0] = U;
    out[1] = W;
    out[2] = pairs;
    return 0;
}

/* nsteps of orc_lj_nve (velocity Verlet, Listing 4.1's time loop) with the
 * force sweep and both half steps spread over the host's cores. */
int orc_lj_nve_omp(int n, double *pos4, double *vel4, const double L[3], const int periodic[3],
                   double eps, double sigma, double rc, double dt, int nsteps)
{
    double *f = (double *)malloc(sizeof(double) * 4 * (size_t)(n > 0 ? n : 1));
    double out[3];
    if (orc_lj_forces_omp(n, pos4, L, periodic, eps, sigma, rc, f, out)) { free(f); return 1; }
    for (int s = 1; s <= nsteps; ++s) {
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; ++i)
            for (int d = 0; d < 3; ++d) {
                size_t k = 4 * (size_t)i + d;
                vel4[k] = vel4[k] + 0.5 * dt * f[k];
                pos4[k] = pos4[k] + dt * vel4[k];
                if (periodic[d]) pos4[k] = wrap_f64(pos4[k], L[d]);
            }
        orc_lj_forces_omp(n, pos4, L, periodic, eps, sigma, rc, f, out);
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; ++i)
            for (int d = 0; d < 3; ++d) {
                size_t k = 4 * (size_t)i + d;
                vel4[k] = vel4[k] + 0.5 * dt * f[k];
            }
    }
    free(f);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the LJ force (not in the paper; the differentiable workload)  */
/* ------------------------------------------------------------------------ */

/* Hessian-vector product of the LJ force field and parameter derivatives.
 * With s = r^2, phi(s) = 24 eps (2 sigma^12 s^-7 - sigma^6 s^-4) the pair
 * force factor (F_i = sum_j phi r_ij, r_ij = x_i - x_j) and
 * dphi/ds = 24 eps (-14 sigma^12 s^-8 + 4 sigma^6 s^-5):
 *   out_i  += sum_j [phi (a_i - a_j) + 2 dphi/ds (r_ij . (a_i - a_j)) r_ij]
 *             = (J a)_i with J = dF/dx (symmetric),
 *   dth[0] += sum_i a_i . dF_i/d eps   = sum_pairs (a_i - a_j) . r_ij phi / eps,
 *   dth[1] += sum_i a_i . dF_i/d sigma = sum_pairs (a_i - a_j) . r_ij
 *             24 eps (24 sigma^11 s^-7 - 6 sigma^5 s^-4),
 *   dU[0]  += dU/d eps   = sum_pairs 4 (sigma^12 s^-6 - sigma^6 s^-3),
 *   dU[1]  += dU/d sigma = sum_pairs 4 eps (12 sigma^11 s^-6 - 6 sigma^5 s^-3).
 * Pairs inside rc exactly as in orc_lj_forces (mask_f32 likewise).  out4 is
 * [n][4] and is overwritten (w = 0). Returns 0 or 1 (box too small). */
int orc_lj_hvp(int n, const double *pos4, const double L[3], const int periodic[3],
               double eps, double sigma, double rc, int mask_f32, const double *a4,
               double *out4, double dth[2], double dU[2])
{
    orc_cells cl;
    double r_cell = mask_f32 ? rc * (1.0 + 1.0 / 65536.0) : rc;
    if (cells_build(&cl, n, NULL, pos4, L, periodic, r_cell)) return 1;
    memset(out4, 0, sizeof(double) * 4 * (size_t)n);
    dth[0] = dth[1] = dU[0] = dU[1] = 0.0;
    double s2 = sigma * sigma, s6 = s2 * s2 * s2, s12 = s6 * s6;
    double s5 = s6 / sigma, s11 = s12 / sigma;
    uint32_t *cand = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        const double *xi = pos4 + 4 * (size_t)i;
        int m = stencil_candidates(&cl, periodic, cl.cell[i], cand);
        for (int t = 0; t < m; ++t) {
            uint32_t j = cand[t];
            if (j <= (uint32_t)i) continue;
            double r[3];
            if (!pair_inside(xi, pos4 + 4 * (size_t)j, L, periodic, rc, mask_f32, r)) continue;
            double s = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
            double s3 = s * s * s, s4 = s3 * s, s5p = s4 * s, s6p = s3 * s3, s7 = s6p * s, s8 = s7 * s;
            double phi = 24.0 * eps * (2.0 * s12 / s7 - s6 / s4);
            double dphi = 24.0 * eps * (-14.0 * s12 / s8 + 4.0 * s6 / s5p);
            double da[3], rda = 0.0;
            for (int d = 0; d < 3; ++d) {
                da[d] = a4[4 * (size_t)i + d] - a4[4 * (size_t)j + d];
                rda += r[d] * da[d];
            }
            for (int d = 0; d < 3; ++d) {
                double h = phi * da[d] + 2.0 * dphi * rda * r[d];
                out4[4 * (size_t)i + d] += h;
                out4[4 * (size_t)j + d] -= h;
            }
            dth[0] += rda * phi / eps;
            dth[1] += rda * 24.0 * eps * (24.0 * s11 / s7 - 6.0 * s5 / s4);
            dU[0] += 4.0 * (s12 / s6p - s6 / s3);
            dU[1] += 4.0 * eps * (12.0 * s11 / s6p - 6.0 * s5 / s3);
        }
    }
    free(cand);
    cells_free(&cl);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Weakly compressible SPH (Sec. 4.2, Eqs. 1-5)                              */
/* ------------------------------------------------------------------------ */

/* Parameters.  kernel 0: Wendland C2, W = a (1 - q/2)^4 (2q + 1),
 * a = 21 / (16 pi h^3), q = r/h in [0, 2]; kernel 1: cubic spline,
 * W = s [1 - 1.5 q^2 + 0.75 q^3] (q < 1), s 0.25 (2 - q)^3 (1 <= q < 2),
 * s = 1 / (pi h^3).  Both have support 2h. */
typedef struct {
    double h, m, rho0, c0, gamma, alpha, eta2, g[3];
    int kernel;
} orc_sph_params;

/* W(r) and dW/dr for one distance r >= 0. */
void orc_sph_kernel(int kernel, double h, double r, double *W, double *dWdr)
{
    const double pi = 3.14159265358979323846;
    double q = r / h;
    *W = 0.0;
    *dWdr = 0.0;
    if (q >= 2.0) return;
    if (kernel == 0) {
        double a = 21.0 / (16.0 * pi * h * h * h);
        double t = 1.0 - 0.5 * q;
        *W = a * t * t * t * t * (2.0 * q + 1.0);
        *dWdr = a / h * (-2.0 * t * t * t * (2.0 * q + 1.0) + 2.0 * t * t * t * t);
    } else {
        double s = 1.0 / (pi * h * h * h);
        if (q < 1.0) {
            *W = s * (1.0 - 1.5 * q * q + 0.75 * q * q * q);
            *dWdr = s / h * (-3.0 * q + 2.25 * q * q);
        } else {
            double t = 2.0 - q;
            *W = s * 0.25 * t * t * t;
            *dWdr = s / h * (-0.75 * t * t);
        }
    }
}

/* Tait equation of state (Eqs. 3-4): P = b [(rho/rho0)^gamma - 1],
 * b = c0^2 rho0 / gamma. */
double orc_sph_eos(const orc_sph_params *p, double rho)
{
    double b = p->c0 * p->c0 * p->rho0 / p->gamma;
    return b * (pow(rho / p->rho0, p->gamma) - 1.0);
}

/* Density by summation, sum_j m W(|x_i - x_j|) including j = i. */
int orc_sph_density_sum(int n, const double *pos4, const double L[3], const int periodic[3],
                        const orc_sph_params *p, double *rho)
{
    orc_cells cl;
    double rcut = 2.0 * p->h;
    if (cells_build(&cl, n, NULL, pos4, L, periodic, rcut)) return 1;
    uint32_t *cand = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        double W, dW;
        orc_sph_kernel(p->kernel, p->h, 0.0, &W, &dW);
        double s = p->m * W;
        int m = stencil_candidates(&cl, periodic, cl.cell[i], cand);
        for (int t = 0; t < m; ++t) {
            uint32_t j = cand[t];
            if (j == (uint32_t)i) continue;
            double r[3];
            double r2 = sep_f64(pos4 + 4 * (size_t)i, pos4 + 4 * (size_t)j, L, periodic, r);
            if (!(r2 < rcut * rcut)) continue;
            orc_sph_kernel(p->kernel, p->h, sqrt(r2), &W, &dW);
            s += p->m * W;
        }
        rho[i] = s;
    }
    free(cand);
    cells_free(&cl);
    return 0;
}

/* Rates of Eqs. 1-2 for every particle.  pos4 w holds the type: 0 fluid,
 * 1 fixed boundary particle.  For each pair p<q inside the support 2h (the
 * test r^2 < (2h)^2 in single precision when mask_f32):
 *   grad_p W = (dW/dr) (x_p - x_q) / r,  v_pq = v_p - v_q,
 *   drho_p += m v_pq . grad_p W,   drho_q += the same,
 *   Pi = -alpha c0 mu / rhobar with mu = h v_pq.(x_p - x_q) / (r^2 + eta^2),
 *        rhobar = (rho_p + rho_q)/2, when v_pq.(x_p - x_q) < 0, else 0,
 *   acc_p += -m ((P_p + P_q)/(rho_p rho_q) + Pi) grad_p W,  acc_q -= the same;
 * then acc += g for fluid particles and acc = 0 for boundary particles.
 * dtc[0] = max |acc| over fluid particles, dtc[1] = max |mu| over pairs. */
int orc_sph_rates(int n, const double *pos4, const double *vel4, const double *rho, const double L[3],
                  const int periodic[3], const orc_sph_params *p, int mask_f32, double *acc4, double *drho,
                  double dtc[2])
{
    orc_cells cl;
    double rcut = 2.0 * p->h;
    double r_cell = mask_f32 ? rcut * (1.0 + 1.0 / 65536.0) : rcut;
    if (cells_build(&cl, n, NULL, pos4, L, periodic, r_cell)) return 1;
    memset(acc4, 0, sizeof(double) * 4 * (size_t)n);
    memset(drho, 0, sizeof(double) * (size_t)n);
    double *P = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) P[i] = orc_sph_eos(p, rho[i]);
    double mumax = 0.0;
    uint32_t *cand = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        const double *xi = pos4 + 4 * (size_t)i;
        int m = stencil_candidates(&cl, periodic, cl.cell[i], cand);
        for (int t = 0; t < m; ++t) {
            uint32_t j = cand[t];
            if (j <= (uint32_t)i) continue;
            const double *xj = pos4 + 4 * (size_t)j;
            double r[3];
            if (!pair_inside(xi, xj, L, periodic, rcut, mask_f32, r)) continue;
            double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
            double rr = sqrt(r2);
            double W, dW;
            orc_sph_kernel(p->kernel, p->h, rr, &W, &dW);
            double gw[3], vr = 0.0, vdg = 0.0;
            for (int d = 0; d < 3; ++d) {
                gw[d] = rr > 0.0 ? dW * r[d] / rr : 0.0;
                double v = vel4[4 * (size_t)i + d] - vel4[4 * (size_t)j + d];
                vr += v * r[d];
                vdg += v * gw[d];
            }
            drho[i] += p->m * vdg;
            drho[j] += p->m * vdg;
            double mu = p->h * vr / (r2 + p->eta2);
            if (fabs(mu) > mumax) mumax = fabs(mu);
            double Pi = 0.0;
            if (vr < 0.0) Pi = -p->alpha * p->c0 * mu / (0.5 * (rho[i] + rho[j]));
            double c = -p->m * ((P[i] + P[j]) / (rho[i] * rho[j]) + Pi);
            for (int d = 0; d < 3; ++d) {
                acc4[4 * (size_t)i + d] += c * gw[d];
                acc4[4 * (size_t)j + d] -= c * gw[d];
            }
        }
    }
    double amax = 0.0;
    for (int i = 0; i < n; ++i) {
        if (pos4[4 * (size_t)i + 3] != 0.0) {
            acc4[4 * (size_t)i] = acc4[4 * (size_t)i + 1] = acc4[4 * (size_t)i + 2] = 0.0;
            continue;
        }
        double a2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            acc4[4 * (size_t)i + d] += p->g[d];
            a2 += acc4[4 * (size_t)i + d] * acc4[4 * (size_t)i + d];
        }
        if (sqrt(a2) > amax) amax = sqrt(a2);
    }
    dtc[0] = amax;
    dtc[1] = mumax;
    free(cand);
    free(P);
    cells_free(&cl);
    return 0;
}

/* Time step from the constraints: dt = cfl min(sqrt(h / max|a|), h / (c0 + max|mu|)). */
double orc_sph_dt(const orc_sph_params *p, const double dtc[2], double cfl)
{
    double dtf = dtc[0] > 0.0 ? sqrt(p->h / dtc[0]) : 1e300;
    double dtv = p->h / (p->c0 + dtc[1]);
    return cfl * (dtf < dtv ? dtf : dtv);
}

/* One symplectic step (predictor-corrector, the time stepping of Sec. 4.2):
 *   dt from the constraints of the rates at t^n;
 *   half: x += dt/2 v, v += dt/2 a, rho += dt/2 Drho (boundary: rho only);
 *   rates at the half step;
 *   v1 = v0 + dt a, x1 = x0 + dt (v1 + v0)/2 (fluid only),
 *   rho1 = rho0 (2 - e)/(2 + e), e = -(Drho / rho_half) dt (all particles).
 * Returns the dt used (negative on error). */
double orc_sph_step(int n, double *pos4, double *vel4, double *rho, const double L[3], const int periodic[3],
                    const orc_sph_params *p, double cfl)
{
    size_t m4 = 4 * (size_t)(n > 0 ? n : 1), m1 = (size_t)(n > 0 ? n : 1);
    double *acc = (double *)malloc(sizeof(double) * m4), *dr = (double *)malloc(sizeof(double) * m1);
    double *ph = (double *)malloc(sizeof(double) * m4), *vh = (double *)malloc(sizeof(double) * m4);
    double *rh = (double *)malloc(sizeof(double) * m1);
    double dtc[2];
    double dt = -1.0;
    if (orc_sph_rates(n, pos4, vel4, rho, L, periodic, p, 0, acc, dr, dtc)) goto done;
    dt = orc_sph_dt(p, dtc, cfl);
    memcpy(ph, pos4, sizeof(double) * 4 * (size_t)n);
    memcpy(vh, vel4, sizeof(double) * 4 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        rh[i] = rho[i] + 0.5 * dt * dr[i];
        if (pos4[4 * (size_t)i + 3] != 0.0) continue;
        for (int d = 0; d < 3; ++d) {
            ph[4 * (size_t)i + d] = pos4[4 * (size_t)i + d] + 0.5 * dt * vel4[4 * (size_t)i + d];
            vh[4 * (size_t)i + d] = vel4[4 * (size_t)i + d] + 0.5 * dt * acc[4 * (size_t)i + d];
        }
    }
    if (orc_sph_rates(n, ph, vh, rh, L, periodic, p, 0, acc, dr, dtc)) { dt = -1.0; goto done; }
    for (int i = 0; i < n; ++i) {
        double e = -(dr[i] / rh[i]) * dt;
        rho[i] = rho[i] * (2.0 - e) / (2.0 + e);
        if (pos4[4 * (size_t)i + 3] != 0.0) continue;
        for (int d = 0; d < 3; ++d) {
            double v0 = vel4[4 * (size_t)i + d];
            double v1 = v0 + dt * acc[4 * (size_t)i + d];
            vel4[4 * (size_t)i + d] = v1;
            pos4[4 * (size_t)i + d] += dt * 0.5 * (v1 + v0);
        }
    }
done:
    free(acc); free(dr); free(ph); free(vh); free(rh);
    return dt;
}

/* ------------------------------------------------------------------------ */
/* DEM: the Silbert grain model with Hertzian contacts (Sec. 4.5, Eqs. 9-13) */
/* ------------------------------------------------------------------------ */
/* Readings (the paper states Eqs. 9-13 and defers the rest to its refs):
 *  - n = r_pq / |r_pq| with r_pq = r_p - r_q (minimum image); contact iff
 *    r2 < (2R)^2, i.e. delta = 2R - r > 0 (Eq. 9).
 *  - Relative velocity of the contact points: v_pq = v_p - v_q,
 *    v_n = (v_pq . n) n and v_t = v_pq - v_n - R (w_p + w_q) x n (the surface
 *    points of p and q at the contact move with v_p - R w_p x n and
 *    v_q + R w_q x n).
 *  - Eq. 10 is applied first in a step: u_t = u_t(previous step) + v_t dt,
 *    with u_t = 0 for a contact that is new in this step; a contact that has
 *    ended (delta <= 0) forgets its u_t.
 *  - Eqs. 11-12 with m_eff = m/2 and f = sqrt(delta / 2R).
 *  - Coulomb's law: when |F_t| > mu |F_n|, F_t is scaled to length mu |F_n|
 *    and u_t is set to the value that gives that F_t in Eq. 12,
 *    u_t = -(F_t / f + gt m_eff v_t) / kt.
 *  - Torque on p from the contact: -1/2 r_pq x F_t (with this form the pair
 *    conserves total angular momentum exactly).
 *  - Particles with w != 0 are fixed (walls): they take part in contacts and
 *    receive force and torque sums, but Eq. 13 does not move them.  Eq. 13 adds
 *    gravity: v += dt (F / m + g).
 * History: per particle (in input order) up to ORC_DEM_MAXC contacts, each a
 * partner index and its u_t, in the order the contacts were found. */
#define ORC_DEM_MAXC 32

typedef struct {
    double R, m, I, kn, kt, gn, gt, mu, dt;
    double g[3];
} orc_dem_params;

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double norm3(const double a[3]) { return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

/* One contact of p with q: dv = r_p - r_q, r2 = |dv|^2 < (2R)^2.  Writes the
 * force and torque on p and the contact's new u_t. */
static void dem_contact(const orc_dem_params *P, const double dv[3], double r2, const double *vp, const double *vq,
                        const double *wp, const double *wq, const double u_old[3], double F[3], double T[3],
                        double u_new[3])
{
    const double r = sqrt(r2);
    const double delta = 2.0 * P->R - r; /* Eq. 9 */
    double n[3], vpq[3], w[3], wxn[3], vn[3], vt[3], Fn[3], Ft[3];
    for (int d = 0; d < 3; ++d) {
        n[d] = dv[d] / r;
        vpq[d] = vp[d] - vq[d];
        w[d] = wp[d] + wq[d];
    }
    const double vn_s = vpq[0] * n[0] + vpq[1] * n[1] + vpq[2] * n[2];
    cross3(w, n, wxn);
    for (int d = 0; d < 3; ++d) {
        vn[d] = vn_s * n[d];
        vt[d] = vpq[d] - vn[d] - P->R * wxn[d];
        u_new[d] = u_old[d] + vt[d] * P->dt; /* Eq. 10 */
    }
    const double f = sqrt(delta / (2.0 * P->R));
    const double meff = 0.5 * P->m;
    for (int d = 0; d < 3; ++d) {
        Fn[d] = f * (P->kn * delta * n[d] - P->gn * meff * vn[d]); /* Eq. 11 */
        Ft[d] = f * (-P->kt * u_new[d] - P->gt * meff * vt[d]);   /* Eq. 12 */
    }
    const double fn = norm3(Fn), ft = norm3(Ft);
    if (ft > P->mu * fn) { /* Coulomb */
        const double s = P->mu * fn / ft;
        for (int d = 0; d < 3; ++d) {
            Ft[d] *= s;
            u_new[d] = P->kt > 0.0 ? -(Ft[d] / f + P->gt * meff * vt[d]) / P->kt : 0.0;
        }
    }
    double tq[3];
    cross3(dv, Ft, tq);
    for (int d = 0; d < 3; ++d) {
        F[d] = Fn[d] + Ft[d];
        T[d] = -0.5 * tq[d];
    }
}

/* Contact forces and torques at one state (Eqs. 9-12), with the contact
 * history of the previous step (cnt_in/id_in/u_in, may be NULL for none)
 * turned into that of this step (cnt_out/id_out/u_out).  Contacts are
 * found by a cell list of cell size 2R.  Returns the number of (ordered)
 * contacts, -1 if a particle has more than ORC_DEM_MAXC, -2 on a bad box. */
int64_t orc_dem_forces(int n, const double *pos4, const double *vel4, const double *om4, const double L[3],
                       const int periodic[3], const orc_dem_params *P, const int32_t *cnt_in, const uint32_t *id_in,
                       const double *u_in, double *force4, double *torque4, int32_t *cnt_out, uint32_t *id_out,
                       double *u_out)
{
    orc_cells cl;
    if (cells_build(&cl, n, NULL, pos4, L, periodic, 2.0 * P->R)) return -2;
    const double c2 = (2.0 * P->R) * (2.0 * P->R);
    uint32_t *cand = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    int64_t total = 0;
    int over = 0;
    for (int i = 0; i < n; ++i) {
        double Fs[3] = {0, 0, 0}, Ts[3] = {0, 0, 0};
        int c = 0;
        const int m = stencil_candidates(&cl, periodic, cl.cell[i], cand);
        for (int t = 0; t < m; ++t) {
            const uint32_t j = cand[t];
            if (j == (uint32_t)i) continue;
            double dv[3];
            const double r2 = sep_f64(pos4 + 4 * (size_t)i, pos4 + 4 * (size_t)j, L, periodic, dv);
            if (!(r2 < c2)) continue;
            double u_old[3] = {0, 0, 0}, F[3], T[3], u_new[3];
            if (cnt_in)
                for (int k = 0; k < cnt_in[i]; ++k)
                    if (id_in[(size_t)i * ORC_DEM_MAXC + k] == j)
                        for (int d = 0; d < 3; ++d) u_old[d] = u_in[((size_t)i * ORC_DEM_MAXC + k) * 3 + d];
            dem_contact(P, dv, r2, vel4 + 4 * (size_t)i, vel4 + 4 * (size_t)j, om4 + 4 * (size_t)i,
                        om4 + 4 * (size_t)j, u_old, F, T, u_new);
            for (int d = 0; d < 3; ++d) {
                Fs[d] += F[d];
                Ts[d] += T[d];
            }
            if (c < ORC_DEM_MAXC) {
                id_out[(size_t)i * ORC_DEM_MAXC + c] = j;
                for (int d = 0; d < 3; ++d) u_out[((size_t)i * ORC_DEM_MAXC + c) * 3 + d] = u_new[d];
            } else {
                over = 1;
            }
            ++c;
            ++total;
        }
        cnt_out[i] = c < ORC_DEM_MAXC ? c : ORC_DEM_MAXC;
        for (int d = 0; d < 3; ++d) {
            force4[4 * (size_t)i + d] = Fs[d];
            torque4[4 * (size_t)i + d] = Ts[d];
        }
        force4[4 * (size_t)i + 3] = 0.0;
        torque4[4 * (size_t)i + 3] = 0.0;
    }
    free(cand);
    cells_free(&cl);
    return over ? -1 : total;
}

/* Leapfrog of Eq. 13 for the particles with w == 0: v += dt (F/m + g),
 * r += dt v (the new v), w += dt T / I. */
void orc_dem_leapfrog(int n, double *pos4, double *vel4, double *om4, const double *force4, const double *torque4,
                      const orc_dem_params *P)
{
    for (int i = 0; i < n; ++i) {
        if (pos4[4 * (size_t)i + 3] != 0.0) continue;
        for (int d = 0; d < 3; ++d) {
            const size_t k = 4 * (size_t)i + d;
            vel4[k] = vel4[k] + P->dt * (force4[k] / P->m + P->g[d]);
            pos4[k] = pos4[k] + P->dt * vel4[k];
            om4[k] = om4[k] + P->dt * torque4[k] / P->I;
        }
    }
}

/* nsteps DEM steps (forces of Eqs. 9-12 at the current state, then Eq. 13),
 * carrying the contact history (cnt/id/u, updated in place; start with
 * cnt = 0 for none).  force4/torque4 receive those of the last step.
 * Returns the contacts of the last step, or a negative error of
 * orc_dem_forces. */
int64_t orc_dem_run(int n, int nsteps, double *pos4, double *vel4, double *om4, const double L[3],
                    const int periodic[3], const orc_dem_params *P, int32_t *cnt, uint32_t *id, double *u,
                    double *force4, double *torque4)
{
    const size_t nc = (size_t)(n > 0 ? n : 1) * ORC_DEM_MAXC;
    int32_t *cnt2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    uint32_t *id2 = (uint32_t *)malloc(sizeof(uint32_t) * nc);
    double *u2 = (double *)malloc(sizeof(double) * nc * 3);
    int64_t r = 0;
    for (int s = 0; s < nsteps && r >= 0; ++s) {
        r = orc_dem_forces(n, pos4, vel4, om4, L, periodic, P, cnt, id, u, force4, torque4, cnt2, id2, u2);
        memcpy(cnt, cnt2, sizeof(int32_t) * (size_t)n);
        memcpy(id, id2, sizeof(uint32_t) * nc);
        memcpy(u, u2, sizeof(double) * nc * 3);
        if (r >= 0) orc_dem_leapfrog(n, pos4, vel4, om4, force4, torque4, P);
    }
    free(cnt2);
    free(id2);
    free(u2);
    return r;
}
