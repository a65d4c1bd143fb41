/*
 * fpm.h -- C ABI of libfpm, the GB300 (sm_103a) particle hot path of
 * OpenFPM (arXiv 1804.07598): cell lists, Verlet lists, the Lennard-Jones and
 * SPH pair sweeps, velocity Verlet and the adjoint of the LJ force.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every array argument is a DEVICE pointer owned by the caller (the library
 *    allocates nothing).  The library never frees or retains a pointer after
 *    the call returns.
 *  - Calls are asynchronous on the given stream (0 = the legacy default
 *    stream).  FPM_OK means the arguments were valid and the work was
 *    enqueued; conditions found on the device (neighbour-list overflow, a
 *    particle outside a non-periodic box, a device wait that gave up) are
 *    latched in the caller's fpm_dev_status block, read back by the caller
 *    and turned into a status by fpm_status_from_device().
 *  - Host-side argument errors return FPM_ERR_INVALID (or FPM_ERR_WORKSPACE)
 *    and enqueue nothing; a failed launch returns FPM_ERR_CUDA.  The text of
 *    the last error of the calling thread is returned by fpm_last_error().
 *  - No call synchronises the device, allocates, or touches host memory other
 *    than its by-value / by-pointer host arguments, so every call may be
 *    captured into a CUDA graph.
 *  - Particle arrays are 4-vectors: FPM_F32 -> float4 (16 B, 16-B aligned),
 *    FPM_F64 -> double4 (32 B, 32-B aligned), component w unused on input
 *    unless stated.  Positions
 *    live in the box [0,L0) x [0,L1) x [0,L2); mass is 1 (reduced units).
 *  - A Verlet list is an object in caller memory (fpm_verlet_list_bytes):
 *    per-tile descriptors followed by 16-bit entries laid out column-major
 *    (entry k of particle i in word (k/2)*ld + i, ld = fpm_nbr_ld(n)), so
 *    that consecutive particles read consecutive words.  Entries index the
 *    tile's staged neighbourhood, not particles; fpm_verlet_decode turns a
 *    list into particle indices.
 */
#ifndef FPM_H
#define FPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque CUDA stream (a cudaStream_t / CUstream). */
typedef struct CUstream_st *fpm_stream;

typedef enum {
    FPM_OK = 0,
    FPM_ERR_INVALID = 1,   /* bad argument; nothing enqueued                     */
    FPM_ERR_CAPACITY = 2,  /* a neighbour list needed more than `cap` entries    */
    FPM_ERR_DOMAIN = 3,    /* a particle lay outside a non-periodic dimension    */
    FPM_ERR_CUDA = 4,      /* CUDA launch / runtime error                        */
    FPM_ERR_TIMEOUT = 5,   /* a bounded device wait gave up                      */
    FPM_ERR_WORKSPACE = 6  /* workspace pointer null or smaller than required    */
} fpm_status;

typedef enum { FPM_F32 = 0, FPM_F64 = 1 } fpm_prec;

/* The simulation domain: the paper's Box and per-dimension boundary
 * conditions (Listing 4.1, Sec. 4.1: Box<3> + bc[3] = {PERIODIC,...}).
 * The box starts at the origin; a periodic dimension requires
 * L > 2 * r_cell * (1 + 2^-10) for the cutoff r_cell it is used with. */
typedef struct {
    double L[3];
    int32_t periodic[3];
} fpm_box;

/* Cell grid of a cell list (Sec. 2 "Cell Lists [45]"; getCellListSym,
 * Listing 4.1).  nc[d] = floor(L[d] / (r_cell * (1 + 2^-12))), forced to 1 in
 * a periodic dimension where it would be < 3 (every particle of that
 * dimension is then a candidate); inv[d] = (float)(nc[d] / L[d]).
 * tiles_x: the pair sweeps work on tiles of consecutive cells along x; each
 * row of nc[0] cells is split into tiles_x tiles of near-equal width (at most
 * 14 cells).  ntiles = tiles_x * nc[1] * nc[2].
 * stage_cap: particles of a tile's neighbourhood that a sweep stages in shared
 * memory (0: estimated from the mean density).  A tile with a larger
 * neighbourhood is still computed correctly, reading neighbours from global
 * memory, and counted in fpm_dev_status.spilled; fpm_dev_status.max_staged
 * after a Verlet build tells the caller what to set.
 * sweep_blocks: blocks of the tile sweeps (Verlet scan, LJ, SPH, adjoint),
 * which take tiles by ticket: 0 = as many as fit on the GPU at once, > 0 =
 * that many, -1 = one block per tile.  A launch-shape choice only: results
 * do not depend on it. */
typedef struct {
    int32_t nc[3];
    int32_t ncell;
    float inv[3];
    int32_t tiles_x;
    int32_t stage_cap;
    int32_t sweep_blocks;
} fpm_grid;

/* Device-side status block (caller-allocated in device memory, 64 bytes,
 * zero-filled before first use).  Written by the kernels with atomics. */
typedef struct {
    uint32_t flags;        /* bit 0 capacity, bit 1 domain, bit 2 timeout        */
    uint32_t max_nn;       /* largest neighbour count seen by a Verlet build      */
    uint32_t rebuild;      /* 1 after fpm_verlet_check found a displacement > skin/2 */
    uint32_t nrebuild;     /* number of gated rebuilds performed                  */
    uint32_t max_disp2;    /* float bits of the largest squared displacement      */
    uint32_t bad_index;    /* a particle index that raised FPM_ERR_DOMAIN         */
    uint32_t max_staged;   /* largest tile neighbourhood seen by a Verlet build   */
    uint32_t spilled;      /* tile sweeps whose neighbourhood exceeded stage_cap  */
    uint32_t reserved[8];
} fpm_dev_status;

#define FPM_FLAG_CAPACITY 1u
#define FPM_FLAG_DOMAIN 2u
#define FPM_FLAG_TIMEOUT 4u

/* ------------------------------------------------------------------ */
/* Errors and helpers (host only)                                       */
/* ------------------------------------------------------------------ */

/* Static text of a status code. */
const char *fpm_status_string(fpm_status s);

/* Text of the last error raised on the calling thread ("" if none). */
const char *fpm_last_error(void);

/* Maps a host copy of the device status block to the first latched error
 * (CAPACITY, then DOMAIN, then TIMEOUT) or FPM_OK. */
fpm_status fpm_status_from_device(const fpm_dev_status *host_copy);

/* Leading dimension of an ELL neighbour list for n particles:
 * (n + 31) rounded down to a multiple of 32. */
int64_t fpm_nbr_ld(int32_t n);

/* A branch decided on the device inside a CUDA graph being captured on
 * `stream`: fpm_graph_if_begin adds a conditional (IF) node, whose body runs
 * in a replay only when *d_flag != 0 at that point of the replay, and starts
 * capturing that body on `body_stream` (a different stream, not capturing);
 * the caller enqueues the conditional work on body_stream and then calls
 * fpm_graph_if_end(body_stream).  Work enqueued on `stream` afterwards runs
 * after the conditional node.  When `stream` is not capturing, *capturing is
 * set to 0 and nothing is added (the caller enqueues the work on `stream`,
 * gated by the same flag).  Used for the Verlet rebuild of a step, so that a
 * step without a rebuild does not launch the rebuild kernels. */
fpm_status fpm_graph_if_begin(const uint32_t *d_flag, fpm_stream stream, fpm_stream body_stream, int32_t *capturing);
fpm_status fpm_graph_if_end(fpm_stream body_stream);

/* Cell grid for cutoff r_cell in box (see fpm_grid).  Host only.  n_hint,
 * the expected particle count (<= 0: unknown), only sets the tile width:
 * about 200 particles per tile, i.e. round(200 ncell / n_hint) cells.
 * FPM_ERR_INVALID if r_cell <= 0, a length <= 0, a periodic length below
 * 2 r_cell (1 + 2^-10) or more than 2^24 cells. */
fpm_status fpm_grid_make(const fpm_box *box, double r_cell, int32_t n_hint, fpm_grid *out);

/* ------------------------------------------------------------------ */
/* Cell list (Sec. 2, cell lists [45]; Sec. 3.6, cache-friendly         */
/* re-sorting; getCellListSym / updateCellListSym, Listing 4.1)         */
/* ------------------------------------------------------------------ */

/* Bytes of device workspace fpm_celllist_build needs for n particles on the
 * given grid at precision prec (16-byte aligned base required). */
fpm_status fpm_celllist_workspace(int32_t n, const fpm_grid *grid, fpm_prec prec, size_t *bytes);

/* Builds the cell list of n particles:
 *   1. wrap every periodic coordinate into [0,L) (one correction step),
 *   2. cell coordinate ci = min((int)((float)x * inv), nc-1) per dimension,
 *      linear cell id (cz*ncy + cy)*ncx + cx,
 *   3. stable counting sort by cell (ties keep the input order),
 *   4. exclusive scan of the cell counts into cell_start[ncell+1],
 *   5. reorder: pos_out[k] = wrapped pos_in[perm[k]], vel_out[k] =
 *      vel_in[perm[k]], id_out[k] = id_in[perm[k]] (or perm[k] when id_in is
 *      NULL).
 * pos_in/pos_out : [n] float4|double4; may alias (in-place reorder).
 * vel_in/vel_out : [n] float4|double4 or both NULL; may alias.
 * id_in          : [n] uint32 or NULL; id_out : [n] uint32 or NULL; may alias.
 * cell_start     : [grid->ncell + 1] uint32 (output).
 * perm           : [n] uint32 (output), input index of sorted slot k.
 * workspace      : >= fpm_celllist_workspace() bytes, contents need no init.
 * d_status       : device status block or NULL; FPM_FLAG_DOMAIN is latched
 *                  (and the particle binned into the nearest cell) for a
 *                  particle outside a non-periodic dimension.
 * d_gate         : NULL, or a device word; when it holds 0 at run time every
 *                  kernel of the call returns at once (device-gated rebuild).
 * Deterministic: identical inputs give bit-identical outputs. */
fpm_status fpm_celllist_build(const fpm_box *box, const fpm_grid *grid, int32_t n, fpm_prec prec,
                              const void *pos_in, const void *vel_in, const uint32_t *id_in,
                              void *pos_out, void *vel_out, uint32_t *id_out,
                              uint32_t *cell_start, uint32_t *perm,
                              void *workspace, size_t workspace_bytes,
                              fpm_dev_status *d_status, const uint32_t *d_gate, fpm_stream stream);

/* Gathers a per-particle property into sorted order: dst[k] = src[perm[k]],
 * elem_bytes in {4, 8, 16, 32}; src and dst must not alias. */
fpm_status fpm_reorder(int32_t n, int32_t elem_bytes, const uint32_t *perm, const void *src, void *dst,
                       const uint32_t *d_gate, fpm_stream stream);

/* ------------------------------------------------------------------ */
/* Verlet lists (Sec. 2, Verlet lists [46]; Sec. 4.1)                   */
/* ------------------------------------------------------------------ */

/* Bytes of the Verlet-list object for n particles, grid and capacity cap
 * (entries per particle).  The object must be 256-byte aligned. */
fpm_status fpm_verlet_list_bytes(int32_t n, const fpm_grid *grid, int32_t cap, size_t *bytes);

/* Full Verlet list of n particles sorted by fpm_celllist_build on a grid
 * made with r_cell >= r_list, positions unchanged since: for every i, every
 * j != i of the 27 (or fewer) neighbouring cells with r2 < (T)(r_list^2),
 * where per periodic dimension d = x_i - x_j, replaced by (x_i - L) - x_j
 * when j is seen through the upper wall and by x_i - (x_j - L) through the
 * lower wall (the exact image shift first, then one rounded subtraction),
 * and r2 = fma(dz,dz, fma(dy,dy, dx*dx)), all in the positions' precision.
 * (The image is chosen by the cell stencil; for every pair inside r_list it
 * is the minimum image.)
 * pos     : [n] sorted positions.     cell_start : [ncell+1].
 * cap     : entries reserved per particle.
 * list    : fpm_verlet_list_bytes() bytes, written.  nn : [n] uint32, the
 *           number of stored entries (min(count, cap)).  A count above cap
 *           latches FPM_FLAG_CAPACITY (so does a tile neighbourhood of more
 *           than 65535 particles, whose particles then get nn = 0);
 *           d_status->max_nn receives the largest count.
 * pos_ref : [n] (same type as pos) receives pos, the reference positions of
 *           the displacement test (may be NULL).
 * d_gate  : as in fpm_celllist_build.  After a gated build the gate word is
 *           cleared and d_status->nrebuild incremented.
 * Until the next build the positions may move but must not be wrapped: the
 * image of every listed pair is fixed by the build. */
fpm_status fpm_verlet_build(const fpm_box *box, const fpm_grid *grid, int32_t n, fpm_prec prec,
                            const void *pos, const uint32_t *cell_start, double r_list, int32_t cap,
                            void *list, size_t list_bytes, uint32_t *nn, void *pos_ref,
                            fpm_dev_status *d_status, uint32_t *d_gate, fpm_stream stream);

/* fpm_verlet_build for the symmetric sweep (fpm_lj_forces_half): a half list
 * that holds each pair {i, j} with r2 < (T)(r_list^2) once, in the list of
 * the particle whose cell comes first in the half stencil: the cells
 * (dz, dy, dx) lexicographically after (0, 0, 0), and in the particle's own
 * cell the particles after it in the sorted order (the cell list of
 * getCellListSym, Listing 4.1).  A tile stages its own row and the four rows
 * after it, each piece of the staging at an offset of the parity of its
 * first particle index (free slots between pieces belong to no particle).
 * Same arguments, layout and errors as fpm_verlet_build; about half the
 * entries, so cap can be about half. */
fpm_status fpm_verlet_build_half(const fpm_box *box, const fpm_grid *grid, int32_t n, fpm_prec prec, const void *pos,
                                 const uint32_t *cell_start, double r_list, int32_t cap, void *list,
                                 size_t list_bytes, uint32_t *nn, void *pos_ref, fpm_dev_status *d_status,
                                 uint32_t *d_gate, fpm_stream stream);

/* Particle indices of a Verlet list: out[k*ld + i] = j for k < nn[i]
 * (out : [cap * fpm_nbr_ld(n)] uint32; other slots untouched).  The order of
 * entries within a list is not part of the contract; the set is. */
fpm_status fpm_verlet_decode(const fpm_grid *grid, int32_t n, int32_t cap, const void *list,
                             const uint32_t *nn, uint32_t *out, fpm_stream stream);

/* Verlet rebuild test: sets d_status->rebuild = 1 when some particle moved
 * (minimum image) by more than skin/2 since pos_ref, judged in the
 * positions' precision as d2 > (T)(skin^2 / 4); d_status->max_disp2 receives
 * the largest d2 (atomic max; as float bits).  Never clears the flag. */
fpm_status fpm_verlet_check(const fpm_box *box, int32_t n, fpm_prec prec, const void *pos,
                            const void *pos_ref, double skin, fpm_dev_status *d_status,
                            fpm_stream stream);

/* ------------------------------------------------------------------ */
/* Lennard-Jones pair sweep (Sec. 4.1: V(r) = 4 eps[(s/r)^12 - (s/r)^6],  */
/* pair force 24 eps (2 s^12 / r^14 - s^6 / r^8) (x_p - x_q) of           */
/* Listing 4.1, truncated at r_cut, applied over the Verlet list)          */
/* ------------------------------------------------------------------ */

/* Bytes of workspace for the tile sweeps (fpm_lj_forces, fpm_lj_backward,
 * fpm_sph_forces: tile-scheduling counters and per-tile FP64 partial sums)
 * and for fpm_kinetic (per-block partial sums), for n particles on grid (grid
 * may be NULL for fpm_kinetic alone).  The workspace must be ZERO-FILLED once
 * before its first use; every call leaves its counters at zero again.  Calls
 * sharing a workspace must not run concurrently. */
fpm_status fpm_reduce_workspace(int32_t n, const fpm_grid *grid, size_t *bytes);

/* Forces of the truncated (unshifted) LJ potential over the full Verlet
 * list: F_i = sum_j 24 eps (2 s^12/r^14 - s^6/r^8) (x_i - x_j) over entries
 * with r2 < (T)(rc^2) (separation and r2 as in fpm_verlet_build).  Pair
 * arithmetic and the per-particle accumulation run in the positions'
 * precision.  box, grid, cap, list and nn as given to fpm_verlet_build.
 * force     : [n] float4|double4; w = 1/2 sum_j V(r_ij), the particle's share
 *             of the potential energy.
 * d_energy  : [3] double: U = sum_{i<j} V, W = sum_{i<j} r_ij . F_ij and
 *             the number of interacting pairs.  Reduced in FP64 in a fixed
 *             order (bit-reproducible).  May be NULL (no reduction).
 *             With n == 0 it receives zeros and nothing is launched.
 * workspace : fpm_reduce_workspace(n, grid) bytes (zero-filled once; always
 *             needed: it holds the sweep's tile-scheduling counters).
 * d_status  : device status block or NULL; FPM_FLAG_TIMEOUT is latched if a
 *             tile's bulk copy into shared memory did not complete within
 *             about 2 s (its particles' forces are then not written). */
fpm_status fpm_lj_forces(const fpm_box *box, const fpm_grid *grid, int32_t n, fpm_prec prec, const void *pos,
                         const void *list, const uint32_t *nn, int32_t cap,
                         double eps, double sigma, double rc,
                         void *force, double *d_energy, void *workspace, size_t workspace_bytes,
                         fpm_dev_status *d_status, fpm_stream stream);

/* fpm_lj_forces and the closing half-kick of velocity Verlet (Listing 4.1's
 * time loop) in one launch: after F_i is written, vel[i] += dt/2 F_i, with
 * the arithmetic of fpm_vv_step(half = 1), so the result is bit-identical to
 * fpm_lj_forces followed by fpm_vv_step(half = 1) on the same stream.
 * vel : [n] float4|double4 (same type as pos), updated; w kept.  It must not
 *       alias pos or force.  Other arguments and results as fpm_lj_forces. */
fpm_status fpm_lj_forces_kick(const fpm_box *box, const fpm_grid *grid, int32_t n, fpm_prec prec, const void *pos,
                              const void *list, const uint32_t *nn, int32_t cap,
                              double eps, double sigma, double rc,
                              void *force, double *d_energy, void *workspace, size_t workspace_bytes,
                              fpm_dev_status *d_status, void *vel, double dt, fpm_stream stream);

/* fpm_lj_forces without a workspace argument, for callers that cannot
 * allocate device memory at all: a host program whose device memory is owned
 * by another runtime or a fixed pool it must not grow, or a real-time loop in
 * which the implicit synchronisation of cudaMalloc is not acceptable.  (The
 * paper has no counterpart; this is a deployment convenience.)
 * Same arguments and results as fpm_lj_forces.  The energy reduction uses a
 * scratch array compiled into the library (4 MiB + 256 B of device memory on
 * every GPU that loads it, held until the process exits), which limits n to
 * 2^24 = 16,777,216 particles and the grid to 65,536 tiles; larger sizes
 * return FPM_ERR_INVALID.  The call allocates and frees nothing.
 * - The first call on each device looks the scratch address up (with that
 *   device current); make that first call before any stream capture.
 * - Every call uses the scratch, with or without d_energy: it clears the
 *   tile-scheduling counters held there (on `stream`), its blocks take their
 *   tiles from those counters, and with d_energy it keeps the per-tile
 *   energy partial sums there too.  All calls on a device share the one
 *   array, which keeps whatever the last call left in it.
 * - Calls that may run at the same time on the GPU (different streams, or
 *   graphs replayed concurrently) race on that array: one call's blocks can
 *   take another call's tiles, or its clear can reset counters still in
 *   use, so forces can come out wrong or unwritten, not only energies.
 *   Serialise such calls. */
fpm_status fpm_lj_forces_noalloc(const fpm_box *box, const fpm_grid *grid, int32_t n, fpm_prec prec,
                                 const void *pos, const void *list, const uint32_t *nn, int32_t cap,
                                 double eps, double sigma, double rc,
                                 void *force, double *d_energy, fpm_dev_status *d_status, fpm_stream stream);

/* The symmetric sweep of Sec. 4.1 (each pair once, the force applied to both
 * particles, the reactions summed back as Sec. 3.4's ghost_put with a sum
 * does), single precision, over a half list from fpm_verlet_build_half:
 *   F_i = sum over pairs {i, j} with r2 < (float)(rc^2) of
 *         24 eps (2 s^12/r^14 - s^6/r^8) (x_i - x_j),
 * the same forces as fpm_lj_forces up to rounding.  Each home particle's own
 * sum runs in FP32; every contribution is then added as a 64-bit fixed-point
 * integer (units of 2^-32 of force), so the result does not depend on the
 * order of the additions: bit-reproducible.
 * force    : [n] float4, w = 0 (the per-particle energy share is not formed).
 * d_energy : [3] double, U, W and the pair count as fpm_lj_forces, or NULL.
 * acc      : fpm_lj_half_acc_bytes(n) bytes, 16-byte aligned, ZERO-FILLED
 *            before the first call; every call leaves it zero again.
 * workspace: fpm_reduce_workspace(n, grid) bytes, as fpm_lj_forces.
 * vel      : NULL, or [n] float4 receiving the closing half-kick
 *            v += dt/2 F (as fpm_lj_forces_kick).
 * Two launches on `stream`.  Single precision only (the fixed-point unit
 * 2^-32 is far below FP32 rounding of forces, not below FP64's). */
fpm_status fpm_lj_forces_half(const fpm_box *box, const fpm_grid *grid, int32_t n, const void *pos, const void *list,
                              const uint32_t *nn, int32_t cap, double eps, double sigma, double rc, void *force,
                              double *d_energy, void *acc, size_t acc_bytes, void *workspace, size_t workspace_bytes,
                              fpm_dev_status *d_status, void *vel, double dt, fpm_stream stream);

/* Bytes of the fixed-point array of fpm_lj_forces_half: three int64 per
 * particle, n rounded up to even. */
fpm_status fpm_lj_half_acc_bytes(int32_t n, size_t *bytes);

/* Test hook (the paper has no counterpart): the budget, in SM clock cycles,
 * of the first bounded wait per tile of the force sweeps of fpm_lj_forces,
 * fpm_lj_forces_kick and fpm_lj_forces_noalloc launched after the call, from
 * any thread (the wait for the tile's neighbourhood to land in shared
 * memory).  cycles <= 0 restores the default of about 2 s.  A short budget
 * drives the expiry path that a stalled copy would take: FPM_FLAG_TIMEOUT is
 * latched in d_status (fpm_status_from_device gives FPM_ERR_TIMEOUT); the
 * kernel then waits for the copies with the full budget, so that none is
 * still in flight when it exits, and sweeps the tile if they have landed
 * (a tile whose copies never land is not swept: its forces are not
 * written).  The other waits keep their budget. */
fpm_status fpm_test_wait_budget(int64_t cycles);

/* ------------------------------------------------------------------ */
/* Velocity Verlet (Listing 4.1 time loop: v += dt/2 F; x += dt v; ...;   */
/* v += dt/2 F), unit mass                                                */
/* ------------------------------------------------------------------ */

/* half = 0: v += dt/2 F; x += dt v.  Positions are not wrapped here (a
 * Verlet list fixes the periodic image of each pair until the next build);
 * fpm_celllist_build wraps them.
 * half = 1: v += dt/2 F.  pos is untouched when half = 1 (may be NULL). */
fpm_status fpm_vv_step(const fpm_box *box, int32_t n, fpm_prec prec, int32_t half, double dt,
                       void *pos, void *vel, const void *force, fpm_stream stream);

/* fpm_vv_step(half = 0) followed by fpm_verlet_check on the new positions,
 * in one pass over the particles (same results as the two calls). */
fpm_status fpm_vv_drift_check(const fpm_box *box, int32_t n, fpm_prec prec, double dt, void *pos, void *vel,
                              const void *force, const void *pos_ref, double skin, fpm_dev_status *d_status,
                              fpm_stream stream);

/* Transfers in the host's layout: packed (x, y, z) triples (float or double
 * [3n]) to and from the 4-vector state (float4|double4 [n], device memory).
 * unpack writes x, y, z of dst4 and keeps its w; pack writes 3n values.
 * With these, an end-to-end step moves 12 (24) bytes per vector across the
 * host link instead of 16 (32).  The packed array may be device memory or
 * page-locked host memory mapped into the device's address space (what
 * cudaHostAlloc gives under unified addressing): the kernel then reads or
 * writes the host's buffer directly across the host link, with no separate
 * copy.  Single precision with a 16-byte aligned packed array moves four
 * particles per thread in 16-byte words. */
fpm_status fpm_unpack_xyz(int32_t n, fpm_prec prec, const void *src_xyz, void *dst4, fpm_stream stream);
fpm_status fpm_pack_xyz(int32_t n, fpm_prec prec, const void *src4, void *dst_xyz, fpm_stream stream);

/* Kinetic energy and momentum in FP64 (fixed-order, bit-reproducible):
 * d_out[0] = 1/2 sum |v|^2, d_out[1..3] = sum v. */
fpm_status fpm_kinetic(int32_t n, fpm_prec prec, const void *vel, double *d_out,
                       void *workspace, size_t workspace_bytes, fpm_stream stream);

/* ------------------------------------------------------------------ */
/* Weakly compressible SPH (Sec. 4.2, Eqs. 1-5), single precision        */
/* ------------------------------------------------------------------ */

/* SPH constants.  kernel 0: Wendland C2, W = a (1-q/2)^4 (2q+1),
 * a = 21/(16 pi h^3); kernel 1: cubic spline, s [1 - 1.5q^2 + 0.75q^3] for
 * q < 1, s 0.25 (2-q)^3 for q < 2, s = 1/(pi h^3); q = r/h, support 2h.
 * Tait EOS P = b[(rho/rho0)^gamma - 1], b = c0^2 rho0 / gamma (Eqs. 3-4;
 * gamma an integer in [1,8]); artificial viscosity alpha, eta2 (Eq. 5);
 * gravity g. */
typedef struct {
    double h, mass, rho0, c0, gamma, alpha, eta2, g[3];
    int32_t kernel;
} fpm_sph_params;

/* Rates of Eqs. 1-2 over a Verlet list built with r_list >= 2h (same box,
 * grid, list, nn, cap conventions as fpm_lj_forces):
 *   pos : [n] float4 (x, y, z, type), type 0 fluid, 1 fixed boundary particle;
 *   vr  : [n] float4 (vx, vy, vz, rho - rho0);
 *   acc : [n] float4 (ax, ay, az, Drho/Dt): for each pair inside 2h,
 *         grad_p W = (dW/dr)(x_p - x_q)/r, Drho_p += m (v_p - v_q).grad_p W,
 *         a_p += -m [(P_p+P_q)/(rho_p rho_q) + Pi_pq] grad_p W with
 *         Pi_pq = -alpha c0 mu / ((rho_p+rho_q)/2) when (v_p-v_q).(x_p-x_q) < 0,
 *         mu = h (v_p-v_q).(x_p-x_q) / (r^2 + eta2); fluid: a += g;
 *         boundary: a = 0 (Drho still computed).
 *   d_dtcons : [2] float, raised (atomic max) to max |a| over fluid particles
 *         and max |mu| over pairs; must hold 0 (or smaller values) on entry
 *         (fpm_sph_predict / fpm_sph_correct clear the buffers they consume).
 * The pressure is evaluated from rho - rho0 by the binomial expansion of
 * (1+x)^gamma - 1 (no cancellation in single precision).
 * workspace : fpm_reduce_workspace(n, grid) bytes, zero-filled once (it holds
 *             the tile-scheduling counters of the sweep). */
fpm_status fpm_sph_forces(const fpm_box *box, const fpm_grid *grid, int32_t n, const void *pos, const void *vr,
                          const void *list, const uint32_t *nn, int32_t cap, const fpm_sph_params *params,
                          void *acc, float *d_dtcons, void *workspace, size_t workspace_bytes,
                          fpm_dev_status *d_status, fpm_stream stream);

/* Density by summation over the kernel of Sec. 4.2 (the SPH estimate
 * rho_i = sum_j m W(|x_i - x_j|), the particle itself included, that Eqs. 1-2
 * differentiate; a variant of evolving rho by Eq. 2):
 *   rho[i] = m W(0) + sum over list entries with r2 < (2h)^2 of m W(r),
 * W as in fpm_sph_params (kernel 0 Wendland C2, 1 cubic spline), r2 and the
 * support test in single precision as in fpm_sph_forces.  Every particle
 * (fluid and boundary) sums over every neighbour.  Same box, grid, list, nn,
 * cap, workspace and status conventions as fpm_sph_forces; the list must be
 * built with r_list >= 2h.
 * rho : [n] float, the summed density of each particle (sorted order). */
fpm_status fpm_sph_density(const fpm_box *box, const fpm_grid *grid, int32_t n, const void *pos, const void *list,
                           const uint32_t *nn, int32_t cap, const fpm_sph_params *params, float *rho,
                           void *workspace, size_t workspace_bytes, fpm_dev_status *d_status, fpm_stream stream);

/* Symplectic predictor (the "Verlet time-stepping with dynamic step size" of
 * Sec. 4.2, read as the predictor-corrector of the DualSPHysics scheme):
 *   dt = cfl min( sqrt(h / max|a|), h / (c0 + max|mu|) ) from d_dtcons (the
 *   rates at t^n), written to d_dt[0];
 *   pos_h = pos + dt/2 v, vr_h.xyz = v + dt/2 a (fluid; boundary unchanged),
 *   vr_h.w = (rho - rho0) + dt/2 Drho (all);  d_dtcons_h[0..1] = 0.
 * With pos_ref, the displacement test of fpm_verlet_check runs on pos_h. */
fpm_status fpm_sph_predict(const fpm_box *box, int32_t n, const fpm_sph_params *params, double cfl,
                           const void *pos, const void *vr, const void *acc, const float *d_dtcons,
                           void *pos_h, void *vr_h, float *d_dt, float *d_dtcons_h,
                           const void *pos_ref, double skin, fpm_dev_status *d_status, fpm_stream stream);

/* Symplectic corrector with the rates at the half step (acc_h):
 *   v1 = v0 + dt a, x1 = x0 + dt (v0 + v1)/2 (fluid only),
 *   rho1 = rho0 (2 - e)/(2 + e) with e = -(Drho / rho_half) dt (all), in place
 *   on pos, vr; d_dtcons[0..1] = 0.  With pos_ref, sets d_status->rebuild when
 *   |x1 - x_ref| + dt |v1| > skin/2 (room for the next half step).  With
 *   d_time (optional, one double), *d_time += dt: the simulated time. */
fpm_status fpm_sph_correct(const fpm_box *box, int32_t n, const fpm_sph_params *params, void *pos, void *vr,
                           const void *vr_h, const void *acc_h, const float *d_dt, float *d_dtcons,
                           const void *pos_ref, double skin, fpm_dev_status *d_status, double *d_time,
                           fpm_stream stream);

/* ------------------------------------------------------------------ */
/* DEM: the Silbert grain model with Hertzian contacts (Sec. 4.5,        */
/* Eqs. 9-13).  FP32 state, float4 arrays in the sorted order.            */
/* ------------------------------------------------------------------ */

/* R: particle radius (contact iff r < 2R, delta = 2R - r, Eq. 9); m, I:
 * mass and moment of inertia of every particle; kn, kt, gn, gt: the elastic
 * and damping constants of Eqs. 11-12 (m_eff = m/2); mu: Coulomb friction
 * coefficient; dt: time step (Eqs. 10, 13); g: gravity (Eq. 13). */
typedef struct {
    double R, m, I, kn, kt, gn, gt, mu, dt, g[3];
} fpm_dem_params;

/* Contact forces and torques over a Verlet list built with r_list >= 2R
 * (box, grid, list, nn, cap as for fpm_lj_forces), float4 [n] arrays:
 *   pos (x, y, z, type): type 0 moving grain, nonzero fixed (wall) grain;
 *   vel (vx, vy, vz, -), omega (wx, wy, wz, -);
 *   force, torque (output, w = 0): for every list entry inside 2R, with
 *   n = (x_p - x_q)/r, v_pq = v_p - v_q, v_n = (v_pq.n) n and the
 *   contact-point velocity v_t = v_pq - v_n - R (w_p + w_q) x n:
 *     u_t += v_t dt (Eq. 10; u_t from the entry's history),
 *     F_n = f (kn delta n - gn m_eff v_n), F_t = f (-kt u_t - gt m_eff v_t),
 *     f = sqrt(delta / 2R) (Eqs. 11-12); if |F_t| > mu |F_n| then F_t is
 *     scaled to mu |F_n| and u_t = -(F_t/f + gt m_eff v_t)/kt (Coulomb);
 *     force_p += F_n + F_t, torque_p += -1/2 (x_p - x_q) x F_t.
 *   hist : float4 [cap * fpm_nbr_ld(n)], entry k of particle i at
 *     k * ld + i: the tangential deformation (x, y, z, -) of that list entry,
 *     read and rewritten by every call (0 for an entry not in contact; zero
 *     it after a Verlet build that is not followed by fpm_dem_hist_unpack).
 *   d_ncontact : optional uint32 [1], incremented by the number of (ordered)
 *     contacts.
 * workspace : fpm_reduce_workspace(n, grid) bytes, zero-filled once. */
fpm_status fpm_dem_forces(const fpm_box *box, const fpm_grid *grid, int32_t n, const void *pos, const void *vel,
                          const void *omega, const void *list, const uint32_t *nn, int32_t cap,
                          const fpm_dem_params *params, void *hist, void *force, void *torque,
                          uint32_t *d_ncontact, void *workspace, size_t workspace_bytes, fpm_dev_status *d_status,
                          fpm_stream stream);

/* Leapfrog of Eq. 13 for grains of type 0 (in place):
 *   v += dt (force/m + g), x += dt v (the new v), w += dt torque / I.
 * With pos_ref, sets d_status->rebuild when a grain moved (minimum image)
 * by more than skin/2 since pos_ref (as fpm_verlet_check). */
fpm_status fpm_dem_leapfrog(const fpm_box *box, int32_t n, const fpm_dem_params *params, void *pos, void *vel,
                            void *omega, const void *force, const void *torque, const void *pos_ref, double skin,
                            fpm_dev_status *d_status, fpm_stream stream);

/* The DEM state across a Verlet rebuild: the contacts' u_t follow their
 * particle pairs, and omega follows its particle, through the cell-list
 * reorder.  A rebuild is
 *   fpm_dem_rebuild_begin -> fpm_celllist_build (pos, vel, ids) ->
 *   fpm_verlet_build -> fpm_dem_rebuild_end,
 * all gated by the same rebuild flag (the Verlet build clears it; `pending`,
 * a caller-owned device uint32 that starts at 0, carries it to the end call).
 * Bytes of the `packed` buffer (device memory, no initialisation needed): */
size_t fpm_dem_packed_bytes(int32_t n);

/* Runs only when *d_gate != 0 (always when d_gate is NULL), and then sets
 * *d_pending = 1.  For every particle i (current order) the list entries with
 * nonzero u_t are saved in `packed` as (partner's current index, u_t), at most
 * 16 per particle (more latches FPM_FLAG_CAPACITY in d_status and drops the
 * rest), and omega is saved.  list, nn, cap, grid: the list that hist
 * belongs to. */
fpm_status fpm_dem_rebuild_begin(const fpm_grid *grid, int32_t n, int32_t cap, const void *list, const uint32_t *nn,
                                 const void *hist, const void *omega, void *packed, const uint32_t *d_gate,
                                 uint32_t *d_pending, fpm_dev_status *d_status, fpm_stream stream);

/* Runs only when *d_pending != 0, and clears it.  With perm from the
 * rebuild's fpm_celllist_build (new index -> previous index) and the new
 * list: omega[i] = saved omega[perm[i]], and hist entry k of new particle i
 * receives the saved u_t of the pair (perm[i], perm[j]), j that entry's
 * partner, or 0 when the pair had none. */
fpm_status fpm_dem_rebuild_end(const fpm_grid *grid, int32_t n, int32_t cap, const void *list, const uint32_t *nn,
                               const uint32_t *perm, const void *packed, void *hist, void *omega,
                               uint32_t *d_pending, fpm_stream stream);

/* ------------------------------------------------------------------ */
/* Particle-mesh interpolation with the moment-conserving M'4 kernel     */
/* (Sec. 4.4: the vortex method's particle-to-mesh and mesh-to-particle  */
/* interpolations).  FP32.                                                */
/* ------------------------------------------------------------------ */
/* Mesh: N[d] nodes per dimension at x = i L_d / N_d, periodic in every
 * dimension; node (i, j, k) at index (k N1 + j) N0 + i of a float4 array.  A
 * particle with s = x N / L in cell c = floor(s) touches the nodes
 * c - 1 .. c + 2 (mod N) with weight prod_d M'4(s_d - node_d), M'4(x) =
 * 1 - 5/2 x^2 + 3/2 |x|^3 (|x| < 1), (2 - |x|)^2 (1 - |x|)/2 (1 <= |x| < 2),
 * 0 beyond. */

/* The cell grid whose cells are the mesh cells (nc = N), for binning the
 * particles with fpm_celllist_build before fpm_p2m.  Host only.
 * FPM_ERR_INVALID unless N[d] >= 3 and the box is periodic in every
 * dimension, or for more than 2^24 nodes. */
fpm_status fpm_mesh_grid(const fpm_box *box, const int32_t N[3], fpm_grid *out);

/* mesh[node] = sum_p val_p W(x_node - x_p) (every node written).  pos and
 * val : float4 [n] binned by mesh cell, with cell_start, by
 * fpm_celllist_build(box, mesh_grid, ...) (val as its vel); w of val is
 * interpolated like x, y, z.  A gather over each node's 4x4x4 cells:
 * deterministic, no atomics.  A node tile whose cells hold more particles
 * than the staging room reads them from global memory (counted in
 * d_status->spilled when d_status is given). */
fpm_status fpm_p2m(const fpm_box *box, const fpm_grid *mesh_grid, int32_t n, const void *pos, const void *val,
                   const uint32_t *cell_start, void *mesh, fpm_dev_status *d_status, fpm_stream stream);

/* val[p] = sum_nodes mesh[node] W(x_node - x_p), float4 [n]; pos in any
 * order (wrapped into the box as the cell-list build does).  order
 * (optional, a permutation of 0..n-1, e.g. the perm of the binning of the
 * same positions): the particles are taken in that order, which only
 * changes speed (neighbouring threads share nodes); each val[p] is the same. */
fpm_status fpm_m2p(const fpm_box *box, const fpm_grid *mesh_grid, int32_t n, const void *pos, const void *mesh,
                   const uint32_t *order, void *val, fpm_stream stream);

/* ------------------------------------------------------------------ */
/* Adjoint of the LJ force and of velocity Verlet (not in the paper:     */
/* the chain rule applied to the force of Sec. 4.1 and the integrator    */
/* of Listing 4.1, for gradients w.r.t. positions, eps and sigma)        */
/* ------------------------------------------------------------------ */

/* Backward sweep of the LJ force over a Verlet list (same box, grid, list,
 * nn, cap and cutoff as fpm_lj_forces).  With J = dF/dx (symmetric):
 *   adj_pos[i].xyz += scale * (J a)_i                       (FP64, double4 [n])
 *   d_params[0]    += scale * sum_i a_i . dF_i/d eps
 *   d_params[1]    += scale * sum_i a_i . dF_i/d sigma
 *   d_params[2]    += dU/d eps,  d_params[3] += dU/d sigma    (U as in fpm_lj_forces)
 * a : [n] float4|double4 in the positions' precision (w ignored).  Pair
 * arithmetic in the positions' precision; adj_pos and d_params accumulate in
 * FP64 (d_params in a fixed order, bit-reproducible).  d_params may be NULL.
 * workspace : fpm_reduce_workspace(n, grid) bytes (zero-filled once).
 * adj_pos 32-byte aligned. */
fpm_status fpm_lj_backward(const fpm_box *box, const fpm_grid *grid, int32_t n, fpm_prec prec, const void *pos,
                           const void *list, const uint32_t *nn, int32_t cap,
                           double eps, double sigma, double rc,
                           const void *a, double scale, double *adj_pos, double *d_params,
                           void *workspace, size_t workspace_bytes, fpm_dev_status *d_status, fpm_stream stream);

/* One reverse velocity-Verlet update of the FP64 adjoint state (xbar, vbar:
 * double4 [n]).  For every k, with j = perm[k] (perm from the cell-list build
 * that reordered the particles during this step) or j = k (perm NULL, or
 * d_gate given and *d_gate == 0):
 *   xbar_out[j] = xbar_in[k];  vbar_out[j] = vbar_in[k] + dt * xbar_in[k];
 *   a_out[j] = (T)(c * vbar_out[j])   (float4|double4, the vector for the next
 *                                      fpm_lj_backward).
 * d_gate (device word, may be NULL) lets a captured graph apply perm only in
 * the steps whose rebuild ran.  With perm, inputs and outputs must be
 * distinct arrays; without, they may alias. */
fpm_status fpm_vv_adjoint(int32_t n, fpm_prec prec, const uint32_t *perm, const uint32_t *d_gate, double dt,
                          double c, const double *xbar_in, const double *vbar_in, double *xbar_out,
                          double *vbar_out, void *a_out, fpm_stream stream);

/* Seed of the loss L = U(x_T) + sum_i |F_i(x_T)|^2: xbar = -F, vbar = 0,
 * a_out = F (so that fpm_lj_backward(a_out, scale = 2) adds 2 J F and
 * 2 F . dF/d(eps, sigma), and its d_params[2..3] add dU/d(eps, sigma)). */
fpm_status fpm_adjoint_seed(int32_t n, fpm_prec prec, const void *force, double *xbar, double *vbar,
                            void *a_out, fpm_stream stream);

/* The loss of the differentiable rollout, L = U(x_T) + sum_i |F_i(x_T)|^2,
 * on the device: d_loss[0] = d_energy[0] + 2 d_half_sumf2[0], with d_energy
 * the [3] output of fpm_lj_forces at x_T and d_half_sumf2[0] = 1/2 sum |F|^2
 * (fpm_kinetic applied to the forces).  All three are device pointers to
 * FP64; one single-thread launch. */
fpm_status fpm_adjoint_loss(const double *d_energy, const double *d_half_sumf2, double *d_loss,
                            fpm_stream stream);

/* The results of the reverse pass, assembled on the device:
 *   grad_x[3 ids[k] + c] = xbar[k][c], grad_v[3 ids[k] + c] = vbar[k][c]
 *     (c = 0..2): dL/dx0 and dL/dv0 as [n][3] FP64 rows in the order the
 *     particles had before the first cell-list build, ids being the particle
 *     ids held in sorted slot k at step 0 (a permutation of 0..n-1);
 *   d_grad_theta[0] = seed[0] + seed[2] + steps[0]   (dL/d eps),
 *   d_grad_theta[1] = seed[1] + seed[3] + steps[1]   (dL/d sigma),
 *     with d_theta_seed the [4] d_params of the seed's fpm_lj_backward
 *     (2 F.dF/dtheta, then dU/dtheta) and d_theta_steps the [4] d_params
 *     accumulated by the reverse steps (a.dF/dtheta; their dU entries unused).
 * xbar, vbar: [n] double4.  grad_x and grad_v must not alias. */
fpm_status fpm_adjoint_finish(int32_t n, const uint32_t *ids, const double *xbar, const double *vbar,
                              const double *d_theta_seed, const double *d_theta_steps, double *grad_x,
                              double *grad_v, double *d_grad_theta, fpm_stream stream);

/* ------------------------------------------------------------------ */
/* Batched replicas: R independent periodic LJ systems of uneven size    */
/* advanced together (an ensemble of the MD system of Sec. 4.1; the      */
/* paper runs one system per process), single precision                  */
/* ------------------------------------------------------------------ */

/* One replica of a batch.  Its particles are [p0, p0 + n) of the batch's
 * concatenated arrays; its cells are entries [c0, c0 + grid.ncell] of the
 * batch's cell_start (whose values are indices into the concatenated
 * arrays); its tiles are [t0, t0 + grid.tiles_x * grid.nc[1] * grid.nc[2])
 * of the batch's Verlet-list object.  Written by fpm_batch_plan; the calls
 * below read a DEVICE copy of the array (d_reps), which the caller makes. */
typedef struct {
    fpm_box box;
    fpm_grid grid;
    int32_t p0, n;
    int32_t c0, t0;
} fpm_replica;

/* Sizes of a batch (host struct, passed by pointer to every batched call).
 * stage_cap and sweep_blocks act as in fpm_grid, for every replica; the
 * plan sets stage_cap to an estimate and sweep_blocks, sweep_threads and
 * step_blocks_per_sm to 0, and the caller may change them between calls
 * (launch-shape choices: lists and forces do not depend on them, and the
 * per-replica energies only up to the FP32 rounding of the per-tile sums,
 * which group by block size; a tile whose neighbourhood exceeds stage_cap
 * reads it from global memory and is counted in d_status->spilled). */
typedef struct {
    int32_t R;
    int32_t n_total;
    int32_t ncell_total;   /* cell_start has ncell_total + 1 entries */
    int32_t ntiles_total;
    int32_t max_n;
    int32_t max_ncell;
    int32_t stage_cap;
    int32_t sweep_blocks;
    int32_t sweep_threads;  /* threads per block of the batched force sweep: 128, 256 or 512 (0: 256) */
    int32_t step_blocks_per_sm;  /* fpm_batch_step: blocks per SM its registers are bounded for, 2, 3 or 4
                                    (0: 4); fewer blocks, more registers per thread */
} fpm_batch;

/* Plans a batch of R replicas (host only): replica r has counts[r]
 * particles in boxes[r] (every dimension periodic, L > 2 r_cell (1 + 2^-10)),
 * a cell grid made as by fpm_grid_make(boxes[r], r_cell, counts[r]) but with
 * tile widths aimed at tile_target particles per tile (0: 200), and the
 * offsets p0, c0, t0 in replica order.  reps : [R] host array, written.
 * Limits: R <= 65535, max_ncell <= 32768 cells per replica. */
fpm_status fpm_batch_plan(int32_t R, const fpm_box *boxes, const int32_t *counts, double r_cell,
                          int32_t tile_target, fpm_replica *reps, fpm_batch *batch);

/* v += dt/2 F; x += dt v (no wrap) for all particles of the batch, then the
 * rebuild test of each replica: d_rep_flag[r] |= 1 when a particle of
 * replica r moved by more than skin/2 since pos_ref (d2 > (float)(skin^2/4),
 * d = x - x_ref per component).  d_rep_flag : [R] uint32. */
fpm_status fpm_batch_drift_check(const fpm_batch *batch, const fpm_replica *d_reps, double dt, void *pos,
                                 void *vel, const void *force, const void *pos_ref, double skin,
                                 uint32_t *d_rep_flag, fpm_stream stream);

/* Bytes of device workspace of fpm_batch_celllist_build and fpm_batch_step
 * (for fpm_batch_step zero-filled once before first use: it holds cell
 * counters that every step leaves at zero again). */
fpm_status fpm_batch_celllist_workspace(const fpm_batch *batch, size_t *bytes);

/* Cell lists of the replicas whose d_rep_flag is set (all replicas when
 * d_rep_flag is NULL), each as fpm_celllist_build on its own box and grid:
 * wrap, cell index, the stable counting sort by (cell, index), and the
 * in-place reorder of pos, vel (float4 [n_total]) and ids (uint32, may be
 * NULL), within the replica's range.  cell_start : [ncell_total + 1];
 * perm[k] = the index before the reorder of the particle now at k (entries
 * of replicas not rebuilt are untouched).  One block per replica.  A
 * particle outside its box (a non-finite coordinate) latches
 * FPM_FLAG_DOMAIN. */
fpm_status fpm_batch_celllist_build(const fpm_batch *batch, const fpm_replica *d_reps, void *pos, void *vel,
                                    uint32_t *ids, uint32_t *cell_start, uint32_t *perm, void *workspace,
                                    size_t workspace_bytes, const uint32_t *d_rep_flag,
                                    fpm_dev_status *d_status, fpm_stream stream);

/* Bytes of the batch's Verlet-list object for capacity cap (256-B aligned). */
fpm_status fpm_batch_list_bytes(const fpm_batch *batch, int32_t cap, size_t *bytes);

/* Verlet lists (as fpm_verlet_build, per replica) of the replicas whose
 * d_rep_flag is set (all when NULL), then clears every d_rep_flag and adds
 * the number of rebuilt replicas to d_status->nrebuild.  pos_ref receives
 * the positions of the rebuilt replicas.  The list object must have been
 * built for all replicas once (d_rep_flag NULL) before a gated build. */
fpm_status fpm_batch_verlet_build(const fpm_batch *batch, const fpm_replica *d_reps, const void *pos,
                                  const uint32_t *cell_start, double r_list, int32_t cap, void *list,
                                  size_t list_bytes, uint32_t *nn, void *pos_ref, uint32_t *d_rep_flag,
                                  fpm_dev_status *d_status, fpm_stream stream);

/* As fpm_verlet_decode, for the batch's list (indices into the concatenated
 * arrays; out : [cap * fpm_nbr_ld(n_total)]). */
fpm_status fpm_batch_verlet_decode(const fpm_batch *batch, int32_t cap, const void *list, const uint32_t *nn,
                                   uint32_t *out, fpm_stream stream);

/* Bytes of workspace of fpm_batch_lj_forces and fpm_batch_step (zero-filled
 * once before first use; every call leaves its counters at zero again). */
fpm_status fpm_batch_workspace(const fpm_batch *batch, size_t *bytes);

/* LJ forces of every replica (as fpm_lj_forces on its own box, single
 * precision) in one persistent launch over all tiles of the batch.
 * d_energy : [R][3] double (U, W, pairs of each replica, FP64, fixed order)
 * or NULL. */
fpm_status fpm_batch_lj_forces(const fpm_batch *batch, const fpm_replica *d_reps, const void *pos,
                               const void *list, const uint32_t *nn, int32_t cap, double eps, double sigma,
                               double rc, void *force, double *d_energy, void *workspace,
                               size_t workspace_bytes, fpm_dev_status *d_status, fpm_stream stream);

/* fpm_batch_lj_forces and the closing half-kick of velocity Verlet in the same
 * launch (as fpm_lj_forces_kick): after F_i is written, vel[i] += dt/2 F_i,
 * bit-identical to fpm_batch_lj_forces followed by fpm_vv_step(half = 1).
 * vel: [n_total] float4, not aliasing pos or force. */
fpm_status fpm_batch_lj_forces_kick(const fpm_batch *batch, const fpm_replica *d_reps, const void *pos,
                                    const void *list, const uint32_t *nn, int32_t cap, double eps, double sigma,
                                    double rc, void *force, double *d_energy, void *workspace,
                                    size_t workspace_bytes, fpm_dev_status *d_status, void *vel, double dt,
                                    fpm_stream stream);

/* One velocity-Verlet step of the whole batch in ONE cooperative launch:
 * the work of fpm_batch_drift_check, fpm_batch_celllist_build and
 * fpm_batch_verlet_build gated by d_rep_flag, then fpm_batch_lj_forces_kick,
 * as phases of a persistent kernel separated by grid barriers, with the same
 * arguments as those four calls (cell_ws: fpm_batch_celllist_workspace bytes;
 * workspace: fpm_batch_workspace bytes).  The cell lists of the flagged
 * replicas are built by the whole grid (particles binned with global
 * counters, a scan per replica, a warp per cell), and the Verlet scans of
 * their tiles share one ticket queue with the force tiles: the tiles of the
 * replicas not rebuilt first, those of the rebuilt replicas once every tile
 * of their replica is scanned.  A step that flags no replica skips the
 * rebuild phases.  The results (pos, vel, force, ids, perm, cell_start, nn,
 * the list, pos_ref, d_energy, d_status->nrebuild and max_nn) are those of
 * the four calls bit for bit when the batch's sweep_threads is 0 or 256; the
 * flags are clear afterwards.
 * Preconditions: cell_ws and workspace zero-filled once; the cell lists and
 * the list built for every replica once with this cell_ws and list
 * (fpm_batch_celllist_build and fpm_batch_verlet_build, d_rep_flag NULL: the
 * cell build also records the replica of every particle and cell in cell_ws);
 * force holds the forces of the current positions.
 * The grid is every block that fits on the GPU at once (or sweep_blocks when
 * smaller); a grid that cannot be resident is refused by the launch
 * (FPM_ERR_CUDA), never run.  The grid barrier's state lives in the list
 * object (bytes 32..39).  Every wait (grid barrier, scanned-tile count, bulk
 * copy) is bounded (about 2 s of SM clock); on expiry the kernel latches
 * FPM_FLAG_TIMEOUT and returns.  The results of that step are then undefined:
 * zero-fill cell_ws and workspace again and run fpm_batch_celllist_build and
 * fpm_batch_verlet_build (which resets the barrier) on every replica before
 * the next step. */
fpm_status fpm_batch_step(const fpm_batch *batch, const fpm_replica *d_reps, double dt, double skin, double r_list,
                          int32_t cap, double eps, double sigma, double rc, void *pos, void *vel, void *force,
                          void *pos_ref, uint32_t *ids, uint32_t *cell_start, uint32_t *perm, void *list,
                          size_t list_bytes, uint32_t *nn, uint32_t *d_rep_flag, void *cell_ws,
                          size_t cell_ws_bytes, void *workspace, size_t workspace_bytes, double *d_energy,
                          fpm_dev_status *d_status, fpm_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* FPM_H */
