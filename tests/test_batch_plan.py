"""Host-side logic of the batched replicas (no GPU): the plan's offsets and
grids, its argument checks, and the ensemble generator's statistics."""
import numpy as np
import pytest

from paper_1804_07598_gb300 import fpm, inputs


def boxes_of(Ls):
    return [fpm.make_box(np.array([L, L, L]), (1, 1, 1)) for L in Ls]


def test_plan_offsets_and_grids(fpm_lib):
    counts = [256, 700, 0, 5000, 1200]
    rho = [0.95, 0.80, 0.80, 0.75, 0.90]
    Ls = [max((c / r) ** (1 / 3), 6.0) for c, r in zip(counts, rho)]
    reps, b = fpm.fpm_batch_plan(boxes_of(Ls), counts, 2.8, 0)
    assert b.R == 5 and b.n_total == sum(counts) and b.max_n == max(counts)
    p0 = c0 = t0 = 0
    for r in range(5):
        g = fpm.fpm_grid_make(boxes_of([Ls[r]])[0], 2.8, counts[r])
        assert tuple(reps[r].grid.nc) == tuple(g.nc) and reps[r].grid.ncell == g.ncell
        assert list(reps[r].grid.inv) == list(g.inv)
        assert (reps[r].p0, reps[r].n, reps[r].c0, reps[r].t0) == (p0, counts[r], c0, t0)
        p0 += counts[r]
        c0 += g.ncell
        t0 += reps[r].grid.tiles_x * g.nc[1] * g.nc[2]
        assert 1 <= reps[r].grid.tiles_x <= g.nc[0]
        assert (g.nc[0] + reps[r].grid.tiles_x - 1) // reps[r].grid.tiles_x <= 14
    assert (b.ncell_total, b.ntiles_total) == (c0, t0)
    assert reps[0].grid.nc[0] == 1  # L = 6.46 < 3 r_cell: all-pairs replica
    assert b.stage_cap > 0 and b.sweep_blocks == 0


def test_plan_tile_target_sets_tile_width(fpm_lib):
    L = (16000 / 0.7) ** (1 / 3)
    _, b_small = fpm.fpm_batch_plan(boxes_of([L]), [16000], 2.8, 64)
    _, b_big = fpm.fpm_batch_plan(boxes_of([L]), [16000], 2.8, 512)
    assert b_small.ntiles_total > b_big.ntiles_total


def test_plan_rejects_bad_replicas(fpm_lib):
    with pytest.raises(fpm.FpmError):
        fpm.fpm_batch_plan([fpm.make_box(np.array([10.0, 10.0, 10.0]), (1, 0, 1))], [100], 2.8)
    with pytest.raises(fpm.FpmError):  # periodic L must exceed 2 r_cell
        fpm.fpm_batch_plan(boxes_of([5.0]), [100], 2.8)
    with pytest.raises(fpm.FpmError):
        fpm.fpm_batch_plan(boxes_of([10.0]), [-1], 2.8)


def test_ensemble_statistics():
    N, rho, T = inputs.batched_replicas(512, 2024)
    assert N.min() >= 256 and N.max() <= 16384
    assert 0.70 <= rho.min() and rho.max() <= 0.95 and 0.6 <= T.min() and T.max() <= 1.5
    # log-uniform sizes: the median is near the geometric mean of the bounds
    assert 1000 < np.median(N) < 4000
    x, v, L = inputs.replica_state(1000, 0.8, 1.0, 3)
    assert x.shape == (1000, 4) and np.all(x[:, :3] >= 0) and np.all(x[:, :3] < L[0])
    assert abs(1000 / L[0] ** 3 - 0.8) < 1e-12
    assert len({tuple(p) for p in np.round(x[:, :3], 9)}) == 1000  # distinct sites
    assert np.allclose(v[:, :3].sum(0), 0, atol=1e-10)


def test_step_rejects_bad_arguments(fpm_lib):
    """fpm_batch_step checks its arguments before any device work: a bad
    register bound, pos / vel aliasing, no flag array, and a list object or a
    workspace below the sizes the size queries give.  The pointers are
    aligned fakes that a valid call would dereference; none is touched."""
    import ctypes
    counts = [300, 1200]
    Ls = [max((c / 0.8) ** (1 / 3), 6.0) for c in counts]
    reps, b = fpm.fpm_batch_plan(boxes_of(Ls), counts, 2.8, 0)
    cap = 96
    lb = fpm.fpm_batch_list_bytes(b, cap)
    cb = fpm.fpm_batch_celllist_workspace(b)
    wb = fpm.fpm_batch_workspace(b)
    # the step's regions: flagged list, scanned-tile counts, tile queue; cell counters, replica ids
    assert wb >= 256 + 24 * b.ntiles_total + 4 * (3 * b.R + b.ntiles_total)
    assert cb >= 4 * (7 * b.n_total + 2 * b.ncell_total)
    P, Q, V, F = 0x100000, 0x200000, 0x300000, 0x400000
    L, C, W = 0x1000000, 0x2000000, 0x3000000

    def step(batch, pos=P, vel=V, list_bytes=lb, flag=Q, cell_bytes=cb, ws_bytes=wb):
        return fpm_lib.fpm_batch_step(ctypes.byref(batch), P, 0.005, 0.3, 2.8, cap, 1.0, 1.0, 2.5, pos, vel, F, P,
                                      None, Q, None, L, list_bytes, Q, flag, C, cell_bytes, W, ws_bytes, None,
                                      None, None)

    bad_b = fpm.fpm_batch.from_buffer_copy(b)
    bad_b.step_blocks_per_sm = 1
    assert step(bad_b) == fpm.FPM_ERR_INVALID
    assert "step_blocks_per_sm" in fpm.fpm_last_error()
    assert step(b, vel=P) == fpm.FPM_ERR_INVALID
    assert step(b, flag=None) == fpm.FPM_ERR_INVALID
    assert step(b, list_bytes=lb - 4) == fpm.FPM_ERR_WORKSPACE
    assert step(b, cell_bytes=cb - 4) == fpm.FPM_ERR_WORKSPACE
    assert step(b, ws_bytes=wb - 4) == fpm.FPM_ERR_WORKSPACE
