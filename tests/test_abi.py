"""The C ABI library builds, loads and exports every function its header
declares; host-side argument checks work without a GPU."""
import ctypes

import numpy as np
import pytest

from paper_1804_07598_gb300 import fpm


def test_header_symbols_exported(fpm_lib):
    names = fpm.header_functions()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(fpm_lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    """The Python binding declares every header function (same names)."""
    assert set(fpm.header_functions()) <= set(fpm._SIG)


def test_grid_rule(fpm_lib):
    import oracle
    for L, per, r in [((16.79596, 16.79596, 16.79596), (1, 1, 1), 2.8), ((105.81456,) * 3, (1, 1, 1), 2.8),
                      ((6.46, 6.46, 6.46), (1, 1, 1), 2.8), ((1.6, 0.67, 0.4), (0, 0, 0), 0.0098),
                      ((9.0, 12.0, 5.7), (1, 1, 1), 2.8), ((6.0, 6.0, 6.0), (0, 0, 0), 2.8)]:
        g = fpm.fpm_grid_make(fpm.make_box(L, per), r, 1000)
        nc, inv = oracle.cell_grid(L, per, r)
        assert tuple(g.nc) == tuple(int(x) for x in nc)
        assert np.array_equal(np.array(g.inv, np.float32), inv)
        assert g.ncell == int(np.prod(nc))


def test_invalid_arguments_rejected(fpm_lib):
    with pytest.raises(fpm.FpmError) as e:
        fpm.fpm_grid_make(fpm.make_box((5.0, 5.0, 5.0)), 2.8)
    assert e.value.status == fpm.FPM_ERR_INVALID
    assert "2*r_cell" in fpm.fpm_last_error()
    with pytest.raises(fpm.FpmError):
        fpm.fpm_grid_make(fpm.make_box((5.0, 5.0, 5.0)), -1.0)
    g = fpm.fpm_grid_make(fpm.make_box((10.0, 10.0, 10.0)), 2.8)
    # null pointers / bad sizes return before touching the device
    assert fpm_lib.fpm_celllist_build(ctypes.byref(fpm.make_box((10.0,) * 3)), ctypes.byref(g), 10, 0, None, None,
                                      None, None, None, None, None, None, None, 0, None, None, None) \
        == fpm.FPM_ERR_INVALID
    assert fpm_lib.fpm_lj_forces(ctypes.byref(fpm.make_box((10.0,) * 3)), ctypes.byref(g), 10, 0, None, None, None, 0,
                                 1.0, 1.0, 2.5, None, None, None, 0, None, None) == fpm.FPM_ERR_INVALID
    assert fpm_lib.fpm_vv_step(ctypes.byref(fpm.make_box((10.0,) * 3)), 10, 0, 2, 0.005, None, None, None, None) \
        == fpm.FPM_ERR_INVALID
    assert fpm.fpm_status_string(fpm.FPM_ERR_CAPACITY).startswith("neighbour")


def test_status_decode(fpm_lib):
    s = fpm.fpm_dev_status()
    assert fpm.fpm_status_from_device(s) == fpm.FPM_OK
    s.flags = fpm.FPM_FLAG_DOMAIN
    assert fpm.fpm_status_from_device(s) == fpm.FPM_ERR_DOMAIN
    s.flags = fpm.FPM_FLAG_DOMAIN | fpm.FPM_FLAG_CAPACITY
    assert fpm.fpm_status_from_device(s) == fpm.FPM_ERR_CAPACITY
    assert ctypes.sizeof(fpm.fpm_dev_status) == fpm.STATUS_BYTES


def test_workspace_sizes(fpm_lib):
    g = fpm.fpm_grid_make(fpm.make_box((105.81456,) * 3), 2.8)
    b32 = fpm.fpm_celllist_workspace(1000188, g, fpm.FPM_F32)
    b64 = fpm.fpm_celllist_workspace(1000188, g, fpm.FPM_F64)
    assert b64 > b32 > 1000188 * 16
    assert fpm.fpm_reduce_workspace(1000188) >= 256 + (1000188 // 256) * 24
    g = fpm.fpm_grid_make(fpm.make_box((105.81456,) * 3), 2.8, 1000188)
    ntiles = g.tiles_x * g.nc[1] * g.nc[2]
    assert fpm.fpm_reduce_workspace(1000188, g) >= 256 + ntiles * 24
    assert fpm.fpm_verlet_list_bytes(1000188, g, 120) >= 60 * fpm.fpm_nbr_ld(1000188) * 4


def test_tile_width_rule(fpm_lib):
    """About 200 particles per tile (below the 256 threads of a tile block),
    at most 14 cells wide; every tile at least one cell."""
    for L, n in [((105.81456,) * 3, 1000188), ((16.79596,) * 3, 4000), ((6.46,) * 3, 256), ((60.0,) * 3, 1000)]:
        g = fpm.fpm_grid_make(fpm.make_box(L), 2.8, n)
        width = -(-g.nc[0] // g.tiles_x)
        assert 1 <= g.tiles_x <= g.nc[0] and width <= 14
        if g.nc[0] > 1:
            per_tile = n / (g.nc[1] * g.nc[2] * g.tiles_x)
            assert per_tile < 2 * 200 + 2 * n / g.ncell
    assert fpm.fpm_nbr_ld(1000188) % 32 == 0 and fpm.fpm_nbr_ld(1000188) >= 1000188


def test_later_entry_points_reject_bad_arguments(fpm_lib):
    """Argument errors of the fused force-and-kick, DEM, SPH and particle-mesh
    calls return FPM_ERR_INVALID before any device work.  The pointers are
    aligned fakes that a valid call would dereference; none is touched."""
    box = fpm.make_box((10.0,) * 3)
    g = fpm.fpm_grid_make(box, 2.8, 100)
    P, Q = 0x100000, 0x200000
    bad = fpm.FPM_ERR_INVALID
    # forces + kick: no vel, vel aliasing pos
    assert fpm_lib.fpm_lj_forces_kick(ctypes.byref(box), ctypes.byref(g), 10, 0, P, P, P, 8, 1.0, 1.0, 2.5, Q, None,
                                      None, 0, None, None, 0.005, None) == bad
    assert "vel" in fpm.fpm_last_error()
    assert fpm_lib.fpm_lj_forces_kick(ctypes.byref(box), ctypes.byref(g), 10, 0, P, P, P, 8, 1.0, 1.0, 2.5, Q, None,
                                      None, 0, None, P, 0.005, None) == bad
    # DEM: a non-positive radius; a history array off its 16-byte alignment
    dp = fpm.dem_params(R=-0.06)
    assert fpm_lib.fpm_dem_forces(ctypes.byref(box), ctypes.byref(g), 10, P, P, P, P, P, 8, ctypes.byref(dp), P, P,
                                  P, None, None, 0, None, None) == bad
    assert "DEM parameters" in fpm.fpm_last_error()
    dp = fpm.dem_params()
    assert fpm_lib.fpm_dem_forces(ctypes.byref(box), ctypes.byref(g), 10, P, P, P, P, P, 8, ctypes.byref(dp), P + 4,
                                  P, P, None, None, 0, None, None) == bad
    # SPH: a non-integer EOS exponent; an unknown kernel
    sp = fpm.fpm_sph_params()
    sp.h, sp.mass, sp.rho0, sp.c0, sp.gamma, sp.alpha, sp.eta2 = 0.01, 1e-3, 1000.0, 30.0, 7.5, 0.1, 1e-6
    assert fpm_lib.fpm_sph_forces(ctypes.byref(box), ctypes.byref(g), 10, P, P, P, P, 8, ctypes.byref(sp), P, None,
                                  None, 0, None, None) == bad
    assert "gamma" in fpm.fpm_last_error()
    sp.gamma, sp.kernel = 7.0, 2
    assert fpm_lib.fpm_sph_forces(ctypes.byref(box), ctypes.byref(g), 10, P, P, P, P, 8, ctypes.byref(sp), P, None,
                                  None, 0, None, None) == bad
    # particle-mesh: a mesh under 3 nodes, an open dimension, no cell_start
    with pytest.raises(fpm.FpmError):
        fpm.fpm_mesh_grid(fpm.make_box((1.0,) * 3), (2, 8, 8))
    with pytest.raises(fpm.FpmError):
        fpm.fpm_mesh_grid(fpm.make_box((1.0,) * 3, (1, 0, 1)), (8, 8, 8))
    mg = fpm.fpm_mesh_grid(fpm.make_box((1.0,) * 3), (8, 8, 8))
    assert fpm_lib.fpm_p2m(ctypes.byref(fpm.make_box((1.0,) * 3)), ctypes.byref(mg), 10, P, P, None, P, None,
                           None) == bad
