"""Degenerate inputs through the C-ABI path: the empty system (n = 0) at every
entry point of a step, one particle alone, and particle pairs against the
closed-form Lennard-Jones force, energy and virial (the pair law of Sec.
4.1), in an open box and through the minimum image of a periodic box too
small for a cell stencil (one cell per dimension)."""
import numpy as np
import pytest
import torch

from gpu_util import status_tensor
from paper_1804_07598_gb300 import fpm
from paper_1804_07598_gb300.md import LJSystem

pytestmark = pytest.mark.gpu


def tdt(prec):
    return torch.float32 if prec == "f32" else torch.float64


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_empty_system_every_entry_point(cuda, prec):
    """n = 0: every call of an LJ step, the SPH rates and the DEM sweep
    return FPM_OK; the energies and the kinetic sums are zeros (not left
    over from the buffer's previous contents), the cell list is empty and no
    status flag is raised."""
    P = fpm.FPM_F32 if prec == "f32" else fpm.FPM_F64
    dev, dt = "cuda", tdt(prec)
    box = fpm.make_box((10.0, 10.0, 10.0))
    grid = fpm.fpm_grid_make(box, 2.8, 0)
    cap = 32

    def v4():
        return torch.zeros((1, 4), dtype=dt, device=dev)

    pos, vel, force, ref = v4(), v4(), v4(), v4()
    ids = torch.zeros(1, dtype=torch.int32, device=dev)
    perm = torch.zeros(1, dtype=torch.int32, device=dev)
    cs = torch.full((grid.ncell + 1,), -1, dtype=torch.int32, device=dev)
    ws = torch.zeros(max(fpm.fpm_celllist_workspace(0, grid, P), 16), dtype=torch.uint8, device=dev)
    st = status_tensor()
    fpm.fpm_celllist_build(box, grid, 0, P, pos, vel, ids, pos, vel, ids, cs, perm, ws, st)
    lst = torch.zeros(fpm.fpm_verlet_list_bytes(0, grid, cap), dtype=torch.uint8, device=dev)
    nn = torch.zeros(1, dtype=torch.int32, device=dev)
    fpm.fpm_verlet_build(box, grid, 0, P, pos, cs, 2.8, cap, lst, nn, ref, st)
    red = torch.zeros(fpm.fpm_reduce_workspace(0, grid), dtype=torch.uint8, device=dev)
    energy = torch.full((3,), 7.0, dtype=torch.float64, device=dev)
    fpm.fpm_lj_forces(box, grid, 0, P, pos, lst, nn, cap, 1.0, 1.0, 2.5, force, energy, red, st)
    energy2 = torch.full((3,), 7.0, dtype=torch.float64, device=dev)
    fpm.fpm_lj_forces_noalloc(box, grid, 0, P, pos, lst, nn, cap, 1.0, 1.0, 2.5, force, energy2, st)
    fpm.fpm_vv_drift_check(box, 0, P, 0.005, pos, vel, force, ref, 0.3, st)
    fpm.fpm_vv_step(box, 0, P, 1, 0.005, None, vel, force)
    fpm.fpm_verlet_check(box, 0, P, pos, ref, 0.3, st)
    kin = torch.full((4,), 7.0, dtype=torch.float64, device=dev)
    fpm.fpm_kinetic(0, P, vel, kin, red)
    adj = v4()
    fpm.fpm_lj_backward(box, grid, 0, P, pos, lst, nn, cap, 1.0, 1.0, 2.5, vel, 1.0, adj, None, red, st)
    if prec == "f32":
        sp = fpm.fpm_sph_params()
        sp.h, sp.mass, sp.rho0, sp.c0, sp.gamma, sp.alpha, sp.eta2 = 0.01, 1e-3, 1000.0, 30.0, 7.0, 0.1, 1e-6
        sp.g[2] = -9.81
        dtc = torch.zeros(2, dtype=torch.float32, device=dev)
        fpm.fpm_sph_forces(box, grid, 0, pos, vel, lst, nn, cap, sp, force, dtc, red, st)
        hist = torch.zeros((cap, 4), dtype=torch.float32, device=dev)
        ncon = torch.zeros(1, dtype=torch.int32, device=dev)
        dp = fpm.dem_params()
        fpm.fpm_dem_forces(box, grid, 0, pos, vel, v4(), lst, nn, cap, dp, hist, force, v4(), ncon, red, st)
        fpm.fpm_dem_leapfrog(box, 0, dp, pos, vel, v4(), force, v4(), ref, 0.1, st)
        assert torch.all(dtc == 0) and int(ncon[0]) == 0
    torch.cuda.synchronize()
    assert torch.all(cs == 0)
    assert torch.all(energy == 0) and torch.all(energy2 == 0)
    assert torch.all(kin == 0)
    assert torch.all(force == 0) and torch.all(adj == 0)
    assert fpm.read_status(st).flags == 0


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("L", [10.0, 6.0])
def test_single_particle(cuda, prec, L):
    """One particle in a periodic box: its own images lie beyond r_list (L =
    10 with three cells per dimension, L = 6 with one), so it has no
    neighbour, no force and no energy."""
    s = LJSystem(np.array([[1.3, 4.2, 0.7]]), np.array([[0.5, -0.2, 0.1]]), L, precision=prec)
    torch.cuda.synchronize()
    assert int(s.nn[0]) == 0
    assert torch.all(s.force == 0)
    assert torch.all(s.energy == 0)
    s.step(3)
    torch.cuda.synchronize()
    x = s.pos[0, :3].cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(x, np.mod(np.array([1.3, 4.2, 0.7]) + 3 * 0.005 * np.array([0.5, -0.2, 0.1]), L),
                               rtol=0, atol=1e-5)
    assert fpm.read_status(s.status).flags == 0


def lj_closed_form(d, eps=1.0, sigma=1.0, rc=2.5):
    """Force on particle 0 of a pair with separation d = x_0 - x_1, the pair
    energy and the pair virial r . F, from the pair law of Sec. 4.1, and the
    scales their rounding errors follow: the sums of the magnitudes of the
    repulsive and attractive terms (near the minimum the terms cancel, and a
    relative error of each term shows against that sum, not against the
    nearly zero difference)."""
    r2 = float(np.dot(d, d))
    if r2 >= rc * rc:
        return np.zeros(3), 0.0, 0.0, (1.0, 1.0, 1.0)
    s6 = (sigma * sigma / r2) ** 3
    f = 24.0 * eps * (2.0 * s6 * s6 - s6) / r2
    scales = (24.0 * eps * (2.0 * s6 * s6 + s6) / r2 * np.sqrt(r2), 4.0 * eps * (s6 * s6 + s6),
              24.0 * eps * (2.0 * s6 * s6 + s6))
    return f * d, 4.0 * eps * (s6 * s6 - s6), 24.0 * eps * (2.0 * s6 * s6 - s6), scales


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("r", [0.95, 1.0, 2.0 ** (1.0 / 6.0), 1.7, 2.49, 2.6])
def test_pair_closed_form_open_box(cuda, prec, r):
    """Two particles r apart along an oblique direction in an open box: the
    GPU force, U, W and pair count against the closed form, evaluated at the
    separation of the stored positions.  r = 2^(1/6) is the minimum (force
    zero up to rounding); r = 2.6 lies inside r_list but beyond rc (in the
    list, masked by the cutoff)."""
    u = np.array([0.48, -0.6, 0.64])
    c = np.array([5.1, 4.9, 5.3])
    x = np.stack([c + 0.5 * r * u, c - 0.5 * r * u])
    s = LJSystem(x, np.zeros((2, 3)), 10.0, periodic=(0, 0, 0), precision=prec)
    torch.cuda.synchronize()
    p = s.pos.cpu().numpy().astype(np.float64)[:, :3]
    f = s.force.cpu().numpy().astype(np.float64)
    e = s.energy.cpu().numpy()
    F0, U, W, (sf, su, sw) = lj_closed_form(p[0] - p[1])
    tol = 1e-12 if prec == "f64" else 4e-6
    assert np.max(np.abs(f[0, :3] - F0)) <= tol * sf
    assert np.max(np.abs(f[1, :3] + F0)) <= tol * sf
    assert abs(e[0] - U) <= tol * su
    assert abs(e[1] - W) <= tol * sw
    assert int(round(e[2])) == (1 if r < 2.5 else 0)
    assert abs(f[0, 3] - 0.5 * U) <= tol * su
    assert int(s.nn[0]) == 1 and int(s.nn[1]) == 1


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_pair_minimum_image_one_cell(cuda, prec):
    """A periodic box of L = 6 (< 3 r_list: one cell per dimension, every
    particle a candidate of every other): two particles 4.8 apart in x see
    each other at 1.2 through the wall, and at no other image."""
    x = np.array([[0.5, 3.0, 3.0], [5.3, 3.4, 2.9]])
    s = LJSystem(x, np.zeros((2, 3)), 6.0, precision=prec)
    torch.cuda.synchronize()
    p = s.pos.cpu().numpy().astype(np.float64)[:, :3]
    f = s.force.cpu().numpy().astype(np.float64)
    e = s.energy.cpu().numpy()
    d = p[0] - p[1]
    d -= 6.0 * np.round(d / 6.0)
    F0, U, W, (sf, su, sw) = lj_closed_form(d)
    tol = 1e-12 if prec == "f64" else 4e-6
    assert np.max(np.abs(f[0, :3] - F0)) <= tol * sf
    assert np.max(np.abs(f[1, :3] + F0)) <= tol * sf
    assert abs(e[0] - U) <= tol * su
    assert abs(e[1] - W) <= tol * sw
    assert int(round(e[2])) == 1
    assert int(s.nn[0]) == 1 and int(s.nn[1]) == 1
