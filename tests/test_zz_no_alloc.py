"""fpm_lj_forces_noalloc: the force sweep for callers that cannot allocate
device memory (their memory belongs to another runtime or a fixed pool, or a
cudaMalloc would stall a real-time loop).  It must give the same forces and
energies as fpm_lj_forces, on consecutive calls, because its built-in scratch
keeps the previous call's contents.

Collected last on purpose, so that a run stopping at its first failure has
already run every other test.  It passes alone in a fresh process too.
"""
import numpy as np
import pytest
import torch

from paper_1804_07598_gb300 import fpm, inputs
from paper_1804_07598_gb300.md import LJSystem

pytestmark = pytest.mark.gpu

TOL_F = {"f32": 1e-5, "f64": 1e-12}   # same as the force parity tests
TOL_E = {"f32": 1e-6, "f64": 1e-12}


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_noalloc_matches_workspace_version(cuda, prec):
    wl = inputs.WORKLOADS["lj_small"]
    pos, vel, L = inputs.lj_state(wl, jitter=0.06)
    s = LJSystem(pos, vel, L, precision=prec)
    s.compute_forces()
    torch.cuda.synchronize()
    f_ref = s.force.cpu().numpy().astype(np.float64)
    e_ref = s.energy.cpu().numpy()
    rms = np.sqrt(np.mean(np.sum(f_ref[:, :3] ** 2, axis=1)))
    for call in range(2):  # two calls in a row share the scratch array
        f = torch.full_like(s.force, float("nan"))
        e = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        fpm.fpm_lj_forces_noalloc(s.box, s.grid, s.n, s.prec, s.pos, s.nbr, s.nn, s.cap, s.eps, s.sigma, s.rc, f, e)
        torch.cuda.synchronize()
        fn = f.cpu().numpy().astype(np.float64)
        en = e.cpu().numpy()
        err = np.max(np.linalg.norm(fn[:, :3] - f_ref[:, :3], axis=1)) / rms
        assert err <= TOL_F[prec], (call, err)
        assert np.all(np.abs(en[:2] - e_ref[:2]) <= TOL_E[prec] * np.abs(e_ref[:2])), (call, en, e_ref)
        assert en[2] == e_ref[2]


def test_noalloc_rejects_oversize(fpm_lib):
    box = fpm.make_box((10.0, 10.0, 10.0))
    grid = fpm.fpm_grid_make(box, 2.8, 1000)
    with pytest.raises(fpm.FpmError) as e:
        fpm.fpm_lj_forces_noalloc(box, grid, (1 << 24) + 1, fpm.FPM_F32, 1, 256, 1, 64, 1.0, 1.0, 2.5, 1, 1, None, 0)
    assert e.value.status == fpm.FPM_ERR_INVALID
    assert "scratch limit" in fpm.fpm_last_error()


def test_noalloc_allocates_nothing(cuda):
    """After a first call on the device (which looks the scratch address up),
    further calls change neither torch's allocation count nor the device's
    free memory: no cudaMalloc, no caching-allocator growth."""
    wl = inputs.WORKLOADS["lj_small"]
    pos, vel, L = inputs.lj_state(wl, jitter=0.06)
    s = LJSystem(pos, vel, L, precision="f32")
    f = torch.empty_like(s.force)
    e = torch.empty(3, dtype=torch.float64, device="cuda")

    def call():
        fpm.fpm_lj_forces_noalloc(s.box, s.grid, s.n, s.prec, s.pos, s.nbr, s.nn, s.cap, s.eps, s.sigma, s.rc, f, e)

    call()
    torch.cuda.synchronize()
    alloc0, reserved0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        call()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == reserved0
    assert free1 == free0


def test_noalloc_rejects_too_many_tiles(cuda):
    """A grid of more than 65,536 tiles (300^3 box, cells of 2.8: 8 x 107 x 107
    tiles) is rejected before any device work, whatever n.  The buffers are
    real and the list is empty, so nothing could go astray even if it were
    not."""
    box = fpm.make_box((300.0, 300.0, 300.0))
    n, cap = 1000, 64
    grid = fpm.fpm_grid_make(box, 2.8, n)
    assert grid.tiles_x * grid.nc[1] * grid.nc[2] > 65536
    pos = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    lst = torch.zeros(fpm.fpm_verlet_list_bytes(n, grid, cap), dtype=torch.uint8, device="cuda")
    nn = torch.zeros(n, dtype=torch.int32, device="cuda")
    f = torch.zeros_like(pos)
    with pytest.raises(fpm.FpmError) as err:
        fpm.fpm_lj_forces_noalloc(box, grid, n, fpm.FPM_F32, pos, lst, nn, cap, 1.0, 1.0, 2.5, f, None)
    assert err.value.status == fpm.FPM_ERR_INVALID
    assert "scratch limit" in fpm.fpm_last_error()
