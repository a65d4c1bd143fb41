"""Particle-mesh interpolation with the M'4 kernel (Sec. 4.4) on the GPU.

    pm = ParticleMesh(L, (Nx, Ny, Nz), n_max)
    mesh = pm.p2m(pos, val)      # bins (fpm_celllist_build on the mesh cells), then fpm_p2m
    out = pm.m2p(pos, mesh)      # fpm_m2p

pos: float4 [n] device tensor (x, y, z, -); val: float4 [n]; mesh: float4
[Nz, Ny, Nx, 4].  The box is periodic in every dimension.
"""
from __future__ import annotations

import torch

from . import fpm


class ParticleMesh:
    def __init__(self, L, N, n_max: int, device="cuda"):
        self.device = torch.device(device)
        self.N = tuple(int(v) for v in N)
        self.box = fpm.make_box(L, (1, 1, 1))
        self.grid = fpm.fpm_mesh_grid(self.box, self.N)
        self.n_max = int(n_max)
        dev, f32 = self.device, torch.float32
        self.pos_s = torch.zeros((max(self.n_max, 1), 4), dtype=f32, device=dev)
        self.val_s = torch.zeros((max(self.n_max, 1), 4), dtype=f32, device=dev)
        self.perm = torch.zeros(max(self.n_max, 1), dtype=torch.int32, device=dev)
        self.cell_start = torch.zeros(self.grid.ncell + 1, dtype=torch.int32, device=dev)
        self.ws_cell = torch.zeros(fpm.fpm_celllist_workspace(self.n_max, self.grid, fpm.FPM_F32), dtype=torch.uint8,
                                   device=dev)
        self.status = torch.zeros(fpm.STATUS_BYTES // 4, dtype=torch.int32, device=dev)
        self.mesh = torch.zeros((self.N[2], self.N[1], self.N[0], 4), dtype=f32, device=dev)

    def bin(self, pos, val, stream=None):
        """Sort a copy of (pos, val) by mesh cell (pos_s, val_s, cell_start)."""
        n = pos.shape[0]
        if n > self.n_max:
            raise ValueError(f"{n} particles > n_max {self.n_max}")
        if n == 0:
            self.cell_start.zero_()
            return
        fpm.fpm_celllist_build(self.box, self.grid, n, fpm.FPM_F32, pos, val, None, self.pos_s, self.val_s, None,
                               self.cell_start, self.perm, self.ws_cell, self.status, None, stream=stream)

    def p2m(self, pos, val, stream=None):
        """mesh = the M'4 interpolation of the particles' val onto the mesh."""
        self.bin(pos, val, stream=stream)
        fpm.fpm_p2m(self.box, self.grid, pos.shape[0], self.pos_s, self.val_s, self.cell_start, self.mesh,
                    self.status, stream=stream)
        return self.mesh

    def m2p(self, pos, mesh=None, out=None, binned=False, stream=None):
        """The M'4 interpolation of the mesh at the particles.  binned=True:
        `pos` are the positions last given to p2m/bin, whose permutation then
        orders the work (faster; the same values)."""
        mesh = self.mesh if mesh is None else mesh
        if out is None:
            out = torch.empty((pos.shape[0], 4), dtype=torch.float32, device=self.device)
        order = self.perm if binned and pos.shape[0] > 0 else None
        fpm.fpm_m2p(self.box, self.grid, pos.shape[0], pos, mesh, out, order=order, stream=stream)
        return out

    def check_status(self):
        st = fpm.read_status(self.status)
        code = fpm.fpm_status_from_device(st)
        if code != fpm.FPM_OK:
            raise fpm.FpmError(code, f"device status flags={st.flags}")
        return st
