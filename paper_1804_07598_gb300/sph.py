"""Weakly compressible SPH driver over libfpm (the dam-break test case of
Sec. 4.2): state buffers, the symplectic step with dynamic dt, a device-gated
Verlet rebuild, and CUDA-graph capture.

One step (all on the current stream):
    fpm_sph_forces   (pos, vr)      -> acc,   dt constraints at t^n
    fpm_sph_predict                 -> pos_h, vr_h, dt
    fpm_sph_forces   (pos_h, vr_h)  -> acc_h
    fpm_sph_correct                 -> pos, vr (in place), rebuild flag
    fpm_celllist_build [gated]         re-bin and reorder pos, vr, ids
    fpm_verlet_build   [gated]         new list with r_list = 2h + skin
Under CUDA-graph capture the gated calls sit in the body of a conditional
node on the rebuild flag (fpm_graph_if_begin).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import fpm


class SPHSystem:
    def __init__(self, pos, vel, rho, L, h, m, rho0=1000.0, c0=None, gamma=7.0, alpha=0.1, g=(0.0, 0.0, -9.81),
                 kernel="wendland", periodic=(0, 0, 0), skin=None, cfl=0.2, cap=None, h_swl=0.3, tile_target=170,
                 device="cuda"):
        self.device = torch.device(device)
        pos = np.asarray(pos, np.float64)
        n = pos.shape[0]
        self.n = n
        self.L = np.broadcast_to(np.asarray(L, np.float64), (3,)).copy()
        self.periodic = tuple(int(p) for p in periodic)
        self.box = fpm.make_box(self.L, self.periodic)
        if c0 is None:
            c0 = 20.0 * math.sqrt(float(np.linalg.norm(g)) * h_swl)
        P = fpm.fpm_sph_params()
        P.h, P.mass, P.rho0, P.c0, P.gamma, P.alpha, P.eta2 = h, m, rho0, c0, gamma, alpha, 0.01 * h * h
        for d in range(3):
            P.g[d] = g[d]
        P.kernel = 0 if kernel == "wendland" else 1
        self.params = P
        self.cfl = float(cfl)
        self.skin = float(skin) if skin is not None else 0.25 * h
        self.r_list = 2.0 * h + self.skin
        self.grid = fpm.fpm_grid_make(self.box, self.r_list, n)
        self._dp = (m / rho0) ** (1.0 / 3.0)
        self._set_tiles(tile_target)
        self.cap = int(cap) if cap else max(32, int(math.ceil(1.6 * 4.0 / 3.0 * math.pi * (self.r_list / (m / rho0)
                                                                                           ** (1 / 3)) ** 3 / 8)) * 8)
        dev = self.device
        f32 = torch.float32
        self.pos = torch.zeros((n, 4), dtype=f32, device=dev)
        self.pos[:] = torch.as_tensor(pos[:, :4] if pos.shape[1] == 4 else np.c_[pos, np.zeros(n)], dtype=f32)
        self.vr = torch.zeros((n, 4), dtype=f32, device=dev)
        self.vr[:, :3] = torch.as_tensor(np.asarray(vel, np.float64)[:, :3], dtype=f32)
        self.vr[:, 3] = torch.as_tensor(np.asarray(rho, np.float64) - rho0, dtype=f32)
        self.pos_h = torch.zeros_like(self.pos)
        self.vr_h = torch.zeros_like(self.vr)
        self.acc = torch.zeros_like(self.pos)
        self.acc_h = torch.zeros_like(self.pos)
        self.pos_ref = torch.zeros_like(self.pos)
        self.ids = torch.arange(n, dtype=torch.int32, device=dev)
        self.perm = torch.zeros(max(n, 1), dtype=torch.int32, device=dev)
        self.cell_start = torch.zeros(self.grid.ncell + 1, dtype=torch.int32, device=dev)
        self.nbr = torch.zeros(fpm.fpm_verlet_list_bytes(n, self.grid, self.cap), dtype=torch.uint8, device=dev)
        self.nn = torch.zeros(max(n, 1), dtype=torch.int32, device=dev)
        self.status = torch.zeros(fpm.STATUS_BYTES // 4, dtype=torch.int32, device=dev)
        self.ws_cell = torch.zeros(fpm.fpm_celllist_workspace(n, self.grid, fpm.FPM_F32), dtype=torch.uint8,
                                   device=dev)
        self.dtcons = torch.zeros(2, dtype=f32, device=dev)
        self.dtcons_h = torch.zeros(2, dtype=f32, device=dev)
        self.dt = torch.zeros(1, dtype=f32, device=dev)
        self.t_sim = torch.zeros(1, dtype=torch.float64, device=dev)  # simulated time (sum of the steps' dt)
        self.ws_red = torch.zeros(fpm.fpm_reduce_workspace(n, self.grid), dtype=torch.uint8, device=dev)
        self._body = torch.cuda.Stream(device=dev)  # captures the conditional rebuild
        self._graph = None
        self.rebuild()
        self.size_staging()

    def _set_tiles(self, tile_target):
        """Tile width for about `tile_target` particles per tile at the
        fluid's own density (the box is mostly empty)."""
        g = self.grid
        per_cell = (self.L[0] / g.nc[0]) * (self.L[1] / g.nc[1]) * (self.L[2] / g.nc[2]) / self._dp ** 3
        width = int(min(14, max(1, round(float(tile_target) / per_cell))))
        g.tiles_x = (g.nc[0] + width - 1) // width
        g.stage_cap = 0
        self.tile_target = int(tile_target)

    def retile(self, tile_target, sweep_blocks=None):
        """New tile width (a launch-shape choice): reallocates the list,
        rebuilds it and resizes the staging (synchronises)."""
        self._set_tiles(tile_target)
        if sweep_blocks is not None:
            self.grid.sweep_blocks = int(sweep_blocks)
        self.nbr = torch.zeros(fpm.fpm_verlet_list_bytes(self.n, self.grid, self.cap), dtype=torch.uint8,
                               device=self.device)
        self.ws_red = torch.zeros(fpm.fpm_reduce_workspace(self.n, self.grid), dtype=torch.uint8, device=self.device)
        self._graph = None
        self.status[fpm.STATUS_MAX_STAGED] = 0  # the staging size follows the new tiles
        self.rebuild()
        self.size_staging()

    def size_staging(self, margin: float = 1.15):
        """Set the grid's shared-memory staging capacity from the largest tile
        neighbourhood the last Verlet build saw (synchronises)."""
        st = fpm.read_status(self.status)
        self.grid.stage_cap = int(math.ceil((margin * st.max_staged + 64) / 32.0)) * 32

    @property
    def gate_ptr(self) -> int:
        return self.status.data_ptr() + 8

    def rebuild(self, gated: bool = False, stream=None):
        gate = self.gate_ptr if gated else None
        fpm.fpm_celllist_build(self.box, self.grid, self.n, fpm.FPM_F32, self.pos, self.vr, self.ids, self.pos,
                               self.vr, self.ids, self.cell_start, self.perm, self.ws_cell, self.status, gate,
                               stream=stream)
        fpm.fpm_verlet_build(self.box, self.grid, self.n, fpm.FPM_F32, self.pos, self.cell_start, self.r_list,
                             self.cap, self.nbr, self.nn, self.pos_ref, self.status, gate, stream=stream)

    def rates(self, pos=None, vr=None, acc=None, dtcons=None):
        fpm.fpm_sph_forces(self.box, self.grid, self.n, self.pos if pos is None else pos,
                           self.vr if vr is None else vr, self.nbr, self.nn, self.cap, self.params,
                           self.acc if acc is None else acc, self.dtcons if dtcons is None else dtcons, self.ws_red,
                           self.status)

    def density(self, out=None):
        """Density by summation, sum_j m W(r_ij) over the current list
        (the particle itself included), [n] float32 in sorted order."""
        rho = out if out is not None else torch.empty(self.n, dtype=torch.float32, device=self.device)
        fpm.fpm_sph_density(self.box, self.grid, self.n, self.pos, self.nbr, self.nn, self.cap, self.params, rho,
                            self.ws_red, self.status)
        return rho

    def _step(self):
        self.rates()
        fpm.fpm_sph_predict(self.box, self.n, self.params, self.cfl, self.pos, self.vr, self.acc, self.dtcons,
                            self.pos_h, self.vr_h, self.dt, self.dtcons_h, self.pos_ref, self.skin, self.status)
        self.rates(self.pos_h, self.vr_h, self.acc_h, self.dtcons_h)
        fpm.fpm_sph_correct(self.box, self.n, self.params, self.pos, self.vr, self.vr_h, self.acc_h, self.dt,
                            self.dtcons, self.pos_ref, self.skin, self.status, d_time=self.t_sim)
        if fpm.fpm_graph_if_begin(self.gate_ptr, self._body):
            self.rebuild(gated=True, stream=self._body)
            fpm.fpm_graph_if_end(self._body)
        else:
            self.rebuild(gated=True)

    def step(self, nsteps: int = 1):
        for _ in range(int(nsteps)):
            self._step()

    def capture(self, steps_per_graph: int = 1):
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        while s.cuda_stream == self._body.cuda_stream:  # torch hands out streams from a small pool
            s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                for _ in range(steps_per_graph):
                    self._step()
        torch.cuda.current_stream().wait_stream(s)
        self._graph = (g, steps_per_graph)
        return g

    def run(self, nsteps: int):
        if self._graph is None:
            self.step(nsteps)
            return
        g, k = self._graph
        for _ in range(nsteps // k):
            g.replay()
        self.step(nsteps % k)

    def simulated_time(self) -> float:
        """Simulated time so far (synchronises)."""
        return float(self.t_sim.item())

    def check_status(self):
        st = fpm.read_status(self.status)
        code = fpm.fpm_status_from_device(st)
        if code != fpm.FPM_OK:
            raise fpm.FpmError(code, f"device status flags={st.flags} max_nn={st.max_nn} cap={self.cap}")
        return st

    def state_numpy(self):
        """(pos [n,4] with type in w, vel [n,3], rho [n], ids) in sorted order."""
        p = self.pos.cpu().numpy()
        vr = self.vr.cpu().numpy()
        return p, vr[:, :3], vr[:, 3].astype(np.float64) + self.params.rho0, self.ids.cpu().numpy().view(np.uint32)
