"""DEM driver: the Silbert grain model of Sec. 4.5 (Eqs. 9-13) on the GPU.

One step (FP32 state in the sorted order, float4 arrays):

    [rebuild, gated by the flag of the previous leapfrog]
        fpm_dem_rebuild_begin   save the contacts' u_t and omega
        fpm_celllist_build      wrap, re-bin and reorder pos, vel, ids
        fpm_verlet_build        the list of r_list = 2R + skin
        fpm_dem_rebuild_end     u_t and omega into the new order
    fpm_dem_forces              contact forces, torques, u_t (Eqs. 9-12)
    fpm_dem_leapfrog            Eq. 13 + the displacement test (sets the flag)

The cell size is `cell_factor` times r_list: grains are about 2R apart, so
cells of r_list hold one or two grains and a tile (at most 14 cells along x)
only a few dozen.  On the 688k-grain avalanche (cell factor: contact sweep /
whole step) 1.5: 209 / 258 us, 2.0: 115 / 148, 2.3: 99 / 132, 2.6: 91 / 127,
3.0: 88 / 123; larger cells cost only in the (rare) rebuild's candidate scan.
Under graph capture the rebuild is a conditional node.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import fpm


class DEMSystem:
    def __init__(self, pos, vel, omega, L, periodic, params: dict, skin: float, cell_factor: float = 3.0,
                 cap: int = 32, device="cuda"):
        self.device = torch.device(device)
        pos = np.asarray(pos, np.float64)
        n = pos.shape[0]
        self.n = n
        self.L = np.broadcast_to(np.asarray(L, np.float64), (3,)).copy()
        self.periodic = tuple(int(p) for p in periodic)
        self.params = dict(params)
        self.p = fpm.dem_params(**self.params)
        self.R = float(self.params["R"])
        self.skin = float(skin)
        self.r_list = 2.0 * self.R + self.skin
        self.box = fpm.make_box(self.L, self.periodic)
        # cells of cell_factor * r_list, no wider than a periodic length allows
        # (the grid needs L > 2 r_cell (1 + 2^-10) there), and never below r_list
        r_cell = cell_factor * self.r_list
        for d in range(3):
            if self.periodic[d]:
                r_cell = min(r_cell, self.L[d] / (2.0 * (1.0 + 2.0 ** -9)))
        self.grid = fpm.fpm_grid_make(self.box, max(r_cell, self.r_list), n)
        self.cap = int(cap) + int(cap) % 2
        self.ld = fpm.fpm_nbr_ld(n)
        dev, f32 = self.device, torch.float32

        def arr4(a):
            t = torch.zeros((n, 4), dtype=f32, device=dev)
            a = np.asarray(a, np.float64)
            t[:, : a.shape[1]] = torch.as_tensor(a[:, :4], dtype=f32)
            return t

        self.pos = arr4(pos)
        self.vel = arr4(vel)
        self.vel[:, 3] = 0
        self.omega = arr4(omega)
        self.omega[:, 3] = 0
        self.force = torch.zeros((n, 4), dtype=f32, device=dev)
        self.torque = torch.zeros((n, 4), dtype=f32, device=dev)
        self.pos_ref = torch.zeros((n, 4), dtype=f32, device=dev)
        self.ids = torch.arange(n, dtype=torch.int32, device=dev)
        self.perm = torch.zeros(max(n, 1), dtype=torch.int32, device=dev)
        self.cell_start = torch.zeros(self.grid.ncell + 1, dtype=torch.int32, device=dev)
        self.nbr = torch.zeros(fpm.fpm_verlet_list_bytes(n, self.grid, self.cap), dtype=torch.uint8, device=dev)
        self.nn = torch.zeros(max(n, 1), dtype=torch.int32, device=dev)
        self.hist = torch.zeros((self.cap * self.ld, 4), dtype=f32, device=dev)
        self.packed = torch.zeros(fpm.fpm_dem_packed_bytes(n), dtype=torch.uint8, device=dev)
        self.pending = torch.zeros(4, dtype=torch.int32, device=dev)
        self.ncontact = torch.zeros(4, dtype=torch.int32, device=dev)
        self.status = torch.zeros(fpm.STATUS_BYTES // 4, dtype=torch.int32, device=dev)
        self.ws_cell = torch.zeros(fpm.fpm_celllist_workspace(n, self.grid, fpm.FPM_F32), dtype=torch.uint8,
                                   device=dev)
        self.ws_red = torch.zeros(fpm.fpm_reduce_workspace(n, self.grid), dtype=torch.uint8, device=dev)
        self._body = torch.cuda.Stream(device=dev)
        self._graph = None
        self.rebuild()
        self.size_staging()

    # -- pieces ---------------------------------------------------------
    @property
    def gate_ptr(self) -> int:
        return self.status.data_ptr() + 8  # fpm_dev_status.rebuild

    def size_staging(self, margin: float = 1.15):
        """The staging capacity from the largest tile neighbourhood of the last
        Verlet build (synchronises)."""
        st = fpm.read_status(self.status)
        self.grid.stage_cap = int(math.ceil((margin * st.max_staged + 64) / 32.0)) * 32

    def rebuild(self, gated: bool = False, stream=None):
        gate = self.gate_ptr if gated else None
        fpm.fpm_dem_rebuild_begin(self.grid, self.n, self.cap, self.nbr, self.nn, self.hist, self.omega,
                                  self.packed, gate, self.pending, self.status, stream=stream)
        fpm.fpm_celllist_build(self.box, self.grid, self.n, fpm.FPM_F32, self.pos, self.vel, self.ids, self.pos,
                               self.vel, self.ids, self.cell_start, self.perm, self.ws_cell, self.status, gate,
                               stream=stream)
        fpm.fpm_verlet_build(self.box, self.grid, self.n, fpm.FPM_F32, self.pos, self.cell_start, self.r_list,
                             self.cap, self.nbr, self.nn, self.pos_ref, self.status, gate, stream=stream)
        fpm.fpm_dem_rebuild_end(self.grid, self.n, self.cap, self.nbr, self.nn, self.perm, self.packed, self.hist,
                                self.omega, self.pending, stream=stream)

    def _gated_rebuild(self):
        if fpm.fpm_graph_if_begin(self.gate_ptr, self._body):
            self.rebuild(gated=True, stream=self._body)
            fpm.fpm_graph_if_end(self._body)
        else:
            self.rebuild(gated=True)

    def compute_forces(self):
        fpm.fpm_dem_forces(self.box, self.grid, self.n, self.pos, self.vel, self.omega, self.nbr, self.nn, self.cap,
                           self.p, self.hist, self.force, self.torque, self.ncontact, self.ws_red, self.status)

    def _step(self):
        self._gated_rebuild()
        self.compute_forces()
        fpm.fpm_dem_leapfrog(self.box, self.n, self.p, self.pos, self.vel, self.omega, self.force, self.torque,
                             self.pos_ref, self.skin, self.status)

    # -- public -----------------------------------------------------------
    def step(self, nsteps: int = 1):
        for _ in range(int(nsteps)):
            self._step()

    def capture(self, steps_per_graph: int = 1):
        """Capture `steps_per_graph` whole steps into one CUDA graph."""
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

    def contacts(self) -> int:
        """Ordered contacts counted by the force sweeps so far (synchronises)."""
        return int(self.ncontact[0].item())

    def device_status(self) -> fpm.fpm_dev_status:
        return fpm.read_status(self.status)

    def check_status(self):
        st = self.device_status()
        code = fpm.fpm_status_from_device(st)
        if code != fpm.FPM_OK:
            raise fpm.FpmError(code, f"device status flags={st.flags} max_nn={st.max_nn} cap={self.cap}")
        return st

    def state_by_id(self):
        """(pos, vel, omega, force, torque) as numpy [n,4] in input (id) order."""
        ids = self.ids.cpu().numpy().view(np.uint32)
        out = []
        for t in (self.pos, self.vel, self.omega, self.force, self.torque):
            a = np.empty((self.n, 4), np.float32)
            a[ids] = t.cpu().numpy()
            out.append(a)
        return tuple(out)

    def history_by_id(self) -> dict:
        """{(id_p, id_q): u_t} of the entries with nonzero u_t (synchronises)."""
        dec = torch.full((self.cap * self.ld,), -1, dtype=torch.int32, device=self.device)
        fpm.fpm_verlet_decode(self.grid, self.n, self.cap, self.nbr, self.nn, dec)
        dec = dec.cpu().numpy().view(np.uint32).reshape(self.cap, self.ld)
        nn = self.nn[: self.n].cpu().numpy()
        ids = self.ids.cpu().numpy().view(np.uint32)
        h = self.hist.cpu().numpy().reshape(self.cap, self.ld, 4)
        out = {}
        for i in range(self.n):
            for k in range(int(nn[i])):
                u = h[k, i, :3]
                if np.any(u != 0):
                    out[(int(ids[i]), int(ids[dec[k, i]]))] = u.astype(np.float64)
        return out

    def set_history_by_id(self, hist: dict):
        """Load {(id_p, id_q): u_t} into the current list's entries (0 for the
        pairs not in `hist`)."""
        dec = torch.full((self.cap * self.ld,), -1, dtype=torch.int32, device=self.device)
        fpm.fpm_verlet_decode(self.grid, self.n, self.cap, self.nbr, self.nn, dec)
        dec = dec.cpu().numpy().view(np.uint32).reshape(self.cap, self.ld)
        nn = self.nn[: self.n].cpu().numpy()
        ids = self.ids.cpu().numpy().view(np.uint32)
        h = np.zeros((self.cap, self.ld, 4), np.float32)
        for i in range(self.n):
            for k in range(int(nn[i])):
                u = hist.get((int(ids[i]), int(ids[dec[k, i]])))
                if u is not None:
                    h[k, i, :3] = u
        self.hist.copy_(torch.as_tensor(h.reshape(-1, 4), device=self.device))
