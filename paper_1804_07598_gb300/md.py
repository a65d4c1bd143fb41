"""Lennard-Jones NVE driver over libfpm (the MD test case of Sec. 4.1 /
Listing 4.1): state buffers in device memory, the velocity-Verlet step with a
device-gated Verlet rebuild, and CUDA-graph capture of whole steps.

One step (all on the current stream, no host synchronisation):
    fpm_vv_drift_check          v += dt/2 F; x += dt v (no wrap until the rebuild);
                                rebuild flag := max |x - x_ref| > skin/2
    fpm_celllist_build [gated]  wrap, re-bin and reorder in place
    fpm_verlet_build   [gated]  new list, x_ref := x, flag cleared
    fpm_lj_forces_kick          F, U, W, pairs; then v += dt/2 F in the same launch
Under CUDA-graph capture the two gated calls sit in the body of a
conditional node on the rebuild flag (fpm_graph_if_begin), so a replayed
step without a rebuild launches none of their kernels.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import fpm


def default_cap(rho: float, r_list: float) -> int:
    """Neighbour-list capacity: 1.5x the mean full-list count at density rho,
    rounded up to a multiple of 8 (at least 32)."""
    mean = 4.0 / 3.0 * math.pi * r_list ** 3 * rho
    return max(32, int(math.ceil(1.5 * mean / 8.0)) * 8)


# Systems of at most SMALL_N particles take tiles of about SMALL_TILE
# particles (the library's force sweep splits each list over several threads
# for such tiles).  Larger systems fill the GPU with the default tiles, which
# the other tile sweeps (the Verlet scan, the adjoint's Hessian-vector sweep)
# also run best on: at 32,768 particles the finer tiles cost the adjoint's
# sweep 36 -> 50 us.
SMALL_N = 16384
SMALL_TILE = 40


class LJSystem:
    def __init__(self, pos, vel, L, periodic=(1, 1, 1), eps=1.0, sigma=1.0, rc=2.5, skin=0.3, dt=0.005,
                 precision="f32", cap=None, device="cuda", half=False):
        """half: the symmetric sweep over a half list (each pair once,
        fpm_verlet_build_half + fpm_lj_forces_half; single precision only)."""
        if half and precision != "f32":
            raise ValueError("the half-list sweep is single precision only")
        self.half = bool(half)
        self.dtype = torch.float32 if precision == "f32" else torch.float64
        self.prec = fpm.FPM_F32 if precision == "f32" else fpm.FPM_F64
        self.device = torch.device(device)
        pos = torch.as_tensor(np.asarray(pos), dtype=torch.float64)
        vel = torch.as_tensor(np.asarray(vel), dtype=torch.float64)
        n = pos.shape[0]
        self.n = n
        self.L = np.broadcast_to(np.asarray(L, np.float64), (3,)).copy()
        self.periodic = tuple(int(p) for p in periodic)
        self.eps, self.sigma, self.rc, self.skin, self.dt = float(eps), float(sigma), float(rc), float(skin), float(dt)
        self.r_list = self.rc + self.skin
        self.box = fpm.make_box(self.L, self.periodic)
        self.grid = fpm.fpm_grid_make(self.box, self.r_list, n)
        if 0 < n <= SMALL_N and not self.half:
            # a small system has too few tiles of the default width to fill
            # the GPU: tiles of about SMALL_TILE particles, whose force sweep
            # gives each home particle several threads (a launch shape only)
            per_cell = n / max(1, int(self.grid.ncell))
            w = max(1, int(round(SMALL_TILE / per_cell)))
            nc0 = int(self.grid.nc[0])
            self.grid.tiles_x = min(nc0, max(int(self.grid.tiles_x), -(-nc0 // w)))
        vol = float(np.prod(self.L))
        self.cap = int(cap) if cap else default_cap(max(n, 1) / vol, self.r_list)
        if self.half and not cap:
            # a half list holds about half the entries, but its counts spread
            # more (a particle early in its cell's order lists the rest of it)
            self.cap = max(32, (4 * self.cap // 5 + 7) // 8 * 8)
        self.ld = fpm.fpm_nbr_ld(n)
        dev, dt_ = self.device, self.dtype
        self.pos = torch.zeros((n, 4), dtype=dt_, device=dev)
        self.vel = torch.zeros((n, 4), dtype=dt_, device=dev)
        self.pos[:, :pos.shape[1]] = pos[:, :4].to(dt_)
        self.vel[:, :vel.shape[1]] = vel[:, :4].to(dt_)
        self.pos[:, 3] = 0
        self.vel[:, 3] = 0
        self.force = torch.zeros((n, 4), dtype=dt_, device=dev)
        self.pos_ref = torch.zeros((n, 4), dtype=dt_, device=dev)
        self.ids = torch.arange(n, dtype=torch.int32, device=dev)
        self.perm = torch.zeros(max(n, 1), dtype=torch.int32, device=dev)
        self.cell_start = torch.zeros(self.grid.ncell + 1, dtype=torch.int32, device=dev)
        self.nbr = torch.zeros(fpm.fpm_verlet_list_bytes(n, self.grid, self.cap), dtype=torch.uint8, device=dev)
        self.nn = torch.zeros(max(n, 1), dtype=torch.int32, device=dev)
        self.status = torch.zeros(fpm.STATUS_BYTES // 4, dtype=torch.int32, device=dev)
        self.ws_cell = torch.zeros(fpm.fpm_celllist_workspace(n, self.grid, self.prec), dtype=torch.uint8, device=dev)
        self.ws_red = torch.zeros(fpm.fpm_reduce_workspace(n, self.grid), dtype=torch.uint8, device=dev)
        self.energy = torch.zeros(3, dtype=torch.float64, device=dev)
        self.acc = (torch.zeros(fpm.fpm_lj_half_acc_bytes(n) // 8, dtype=torch.int64, device=dev) if self.half
                    else None)
        self.kin = torch.zeros(4, dtype=torch.float64, device=dev)
        self._body = torch.cuda.Stream(device=dev)  # captures the conditional rebuild
        self._graph = None
        self.rebuild()
        self.size_staging()
        self.compute_forces()

    def retile(self, tiles_x, sweep_blocks=None):
        """New number of tiles per cell row (a launch-shape choice):
        reallocates the list, rebuilds it and resizes the staging
        (synchronises)."""
        self.grid.tiles_x = int(tiles_x)
        self.grid.stage_cap = 0
        if sweep_blocks is not None:
            self.grid.sweep_blocks = int(sweep_blocks)
        self.nbr = torch.zeros(fpm.fpm_verlet_list_bytes(self.n, self.grid, self.cap), dtype=torch.uint8,
                               device=self.device)
        self.ws_red = torch.zeros(fpm.fpm_reduce_workspace(self.n, self.grid), dtype=torch.uint8, device=self.device)
        self._graph = None
        self.status[fpm.STATUS_MAX_STAGED] = 0  # the staging size follows the new tiles
        self.rebuild()
        self.size_staging()
        self.compute_forces()

    def size_staging(self, margin: float = 1.15):
        """Set the grid's shared-memory staging capacity from the largest tile
        neighbourhood the last Verlet build saw (synchronises)."""
        st = fpm.read_status(self.status)
        self.grid.stage_cap = int(math.ceil((margin * st.max_staged + 64) / 32.0)) * 32

    # -- pieces ---------------------------------------------------------
    @property
    def gate_ptr(self) -> int:
        return self.status.data_ptr() + 8  # fpm_dev_status.rebuild

    def rebuild(self, gated: bool = False, stream=None):
        gate = self.gate_ptr if gated else None
        fpm.fpm_celllist_build(self.box, self.grid, self.n, self.prec, self.pos, self.vel, self.ids, self.pos,
                               self.vel, self.ids, self.cell_start, self.perm, self.ws_cell, self.status, gate,
                               stream=stream)
        build = fpm.fpm_verlet_build_half if self.half else fpm.fpm_verlet_build
        build(self.box, self.grid, self.n, self.prec, self.pos, self.cell_start, self.r_list, self.cap, self.nbr,
              self.nn, self.pos_ref, self.status, gate, stream=stream)

    def _gated_rebuild(self):
        """The step's rebuild: a conditional graph node under capture, gated
        launches otherwise."""
        if fpm.fpm_graph_if_begin(self.gate_ptr, self._body):
            self.rebuild(gated=True, stream=self._body)
            fpm.fpm_graph_if_end(self._body)
        else:
            self.rebuild(gated=True)

    def compute_forces(self):
        if self.half:
            fpm.fpm_lj_forces_half(self.box, self.grid, self.n, self.pos, self.nbr, self.nn, self.cap, self.eps,
                                   self.sigma, self.rc, self.force, self.energy, self.acc, self.ws_red, self.status)
            return
        fpm.fpm_lj_forces(self.box, self.grid, self.n, self.prec, self.pos, self.nbr, self.nn, self.cap, self.eps,
                          self.sigma, self.rc, self.force, self.energy, self.ws_red, self.status)

    def forces_and_kick(self):
        """compute_forces, then the closing half-kick v += dt/2 F, in one
        launch (bit-identical to the two calls)."""
        if self.half:
            fpm.fpm_lj_forces_half(self.box, self.grid, self.n, self.pos, self.nbr, self.nn, self.cap, self.eps,
                                   self.sigma, self.rc, self.force, self.energy, self.acc, self.ws_red, self.status,
                                   self.vel, self.dt)
            return
        fpm.fpm_lj_forces_kick(self.box, self.grid, self.n, self.prec, self.pos, self.nbr, self.nn, self.cap,
                               self.eps, self.sigma, self.rc, self.force, self.energy, self.ws_red, self.status,
                               self.vel, self.dt)

    def _step(self):
        fpm.fpm_vv_drift_check(self.box, self.n, self.prec, self.dt, self.pos, self.vel, self.force, self.pos_ref,
                               self.skin, self.status)
        self._gated_rebuild()
        self.forces_and_kick()

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

    def run(self, nsteps: int):
        """nsteps steps, through the captured graph when there is one."""
        if self._graph is None:
            self.step(nsteps)
            return
        g, k = self._graph
        for _ in range(nsteps // k):
            g.replay()
        self.step(nsteps % k)

    def kinetic(self):
        fpm.fpm_kinetic(self.n, self.prec, self.vel, self.kin, self.ws_red)
        return self.kin

    def observables(self) -> dict:
        """KE, U, W, pairs, momentum (host values; synchronises)."""
        k = self.kinetic().cpu().numpy()
        e = self.energy.cpu().numpy()
        return dict(KE=float(k[0]), U=float(e[0]), W=float(e[1]), pairs=int(round(e[2])), P=k[1:4].copy())

    def device_status(self) -> fpm.fpm_dev_status:
        return fpm.read_status(self.status)

    def check_status(self):
        st = self.device_status()
        code = fpm.fpm_status_from_device(st)
        if code != fpm.FPM_OK:
            raise fpm.FpmError(code, f"device status flags={st.flags} max_nn={st.max_nn} cap={self.cap}")
        return st

    def neighbor_lists(self):
        """The Verlet list as particle indices: (nbr [cap, ld] uint32, nn [n])."""
        out = torch.full((self.cap * self.ld,), -1, dtype=torch.int32, device=self.device)
        fpm.fpm_verlet_decode(self.grid, self.n, self.cap, self.nbr, self.nn, out)
        return (out.cpu().numpy().view(np.uint32).reshape(self.cap, self.ld),
                self.nn[: self.n].cpu().numpy().view(np.uint32))

    def state_numpy(self):
        """(pos, vel, ids) in the current (sorted) order, as numpy."""
        return (self.pos.cpu().numpy(), self.vel.cpu().numpy(), self.ids.cpu().numpy().view(np.uint32))
