"""Batched Lennard-Jones replicas over libfpm: R independent periodic systems
of uneven size (an ensemble of the MD system of Sec. 4.1) advanced together,
one launch per operation for the whole batch.

One step (all on the current stream, no host synchronisation) is one
launch, fpm_batch_step, whose phases do the work of the four separate calls
below (fused=False runs those instead; the results are the same bit for bit):
    fpm_batch_drift_check           v += dt/2 F; x += dt v; flag the replicas
                                    in which a particle moved > skin/2
    fpm_batch_celllist_build        re-bin and reorder the flagged replicas
    fpm_batch_verlet_build          their tiles and lists; flags cleared
    fpm_batch_lj_forces_kick        F, and U, W, pairs per replica; then
                                    v += dt/2 F in the same launch
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import fpm
from .md import default_cap


class LJBatch:
    def __init__(self, replicas, eps=1.0, sigma=1.0, rc=2.5, skin=0.3, dt=0.005, tile_target=0, cap=None,
                 device="cuda", fused=True):
        """replicas: sequence of (pos [n, >=3], vel [n, >=3], L [3]) per replica.
        fused: a step is the one launch fpm_batch_step (else four calls)."""
        self.device = torch.device(device)
        self.fused = bool(fused)
        self.eps, self.sigma, self.rc, self.skin, self.dt = float(eps), float(sigma), float(rc), float(skin), float(dt)
        self.r_list = self.rc + self.skin
        self.L = [np.broadcast_to(np.asarray(L, np.float64), (3,)).copy() for (_, _, L) in replicas]
        self.counts = [int(np.asarray(p).shape[0]) for (p, _, _) in replicas]
        self.boxes = [fpm.make_box(L, (1, 1, 1)) for L in self.L]
        self.R = len(replicas)
        rho_max = max(c / float(np.prod(L)) for c, L in zip(self.counts, self.L))
        self.cap = int(cap) if cap else default_cap(rho_max, self.r_list)
        n = sum(self.counts)
        self.n = n
        dev = self.device
        pos = np.zeros((n, 4), np.float32)
        vel = np.zeros((n, 4), np.float32)
        o = 0
        for (p, v, _), c in zip(replicas, self.counts):
            pos[o:o + c, :3] = np.asarray(p, np.float64)[:, :3]
            vel[o:o + c, :3] = np.asarray(v, np.float64)[:, :3]
            o += c
        self.pos = torch.as_tensor(pos, device=dev)
        self.vel = torch.as_tensor(vel, device=dev)
        self.force = torch.zeros_like(self.pos)
        self.pos_ref = torch.zeros_like(self.pos)
        self.ids = torch.arange(n, dtype=torch.int32, device=dev)
        self.perm = torch.zeros(max(n, 1), dtype=torch.int32, device=dev)
        self.nn = torch.zeros(max(n, 1), dtype=torch.int32, device=dev)
        self.status = torch.zeros(fpm.STATUS_BYTES // 4, dtype=torch.int32, device=dev)
        self.flags = torch.zeros(self.R, dtype=torch.int32, device=dev)
        self.energy = torch.zeros((self.R, 3), dtype=torch.float64, device=dev)
        self._graph = None
        self.plan(tile_target)

    # -- plan / tiles -------------------------------------------------------
    def plan(self, tile_target: int = 0, sweep_blocks: int = 0):
        """(Re)plan the batch's grids and tiles (tile_target particles per
        tile, 0 = default) and rebuild every replica's lists."""
        reps, b = fpm.fpm_batch_plan(self.boxes, self.counts, self.r_list, tile_target)
        b.sweep_blocks = int(sweep_blocks)
        if hasattr(self, "batch"):  # launch-shape choices are kept across re-plans
            b.sweep_threads = self.batch.sweep_threads
            b.step_blocks_per_sm = self.batch.step_blocks_per_sm
        self.reps, self.batch = reps, b
        self.tile_target = int(tile_target)
        raw = np.frombuffer(bytes(reps), dtype=np.uint8).copy()
        self.d_reps = torch.as_tensor(raw, device=self.device)
        self.p0 = np.array([reps[r].p0 for r in range(self.R)], np.int64)
        dev = self.device
        self.cell_start = torch.zeros(b.ncell_total + 1, dtype=torch.int32, device=dev)
        self.nbr = torch.zeros(fpm.fpm_batch_list_bytes(b, self.cap), dtype=torch.uint8, device=dev)
        self.ws_cell = torch.zeros(fpm.fpm_batch_celllist_workspace(b), dtype=torch.uint8, device=dev)
        self.ws_red = torch.zeros(fpm.fpm_batch_workspace(b), dtype=torch.uint8, device=dev)
        self._graph = None
        self.status[fpm.STATUS_MAX_STAGED] = 0  # the staging size follows the new tiles
        self.rebuild()
        self.size_staging()
        self.compute_forces()

    def size_staging(self, margin: float = 1.15):
        """Staging capacity from the largest tile neighbourhood of the last
        build (synchronises)."""
        st = fpm.read_status(self.status)
        self.batch.stage_cap = int(math.ceil((margin * st.max_staged + 64) / 32.0)) * 32

    def set_sweep_blocks(self, blocks: int):
        self.batch.sweep_blocks = int(blocks)
        self._graph = None

    def set_step_blocks_per_sm(self, blocks: int):
        """Blocks per SM the one-launch step's registers are bounded for
        (2, 3 or 4; 0: 4)."""
        self.batch.step_blocks_per_sm = int(blocks)
        self._graph = None

    def set_sweep_threads(self, threads: int):
        """Threads per block of the force sweep (128, 256 or 512; 0: 256)."""
        self.batch.sweep_threads = int(threads)
        self._graph = None

    # -- pieces ---------------------------------------------------------
    def rebuild(self, gated: bool = False):
        flag = self.flags if gated else None
        fpm.fpm_batch_celllist_build(self.batch, self.d_reps, self.pos, self.vel, self.ids, self.cell_start, self.perm,
                                     self.ws_cell, flag, self.status)
        fpm.fpm_batch_verlet_build(self.batch, self.d_reps, self.pos, self.cell_start, self.r_list, self.cap, self.nbr,
                                   self.nn, self.pos_ref, flag, self.status)

    def compute_forces(self):
        fpm.fpm_batch_lj_forces(self.batch, self.d_reps, self.pos, self.nbr, self.nn, self.cap, self.eps, self.sigma,
                                self.rc, self.force, self.energy, self.ws_red, self.status)

    def forces_and_kick(self):
        """compute_forces and the closing half-kick v += dt/2 F in one launch."""
        fpm.fpm_batch_lj_forces_kick(self.batch, self.d_reps, self.pos, self.nbr, self.nn, self.cap, self.eps,
                                     self.sigma, self.rc, self.force, self.energy, self.ws_red, self.status,
                                     self.vel, self.dt)

    def _step(self):
        if self.fused:
            fpm.fpm_batch_step(self.batch, self.d_reps, self.dt, self.skin, self.r_list, self.cap, self.eps,
                               self.sigma, self.rc, self.pos, self.vel, self.force, self.pos_ref, self.ids,
                               self.cell_start, self.perm, self.nbr, self.nn, self.flags, self.ws_cell, self.ws_red,
                               self.energy, self.status)
            return
        fpm.fpm_batch_drift_check(self.batch, self.d_reps, self.dt, self.pos, self.vel, self.force, self.pos_ref,
                                  self.skin, self.flags)
        self.rebuild(gated=True)
        self.forces_and_kick()

    # -- public -----------------------------------------------------------
    def step(self, nsteps: int = 1):
        for _ in range(int(nsteps)):
            self._step()

    def capture(self, steps_per_graph: int = 1):
        torch.cuda.synchronize()
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

    def check_status(self):
        st = fpm.read_status(self.status)
        code = fpm.fpm_status_from_device(st)
        if code != fpm.FPM_OK:
            raise fpm.FpmError(code, f"device status flags={st.flags} max_nn={st.max_nn} cap={self.cap}")
        return st

    def replica_range(self, r: int):
        return int(self.reps[r].p0), int(self.reps[r].p0) + int(self.reps[r].n)

    def energies(self) -> np.ndarray:
        """[R, 3]: U, W, pairs of each replica (synchronises)."""
        return self.energy.cpu().numpy()

    def neighbor_lists(self):
        """(nbr [cap, ld] uint32 of concatenated indices, nn [n])."""
        ld = fpm.fpm_nbr_ld(self.n)
        out = torch.full((self.cap * ld,), -1, dtype=torch.int32, device=self.device)
        fpm.fpm_batch_verlet_decode(self.batch, self.cap, self.nbr, self.nn, out)
        return (out.cpu().numpy().view(np.uint32).reshape(self.cap, ld),
                self.nn[: self.n].cpu().numpy().view(np.uint32))

    def state_numpy(self):
        """(pos, vel, ids) of the whole batch in the current (sorted) order."""
        return self.pos.cpu().numpy(), self.vel.cpu().numpy(), self.ids.cpu().numpy().view(np.uint32)
