"""Differentiable LJ rollout: the hand-written adjoint of the force sweep and of
velocity Verlet (libfpm's fpm_lj_backward / fpm_vv_adjoint / fpm_adjoint_seed)
behind a torch.autograd.Function, with step checkpointing and recomputation.

Loss: L = U(x_T) + sum_i |F_i(x_T)|^2 after T NVE steps from (x0, v0).
Gradients: dL/dx0, dL/dv0, dL/deps, dL/dsigma.

Forward: T steps of LJSystem; every `every` steps the full state (positions,
velocities, ids, reference positions, force, cell list and Verlet list) is
copied aside.  Backward, segment by segment from the last: restore the
checkpoint, recompute the segment (bit-identical: every kernel is
deterministic), keeping each step's positions, the list in force at each step
and the permutation of each rebuild, then walk the steps in reverse:

    seed      xbar = -F_T + 2 J(x_T) F_T,  vbar = 0,  thbar = dU/dth + 2 F_T.dF/dth
    step n    undo the reorder of step n's rebuild (if any); vbar += dt xbar;
              xbar += J(x_n) (c vbar);  thbar += (c vbar).dF/dth(x_n)
              with c = dt, and c = dt/2 for n = 0

(the two half-kick terms that meet at x_n are merged into one sweep with
c = dt).  The adjoint state is FP64; pair arithmetic is in the positions'
precision.  Every numeric step runs in libfpm's kernels; this module only
orders the calls and keeps the buffers.
"""
from __future__ import annotations

import numpy as np
import torch

from . import fpm
from .md import LJSystem

_STATE = ("pos", "vel", "ids", "pos_ref", "force", "cell_start", "nbr", "nn")


class LJAdjointRunner:
    def __init__(self, pos, vel, L, eps=1.0, sigma=1.0, rc=2.5, skin=0.3, dt=0.005, nsteps=200, every=20,
                 precision="f32", periodic=(1, 1, 1), cap=None):
        self.sys = LJSystem(pos, vel, L, periodic=periodic, eps=eps, sigma=sigma, rc=rc, skin=skin, dt=dt,
                            precision=precision, cap=cap)
        self.nsteps = int(nsteps)
        self.every = max(1, int(every))
        self.checkpoints = []
        self.x_final = None
        s = self.sys
        dev = s.device
        self.adtype = s.dtype
        self.xbar = torch.zeros((s.n, 4), dtype=torch.float64, device=dev)
        self.vbar = torch.zeros_like(self.xbar)
        self.xbar2 = torch.zeros_like(self.xbar)
        self.vbar2 = torch.zeros_like(self.xbar)
        self.avec = torch.zeros((s.n, 4), dtype=s.dtype, device=dev)
        self.theta_seed = torch.zeros(4, dtype=torch.float64, device=dev)
        self.theta_steps = torch.zeros(4, dtype=torch.float64, device=dev)
        self.sumf2 = torch.zeros(4, dtype=torch.float64, device=dev)

    # -- forward -----------------------------------------------------------
    def _save(self):
        s = self.sys
        return {k: getattr(s, k).clone() for k in _STATE}

    def _restore(self, ck):
        s = self.sys
        for k in _STATE:
            getattr(s, k).copy_(ck[k])
        s.status.zero_()

    def forward(self) -> float:
        s = self.sys
        self.checkpoints = []
        for n in range(self.nsteps):
            if n % self.every == 0:
                self.checkpoints.append(self._save())
            s.step(1)
        s.check_status()
        self.x_final = s.pos.clone()
        return self.loss()

    def loss(self) -> float:
        """U(x_T) + sum |F(x_T)|^2 from the current force and energy."""
        s = self.sys
        fpm.fpm_kinetic(s.n, s.prec, s.force, self.sumf2, s.ws_red)  # 1/2 sum |F|^2 in FP64
        return float(s.energy[0].item() + 2.0 * self.sumf2[0].item())

    # -- backward ------------------------------------------------------------
    def _recompute(self, k):
        """Re-run segment k from its checkpoint; returns per-step positions, the
        list in force at each step and the permutations of rebuilds."""
        s = self.sys
        start = k * self.every
        end = min(start + self.every, self.nsteps)
        self._restore(self.checkpoints[k])
        xs = {start: s.pos.clone()}
        cur = (s.nbr.clone(), s.nn.clone())
        lists = {start: cur}
        perms = {}
        nr = s.device_status().nrebuild
        for n in range(start, end):
            s.step(1)
            nr1 = s.device_status().nrebuild
            if nr1 != nr:
                perms[n] = s.perm.clone()
                cur = (s.nbr.clone(), s.nn.clone())
                nr = nr1
            xs[n + 1] = s.pos.clone()
            lists[n + 1] = cur
        s.check_status()
        return xs, lists, perms, start, end

    def _sweep(self, pos, lst, scale, theta):
        s = self.sys
        nbr, nn = lst
        fpm.fpm_lj_backward(s.box, s.grid, s.n, s.prec, pos, nbr, nn, s.cap, s.eps, s.sigma, s.rc, self.avec, scale,
                            self.xbar, theta, s.ws_red, s.status)

    def backward(self):
        """Returns (dL/dx0 [n,3], dL/dv0 [n,3], dL/deps, dL/dsigma) as FP64 tensors,
        rows in the order of the particles given to the constructor."""
        s = self.sys
        dt = s.dt
        self.theta_seed.zero_()
        self.theta_steps.zero_()
        self.reorders_undone = 0
        # seed at x_T (the current state after forward / the last recomputation)
        segs = list(range(len(self.checkpoints)))
        xs, lists, perms, start, end = self._recompute(segs[-1])
        if not torch.equal(xs[end], self.x_final):
            raise RuntimeError("checkpoint recomputation is not bit-identical to the forward pass")
        fpm.fpm_adjoint_seed(s.n, s.prec, s.force, self.xbar, self.vbar, self.avec)
        # xbar += 2 J F; theta[0:2] += 2 F.dF/dth; theta[2:4] += dU/dth
        self._sweep(xs[end], lists[end], 2.0, self.theta_seed)
        for k in reversed(segs):
            if k != segs[-1]:
                xs, lists, perms, start, end = self._recompute(k)
            for n in range(end - 1, start - 1, -1):
                c = dt if n > 0 else 0.5 * dt
                perm = perms.get(n)
                if perm is not None:
                    self.reorders_undone += 1
                    fpm.fpm_vv_adjoint(s.n, s.prec, perm, dt, c, self.xbar, self.vbar, self.xbar2, self.vbar2,
                                       self.avec)
                    self.xbar, self.xbar2 = self.xbar2, self.xbar
                    self.vbar, self.vbar2 = self.vbar2, self.vbar
                else:
                    fpm.fpm_vv_adjoint(s.n, s.prec, None, dt, c, self.xbar, self.vbar, self.xbar, self.vbar,
                                       self.avec)
                self._sweep(xs[n], lists[n], 1.0, self.theta_steps)  # J(x_n) (c vbar)
        s.check_status()
        # back to the caller's particle order (host-side): sorted slot k holds particle ids[k]
        ids = self.checkpoints[0]["ids"].cpu().numpy().view(np.uint32).astype(np.int64)  # order at step 0
        xb, vb = self.xbar.cpu().numpy(), self.vbar.cpu().numpy()
        gx = np.empty((s.n, 3))
        gv = np.empty((s.n, 3))
        gx[ids] = xb[:, :3]
        gv[ids] = vb[:, :3]
        ts, tt = self.theta_seed.cpu().numpy(), self.theta_steps.cpu().numpy()
        # the seed sweep holds 2 F.dF/dth and dU/dth; the step sweeps hold a.dF/dth (their dU terms are unused)
        return torch.from_numpy(gx), torch.from_numpy(gv), float(ts[0] + ts[2] + tt[0]), float(ts[1] + ts[3] + tt[1])


class LJRollout(torch.autograd.Function):
    """loss = LJRollout.apply(x0, v0, eps, sigma, cfg) with cfg a dict of
    LJAdjointRunner arguments (L, rc, skin, dt, nsteps, every, precision).
    x0, v0: [n,3] float64 tensors; eps, sigma: 0-dim float64 tensors."""

    @staticmethod
    def forward(ctx, x0, v0, eps, sigma, cfg):
        runner = LJAdjointRunner(x0.detach().cpu().numpy(), v0.detach().cpu().numpy(), cfg["L"],
                                 eps=float(eps), sigma=float(sigma), rc=cfg.get("rc", 2.5), skin=cfg.get("skin", 0.3),
                                 dt=cfg.get("dt", 0.005), nsteps=cfg.get("nsteps", 200), every=cfg.get("every", 20),
                                 precision=cfg.get("precision", "f32"))
        loss = runner.forward()
        ctx.runner = runner
        ctx.dev = x0.device
        return torch.tensor(loss, dtype=torch.float64, device=x0.device)

    @staticmethod
    def backward(ctx, gout):
        gx, gv, ge, gs = ctx.runner.backward()
        g = gout.to(torch.float64)
        return ((g * gx).to(ctx.dev), (g * gv).to(ctx.dev), g * ge, g * gs, None)
