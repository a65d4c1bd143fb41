"""Differentiable LJ rollout: the hand-written adjoint of the force sweep and of
velocity Verlet (libfpm's fpm_lj_backward / fpm_vv_adjoint / fpm_adjoint_seed)
behind a torch.autograd.Function, with step checkpointing and recomputation.

Loss: L = U(x_T) + sum_i |F_i(x_T)|^2 after T NVE steps from (x0, v0).
Gradients: dL/dx0, dL/dv0, dL/deps, dL/dsigma.

Forward: T steps of LJSystem in segments of `every` steps, each segment one
CUDA-graph replay; before each segment the full state (positions,
velocities, ids, reference positions, force, cell list and Verlet list) is
copied aside on the device.  Backward, segment by segment from the last:
restore the checkpoint and replay a recording graph of the segment
(bit-identical to the forward: every kernel is deterministic) that also keeps
each step's positions, the list in force at each step, the permutation of
the step's cell-list build and whether that build ran; then replay a reverse
graph of the segment:

    seed      xbar = -F_T + 2 J(x_T) F_T,  vbar = 0,  thbar = dU/dth + 2 F_T.dF/dth
    step n    undo the reorder of step n's rebuild (if it ran: a device-side
              gate); vbar += dt xbar; xbar += J(x_n) (c vbar);
              thbar += (c vbar).dF/dth(x_n), with c = dt, and c = dt/2 for n = 0

(the two half-kick terms that meet at x_n are merged into one sweep with
c = dt).  The adjoint state is FP64; pair arithmetic is in the positions'
precision.  No host synchronisation inside either pass: the rebuild
decisions stay on the device.  Every numeric step runs in libfpm's kernels;
this module only orders the calls and keeps the buffers.
"""
from __future__ import annotations

import torch

from . import fpm
from .md import LJSystem

_STATE = ("pos", "vel", "ids", "pos_ref", "force", "cell_start", "nbr", "nn")
_REBUILD_WORD = 2  # int32 word of fpm_dev_status.rebuild in a status tensor


def _capture(fn):
    """fn() captured into a CUDA graph on a side stream (nothing runs)."""
    torch.cuda.synchronize()
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            fn()
    torch.cuda.current_stream().wait_stream(st)
    return g


class LJAdjointRunner:
    def __init__(self, pos, vel, L, eps=1.0, sigma=1.0, rc=2.5, skin=0.3, dt=0.005, nsteps=200, every=20,
                 precision="f32", periodic=(1, 1, 1), cap=None):
        self.sys = LJSystem(pos, vel, L, periodic=periodic, eps=eps, sigma=sigma, rc=rc, skin=skin, dt=dt,
                            precision=precision, cap=cap)
        self.nsteps = int(nsteps)
        self.every = max(1, int(every))
        self.nseg = -(-self.nsteps // self.every)
        self.x_final = None
        s = self.sys
        dev = s.device
        self.adtype = s.dtype
        self.checkpoints = [{k: torch.empty_like(getattr(s, k)) for k in _STATE} for _ in range(self.nseg)]
        E = self.every
        self.xs = [torch.empty_like(s.pos) for _ in range(E + 1)]
        self.nbrs = [torch.empty_like(s.nbr) for _ in range(E + 1)]
        self.nns = [torch.empty_like(s.nn) for _ in range(E + 1)]
        self.perms = [torch.empty_like(s.perm) for _ in range(E)]
        self.rebuilt = torch.zeros(E, dtype=torch.int32, device=dev)
        self.rebuilt_total = torch.zeros(1, dtype=torch.int64, device=dev)
        self.xbar = torch.zeros((s.n, 4), dtype=torch.float64, device=dev)
        self.vbar = torch.zeros_like(self.xbar)
        self.xbar2 = torch.zeros_like(self.xbar)
        self.vbar2 = torch.zeros_like(self.xbar)
        self.avec = torch.zeros((s.n, 4), dtype=s.dtype, device=dev)
        self.theta_seed = torch.zeros(4, dtype=torch.float64, device=dev)
        self.theta_steps = torch.zeros(4, dtype=torch.float64, device=dev)
        self.sumf2 = torch.zeros(4, dtype=torch.float64, device=dev)
        self.loss_dev = torch.zeros(1, dtype=torch.float64, device=dev)
        self.grad_x = torch.zeros((s.n, 3), dtype=torch.float64, device=dev)
        self.grad_v = torch.zeros_like(self.grad_x)
        self.grad_theta = torch.zeros(2, dtype=torch.float64, device=dev)
        self._graphs = {}
        self.reorders_undone = 0

    def _seg_len(self, k: int) -> int:
        return min(self.every, self.nsteps - k * self.every)

    def _graph(self, key, fn):
        g = self._graphs.get(key)
        if g is None:
            g = self._graphs[key] = _capture(fn)
        return g

    # -- forward -----------------------------------------------------------
    def _save(self, k):
        s = self.sys
        for name in _STATE:
            self.checkpoints[k][name].copy_(getattr(s, name))

    def _restore(self, k):
        s = self.sys
        for name in _STATE:
            getattr(s, name).copy_(self.checkpoints[k][name])
        s.status.zero_()

    def _steps(self, L):
        for _ in range(L):
            self.sys._step()

    def forward(self) -> float:
        s = self.sys
        for k in range(self.nseg):
            L = self._seg_len(k)
            self._save(k)
            self._graph(("fwd", L), lambda L=L: self._steps(L)).replay()
        s.check_status()
        self.x_final = s.pos.clone()
        return self.loss()

    def loss(self) -> float:
        """U(x_T) + sum |F(x_T)|^2 from the current force and energy."""
        s = self.sys
        fpm.fpm_kinetic(s.n, s.prec, s.force, self.sumf2, s.ws_red)  # 1/2 sum |F|^2 in FP64
        fpm.fpm_adjoint_loss(s.energy, self.sumf2, self.loss_dev)
        return float(self.loss_dev.item())

    # -- backward ------------------------------------------------------------
    def _record(self, L):
        """The forward steps of one segment (the same calls as LJSystem._step)
        keeping, per step j, x_j, the list in force at x_j, the permutation of
        the step's cell-list build and its gate word."""
        s = self.sys
        self.xs[0].copy_(s.pos)
        self.nbrs[0].copy_(s.nbr)
        self.nns[0].copy_(s.nn)
        for j in range(L):
            fpm.fpm_vv_drift_check(s.box, s.n, s.prec, s.dt, s.pos, s.vel, s.force, s.pos_ref, s.skin, s.status)
            self.rebuilt[j:j + 1].copy_(s.status[_REBUILD_WORD:_REBUILD_WORD + 1])
            s.rebuild(gated=True)
            self.perms[j].copy_(s.perm)
            s.forces_and_kick()
            self.xs[j + 1].copy_(s.pos)
            self.nbrs[j + 1].copy_(s.nbr)
            self.nns[j + 1].copy_(s.nn)
        self.rebuilt_total += (self.rebuilt[:L] != 0).sum()

    def _sweep(self, j, scale, theta):
        s = self.sys
        fpm.fpm_lj_backward(s.box, s.grid, s.n, s.prec, self.xs[j], self.nbrs[j], self.nns[j], s.cap, s.eps, s.sigma,
                            s.rc, self.avec, scale, self.xbar, theta, s.ws_red, s.status)

    def _reverse(self, L, first):
        """The reverse steps of one segment, from xbar/vbar back into them."""
        s = self.sys
        dt = s.dt
        xa, va, xb, vb = self.xbar, self.vbar, self.xbar2, self.vbar2
        for j in range(L - 1, -1, -1):
            c = 0.5 * dt if (first and j == 0) else dt
            fpm.fpm_vv_adjoint(s.n, s.prec, self.perms[j], dt, c, xa, va, xb, vb, self.avec,
                               d_gate=self.rebuilt[j:j + 1])
            xa, xb, va, vb = xb, xa, vb, va
            fpm.fpm_lj_backward(s.box, s.grid, s.n, s.prec, self.xs[j], self.nbrs[j], self.nns[j], s.cap, s.eps,
                                s.sigma, s.rc, self.avec, 1.0, xa, self.theta_steps, s.ws_red, s.status)
        if xa is not self.xbar:  # odd segment length: the state ends in the second buffers
            self.xbar.copy_(xa)
            self.vbar.copy_(va)

    def backward(self):
        """Returns (dL/dx0 [n,3], dL/dv0 [n,3], dL/deps, dL/dsigma) as FP64 tensors,
        rows in the order of the particles given to the constructor."""
        s = self.sys
        self.theta_seed.zero_()
        self.theta_steps.zero_()
        self.rebuilt_total.zero_()
        last = self.nseg - 1
        for k in range(last, -1, -1):
            L = self._seg_len(k)
            self._restore(k)
            self._graph(("rec", L), lambda L=L: self._record(L)).replay()
            if k == last:
                if not torch.equal(self.xs[L], self.x_final):
                    raise RuntimeError("checkpoint recomputation is not bit-identical to the forward pass")
                # seed at x_T: xbar = -F, vbar = 0, a = F; xbar += 2 J F; theta += 2 F.dF/dth + dU/dth
                fpm.fpm_adjoint_seed(s.n, s.prec, s.force, self.xbar, self.vbar, self.avec)
                self._sweep(L, 2.0, self.theta_seed)
            self._graph(("rev", L, k == 0), lambda L=L, f=(k == 0): self._reverse(L, f)).replay()
        s.check_status()
        self.reorders_undone = int(self.rebuilt_total.item())
        # rows back to the caller's order (sorted slot k held particle ids[k] at
        # step 0) and dL/d(eps, sigma) from the seed's and the steps' partials
        fpm.fpm_adjoint_finish(s.n, self.checkpoints[0]["ids"], self.xbar, self.vbar, self.theta_seed,
                               self.theta_steps, self.grad_x, self.grad_v, self.grad_theta)
        gt = self.grad_theta.cpu().numpy()
        return self.grad_x.cpu(), self.grad_v.cpu(), float(gt[0]), float(gt[1])


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
