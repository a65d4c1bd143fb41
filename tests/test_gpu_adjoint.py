"""GPU parity of the hand-written LJ adjoint against the oracle.

* fpm_lj_backward (J a, a.dF/d(eps,sigma), dU/d(eps,sigma)) on identical
  positions and vectors: FP64 to 1e-11, FP32 to 1e-4 of the RMS (the HVP
  carries r^-16 terms, one power of r^-2 steeper than the force).
* The full reverse pass (checkpointed, with rebuild reorders undone) in FP64
  against the oracle's gradient of the same rollout: 1e-8 relative.
* The FP32-forward / FP64-accumulation gradient of the 32,768-particle
  workload against the FP64 oracle gradient: the error is measured and bounded
  (the FP32 trajectory differs from the FP64 one by rounding, amplified by the
  chaotic dynamics), see the test.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1804_07598_gb300 import fpm, inputs
from paper_1804_07598_gb300.adjoint import LJAdjointRunner, LJRollout
from paper_1804_07598_gb300.md import LJSystem

pytestmark = pytest.mark.gpu


def box_of(L, prec):
    L = np.asarray(L, np.float64)
    return L.astype(np.float32).astype(np.float64) if prec == "f32" else L


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_hvp_matches_oracle(cuda, prec):
    wl = inputs.WORKLOADS["lj_small"]
    pos, vel, L = inputs.lj_state(wl, jitter=0.06)
    s = LJSystem(pos, vel, L, precision=prec)
    rng = np.random.default_rng(5)
    a = np.zeros((s.n, 4))
    a[:, :3] = rng.normal(size=(s.n, 3))
    at = torch.tensor(a, dtype=s.dtype, device="cuda")
    out = torch.zeros((s.n, 4), dtype=torch.float64, device="cuda")
    par = torch.zeros(4, dtype=torch.float64, device="cuda")
    fpm.fpm_lj_backward(s.box, s.grid, s.n, s.prec, s.pos, s.nbr, s.nn, s.cap, 1.0, 1.0, 2.5, at, 1.0, out, par,
                        s.ws_red, s.status)
    torch.cuda.synchronize()
    s.check_status()
    p = s.pos.cpu().numpy().astype(np.float64)
    a_used = at.cpu().numpy().astype(np.float64)
    Ja, dth, dU = oracle.lj_hvp(p, a_used, box_of(L, prec), (1, 1, 1), 1.0, 1.0, 2.5, mask_f32=(prec == "f32"))
    g = out.cpu().numpy()
    rms = np.sqrt(np.mean(np.sum(Ja[:, :3] ** 2, axis=1)))
    err = np.max(np.linalg.norm(g[:, :3] - Ja[:, :3], axis=1)) / rms
    tol = 1e-11 if prec == "f64" else 1e-4
    assert err <= tol, err
    pv = par.cpu().numpy()
    ref = np.array([dth[0], dth[1], dU[0], dU[1]])
    tolp = 1e-11 if prec == "f64" else 1e-5
    assert np.all(np.abs(pv - ref) <= tolp * np.maximum(np.abs(ref), 1.0)), (pv, ref)


def _rollout_inputs(cells=(4, 4, 4), jitter=0.04):
    wl = inputs.LJWorkload("t", cells)
    x, v, L = inputs.lj_state(wl, jitter=jitter)
    return x, v, L


def test_full_gradient_fp64_matches_oracle(cuda):
    """40 steps, checkpoints every 7 (segments of uneven length), FP64 GPU path
    against the oracle's reverse pass of the same rollout."""
    x, v, L = _rollout_inputs()
    steps, dt = 40, 0.005
    r = LJAdjointRunner(x, v, L, nsteps=steps, every=7, precision="f64", dt=dt)
    loss = r.forward()
    gx, gv, ge, gs = r.backward()
    assert r.reorders_undone >= 1  # the reverse pass crossed a rebuild's reorder
    oloss, xb, vb, th = oracle.lj_rollout_grad(x, v, L, (1, 1, 1), 1.0, 1.0, 2.5, dt, steps)
    assert abs(loss - oloss) <= 1e-10 * abs(oloss)
    for got, ref in ((gx.numpy(), xb), (gv.numpy(), vb)):
        assert np.max(np.abs(got - ref)) <= 1e-8 * np.max(np.abs(ref))
    assert abs(ge - th[0]) <= 1e-8 * abs(th[0]) and abs(gs - th[1]) <= 1e-8 * abs(th[1])


def test_fp32_gradient_against_fp64_oracle(cuda):
    """The 32,768-particle workload (FCC 16x16x32), its full 200 steps,
    checkpoints every 20 (the bench's configuration): FP32 forward with FP64
    adjoint accumulation against the FP64 oracle gradient.  Observed relative error (max over particles of the
    gradient row difference / max row norm) is printed; bound 1e-2."""
    wl = inputs.WORKLOADS["lj_adjoint"]
    x, v, L = inputs.lj_state(wl)
    steps = 200
    r = LJAdjointRunner(x, v, L, nsteps=steps, every=20, precision="f32", dt=wl.dt)
    loss = r.forward()
    gx, gv, ge, gs = r.backward()
    oloss, xb, vb, th = oracle.lj_rollout_grad(x, v, L, (1, 1, 1), 1.0, 1.0, 2.5, wl.dt, steps)
    ex = np.max(np.linalg.norm(gx.numpy() - xb, axis=1)) / np.max(np.linalg.norm(xb, axis=1))
    ev = np.max(np.linalg.norm(gv.numpy() - vb, axis=1)) / np.max(np.linalg.norm(vb, axis=1))
    ee, es = abs(ge - th[0]) / abs(th[0]), abs(gs - th[1]) / abs(th[1])
    print(f"FP32 adjoint vs FP64 oracle, {steps} steps: loss {abs(loss - oloss) / abs(oloss):.2e}, "
          f"x0 {ex:.2e}, v0 {ev:.2e}, eps {ee:.2e}, sigma {es:.2e}")
    assert abs(loss - oloss) <= 1e-4 * abs(oloss)
    assert ex <= 1e-2 and ev <= 1e-2 and ee <= 1e-2 and es <= 1e-2


def test_autograd_function(cuda):
    x, v, L = _rollout_inputs(cells=(4, 4, 4))
    cfg = dict(L=L, nsteps=15, every=5, precision="f64")
    x0 = torch.tensor(x[:, :3], dtype=torch.float64, requires_grad=True)
    v0 = torch.tensor(v[:, :3], dtype=torch.float64, requires_grad=True)
    eps = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    sig = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    loss = LJRollout.apply(x0, v0, eps, sig, cfg)
    loss.backward()
    oloss, xb, vb, th = oracle.lj_rollout_grad(x, v, L, (1, 1, 1), 1.0, 1.0, 2.5, 0.005, 15)
    assert abs(loss.item() - oloss) <= 1e-10 * abs(oloss)
    assert np.max(np.abs(x0.grad.numpy() - xb)) <= 1e-8 * np.max(np.abs(xb))
    assert np.max(np.abs(v0.grad.numpy() - vb)) <= 1e-8 * np.max(np.abs(vb))
    assert abs(eps.grad.item() - th[0]) <= 1e-8 * abs(th[0])
    assert abs(sig.grad.item() - th[1]) <= 1e-8 * abs(th[1])
