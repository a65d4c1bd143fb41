"""Pins of the oracle's adjoint against central finite differences in FP64
(independent of the adjoint code: only the forward force/energy routines are
re-evaluated) and against the symmetry of the Hessian."""
import numpy as np
import pytest

import oracle
from paper_1804_07598_gb300 import inputs

PER = (1, 1, 1)


def small_state(cells=(3, 3, 3), jitter=0.07, seed=7):
    wl = inputs.LJWorkload("t", cells)
    x, v, L = inputs.lj_state(wl, jitter=jitter, jitter_seed=seed)
    return x, v, L


def test_hvp_matches_force_differences():
    """J a = (F(x + h a) - F(x - h a)) / 2h."""
    x, _, L = small_state()
    rng = np.random.default_rng(1)
    a = np.zeros_like(x)
    a[:, :3] = rng.normal(size=(x.shape[0], 3))
    Ja, _, _ = oracle.lj_hvp(x, a, L, PER, 1.0, 1.0, 2.5)
    h = 1e-6
    fp, _, _, np1 = oracle.lj_forces(x + h * a, L, PER, 1.0, 1.0, 2.5)
    fm, _, _, np2 = oracle.lj_forces(x - h * a, L, PER, 1.0, 1.0, 2.5)
    assert np1 == np2
    fd = (fp - fm)[:, :3] / (2 * h)
    assert np.max(np.abs(fd - Ja[:, :3])) <= 1e-6 * np.max(np.abs(fd))


def test_hessian_symmetric():
    x, _, L = small_state()
    rng = np.random.default_rng(2)
    a, b = np.zeros_like(x), np.zeros_like(x)
    a[:, :3] = rng.normal(size=(x.shape[0], 3))
    b[:, :3] = rng.normal(size=(x.shape[0], 3))
    Ja, _, _ = oracle.lj_hvp(x, a, L, PER, 1.0, 1.0, 2.5)
    Jb, _, _ = oracle.lj_hvp(x, b, L, PER, 1.0, 1.0, 2.5)
    lhs, rhs = np.sum(b[:, :3] * Ja[:, :3]), np.sum(a[:, :3] * Jb[:, :3])
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


@pytest.mark.parametrize("which", [0, 1])
def test_parameter_derivatives(which):
    """a . dF/d(eps, sigma) and dU/d(eps, sigma) by central differences."""
    x, _, L = small_state()
    rng = np.random.default_rng(3)
    a = np.zeros_like(x)
    a[:, :3] = rng.normal(size=(x.shape[0], 3))
    eps, sig = 0.9, 1.05
    _, dth, dU = oracle.lj_hvp(x, a, L, PER, eps, sig, 2.5)
    h = 1e-6
    pe = [eps + h, sig] if which == 0 else [eps, sig + h]
    me = [eps - h, sig] if which == 0 else [eps, sig - h]
    fp, Up, _, _ = oracle.lj_forces(x, L, PER, pe[0], pe[1], 2.5)
    fm, Um, _, _ = oracle.lj_forces(x, L, PER, me[0], me[1], 2.5)
    fd_th = np.sum(a[:, :3] * (fp - fm)[:, :3]) / (2 * h)
    fd_U = (Up - Um) / (2 * h)
    assert abs(dth[which] - fd_th) <= 1e-6 * max(abs(fd_th), 1.0)
    assert abs(dU[which] - fd_U) <= 1e-6 * max(abs(fd_U), 1.0)


def test_rollout_gradient_matches_finite_differences():
    """Full adjoint of 20 VV steps + loss U + sum|F|^2, against central
    differences (h = 1e-6) of the loss for sampled initial coordinates,
    velocities and both parameters; a sample is skipped if the pair set at the
    last step differs between +h and -h (the cutoff makes the loss
    non-differentiable there)."""
    x, v, L = small_state(cells=(3, 3, 3), jitter=0.05)
    steps, dt = 20, 0.005
    eps, sig, rc = 1.0, 1.0, 2.5
    loss, xbar, vbar, thbar = oracle.lj_rollout_grad(x, v, L, PER, eps, sig, rc, dt, steps)
    rng = np.random.default_rng(11)
    h = 1e-6
    checked = 0
    for _ in range(8):
        i, d = int(rng.integers(0, x.shape[0])), int(rng.integers(0, 3))
        for arr, bar in ((x, xbar), (v, vbar)):
            ap, am = arr.copy(), arr.copy()
            ap[i, d] += h
            am[i, d] -= h
            if arr is x:
                lp = oracle.lj_rollout_loss(ap, v, L, PER, eps, sig, rc, dt, steps)
                lm = oracle.lj_rollout_loss(am, v, L, PER, eps, sig, rc, dt, steps)
            else:
                lp = oracle.lj_rollout_loss(x, ap, L, PER, eps, sig, rc, dt, steps)
                lm = oracle.lj_rollout_loss(x, am, L, PER, eps, sig, rc, dt, steps)
            fd = (lp - lm) / (2 * h)
            if abs(fd - bar[i, d]) > 1e-5 * max(abs(fd), 1.0):
                # accept only if a pair crossed the cutoff between +h and -h
                pp, _, _ = oracle.lj_nve(ap if arr is x else x, v if arr is x else ap, L, PER, eps, sig, rc, dt,
                                         steps, record=False)
                pm, _, _ = oracle.lj_nve(am if arr is x else x, v if arr is x else am, L, PER, eps, sig, rc, dt,
                                         steps, record=False)
                n1 = oracle.lj_forces(pp, L, PER, eps, sig, rc)[3]
                n2 = oracle.lj_forces(pm, L, PER, eps, sig, rc)[3]
                assert n1 != n2, (i, d, fd, bar[i, d])
            else:
                checked += 1
    assert checked >= 12
    for k, (pe, me) in enumerate((((eps + h, sig), (eps - h, sig)), ((eps, sig + h), (eps, sig - h)))):
        lp = oracle.lj_rollout_loss(x, v, L, PER, pe[0], pe[1], rc, dt, steps)
        lm = oracle.lj_rollout_loss(x, v, L, PER, me[0], me[1], rc, dt, steps)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - thbar[k]) <= 1e-5 * max(abs(fd), 1.0), (k, fd, thbar[k])
