"""GPU parity of the symmetric (half-list) Lennard-Jones path against the
oracle: the half list (fpm_verlet_build_half) holds every pair inside r_list
exactly once, so its pairs are the oracle's full neighbour sets with each
pair counted once; the sweep (fpm_lj_forces_half) gives the oracle's forces,
energy, virial and pair count within the FP32 tolerances of the full-list
sweep; its fixed-point sums make it bit-reproducible; and the half-kick in
its finishing pass equals a separate kick.

Tolerances: forces max |F - F_ref| / RMS(F_ref) <= 1e-5; U, W relative
<= 1e-6; pair counts exact (the cutoff decided in FP32 on both sides)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1804_07598_gb300 import fpm, inputs
from paper_1804_07598_gb300.md import LJSystem

pytestmark = pytest.mark.gpu

TOL_F, TOL_E = 1e-5, 1e-6


def f32box(L):
    return np.asarray(L, np.float64).astype(np.float32).astype(np.float64)


def half_pairs(s):
    """The list's entries as unordered pairs of sorted indices (a list, so
    that a pair listed twice shows up)."""
    nbr, nn = s.neighbor_lists()
    out = []
    for i in range(s.n):
        for j in nbr[: nn[i], i]:
            out.append((min(i, int(j)), max(i, int(j))))
    return out


def oracle_pairs(pos32, L, periodic, r_list):
    offs, nbr = oracle.neighbors(pos32, f32box(L), periodic, r_list)
    out = set()
    for i in range(pos32.shape[0]):
        for j in nbr[offs[i]:offs[i + 1]]:
            if i < j:
                out.add((i, int(j)))
    return out


def check_forces(s):
    torch.cuda.synchronize()
    s.check_status()
    pos = s.pos.cpu().numpy().astype(np.float64)
    f = s.force.cpu().numpy().astype(np.float64)
    fref, U, W, pairs = oracle.lj_forces(pos, f32box(s.L), s.periodic, s.eps, s.sigma, s.rc, mask_f32=True)
    e = s.energy.cpu().numpy()
    rms = np.sqrt(np.mean(np.sum(fref[:, :3] ** 2, axis=1)))
    err = np.max(np.linalg.norm(f[:, :3] - fref[:, :3], axis=1)) / rms
    assert err <= TOL_F, err
    assert abs(e[0] - U) <= TOL_E * abs(U), (e[0], U)
    assert abs(e[1] - W) <= TOL_E * abs(W), (e[1], W)
    assert int(round(e[2])) == pairs
    assert np.all(f[:, 3] == 0.0)
    return err


def boxes():
    """(name, pos [n,4], L, periodic): the 4000-atom liquid, a box with a
    non-periodic y, a box with one cell per dimension (every pair a
    candidate), and a jittered box of three cells per dimension (staged cells
    repeat through the periodic walls)."""
    wl = inputs.WORKLOADS["lj_small"]
    pos, _, L = inputs.lj_state(wl, jitter=0.06)
    out = [("lj_small", pos, L, (1, 1, 1))]
    for L, per, n in [((14.0, 14.0, 14.0), (1, 0, 1), 2000), ((6.2, 6.2, 6.2), (1, 1, 1), 180),
                      ((8.7, 8.7, 8.7), (1, 1, 1), 560)]:
        m = int(np.ceil(n ** (1 / 3)))
        g = (np.stack(np.meshgrid(*[np.arange(m)] * 3, indexing="ij"), -1).reshape(-1, 3)[:n] + 0.5) / m
        x = inputs.random_box(n, np.array(L), seed=n)
        x = g * np.array(L) + (x / np.array(L) - 0.5) * 0.3
        x = np.clip(x, 1e-3, np.array(L) - 1e-3)
        out.append((f"box{n}", inputs.as4(x), np.array(L), per))
    return out


@pytest.mark.parametrize("case", range(4))
def test_half_list_holds_each_pair_once(cuda, case):
    name, pos, L, per = boxes()[case]
    s = LJSystem(pos, np.zeros_like(pos), L, periodic=per, half=True, cap=None if case == 0 else 256)
    s.check_status()
    got = half_pairs(s)
    assert len(got) == len(set(got)), "a pair is listed twice"
    want = oracle_pairs(s.pos.cpu().numpy(), s.L, s.periodic, s.r_list)
    assert set(got) == want


@pytest.mark.parametrize("case", range(4))
def test_half_forces_match_oracle(cuda, case):
    name, pos, L, per = boxes()[case]
    s = LJSystem(pos, np.zeros_like(pos), L, periodic=per, half=True, cap=None if case == 0 else 256)
    err = check_forces(s)
    print(f"half-list forces ({name}): max error / RMS {err:.2e}")


def test_half_forces_1m(cuda):
    """The 1,000,188-atom liquid after 20 steps of the half-list path (a
    rebuild on the way): forces, U, W and the pair count against the oracle."""
    wl = inputs.WORKLOADS["lj_1m"]
    pos, vel, L = inputs.lj_state(wl)
    s = LJSystem(pos, vel, L, eps=wl.eps, sigma=wl.sigma, rc=wl.rc, skin=wl.skin, dt=wl.dt, half=True)
    s.step(20)
    s.compute_forces()
    err = check_forces(s)
    print(f"half-list forces (1M, after 20 steps): max error / RMS {err:.2e}")


def test_half_deterministic_and_kick(cuda):
    """Two sweeps give the same bits; the finishing pass's half-kick equals
    fpm_vv_step(half = 1) after the plain sweep."""
    wl = inputs.WORKLOADS["lj_small"]
    pos, vel, L = inputs.lj_state(wl, jitter=0.06)
    s = LJSystem(pos, vel, L, half=True)
    s.compute_forces()
    f1, e1 = s.force.clone(), s.energy.clone()
    s.compute_forces()
    torch.cuda.synchronize()
    assert torch.equal(f1, s.force) and torch.equal(e1, s.energy)
    v0 = s.vel.clone()
    fpm.fpm_vv_step(s.box, s.n, s.prec, 1, s.dt, None, s.vel, s.force)
    v_split = s.vel.clone()
    s.vel.copy_(v0)
    s.forces_and_kick()
    torch.cuda.synchronize()
    assert torch.equal(s.vel, v_split) and torch.equal(s.force, f1)


def test_half_nve_graph_equals_eager(cuda):
    """Steps of the half-list path replayed from a CUDA graph equal eager steps
    bit for bit, and the NVE energy drifts by less than 1e-4 over 100 steps of
    the 4000-atom liquid (the shifted energy, as for the full-list path)."""
    wl = inputs.WORKLOADS["lj_small"]
    pos, vel, L = inputs.lj_state(wl)
    a = LJSystem(pos, vel, L, half=True)
    b = LJSystem(pos, vel, L, half=True)
    a.step(12)
    g = b.capture(steps_per_graph=4)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(a.pos, b.pos) and torch.equal(a.vel, b.vel)
    vrc = 4.0 * (2.5 ** -12 - 2.5 ** -6)

    def energy(s):
        o = s.observables()
        return o["KE"] + o["U"] - o["pairs"] * vrc

    e0 = energy(a)
    a.step(100)
    a.check_status()
    assert abs(energy(a) - e0) <= 1e-4 * abs(e0)
