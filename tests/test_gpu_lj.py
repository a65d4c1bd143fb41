"""GPU parity of the LJ pair sweep, velocity Verlet and the FP64 reductions
against the oracle, on identical positions.

Tolerances (the FP32 bounds are this project's stated accuracy targets; the
FP64 ones follow from the arithmetic: a few ulps per pair term summed over
~80 terms):
  forces  max_i |F_i - F_i^ref| / RMS(F^ref)  <= 1e-5 (FP32), 1e-12 (FP64)
  U, W    relative                           <= 1e-6 (FP32), 1e-12 (FP64)
  pairs   exact (the cutoff test is taken in the path's precision on both
          sides)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1804_07598_gb300 import fpm, inputs
from paper_1804_07598_gb300.md import LJSystem

pytestmark = pytest.mark.gpu

TOL_F = {"f32": 1e-5, "f64": 1e-12}
TOL_E = {"f32": 1e-6, "f64": 1e-12}


def box_of(L, prec):
    """The box the path simulates: an FP32 run holds its box lengths in FP32,
    so the oracle takes L rounded to single precision (then held in FP64)."""
    L = np.asarray(L, np.float64)
    return L.astype(np.float32).astype(np.float64) if prec == "f32" else L


def force_error(f, fref):
    rms = np.sqrt(np.mean(np.sum(fref[:, :3] ** 2, axis=1)))
    return np.max(np.linalg.norm(f[:, :3] - fref[:, :3], axis=1)) / rms


def make(name, prec, jitter=0.06, **kw):
    wl = inputs.WORKLOADS[name]
    pos, vel, L = inputs.lj_state(wl, jitter=jitter)
    return wl, LJSystem(pos, vel, L, eps=wl.eps, sigma=wl.sigma, rc=wl.rc, skin=wl.skin, dt=wl.dt, precision=prec,
                        **kw)


def check_forces(sys_, prec):
    torch.cuda.synchronize()
    pos = sys_.pos.cpu().numpy().astype(np.float64)
    f = sys_.force.cpu().numpy().astype(np.float64)
    fref, U, W, pairs = oracle.lj_forces(pos, box_of(sys_.L, prec), sys_.periodic, sys_.eps, sys_.sigma, sys_.rc,
                                         mask_f32=(prec == "f32"))
    e = sys_.energy.cpu().numpy()
    err = force_error(f, fref)
    assert err <= TOL_F[prec], err
    assert abs(e[0] - U) <= TOL_E[prec] * abs(U), (e[0], U)
    assert abs(e[1] - W) <= TOL_E[prec] * abs(W), (e[1], W)
    assert int(round(e[2])) == pairs
    # per-particle energy share
    assert np.max(np.abs(f[:, 3] - fref[:, 3])) <= 10 * TOL_E[prec] * np.max(np.abs(fref[:, 3])) + 1e-6 * (prec == "f32")
    return err


@pytest.mark.parametrize("name,prec", [("lj_small", "f64"), ("lj_small", "f32"), ("lj_1m", "f32"),
                                       ("lj_1m", "f64"), ("lj_adjoint", "f32")])
def test_lj_forces_match_oracle(cuda, name, prec):
    wl, s = make(name, prec)
    s.check_status()
    check_forces(s, prec)


def test_lj_forces_deterministic(cuda):
    wl, s = make("lj_small", "f32")
    f1, e1 = s.force.clone(), s.energy.clone()
    s.compute_forces()
    assert torch.equal(f1, s.force) and torch.equal(e1, s.energy)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_lj_open_and_mixed_boxes(cuda, prec):
    """A box with one wall (non-periodic y) and a small box with one cell per
    dimension: forces still equal the oracle's."""
    for L, per, n in [((14.0, 14.0, 14.0), (1, 0, 1), 2000), ((6.2, 6.2, 6.2), (1, 1, 1), 180)]:
        x = inputs.random_box(n, np.array(L), seed=n)
        # push apart overlapping particles a little by using a coarse lattice + jitter
        m = int(np.ceil(n ** (1 / 3)))
        grid = (np.stack(np.meshgrid(*[np.arange(m)] * 3, indexing="ij"), -1).reshape(-1, 3)[:n] + 0.5) / m
        x = grid * np.array(L) + (x / np.array(L) - 0.5) * 0.3
        x = np.clip(x, 1e-3, np.array(L) - 1e-3)
        s = LJSystem(inputs.as4(x), np.zeros((n, 4)), L, periodic=per, precision=prec, cap=256)
        s.check_status()
        check_forces(s, prec)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_vv_step_matches_oracle(cuda, prec):
    wl, s = make("lj_small", prec)
    pos0 = s.pos.cpu().numpy().astype(np.float64)
    vel0 = s.vel.cpu().numpy().astype(np.float64)
    f0 = s.force.cpu().numpy().astype(np.float64)
    fpm.fpm_vv_step(s.box, s.n, s.prec, 0, s.dt, s.pos, s.vel, s.force)
    p1, v1 = oracle.vv_kick_drift(pos0, vel0, f0, s.dt, s.L, s.periodic)
    tol = 1e-6 if prec == "f32" else 1e-14
    d = s.pos.cpu().numpy()[:, :3] - p1[:, :3]
    d -= s.L * np.round(d / s.L)
    assert np.max(np.abs(d)) <= tol * np.max(s.L)
    assert np.max(np.abs(s.vel.cpu().numpy()[:, :3] - v1[:, :3])) <= tol * np.max(np.abs(v1[:, :3]))
    fpm.fpm_vv_step(s.box, s.n, s.prec, 1, s.dt, None, s.vel, s.force)
    v2 = oracle.vv_kick(v1, f0, s.dt)
    assert np.max(np.abs(s.vel.cpu().numpy()[:, :3] - v2[:, :3])) <= tol * np.max(np.abs(v2[:, :3]))


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_kinetic_reduction(cuda, prec):
    wl, s = make("lj_small", prec)
    o = s.observables()
    v = s.vel.cpu().numpy().astype(np.float64)[:, :3]
    assert abs(o["KE"] - 0.5 * np.sum(v * v)) <= 1e-12 * o["KE"]
    assert np.max(np.abs(o["P"] - v.sum(0))) <= 1e-9


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_nve_run(cuda, prec):
    """100 NVE steps of the 4000-particle workload: momentum stays ~0, the
    shifted total energy drifts < 1e-4 relative, the Verlet list gets rebuilt,
    and the forces at the final positions still equal the oracle's."""
    wl, s = make("lj_small", prec, jitter=0.0)
    vrc = 4.0 * (wl.rc ** -12 - wl.rc ** -6)
    o0 = s.observables()
    E0 = o0["KE"] + o0["U"] - o0["pairs"] * vrc
    s.step(wl.steps)
    st = s.check_status()
    o1 = s.observables()
    E1 = o1["KE"] + o1["U"] - o1["pairs"] * vrc
    assert abs(E1 - E0) / abs(E0) < 1e-4
    assert np.max(np.abs(o1["P"])) < (1e-9 if prec == "f64" else 1e-3)
    assert st.nrebuild >= 1
    check_forces(s, prec)


def test_graph_replay_equals_eager(cuda):
    """Steps replayed from a CUDA graph give bit-identical states to the same
    steps issued eagerly (the kernels are deterministic)."""
    wl = inputs.WORKLOADS["lj_small"]
    pos, vel, L = inputs.lj_state(wl)
    a = LJSystem(pos, vel, L, precision="f32")
    b = LJSystem(pos, vel, L, precision="f32")
    a.step(30)
    b.capture(steps_per_graph=10)
    b.run(30)
    torch.cuda.synchronize()
    assert torch.equal(a.pos, b.pos) and torch.equal(a.vel, b.vel) and torch.equal(a.ids, b.ids)
    assert torch.equal(a.energy, b.energy)
    assert a.device_status().nrebuild == b.device_status().nrebuild >= 1


def test_graph_steps_1m_match_oracle(cuda):
    """The benchmark configuration: the 1M-atom FP32 system stepped by CUDA
    graph replays (the rebuild as a conditional graph node) over several
    rebuilds; then the forces and energies at the final positions against
    the oracle, every particle within skin/2 of its reference position, and
    the Verlet list of sampled particles against an O(n) scan of the
    reference positions."""
    wl, s = make("lj_1m", "f32", jitter=0.0)
    s.step(2)
    s.capture(steps_per_graph=1)
    s.run(40)
    torch.cuda.synchronize()
    st = s.check_status()
    assert st.nrebuild >= 3
    check_forces(s, "f32")
    pos = s.pos.cpu().numpy().astype(np.float64)
    ref = s.pos_ref.cpu().numpy()
    d = pos[:, :3] - ref[:, :3].astype(np.float64)
    assert np.max(np.sum(d * d, axis=1)) <= (0.5 * s.skin) ** 2 * (1 + 1e-5)
    nbr, nn = s.neighbor_lists()
    rng = np.random.default_rng(1)
    for i in rng.choice(s.n, 12, replace=False):
        want = np.sort(oracle.neighbors_one(ref, s.L, s.periodic, s.r_list, int(i)).astype(np.int64))
        got = np.sort(nbr[:nn[i], i].astype(np.int64))
        assert np.array_equal(got, want), i


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_pack_unpack_xyz(cuda, prec):
    """fpm_pack_xyz / fpm_unpack_xyz move x, y, z between the packed host
    layout and the 4-vector state exactly, keeping the state's w."""
    dt_ = torch.float32 if prec == "f32" else torch.float64
    fp = fpm.FPM_F32 if prec == "f32" else fpm.FPM_F64
    n = 100003
    g = torch.Generator().manual_seed(3)
    x4 = torch.rand((n, 4), generator=g, dtype=dt_).cuda()
    w = x4[:, 3].clone()
    xyz = torch.empty((n, 3), dtype=dt_, device="cuda")
    fpm.fpm_pack_xyz(n, fp, x4, xyz)
    y4 = torch.full_like(x4, -1.0)
    y4[:, 3] = w
    fpm.fpm_unpack_xyz(n, fp, xyz, y4)
    torch.cuda.synchronize()
    assert torch.equal(xyz, x4[:, :3]) and torch.equal(y4, x4)
    # the packed side in pinned host memory (read and written across the host
    # link by the kernels), and a packed array that starts off a 16-byte
    # boundary (the one-particle-per-thread path); n = 100003 leaves a tail of 3
    hb = torch.zeros(3 * n + 1, dtype=dt_).pin_memory()
    for off in (0, 1):
        h = hb[off:off + 3 * n]
        fpm.fpm_pack_xyz(n, fp, x4, h)
        torch.cuda.synchronize()
        assert torch.equal(h.view(n, 3), x4[:, :3].cpu())
        z4 = torch.full_like(x4, -1.0)
        z4[:, 3] = w
        fpm.fpm_unpack_xyz(n, fp, h, z4)
        torch.cuda.synchronize()
        assert torch.equal(z4, x4)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_forces_kick_equals_forces_then_kick(cuda, prec):
    """fpm_lj_forces_kick writes the same forces and energies as
    fpm_lj_forces and the same velocities as fpm_vv_step(half = 1) after it,
    bit for bit."""
    wl, s = make("lj_small", prec)
    v0 = s.vel.clone()
    s.compute_forces()
    fpm.fpm_vv_step(s.box, s.n, s.prec, 1, s.dt, None, s.vel, s.force)
    torch.cuda.synchronize()
    f_ref, e_ref, v_ref = s.force.clone(), s.energy.clone(), s.vel.clone()
    s.vel.copy_(v0)
    s.force.zero_()
    s.energy.zero_()
    s.forces_and_kick()
    torch.cuda.synchronize()
    assert torch.equal(s.force, f_ref)
    assert torch.equal(s.energy, e_ref)
    assert torch.equal(s.vel, v_ref)
    assert not torch.equal(v_ref, v0)


def test_sweep_wait_expiry_latches_timeout(cuda):
    """The bounded wait of the force sweep driven to expiry through the test
    hook (a 1-cycle budget for the first wait of each work item on its tile's
    copies): the call completes, FPM_FLAG_TIMEOUT is latched
    (FPM_ERR_TIMEOUT from the device status), and with the default budget
    restored the next sweep is clean and gives the earlier forces bit for
    bit."""
    wl = inputs.WORKLOADS["lj_small"]
    pos, vel, L = inputs.lj_state(wl, jitter=0.06)
    s = LJSystem(pos, vel, L, precision="f32")
    s.compute_forces()
    torch.cuda.synchronize()
    s.check_status()
    f0 = s.force.clone()
    latched = False
    try:
        for _ in range(5):
            s.status.zero_()
            fpm.fpm_test_wait_budget(1)
            s.compute_forces()
            torch.cuda.synchronize()
            if fpm.fpm_status_from_device(fpm.read_status(s.status)) == fpm.FPM_ERR_TIMEOUT:
                latched = True
                break
    finally:
        fpm.fpm_test_wait_budget(0)
    assert latched
    s.status.zero_()
    s.compute_forces()
    torch.cuda.synchronize()
    s.check_status()
    assert torch.equal(s.force, f0)
