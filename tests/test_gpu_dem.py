"""GPU parity of the DEM path (Sec. 4.5, Eqs. 9-13) against the oracle:
contact forces, torques and tangential histories at identical states (with
and without stored histories), the histories carried through Verlet
rebuilds, multi-step runs with rebuilds and walls, conservation of momentum
and angular momentum, graph replays against eager steps, and single
contacts against the closed forms of Eqs. 10-12."""
import numpy as np
import pytest
import torch

import oracle
from paper_1804_07598_gb300 import inputs
from paper_1804_07598_gb300.dem import DEMSystem

pytestmark = pytest.mark.gpu

R = 0.06
SKIN = inputs.DEM_SKIN


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def dense_box(k, seed, spacing=0.116, jitter=0.003, v=0.05, w=0.5):
    """k^3 grains on a jittered cubic lattice (overlaps of ~4e-3 with the
    axis neighbours) in a periodic box, random velocities and spins; FP32
    values."""
    rng = np.random.default_rng(seed)
    g = np.stack(np.meshgrid(*[np.arange(k)] * 3, indexing="ij"), -1).reshape(-1, 3)
    n = len(g)
    pos = np.zeros((n, 4))
    pos[:, :3] = (g + 0.5) * spacing + rng.uniform(-jitter, jitter, size=(n, 3))
    vel = np.zeros((n, 4))
    vel[:, :3] = rng.normal(scale=v, size=(n, 3))
    om = np.zeros((n, 4))
    om[:, :3] = rng.normal(scale=w, size=(n, 3))
    L = np.full(3, k * spacing)
    return f32(pos), f32(vel), f32(om), L


def params(**kw):
    p = dict(inputs.DEM_PARAMS)
    p.update(kw)
    return p


def oracle_p(pd):
    return oracle.dem_params(**pd)


def rms(a):
    return float(np.sqrt((a[:, :3] ** 2).sum(1).mean()))


def dict_to_hist(n, d):
    cnt, ids, u = oracle.dem_empty_history(n)
    for (i, j), val in sorted(d.items()):
        c = cnt[i]
        ids[i, c] = j
        u[i, c] = val
        cnt[i] += 1
    return cnt, ids, u


def delta_of(pos, L, per, i, j):
    d = pos[i, :3] - pos[j, :3]
    for a in range(3):
        if per[a]:
            d[a] -= L[a] * np.round(d[a] / L[a])
    return 2 * R - np.linalg.norm(d)


def compare_hist(gd, od, pos, L, per, tol):
    """Same contacts (up to pairs within 1e-6 of touching, where FP32 and FP64
    may decide differently) and u_t within tol."""
    for key in set(gd) ^ set(od):
        assert abs(delta_of(pos, L, per, *key)) < 1e-6, key
    common = set(gd) & set(od)
    assert len(common) > 0.9 * max(len(od), 1)
    err = max(np.abs(gd[k] - od[k]).max() for k in common)
    assert err <= tol, err


# FP32 bound on forces and torques, as a fraction of their RMS.  The overlap
# delta = 2R - r is a difference of nearly equal numbers: in FP32 it carries an
# absolute error of a few ulps of 2R (~1e-8), and f = sqrt(delta / 2R)
# magnifies that without limit as a contact opens (d ln f / d delta =
# 1 / (2 delta)), while the damping force f gn m_eff v_n stays finite there.
# Contacts within ~1e-5 of touching therefore carry errors of order 1e-5 of
# a typical contact force, above the 1e-5-of-RMS bound of the smooth LJ pair;
# the DEM bound is 1e-4 of RMS.
TOL_F = 1e-4


def test_dem_forces_match_oracle(cuda):
    """One force evaluation at a state with fresh contacts: F and T within
    TOL_F of their RMS, u_t = v_t dt per contact."""
    pos, vel, om, L = dense_box(12, 1)
    pd = params()
    s = DEMSystem(pos, vel, om, L, (1, 1, 1), pd, SKIN)
    s.compute_forces()
    torch.cuda.synchronize()
    s.check_status()
    _, _, _, F, T = s.state_by_id()
    Fo, To, ho, c = oracle.dem_forces(pos, vel, om, L, (1, 1, 1), oracle_p(pd))
    assert c > 3 * len(pos)
    assert np.abs(F[:, :3] - Fo[:, :3]).max() <= TOL_F * rms(Fo)
    assert np.abs(T[:, :3] - To[:, :3]).max() <= TOL_F * rms(To)
    od = oracle.dem_history_dict(ho)
    umax = max(np.abs(u).max() for u in od.values())
    compare_hist(s.history_by_id(), od, pos, L, (1, 1, 1), 1e-5 * umax)
    assert s.contacts() == c or abs(s.contacts() - c) <= 4



def test_dem_forces_full_avalanche(cuda):
    """The avalanche the benchmark times, at full size (166 x 62 x 64 moving
    grains + 28,304 fixed floor and wall grains, the default cells of 3
    r_list, the benchmark's launch shape): one force evaluation with fresh
    contacts, every grain against the oracle, and the same contact count.
    The lattice's closest non-contacts (floor and wall grains) lie ~4e-6
    beyond touching, far above the FP32 resolution of r^2 there, so both
    sides find the same contacts.  A grain's net force is a sum of nearly
    cancelling contact forces (opposite lattice neighbours), so its FP32
    error follows the contact forces, not the net force: each carries the
    rounding of delta = 2R - r (a few ulps of 2R, 5e-5 of the lattice's
    overlap 6e-4, x 1.5 through delta^1.5).  The bound is TOL_F of 8 times
    the largest contact force (elastic at that overlap plus damping at twice
    the largest speed), and likewise for the torques."""
    pos, vel, om, L, per, g = inputs.dem_avalanche(166, 62, 64, gap=-0.005)
    pos, vel, om = f32(pos), f32(vel), f32(om)
    pd = params(g=g)
    s = DEMSystem(pos, vel, om, L, per, pd, SKIN)
    s.compute_forces()
    torch.cuda.synchronize()
    s.check_status()
    _, _, _, F, T = s.state_by_id()
    Fo, To, _, c = oracle.dem_forces(pos, vel, om, L, per, oracle_p(pd))
    assert len(pos) == 686992 and c > 3_900_000
    assert s.contacts() == c
    dmax = -2 * R * (-0.005)  # 2R - s: the lattice's overlap
    f = np.sqrt(dmax / (2 * R))
    vmax = 2 * np.linalg.norm(vel[:, :3], axis=1).max()  # largest relative speed
    m_eff = 0.5 * pd["m"]
    fc = f * (pd["kn"] * dmax + pd["gn"] * m_eff * vmax)
    tc = R * f * (pd["kt"] * vmax * pd["dt"] + pd["gt"] * m_eff * vmax)
    assert np.abs(F[:, :3] - Fo[:, :3]).max() <= TOL_F * 8 * fc
    assert np.abs(T[:, :3] - To[:, :3]).max() <= TOL_F * 8 * tc

def test_dem_forces_with_stored_history(cuda):
    """A state with aged contacts (sliding ones at the Coulomb limit): the GPU
    loads the oracle's u_t, then both evaluate the forces once."""
    pos, vel, om, L = dense_box(10, 2)
    pd = params()
    po = oracle_p(pd)
    x, v, w, _, _, h, c = oracle.dem_run(pos, vel, om, L, (1, 1, 1), po, 25)
    x, v, w = f32(x), f32(v), f32(w)
    hd = {k: f32(u) for k, u in oracle.dem_history_dict(h).items()}
    s = DEMSystem(x, v, w, L, (1, 1, 1), pd, SKIN)
    s.set_history_by_id(hd)
    s.compute_forces()
    torch.cuda.synchronize()
    s.check_status()
    _, _, _, F, T = s.state_by_id()
    Fo, To, ho, c = oracle.dem_forces(x, v, w, L, (1, 1, 1), po, hist=dict_to_hist(len(x), hd))
    assert np.abs(F[:, :3] - Fo[:, :3]).max() <= TOL_F * rms(Fo)
    assert np.abs(T[:, :3] - To[:, :3]).max() <= TOL_F * rms(To)
    od = oracle.dem_history_dict(ho)
    umax = max(np.abs(u).max() for u in od.values())
    compare_hist(s.history_by_id(), od, x, L, (1, 1, 1), 1e-5 * umax)


def test_dem_history_and_spin_survive_rebuild(cuda):
    """A rebuild reorders the grains; every contact's u_t and every grain's
    omega stay with their ids, bit for bit."""
    pos, vel, om, L = dense_box(10, 3, v=0.2)
    s = DEMSystem(pos, vel, om, L, (1, 1, 1), params(), SKIN, cell_factor=1.0)  # 8^3 cells: grains change cells
    s.step(6)
    s.compute_forces()
    torch.cuda.synchronize()
    before = s.history_by_id()
    om0 = s.state_by_id()[2]
    ids0 = s.ids.cpu().numpy().copy()
    s.rebuild()
    torch.cuda.synchronize()
    s.check_status()
    assert not np.array_equal(s.ids.cpu().numpy(), ids0)  # the order did change
    after = s.history_by_id()
    assert set(after) == set(before) and len(before) > 100
    assert all(np.array_equal(after[k], before[k]) for k in before)
    np.testing.assert_array_equal(s.state_by_id()[2], om0)


def run_pair(pos, vel, om, L, per, pd, steps, seed=9, cell_factor=3.0):
    """GPU run and oracle run of `steps` steps, plus the oracle from inputs
    one FP32 ulp away: the spread of the two oracle runs is the dynamics'
    own sensitivity, the scale the GPU's FP32 error is held to."""
    s = DEMSystem(pos, vel, om, L, per, pd, SKIN, cell_factor=cell_factor)
    s.step(steps)
    torch.cuda.synchronize()
    st = s.check_status()
    po = oracle_p(pd)
    A = oracle.dem_run(pos, vel, om, L, per, po, steps)
    rng = np.random.default_rng(seed)
    moving = pos[:, 3] == 0
    pert = pos.copy()
    pert[moving, :3] *= 1.0 + rng.choice([-1.0, 1.0], size=(moving.sum(), 3)) * 2.0 ** -24
    B = oracle.dem_run(pert, vel, om, L, per, po, steps)
    return s, st, A, B


@pytest.mark.parametrize("case", ["periodic", "avalanche"])
def test_dem_run_matches_oracle(cuda, case):
    """Steps with Verlet rebuilds (the history crossing each reorder): final
    positions, velocities and spins within 20x the oracle's own one-ulp
    spread (plus a floor of a few FP32 ulps)."""
    if case == "periodic":  # cells of r_list: wrapped tiles, grains crossing cells
        pos, vel, om, L = dense_box(10, 4, v=0.1)
        per, pd, steps, cf = (1, 1, 1), params(), 40, 1.0
    else:  # the default cells; y (periodic, 2 cells wide) in all-pairs mode
        pos, vel, om, L, per, g = inputs.dem_avalanche(12, 8, 8, vel_scale=0.02)
        pos, vel, om = f32(pos), f32(vel), f32(om)
        per, pd, steps, cf = per, params(g=g), 60, 3.0
    s, st, A, B = run_pair(pos, vel, om, L, per, pd, steps, cell_factor=cf)
    assert st.nrebuild >= 2
    x, v, w, F, T = s.state_by_id()

    def diff(a, b, is_pos):
        d = a[:, :3].astype(np.float64) - b[:, :3]
        if is_pos:  # the GPU's rebuilds wrap positions into the box
            for ax in range(3):
                if per[ax]:
                    d[:, ax] -= L[ax] * np.round(d[:, ax] / L[ax])
        return np.abs(d).max()

    for k, (g_, a_, b_) in enumerate([(x, A[0], B[0]), (v, A[1], B[1]), (w, A[2], B[2])]):
        spread = diff(a_, b_, k == 0)
        floor = 4 * 2.0 ** -24 * max(np.abs(a_[:, :3]).max(), 1e-30)
        err = diff(g_, a_, k == 0)
        assert err <= 20 * spread + floor, (k, err, spread)
    if case == "avalanche":
        fixed = pos[:, 3] != 0
        np.testing.assert_array_equal(x[fixed], pos[fixed].astype(np.float32))


def test_dem_conserves_momentum_and_angular_momentum(cuda):
    """An isolated cluster (open box, no gravity): total P and L stay within
    FP32 rounding of their start over 100 steps with rebuilds."""
    k, sp = 8, 0.115
    rng = np.random.default_rng(6)
    g = np.stack(np.meshgrid(*[np.arange(k)] * 3, indexing="ij"), -1).reshape(-1, 3)
    n = len(g)
    pos = np.zeros((n, 4))
    pos[:, :3] = 1.0 + g * sp + rng.uniform(-0.003, 0.003, size=(n, 3))
    vel = np.zeros((n, 4))
    vel[:, :3] = rng.normal(scale=0.05, size=(n, 3))
    om = np.zeros((n, 4))
    om[:, :3] = rng.normal(scale=0.5, size=(n, 3))
    pos, vel, om = f32(pos), f32(vel), f32(om)
    pd = params(gt=1.0)
    s = DEMSystem(pos, vel, om, (4.0, 4.0, 4.0), (0, 0, 0), pd, SKIN)

    def momenta():
        x, v, w, _, _ = s.state_by_id()
        x, v, w = x.astype(np.float64), v.astype(np.float64), w.astype(np.float64)
        P = pd["m"] * v[:, :3].sum(0)
        Lm = pd["m"] * np.cross(x[:, :3], v[:, :3]).sum(0) + pd["I"] * w[:, :3].sum(0)
        return P, Lm

    P0, L0 = momenta()
    s.step(100)
    torch.cuda.synchronize()
    assert s.check_status().nrebuild >= 1
    P1, L1 = momenta()
    scale_p = pd["m"] * np.abs(vel[:, :3]).sum()
    scale_l = pd["m"] * np.abs(np.cross(pos[:, :3], vel[:, :3])).sum() + pd["I"] * np.abs(om[:, :3]).sum()
    assert np.abs(P1 - P0).max() <= 1e-5 * scale_p
    assert np.abs(L1 - L0).max() <= 1e-5 * scale_l


def test_dem_graph_replay_equals_eager(cuda):
    """Steps replayed from a CUDA graph (rebuild in a conditional node) give
    the same state, bit for bit, as the same steps launched eagerly."""
    pos, vel, om, L = dense_box(10, 5, v=0.15)
    a = DEMSystem(pos, vel, om, L, (1, 1, 1), params(), SKIN)
    b = DEMSystem(pos, vel, om, L, (1, 1, 1), params(), SKIN)
    a.step(20)
    g = b.capture(1)
    for _ in range(20):
        g.replay()
    torch.cuda.synchronize()
    assert a.check_status().nrebuild == b.check_status().nrebuild >= 2
    for x, y in zip(a.state_by_id(), b.state_by_id()):
        np.testing.assert_array_equal(x, y)
    assert a.history_by_id().keys() == b.history_by_id().keys()


def contact_pair(n, delta, c=(1.0, 1.0, 1.0)):
    """Grains 0 and 1 whose centres are 2R - delta apart along n (0 at
    c + r n / 2), positions rounded to FP32."""
    r = 2 * R - delta
    x = np.zeros((2, 4))
    x[0, :3] = np.asarray(c) + 0.5 * r * n
    x[1, :3] = np.asarray(c) - 0.5 * r * n
    return f32(x)


@pytest.mark.parametrize("seed,delta", [(1, 1e-3), (2, 5e-3), (3, 2e-2)])
def test_dem_static_contact_closed_form(cuda, seed, delta):
    """One contact at rest, on the GPU: Eq. 11 alone, F_0 = sqrt(delta / 2R)
    kn delta n = -F_1 with delta taken from the stored positions; no torque,
    no tangential history, two ordered contacts."""
    n = np.random.default_rng(seed).normal(size=3)
    n /= np.linalg.norm(n)
    x = contact_pair(n, delta)
    pd = params()
    ds = DEMSystem(x, np.zeros((2, 3)), np.zeros((2, 3)), (3.0, 3.0, 3.0), (1, 1, 1), pd, SKIN)
    ds.compute_forces()
    torch.cuda.synchronize()
    _, _, _, F, T = ds.state_by_id()
    d = x[0, :3] - x[1, :3]
    r = np.linalg.norm(d)
    dl = 2 * R - r
    ref = np.sqrt(dl / (2 * R)) * pd["kn"] * dl * d / r
    scale = np.linalg.norm(ref)
    # delta = 2R - r carries a few ulps of 2R (TOL_F above): 1e-5 of delta at
    # delta = 1e-3, 1.5e-5 of the force
    assert np.max(np.abs(F[0, :3] - ref)) <= TOL_F * scale
    assert np.max(np.abs(F[1, :3] + ref)) <= TOL_F * scale
    assert np.all(np.abs(T[:, :3]) <= 1e-6 * scale * R)
    assert ds.contacts() == 2
    assert all(np.all(v == 0) for v in ds.history_by_id().values())


def test_dem_sliding_contact_first_step_closed_form(cuda):
    """A new contact sliding at v_t with no spin, on the GPU: Eq. 10 stores
    u = v_t dt (and -u for the mirror entry), Eq. 12 gives F_t = f (-kt u -
    gt m_eff v_t), the torque on each grain is -1/2 r_pq x F_t, and the two
    grains get opposite forces."""
    rng = np.random.default_rng(7)
    n = np.array([1.0, 0.2, -0.3])
    n /= np.linalg.norm(n)
    t = rng.normal(size=3)
    t -= t.dot(n) * n
    t /= np.linalg.norm(t)
    delta = 3e-3
    x = contact_pair(n, delta)
    v = f32(np.stack([0.4 * t, -0.1 * t]))
    pd = params(gt=1.7, mu=1e3)  # no Coulomb limit here
    ds = DEMSystem(x, v, np.zeros((2, 3)), (3.0, 3.0, 3.0), (1, 1, 1), pd, SKIN)
    ds.compute_forces()
    torch.cuda.synchronize()
    _, _, _, F, T = ds.state_by_id()
    d = x[0, :3] - x[1, :3]
    r = np.linalg.norm(d)
    nn_ = d / r
    dl = 2 * R - r
    f = np.sqrt(dl / (2 * R))
    vpq = v[0] - v[1]
    vt = vpq - vpq.dot(nn_) * nn_
    u = vt * pd["dt"]
    m_eff = 0.5 * pd["m"]
    Fn = f * (pd["kn"] * dl * nn_ - pd["gn"] * m_eff * vpq.dot(nn_) * nn_)
    Ft = f * (-pd["kt"] * u - pd["gt"] * m_eff * vt)
    scale = np.linalg.norm(Fn + Ft)
    assert np.max(np.abs(F[0, :3] - (Fn + Ft))) <= TOL_F * scale
    assert np.max(np.abs(F[1, :3] + (Fn + Ft))) <= TOL_F * scale
    Tref = -0.5 * np.cross(d, Ft)
    tscale = max(np.linalg.norm(Tref), 1e-30)
    assert np.max(np.abs(T[0, :3] - Tref)) <= 1e-4 * tscale
    assert np.max(np.abs(T[1, :3] - Tref)) <= 1e-4 * tscale
    hd = ds.history_by_id()
    np.testing.assert_allclose(hd[(0, 1)], u, rtol=1e-5, atol=1e-5 * np.linalg.norm(u))
    np.testing.assert_allclose(hd[(1, 0)], -u, rtol=1e-5, atol=1e-5 * np.linalg.norm(u))
