"""Pins of the DEM oracle (Sec. 4.5, Eqs. 9-13) against facts that do not come
from the oracle itself: closed forms of a single contact, a contact that rolls
without slipping, Coulomb's limit, conservation of linear and angular
momentum, a brute-force contact count, and the Hertz collision's restitution
and maximum overlap."""
import numpy as np
import pytest

import oracle

R = 0.06


def unit(v):
    v = np.asarray(v, float)
    return v / np.linalg.norm(v)


def perp(n, seed):
    a = np.random.default_rng(seed).normal(size=3)
    a -= a.dot(n) * n
    return unit(a)


def pair(n, delta, c=(1.0, 1.0, 1.0)):
    """Two particles whose centres are 2R - delta apart along n (p = 0 at
    c + r n / 2, q = 1 at c - r n / 2)."""
    r = 2 * R - delta
    x = np.zeros((2, 4))
    x[0, :3] = np.asarray(c) + 0.5 * r * n
    x[1, :3] = np.asarray(c) - 0.5 * r * n
    return x


P_BOX = ((3.0, 3.0, 3.0), (1, 1, 1))


def test_static_overlap_closed_form():
    """Eq. 11 with no motion: F_p = sqrt(delta/2R) kn delta n, F_q = -F_p."""
    p = oracle.dem_params()
    for seed, delta in [(1, 1e-3), (2, 5e-3), (3, 2e-2)]:
        n = unit(np.random.default_rng(seed).normal(size=3))
        x = pair(n, delta)
        F, T, h, c = oracle.dem_forces(x, np.zeros((2, 4)), np.zeros((2, 4)), *P_BOX, p)
        ref = np.sqrt(delta / (2 * R)) * p.kn * delta * n
        assert c == 2
        np.testing.assert_allclose(F[0, :3], ref, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(F[1, :3], -ref, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(T[:, :3], 0.0, atol=1e-18)
        assert np.all(h[2][:, 0] == 0.0)


def test_no_force_without_overlap():
    p = oracle.dem_params()
    n = unit([1.0, 2.0, 0.5])
    x = pair(n, -1e-6)  # 2R + 1e-6 apart
    F, T, h, c = oracle.dem_forces(x, np.zeros((2, 4)), np.zeros((2, 4)), *P_BOX, p)
    assert c == 0 and np.all(F == 0) and np.all(T == 0) and np.all(h[0] == 0)


def test_normal_damping_closed_form():
    """Eq. 11 with approach speed: F_p = f (kn delta n - gn m_eff (v_pq . n) n)."""
    p = oracle.dem_params()
    n, delta, s = unit([0.3, -0.4, 0.8]), 4e-3, -0.7  # v_pq . n = s < 0: approaching
    x = pair(n, delta)
    v = np.zeros((2, 4))
    v[0, :3] = 0.5 * s * n
    v[1, :3] = -0.5 * s * n
    F, T, h, c = oracle.dem_forces(x, v, np.zeros((2, 4)), *P_BOX, p)
    f = np.sqrt(delta / (2 * R))
    ref = f * (p.kn * delta * n - p.gn * 0.5 * p.m * s * n)
    np.testing.assert_allclose(F[0, :3], ref, rtol=1e-12)
    np.testing.assert_allclose(T[0, :3], 0.0, atol=1e-15)


def test_tangential_first_step_closed_form():
    """A new contact sliding at v_t (no spin): Eq. 10 gives u = v_t dt, Eq. 12
    F_t = f (-kt u - gt m_eff v_t), and the torque -1/2 r_pq x F_t."""
    p = oracle.dem_params(gt=1.7, mu=1e3)  # no Coulomb limit here
    n, delta = unit([1.0, 0.2, -0.3]), 3e-3
    t = perp(n, 7)
    x = pair(n, delta)
    v = np.zeros((2, 4))
    v[0, :3] = 0.4 * t
    v[1, :3] = -0.1 * t  # v_pq = 0.5 t, purely tangential
    F, T, h, c = oracle.dem_forces(x, v, np.zeros((2, 4)), *P_BOX, p)
    f = np.sqrt(delta / (2 * R))
    vt = 0.5 * t
    u = vt * p.dt
    Ft = f * (-p.kt * u - p.gt * 0.5 * p.m * vt)
    Fn = f * p.kn * delta * n
    np.testing.assert_allclose(F[0, :3], Fn + Ft, rtol=1e-12, atol=1e-16)
    r_pq = x[0, :3] - x[1, :3]
    np.testing.assert_allclose(T[0, :3], -0.5 * np.cross(r_pq, Ft), rtol=1e-12, atol=1e-18)
    # q sees the mirror contact: the same torque, the opposite force
    np.testing.assert_allclose(T[1, :3], T[0, :3], rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(F[1, :3], -F[0, :3], rtol=1e-12, atol=1e-16)
    hd = oracle.dem_history_dict(h)
    np.testing.assert_allclose(hd[(0, 1)], u, rtol=1e-12)
    np.testing.assert_allclose(hd[(1, 0)], -u, rtol=1e-12)


def test_rolling_without_slip_has_no_tangential_force():
    """Spins that make the surface points move together, v_p - v_q = R (w_p +
    w_q) x n, give v_t = 0: no tangential force and no history.  (The opposite
    sign of the rotational term would double v_t instead.)"""
    p = oracle.dem_params(gt=2.0)
    n, delta = unit([0.2, 0.9, 0.1]), 2e-3
    w = 3.0 * perp(n, 11)
    x = pair(n, delta)
    vpq = R * np.cross(2 * w, n)
    v = np.zeros((2, 4))
    v[0, :3] = 0.5 * vpq
    v[1, :3] = -0.5 * vpq
    om = np.zeros((2, 4))
    om[0, :3] = w
    om[1, :3] = w
    F, T, h, c = oracle.dem_forces(x, v, om, *P_BOX, p)
    f = np.sqrt(delta / (2 * R))
    np.testing.assert_allclose(F[0, :3], f * p.kn * delta * n, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(T[:, :3], 0.0, atol=1e-15)
    np.testing.assert_allclose(h[2][0, 0], 0.0, atol=1e-16)


def test_coulomb_limit():
    """A large stored u_t: |F_t| is cut to mu |F_n| along -u_t, and the new u_t
    gives that F_t through Eq. 12."""
    p = oracle.dem_params(mu=0.5)
    n, delta = unit([0.0, 0.0, 1.0]), 4e-3
    t = unit([1.0, 1.0, 0.0])
    x = pair(n, delta)
    hist = oracle.dem_empty_history(2)
    hist[0][:] = 1
    hist[1][0, 0], hist[1][1, 0] = 1, 0
    hist[2][0, 0] = 0.05 * t
    hist[2][1, 0] = -0.05 * t
    F, T, h, c = oracle.dem_forces(x, np.zeros((2, 4)), np.zeros((2, 4)), *P_BOX, p, hist=hist)
    f = np.sqrt(delta / (2 * R))
    Fn = f * p.kn * delta * n
    Ft = F[0, :3] - Fn
    assert np.isclose(np.linalg.norm(Ft), p.mu * np.linalg.norm(Fn), rtol=1e-12)
    np.testing.assert_allclose(unit(Ft), -t, atol=1e-12)
    u_new = oracle.dem_history_dict(h)[(0, 1)]
    np.testing.assert_allclose(f * (-p.kt * u_new), Ft, rtol=1e-12, atol=1e-15)
    assert np.linalg.norm(u_new) < 0.05


def test_history_accumulates_then_resets():
    """Sustained sliding: u_t grows by v_t dt per step (below the Coulomb
    limit); after the contact opens it is forgotten and restarts at v_t dt."""
    p = oracle.dem_params(mu=100.0)
    n, delta = unit([1.0, 0.0, 0.0]), 2e-3
    t = unit([0.0, 1.0, 0.0])
    x = pair(n, delta)
    v = np.zeros((2, 4))
    v[0, :3] = 0.2 * t
    h = None
    for k in range(1, 6):
        F, T, h, c = oracle.dem_forces(x, v, np.zeros((2, 4)), *P_BOX, p, hist=h)
        np.testing.assert_allclose(oracle.dem_history_dict(h)[(0, 1)], k * 0.2 * p.dt * t, rtol=1e-12)
    F, T, h, c = oracle.dem_forces(pair(n, -1e-4), v, np.zeros((2, 4)), *P_BOX, p, hist=h)
    assert c == 0 and np.all(h[0] == 0)
    F, T, h, c = oracle.dem_forces(x, v, np.zeros((2, 4)), *P_BOX, p, hist=h)
    np.testing.assert_allclose(oracle.dem_history_dict(h)[(0, 1)], 0.2 * p.dt * t, rtol=1e-12)


def cluster(n, seed, spacing=0.115):
    """A compact cubic cluster with small overlaps and random v, w."""
    k = int(np.ceil(n ** (1 / 3)))
    g = np.stack(np.meshgrid(*[np.arange(k)] * 3, indexing="ij"), -1).reshape(-1, 3)[:n]
    rng = np.random.default_rng(seed)
    x = np.zeros((n, 4))
    x[:, :3] = 1.0 + g * spacing + rng.uniform(-0.004, 0.004, size=(n, 3))
    v = np.zeros((n, 4))
    v[:, :3] = rng.normal(scale=0.05, size=(n, 3))
    w = np.zeros((n, 4))
    w[:, :3] = rng.normal(scale=0.5, size=(n, 3))
    return x, v, w


def momenta(x, v, w, p):
    P = p.m * v[:, :3].sum(0)
    L = p.m * np.cross(x[:, :3], v[:, :3]).sum(0) + p.I * w[:, :3].sum(0)
    return P, L


def test_conservation_of_linear_and_angular_momentum():
    """An isolated cluster (open box, no gravity, damping on): every contact
    force acts equally and oppositely, and the torques -1/2 r_pq x F_t cancel
    the orbital moment of F_t, so the leapfrog of Eq. 13 keeps the total
    linear and angular momentum up to rounding."""
    p = oracle.dem_params(gt=1.0, dt=0.01)
    x, v, w = cluster(125, 3)
    P0, L0 = momenta(x, v, w, p)
    x1, v1, w1, F, T, h, c = oracle.dem_run(x, v, w, (5.0, 5.0, 5.0), (0, 0, 0), p, 150)
    assert c > 100  # the cluster stays in contact
    P1, L1 = momenta(x1, v1, w1, p)
    scale_p = p.m * np.abs(v[:, :3]).sum()
    scale_l = p.m * np.abs(np.cross(x[:, :3], v[:, :3])).sum() + p.I * np.abs(w[:, :3]).sum()
    assert np.all(np.abs(P1 - P0) < 1e-12 * scale_p)
    assert np.all(np.abs(L1 - L0) < 1e-11 * scale_l)
    # a torque of -R n x F_t instead (contact-point lever arm) would not conserve L
    assert np.abs(w1 - w).max() > 1e-3


def test_contact_count_brute_force():
    """The cell-list contact search finds exactly the pairs with minimum-image
    distance below 2R (brute force over all pairs)."""
    rng = np.random.default_rng(5)
    L = np.array([1.3, 1.1, 1.2])
    n = 900
    x = np.zeros((n, 4))
    x[:, :3] = rng.uniform(0, 1, size=(n, 3)) * L
    p = oracle.dem_params()
    F, T, h, c = oracle.dem_forces(x, np.zeros((n, 4)), np.zeros((n, 4)), L, (1, 1, 1), p)
    d = x[:, None, :3] - x[None, :, :3]
    d -= L * np.round(d / L)
    r2 = (d ** 2).sum(-1)
    np.fill_diagonal(r2, np.inf)
    assert c == int((r2 < (2 * R) ** 2).sum())
    assert np.array_equal(h[0], (r2 < (2 * R) ** 2).sum(1))


def test_elastic_head_on_collision():
    """gn = gt = 0: the Hertz contact conserves energy, so the particles leave
    with their approach speed, and the deepest overlap solves
    1/2 m_eff v0^2 = (2/5) kn delta^(5/2) / sqrt(2R)."""
    p = oracle.dem_params(gn=0.0, gt=0.0, dt=2e-4)
    v0 = 0.05
    x = np.zeros((2, 4))
    x[0, :3] = [1.0 - R - 0.002, 1.0, 1.0]
    x[1, :3] = [1.0 + R + 0.002, 1.0, 1.0]
    v = np.zeros((2, 4))
    v[0, 0], v[1, 0] = 0.5 * v0, -0.5 * v0
    om = np.zeros((2, 4))
    dmax, h = 0.0, None
    for _ in range(20000):
        F, T, h, c = oracle.dem_forces(x, v, om, *P_BOX, p, hist=h)
        x, v, om = oracle.dem_leapfrog(x, v, om, F, T, p)
        dmax = max(dmax, 2 * R - abs(x[1, 0] - x[0, 0]))
        if c == 0 and v[1, 0] - v[0, 0] > 0:
            break
    assert v[1, 0] - v[0, 0] == pytest.approx(v0, rel=1e-3)
    meff = 0.5 * p.m
    ref = (5.0 * meff * v0 ** 2 * np.sqrt(2 * R) / (4.0 * p.kn)) ** 0.4
    assert dmax == pytest.approx(ref, rel=2e-3)


def test_leapfrog_gravity_and_fixed_particles():
    """Eq. 13 without contacts: v1 = v0 + dt g, r1 = r0 + dt v1, w unchanged;
    a particle with w != 0 does not move."""
    p = oracle.dem_params(dt=0.02, g=(0.5, 0.0, -0.866))
    x = np.array([[1.0, 1.0, 1.0, 0.0], [2.0, 2.0, 2.0, 1.0]])
    v = np.array([[0.1, -0.2, 0.3, 0.0], [0.0, 0.0, 0.0, 0.0]])
    om = np.array([[1.0, 2.0, 3.0, 0.0], [0.0, 0.0, 0.0, 0.0]])
    F, T, h, c = oracle.dem_forces(x, v, om, *P_BOX, p)
    x1, v1, w1 = oracle.dem_leapfrog(x, v, om, F, T, p)
    np.testing.assert_allclose(v1[0, :3], v[0, :3] + p.dt * np.array(p.g), rtol=1e-15)
    np.testing.assert_allclose(x1[0, :3], x[0, :3] + p.dt * v1[0, :3], rtol=1e-15)
    np.testing.assert_array_equal(w1[0], om[0])
    np.testing.assert_array_equal(x1[1], x[1])
    np.testing.assert_array_equal(v1[1], v[1])
