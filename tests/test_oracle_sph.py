"""Pins of the SPH oracle (Sec. 4.2, Eqs. 1-5) against facts fixed by the
mathematics: kernel normalisation and derivative, the density of a uniform
lattice, the rest state, momentum conservation, the sign of the artificial
viscosity's work, the equation of state, the pressure force of a particle
pair in closed form, the response to a linear pressure field (a = -grad P /
rho), and the symplectic corrector written out.  The last three are shown to
reject planted mistakes (a flipped sign, P_p - P_q, a lost mass factor, a
wrong corrector) in copies of the oracle built for the purpose."""
import math

import numpy as np
import pytest

import oracle
from oracle_mutants import mutant

KERNELS = ["wendland", "cubic"]


def lattice(nx, ny, nz, dp, offset=0.5):
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1).reshape(-1, 3)
    return (g + offset) * dp


@pytest.mark.parametrize("kind", KERNELS)
def test_kernel_normalised_and_derivative(kind):
    """4 pi int_0^{2h} W r^2 dr = 1; dW/dr = d/dr W by central differences;
    W(2h) = 0 and W decreases."""
    h = 0.013
    p = oracle.sph_params(h, 1.0, kernel=kind)
    r = np.linspace(0.0, 2 * h, 20001)
    W, D = oracle.sph_kernel(p, r)
    integral = np.trapezoid(4 * math.pi * r * r * W, r)
    assert abs(integral - 1.0) < 1e-6
    e = 1e-9
    Wp, _ = oracle.sph_kernel(p, r[1:-1] + e)
    Wm, _ = oracle.sph_kernel(p, r[1:-1] - e)
    assert np.max(np.abs((Wp - Wm) / (2 * e) - D[1:-1])) <= 1e-5 * np.max(np.abs(D))
    assert W[-1] == 0.0 and np.all(np.diff(W) <= 1e-12 * W[0])


@pytest.mark.parametrize("kind", KERNELS)
def test_uniform_lattice_density(kind):
    """Cubic lattice of spacing dp, h = 1.3 dp, m = rho0 dp^3: the summed
    density of an interior particle is rho0 within 1 %."""
    dp = 0.01
    x = lattice(12, 12, 12, dp)
    L = np.array([12 * dp] * 3)
    p = oracle.sph_params(1.3 * dp, 1000.0 * dp ** 3, kernel=kind)
    rho = oracle.sph_density_sum(x, L, (1, 1, 1), p)
    assert np.max(np.abs(rho / 1000.0 - 1.0)) < 0.01
    assert np.max(rho) - np.min(rho) < 1e-9 * 1000.0  # periodic lattice: all equal


def test_rest_state():
    """Uniform lattice at rest with uniform density (periodic): Drho = 0 and
    a = g for every particle."""
    dp = 0.01
    x = lattice(10, 10, 10, dp)
    L = np.array([10 * dp] * 3)
    p = oracle.sph_params(1.3 * dp, 1000.0 * dp ** 3)
    rho = np.full(x.shape[0], 1003.0)
    acc, dr, dtc = oracle.sph_rates(x, np.zeros_like(x), rho, L, (1, 1, 1), p)
    assert np.max(np.abs(dr)) < 1e-9
    assert np.max(np.abs(acc[:, :3] - np.array([0.0, 0.0, -9.81]))) < 1e-9
    assert dtc[1] == 0.0


def test_momentum_conservation_and_viscous_dissipation():
    """Random fluid in a periodic box: sum_p m a_p = M g (pairwise
    antisymmetry); with P = 0 (rho = rho0) and g = 0, the artificial
    viscosity does non-positive work: sum_p m v_p . a_p <= 0."""
    rng = np.random.default_rng(3)
    dp = 0.01
    x = lattice(9, 9, 9, dp) + rng.uniform(-0.2, 0.2, (729, 3)) * dp
    L = np.array([9 * dp] * 3)
    v = rng.normal(0, 0.5, (729, 3))
    m = 1000.0 * dp ** 3
    p = oracle.sph_params(1.3 * dp, m)
    rho = 1000.0 + rng.uniform(-5, 5, 729)
    acc, dr, _ = oracle.sph_rates(x, v, rho, L, (1, 1, 1), p)
    tot = np.sum(m * acc[:, :3], axis=0)
    assert np.max(np.abs(tot - m * 729 * np.array([0, 0, -9.81]))) < 1e-9 * np.sum(np.abs(m * acc[:, :3]))
    p0 = oracle.sph_params(1.3 * dp, m, g=(0.0, 0.0, 0.0))
    acc0, _, _ = oracle.sph_rates(x, v, np.full(729, 1000.0), L, (1, 1, 1), p0)
    assert np.sum(m * np.sum(v * acc0[:, :3], axis=1)) <= 0.0


def test_translation_and_divergence():
    """A uniform translation gives Drho = 0; a uniform expansion v = k x gives
    Drho ~ -3 k rho in the interior (continuity, Eq. 2) within 3 % (the kernel
    gradient sum of a lattice at h = 1.3 dp reproduces the identity to about
    2 %: a discretisation property, not rounding)."""
    dp = 0.01
    n = 14
    x = lattice(n, n, n, dp)
    L = np.array([n * dp] * 3)
    p = oracle.sph_params(1.3 * dp, 1000.0 * dp ** 3, g=(0, 0, 0))
    rho = np.full(x.shape[0], 1000.0)
    _, dr, _ = oracle.sph_rates(x, np.tile([0.3, -0.2, 0.1], (x.shape[0], 1)), rho, L, (0, 0, 0), p)
    assert np.max(np.abs(dr)) < 1e-9
    k = 0.5
    _, dr, _ = oracle.sph_rates(x, k * x, rho, L, (0, 0, 0), p)
    interior = np.all((x > 3 * dp) & (x < (n - 3) * dp), axis=1)
    assert np.max(np.abs(dr[interior] / (-3 * k * 1000.0) - 1.0)) < 0.03


def test_eos_and_dt():
    """The Tait law of Eqs. 3-4 has zero pressure at the rest density, and its
    slope there is the squared sound speed, dP/drho (rho0) = c0^2 (the
    physical meaning of c0; b = c0^2 rho0 / gamma is what makes it hold)."""
    p = oracle.sph_params(0.01, 1.0)
    assert abs(p.c0 - 20 * math.sqrt(9.81 * 0.3)) < 1e-12
    assert abs(oracle.sph_eos(p, 1000.0)[0]) < 1e-9
    e = 1e-4
    slope = (oracle.sph_eos(p, 1000.0 + e)[0] - oracle.sph_eos(p, 1000.0 - e)[0]) / (2 * e)
    assert abs(slope / p.c0 ** 2 - 1.0) < 1e-7
    # the pressure grows with the density (a stiff fluid: 1 % of compression
    # is about 7 % of rho0 c0^2 / gamma)
    assert oracle.sph_eos(p, 1010.0)[0] > 0.0 > oracle.sph_eos(p, 990.0)[0]
    assert abs(oracle.sph_dt(p, [9.81, 0.0]) - 0.2 * min(math.sqrt(0.01 / 9.81), 0.01 / p.c0)) < 1e-15


def test_symplectic_step_free_fall():
    """A single fluid particle far from others falls freely: after one step
    v = dt g and x = x0 + dt^2 g / 2 exactly (symplectic scheme with constant
    acceleration), and its density is unchanged."""
    p = oracle.sph_params(0.01, 1.0)
    x = np.array([[0.5, 0.5, 0.5]])
    L = np.array([1.0, 1.0, 1.0])
    xp, vp, rp, dt = oracle.sph_step(x, np.zeros((1, 3)), np.array([1000.0]), L, (0, 0, 0), p)
    assert abs(dt - 0.2 * min(math.sqrt(0.01 / 9.81), 0.01 / p.c0)) < 1e-15
    assert abs(vp[0, 2] + 9.81 * dt) < 1e-15
    assert abs(xp[0, 2] - (0.5 - 0.5 * 9.81 * dt * dt)) < 1e-15
    assert rp[0] == 1000.0


# ---------------------------------------------------------------------------
# The pressure term of Eq. 1 and the symplectic corrector, pinned by closed
# forms, and shown to reject planted mistakes.

C0 = 34.31  # sound speed of the dam-break workload, 20 sqrt(g 0.3)


def wendland_dwdr(r, h):
    """dW/dr of the Wendland C2 kernel W = a (1 - q/2)^4 (2q + 1),
    a = 21 / (16 pi h^3), q = r/h: differentiating the product gives
    dW/dq = -5 a q (1 - q/2)^3."""
    q = r / h
    a = 21.0 / (16.0 * math.pi * h ** 3)
    return -5.0 * a * q * (1.0 - 0.5 * q) ** 3 / h


def tait(rho, rho0=1000.0, gamma=7.0, c0=C0):
    b = c0 * c0 * rho0 / gamma
    return b * ((rho / rho0) ** gamma - 1.0)


def check_pair_pressure(orc):
    """Two fluid particles at rest (no gravity, no viscosity since v = 0), at
    distance r = 0.9 h along a skew direction, with unequal densities above
    rho0 (unequal, positive pressures): Eq. 1 with the gradient convention
    grad_p W = W'(r) (x_p - x_q)/r gives a_p = -m (P_p + P_q)/(rho_p rho_q)
    W'(r) (x_p - x_q)/r and a_q = -a_p.  W' < 0, so positive pressures push
    the particles apart; the densities do not change (Eq. 2, v = 0)."""
    h, m = 0.013, 2.197
    p = orc.sph_params(h, m, g=(0.0, 0.0, 0.0), c0=C0)
    u = np.array([0.48, -0.6, 0.64])
    u /= np.linalg.norm(u)
    r = 0.9 * h
    xq = np.array([0.5, 0.5, 0.5])
    x = np.stack([xq + r * u, xq])
    rho = np.array([1002.0, 1005.0])
    acc, dr, _ = orc.sph_rates(x, np.zeros_like(x), rho, [1.0, 1.0, 1.0], (0, 0, 0), p)
    P = tait(rho)
    expect = -m * (P[0] + P[1]) / (rho[0] * rho[1]) * wendland_dwdr(r, h) * u
    scale = np.linalg.norm(expect)
    assert np.max(np.abs(acc[0, :3] - expect)) <= 1e-12 * scale
    assert np.max(np.abs(acc[1, :3] + expect)) <= 1e-12 * scale
    assert np.dot(acc[0, :3], u) > 0.0  # repulsive
    assert np.max(np.abs(dr)) == 0.0


def lattice_linear_pressure(orc, kind):
    """An open 16^3 lattice at rest (dp = 0.01, h = 1.3 dp, m = rho0 dp^3, no
    gravity) whose densities make the Tait pressure linear in x,
    P = k (x - x_c) (|P| <= 0.01 b): the particles at least 3 dp from every
    face (outside the support's reach of the free surface) accelerate by
    a = -grad P / rho = (-k / rho, 0, 0) up to the discretisation error of the
    kernel-gradient sum (2.3 % for Wendland, 0.9 % for the cubic spline at
    this h / dp); the y and z components cancel by the lattice's symmetry."""
    dp, n = 0.01, 16
    x = lattice(n, n, n, dp)
    p = orc.sph_params(1.3 * dp, 1000.0 * dp ** 3, g=(0.0, 0.0, 0.0), c0=C0, kernel=kind)
    b = C0 * C0 * 1000.0 / 7.0
    k = 0.02 * b / (n * dp)
    P = k * (x[:, 0] - n * dp / 2)
    rho = 1000.0 * (1.0 + P / b) ** (1.0 / 7.0)
    assert np.max(np.abs(tait(rho) - P)) < 1e-9 * b  # the densities carry the intended field
    acc, _, _ = orc.sph_rates(x, np.zeros_like(x), rho, [n * dp] * 3, (0, 0, 0), p)
    inner = np.all((x > 3 * dp) & (x < (n - 3) * dp), axis=1)
    ax = -k / rho[inner]
    return np.max(np.abs(acc[inner, 0] / ax - 1.0)), np.max(np.abs(acc[inner, 1:3])) / np.max(np.abs(ax))


def check_linear_pressure(orc):
    for kind, bound in (("wendland", 0.03), ("cubic", 0.015)):
        rel, cross = lattice_linear_pressure(orc, kind)
        assert rel < bound, (kind, rel)
        assert cross < 1e-12, (kind, cross)


def check_corrector(orc):
    """One symplectic step of a jittered, moving fluid box with fixed boundary
    particles, against the scheme written out: rates at t^n give dt; the half
    state x + dt/2 v, v + dt/2 a, rho + dt/2 Drho (boundary particles: rho
    only); rates at the half state (a_h, Drho_h); then v1 = v0 + dt a_h,
    x1 = x0 + dt (v0 + v1)/2 for fluid particles and
    rho1 = rho0 (2 - e)/(2 + e), e = -(Drho_h / rho_h) dt for all.  The rates
    come from the oracle's own rate routine, pinned above; this pins the
    composition.  Also: every rate is nonzero (Drho and a vary along the
    step), and for the small e of one step rho1 - rho0 = dt Drho_h rho0 /
    rho_h to O(e^2) (the density update integrates Eq. 2)."""
    rng = np.random.default_rng(11)
    dp, n = 0.01, 8
    x = lattice(n, n, n, dp) + rng.uniform(-0.1, 0.1, (n ** 3, 3)) * dp
    typ = (x[:, 2] < 1.5 * dp).astype(np.float64)  # the bottom layer is fixed boundary
    x4 = np.concatenate([x, typ[:, None]], axis=1)
    v = rng.normal(0.0, 0.4, (n ** 3, 3)) * (1.0 - typ)[:, None]
    rho = 1000.0 + rng.uniform(-3.0, 3.0, n ** 3)
    L = [n * dp] * 3
    p = orc.sph_params(1.3 * dp, 1000.0 * dp ** 3, c0=C0)
    acc0, dr0, dtc = orc.sph_rates(x4, v, rho, L, (1, 1, 1), p)
    dt = orc.sph_dt(p, dtc, 0.2)
    fluid = typ == 0.0
    xh = x4.copy()
    vh = v.copy()
    xh[fluid, :3] += 0.5 * dt * v[fluid]
    vh[fluid] += 0.5 * dt * acc0[fluid, :3]
    rh = rho + 0.5 * dt * dr0
    acch, drh, _ = orc.sph_rates(xh, vh, rh, L, (1, 1, 1), p)
    assert np.min(np.abs(drh)) > 0.0 and np.min(np.linalg.norm(acch[fluid, :3] - acc0[fluid, :3], axis=1)) > 0.0
    v1 = v.copy()
    x1 = x4[:, :3].copy()
    v1[fluid] = v[fluid] + dt * acch[fluid, :3]
    x1[fluid] = x[fluid] + dt * 0.5 * (v[fluid] + v1[fluid])
    e = -(drh / rh) * dt
    rho1 = rho * (2.0 - e) / (2.0 + e)
    xs, vs, rs, dts = orc.sph_step(x4, v, rho, L, (1, 1, 1), p, cfl=0.2)
    assert dts == dt
    assert np.max(np.abs(xs[:, :3] - x1)) <= 1e-15 * 8
    assert np.max(np.abs(vs[:, :3] - v1)) <= 1e-13 * np.max(np.abs(v1))
    assert np.max(np.abs(rs - rho1)) <= 1e-13 * 1000.0
    assert np.max(np.abs(xs[~fluid, :3] - x[~fluid])) == 0.0 and np.max(np.abs(vs[~fluid, :3])) == 0.0
    cont = dt * drh * rho / rh
    assert np.max(np.abs((rs - rho) - cont)) <= 4.0 * np.max(np.abs(e)) ** 2 * 1000.0


def test_pair_pressure_closed_form():
    check_pair_pressure(oracle)


def test_linear_pressure_field():
    check_linear_pressure(oracle)


def test_symplectic_corrector_written_out():
    check_corrector(oracle)


PRESSURE_MISTAKES = {
    "sign": ("double c = -p->m * ((P[i] + P[j])", "double c = p->m * ((P[i] + P[j])"),
    "difference": ("double c = -p->m * ((P[i] + P[j])", "double c = -p->m * ((P[i] - P[j])"),
    "mass": ("double c = -p->m * ((P[i] + P[j])", "double c = -((P[i] + P[j])"),
    "density product": ("(P[i] + P[j]) / (rho[i] * rho[j])", "(P[i] + P[j]) / (rho[i] * rho[i])"),
}

CORRECTOR_MISTAKES = {
    "density update": ("rho[i] = rho[i] * (2.0 - e) / (2.0 + e);", "rho[i] = rho[i] * (2.0 + e) / (2.0 - e);"),
    "sign of e": ("double e = -(dr[i] / rh[i]) * dt;", "double e = (dr[i] / rh[i]) * dt;"),
    "position update": ("pos4[4 * (size_t)i + d] += dt * 0.5 * (v1 + v0);", "pos4[4 * (size_t)i + d] += dt * v1;"),
    "half-step density": ("rh[i] = rho[i] + 0.5 * dt * dr[i];", "rh[i] = rho[i] + dt * dr[i];"),
}


@pytest.mark.parametrize("what", list(PRESSURE_MISTAKES))
def test_pressure_pins_reject_planted_mistakes(tmp_path, what):
    """Each planted mistake in the pressure term fails the pair closed form;
    the sign, the difference and the lost mass fail the linear-field pin too
    (a density product rho_p rho_p differs from rho_p rho_q by 0.1 % in that
    nearly incompressible field, inside its discretisation bound)."""
    orc = mutant(tmp_path, *PRESSURE_MISTAKES[what])
    with pytest.raises(AssertionError):
        check_pair_pressure(orc)
    if what != "density product":
        with pytest.raises(AssertionError):
            check_linear_pressure(orc)


@pytest.mark.parametrize("what", list(CORRECTOR_MISTAKES))
def test_corrector_pin_rejects_planted_mistakes(tmp_path, what):
    orc = mutant(tmp_path, *CORRECTOR_MISTAKES[what])
    with pytest.raises(AssertionError):
        check_corrector(orc)
