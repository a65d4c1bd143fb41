"""Pins of the SPH oracle (Sec. 4.2, Eqs. 1-5) against facts fixed by the
mathematics: kernel normalisation and derivative, the density of a uniform
lattice, the rest state, momentum conservation, the sign of the artificial
viscosity's work, and the equation of state."""
import math

import numpy as np
import pytest

import oracle

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
    p = oracle.sph_params(0.01, 1.0)
    assert abs(p.c0 - 20 * math.sqrt(9.81 * 0.3)) < 1e-12
    assert abs(oracle.sph_eos(p, 1000.0)[0]) < 1e-9
    b = p.c0 ** 2 * 1000.0 / 7.0
    assert abs(oracle.sph_eos(p, 1010.0)[0] - b * ((1.01) ** 7 - 1.0)) < 1e-9 * b
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
