"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the method itself (no cell index, neighbour
test, force or integrator): only lattices, seeded velocity draws and the
workload parameters.  It imports nothing from the CUDA library or the oracle.

Workloads (all synthetic; the paper's inputs are a 60^3 grid in a unit cube,
Sec. 4.1, whose printed sigma makes it implausible, so the LJ workloads are
the standard reduced-unit LJ fluid at density 0.8442):

* ``lj_small``   : 4000 particles, FCC 10^3 cells, FP64 path, 100 NVE steps.
* ``lj_1m``      : 1,000,188 particles, FCC 63^3 cells, FP32 path, 1000 steps.
* ``lj_adjoint`` : 32,768 particles, FCC 16x16x32 cells (orthorhombic box).
* ``lj_batched`` : 512 replicas, log-uniform sizes in [256, 16384].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

RHO_LJ = 0.8442


@dataclass
class LJWorkload:
    name: str
    cells: tuple          # FCC unit cells per dimension
    rho: float = RHO_LJ
    T: float = 0.72
    eps: float = 1.0
    sigma: float = 1.0
    rc: float = 2.5
    skin: float = 0.3
    dt: float = 0.005
    steps: int = 100
    seed: int = 12345
    precision: str = "f32"
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return 4 * int(np.prod(self.cells))

    @property
    def a(self) -> float:
        return (4.0 / self.rho) ** (1.0 / 3.0)

    @property
    def L(self) -> np.ndarray:
        return np.array(self.cells, np.float64) * self.a


WORKLOADS = {
    "lj_small": LJWorkload("lj_small", (10, 10, 10), steps=100, precision="f64"),
    "lj_1m": LJWorkload("lj_1m", (63, 63, 63), steps=1000, precision="f32"),
    "lj_adjoint": LJWorkload("lj_adjoint", (16, 16, 32), steps=200, precision="f32"),
}


def fcc_lattice(cells, a, offset=None) -> np.ndarray:
    """FCC sites [4*prod(cells), 3] in float64, origin shifted by offset (a/4 by
    default so that, at the lattice constants used here, no site sits on a cell
    wall)."""
    cells = tuple(int(c) for c in cells)
    if offset is None:
        offset = 0.25 * a
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    iz, iy, ix = np.meshgrid(np.arange(cells[2]), np.arange(cells[1]), np.arange(cells[0]), indexing="ij")
    corners = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    sites = (corners[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    return sites * a + offset


def maxwell_boltzmann(n: int, T: float, seed: int, mass: float = 1.0) -> np.ndarray:
    """Velocities [n, 3] (float64): normal draws with zero net momentum,
    rescaled so that the kinetic energy is exactly (3n-3)/2 * T."""
    rng = np.random.default_rng(seed)
    v = rng.normal(0.0, math.sqrt(T / mass), size=(n, 3))
    v -= v.mean(axis=0, keepdims=True)
    ke = 0.5 * mass * float(np.sum(v * v))
    target = 0.5 * (3 * n - 3) * T
    if ke > 0:
        v *= math.sqrt(target / ke)
    return v


def as4(x: np.ndarray, dtype=np.float64, w=0.0) -> np.ndarray:
    """Pad [n,3] to the [n,4] (x, y, z, w) layout."""
    out = np.full((x.shape[0], 4), w, dtype)
    out[:, :3] = x
    return out


def lj_state(wl: LJWorkload, jitter: float = 0.0, jitter_seed: int = 7):
    """(pos4, vel4, L) for an LJ workload; optional uniform position jitter of
    +-jitter*a (to leave the perfect lattice for parity tests)."""
    x = fcc_lattice(wl.cells, wl.a)
    if jitter > 0:
        rng = np.random.default_rng(jitter_seed)
        x = x + rng.uniform(-jitter * wl.a, jitter * wl.a, size=x.shape)
        x = np.mod(x, wl.L)
    v = maxwell_boltzmann(wl.n, wl.T, wl.seed)
    return as4(x), as4(v), wl.L.copy()


def random_box(n: int, L, seed: int, snap: float = 0.0, snap_to=None) -> np.ndarray:
    """Uniform random positions in [0,L)^3 [n,3] float64.  With snap>0, that
    fraction of the coordinates is moved exactly onto multiples of snap_to
    (cell walls), including 0."""
    rng = np.random.default_rng(seed)
    L = np.broadcast_to(np.asarray(L, np.float64), (3,))
    x = rng.uniform(0.0, 1.0, size=(n, 3)) * L
    if snap > 0 and snap_to is not None:
        w = np.broadcast_to(np.asarray(snap_to, np.float64), (3,))
        m = rng.uniform(size=(n, 3)) < snap
        k = np.floor(x / w)
        x = np.where(m, k * w, x)
        x = np.minimum(x, np.nextafter(L, 0))
    return x


def batched_replicas(count: int = 512, seed: int = 2024, nmin: int = 256, nmax: int = 16384):
    """Replica sizes, densities and temperatures: N log-uniform in [nmin, nmax],
    rho uniform in [0.70, 0.95], T uniform in [0.6, 1.5]."""
    rng = np.random.default_rng(seed)
    N = np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=count))).astype(np.int64)
    rho = rng.uniform(0.70, 0.95, size=count)
    T = rng.uniform(0.6, 1.5, size=count)
    return N, rho, T


def replica_state(N: int, rho: float, T: float, seed: int):
    """A cubic FCC-like fill of one replica: ceil((N/4)^(1/3)) cells per side,
    first N sites; box side from the density."""
    m = int(math.ceil((N / 4.0) ** (1.0 / 3.0) - 1e-9))
    L = (N / rho) ** (1.0 / 3.0)
    a = L / m
    x = fcc_lattice((m, m, m), a)[:N]
    v = maxwell_boltzmann(N, T, seed)
    return as4(x), as4(v), np.array([L, L, L])
