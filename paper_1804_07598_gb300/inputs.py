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
* ``lj_8m``      : 8,001,504 particles, FCC 126^3 cells: the cell-list build
  measured from HBM (its positions and velocities alone, 256 MB in FP32, are
  twice the GPU's L2).
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
    "lj_8m": LJWorkload("lj_8m", (126, 126, 126), steps=0, precision="f32"),
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


def replica_state(N: int, rho: float, T: float, seed: int, jitter: float = 0.06):
    """One replica of the ensemble: a cubic box of side (N/rho)^(1/3) with N
    sites drawn without replacement (seeded) from an FCC lattice of
    m = ceil((N/4)^(1/3)) cells per side (so the density is rho on average,
    with vacancies spread uniformly), each moved by a uniform jitter of
    +-jitter*a off the lattice, and Maxwell-Boltzmann velocities at T."""
    m = int(math.ceil((N / 4.0) ** (1.0 / 3.0) - 1e-9))
    L = (N / rho) ** (1.0 / 3.0)
    a = L / m
    sites = fcc_lattice((m, m, m), a)
    rng = np.random.default_rng(seed)
    keep = np.sort(rng.choice(sites.shape[0], size=N, replace=False))
    x = sites[keep]
    if jitter > 0:
        x = np.mod(x + rng.uniform(-jitter * a, jitter * a, size=x.shape), L)
    v = maxwell_boltzmann(N, T, seed + 1)
    return as4(x), as4(v), np.array([L, L, L])


def ensemble(count: int = 512, seed: int = 2024, nmin: int = 256, nmax: int = 16384):
    """The batched LJ ensemble: `count` replicas from batched_replicas, each
    filled by replica_state with its own seed.  Returns (list of
    (pos [N,4], vel [N,4], L [3]), N, rho, T)."""
    N, rho, T = batched_replicas(count, seed, nmin, nmax)
    reps = [replica_state(int(N[r]), float(rho[r]), float(T[r]), seed * 1000 + r) for r in range(count)]
    return reps, N, rho, T


# ---------------------------------------------------------------------------
# SPH dam break (Sec. 4.2 test case, the tank shape of the SPH workload)
# ---------------------------------------------------------------------------

# The fixed obstacle of the paper's dam break (shown, not dimensioned there):
# a box of (0.12, 0.12, 0.45) with its low corner at (0.9, 0.24, 0) of the
# tank's interior.
DAM_OBSTACLE = ((0.9, 0.24, 0.0), (0.12, 0.12, 0.45))


def dam_break(dp: float, tank=(1.6, 0.67, 0.4), column=(0.4, 0.67, 0.3), layers: int = 3, lz: float = 1.0,
              rho0: float = 1000.0, g: float = 9.81, gamma: float = 7.0, coef: float = 20.0, obstacle=None):
    """A fluid column at one end of an open-top tank with `layers` layers of
    fixed boundary particles on the floor and the four walls, all on a cubic
    lattice of spacing dp.  Coordinates start at 0 (the boundary layers fill
    [0, layers*dp) on the low sides).  Returns a dict with pos [n,4] (w = type,
    0 fluid / 1 boundary), vel [n,3] (zero), rho [n] (hydrostatic:
    rho0 (1 + rho0 g depth / b)^(1/gamma), b = c0^2 rho0 / gamma,
    c0 = coef sqrt(g h_swl)), the box L, and the SPH constants h = 1.3 dp,
    m = rho0 dp^3.  obstacle ((x0, y0, z0), (sx, sy, sz)) in the tank's
    interior coordinates (e.g. DAM_OBSTACLE) adds a box filled with fixed
    boundary particles on the lattice."""
    nb = int(layers)
    nxt, nyt, nzt = (int(round(t / dp)) for t in tank)
    nxf, nyf, nzf = (int(round(c / dp)) for c in column)
    off = nb * dp

    def grid(nx, ny, nz, x0, y0, z0):
        iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        return np.stack([x0 + (ix.ravel() + 0.5) * dp, y0 + (iy.ravel() + 0.5) * dp, z0 + (iz.ravel() + 0.5) * dp], 1)

    fluid = grid(nxf, nyf, nzf, off, off, off)
    floor = grid(nxt + 2 * nb, nyt + 2 * nb, nb, 0.0, 0.0, 0.0)
    xw = np.concatenate([grid(nb, nyt + 2 * nb, nzt, 0.0, 0.0, off),
                         grid(nb, nyt + 2 * nb, nzt, off + nxt * dp, 0.0, off)])
    yw = np.concatenate([grid(nxt, nb, nzt, off, 0.0, off), grid(nxt, nb, nzt, off, off + nyt * dp, off)])
    bnd = [floor, xw, yw]
    if obstacle is not None:
        (ox, oy, oz), (sx, sy, sz) = obstacle
        sz = min(sz, nzt * dp - oz)
        bnd.append(grid(int(round(sx / dp)), int(round(sy / dp)), int(round(sz / dp)), off + ox, off + oy, off + oz))
    bnd = np.concatenate(bnd)
    h_swl = column[2]  # the nominal fluid height of the paper's setup
    c0 = coef * math.sqrt(g * h_swl)
    b = c0 * c0 * rho0 / gamma
    x = np.concatenate([fluid, bnd])
    depth = np.maximum(h_swl - (x[:, 2] - off), 0.0)
    rho = rho0 * (1.0 + rho0 * g * depth / b) ** (1.0 / gamma)
    pos = np.zeros((x.shape[0], 4))
    pos[:, :3] = x
    pos[fluid.shape[0]:, 3] = 1.0
    L = np.array([(nxt + 2 * nb) * dp, (nyt + 2 * nb) * dp, lz])
    return dict(pos=pos, vel=np.zeros((x.shape[0], 3)), rho=rho, L=L, n_fluid=fluid.shape[0],
                n_boundary=bnd.shape[0], h=1.3 * dp, m=rho0 * dp ** 3, c0=c0, b=b, rho0=rho0, dp=dp,
                h_swl=h_swl)


SPH_DP = 3.7704e-3  # dam break with ~1.51M fluid particles (106 x 178 x 80)


# ---------------------------------------------------------------------------
# DEM avalanche (Sec. 4.5): grains on a cubic lattice in the upstream part of
# a box inclined by 30 degrees (gravity rotated), a floor and two x-walls of
# fixed grains (type 1), periodic in y, open in z.  The printed constants
# are kept (R = 0.06, m = 1, I = 1.44e-3, kn = 7.849, kt = 2.243,
# gn = 3.401); gamma_t = 0 and mu = 0.5 (not printed).  |g| and dt are not
# printed either: |g| is chosen so that the weight of an nz-grain column
# compresses the lowest contact by about 1 % of 2R under that kn, and dt
# resolves the contact oscillation (period ~2 pi sqrt(m_eff / (kn f)) ~ 5)
# with ~100 steps.

DEM_PARAMS = dict(R=0.06, m=1.0, I=1.44e-3, kn=7.849, kt=2.243, gn=3.401, gt=0.0, mu=0.5, dt=0.05)
DEM_SKIN = 0.012  # 0.2 R: r_list = 2R + skin


def dem_gravity(nz: int, R: float = 0.06, kn: float = 7.849, tilt_deg: float = 30.0, overlap: float = 0.01):
    """Gravity vector for an nz-high pile: nz m |g| = kn sqrt(d / 2R) d with
    d = overlap * 2R, tilted by tilt_deg about y (down-slope along +x)."""
    d = overlap * 2.0 * R
    gmag = kn * math.sqrt(d / (2.0 * R)) * d / nz
    t = math.radians(tilt_deg)
    return (gmag * math.sin(t), 0.0, -gmag * math.cos(t))


def dem_avalanche(nx: int, ny: int, nz: int, R: float = 0.06, gap: float = 0.02, seed: int = 17,
                  vel_scale: float = 1e-3):
    """(pos4, vel4, omega4, L, periodic, gravity) of the avalanche: nx*ny*nz
    moving grains (lattice spacing s = 2R(1 + gap)) from x = 3R, z = 3R; a
    floor of fixed grains at z = R (spacing >= 2R, periodic in y); fixed walls
    at x = R and x = L_x - R up to the block's top; the box is 2 nx + 4
    diameters long (room to flow), ny spacings wide (periodic), and open above
    (twice the block's height).  Small seeded random velocities."""
    s = 2.0 * R * (1.0 + gap)
    Lx = (2 * nx + 4) * 2.0 * R
    Ly = ny * s
    Lz = 2.0 * (nz * s + 4.0 * R)
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    moving = np.stack([3.0 * R + ix.ravel() * s, 0.5 * s + iy.ravel() * s, 3.0 * R + iz.ravel() * s], 1)
    nfx = int(math.floor(Lx / (2.0 * R)))
    nfy = int(math.floor(Ly / (2.0 * R)))
    fx, fy = np.meshgrid(np.arange(nfx), np.arange(nfy), indexing="ij")
    floor = np.stack([R + fx.ravel() * (Lx - 2.0 * R) / max(nfx - 1, 1), (fy.ravel() + 0.5) * (Ly / nfy),
                      np.full(fx.size, R)], 1)
    top = 3.0 * R + (nz - 1) * s + R
    nwz = int(math.floor((top - 2.0 * R) / (2.0 * R))) + 1
    wy, wz = np.meshgrid(np.arange(nfy), np.arange(1, nwz + 1), indexing="ij")
    wall = np.stack([np.zeros(wy.size), (wy.ravel() + 0.5) * (Ly / nfy), R + wz.ravel() * 2.0 * R], 1)
    walls = np.concatenate([wall + [R, 0.0, 0.0], wall + [Lx - R, 0.0, 0.0]])
    x = np.concatenate([moving, floor, walls])
    kind = np.concatenate([np.zeros(len(moving)), np.ones(len(floor) + len(walls))])
    pos = np.zeros((len(x), 4))
    pos[:, :3] = x
    pos[:, 3] = kind
    rng = np.random.default_rng(seed)
    vel = np.zeros_like(pos)
    vel[: len(moving), :3] = rng.normal(scale=vel_scale, size=(len(moving), 3))
    om = np.zeros_like(pos)
    return pos, vel, om, np.array([Lx, Ly, Lz]), (0, 1, 0), dem_gravity(nz, R)
