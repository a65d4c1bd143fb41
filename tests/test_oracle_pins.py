"""Pins of the oracle against facts fixed by the paper and by mathematics
(no GPU involved).  Each test names what it pins and why a plausible mistake in
the oracle (a dropped term, a wrong sign or index, a transposed operand) would
fail it.
"""
import itertools
import os
import math

import numpy as np
import pytest

import oracle
from paper_1804_07598_gb300 import inputs

PER = [1, 1, 1]


# ---------------------------------------------------------------- helpers ---

def brute_neighbors(x, L, periodic, r):
    """O(n^2) neighbour sets by checking every periodic image explicitly
    (27 shifts), independent of the oracle's minimum-image formula and cells."""
    x = np.asarray(x, np.float64)[:, :3]
    n = x.shape[0]
    shifts = [np.array(s) * np.asarray(L) for s in itertools.product(
        *[(-1, 0, 1) if periodic[d] else (0,) for d in range(3)])]
    d2min = np.full((n, n), np.inf)
    for s in shifts:
        d = x[:, None, :] - x[None, :, :] + s[None, None, :]
        d2min = np.minimum(d2min, np.sum(d * d, axis=2))
    np.fill_diagonal(d2min, np.inf)
    return [set(np.nonzero(d2min[i] < r * r)[0].tolist()) for i in range(n)]


def csr_sets(offs, nbr):
    return [set(nbr[offs[i]:offs[i + 1]].tolist()) for i in range(len(offs) - 1)]


def lj_pair(r, eps=1.0, sigma=1.0, rc=10.0):
    """Two particles on the x axis in a large open box; returns (F on 0, U)."""
    L = [100.0, 100.0, 100.0]
    x = np.array([[50.0, 50.0, 50.0], [50.0 + r, 50.0, 50.0]])
    f, U, W, npairs = oracle.lj_forces(x, L, [0, 0, 0], eps, sigma, rc)
    return f, U, W, npairs


# ------------------------------------------------------------ cell lists ---

def test_cell_index_edges_and_containment():
    """x=0 -> cell 0, x just below L -> nc-1, and every particle lies inside
    the geometric bounds of its cell (up to single-precision rounding, far
    inside the 2^-12 cell-size margin) -- the property neighbour search needs."""
    L = np.array([16.79596191, 7.3, 11.0])
    r = 2.8
    nc, inv = oracle.cell_grid(L, PER, r)
    assert list(nc) == [5, 1, 3]  # 7.3 < 3*2.8 -> one cell in y
    edge = np.array([[0.0, 0.0, 0.0], np.nextafter(L, 0)], np.float64)
    for dt in (np.float32, np.float64):
        e = edge.astype(dt)
        if dt == np.float32:
            e[1] = np.nextafter(L.astype(np.float32), np.float32(0))
        cell, nbad, _ = oracle.cell_index(e, L, PER, r)
        assert nbad == 0
        assert cell[0] == 0 and cell[1] == int(np.prod(nc)) - 1
    x = inputs.random_box(5000, L, seed=3, snap=0.3, snap_to=L / nc)
    for dt in (np.float32, np.float64):
        xx = x.astype(dt)
        cell, nbad, _ = oracle.cell_index(xx, L, PER, r)
        assert nbad == 0
        c = np.stack([cell % nc[0], (cell // nc[0]) % nc[1], cell // (nc[0] * nc[1])], 1)
        assert np.all(c >= 0) and np.all(c < nc)
        w = L / nc
        tol = 1e-5 * L
        xd = xx.astype(np.float64)
        assert np.all(xd >= c * w - tol) and np.all(xd < (c + 1) * w + tol)


def test_cell_grid_rules():
    """Cell width >= r_cell always; periodic boxes too small for the minimum
    image are rejected; non-periodic dims may keep two cells."""
    for Ld in [5.7, 8.4, 8.41, 10.0, 105.81456]:
        nc, _ = oracle.cell_grid([Ld] * 3, PER, 2.8)
        assert Ld / nc[0] >= 2.8
        assert nc[0] == 1 or nc[0] >= 3
    with pytest.raises(ValueError):
        oracle.cell_grid([5.6, 10, 10], PER, 2.8)
    nc, _ = oracle.cell_grid([5.7, 10, 10], [0, 1, 1], 2.8)
    assert nc[0] == 2


def test_counting_sort_is_stable_sort():
    """Pinned to numpy's stable sort (a different algorithm): perm = stable
    argsort of the cell ids; cell_start = exclusive scan of the histogram."""
    rng = np.random.default_rng(1)
    for ncell, n in [(1, 10), (7, 1000), (1000, 20000), (50, 0)]:
        cell = rng.integers(0, ncell, size=n).astype(np.uint32)
        cs, perm = oracle.counting_sort(cell, ncell)
        assert np.array_equal(perm, np.argsort(cell, kind="stable").astype(np.uint32))
        assert cs[0] == 0 and cs[-1] == n
        assert np.array_equal(np.diff(cs.astype(np.int64)), np.bincount(cell, minlength=ncell))


# --------------------------------------------------------- neighbour sets ---

@pytest.mark.parametrize("case", [
    dict(n=64, L=[6.0, 6.0, 6.0], per=[1, 1, 1], r=2.8),           # nc = 1 in all dims
    dict(n=150, L=[9.0, 12.0, 5.7], per=[1, 1, 1], r=2.8),          # 3, 4, 1 cells
    dict(n=200, L=[10.0, 10.0, 10.0], per=[1, 0, 1], r=2.8),        # a wall in y
    dict(n=120, L=[6.0, 6.0, 6.0], per=[0, 0, 0], r=2.8),           # open box, 2 cells
    dict(n=300, L=[14.0, 14.0, 14.0], per=[1, 1, 1], r=2.5),
])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_neighbor_sets_equal_brute_force(case, dtype):
    """Pinned to an O(n^2) search over all 27 explicit periodic images, with
    particles on cell walls, at x=0 and just below L."""
    L = np.array(case["L"])
    nc, _ = oracle.cell_grid(L, case["per"], case["r"])
    x = inputs.random_box(case["n"], L, seed=case["n"], snap=0.25, snap_to=L / nc)
    x[0] = 0.0
    x[1] = np.nextafter(L, 0)
    xx = x.astype(dtype)
    offs, nbr = oracle.neighbors(xx, L, case["per"], case["r"])
    got = csr_sets(offs, nbr)
    want = brute_neighbors(xx.astype(np.float64), L, case["per"], case["r"])
    assert got == want
    # symmetry: j in N(i) <=> i in N(j)
    for i, s in enumerate(got):
        for j in s:
            assert i in got[j]
    # the single-particle scan agrees too
    for i in (0, 1, 5):
        assert set(oracle.neighbors_one(xx, L, case["per"], case["r"], i).tolist()) == want[i]


@pytest.mark.parametrize("r,count", [(0.8, 12), (1.1, 18), (1.3, 42), (1.45, 54), (1.6, 78)])
def test_fcc_shell_counts(r, count):
    """Textbook FCC coordination shells: 12, 6, 24, 12, 24 neighbours at
    r/a = sqrt(1/2), 1, sqrt(3/2), sqrt(2), sqrt(5/2)."""
    x = inputs.fcc_lattice((4, 4, 4), 1.0)
    offs, nbr = oracle.neighbors(x, [4.0] * 3, PER, r)
    assert np.all(np.diff(offs) == count)


# --------------------------------------------------------- Lennard-Jones ---

def test_lj_closed_forms():
    """V(sigma) = 0; V(2^(1/6) sigma) = -eps with zero force; the force is
    repulsive inside the minimum and attractive outside."""
    for eps, sigma in [(1.0, 1.0), (0.7, 1.3)]:
        rmin = 2 ** (1 / 6) * sigma
        f, U, W, npairs = lj_pair(rmin, eps, sigma)
        assert npairs == 1
        assert abs(U + eps) < 1e-13
        assert np.max(np.abs(f[:, :3])) < 1e-12
        f, U, _, _ = lj_pair(sigma, eps, sigma)
        assert abs(U) < 1e-13
        f, _, _, _ = lj_pair(0.95 * rmin, eps, sigma)
        assert f[0, 0] < 0 < f[1, 0]        # particle 0 pushed towards -x
        f, _, _, _ = lj_pair(1.2 * rmin, eps, sigma)
        assert f[0, 0] > 0 > f[1, 0]


def test_lj_force_is_minus_energy_gradient():
    """F = -dU/dx by central differences of the oracle's own energy (a code
    path separate from its force), on a jittered periodic LJ liquid."""
    wl = inputs.LJWorkload("t", (3, 3, 3))
    x, _, L = inputs.lj_state(wl, jitter=0.08)
    f, U, W, _ = oracle.lj_forces(x, L, PER, 1.0, 1.0, 2.5)
    h = 1e-6
    rng = np.random.default_rng(0)
    for _ in range(12):
        i, d = int(rng.integers(0, wl.n)), int(rng.integers(0, 3))
        xp, xm = x.copy(), x.copy()
        xp[i, d] += h
        xm[i, d] -= h
        _, Up, _, np1 = oracle.lj_forces(xp, L, PER, 1.0, 1.0, 2.5)
        _, Um, _, np2 = oracle.lj_forces(xm, L, PER, 1.0, 1.0, 2.5)
        if np1 != np2:
            continue
        assert abs(-(Up - Um) / (2 * h) - f[i, d]) < 1e-6 * max(1.0, abs(f[i, d]))


def test_lj_newton3_and_energy_bookkeeping():
    """Sum of forces vanishes (pairwise antisymmetry); per-particle half
    energies sum to U."""
    wl = inputs.LJWorkload("t", (5, 5, 5))
    x, _, L = inputs.lj_state(wl, jitter=0.1)
    f, U, W, _ = oracle.lj_forces(x, L, PER, 1.0, 1.0, 2.5)
    scale = np.sum(np.abs(f[:, :3]))
    assert np.all(np.abs(f[:, :3].sum(0)) <= 1e-13 * scale)
    assert abs(f[:, 3].sum() - U) < 1e-10 * abs(U)


def test_fcc_lattice_sum():
    """Perfect FCC at T=0: all forces vanish by symmetry and U/N equals the
    lattice sum 1/2 * sum_shells n_s V(r_s) over the shells inside rc
    (12, 6, 24, 12 sites at r/a = sqrt(1/2), 1, sqrt(3/2), sqrt(2))."""
    wl = inputs.WORKLOADS["lj_small"]
    x, _, L = inputs.lj_state(wl)
    f, U, W, npairs = oracle.lj_forces(x, L, PER, 1.0, 1.0, 2.5)
    assert np.max(np.abs(f[:, :3])) < 1e-11
    a = wl.a

    def V(r):
        return 4.0 * ((1.0 / r) ** 12 - (1.0 / r) ** 6)

    shells = [(12, math.sqrt(0.5)), (6, 1.0), (24, math.sqrt(1.5)), (12, math.sqrt(2.0))]
    want = 0.5 * sum(c * V(s * a) for c, s in shells)
    assert abs(U / wl.n - want) < 1e-12 * abs(want)
    assert npairs == wl.n * 27


def test_virial_open_cluster():
    """For a non-periodic cluster the pair virial sum_{i<j} r_ij.F_ij equals
    sum_i x_i.F_i (a geometric identity)."""
    rng = np.random.default_rng(5)
    x = inputs.fcc_lattice((3, 3, 3), 1.6796) + 20.0 + rng.uniform(-0.1, 0.1, (108, 3))
    f, U, W, _ = oracle.lj_forces(x, [60.0] * 3, [0, 0, 0], 1.0, 1.0, 2.5)
    assert abs(W - np.sum(x * f[:, :3])) < 1e-10 * abs(W)


def test_lj_mask_f32_matches_f64_away_from_cutoff():
    """The single-precision cutoff decision differs from FP64 only for pairs
    within rounding of rc: forces agree to 1e-9 once those are absent."""
    wl = inputs.LJWorkload("t", (4, 4, 4))
    x, _, L = inputs.lj_state(wl, jitter=0.1)
    x32 = x.astype(np.float32).astype(np.float64)
    f1, U1, _, p1 = oracle.lj_forces(x32, L, PER, 1.0, 1.0, 2.5, mask_f32=False)
    f2, U2, _, p2 = oracle.lj_forces(x32, L, PER, 1.0, 1.0, 2.5, mask_f32=True)
    assert p1 == p2
    assert np.max(np.abs(f1 - f2)) < 1e-9


def test_force_one_matches_all():
    wl = inputs.LJWorkload("t", (4, 4, 4))
    x, _, L = inputs.lj_state(wl, jitter=0.1)
    f, *_ = oracle.lj_forces(x, L, PER, 1.0, 1.0, 2.5)
    for i in (0, 17, 255):
        assert np.allclose(oracle.lj_force_one(x, L, PER, 1.0, 1.0, 2.5, i), f[i], atol=1e-12)


# --------------------------------------------------------- velocity Verlet ---

def test_vv_free_flight_and_wrap():
    """eps = 0: particles move ballistically, x(t) = wrap(x0 + t v0)."""
    L = np.array([10.0, 10.0, 10.0])
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 10, (50, 3))
    v = rng.normal(0, 3, (50, 3))
    p, vv, _ = oracle.lj_nve(x, v, L, PER, 0.0, 1.0, 2.5, 0.01, 40, record=False)
    want = np.mod(x + 40 * 0.01 * v, L)
    d = p[:, :3] - want
    d -= L * np.round(d / L)
    assert np.max(np.abs(d)) < 1e-12
    assert np.allclose(vv[:, :3], v)


def test_vv_momentum_reversibility_energy():
    """NVE velocity Verlet on the small LJ workload: total momentum stays zero,
    the scheme is time-reversible (negate v, run back, recover x0) and the
    total energy (with U shifted by V(rc) per pair to remove the jump at the
    cutoff) drifts by < 1e-4 relative over 100 steps."""
    wl = inputs.WORKLOADS["lj_small"]
    x, v, L = inputs.lj_state(wl)
    p, vv, e = oracle.lj_nve(x, v, L, PER, 1.0, 1.0, 2.5, wl.dt, wl.steps)
    assert np.max(np.abs(vv[:, :3].sum(0))) < 1e-10
    vrc = 4.0 * (2.5 ** -12 - 2.5 ** -6)
    E = e[:, 0] + e[:, 1] - e[:, 3] * vrc
    assert np.max(np.abs(E - E[0])) / abs(E[0]) < 1e-4
    back, vb, _ = oracle.lj_nve(p, -vv, L, PER, 1.0, 1.0, 2.5, wl.dt, wl.steps, record=False)
    d = back[:, :3] - x[:, :3]
    d -= L * np.round(d / L)
    assert np.max(np.abs(d)) < 1e-8
    assert np.max(np.abs(vb[:, :3] + v[:, :3])) < 1e-8


def test_vv_single_step_matches_definition():
    """One kick-drift-kick step equals its definition written out."""
    wl = inputs.LJWorkload("t", (3, 3, 3))
    x, v, L = inputs.lj_state(wl, jitter=0.05)
    f0, *_ = oracle.lj_forces(x, L, PER, 1.0, 1.0, 2.5)
    p1, v1 = oracle.vv_kick_drift(x, v, f0, 0.005, L, PER)
    vh = v[:, :3] + 0.0025 * f0[:, :3]
    assert np.allclose(v1[:, :3], vh, rtol=0, atol=1e-15)
    assert np.allclose(p1[:, :3], np.mod(x[:, :3] + 0.005 * vh, L), rtol=0, atol=1e-13)


def test_max_disp():
    L = [10.0, 10.0, 10.0]
    ref = np.array([[0.05, 5.0, 5.0], [5.0, 5.0, 5.0]])
    pos = ref.copy()
    pos[0, 0] = 9.95  # moved by -0.1 through the periodic wall
    flag, m = oracle.max_disp(pos, ref, L, PER, 0.3)
    assert flag == 0 and abs(m - 0.01) < 1e-12
    pos[1, 1] += 0.16
    flag, m = oracle.max_disp(pos, ref, L, PER, 0.3)
    assert flag == 1


def _golden(name):
    vals = {}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


@pytest.mark.parametrize("m,R,d", [(11, 7.1, 1.1), (12, 8.1, 1.1), (12, 8.1, 1.0)])
def test_fcc_lattice_sums_published(m, R, d):
    """The oracle's LJ energy and virial of a perfect FCC crystal with a long
    cutoff R*d equal the published FCC lattice sums A12, A6
    (tests/golden/fcc_lattice_sums.txt) minus the sites beyond the cutoff,
    counted as a continuum of density sqrt(2)/d^3:
    tail_n = 4 pi sqrt(2) / ((n - 3) R^(n-3)).  (R^2 is not an integer, so no
    shell sits on the cutoff.)  The tolerance is relative to the sum of the
    two terms' magnitudes (the energy and virial are differences of them);
    the continuum tail is good to about 1e-5 of it.  Checks the pair
    potential, the 1/2 of the energy bookkeeping and the virial sign and
    scale."""
    g = _golden("fcc_lattice_sums.txt")
    a = d * math.sqrt(2.0)
    x = inputs.fcc_lattice((m, m, m), a)
    L = np.array([m * a] * 3)
    f, U, W, _ = oracle.lj_forces(x, L, PER, 1.0, 1.0, R * d)
    n = x.shape[0]
    a12 = g["A12"] - 4 * math.pi * math.sqrt(2.0) / (9 * R ** 9)
    a6 = g["A6"] - 4 * math.pi * math.sqrt(2.0) / (3 * R ** 3)
    u = 2.0 * (a12 * d ** -12 - a6 * d ** -6)
    w = 12.0 * (2.0 * a12 * d ** -12 - a6 * d ** -6)
    assert abs(U / n - u) < 3e-5 * 2.0 * (a12 * d ** -12 + a6 * d ** -6), (U / n, u)
    assert abs(W / n - w) < 3e-5 * 12.0 * (2.0 * a12 * d ** -12 + a6 * d ** -6), (W / n, w)
    assert np.max(np.abs(f[:, :3])) < 1e-10


def test_multicore_oracle_matches_serial():
    """The all-core timing variant (each particle's sum from its own side)
    gives the serial half-list sums up to rounding order, and the same NVE
    trajectory over a few steps."""
    from paper_1804_07598_gb300 import inputs
    wl = inputs.LJWorkload("omp_check", (5, 5, 5))
    pos, vel, L = inputs.lj_state(wl, jitter=0.06)
    f, U, W, npairs = oracle.lj_forces(pos, L, (1, 1, 1), 1.0, 1.0, 2.5)
    fo, outo = oracle.lj_forces_omp(pos, L, (1, 1, 1), 1.0, 1.0, 2.5)
    rms = np.sqrt(np.mean(np.sum(f[:, :3] ** 2, axis=1)))
    assert np.max(np.abs(fo - f)) <= 1e-12 * rms
    assert np.allclose(outo[:2], [U, W], rtol=1e-12) and outo[2] == npairs
    p1, v1, _ = oracle.lj_nve(pos, vel, L, (1, 1, 1), 1.0, 1.0, 2.5, 0.005, 5, record=False)
    p2, v2 = oracle.lj_nve_omp(pos, vel, L, (1, 1, 1), 1.0, 1.0, 2.5, 0.005, 5)
    assert np.max(np.abs(p2 - p1)) < 1e-10 and np.max(np.abs(v2 - v1)) < 1e-10
    assert oracle.threads() >= 1
