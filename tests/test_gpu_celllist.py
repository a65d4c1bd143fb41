"""GPU parity of fpm_celllist_build against the oracle: cell ids, the stable
permutation, cell_start and the reordered (wrapped) arrays must be bit-exact."""
import numpy as np
import pytest

import oracle
from gpu_util import gpu_celllist
from paper_1804_07598_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = [
    dict(n=1, L=(10.0, 10.0, 10.0), per=(1, 1, 1), r=2.8),
    dict(n=33, L=(6.0, 6.0, 6.0), per=(1, 1, 1), r=2.8),            # one cell, > 32 particles
    dict(n=700, L=(6.5, 6.5, 6.5), per=(1, 1, 1), r=2.8),           # one cell, rank-count path
    dict(n=257, L=(9.0, 12.0, 5.7), per=(1, 1, 1), r=2.8),          # 3 x 4 x 1 cells
    dict(n=1000, L=(10.0, 10.0, 10.0), per=(1, 0, 1), r=2.8),       # a wall in y
    dict(n=513, L=(6.0, 6.0, 6.0), per=(0, 0, 0), r=2.8),           # open box, 2 cells per dim
    dict(n=20000, L=(30.0, 25.0, 28.0), per=(1, 1, 1), r=2.5),
]


def oracle_cells(pos, L, per, r, vel=None, ids=None):
    return oracle.celllist_build(pos, L, per, r, vel=vel, ids=ids)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c['n']}")
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_celllist_random_boxes(cuda, case, prec):
    L = np.array(case["L"])
    nc, _ = oracle.cell_grid(L, case["per"], case["r"])
    x = inputs.random_box(case["n"], L, seed=case["n"] + 11, snap=0.2, snap_to=L / nc)
    if case["n"] > 2:
        x[0] = 0.0
        x[1] = np.nextafter(L, 0) if prec == "f64" else np.nextafter(L.astype(np.float32), np.float32(0))
    # periodic coordinates up to one box length outside are wrapped by the build
    rng = np.random.default_rng(3)
    shift = rng.integers(-1, 2, size=x.shape) * L * np.asarray(case["per"])
    x = x + np.where(rng.uniform(size=x.shape) < 0.1, shift, 0.0)
    dt = np.float32 if prec == "f32" else np.float64
    pos = inputs.as4(x, dt)
    vel = inputs.as4(rng.normal(size=x.shape), dt)
    ids = rng.permutation(case["n"]).astype(np.uint32)
    g = gpu_celllist(pos, L, case["per"], case["r"], prec, vel4=vel, ids=ids)
    o = oracle_cells(pos, L, case["per"], case["r"], vel=vel, ids=ids)
    assert fpm_ok(g)
    assert np.array_equal(g["cell_start"], o["cell_start"])
    assert np.array_equal(g["perm"], o["perm"])
    assert np.array_equal(g["pos"].view(np.uint8), o["pos"].astype(dt).view(np.uint8))
    assert np.array_equal(g["vel"], o["vel"])
    assert np.array_equal(g["ids"], o["ids"])


def fpm_ok(g):
    return g["status"].flags == 0


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_celllist_inplace_equals_out_of_place(cuda, prec):
    L = np.array([20.0, 20.0, 20.0])
    x = inputs.random_box(5000, L, seed=9)
    dt = np.float32 if prec == "f32" else np.float64
    pos = inputs.as4(x, dt)
    vel = inputs.as4(x[::-1].copy(), dt)
    a = gpu_celllist(pos, L, (1, 1, 1), 2.8, prec, vel4=vel, ids=np.arange(5000))
    b = gpu_celllist(pos, L, (1, 1, 1), 2.8, prec, vel4=vel, ids=np.arange(5000), inplace=True)
    for k in ("pos", "vel", "ids", "perm", "cell_start"):
        assert np.array_equal(a[k], b[k]), k
    c = gpu_celllist(pos, L, (1, 1, 1), 2.8, prec, vel4=vel, ids=None, inplace=True)
    assert np.array_equal(c["ids"], a["perm"])  # ids default to the input index


@pytest.mark.parametrize("name,prec", [("lj_small", "f64"), ("lj_1m", "f32"), ("lj_1m", "f64")])
def test_celllist_workloads(cuda, name, prec):
    """Full-size FCC workloads (4000 and 1,000,188 particles): whole-array
    bit-exact comparison, plus determinism over two runs."""
    wl = inputs.WORKLOADS[name]
    pos, vel, L = inputs.lj_state(wl, jitter=0.05)
    dt = np.float32 if prec == "f32" else np.float64
    pos, vel = pos.astype(dt), vel.astype(dt)
    r = wl.rc + wl.skin
    g = gpu_celllist(pos, L, (1, 1, 1), r, prec, vel4=vel)
    o = oracle_cells(pos, L, (1, 1, 1), r, vel=vel)
    assert fpm_ok(g)
    assert np.array_equal(g["cell_start"], o["cell_start"])
    assert np.array_equal(g["perm"], o["perm"])
    assert np.array_equal(g["pos"], o["pos"].astype(dt))
    g2 = gpu_celllist(pos, L, (1, 1, 1), r, prec, vel4=vel)
    assert np.array_equal(g2["perm"], g["perm"]) and np.array_equal(g2["pos"], g["pos"])


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_celllist_crowded_cells_among_many(cuda, prec):
    """More cells than the sort kernel has warps (31^3), so each warp sorts
    cells two at a time, with a dense cluster whose cells hold hundreds of
    particles next to ordinary ones: bit-exact against the oracle."""
    L = np.array([80.0, 80.0, 80.0])
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.uniform(0.0, 80.0, size=(200000, 3)), rng.uniform(40.0, 47.5, size=(20000, 3))])
    x = x[rng.permutation(x.shape[0])]
    dt = np.float32 if prec == "f32" else np.float64
    pos = inputs.as4(x, dt)
    vel = inputs.as4(rng.normal(size=x.shape), dt)
    o = oracle_cells(pos, L, (1, 1, 1), 2.5, vel=vel)
    k = np.diff(o["cell_start"])
    assert len(k) > 20000 and k.max() > 32 and np.sum(k > 32) < len(k) // 100
    g = gpu_celllist(pos, L, (1, 1, 1), 2.5, prec, vel4=vel)
    assert fpm_ok(g)
    assert np.array_equal(g["cell_start"], o["cell_start"])
    assert np.array_equal(g["perm"], o["perm"])
    assert np.array_equal(g["pos"], o["pos"].astype(dt))
    assert np.array_equal(g["vel"], o["vel"])


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_celllist_sparse_grid(cuda, prec):
    """Far fewer particles than cells (the sparse sort: a lane per cell of up
    to 8), with cells of 9-32 and of hundreds of particles among them (taken
    by the warp): bit-exact against the oracle."""
    L = np.array([20.0, 20.0, 20.0])
    rng = np.random.default_rng(12)
    parts = [rng.uniform(0.0, 20.0, size=(40000, 3)),  # ~0.04 per cell
             rng.uniform(5.0, 5.19, size=(600, 3)),    # one crowded cell
             rng.uniform(11.0, 11.19, size=(20, 3))]   # a cell of ~20
    parts += [rng.uniform(c, c + 0.19, size=(int(k), 3)) for c, k in zip(np.linspace(1.0, 18.0, 40),
                                                                         rng.integers(2, 12, 40))]
    x = np.concatenate(parts)
    x = x[rng.permutation(len(x))]
    dt = np.float32 if prec == "f32" else np.float64
    pos = inputs.as4(x, dt)
    vel = inputs.as4(rng.normal(size=x.shape), dt)
    o = oracle_cells(pos, L, (1, 1, 1), 0.2, vel=vel)
    k = np.diff(o["cell_start"])
    assert len(x) < 4 * len(k) and k.max() > 32 and np.sum((k > 8) & (k <= 32)) >= 1 and np.sum(k == 0) > 0
    g = gpu_celllist(pos, L, (1, 1, 1), 0.2, prec, vel4=vel)
    assert fpm_ok(g)
    assert np.array_equal(g["cell_start"], o["cell_start"])
    assert np.array_equal(g["perm"], o["perm"])
    assert np.array_equal(g["pos"], o["pos"].astype(dt))
    assert np.array_equal(g["vel"], o["vel"])


def test_celllist_empty(cuda):
    g = gpu_celllist(np.zeros((0, 4), np.float32), (10.0, 10.0, 10.0), (1, 1, 1), 2.8, "f32")
    assert np.all(g["cell_start"] == 0)


def test_celllist_domain_flag(cuda):
    """A particle outside a non-periodic dimension latches FPM_FLAG_DOMAIN and
    is binned into the nearest cell, like the oracle does."""
    L = np.array([10.0, 10.0, 10.0])
    x = inputs.random_box(100, L, seed=4)
    x[17, 1] = 10.5   # above the wall in y
    x[42, 1] = -0.25  # below it
    pos = inputs.as4(x, np.float32)
    g = gpu_celllist(pos, L, (1, 0, 1), 2.8, "f32")
    assert g["status"].flags & 2
    assert g["status"].bad_index in (17, 42)
    o = oracle_cells(pos, L, (1, 0, 1), 2.8)
    assert o["nbad"] == 2
    assert np.array_equal(g["perm"], o["perm"])
