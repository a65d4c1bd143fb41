"""GPU parity of fpm_verlet_build / fpm_verlet_check against the oracle:
neighbour sets bit-exact (decided in the same precision), capacity overflow
reported, rebuild flag identical."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import ell_equal_csr, gpu_celllist, gpu_verlet, status_tensor, dev, fprec, tdtype
from paper_1804_07598_gb300 import fpm, inputs

pytestmark = pytest.mark.gpu

CASES = [
    dict(n=64, L=(6.0, 6.0, 6.0), per=(1, 1, 1), r=2.8),
    dict(n=150, L=(9.0, 12.0, 5.7), per=(1, 1, 1), r=2.8),
    dict(n=200, L=(10.0, 10.0, 10.0), per=(1, 0, 1), r=2.8),
    dict(n=120, L=(6.0, 6.0, 6.0), per=(0, 0, 0), r=2.8),
    dict(n=3001, L=(14.0, 15.0, 16.0), per=(1, 1, 1), r=2.5),
    dict(n=5000, L=(18.0, 9.0, 17.0), per=(0, 1, 1), r=2.8),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c['n']}")
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_verlet_sets_random(cuda, case, prec):
    L = np.array(case["L"])
    nc, _ = oracle.cell_grid(L, case["per"], case["r"])
    x = inputs.random_box(case["n"], L, seed=case["n"], snap=0.25, snap_to=L / nc)
    dt = np.float32 if prec == "f32" else np.float64
    g = gpu_celllist(inputs.as4(x, dt), L, case["per"], case["r"], prec)
    v = gpu_verlet(g, case["r"], prec, cap=256)
    assert v["status"].flags == 0
    offs, onbr = oracle.neighbors(g["pos"], L, case["per"], case["r"])
    ok, msg = ell_equal_csr(v, offs, onbr, case["n"])
    assert ok, msg
    assert v["status"].max_nn == int(np.diff(offs).max())
    assert np.array_equal(v["ref"].cpu().numpy(), g["pos"])


@pytest.mark.parametrize("name,prec", [("lj_small", "f64"), ("lj_small", "f32"), ("lj_1m", "f32")])
def test_verlet_sets_workloads(cuda, name, prec):
    """Every neighbour set of the full workload (4000 / 1,000,188 particles,
    jittered FCC) equals the oracle's."""
    wl = inputs.WORKLOADS[name]
    pos, _, L = inputs.lj_state(wl, jitter=0.06)
    dt = np.float32 if prec == "f32" else np.float64
    r = wl.rc + wl.skin
    g = gpu_celllist(pos.astype(dt), L, (1, 1, 1), r, prec)
    v = gpu_verlet(g, r, prec, cap=128)
    assert v["status"].flags == 0
    offs, onbr = oracle.neighbors(g["pos"], L, (1, 1, 1), r)
    ok, msg = ell_equal_csr(v, offs, onbr, g["pos"].shape[0])
    assert ok, msg


def test_verlet_capacity_overflow(cuda):
    wl = inputs.WORKLOADS["lj_small"]
    pos, _, L = inputs.lj_state(wl, jitter=0.06)
    g = gpu_celllist(pos.astype(np.float32), L, (1, 1, 1), 2.8, "f32")
    v = gpu_verlet(g, 2.8, "f32", cap=40)
    assert v["status"].flags & fpm.FPM_FLAG_CAPACITY
    assert fpm.fpm_status_from_device(v["status"]) == fpm.FPM_ERR_CAPACITY
    offs, _ = oracle.neighbors(g["pos"], L, (1, 1, 1), 2.8)
    assert v["status"].max_nn == int(np.diff(offs).max()) > 40
    assert np.all(v["nn"] == np.minimum(np.diff(offs), 40))


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_verlet_gate(cuda, prec):
    """A zero gate word skips the build; a set one builds, then clears the
    word and counts the rebuild."""
    L = np.array([12.0, 12.0, 12.0])
    x = inputs.random_box(800, L, seed=1)
    dt = np.float32 if prec == "f32" else np.float64
    g = gpu_celllist(inputs.as4(x, dt), L, (1, 1, 1), 2.8, prec)
    st = status_tensor()
    gate = st.data_ptr() + 8
    n = 800
    cap = 128
    nbr = torch.zeros((fpm.fpm_verlet_list_bytes(n, g["grid"], cap),), dtype=torch.uint8, device="cuda")
    nn = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    fpm.fpm_verlet_build(g["box"], g["grid"], n, fprec(prec), g["dev"]["pos"], g["dev"]["cs"], 2.8, cap, nbr, nn,
                         None, st, gate)
    torch.cuda.synchronize()
    assert torch.all(nn == -1)
    st[2] = 1
    fpm.fpm_verlet_build(g["box"], g["grid"], n, fprec(prec), g["dev"]["pos"], g["dev"]["cs"], 2.8, cap, nbr, nn,
                         None, st, gate)
    s = fpm.read_status(st)
    assert s.rebuild == 0 and s.nrebuild == 1
    assert torch.all(nn >= 0)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_verlet_check_matches_oracle(cuda, prec):
    L = np.array([15.0, 15.0, 15.0])
    rng = np.random.default_rng(8)
    ref = inputs.random_box(10000, L, seed=2)
    dt = np.float32 if prec == "f32" else np.float64
    for amp, expect in [(0.05, 0), (0.2, None)]:
        pos = np.mod(ref + rng.uniform(-amp, amp, ref.shape), L)
        p4, r4 = inputs.as4(pos, dt), inputs.as4(ref, dt)
        st = status_tensor()
        fpm.fpm_verlet_check(fpm.make_box(L), 10000, fprec(prec), dev(p4, tdtype(prec)), dev(r4, tdtype(prec)), 0.3,
                             st)
        s = fpm.read_status(st)
        flag, m = oracle.max_disp(p4, r4, L, (1, 1, 1), 0.3)
        assert s.rebuild == flag
        if expect is not None:
            assert flag == expect
        assert abs(np.array(s.max_disp2, np.uint32).view(np.float32) - m) <= 1e-6 * m
