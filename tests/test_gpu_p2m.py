"""GPU parity of the M'4 particle-mesh interpolation (Sec. 4.4) against the
oracle: particle-to-mesh on ragged and tiny periodic meshes, with particles
given outside the box, a clustered case past the staging room, bit-for-bit
repeatability, mesh-to-particle, and the paper's size (2M particles on 128^3)
on sampled nodes and the exact total."""
import numpy as np
import pytest
import torch

import oracle
from paper_1804_07598_gb300.p2m import ParticleMesh

pytestmark = pytest.mark.gpu


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def rms(a):
    return float(np.sqrt(np.mean(a ** 2)))


def setup(n, L, seed, cluster=None):
    rng = np.random.default_rng(seed)
    L = np.asarray(L, np.float64)
    x = np.zeros((n, 4))
    if cluster is None:
        x[:, :3] = rng.uniform(0.0, 1.0, size=(n, 3)) * L
    else:
        c, r = cluster
        x[:, :3] = np.asarray(c) + rng.uniform(-r, r, size=(n, 3))
    v = rng.normal(size=(n, 4))
    return f32(x), f32(v), L


def close(g, o, x, v, L, N):
    """Node by node within 2e-5 of the RMS plus 2e-6 of sum w |v| over the
    node's terms.  Two FP32 error sources: the scaled coordinate s = x N / L
    carries a few ulps of s, so every weight is off by up to ~1e-6 (absolute),
    which over a node's terms shows at ~1e-5 of the RMS; and a node sums every
    particle of its 4x4x4 cells, so its rounding grows with that absolute sum
    (thousands of terms on a coarse mesh or in a cluster)."""
    scale = oracle.p2m(x, np.abs(v), L, N)
    return bool(np.all(np.abs(g - o) <= 2e-6 * np.abs(scale) + 2e-5 * rms(o)))


def gpu_p2m(x, v, L, N):
    pm = ParticleMesh(L, N, len(x))
    mesh = pm.p2m(torch.as_tensor(x, dtype=torch.float32, device="cuda"),
                  torch.as_tensor(v, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    st = pm.check_status()
    return mesh.cpu().numpy().astype(np.float64), st, pm


@pytest.mark.parametrize("N", [(16, 20, 12), (8, 8, 8), (3, 4, 5)])
def test_p2m_matches_oracle(cuda, N):
    x, v, L = setup(20000, (1.0, 1.3, 0.8), 1)
    # a tenth of the particles given up to one box length outside: the binning wraps them
    x[::10, :3] += np.round(np.random.default_rng(2).uniform(-1, 1, size=(len(x[::10]), 3))) * L
    x = f32(x)
    g, st, _ = gpu_p2m(x, v, L, N)
    o = oracle.p2m(x, v, L, N)
    assert close(g, o, x, v, L, N)
    np.testing.assert_allclose(g.sum(axis=(0, 1, 2)), v.sum(0), rtol=1e-4)


def test_p2m_is_repeatable(cuda):
    x, v, L = setup(50000, (1.0, 1.0, 1.0), 3)
    a, _, _ = gpu_p2m(x, v, L, (32, 32, 32))
    b, _, _ = gpu_p2m(x[::-1].copy(), v[::-1].copy(), L, (32, 32, 32))  # other input order: same cells, same sort
    np.testing.assert_array_equal(a, gpu_p2m(x, v, L, (32, 32, 32))[0])
    assert close(a, b, x, v, L, (32, 32, 32))


def test_p2m_clustered_past_the_staging_room(cuda):
    """All particles in a few cells: tiles past the staging room read their
    particles from global memory, with the same result."""
    x, v, L = setup(30000, (1.0, 1.0, 1.0), 4, cluster=((0.5, 0.5, 0.5), 0.03))
    g, st, _ = gpu_p2m(x, v, L, (32, 32, 32))
    assert st.spilled > 0
    o = oracle.p2m(x, v, L, (32, 32, 32))
    assert close(g, o, x, v, L, (32, 32, 32))


def test_p2m_empty(cuda):
    g, st, _ = gpu_p2m(np.zeros((0, 4)), np.zeros((0, 4)), (1.0, 1.0, 1.0), (8, 8, 8))
    assert np.all(g == 0)


def test_m2p_matches_oracle(cuda):
    rng = np.random.default_rng(5)
    L, N = np.array([1.0, 0.7, 1.2]), (10, 7, 12)
    mesh = f32(rng.normal(size=(N[2], N[1], N[0], 4)))
    x, _, _ = setup(5000, L, 6)
    x[::7, :3] -= L  # outside the box: wrapped
    pm = ParticleMesh(L, N, len(x))
    out = pm.m2p(torch.as_tensor(x, dtype=torch.float32, device="cuda"),
                 torch.as_tensor(mesh, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    o = oracle.m2p(x, mesh, L)
    assert np.abs(out.cpu().numpy() - o).max() <= 1e-5 * rms(o)
    # taken in the binning's order: the same values, bit for bit
    xt = torch.as_tensor(x, dtype=torch.float32, device="cuda")
    pm.bin(xt, torch.zeros_like(xt))
    out2 = pm.m2p(xt, torch.as_tensor(mesh, dtype=torch.float32, device="cuda"), binned=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out2.cpu().numpy(), out.cpu().numpy())


def test_p2m_paper_size_sampled(cuda):
    """2M particles on a 128^3 mesh (the paper's interpolation benchmark):
    100 sampled nodes against the direct sum over the particles near each,
    and the exact total."""
    x, v, L = setup(2_000_000, (1.0, 1.0, 1.0), 7)
    N = (128, 128, 128)
    g, st, _ = gpu_p2m(x, v, L, N)
    h = 1.0 / 128
    rng = np.random.default_rng(8)
    nodes = rng.integers(0, 128, size=(100, 3))
    ref = np.zeros((100, 4))
    for k, (i, j, l) in enumerate(nodes):
        d = x[:, :3] - np.array([i, j, l]) * h
        d -= np.round(d)  # periodic, L = 1
        near = np.all(np.abs(d) < 2 * h, axis=1)
        w = np.prod(oracle.m4p(d[near] / h), axis=1)
        ref[k] = (w[:, None] * v[near]).sum(0)
    got = g[nodes[:, 2], nodes[:, 1], nodes[:, 0]]
    assert np.abs(got - ref).max() <= 1e-5 * rms(ref)
    np.testing.assert_allclose(g.sum(axis=(0, 1, 2)), v.sum(0), rtol=1e-4, atol=1e-2)
