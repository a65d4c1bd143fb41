"""Pins of the M'4 particle-mesh interpolation oracle (Sec. 4.4) against the
kernel's published properties: its closed-form values, partition of unity,
conservation of the first and second moments, interpolation at the nodes,
and exact reproduction of quadratic fields by mesh-to-particle."""
import numpy as np

import oracle


def test_m4p_closed_form_values():
    x = np.array([0.0, 0.5, 1.0, 1.5, 2.0, 2.5, -0.5, -1.5])
    ref = np.array([1.0, 0.5625, 0.0, -0.0625, 0.0, 0.0, 0.5625, -0.0625])
    np.testing.assert_allclose(oracle.m4p(x), ref, atol=1e-15)


def test_m4p_partition_of_unity_and_moments():
    """For every offset t in [0, 1): sum_k M'4(t - k) = 1, sum_k k M'4(t-k) = t,
    sum_k k^2 M'4(t - k) = t^2 (k = -1..2): the kernel conserves the zeroth,
    first and second moments."""
    t = np.linspace(0.0, 1.0, 101, endpoint=False)
    k = np.arange(-1, 3)[None, :]
    w = oracle.m4p(t[:, None] - k)
    np.testing.assert_allclose(w.sum(1), 1.0, atol=1e-14)
    np.testing.assert_allclose((w * k).sum(1), t, atol=1e-14)
    np.testing.assert_allclose((w * k ** 2).sum(1), t ** 2, atol=1e-14)


def test_p2m_conserves_total_and_moments():
    """Scattered strength sums to the particles' total; the mesh's first and
    second moments equal the particles' (particles away from the periodic
    seam, so that unwrapped node coordinates apply)."""
    rng = np.random.default_rng(1)
    L, N = np.array([2.0, 3.0, 4.0]), (16, 24, 32)
    h = L / np.array(N)
    x = np.zeros((300, 4))
    x[:, :3] = rng.uniform(3 * h, L - 3 * h, size=(300, 3))
    q = rng.normal(size=(300, 1))
    mesh = oracle.p2m(x, q, L, N)[..., 0]
    assert np.isclose(mesh.sum(), q.sum(), rtol=1e-12)
    grids = np.meshgrid(np.arange(N[2]) * h[2], np.arange(N[1]) * h[1], np.arange(N[0]) * h[0], indexing="ij")
    for d, g in zip((2, 1, 0), grids):
        assert np.isclose((mesh * g).sum(), (q[:, 0] * x[:, d]).sum(), rtol=1e-11)
        assert np.isclose((mesh * g ** 2).sum(), (q[:, 0] * x[:, d] ** 2).sum(), rtol=1e-11)


def test_particle_on_a_node():
    """M'4 interpolates: a particle exactly on a node gives that node its
    strength and every other node 0 (M'4(1) = M'4(2) = 0)."""
    L, N = np.array([1.0, 1.0, 1.0]), (8, 8, 8)
    x = np.array([[3 / 8, 5 / 8, 0.0, 0.0]])
    mesh = oracle.p2m(x, np.array([[2.5, -1.0]]), L, N)
    nz = np.argwhere(np.abs(mesh[..., 0]) > 1e-15)
    assert nz.tolist() == [[0, 5, 3]]
    np.testing.assert_allclose(mesh[0, 5, 3], [2.5, -1.0], rtol=1e-15)


def test_m2p_reproduces_quadratics():
    """Mesh-to-particle of a quadratic field sampled at the nodes is exact
    (away from the periodic seam)."""
    rng = np.random.default_rng(2)
    L, N = np.array([1.0, 1.5, 2.0]), (10, 15, 20)
    h = L / np.array(N)
    zz, yy, xx = np.meshgrid(np.arange(N[2]) * h[2], np.arange(N[1]) * h[1], np.arange(N[0]) * h[0], indexing="ij")

    def f(x, y, z):
        return 1.0 + 2.0 * x - 3.0 * y + 0.5 * z + x * x - 2.0 * x * y + 1.5 * z * z

    mesh = f(xx, yy, zz)[..., None]
    p = np.zeros((200, 4))
    p[:, :3] = rng.uniform(2 * h, L - 3 * h, size=(200, 3))
    np.testing.assert_allclose(oracle.m2p(p, mesh, L)[:, 0], f(p[:, 0], p[:, 1], p[:, 2]), rtol=1e-12)


def test_p2m_periodic_wrap():
    """A particle near x = 0 spreads to the nodes at the far end, and a
    particle given one box length out lands exactly where its image does."""
    L, N = np.array([1.0, 1.0, 1.0]), (8, 8, 8)
    x = np.array([[0.01, 0.5, 0.5, 0.0]])
    a = oracle.p2m(x, np.ones((1, 1)), L, N)
    assert np.abs(a[4, 4, 7, 0]) > 0 and np.abs(a[4, 4, 6, 0]) == 0
    b = oracle.p2m(x + [1.0, -1.0, 0.0, 0.0], np.ones((1, 1)), L, N)
    np.testing.assert_allclose(a, b, atol=1e-15)
