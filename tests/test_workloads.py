"""The seeded synthetic inputs follow their stated recipes (CPU): grid geometry, the
refined grid's point count, the batched workload's size and pressure draws, the paper's
multi-peak source, and determinism of every seeded generator."""
import numpy as np
import pytest

from paper_2006_03515_gb300 import workloads as W


def test_uniform_grid_cell_centres():
    pts, h = W.uniform_grid(4, 2.0)
    assert h == 0.5 and pts.shape == (64, 3)
    np.testing.assert_array_equal(pts[0], [0.25, 0.25, 0.25])
    np.testing.assert_array_equal(pts[1], [0.75, 0.25, 0.25])      # x fastest
    np.testing.assert_array_equal(pts[4], [0.25, 0.75, 0.25])
    np.testing.assert_array_equal(pts[16], [0.25, 0.25, 0.75])
    pts, h = W.uniform_grid(None, n_xyz=(8, 6, 4), Lxyz=(0.4, 0.3, 0.2))
    assert h == pytest.approx(0.05) and pts.shape == (192, 3)
    assert pts[:, 0].max() == pytest.approx(0.375) and pts[:, 2].max() == pytest.approx(0.175)
    with pytest.raises(ValueError):
        W.uniform_grid(None, n_xyz=(8, 8, 8), Lxyz=(1.0, 1.0, 2.0))


def test_refined_grid_point_count():
    # 2 cm cube, base h = 1/64 cm; the 13^3 base cells around the head each split into 8^3:
    # 128^3 - 13^3 + (13 * 8)^3 = 3,219,819 points (the adaptive workload)
    pts, h = W.refined_grid(2.0, 128, 8, (1.0, 1.0, 1.5), 6)
    assert len(pts) == 128 ** 3 - 13 ** 3 + 104 ** 3 == 3219819
    assert set(np.unique(h)) == {2.0 / 128, 2.0 / 1024}
    fine = h < 2.0 / 128
    lo, hi = pts[fine].min(0), pts[fine].max(0)
    assert np.all(hi - lo < 13 * 2.0 / 128)
    # cells tile the cube: total volume 8 cm^3
    assert float(np.sum(h ** 3)) == pytest.approx(8.0, rel=1e-12)


def test_batched_fields_follow_their_draws():
    seen_p = set()
    for k in range(12):
        pts, h, I, p = W.two_channel_field(k, n_min=10, n_max=20)
        n = round(len(pts) ** (1 / 3))
        assert n ** 3 == len(pts) and 10 <= n <= 20
        assert h[0] == pytest.approx(1.0 / n) and p in (760.0, 76.0)
        assert np.all(I >= 0) and I.max() > 0
        seen_p.add(p)
        pts2, _, I2, p2 = W.two_channel_field(k, n_min=10, n_max=20)
        assert p2 == p and np.array_equal(I2, I)      # seeded per field
    assert seen_p == {760.0, 76.0}


def test_multipeak_source():
    # Sec. 4.3: amp sin^2(50 pi x) sin^2(50 pi y) sin^2(50 pi z) in the middle half, 0 outside
    dims = (0.4, 0.4, 0.2)
    pts, h = W.uniform_grid(None, n_xyz=(32, 32, 16), Lxyz=dims)
    I = W.multipeak(pts, dims)
    inside = np.all((pts >= 0.25 * np.array(dims)) & (pts <= 0.75 * np.array(dims)), axis=1)
    assert np.all(I[~inside] == 0) and np.all(I >= 0) and I.max() <= 1.53e25
    j = int(np.flatnonzero(inside)[7])
    x, y, z = pts[j]
    want = 1.53e25 * (np.sin(50 * np.pi * x) * np.sin(50 * np.pi * y) * np.sin(50 * np.pi * z)) ** 2
    assert I[j] == pytest.approx(want, rel=1e-12)


def test_seeded_generators_are_deterministic():
    a = W.random_cloud(100, 5)
    b = W.random_cloud(100, 5)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert len(np.unique(a[0], axis=0)) == 100
    pts, _ = W.uniform_grid(8, 1.0)
    np.testing.assert_array_equal(W.gaussian_mixture(pts, 3), W.gaussian_mixture(pts, 3))
    assert not np.array_equal(W.gaussian_mixture(pts, 3), W.gaussian_mixture(pts, 4))
