"""Host-side scene helpers (no GPU)."""
import numpy as np

from paper_2401_11882_gb300 import scenes


def test_spatial_order_is_a_permutation_along_the_z_curve():
    rng = np.random.default_rng(0)
    p = rng.uniform(0, 1, (500, 2))
    o = scenes.spatial_order(p)
    assert np.array_equal(np.sort(o), np.arange(500))
    q = p[o]
    # consecutive points are close (random order: mean step ~0.52)
    assert np.hypot(*(q[1:] - q[:-1]).T).mean() < 0.15
    # the four quadrants come in Z order: (0,0), (1,0), (0,1), (1,1)
    quad = (q[:, 0] >= 0.5).astype(int) + 2 * (q[:, 1] >= 0.5).astype(int)
    assert np.all(np.diff(quad) >= 0)


def test_spatial_order_of_a_grid_is_exact_morton():
    c = (np.arange(4) + 0.5) / 4
    xx, yy = np.meshgrid(c, c, indexing="xy")
    p = np.stack([xx.ravel(), yy.ravel()], 1)
    o = scenes.spatial_order(p, bits=2)
    # cell (i, j) of the 4 x 4 grid -> Morton key with x bits in even positions
    ij = [(int(p[k, 0] * 4), int(p[k, 1] * 4)) for k in o]
    keys = [sum(((i >> b) & 1) << (2 * b) | ((j >> b) & 1) << (2 * b + 1) for b in range(2))
            for i, j in ij]
    assert keys == sorted(keys) and len(set(keys)) == 16


def test_scene_batch3_layout():
    b = scenes.scene_batch3(6, 3, segments_range=(2, 5), rx_range=(10, 20), orders=(0, 2), n_tx=2)
    assert b.n_scenes == 6 and b.tx0.shape == (6, 2, 3)
    assert b.wall_off[0] == 0 and b.wall_off[-1] == b.tris.shape[0]
    assert b.rx_off[0] == 0 and b.rx_off[-1] == b.rx.shape[0]
    n_tris = np.diff(b.wall_off)
    # 2 triangles per wall (the square's 4 and the segments) plus floor and ceiling
    assert np.all((n_tris - 4) % 2 == 0) and np.all((n_tris - 4) // 2 - 4 >= 2)
    assert set(b.max_order.tolist()) <= {0, 2}
    assert b.tris.dtype == np.float32 and b.rx.dtype == np.float32
    sc = b.scene(4, 1)
    assert sc.n_tris == n_tris[4] and np.array_equal(sc.tx, b.tx0[4, 1])
    assert np.all((b.rx[:, 2] >= 0.1) & (b.rx[:, 2] <= 0.9))
    # seeded: the same arguments give the same batch
    c = scenes.scene_batch3(6, 3, segments_range=(2, 5), rx_range=(10, 20), orders=(0, 2), n_tx=2)
    assert np.array_equal(b.tris, c.tris) and np.array_equal(b.tx0, c.tx0)
