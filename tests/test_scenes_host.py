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
