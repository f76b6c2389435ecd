"""Host-side parts of the surrogate search (no GPU): the target transform, the
grid's local minima and the greedy separated selection of proposals."""
import numpy as np

from paper_2401_11882_gb300.surrogate import grid_local_minima, separated_minima, target_of


def test_target_is_decreasing_in_F_and_finite_at_zero():
    F = np.array([0.0, 1e-9, 1e-3, 0.5, 2.0])
    t = target_of(F)
    assert np.all(np.isfinite(t)) and np.all(np.diff(t) < 0)
    np.testing.assert_allclose(t[-1], -np.log(2.0 + 1e-12))


def test_grid_local_minima_finds_the_wells_of_a_known_function():
    n = 64
    c = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(c, c, indexing="xy")
    # two wells and a shallow bowl, each centred on a grid point
    w1, w2, b = (c[16], c[16]), (c[48], c[38]), (c[32], c[32])
    f = (-np.exp(-((X - w1[0]) ** 2 + (Y - w1[1]) ** 2) / 0.005)
         - 0.8 * np.exp(-((X - w2[0]) ** 2 + (Y - w2[1]) ** 2) / 0.005)
         + 0.2 * ((X - b[0]) ** 2 + (Y - b[1]) ** 2))
    m = grid_local_minima(f)
    got = sorted(map(tuple, np.stack([X[m], Y[m]], 1).round(7)))
    assert got == sorted(tuple(np.round(p, 7)) for p in (w1, w2, b))
    # a constant grid: every point ties with its neighbours
    assert grid_local_minima(np.zeros((5, 7))).all()


def test_separated_minima_is_greedy_by_value_with_a_minimum_distance():
    rng = np.random.default_rng(0)
    pts = rng.uniform(0, 1, (400, 2))
    vals = rng.normal(size=400)
    out = separated_minima(pts, vals, 12, 0.1)
    assert out.shape == (12, 2)
    d = np.hypot(*(out[:, None, :] - out[None, :, :]).transpose(2, 0, 1))
    assert np.all(d[np.triu_indices(12, 1)] >= 0.1)
    # the first choice is the global minimum; every later one is the best point
    # far enough from the earlier choices
    order = np.argsort(vals, kind="stable")
    assert np.array_equal(out[0], pts[order[0]])
    chosen = [out[0]]
    for p in out[1:]:
        i = np.nonzero((pts == p).all(1))[0][0]
        better = [j for j in order[:np.nonzero(order == i)[0][0]]
                  if np.min(np.hypot(*(np.array(chosen) - pts[j]).T)) >= 0.1]
        assert not better
        chosen.append(p)
    # asking for more than fit returns what fits
    assert separated_minima(pts, vals, 10_000, 0.5).shape[0] < 30
