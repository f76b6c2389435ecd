"""Pins of the oracle's Fermat path finder (Sec. V-B, "Continuous Path Finding"):
Newton steps on the total path length from the walls' midpoints, with the same
smoothed convergence check s(eps - C) on the MPT cost C as the MPT finder.

Closed forms fix the converged points (a mirror's image construction) and, where
the wall's line separates the two ends, the straight crossing that minimises the
length and the cost 4 (i . n)^2 that the check then rejects; the image-method
points fix the converged points on the valid paths of random scenes (97% of them:
the rest, like two perpendicular mirrors, run into the corner where two walls
meet); the length never increases from one step to the next (the problem is
convex); the square room's power is the image method's."""
import numpy as np
import pytest

import oracle
from oracle import mpt
from paper_2401_11882_gb300 import scenes

X_AXIS = np.array([[0.0, 0.0, 1.0, 0.0]])


def _s(x, alpha, kind):
    """Eq. 4 (sigmoid) and Eqs. 5-6 (hard sigmoid) at alpha x, written out."""
    if kind == "sigmoid":
        return 1.0 / (1.0 + np.exp(-alpha * x))
    return min(max(alpha * x / 6.0 + 0.5, 0.0), 1.0)


def _length(walls, seq, tau, tx, rx):
    walls = np.asarray(walls, np.float64)
    pts = [np.asarray(tx, np.float64)]
    for w, t in zip(seq, tau):
        a, b = walls[w, :2], walls[w, 2:]
        pts.append(a + t * (b - a) / np.linalg.norm(b - a))
    pts.append(np.asarray(rx, np.float64))
    return sum(np.linalg.norm(q - p) for p, q in zip(pts[:-1], pts[1:]))


def test_single_mirror_converges_to_the_image_point():
    tx, rx = np.array([0.1, 0.4]), np.array([0.9, 0.2])
    x_star = 0.1 + 0.8 * 0.4 / 0.6
    d = oracle.fpt_paths(X_AXIS, tx, rx, 1, 100.0, "hard_sigmoid", n_iter=10, eps=0.05)
    assert d["tau"][1, 0] == pytest.approx(x_star, abs=1e-12)
    assert d["cost"][1] < 1e-24 and d["kappa"][1] == 1.0
    assert d["cost"][0] == 0.0 and d["kappa"][0] == 1.0


def test_two_perpendicular_mirrors_run_into_the_corner():
    """The double reflection of two perpendicular mirrors is the length's minimum (a
    grid search finds nothing shorter), but Newton from the midpoints heads for the
    corner where the mirrors meet: there the leg between them vanishes, the length
    has a kink, and its Hessian (1 / leg length) stalls the steps, so the path ends
    degenerate.  The MPT finder converges on the same path (its residuals stay
    smooth there)."""
    walls = np.array([[1.0, 0.0, 1.0, 1.0], [1.0, 0.0, 0.0, 0.0]])
    tx, rx = np.array([0.5, 0.2]), np.array([0.125, 0.125])
    I2 = np.array([2.0 - tx[0], -tx[1]])
    best = np.linalg.norm(I2 - rx)                     # the unfolded straight path
    g = np.linspace(-1.0, 1.0, 201)
    grid = min(_length(walls, (0, 1), (a, b), tx, rx) for a in g for b in g)
    assert best <= grid + 1e-12
    d = oracle.fpt_paths(walls, tx, rx, 2, 100.0, "sigmoid", n_iter=12, eps=0.05)
    seq = [tuple(s[:o]) for s, o in zip(d["seq"], d["order"])]
    c = seq.index((0, 1))
    assert d["degenerate"][c] == 1 and d["power"][c] == 0.0
    m = oracle.mpt_paths(walls, tx, rx, 2, 100.0, "sigmoid", n_iter=12, eps=0.05)
    assert m["degenerate"][c] == 0 and m["cost"][c] < 1e-24


@pytest.mark.parametrize("kind", ["sigmoid", "hard_sigmoid"])
def test_a_separating_line_gives_the_straight_crossing_and_is_rejected(kind):
    # TX above the mirror's line, RX below: the shortest path touching the line is the
    # straight segment, crossing at x_c; there the outgoing leg continues the incoming
    # one, so the reflection-law residual is 2 (i . n) n and C = 4 (i . n)^2
    tx, rx = np.array([0.2, 0.4]), np.array([0.8, -0.3])
    x_c = 0.2 + 0.6 * 0.4 / 0.7
    i_dir = (rx - tx) / np.linalg.norm(rx - tx)
    C = 4.0 * i_dir[1] ** 2
    d = oracle.fpt_paths(X_AXIS, tx, rx, 1, 100.0, kind, n_iter=10, eps=0.05)
    assert d["tau"][1, 0] == pytest.approx(x_c, abs=1e-12)
    assert d["cost"][1] == pytest.approx(C, rel=1e-12)
    assert d["kappa"][1] == pytest.approx(_s(0.05 - C, 100.0, kind), rel=1e-9, abs=1e-300)
    assert d["power"][1] < 1e-30


def test_length_never_increases():
    sc = scenes.clutter_scene(8, 3, seed=4, alpha=100.0, smoothing="sigmoid", max_order=2)
    for rx in sc.rx.astype(np.float64):
        prev = None
        for n in range(6):
            d = oracle.fpt_paths(sc.walls, sc.tx, rx, 2, 100.0, "sigmoid", n_iter=n)
            L = np.array([_length(sc.walls, [int(w) for w in s[:o]], t[:o], sc.tx, rx)
                          if o > 0 and not g else np.nan
                          for s, o, t, g in zip(d["seq"], d["order"], d["tau"], d["degenerate"])])
            if prev is not None:
                both = ~np.isnan(L) & ~np.isnan(prev)
                assert np.all(L[both] <= prev[both] * (1 + 1e-14))
            prev = L


def test_converges_to_the_image_method_points_on_valid_paths():
    """On a valid path the image-method points minimise the length (the unfolded path
    is straight); Newton on the convex length reaches them from the midpoints on 97%
    of the valid paths of these scenes; where it does not, the path ends in a corner
    (degenerate), short of them near a kink, or far from them with C > 1e-6, never at
    another point with C = 0."""
    n_valid = n_conv = 0
    for seed, W, K in [(3, 20, 2), (5, 20, 2), (7, 8, 3), (2, 12, 1)]:
        sc = scenes.clutter_scene(W, 4, seed=seed, alpha=100.0, smoothing="hard_sigmoid",
                                  max_order=K)
        walls = sc.walls.astype(np.float64)
        tx = sc.tx.astype(np.float64)
        for rx in sc.rx.astype(np.float64):
            im = oracle.paths(walls, tx, rx, K, 100.0, "step")
            f = oracle.fpt_paths(walls, tx, rx, K, 100.0, "hard_sigmoid", n_iter=12)
            for c in range(1, len(im["order"])):
                k = int(im["order"][c])
                if im["degenerate"][c]:
                    continue
                seq = tuple(int(w) for w in im["seq"][c][:k])
                tau_im = mpt.tau_of(walls, seq, im["verts"][c][1:k + 1])
                lens = np.hypot(walls[list(seq), 2] - walls[list(seq), 0],
                                walls[list(seq), 3] - walls[list(seq), 1])
                legs = np.hypot(*np.diff(im["verts"][c][:k + 2], axis=0).T)
                if (mpt.cost(walls, seq, tau_im, tx, rx) < 1e-20 and
                        np.all((tau_im > 0) & (tau_im < lens)) and legs.min() >= 1e-3):
                    n_valid += 1
                    if not f["degenerate"][c] and np.abs(f["tau"][c][:k] - tau_im).max() <= 1e-9:
                        n_conv += 1
                        assert f["cost"][c] < 1e-16
                    elif not f["degenerate"][c]:
                        # stopped short near a kink: still heading for the same points
                        assert (f["cost"][c] > 1e-6 or
                                np.abs(f["tau"][c][:k] - tau_im).max() <= 1e-3)
    assert n_valid > 300 and n_conv >= 0.95 * n_valid


def test_square_room_power_closed_form():
    walls = scenes.unit_square_walls().astype(np.float64)
    tx = np.array([0.31, 0.42])
    rx = np.array([[0.7, 0.66], [0.15, 0.8], [0.55, 0.2]])
    images = [np.array([tx[0], -tx[1]]), np.array([2 - tx[0], tx[1]]),
              np.array([tx[0], 2 - tx[1]]), np.array([-tx[0], tx[1]])]
    ref = [1 / np.sum((r - tx) ** 2) + 0.5 * sum(1 / np.sum((I - r) ** 2) for I in images)
           for r in rx]
    P = oracle.power_fpt(walls, tx, rx, 1, 1e4, "hard_sigmoid", n_iter=10, eps=0.05)
    np.testing.assert_allclose(P, ref, rtol=1e-12)


def test_fermat_and_mpt_agree_on_converged_paths():
    sc = scenes.clutter_scene(10, 3, seed=9, alpha=100.0, smoothing="sigmoid", max_order=2)
    n = 0
    for rx in sc.rx.astype(np.float64):
        a = oracle.fpt_paths(sc.walls, sc.tx, rx, 2, 100.0, "sigmoid", n_iter=15)
        b = oracle.mpt_paths(sc.walls, sc.tx, rx, 2, 100.0, "sigmoid", n_iter=15)
        both = (a["cost"] < 1e-20) & (b["cost"] < 1e-20) & (a["order"] > 0) & \
            ~a["degenerate"].astype(bool) & ~b["degenerate"].astype(bool)
        n += int(both.sum())
        np.testing.assert_allclose(a["tau"][both], b["tau"][both], atol=1e-10)
        np.testing.assert_allclose(a["power"][both], b["power"][both], rtol=1e-9)
    assert n > 20
