"""Pins of the oracle's iterative path finder (Sec. V-B, "Continuous Path
Finding"): Min-Path-Tracing steps on the reflection law from the walls'
midpoints, and the smoothed convergence check s(eps - C) on its MPT cost C.

Closed forms fix the converged points (a mirror's image construction, two
perpendicular mirrors' double image), the cost of configurations that have no
reflection, and the square room's received power; the independent Python cost
(``oracle/mpt.py``, pinned in test_oracle_convergence_check.py) fixes C at the
finder's points; the oracle's image-method points fix the converged points on
every valid path of random scenes."""
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


def test_single_mirror_converges_to_the_image_point():
    tx, rx = np.array([0.1, 0.4]), np.array([0.9, 0.2])
    x_star = 0.1 + 0.8 * 0.4 / 0.6          # TX's image (0.1, -0.4) sees RX through it
    d = oracle.mpt_paths(X_AXIS, tx, rx, 1, 100.0, "hard_sigmoid", n_iter=10, eps=0.05)
    assert d["tau"][1, 0] == pytest.approx(x_star, abs=1e-12)
    assert d["cost"][1] < 1e-24
    # converged: the check passes (hard sigmoid: s(eps - 0) = 1 once eps >= 3 / alpha)
    assert d["kappa"][1] == 1.0
    # the line of sight (no reflection) has nothing to converge: C = 0
    assert d["cost"][0] == 0.0 and d["kappa"][0] == 1.0
    # quadratic convergence: one more step leaves the point where it is
    d2 = oracle.mpt_paths(X_AXIS, tx, rx, 1, 100.0, "hard_sigmoid", n_iter=11)
    assert d2["tau"][1, 0] == pytest.approx(d["tau"][1, 0], abs=1e-15)


def test_two_perpendicular_mirrors_converge_to_the_double_image():
    # walls on the lines x = 1 and y = 0 meeting at the corner (1, 0); TX -> wall 0 (x = 1)
    # -> wall 1 (y = 0) -> RX.  TX's image in x = 1, then in y = 0: (2 - tx_x, -tx_y); the
    # line from it to RX crosses y = 0 at X2 and the first image's line crosses x = 1 at X1.
    walls = np.array([[1.0, 0.0, 1.0, 1.0], [1.0, 0.0, 0.0, 0.0]])
    tx, rx = np.array([0.5, 0.2]), np.array([0.125, 0.125])
    I1 = np.array([2.0 - tx[0], tx[1]])
    I2 = np.array([I1[0], -I1[1]])
    t2 = rx[1] / (rx[1] - I2[1])
    X2 = rx + t2 * (I2 - rx)
    t1 = (1.0 - X2[0]) / (I1[0] - X2[0])
    X1 = X2 + t1 * (I1 - X2)
    d = oracle.mpt_paths(walls, tx, rx, 2, 100.0, "sigmoid", n_iter=12, eps=0.05)
    seq = [tuple(s[:o]) for s, o in zip(d["seq"], d["order"])]
    c = seq.index((0, 1))
    # along-wall coordinates: wall 0 runs up from (1, 0), wall 1 runs left from (1, 0)
    assert d["tau"][c, 0] == pytest.approx(X1[1], abs=1e-12)
    assert d["tau"][c, 1] == pytest.approx(1.0 - X2[0], abs=1e-12)
    assert d["cost"][c] < 1e-24
    assert d["kappa"][c] == pytest.approx(_s(0.05, 100.0, "sigmoid"), rel=1e-12)


def test_no_reflection_across_a_wall():
    # TX and RX on opposite sides of the mirror: the reflection law has no solution on
    # the line (a reflected ray returns to TX's side), so C stays far from 0 and the
    # smoothed check rejects the path
    tx, rx = np.array([0.2, 0.3]), np.array([0.8, -0.25])
    for kind in ("sigmoid", "hard_sigmoid"):
        d = oracle.mpt_paths(X_AXIS, tx, rx, 1, 100.0, kind, n_iter=20, eps=0.05)
        assert d["cost"][1] > 0.5
        assert d["kappa"][1] == pytest.approx(_s(0.05 - d["cost"][1], 100.0, kind), abs=1e-300)
        assert d["kappa"][1] < 1e-10 and d["power"][1] < 1e-10


def test_cost_agrees_with_the_independent_cost():
    rng = np.random.default_rng(4)
    sc = scenes.random_small_scene(rng, 6, 5, 3, 50.0, "sigmoid", boundary=True)
    for rx in sc.rx:
        d = oracle.mpt_paths(sc.walls, sc.tx, rx, 3, 50.0, "sigmoid", n_iter=3)
        for c in range(1, len(d["order"])):
            if d["degenerate"][c]:
                continue
            k = int(d["order"][c])
            seq = tuple(int(w) for w in d["seq"][c][:k])
            C = mpt.cost(sc.walls, seq, d["tau"][c][:k], sc.tx, rx)
            assert d["cost"][c] == pytest.approx(C, rel=1e-9, abs=1e-15)


def test_converges_to_the_image_method_points_on_valid_paths():
    """Gauss-Newton on the (nonconvex) MPT cost reaches the image-method points of
    nearly every valid path from the walls' midpoints; where it settles elsewhere the
    cost stays far from zero, so its convergence check rejects the path; and every
    point it reports as converged is the image-method point."""
    n_valid = n_conv = 0
    for seed, W, K in [(3, 20, 2), (5, 20, 2), (7, 8, 3), (9, 12, 2), (1, 6, 3), (2, 12, 1)]:
        sc = scenes.clutter_scene(W, 4, seed=seed, alpha=100.0, smoothing="hard_sigmoid",
                                  max_order=K)
        walls = sc.walls.astype(np.float64)
        tx = sc.tx.astype(np.float64)
        for rx in sc.rx.astype(np.float64):
            im = oracle.paths(walls, tx, rx, K, 100.0, "step")
            f = oracle.mpt_paths(walls, tx, rx, K, 100.0, "hard_sigmoid", n_iter=12)
            for c in range(1, len(im["order"])):
                k = int(im["order"][c])
                if im["degenerate"][c]:
                    continue
                seq = tuple(int(w) for w in im["seq"][c][:k])
                tau_im = mpt.tau_of(walls, seq, im["verts"][c][1:k + 1])
                if not f["degenerate"][c] and f["cost"][c] < 1e-20:
                    np.testing.assert_allclose(f["tau"][c][:k], tau_im, atol=1e-8)
                lens = np.hypot(walls[list(seq), 2] - walls[list(seq), 0],
                                walls[list(seq), 3] - walls[list(seq), 1])
                legs = np.hypot(*np.diff(im["verts"][c][:k + 2], axis=0).T)
                if (mpt.cost(walls, seq, tau_im, tx, rx) < 1e-20 and
                        np.all((tau_im > 0) & (tau_im < lens))):
                    n_valid += 1
                    # a leg shorter than 1e-3 makes the path degenerate by definition
                    assert bool(f["degenerate"][c]) == bool(legs.min() < 1e-3)
                    if f["degenerate"][c]:
                        continue
                    if np.abs(f["tau"][c][:k] - tau_im).max() <= 1e-10:
                        n_conv += 1
                        assert f["cost"][c] < 1e-18 and f["kappa"][c] == 1.0
                    else:
                        assert f["cost"][c] > 0.1 and f["kappa"][c] == 0.0
    assert n_valid > 400 and n_conv >= 0.98 * n_valid


def test_square_room_power_closed_form():
    # the unit square, an interior receiver, K <= 1: the line of sight and four valid
    # single reflections, P = 1/d0^2 + Gamma sum_i 1/|I_i - RX|^2 (hard sigmoid at a
    # sharpness where every smoothed value saturates), as for the image method
    walls = scenes.unit_square_walls().astype(np.float64)
    tx = np.array([0.31, 0.42])
    rx = np.array([[0.7, 0.66], [0.15, 0.8], [0.55, 0.2]])
    images = [np.array([tx[0], -tx[1]]), np.array([2 - tx[0], tx[1]]),
              np.array([tx[0], 2 - tx[1]]), np.array([-tx[0], tx[1]])]
    ref = [1 / np.sum((r - tx) ** 2) + 0.5 * sum(1 / np.sum((I - r) ** 2) for I in images)
           for r in rx]
    P = oracle.power_mpt(walls, tx, rx, 1, 1e4, "hard_sigmoid", n_iter=10, eps=0.05)
    np.testing.assert_allclose(P, ref, rtol=1e-12)


def test_check_replaces_the_same_side_test():
    # image-method power and MPT power agree path by path wherever the image-method
    # point is valid: there the same-side product and the check are both 1 (hard sigmoid,
    # every smoothed value saturated), elsewhere the MPT path is rejected by its check
    sc = scenes.clutter_scene(12, 3, seed=2, alpha=3e3, smoothing="hard_sigmoid", max_order=2)
    n = 0
    for rx in sc.rx.astype(np.float64):
        im = oracle.paths(sc.walls, sc.tx, rx, 2, 3e3, "hard_sigmoid")
        f = oracle.mpt_paths(sc.walls, sc.tx, rx, 2, 3e3, "hard_sigmoid", n_iter=12)
        ok = (f["kappa"] == 1.0) & (im["power"] > 0)
        n += int(ok.sum())
        np.testing.assert_allclose(f["power"][ok], im["power"][ok], rtol=1e-9)
        assert np.all(f["power"][f["kappa"] == 0.0] == 0.0)
    assert n > 40


def test_a_leg_shorter_than_the_limit_makes_the_path_degenerate():
    # a receiver h = 2e-4 above the mirror: the converged reflection point lies 4e-4 to
    # its left, so the last leg (sqrt(5) h) is shorter than 1e-3 and the path contributes
    # nothing; 2e-3 above the mirror it is an ordinary path
    tx = np.array([0.1, 0.4])
    for h, deg in ((2e-4, 1), (2e-3, 0)):
        rx = np.array([0.9, h])
        d = oracle.mpt_paths(X_AXIS, tx, rx, 1, 100.0, "hard_sigmoid", n_iter=12)
        assert d["degenerate"][1] == deg
        if deg:
            assert d["power"][1] == 0.0 and d["kappa"][1] == 0.0 and np.isnan(d["tau"][1, 0])
        else:
            assert d["tau"][1, 0] == pytest.approx(0.1 + 0.8 * 0.4 / (0.4 + h), abs=1e-10)
