"""The convergence check of the iterative path finders (Sec. V-B) on image-method paths.

Sec. V-B: every path finder checks convergence with the Min-Path-Tracing cost,
which vanishes exactly on a valid path.  These tests pin that cost (``oracle.mpt``)
by closed forms and show what it evaluates to on the image-method paths of the
oracle: zero when both neighbours of every reflection point lie on the same side
of its wall (where the Fermat minimiser over the walls' lines gives the same
points), and exactly 4 for each reflection whose neighbours lie on opposite
sides.  A smoothed check s(eps - C) on these paths is therefore a step in the
same-side test, which the path's validity already carries as the smooth product
s(p) s(q) + s(-p) s(-q).
"""
import numpy as np
import pytest

from classical_rt import fermat_points
from oracle import mpt
from paper_2401_11882_gb300 import scenes


def test_cost_closed_forms():
    wall = np.array([[0.0, 0.0, 1.0, 0.0]])            # the x axis, normal +y
    tx = np.array([0.1, 0.4])
    # mirror reflection at the image-method point: cost 0
    rx = np.array([0.9, 0.2])
    x = 0.1 + 0.8 * 0.4 / 0.6                           # where TX's image (0.1, -0.4) sees RX
    assert mpt.cost(wall, (0,), [x], tx, rx) == pytest.approx(0.0, abs=1e-30)
    # any other point: |o - r|^2 = 2 - 2 cos(angle between o and the mirrored i)
    for xo in (0.2, 0.5, 0.8):
        i = np.array([xo, 0.0]) - tx
        o = rx - np.array([xo, 0.0])
        r = np.array([i[0], -i[1]]) / np.hypot(*i)
        o = o / np.hypot(*o)
        assert mpt.cost(wall, (0,), [xo], tx, rx) == pytest.approx(2.0 - 2.0 * (o @ r), rel=1e-12)
    # straight crossing to the other side: i = o, so C = 4 (i . n)^2
    rx2 = np.array([0.7, -0.3])
    xc = 0.1 + 0.6 * 0.4 / 0.7
    i = (rx2 - tx) / np.hypot(*(rx2 - tx))
    assert mpt.cost(wall, (0,), [xc], tx, rx2) == pytest.approx(4.0 * i[1] ** 2, rel=1e-12)


def _same_side(walls, seq, verts):
    a, _, n = mpt._frames(walls, seq)
    return [np.dot(n[j], verts[j] - a[j]) * np.dot(n[j], verts[j + 2] - a[j]) > 0
            for j in range(len(seq))]


def test_cost_on_image_method_paths(oracle_mod):
    sc = scenes.large_scene(alpha=100.0, smoothing="step")
    walls = np.asarray(sc.walls, np.float64)[:10]
    tx = np.asarray(sc.tx, np.float64)
    rng = np.random.default_rng(11)
    seen = {0: 0, 1: 0, 2: 0}
    fermat_checked = 0
    for rx in rng.uniform(0.05, 0.95, (6, 2)):
        d = oracle_mod.paths(walls, tx, rx, 2, 100.0, "step")
        for c in range(1, d["seq"].shape[0]):
            k = int(d["order"][c])
            if d["degenerate"][c]:
                continue
            seq = tuple(int(w) for w in d["seq"][c][:k])
            v = d["verts"][c]
            same = _same_side(walls, seq, v)
            n = mpt._frames(walls, seq)[2]
            if any(abs(np.dot(n[j], v[j + 1] - v[j])) < 1e-9 for j in range(k)):
                continue                      # a leg grazing its wall: the sides are undecided
            C = mpt.cost(walls, seq, mpt.tau_of(walls, seq, v[1:k + 1]), tx, rx)
            bad = same.count(False)
            seen[bad] += 1
            assert C == pytest.approx(4.0 * bad, abs=1e-12), (seq, same, C)
            if bad == 0 and fermat_checked < 40:
                pts, _ = fermat_points(walls, tx, rx, seq)
                np.testing.assert_allclose(np.array(pts[1:k + 1]), v[1:k + 1], atol=1e-7)
                fermat_checked += 1
    assert min(seen.values()) > 10 and fermat_checked == 40
