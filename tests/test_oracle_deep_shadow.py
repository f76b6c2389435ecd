"""Pins of the oracle's sigmoid obstruction factor where a wall all but blocks a leg
(Sec. V-A with the sigmoid of Eq. 4 at large alpha): the factor 1 - X1 X2 (2D) or
1 - X in (3D) is then far below the rounding of 1, and only a cancellation-free
evaluation keeps its value.  The expected values are the same definitions
evaluated with 60 significant digits (mpmath), on line-of-sight paths blocked by
one wall or one triangle, so that the received power is the factor over L^2."""
import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

mp.mp.dps = 60


def _s(z, alpha):
    """Eq. 4 at alpha z, 60 digits."""
    return 1 / (1 + mp.exp(-alpha * mp.mpf(z)))


def _X(x, y, alpha):
    """x and y on opposite sides: s(x) s(-y) + s(-x) s(y)."""
    return _s(x, alpha) * _s(-y, alpha) + _s(-x, alpha) * _s(y, alpha)


@pytest.mark.parametrize("alpha", [20.0, 100.0, 150.0, 200.0])
def test_2d_wall_blocking_the_line_of_sight(oracle_mod, alpha):
    # wall x = 0.5 from y = -0.5 to 0.5; TX (0.2, 0), RX (0.8, 0): the leg crosses the
    # wall's line 0.3 from both end points and the wall's end points lie 0.5 off the
    # leg's line on either side
    walls = np.array([[0.5, -0.5, 0.5, 0.5]])
    tx, rx = np.array([0.2, 0.0]), np.array([[0.8, 0.0]])
    f = 1 - _X(mp.mpf("0.3"), mp.mpf("-0.3"), alpha) * _X(mp.mpf("-0.5"), mp.mpf("0.5"), alpha)
    want = float(f / mp.mpf("0.36"))
    got = oracle_mod.power(walls, tx, rx, 0, alpha, "sigmoid")[0]
    assert got == pytest.approx(want, rel=1e-12, abs=0.0)
    assert want > 0.0


def _edge_dist(P, a, b, c):
    """Signed in-plane distance of P to the edge line a-b, positive on c's side."""
    ab = [b[i] - a[i] for i in range(3)]
    ap = [P[i] - a[i] for i in range(3)]
    ac = [c[i] - a[i] for i in range(3)]
    l2 = sum(v * v for v in ab)
    # the component of AP (and AC) orthogonal to AB, in the plane
    kp = sum(ap[i] * ab[i] for i in range(3)) / l2
    kc = sum(ac[i] * ab[i] for i in range(3)) / l2
    op = [ap[i] - kp * ab[i] for i in range(3)]
    oc = [ac[i] - kc * ab[i] for i in range(3)]
    norm_oc = mp.sqrt(sum(v * v for v in oc))
    return sum(op[i] * oc[i] for i in range(3)) / norm_oc


@pytest.mark.parametrize("alpha", [20.0, 100.0, 150.0, 200.0])
def test_3d_triangle_blocking_the_line_of_sight(oracle_mod, alpha):
    # triangle in the plane x = 0.5 around the point (0.5, 0, 0) where the leg from
    # TX (0.2, 0, 0) to RX (0.8, 0, 0) crosses it
    corners = [mp.matrix([0.5, -1.0, -1.0]), mp.matrix([0.5, 1.0, -1.0]),
               mp.matrix([0.5, 0.0, 1.0])]
    tris = np.array([[0.5, -1.0, -1.0, 0.5, 1.0, -1.0, 0.5, 0.0, 1.0]])
    tx, rx = np.array([0.2, 0.0, 0.0]), np.array([[0.8, 0.0, 0.0]])
    hit = mp.matrix([0.5, 0.0, 0.0])
    inside = mp.mpf(1)
    for k in range(3):
        a, b, c = corners[k], corners[(k + 1) % 3], corners[(k + 2) % 3]
        inside *= _s(_edge_dist(hit, a, b, c), alpha)
    f = 1 - _X(mp.mpf("-0.3"), mp.mpf("0.3"), alpha) * inside
    want = float(f / mp.mpf("0.36"))
    got = oracle_mod.power3(tris, tx, rx, 0, alpha, "sigmoid")[0]
    assert got == pytest.approx(want, rel=1e-12, abs=0.0)
    assert want > 0.0
