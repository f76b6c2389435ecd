"""Pins of the oracle's 3D extension (Sec. VI: the method for triangle walls).

Closed forms (free-space LOS, blocking, a ground reflection, alpha = 0), the 2D
oracle reproduced exactly by extruded scenes in the hard limit, classical 3D ray
tracing by brute force on arbitrary triangles (``classical_rt3``), invariance
under rigid motions, and reciprocity."""
import itertools

import numpy as np
import pytest

from classical_rt3 import classical_power3
from test_oracle_bruteforce import CASES, _scene

GAMMA = 0.5


def _P3(o, tris, tx, rx, K, alpha, fn):
    return o.power3(tris, tx, np.atleast_2d(rx), K, alpha, fn, GAMMA)


def _extrude(walls2d, h=5.0):
    """Each 2D wall becomes a vertical rectangle z in [-h, h] made of two triangles."""
    tris = []
    for x0, y0, x1, y1 in np.asarray(walls2d, np.float64):
        a, b = np.array([x0, y0, -h]), np.array([x1, y1, -h])
        c, d = np.array([x1, y1, h]), np.array([x0, y0, h])
        tris.append(np.concatenate([a, b, c]))
        tris.append(np.concatenate([a, c, d]))
    return np.array(tris)


def test_line_of_sight_clear_and_blocked(oracle_mod):
    far = np.array([[5.0, 5.0, 5.0, 6.0, 5.0, 5.0, 5.0, 6.0, 5.0]])
    tx = np.array([0.1, 0.2, 0.3])
    rx = np.array([[0.7, 0.1, -0.2], [0.4, 0.9, 0.5]])
    d2 = ((rx - tx) ** 2).sum(1)
    for fn, alpha in (("step", 1.0), ("hard_sigmoid", 100.0), ("sigmoid", 1e4)):
        np.testing.assert_allclose(_P3(oracle_mod, far, tx, rx, 0, alpha, fn), 1.0 / d2,
                                   rtol=1e-14)
    # a large triangle in the plane x = 0.5 between TX and RX blocks the direct path
    wall = np.array([[0.5, -10.0, -10.0, 0.5, 10.0, -10.0, 0.5, 0.0, 10.0]])
    tx, rx = np.array([0.0, 0.0, 0.0]), np.array([[1.0, 0.1, 0.2]])
    for fn, alpha in (("step", 1.0), ("hard_sigmoid", 100.0)):
        assert _P3(oracle_mod, wall, tx, rx, 0, alpha, fn)[0] == 0.0


def test_ground_reflection(oracle_mod):
    ground = np.array([[-50.0, -50.0, 0.0, 50.0, -50.0, 0.0, 0.0, 50.0, 0.0]])
    tx = np.array([0.0, 0.0, 1.0])
    rx = np.array([[2.0, 0.5, 0.5], [1.0, -1.0, 2.0]])
    d0 = ((rx - tx) ** 2).sum(1)
    img = np.array([0.0, 0.0, -1.0])
    d1 = ((rx - img) ** 2).sum(1)
    for fn, alpha in (("step", 1.0), ("hard_sigmoid", 100.0)):
        P = _P3(oracle_mod, ground, tx, rx, 1, alpha, fn)
        np.testing.assert_allclose(P, 1.0 / d0 + GAMMA / d1, rtol=1e-13)


@pytest.mark.parametrize("seed,W,K", CASES)
def test_extruded_scenes_equal_the_2d_oracle_in_the_hard_limit(oracle_mod, seed, W, K):
    # a 2D scene extruded into tall vertical walls, TX and RX in the plane z = 0:
    # every path stays in that plane, so the 3D power is the 2D power (the extra
    # sequences over the two triangles of one wall are degenerate or invalid)
    walls, tx, rx = _scene(seed, W, 5)
    P2 = oracle_mod.power(walls, tx, rx, K, 1.0, "step", GAMMA)
    tris = _extrude(walls)
    tx3 = np.array([tx[0], tx[1], 0.0])
    rx3 = np.concatenate([rx, np.zeros((rx.shape[0], 1))], 1)
    P3 = _P3(oracle_mod, tris, tx3, rx3, K, 1.0, "step")
    np.testing.assert_allclose(P3, P2, rtol=1e-9, atol=1e-300)
    np.testing.assert_array_equal(_P3(oracle_mod, tris, tx3, rx3, K, 1e9, "hard_sigmoid"), P3)
    assert np.count_nonzero(P2) >= 1


def _random_tris(rng, n):
    centre = rng.uniform(-1, 1, (n, 1, 3))
    return (centre + rng.uniform(-0.6, 0.6, (n, 3, 3))).reshape(n, 9)


def _rotation(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q *= np.sign(np.diag(r))
    return q if np.linalg.det(q) > 0 else -q


@pytest.mark.parametrize("fn,alpha", [("sigmoid", 30.0), ("hard_sigmoid", 50.0)])
def test_rigid_motion_invariance(oracle_mod, fn, alpha):
    rng = np.random.default_rng(3)
    tris = _random_tris(rng, 5)
    tx = rng.uniform(-1, 1, 3)
    rx = rng.uniform(-1, 1, (6, 3))
    P = _P3(oracle_mod, tris, tx, rx, 2, alpha, fn)
    Rm, t = _rotation(rng), rng.normal(size=3)
    mv = lambda p: p.reshape(-1, 3) @ Rm.T + t
    P_mv = _P3(oracle_mod, mv(tris).reshape(-1, 9), mv(tx)[0], mv(rx), 2, alpha, fn)
    np.testing.assert_allclose(P_mv, P, rtol=1e-10)
    assert np.all(P > 0)


def test_reciprocity(oracle_mod):
    rng = np.random.default_rng(4)
    tris = _random_tris(rng, 4)
    a, b = rng.uniform(-1, 1, 3), rng.uniform(-1, 1, 3)
    for fn, alpha in (("sigmoid", 20.0), ("hard_sigmoid", 40.0), ("step", 1.0)):
        pa = _P3(oracle_mod, tris, a, b, 2, alpha, fn)[0]
        pb = _P3(oracle_mod, tris, b, a, 2, alpha, fn)[0]
        assert pa == pytest.approx(pb, rel=1e-12)


def _mirror(p, tri):
    a, b, c = tri.reshape(3, 3)
    n = np.cross(b - a, c - a)
    n /= np.linalg.norm(n)
    return p - 2.0 * np.dot(p - a, n) * n


def _backtrace_length(tx, rx, seq, tris):
    """Sum of the leg lengths of the image-method path, each reflection point found as
    a line-plane intersection (parametric solve), independently of the oracle."""
    imgs = [tx]
    for w in seq:
        imgs.append(_mirror(imgs[-1], tris[w]))
    pts = [rx]
    for j in range(len(seq), 0, -1):
        a, b, c = tris[seq[j - 1]].reshape(3, 3)
        n = np.cross(b - a, c - a)
        q, i = pts[-1], imgs[j]
        s = np.dot(a - q, n) / np.dot(i - q, n)
        pts.append(q + s * (i - q))
    pts.append(tx)
    return sum(np.linalg.norm(pts[i + 1] - pts[i]) for i in range(len(pts) - 1))


def test_alpha_zero_closed_form(oracle_mod):
    # alpha = 0: every s = 1/2, so a reflection's validity is (1/8)(1/2) = 1/16 and each
    # tested (leg, triangle) pair passes 1 - (1/2)(1/8) = 15/16; L is the sum of the legs
    # (|I_k - RX| only on paths whose reflections are valid)
    rng = np.random.default_rng(5)
    W = 4
    tris = _random_tris(rng, W)
    tx = rng.uniform(-1, 1, 3)
    rx = rng.uniform(-1, 1, (3, 3))
    for K in (0, 1, 2):
        P = _P3(oracle_mod, tris, tx, rx, K, 0.0, "sigmoid")
        ref = np.zeros(rx.shape[0])
        for k in range(K + 1):
            for seq in itertools.product(range(W), repeat=k):
                if any(seq[i] == seq[i + 1] for i in range(k - 1)):
                    continue
                L = np.array([_backtrace_length(tx, r, seq, tris) for r in rx])
                tests = (k + 1) * W - 2 * k
                ref += GAMMA ** k * 16.0 ** -k * (15.0 / 16.0) ** tests / L ** 2
        np.testing.assert_allclose(P, ref, rtol=1e-12)


def test_two_triangles_of_one_mirror_reflect_once(oracle_mod):
    # a square mirror made of two triangles: a path cannot reflect on it twice in a
    # row (the leg between the two reflections has zero length), so K = 2 adds nothing
    # to K = 1, even with the reflection point on the shared diagonal, where the
    # smoothed on-object tests of both triangles are 1/2
    sq = np.array([[-1.0, -1.0, 0.0, 1.0, -1.0, 0.0, 1.0, 1.0, 0.0],
                   [-1.0, -1.0, 0.0, 1.0, 1.0, 0.0, -1.0, 1.0, 0.0]])
    tx = np.array([0.3, 0.3, 1.0])
    rx = np.array([[-0.3, -0.3, 1.0], [-0.2, -0.25, 0.7]])
    for fn, alpha in (("hard_sigmoid", 10.0), ("sigmoid", 10.0)):
        P1 = _P3(oracle_mod, sq, tx, rx, 1, alpha, fn)
        P2 = _P3(oracle_mod, sq, tx, rx, 2, alpha, fn)
        np.testing.assert_array_equal(P2, P1)
    # on the diagonal the two halves' on-object tests add up to one (C4), and neither
    # half blocks a leg that starts or ends on the other (same plane)
    d1 = np.sum((rx[0] - np.array([0.3, 0.3, -1.0])) ** 2)
    P = _P3(oracle_mod, sq, tx, rx[:1], 1, 10.0, "hard_sigmoid")[0]
    d0 = np.sum((rx[0] - tx) ** 2)
    assert P == pytest.approx(1.0 / d0 + GAMMA / d1, rel=1e-12)


def test_3d_gradient_closed_form_ground_reflection(oracle_mod):
    # d/dTX of 1/|RX - TX|^2 + Gamma/|RX - TX'|^2, TX' the image of TX in z = 0
    ground = np.array([[-50.0, -50.0, 0.0, 50.0, -50.0, 0.0, 0.0, 50.0, 0.0]])
    tx = np.array([0.2, -0.1, 1.0])
    rx = np.array([[2.0, 0.5, 0.5], [1.0, -1.0, 2.0]])
    g = np.array([0.7, -1.3])
    got = oracle_mod.gradient3_tx(ground, tx, rx, 1, 1.0, "step", g, GAMMA)
    ref = np.zeros(3)
    for r, gr in zip(rx, g):
        d = r - tx
        ref += gr * 2.0 * d / np.dot(d, d) ** 2
        img = tx * np.array([1.0, 1.0, -1.0])
        e = r - img
        ref += gr * GAMMA * 2.0 * e * np.array([1.0, 1.0, -1.0]) / np.dot(e, e) ** 2
    np.testing.assert_allclose(got, ref, rtol=1e-12)


def test_3d_corner_derivative_closed_form_ground_height(oracle_mod):
    # raising the ground plane z = h (all corners of its triangle) moves TX's image
    # (tx, ty, 2h - tz): d/dh Gamma / |RX - I|^2 = 4 Gamma (rz - Iz) / |RX - I|^4, and the
    # line of sight does not move; per corner the derivatives must add up to it
    h = 0.15
    ground = np.array([[-50.0, -50.0, h, 50.0, -50.0, h, 0.0, 50.0, h]])
    tx = np.array([0.2, -0.1, 1.0])
    rx = np.array([[2.0, 0.5, 0.5], [1.0, -1.0, 2.0]])
    g = np.array([0.7, -1.3])
    gtx, gtris = oracle_mod.gradient3(ground, tx, rx, 1, 1.0, "step", g, GAMMA)
    img = np.array([tx[0], tx[1], 2 * h - tx[2]])
    ref = sum(gr * 4 * GAMMA * (r[2] - img[2]) / np.dot(r - img, r - img) ** 2
              for r, gr in zip(rx, g))
    assert gtris[0, [2, 5, 8]].sum() == pytest.approx(ref, rel=1e-12)
    # in-plane moves of the corners change nothing while the reflection point stays inside
    np.testing.assert_allclose(gtris[0, [0, 1, 3, 4, 6, 7]], 0.0, atol=1e-12)
    np.testing.assert_allclose(gtx, oracle_mod.gradient3_tx(ground, tx, rx, 1, 1.0, "step", g,
                                                            GAMMA), rtol=1e-14)


@pytest.mark.parametrize("fn,alpha", [("sigmoid", 25.0), ("hard_sigmoid", 40.0)])
def test_3d_jvp_equals_central_differences(oracle_mod, fn, alpha):
    rng = np.random.default_rng(6)
    tris = _random_tris(rng, 4)
    tx = rng.uniform(-1, 1, 3)
    rx = rng.uniform(-1, 1, (4, 3))
    for _ in range(3):
        dw = rng.normal(size=tris.shape)
        dtx = rng.normal(size=3)
        _, dP = oracle_mod.power3_jvp(tris, tx, rx, 2, alpha, fn, dw, dtx, GAMMA)
        h = 1e-6
        Pp = _P3(oracle_mod, tris + h * dw, tx + h * dtx, rx, 2, alpha, fn)
        Pm = _P3(oracle_mod, tris - h * dw, tx - h * dtx, rx, 2, alpha, fn)
        np.testing.assert_allclose(dP, (Pp - Pm) / (2 * h), rtol=1e-5,
                                   atol=1e-5 * np.abs(dP).max())


@pytest.mark.parametrize("seed,W,K", [(1, 4, 1), (2, 3, 2), (3, 4, 2), (4, 5, 1), (5, 3, 2)])
def test_step_mode_equals_classical_3d_ray_tracing(oracle_mod, seed, W, K):
    # arbitrary triangles: reflection points by Fermat minimisation over the planes,
    # exact barycentric and segment-triangle predicates (no image method, no smoothing)
    rng = np.random.default_rng(100 + seed)
    tris = _random_tris(rng, W)
    tx = rng.uniform(-1, 1, 3)
    rx = rng.uniform(-1, 1, (4, 3))
    P = _P3(oracle_mod, tris, tx, rx, K, 1.0, "step")
    P0 = _P3(oracle_mod, tris, tx, rx, 0, 1.0, "step")
    for r in range(rx.shape[0]):
        ref, margin = classical_power3(tris, tx, rx[r], K, GAMMA)
        assert margin > 1e-6, "a predicate sits on a tie; pick another seed"
        assert P[r] == pytest.approx(ref, rel=1e-9, abs=1e-300)
    assert np.any(P > P0)   # some reflection path is valid and unblocked
