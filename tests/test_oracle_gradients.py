"""Pins of the oracle's derivatives (Sec. III: the loss gradient w.r.t. the scene
parameters) against closed forms, complex-step differentiation and finite differences."""
import numpy as np
import pytest

from classical_rt import mirror_point

GAMMA = 0.5


def _scene(seed, W=4, R=5):
    rng = np.random.default_rng(seed)
    mid = rng.uniform(0.15, 0.85, (W, 2))
    ang = rng.uniform(0, np.pi, W)
    ln = rng.uniform(0.15, 0.45, W)
    h = 0.5 * ln[:, None] * np.stack([np.cos(ang), np.sin(ang)], 1)
    return (np.concatenate([mid - h, mid + h], 1), rng.uniform(0.1, 0.9, 2),
            rng.uniform(0.05, 0.95, (R, 2)))


def _dirs(W, rng, n):
    for _ in range(n):
        yield rng.normal(size=(W, 4)), rng.normal(size=2)


@pytest.mark.parametrize("fn,alpha", [("sigmoid", 25.0), ("hard_sigmoid", 15.0)])
def test_dual_equals_complex_step(oracle_mod, fn, alpha):
    walls, tx, rx = _scene(0)
    rng = np.random.default_rng(1)
    for dw, dt in _dirs(walls.shape[0], rng, 3):
        _, jvp = oracle_mod.power_jvp(walls, tx, rx, 2, alpha, fn, dw, dt, GAMMA)
        cs = oracle_mod.power_cstep(walls, tx, rx, 2, alpha, fn, dw, dt, 1e-30, GAMMA)
        np.testing.assert_allclose(jvp, cs, rtol=1e-10, atol=1e-12 * np.abs(cs).max())


@pytest.mark.parametrize("fn,alpha", [("sigmoid", 5.0), ("sigmoid", 40.0)])
def test_dual_equals_central_differences(oracle_mod, fn, alpha):
    walls, tx, rx = _scene(2)
    rng = np.random.default_rng(3)
    h = 1e-6
    for dw, dt in _dirs(walls.shape[0], rng, 2):
        _, jvp = oracle_mod.power_jvp(walls, tx, rx, 2, alpha, fn, dw, dt, GAMMA)
        Pp = oracle_mod.power(walls + h * dw, tx + h * dt, rx, 2, alpha, fn, GAMMA)
        Pm = oracle_mod.power(walls - h * dw, tx - h * dt, rx, 2, alpha, fn, GAMMA)
        fd = (Pp - Pm) / (2 * h)
        np.testing.assert_allclose(jvp, fd, rtol=2e-5, atol=1e-7 * np.abs(fd).max())


def test_los_gradient_closed_form(oracle_mod):
    # P = 1/|TX - RX|^2 in a clear scene: dP/dTX = -2 (TX - RX) / |TX - RX|^4.
    walls = np.array([[0.0, 0.95, 0.2, 0.99]])
    tx = np.array([0.3, 0.2])
    rx = np.array([[0.7, 0.6], [0.2, 0.7]])
    for r in rx:
        g = oracle_mod.gradient(walls, tx, r[None], 0, 100.0, "hard_sigmoid", [1.0], "tx", GAMMA)
        d = tx - r
        np.testing.assert_allclose(g, -2 * d / (d @ d) ** 2, rtol=1e-13)


def test_single_reflection_gradient_closed_form(oracle_mod):
    # With LOS blocked, P = Gamma / |M(TX) - RX|^2.  dP/dTX = -2 Gamma H (I1 - RX)/|I1 - RX|^4,
    # H = I - 2 n n^T.  Translating the wall along its normal by eps moves the image by
    # 2 eps n; sliding it along itself changes nothing.
    walls = np.array([[0.0, 0.0, 1.0, 0.0],          # floor reflector
                      [0.5, 0.15, 0.5, 0.9]])        # blocks the direct path
    tx, rx = np.array([0.2, 0.5]), np.array([0.8, 0.45])
    P = oracle_mod.power(walls, tx, rx[None], 1, 1e3, "hard_sigmoid", GAMMA)[0]
    img = mirror_point(tx, walls[0, :2], walls[0, 2:])
    assert P == pytest.approx(GAMMA / ((img - rx) ** 2).sum(), rel=1e-13)
    n = np.array([0.0, 1.0])
    H = np.eye(2) - 2 * np.outer(n, n)
    d = img - rx
    g = oracle_mod.gradient(walls, tx, rx[None], 1, 1e3, "hard_sigmoid", [1.0], "all", GAMMA)
    np.testing.assert_allclose(g[:2], -2 * GAMMA * H @ d / (d @ d) ** 2, rtol=1e-12)
    gw = g[2:].reshape(2, 4)
    normal_shift = gw[0, 1] + gw[0, 3]                 # d/deps of (y0 + eps, y1 + eps)
    assert normal_shift == pytest.approx(-2 * GAMMA * (d @ (2 * n)) / (d @ d) ** 2, rel=1e-12)
    assert gw[0, 0] + gw[0, 2] == pytest.approx(0.0, abs=1e-12)   # slide along the wall
    np.testing.assert_allclose(gw[1], 0.0, atol=1e-12)            # the blocker is saturated


def test_tiny_scene_gradient_symmetry(oracle_mod):
    from paper_2401_11882_gb300 import scenes
    sc = scenes.tiny_scene()
    walls = sc.walls.astype(np.float64)
    rx = np.array([[0.5, 0.8], [0.5, 0.35], [0.3, 0.7], [0.7, 0.7]])
    for fn in ("sigmoid", "hard_sigmoid"):
        gx = [oracle_mod.gradient(walls, sc.tx, r[None], 1, 100.0, fn, [1.0], "tx", GAMMA)
              for r in rx]
        assert gx[0][0] == pytest.approx(0.0, abs=1e-10 * abs(gx[0][1]) + 1e-300)
        assert gx[1][0] == pytest.approx(0.0, abs=1e-10 * abs(gx[1][1]) + 1e-300)
        assert gx[2][0] == pytest.approx(-gx[3][0], rel=1e-10)
        assert gx[2][1] == pytest.approx(gx[3][1], rel=1e-10)


def test_gradient_is_weighted_sum_of_jvps(oracle_mod):
    walls, tx, rx = _scene(4)
    g = np.array([0.3, 0.0, -1.2, 2.0, 0.5])
    idx = [0, 1, 2 + 5, 2 + 12]
    got = oracle_mod.gradient(walls, tx, rx, 2, 30.0, "sigmoid", g, idx, GAMMA)
    for n, p in enumerate(idx):
        dw, dt = np.zeros(walls.size), np.zeros(2)
        if p < 2:
            dt[p] = 1.0
        else:
            dw[p - 2] = 1.0
        _, dP = oracle_mod.power_jvp(walls, tx, rx, 2, 30.0, "sigmoid", dw, dt, GAMMA)
        assert got[n] == pytest.approx(g @ dP, rel=1e-13)
