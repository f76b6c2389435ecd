"""Pins of the oracle's coherent field (Eq. 7 as a sum of complex path fields).

Closed forms (free-space line of sight, the two-ray ground reflection with the
Fresnel coefficient, its limits), the hard limit against classical ray tracing
by brute force (Fermat points, exact predicates; ``classical_rt.classical_field``),
and reciprocity."""
import numpy as np
import pytest

from classical_rt import classical_field
from test_oracle_bruteforce import CASES, _scene

GAMMA = 0.5


def _E(o, walls, tx, rx, K, alpha, fn, lam, eps):
    return o.field(walls, tx, np.atleast_2d(rx), K, alpha, fn, lam, eps, GAMMA)


def _fresnel_te(c, eps):
    # textbook form with the angle of incidence theta from the normal
    st = np.sqrt(1.0 - c * c)
    return (c - np.sqrt(eps - st * st)) / (c + np.sqrt(eps - st * st))


def test_line_of_sight_is_a_spherical_wave(oracle_mod):
    walls = np.array([[0.1, 0.9, 0.3, 0.95]])            # far from the direct path
    tx = np.array([0.2, 0.1])
    rx = np.array([[0.7, 0.3], [0.8, 0.2], [0.5, 0.4]])
    d = np.hypot(*(rx - tx).T)
    for lam in (0.05, 0.013, 1.7):
        for fn, alpha in (("step", 1.0), ("hard_sigmoid", 100.0), ("sigmoid", 1e4)):
            E = _E(oracle_mod, walls, tx, rx, 0, alpha, fn, lam, 5.0)
            np.testing.assert_allclose(E, np.exp(-2j * np.pi * d / lam) / d, rtol=1e-13)
            np.testing.assert_allclose(np.abs(E) ** 2, 1.0 / d ** 2, rtol=1e-13)
    E, mag, lmax = oracle_mod.field(walls, tx, rx, 0, 1.0, "step", 0.05, 5.0, GAMMA, scales=True)
    np.testing.assert_allclose(mag, 1.0 / d, rtol=1e-13)
    np.testing.assert_allclose(lmax, d, rtol=1e-13)


@pytest.mark.parametrize("eps", [2.0, 15.0, 81.0])
def test_two_ray_ground_reflection(oracle_mod, eps):
    # The classic two-ray model over a flat ground: direct ray plus one ray reflected
    # with the Fresnel coefficient at grazing angle set by the antenna heights.
    ground = np.array([[-50.0, 0.0, 50.0, 0.0]])
    ht, hr, lam = 0.3, 0.2, 0.01
    tx = np.array([0.0, ht])
    xs = np.array([0.15, 0.4, 0.9, 2.5])
    rx = np.stack([xs, np.full_like(xs, hr)], 1)
    d0 = np.hypot(xs, ht - hr)
    d1 = np.hypot(xs, ht + hr)
    gam = _fresnel_te((ht + hr) / d1, eps)
    ref = np.exp(-2j * np.pi * d0 / lam) / d0 + gam * np.exp(-2j * np.pi * d1 / lam) / d1
    E = _E(oracle_mod, ground, tx, rx, 1, 1.0, "step", lam, eps)
    np.testing.assert_allclose(E, ref, rtol=1e-12)
    assert np.all(gam < 0) and np.all(gam > -1)


def test_fresnel_limits(oracle_mod):
    ground = np.array([[-5.0, 0.0, 5.0, 0.0]])
    tx, lam = np.array([0.0, 1.0]), 0.07
    # eps = 1: the wall is free space, nothing reflects
    rx = np.array([[0.6, 0.5]])
    d0 = np.hypot(0.6, 0.5)
    E = _E(oracle_mod, ground, tx, rx, 1, 1.0, "step", lam, 1.0)
    np.testing.assert_allclose(E, np.exp(-2j * np.pi * d0 / lam) / d0, rtol=1e-13)
    # normal incidence: (1 - sqrt(eps)) / (1 + sqrt(eps)); the image is 3 away
    rx = np.array([[0.0, 2.0]])
    for eps in (4.0, 9.0):
        g = (1.0 - np.sqrt(eps)) / (1.0 + np.sqrt(eps))
        E = _E(oracle_mod, ground, tx, rx, 1, 1.0, "step", lam, eps)
        ref = np.exp(-2j * np.pi / lam) + g * np.exp(-2j * np.pi * 3.0 / lam) / 3.0
        np.testing.assert_allclose(E, ref, rtol=1e-13)
    # grazing incidence: the coefficient tends to -1
    rx = np.array([[4000.0, 1.0]])
    ground = np.array([[-1.0, 0.0, 5000.0, 0.0]])
    E0 = _E(oracle_mod, ground, tx, rx, 0, 1.0, "step", lam, 9.0)
    E1 = _E(oracle_mod, ground, tx, rx, 1, 1.0, "step", lam, 9.0) - E0
    d1 = np.hypot(4000.0, 2.0)
    assert (E1 * d1 * np.exp(2j * np.pi * d1 / lam))[0].real == pytest.approx(-1.0, abs=2e-3)
    # the constant coefficient: -sqrt(Gamma), so the reflected power is Gamma / L^2
    E1 = _E(oracle_mod, ground, tx, rx, 1, 1.0, "step", lam, 0.0) - E0
    assert (E1 * d1 * np.exp(2j * np.pi * d1 / lam))[0] == pytest.approx(-np.sqrt(GAMMA), rel=1e-9)


@pytest.mark.parametrize("seed,W,K", CASES)
@pytest.mark.parametrize("eps", [0.0, 6.0])
def test_step_mode_equals_classical_ray_tracing(oracle_mod, seed, W, K, eps):
    walls, tx, rx = _scene(seed, W, 5)
    lam = 0.031
    E_step = _E(oracle_mod, walls, tx, rx, K, 1.0, "step", lam, eps)
    E_hard = _E(oracle_mod, walls, tx, rx, K, 1e9, "hard_sigmoid", lam, eps)
    n_paths = 0
    for r in range(rx.shape[0]):
        ref, margin = classical_field(walls, tx, rx[r], K, lam, eps, GAMMA)
        assert margin > 1e-6
        assert abs(E_step[r] - ref) <= 1e-9 * max(abs(ref), 1e-300)
        assert E_hard[r] == E_step[r]
        n_paths += ref != 0
    assert n_paths >= 1


@pytest.mark.parametrize("eps", [0.0, 3.0])
def test_reciprocity_in_the_hard_limit(oracle_mod, eps):
    walls, tx, rx = _scene(3, 4, 6)
    for r in range(rx.shape[0]):
        a = _E(oracle_mod, walls, tx, rx[r], 2, 1.0, "step", 0.02, eps)[0]
        b = _E(oracle_mod, walls, rx[r], tx, 2, 1.0, "step", 0.02, eps)[0]
        assert abs(a - b) <= 1e-12 * max(abs(a), 1e-300)


def _two_ray_power_cs(tx, ground_y, rx, lam, eps):
    """|E|^2 of the two-ray model as a real-analytic expression of (tx, ground height),
    so complex-step differentiation applies (no abs, no conjugate)."""
    ht, hr = tx[1] - ground_y, rx[1] - ground_y
    dx = rx[0] - tx[0]
    d0 = np.sqrt(dx * dx + (ht - hr) ** 2)
    d1 = np.sqrt(dx * dx + (ht + hr) ** 2)
    c = (ht + hr) / d1
    root = np.sqrt(eps - 1.0 + c * c)
    gam = (c - root) / (c + root)
    k = 2 * np.pi / lam
    re = np.cos(k * d0) / d0 + gam * np.cos(k * d1) / d1
    im = -np.sin(k * d0) / d0 - gam * np.sin(k * d1) / d1
    return re * re + im * im


@pytest.mark.parametrize("eps", [2.0, 15.0])
def test_field_gradient_of_the_two_ray_model(oracle_mod, eps):
    # d|E|^2 / d(TX x, TX y, ground height) against complex-step derivatives of the
    # closed form (an independent expression of the same model)
    tx = np.array([0.1, 0.3])
    rx = np.array([[0.9, 0.25]])
    lam, gy = 0.05, 0.0
    ground = np.array([[-50.0, gy, 50.0, gy]])
    g = np.array([1.0])
    # parameters: TX x, TX y, and the wall's two y coordinates (flat indices 2 + 1, 2 + 3)
    got = oracle_mod.field_gradient(ground, tx, rx, 1, 1.0, "step", lam, eps, g, [0, 1, 3, 5],
                                    GAMMA)
    h = 1e-30
    ref_tx = [_two_ray_power_cs(tx + 1j * h * e, gy, rx[0], lam, eps).imag / h
              for e in np.eye(2)]
    ref_gy = _two_ray_power_cs(tx, gy + 1j * h, rx[0], lam, eps).imag / h
    np.testing.assert_allclose(got[:2], ref_tx, rtol=1e-9)
    assert got[2] + got[3] == pytest.approx(ref_gy, rel=1e-9)


@pytest.mark.parametrize("fn,alpha", [("sigmoid", 30.0), ("hard_sigmoid", 40.0)])
@pytest.mark.parametrize("eps", [0.0, 4.0])
def test_field_jvp_equals_central_differences(oracle_mod, fn, alpha, eps):
    walls, tx, rx = _scene(8, 4, 3)
    lam = 0.06
    rng = np.random.default_rng(1)
    for _ in range(3):
        dw = rng.normal(size=walls.shape)
        dtx = rng.normal(size=2)
        E, dE = oracle_mod.field_jvp(walls, tx, rx, 2, alpha, fn, lam, eps, dw, dtx, GAMMA)
        h = 1e-6
        Ep = oracle_mod.field(walls + h * dw, tx + h * dtx, rx, 2, alpha, fn, lam, eps, GAMMA)
        Em = oracle_mod.field(walls - h * dw, tx - h * dtx, rx, 2, alpha, fn, lam, eps, GAMMA)
        fd = (Ep - Em) / (2 * h)
        np.testing.assert_allclose(dE, fd, rtol=2e-5, atol=2e-5 * np.abs(fd).max())
