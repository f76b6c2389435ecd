"""Pins of the oracle's smoothing functions (Sec. IV) to what the paper fixes."""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SMOOTH = ("sigmoid", "hard_sigmoid")


def _read(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


@pytest.mark.parametrize("alpha", [0.5, 1.0, 7.0, 100.0])
def test_fig2_printed_values(oracle_mod, alpha):
    # Fig. 2: the sigmoid reaches e/(e+1) at 1/alpha; the hard sigmoid reaches 1 at 3/alpha.
    for fn, ax, val in _read("fig2_smoothing.txt"):
        s, _ = oracle_mod.smooth(float(ax) / alpha, alpha, fn)
        assert s == pytest.approx(float(val), abs=1e-15)
    assert oracle_mod.smooth(1.0 / alpha, alpha, "sigmoid")[0] == pytest.approx(
        math.e / (math.e + 1.0), abs=1e-15)
    for ax, printed, tol in _read("fig2_marker_rounded.txt"):
        s, _ = oracle_mod.smooth(float(ax) / alpha, alpha, "sigmoid")
        assert abs(s - float(printed)) <= float(tol)


@pytest.mark.parametrize("fn", SMOOTH)
@pytest.mark.parametrize("alpha", [0.3, 1.0, 50.0, 1000.0])
def test_properties_c1_to_c4(oracle_mod, fn, alpha):
    xs = np.linspace(-10.0 / alpha, 10.0 / alpha, 401)
    s = np.array([oracle_mod.smooth(x, alpha, fn)[0] for x in xs])
    # range [0, 1]
    assert s.min() >= 0.0 and s.max() <= 1.0
    # C1: limits at -inf / +inf
    assert oracle_mod.smooth(-1e6 / alpha, alpha, fn)[0] == pytest.approx(0.0, abs=1e-12)
    assert oracle_mod.smooth(1e6 / alpha, alpha, fn)[0] == pytest.approx(1.0, abs=1e-12)
    # C2: monotonically increasing
    assert np.all(np.diff(s) >= 0.0)
    # C3: s(0) = 1/2
    assert oracle_mod.smooth(0.0, alpha, fn)[0] == 0.5
    # C4: s(x) - s(0) = s(0) - s(-x)
    s_neg = np.array([oracle_mod.smooth(-x, alpha, fn)[0] for x in xs])
    np.testing.assert_allclose(s - 0.5, 0.5 - s_neg, atol=1e-15)


@pytest.mark.parametrize("fn", SMOOTH)
def test_scaling_parametrisation(oracle_mod, fn):
    # Eq. 3: s(x; alpha) = s(alpha x; 1)
    for alpha in (0.25, 3.0, 80.0):
        for x in (-0.7, -0.01, 0.004, 0.3):
            assert oracle_mod.smooth(x, alpha, fn)[0] == pytest.approx(
                oracle_mod.smooth(alpha * x, 1.0, fn)[0], abs=1e-15)


@pytest.mark.parametrize("fn", SMOOTH)
def test_limit_is_unit_step(oracle_mod, fn):
    # Eq. 2: s(x; alpha) -> theta(x) as alpha -> infinity, for x != 0 (Eq. 1: theta(0) = 0).
    for x in (-1e-3, -1e-6, 1e-6, 1e-3):
        theta = 1.0 if x > 0 else 0.0
        assert oracle_mod.smooth(x, 1e12, fn)[0] == pytest.approx(theta, abs=1e-12)
        assert oracle_mod.smooth(x, 1e12, "step")[0] == theta
    assert oracle_mod.smooth(0.0, 1.0, "step")[0] == 0.0


def test_sigmoid_closed_form_and_derivative(oracle_mod):
    # Eq. 4 and its derivative alpha s (1 - s).
    for alpha in (1.0, 30.0):
        for x in (-0.2, -0.01, 0.0, 0.05, 0.3):
            s, ds = oracle_mod.smooth(x, alpha, "sigmoid")
            ref = 1.0 / (1.0 + math.exp(-alpha * x))
            assert s == pytest.approx(ref, rel=1e-14)
            assert ds == pytest.approx(alpha * ref * (1.0 - ref), rel=1e-12)


def test_hard_sigmoid_kinks(oracle_mod):
    # Eqs. 5-6: slope alpha/6 on (-3/alpha, 3/alpha), 0 outside; the derivative is
    # not continuous at +-3/alpha, where the oracle takes 0.
    alpha = 12.0
    for x in (-0.2, -0.1, -0.01, 0.0, 0.05, 0.2):
        s, ds = oracle_mod.smooth(x, alpha, "hard_sigmoid")
        z = alpha * x + 3.0
        assert s == pytest.approx(min(max(z, 0.0), 6.0) / 6.0, abs=1e-15)
        inside = -3.0 / alpha < x < 3.0 / alpha
        assert ds == (alpha / 6.0 if inside else 0.0)
    assert oracle_mod.smooth(3.0 / alpha, alpha, "hard_sigmoid")[1] == 0.0
    assert oracle_mod.smooth(-3.0 / alpha, alpha, "hard_sigmoid")[1] == 0.0


def test_alpha_zero_is_half(oracle_mod):
    for fn in SMOOTH:
        for x in (-5.0, 0.0, 3.0):
            assert oracle_mod.smooth(x, 0.0, fn)[0] == 0.5
