"""Hard-limit pins: the oracle's step mode, and the smoothed modes at very large alpha,
must reproduce classical 0/1 ray tracing computed by brute force (Eq. 2: the
smoothing tends to the unit step as alpha grows)."""
import numpy as np
import pytest

from classical_rt import classical_power

GAMMA = 0.5


def _scene(seed, W, R):
    rng = np.random.default_rng(seed)
    mid = rng.uniform(0.15, 0.85, (W, 2))
    ang = rng.uniform(0, np.pi, W)
    ln = rng.uniform(0.15, 0.5, W)
    h = 0.5 * ln[:, None] * np.stack([np.cos(ang), np.sin(ang)], 1)
    walls = np.concatenate([mid - h, mid + h], 1)
    tx = rng.uniform(0.1, 0.9, 2)
    rx = rng.uniform(0.05, 0.95, (R, 2))
    return walls, tx, rx


CASES = [(seed, W, K) for seed, W, K in [(0, 3, 1), (1, 4, 1), (2, 3, 2), (3, 4, 2), (4, 2, 2),
                                          (5, 4, 2)]]


@pytest.mark.parametrize("seed,W,K", CASES)
def test_step_mode_equals_classical_ray_tracing(oracle_mod, seed, W, K):
    walls, tx, rx = _scene(seed, W, 5)
    P_step = oracle_mod.power(walls, tx, rx, K, 1.0, "step", GAMMA)
    P_hard = oracle_mod.power(walls, tx, rx, K, 1e9, "hard_sigmoid", GAMMA)
    P_sig = oracle_mod.power(walls, tx, rx, K, 1e9, "sigmoid", GAMMA)
    n_nonzero = 0
    for r in range(rx.shape[0]):
        ref, margin = classical_power(walls, tx, rx[r], K, GAMMA)
        assert margin > 1e-6, "a predicate sits on a tie; pick another seed"
        assert P_step[r] == pytest.approx(ref, rel=1e-9, abs=1e-300)
        # |x| > 3/alpha for every argument: the hard sigmoid is exactly 0 or 1 (Eqs. 5-6)
        assert P_hard[r] == P_step[r]
        assert P_sig[r] == pytest.approx(P_step[r], rel=1e-12, abs=1e-300)
        n_nonzero += ref > 0
    assert n_nonzero >= 1


def test_bruteforce_sees_blocking_and_reflections(oracle_mod):
    # Sanity of the fixture itself: a scene where a wall blocks LOS but a reflection gets through.
    walls = np.array([[0.45, 0.2, 0.45, 0.8], [0.0, 0.0, 1.0, 0.0]])
    tx, rx = np.array([0.2, 0.5]), np.array([0.8, 0.5])
    ref, margin = classical_power(walls, tx, rx, 1, GAMMA)
    assert margin > 1e-3
    # LOS is blocked; the floor reflection at (0.5, 0) passes below the wall's lower tip:
    # its first leg crosses x = 0.45 at y = 0.083 < 0.2.
    img = np.array([0.2, -0.5])
    assert ref == pytest.approx(GAMMA / ((img - rx) ** 2).sum(), rel=1e-9)
    P = oracle_mod.power(walls, tx, rx[None], 1, 1.0, "step", GAMMA)
    assert P[0] == pytest.approx(ref, rel=1e-9)
