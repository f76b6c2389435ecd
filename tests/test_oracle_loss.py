"""Pins of the oracle's loss (Eq. 8 and Sec. III): L = -min_r P_r, with ties
going to the lowest receiver index (reading R7).

Hand-worked vectors fix the sign, the tie rule and the degenerate shapes; a
scene whose powers have a closed form (line of sight only, nothing in the way:
P = 1/d^2) fixes that the loss is taken over the oracle's own powers and lands
on the receiver farthest from the transmitter.  A dropped minus sign, a max
instead of a min, or a tie going to the last index fails one of these."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("P, L, i", [
    ([3.0, 1.0, 2.0], -1.0, 1),             # sign: the loss is the negated minimum
    ([0.5], -0.5, 0),                       # a single receiver
    ([2.0, 2.0, 2.0, 2.0], -2.0, 0),        # all equal: the first index
    ([4.0, 1.0, 7.0, 1.0, 1.0], -1.0, 1),   # ties inside: the lowest index of the minimum
    ([1e-30, 5.0, 1e-30], -1e-30, 0),       # tiny powers keep their value
    ([0.0, 0.0, 3.0], -0.0, 0),             # a fully shadowed receiver has loss 0
    ([9.0, 8.0, 7.0, 6.0], -6.0, 3),        # the minimum at the end
])
def test_hand_worked_vectors(P, L, i):
    got_L, got_i = oracle.loss(np.array(P))
    assert got_i == i
    assert got_L == L


def test_integer_and_float32_inputs_give_the_same_loss():
    assert oracle.loss([5, 2, 2]) == (-2.0, 1)
    assert oracle.loss(np.array([5, 2, 2], np.float32)) == (-2.0, 1)


def test_loss_of_a_clear_scene_is_the_farthest_receiver():
    """Line of sight only (K = 0), one wall far outside the receivers' region and
    the hard sigmoid at alpha = 100 (so every smoothed test saturates): each
    receiver gets exactly 1/d^2 (Eq. 7 with no reflection), the minimum is the
    farthest receiver, and of two receivers at that distance the lower index wins."""
    walls = np.array([[10.0, 10.0, 10.5, 10.0]])
    tx = np.array([0.5, 0.5])
    rx = np.array([[0.6, 0.5], [0.5, 0.9], [0.1, 0.5], [0.9, 0.5], [0.5, 0.1], [0.45, 0.55]])
    P = oracle.power(walls, tx, rx, 0, 100.0, "hard_sigmoid")
    d2 = ((rx - tx) ** 2).sum(1)
    np.testing.assert_allclose(P, 1.0 / d2, rtol=1e-14)
    L, i = oracle.loss(P)
    # receivers 1, 2, 3 and 4 are all 0.4 away: the tie goes to receiver 1
    assert i == 1
    assert L == pytest.approx(-1.0 / 0.16, rel=1e-14)
    # moving receiver 1 inwards hands the minimum to the next farthest in index order
    rx2 = rx.copy()
    rx2[1] = [0.5, 0.8]
    L2, i2 = oracle.loss(oracle.power(walls, tx, rx2, 0, 100.0, "hard_sigmoid"))
    assert i2 == 2 and L2 == pytest.approx(-1.0 / 0.16, rel=1e-14)
