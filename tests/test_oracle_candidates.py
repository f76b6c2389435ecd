"""Pins of the candidate list (Sec. V: every wall sequence allowed by the visibility
matrix, here all pairs except a wall with itself)."""
import itertools

import numpy as np
import pytest


@pytest.mark.parametrize("W,K,n", [(5, 1, 6), (64, 2, 4097), (128, 2, 16385), (4, 3, 1 + 4 + 12 + 36),
                                   (7, 0, 1)])
def test_candidate_counts(oracle_mod, W, K, n):
    assert oracle_mod.num_candidates(W, K) == n


@pytest.mark.parametrize("W,K", [(3, 2), (4, 3), (5, 2)])
def test_candidate_table_is_the_lexicographic_list(oracle_mod, W, K):
    seq, order = oracle_mod.candidates(W, K)
    ref = [()]
    for k in range(1, K + 1):
        ref += [s for s in itertools.product(range(W), repeat=k)
                if all(s[i] != s[i + 1] for i in range(k - 1))]
    got = [tuple(int(w) for w in row[:o]) for row, o in zip(seq, order)]
    assert got == ref
    assert np.all(seq[np.arange(K)[None, :] >= order[:, None]] == -1)
