"""FP64 Min-Path-Tracing cost of Sec. V-B ("Continuous Path Finding") for reflections
on the infinite lines through the walls.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``): the tests use it
to show what the convergence check of the iterative path finders evaluates to on
the image-method paths; nothing in the CUDA library calls it.

Sec. V-B: the image method (IM), the Fermat-principle minimisation of the path
length (FPT) and Min-Path-Tracing (MPT) all check convergence with the MPT cost,
which is zero exactly on a valid path, the comparison with zero being smoothed
by s.  The paper gives no formula; this module reads the cost for reflections as

    C = sum_j | o_j - (i_j - 2 (i_j . n_j) n_j) |^2

with i_j, o_j the unit directions of the legs into and out of reflection point
X_j and n_j the unit normal of its wall: zero iff the reflection law holds at
every point.  Points are parametrised along their walls' lines,
X_j = A_j + tau_j u_j, so the cost's "point on the object" term is zero by
construction.
"""
from __future__ import annotations

import numpy as np


def _frames(walls, seq):
    w = np.asarray(walls, dtype=np.float64).reshape(-1, 4)[list(seq)]
    a = w[:, :2]
    e = w[:, 2:] - a
    u = e / np.hypot(e[:, 0], e[:, 1])[:, None]
    n = np.stack([-u[:, 1], u[:, 0]], 1)
    return a, u, n


def tau_of(walls, seq, xs) -> np.ndarray:
    """Along-wall coordinates of points ``xs`` [k, 2] that lie on the walls' lines."""
    a, u, _ = _frames(walls, seq)
    return np.einsum("ij,ij->i", np.asarray(xs, np.float64).reshape(-1, 2) - a, u)


def points(walls, seq, tau, tx, rx) -> np.ndarray:
    """Vertices [TX, X_1 .. X_k, RX] for along-wall coordinates ``tau``."""
    a, u, _ = _frames(walls, seq)
    x = a + np.asarray(tau, dtype=np.float64)[:, None] * u
    return np.vstack([np.asarray(tx, np.float64)[None], x, np.asarray(rx, np.float64)[None]])


def residuals(walls, seq, tau, tx, rx) -> np.ndarray:
    """[2k] residuals o_j - reflect(i_j) of the reflection law, one pair per point."""
    _, _, n = _frames(walls, seq)
    d = np.diff(points(walls, seq, tau, tx, rx), axis=0)
    dh = d / np.hypot(d[:, 0], d[:, 1])[:, None]
    r = [dh[j + 1] - (dh[j] - 2.0 * np.dot(dh[j], n[j]) * n[j]) for j in range(len(seq))]
    return np.concatenate(r) if r else np.zeros(0)


def cost(walls, seq, tau, tx, rx) -> float:
    """The MPT cost C (zero iff the reflection law holds at every point)."""
    r = residuals(walls, seq, tau, tx, rx)
    return float(np.dot(r, r))
