"""Classical (unsmoothed) 3D ray tracing by brute force, for pinning the 3D oracle.

Written independently of the oracle: the reflection points of a triangle
sequence minimise the total path length over the triangles' planes (Fermat's
principle; convex in the points' plane coordinates), not the image method; a
point is on a triangle when its barycentric coordinates are all positive; a leg
is blocked when its end points lie strictly on opposite sides of a triangle's
plane and the crossing point is strictly inside the triangle.  A path counts
when every reflection point is inside its triangle, the neighbouring vertices
lie strictly on the same side of its plane, and no leg is blocked by a
triangle other than the ones its end points lie on.  Power: Gamma^k / L^2 per
path.  ``margin`` is the smallest predicate value met on the valid paths, so a
test can check that no decision sat on a tie.
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy.optimize import minimize


def _frame(tri):
    a, b, c = np.asarray(tri, np.float64).reshape(3, 3)
    return a, b - a, c - a


def _signed_dist(tri, p):
    a, e1, e2 = _frame(tri)
    n = np.cross(e1, e2)
    return np.dot(p - a, n) / np.linalg.norm(n)


def _barycentric(tri, p):
    """(u, v, w) with p = w A + u B + v C for a point p of the triangle's plane."""
    a, e1, e2 = _frame(tri)
    G = np.array([[e1 @ e1, e1 @ e2], [e1 @ e2, e2 @ e2]])
    u, v = np.linalg.solve(G, np.array([e1 @ (p - a), e2 @ (p - a)]))
    return np.array([u, v, 1.0 - u - v])


def fermat_points3(tris, tx, rx, seq):
    k = len(seq)
    frames = [_frame(tris[w]) for w in seq]

    def pts(z):
        out = [tx]
        for j, (a, e1, e2) in enumerate(frames):
            out.append(a + z[2 * j] * e1 + z[2 * j + 1] * e2)
        out.append(rx)
        return out

    def f(z):
        P = pts(z)
        legs = [P[j + 1] - P[j] for j in range(k + 1)]
        lens = [np.linalg.norm(v) for v in legs]
        dirs = [v / n if n > 0 else np.zeros(3) for v, n in zip(legs, lens)]
        g = np.zeros(2 * k)
        for j, (a, e1, e2) in enumerate(frames):
            d = dirs[j] - dirs[j + 1]
            g[2 * j] = e1 @ d
            g[2 * j + 1] = e2 @ d
        return sum(lens), g

    best = None
    for z0 in (0.33, 0.1, 0.6):
        r = minimize(f, np.full(2 * k, z0), jac=True, method="BFGS",
                     options={"gtol": 1e-13, "maxiter": 4000})
        if best is None or r.fun < best.fun:
            best = r
    return pts(best.x)


def classical_power3(tris, tx, rx, max_order, gamma=0.5):
    """(P, min_margin) for one receiver of a triangle scene [W, 9]."""
    tris = np.asarray(tris, np.float64).reshape(-1, 9)
    tx = np.asarray(tx, np.float64)
    rx = np.asarray(rx, np.float64)
    W = tris.shape[0]
    total, margin = 0.0, np.inf
    for k in range(max_order + 1):
        for seq in itertools.product(range(W), repeat=k):
            if any(seq[i] == seq[i + 1] for i in range(k - 1)):
                continue
            P = fermat_points3(tris, tx, rx, seq) if k else [tx, rx]
            ok, m = True, np.inf
            for j in range(1, k + 1):
                tri = tris[seq[j - 1]]
                bc = _barycentric(tri, P[j])
                m = min(m, np.abs(bc).min())
                sp, sq = _signed_dist(tri, P[j - 1]), _signed_dist(tri, P[j + 1])
                m = min(m, abs(sp), abs(sq))
                if not (bc.min() > 0 and sp * sq > 0):
                    ok = False
            if not ok:
                # no specular path for this sequence: a valid image-method path would be
                # the unique length minimiser, so the oracle's path is invalid as well
                continue
            for j in range(k + 1):
                skip = set()
                if j >= 1:
                    skip.add(seq[j - 1])
                if j + 1 <= k:
                    skip.add(seq[j])
                for w in range(W):
                    if w in skip:
                        continue
                    x, y = _signed_dist(tris[w], P[j]), _signed_dist(tris[w], P[j + 1])
                    m = min(m, abs(x), abs(y))
                    if x * y < 0:
                        hit = P[j] + (x / (x - y)) * (P[j + 1] - P[j])
                        bc = _barycentric(tris[w], hit)
                        m = min(m, np.abs(bc).min())
                        if bc.min() > 0:
                            ok = False
            margin = min(margin, m)
            if ok:
                L = sum(np.linalg.norm(P[j + 1] - P[j]) for j in range(k + 1))
                total += gamma ** k / L ** 2
    return total, margin
