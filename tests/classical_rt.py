"""Classical (unsmoothed) 2D ray tracing by brute force, for pinning the oracle.

Written independently of the oracle: the reflection points of a wall
sequence come from minimising the total path length over the walls'
infinite lines (Fermat's principle, a convex problem), not from the image
method; validity and obstruction use exact orientation predicates (proper
segment intersection), not smoothing functions.  A path is counted when
every reflection point lies strictly inside its segment, the previous and
next vertices lie strictly on the same side of the reflecting line, and no
leg properly crosses a wall other than the ones its end points lie on.

Its power model is the same reading as the oracle's: Gamma^k / L^2 per valid
path, summed over paths.  ``min_margin`` reports the smallest predicate
margin seen on the specular paths, so a test can check that no deciding
predicate sat on a tie.
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy.optimize import minimize


def _orient(a, b, p):
    """Signed distance of p from the line a->b (positive on the left)."""
    d = b - a
    return (d[0] * (p[1] - a[1]) - d[1] * (p[0] - a[0])) / np.hypot(d[0], d[1])


def sequences(n_walls, max_order):
    out = [()]
    for k in range(1, max_order + 1):
        for s in itertools.product(range(n_walls), repeat=k):
            if all(s[i] != s[i + 1] for i in range(k - 1)):
                out.append(s)
    return out


def fermat_points(walls, tx, rx, seq):
    """Minimise sum of leg lengths over points on the walls' lines."""
    k = len(seq)
    if k == 0:
        return [tx, rx], np.zeros(0)
    A = np.array([walls[w][:2] for w in seq])
    D = np.array([walls[w][2:] - walls[w][:2] for w in seq])

    def pts(t):
        return [tx] + [A[j] + t[j] * D[j] for j in range(k)] + [rx]

    def f(t):
        # a zero-length leg at a junction of two lines has no direction: give it none
        P = pts(t)
        legs = [P[j + 1] - P[j] for j in range(k + 1)]
        lens = [np.hypot(*v) for v in legs]
        dirs = [v / n if n > 0 else np.zeros(2) for v, n in zip(legs, lens)]
        g = np.zeros(k)
        for j in range(k):
            g[j] = D[j] @ (dirs[j] - dirs[j + 1])
        return sum(lens), g

    best = None
    for t0 in (np.full(k, 0.5), np.full(k, 0.1), np.full(k, 0.9)):
        r = minimize(f, t0, jac=True, method="BFGS", options={"gtol": 1e-14, "maxiter": 2000})
        if best is None or r.fun < best.fun:
            best = r
    return pts(best.x), best.x


def classical_paths(walls, tx, rx, max_order):
    """(paths, min_margin) for one receiver: every specular, unobstructed path as
    (wall sequence, vertices [TX, X_1 .. X_k, RX])."""
    walls = [np.asarray(w, dtype=np.float64) for w in walls]
    tx = np.asarray(tx, np.float64)
    rx = np.asarray(rx, np.float64)
    paths, margin = [], np.inf
    for seq in sequences(len(walls), max_order):
        k = len(seq)
        P, t = fermat_points(walls, tx, rx, seq)
        ok = True
        m = np.inf          # smallest margin among this path's predicates
        for j in range(1, k + 1):
            w = walls[seq[j - 1]]
            a, b = w[:2], w[2:]
            ell = np.hypot(*(b - a))
            along = t[j - 1] * ell
            m = min(m, abs(along), abs(ell - along))
            if not (0.0 < along < ell):
                ok = False
            sp, sq = _orient(a, b, P[j - 1]), _orient(a, b, P[j + 1])
            m = min(m, abs(sp), abs(sq))
            if not (sp * sq > 0):
                ok = False
        if not ok:
            # An invalid Fermat path cannot be a specular path, whatever its margins:
            # a valid image-method path would be the (unique) length minimiser.
            continue
        for j in range(k + 1):
            p0, p1 = P[j], P[j + 1]
            skip = set()
            if j >= 1:
                skip.add(seq[j - 1])
            if j + 1 <= k:
                skip.add(seq[j])
            for wi, w in enumerate(walls):
                if wi in skip:
                    continue
                a, b = w[:2], w[2:]
                o1, o2 = _orient(a, b, p0), _orient(a, b, p1)
                o3, o4 = _orient(p0, p1, a), _orient(p0, p1, b)
                m = min(m, abs(o1), abs(o2), abs(o3), abs(o4))
                if o1 * o2 < 0 and o3 * o4 < 0:
                    ok = False
        margin = min(margin, m)
        if ok:
            paths.append((seq, P))
    return paths, margin


def _length(P):
    return sum(np.hypot(*(P[j + 1] - P[j])) for j in range(len(P) - 1))


def classical_power(walls, tx, rx, max_order, gamma=0.5):
    """(P, min_margin) for one receiver."""
    paths, margin = classical_paths(walls, tx, rx, max_order)
    return sum(gamma ** len(seq) / _length(P) ** 2 for seq, P in paths), margin


def classical_field(walls, tx, rx, max_order, wavelength, eps_r, gamma=0.5):
    """(E, min_margin) for one receiver: the coherent sum over the specular paths of
    prod_j C_j exp(-2 pi i L / wavelength) / L, C_j the Fresnel coefficient for a field
    normal to the plane of incidence, from the angle between the incoming leg and the
    wall's normal (eps_r > 0), or -sqrt(gamma) (eps_r = 0)."""
    paths, margin = classical_paths(walls, tx, rx, max_order)
    E = 0j
    for seq, P in paths:
        coef = 1.0
        for j, w in enumerate(seq, start=1):
            if eps_r > 0:
                a, b = np.asarray(walls[w][:2], np.float64), np.asarray(walls[w][2:], np.float64)
                d = P[j] - P[j - 1]
                # cosine of incidence from the normal, via the 2D cross product
                e = b - a
                c = abs(e[0] * d[1] - e[1] * d[0]) / (np.hypot(*e) * np.hypot(*d))
                root = np.sqrt(eps_r - (1.0 - c * c))
                coef *= (c - root) / (c + root)
            else:
                coef *= -np.sqrt(gamma)
        L = _length(P)
        E += coef * np.exp(-2j * np.pi * L / wavelength) / L
    return E, margin


def mirror_point(p, a, b):
    """Reflection of p across the line through a and b (projection form)."""
    d = b - a
    foot = a + d * ((p - a) @ d) / (d @ d)
    return 2.0 * foot - p


def line_intersection(p0, p1, a, b):
    """Intersection of the lines (p0, p1) and (a, b) by solving a 2x2 system."""
    M = np.array([[p1[0] - p0[0], a[0] - b[0]], [p1[1] - p0[1], a[1] - b[1]]])
    s = np.linalg.solve(M, a - p0)
    return p0 + s[0] * (p1 - p0)


def relaxed_path(walls, tx, rx, seq):
    """Image-method vertices on the infinite lines, by projection mirrors and 2x2 solves."""
    walls = [np.asarray(w, np.float64) for w in walls]
    imgs = [np.asarray(tx, np.float64)]
    for w in seq:
        imgs.append(mirror_point(imgs[-1], walls[w][:2], walls[w][2:]))
    Q = [None] * (len(seq) + 2)
    Q[0] = np.asarray(tx, np.float64)
    Q[-1] = np.asarray(rx, np.float64)
    for j in range(len(seq), 0, -1):
        w = walls[seq[j - 1]]
        Q[j] = line_intersection(Q[j + 1], imgs[j], w[:2], w[2:])
    return Q, imgs
