"""Seeded synthetic scene generators.

This module only draws inputs: wall segments, transmitter (TX) and receiver
(RX) positions, and the per-scene knobs (maximum reflection order K, smoothing
sharpness alpha, smoothing function).  It contains none of the ray-tracing
arithmetic, and it is the one module that both the CUDA path and the CPU
oracle consume, so that both see the exact same FP32 bits.

The scenes follow the setting of the paper's application (Sec. VII): one TX,
many RX, 2D walls given as segments (Sec. III, Sec. VI).  The paper publishes
no scene data, so every scene here is synthetic:

* ``unit_square_walls``: the four sides of [0, 1]^2.
* ``random_segments``: segment midpoints uniform in [0, 1]^2, lengths uniform
  in [0.02, 0.2], orientation uniform in [0, pi).
* ``rx_grid``: receivers at the cell centres of an n x n grid of [0, 1]^2.

Random numbers come from ``numpy.random.default_rng(seed)`` (PCG64); the draw
order is fixed by the code below.  Arrays are float32, C-contiguous: walls
``[W, 4]`` as (x0, y0, x1, y1), tx ``[2]``, rx ``[R, 2]``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SMOOTHINGS = ("sigmoid", "hard_sigmoid", "step")


@dataclass
class Scene:
    """One scene: walls, one TX, a set of RX, and the smoothing knobs."""

    walls: np.ndarray          # float32 [W, 4]: x0, y0, x1, y1
    tx: np.ndarray             # float32 [2]
    rx: np.ndarray             # float32 [R, 2]
    max_order: int = 1         # K: paths with 0..K reflections
    alpha: float = 100.0       # smoothing sharpness (Eq. 3)
    smoothing: str = "hard_sigmoid"
    refl_coef: float = 0.5     # per-reflection power coefficient Gamma
    name: str = ""
    meta: dict = field(default_factory=dict)

    def __post_init__(self):
        self.walls = np.ascontiguousarray(self.walls, dtype=np.float32).reshape(-1, 4)
        self.tx = np.ascontiguousarray(self.tx, dtype=np.float32).reshape(2)
        self.rx = np.ascontiguousarray(self.rx, dtype=np.float32).reshape(-1, 2)
        if self.smoothing not in SMOOTHINGS:
            raise ValueError(f"unknown smoothing {self.smoothing!r}")

    @property
    def n_walls(self) -> int:
        return int(self.walls.shape[0])

    @property
    def n_rx(self) -> int:
        return int(self.rx.shape[0])

    def replace(self, **kw) -> "Scene":
        d = dict(walls=self.walls, tx=self.tx, rx=self.rx, max_order=self.max_order,
                 alpha=self.alpha, smoothing=self.smoothing, refl_coef=self.refl_coef,
                 name=self.name, meta=dict(self.meta))
        d.update(kw)
        return Scene(**d)


def unit_square_walls() -> np.ndarray:
    """The four sides of the unit square, counter-clockwise from the origin."""
    return np.array([[0, 0, 1, 0], [1, 0, 1, 1], [1, 1, 0, 1], [0, 1, 0, 0]],
                    dtype=np.float32)


def random_segments(rng: np.random.Generator, n: int,
                    length_range=(0.02, 0.2)) -> np.ndarray:
    """n segments: midpoints U[0,1]^2, then lengths, then angles U[0, pi)."""
    mid = rng.uniform(0.0, 1.0, size=(n, 2))
    length = rng.uniform(length_range[0], length_range[1], size=n)
    angle = rng.uniform(0.0, np.pi, size=n)
    half = 0.5 * length[:, None] * np.stack([np.cos(angle), np.sin(angle)], axis=1)
    return np.concatenate([mid - half, mid + half], axis=1).astype(np.float32)


def spatial_order(points: np.ndarray, bits: int = 16) -> np.ndarray:
    """Permutation that sorts 2D points in [0, 1]^2 along a Z-order (Morton) curve,
    so that consecutive points (the lanes of a warp) are near each other."""
    q = np.clip(np.asarray(points, np.float64), 0.0, 1.0)
    n = (1 << bits) - 1
    ix = np.round(q[:, 0] * n).astype(np.uint64)
    iy = np.round(q[:, 1] * n).astype(np.uint64)
    key = np.zeros(len(q), np.uint64)
    for b in range(bits):
        key |= ((ix >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b)
        key |= ((iy >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b + 1)
    return np.argsort(key, kind="stable")


def rx_grid(n: int) -> np.ndarray:
    """RX at the cell centres ((i + 1/2)/n, (j + 1/2)/n), row-major in (j, i)."""
    c = (np.arange(n, dtype=np.float64) + 0.5) / n
    xx, yy = np.meshgrid(c, c, indexing="xy")
    return np.stack([xx.ravel(), yy.ravel()], axis=1).astype(np.float32)


def rx_uniform(rng: np.random.Generator, n: int, lo=0.05, hi=0.95) -> np.ndarray:
    return rng.uniform(lo, hi, size=(n, 2)).astype(np.float32)


def _check_rx_clear_of_tx(rx: np.ndarray, tx: np.ndarray, min_dist=1e-3) -> None:
    d = np.hypot(rx[:, 0].astype(np.float64) - tx[0], rx[:, 1].astype(np.float64) - tx[1])
    if rx.shape[0] and d.min() < min_dist:
        raise ValueError("an RX lies within %g of the TX" % min_dist)


def tiny_scene(alpha: float = 100.0, smoothing: str = "hard_sigmoid", max_order: int = 1) -> Scene:
    """Unit square + interior wall (0.3,0.5)-(0.7,0.5); TX (0.5,0.2); 16 RX
    uniform in [0.05, 0.95]^2 from seed 0; K <= 1."""
    walls = np.concatenate([unit_square_walls(),
                            np.array([[0.3, 0.5, 0.7, 0.5]], dtype=np.float32)])
    rx = rx_uniform(np.random.default_rng(0), 16)
    tx = np.array([0.5, 0.2], dtype=np.float32)
    _check_rx_clear_of_tx(rx, tx)
    return Scene(walls, tx, rx, max_order=max_order, alpha=alpha, smoothing=smoothing,
                 name="square+1 wall, 16 RX, K<=1")


def clutter_scene(n_segments: int = 60, grid: int = 256, seed: int = 0, alpha: float = 100.0,
                  smoothing: str = "hard_sigmoid", max_order: int = 2, boundary: bool = True,
                  tx=(0.5, 0.2), rx: np.ndarray | None = None) -> Scene:
    """Square boundary (optional) + n random segments; RX grid (or given RX)."""
    rng = np.random.default_rng(seed)
    segs = random_segments(rng, n_segments)
    walls = np.concatenate([unit_square_walls(), segs]) if boundary else segs
    rx = rx_grid(grid) if rx is None else rx
    tx = np.asarray(tx, dtype=np.float32)
    _check_rx_clear_of_tx(rx, tx)
    return Scene(walls, tx, rx, max_order=max_order, alpha=alpha, smoothing=smoothing,
                 name=f"{'square+' if boundary else ''}{n_segments} segments, "
                      f"{rx.shape[0]} RX, K<={max_order}")


def large_scene(alpha: float = 100.0, smoothing: str = "hard_sigmoid") -> Scene:
    """Square + 60 random segments (seed 0), 256 x 256 RX grid, K <= 2 (4097 sequences)."""
    return clutter_scene(60, 256, 0, alpha, smoothing, 2, True)


def gradient_scene(alpha: float = 100.0, smoothing: str = "hard_sigmoid") -> Scene:
    """128 random segments (seed 0, no boundary), 128 x 128 RX grid, K <= 2 (16385 sequences)."""
    return clutter_scene(128, 128, 0, alpha, smoothing, 2, False)


def surrogate_scene(alpha: float = 100.0, smoothing: str = "hard_sigmoid", seed: int = 0,
                    n_rx: int = 256) -> Scene:
    """Square + 60 random segments (64 walls), 256 RX uniform in [0.05, 0.95]^2, K <= 2."""
    rng = np.random.default_rng(seed)
    segs = random_segments(rng, 60)
    walls = np.concatenate([unit_square_walls(), segs])
    rx = rx_uniform(rng, n_rx)
    return Scene(walls, np.array([0.5, 0.5], np.float32), rx, max_order=2, alpha=alpha,
                 smoothing=smoothing, name="square+60 segments, 256 random RX, K<=2")


def random_small_scene(rng: np.random.Generator, n_walls: int, n_rx: int, max_order: int,
                       alpha: float, smoothing: str, boundary: bool = False) -> Scene:
    """A small random scene for parity sweeps (walls, then TX, then RX drawn in that order)."""
    segs = random_segments(rng, n_walls - (4 if boundary else 0), (0.05, 0.4))
    walls = np.concatenate([unit_square_walls(), segs]) if boundary else segs
    tx = rng.uniform(0.1, 0.9, size=2).astype(np.float32)
    rx = rx_uniform(rng, n_rx)
    keep = np.hypot(rx[:, 0] - tx[0], rx[:, 1] - tx[1]) > 1e-2
    return Scene(walls, tx, rx[keep], max_order=max_order, alpha=alpha, smoothing=smoothing,
                 name=f"random {n_walls} walls")


@dataclass
class SceneBatch:
    """Many scenes of uneven size, concatenated (CSR offsets)."""

    walls: np.ndarray        # float32 [sum W, 4]
    wall_off: np.ndarray     # int32 [S + 1]
    rx: np.ndarray           # float32 [sum R, 2]
    rx_off: np.ndarray       # int32 [S + 1]
    max_order: np.ndarray    # int32 [S]
    tx0: np.ndarray          # float32 [S, T, 2] initial TX positions
    alpha: float = 100.0
    smoothing: str = "hard_sigmoid"
    refl_coef: float = 0.5

    @property
    def n_scenes(self) -> int:
        return int(self.max_order.shape[0])

    def scene(self, s: int, t: int = 0) -> Scene:
        w = self.walls[self.wall_off[s]:self.wall_off[s + 1]]
        r = self.rx[self.rx_off[s]:self.rx_off[s + 1]]
        return Scene(w, self.tx0[s, t], r, max_order=int(self.max_order[s]), alpha=self.alpha,
                     smoothing=self.smoothing, refl_coef=self.refl_coef)


def scene_batch(n_scenes: int = 4096, seed: int = 0, walls_range=(8, 256), rx_range=(64, 4096),
                orders=(0, 1, 2), n_tx: int = 4, alpha: float = 100.0,
                smoothing: str = "hard_sigmoid") -> SceneBatch:
    """Uneven batch: per scene W ~ U{walls_range} (4 boundary + W-4 random segments),
    R ~ U{rx_range} uniform in [0.05, 0.95]^2, K ~ U{orders}, n_tx TX starts in
    [0.05, 0.95]^2.  Draw order per scene: W, R, K, segments, RX, TX starts."""
    rng = np.random.default_rng(seed)
    walls, rxs, w_off, r_off, ks, txs = [], [], [0], [0], [], []
    for _ in range(n_scenes):
        W = int(rng.integers(walls_range[0], walls_range[1] + 1))
        R = int(rng.integers(rx_range[0], rx_range[1] + 1))
        K = int(rng.choice(orders))
        segs = random_segments(rng, W - 4)
        w = np.concatenate([unit_square_walls(), segs])
        r = rx_uniform(rng, R)
        t = rx_uniform(rng, n_tx)
        walls.append(w); rxs.append(r); ks.append(K); txs.append(t)
        w_off.append(w_off[-1] + W); r_off.append(r_off[-1] + R)
    return SceneBatch(np.concatenate(walls), np.asarray(w_off, np.int32), np.concatenate(rxs),
                      np.asarray(r_off, np.int32), np.asarray(ks, np.int32),
                      np.stack(txs).astype(np.float32), alpha, smoothing)


# --------------------------------------------------------------------------- 3D scenes
@dataclass
class Scene3:
    """One 3D scene: triangle walls, one TX, a set of RX, and the smoothing knobs."""

    tris: np.ndarray           # float32 [W, 9]: corners A, B, C as x, y, z
    tx: np.ndarray             # float32 [3]
    rx: np.ndarray             # float32 [R, 3]
    max_order: int = 1
    alpha: float = 100.0
    smoothing: str = "hard_sigmoid"
    refl_coef: float = 0.5
    name: str = ""

    def __post_init__(self):
        self.tris = np.ascontiguousarray(self.tris, dtype=np.float32).reshape(-1, 9)
        self.tx = np.ascontiguousarray(self.tx, dtype=np.float32).reshape(3)
        self.rx = np.ascontiguousarray(self.rx, dtype=np.float32).reshape(-1, 3)
        if self.smoothing not in SMOOTHINGS:
            raise ValueError(f"unknown smoothing {self.smoothing!r}")

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])

    @property
    def n_rx(self) -> int:
        return int(self.rx.shape[0])


def extrude(walls: np.ndarray, z0: float, z1: float) -> np.ndarray:
    """Vertical rectangles z in [z0, z1] over 2D walls [W, 4], two triangles each ([2W, 9])."""
    out = []
    for x0, y0, x1, y1 in np.asarray(walls, np.float64):
        a, b = (x0, y0, z0), (x1, y1, z0)
        c, d = (x1, y1, z1), (x0, y0, z1)
        out.append(a + b + c)
        out.append(a + c + d)
    return np.array(out, dtype=np.float32).reshape(-1, 9)


def room3d(grid: int = 128, alpha: float = 100.0, smoothing: str = "hard_sigmoid",
           max_order: int = 2) -> Scene3:
    """The 64-wall scene of ``large_scene`` as a room of height 1: its walls extruded over
    z in [0, 1] (128 triangles) plus a floor and a ceiling (2 triangles each), 132
    triangles; TX (0.5, 0.2, 0.5); a grid x grid receiver plane at z = 0.3."""
    base = clutter_scene(60, 2, 0, alpha, smoothing, 2, True)
    corners = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float64)
    slabs = []
    for z, order in ((0.0, (0, 1, 2, 3)), (1.0, (0, 3, 2, 1))):
        p = [tuple(corners[i]) + (z,) for i in order]
        slabs.append(p[0] + p[1] + p[2])
        slabs.append(p[0] + p[2] + p[3])
    tris = np.concatenate([extrude(base.walls, 0.0, 1.0),
                           np.array(slabs, dtype=np.float32).reshape(-1, 9)])
    rx2 = rx_grid(grid)
    rx = np.concatenate([rx2, np.full((rx2.shape[0], 1), 0.3, np.float32)], 1)
    return Scene3(tris, np.array([0.5, 0.2, 0.5], np.float32), rx, max_order=max_order,
                  alpha=alpha, smoothing=smoothing, name="room3d")


def random_scene3(rng: np.random.Generator, n_tris: int, n_rx: int, max_order: int, alpha: float,
                  smoothing: str) -> Scene3:
    """Random triangles (corners within 0.35 of a centre in [0.1, 0.9]^3), TX and RX in the
    unit cube (triangles, then TX, then RX drawn in that order)."""
    centre = rng.uniform(0.1, 0.9, (n_tris, 1, 3))
    tris = (centre + rng.uniform(-0.35, 0.35, (n_tris, 3, 3))).reshape(n_tris, 9)
    tx = rng.uniform(0.1, 0.9, 3)
    rx = rng.uniform(0.05, 0.95, (n_rx, 3))
    rx = rx[np.linalg.norm(rx - tx, axis=1) > 1e-2]
    return Scene3(tris, tx, rx, max_order=max_order, alpha=alpha, smoothing=smoothing,
                  name=f"random {n_tris} triangles")


@dataclass
class SceneBatch3:
    """Many 3D scenes of uneven size, concatenated (CSR offsets)."""

    tris: np.ndarray         # float32 [sum W, 9]
    wall_off: np.ndarray     # int32 [S + 1]
    rx: np.ndarray           # float32 [sum R, 3]
    rx_off: np.ndarray       # int32 [S + 1]
    max_order: np.ndarray    # int32 [S]
    tx0: np.ndarray          # float32 [S, T, 3] initial TX positions
    alpha: float = 100.0
    smoothing: str = "hard_sigmoid"
    refl_coef: float = 0.5

    @property
    def n_scenes(self) -> int:
        return int(self.max_order.shape[0])

    def scene(self, s: int, t: int = 0) -> Scene3:
        w = self.tris[self.wall_off[s]:self.wall_off[s + 1]]
        r = self.rx[self.rx_off[s]:self.rx_off[s + 1]]
        return Scene3(w, self.tx0[s, t], r, max_order=int(self.max_order[s]), alpha=self.alpha,
                      smoothing=self.smoothing, refl_coef=self.refl_coef)


def scene_batch3(n_scenes: int = 64, seed: int = 0, segments_range=(2, 30), rx_range=(16, 512),
                 orders=(0, 1, 2), n_tx: int = 4, alpha: float = 100.0,
                 smoothing: str = "hard_sigmoid") -> SceneBatch3:
    """Uneven batch of rooms: per scene n ~ U{segments_range} random segments
    (``random_segments``) inside the unit square, extruded with the square's four
    walls over z in [0, 1] and closed by a floor and a ceiling (2 (n + 4) + 4
    triangles); R ~ U{rx_range} receivers uniform in [0.05, 0.95]^2 x [0.1, 0.9];
    K ~ U{orders}; n_tx TX starts drawn the same way.  Draw order per scene: n, R,
    K, segments, RX, TX starts."""
    rng = np.random.default_rng(seed)
    corners = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float64)
    slabs = []
    for z, order in ((0.0, (0, 1, 2, 3)), (1.0, (0, 3, 2, 1))):
        p = [tuple(corners[i]) + (z,) for i in order]
        slabs.append(p[0] + p[1] + p[2])
        slabs.append(p[0] + p[2] + p[3])
    slabs = np.array(slabs, dtype=np.float32).reshape(-1, 9)

    def points(n):
        return np.concatenate([rx_uniform(rng, n), rng.uniform(0.1, 0.9, (n, 1))],
                              1).astype(np.float32)

    tris, rxs, w_off, r_off, ks, txs = [], [], [0], [0], [], []
    for _ in range(n_scenes):
        n = int(rng.integers(segments_range[0], segments_range[1] + 1))
        R = int(rng.integers(rx_range[0], rx_range[1] + 1))
        K = int(rng.choice(orders))
        walls2 = np.concatenate([unit_square_walls(), random_segments(rng, n)])
        t3 = np.concatenate([extrude(walls2, 0.0, 1.0), slabs])
        r = points(R)
        t = points(n_tx)
        tris.append(t3); rxs.append(r); ks.append(K); txs.append(t)
        w_off.append(w_off[-1] + t3.shape[0]); r_off.append(r_off[-1] + R)
    return SceneBatch3(np.concatenate(tris), np.asarray(w_off, np.int32), np.concatenate(rxs),
                       np.asarray(r_off, np.int32), np.asarray(ks, np.int32),
                       np.stack(txs).astype(np.float32), alpha, smoothing)
