"""Writes shadow_receivers_large_scene.txt: the oracle's lowest-power receivers of
the benchmark scene (square + 60 random segments, seed 0; 256 x 256 receiver
grid; K <= 2; hard sigmoid at alpha 10, 100 and 1000).

The min-power loss (Eq. 8) lands on these receivers, whose power is many
decades below the scene's brightest one, so a parity sample drawn uniformly
from the grid rarely holds them.  This script runs the FP64 oracle over the
whole grid once (about a minute per alpha on 16 cores) and keeps, per alpha,
the N lowest receivers and the N lowest with a positive power (where the
hard sigmoid saturates, the lowest are in full shadow, exactly 0): their indices
and powers.  Only ``oracle`` computes the stored values.

    python tests/golden/make_shadow_receivers.py
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2401_11882_gb300 import scenes  # noqa: E402

ALPHAS = (10.0, 100.0, 1000.0)
N_LOWEST = 24
OUT = os.path.join(HERE, "shadow_receivers_large_scene.txt")


def main() -> None:
    oracle.build()
    lines = [
        "# The oracle's lowest-power receivers of the benchmark scene: square + 60 random",
        "# segments (seed 0), 256 x 256 cell-centre receiver grid, TX (0.5, 0.2), K <= 2,",
        "# hard sigmoid, Gamma 0.5.  Written by make_shadow_receivers.py from the FP64 oracle",
        "# over every receiver: per alpha the 24 lowest receivers and the 24 lowest with a",
        "# positive power.  Columns: alpha, receiver index (row-major grid), rank of its power",
        "# among all receivers (0 = the minimum, the loss's receiver; ties by index), FP64",
        "# power, and the scene's largest power at that alpha.",
    ]
    for alpha in ALPHAS:
        sc = scenes.large_scene(alpha=alpha, smoothing="hard_sigmoid")
        P = oracle.power(sc.walls, sc.tx, sc.rx, sc.max_order, sc.alpha, sc.smoothing,
                         sc.refl_coef)
        ranked = np.argsort(P, kind="stable")
        rank_of = np.empty_like(ranked)
        rank_of[ranked] = np.arange(ranked.size)
        positive = ranked[P[ranked] > 0.0]
        keep = sorted(set(ranked[:N_LOWEST].tolist()) | set(positive[:N_LOWEST].tolist()),
                      key=lambda i: rank_of[i])
        for i in keep:
            lines.append(f"{alpha:g} {int(i)} {int(rank_of[i])} {P[i]:.17g} {P.max():.17g}")
        print(f"alpha {alpha:g}: min {P[ranked[0]]:.6g} at {int(ranked[0])}, lowest positive "
              f"{P[positive[0]]:.6g}, max {P.max():.6g}", flush=True)
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
