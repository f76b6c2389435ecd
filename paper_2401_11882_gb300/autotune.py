"""Autotuner for the path kernels' work decomposition.

Times a set of candidate tile shapes (warps per CTA, candidates per work
unit, resident CTAs per SM, one or two receivers per lane) with CUDA events on
the current stream (inside the library: drt_tune_forward) and keeps the
fastest.  Results are cached on disk, keyed by GPU name, smoothing, order
K and the power-of-two buckets of the wall and receiver counts; a later call
with a key in the cache costs no timing.  Cache file: $DRT_TUNE_CACHE, else
~/.cache/drt_gb300/tune.json.
"""
from __future__ import annotations

import json
import math
import os
import threading
from dataclasses import asdict, replace

from .ops import TileConfig

_lock = threading.Lock()

FORWARD_CANDIDATES = [
    TileConfig(warps_per_cta=w, cands_per_unit=c, ctas_per_sm=o)
    for w in (4, 8) for c in (16, 32, 64, 128) for o in (0, 2)
]

BATCH_CANDIDATES = [TileConfig(warps_per_cta=w, ctas_per_sm=o) for w in (4, 8) for o in (0, 1, 2)]


def cache_path() -> str:
    return os.environ.get("DRT_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "drt_gb300", "tune.json")


def _bucket(n: int) -> int:
    return 1 << max(0, math.ceil(math.log2(max(1, n))))


def forward_key(gpu: str, smoothing: str, max_order: int, n_walls: int, n_rx: int) -> str:
    return f"fwd|{gpu}|{smoothing}|K{max_order}|W{_bucket(n_walls)}|R{_bucket(n_rx)}"


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str | None = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def pick_best(timings: list[tuple[TileConfig, float]]) -> TileConfig:
    """Fastest configuration; ties go to the earlier candidate."""
    best = min(range(len(timings)), key=lambda i: (timings[i][1], i))
    return timings[best][0]


def time_fn(fn, reps: int = 3) -> float:
    """Mean milliseconds of fn() over reps runs after one warm-up, on the current stream."""
    import torch
    fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    b.synchronize()
    return a.elapsed_time(b) / reps


def tune_forward(walls, tx, rx, max_order: int, alpha: float, smoothing: str = "hard_sigmoid",
                 refl_coef: float = 0.5, candidates=None, reps: int = 3, use_cache: bool = True,
                 timer=None) -> TileConfig:
    """Best tile for drt_forward on this scene shape (cached)."""
    import torch
    from . import ops
    gpu = torch.cuda.get_device_name(walls.device)
    key = forward_key(gpu, smoothing, max_order, walls.shape[0], rx.shape[0])
    with _lock:
        cache = load_cache() if use_cache else {}
        if key in cache:
            return TileConfig(**cache[key]["tile"])
    cands = candidates or FORWARD_CANDIDATES
    if candidates is None and smoothing in ("hard_sigmoid", "sigmoid"):
        # these smoothings have a one-receiver-per-lane variant of every shape
        cands = cands + [replace(c, single_rx=True) for c in cands]
    if timer is None:
        # timed inside the library (drt_tune_forward, CUDA events)
        _, ms = ops.tune_forward_timings(walls, tx, rx, max_order, alpha, smoothing, cands,
                                         refl_coef, reps)
        timings = list(zip(cands, ms))
    else:
        timings = []
        for cfg in cands:
            ms = timer(lambda: ops.forward(walls, tx, rx, max_order, alpha, smoothing, refl_coef,
                                           tile=cfg), reps)
            timings.append((cfg, ms))
    best = pick_best(timings)
    if use_cache:
        with _lock:
            cache = load_cache()
            cache[key] = {"tile": asdict(best), "ms": min(t for _, t in timings),
                          "tried": [[asdict(c), t] for c, t in timings]}
            save_cache(cache)
    return best


def tune_batch(batch, n_scenes: int | None = None, candidates=None, steps: int = 1,
               timer=None, return_timings: bool = False, **descent_kw):
    """Best tile for the batched descent, timed on (the first n_scenes of) the batch:
    each candidate builds its own plan and runs ``steps`` descent steps once to warm
    up and once timed.  Returns the tile, or (tile, [(tile, ms), ...]) with
    ``return_timings``."""
    from .batched import BatchedDescent
    from . import scenes
    sub = batch
    if n_scenes is not None and n_scenes < batch.n_scenes:
        n = n_scenes
        sub = scenes.SceneBatch(batch.walls[:batch.wall_off[n]], batch.wall_off[:n + 1],
                                batch.rx[:batch.rx_off[n]], batch.rx_off[:n + 1],
                                batch.max_order[:n], batch.tx0[:n], batch.alpha,
                                batch.smoothing, batch.refl_coef)
    timer = timer or time_fn
    timings = []
    for cfg in candidates or BATCH_CANDIDATES:
        bd = BatchedDescent(sub, tile=cfg, **descent_kw)
        ms = timer(lambda: bd.run(steps), 1)
        bd.close()
        timings.append((cfg, ms))
    best = pick_best(timings)
    return (best, timings) if return_timings else best
